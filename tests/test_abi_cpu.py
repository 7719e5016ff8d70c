"""The C-ABI library on a machine without a GPU.

Checks that libbridge.so loads, exports every entry point that
include/bridge.h declares, fails loudly (BRIDGE_ECUDA) instead of falling
back to the CPU, and that the host-side index arithmetic the kernels use
(even-odd half-lattice neighbours with wrap flags) matches the oracle's
lattice.  No compute call is made.
"""

import os
import re
import subprocess

import numpy as np
import pytest

from oracle.lattice import Lattice

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2303_05883_gb300", "libbridge.so")


@pytest.fixture(scope="session")
def built():
    import __graft_entry__ as g

    g.build()
    from paper_2303_05883_gb300 import _abi

    return _abi.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "bridge.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|long|const char\*|void\*)\s*\*?\s*(bridge_\w+)\s*\(", src, re.M)))


def test_every_declared_symbol_is_exported(built):
    names = declared_symbols()
    assert len(names) >= 30
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (bridge_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(built, n)


def test_binding_declares_every_symbol(built):
    from paper_2303_05883_gb300 import _abi

    assert set(declared_symbols()) == set(_abi.SIGNATURES)


def test_no_gpu_means_ecuda_not_fallback(built):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2303_05883_gb300 import _abi, api

    with pytest.raises(_abi.BridgeError) as e:
        api.bridge_lattice_create((4, 4, 4, 4))
    assert e.value.status == _abi.BRIDGE_ECUDA


def test_strerror_and_defaults(built):
    from paper_2303_05883_gb300 import api

    assert api.bridge_strerror(0) == "ok"
    assert "converge" in api.bridge_strerror(-3)
    s = api.make_solver()
    assert s.tol == 1e-10 and s.mixed == 1 and s.check_every == 16
    m = api.make_mg_params()
    assert list(m.block) == [4, 4, 4, 4] and m.nvec == 16 and m.setup_steps == 1
    assert (m.sap_cycles, m.mr_steps, m.coarse_maxiter) == (2, 4, 200)
    assert m.coarse_tol == 5e-2 and m.coarse_half == 1 and m.coarse_eo == 1
    m = api.make_mg_params(block=(2, 2, 4, 4), nvec=12, coarse_eo=0, coarse_tol=0.1)
    assert list(m.block) == [2, 2, 4, 4] and m.nvec == 12 and m.coarse_eo == 0 and m.coarse_tol == 0.1


def test_invalid_extents_rejected(built):
    from paper_2303_05883_gb300 import _abi, api

    for dims in [(4, 3, 4, 4), (0, 4, 4, 4), (4, 4, 4, 1)]:
        with pytest.raises(_abi.BridgeError) as e:
            api.bridge_lattice_create(dims)
        assert e.value.status == _abi.BRIDGE_EINVAL


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 6, 8, 10), (8, 4, 2, 6), (6, 2, 4, 4)])
def test_neighbour_map_matches_oracle(built, dims):
    from paper_2303_05883_gb300 import api

    lat = Lattice(dims)
    for parity in (0, 1):
        sites = lat.sites_of(parity)
        for ih in range(0, len(sites), max(1, len(sites) // 37)):
            x = sites[ih]
            got, wraps = api.bridge_debug_neighbours(dims, parity, ih)
            for mu in range(4):
                for k, step in enumerate((+1, -1)):
                    (y,), (w,) = lat.neighbor(np.array([x]), mu, step)
                    assert got[2 * mu + k] == y // 2, (dims, parity, ih, mu, step)
                    assert wraps[2 * mu + k] == int(w)
