"""Python binding of libbridge: the C-ABI entry points under the same names.

Argument marshalling only -- every step of the operator and the solver runs
in the CUDA kernels of libbridge.so.  Host arrays are numpy complex128 in the
canonical layouts of include/bridge.h (spinors ``(V, 4, 3)`` or
``(nrhs, V, 4, 3)``, links ``(4, V, 3, 3)``); device arrays are torch CUDA
complex128 tensors of the same shapes, which route to the ``*_dev`` entry
points.  PyTorch is used for device memory and streams only.
"""

from __future__ import annotations

import ctypes
from ctypes import POINTER, byref, c_double, c_int, c_long, c_void_p
from dataclasses import dataclass, field

import numpy as np

from . import _abi
from ._abi import BRIDGE_CLOVER, BRIDGE_MOBIUS, BRIDGE_STAGGERED, BRIDGE_WILSON, bridge_info, bridge_kstat, bridge_op, bridge_solver, check

PRECISIONS = {"f64": _abi.BRIDGE_F64, "f32": _abi.BRIDGE_F32, "f16": _abi.BRIDGE_F16, "bf16": _abi.BRIDGE_BF16}


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def make_op(kind="wilson", kappa=0.12, csw=0.0, bc=(1, 1, 1, -1), Ls=0, M5=0.0, b5=0.0, c5=0.0, mf=0.0,
            mass=0.0) -> bridge_op:
    k = {"wilson": BRIDGE_WILSON, "clover": BRIDGE_CLOVER, "mobius": BRIDGE_MOBIUS, "staggered": BRIDGE_STAGGERED}.get(
        kind, kind)
    return bridge_op(int(k), float(kappa), float(csw), (c_int * 4)(*[int(b) for b in bc]), int(Ls), float(M5),
                     float(b5), float(c5), float(mf), float(mass))


def make_staggered(mass, bc=(1, 1, 1, -1)) -> bridge_op:
    """Staggered operator with quark mass ``mass``; fields hold one colour vector per site."""
    return make_op("staggered", bc=bc, mass=mass)


def make_mobius(Ls, M5, b5, c5, mf, bc=(1, 1, 1, -1)) -> bridge_op:
    """Moebius domain-wall operator; b5 = 1, c5 = 0 gives the Shamir operator."""
    return make_op("mobius", 0.0, 0.0, bc, Ls, M5, b5, c5, mf)


def _nrhs(op, a) -> int:
    """Right-hand sides in a canonical array: its leading dimensions count
    four-dimensional fields, Ls of them per right-hand side for MOBIUS;
    STAGGERED fields end in (sites, 3)."""
    if op.kind == BRIDGE_STAGGERED:
        return int(np.prod(a.shape[:-2])) if a.ndim > 2 else 1
    n4 = int(np.prod(a.shape[:-3])) if a.ndim > 3 else 1
    if op.kind == BRIDGE_MOBIUS and op.Ls >= 1:  # (Ls < 1 is left to the library to refuse)
        if n4 % op.Ls:
            raise ValueError(f"a MOBIUS field holds a multiple of Ls = {op.Ls} slices, got {n4}")
        return n4 // op.Ls
    return n4


def make_solver(**kw) -> bridge_solver:
    s = bridge_solver()
    _abi.load().bridge_solver_defaults(byref(s))
    for k, v in kw.items():
        if k == "inner_prec":
            v = _prec(v)
        setattr(s, k, v)
    return s


def _is_torch_cuda(a) -> bool:
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(a, torch.Tensor) and a.is_cuda


def _host(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_double))


def _torch_sync():
    import torch

    torch.cuda.current_stream().synchronize()


# --- lattice ------------------------------------------------------------------


def bridge_lattice_create(dims) -> int:
    lib = _abi.load()
    h = c_void_p()
    check(lib.bridge_lattice_create((c_int * 4)(*[int(d) for d in dims]), byref(h)), "bridge_lattice_create")
    return h.value


def bridge_lattice_destroy(lat) -> None:
    check(_abi.load().bridge_lattice_destroy(lat), "bridge_lattice_destroy")


def bridge_lattice_stream(lat) -> int:
    return _abi.load().bridge_lattice_stream(lat) or 0


def bridge_sync(lat) -> None:
    check(_abi.load().bridge_sync(lat), "bridge_sync")


def bridge_gauge_upload(lat, U, op: bridge_op | None = None) -> None:
    lib = _abi.load()
    opp = byref(op) if op is not None else None
    if _is_torch_cuda(U):
        _torch_sync()
        check(lib.bridge_gauge_upload_dev(lat, c_void_p(U.contiguous().data_ptr()), opp), "bridge_gauge_upload_dev")
    else:
        U = _host(U)
        check(lib.bridge_gauge_upload(lat, _dptr(U), opp), "bridge_gauge_upload")


# --- operators ------------------------------------------------------------------


def _mult(name, lat, op, prec, psi, *extra):
    lib = _abi.load()
    nrhs = _nrhs(op, psi)
    if _is_torch_cuda(psi):
        import torch

        src = psi.contiguous()
        out = torch.empty_like(src)
        _torch_sync()
        fn = getattr(lib, name + "_dev")
        check(fn(lat, byref(op), _prec(prec), *extra, c_void_p(src.data_ptr()), c_void_p(out.data_ptr()), nrhs), name)
        bridge_sync(lat)
        return out
    src = _host(psi)
    out = np.empty_like(src)
    fn = getattr(lib, name)
    check(fn(lat, byref(op), _prec(prec), *extra, _dptr(src), _dptr(out), nrhs), name)
    return out


def bridge_mult_D(lat, op, prec, psi):
    """D psi on the full lattice."""
    return _mult("bridge_mult_D", lat, op, prec, psi)


def bridge_mult_Deo(lat, op, prec, out_parity, psi_half):
    """D_eo psi_o (out_parity 0) or D_oe psi_e (out_parity 1) on half-lattice vectors."""
    return _mult("bridge_mult_Deo", lat, op, prec, psi_half, int(out_parity))


def bridge_mult_Dhat(lat, op, prec, psi_even):
    """The Schur operator of Eq. 1 on even half-lattice vectors."""
    return _mult("bridge_mult_Dhat", lat, op, prec, psi_even)


def bridge_mult_Dhat_dag(lat, op, prec, psi_even):
    """The adjoint of the Schur operator (MOBIUS operators)."""
    return _mult("bridge_mult_Dhat_dag", lat, op, prec, psi_even)


# --- solver -----------------------------------------------------------------------


def _infos(arr, n):
    return [
        dict(
            status=arr[k].status,
            outer_iters=arr[k].outer_iters,
            inner_iters=arr[k].inner_iters,
            restarts=arr[k].restarts,
            true_rel_residual=arr[k].true_rel_residual,
            seconds=arr[k].seconds,
            cgnr_passes=arr[k].cgnr_passes,
        )
        for k in range(n)
    ]


def bridge_solve(lat, op, solver, b, x0=None, raise_on_fail=True):
    """Solve D x = b; returns (x, per-rhs info dicts)."""
    lib = _abi.load()
    nrhs = _nrhs(op, b)
    info = (bridge_info * nrhs)()
    if _is_torch_cuda(b):
        import torch

        bb = b.contiguous()
        x = torch.zeros_like(bb) if x0 is None else x0.contiguous().clone()
        _torch_sync()
        st = lib.bridge_solve_dev(lat, byref(op), byref(solver), c_void_p(bb.data_ptr()), c_void_p(x.data_ptr()), nrhs, info)
    else:
        bb = _host(b)
        x = np.zeros_like(bb) if x0 is None else _host(x0).copy()
        st = lib.bridge_solve(lat, byref(op), byref(solver), _dptr(bb), _dptr(x), nrhs, info)
    if raise_on_fail:
        check(st, "bridge_solve")
    return x, _infos(info, nrhs)


# --- fields -------------------------------------------------------------------------


def bridge_field_create(lat, prec, subset, nrhs=1) -> int:
    h = c_void_p()
    check(_abi.load().bridge_field_create(lat, _prec(prec), int(subset), int(nrhs), byref(h)), "bridge_field_create")
    return h.value


def bridge_field_destroy(f) -> None:
    check(_abi.load().bridge_field_destroy(f), "bridge_field_destroy")


def bridge_field_import(f, src) -> None:
    if _is_torch_cuda(src):
        _torch_sync()
        check(_abi.load().bridge_field_import(f, c_void_p(src.contiguous().data_ptr()), 1), "bridge_field_import")
    else:
        a = _host(src)
        check(_abi.load().bridge_field_import(f, c_void_p(a.ctypes.data), 0), "bridge_field_import")


def bridge_field_export(f, dst) -> None:
    if _is_torch_cuda(dst):
        check(_abi.load().bridge_field_export(f, c_void_p(dst.data_ptr()), 1), "bridge_field_export")
    else:
        assert dst.flags.c_contiguous and dst.dtype == np.complex128
        check(_abi.load().bridge_field_export(f, c_void_p(dst.ctypes.data), 0), "bridge_field_export")


def bridge_apply(lat, op, which, out, inp) -> None:
    check(_abi.load().bridge_apply(lat, byref(op), int(which), out, inp), "bridge_apply")


# --- serving --------------------------------------------------------------------------


def bridge_engine_config(budget_bytes=0, max_active=0) -> None:
    check(_abi.load().bridge_engine_config(int(budget_bytes), int(max_active)), "bridge_engine_config")


@dataclass
class Request:
    handle: int
    shape: tuple
    nrhs: int
    _b: np.ndarray = field(repr=False, default=None)


def bridge_submit(lat, op, solver, b, borrow=False) -> Request:
    """Queue a solve.  borrow=True: the library reads b in place at admission
    (no host copy); the returned Request keeps the array alive."""
    bb = _host(b)
    nrhs = 1 if bb.ndim == 3 else bb.shape[0]
    h = c_void_p()
    fn = _abi.load().bridge_submit_borrowed if borrow else _abi.load().bridge_submit
    check(fn(lat, byref(op), byref(solver), _dptr(bb), nrhs, byref(h)), "bridge_submit")
    # without borrow the library keeps its own copy of b
    return Request(h.value, bb.shape, nrhs, bb if borrow else None)


def bridge_poll(req: Request):
    """None while pending, else (status, x, infos)."""
    x = np.empty(req.shape, dtype=np.complex128)
    info = (bridge_info * req.nrhs)()
    st = _abi.load().bridge_poll(req.handle, _dptr(x), info)
    if st == _abi.BRIDGE_PENDING:
        return None
    return st, x, _infos(info, req.nrhs)


def bridge_wait(req: Request, timeout_ms=-1, want_x=True):
    """None on timeout, else (status, x or None, infos)."""
    x = np.empty(req.shape, dtype=np.complex128) if want_x else None
    info = (bridge_info * req.nrhs)()
    st = _abi.load().bridge_wait(req.handle, int(timeout_ms), _dptr(x) if want_x else None, info)
    if st == _abi.BRIDGE_ETIMEDOUT:
        return None
    return st, x, _infos(info, req.nrhs)


def bridge_request_times(req: Request):
    a, b, c = c_double(), c_double(), c_double()
    check(_abi.load().bridge_request_times(req.handle, byref(a), byref(b), byref(c)), "bridge_request_times")
    return a.value, b.value, c.value


def bridge_request_release(req: Request) -> None:
    check(_abi.load().bridge_request_release(req.handle), "bridge_request_release")


# --- diagnostics ------------------------------------------------------------------------


def bridge_stats(lat):
    arr = (bridge_kstat * 64)()
    n = _abi.load().bridge_stats(lat, arr, 64)
    check(n, "bridge_stats")
    return {
        arr[k].name.decode(): dict(launches=arr[k].launches, bytes=arr[k].bytes, flops=arr[k].flops, ms=arr[k].ms)
        for k in range(n)
    }


def bridge_stats_reset(lat) -> None:
    check(_abi.load().bridge_stats_reset(lat), "bridge_stats_reset")


def bridge_profile(lat, enable=True) -> None:
    check(_abi.load().bridge_profile(lat, 1 if enable else 0), "bridge_profile")


def bridge_launch_count() -> int:
    return int(_abi.load().bridge_launch_count())


def bridge_alu_peak(prec="f32") -> float:
    """Measured FMA throughput of the device in flop/s (2 per FMA)."""
    v = ctypes.c_double(0.0)
    check(_abi.load().bridge_alu_peak(_prec(prec), ctypes.byref(v)), "bridge_alu_peak")
    return v.value


def bridge_debug_neighbours(dims, parity, ih):
    out = (c_long * 8)()
    wr = (c_int * 8)()
    check(
        _abi.load().bridge_debug_neighbours((c_int * 4)(*[int(d) for d in dims]), int(parity), int(ih), out, wr),
        "bridge_debug_neighbours",
    )
    return list(out), list(wr)


def bridge_tune(lat, op, prec="f32", nrhs=1) -> None:
    check(_abi.load().bridge_tune(lat, byref(op), _prec(prec), int(nrhs)), "bridge_tune")


def bridge_tune_table(lat) -> dict:
    buf = ctypes.create_string_buffer(1 << 16)
    _abi.load().bridge_tune_table(lat, buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        k, b, n, v = line.split()
        out[k] = (int(b), int(n), int(v))
    return out


def bridge_tune_set(lat, key: str, block: int, nblk: int, variant: int) -> None:
    check(_abi.load().bridge_tune_set(lat, key.encode(), int(block), int(nblk), int(variant)), "bridge_tune_set")


def bridge_strerror(status: int) -> str:
    return _abi.load().bridge_strerror(int(status)).decode()


# --- two-level multigrid ------------------------------------------------------------------


def make_mg_params(**kw) -> "_abi.bridge_mg_params":
    p = _abi.bridge_mg_params()
    _abi.load().bridge_mg_defaults(byref(p))
    for k, v in kw.items():
        if k == "block":
            v = (c_int * 4)(*[int(b) for b in v])
        setattr(p, k, v)
    return p


class Multigrid:
    """Owning wrapper of a multigrid hierarchy (bridge_mg_setup .. bridge_mg_destroy)."""

    def __init__(self, lattice, op, params=None, null_vectors=None):
        lib = _abi.load()
        self.lattice, self.op = lattice, op
        self.params = params or make_mg_params()
        h = c_void_p()
        nv = None if null_vectors is None else _host(null_vectors)
        check(lib.bridge_mg_setup(lattice.handle, byref(op), byref(self.params), None if nv is None else _dptr(nv),
                                  byref(h)), "bridge_mg_setup")
        self.handle = h.value
        nb, nvec = c_int(), c_int()
        check(lib.bridge_mg_info(self.handle, byref(nb), byref(nvec)), "bridge_mg_info")
        self.nblocks, self.nvec = nb.value, nvec.value

    def close(self):
        if getattr(self, "handle", None):
            _abi.load().bridge_mg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b, solver=None, x0=None, raise_on_fail=True):
        lib = _abi.load()
        solver = solver or make_solver()
        bb = _host(b)
        nrhs = 1 if bb.ndim == 3 else bb.shape[0]
        x = np.zeros_like(bb) if x0 is None else _host(x0).copy()
        info = (bridge_info * nrhs)()
        st = lib.bridge_mg_solve(self.handle, byref(solver), _dptr(bb), _dptr(x), nrhs, info)
        if raise_on_fail:
            check(st, "bridge_mg_solve")
        return x, _infos(info, nrhs)

    def apply(self, which, v):
        """One piece of the cycle (bridge_mg_apply_op) on a canonical array."""
        fine_out = which in (_abi.BRIDGE_MG_PROLONG, _abi.BRIDGE_MG_SAP, _abi.BRIDGE_MG_CYCLE)
        V = self.lattice.V
        out = np.empty((V, 4, 3) if fine_out else (self.nblocks, 2, self.nvec), dtype=np.complex128)
        vin = _host(v)
        check(_abi.load().bridge_mg_apply(self.handle, int(which), _dptr(vin), _dptr(out)), "bridge_mg_apply")
        return out

    def counters(self):
        """(coarse solves, coarse BiCGStab iterations) so far."""
        a, b = c_long(), c_long()
        check(_abi.load().bridge_mg_counters(self.handle, byref(a), byref(b)), "bridge_mg_counters")
        return a.value, b.value

    def coarse_matrix(self):
        """[block][coupling][column][row] complex."""
        n2 = 2 * self.nvec
        out = np.empty((self.nblocks, 9, n2, n2), dtype=np.complex128)
        check(_abi.load().bridge_mg_coarse_matrix(self.handle, _dptr(out)), "bridge_mg_coarse_matrix")
        return out


# --- convenience ---------------------------------------------------------------------------


class Lattice:
    """Owning wrapper of a lattice handle."""

    def __init__(self, dims):
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.handle = bridge_lattice_create(self.dims)

    def close(self):
        if self.handle:
            bridge_lattice_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload(self, U, op=None):
        bridge_gauge_upload(self.handle, U, op)

    def D(self, op, psi, prec="f64"):
        return bridge_mult_D(self.handle, op, prec, psi)

    def Deo(self, op, psi, out_parity=0, prec="f64"):
        return bridge_mult_Deo(self.handle, op, prec, out_parity, psi)

    def Dhat(self, op, psi, prec="f64"):
        return bridge_mult_Dhat(self.handle, op, prec, psi)

    def Dhat_dag(self, op, psi, prec="f64"):
        return bridge_mult_Dhat_dag(self.handle, op, prec, psi)

    def solve(self, op, b, solver=None, x0=None, raise_on_fail=True):
        return bridge_solve(self.handle, op, solver or make_solver(), b, x0, raise_on_fail)

    @property
    def stream(self):
        import torch

        return torch.cuda.ExternalStream(bridge_lattice_stream(self.handle))


# --- domain decomposition with halo exchange ---------------------------------------------


def bridge_dd_plan_of(dims, nparts, rank) -> dict:
    """Face schedule of one slab (host arithmetic only)."""
    pl = _abi.bridge_dd_plan()
    d = (c_int * 4)(*[int(x) for x in dims])
    check(_abi.load().bridge_dd_plan_of(d, int(nparts), int(rank), byref(pl)), "bridge_dd_plan_of")
    return dict(local_dims=tuple(pl.local_dims), t0=pl.t0, rank_up=pl.rank_up, rank_down=pl.rank_down,
                face_sites=pl.face_sites, up_wraps=pl.up_wraps, down_wraps=pl.down_wraps,
                canon_offset_sites=pl.canon_offset_sites)


class Decomposition:
    """A lattice cut into nparts slabs along t, joined by a halo exchange
    (bridge_dd_*).  Inputs may be host arrays or CUDA tensors; results come
    back in the same kind."""

    def __init__(self, lattice, op, nparts):
        self.lattice, self.op, self.nparts = lattice, op, int(nparts)
        h = c_void_p()
        check(_abi.load().bridge_dd_create(lattice.handle, byref(op), self.nparts, byref(h)), "bridge_dd_create")
        self.handle = h.value

    def close(self):
        if self.handle:
            check(_abi.load().bridge_dd_destroy(self.handle), "bridge_dd_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _dev(a):
        import torch

        if _is_torch_cuda(a):
            return a.contiguous(), True
        return torch.from_numpy(np.ascontiguousarray(_host(a))).cuda(), False

    def _mult(self, name, prec, psi, *extra):
        src, on_dev = self._dev(psi)
        out = src.new_empty(src.shape)
        nrhs = 1 if src.dim() == 3 else src.shape[0]
        _torch_sync()
        check(getattr(_abi.load(), name)(self.handle, _prec(prec), *extra, c_void_p(src.data_ptr()),
                                         c_void_p(out.data_ptr()), nrhs), name)
        return out if on_dev else out.cpu().numpy()

    def D(self, psi, prec="f64"):
        return self._mult("bridge_dd_mult_D_dev", prec, psi)

    def Deo(self, psi, out_parity=0, prec="f64"):
        return self._mult("bridge_dd_mult_Deo_dev", prec, psi, int(out_parity))

    def Dhat(self, psi, prec="f64"):
        return self._mult("bridge_dd_mult_Dhat_dev", prec, psi)

    def solve(self, b, solver=None, raise_on_fail=True):
        solver = solver or make_solver()
        src, on_dev = self._dev(b)
        x = src.new_zeros(src.shape)
        nrhs = 1 if src.dim() == 3 else src.shape[0]
        info = (bridge_info * nrhs)()
        _torch_sync()
        check(_abi.load().bridge_dd_solve_dev(self.handle, byref(solver), c_void_p(src.data_ptr()),
                                              c_void_p(x.data_ptr()), nrhs, info), "bridge_dd_solve_dev")
        infos = _infos(info, nrhs)
        if raise_on_fail and any(i["status"] != 0 for i in infos):
            raise _abi.BridgeError(infos[0]["status"], "bridge_dd_solve_dev")
        return (x if on_dev else x.cpu().numpy()), infos
