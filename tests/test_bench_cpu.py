"""The bench's reference arm (the FP64 oracle timed on the host cores) runs
without a GPU and prints one JSON line in the bench contract."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload", ["clover_32x32x32x64", "mobius_24x24x24x48x16", "staggered_32x32x32x32"])
def test_reference_arm_prints_contract_line(workload):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload, "--steps", "1",
                          "--warmup", "0", "--oracle-sites", "1024"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == workload


def test_oracle_sample_on_all_cores_matches_work():
    """The all-cores oracle baseline: the sampled sites split over spawned
    workers reading the fields from shared memory; every site is computed."""
    sys.path.insert(0, ROOT)
    import bench
    import synth

    w = synth.WORKLOADS["wilson_8x8x8x8"]
    U = w.gauge()
    b = synth.gaussian_spinor(w.dims, 1)
    v, secs, procs = bench.oracle_sample_pool(w, U, b, 1024, seed=3, procs=2)
    assert procs == 2 and secs > 0 and v == pytest.approx(1024 * bench.FP64_D_BYTES_PER_SITE / secs / 1e9)


def test_oracle_samples_never_exceed_the_lattice():
    """A sample asked for more sites than the lattice has takes every site once."""
    sys.path.insert(0, ROOT)
    import bench
    import synth

    w = synth.WORKLOADS["wilson_8x8x8x8"]
    U = w.gauge()
    b = synth.gaussian_spinor(w.dims, 1)
    v, secs, _ = bench.oracle_sample(w, U, b, 10 * 4096, seed=0)
    assert v == pytest.approx(4096 * bench.FP64_D_BYTES_PER_SITE / secs / 1e9)
    v, secs, _ = bench.oracle_sample_pool(w, U, b, 10 * 4096, seed=0, procs=2)
    assert v == pytest.approx(4096 * bench.FP64_D_BYTES_PER_SITE / secs / 1e9)
