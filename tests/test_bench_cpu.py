"""Host logic of bench.py (no GPU): the algorithmic-byte counts behind the
roofline fractions, the guard that drops profiled DRAM traffic once the
kernel sources change, and the config object both arms print."""
import argparse
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_sweep_bytes_without_absorbing_layer(bench):
    """3D, N = 4, FP32, no layer: velocity reads p, v (3), psi1 (12), rho,
    class and writes v, psi1; pressure reads v (3), p, psi2 (4), K dt, class
    and writes p, psi2; the single pass reads and writes every state array
    once and reads each map once."""
    vel, pres, single = bench.alg_bytes(3, 4, "f32", False, 0, (64, 64, 64))
    assert vel == 4 + 2 * 3 * 4 + 2 * 12 * 4 + 4 + 2
    assert pres == 3 * 4 + 2 * 4 + 2 * 4 * 4 + 4 + 2
    state = 1 + 3 + 12 + 4
    assert single == 2 * state * 4 + 4 + 4 + 2
    # 16-bit memory variables halve the psi bytes only; beta adds 2 beta dt to the pressure sweep
    v16, p16, _ = bench.alg_bytes(3, 4, "f16", False, 0, (64, 64, 64))
    assert vel - v16 == 2 * 12 * 2 and pres - p16 == 2 * 4 * 2
    assert bench.alg_bytes(2, 4, "f32", True, 0, (64, 64))[1] == bench.alg_bytes(2, 4, "f32", False, 0, (64, 64))[1] + 4


def test_absorbing_layer_share(bench):
    """The layer's memory variables count only over the layer's share of
    each axis: two read-write arrays of 4 B per direction."""
    n, w = 100, 10
    vel0, pres0, _ = bench.alg_bytes(2, 2, "f32", False, 0, (n, n))
    vel, pres, _ = bench.alg_bytes(2, 2, "f32", False, w, (n, n))
    assert vel - vel0 == pytest.approx(2 * (2 * w - 1) / n * 2 * 4)
    assert pres - pres0 == pytest.approx(2 * (2 * w) / n * 2 * 4)


def test_adjoint_bytes(bench):
    vel, pres, _ = bench.alg_bytes(2, 3, "f32", False, 0, (32, 32))
    state = (1 + 2 + 6 + 3) * 4
    assert bench.adjoint_alg_bytes(2, 3, 0, (32, 32)) == 2 * (vel + pres) + 4 * state + 32 + 10


def test_traffic_dropped_when_kernels_change(bench, monkeypatch):
    t = bench.profiled_traffic(1000, "velocity")
    if t is None:
        pytest.skip("committed traffic does not match these kernel sources")
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
    assert bench.profiled_traffic(1000, "velocity") is None


@pytest.mark.parametrize("workload", ["voronoi3d", "twolayer2d"])
def test_reference_arm_names_the_crop_it_runs(bench, workload):
    """The reference arm's config names the crop the oracle runs and the
    workload it is cut from; its voxel count is the crop's."""
    a = argparse.Namespace(workload=workload, size=512, storage="f32")
    gpu = bench.workload_config(a, "x", "single GPU")
    ref = bench.reference_config(a)
    crop = bench.ORACLE_CROP[workload]
    assert ref["voxels"] == (crop ** 2 if workload == "twolayer2d" else crop ** 3)
    assert ref["voxels"] < gpu["voxels"]
    assert gpu["workload"] in ref["workload"] and bench.oracle_sample(workload) in ref["workload"]
    assert ref["storage"] == "f64"
