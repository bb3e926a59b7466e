"""Serving runtime (fw_server_*): continuous batching of simulation requests.

Each request's traces must be the same alone and in the mix (the kernels are
deterministic and every request owns its medium, so the comparison is
bitwise), admission must respect the footprint budget, and failures are
injected on the host (a request above the budget, a CFL above the stability
limit, a non-finite source waveform, cancellation) without disturbing the
other requests."""
import ctypes as C
import time

import numpy as np
import pytest

from gpu_util import oracle_params, to_c
from synthetic import gaussian_pulse, voronoi_classes, voronoi_medium

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_11103_gb300 as fw
    from paper_2606_11103_gb300 import build
    build.build()
    return fw


@pytest.fixture(scope="module")
def lut(fw):
    """Small table of calibrated (alpha0, y) classes shared by the requests."""
    pairs = [(0.5, 1.1), (0.9, 1.6), (0.2, 0.7), (0.0, 1.0)]
    return [to_c(oracle_params(a, y, 2), fw) for a, y in pairs]


def make_request(lut, shape, seed, n_steps, f0=3e6):
    rng = np.random.default_rng(seed)
    dx = 1540.0 / (f0 * 10)
    vc = voronoi_classes(seed, shape, n_seed=6, n_class=len(lut))
    med = voronoi_medium(vc, shape, seed=seed)
    dt = 0.3 * dx / (1650.0 * 1.06)
    src = np.zeros(shape, np.uint8)
    src[(6,) + tuple(rng.integers(8, n - 8) for n in shape[1:])] = 1
    rcv = np.zeros(shape, np.uint8)
    rcv[tuple([12] + [slice(6, n - 6, 5) for n in shape[1:]])] = 1
    amp = 1e-7 if len(shape) == 2 else 1e-11
    w = gaussian_pulse(f0, dt, n_steps, amp)[None].astype(np.float32)
    return dict(shape=shape, dx=dx, dt=dt, c=med["c"], rho=med["rho"], class_idx=med["class_idx"], classes=lut,
                n_steps=n_steps, src_mask=src, waves=w, rcv_mask=rcv, pml=5, f0=f0)


def run_alone(fw, q):
    m = fw.Medium.from_classes(q["shape"], q["dx"], q["c"], q["rho"], q["class_idx"], q["classes"], dt=q["dt"],
                               pml=q["pml"], f0=q["f0"])
    m.set_sources(q["src_mask"], q["waves"])
    m.set_receivers(q["rcv_mask"], q["n_steps"])
    m.run(q["n_steps"])
    tr = m.receivers()
    m.close()
    return tr


def drain(srv, n, timeout=120.0):
    got = {}
    t_end = time.time() + timeout
    while len(got) < n and time.time() < t_end:
        for d in srv.poll(timeout=0.5):
            got[d["id"]] = d
    assert len(got) == n, (len(got), n)
    return got


def footprint(fw, q):
    """The server's admission estimate of a request (fw_server_submit)."""
    g = fw.make_grid(q["shape"], q["dx"], q["dt"], pml=q["pml"], f0=q["f0"])
    b = C.c_size_t()
    fw.check(fw.lib().fw_medium_bytes(C.byref(g), q["classes"][0].n_mech, 0, 0, C.byref(b)))
    shape = q["shape"]
    padded = -(-shape[-1] // 32) * 32 * int(np.prod(shape[:-1]))
    n_src, n_rcv = int(q["src_mask"].sum()), int(q["rcv_mask"].sum())
    return b.value + padded * 8 + n_src * 16 + q["waves"].shape[0] * q["n_steps"] * 8 + \
        n_rcv * (8 + 4 * q["n_steps"]) + (16 << 20)


def test_results_equal_alone_and_in_the_mix(fw, lut):
    shapes = [(96, 80), (160, 128), (48, 40, 36), (128, 128), (40, 44, 52), (200, 96), (56, 48, 40),
              (112, 144), (36, 36, 60), (150, 150)]
    reqs = [make_request(lut, s, seed=100 + i, n_steps=160 + 23 * i) for i, s in enumerate(shapes)]
    srv = fw.Server(hbm_budget=4 << 30, max_active=4, chunk_steps=32, n_streams=4)
    ids = {}
    for i, q in enumerate(reqs):
        rid, _ = srv.submit(tag=i, **q)
        ids[rid] = i
        if i % 3 == 2:
            time.sleep(0.01)          # later arrivals join while earlier ones run
    got = drain(srv, len(reqs))
    srv.close()
    for rid, d in got.items():
        i = ids[rid]
        assert d["status"] == 0, d
        assert d["t_submit"] <= d["t_admit"] <= d["t_done"]
        assert d["voxel_steps"] == int(np.prod(shapes[i])) * reqs[i]["n_steps"]
        alone = run_alone(fw, reqs[i])
        assert np.abs(alone).max() > 0
        assert np.array_equal(d["traces"], alone), i


def test_admission_respects_the_budget(fw, lut):
    q = make_request(lut, (64, 60, 56), seed=7, n_steps=200)
    srv = fw.Server(hbm_budget=int(2.5 * footprint(fw, q)), max_active=8, chunk_steps=16, n_streams=4)
    for i in range(6):
        srv.submit(tag=i, **q)
    peak_active, peak_reserved = 0, 0
    got = {}
    t_end = time.time() + 120
    while len(got) < 6 and time.time() < t_end:
        st = srv.stats()
        peak_active = max(peak_active, st["active"] + st["building"])
        peak_reserved = max(peak_reserved, st["bytes_reserved"])
        assert st["bytes_reserved"] <= st["bytes_budget"]
        for d in srv.poll(timeout=0.002):
            got[d["id"]] = d
    srv.close()
    assert len(got) == 6 and all(d["status"] == 0 for d in got.values())
    ref = run_alone(fw, q)
    for d in got.values():
        assert np.array_equal(d["traces"], ref)
    assert 1 <= peak_active <= 2         # the budget (2.5 footprints), not the 8 slots, limited admission
    assert peak_reserved > 0


def test_failures_stay_with_their_request(fw, lut):
    good = [make_request(lut, (120, 100), seed=20 + i, n_steps=200) for i in range(3)]
    bad_cfl = make_request(lut, (80, 80), seed=30, n_steps=50)
    bad_cfl["dt"] = 0.7 * bad_cfl["dx"] / 1500.0                  # above the 2D limit 0.5497
    bad_nan = make_request(lut, (90, 70), seed=31, n_steps=80)
    bad_nan["waves"] = bad_nan["waves"].copy()
    bad_nan["waves"][0, 40] = np.nan                               # non-finite input -> unstable run
    huge = make_request(lut, (64, 64), seed=32, n_steps=10)
    srv = fw.Server(hbm_budget=256 << 20, max_active=4, chunk_steps=32, n_streams=4)
    rid_huge, _ = srv.submit(tag=99, **dict(huge, shape=(4096, 4096), c=np.full((4096, 4096), 1500, np.float32),
                                            rho=np.full((4096, 4096), 1000, np.float32),
                                            class_idx=np.zeros((4096, 4096), np.uint16),
                                            src_mask=None, rcv_mask=None))
    tags = {}
    for i, q in enumerate([good[0], bad_cfl, good[1], bad_nan, good[2]]):
        rid, _ = srv.submit(tag=i, **q)
        tags[rid] = i
    got = drain(srv, 6)
    srv.close()
    assert got[rid_huge]["status"] == fw.FW_ERR_NOMEM and got[rid_huge]["t_admit"] < 0
    st = {tags[r]: d for r, d in got.items() if r in tags}
    assert st[1]["status"] == fw.FW_ERR_ARG
    assert st[3]["status"] == fw.FW_ERR_UNSTABLE
    for i, q in ((0, good[0]), (2, good[1]), (4, good[2])):
        assert st[i]["status"] == 0
        assert np.array_equal(st[i]["traces"], run_alone(fw, q))


def test_cancel_queued_and_running(fw, lut):
    q = make_request(lut, (256, 256), seed=40, n_steps=3000)
    srv = fw.Server(hbm_budget=2 << 30, max_active=1, chunk_steps=32, n_streams=2)
    r1, _ = srv.submit(tag=1, **q)
    r2, _ = srv.submit(tag=2, **q)
    srv.cancel(r2)                      # still queued: cancelled at once
    t_end = time.time() + 30
    while srv.stats()["active"] == 0 and time.time() < t_end:
        time.sleep(0.005)
    srv.cancel(r1)                      # running: ends after its in-flight chunks
    got = drain(srv, 2)
    srv.close()
    assert got[r2]["status"] == fw._lib.FW_CANCELLED and got[r2]["t_admit"] < 0
    assert got[r1]["status"] == fw._lib.FW_CANCELLED


@pytest.mark.parametrize("policy", [0, 1])
def test_short_requests_are_admitted_ahead_of_long_ones(fw, lut, policy):
    """Size-class policy (0): with one slot, a short request queued behind a
    long one is admitted first when the slot frees up; in arrival order (1)
    it waits its turn.  Results are the same either way."""
    long_q = make_request(lut, (384, 384), seed=50, n_steps=1500)
    short_q = make_request(lut, (64, 64), seed=51, n_steps=100)
    srv = fw.Server(hbm_budget=2 << 30, max_active=1, chunk_steps=32, n_streams=2, policy=policy, short_work=1e6)
    ra, _ = srv.submit(tag=0, **long_q)
    t_end = time.time() + 30
    while srv.stats()["active"] == 0 and time.time() < t_end:
        time.sleep(0.002)
    rb, _ = srv.submit(tag=1, **long_q)
    rc, _ = srv.submit(tag=2, **short_q)
    got = drain(srv, 3)
    srv.close()
    assert all(d["status"] == 0 for d in got.values())
    if policy == 0:
        assert got[rc]["t_admit"] < got[rb]["t_admit"] and got[rc]["t_done"] < got[rb]["t_done"]
    else:
        assert got[rb]["t_admit"] < got[rc]["t_admit"]
    assert np.array_equal(got[rc]["traces"], run_alone(fw, short_q))
    assert np.array_equal(got[rb]["traces"], got[ra]["traces"])
