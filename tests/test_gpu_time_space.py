"""GPU parity of the time-space stencil (Sec. 3.3: 2M-th order in space,
fourth order in time, after Tan & Huang 2014; fw_grid.time_order = 4)
against the FP64 oracle's time-space stencil on the same seeded inputs.
Tolerances (relative L2 of p, every v_d and the receiver traces): 1e-5
for FP32 arithmetic, 1e-11 for the FP64 build of the kernels (measured
1e-14 and below).  Also: the stability limit
that creation enforces against the oracle's, the bf16 / binary16 memory
variables with this stencil at the precision bounds of the leapfrog, and
the refusal of gradients."""
import ctypes as C

import numpy as np
import pytest

from gpu_util import Pair, oracle_params, rel_l2, to_c
from oracle.medium import time_space_cfl_limit
from synthetic import config_c1, config_c2, config_c3, gaussian_pulse

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-11, "bf16": 1e-2, "f16": 2e-3}


@pytest.fixture(scope="module")
def fw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_11103_gb300 as fw
    from paper_2606_11103_gb300 import build
    build.build()
    return fw


def _check(res, tol):
    print(res)
    for k, v in res.items():
        assert v < tol, (k, v, res)


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16"])
def test_c1_homogeneous_2d_time_space(fw, storage):
    """256^2, N=2, 20-cell layer, line source, CFL 0.4, 1000 steps."""
    spec = config_c1()
    prm = oracle_params(0.5, 1.1, 2)
    cls = np.zeros(spec.shape, np.uint16)
    pr = Pair(fw, spec.shape, spec.dx, spec.dt, spec.maps["c"], spec.maps["rho"], cls, [prm],
              pml=spec.pml, f0=spec.f0, storage=storage, time_order=4)
    pr.sources(spec.src_mask, spec.src_waves)
    pr.receivers(spec.rcv_mask, spec.n_steps)
    _check(pr.run_compare(spec.n_steps, checks=4, f64=storage == "f64"), TOL[storage])


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_c3_voronoi_3d_crop_time_space(fw, storage):
    """64^3 crop of the 512^3 Voronoi map (8 classes, N=4, jittered c/rho:
    every cell has its own weights), focused aperture, 100 steps."""
    box = ((0, 64), (224, 288), (224, 288))
    spec = config_c3(n_steps=100, box=box)
    params = [oracle_params(a, y, 4) for a, y in zip(spec.classes["alpha0"], spec.classes["y"])]
    pr = Pair(fw, spec.shape, spec.dx, spec.dt, spec.maps["c"], spec.maps["rho"], spec.maps["class_idx"],
              params, pml=spec.pml, f0=spec.f0, storage=storage, time_order=4)
    pr.sources(spec.src_mask, spec.src_waves, spec.src_wave_of)
    pr.receivers(spec.rcv_mask, 100)
    _check(pr.run_compare(100, f64=storage == "f64"), TOL[storage])


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("shape,nmech,pml,lt", [((203, 157), 1, 12, 6), ((37, 45, 51), 3, 6, 3),
                                                 ((20, 19, 133), 2, 4, 0), ((9, 9, 9), 4, 2, 0)])
def test_ragged_shapes_time_space(fw, storage, shape, nmech, pml, lt):
    """Shapes that are not multiples of the tiles (edges of the x strips and
    of the row blocks, where the cross terms reach the tile corners), a
    random class map, a transition layer and a point source."""
    rng = np.random.default_rng(12)
    dx = 5e-5
    c = (1500 + 80 * rng.uniform(size=shape)).astype(np.float32)
    rho = (950 + 100 * rng.uniform(size=shape)).astype(np.float32)
    cls = rng.integers(0, 3, size=shape).astype(np.uint16)
    params = [oracle_params(a, y, nmech) for a, y in ((0.5, 1.1), (0.9, 1.6), (0.0, 1.0))]
    dt = 0.4 * dx / 1580.0
    pr = Pair(fw, shape, dx, dt, c, rho, cls, params, pml=pml, transition=lt, f0=3e6, storage=storage,
              time_order=4)
    src = np.zeros(shape, np.uint8)
    src[tuple(n // 2 for n in shape)] = 1
    nt = 150
    pr.sources(src, gaussian_pulse(3e6, dt, nt, 1e-9)[None].astype(np.float32))
    rcv = np.zeros(shape, np.uint8)
    rcv[tuple(n // 3 for n in shape)] = 1
    rcv[tuple(n - 2 for n in shape)] = 1
    pr.receivers(rcv, nt, 2)
    _check(pr.run_compare(nt, graphs=False, f64=storage == "f64"), TOL[storage])


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_c2_two_layer_nonlinear_crop_time_space(fw, storage):
    spec = config_c2(n=320, n_steps=400, amp=1e6)
    shape = (320, 301)
    maps = {k: np.ascontiguousarray(v[:, :301]) for k, v in spec.maps.items()}
    cls = (np.arange(320)[:, None] >= 160).astype(np.uint16) * np.ones(shape, np.uint16)
    params = [oracle_params(1.09, 1.0, 4), oracle_params(0.6, 1.5, 4)]
    pr = Pair(fw, shape, spec.dx, spec.dt, maps["c"], maps["rho"], cls, params, beta=maps["beta"],
              pml=spec.pml, f0=spec.f0, storage=storage, time_order=4)
    pr.sources(np.ascontiguousarray(spec.src_mask[:, :301]), spec.src_waves)
    pr.receivers(np.ascontiguousarray(spec.rcv_mask[:, :301]), 400)
    _check(pr.run_compare(400, f64=storage == "f64"), TOL[storage])


@pytest.mark.parametrize("nd", [2, 3])
def test_stability_limit_matches_the_oracle(fw, nd):
    """Creation accepts a homogeneous lossless medium just below the
    oracle's stability limit of the time-space scheme (above the leapfrog's)
    and refuses it just above."""
    lim = time_space_cfl_limit(nd)
    shape = (16,) * nd
    one = np.ones(shape, np.float32)
    lossless = [fw.relax_params(1, 1, [0], [1e9], [0], [1e9])]
    dx, c = 1e-4, 1540.0
    m = fw.Medium.from_classes(shape, dx, one * c, one * 1000, np.zeros(shape, np.uint16), lossless,
                               dt=0.995 * lim * dx / c, time_order=4)
    assert m.info()["time_order"] == 4
    m.close()
    with pytest.raises(fw.FwError):
        fw.Medium.from_classes(shape, dx, one * c, one * 1000, np.zeros(shape, np.uint16), lossless,
                               dt=1.01 * lim * dx / c, time_order=4)


def test_gradient_refused_with_time_space(fw):
    spec = config_c1(n=64, n_steps=20)
    prm = oracle_params(0.5, 1.1, 2)
    m = fw.Medium.from_classes(spec.shape, spec.dx, spec.maps["c"], spec.maps["rho"],
                               np.zeros(spec.shape, np.uint16), [to_c(prm, fw)], dt=spec.dt, pml=spec.pml,
                               f0=spec.f0, time_order=4)
    m.set_sources(spec.src_mask, spec.src_waves)
    m.set_receivers(spec.rcv_mask, 20)
    G = np.zeros((int(spec.rcv_mask.sum()), 20), np.float32)
    gc = np.zeros(spec.shape, np.float32)
    rc = fw.lib().fw_gradient(m.h, 20, 0, C.c_void_p(G.ctypes.data), None, C.c_void_p(gc.ctypes.data), None, 0,
                              C.c_void_p(0))
    assert rc == fw.FW_ERR_UNSUPPORTED
    m.close()


def test_time_space_lowers_the_dispersion_error(fw):
    """The point of the stencil (Sec. 3.3): at CFL 0.4 and 12 points per
    wavelength, a plane pulse on the GPU arrives with a smaller phase error
    than with the leapfrog, both against the exact travel time c t."""
    spec = config_c1(n=256, n_steps=900)
    lossless = fw.relax_params(1, 1, [0, 0], [1e9, 1e9], [0, 0], [1e9, 1e9])
    cls = np.zeros(spec.shape, np.uint16)
    rows = (60, 220)
    rcv = np.zeros(spec.shape, np.uint8)
    rcv[rows[0], 128] = rcv[rows[1], 128] = 1
    delay = {}
    exact = (rows[1] - rows[0]) * spec.dx / 1540.0
    for to in (2, 4):
        m = fw.Medium.from_classes(spec.shape, spec.dx, spec.maps["c"], spec.maps["rho"], cls, [lossless],
                                   dt=spec.dt, pml=spec.pml, f0=spec.f0, time_order=to)
        m.set_sources(spec.src_mask, spec.src_waves)
        m.set_receivers(rcv, spec.n_steps)
        m.run(spec.n_steps)
        tr = m.receivers(f64=True)
        m.close()
        n = 1 << 14
        f = np.fft.rfftfreq(n, spec.dt)
        P1, P2 = np.fft.rfft(tr[0], n), np.fft.rfft(tr[1], n)
        k = np.argmin(np.abs(f - spec.f0))
        ph = np.angle(P2[k] * np.conj(P1[k]))          # -2 pi f delay, wrapped
        w = 2 * np.pi * f[k]
        cycles = np.round((w * exact + ph) / (2 * np.pi))    # whole periods from the nominal delay
        delay[to] = (2 * np.pi * cycles - ph) / w
    err = {to: abs(d - exact) / exact for to, d in delay.items()}
    print("relative travel-time error at f0: leapfrog %.2e, time-space %.2e" % (err[2], err[4]))
    assert err[4] < err[2] / 5
