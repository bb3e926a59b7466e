"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Tolerances (relative L2 over the field / traces;
velocity components share the largest component's norm):

* FP32 arithmetic: 1e-5, the stated target.
* FP64 build of the same kernels: 2e-10.  This is the rounding floor, not a
  loosened target: perturbing the oracle's own K dt and dt/rho by one ulp
  moves its 1000-step 256^2 result by 9.6e-12 (p) and 7.2e-11 (v), the same
  size as the GPU-vs-oracle differences, because the phase error of a
  one-ulp speed change grows with the distance travelled."""
import numpy as np
import pytest

from gpu_util import Pair, oracle_params, rel_l2, to_c
from synthetic import config_c1, config_c2, config_c3, config_c5, gaussian_pulse, voronoi_classes, voronoi_medium

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 2e-10}


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


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_c1_homogeneous_2d_1000_steps(fw, storage):
    """256^2, N=2, 20-cell PML, line source, centre-column receivers, 1000 steps."""
    spec = config_c1()
    prm = oracle_params(0.5, 1.1, 2)
    cls = np.zeros(spec.shape, np.uint16)
    pr = Pair(fw, spec.shape, spec.dx, spec.dt, spec.maps["c"], spec.maps["rho"], cls, [prm],
              pml=spec.pml, f0=spec.f0, storage=storage)
    pr.sources(spec.src_mask, spec.src_waves)
    pr.receivers(spec.rcv_mask, spec.n_steps)
    _check(pr.run_compare(spec.n_steps, checks=4, f64=storage == "f64"), TOL[storage])


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_c2_two_layer_nonlinear_crop(fw, storage):
    """Two-layer medium (N=4 per layer, beta 3.5 / 6, 30-cell PML) on a
    cropped grid with a ragged x extent, 1 MPa source for the nonlinear term."""
    spec = config_c2(n=320, n_steps=500, amp=1e6)
    shape = (320, 301)
    maps = {k: np.ascontiguousarray(v[:, :301]) for k, v in spec.maps.items()}
    cls = (np.arange(320)[:, None] >= 160).astype(np.uint16) * np.ones(shape, np.uint16)
    params = [oracle_params(1.09, 1.0, 4), oracle_params(0.6, 1.5, 4)]
    pr = Pair(fw, shape, spec.dx, spec.dt, maps["c"], maps["rho"], cls, params, beta=maps["beta"],
              pml=spec.pml, f0=spec.f0, storage=storage)
    pr.sources(np.ascontiguousarray(spec.src_mask[:, :301]), spec.src_waves)
    rcv = np.ascontiguousarray(spec.rcv_mask[:, :301])
    pr.receivers(rcv, 500)
    _check(pr.run_compare(500, f64=storage == "f64"), TOL[storage])


@pytest.mark.parametrize("shape", [(80, 72), (24, 30, 28)])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_receivers_on_source_cells(fw, shape, storage):
    """Injection and recording share one launch: receivers on some source
    cells record p after the injection (as the oracle does), receivers beside
    them record as usual, every second step (decimation 2), and the waveform
    ends before the run does (the last 60 steps record without injection)."""
    f0 = 3e6
    dx = 1540.0 / (f0 * 12)
    one = np.ones(shape, np.float32)
    dt = 0.3 * dx / 1540.0
    n_steps = 200
    src = np.zeros(shape, np.uint8)
    src[(8,) + tuple(slice(4, n - 4) for n in shape[1:])] = 1
    rcv = np.zeros(shape, np.uint8)
    rcv[(8,) + tuple(slice(2, n - 2, 3) for n in shape[1:])] = 1      # on and beside the source cells
    rcv[(shape[0] - 9,) + tuple(slice(2, n - 2, 5) for n in shape[1:])] = 1
    assert (src & rcv).sum() > 1 and (rcv & ~src).sum() > 1
    waves = gaussian_pulse(f0, dt, n_steps - 60, 1e-3 if len(shape) == 2 else 1e-6)[None].astype(np.float32)
    pr = Pair(fw, shape, dx, dt, 1540 * one, 1000 * one, np.zeros(shape, np.uint16), [oracle_params(0.5, 1.1, 2)],
              pml=6, f0=f0, storage=storage)
    pr.sources(src, waves)
    pr.receivers(rcv, n_steps, decim=2)
    _check(pr.run_compare(n_steps, f64=storage == "f64"), TOL[storage])


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_c3_voronoi_3d_crop(fw, storage):
    """96^3 crop of the 512^3 Voronoi map (8 classes, N=4, jittered c/rho),
    focused aperture source, 20-cell PML on the crop, 120 steps."""
    box = ((0, 96), (208, 304), (208, 304))
    spec = config_c3(n_steps=120, box=box)
    params = [oracle_params(a, y, 4) for a, y in zip(spec.classes["alpha0"], spec.classes["y"])]
    pr = Pair(fw, spec.shape, spec.dx, spec.dt, spec.maps["c"], spec.maps["rho"], spec.maps["class_idx"],
              params, pml=spec.pml, f0=spec.f0, storage=storage)
    pr.sources(spec.src_mask, spec.src_waves, spec.src_wave_of)
    pr.receivers(spec.rcv_mask, 120)
    _check(pr.run_compare(120, f64=storage == "f64"), TOL[storage])


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("shape,nmech,pml,lt", [((203, 157), 1, 12, 6), ((37, 45, 51), 3, 6, 3),
                                                 ((20, 19, 133), 2, 4, 0), ((9, 9, 9), 4, 2, 0)])
def test_ragged_shapes_and_transition(fw, storage, shape, nmech, pml, lt):
    """Shapes that are not multiples of the tiles, several mechanism counts,
    a transition layer, a random class map and a point source."""
    rng = np.random.default_rng(11)
    dx = 5e-5
    c = (1500 + 80 * rng.uniform(size=shape)).astype(np.float32)
    rho = (950 + 100 * rng.uniform(size=shape)).astype(np.float32)
    cls = rng.integers(0, 3, size=shape).astype(np.uint16)
    params = [oracle_params(a, y, nmech) for a, y in ((0.5, 1.1), (0.9, 1.6), (0.0, 1.0))]
    dt = 0.35 * dx / 1580.0
    pr = Pair(fw, shape, dx, dt, c, rho, cls, params, pml=pml, transition=lt, f0=3e6, storage=storage)
    src = np.zeros(shape, np.uint8)
    src[tuple(n // 2 for n in shape)] = 1
    nt = 150
    pr.sources(src, gaussian_pulse(3e6, dt, nt, 1e-9)[None].astype(np.float32))
    rcv = np.zeros(shape, np.uint8)
    rcv[tuple(n // 3 for n in shape)] = 1
    rcv[tuple(n - 2 for n in shape)] = 1
    pr.receivers(rcv, nt, 2)
    _check(pr.run_compare(nt, graphs=False, f64=storage == "f64"), TOL[storage])


def test_c5_voronoi_2d_crop(fw):
    spec = config_c5(n=256, n_steps=400)
    params = [oracle_params(a, y, 3) for a, y in zip(spec.classes["alpha0"], spec.classes["y"])]
    pr = Pair(fw, spec.shape, spec.dx, spec.dt, spec.maps["c"], spec.maps["rho"], spec.maps["class_idx"],
              params, pml=spec.pml, f0=spec.f0, storage="f32")
    pr.sources(spec.src_mask, spec.src_waves)
    pr.receivers(spec.rcv_mask, 400)
    _check(pr.run_compare(400), TOL["f32"])


def test_graph_run_equals_plain_steps(fw):
    spec = config_c1(n=128, n_steps=100)
    prm = oracle_params(0.5, 1.1, 2)
    cls = np.zeros(spec.shape, np.uint16)
    outs = []
    for graphs in (True, False):
        m = fw.Medium.from_classes(spec.shape, spec.dx, spec.maps["c"], spec.maps["rho"], cls,
                                   [fw.relax_params(prm.kappa1, prm.kappa2, prm.d1, prm.alpha1, prm.d2, prm.alpha2)],
                                   dt=spec.dt, pml=spec.pml, f0=spec.f0)
        m.set_sources(spec.src_mask, spec.src_waves)
        m.set_receivers(spec.rcv_mask, 100)
        (m.run if graphs else m.step)(100)
        outs.append((m.read_field(0), m.receivers()))
        m.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_checkpoint_resume_bit_exact(fw):
    spec = config_c1(n=96, n_steps=200)
    prm = oracle_params(0.5, 1.1, 2)
    cp = fw.relax_params(prm.kappa1, prm.kappa2, prm.d1, prm.alpha1, prm.d2, prm.alpha2)
    cls = np.zeros(spec.shape, np.uint16)

    def new():
        m = fw.Medium.from_classes(spec.shape, spec.dx, spec.maps["c"], spec.maps["rho"], cls, [cp],
                                   dt=spec.dt, pml=spec.pml, f0=spec.f0)
        m.set_sources(spec.src_mask, spec.src_waves)
        return m

    a = new()
    a.run(200)
    b = new()
    b.run(90)
    img = b.save_state()
    b.close()
    c = new()
    c.load_state(img)
    assert c.info()["step"] == 90
    c.run(110)
    assert np.array_equal(a.read_field(0), c.read_field(0))
    for d in range(2):
        assert np.array_equal(a.read_field(1, d), c.read_field(1, d))


def test_field_roundtrip_and_zero_steps(fw):
    shape = (33, 70)
    rng = np.random.default_rng(2)
    m = fw.Medium.from_classes(shape, 1e-4, np.full(shape, 1540, np.float32), np.full(shape, 1000, np.float32),
                               np.zeros(shape, np.uint16), [fw.relax_params(1, 1, [0], [1e9], [0], [1e9])],
                               dt=2e-8, pml=4)
    x = rng.standard_normal(shape).astype(np.float32)
    m.write_field(0, 0, x)
    assert np.array_equal(m.read_field(0), x)
    m.run(0)
    assert np.array_equal(m.read_field(0), x)
    m.close()


def test_monitor_flags_nonfinite(fw):
    """A non-finite value written into p is caught by the stability monitor
    of the next step and the error is sticky (Sec. 4.6 instability check)."""
    shape = (40, 40)
    m = fw.Medium.from_classes(shape, 1e-4, np.full(shape, 1540, np.float32), np.full(shape, 1000, np.float32),
                               np.zeros(shape, np.uint16), [fw.relax_params(1, 1, [0], [1e9], [0], [1e9])],
                               dt=2e-8, pml=4)
    x = np.zeros(shape, np.float32)
    x[20, 20] = 1.0
    m.write_field(0, 0, x)
    m.run(3)
    rc, pmax = m.status()
    assert rc == 0 and 0 < pmax < 2
    x[20, 20] = np.nan
    m.write_field(0, 0, x)
    m.run(1)
    rc, _ = m.status()
    assert rc == fw.FW_ERR_UNSTABLE
    with pytest.raises(fw.FwError):
        m.run(1)
    m.close()


def test_rejects_bad_inputs(fw):
    shape = (16, 16)
    one = np.ones(shape, np.float32)
    cls = np.zeros(shape, np.uint16)
    lossless = [fw.relax_params(1, 1, [0], [1e9], [0], [1e9])]
    with pytest.raises(fw.FwError):       # CFL above the 2D limit (0.5497)
        fw.Medium.from_classes(shape, 1e-4, one * 1540, one * 1000, cls, lossless, dt=0.6 * 1e-4 / 1540)
    with pytest.raises(fw.FwError):       # non-positive density
        fw.Medium.from_classes(shape, 1e-4, one * 1540, one * 0, cls, lossless, dt=1e-8)
    with pytest.raises(fw.FwError):       # class index out of range
        fw.Medium.from_classes(shape, 1e-4, one * 1540, one * 1000, cls + 3, lossless, dt=1e-8)
    m = fw.Medium.from_classes(shape, 1e-4, one * 1540, one * 1000, cls, lossless, cfl=0.5)
    assert abs(m.info()["dt"] - 0.5 * 1e-4 / 1540) < 1e-15
    m.close()


def test_create_from_maps_fits_each_class(fw):
    """fw_create_medium: distinct (alpha0, y) pairs become classes fitted on
    the host with the class's mean c as c0."""
    shape = (24, 40)
    spec_c = np.full(shape, 1540, np.float32)
    a0 = np.full(shape, 0.5, np.float32)
    y = np.full(shape, 1.1, np.float32)
    a0[12:] = 0.0
    m = fw.Medium.from_maps(shape, 1e-4, spec_c, spec_c * 0 + 1000, a0, y, n_mech=2, dt=2e-8, pml=4,
                            maxiter=300, w=(0.5,))
    assert m.info()["n_classes"] == 2
    m.run(10)
    assert m.status()[0] == 0
    m.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_tma_staging_equals_cp_async_staging(fw, storage, monkeypatch):
    """The 3D sweeps stage their streams by TMA; FWGB_NO_TMA=1 at medium
    creation selects the per-thread cp.async staging instead.  Both feed the
    same arithmetic, so the fields after 150 steps (the pulse well under way)
    agree bitwise (ragged crop: partial tiles in x and y, both halo edges)."""
    box = ((0, 40), (230, 283), (221, 290))
    spec = config_c3(n_steps=150, box=box)
    params = [oracle_params(a, y, 4) for a, y in zip(spec.classes["alpha0"], spec.classes["y"])]
    out = []
    for no_tma in ("0", "1"):
        monkeypatch.setenv("FWGB_NO_TMA", no_tma)
        m = fw.Medium.from_classes(spec.shape, spec.dx, spec.maps["c"], spec.maps["rho"], spec.maps["class_idx"],
                                   [to_c(p, fw) for p in params], dt=spec.dt, pml=8, f0=spec.f0, storage=storage)
        m.set_sources(spec.src_mask, spec.src_waves, spec.src_wave_of)
        m.run(150)
        out.append([m.read_field(0, 0)] + [m.read_field(1, d) for d in range(3)] + [m.read_field(3, 1)])
        assert m.status()[0] == 0
        m.close()
    assert np.abs(out[0][0]).max() > 0
    for name, a, b in zip(("p", "v0", "v1", "v2", "psi2"), *out):
        d = np.abs(a.astype(np.float64) - b)
        print(name, "max |TMA - cp.async| %.3e at %s of max %.3e" % (d.max(), np.unravel_index(d.argmax(), d.shape),
                                                                    np.abs(b).max()))
    for a, b in zip(*out):
        assert np.array_equal(a, b)
