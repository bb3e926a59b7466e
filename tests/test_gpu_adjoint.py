"""GPU adjoint (fw_gradient): gradients of a receiver functional with respect
to c(x) and alpha0(x) against the FP64 oracle's discrete adjoint and against
central finite differences of the GPU forward run.

Tolerances (relative L2 over the whole gradient map unless stated):
* FP64 build of the kernels vs the oracle: 1e-12 (same arithmetic up to the
  order of rounding; the forward parity floor is 2e-10);
* FP32 kernels vs the FP64 oracle: 1e-4 (the stated target);
* finite differences (FP64 forward, h = 1e-5 relative, truncation ~h^2):
  each voxel within 1e-5 of the largest gradient magnitude plus 1e-4 of its
  own; the FP32 gradient within 1e-3 of the largest magnitude."""
import numpy as np
import pytest

from gpu_util import oracle_params, rel_l2, to_c
from oracle.adjoint import misfit_gradient
from synthetic import config_c5, gaussian_pulse, plane_amplitude_rate

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


def _problem(shape, seed, n_steps=160, pml=6):
    rng = np.random.default_rng(seed)
    params = [oracle_params(0.6, 1.2, 2), oracle_params(1.0, 1.6, 2), oracle_params(0.0, 1.0, 2)]
    a0 = np.array([0.6, 1.0, 0.0])
    f0 = 3e6
    dx = 1540.0 / (f0 * 10)
    dt = 0.3 * dx / 1650.0
    c = (1500 + 60 * rng.uniform(size=shape)).astype(np.float32)
    rho = (950 + 100 * rng.uniform(size=shape)).astype(np.float32)
    cls = rng.integers(0, 3, size=shape).astype(np.uint16)
    src = np.zeros(shape, np.uint8)
    src[(pml + 2,) + tuple(n // 2 for n in shape[1:])] = 1
    rcv = np.zeros(shape, np.uint8)
    idx = tuple([shape[0] - pml - 3] + [slice(pml + 1, n - pml - 1, 3) for n in shape[1:]])
    rcv[idx] = 1
    w = gaussian_pulse(f0, dt, n_steps, 1e-7 if len(shape) == 2 else 1e-11)[None].astype(np.float32)
    G = rng.standard_normal((int(rcv.sum()), n_steps))
    return dict(shape=shape, dx=dx, dt=dt, c=c, rho=rho, cls=cls, params=params, a0=a0, src=src, rcv=rcv, w=w,
                G=G, pml=pml, f0=f0, n=n_steps)


def _gpu_grad(fw, P, storage, checkpoint=37, cls=None, params=None):
    cls = P["cls"] if cls is None else cls
    params = P["params"] if params is None else params
    m = fw.Medium.from_classes(P["shape"], P["dx"], P["c"], P["rho"], cls, [to_c(p, fw) for p in params],
                               dt=P["dt"], pml=P["pml"], f0=P["f0"], storage=storage)
    m.set_sources(P["src"], P["w"])
    m.set_receivers(P["rcv"], P["n"])
    f64 = storage == "f64"
    a0map = P["a0"][P["cls"]].astype(np.float64 if f64 else np.float32)
    gc, ga = m.gradient(P["n"], P["G"], alpha0=a0map, checkpoint=checkpoint, f64=f64)
    tr = m.receivers(f64=True)
    info = m.info()
    m.close()
    return gc.astype(np.float64), ga.astype(np.float64), tr, info


def _oracle_grad(P, checkpoint=50):
    return misfit_gradient(P["shape"], P["dx"], P["dt"], P["c"].astype(np.float64), P["rho"].astype(np.float64),
                           P["cls"].astype(np.int64), P["params"], P["a0"], P["n"], P["src"],
                           P["w"].astype(np.float64), P["rcv"], G=P["G"], pml=P["pml"], f0=P["f0"],
                           checkpoint=checkpoint)


@pytest.mark.parametrize("shape", [(48, 41), (100, 150), (20, 18, 23)])
def test_gradient_matches_oracle(fw, shape):
    """Random class map (two lossy classes and a lossless one), absorbing
    layer, point source, receiver line; FP64 and FP32 kernels against the
    oracle's FP64 discrete adjoint; the run leaves the medium at the end of
    the window with the traces of a plain run.  The 100 x 150 grid spans
    several tiles of the 2D reverse-step kernel along both axes, with ragged
    last tiles (320 steps: the direct wave reaches its receivers 83 cells
    from the source)."""
    n_steps = (320 if shape[0] == 100 else 160) if len(shape) == 2 else 90
    P = _problem(shape, seed=len(shape), n_steps=n_steps, pml=6 if len(shape) == 2 else 3)
    orc = _oracle_grad(P)
    assert np.abs(orc["grad_c"]).max() > 0 and np.abs(orc["grad_alpha0"]).max() > 0
    for storage, tol in (("f64", 1e-12), ("f32", 1e-4)):
        gc, ga, tr, info = _gpu_grad(fw, P, storage)
        ec, ea = rel_l2(gc, orc["grad_c"]), rel_l2(ga, orc["grad_alpha0"])
        print("\n%s %s: grad_c rel L2 %.2e, grad_alpha0 rel L2 %.2e" % (shape, storage, ec, ea))
        assert ec < tol and ea < tol, (storage, ec, ea)
        assert info["step"] == P["n"]
        assert rel_l2(tr, orc["traces"]) < (2e-10 if storage == "f64" else 1e-5)


@pytest.mark.parametrize("shape", [(60, 52), (18, 16, 20)])
def test_gradient_receiver_on_the_source_cell(fw, shape):
    """A receiver on the source cell and one beside it: the transpose of the
    combined injection and recording adds that receiver's adjoint before the
    source-gain term reads the pressure adjoint there."""
    n_steps = 140 if len(shape) == 2 else 80
    P = _problem(shape, seed=11, n_steps=n_steps, pml=6 if len(shape) == 2 else 3)
    at_src = tuple(int(i[0]) for i in np.nonzero(P["src"]))
    beside = (at_src[0] + 1,) + at_src[1:]
    P["rcv"][at_src] = 1
    P["rcv"][beside] = 1
    P["G"] = np.random.default_rng(12).standard_normal((int(P["rcv"].sum()), n_steps))
    orc = _oracle_grad(P)
    for storage, tol in (("f64", 1e-12), ("f32", 1e-4)):
        gc, ga, tr, _ = _gpu_grad(fw, P, storage)
        ec, ea = rel_l2(gc, orc["grad_c"]), rel_l2(ga, orc["grad_alpha0"])
        print("\n%s %s: grad_c rel L2 %.2e, grad_alpha0 rel L2 %.2e" % (shape, storage, ec, ea))
        assert ec < tol and ea < tol, (storage, ec, ea)
        assert rel_l2(tr, orc["traces"]) < (2e-10 if storage == "f64" else 1e-5)


def test_gradient_checkpoint_interval_does_not_matter(fw):
    P = _problem((40, 36), seed=7, n_steps=120)
    ref = _gpu_grad(fw, P, "f64", checkpoint=120)
    for k in (1, 13, 50):
        gc, ga, _, _ = _gpu_grad(fw, P, "f64", checkpoint=k)
        # the fold onto the user's grid adds with FP64 atomics (order free)
        assert np.allclose(gc, ref[0], rtol=1e-12, atol=0) and np.allclose(ga, ref[1], rtol=1e-12, atol=0), k


def test_c5_gradient_vs_finite_differences_and_oracle(fw):
    """Adjoint workload: 1024^2 Voronoi medium (6 classes, N = 3), 64
    receivers, 3000 steps, checkpoint every 100; misfit 1/2 |traces - d_obs|^2
    with d_obs from the perturbed medium (c +1 %, alpha0 +20 % in a Gaussian
    blob; the alpha0 factor on every d of the class, in 64 levels).  The FP32 and FP64 gradients at 32 seeded voxels against central
    differences of the FP64 forward run (c: the voxel's c; alpha0: the voxel
    gets its own class with every d scaled, the reading of fw_gradient)."""
    import time
    spec = config_c5()
    true = config_c5(perturbed=True)
    params = [oracle_params(a, y, 3) for a, y in zip(spec.classes["alpha0"], spec.classes["y"])]
    cp = [to_c(p, fw) for p in params]
    cls = spec.maps["class_idx"]
    a0c = np.asarray(spec.classes["alpha0"], np.float64)

    def medium(c, storage, cls_map=cls, classes=cp):
        m = fw.Medium.from_classes(spec.shape, spec.dx, c, spec.maps["rho"], cls_map, classes, dt=spec.dt,
                                   pml=spec.pml, f0=spec.f0, storage=storage)
        m.set_sources(spec.src_mask, spec.src_waves)
        m.set_receivers(spec.rcv_mask, spec.n_steps)
        return m

    # observed data: the perturbed medium, c +1 % and alpha0 +20 % in the blob.  The alpha0 factor
    # s(x) = alpha0_true(x) / alpha0_class scales every d of the voxel's class (the reading of
    # fw_gradient); s is quantised to 64 levels across its range, one class per (class, level).
    levels = 64
    s_true = np.where(a0c[cls] > 0, true.maps["alpha0"].astype(np.float64) / np.maximum(a0c[cls], 1e-30), 1.0)
    lev = np.clip(np.rint((s_true - 1.0) / 0.2 * (levels - 1)), 0, levels - 1).astype(np.int64)
    assert lev.max() >= levels - 8   # the blob's centre reaches the top levels
    blob_classes = []
    for q in params:
        for lv in range(levels):
            sc = 1.0 + 0.2 * lv / (levels - 1)
            blob_classes.append(fw.relax_params(q.kappa1, q.kappa2, [x * sc for x in q.d1], q.alpha1,
                                                [x * sc for x in q.d2], q.alpha2))
    mt = medium(true.maps["c"], "f64", cls_map=(cls.astype(np.int64) * levels + lev).astype(np.uint16),
                classes=blob_classes)
    mt.run(spec.n_steps)
    d_obs = mt.receivers(f64=True)
    mt.close()

    def misfit(c, storage="f64", cls_map=cls, classes=cp):
        m = medium(c, storage, cls_map, classes)
        m.run(spec.n_steps)
        r = m.receivers(f64=True) - d_obs
        m.close()
        return 0.5 * float(np.sum(r * r)), r

    L0, resid = misfit(spec.maps["c"])
    grads = {}
    for storage in ("f64", "f32"):
        m = medium(spec.maps["c"], storage)
        t0 = time.perf_counter()
        gc, ga = m.gradient(spec.n_steps, resid, alpha0=a0c[cls], checkpoint=100, f64=True)
        grads[storage] = (gc, ga, time.perf_counter() - t0)
        m.close()
    print("\nC5 gradient time: f64 %.2f s, f32 %.2f s" % (grads["f64"][2], grads["f32"][2]))
    rng = np.random.default_rng(44)
    n = spec.shape[0]
    w = spec.pml + 8
    cmax = float(spec.maps["c"].max())
    picks = []
    while len(picks) < 32:
        v = (int(rng.integers(w, n - w)), int(rng.integers(w, n - w)))
        if spec.maps["c"][v] * 1.001 < cmax and a0c[cls[v]] > 0 and v not in picks:
            picks.append(v)
    h = 1e-5
    gmax_c = np.abs(grads["f64"][0]).max()
    gmax_a = np.abs(grads["f64"][1]).max()
    worst = {"c64": 0.0, "a64": 0.0, "c32": 0.0, "a32": 0.0}
    for v in picks:
        c1, c2 = spec.maps["c"].copy(), spec.maps["c"].copy()
        c1[v] = np.float32(spec.maps["c"][v] * (1 + h))
        c2[v] = np.float32(spec.maps["c"][v] * (1 - h))
        fd_c = (misfit(c1)[0] - misfit(c2)[0]) / (float(c1[v]) - float(c2[v]))
        k = int(cls[v])
        cl2 = cls.copy()
        cl2[v] = len(cp)
        fds = []
        for sgn in (1, -1):
            q = params[k]
            sc = 1 + sgn * h
            extra = fw.relax_params(q.kappa1, q.kappa2, [x * sc for x in q.d1], q.alpha1, [x * sc for x in q.d2],
                                    q.alpha2)
            fds.append(misfit(spec.maps["c"], cls_map=cl2, classes=cp + [extra])[0])
        fd_a = (fds[0] - fds[1]) / (2 * h * a0c[k])
        for key, fd, g, gm in (("c64", fd_c, grads["f64"][0][v], gmax_c), ("a64", fd_a, grads["f64"][1][v], gmax_a),
                               ("c32", fd_c, grads["f32"][0][v], gmax_c), ("a32", fd_a, grads["f32"][1][v], gmax_a)):
            worst[key] = max(worst[key], abs(g - fd) / gm)
            tol = 1e-5 * gm + 1e-4 * abs(fd) if key.endswith("64") else 1e-3 * gm
            assert abs(g - fd) <= tol, (key, v, g, fd, gm)
    print("C5 finite differences, worst |grad - fd| / max|grad|: %s" % {k: "%.1e" % x for k, x in worst.items()})
    e = rel_l2(grads["f32"][0], grads["f64"][0]), rel_l2(grads["f32"][1], grads["f64"][1])
    print("C5 FP32 vs FP64 gradient rel L2: c %.2e alpha0 %.2e" % e)
    assert max(e) < 1e-4


def test_autograd_function_matches_fw_gradient(fw):
    import torch
    from paper_2606_11103_gb300.autograd import simulate
    P = _problem((40, 44), seed=9, n_steps=120)
    setup = dict(shape=P["shape"], dx=P["dx"], dt=P["dt"], rho=P["rho"], n_steps=P["n"], src_mask=P["src"],
                 waves=P["w"], rcv_mask=P["rcv"], pml=P["pml"], f0=P["f0"], storage="f64",
                 classes=(P["cls"], [to_c(p, fw) for p in P["params"]], P["a0"]), checkpoint=30)
    c = torch.tensor(P["c"], dtype=torch.float32, device="cuda", requires_grad=True)
    a0 = torch.tensor(P["a0"][P["cls"]], dtype=torch.float64, device="cuda", requires_grad=True)
    tr = simulate(c, a0, setup)
    G = torch.tensor(P["G"], device="cuda")
    (tr * G).sum().backward()
    gc, ga, _, _ = _gpu_grad(fw, P, "f64", checkpoint=30)
    assert c.grad.dtype == torch.float32 and a0.grad.dtype == torch.float64
    assert torch.allclose(c.grad.double().cpu(), torch.from_numpy(gc).float().double(), rtol=1e-6, atol=0)
    assert np.allclose(a0.grad.cpu().numpy(), ga, rtol=1e-12, atol=0)
