"""Pins of the oracle's discrete adjoint (gradients with respect to c(x) and
alpha0(x)): the transpose identity of one time step, the closed-form
derivatives of the recursion coefficients, and central finite differences
of the oracle's own forward run."""
import math

import numpy as np
import pytest

from oracle import fit
from oracle.adjoint import Adjoint, _Snapshot, misfit_gradient, recursion_ab_dscale
from oracle.medium import OracleMedium, recursion_ab
from oracle.stepper import OracleSim
from synthetic import gaussian_pulse, plane_amplitude_rate


def _params():
    # two tissue classes and a lossless one (cheap fits; exact values do not matter here)
    p1, _ = fit.fit_relaxation(0.6, 1.2, 2, maxiter=200, w_list=(0.5,))
    p2, _ = fit.fit_relaxation(1.0, 1.6, 2, maxiter=200, w_list=(0.5,))
    return [p1, p2, fit.RelaxParams.lossless(2)], np.array([0.6, 1.0, 0.0])


def _states(sim):
    """Every state array of a simulator (or snapshot), in a fixed order."""
    out = [sim.p] + list(sim.v)
    out += [a for row in sim.psi1 for a in row] + [a for row in sim.psi2 for a in row]
    out += [a for a in list(sim.psi1p) + list(sim.psi2p) if a is not None]
    return out


def _dot(a, b):
    return sum(float(np.sum(x * y)) for x, y in zip(_states(a), _states(b)))


def test_recursion_derivatives_match_central_differences():
    rng = np.random.default_rng(0)
    d = 10 ** rng.uniform(2, 10, 50)
    al = 10 ** rng.uniform(5, 12, 50)
    ka = rng.uniform(0.98, 1.0, 50)
    dt = 1e-8
    for s in (1.0, 0.7, 1.3):
        da, db = recursion_ab_dscale(d, al, ka, dt, s)
        # fourth-order central difference: truncation ~h^4, rounding ~eps/h
        h = 1e-3
        ev = [recursion_ab(d * (s + k * h), al, ka, dt) for k in (-2, -1, 1, 2)]
        fd = [(e0 - 8 * e1 + 8 * e2 - e3) / (12 * h) for e0, e1, e2, e3 in zip(*ev)]
        np.testing.assert_allclose(da, fd[0], rtol=1e-7, atol=1e-12)
        np.testing.assert_allclose(db, fd[1], rtol=1e-7, atol=1e-12)


@pytest.mark.parametrize("shape,pml,periodic", [((30, 26), 5, None), ((14, 12, 16), 3, None),
                                                ((24, 20), 4, (False, True))])
def test_adjoint_step_is_the_transpose(shape, pml, periodic, oracle_lib):
    """<M du, lam> = <du, M^T lam> for one time step M of the linear system
    (all state arrays random, heterogeneous c, rho, classes, absorbing layer)."""
    rng = np.random.default_rng(1)
    params, _ = _params()
    dx = 5e-5
    c = 1500 + 80 * rng.uniform(size=shape)
    rho = 950 + 100 * rng.uniform(size=shape)
    cls = rng.integers(0, 3, size=shape)
    dscale = rng.uniform(0.5, 1.5, size=shape)
    med = OracleMedium(shape, dx, 0.3 * dx / 1580, c, rho, cls, params, pml=pml, f0=3e6, periodic=periodic,
                       dscale=dscale)
    sim = OracleSim(med)
    adj = Adjoint(sim)
    for a in _states(sim):
        a[...] = rng.standard_normal(a.shape)
    du = _Snapshot(sim)
    sim.run(1)
    Mdu = _Snapshot(sim)
    lam = adj.zero_like_state()
    for a in _states(lam):
        a[...] = rng.standard_normal(a.shape)
    lam0 = _Snapshot.__new__(_Snapshot)
    lam0.__dict__ = {k: (v.copy() if isinstance(v, np.ndarray) else
                         [[x.copy() for x in r] if isinstance(r, list) else (None if r is None else r.copy())
                          for r in v] if isinstance(v, list) else v)
                     for k, v in lam.__dict__.items()}
    gk = np.zeros(shape)
    gs = np.zeros(shape)
    adj.step_transpose(du, Mdu.v, lam, gk, gs)
    lhs = _dot(Mdu, lam0)
    rhs = _dot(du, lam)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def _small_problem(shape=(40, 36), pml=6, n_steps=160, seed=3):
    rng = np.random.default_rng(seed)
    params, a0 = _params()
    f0 = 3e6
    dx = 1540.0 / (f0 * 10)
    dt = 0.3 * dx / 1650.0
    c = (1500 + 60 * rng.uniform(size=shape)).astype(np.float32).astype(np.float64)
    rho = 950 + 100 * rng.uniform(size=shape)
    cls = np.zeros(shape, np.int64)
    cls[shape[0] // 2:] = 1
    cls[:, : shape[1] // 4] = 2
    src = np.zeros(shape, np.uint8)
    src[pml + 2, pml:-pml] = 1
    rcv = np.zeros(shape, np.uint8)
    rcv[pml + 6, pml + 3::5] = 1
    rcv[shape[0] - pml - 3, pml + 2::4] = 1
    w = gaussian_pulse(f0, dt, n_steps, plane_amplitude_rate(1e3, dx, 2, 1000.0, 1540.0))[None]
    G = rng.standard_normal((int(rcv.sum()), n_steps))
    return dict(shape=shape, dx=dx, dt=dt, c=c, rho=rho, cls=cls, params=params, a0=a0, src=src, rcv=rcv,
                w=w, G=G, pml=pml, f0=f0, n_steps=n_steps)


def _loss(P, c=None, dscale=None):
    med = OracleMedium(P["shape"], P["dx"], P["dt"], P["c"] if c is None else c, P["rho"], P["cls"], P["params"],
                       pml=P["pml"], f0=P["f0"], dscale=dscale)
    sim = OracleSim(med)
    sim.set_sources(P["src"], P["w"])
    sim.set_receivers(P["rcv"], P["n_steps"])
    sim.run(P["n_steps"])
    return float(np.sum(P["G"] * sim.traces))


def test_gradient_matches_central_differences(oracle_lib):
    """dL/dc and dL/dalpha0 of L = sum G * traces against central differences
    of the forward run at single voxels: interior voxels, a source-row voxel
    (volume-source gain), and a voxel on the inner edge of the absorbing
    layer (its value is inherited by the layer cells behind it)."""
    P = _small_problem()
    out = misfit_gradient(P["shape"], P["dx"], P["dt"], P["c"], P["rho"], P["cls"], P["params"], P["a0"],
                          P["n_steps"], P["src"], P["w"], P["rcv"], G=P["G"], pml=P["pml"], f0=P["f0"],
                          checkpoint=37)
    pml = P["pml"]
    voxels = [(20, 18), (12, 25), (pml + 2, 20), (pml, 30), (30, pml)]
    h = 1e-5
    for v in voxels:
        cp = P["c"].copy()
        cp[v] *= 1 + h
        cm = P["c"].copy()
        cm[v] *= 1 - h
        fd = (_loss(P, c=cp) - _loss(P, c=cm)) / (2 * h * P["c"][v])
        assert abs(fd - out["grad_c"][v]) <= 2e-6 * abs(fd) + 1e-12 * np.abs(out["grad_c"]).max(), (v, fd, out["grad_c"][v])
        if P["a0"][P["cls"][v]] > 0:
            sp = np.ones(P["shape"])
            sp[v] = 1 + h
            sm = np.ones(P["shape"])
            sm[v] = 1 - h
            a0 = P["a0"][P["cls"][v]]
            fd = (_loss(P, dscale=sp) - _loss(P, dscale=sm)) / (2 * h * a0)
            ga = out["grad_alpha0"][v]
            assert abs(fd - ga) <= 2e-6 * abs(fd) + 1e-12 * np.abs(out["grad_alpha0"]).max(), (v, fd, ga)


def test_gradient_directional_derivative_and_misfit(oracle_lib):
    """Along random smooth perturbations of c and of s, the directional
    derivative <grad, dm> equals the central difference of the misfit
    1/2 |traces - d_obs|^2 (all voxels at once), and the forward traces of
    the gradient run equal a plain forward run."""
    P = _small_problem(shape=(34, 30), pml=5, n_steps=140, seed=5)
    rng = np.random.default_rng(9)
    d_obs = rng.standard_normal(P["G"].shape) * 1e-3
    out = misfit_gradient(P["shape"], P["dx"], P["dt"], P["c"], P["rho"], P["cls"], P["params"], P["a0"],
                          P["n_steps"], P["src"], P["w"], P["rcv"], d_obs=d_obs, pml=P["pml"], f0=P["f0"],
                          checkpoint=50)

    def misfit(c=None, dscale=None):
        med = OracleMedium(P["shape"], P["dx"], P["dt"], P["c"] if c is None else c, P["rho"], P["cls"],
                           P["params"], pml=P["pml"], f0=P["f0"], dscale=dscale)
        sim = OracleSim(med)
        sim.set_sources(P["src"], P["w"])
        sim.set_receivers(P["rcv"], P["n_steps"])
        sim.run(P["n_steps"])
        return 0.5 * float(np.sum((sim.traces - d_obs) ** 2)), sim.traces

    L0, tr0 = misfit()
    assert np.array_equal(tr0, out["traces"])
    yy, xx = np.meshgrid(np.arange(P["shape"][0]), np.arange(P["shape"][1]), indexing="ij")
    bump = np.exp(-((yy - 17) ** 2 + (xx - 14) ** 2) / 40.0)
    h = 1e-5
    dc = 20.0 * bump
    # c_max (over the map with the absorbing layer inherited) sets the
    # absorbing profile, which the gradient holds fixed: leave the fastest
    # cell alone
    c_int = OracleMedium(P["shape"], P["dx"], P["dt"], P["c"], P["rho"], P["cls"], P["params"], pml=P["pml"]).c
    dc[P["c"] >= c_int.max()] = 0.0
    fd = (misfit(c=P["c"] + h * dc)[0] - misfit(c=P["c"] - h * dc)[0]) / (2 * h)
    an = float(np.sum(out["grad_c"] * dc))
    assert abs(fd - an) <= 1e-6 * abs(fd), (fd, an)
    ds = 0.3 * bump
    fd = (misfit(dscale=1 + h * ds)[0] - misfit(dscale=1 - h * ds)[0]) / (2 * h)
    an = float(np.sum(out["grad_s_user"] * ds))
    assert abs(fd - an) <= 1e-6 * abs(fd), (fd, an)


def test_gradient_3d_single_voxels(oracle_lib):
    rng = np.random.default_rng(4)
    shape = (20, 18, 16)
    params, a0 = _params()
    f0 = 3e6
    dx = 1540.0 / (f0 * 8)
    dt = 0.25 * dx / 1650.0
    c = 1500 + 60 * rng.uniform(size=shape)
    rho = 950 + 100 * rng.uniform(size=shape)
    cls = rng.integers(0, 2, size=shape)
    src = np.zeros(shape, np.uint8)
    src[5, 8, 7] = 1
    rcv = np.zeros(shape, np.uint8)
    rcv[14, 5:13:3, 4:12:3] = 1
    n = 90
    w = gaussian_pulse(f0, dt, n, 1e-9)[None]
    G = rng.standard_normal((int(rcv.sum()), n))
    out = misfit_gradient(shape, dx, dt, c, rho, cls, params, a0, n, src, w, rcv, G=G, pml=3, f0=f0, checkpoint=30)

    def loss(cc=c, ds=None):
        med = OracleMedium(shape, dx, dt, cc, rho, cls, params, pml=3, f0=f0, dscale=ds)
        sim = OracleSim(med)
        sim.set_sources(src, w)
        sim.set_receivers(rcv, n)
        sim.run(n)
        return float(np.sum(G * sim.traces))

    h = 1e-5
    for v in [(9, 8, 8), (12, 6, 9), (3, 8, 8)]:
        cp, cm = c.copy(), c.copy()
        cp[v] *= 1 + h
        cm[v] *= 1 - h
        fd = (loss(cp) - loss(cm)) / (2 * h * c[v])
        assert math.isclose(fd, out["grad_c"][v], rel_tol=2e-6), (v, fd, out["grad_c"][v])
        sp, sm = np.ones(shape), np.ones(shape)
        sp[v], sm[v] = 1 + h, 1 - h
        fd = (loss(ds=sp) - loss(ds=sm)) / (2 * h * a0[cls[v]])
        assert math.isclose(fd, out["grad_alpha0"][v], rel_tol=2e-6), (v, fd, out["grad_alpha0"][v])
