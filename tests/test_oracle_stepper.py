"""Pins of the FP64 oracle time stepper against closed forms and physics
(no GPU).  Each test derives its expectation independently of the oracle's
own code: Taylor weights from their defining linear system, exact discrete
plane waves and eigenmodes from the scheme's z-transform, energy identities,
the 2D Green's function, the paper's PML and attenuation bounds, and the
Fubini solution for the nonlinear term."""
import math

import numpy as np
import pytest

from oracle import fit, measure
from oracle.medium import OracleMedium, recursion_ab
from oracle.stepper import OracleSim
from synthetic import gaussian_pulse, plane_amplitude_rate


def taylor_weights(M=4):
    """Staggered first-derivative weights: sum_m c_m (2m-1)^(2j-1) = [j == 1]."""
    A = np.array([[(2 * m - 1) ** (2 * j - 1) for m in range(1, M + 1)] for j in range(1, M + 1)], float)
    b = np.zeros(M)
    b[0] = 1.0
    return np.linalg.solve(A, b)


def modified_wavenumber(k, dx):
    c = taylor_weights()
    return 2.0 * sum(c[m] * math.sin((2 * m + 1) * k * dx / 2) for m in range(4)) / dx


def sim_of(shape, dx, dt, c=1540.0, rho=1000.0, params=None, periodic=None, pml=0, transition=0,
           beta=None, f0=1e6, cls=None, layer_relax=False):
    params = params or [fit.RelaxParams.lossless(2)]
    cmap = np.broadcast_to(np.asarray(c, float), shape)
    rmap = np.broadcast_to(np.asarray(rho, float), shape)
    cls = np.zeros(shape, np.int64) if cls is None else cls
    med = OracleMedium(shape, dx, dt, cmap, rmap, cls, params, beta=beta, pml=pml,
                       transition=transition, f0=f0, periodic=periodic, layer_relax=layer_relax)
    return OracleSim(med)


# ---------------------------------------------------------------------------
# p1: finite-difference operator


@pytest.mark.parametrize("ndim,d", [(2, 0), (2, 1), (3, 0), (3, 1), (3, 2)])
def test_fd_polynomials_exact_to_degree_8(ndim, d, oracle_lib):
    n = 24
    shape = (n,) * ndim
    sim = sim_of(shape, 1.0, 1e-9)
    ax = ndim - 1 - d
    coord = np.arange(n, dtype=float) - n / 2
    sl = [None] * ndim
    sl[ax] = slice(None)
    interior = [slice(None)] * ndim
    interior[ax] = slice(4, n - 4)
    for k in range(0, 10):
        # D+ : input at integer points, output at i + 1/2
        f = np.broadcast_to((coord / 8.0)[tuple(sl)] ** k, shape).copy()
        dp = sim.dplus(f, d)
        xh = (coord + 0.5) / 8.0
        want_p = np.broadcast_to((k * xh ** max(k - 1, 0) / 8.0 * (k > 0))[tuple(sl)], shape)
        # D- : input at half points j + 1/2, output at integer points
        g = np.broadcast_to(((coord + 0.5) / 8.0)[tuple(sl)] ** k, shape).copy()
        dm = sim.dminus(g, d)
        xi = coord / 8.0
        want_m = np.broadcast_to((k * xi ** max(k - 1, 0) / 8.0 * (k > 0))[tuple(sl)], shape)
        err_p = np.max(np.abs(dp[tuple(interior)] - want_p[tuple(interior)]))
        err_m = np.max(np.abs(dm[tuple(interior)] - want_m[tuple(interior)]))
        if k <= 8:
            assert err_p < 1e-11 and err_m < 1e-11, (k, err_p, err_m)
        else:
            assert err_p > 1e-8          # exactly 8th order: degree 9 is not exact


def test_fd_weights_are_the_taylor_weights(oracle_lib):
    """D+ sin(kx) at x+1/2 must be K_d cos(k(x+1/2)) with K_d built from the
    independently solved Taylor weights (periodic wrap included)."""
    n, dx = 32, 2e-4
    sim = sim_of((4, n), dx, 1e-9, periodic=(True, True))
    x = np.arange(n) * dx
    for m in (1, 3, 7, 15):
        k = 2 * math.pi * m / (n * dx)
        f = np.broadcast_to(np.sin(k * x), (4, n)).copy()
        dp = sim.dplus(f, 0)
        np.testing.assert_allclose(dp[0], modified_wavenumber(k, dx) * np.cos(k * (x + dx / 2)),
                                   atol=1e-9 * abs(modified_wavenumber(k, dx)))


def test_source_and_receiver_convention(oracle_lib):
    """Step n adds gain*wave[n] after the update, gain = dt K / dx^D, and
    records p^(n+1) at every decim-th step."""
    shape = (12, 12)
    dx, dt = 1e-4, 2e-8
    sim = sim_of(shape, dx, dt)
    src = np.zeros(shape, np.uint8)
    src[6, 5] = 1
    sim.set_sources(src, np.array([[3.0, -1.0, 0.5, 2.0]]))
    sim.set_receivers(src, 4, 1)
    sim.run(1)
    K = 1000.0 * 1540.0 ** 2
    g = dt * K / dx ** 2
    assert sim.p[6, 5] == pytest.approx(3.0 * g, rel=1e-15)
    assert sim.traces[0, 0] == sim.p[6, 5]
    assert np.count_nonzero(sim.p) == 1


# ---------------------------------------------------------------------------
# p2: lossless stepper


def _plane_wave_check(shape, dx, modes, kappa=(1.0, 1.0), n_steps=600):
    c, rho = 1500.0, 1100.0
    nd = len(shape)
    dt = 0.3 * dx / c
    p0 = fit.RelaxParams(kappa[0], kappa[1], np.zeros(2), np.full(2, 1e9), np.zeros(2), np.full(2, 1e9))
    sim = sim_of(shape, dx, dt, c, rho, params=[p0], periodic=(True,) * nd)
    kvec = [2 * math.pi * m / (shape[nd - 1 - d] * dx) for d, m in enumerate(modes)]
    Kd = [modified_wavenumber(k, dx) for k in kvec]
    ceff = c / math.sqrt(kappa[0] * kappa[1])
    om = 2.0 / dt * math.asin(0.5 * dt * ceff * math.sqrt(sum(K * K for K in Kd)))
    grids = np.meshgrid(*[np.arange(n) * dx for n in shape], indexing="ij")
    pos = [grids[nd - 1 - d] for d in range(nd)]          # pos[d] = coordinate along d
    phase = sum(k * x for k, x in zip(kvec, pos))
    sim.p[...] = np.cos(phase)
    s = math.sin(om * dt / 2)
    for d in range(nd):
        A = dt * Kd[d] / (kappa[0] * 2 * rho * s)
        sim.v[d][...] = A * np.cos(phase + kvec[d] * dx / 2 + om * dt / 2)
    sim.run(n_steps)
    want = np.cos(phase - om * n_steps * dt)
    return np.max(np.abs(sim.p - want))


def test_lossless_plane_wave_exact_2d(oracle_lib):
    assert _plane_wave_check((16, 32), 1e-4, (3, 2)) < 1e-10


def test_lossless_plane_wave_exact_2d_kappa(oracle_lib):
    # the 1/kappa factors of both stretches change the speed to c/sqrt(k1 k2)
    assert _plane_wave_check((8, 40), 1e-4, (5, 1), kappa=(0.99, 0.985)) < 1e-10


def test_lossless_plane_wave_exact_3d(oracle_lib):
    assert _plane_wave_check((8, 8, 16), 1e-4, (2, 1, 3), n_steps=300) < 1e-10


def test_energy_conserved_lossless_heterogeneous(oracle_lib):
    """E = sum p^2/(2K) + sum rho_f v^(n-1/2) v^(n+1/2)/2 is an exact invariant
    of the staggered leapfrog (summation by parts), with zero boundaries."""
    rng = np.random.default_rng(3)
    shape = (20, 24)
    dx = 1e-4
    c = 1500 + 100 * rng.uniform(size=shape)
    rho = 1000 + 200 * rng.uniform(size=shape)
    dt = 0.4 * dx / c.max()
    sim = sim_of(shape, dx, dt, c, rho)
    sim.p[...] = rng.standard_normal(shape)
    K = rho * c * c
    rho_f = [dt / sim.med.dt_rho[d] for d in range(2)]

    def energy(v_old):
        return np.sum(sim.p ** 2 / (2 * K)) + sum(np.sum(rho_f[d] * v_old[d] * sim.v[d]) / 2 for d in range(2))

    E = []
    for _ in range(300):
        v_old = [v.copy() for v in sim.v]     # v^(n-1/2); p holds p^n
        p_n = sim.p.copy()
        sim.run(1)                             # -> v^(n+1/2), p^(n+1)
        p_next = sim.p.copy()
        sim.p[...] = p_n
        E.append(energy(v_old))
        sim.p[...] = p_next
    E = np.array(E)
    assert np.max(np.abs(E - E[0])) < 1e-12 * E[0]


# ---------------------------------------------------------------------------
# p3: lossy stepper against the scheme's closed form


def _S(a, b, kappa, om, dt):
    """Discrete stretch of the scheme: psi_n = b psi_(n-1) + a g_n drives the
    derivative through (psi_(n-1) + psi_n)/2, i.e. a (1 + z^-1)/2 / (1 - b z^-1)."""
    z = np.exp(-1j * om * dt)
    return 1.0 / kappa + sum(aa * 0.5 * (1.0 + z) / (1.0 - bb * z) for aa, bb in zip(a, b))


def test_discrete_stretch_tends_to_paper_gamma():
    """The z-transform of the scheme's stretch converges at SECOND order in dt
    to 1/kappa - gamma(w) (Eq. gamma1): ties Eqs. relaxation_a/b and the
    midpoint time index of Eq. relaxation_psi to the dispersion relation of
    Sec. 2.2."""
    d = np.array([3e5, 2e7, 4e8])
    al = np.array([5e6, 8e8, 2e10])
    kap = 0.985
    om = 2 * math.pi * np.array([1e6, 5e6, 20e6])
    ref = 1.0 / kap - fit.gamma(d, al, kap, om)
    errs = []
    for dt in (1e-11, 1e-12):
        a, b = recursion_ab(d, al, kap, dt)
        errs.append(np.max(np.abs(_S(a, b, kap, om, dt) - ref) / np.abs(ref)))
    assert errs[0] < 1e-3 and 80 < errs[0] / errs[1] < 120, errs


def test_lossy_eigenmode_exact(oracle_lib):
    """A travelling eigenmode of the discrete lossy scheme, built from its
    dispersion relation [2 sin(w dt/2)/dt]^2 = c^2 K_d^2 S1(w) S2(w), must be
    followed to rounding error for hundreds of steps (per-direction psi_2)."""
    nx, dx = 64, 1e-4
    c, rho = 1500.0, 1000.0
    dt = 0.35 * dx / c
    prm = fit.RelaxParams(0.995, 0.99, np.array([3e5, 2e7]), np.array([5e6, 8e8]),
                          np.array([1e6, 4e7]), np.array([2e7, 3e9]))
    sim = sim_of((4, nx), dx, dt, c, rho, params=[prm], periodic=(True, True))
    m = sim.med
    a1 = [m.a1[nu][0, 0] for nu in range(2)]
    b1 = [m.b1[nu][0, 0] for nu in range(2)]
    a2 = [m.a2[nu][0, 0] for nu in range(2)]
    b2 = [m.b2[nu][0, 0] for nu in range(2)]
    k = 2 * math.pi * 3 / (nx * dx)
    Kd = modified_wavenumber(k, dx)

    def F(om):
        return (2 * np.sin(om * dt / 2) / dt) ** 2 - c * c * Kd * Kd * _S(a1, b1, prm.kappa1, om, dt) * _S(a2, b2, prm.kappa2, om, dt)

    om = complex(c * Kd)
    for _ in range(60):
        h = 1e-7 * abs(om)
        step = F(om) / ((F(om + h) - F(om - h)) / (2 * h))
        om -= step
        if abs(step) < 1e-15 * abs(om):
            break
    assert abs(F(om)) < 1e-9 * (c * Kd) ** 2
    assert om.imag > 0                         # decays as e^(i w t)
    z = np.exp(-1j * om * dt)
    s = np.sin(om * dt / 2)
    P = 1.0
    g = -1j * Kd * P
    S1 = _S(a1, b1, prm.kappa1, om, dt)
    psi1 = [a1[nu] * g / (1 - b1[nu] * z) for nu in range(2)]
    V = -(dt / rho) * S1 * g / (2j * s)
    q = -1j * Kd * V
    psi2 = [a2[nu] * q / (1 - b2[nu] * z) for nu in range(2)]
    x = np.arange(nx) * dx
    xi = np.broadcast_to(x, (4, nx))
    xh = xi + dx / 2
    ph = lambda X: np.exp(-1j * k * X)  # noqa: E731
    sim.p[...] = np.real(P * ph(xi))
    sim.v[0][...] = np.real(V * np.exp(-1j * om * dt / 2) * ph(xh))
    for nu in range(2):
        sim.psi1[nu][0][...] = np.real(psi1[nu] * np.exp(-1j * om * dt) * ph(xh))
        sim.psi2[nu][0][...] = np.real(psi2[nu] * np.exp(-1j * om * dt / 2) * ph(xi))
    n = 500
    sim.run(n)
    want = np.real(P * np.exp(1j * om * n * dt) * ph(xi))
    amp = abs(np.exp(1j * om * n * dt))
    assert amp < 0.999                          # the mode really decays
    assert np.max(np.abs(sim.p - want)) < 1e-10


def test_lossy_energy_never_exceeds_initial(oracle_lib):
    """Passivity: with relaxation (energy flows into the memory variables and
    is dissipated) the mechanical energy stays below its initial value."""
    rng = np.random.default_rng(5)
    shape = (24, 24)
    dx = 1e-4
    c, rho = 1540.0, 1000.0
    dt = 0.4 * dx / c
    prm, _ = fit.fit_relaxation(0.8, 1.2, 2, maxiter=600, w_list=(0.5,))
    sim = sim_of(shape, dx, dt, c, rho, params=[prm], periodic=(True, True))
    sim.p[...] = rng.standard_normal(shape)
    K = rho * c * c
    E = []
    for _ in range(400):
        v_old = [v.copy() for v in sim.v]
        p_n = sim.p.copy()
        sim.run(1)
        E.append(np.sum(p_n ** 2 / (2 * K)) + sum(np.sum(rho * v_old[d] * sim.v[d]) / 2 for d in range(2)))
    E = np.array(E)
    assert np.all(E <= E[0] * (1 + 1e-12))
    assert E[-1] < 0.99 * E[0]


# ---------------------------------------------------------------------------
# continuous pins


def test_point_source_matches_2d_green_function(oracle_lib):
    """Lossless point source: P(f)/S(f) = (rho w/4) H0^(2)(k r) (e^{+iwt}
    convention, volume-injection rate S), after the half-step delay that the
    injection convention introduces and the sample-time offset of traces."""
    special = pytest.importorskip("scipy.special")
    c, rho, f0 = 1500.0, 1000.0, 1e6
    dx = c / (f0 * 16)
    dt = 0.3 * dx / c
    n = 300
    shape = (n, n)
    sim = sim_of(shape, dx, dt, c, rho, pml=24, f0=f0)
    src = np.zeros(shape, np.uint8)
    src[n // 2, n // 2] = 1
    rcv = np.zeros(shape, np.uint8)
    r_cells = 32
    rcv[n // 2, n // 2 + r_cells] = 1
    nt = 1400
    w = gaussian_pulse(f0, dt, nt, 1.0)
    sim.set_sources(src, w[None])
    sim.set_receivers(rcv, nt)
    sim.run(nt)
    tr = sim.traces[0]
    N = 1 << 14
    f = np.fft.rfftfreq(N, dt)
    P = np.fft.rfft(tr, N)
    S = np.fft.rfft(w, N)
    om = 2 * math.pi * f
    sel = (f > 0.7 * f0) & (f < 1.3 * f0)
    H = P[sel] / S[sel] * np.exp(-1j * om[sel] * dt / 2)     # trace sample n is p((n+1) dt)
    r = r_cells * dx
    want = rho * om[sel] / 4 * special.hankel2(0, om[sel] / c * r)
    assert np.max(np.abs(np.abs(H) / np.abs(want) - 1)) < 0.01
    assert np.max(np.abs(np.angle(H / want))) < 0.03


def _plane_run(params, f0, depth_cells, rcv_rows, nt, ppw=16, cfl=0.2, pml=20, transition=0,
               c=1540.0, rho=1000.0, beta=None, amp=1e3, tau=None, cls=None, layer_class=None):
    """1D-like plane wave: 4 periodic columns, source row pml+transition+2.
    layer_class: one fixed class in the whole absorbing layer (layer_relax)."""
    dx = c / (f0 * ppw)
    dt = cfl * dx / c
    width = pml + transition
    ny = depth_cells + 2 * width
    shape = (ny, 4)
    if cls is None:
        cls = np.zeros(shape, np.int64)
    if layer_class is not None:
        cls = cls.copy()
        cls[:width] = layer_class
        cls[ny - width:] = layer_class
    sim = sim_of(shape, dx, dt, c, rho, params=params, periodic=(False, True), pml=pml,
                 transition=transition, beta=None if beta is None else np.full(shape, beta), f0=f0, cls=cls,
                 layer_relax=layer_class is not None)
    row = width + 2
    src = np.zeros(shape, np.uint8)
    src[row] = 1
    rcv = np.zeros(shape, np.uint8)
    for r in rcv_rows:
        rcv[row + r, 0] = 1
    w = gaussian_pulse(f0, dt, nt, plane_amplitude_rate(amp, dx, 2, rho, c), tau=tau)
    sim.set_sources(src, w[None])
    sim.set_receivers(rcv, nt)
    sim.run(nt)
    return sim, dx, dt


@pytest.mark.parametrize("a0,y", [(0.5, 1.0), (0.75, 1.5), (0.3, 0.7)])
def test_pml_reflection_below_minus_50db(a0, y, oracle_lib):
    """Two-stage absorbing layer, L_T = L_B = 3 lambda at 1 MHz, D = 5 lambda
    (Sec. 4.3): R < -50 dB for y <= 1.5 (abstract, Sec. 5.4)."""
    prm, _ = fit.fit_relaxation(a0, y, 2, maxiter=1500, w_list=(0.5,))
    f0, ppw = 1e6, 16
    L = 3 * ppw
    D = 5 * ppw
    rows = [D - 8]
    nt = 2000
    small, _, _ = _plane_run([prm], f0, D, rows, nt, ppw=ppw, pml=L, transition=L)
    big, _, _ = _plane_run([prm], f0, D + 600, rows, nt, ppw=ppw, pml=L, transition=L)
    R = measure.reflection_db(small.traces[0], big.traces[0])
    assert R < -50.0, R


def test_homogeneous_layer_reflects_away_from_its_design_point(oracle_lib):
    """Homogeneous layers (Sec. 4.6): one relaxation class, fitted for
    (0.5, 1.0), in the whole layer instead of the inherited interior class.
    At its own (alpha0, y) the medium is the adaptive one, so R is equal; for
    an interior tissue away from it the relaxation set changes abruptly at the
    layer's inner edge and R rises well above the adaptive layer's (Sec. 5.5:
    the homogeneous layers degrade away from the design point)."""
    ref, _ = fit.fit_relaxation(0.5, 1.0, 2, maxiter=1500, w_list=(0.5,))
    f0, ppw = 1e6, 16
    L = 3 * ppw
    D = 5 * ppw
    rows = [D - 8]
    nt = 2000
    out = {}
    for a0, y in ((0.5, 1.0), (0.3, 0.7)):
        prm, _ = fit.fit_relaxation(a0, y, 2, maxiter=1500, w_list=(0.5,))
        for lc in (None, 1):
            small, _, _ = _plane_run([prm, ref], f0, D, rows, nt, ppw=ppw, pml=L, transition=L, layer_class=lc)
            big, _, _ = _plane_run([prm, ref], f0, D + 600, rows, nt, ppw=ppw, pml=L, transition=L, layer_class=lc)
            out[(a0, y, lc)] = measure.reflection_db(small.traces[0], big.traces[0])
    assert abs(out[(0.5, 1.0, None)] - out[(0.5, 1.0, 1)]) < 1e-6, out
    assert out[(0.3, 0.7, None)] < -60.0, out
    assert out[(0.3, 0.7, 1)] > out[(0.3, 0.7, None)] + 10.0, out


def test_simulated_attenuation_and_dispersion(oracle_lib):
    """Spectral attenuation between receivers at 0.05 D and 0.8 D, D = 10
    lambda, 16 ppw, CFL 0.2 (Sec. 3.3, 4.1), centre frequencies 1-20 MHz in
    2.71 MHz steps: NRMSE vs alpha0 f^y below 3 % and phase velocity within
    5 m/s of the Kramers-Kronig target (Sec. 5.1)."""
    a0, y, c = 0.5, 1.1, 1540.0
    prm, rep = fit.fit_relaxation(a0, y, 2, maxiter=2500, w_list=(0.1, 0.5, 0.9))
    fs, al, al_model, cerr = [], [], [], []
    for f0 in np.arange(1e6, 20.01e6, 2.71e6):
        D = 160
        r1, r2 = int(round(0.05 * D)), int(round(0.8 * D))
        nt = int((r2 + 100) / 0.2)
        sim, dx, dt = _plane_run([prm], f0, D + 20, [r1, r2], nt)
        d = (r2 - r1) * dx
        f, a = measure.attenuation_spectrum(sim.traces[0], sim.traces[1], dt, d)
        keep = (f > 0.7 * f0) & (f < 1.3 * f0)
        fs.append(f[keep])
        al.append(a[keep])
        fc, cm = measure.phase_velocity(sim.traces[0], sim.traces[1], dt, d, c)
        keep = (fc > 0.7 * f0) & (fc < 1.3 * f0)
        ct = 1.0 / fit.inv_c_target(a0, y, 2 * math.pi * fc[keep], c)
        cerr.append(cm[keep] - ct)
    fs, al = np.concatenate(fs), np.concatenate(al)
    target = fit.alpha_target(a0, y, fs)
    assert measure.nrmse(al, target) < 0.03
    # against the closed form of the fitted model the error is discretisation only
    assert measure.nrmse(al, fit.attenuation_model(prm, fs, c)) < 0.02
    assert math.sqrt(np.mean(np.concatenate(cerr) ** 2)) < 5.0


def test_fubini_second_harmonic(oracle_lib):
    """Lossless plane wave with the nonlinear term, before shock: harmonic
    ratio B2/B1 = J2(2 s)/(2 J1(s)) (Fubini), s = x/x_sh, x_sh = rho c^3/(beta w p0)."""
    special = pytest.importorskip("scipy.special")
    f0, c, rho, beta, p0 = 2e6, 1500.0, 1000.0, 6.0, 2e6
    ppw = 24
    nt = 3200
    rows = [10, 250]
    sim, dx, dt = _plane_run([fit.RelaxParams.lossless(1)], f0, 420, rows, nt, ppw=ppw, cfl=0.25,
                             c=c, rho=rho, beta=beta, amp=p0, tau=6.0 / f0)
    N = 1 << 15
    f = np.fft.rfftfreq(N, dt)

    def envelope_peak(tr, fc):
        # analytic signal of the band fc +- 0.4 f0, then its peak magnitude
        S = np.fft.fft(tr, N)
        ff = np.fft.fftfreq(N, dt)
        S[(ff < fc - 0.4 * f0) | (ff > fc + 0.4 * f0)] = 0.0
        return np.max(np.abs(np.fft.ifft(2 * S)))

    amps = [(envelope_peak(sim.traces[i], f0), envelope_peak(sim.traces[i], 2 * f0)) for i in range(2)]
    p_meas = amps[0][0]                         # fundamental amplitude near the source
    xsh = rho * c ** 3 / (beta * 2 * math.pi * f0 * p_meas)
    fub = lambda s: special.jv(2, 2 * s) / (2 * special.jv(1, s))  # noqa: E731
    s1, s2 = (rows[0] * dx / xsh, rows[1] * dx / xsh)
    # growth of the second harmonic (at the envelope peak) between the receivers
    want = fub(s2) - fub(s1)
    got = amps[1][1] / amps[1][0] - amps[0][1] / amps[0][0]
    assert 0.1 < s2 < 0.5
    assert 0.5 * p0 < p_meas < 1.5 * p0
    assert abs(got / want - 1) < 0.05, (got, want)


def test_tissue_ramp_keeps_the_absorbing_layer_stable(oracle_lib):
    """Long-time stability of the absorbing layer (Sec. 5.4: the transition
    layer removes the divergent cells).  A point source in a strongly lossy
    medium (alpha0 1.0, y 2.0, N = 4) with a 20-cell layer and no transition:
    with the tissue mechanisms ramped out across the layer the field decays
    after the pulse has left; with them kept at full strength up to the
    outer edge, where the absorbing mechanism's alpha vanishes, the
    low-frequency stretch turns negative there and the run diverges."""
    prm, _ = fit.fit_relaxation(1.0, 2.0, 4, maxiter=3000, w_list=(0.1, 0.5, 0.9))
    f0 = 3e6
    dx = 1540.0 / (f0 * 12)
    dt = 0.4 * dx / 1700.0
    shape = (96, 96)
    out = {}
    for ramp in (True, False):
        med = OracleMedium(shape, dx, dt, np.full(shape, 1540.0), np.full(shape, 1000.0), np.zeros(shape, np.int64),
                           [prm], pml=20, f0=f0, tissue_ramp_on=ramp)
        sim = OracleSim(med)
        src = np.zeros(shape, np.uint8)
        src[48, 48] = 1
        sim.set_sources(src, gaussian_pulse(f0, dt, 1200, 1e-6)[None])
        sim.run(100)
        peak = np.abs(sim.p).max()
        sim.run(1100)
        out[ramp] = np.abs(sim.p).max() / peak
    assert out[True] < 1e-4, out
    assert out[False] > 1e3, out


def _layer_wkb_db(n, l_t, l_b, r0, c, dx, f0):
    """Round trip through the bottom absorbing layer in the WKB limit:
    exp(-2 sum_cells a dx), a = -Im k of the layer's Debye mechanism on both
    stretches (kappa = 1, lossless tissue), with the profile written out from
    its definition: depth s from the inner edge (half points for the
    gradient side, integer points for the divergence side), d(s) = 0.1 d_max
    (s/L_T)^2 in the transition, d_max (0.1 + 0.9 ((s - L_T)/L_B)^2) beyond
    (d_max (s/L_B)^2 without transition), d_max = -3 c ln(R0) / (2 L_B dx),
    alpha(s) = pi f0 (1 - s/(L_T + L_B))."""
    w = l_t + l_b
    d_max = -3.0 * c * math.log(r0) / (2.0 * l_b * dx)
    om = 2 * math.pi * f0
    total = 0.0
    for i in range(n - w - 1, n):
        k = om / c
        for s in (max(0.0, i + 0.5 - (n - w - 0.5)), max(0.0, i - (n - w - 0.5))):
            if s <= 0:
                d = 0.0
            elif l_t > 0 and s <= l_t:
                d = 0.1 * d_max * (s / l_t) ** 2
            elif l_t > 0:
                d = d_max * (0.1 + 0.9 * ((s - l_t) / l_b) ** 2)
            else:
                d = d_max * (s / l_b) ** 2
            alpha = math.pi * f0 * (1.0 - s / w)
            k = k / np.sqrt(1.0 - d / (d + alpha + 1j * om))      # stretch 1 - gamma, kappa = 1
        total += -k.imag * dx
    return 20.0 * math.log10(math.exp(-2.0 * total))


@pytest.mark.parametrize("l_t,l_b,r0", [(0, 40, 1e-2), (0, 40, 1e-3), (24, 24, 1e-2)])
def test_absorbing_layer_round_trip(l_t, l_b, r0, oracle_lib):
    """Absorbing-profile constants (the reading of Sec. 4.3's C-PML): a 1 MHz
    plane wave crosses the bottom layer, meets the zero field beyond the grid
    and crosses back.  Its amplitude at f0, against the same run on a much
    deeper grid, equals the WKB round trip of the profile to 1.5 dB, and a
    layer without transition returns the design reflection R0 to 1 dB."""
    c, rho, f0, ppw = 1540.0, 1000.0, 1e6, 16
    dx = c / (f0 * ppw)
    dt = 0.2 * dx / c
    w = l_t + l_b
    src_off, depth = 300, 340

    def run(extra):
        shape = (w + src_off + depth + extra + w, 4)
        med = OracleMedium(shape, dx, dt, np.full(shape, c), np.full(shape, rho), np.zeros(shape, np.int64),
                           [fit.RelaxParams.lossless(1)], pml=l_b, transition=l_t, f0=f0, R0=r0,
                           periodic=(False, True))
        sim = OracleSim(med)
        src = np.zeros(shape, np.uint8)
        src[w + src_off] = 1
        rcv = np.zeros(shape, np.uint8)
        rcv[w + src_off + depth - 20, 0] = 1
        nt = int((depth + 2 * (20 + w) + 200) / 0.2)
        sim.set_sources(src, gaussian_pulse(f0, dt, nt, 1.0, tau=3.0 / f0)[None])
        sim.set_receivers(rcv, nt)
        sim.run(nt)
        return sim.traces[0], shape[0]

    near, n = run(0)
    far, _ = run(2000)
    N = 1 << 16
    f = np.fft.rfftfreq(N, dt)
    k0 = int(np.argmin(np.abs(f - f0)))
    got = 20 * math.log10(abs(np.fft.rfft(near - far, N)[k0]) / abs(np.fft.rfft(far, N)[k0]))
    want = _layer_wkb_db(n, l_t, l_b, r0, c, dx, f0)
    assert abs(got - want) < 1.5, (got, want)
    if l_t == 0:
        assert abs(got - 20 * math.log10(r0)) < 1.0, got
