"""Pins of the oracle's time-space stencil (Sec. 3.3: 2M-th order in space,
fourth order in time, after Tan & Huang, J. Comput. Phys. 276 (2014)), no
GPU.  The expectations come from outside the stepper's code: the Taylor
weights of the textbook staggered derivative, the exact plane-wave relation
of the leapfrog scheme with the stencil's Fourier symbol written out here,
the order of the phase error measured on simulated waves against the exact
continuous solution, and growth or boundedness of simulated noise on either
side of the stability limit."""
import math

import numpy as np
import pytest

from oracle import fit
from oracle.medium import OracleMedium, time_space_cfl_limit, time_space_coefficients
from oracle.stepper import OracleSim

# 8th-order staggered Taylor weights (textbook values)
TAYLOR = (1225.0 / 1024.0, -245.0 / 3072.0, 49.0 / 5120.0, -5.0 / 7168.0)


def _sim(shape, dx, dt, c=1500.0, rho=1100.0, time_order=4, kappa=(1.0, 1.0)):
    p0 = fit.RelaxParams(kappa[0], kappa[1], np.zeros(2), np.full(2, 1e9), np.zeros(2), np.full(2, 1e9))
    nd = len(shape)
    med = OracleMedium(shape, dx, dt, np.full(shape, c), np.full(shape, rho), np.zeros(shape, np.int64), [p0],
                       periodic=(True,) * nd, time_order=time_order)
    return OracleSim(med)


def _symbol(kvec, dx, a, b):
    """K_d of the time-space first derivative: the stencil
    sum_m a_m (f(+m) - f(-m+1)) + b sum_{e != d, s = +-1} (f(+1, s e) - f(0, s e))
    applied to exp(i k.x) is i K_d exp(i k.x) dx (half-point shift aside)."""
    nd = len(kvec)
    out = []
    for d in range(nd):
        on = sum(a[m] * 2.0 * math.sin((2 * m + 1) * kvec[d] * dx / 2.0) for m in range(4))
        cross = b * 2.0 * math.sin(kvec[d] * dx / 2.0) * sum(2.0 * math.cos(kvec[e] * dx)
                                                            for e in range(nd) if e != d)
        out.append((on + cross) / dx)
    return out


def test_time_space_weights_reduce_to_taylor_at_zero_courant():
    for nd in (2, 3):
        a, b = time_space_coefficients(0.0, nd)
        assert b == 0.0
        assert np.allclose(a, TAYLOR, rtol=1e-13, atol=0)


def test_time_space_weights_shift_with_courant_number():
    """At r > 0 the on-axis weights move away from Taylor's by O(r^2), and
    the 3D set differs from the 2D one only by 2 b in the first weight (one
    more transverse axis, sum of 2 (D-1) b terms)."""
    a2, b2 = time_space_coefficients(0.4, 2)
    a3, b3 = time_space_coefficients(0.4, 3)
    assert b2 == b3 == pytest.approx(0.16 / 24.0, rel=1e-15)
    assert np.all(np.abs(np.asarray(a2) - TAYLOR) > 1e-5)
    # the 2 (D-1) b term of the j-conditions enters like a weight on (2m-1) = 1: a_1 only
    assert a3[0] - a2[0] == pytest.approx(-2.0 * b2, rel=1e-12)
    assert np.allclose(a3[1:], a2[1:], rtol=1e-12, atol=0)


def _plane_wave_exact(shape, dx, modes, r=0.4, n_steps=400, kappa=(1.0, 1.0)):
    """p after n_steps of an exact discrete plane wave (periodic, lossless)
    minus the closed form with omega from sin(omega dt/2) = (dt/2) c_eff |K|."""
    c, rho = 1500.0, 1100.0
    nd = len(shape)
    dt = r * dx / c
    sim = _sim(shape, dx, dt, c, rho, kappa=kappa)
    a, b = time_space_coefficients(r, nd)
    kvec = [2 * math.pi * m / (shape[nd - 1 - d] * dx) for d, m in enumerate(modes)]
    Kd = _symbol(kvec, dx, a, b)
    ceff = c / math.sqrt(kappa[0] * kappa[1])
    om = 2.0 / dt * math.asin(0.5 * dt * ceff * math.sqrt(sum(K * K for K in Kd)))
    grids = np.meshgrid(*[np.arange(n) * dx for n in shape], indexing="ij")
    pos = [grids[nd - 1 - d] for d in range(nd)]
    phase = sum(k * x for k, x in zip(kvec, pos))
    sim.p[...] = np.cos(phase)
    s = math.sin(om * dt / 2)
    for d in range(nd):
        amp = dt * Kd[d] / (kappa[0] * 2 * rho * s)
        sim.v[d][...] = amp * np.cos(phase + kvec[d] * dx / 2 + om * dt / 2)
    sim.run(n_steps)
    return float(np.max(np.abs(sim.p - np.cos(phase - om * n_steps * dt))))


def test_time_space_plane_wave_exact_2d():
    assert _plane_wave_exact((16, 32), 1e-4, (3, 2)) < 1e-10


def test_time_space_plane_wave_exact_2d_kappa():
    assert _plane_wave_exact((8, 40), 1e-4, (2, 3), r=0.3, kappa=(0.99, 0.985)) < 1e-10


def test_time_space_plane_wave_exact_3d():
    assert _plane_wave_exact((8, 8, 16), 1e-4, (2, 1, 3), n_steps=250) < 1e-10


def _phase_error(ppw, time_order, nd, r=0.4, periods=2.0):
    """Largest |p - cos(k.x - c|k|t)| of a simulated oblique plane wave (one
    wavelength per axis of a periodic box of ppw cells per side) after
    `periods` periods, started from the exact continuous solution."""
    c, rho, dx = 1500.0, 1000.0, 1e-4
    shape = (ppw,) * nd
    dt = r * dx / c
    sim = _sim(shape, dx, dt, c, rho, time_order=time_order)
    k1 = 2.0 * math.pi / (ppw * dx)
    kabs = k1 * math.sqrt(nd)
    om = c * kabs
    grids = np.meshgrid(*[np.arange(n) * dx for n in shape], indexing="ij")
    phase = sum(k1 * g for g in grids)
    sim.p[...] = np.cos(phase)
    for d in range(nd):
        # v_d at its half point, half a step before p (continuous plane wave)
        sim.v[d][...] = (k1 / (rho * om)) * np.cos(phase + k1 * dx / 2 + om * dt / 2)
    n = int(round(periods * 2.0 * math.pi / om / dt))
    sim.run(n)
    return float(np.max(np.abs(sim.p - np.cos(phase - om * n * dt))))


@pytest.mark.parametrize("nd", [2, 3])
def test_time_space_error_is_fourth_order_at_fixed_courant(nd):
    """At CFL 0.4 the simulated phase error of an oblique wave falls 16-fold
    per halving of the cell (fourth order); the leapfrog's falls 4-fold."""
    ppws = (8, 16, 32) if nd == 2 else (8, 16)
    th = [_phase_error(p, 4, nd) for p in ppws]
    lf = [_phase_error(p, 2, nd) for p in ppws]
    for i in range(len(ppws) - 1):
        assert 12.0 < th[i] / th[i + 1] < 20.0, th
        assert 3.0 < lf[i] / lf[i + 1] < 5.0, lf
    assert th[0] < lf[0] / 20.0


@pytest.mark.parametrize("nd", [2, 3])
def test_time_space_stability_limit(nd):
    """Noise in a periodic box stays bounded just below the computed limit
    of the Courant number and grows without bound just above it."""
    lim = time_space_cfl_limit(nd)
    assert lim > (0.62 if nd == 2 else 0.50)            # above the leapfrog's 0.5497 / 0.4488
    shape = (16,) * nd if nd == 2 else (8, 8, 8)
    dx, c = 1e-4, 1500.0
    out = {}
    for f in (0.98, 1.02):
        sim = _sim(shape, dx, f * lim * dx / c, c, 1000.0)
        rng = np.random.default_rng(7)
        sim.p[...] = rng.standard_normal(shape)
        sim.run(1500)
        out[f] = float(np.max(np.abs(sim.p)))
    assert out[0.98] < 50.0, out
    assert out[1.02] > 1e6, out
