"""Pins of the FP64 calibration oracle (oracle/fit.py) against closed forms,
the paper's printed values and a library routine -- CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import fit

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_table2_variables_match_paper():
    g = _gold("table2_bounds.json")
    for n in (1, 2, 4):
        lo, hi = fit.theta_bounds(n)
        x0 = fit.theta_initial(n)
        assert lo[0] == g["kappa"]["range"][0] and hi[1] == g["kappa"]["range"][1]
        assert x0[0] == g["kappa"]["init"] and x0[1] == g["kappa"]["init"]
        blk_lo, blk_hi, blk_x = lo[2:].reshape(n, 4), hi[2:].reshape(n, 4), x0[2:].reshape(n, 4)
        # per mechanism: log10 d1, log10 d2, log10 alpha1, log10 alpha2
        np.testing.assert_allclose(10 ** blk_lo[:, :2], g["d"]["range"][0])
        np.testing.assert_allclose(10 ** blk_hi[:, :2], g["d"]["range"][1])
        np.testing.assert_allclose(10 ** blk_lo[:, 2:], g["alpha"]["range"][0])
        np.testing.assert_allclose(10 ** blk_hi[:, 2:], g["alpha"]["range"][1])
        np.testing.assert_allclose(10 ** blk_x[:, :2], g["d"]["init"])
        np.testing.assert_allclose(10 ** blk_x[:, 2:], g["alpha"]["init"])
    assert tuple(fit.W_SWEEP) == tuple(g["w_sweep"]["values"])


def test_theta_roundtrip_and_order():
    p = fit.RelaxParams(0.99, 0.985, np.array([1e3, 1e7]), np.array([2e6, 3e9]),
                        np.array([4e5, 5e8]), np.array([6e10, 7e7]))
    th = fit.theta_from_params(p)
    # paper's listing order: k1, k2, d1^1, d2^1, a1^1, a2^1, d1^2, ...
    np.testing.assert_allclose(th[:6], [0.99, 0.985, 3.0, math.log10(4e5), math.log10(2e6), math.log10(6e10)])
    q = fit.params_from_theta(th)
    for name in ("d1", "alpha1", "d2", "alpha2"):
        np.testing.assert_allclose(getattr(q, name), getattr(p, name), rtol=1e-14)


def test_db_per_neper_textbook():
    # 1 Np = 20 log10(e) dB = 8.685889638 dB; 1 dB/(MHz cm) at 1 MHz = 11.5129 Np/m
    assert abs(fit.alpha_target(1.0, 1.0, 1e6) - 100.0 / 8.685889638065035) < 1e-12
    # power law: doubling f multiplies alpha by 2^y
    a = fit.alpha_target(0.5, 1.3, np.array([2e6, 4e6]))
    assert abs(a[1] / a[0] - 2 ** 1.3) < 1e-12


@pytest.mark.parametrize("y", [0.4, 0.7, 1.3, 1.5, 1.9])
def test_kk_target_is_causal_power_law(y):
    """k_GT(w) - w/c_inf must be a constant times (i w)^y (the causal power-law
    form with k(-w) = -conj k(w)); this fixes both the tan(pi y/2) factor and
    its sign, and the -i alpha sign reading."""
    c0, a0 = 1540.0, 0.6
    f = np.logspace(5.5, 7.5, 40)
    w = 2 * math.pi * f
    k = fit.k_target(a0, y, f, c0)
    a0p = a0 * 100.0 / fit.DB_PER_NP / (2 * math.pi * 1e6) ** y
    inv_cinf = 1.0 / c0 - a0p * math.tan(math.pi * y / 2) * (2 * math.pi * 1e6) ** (y - 1)
    ratio = (k - w * inv_cinf) / (1j * w) ** y
    assert np.allclose(ratio, ratio[0], rtol=1e-9, atol=0)
    assert abs(ratio[0].real) < 1e-9 * abs(ratio[0])          # purely imaginary
    # the constant is -i a0'/cos(pi y/2): then -Im k = a0' w^y on w > 0
    assert abs(ratio[0] - (-1j * a0p / math.cos(math.pi * y / 2))) < 1e-9 * abs(ratio[0])


def test_kk_reference_and_y1_limit():
    c0 = 1540.0
    w0 = 2 * math.pi * 1e6
    for y in (0.6, 1.0, 1.7):
        assert abs(1.0 / fit.inv_c_target(0.5, y, w0, c0) - c0) < 1e-9
    f = np.logspace(6, 7.3, 20)
    w = 2 * math.pi * f
    lim = fit.inv_c_target(0.5, 1.0, w, c0)
    for dy in (1e-3, -1e-3):
        near = fit.inv_c_target(0.5, 1.0 + dy, w, c0)
        assert np.max(np.abs(near - lim) / lim) < 5e-6
    # positive dispersion: phase velocity grows with frequency
    for y in (0.5, 1.0, 1.5):
        c = 1.0 / fit.inv_c_target(0.5, y, w, c0)
        assert np.all(np.diff(c) > 0)


def test_k_model_closed_forms():
    f = np.logspace(6, 7.3, 30)
    w = 2 * math.pi * f
    c = 1500.0
    # no mechanisms active: k = (w/c) sqrt(k1 k2)
    p = fit.RelaxParams(0.99, 0.985, np.zeros(2), np.full(2, 1e9), np.zeros(2), np.full(2, 1e9))
    np.testing.assert_allclose(fit.k_model(p, f, c), (w / c) * math.sqrt(0.99 * 0.985), rtol=1e-14)
    # one mechanism on stretch 1 only, kappa = 1: s1^-1 = (alpha + i w)/(d + alpha + i w),
    # so k = (w/c) sqrt((d + alpha + i w)/(alpha + i w)); low-frequency phase speed
    # c sqrt(alpha/(d + alpha)), high-frequency c
    d, al = 3e6, 2e7
    p = fit.RelaxParams(1.0, 1.0, np.array([d]), np.array([al]), np.array([0.0]), np.array([1e9]))
    k = fit.k_model(p, f, c)
    direct = (w / c) * np.sqrt((d + al + 1j * w) / (al + 1j * w))
    np.testing.assert_allclose(k, direct, rtol=1e-13)
    lo = fit.phase_velocity_model(p, np.array([1.0]), c)[0]
    hi = fit.phase_velocity_model(p, np.array([1e12]), c)[0]
    assert abs(lo - c * math.sqrt(al / (d + al))) < 1e-6 * c
    assert abs(hi - c) < 1e-3 * c
    # passivity: attenuation positive for d > 0 (sign reading of the target)
    assert np.all(fit.attenuation_model(p, f, c) > 0)


def test_objective_zero_at_target_and_weighting():
    f = fit.freq_grid()
    obj = fit.Objective(0.5, 1.1, 1540.0, 0.3, f)
    # the normalised target vs itself is exactly zero
    assert np.mean(np.abs(obj.kgt_n - obj._normalise(fit.k_target(0.5, 1.1, f, 1540.0))) ** 2) == 0.0
    # a pure imaginary error of one range unit costs w^2, a real one (1-w)^2
    k = fit.k_target(0.5, 1.1, f, 1540.0)
    e_im = np.mean(np.abs(obj.kgt_n - obj._normalise(k + 1j * obj.r_im)) ** 2)
    e_re = np.mean(np.abs(obj.kgt_n - obj._normalise(k + obj.r_re)) ** 2)
    assert abs(e_im - 0.3 ** 2) < 1e-12 and abs(e_re - 0.7 ** 2) < 1e-12


def test_freq_grid_log_spaced():
    f = fit.freq_grid()
    assert len(f) == 200 and abs(f[0] - 1e6) < 1e-6 and abs(f[-1] - 20e6) < 1e-3
    r = f[1:] / f[:-1]
    assert np.allclose(r, r[0], rtol=1e-12)


def test_nelder_mead_matches_scipy_adaptive_bounded():
    """On tie-free objectives the oracle's simplex visits exactly the points
    SciPy's adaptive, bounded Nelder-Mead visits (the routine the paper used)."""
    opt = pytest.importorskip("scipy.optimize")
    lo = np.array([-2.0, -1.5, -2, -1, -3])
    hi = np.array([2.0, 1.1, 2, 3, 1.0])
    x0 = np.array([-1.2, 1.0, 0.3, 0.0, 1.0])
    A, B = [], []
    fa = lambda x: (A.append(np.array(x)), opt.rosen(x))[1]  # noqa: E731
    fb = lambda x: (B.append(np.array(x)), opt.rosen(x))[1]  # noqa: E731
    r = opt.minimize(fa, x0, method="Nelder-Mead", bounds=list(zip(lo, hi)),
                     options=dict(adaptive=True, maxiter=1500, xatol=1e-14, fatol=1e-14))
    res = fit.nelder_mead(fb, x0, lo, hi, maxiter=1500, xatol=1e-14, fatol=1e-14)
    assert len(A) == len(B)
    for a, b in zip(A, B):
        assert np.array_equal(a, b)
    assert res.fun == r.fun


def test_nelder_mead_quadratic_minimum():
    rng = np.random.default_rng(7)
    M = rng.standard_normal((6, 6))
    H = M @ M.T + 6 * np.eye(6)
    xs = rng.standard_normal(6)
    f = lambda x: float((x - xs) @ H @ (x - xs))  # noqa: E731
    res = fit.nelder_mead(f, np.zeros(6), maxiter=20000, xatol=1e-12, fatol=1e-20)
    np.testing.assert_allclose(res.x, xs, atol=1e-8)


def test_nelder_mead_respects_bounds():
    f = lambda x: float(np.sum((x - 5.0) ** 2))  # noqa: E731
    res = fit.nelder_mead(f, np.zeros(3), np.full(3, -1.0), np.full(3, 1.0), maxiter=3000,
                          xatol=1e-12, fatol=1e-20)
    np.testing.assert_allclose(res.x, 1.0, atol=1e-9)


@pytest.mark.parametrize("a0,y", [(0.5, 1.1), (0.15, 1.0), (1.0, 0.7)])
def test_fit_core_accuracy(a0, y):
    """Closed-form attenuation NRMSE of the fitted N=2 set is below the paper's
    3 % core bound and the dispersion error is of the paper's order (Sec. 5.1)."""
    g = _gold("paper_accuracy.json")
    p, rep = fit.fit_relaxation(a0, y, 2, maxiter=2500, w_list=(0.1, 0.5, 0.9))
    assert rep.nrmse < g["nrmse_core_bound"]
    assert rep.disp_rmse < 5.0
    assert not rep.failed
    # the returned set is admissible (Sec. 3.2)
    assert 0.98 <= p.kappa1 <= 1.0 and 0.98 <= p.kappa2 <= 1.0
    assert np.all(p.d1 >= 1e2) and np.all(p.alpha1 >= 1e5)


def test_fit_lossless_class():
    p, rep = fit.fit_relaxation(0.0, 1.5, 3)
    assert p.n_mech == 3 and np.all(p.d1 == 0) and np.all(p.d2 == 0) and p.kappa1 == 1.0
    assert not rep.failed


def test_fit_selection_prefers_lowest_nrmse():
    p, rep = fit.fit_relaxation(0.5, 1.3, 2, maxiter=800, w_list=(0.1, 0.9))
    best = min(rep.per_w, key=lambda e: (e["nrmse"], e["disp"]))
    assert rep.w == best["w"] and rep.nrmse == best["nrmse"]
