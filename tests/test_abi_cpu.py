"""C-ABI library: loads, exports every declared symbol, and its host-side
calibration (FP64, no GPU) agrees with the oracle -- CPU only."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

import paper_2606_11103_gb300 as fw
from paper_2606_11103_gb300 import _lib
from oracle import fit

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2606_11103_gb300 import build
    build.build()
    return fw.lib()


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(fw_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported_and_bound(L):
    names = declared_functions()
    assert len(names) >= 25
    for n in sorted(names):
        assert hasattr(L, n), n
        assert n in _lib.SIGNATURES, n


def test_version_and_errors(L):
    assert L.fw_version() >= 100
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert L.fw_strerror(code)
    assert L.fw_strerror(-99) == b"unknown error"


def test_argument_errors_without_a_gpu(L):
    h = C.c_void_p()
    g = fw.make_grid((8, 8), 1e-4, dt=1e-8)
    g.ndim = 4
    c = np.ones(64, np.float32)
    p = fw.relax_params(1, 1, [0], [1e9], [0], [1e9])
    rc = L.fw_create_medium_classes(C.byref(g), c.ctypes.data, c.ctypes.data, None, c.ctypes.data,
                                    C.byref(p), 1, 0, None, C.byref(h))
    assert rc == fw.FW_ERR_ARG
    nb = C.c_size_t()
    assert L.fw_medium_bytes(C.byref(g), 2, 0, 0, C.byref(nb)) == fw.FW_ERR_ARG
    g = fw.make_grid((8, 8), 1e-4, dt=1e-8)
    assert L.fw_medium_bytes(C.byref(g), 5, 0, 0, C.byref(nb)) == fw.FW_ERR_ARG
    assert L.fw_medium_bytes(C.byref(g), 2, 7, 0, C.byref(nb)) == fw.FW_ERR_ARG
    o = fw.fit_opts()
    out, rep = fw.fw_relax_params(), fw.fw_fit_report()
    assert L.fw_fit_relaxation(0.5, 5.0, 2, C.byref(o), C.byref(out), C.byref(rep)) == fw.FW_ERR_ARG
    assert L.fw_fit_relaxation(0.5, 1.0, 0, C.byref(o), C.byref(out), C.byref(rep)) == fw.FW_ERR_ARG
    # y outside the valid range [0.4, 2.0] of the power law (abstract, Sec. 3.1), for a lossy class only
    for y in (0.39, 2.01):
        assert L.fw_fit_relaxation(0.5, y, 2, C.byref(o), C.byref(out), C.byref(rep)) == fw.FW_ERR_ARG
    assert L.fw_fit_relaxation(0.0, 3.0, 2, C.byref(o), C.byref(out), C.byref(rep)) == fw.FW_OK
    f = np.array([1e6, 5e6])
    al, cp = np.zeros(2), np.zeros(2)
    P = C.POINTER(C.c_double)
    args = (f.ctypes.data_as(P), 2, al.ctypes.data_as(P), cp.ctypes.data_as(P))
    assert L.fw_fit_targets(0.5, 2.5, 1540.0, 1e6, *args) == fw.FW_ERR_ARG
    assert L.fw_fit_targets(0.5, 1.1, -1.0, 1e6, *args) == fw.FW_ERR_ARG
    assert L.fw_fit_targets(0.5, 1.1, 1540.0, 1e6, *args) == fw.FW_OK


def test_medium_bytes_scale_with_grid(L):
    nb1, nb2 = C.c_size_t(), C.c_size_t()
    g1 = fw.make_grid((64, 64, 64), 1e-4, dt=1e-8, pml=8)
    g2 = fw.make_grid((128, 128, 128), 1e-4, dt=1e-8, pml=8)
    assert L.fw_medium_bytes(C.byref(g1), 4, 0, 0, C.byref(nb1)) == 0
    assert L.fw_medium_bytes(C.byref(g2), 4, 0, 0, C.byref(nb2)) == 0
    # 3D N=4 FP32: 20 state arrays + 6 absorbing-memory arrays + maps (~114 B/voxel)
    per_voxel = nb2.value / 128 ** 3
    assert 100 < per_voxel < 130
    assert 6.0 < nb2.value / nb1.value < 8.5      # plus a fixed 8 MB class-table reserve
    nb16 = C.c_size_t()
    assert L.fw_medium_bytes(C.byref(g2), 4, fw.FW_STORE_BF16, 0, C.byref(nb16)) == 0
    assert nb16.value < nb2.value * 0.75


def test_objective_matches_oracle(L):
    rng = np.random.default_rng(0)
    f = fit.freq_grid()
    for n_mech in (1, 2, 4):
        lo, hi = fit.theta_bounds(n_mech)
        for _ in range(5):
            th = lo + (hi - lo) * rng.uniform(size=lo.size)
            for (a0, y, w) in ((0.5, 1.1, 0.3), (0.9, 1.0, 0.7), (0.05, 1.8, 0.5)):
                J = C.c_double()
                thc = np.ascontiguousarray(th)
                o = fw.fit_opts()
                rc = L.fw_fit_objective(a0, y, w, C.byref(o), thc.ctypes.data_as(C.POINTER(C.c_double)),
                                        n_mech, C.byref(J))
                assert rc == 0
                ref = fit.Objective(a0, y, 1540.0, w, f)(th)
                assert abs(J.value - ref) <= 1e-11 * abs(ref), (J.value, ref)


def test_model_wavenumber_matches_oracle(L):
    p = fw.relax_params(0.99, 0.985, [3e5, 2e7], [5e6, 8e8], [1e6, 4e7], [2e7, 3e9])
    f = np.logspace(5, 8, 50)
    k = fw.model_wavenumber(p, 1500.0, f)
    ref = fit.k_model(fit.RelaxParams(0.99, 0.985, np.array([3e5, 2e7]), np.array([5e6, 8e8]),
                                      np.array([1e6, 4e7]), np.array([2e7, 3e9])), f, 1500.0)
    np.testing.assert_allclose(k, ref, rtol=1e-13)


def test_nelder_mead_matches_oracle_bitwise(L):
    lo = np.array([-2.0, -1.5, -2, -1, -3])
    hi = np.array([2.0, 1.1, 2, 3, 1.0])
    x0 = np.array([-1.2, 1.0, 0.3, 0.0, 1.0])

    def rosen(x):
        return float(np.sum(100.0 * (x[1:] - x[:-1] ** 2) ** 2 + (1 - x[:-1]) ** 2))

    seq = []

    @_lib.OBJFN
    def cb(xp, ctx):
        x = np.ctypeslib.as_array(xp, shape=(5,)).copy()
        seq.append(x)
        return rosen(x)

    x = x0.copy()
    D = C.POINTER(C.c_double)
    fmin, it, ne = C.c_double(), C.c_int(), C.c_int()
    rc = L.fw_nelder_mead(5, x.ctypes.data_as(D), lo.ctypes.data_as(D), hi.ctypes.data_as(D), cb, None,
                          1500, 1e-14, 1e-14, C.byref(fmin), C.byref(it), C.byref(ne))
    assert rc == 0
    ref_seq = []
    res = fit.nelder_mead(lambda v: (ref_seq.append(v.copy()), rosen(v))[1], x0, lo, hi, maxiter=1500,
                          xatol=1e-14, fatol=1e-14)
    assert ne.value == res.n_eval and it.value == res.n_iter
    for a, b in zip(seq, ref_seq):
        assert np.array_equal(a, b)
    assert np.array_equal(x, res.x)


@pytest.mark.parametrize("a0,y,n", [(0.5, 1.1, 2), (0.75, 1.5, 2), (0.3, 0.7, 3)])
def test_fit_matches_oracle(L, a0, y, n):
    """Same algorithm, same objective: the library's calibration reaches the
    oracle's objective value (to 1 %) and its attenuation accuracy."""
    kw = dict(maxiter=1200, w=(0.3, 0.7))
    p, rep = fw.fit_relaxation(a0, y, n, **kw)
    rp, rrep = fit.fit_relaxation(a0, y, n, maxiter=1200, w_list=(0.3, 0.7))
    assert rep.w == rrep.w
    assert abs(rep.J - rrep.J) <= 0.01 * rrep.J
    assert abs(rep.nrmse - rrep.nrmse) <= 0.01 * rrep.nrmse + 1e-6
    # the library's parameters, evaluated by the oracle, give the reported values
    q = fit.RelaxParams(p.kappa1, p.kappa2, np.array(p.d1[:n]), np.array(p.alpha1[:n]),
                        np.array(p.d2[:n]), np.array(p.alpha2[:n]))
    nr, dsp = fit.accuracy(q, a0, y, 1540.0, fit.freq_grid())
    assert abs(nr - rep.nrmse) < 1e-9 and abs(dsp - rep.disp_rmse) < 1e-7
    assert rep.failed == int(nr > 0.1 or dsp > 5.0)


def test_fit_lossless_and_threads(L):
    p, rep = fw.fit_relaxation(0.0, 1.0, 3)
    assert p.n_mech == 3 and p.kappa1 == 1.0 and list(p.d1[:3]) == [0, 0, 0]
    p1, r1 = fw.fit_relaxation(0.4, 1.2, 2, maxiter=500, n_threads=1)
    p4, r4 = fw.fit_relaxation(0.4, 1.2, 2, maxiter=500, n_threads=4)
    assert r1.J == r4.J and r1.w == r4.w


def test_missing_library_fails_loudly(tmp_path):
    """No fallback path: loading from a path without the library raises."""
    from paper_2606_11103_gb300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            _lib.load(str(tmp_path / "libfullwave_gb.so"))
    finally:
        _lib._lib = saved
