"""ctypes driver of the FP64 C stepper ``fw_oracle.c`` (test infrastructure only)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from .medium import OracleMedium

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_fw.so")
MAXMECH = 4

_P = C.POINTER(C.c_double)


class _Coeffs(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("n", C.c_int * 3), ("periodic", C.c_int * 3), ("nmech", C.c_int),
        ("dx", C.c_double),
        ("kdt", _P), ("b2dt", _P), ("dt_rho", _P * 3), ("ik1", _P * 3), ("ik2", _P),
        ("a1", (_P * 3) * MAXMECH), ("b1", (_P * 3) * MAXMECH),
        ("a2", (_P * 3) * MAXMECH), ("b2", (_P * 3) * MAXMECH),
        ("a1p", _P * 3), ("b1p", _P * 3), ("a2p", _P * 3), ("b2p", _P * 3),
        ("tha", _P * 4), ("thb", _P),
    ]


class _State(C.Structure):
    _fields_ = [
        ("p", _P), ("v", _P * 3),
        ("psi1", (_P * 3) * MAXMECH), ("psi2", (_P * 3) * MAXMECH),
        ("psi1p", _P * 3), ("psi2p", _P * 3),
    ]


def build(force=False):
    """Compile fw_oracle.c with gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_run.restype = C.c_int
        _lib.orc_run.argtypes = [C.POINTER(_Coeffs), C.POINTER(_State), C.c_int, C.c_int,
                                 C.c_int, C.POINTER(C.c_long), _P, C.POINTER(C.c_int), _P, C.c_int,
                                 C.c_int, C.POINTER(C.c_long), _P, C.c_int, C.c_int]
        _lib.orc_dplus.argtypes = [C.POINTER(_Coeffs), _P, _P, C.c_int]
        _lib.orc_dminus.argtypes = [C.POINTER(_Coeffs), _P, _P, C.c_int]
        _lib.orc_threads.restype = C.c_int
    return _lib


def threads():
    """Host threads the C stepper runs on."""
    return int(lib().orc_threads())


def _ptr(a):
    if a is None:
        return _P()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


class OracleSim:
    """State + coefficients of one oracle run; numpy views in C order."""

    def __init__(self, med: OracleMedium):
        self.med = med
        self.it = 0
        shape = med.shape
        nd = med.ndim
        z = lambda: np.zeros(shape, np.float64)  # noqa: E731
        self.p = z()
        self.v = [z() for _ in range(nd)]
        self.psi1 = [[z() for _ in range(nd)] for _ in range(med.nmech)]
        self.psi2 = [[z() for _ in range(nd)] for _ in range(med.nmech)]
        self.psi1p = [z() if med.a1p[d] is not None else None for d in range(nd)]
        self.psi2p = [z() if med.a2p[d] is not None else None for d in range(nd)]
        self._keep = []
        self._c = self._coeffs()
        self._s = self._state()
        self.sources = None
        self.receivers = None

    def _arr(self, a):
        a = np.ascontiguousarray(np.broadcast_to(a, self.med.shape), dtype=np.float64)
        self._keep.append(a)
        return a

    def _coeffs(self):
        m = self.med
        c = _Coeffs()
        c.ndim = m.ndim
        dims = list(reversed(m.shape)) + [1] * (3 - m.ndim)
        for i in range(3):
            c.n[i] = dims[i]
            c.periodic[i] = int(m.periodic[m.ndim - 1 - i]) if i < m.ndim else 0
        c.nmech = m.nmech
        c.dx = m.dx
        c.kdt = _ptr(self._arr(m.kdt))
        c.b2dt = _ptr(None if m.b2dt is None else self._arr(m.b2dt))
        ik2 = self._arr(m.ik2)
        c.ik2 = _ptr(ik2)
        ik1 = self._arr(m.ik1)
        for d in range(m.ndim):
            c.dt_rho[d] = _ptr(self._arr(m.dt_rho[d]))
            c.ik1[d] = _ptr(ik1)
            for nu in range(m.nmech):
                a1, b1 = self._arr(m.a1[nu]), self._arr(m.b1[nu])
                a2, b2 = self._arr(m.a2[nu]), self._arr(m.b2[nu])
                c.a1[nu][d], c.b1[nu][d] = _ptr(a1), _ptr(b1)
                c.a2[nu][d], c.b2[nu][d] = _ptr(a2), _ptr(b2)
            if m.a1p[d] is not None:
                c.a1p[d], c.b1p[d] = _ptr(self._arr(m.a1p[d])), _ptr(self._arr(m.b1p[d]))
                c.a2p[d], c.b2p[d] = _ptr(self._arr(m.a2p[d])), _ptr(self._arr(m.b2p[d]))
        if getattr(m, "thb", None) is not None:
            for k in range(4):
                c.tha[k] = _ptr(self._arr(m.tha[k]))
            c.thb = _ptr(self._arr(m.thb))
        return c

    def _state(self):
        s = _State()
        s.p = _ptr(self.p)
        for d in range(self.med.ndim):
            s.v[d] = _ptr(self.v[d])
            for nu in range(self.med.nmech):
                s.psi1[nu][d] = _ptr(self.psi1[nu][d])
                s.psi2[nu][d] = _ptr(self.psi2[nu][d])
            s.psi1p[d] = _ptr(self.psi1p[d])
            s.psi2p[d] = _ptr(self.psi2p[d])
        return s

    # -- sources / receivers --------------------------------------------------

    def set_sources(self, mask, waves, wave_of=None):
        idx = np.flatnonzero(np.asarray(mask).ravel()).astype(np.int64)
        waves = np.ascontiguousarray(np.atleast_2d(waves), dtype=np.float64)
        if wave_of is None:
            wave_of = np.zeros(idx.size, np.int32) if waves.shape[0] == 1 else np.arange(idx.size, dtype=np.int32)
        self.sources = dict(idx=idx, gain=np.ascontiguousarray(self.med.source_gain(idx), dtype=np.float64),
                            wave_of=np.ascontiguousarray(wave_of, dtype=np.int32), waves=waves)

    def set_receivers(self, mask, n_steps, decim=1):
        idx = np.flatnonzero(np.asarray(mask).ravel()).astype(np.int64)
        n_rec = (n_steps + decim - 1) // decim
        self.receivers = dict(idx=idx, traces=np.zeros((idx.size, n_rec), np.float64), decim=decim)

    def run(self, n_steps):
        L = lib()
        s = self.sources
        r = self.receivers
        if s is not None:
            src = (int(s["idx"].size), s["idx"].ctypes.data_as(C.POINTER(C.c_long)), _ptr(s["gain"]),
                   s["wave_of"].ctypes.data_as(C.POINTER(C.c_int)), _ptr(s["waves"]), int(s["waves"].shape[1]))
        else:
            src = (0, C.POINTER(C.c_long)(), _P(), C.POINTER(C.c_int)(), _P(), 0)
        if r is not None:
            rcv = (int(r["idx"].size), r["idx"].ctypes.data_as(C.POINTER(C.c_long)), _ptr(r["traces"]),
                   int(r["traces"].shape[1]), int(r["decim"]))
        else:
            rcv = (0, C.POINTER(C.c_long)(), _P(), 0, 1)
        rc = L.orc_run(C.byref(self._c), C.byref(self._s), int(n_steps), int(self.it), *src, *rcv)
        assert rc == 0
        self.it += n_steps

    @property
    def traces(self):
        return None if self.receivers is None else self.receivers["traces"]

    # -- derivative operators (pin tests) ------------------------------------

    def dplus(self, f, d):
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros_like(f)
        lib().orc_dplus(C.byref(self._c), _ptr(f), _ptr(out), d)
        return out

    def dminus(self, f, d):
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros_like(f)
        lib().orc_dminus(C.byref(self._c), _ptr(f), _ptr(out), d)
        return out


def simulate(spec, params, n_steps=None, periodic=None, beta=True, cls=None, dscale=None):
    """Run a synthetic workload spec on the oracle; returns the OracleSim."""
    n_steps = spec.n_steps if n_steps is None else n_steps
    cls = spec.maps["class_idx"] if cls is None else cls
    med = OracleMedium(spec.shape, spec.dx, spec.dt, spec.maps["c"], spec.maps["rho"], cls, params,
                       beta=spec.maps.get("beta") if beta else None, pml=spec.pml,
                       transition=spec.transition, f0=spec.f0, periodic=periodic, dscale=dscale)
    sim = OracleSim(med)
    sim.set_sources(spec.src_mask, spec.src_waves, spec.src_wave_of)
    sim.set_receivers(spec.rcv_mask, n_steps, spec.decim)
    sim.run(n_steps)
    return sim
