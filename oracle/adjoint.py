"""Gradient of a receiver functional by the discrete adjoint, FP64 (test
infrastructure only).

The forward problem is the oracle stepper (Sec. 2.1, Sec. 3.3); the paper
uses full-wave simulation as the forward model of inverse problems but gives
no gradient method, so this module takes the plainest exact one: the
transpose of the discrete time step (reverse-mode differentiation of the
stepper, written out in ``orc_adjoint_step`` of ``fw_oracle.c``), run
backwards over forward states recomputed from checkpoints.

Functional:  L = sum_{r, col} G[r, col] * trace[r, col]   (G = dL/dtraces,
e.g. the residual trace - d_obs of the misfit 1/2 |trace - d_obs|^2).

Parameters (readings stated in the design notes):

* c(x): enters through K dt = rho c^2 dt (the pressure update and the
  volume-source gain K dt / dx^D); dt, the absorbing profile (through
  c_max) and the relaxation parameters are held fixed;
* alpha0(x): per voxel the mechanisms of the voxel's class are scaled as
  d^nu(x) = d^nu_class * s(x), s(x) = alpha0(x) / alpha0_class, with kappa
  and alpha^nu at the class values, so dL/dalpha0 = dL/ds / alpha0_class;
* every map of the absorbing layer is inherited from the nearest interior
  cell, so the gradient with respect to the user's map folds the layer's
  values back onto the cells they came from.

Only the linear system (no nonlinear factor) is differentiated.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .medium import OracleMedium
from .stepper import MAXMECH, OracleSim, _P, _ptr, lib


class _DCoeffs(C.Structure):
    _fields_ = [("da1", (_P * 3) * MAXMECH), ("db1", (_P * 3) * MAXMECH),
                ("da2", (_P * 3) * MAXMECH), ("db2", (_P * 3) * MAXMECH)]


def recursion_ab_dscale(d, alpha, kappa, dt, s):
    """Derivatives with respect to s of (a, b) of Eqs. relaxation_a /
    relaxation_b evaluated at d*s:
        b = exp(-(d s / kappa + alpha) dt),   db/ds = -(d dt / kappa) b,
        a = D / (kappa (D + kappa alpha)) (b - 1),  D = d s,
        da/ds = d alpha (b - 1) / (D + kappa alpha)^2 + D / (kappa (D + kappa alpha)) db/ds."""
    d = np.asarray(d, np.float64)
    alpha = np.asarray(alpha, np.float64)
    kappa = np.asarray(kappa, np.float64)
    D = d * s
    b = np.exp(-(D / kappa + alpha) * dt)
    db = -(d * dt / kappa) * b
    da = d * alpha * (b - 1.0) / (D + kappa * alpha) ** 2 + D / (kappa * (D + kappa * alpha)) * db
    return da, db


def fold_inherited(g, med: OracleMedium):
    """Transpose of the absorbing-layer inheritance: sum every internal value
    onto the interior cell it was copied from."""
    g = np.asarray(g, np.float64)
    if med.width <= 0:
        return g.copy()
    idx = []
    for ax, n in enumerate(g.shape):
        if ax in med.abs_axes:
            lo, hi = min(med.width, n - 1), max(n - 1 - med.width, 0)
            if lo > hi:
                lo = hi = n // 2
            idx.append(np.clip(np.arange(n), lo, hi))
        else:
            idx.append(np.arange(n))
    out = np.zeros_like(g)
    np.add.at(out, np.ix_(*idx), g)
    return out


class _Snapshot:
    """Copy of every state array of an OracleSim."""

    def __init__(self, sim: OracleSim):
        self.p = sim.p.copy()
        self.v = [a.copy() for a in sim.v]
        self.psi1 = [[a.copy() for a in row] for row in sim.psi1]
        self.psi2 = [[a.copy() for a in row] for row in sim.psi2]
        self.psi1p = [None if a is None else a.copy() for a in sim.psi1p]
        self.psi2p = [None if a is None else a.copy() for a in sim.psi2p]
        self.it = sim.it

    def restore(self, sim: OracleSim):
        np.copyto(sim.p, self.p)
        for a, b in zip(sim.v, self.v):
            np.copyto(a, b)
        for ra, rb in zip(sim.psi1, self.psi1):
            for a, b in zip(ra, rb):
                np.copyto(a, b)
        for ra, rb in zip(sim.psi2, self.psi2):
            for a, b in zip(ra, rb):
                np.copyto(a, b)
        for a, b in zip(sim.psi1p + sim.psi2p, self.psi1p + self.psi2p):
            if a is not None:
                np.copyto(a, b)
        sim.it = self.it


def _state_struct(snap, keep):
    from .stepper import _State
    s = _State()
    s.p = _ptr(snap.p)
    for d in range(len(snap.v)):
        s.v[d] = _ptr(snap.v[d])
        for nu in range(len(snap.psi1)):
            s.psi1[nu][d] = _ptr(snap.psi1[nu][d])
            s.psi2[nu][d] = _ptr(snap.psi2[nu][d])
        s.psi1p[d] = _ptr(snap.psi1p[d])
        s.psi2p[d] = _ptr(snap.psi2p[d])
    keep.append(snap)
    return s


class Adjoint:
    """Discrete adjoint of one OracleSim set-up (sources and receivers set)."""

    def __init__(self, sim: OracleSim):
        med = sim.med
        if med.b2dt is not None:
            raise ValueError("the adjoint differentiates the linear system only")
        self.sim = sim
        self.med = med
        tab, cls, dt = med.table, med.cls, med.dt
        s = 1.0 if med.dscale is None else med.dscale
        ramp = med.ramp
        k1 = tab["kappa1"][cls]
        k2 = tab["kappa2"][cls]
        self._keep = []
        dc = _DCoeffs()
        for nu in range(med.nmech):
            # the layer ramp scales a (not b): a = r a_class(d s), so da/ds = r da_class/ds
            da1, db1 = recursion_ab_dscale(tab["d1"][cls, nu], tab["alpha1"][cls, nu], k1, dt, s)
            da2, db2 = recursion_ab_dscale(tab["d2"][cls, nu], tab["alpha2"][cls, nu], k2, dt, s)
            da1, da2 = da1 * ramp, da2 * ramp
            arrs = [np.ascontiguousarray(np.broadcast_to(a, med.shape), np.float64) for a in (da1, db1, da2, db2)]
            self._keep += arrs
            for d in range(med.ndim):
                dc.da1[nu][d], dc.db1[nu][d] = _ptr(arrs[0]), _ptr(arrs[1])
                dc.da2[nu][d], dc.db2[nu][d] = _ptr(arrs[2]), _ptr(arrs[3])
        self.dc = dc
        L = lib()
        L.orc_adjoint_step.restype = C.c_int
        L.orc_adjoint_step.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(_P), C.c_void_p, C.c_void_p,
                                       _P, _P, C.POINTER(_P), C.POINTER(_P)]

    # -- one reverse step -------------------------------------------------------
    def step_transpose(self, fwd: _Snapshot, v_after, lam: _Snapshot, grad_kdt, grad_s):
        """lam: adjoint of the state after the step -> before it (in place)."""
        med = self.med
        keep = []
        f = _state_struct(fwd, keep)
        ls = _state_struct(lam, keep)
        vh = (_P * 3)(*[_ptr(v_after[d]) for d in range(med.ndim)] + [_P()] * (3 - med.ndim))
        wq = [np.zeros(med.shape) for _ in range(med.ndim)]
        wg = [np.zeros(med.shape) for _ in range(med.ndim)]
        pq = (_P * 3)(*[_ptr(a) for a in wq] + [_P()] * (3 - med.ndim))
        pg = (_P * 3)(*[_ptr(a) for a in wg] + [_P()] * (3 - med.ndim))
        rc = lib().orc_adjoint_step(C.addressof(self.sim._c), C.addressof(f), vh, C.addressof(ls),
                                    C.addressof(self.dc), _ptr(grad_kdt), _ptr(grad_s), pq, pg)
        assert rc == 0

    def zero_like_state(self):
        lam = _Snapshot(self.sim)
        for a in [lam.p] + lam.v + [x for r in lam.psi1 for x in r] + [x for r in lam.psi2 for x in r] + \
                [x for x in lam.psi1p + lam.psi2p if x is not None]:
            a[...] = 0.0
        return lam

    # -- full gradient ------------------------------------------------------------
    def gradient(self, n_steps, G, checkpoint=100):
        """Run n_steps forward from the simulator's current state (recording
        traces), then the adjoint of L = sum G * traces.  Returns dict with
        dL/d(K dt) and dL/ds on the internal grid and the folded gradients
        dL/dc and dL/ds on the user's grid."""
        sim, med = self.sim, self.med
        src, rcv = sim.sources, sim.receivers
        it0 = sim.it
        G = np.asarray(G, np.float64)
        ckpt = []
        for k in range(0, n_steps, checkpoint):
            ckpt.append(_Snapshot(sim))
            sim.run(min(checkpoint, n_steps - k))
        traces = None if rcv is None else rcv["traces"].copy()
        final = _Snapshot(sim)
        grad_kdt = np.zeros(med.shape)
        grad_s = np.zeros(med.shape)
        lam = self.zero_like_state()
        flat = lambda a: a.reshape(-1)  # noqa: E731
        inv_dxd = 1.0 / med.dx ** med.ndim
        for si in range(len(ckpt) - 1, -1, -1):
            ckpt[si].restore(sim)
            seg = [_Snapshot(sim)]
            k0 = si * checkpoint
            k1 = min(n_steps, k0 + checkpoint)
            for _ in range(k0, k1):
                sim.run(1)
                seg.append(_Snapshot(sim))
            for k in range(k1 - 1, k0 - 1, -1):
                it = it0 + k
                if rcv is not None and rcv["idx"].size and it % rcv["decim"] == 0 and \
                        it // rcv["decim"] < G.shape[1]:
                    np.add.at(flat(lam.p), rcv["idx"], G[:, it // rcv["decim"]])
                if src is not None and src["idx"].size and it < src["waves"].shape[1]:
                    w = src["waves"][src["wave_of"], it]
                    np.add.at(flat(grad_kdt), src["idx"], w * inv_dxd * flat(lam.p)[src["idx"]])
                self.step_transpose(seg[k - k0], seg[k - k0 + 1].v, lam, grad_kdt, grad_s)
        final.restore(sim)            # leave the simulator at the end of the run
        grad_c_int = grad_kdt * 2.0 * med.rho * med.c * med.dt
        return dict(traces=traces, grad_kdt=grad_kdt, grad_s=grad_s,
                    grad_c=fold_inherited(grad_c_int, med), grad_s_user=fold_inherited(grad_s, med),
                    lam=lam)


def misfit_gradient(shape, dx, dt, c, rho, cls, params, alpha0_class, n_steps, src_mask, waves, rcv_mask,
                    G=None, d_obs=None, wave_of=None, pml=0, transition=0, f0=3e6, checkpoint=100, dscale=None,
                    decim=1):
    """Gradient of L = sum G * traces (or of 1/2 |traces - d_obs|^2 when G is
    None) with respect to c(x) and alpha0(x) on the user's grid."""
    med = OracleMedium(shape, dx, dt, c, rho, cls, params, pml=pml, transition=transition, f0=f0,
                       dscale=dscale)
    sim = OracleSim(med)
    sim.set_sources(src_mask, waves, wave_of)
    sim.set_receivers(rcv_mask, n_steps, decim)
    adj = Adjoint(sim)
    if G is None:
        # the residual needs the traces first: one plain forward run
        probe = OracleSim(med)
        probe.set_sources(src_mask, waves, wave_of)
        probe.set_receivers(rcv_mask, n_steps, decim)
        probe.run(n_steps)
        G = probe.traces - d_obs
    out = adj.gradient(n_steps, G, checkpoint)
    a0c = np.asarray(alpha0_class, np.float64)[np.asarray(cls)]
    out["grad_alpha0"] = np.where(a0c > 0, out["grad_s_user"] / np.where(a0c > 0, a0c, 1.0), 0.0)
    return out
