"""Per-voxel FP64 coefficient arrays in the paper's form (test infrastructure only).

* K = rho c^2 and the p update factor K dt (Eq. wave2 with kappa = 1/K);
* face density: arithmetic mean of the two cells that share the face (the last
  face of a non-periodic axis takes the cell's own rho);
* recursion coefficients per mechanism (Eqs. relaxation_a, relaxation_b):
      b = exp(-(d/kappa + alpha) dt),  a = d / (kappa (d + kappa alpha)) (b - 1);
* a velocity point v_d[i] (at i + 1/2 along d) takes the relaxation class of
  cell i, its lower neighbour;
* absorbing boundary: one more mechanism per direction, same Debye form, in a
  layer of L_T transition + L_B absorbing cells on every side.  The maps of
  that layer are inherited from the nearest interior cell (the adaptive PML
  of Sec. 4.6); the tissue mechanisms continue unchanged through it.
  Reading of the profile (the paper defers it to its Fullwave 2 reference):
  depth s [cells] from the inner edge of the layer,
      d(s) = 0.1 d_max (s/L_T)^2                   for s <= L_T,
      d(s) = d_max (0.1 + 0.9 ((s-L_T)/L_B)^2)     for s >  L_T,
      (L_T = 0: d(s) = d_max (s/L_B)^2),
      d_max = -3 c_max ln(R0) / (2 L_B dx),  R0 = 1e-5,
      alpha(s) = pi f0 (1 - s/(L_T+L_B)),
  and kappa of the mechanism = the tissue kappa of the point's stretch.
* two-stage layer (Sec. 4.6 methods, Sec. 5.4-5.5): the tissue ("higher-order")
  relaxation mechanisms are ramped across the transition region, and within
  the absorbing region when there is no transition layer, so that the
  absorbing mechanism alone acts at the outer edge.  Reading of the ramp:
  the strength of every tissue mechanism of a cell is multiplied by
      r(s) = 1 - (s / L_r)^2  for s < L_r,   0 beyond,
  with its relaxation rate d/kappa + alpha held fixed, i.e. d -> r d and
  alpha -> alpha + (1 - r) d / kappa, which gives a -> r a with b unchanged
  in Eqs. relaxation_a/b; s is the cell's depth into the layer (the largest
  over the axes, at the cell centre), L_r = L_T, or L_B / 2 when L_T = 0.
  Without it, tissue mechanisms added to a strong absorbing mechanism whose
  alpha vanishes at the outer edge make the low-frequency stretch negative
  there, and long runs diverge (the paper's no-transition variant diverged
  in 29 cells).
* time step from a CFL number: dt = CFL dx / max(c / sqrt(kappa_1 kappa_2)).
* time-space stencil (Sec. 3.3: 2M-th order in space and fourth order in
  time, after Tan & Huang, J. Comput. Phys. 276 (2014)), ``time_order=4``:
  every first derivative along d gets, besides its on-axis differences
  f(+m) - f(-m+1) (weights a_m), the two-point difference along d at the
  +-1 neighbours across every other axis (weight b).  Both come from the
  cell's Courant number r = c dt / dx by asking the plane-wave relation of
  the leapfrog scheme, sin(omega dt / 2) = (dt / 2) c |K(k)|, to hold for
  omega = c |k| to the orders the stencil can reach: b = r^2 / 24 from the
  k_d k_e^2 term, and for j = 1..M
      sum_m (2m - 1)^(2j - 1) a_m + 2 (D - 1) b = r^(2j - 2)
  from the k_d^(2j-1) terms along the axes.  r -> 0 gives b = 0 and the
  Taylor weights.  Velocity points use the coefficients of their cell.
"""
from __future__ import annotations

import math

import numpy as np

from .fit import RelaxParams


def class_table(params):
    """Stack a list of RelaxParams into arrays [n_class] / [n_class, N]."""
    n = params[0].n_mech
    for p in params:
        assert p.n_mech == n
    return dict(
        kappa1=np.array([p.kappa1 for p in params], dtype=np.float64),
        kappa2=np.array([p.kappa2 for p in params], dtype=np.float64),
        d1=np.array([p.d1 for p in params], dtype=np.float64).reshape(len(params), n),
        alpha1=np.array([p.alpha1 for p in params], dtype=np.float64).reshape(len(params), n),
        d2=np.array([p.d2 for p in params], dtype=np.float64).reshape(len(params), n),
        alpha2=np.array([p.alpha2 for p in params], dtype=np.float64).reshape(len(params), n),
    )


def recursion_ab(d, alpha, kappa, dt):
    """(a, b) of Eqs. relaxation_a / relaxation_b, elementwise, FP64."""
    d = np.asarray(d, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    kappa = np.asarray(kappa, dtype=np.float64)
    b = np.exp(-(d / kappa + alpha) * dt)
    a = d / (kappa * (d + kappa * alpha)) * (b - 1.0)
    return a, b


def time_space_coefficients(r, ndim, M=4):
    """(a [..., M], b [...]) of the time-space stencil for Courant numbers r
    (any shape), from its plane-wave conditions (module docstring)."""
    r = np.asarray(r, np.float64)
    b = r * r / 24.0
    V = np.array([[(2.0 * m - 1.0) ** (2 * j - 1) for m in range(1, M + 1)] for j in range(1, M + 1)])
    rhs = np.stack([r ** (2 * j - 2) - 2.0 * (ndim - 1) * b for j in range(1, M + 1)], axis=-1)
    a = np.linalg.solve(V, rhs.reshape(-1, M).T).T.reshape(r.shape + (M,))
    return a, b


def time_space_symbol(theta, a, b):
    """dx/2 times the symbol magnitude of each staggered derivative for a
    plane wave of phase advance theta[d] = k_d dx per cell: list over d of
    sum_m a_m sin((2m-1) theta_d / 2) + b sin(theta_d / 2) sum_{e != d} 2 cos theta_e."""
    nd = len(theta)
    out = []
    for d in range(nd):
        s = sum(a[m] * np.sin((2 * m + 1) * theta[d] / 2.0) for m in range(len(a)))
        cross = sum(2.0 * np.cos(theta[e]) for e in range(nd) if e != d)
        out.append(s + b * np.sin(theta[d] / 2.0) * cross)
    return out


def time_space_cfl_limit(ndim, n_theta=65):
    """Largest Courant number at which the lossless time-space scheme is
    stable: r max over theta of sqrt(sum_d symbol_d^2) <= 1 (bisection over
    r, theta on a grid over [0, pi]^D)."""
    g = np.linspace(0.0, np.pi, n_theta)
    th = np.meshgrid(*([g] * ndim), indexing="ij")
    lo, hi = 0.0, 1.0
    for _ in range(50):
        r = 0.5 * (lo + hi)
        a, b = time_space_coefficients(r, ndim)
        amp = r * np.sqrt(sum(s * s for s in time_space_symbol(th, a, b)))
        lo, hi = (r, hi) if amp.max() <= 1.0 else (lo, r)
    return lo


def cfl_dt(cfl, dx, c, cls, table):
    """dt = CFL dx / max over voxels of c/sqrt(kappa_1 kappa_2)."""
    ceff = np.asarray(c, np.float64) / np.sqrt(table["kappa1"][cls] * table["kappa2"][cls])
    return float(cfl * dx / np.max(ceff))


def _inherit(a, width, axes):
    """Replace the outer ``width`` layer of the listed axes by the nearest
    interior value."""
    a = np.asarray(a)
    if width <= 0:
        return a
    idx = []
    for ax, n in enumerate(a.shape):
        if ax in axes:
            lo, hi = min(width, n - 1), max(n - 1 - width, 0)
            if lo > hi:
                lo = hi = n // 2
            idx.append(np.clip(np.arange(n), lo, hi))
        else:
            idx.append(np.arange(n))
    return a[np.ix_(*idx)]


def absorbing_depth(n, width, staggered):
    """Depth s [cells] into the absorbing layer of points 0..n-1 along one axis
    (staggered: the point sits at i + 1/2)."""
    x = np.arange(n, dtype=np.float64) + (0.5 if staggered else 0.0)
    left = (width - 0.5) - x
    right = x - (n - width - 0.5)
    return np.maximum(0.0, np.maximum(left, right))


def tissue_ramp(shape, width, l_t, l_b, axes):
    """Factor r(s) on the strength of the tissue mechanisms of every cell
    (1 in the interior)."""
    s = np.zeros(shape)
    if width <= 0:
        return np.ones(shape)
    for ax in axes:
        bshape = [1] * len(shape)
        bshape[ax] = shape[ax]
        s = np.maximum(s, absorbing_depth(shape[ax], width, False).reshape(bshape))
    lr = l_t if l_t > 0 else 0.5 * l_b
    return np.where(s < lr, 1.0 - (s / lr) ** 2, 0.0)


def absorbing_profile(s, l_t, l_b, d_max, f0):
    s = np.asarray(s, dtype=np.float64)
    if l_t > 0:
        d = np.where(s <= l_t, 0.1 * d_max * (s / l_t) ** 2,
                     d_max * (0.1 + 0.9 * ((s - l_t) / l_b) ** 2))
    else:
        d = d_max * (s / l_b) ** 2
    d = np.where(s > 0.0, d, 0.0)
    alpha = math.pi * f0 * (1.0 - s / (l_t + l_b))
    return d, alpha


class OracleMedium:
    """Coefficient arrays of one medium (numpy C order; axis -1 is x).

    Parameters
    ----------
    shape      : (ny, nx) or (nz, ny, nx)
    c, rho     : maps [m/s], [kg/m^3]
    cls        : integer class map into ``params`` (list of RelaxParams)
    beta       : nonlinearity map or None
    pml, transition : L_B and L_T in cells (0 = no absorbing layer)
    periodic   : per numpy axis, for the pin tests (no absorbing layer on those axes)
    tissue_ramp_on : ramp the tissue mechanisms across the layer (the method);
                 False only to show what happens without it
    dscale     : optional per-voxel factor s on every d of the tissue mechanisms
                 (d^nu(x) = s(x) d^nu_class), a map like alpha0 and inherited
                 into the absorbing layer like the other maps
    layer_relax : keep the caller's class map inside the absorbing layer
                 instead of inheriting it (the homogeneous layers compared
                 with the adaptive one in Sec. 4.6: one fixed class there);
                 c, rho and beta are inherited either way
    time_order : 2 (leapfrog with the Taylor weights) or 4 (the time-space
                 stencil, per-cell coefficients from r = c dt / dx)
    """

    def __init__(self, shape, dx, dt, c, rho, cls, params, beta=None, pml=0, transition=0,
                 f0=3e6, R0=1e-5, periodic=None, dscale=None, tissue_ramp_on=True, layer_relax=False,
                 time_order=2):
        self.shape = tuple(shape)
        self.ndim = len(shape)
        self.dx, self.dt = float(dx), float(dt)
        self.periodic = tuple(periodic) if periodic is not None else (False,) * self.ndim
        width = pml + transition
        self.width = width
        self.pml, self.transition = pml, transition
        # the absorbing layer lines every non-periodic axis
        self.abs_axes = tuple(ax for ax in range(self.ndim) if not self.periodic[ax])
        inh = lambda a, dt_: _inherit(np.asarray(a, dt_), width, self.abs_axes)  # noqa: E731
        c = inh(c, np.float64)
        rho = inh(rho, np.float64)
        cls = np.array(cls, np.int64) if layer_relax else inh(cls, np.int64)
        beta = None if beta is None else inh(beta, np.float64)
        self.c, self.rho, self.cls = c, rho, cls
        self.dscale = None if dscale is None else inh(dscale, np.float64)
        tab = class_table(params)
        self.table = tab
        self.nmech = tab["d1"].shape[1]
        K = rho * c * c
        self.K = K
        self.kdt = K * self.dt
        assert time_order in (2, 4)
        self.time_order = time_order
        self.tha = self.thb = None
        if time_order == 4:
            a, b = time_space_coefficients(c * self.dt / self.dx, self.ndim)
            self.tha = [np.ascontiguousarray(a[..., m]) for m in range(4)]
            self.thb = np.ascontiguousarray(b)
        self.b2dt = None if (beta is None or not np.any(beta)) else 2.0 * beta * self.dt
        # face density per direction (numpy axis ax <-> direction d = ndim-1-ax)
        self.dt_rho = []
        for d in range(self.ndim):
            ax = self.ndim - 1 - d
            nxt = np.roll(rho, -1, axis=ax)
            if not self.periodic[ax]:
                last = [slice(None)] * self.ndim
                last[ax] = -1
                nxt[tuple(last)] = rho[tuple(last)]
            self.dt_rho.append(self.dt / (0.5 * (rho + nxt)))
        # tissue mechanisms, optional per-voxel scale of d (used by gradients w.r.t. alpha0)
        k1 = tab["kappa1"][cls]
        k2 = tab["kappa2"][cls]
        self.ik1 = 1.0 / k1
        self.ik2 = 1.0 / k2
        self.a1, self.b1, self.a2, self.b2 = [], [], [], []
        self.ramp = tissue_ramp(self.shape, width, transition, pml, self.abs_axes) if tissue_ramp_on \
            else np.ones(self.shape)
        for nu in range(self.nmech):
            sc = 1.0 if self.dscale is None else self.dscale
            # ramp: d -> r d at a fixed relaxation rate, i.e. a -> r a, b unchanged
            a, b = recursion_ab(tab["d1"][cls, nu] * sc, tab["alpha1"][cls, nu], k1, self.dt)
            self.a1.append(a * self.ramp)
            self.b1.append(b)
            a, b = recursion_ab(tab["d2"][cls, nu] * sc, tab["alpha2"][cls, nu], k2, self.dt)
            self.a2.append(a * self.ramp)
            self.b2.append(b)
        # absorbing mechanism per direction
        self.a1p = [None] * self.ndim
        self.b1p = [None] * self.ndim
        self.a2p = [None] * self.ndim
        self.b2p = [None] * self.ndim
        if width > 0:
            cmax = float(np.max(c))
            d_max = -3.0 * cmax * math.log(R0) / (2.0 * pml * self.dx)
            for d in range(self.ndim):
                ax = self.ndim - 1 - d
                if ax not in self.abs_axes:
                    continue
                n = self.shape[ax]
                bshape = [1] * self.ndim
                bshape[ax] = n
                for stag, k, dst_a, dst_b in ((True, k1, self.a1p, self.b1p),
                                              (False, k2, self.a2p, self.b2p)):
                    s = absorbing_depth(n, width, stag)
                    dd, al = absorbing_profile(s, transition, pml, d_max, f0)
                    dd = np.broadcast_to(dd.reshape(bshape), self.shape)
                    al = np.broadcast_to(al.reshape(bshape), self.shape)
                    a, b = recursion_ab(dd, al, k, self.dt)
                    dst_a[d] = np.ascontiguousarray(a)
                    dst_b[d] = np.ascontiguousarray(b)

    def source_gain(self, idx):
        """Volume-source gain K dt / dx^D at linear indices ``idx``."""
        return self.kdt.ravel()[idx] / self.dx ** self.ndim
