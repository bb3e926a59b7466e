"""Seeded synthetic media, sources and receivers for the five workloads.

Array conventions (shared by every consumer):

* 2D maps are C-order ``[ny][nx]``; 3D maps are C-order ``[nz][ny][nx]``;
  x is the fastest axis, the first axis is the propagation (depth) axis.
* Materials: ``c`` [m/s], ``rho`` [kg/m^3], ``beta`` [-], ``alpha0`` in
  dB/(MHz^y cm) and ``y`` [-], all float32.
* A source waveform is a volume-injection rate per source cell [m^D/s]; the
  amplitude helper converts a wanted plane-wave pressure amplitude A [Pa] into
  such a rate with the nominal factor 2*A*dx^(D-1)/(rho*c) (a one-cell-thick
  planar source emits two plane waves).
* Waveform sample ``n`` belongs to time ``n*dt`` and is injected by time step n.

Nothing here performs any part of the simulation or of the relaxation fit.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# ---------------------------------------------------------------------------
# waveform and masks


def gaussian_pulse(f0: float, dt: float, n_steps: int, amp: float = 1.0,
                   t0: Optional[float] = None, tau: Optional[float] = None,
                   delay: float = 0.0) -> np.ndarray:
    """Gaussian-modulated sinusoid A sin(2 pi f0 (t-t0)) exp(-((t-t0)/tau)^2).

    Defaults tau = 1/f0 and t0 = 3 tau; ``delay`` shifts the pulse later.
    Returns float64 samples at t = n*dt, n = 0..n_steps-1.
    """
    tau = 1.0 / f0 if tau is None else tau
    t0 = 3.0 * tau if t0 is None else t0
    t = np.arange(n_steps, dtype=np.float64) * dt - t0 - delay
    return amp * np.sin(2.0 * np.pi * f0 * t) * np.exp(-(t / tau) ** 2)


def plane_amplitude_rate(amp_pa: float, dx: float, ndim: int, rho: float, c: float) -> float:
    """Nominal injection-rate amplitude that yields ~amp_pa from a planar source."""
    return 2.0 * amp_pa * dx ** (ndim - 1) / (rho * c)


def line_source_mask(shape, row: int) -> np.ndarray:
    """All cells of depth index ``row`` (a line in 2D, a plane in 3D)."""
    m = np.zeros(shape, dtype=np.uint8)
    m[row] = 1
    return m


# ---------------------------------------------------------------------------
# media


def homogeneous_medium(shape, c=1540.0, rho=1000.0, alpha0=0.5, y=1.1, beta=0.0):
    """Constant maps of the given shape (float32)."""
    f = lambda v: np.full(shape, v, dtype=np.float32)  # noqa: E731
    return dict(c=f(c), rho=f(rho), alpha0=f(alpha0), y=f(y), beta=f(beta))


def two_layer_medium(shape, layer_a: dict, layer_b: dict, interface: Optional[int] = None):
    """Planar interface normal to the depth axis; layer A above ``interface``."""
    n0 = shape[0]
    k = n0 // 2 if interface is None else interface
    out = {}
    for key in ("c", "rho", "alpha0", "y", "beta"):
        a = np.empty(shape, dtype=np.float32)
        a[:k] = layer_a.get(key, 0.0)
        a[k:] = layer_b.get(key, 0.0)
        out[key] = a
    return out


@dataclass
class VoronoiClasses:
    seeds: np.ndarray        # [n_seed, ndim] float64, in cell units, (depth, ..., x) order
    seed_class: np.ndarray   # [n_seed] int
    alpha0: np.ndarray       # [n_class]
    y: np.ndarray
    c: np.ndarray
    rho: np.ndarray


def voronoi_classes(seed: int, shape, n_seed: int, n_class: int,
                    alpha0_range=(0.0022, 1.0), y_range=(0.4, 2.0),
                    c_range=(1450.0, 1600.0), rho_range=(900.0, 1100.0)) -> VoronoiClasses:
    """Seed points and per-class parameters drawn uniformly (seeded)."""
    rng = np.random.default_rng(seed)
    seeds = rng.uniform(0.0, 1.0, size=(n_seed, len(shape))) * np.asarray(shape, dtype=np.float64)
    seed_class = rng.integers(0, n_class, size=n_seed)
    a0 = rng.uniform(*alpha0_range, size=n_class)
    yy = rng.uniform(*y_range, size=n_class)
    cc = rng.uniform(*c_range, size=n_class)
    rr = rng.uniform(*rho_range, size=n_class)
    return VoronoiClasses(seeds, seed_class, a0, yy, cc, rr)


def _nearest_seed_plane(depth: float, inner_axes, seeds: np.ndarray) -> np.ndarray:
    """Nearest seed (squared Euclidean distance, ties -> lowest seed index)
    for every point of one depth plane; ``inner_axes`` holds the cell-centre
    coordinates of the remaining axes.  The squared distance is a sum of
    per-axis terms, evaluated in float64 with torch on the CPU when it is
    importable (multi-threaded), else with numpy."""
    terms = [(depth - seeds[:, 0]) ** 2]
    for a, coords in enumerate(inner_axes):
        terms.append((coords[:, None] - seeds[None, :, a + 1]) ** 2)   # [n_a, n_seed]
    try:
        import torch
        t = [torch.from_numpy(np.ascontiguousarray(x)) for x in terms]
        d2 = t[0].view(*([1] * len(inner_axes)), -1)
        for a in range(len(inner_axes)):
            shp = [1] * len(inner_axes) + [-1]
            shp[a] = t[a + 1].shape[0]
            d2 = d2 + t[a + 1].view(*shp)
        return torch.argmin(d2, dim=-1).numpy()
    except ImportError:  # pragma: no cover
        d2 = terms[0].reshape(*([1] * len(inner_axes)), -1)
        for a in range(len(inner_axes)):
            shp = [1] * len(inner_axes) + [-1]
            shp[a] = terms[a + 1].shape[0]
            d2 = d2 + terms[a + 1].reshape(shp)
        return np.argmin(d2, axis=-1)


def voronoi_medium(vc: VoronoiClasses, shape, seed: int, jitter: float = 0.02,
                   box=None, with_maps: bool = True):
    """Voronoi class map plus per-voxel c/rho jitter, optionally on a sub-box.

    ``box`` = tuple of (start, stop) per axis selects a crop of the full
    ``shape`` grid; the crop is bitwise identical to slicing the full map,
    because the jitter of depth plane k is drawn from its own generator
    seeded with (seed, k) over the full plane.  Jitter is c*(1+j*N(0,1)) with
    N clipped at +-3.
    """
    if box is None:
        box = tuple((0, n) for n in shape)
    sub = tuple(b - a for a, b in box)
    cls = np.empty(sub, dtype=np.uint16)
    cmap = np.empty(sub, dtype=np.float32)
    rmap = np.empty(sub, dtype=np.float32)
    inner_full = shape[1:]
    inner_box = box[1:]
    inner_axes = [np.arange(a, b, dtype=np.float64) + 0.5 for a, b in inner_box]
    for kk, k in enumerate(range(box[0][0], box[0][1])):
        near = _nearest_seed_plane(k + 0.5, inner_axes, vc.seeds)
        cl = vc.seed_class[near].reshape(sub[1:])
        cls[kk] = cl
        if with_maps:
            rng = np.random.default_rng([seed, k])
            n_full = int(np.prod(inner_full))
            jc = np.clip(rng.standard_normal(n_full), -3.0, 3.0).reshape(inner_full)
            jr = np.clip(rng.standard_normal(n_full), -3.0, 3.0).reshape(inner_full)
            sl = tuple(slice(a, b) for a, b in inner_box)
            cmap[kk] = vc.c[cl] * (1.0 + jitter * jc[sl])
            rmap[kk] = vc.rho[cl] * (1.0 + jitter * jr[sl])
    out = dict(class_idx=cls)
    if with_maps:
        out.update(c=cmap, rho=rmap,
                   alpha0=vc.alpha0.astype(np.float32)[cls],
                   y=vc.y.astype(np.float32)[cls],
                   beta=np.zeros(sub, dtype=np.float32))
    return out


# ---------------------------------------------------------------------------
# workload specifications


@dataclass
class WorkloadSpec:
    name: str
    shape: tuple                 # (ny, nx) or (nz, ny, nx)
    dx: float
    dt: float
    f0: float
    pml: int
    transition: int
    n_mech: int
    n_steps: int
    maps: dict                   # c, rho, beta, alpha0, y (float32) [+ class_idx]
    src_mask: np.ndarray
    src_waves: np.ndarray        # [n_wave, n_steps] float32
    src_wave_of: Optional[np.ndarray]  # [n_src] int32 (mask order) or None
    rcv_mask: np.ndarray
    decim: int = 1
    classes: Optional[dict] = None     # {'alpha0': [...], 'y': [...]} when class_idx given
    extra: dict = field(default_factory=dict)

    @property
    def ndim(self):
        return len(self.shape)


def _dt_from_cfl(cfl, dx, c_map):
    return float(cfl * dx / float(np.max(c_map)))


def config_c1(n: int = 256, n_steps: int = 1000, amp: float = 1e3) -> WorkloadSpec:
    """2D homogeneous lossy medium: c 1540, rho 1000, alpha0 0.5, y 1.1, N=2,
    dx = lambda/12 at 3 MHz, 20-cell PML, CFL 0.4, line source at row 24,
    receivers on the centre column."""
    f0 = 3e6
    dx = 1540.0 / (f0 * 12)
    shape = (n, n)
    maps = homogeneous_medium(shape)
    dt = _dt_from_cfl(0.4, dx, maps["c"])
    src = line_source_mask(shape, 24)
    wave = gaussian_pulse(f0, dt, n_steps, plane_amplitude_rate(amp, dx, 2, 1000.0, 1540.0))
    rcv = np.zeros(shape, np.uint8)
    rcv[:, n // 2] = 1
    return WorkloadSpec("c1_2d_homog_256", shape, dx, dt, f0, 20, 0, 2, n_steps, maps,
                        src, wave[None].astype(np.float32), None, rcv, 1)


def config_c2(n: int = 2048, n_steps: int = 5000, amp: float = 1e3, nonlinear: bool = True,
              pml: int = 30) -> WorkloadSpec:
    """2D two-layer medium (A: c 1580 rho 1060 a0 1.09 y 1.0 beta 3.5;
    B: c 1450 rho 950 a0 0.6 y 1.5 beta 6.0), N=4, 30-cell PML, 3 MHz line
    source, receivers on the centre column."""
    f0 = 3e6
    dx = 1450.0 / (f0 * 12)
    shape = (n, n)
    la = dict(c=1580.0, rho=1060.0, alpha0=1.09, y=1.0, beta=3.5 if nonlinear else 0.0)
    lb = dict(c=1450.0, rho=950.0, alpha0=0.6, y=1.5, beta=6.0 if nonlinear else 0.0)
    maps = two_layer_medium(shape, la, lb)
    dt = _dt_from_cfl(0.4, dx, maps["c"])
    row = pml + 4
    src = line_source_mask(shape, row)
    wave = gaussian_pulse(f0, dt, n_steps, plane_amplitude_rate(amp, dx, 2, 1060.0, 1580.0))
    rcv = np.zeros(shape, np.uint8)
    rcv[:, n // 2] = 1
    return WorkloadSpec("c2_2d_twolayer_%d" % n, shape, dx, dt, f0, pml, 0, 4, n_steps, maps,
                        src, wave[None].astype(np.float32), None, rcv, 1,
                        extra=dict(layer_a=la, layer_b=lb, interface=n // 2, src_row=row))


C3_SHAPE = (512, 512, 512)


def c3_classes() -> VoronoiClasses:
    return voronoi_classes(2, C3_SHAPE, n_seed=64, n_class=8)


def config_c3(n_steps: int = 2000, box=None, amp: float = 1e3, aperture: int = 256,
              src_plane: int = 24, focus_cells: int = 256, rcv_stride: int = 8) -> WorkloadSpec:
    """3D seeded Voronoi tissue map 512^3 (64 seeds, 8 classes), 2% c/rho
    jitter, N=4, 20-cell PML, 3 MHz square aperture on plane z=24 focused at
    256 cells depth, receivers on a strided grid of that plane.

    ``box`` selects a crop of the 512^3 map (same generator and seed); the
    source and receivers are clipped to the crop.
    """
    f0 = 3e6
    dx = 1540.0 / (f0 * 12)
    vc = c3_classes()
    full = C3_SHAPE
    if box is None:
        box = tuple((0, n) for n in full)
    med = voronoi_medium(vc, full, seed=2, box=box)
    shape = tuple(b - a for a, b in box)
    # dt from the full-size map's maximum speed bound: class max * (1 + 3*0.02)
    cmax = float(np.max(vc.c)) * 1.06
    dt = float(0.4 * dx / cmax)
    # focused planar aperture, centred laterally in the full grid
    n_y, n_x = full[1], full[2]
    a0y, a0x = (n_y - aperture) // 2, (n_x - aperture) // 2
    yy, xx = np.meshgrid(np.arange(aperture) + a0y, np.arange(aperture) + a0x, indexing="ij")
    r2 = ((yy + 0.5 - n_y / 2) ** 2 + (xx + 0.5 - n_x / 2) ** 2) * dx * dx
    F = focus_cells * dx
    tau = (np.sqrt(r2 + F * F) - F) / 1540.0
    tau = tau.max() - tau                       # outer elements fire first
    # one waveform per distinct delay (radially symmetric aperture)
    uniq, inv = np.unique(np.round(tau / dt * 64.0).astype(np.int64), return_inverse=True)
    src_mask = np.zeros(shape, np.uint8)
    wave_of_full = inv.reshape(aperture, aperture).astype(np.int32)
    z_in = box[0][0] <= src_plane < box[0][1]
    sel = np.zeros((aperture, aperture), bool)
    if z_in:
        sel = ((yy >= box[1][0]) & (yy < box[1][1]) & (xx >= box[2][0]) & (xx < box[2][1]))
        src_mask[src_plane - box[0][0], yy[sel] - box[1][0], xx[sel] - box[2][0]] = 1
    # mask order (C order) matches the row-major order of the selected elements
    wave_of = wave_of_full[sel].astype(np.int32)
    used = np.unique(wave_of) if wave_of.size else np.zeros(0, np.int64)
    remap = -np.ones(len(uniq), np.int64)
    remap[used] = np.arange(len(used))
    wave_of = remap[wave_of].astype(np.int32)
    rate = plane_amplitude_rate(amp, dx, 3, 1000.0, 1540.0)
    waves = np.stack([gaussian_pulse(f0, dt, n_steps, rate, delay=uniq[u] * dt / 64.0)
                      for u in used]) if len(used) else np.zeros((1, n_steps))
    rcv = np.zeros(shape, np.uint8)
    zr = src_plane + 2
    if box[0][0] <= zr < box[0][1]:
        ys = np.arange(a0y, a0y + aperture, rcv_stride)
        xs = np.arange(a0x, a0x + aperture, rcv_stride)
        ys = ys[(ys >= box[1][0]) & (ys < box[1][1])] - box[1][0]
        xs = xs[(xs >= box[2][0]) & (xs < box[2][1])] - box[2][0]
        rcv[zr - box[0][0]][np.ix_(ys, xs)] = 1
    classes = dict(alpha0=vc.alpha0.copy(), y=vc.y.copy(), c=vc.c.copy(), rho=vc.rho.copy())
    return WorkloadSpec("c3_3d_voronoi_512" if shape == full else "c3_3d_voronoi_crop%d" % shape[0],
                        shape, dx, dt, f0, 20, 0, 4, n_steps, med,
                        src_mask, waves.astype(np.float32), wave_of if len(used) else None,
                        rcv, 1, classes=classes, extra=dict(box=box))


def config_c5(n: int = 1024, n_steps: int = 3000, amp: float = 1e3, perturbed: bool = False) -> WorkloadSpec:
    """2D 1024^2 Voronoi (32 seeds, 6 classes), N=3, 20-cell PML, 3 MHz line
    source at the top, 64 receivers on a row 8 cells below it.  With
    ``perturbed`` the 'true' medium: c +1% and alpha0 +20% inside a seeded
    Gaussian blob (weight exp(-r^2/(2 s^2)), s = n/16)."""
    f0 = 3e6
    dx = 1540.0 / (f0 * 12)
    shape = (n, n)
    vc = voronoi_classes(4, shape, n_seed=32, n_class=6)
    med = voronoi_medium(vc, shape, seed=4)
    if perturbed:
        rng = np.random.default_rng(40)
        cy, cx = rng.uniform(0.3, 0.7, size=2) * n
        s = n / 16.0
        yy, xx = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
        wgt = np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * s * s)).astype(np.float32)
        med["c"] = (med["c"] * (1 + 0.01 * wgt)).astype(np.float32)
        med["alpha0"] = (med["alpha0"] * (1 + 0.20 * wgt)).astype(np.float32)
    dt = float(0.4 * dx / (float(np.max(vc.c)) * 1.06 * 1.01))
    row = 24
    src = line_source_mask(shape, row)
    wave = gaussian_pulse(f0, dt, n_steps, plane_amplitude_rate(amp, dx, 2, 1000.0, 1540.0))
    rcv = np.zeros(shape, np.uint8)
    xs = np.linspace(20 + 4, n - 20 - 5, 64).round().astype(int)
    rcv[row + 8, xs] = 1
    classes = dict(alpha0=vc.alpha0.copy(), y=vc.y.copy(), c=vc.c.copy(), rho=vc.rho.copy())
    return WorkloadSpec("c5_2d_voronoi_%d" % n, shape, dx, dt, f0, 20, 0, 3, n_steps, med,
                        src, wave[None].astype(np.float32), None, rcv, 1, classes=classes)


def serving_stream(seed: int = 3, n_req: int = 200, rate_hz: float = 1.0,
                   sides_2d=(512, 1024, 2048, 4096), side_3d=(128, 384),
                   steps=(500, 3000)):
    """Poisson arrival stream of simulation requests (descriptors only).

    Each request: arrival time [s], ndim, shape, n_steps and a per-request
    Voronoi seed; half 2D (side uniform in ``sides_2d``), half 3D (side a
    multiple of 32 uniform in ``side_3d``).
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n_req)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    sides3 = np.arange(side_3d[0], side_3d[1] + 1, 32)
    for i in range(n_req):
        if rng.uniform() < 0.5:
            s = int(rng.choice(sides_2d))
            shape = (s, s)
        else:
            s = int(rng.choice(sides3))
            shape = (s, s, s)
        reqs.append(dict(id=i, arrival=float(t[i]), shape=shape,
                         n_steps=int(rng.integers(steps[0], steps[1] + 1)),
                         seed=int(rng.integers(0, 2 ** 31 - 1))))
    return reqs
