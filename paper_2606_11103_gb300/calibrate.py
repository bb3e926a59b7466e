"""Simulation-based weight selection of the relaxation calibration (Sec. 3.2):
the relaxation set is fitted once per real/imaginary balance weight w, each
candidate is simulated on the GPU in the attenuation and dispersion protocol
of Sec. 4.1-4.2, and the candidate with the lowest simulated attenuation
NRMSE is kept, the absolute dispersion error breaking ties; a calibration
whose best NRMSE exceeds 10 % or whose dispersion error exceeds 5 m/s is
labelled failed.

Protocol (Sec. 4.1-4.2): a plane wave (line source across the top of a
domain D = 10 lambda deep and W = 50 lambda wide, lambda at the centre
frequency) of Gaussian-modulated sinusoidal pulses at centre frequencies
1-20 MHz in 2.71 MHz steps; receivers on the centre column at 0.05 D and
0.8 D below the source.  Per centre frequency f0 the spectra of the two
traces give, over 0.7-1.3 f0 where the first is within -20 dB of its peak,
the attenuation alpha(f) = -ln(|P2|/|P1|)/d and the phase velocity
c(f) = 2 pi f d / phi(f), phi the phase delay between the receivers.
NRMSE = RMS(alpha - alpha0 f^y) / (range of alpha0 f^y over the measured
frequencies); dispersion error = RMS(c - c_KK), c_KK from the
Kramers-Kronig relation of Eq. kk_relation.

The simulations run on the CUDA path (Medium); the spectra are host work.
"""
from __future__ import annotations

import math

import numpy as np

CENTRES = tuple(float(f) for f in np.arange(1e6, 20.01e6, 2.71e6))


def _targets(alpha0, y, f_hz, c0=1540.0, f_ref=1e6):
    """(alpha0 f^y [Np/m], Kramers-Kronig phase velocity [m/s]) at f_hz from
    the library's fw_fit_targets (the fit's own arithmetic)."""
    import ctypes as C

    from . import _lib

    f = np.ascontiguousarray(np.atleast_1d(np.asarray(f_hz, np.float64)))
    al, cp = np.empty_like(f), np.empty_like(f)
    P = C.POINTER(C.c_double)
    _lib.check(_lib.load().fw_fit_targets(float(alpha0), float(y), float(c0), float(f_ref), f.ctypes.data_as(P),
                                          int(f.size), al.ctypes.data_as(P), cp.ctypes.data_as(P)),
               "fw_fit_targets")
    shape = np.shape(f_hz)
    return al.reshape(shape), cp.reshape(shape)


def alpha_target(alpha0, y, f_hz):
    """alpha0 f^y in Np/m (alpha0 in dB/(MHz^y cm)), Eq. power_law_attenuation."""
    return _targets(alpha0, y, f_hz)[0]


def phase_velocity_target(alpha0, y, f_hz, c0, f_ref=1e6):
    """c(w) of the power law through the Kramers-Kronig relation (Eq.
    kk_relation), c(f_ref) = c0; the y = 1 case takes its logarithmic limit."""
    return _targets(alpha0, y, f_hz, c0, f_ref)[1]


def gaussian_pulse(f0, dt, n, amp=1.0):
    """sin(2 pi f0 (t - 3/f0)) exp(-((t - 3/f0) f0)^2) at t = n dt."""
    t = np.arange(n) * dt - 3.0 / f0
    return amp * np.sin(2.0 * math.pi * f0 * t) * np.exp(-(t * f0) ** 2)


def spectra_between(tr1, tr2, dt, f0, db=-20.0):
    """Frequencies over 0.7-1.3 f0 where |P1| is within db of its peak, the
    amplitude ratio |P2|/|P1| and the phase delay phi(f) >= 0 of trace 2
    behind trace 1 (unwrapped along the band)."""
    n = 1 << int(math.ceil(math.log2(8 * len(tr1))))
    f = np.fft.rfftfreq(n, dt)
    p1, p2 = np.fft.rfft(tr1, n), np.fft.rfft(tr2, n)
    mag = np.abs(p1)
    sel = (mag >= mag.max() * 10.0 ** (db / 20.0)) & (f > 0.7 * f0) & (f < 1.3 * f0)
    phase = np.unwrap(-np.angle(p2 * np.conj(p1)))
    return f[sel], np.abs(p2[sel]) / np.abs(p1[sel]), phase[sel]


def plane_wave_traces(params, f0, c=1540.0, rho=1000.0, ppw=16, cfl=0.2, depth_wl=10, width_wl=50, layer_wl=3,
                      storage="f32", stream=None):
    """Traces at 0.05 D and 0.8 D of one plane-wave run on the GPU; returns
    (trace1, trace2, dt, receiver distance [m])."""
    from . import Medium   # the binding (ctypes); no CPU path

    dx = c / (f0 * ppw)
    dt = cfl * dx / c
    lay = layer_wl * ppw
    width = 2 * lay
    depth = depth_wl * ppw
    shape = (depth + 2 * width + 8, width_wl * ppw + 2 * width)
    src = width + 2
    r1, r2 = src + int(round(0.05 * depth)), src + int(round(0.8 * depth))
    n_steps = int((r2 - src + 6 * ppw + 2 * ppw) / cfl)
    smask = np.zeros(shape, np.uint8)
    smask[src] = 1
    rmask = np.zeros(shape, np.uint8)
    rmask[r1, shape[1] // 2] = 1
    rmask[r2, shape[1] // 2] = 1
    amp = 2.0 * 1e3 * dx / (rho * c)          # injection rate of a ~1 kPa plane wave
    m = Medium.from_classes(shape, dx, np.full(shape, c, np.float32), np.full(shape, rho, np.float32),
                            np.zeros(shape, np.uint16), [params], dt=dt, pml=lay, transition=lay, f0=f0,
                            storage=storage, stream=stream)
    try:
        m.set_sources(smask, gaussian_pulse(f0, dt, n_steps, amp)[None].astype(np.float32))
        m.set_receivers(rmask, n_steps)
        m.run(n_steps, stream=stream)
        tr = m.receivers(f64=True, stream=stream)
        rc, _ = m.status()
    finally:
        m.close()
    if rc != 0:
        raise RuntimeError("plane-wave run unstable (status %d)" % rc)
    return tr[0], tr[1], dt, (r2 - r1) * dx


def simulated_accuracy(params, alpha0, y, c0=1540.0, centres=CENTRES, **run_kw):
    """Simulated attenuation NRMSE and dispersion error of one relaxation set
    (module docstring); also returns the measured samples."""
    fs, als, cs = [], [], []
    for f0 in centres:
        t1, t2, dt, d = plane_wave_traces(params, f0, c=c0, **run_kw)
        f, ratio, phi = spectra_between(t1, t2, dt, f0)
        w = 2.0 * math.pi * f
        # whole cycles of the delay from the nominal travel time at the band's centre
        k = np.round((w[len(w) // 2] * d / c0 - phi[len(phi) // 2]) / (2.0 * math.pi))
        phi = phi + 2.0 * math.pi * k
        fs.append(f)
        als.append(-np.log(ratio) / d)
        cs.append(w * d / phi)
    f, al, cm = np.concatenate(fs), np.concatenate(als), np.concatenate(cs)
    tgt = alpha_target(alpha0, y, f)
    nrmse = float(np.sqrt(np.mean((al - tgt) ** 2)) / (tgt.max() - tgt.min()))
    disp = float(np.sqrt(np.mean((cm - phase_velocity_target(alpha0, y, f, c0)) ** 2)))
    return dict(nrmse=nrmse, disp_rmse=disp, f=f, alpha=al, c=cm)


def select_weight(candidates, alpha0, y, c0=1540.0, **kw):
    """Index of the candidate set kept by the simulation-based selection,
    the per-candidate (nrmse, disp_rmse) and whether the calibration failed."""
    scores = []
    for p in candidates:
        try:
            a = simulated_accuracy(p, alpha0, y, c0, **kw)
            scores.append((a["nrmse"], a["disp_rmse"]))
        except RuntimeError:              # the set's run went unstable: never kept
            scores.append((math.inf, math.inf))
    best = min(range(len(scores)), key=lambda i: scores[i])
    failed = scores[best][0] > 0.10 or scores[best][1] > 5.0
    return best, scores, failed


def calibrate(alpha0, y, n_mech=2, weights=(0.1, 0.3, 0.5, 0.7, 0.9), c0=1540.0, **kw):
    """fw_fit_relaxation once per weight, then the simulation-based
    selection; returns (fw_relax_params, index of the kept weight, scores,
    failed)."""
    from . import fit_relaxation
    cands = [fit_relaxation(alpha0, y, n_mech, w=[w], c0=c0)[0] for w in weights]
    best, scores, failed = select_weight(cands, alpha0, y, c0, **kw)
    return cands[best], best, scores, failed
