"""Attenuation, dispersion and reflection measurements (Sec. 4.1-4.3).

Test infrastructure: these post-process receiver traces from any simulator.

* attenuation: the paper takes alpha = -(1/2d) ln(I_att/I_ref) per centre
  frequency (Sec. 4.1).  Reading: intensities are taken per frequency from
  the spectra of the two receiver traces, I ~ |P(f)|^2, so
  alpha(f) = -ln(|P2(f)|/|P1(f)|)/d over the band where the reference
  spectrum is within -20 dB of its peak (same value for a plane wave);
* NRMSE = RMSE / (alpha_max - alpha_min) of the target (Sec. 4.1);
* phase velocity from the spectral phase delay between the receivers,
  c(f) = 2 pi f d / dphi(f) (the time of flight of Sec. 4.2, per frequency);
* reflection R = 20 log10(p_reflected / p_incident) (Eq.
  reflection_coefficient_pml), with the reflected wave isolated by
  subtracting a run on a domain large enough that nothing returns in the
  window.
"""
from __future__ import annotations

import math

import numpy as np


def spectra(tr1, tr2, dt, pad=8):
    n = int(2 ** math.ceil(math.log2(len(tr1) * pad)))
    f = np.fft.rfftfreq(n, dt)
    return f, np.fft.rfft(tr1, n), np.fft.rfft(tr2, n)


def band(f, P, db=-20.0):
    mag = np.abs(P)
    return mag >= mag.max() * 10 ** (db / 20.0)


def attenuation_spectrum(tr1, tr2, dt, dist, db=-20.0):
    """alpha(f) [Np/m] between two receivers ``dist`` metres apart."""
    f, P1, P2 = spectra(tr1, tr2, dt)
    sel = band(f, P1, db) & (f > 0)
    return f[sel], -np.log(np.abs(P2[sel]) / np.abs(P1[sel])) / dist


def phase_velocity_spectrum(tr1, tr2, dt, dist, db=-20.0):
    """c(f) [m/s] from the unwrapped phase delay of receiver 2 behind 1."""
    f, P1, P2 = spectra(tr1, tr2, dt)
    sel = band(f, P1, db) & (f > 0)
    dphi = np.unwrap(np.angle(P1[sel] * np.conj(P2[sel])))
    # resolve the 2 pi ambiguity with the nominal delay at the band centre
    return f[sel], dphi


def phase_velocity(tr1, tr2, dt, dist, c_nominal, db=-20.0):
    f, dphi = phase_velocity_spectrum(tr1, tr2, dt, dist, db)
    w = 2 * math.pi * f
    k_nom = w * dist / c_nominal
    mid = len(f) // 2
    dphi = dphi + 2 * math.pi * np.round((k_nom[mid] - dphi[mid]) / (2 * math.pi))
    return f, w * dist / dphi


def nrmse(measured, target):
    return math.sqrt(np.mean((measured - target) ** 2)) / (np.max(target) - np.min(target))


def reflection_db(p_small, p_big, window=None):
    """20 log10(max|p_small - p_big| / max|p_big|) over ``window`` (slice)."""
    w = slice(None) if window is None else window
    refl = np.max(np.abs(p_small[w] - p_big[w]))
    inc = np.max(np.abs(p_big[w]))
    return 20.0 * math.log10(refl / inc)
