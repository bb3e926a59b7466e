"""Two-layer validation (Sec. 4.4, Sec. 5.2, Table 4): geometry and
measurements shared by the oracle pin and the GPU test.

Reading of the protocol (the paper gives the tissues, the 5 MHz pulse and
"the method of Sec. 4.1 within each layer"):

* c = 1540 m/s and rho = 1000 kg/m^3 in both layers, so any reflection at
  the interface comes from the relaxation sets alone;
* each layer D = 10 lambda deep (the Sec. 4.1 depth), 16 points per
  wavelength unless stated, CFL 0.2, two-stage absorbing layer
  L_T = L_B = 3 lambda;
* attenuation in each layer by the Sec. 4.1 method: plane-wave pulses at
  centre frequencies 1-20 MHz in 2.71 MHz steps, receivers at 0.05 D and
  0.8 D of that layer, alpha(f) from the spectral ratio of the two traces
  over 0.7-1.3 f0, NRMSE = RMS error / (range of alpha0 f^y over the
  measured frequencies).  Each trace is gated to its direct arrival (a
  Tukey window two periods either side of the travel time), which keeps the
  interface echo out of the layer-1 receivers;
* interface reflection at 5 MHz: R = 20 log10 max|p - p_1| / max|p_1| at a
  receiver half a wavelength above the interface, p_1 the same run with
  layer 1 everywhere (so p - p_1 is the reflected wave alone);
* closed form of that reflection.  In the model the velocity equation
  carries the gradient-side stretch s1(w) = 1/kappa1 - gamma1(w) and the
  pressure equation the divergence-side stretch s2(w) = 1/kappa2 -
  gamma2(w) (Eq. dispersion_relations: k = (w/c) (s1 s2)^-1/2), so a plane
  wave has impedance Z = p/v = rho c sqrt(s2/s1), and between two media of
  equal rho c the reflection coefficient is R(w) = (Z2 - Z1)/(Z2 + Z1).
  Applied to the spectrum of the incident pulse, delayed by the round trip
  receiver -> interface -> receiver in medium 1, it predicts the reflected
  wave.  The discrete interface (a velocity point takes the class of its
  lower cell, so the two stretches switch half a cell apart) adds a
  first-order error in dx.
"""
import math

import numpy as np

from oracle import fit, measure
from synthetic import gaussian_pulse, plane_amplitude_rate

C0, RHO = 1540.0, 1000.0
PPW, CFL = 16, 0.2
MARGIN = 8
F_R = 5e6
CENTRES = tuple(np.arange(1e6, 20.01e6, 2.71e6))


class Geometry:
    """Cells of one two-layer run at ppw points per wavelength."""

    def __init__(self, ppw=PPW):
        self.ppw = ppw
        self.lt = self.lb = 3 * ppw
        self.width = self.lt + self.lb
        self.d1 = self.d2 = 10 * ppw
        self.src = self.width + 2
        self.itf = self.src + self.d1
        self.r1 = (self.src + round(0.05 * self.d1), self.src + round(0.8 * self.d1))
        self.r2 = (self.itf + round(0.05 * self.d2), self.itf + round(0.8 * self.d2))
        self.rr = self.itf - ppw // 2
        self.depth = self.width + 2 + self.d1 + self.d2 + MARGIN + self.width
        # the direct wave past the deepest receiver plus six periods of pulse
        self.n_steps = int((self.d1 + self.d2 + 6 * ppw) / CFL)

    def grid(self, f0):
        dx = C0 / (f0 * self.ppw)
        return dx, CFL * dx / C0

    def receivers(self):
        return sorted(set(self.r1) | set(self.r2) | {self.rr})

    def wave(self, f0, ndim):
        dx, dt = self.grid(f0)
        return gaussian_pulse(f0, dt, self.n_steps, plane_amplitude_rate(1e3, dx, ndim, RHO, C0))

    def class_map(self, shape, two_layers):
        """0 above the interface, 1 from it down (two_layers), else 0 everywhere."""
        cls = np.zeros(shape, np.int64)
        if two_layers:
            cls[self.itf:] = 1
        return cls

    def gate(self, trace, f0, row):
        """Tukey window two periods either side of the direct arrival at row."""
        dx, dt = self.grid(f0)
        t = np.arange(len(trace)) * dt
        ta = 3.0 / f0 + (row - self.src) * dx / C0      # pulse delay t0 = 3 tau, tau = 1/f0
        half = 2.0 / f0
        x = np.clip((np.abs(t - ta) - half) / (0.5 / f0), 0.0, 1.0)
        return trace * np.where(np.abs(t - ta) <= half, 1.0, 0.5 * (1 + np.cos(math.pi * x)))

    def layer_attenuation(self, traces_by_f0, layer, tissue):
        """NRMSE of alpha(f) in one layer over all centre frequencies.
        traces_by_f0: {f0: {row: trace}}."""
        a, b = self.r1 if layer == 1 else self.r2
        fs, als = [], []
        for f0, tr in traces_by_f0.items():
            dx, dt = self.grid(f0)
            f, al = measure.attenuation_spectrum(self.gate(tr[a], f0, a), self.gate(tr[b], f0, b), dt, (b - a) * dx)
            keep = (f > 0.7 * f0) & (f < 1.3 * f0)
            fs.append(f[keep])
            als.append(al[keep])
        fs, als = np.concatenate(fs), np.concatenate(als)
        return measure.nrmse(als, fit.alpha_target(tissue[0], tissue[1], fs))

    def predicted_reflection(self, p1, p2, incident):
        """Reflected wave at the reflection receiver from the closed form
        (module docstring), given the incident trace p_1 there."""
        dx, dt = self.grid(F_R)
        n = 1 << int(math.ceil(math.log2(4 * len(incident))))
        f = np.maximum(np.fft.rfftfreq(n, dt), 1e3)
        w = 2.0 * math.pi * f
        z1, z2 = impedance(p1, w), impedance(p2, w)
        k1 = fit.k_model(p1, f, C0)
        trip = 2 * (self.itf - self.rr) * dx
        return np.fft.irfft(np.fft.rfft(incident, n) * (z2 - z1) / (z2 + z1) * np.exp(-1j * k1 * trip),
                            n)[:len(incident)]


def impedance(p, w):
    """rho c sqrt(s2/s1) in units of rho c."""
    s1 = 1.0 / p.kappa1 - fit.gamma(p.d1, p.alpha1, p.kappa1, w)
    s2 = 1.0 / p.kappa2 - fit.gamma(p.d2, p.alpha2, p.kappa2, w)
    return np.sqrt(s2 / s1)


def reflection_db(p_two, p_one):
    return measure.reflection_db(p_two, p_one)


def peak_db(wave, incident):
    return 20.0 * math.log10(np.abs(wave).max() / np.abs(incident).max())
