"""Helpers shared by the GPU tests: run one synthetic workload on the CUDA
path (through the C ABI) and on the FP64 oracle with the same inputs."""
from __future__ import annotations

import numpy as np

from oracle import fit
from oracle.stepper import OracleSim
from oracle.medium import OracleMedium


def oracle_params(alpha0, y, n_mech, maxiter=400):
    """Relaxation sets from the oracle's own calibration (cheap settings)."""
    if alpha0 == 0:
        return fit.RelaxParams.lossless(n_mech)
    p, _ = fit.fit_relaxation(float(alpha0), float(y), n_mech, maxiter=maxiter, w_list=(0.5,))
    return p


def to_c(p, fw):
    return fw.relax_params(p.kappa1, p.kappa2, p.d1, p.alpha1, p.d2, p.alpha2)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class Pair:
    """The same medium on the GPU (fw.Medium) and on the oracle."""

    def __init__(self, fw, shape, dx, dt, c, rho, cls, params, beta=None, pml=0, transition=0, f0=3e6,
                 storage="f32", time_order=2):
        self.shape = tuple(shape)
        self.gpu = fw.Medium.from_classes(shape, dx, c, rho, cls.astype(np.uint16), [to_c(p, fw) for p in params],
                                          dt=dt, beta=beta, pml=pml, transition=transition, f0=f0,
                                          storage=storage, time_order=time_order)
        med = OracleMedium(shape, dx, dt, c, rho, cls.astype(np.int64), params, beta=beta, pml=pml,
                           transition=transition, f0=f0, time_order=time_order)
        self.orc = OracleSim(med)

    def sources(self, mask, waves, wave_of=None):
        self.gpu.set_sources(mask, waves, wave_of)
        self.orc.set_sources(mask, np.asarray(waves, np.float32).astype(np.float64), wave_of)

    def receivers(self, mask, n_steps, decim=1):
        self.gpu.set_receivers(mask, n_steps, decim)
        self.orc.set_receivers(mask, n_steps, decim)

    def run(self, n, graphs=True):
        if graphs:
            self.gpu.run(n)
        else:
            self.gpu.step(n)
        self.orc.run(n)

    def errors(self, f64=False):
        """Absolute differences and reference norms of p and every v_d."""
        out = {}
        p = self.gpu.read_field(0, 0, f64=f64).astype(np.float64)
        out["p"] = (np.linalg.norm(p - self.orc.p), np.linalg.norm(self.orc.p))
        for d in range(len(self.shape)):
            g = self.gpu.read_field(1, d, f64=f64).astype(np.float64)
            out["v%d" % d] = (np.linalg.norm(g - self.orc.v[d]), np.linalg.norm(self.orc.v[d]))
        return out

    def run_compare(self, n_steps, checks=3, graphs=True, f64=False):
        """Run n_steps, comparing fields at `checks` evenly spaced times.

        Each error is an L2 norm divided by the solution's own scale: the
        largest norm the reference field reached at any check (velocity
        components share one scale, since a plane wave has a near-zero
        component).  Receiver traces over the whole run are compared by
        relative L2.  A field that has left the grid through the absorbing
        layer thus does not turn rounding noise into a large relative error.
        """
        bounds = np.linspace(0, n_steps, checks + 1).round().astype(int)
        errs, scale = {}, {}
        for a, b in zip(bounds[:-1], bounds[1:]):
            self.run(int(b - a), graphs=graphs)
            for k, (e, nrm) in self.errors(f64).items():
                key = "v" if k.startswith("v") else k
                errs[k] = max(errs.get(k, 0.0), e)
                scale[key] = max(scale.get(key, 0.0), nrm)
        out = {k: float(e / max(scale["v" if k.startswith("v") else k], 1e-300)) for k, e in errs.items()}
        if self.orc.traces is not None and self.orc.traces.size:
            out["traces"] = rel_l2(self.gpu.receivers(f64=f64), self.orc.traces)
        return out


_SETS = None


def stored_set(alpha0, y):
    """(RelaxParams, report) of the oracle fit at the paper's settings for
    (alpha0, y), from tests/golden/relax_sets.json (written by
    tests/golden/fit_relax_sets.py, which calls only the oracle)."""
    global _SETS
    if _SETS is None:
        import json
        import os
        with open(os.path.join(os.path.dirname(__file__), "golden", "relax_sets.json")) as f:
            _SETS = json.load(f)
    d = _SETS["sets"]["%g,%g" % (alpha0, y)]
    p = fit.RelaxParams(d["kappa1"], d["kappa2"], np.array(d["d1"]), np.array(d["alpha1"]), np.array(d["d2"]),
                        np.array(d["alpha2"]))
    return p, d
