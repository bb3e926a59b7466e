"""The absorbing-layer reflection sweep of Sec. 5.4-5.5 on the FP64 oracle
(host CPU only) under two readings of the two-stage layer, for the record of
how the reading decides the result.

* ramped (the reading the library implements): the tissue mechanisms are
  ramped out across the transition region, or across the first half of the
  absorbing region when there is none (Sec. 4.6);
* full strength: the tissue mechanisms keep their interior strength in every
  layer cell (``OracleMedium(tissue_ramp_on=False)``).

Geometry, source, receiver, reference domain, relaxation sets and the
stability rule are those of tests/test_gpu_pml_reflection.py (Sec. 4.3
protocol, the oracle's stored fits at the paper's settings).  Run:

    python tests/pml_readings_cpu.py [n_pairs] [R0] [configs]

It prints, per reading and layer configuration, the median reflection, the
share below -50 dB and the unstable runs beside the paper's Sec. 5.5 figures.
R0 (default 1e-5) is the design reflection of the absorbing profile;
configs a comma list of adaptive, hom_T, hom_noT (default all three).
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

from gpu_util import stored_set  # noqa: E402
from oracle import measure  # noqa: E402
from oracle.medium import OracleMedium  # noqa: E402
from oracle.stepper import OracleSim  # noqa: E402
import test_gpu_pml_reflection as proto  # noqa: E402

PAPER = {"adaptive": (-58.5, 97.1, 0), "hom_T": (-54.5, 85.1, 0), "hom_noT": (-41.9, 1.1, 29)}


R0 = 1e-5


def trace(params, cfg, extra, ramp, tail=0):
    """Receiver trace of one oracle run; with tail > 0 also whether the run
    stays finite and below the pulse's peak for tail more steps."""
    shape, cls, src, rcv, lt = proto._geometry(cfg, extra)
    med = OracleMedium(shape, proto.DX, proto.DT, np.full(shape, proto.C0), np.full(shape, proto.RHO), cls, params,
                       pml=proto.LB, transition=lt, f0=proto.F0, layer_relax=cfg != "adaptive",
                       tissue_ramp_on=ramp, R0=R0)
    sim = OracleSim(med)
    sim.set_sources(src, proto._wave()[None])
    sim.set_receivers(rcv, proto.NT)
    peak = 0.0                     # largest |p| over the grid in the window, sampled every 50 steps
    for _ in range(proto.NT // 50):
        sim.run(50)
        peak = max(peak, float(np.max(np.abs(sim.p))))
    tr = sim.traces[0].copy()
    stable = None
    if tail:
        sim.run(tail)
        stable = bool(np.all(np.isfinite(sim.p)) and np.abs(sim.p).max() <= peak)
    return tr, stable


def sweep(n_pairs=None, configs=proto.CONFIGS, readings=(True, False)):
    design = stored_set(0.5, 1.0)[0]
    pairs = [(a, y) for y in proto.YS for a in proto.ALPHA0]
    pairs = [p for p in pairs if not stored_set(*p)[1]["failed"]]
    if n_pairs:
        pairs = pairs[::max(1, len(pairs) // n_pairs)][:n_pairs]
    out = {}
    for ramp in readings:
        for cfg in configs:
            refl, bad = [], 0
            for pair in pairs:
                params = [stored_set(*pair)[0], design]
                small, stable = trace(params, cfg, 0, ramp, tail=3 * proto.NT)
                big, _ = trace(params, cfg, proto.EXTRA, ramp)
                bad += 0 if stable else 1
                if np.all(np.isfinite(small)) and np.all(np.isfinite(big)):
                    refl.append(measure.reflection_db(small, big))
            r = np.array(refl)
            out[(ramp, cfg)] = (float(np.median(r)) if r.size else math.nan,
                                100.0 * float(np.mean(r < -50.0)) if r.size else math.nan, bad, len(pairs))
            row = (("ramped" if ramp else "full strength"), cfg) + out[(ramp, cfg)] + PAPER[cfg]
            print("%-13s %-8s median R %6.1f dB, %5.1f %% below -50 dB, %2d of %d unstable   (paper %.1f, %.1f %%, %d)"
                  % row, flush=True)
    return out


if __name__ == "__main__":
    if len(sys.argv) > 2:
        R0 = float(sys.argv[2])
    cfgs = tuple(sys.argv[3].split(",")) if len(sys.argv) > 3 else proto.CONFIGS
    print("design reflection R0 = %g" % R0, flush=True)
    # with a design reflection given: the library's reading (ramped) only
    sweep(int(sys.argv[1]) if len(sys.argv) > 1 and sys.argv[1] else None, cfgs,
          (True,) if len(sys.argv) > 2 else (True, False))
