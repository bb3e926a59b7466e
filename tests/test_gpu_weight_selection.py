"""Simulation-based weight selection on the GPU (Sec. 3.2):
calibrate.py simulates every weight's relaxation set in the Sec. 4.1-4.2
protocol and keeps the lowest simulated attenuation NRMSE.

* parity of the measured quantity: the plane-wave traces of one set at
  three centre frequencies against the FP64 oracle on the same grid (a
  narrower W = 20 lambda domain), traces to the FP32 target, the measured
  attenuation to 1e-4 relative and phase velocity to 0.01 m/s;
* the grid alpha0 in {0.0022, 0.25, 0.5, 0.75, 1.0} x y in {0.4, ..., 2.0}
  with the oracle's per-weight fits at the paper's settings
  (tests/golden/relax_sets.json): the statistics of Sec. 5.1 (mean and
  standard deviation of the simulated NRMSE and dispersion error over the
  valid pairs) printed beside the paper's 2.61 +- 1.83 % and 1.14 +- 0.76
  m/s; asserted: mean NRMSE below the 3 % of the abstract, every valid
  pair below 10 % and 5 m/s by definition, at least half the pairs valid;
* the whole calibration through the C ABI's fitter for (0.5, 1.0)."""
import math

import numpy as np
import pytest

from gpu_util import rel_l2, stored_set, to_c
from oracle.medium import OracleMedium
from oracle.stepper import OracleSim

pytestmark = pytest.mark.gpu

ALPHA0 = (0.0022, 0.25, 0.5, 0.75, 1.0)
YS = (0.4, 0.6, 0.8, 1.0, 1.2, 1.4, 1.6, 1.8, 2.0)


@pytest.fixture(scope="module")
def fw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_11103_gb300 as fw
    from paper_2606_11103_gb300 import build
    build.build()
    return fw


def _oracle_traces(prm, f0, width_wl, c=1540.0, rho=1000.0, ppw=16, cfl=0.2, depth_wl=10, layer_wl=3):
    """The same run as calibrate.plane_wave_traces, on the oracle."""
    from paper_2606_11103_gb300 import calibrate as cal
    dx = c / (f0 * ppw)
    dt = cfl * dx / c
    lay = layer_wl * ppw
    width = 2 * lay
    depth = depth_wl * ppw
    shape = (depth + 2 * width + 8, width_wl * ppw + 2 * width)
    src = width + 2
    r1, r2 = src + int(round(0.05 * depth)), src + int(round(0.8 * depth))
    n_steps = int((r2 - src + 6 * ppw + 2 * ppw) / cfl)
    med = OracleMedium(shape, dx, dt, np.full(shape, c), np.full(shape, rho), np.zeros(shape, np.int64), [prm],
                       pml=lay, transition=lay, f0=f0)
    sim = OracleSim(med)
    smask = np.zeros(shape, np.uint8)
    smask[src] = 1
    rmask = np.zeros(shape, np.uint8)
    rmask[r1, shape[1] // 2] = 1
    rmask[r2, shape[1] // 2] = 1
    sim.set_sources(smask, cal.gaussian_pulse(f0, dt, n_steps, 2.0 * 1e3 * dx / (rho * c))[None])
    sim.set_receivers(rmask, n_steps)
    sim.run(n_steps)
    return sim.traces[0], sim.traces[1], dt, (r2 - r1) * dx


def test_measurement_matches_oracle(fw):
    from paper_2606_11103_gb300 import calibrate as cal
    prm = stored_set(0.5, 1.0)[0]
    for f0 in (1e6, 6.42e6, 17.26e6):
        g1, g2, dt, d = cal.plane_wave_traces(to_c(prm, fw), f0, width_wl=20)
        o1, o2, _, _ = _oracle_traces(prm, f0, 20)
        e = rel_l2(np.stack([g1, g2]), np.stack([o1, o2]))
        fg, rg, pg = cal.spectra_between(g1, g2, dt, f0)
        fo, ro, po = cal.spectra_between(o1, o2, dt, f0)
        assert np.array_equal(fg, fo)
        ag, ao = -np.log(rg) / d, -np.log(ro) / d
        cg, co = 2 * math.pi * fg * d / pg, 2 * math.pi * fo * d / po
        print("\nf0 %.2f MHz: traces rel L2 %.1e, alpha %.1e rel, c %.1e m/s"
              % (f0 / 1e6, e, np.max(np.abs(ag / ao - 1)), np.max(np.abs(cg - co))))
        assert e < 1e-5
        assert np.max(np.abs(ag / ao - 1)) < 1e-4
        assert np.max(np.abs(cg - co)) < 0.01


def test_weight_selection_over_the_grid(fw):
    from paper_2606_11103_gb300 import calibrate as cal
    rows, valid = [], []
    changed = 0
    for y in YS:
        for a in ALPHA0:
            _, d = stored_set(a, y)
            cands = [fw.relax_params(e["kappa1"], e["kappa2"], e["d1"], e["alpha1"], e["d2"], e["alpha2"])
                     for e in d["per_w"]]
            best, scores, failed = cal.select_weight(cands, a, y)
            w_sim = d["per_w"][best]["w"]
            changed += w_sim != d["w"]
            rows.append((a, y, w_sim, d["w"], scores[best][0], scores[best][1], failed))
            if not failed:
                valid.append(scores[best])
    print("\nalpha0  y    w(sim) w(closed form)  NRMSE    dispersion  failed")
    for a, y, ws, wc, nr, dp, fl in rows:
        print("%-7g %-4g %-6g %-15g %6.2f %% %8.2f m/s  %s" % (a, y, ws, wc, 100 * nr, dp, fl))
    v = np.array(valid)
    print("valid %d of %d; simulated NRMSE %.2f +- %.2f %% (paper 2.61 +- 1.83 %%), dispersion %.2f +- %.2f m/s "
          "(paper 1.14 +- 0.76 m/s); the simulation chose another weight than the closed form for %d pairs"
          % (len(v), len(rows), 100 * v[:, 0].mean(), 100 * v[:, 0].std(), v[:, 1].mean(), v[:, 1].std(), changed))
    assert len(v) >= len(rows) // 2
    assert v[:, 0].mean() < 0.03
    assert np.all(v[:, 0] <= 0.10) and np.all(v[:, 1] <= 5.0)


def test_calibrate_end_to_end(fw):
    from paper_2606_11103_gb300 import calibrate as cal
    p, best, scores, failed = cal.calibrate(0.5, 1.0)
    print("\ncalibrate(0.5, 1.0): weight index %d, scores %s" % (best, ["%.4f/%.2f" % s for s in scores]))
    assert not failed
    assert scores[best][0] < 0.03
