"""Reflection of the absorbing layer on the GPU (protocol of Sec. 4.3, results
of Sec. 5.4 and 5.5): the adaptive two-stage layer against the two
homogeneous layers of Sec. 4.6, over an (alpha0, y) grid.

Protocol (Sec. 4.3): 1 MHz plane wave from a line source across the top of a
domain D = 5 lambda deep and W = 20 lambda wide (inside the layer), 16 points
per wavelength, CFL 0.2, L_T = L_B = 3 lambda; one receiver on the centre
column 8 cells above the bottom layer.  R = 20 log10(max|p - p_ref| /
max|p_ref|), p_ref the same trace in a domain 200 cells deeper, whose bottom
echo reaches the receiver after the 2000-step window.  Configurations:

* adaptive: the layer inherits the nearest interior class (the method);
* hom_T: every cell of the layer takes the class fitted for (0.5, 1.0),
  same two-stage geometry (layer_relax);
* hom_noT: the same fixed class, no transition region (the tissue
  mechanisms are then ramped within the absorbing region).

Stability: each short-domain run continues to 4 times the window; it counts
as unstable if the pressure turns non-finite or ends above the peak of the
pulse (the paper's NaN/Inf count).  Relaxation sets: the oracle's fits at
the paper's calibration settings stored in tests/golden/relax_sets.json;
failed fits (NRMSE > 10 % or dispersion error > 5 m/s) are left out of the
statistics, as in Sec. 5.4."""
import math

import numpy as np
import pytest

from gpu_util import rel_l2, stored_set, to_c
from oracle import measure
from oracle.medium import OracleMedium
from oracle.stepper import OracleSim
from synthetic import gaussian_pulse, plane_amplitude_rate

pytestmark = pytest.mark.gpu

F0, PPW, CFL = 1e6, 16, 0.2
C0, RHO = 1540.0, 1000.0
DX = C0 / (F0 * PPW)
DT = CFL * DX / C0
LAM = PPW                      # cells per wavelength
LB = LT = 3 * LAM
D, W = 5 * LAM, 20 * LAM
EXTRA = 200
NT = 2000
CONFIGS = ("adaptive", "hom_T", "hom_noT")
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


def _geometry(cfg, extra):
    """Shape, class map (0 interior, 1 the fixed layer class), source and
    receiver masks, layer widths."""
    lt = 0 if cfg == "hom_noT" else LT
    width = LB + lt
    shape = (D + extra + 2 * width, W + 2 * width)
    cls = np.zeros(shape, np.int64)
    if cfg != "adaptive":
        cls[:] = 1
        cls[width:shape[0] - width, width:shape[1] - width] = 0
    src = np.zeros(shape, np.uint8)
    row = width + 2
    src[row] = 1
    rcv = np.zeros(shape, np.uint8)
    rcv[row + D - 8, shape[1] // 2] = 1
    return shape, cls, src, rcv, lt


def _wave():
    return gaussian_pulse(F0, DT, NT, plane_amplitude_rate(1e3, DX, 2, RHO, C0))


def _gpu_trace(fw, classes, cfg, extra, tail=0):
    """Receiver trace of one run; with tail > 0 also whether the run stays
    stable for tail more steps."""
    shape, cls, src, rcv, lt = _geometry(cfg, extra)
    m = fw.Medium.from_classes(shape, DX, np.full(shape, C0, np.float32), np.full(shape, RHO, np.float32),
                               cls.astype(np.uint16), classes, dt=DT, pml=LB, transition=lt, f0=F0,
                               layer_relax=cfg != "adaptive")
    m.set_sources(src, _wave()[None].astype(np.float32))
    m.set_receivers(rcv, NT)
    m.run(NT)
    tr = m.receivers(f64=True)[0]
    stable = None
    if tail:
        rc, peak = m.status()
        m.run(tail)
        rc, _ = m.status()
        p = m.read_field(0, 0)
        stable = bool(rc == 0 and np.all(np.isfinite(p)) and np.abs(p).max() <= peak)
    m.close()
    return tr, stable


def _oracle_trace(params, cfg, extra):
    shape, cls, src, rcv, lt = _geometry(cfg, extra)
    med = OracleMedium(shape, DX, DT, np.full(shape, C0), np.full(shape, RHO), cls, params, pml=LB,
                       transition=lt, f0=F0, layer_relax=cfg != "adaptive")
    sim = OracleSim(med)
    sim.set_sources(src, _wave()[None])
    sim.set_receivers(rcv, NT)
    sim.run(NT)
    return sim.traces[0]


@pytest.fixture(scope="module")
def design_point():
    return stored_set(0.5, 1.0)[0]


@pytest.mark.parametrize("cfg,a0,y", [("adaptive", 0.5, 1.0), ("hom_T", 0.25, 0.6)])
def test_reflection_matches_oracle(fw, design_point, cfg, a0, y):
    """The measured quantity itself against the FP64 oracle on the same
    geometry: traces to the FP32 target, R to 0.5 dB."""
    params = [stored_set(a0, y)[0], design_point]
    classes = [to_c(p, fw) for p in params]
    got = [_gpu_trace(fw, classes, cfg, e)[0] for e in (0, EXTRA)]
    want = [_oracle_trace(params, cfg, e) for e in (0, EXTRA)]
    r_gpu = measure.reflection_db(got[0], got[1])
    r_orc = measure.reflection_db(want[0], want[1])
    e = [rel_l2(g, w) for g, w in zip(got, want)]
    print("\n%s (%.2f, %.1f): R GPU %.2f dB, oracle %.2f dB; traces rel L2 %.1e %.1e"
          % (cfg, a0, y, r_gpu, r_orc, e[0], e[1]))
    assert max(e) < 1e-5, e
    assert abs(r_gpu - r_orc) < 0.5, (r_gpu, r_orc)


def test_reflection_sweep_adaptive_vs_homogeneous(fw, design_point):
    """R over alpha0 x y = 5 x 9 for the three configurations; the
    statistics Sec. 5.5 reports (median R, share below -50 dB, unstable
    runs) are printed beside the paper's.  Asserted: the adaptive layer is
    below -50 dB for every valid y <= 1.5 and never unstable, equals the
    homogeneous layer at its design point, and has the lower median."""
    pairs = [(a, y) for y in YS for a in ALPHA0]
    refl = {cfg: {} for cfg in CONFIGS}
    unstable = {cfg: 0 for cfg in CONFIGS}
    for pair in pairs:
        prm, rep = stored_set(*pair)
        if rep["failed"]:
            continue
        classes = [to_c(prm, fw), to_c(design_point, fw)]
        for cfg in CONFIGS:
            small, stable = _gpu_trace(fw, classes, cfg, 0, tail=3 * NT)
            big, _ = _gpu_trace(fw, classes, cfg, EXTRA)
            if not stable:
                unstable[cfg] += 1
            if np.all(np.isfinite(small)) and np.all(np.isfinite(big)):
                refl[cfg][pair] = measure.reflection_db(small, big)
    valid = sorted(refl["adaptive"])
    print("\nvalid (alpha0, y) pairs: %d of %d" % (len(valid), len(pairs)))
    print("y    " + " ".join("%6.4g" % a for a in ALPHA0) + "   (adaptive / hom_T / hom_noT, dB)")
    for y in YS:
        row = []
        for a in ALPHA0:
            if (a, y) in refl["adaptive"]:
                row.append("/".join("%.0f" % refl[c].get((a, y), math.nan) for c in CONFIGS))
            else:
                row.append("failed-fit")
        print("%.1f  %s" % (y, "  ".join(row)))
    paper = {"adaptive": (-58.5, 97.1, 0), "hom_T": (-54.5, 85.1, 0), "hom_noT": (-41.9, 1.1, 29)}
    stats = {}
    for cfg in CONFIGS:
        r = np.array([refl[cfg][p] for p in valid if p in refl[cfg]])
        stats[cfg] = (float(np.median(r)), 100.0 * float(np.mean(r < -50.0)), unstable[cfg])
        print("%-8s median R %.1f dB, %.1f %% below -50 dB, %d unstable   (paper: %.1f dB, %.1f %%, %d)"
              % ((cfg,) + stats[cfg] + paper[cfg]))
    assert len(valid) >= len(pairs) // 2
    for (a, y) in valid:
        if y <= 1.5:
            assert refl["adaptive"][(a, y)] < -50.0, ((a, y), refl["adaptive"][(a, y)])
    assert unstable["adaptive"] == 0
    if (0.5, 1.0) in refl["adaptive"]:
        assert abs(refl["adaptive"][(0.5, 1.0)] - refl["hom_T"][(0.5, 1.0)]) < 0.1
    assert stats["adaptive"][0] < stats["hom_T"][0]
