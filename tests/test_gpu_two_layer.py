"""Two-layer validation on the GPU (Sec. 4.4, Sec. 5.2, Table 4), protocol
in tests/two_layer_protocol.py, in the paper's 2D geometry: a line source
across a domain W = 50 lambda wide inside the absorbing layer, receivers on
the centre column, 16 points per wavelength.

* parity of the measured quantity: the 5 MHz muscle -> liver runs on a
  narrower domain (W = 20 lambda) against the FP64 oracle on the same grid,
  traces to the FP32 target and R to 0.5 dB;
* the three tissue pairs at W = 50 lambda: per-layer attenuation NRMSE below
  2.5 % and interface reflection below -50 dB (Table 4); R within 0.5 dB of
  the oracle's 1D-like plane-wave value at the same resolution (the oracle
  pin ties that value to the closed form of the impedance mismatch)."""
import json
import os

import numpy as np
import pytest

from gpu_util import rel_l2, stored_set, to_c
from oracle.medium import OracleMedium
from oracle.stepper import OracleSim
from two_layer_protocol import CENTRES, C0, F_R, RHO, Geometry, reflection_db

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_accuracy.json")))
CASES = [(c["pair"], (c["layer1"]["alpha0"], c["layer1"]["y"]), (c["layer2"]["alpha0"], c["layer2"]["y"]), c)
         for c in GOLD["two_layer"]]
G = Geometry()


@pytest.fixture(scope="module")
def fw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_11103_gb300 as fw
    from paper_2606_11103_gb300 import build
    build.build()
    return fw


def _setup(two_layers, rcv_rows, w_cells):
    """w_cells = 0: the oracle's 1D-like column (four periodic columns)."""
    shape = (G.depth, w_cells + 2 * G.width) if w_cells else (G.depth, 4)
    src = np.zeros(shape, np.uint8)
    src[G.src] = 1
    rcv = np.zeros(shape, np.uint8)
    for r in rcv_rows:
        rcv[r, shape[1] // 2 if w_cells else 0] = 1
    return shape, G.class_map(shape, two_layers), src, rcv


def _gpu(fw, params, f0, two_layers, rcv_rows, w_cells):
    shape, cls, src, rcv = _setup(two_layers, rcv_rows, w_cells)
    dx, dt = G.grid(f0)
    m = fw.Medium.from_classes(shape, dx, np.full(shape, C0, np.float32), np.full(shape, RHO, np.float32),
                               cls.astype(np.uint16), [to_c(p, fw) for p in params], dt=dt, pml=G.lb,
                               transition=G.lt, f0=f0)
    m.set_sources(src, G.wave(f0, 2)[None].astype(np.float32))
    m.set_receivers(rcv, G.n_steps)
    m.run(G.n_steps)
    tr = m.receivers(f64=True)
    rc, _ = m.status()
    m.close()
    assert rc == 0
    return {r: tr[i] for i, r in enumerate(sorted(rcv_rows))}


def _oracle(params, f0, two_layers, rcv_rows, w_cells):
    shape, cls, src, rcv = _setup(two_layers, rcv_rows, w_cells)
    dx, dt = G.grid(f0)
    med = OracleMedium(shape, dx, dt, np.full(shape, C0), np.full(shape, RHO), cls, params, pml=G.lb,
                       transition=G.lt, f0=f0, periodic=None if w_cells else (False, True))
    sim = OracleSim(med)
    sim.set_sources(src, G.wave(f0, 2)[None])
    sim.set_receivers(rcv, G.n_steps)
    sim.run(G.n_steps)
    return {r: sim.traces[i] for i, r in enumerate(sorted(rcv_rows))}


def test_two_layer_runs_match_oracle(fw):
    params = [stored_set(0.15, 1.0)[0], stored_set(0.50, 1.1)[0]]
    rcv = G.receivers()
    w = 20 * G.ppw
    got = {two: _gpu(fw, params, F_R, two, rcv, w) for two in (True, False)}
    want = {two: _oracle(params, F_R, two, rcv, w) for two in (True, False)}
    e = max(rel_l2(np.array([got[t][r] for r in rcv]), np.array([want[t][r] for r in rcv])) for t in got)
    R_gpu = reflection_db(got[True][G.rr], got[False][G.rr])
    R_orc = reflection_db(want[True][G.rr], want[False][G.rr])
    print("\nmuscle->liver 5 MHz, W = 20 lambda: traces rel L2 %.1e, R GPU %.2f dB, oracle %.2f dB" % (e, R_gpu, R_orc))
    assert e < 1e-5
    assert abs(R_gpu - R_orc) < 0.5


@pytest.mark.parametrize("name,t1,t2,gold", CASES, ids=[c[0] for c in CASES])
def test_two_layer_validation(fw, name, t1, t2, gold):
    p1, p2 = stored_set(*t1)[0], stored_set(*t2)[0]
    rcv = G.receivers()
    w = 50 * G.ppw
    traces = {f0: _gpu(fw, [p1, p2], f0, True, rcv, w) for f0 in CENTRES}
    n1 = G.layer_attenuation(traces, 1, t1)
    n2 = G.layer_attenuation(traces, 2, t2)
    R = reflection_db(_gpu(fw, [p1, p2], F_R, True, [G.rr], w)[G.rr], _gpu(fw, [p1, p2], F_R, False, [G.rr], w)[G.rr])
    R1d = reflection_db(_oracle([p1, p2], F_R, True, [G.rr], 0)[G.rr], _oracle([p1, p2], F_R, False, [G.rr], 0)[G.rr])
    print("\n%s (GPU, W = 50 lambda): NRMSE %.2f %% / %.2f %% (Table 4: %.2f / %.2f), R %.1f dB "
          "(oracle 1D-like %.1f, Table 4 %.1f)" % (name, 100 * n1, 100 * n2, 100 * gold["nrmse1"],
                                                  100 * gold["nrmse2"], R, R1d, gold["R_db"]))
    assert n1 < 0.025 and n2 < 0.025, (n1, n2)
    assert R < -50.0, R
    assert abs(R - R1d) < 0.5, (R, R1d)
