"""Write relax_sets.json: relaxation sets fitted by the FP64 oracle (N = 2,
the paper's calibration settings of Sec. 3.2: 1-20 MHz, 200 log-spaced
samples, w in {0.1, 0.3, 0.5, 0.7, 0.9}, 5e4 Nelder-Mead iterations) for
the (alpha0, y) pairs the validation experiments use:

* the absorbing-layer sweep of Sec. 5.4 / 5.5: alpha0 in {0.0022, 0.25,
  0.5, 0.75, 1.0} x y in {0.4, 0.6, ..., 2.0} (the design point of the
  homogeneous layers, (0.5, 1.0), is on the grid);
* the tissues of the two-layer models of Sec. 4.4 / Table 4: muscle
  (0.15, 1.0), fat (0.40, 1.1), liver (0.50, 1.1).

Each pair also keeps the set fitted at every weight (per_w), the
candidates of the simulation-based weight selection of Sec. 3.2.

Only the oracle is called.  Run from the repository root:
    python tests/golden/fit_relax_sets.py
"""
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

SWEEP_ALPHA0 = (0.0022, 0.25, 0.5, 0.75, 1.0)
SWEEP_Y = (0.4, 0.6, 0.8, 1.0, 1.2, 1.4, 1.6, 1.8, 2.0)
TISSUES = {"muscle": (0.15, 1.0), "fat": (0.40, 1.1), "liver": (0.50, 1.1)}


def key(a0, y):
    return "%g,%g" % (a0, y)


def _params(p):
    fl = lambda v: [float(x) for x in v]  # noqa: E731
    return dict(kappa1=float(p.kappa1), kappa2=float(p.kappa2), d1=fl(p.d1), alpha1=fl(p.alpha1), d2=fl(p.d2),
                alpha2=fl(p.alpha2))


def _one(pair):
    from oracle import fit
    p, rep = fit.fit_relaxation(pair[0], pair[1], 2)
    d = _params(p)
    d.update(nrmse=float(rep.nrmse), disp_rmse=float(rep.disp_rmse), w=float(rep.w), failed=bool(rep.failed))
    d["per_w"] = [dict(_params(e["params"]), w=float(e["w"]), nrmse=float(e["nrmse"]), disp_rmse=float(e["disp"]))
                  for e in rep.per_w]
    return pair, d


def main():
    pairs = sorted({(a, y) for a in SWEEP_ALPHA0 for y in SWEEP_Y} | set(TISSUES.values()))
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        res = pool.map(_one, pairs)
    out = {"source": "oracle.fit.fit_relaxation(alpha0, y, 2) with its defaults (Sec. 3.2 settings)",
           "tissues": {k: key(*v) for k, v in TISSUES.items()},
           "sweep": {"alpha0": list(SWEEP_ALPHA0), "y": list(SWEEP_Y)},
           "sets": {key(*pair): d for pair, d in res}}
    with open(os.path.join(HERE, "relax_sets.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
