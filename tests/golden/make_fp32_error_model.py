"""Write fp32_error_model.txt: the FP64 oracle's own response, on the 1D Au a0 = 270 workload,
to a perturbation of the size of FP32 rounding.  Calls only the oracle and the seeded
workload definitions.

The FP32 step rounds the momenta at every step (the positions and optical depths are
compensated float pairs, exact to ~2^-48).  The model: after every step each momentum
component is multiplied by 1 + e, e uniform in [-2^-23, 2^-23] (up to one FP32 ulp), drawn by
numpy.random.default_rng(0) and independent per component, particle and step.  The perturbed
run is compared with the unperturbed one on the electrons whose event words still match:
recorded are the event-match fraction and, for the momentum error relative to
max(|u|, a0), the position error relative to max(|x|, 1) and the optical-depth error relative
to max(|tau|, 1), the fraction of matched electrons below each threshold.  The GPU's FP32 path
is required to do no worse at every threshold, within binomial noise.

Cases (the GPU parity tests use the same electrons):
  small: 48-point tables, seed 2, electrons 0..999, 1500 steps
  full:  256 x 256 tables of the 1e6-electron workload, 256 electron ids drawn by
         numpy.random.default_rng(0).choice(1e6, 256), 4000 steps (the whole job)

Run:  python tests/golden/make_fp32_error_model.py  (about a minute on 16 cores)
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1612_07592_gb300 import workloads as W  # noqa: E402

THRESHOLDS = (1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fp32_error_model.txt")


def cases():
    small_tp = dict(W.tables_small(), n_eta=48, n_y=48, n_E=48, n_s=48)
    small_run = W.base_run(a0=270.0, init_dist=1, T_mev=1.0, seed=2, **W.AU)
    c = W.config2()
    full_ids = np.random.default_rng(0).choice(c["n"], 256, replace=False)
    return {"small": (small_tp, (13.0, 79.0), small_run, np.arange(1000), 1500),
            "full": (c["tables"], c["Z"], c["run"], full_ids, c["steps"])}


def errors(a, b, a0):
    """Per-electron relative errors of b against a: momentum, position, optical depth."""
    eu = np.abs(a[:, 2:5] - b[:, 2:5]).max(1) / np.maximum(np.abs(a[:, 2:5]).max(1), a0)
    ex = np.abs(a[:, 0:2] - b[:, 0:2]).max(1) / np.maximum(np.abs(a[:, 0:2]).max(1), 1.0)
    et = np.abs(a[:, 5] - b[:, 5]) / np.maximum(np.abs(a[:, 5]), 1.0)
    return eu, ex, et


def model(tp, Z, run, ids, steps):
    ot = O.Tables(O.table_params(**{("photon_min" if k == "photon_min_mc2" else k): v for k, v in tp.items()}),
                  list(Z))
    d = dict(run)
    d["iz"] = list(Z).index(d["Z"])
    rp = O.run_params(**d)
    a = O.init(ot, rp, ids)
    b = a.copy()
    ev_a = np.zeros(len(ids), np.uint64)
    ev_b = np.zeros(len(ids), np.uint64)
    O.run(ot, rp, ids, a, 0, steps, capacity=1 << 20, events=ev_a)
    rng = np.random.default_rng(0)
    for s in range(steps):
        b[:, 2:5] *= 1.0 + rng.uniform(-1.0, 1.0, (len(ids), 3)) * 2.0 ** -23
        O.run(ot, rp, ids, b, s, 1, capacity=1 << 12, events=ev_b)
    m = ev_a == ev_b
    eu, ex, et = errors(a, b, run["a0"])
    return m, eu[m], ex[m], et[m]


def main():
    lines = ["# FP64 oracle under a per-step one-ulp momentum perturbation (see make_fp32_error_model.py)",
             "# case quantity n_matched match_fraction frac_below(" + ",".join(f"{t:g}" for t in THRESHOLDS) + ")"]
    for name, (tp, Z, run, ids, steps) in cases().items():
        m, eu, ex, et = model(tp, Z, run, ids, steps)
        for q, e in (("u", eu), ("x", ex), ("tau", et)):
            fr = [float(np.mean(e < t)) for t in THRESHOLDS]
            lines.append(f"{name} {q} {int(m.sum())} {m.mean():.6f} " + " ".join(f"{v:.6f}" for v in fr))
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
