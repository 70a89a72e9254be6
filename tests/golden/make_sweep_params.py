"""Write lbinputs/sweep.json: per-run coexisting phases for the batched sweep (workload c3).

Calls only the CPU oracle (``oracle.thermo``) and the seeded generators of ``lbinputs``.
Run r draws from numpy default_rng(1805072600 + r): D1Q3 runs (r < 256) a length
L ~ U{128..4096}, D2Q9 runs a square side ~ U{64..512}; every run a mole fraction
x ~ U(0.05, 0.95) of component A and kT ~ U(0.6, 0.98) of the one-fluid critical
temperature at x.  The mixture is workload c1's (a = [[1, .7], [.7, 1]], b = .25,
kappa = .1).  The mean total density is the one-fluid critical density 1/(3 b.x); the
oracle's convex-hull common tangent at that mean gives the coexisting gas and liquid,
between which the run's slab is initialised (Sec. V practice: tanh profiles at the
minimiser's bulk values), and gamma_mu = 1/(6 kappa rho_l) / 8 (Sec. V interface
relation, lowered by a factor within the paper's 2-10 range for stability).

Run:  python tests/golden/make_sweep_params.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import lbinputs  # noqa: E402
from oracle import thermo  # noqa: E402


def main():
    runs = lbinputs.sweep_runs(with_phases=False)
    p = lbinputs.base_params("c1")
    a, b, kap = p["a"], p["b"], 0.1
    out = []
    hulls = {}
    for r in runs:
        x = np.array([r["x"], 1 - r["x"]])
        mean = x / (3.0 * float(b @ x))
        key = round(r["kT"], 12)
        hull = hulls.get(key) or thermo.HullPhaseDiagram(r["kT"], a, b, n=300)
        hulls = {key: hull}
        ph = thermo.coexistence(r["kT"], a, b, mean, hull=hull)
        rec = {"mean": mean.tolist()}
        if len(ph) >= 2:
            ph = sorted(ph, key=lambda q: float(q.sum()))
            rec["gas"], rec["liquid"] = ph[0].tolist(), ph[-1].tolist()
            rho_l = float(ph[-1].sum())
        else:
            rho_l = float(mean.sum())
        rec["gamma_mu"] = 1.0 / (6.0 * kap * rho_l) / 8.0
        out.append(rec)
        print(len(out), r["lattice"], r["nx"], r["ny"], round(r["kT"], 4), round(r["x"], 3), len(ph), flush=True)
    with open(lbinputs.SWEEP_JSON, "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
