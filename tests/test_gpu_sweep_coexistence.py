"""The batched phase-diagram sweep (workload c3: 256 D1Q3 + 128 D2Q9 runs of uneven sizes,
temperatures and compositions, FP32 storage with double-float mu) run for its full 20,000
steps, with every run's bulk phases compared against the oracle's common tangent (the
convex-hull tie line through the run's mean, stored per run in lbinputs/sweep.json).

Each two-phase run starts as a liquid slab in its gas at the tie-line densities; after
20,000 steps the densities at the slab centre and at the gas centre (averaged over the
two sublattices of the neutral period-2 mode, and over y for D2Q9) are compared with the
tie line.  At kappa = 0.1 the lattice itself shifts stationary bulk densities by ~2e-3
(pinning of interfaces), so the bars are statistical over the runs: D1Q3 median 2e-3 and
95 % within 5e-3; D2Q9 (where 20,000 steps do not relax every 512^2 slab) median 5e-3 and
85 % within 1e-2.  As in the paper's campaigns (Sec. VI), a 3000-step pre-scan re-tunes
the runs that leave the density domain (deep quenches: interfaces widened by a larger
kappa, gamma_mu lowered); after it at most 8 % of the runs may still leave the domain
over the 20,000 steps, and every run at kT >= 0.75 of its critical temperature must stay
in it."""
import numpy as np
import pytest

import lbinputs

pytestmark = pytest.mark.gpu


def test_sweep_phases_lie_on_the_common_tangent(gpu_lib, parity_bound):
    from paper_1805_07251_gb300.batch import Batch, prescan

    p = lbinputs.base_params("c1")
    recs, _ = prescan(lbinputs.sweep_runs(), lbinputs.sweep_fields, p["a"], p["b"], p["kappa"], p["lam"], 2,
                      precision="fp32_dfmu")
    b = Batch(recs, p["a"], p["b"], p["kappa"], p["lam"], 2, precision="fp32_dfmu")
    b.init([lbinputs.sweep_fields(r) for r in recs])
    b.step(20000)
    err = b.errors()
    devs = {"D1Q3": [], "D2Q9": []}
    for k, r in enumerate(recs):
        if err[k]:
            assert r["kT_frac"] < 0.75, (k, r["kT_frac"])
            continue
        if "liquid" not in r:
            continue
        rho, _ = b.read(k)
        prof = rho.mean(axis=1)
        c = r["nx"] // 2
        liq = 0.5 * (prof[:, c] + prof[:, c + 1])
        gas = 0.5 * (prof[:, 0] + prof[:, 1])
        devs[r["lattice"]].append(max(np.max(np.abs(liq - np.asarray(r["liquid"]))),
                                      np.max(np.abs(gas - np.asarray(r["gas"])))))
    b.close()
    parity_bound("runs leaving the domain (fraction)", float(np.mean(err != 0)), 0.08)
    d1, d2 = np.array(devs["D1Q3"]), np.array(devs["D2Q9"])
    parity_bound("D1Q3 median bulk deviation", np.median(d1), 2e-3)
    parity_bound("D2Q9 median bulk deviation", np.median(d2), 5e-3)
    assert len(d1) > 150 and len(d2) > 80
    assert np.median(d1) < 2e-3 and np.mean(d1 < 5e-3) > 0.95, (np.median(d1), np.mean(d1 < 5e-3))
    assert np.median(d2) < 5e-3 and np.mean(d2 < 1e-2) > 0.85, (np.median(d2), np.mean(d2 < 1e-2))
