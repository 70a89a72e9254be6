"""Phase-diagram runs on the GPU (batched D1Q3 runs) against the Appendix A minimiser:
the paper's baseline mixture (Sec. VI, Fig. graphBaselineCase: theta_cr = 0.4 for both
components, rho_cr = 1, nu = 0.5, kappa = 0.1, theta = 1/3) along two of its two-phase
test paths (Fig. twoPhaseTestPoints), with the "log" and the "nid" forces (Sec. V).

Each run starts from tanh slabs at the minimiser's phases (the paper's practice), runs
50,000 steps, and its bulk densities (averaged over the two sublattices, see the
neutral period-2 mode of the D1Q3 scheme) are compared with the minimiser.  At
kappa = 0.1 the lattice pins interfaces and shifts bulk densities by ~1e-3, so the bar
for "log" is 5e-3; the paper reports "log" as the more accurate and more stable of the
two forces, which the test checks as: "nid" is worse on the median of the points."""
import numpy as np
import pytest

from oracle import appendix_a as AA
from oracle import thermo as T

pytestmark = pytest.mark.gpu

L = 256
STEPS = 50000


def path_points():
    pts = [(1 - t, t) for t in np.linspace(0.15, 0.85, 8)]          # diagonal (1,0) -> (0,1)
    pts += [(1.0, v) for v in np.linspace(0.1, 0.6, 4)]              # vertical from (1,0)
    return pts


def slab_fields(phases):
    """Phases (densities, volume fraction) side by side as tanh slabs of width 2."""
    x = np.arange(L, dtype=float)
    edges = np.cumsum([0.0] + [v for _, v in phases]) * L
    prof = np.zeros((2, L))
    for k, (r, _) in enumerate(phases):
        lo, hi = edges[k] - 0.5, edges[k + 1] - 0.5
        up = 0.5 * (1 + np.tanh((x - lo) / 2.0)) if k > 0 else np.ones(L)
        down = 0.5 * (1 - np.tanh((x - hi) / 2.0)) if k < len(phases) - 1 else np.ones(L)
        prof += np.outer(r, up * down)
    return np.maximum(prof, 1e-6).reshape(2, 1, L), edges


def run_paths(force):
    from paper_1805_07251_gb300.batch import Batch

    a, b, kap = T.mixture_from_critical(0.4, 0.4, 1.0, 0.5, 0.1)
    lam = np.array([[0.0, 1.0], [1.0, 0.0]])
    recs, fields, refs = [], [], []
    for mean in path_points():
        ph = AA.minimise(1 / 3, a, b, mean)
        if len(ph) != 2:       # the middle of the diagonal path is a stable single phase
            continue
        rho, edges = slab_fields(ph)
        rl = max(float(r.sum()) for r, _ in ph)
        # gamma_mu from the interface relation of Sec. V: c_s^2 = 1 - 4 kappa rho_l gamma
        recs.append(dict(lattice="D1Q3", nx=L, ny=1, kT=1 / 3, gamma_mu=(2 / 3) / (4 * 0.1 * rl)))
        fields.append(rho)
        refs.append((ph, edges))
    assert len(recs) >= 6
    bt = Batch(recs, a, b, kap, lam, 2, precision="fp64", force=force)
    bt.init(fields)
    bt.step(STEPS)
    err = bt.errors()
    devs = []
    for k, (ph, edges) in enumerate(refs):
        if err[k]:
            devs.append(np.inf)
            continue
        r, _ = bt.read(k)
        d = 0.0
        for q, (ref, _) in enumerate(ph):
            c = int(0.5 * (edges[q] + edges[q + 1]))
            bulk = 0.5 * (r[:, 0, c] + r[:, 0, c + 1])
            d = max(d, float(np.max(np.abs(bulk - ref))))
        devs.append(d)
    bt.close()
    return np.array(devs)


def test_log_force_recovers_two_phase_coexistence(gpu_lib):
    devs = run_paths("log")
    assert np.all(np.isfinite(devs)), devs
    assert np.max(devs) < 5e-3, devs


def test_nid_force_is_less_accurate_than_log(gpu_lib):
    log = run_paths("log")
    nid = run_paths("nid")
    assert np.median(nid) > np.median(log), (nid, log)
