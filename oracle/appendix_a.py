"""Second coexistence oracle: the quasi-brute-force three-phase minimiser of
Ridl & Wagner, Appendix A (TEST INFRASTRUCTURE ONLY, see the package docstring).

The system has unit volume and mean densities (A, B).  It is split into three phases
k = 1, 2, 3 with particle numbers (A_k, B_k) and volumes V_k; phase 3 follows from
conservation (A = sum A_k, B = sum B_k, 1 = sum V_k).  The total bulk free energy
sum_k V_k f(A_k/V_k, B_k/V_k) is minimised by a coordinate search over the six free
numbers (A_1, B_1, V_1, A_2, B_2, V_2): every one of them is moved by +step and -step
(a 6 x 2 set of trials next to the unchanged state), the best trial is taken when it
lowers the free energy, otherwise the step is halved, until the free energy changes by
less than 1e-12 (the paper's threshold) and the step is small.  The start follows the
appendix: a stability test by the Hessian; for an unstable mean, volumes 1/3 each and
the particles of phases 1 and 2 split along the eigenvector of the negative
eigenvalue, phase 3 starting (almost) empty.  Phases that end with equal densities are
merged; a phase that is still unstable is split again along its own eigenvector.

This module shares the bulk functions of ``thermo`` (the same free energy the paper
minimises) but none of its convex-hull construction, so the two coexistence oracles
check each other.
"""
from __future__ import annotations

import numpy as np

from . import thermo

_EMPTY = 1e-9   # density floor of an (almost) empty phase


def _phase_f(kT, a, b, n, V):
    """V f(n/V) for particle numbers n (2,) in volume V, with f(0) = 0."""
    if V <= 0:
        return np.inf
    rho = np.maximum(np.asarray(n, float) / V, _EMPTY)
    if b @ rho >= 1.0:
        return np.inf
    return V * float(thermo.free_energy_density(kT, a, b, rho))


def _total(kT, a, b, x, tot):
    """x = (A1, B1, V1, A2, B2, V2); tot = (A, B)."""
    n1, V1 = x[0:2], x[2]
    n2, V2 = x[3:5], x[5]
    n3 = tot - n1 - n2
    V3 = 1.0 - V1 - V2
    if np.any(n1 < 0) or np.any(n2 < 0) or np.any(n3 < 0) or V3 <= 0:
        return np.inf
    return _phase_f(kT, a, b, n1, V1) + _phase_f(kT, a, b, n2, V2) + _phase_f(kT, a, b, n3, V3)


def _split_start(kT, a, b, mean, vol):
    """Particles of a phase of density `mean` and volume `vol` split between two halves
    along the unstable eigenvector (Appendix A, step 3)."""
    H = thermo.hessian(kT, a, b, np.maximum(mean, _EMPTY))
    w, v = np.linalg.eigh(H)
    e = v[:, 0]
    if e[0] < 0:
        e = -e
    tot = mean * vol
    # the largest shift keeping both halves non-negative, scaled down
    s = 0.4 * min(tot[0], tot[1]) / max(abs(e[0]), abs(e[1]), 1e-12)
    return tot / 2 + s * e, tot / 2 - s * e


def minimise(kT, a, b, mean, step0=0.05, tol=1e-12, max_iter=200000):
    """Coexisting phases for mean densities (A, B): a list of 1-3 density pairs with the
    volume fraction of each (sorted by total density)."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    mean = np.asarray(mean, float)
    if not thermo.is_unstable(kT, a, b, mean):
        return [(mean.copy(), 1.0)]
    n1, n2 = _split_start(kT, a, b, mean, 2.0 / 3.0)
    x = np.array([n1[0], n1[1], 1 / 3, n2[0], n2[1], 1 / 3])
    tot = mean.copy()
    x = _coordinate_search(kT, a, b, x, tot, step0, tol, max_iter)
    phases = _phases(x, tot)
    # a phase that is still unstable is split again along its eigenvector (step 6)
    for _ in range(3):
        bad = [k for k, (r, V) in enumerate(phases) if V > 1e-6 and thermo.is_unstable(kT, a, b, r)]
        if not bad or len(phases) >= 3:
            break
        k = bad[0]
        r, V = phases[k]
        others = [p for j, p in enumerate(phases) if j != k]
        h1, h2 = _split_start(kT, a, b, r, V)
        # phase 1 and 2: halves of the unstable phase; phase 3: the stable rest
        x = np.array([h1[0], h1[1], V / 2, h2[0], h2[1], V / 2])
        x = _coordinate_search(kT, a, b, x, tot, step0, tol, max_iter)
        phases = _phases(x, tot)
    return phases


def _coordinate_search(kT, a, b, x, tot, step, tol, max_iter):
    F = _total(kT, a, b, x, tot)
    for _ in range(max_iter):
        best, bestF = None, F
        for k in range(6):
            for sgn in (1.0, -1.0):
                y = x.copy()
                y[k] += sgn * step
                Fy = _total(kT, a, b, y, tot)
                if Fy < bestF:
                    best, bestF = y, Fy
        if best is not None and bestF < F:
            dF = F - bestF
            x, F = best, bestF
            if dF < tol and step < 1e-9:
                break
        else:
            step *= 0.5
            if step < 1e-13:
                break
    return x


def _phases(x, tot, merge=1e-4):
    n = [x[0:2], x[3:5], tot - x[0:2] - x[3:5]]
    V = [x[2], x[5], 1.0 - x[2] - x[5]]
    raw = [(n[k] / V[k], V[k]) for k in range(3) if V[k] > 1e-7]
    out = []
    for r, v in raw:
        for k, (q, w) in enumerate(out):
            if np.max(np.abs(q - r)) < merge:
                out[k] = ((q * w + r * v) / (w + v), w + v)
                break
        else:
            out.append((r, v))
    return sorted(out, key=lambda p: float(p[0].sum()))
