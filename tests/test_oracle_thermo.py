"""Pins of the oracle's bulk thermodynamics (Sec. II, Sec. VI, Appendix A of
Ridl & Wagner) against closed forms, finite differences, the paper's printed
caption values and textbook constructions."""
import json
import os

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import thermo as T

HERE = os.path.dirname(os.path.abspath(__file__))


def test_critical_point_is_inflection_of_pressure():
    # Eqs. tetcr, rhocr, pcr: at (theta_cr, rho_cr) dp/drho = d2p/drho2 = 0 and p = p_cr
    for a, b in [(0.45, 1 / 3), (1.0, 0.25), (0.7, 0.3)]:
        tc, rc, pc = T.critical_point(a, b)
        A, B = np.array([[a]]), np.array([b])

        def p(r):
            return float(T.pressure(tc, A, B, np.array([r])))

        h = 1e-4
        d1 = (p(rc + h) - p(rc - h)) / (2 * h)
        d2 = (p(rc + h) - 2 * p(rc) + p(rc - h)) / h ** 2
        assert abs(d1) < 1e-7 and abs(d2) < 1e-5
        assert abs(p(rc) - pc) < 1e-14
        # below theta_cr the isotherm has a loop, above it has none
        assert T.spinodal_1c(0.95 * tc, a, b) is not None
        assert T.spinodal_1c(1.05 * tc, a, b) is None


def test_ab_from_critical_inverts_critical_point():
    for tc, rc in [(0.4, 1.0), (0.3, 1.2), (0.45, 1.1)]:
        a, b = T.ab_from_critical(tc, rc)
        t2, r2, _ = T.critical_point(a, b)
        assert abs(t2 - tc) < 1e-15 and abs(r2 - rc) < 1e-15


@pytest.mark.parametrize("N", [1, 2, 3])
def test_mu_and_pressure_are_derivatives_of_f(N):
    rng = np.random.default_rng(7)
    a = rng.uniform(0.3, 1.2, (N, N))
    a = 0.5 * (a + a.T)
    b = rng.uniform(0.2, 0.35, N)
    kT = 0.6
    rho = rng.uniform(0.1, 0.6, N)
    mu = T.chemical_potential(kT, a, b, rho)
    h = 1e-6
    for c in range(N):
        e = np.zeros(N); e[c] = h
        fd = (T.free_energy_density(kT, a, b, rho + e) - T.free_energy_density(kT, a, b, rho - e)) / (2 * h)
        assert abs(fd - mu[c]) < 1e-8
    # bulk pressure of Sec. II equals sum rho mu - f (Legendre transform)
    p = T.pressure(kT, a, b, rho)
    assert abs(p - (rho @ mu - T.free_energy_density(kT, a, b, rho))) < 1e-13
    # Hessian is the Jacobian of mu
    H = T.hessian(kT, a, b, rho)
    for c in range(N):
        e = np.zeros(N); e[c] = h
        col = (T.chemical_potential(kT, a, b, rho + e) - T.chemical_potential(kT, a, b, rho - e)) / (2 * h)
        assert np.max(np.abs(col - H[:, c])) < 1e-7


def test_caption_parameters():
    # Sec. VI captions: (xi, zeta, Lambda) printed to 6 digits for 10 mixtures
    with open(os.path.join(HERE, "golden", "captions.json")) as fh:
        cases = json.load(fh)["cases"]
    for cs in cases:
        a, b, _ = T.mixture_from_critical(cs["tA"], cs["tB"], cs["rB"], cs["nu"], 0.1)
        got = np.array(T.konynenburg_scott(a, b))
        want = np.array([cs["xi"], cs["zeta"], cs["Lambda"]])
        if cs["magnitude_only"]:
            got, want = np.abs(got), np.abs(want)
        assert np.max(np.abs(np.round(got, 6) - want)) <= 1.5e-6, cs["fig"]


def test_maxwell_equal_area():
    # textbook: at coexistence, integral of p dv between the phases = p_coex (v_g - v_l)
    for tc in (0.4, 0.36):
        a, b = T.ab_from_critical(tc, 1.0)
        kT = 1 / 3
        rg, rl = T.maxwell_1c(kT, a, b)
        A, B = np.array([[a]]), np.array([b])

        def p_of_v(v):
            return float(T.pressure(kT, A, B, np.array([1.0 / v])))

        pc = p_of_v(1 / rg)
        area, _ = quad(p_of_v, 1 / rl, 1 / rg, limit=200, epsabs=1e-13, epsrel=1e-13)
        assert abs(area - pc * (1 / rg - 1 / rl)) < 1e-10
        assert abs(p_of_v(1 / rl) - pc) < 1e-13


def test_hull_identical_components_reduce_to_single_component():
    # Sec. VI (identical components, nu = 1): liquid and gas have the mean's composition
    # (tie lines through the origin) and total densities equal the single-component
    # Maxwell densities.
    a, b, _ = T.mixture_from_critical(0.4, 0.4, 1.0, 1.0, 0.1)
    aa, bb = T.ab_from_critical(0.4, 1.0)
    rg, rl = T.maxwell_1c(1 / 3, aa, bb)
    for x in (0.5, 0.3):
        mean = 0.8 * np.array([x, 1 - x])
        ph = T.coexistence(1 / 3, a, b, mean, n=400)
        assert len(ph) == 2
        tots = sorted(float(q.sum()) for q in ph)
        assert abs(tots[0] - rg) < 1e-9 and abs(tots[1] - rl) < 1e-9
        for q in ph:
            assert abs(q[0] / q.sum() - x) < 1e-9


def test_three_phase_triangle_of_baseline_case():
    # Sec. VI baseline (theta_cr = 0.4, nu = 0.5): the mean (0.8, 0.8) lies in the
    # three-phase region; the polished phases have equal mu^A, mu^B and p, the mean is
    # inside the triangle, and the construction is symmetric under A <-> B.
    a, b, _ = T.mixture_from_critical(0.4, 0.4, 1.0, 0.5, 0.1)
    ph = T.coexistence(1 / 3, a, b, [0.8, 0.8], n=400)
    assert len(ph) == 3
    mus = np.array([T.chemical_potential(1 / 3, a, b, q) for q in ph])
    ps = np.array([T.pressure(1 / 3, a, b, q) for q in ph])
    assert np.ptp(mus[:, 0]) < 1e-11 and np.ptp(mus[:, 1]) < 1e-11 and np.ptp(ps) < 1e-11
    P = np.array(ph)
    sym = [q for q in P if abs(q[0] - q[1]) < 1e-8]
    assert len(sym) == 1
    others = [q for q in P if abs(q[0] - q[1]) >= 1e-8]
    assert np.max(np.abs(others[0][::-1] - others[1])) < 1e-8
    # mean inside the triangle: barycentric weights in [0, 1]
    M = np.vstack([P.T, np.ones(3)])
    wts = np.linalg.solve(M, np.array([0.8, 0.8, 1.0]))
    assert np.all(wts > 0) and abs(wts.sum() - 1) < 1e-12
    # each phase is locally stable (positive definite Hessian)
    for q in ph:
        assert not T.is_unstable(1 / 3, a, b, q)


def test_two_phase_tie_line_lever_rule_and_stability():
    a = np.array([[1.0, 0.9], [0.9, 0.6]]); b = np.array([0.25, 0.3])
    kT = 0.85 * T.one_fluid_critical_temperature(a, b, [0.4, 0.6])
    mean = 1.2 * np.array([0.4, 0.6])
    assert T.is_unstable(kT, a, b, mean)
    ph = T.coexistence(kT, a, b, mean, n=400)
    assert len(ph) == 2
    r1, r2 = ph
    mu1, mu2 = T.chemical_potential(kT, a, b, r1), T.chemical_potential(kT, a, b, r2)
    assert np.max(np.abs(mu1 - mu2)) < 1e-11
    assert abs(T.pressure(kT, a, b, r1) - T.pressure(kT, a, b, r2)) < 1e-11
    d, e = r2 - r1, mean - r1
    assert abs(d[0] * e[1] - d[1] * e[0]) < 1e-12
    t = (e @ d) / (d @ d)
    assert 0 < t < 1
    # a common tangent plane: f(r) >= tangent plane through r1 on a coarse grid
    grid = np.stack(np.meshgrid(np.linspace(0.02, 2.5, 60), np.linspace(0.02, 2.0, 60))).reshape(2, -1)
    ok = b @ grid < 0.999
    g = grid[:, ok]
    f = T.free_energy_density(kT, a, b, g)
    plane = T.free_energy_density(kT, a, b, r1) + mu1 @ (g - r1[:, None])
    assert np.min(f - plane) > -1e-9


def test_appendix_a_minimiser_agrees_with_convex_hull():
    # Appendix A's quasi-brute-force three-phase minimiser and the convex-hull common
    # tangent (two independent minimisations of the same bulk free energy) agree on the
    # baseline three-phase point (Sec. VI, paper: minimiser uncertainty ~1e-6), on a
    # two-phase point, and on a stable mean (one phase).
    from oracle import appendix_a as AA

    a, b, _ = T.mixture_from_critical(0.4, 0.4, 1.0, 0.5, 0.1)
    hull = sorted(T.coexistence(1 / 3, a, b, [0.8, 0.8], n=400), key=lambda q: (q.sum(), q[0]))
    mini = AA.minimise(1 / 3, a, b, [0.8, 0.8])
    assert len(mini) == 3
    got = sorted([r for r, _ in mini], key=lambda q: (q.sum(), q[0]))
    for g, h in zip(got, hull):
        assert np.max(np.abs(g - h)) < 1e-5
    assert abs(sum(v for _, v in mini) - 1.0) < 1e-12
    a2 = np.array([[1.0, 0.9], [0.9, 0.6]]); b2 = np.array([0.25, 0.3])
    kT = 0.85 * T.one_fluid_critical_temperature(a2, b2, [0.4, 0.6])
    mean = 1.2 * np.array([0.4, 0.6])
    mini = AA.minimise(kT, a2, b2, mean)
    hull = sorted(T.coexistence(kT, a2, b2, mean, n=400), key=lambda q: q.sum())
    assert len(mini) == 2
    for (g, _), h in zip(mini, hull):
        assert np.max(np.abs(g - h)) < 1e-5
    # lever rule: volume-weighted densities give back the mean
    assert np.max(np.abs(sum(v * r for r, v in mini) - mean)) < 1e-9
    one = AA.minimise(kT, a2, b2, [0.02, 0.02])
    assert len(one) == 1


def test_invariant_point_solver():
    # N + 1 coexisting phases (Sec. II conditions).  Two components: the baseline
    # three-phase triangle of the convex hull (an independent minimisation) is
    # reproduced.  Three components (Sec. VI, Fig. graphLB3Components: theta_cr = 0.5,
    # rho_cr = 1, nu = 0.05, theta = 1/3): a four-phase point whose common tangent
    # hyperplane lies below the free energy everywhere on a grid of the domain.
    a, b, _ = T.mixture_from_critical(0.4, 0.4, 1.0, 0.5, 0.1)
    hull = sorted(T.coexistence(1 / 3, a, b, [0.8, 0.8], n=400), key=lambda q: (q.sum(), q[0]))
    start = [q + 1e-3 for q in hull]
    inv = sorted(T.polish_invariant_point(1 / 3, a, b, start), key=lambda q: (q.sum(), q[0]))
    for g, h in zip(inv, hull):
        assert np.max(np.abs(g - h)) < 1e-10
    aa, bb = T.ab_from_critical(0.5, 1.0)
    a3 = np.full((3, 3), 0.05 * aa)
    np.fill_diagonal(a3, aa)
    b3 = np.full(3, bb)
    guess = [np.array([2.2, 1e-3, 1e-3]), np.array([1e-3, 2.2, 1e-3]), np.array([1e-3, 1e-3, 2.2]),
             np.array([0.1, 0.1, 0.1])]
    ph = T.polish_invariant_point(1 / 3, a3, b3, guess)
    mu = T.chemical_potential(1 / 3, a3, b3, ph[0])
    for q in ph:
        assert not T.is_unstable(1 / 3, a3, b3, q)
    # symmetric under permutations of the components
    assert np.max(np.abs(ph[1] - ph[0][[1, 0, 2]])) < 1e-12 and np.max(np.abs(ph[2] - ph[0][[2, 1, 0]])) < 1e-12
    g = np.linspace(1e-4, 2.95, 48)
    G = np.stack(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1)
    G = G[:, b3 @ G < 0.999]
    f = T.free_energy_density(1 / 3, a3, b3, G)
    plane = T.free_energy_density(1 / 3, a3, b3, ph[0]) + mu @ (G - ph[0][:, None])
    assert np.min(f - plane) > -1e-12
