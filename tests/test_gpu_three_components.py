"""Three van der Waals fluids (Sec. VI, Fig. graphLB3Components): theta_cr = 0.5 and
rho_cr = 1 for all three components, nu = 0.05 (a^{cc'} = nu a, kappa^{cc'} = nu kappa,
the paper's cross terms), kappa = 2, theta = kT = 1/3.  Four phases coexist: three
liquids, each rich in one component, and a gas.  The run starts from periodic tanh slabs
(liquid A, gas, liquid B, gas, liquid C, gas) at the oracle's invariant point (Newton on
equal mu^c and p in all four phases) and must stay in the density domain, conserve each
component's mass, and keep its bulk densities near the invariant point.

gamma_mu is gamma_0 / 8 (gamma_0 from the interface relation of Sec. V): with gamma_0,
gamma_0/2 and gamma_0/4 the run leaves the domain after about 2e5, 4e5 and 8e5 steps,
while gamma_0/8 runs the paper's 1e6 steps (the paper also tuned its parameters by
hand for stability).  The test runs 2e5 steps; over that time the liquids match the
invariant point to 1e-3, the slow trace components (minority densities in the liquids,
~1.8e-3, and the gas) to 5e-2, and the density ratio is above 1000 (1225 at the
invariant point)."""
import numpy as np
import pytest

from oracle import thermo as T

pytestmark = pytest.mark.gpu

L, STEPS = 384, 200000


def setup():
    aa, bb = T.ab_from_critical(0.5, 1.0)
    nu, kap, N = 0.05, 2.0, 3
    a = np.full((N, N), nu * aa)
    np.fill_diagonal(a, aa)
    K = np.full((N, N), nu * kap)
    np.fill_diagonal(K, kap)
    b = np.full(N, bb)
    guess = [np.array([2.2, 1e-3, 1e-3]), np.array([1e-3, 2.2, 1e-3]), np.array([1e-3, 1e-3, 2.2]),
             np.array([0.1, 0.1, 0.1])]
    ph = T.polish_invariant_point(1 / 3, a, b, guess)
    w = np.sqrt(2 * kap / (0.5 * 3 - 1))  # interface width of Sec. V at theta_cr / kT = 1.5
    x = np.arange(L, dtype=float)
    bounds = [L * k / 6 for k in range(7)]
    order = [0, 3, 1, 3, 2, 3]
    prof = np.zeros((N, L))
    for k in range(6):
        lo, hi = bounds[k] - 0.5, bounds[k + 1] - 0.5
        m = sum(0.5 * (np.tanh((x + s - lo) / w) - np.tanh((x + s - hi) / w)) for s in (-L, 0, L))
        prof += np.outer(ph[order[k]], m)
    gamma = (2 / 3) / (4 * kap * ph[0][0]) / 8
    return a, K, b, ph, order, bounds, prof, gamma


def test_four_phase_coexistence_of_three_components(gpu_lib):
    from paper_1805_07251_gb300 import Simulation

    a, K, b, ph, order, bounds, prof, gamma = setup()
    N = 3
    sim = Simulation(lattice="D1Q3", nx=L, ny=1, ncomp=N, tau=1.0, kT=1 / 3, gamma_mu=gamma, a=a, kappa=K,
                     lam=np.ones((N, N)) - np.eye(N), b=b, precision="fp64")
    rho0 = prof.reshape(N, 1, L)
    sim.init(rho0)
    sim.step(STEPS)
    r, _ = sim.moments()  # raises on a domain error
    _, mass, _ = sim.free_energy()
    sim.close()
    m0 = rho0.reshape(N, -1).sum(axis=1)
    assert np.max(np.abs(mass - m0) / m0) < 1e-13
    r = r[:, 0, :]
    for k in range(6):
        c = int(0.5 * (bounds[k] + bounds[k + 1]))
        bulk = 0.5 * (r[:, c] + r[:, c + 1])  # the two sublattices (neutral period-2 mode)
        ref = ph[order[k]]
        rel = np.abs(bulk - ref) / ref
        if order[k] < 3:
            assert rel[order[k]] < 1e-3
            assert np.max(np.delete(rel, order[k])) < 5e-2
        else:
            assert np.max(rel) < 5e-2
    assert r.max() / r.min() > 1000
