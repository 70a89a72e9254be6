"""GPU tests of the method's dynamics beyond parity of single steps: linear interdiffusion
of a composition wave at the Maxwell-Stefan / Fick rate of Sec. IV (Eq. MaxwellStefan and
its Fickian limit), on the GPU against the rate and against the FP64 oracle's trajectory."""
import numpy as np
import pytest

import oracle
from oracle import thermo as T

pytestmark = pytest.mark.gpu


def _wave_case(lam, lattice):
    a = np.array([[1.0, 0.7], [0.7, 1.0]])
    b = np.array([0.25, 0.25])
    kT = 1.2 * T.one_fluid_critical_temperature(a, b, [0.5, 0.5])
    nx, ny = 128, (1 if lattice == "D1Q3" else 8)
    gam, rA, rho, eps = 0.5, 0.5, 1.0, 2e-3
    k = 2 * np.pi / nx
    x = np.arange(nx)
    wave = np.cos(k * x)[None, :] * np.ones((ny, 1))
    r0 = np.stack([rA + eps * wave, rho - rA - eps * wave])
    H = T.hessian(kT, a, b, np.array([rA, rho - rA]))
    h = H[0, 0] - H[0, 1] - H[1, 0] + H[1, 1]
    predicted = gam * rA * (rho - rA) * h * k * k / (rho * lam)
    kw = dict(lattice=lattice, nx=nx, ny=ny, ncomp=2, tau=1.0, kT=kT, gamma_mu=gam, a=a,
              kappa=np.full((2, 2), 0.1), lam=np.array([[0.0, lam], [lam, 0.0]]), b=b)
    return kw, r0, predicted, k, x


def _amplitude(r, k, x):
    return np.abs(np.mean(0.5 * (r[0] - r[1]).mean(axis=0) * np.exp(-1j * k * x)))


@pytest.mark.parametrize("precision", ["fp64", "fp32_dfmu"])
@pytest.mark.parametrize("lattice", ["D1Q3", "D2Q9"])
@pytest.mark.parametrize("lam", [0.5, 1.0, 4.0])
def test_gpu_interdiffusion_follows_maxwell_stefan_fick_law(gpu_lib, parity_bound, lam, lattice, precision):
    # Sec. IV: at fixed total density the composition mode exp(ikx) relaxes at
    # gamma rho^A rho^B h k^2 / (rho lambda), h the bulk Hessian along the composition
    # direction.  The amplitude is sampled over five predicted decay times and the rate
    # fitted over the last four (after the start-up transient, while the amplitude stays
    # far above the rounding floor of the storage precision); it must be within 1 % of the
    # prediction, and in FP64 the amplitude history must follow the oracle's.
    from paper_1805_07251_gb300 import Simulation

    kw, r0, predicted, k, x = _wave_case(lam, lattice)
    chunk = max(1, int(round(5.0 / predicted / 40)))
    sim = Simulation(precision=precision, **kw)
    sim.init(r0)
    ts, amps = [], []
    for t in range(1, 41):
        sim.step(chunk)
        r, _ = sim.moments()
        ts.append(chunk * t)
        amps.append(_amplitude(r, k, x))
    sim.close()
    rate = -np.polyfit(ts[8:], np.log(amps[8:]), 1)[0]
    parity_bound("decay rate / Fick rate - 1", abs(rate / predicted - 1), 0.01)
    if precision == "fp64":
        L = oracle.Lattice(lattice, kw["nx"], kw["ny"], 2, kw["tau"], kw["kT"], kw["gamma_mu"], kw["a"],
                           kw["kappa"], kw["lam"], kw["b"])
        f = L.equilibrium(r0)
        worst = 0.0
        for t in range(1, 41):
            f = L.run(f, chunk)
            ro, _ = L.moments(f)
            worst = max(worst, abs(_amplitude(ro, k, x) - amps[t - 1]) / amps[t - 1])
        parity_bound("amplitude vs oracle (rel.)", worst, 1e-9)
