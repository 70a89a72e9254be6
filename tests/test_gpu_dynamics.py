"""GPU tests of the method's dynamics beyond parity of single steps: linear interdiffusion
of a composition wave at the Maxwell-Stefan / Fick rate of Sec. IV (Eq. MaxwellStefan and
its Fickian limit), on the GPU against the rate and against the FP64 oracle's trajectory;
the large-amplitude interdiffusion of an ideal mixture, linear at any composition; the
moment-space collision against the oracle."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32_dfmu"])
@pytest.mark.parametrize("force", ["nid", "log"])
def test_gpu_ideal_mixture_interdiffusion_is_linear_at_large_amplitude(gpu_lib, parity_bound, force, precision):
    # Sec. IV (Eq. MaxwellStefan): an ideal mixture (a = kappa = 0, equal b) at uniform
    # total density interdiffuses by linear diffusion at any composition, flux
    # -(gamma kT / lambda) D rho^A ("nid" at gamma kT = theta: theta / lambda).  A
    # composition wave from x = 0.1 to 0.9 must decay at the small-amplitude rate and at
    # the Fick rate, as it does in the oracle, and in FP64 follow the oracle's amplitudes.
    from paper_1805_07251_gb300 import Simulation

    nx, rho, kT, lam = 256, 1.6, 0.5, 2.0
    theta = 1.0 / 3.0
    gam = theta / kT if force == "nid" else 0.6
    k = 2 * np.pi / nx
    x = np.arange(nx)
    kw = dict(lattice="D1Q3", nx=nx, ny=1, ncomp=2, tau=1.0, kT=kT, gamma_mu=gam, a=np.zeros((2, 2)),
              kappa=np.zeros((2, 2)), lam=np.array([[0.0, lam], [lam, 0.0]]), b=np.array([0.2, 0.2]))
    rates, hist = {}, {}
    for A in (0.005, 0.4):
        xa = 0.5 + A * np.cos(k * x)[None, :]
        r0 = np.stack([rho * xa, rho * (1 - xa)])
        sim = Simulation(precision=precision, force=force, **kw)
        sim.init(r0)
        ts, amps = [], []
        for t in range(1, 41):
            sim.step(250)
            r, _ = sim.moments()
            ts.append(250 * t)
            amps.append(_amplitude(r, k, x))
        sim.close()
        rates[A] = -np.polyfit(ts[5:], np.log(amps[5:]), 1)[0]
        hist[A] = (r0, amps)
    predicted = (theta if force == "nid" else gam * kT) * k * k / lam
    parity_bound("small-amplitude rate / Fick rate - 1", abs(rates[0.005] / predicted - 1), 0.005)
    # FP32 storage: the small wave's amplitude (8e-3) sits ~1e5 above the rounding floor
    parity_bound("large / small amplitude rate - 1", abs(rates[0.4] / rates[0.005] - 1),
                 5e-5 if precision == "fp64" else 2e-4)
    if precision == "fp64":
        r0, amps = hist[0.4]
        L = oracle.Lattice("D1Q3", nx, 1, 2, 1.0, kT, gam, kw["a"], kw["kappa"], kw["lam"], kw["b"],
                           force_method=1 if force == "nid" else 0)
        f = L.equilibrium(r0)
        worst = 0.0
        for t in range(1, 41):
            f = L.run(f, 250)
            ro, _ = L.moments(f)
            worst = max(worst, abs(_amplitude(ro, k, x) - amps[t - 1]) / amps[t - 1])
        parity_bound("large-amplitude history vs oracle (rel.)", worst, 1e-9)


# ------------------------------------------------------------ moment-space collision

def _mrt_pair(precision, tau_s, tau_g, nx, ny, kT=None, **over):
    from paper_1805_07251_gb300 import Simulation
    import lbinputs

    p = lbinputs.base_params("c2")
    kw = lbinputs.lib_kwargs(p, **over)
    kw["nx"], kw["ny"] = nx, ny
    if kT is not None:
        kw["kT"] = kT
    sim = Simulation(precision=precision, tau_shear=tau_s, tau_ghost=tau_g, **kw)
    orc = oracle.Lattice("D2Q9", nx, ny, 2, kw["tau"], kw["kT"], kw["gamma_mu"], kw["a"], kw["kappa"], kw["lam"],
                         kw["b"], tau_s=tau_s, tau_g=tau_g)
    return sim, orc


@pytest.mark.parametrize("tau_s,tau_g", [(0.7, 0.9), (1.0, 0.6), (0.55, 1.0)])
def test_mrt_fp64_trajectory_and_step_match_oracle(gpu_lib, parity_bound, tau_s, tau_g):
    # Eq. BGKcollisionOperator with distinct relaxation times on the GPU (FP64) against the
    # oracle's moment-space collision: the one-phase config-2 mixture over 1000 steps, and
    # one step restarted from the GPU state of the spinodal mixture
    import lbinputs

    p = lbinputs.base_params("c2")
    kT1 = 1.1 * lbinputs.one_fluid_critical_kT(p["a"], p["b"], p["x"])
    sim, orc = _mrt_pair("fp64", tau_s, tau_g, 70, 45, kT=kT1)
    rho = lbinputs.fields("c2", nx=70, ny=45)
    sim.init(rho)
    sim.step(1000)
    r_g, j_g = sim.moments()
    r_o, j_o = orc.moments(orc.run(orc.equilibrium(rho), 1000))
    parity_bound("rho rel. max, 1000 steps", np.max(np.abs(r_g - r_o)) / np.max(np.abs(r_o)), 1e-12)
    parity_bound("j / max rho, 1000 steps", np.max(np.abs(j_g - j_o)) / np.max(np.abs(r_o)), 1e-12)
    sim.close()
    sim, orc = _mrt_pair("fp64", tau_s, tau_g, 70, 45)
    sim.init(rho)
    sim.step(200)
    fshape = orc.fshape()
    buf = sim.save_state()
    f_t = np.frombuffer(buf[64:].tobytes(), dtype=np.float64).reshape(fshape).copy()
    sim.step(1)
    buf = sim.save_state()
    f_n = np.frombuffer(buf[64:].tobytes(), dtype=np.float64).reshape(fshape).copy()
    parity_bound("one step at 200", np.max(np.abs(f_n - orc.run(f_t, 1))), 1e-14)
    sim.close()


@pytest.mark.parametrize("precision", ["fp32_dfmu", "fp32_mixed"])
def test_mrt_fp32_one_phase_within_1e5(gpu_lib, parity_bound, precision):
    import lbinputs

    p = lbinputs.base_params("c2")
    kT1 = 1.1 * lbinputs.one_fluid_critical_kT(p["a"], p["b"], p["x"])
    sim, orc = _mrt_pair(precision, 0.7, 0.9, 70, 45, kT=kT1)
    rho = lbinputs.fields("c2", nx=70, ny=45)
    sim.init(rho)
    sim.step(1000)
    r_g, _ = sim.moments()
    r_o, _ = orc.moments(orc.run(orc.equilibrium(rho), 1000))
    parity_bound("rho max abs, 1000 steps", np.max(np.abs(r_g - r_o)), 1e-5)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_dfmu"])
def test_mrt_shear_wave_decays_at_shear_viscosity_on_gpu(gpu_lib, parity_bound, precision):
    # nu = theta (tau_s - 1/2): a transverse wave in an ideal gas (a = kappa = 0, b small)
    from paper_1805_07251_gb300 import Simulation

    nx, ny, tau_s = 128, 8, 0.6
    k = 2 * np.pi / nx
    x = np.arange(nx)
    sim = Simulation(lattice="D2Q9", nx=nx, ny=ny, ncomp=1, tau=1.0, kT=1.0 / 3.0, gamma_mu=1.0, a=[[0.0]],
                     kappa=[[0.0]], lam=[[0.0]], b=[1e-9], precision=precision, tau_shear=tau_s, tau_ghost=0.9)
    mom = np.zeros((1, 2, ny, nx))
    mom[0, 1] = 1e-3 * np.sin(k * x)[None, :]
    sim.init(np.ones((1, ny, nx)), mom)
    ts, amps = [], []
    for t in range(1, 21):
        sim.step(50)
        _, j = sim.moments()
        ts.append(50 * t)
        amps.append(np.abs(np.mean(j[0, 1].mean(axis=0) * np.exp(-1j * k * x))))
    sim.close()
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    parity_bound("shear decay / nu k^2 - 1", abs(rate / ((tau_s - 0.5) / 3.0 * k * k) - 1), 1e-3)
