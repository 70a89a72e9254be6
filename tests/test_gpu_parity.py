"""GPU parity of the fused CUDA timestep against the CPU oracle, through the C ABI.

Bars: FP64 densities within 1e-12 relative (max norm) after 1000 steps and mass
conserved to 1e-13; FP32-mixed densities within 1e-5 of the FP64 oracle after
1000 steps.  Inputs are the seeded synthetic fields of ``lbinputs``."""
import numpy as np
import pytest

import lbinputs
import oracle
from oracle_windows import oracle_two_steps_at

pytestmark = pytest.mark.gpu


def make_pair(p, precision="fp64", force="log", tile=None, nx=None, ny=None, **over):
    from paper_1805_07251_gb300 import Simulation

    kw = lbinputs.lib_kwargs(p, **over)
    if nx is not None:
        kw["nx"], kw["ny"] = nx, ny
    sim = Simulation(precision=precision, force=force, tile=tile, **kw)
    orc = oracle.Lattice(kw["lattice"], kw["nx"], kw["ny"], kw["ncomp"], kw["tau"], kw["kT"], kw["gamma_mu"],
                         kw["a"], kw["kappa"], kw["lam"], kw["b"], force_method=1 if force == "nid" else 0)
    return sim, orc


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def run_both(sim, orc, rho, steps, mom=None):
    sim.init(rho, mom)
    sim.step(steps)
    r_gpu, j_gpu = sim.moments()
    f = orc.run(orc.equilibrium(rho, mom), steps)
    r_orc, j_orc = orc.moments(f)
    return r_gpu, j_gpu, r_orc, j_orc


# ------------------------------------------------------------------ FP64

def gpu_populations(sim, fshape, dtype=np.float64):
    buf = sim.save_state()
    return np.frombuffer(buf[64:].tobytes(), dtype=dtype).reshape(fshape).copy()


def ulp_amplification(orc, rho, steps, seed=0):
    """Growth of a one-ulp relative perturbation of the initial densities over
    ``steps`` oracle steps: the conditioning of the trajectory itself."""
    s = np.random.default_rng(seed).choice([-1.0, 1.0], size=rho.shape)
    r0, _ = orc.moments(orc.run(orc.equilibrium(rho), steps))
    r1, _ = orc.moments(orc.run(orc.equilibrium(rho * (1 + 2.0 ** -52 * s)), steps))
    return rel_err(r1, r0)


def test_fp64_d2q9_one_phase_1000_steps(gpu_lib, parity_bound):
    # config-2 mixture above its critical temperature: fluctuations decay, so rounding
    # differences are not amplified and the 1000-step trajectories must agree to 1e-12
    p = lbinputs.base_params("c2")
    kT = 1.1 * lbinputs.one_fluid_critical_kT(p["a"], p["b"], p["x"])
    sim, orc = make_pair(p, nx=70, ny=45, kT=kT)
    rho = lbinputs.fields("c2", nx=70, ny=45)
    r_g, j_g, r_o, j_o = run_both(sim, orc, rho, 1000)
    parity_bound("rho rel. max, 1000 steps", rel_err(r_g, r_o), 1e-12)
    parity_bound("j / max rho, 1000 steps", np.max(np.abs(j_g - j_o)) / np.max(np.abs(r_o)), 1e-12)
    m0 = rho.reshape(2, -1).sum(axis=1)
    _, mass, _ = sim.free_energy()
    parity_bound("mass drift", np.max(np.abs(mass - m0) / m0), 1e-13)


def test_fp64_d2q9_spinodal_1000_steps(gpu_lib, parity_bound):
    # config-2 mixture (spinodal decomposition), ragged lattice spanning several tiles.
    # Unstable modes amplify every rounding difference, so the trajectory bound is
    # 1e-12 or 100x the oracle's own amplification of a one-ulp input change,
    # whichever is larger; the step itself is checked to 1e-14 by restarting the
    # oracle from the GPU state along the trajectory.
    p = lbinputs.base_params("c2")
    sim, orc = make_pair(p, nx=70, ny=45)
    rho = lbinputs.fields("c2", nx=70, ny=45)
    fshape = orc.fshape()
    sim.init(rho)
    for t in range(4):
        f_t = gpu_populations(sim, fshape)
        sim.step(1)
        f_next = gpu_populations(sim, fshape)
        parity_bound(f"one step at {333 * t}", np.max(np.abs(f_next - orc.run(f_t, 1))), 1e-14)
        sim.step(332)
    sim.init(rho)
    sim.step(1000)
    r_g, _ = sim.moments()
    r_o, _ = orc.moments(orc.run(orc.equilibrium(rho), 1000))
    amp = ulp_amplification(orc, rho, 1000)
    parity_bound("oracle 1-ulp amplification", amp, 1.0)
    parity_bound("rho rel. max, 1000 steps", rel_err(r_g, r_o), max(1e-12, 100.0 * amp))
    m0 = rho.reshape(2, -1).sum(axis=1)
    _, mass, _ = sim.free_energy()
    parity_bound("mass drift", np.max(np.abs(mass - m0) / m0), 1e-13)


def test_fp64_config2_recipe_256_1000_steps(gpu_lib, parity_bound):
    # the headline recipe (config-2 mixture, spinodal decomposition) on a 256 x 256
    # lattice (32 x 32 tiles), 1000 FP64 steps against the oracle.  The oracle's own
    # amplification of a one-ulp input change over the same 1000 steps measures how far
    # two correct FP64 implementations that round differently can drift apart; the bound
    # is 1e-12 or 100x that amplification, whichever is larger, and both are recorded.
    p = lbinputs.base_params("c2")
    sim, orc = make_pair(p, nx=256, ny=256)
    rho = lbinputs.fields("c2", nx=256, ny=256)
    r_g, j_g, r_o, j_o = run_both(sim, orc, rho, 1000)
    amp = ulp_amplification(orc, rho, 1000)
    parity_bound("oracle 1-ulp amplification", amp, 1.0)
    parity_bound("rho rel. max, 1000 steps", rel_err(r_g, r_o), max(1e-12, 100.0 * amp))
    parity_bound("j / max rho, 1000 steps", np.max(np.abs(j_g - j_o)) / np.max(np.abs(r_o)),
                 max(1e-12, 100.0 * amp))
    m0 = rho.reshape(2, -1).sum(axis=1)
    _, mass, _ = sim.free_energy()
    parity_bound("mass drift", np.max(np.abs(mass - m0) / m0), 1e-13)


def test_fp64_full_size_config2_restarts_along_trajectory(gpu_lib, parity_bound):
    # the benchmark's lattice (1024 x 1024, config 2) in FP64: at steps 0, 500 and 1000 of
    # the GPU's own trajectory, one GPU step against the oracle's step restarted from the
    # GPU state on 9 x 9 periodic windows around sampled nodes (the step's dependency
    # radius is 3, so the window centre is exact); every population of the centre node.
    p = lbinputs.base_params("c2")
    sim, _ = make_pair(p)
    rho = lbinputs.fields("c2")
    kw = lbinputs.lib_kwargs(p)
    win = oracle.Lattice("D2Q9", 9, 9, 2, kw["tau"], kw["kT"], kw["gamma_mu"], kw["a"], kw["kappa"],
                         kw["lam"], kw["b"])
    fshape = (2, 9, 1024, 1024)
    r = np.random.default_rng(79)
    sim.init(rho)
    done = 0
    for t in (0, 500, 1000):
        sim.step(t - done)
        f_t = gpu_populations(sim, fshape)
        sim.step(1)
        done = t + 1
        f_next = gpu_populations(sim, fshape)
        pts = [(0, 0), (1023, 1023), (512, 0), (0, 777)] + [tuple(r.integers(0, 1024, 2)) for _ in range(30)]
        worst = 0.0
        for (y, x) in pts:
            ys = (np.arange(-4, 5) + y) % 1024
            xs = (np.arange(-4, 5) + x) % 1024
            fo = win.run(f_t[:, :, ys][:, :, :, xs], 1)
            worst = max(worst, float(np.max(np.abs(f_next[:, :, y, x] - fo[:, :, 4, 4]))))
        parity_bound(f"one step at {t}, populations", worst, 1e-14)


def test_fp64_d1q3_config1_full_size(gpu_lib, parity_bound):
    p = lbinputs.base_params("c1")
    sim, orc = make_pair(p)
    rho = lbinputs.fields("c1")
    r_g, j_g, r_o, j_o = run_both(sim, orc, rho, 1000)
    parity_bound("rho rel. max, 1000 steps", rel_err(r_g, r_o), 1e-12)
    m0 = rho.reshape(2, -1).sum(axis=1)
    _, mass, _ = sim.free_energy()
    parity_bound("mass drift", np.max(np.abs(mass - m0) / m0), 1e-13)


@pytest.mark.parametrize("N", [1, 3, 4])
@pytest.mark.parametrize("lattice", ["D1Q3", "D2Q9"])
def test_fp64_component_counts(gpu_lib, parity_bound, N, lattice):
    r = np.random.default_rng(100 + N)
    a = r.uniform(0.5, 1.2, (N, N)); a = 0.5 * (a + a.T); np.fill_diagonal(a, 1.0)
    b = r.uniform(0.2, 0.35, N)
    x = np.full(N, 1.0 / N)
    kT = 0.9 * lbinputs.one_fluid_critical_kT(a, b, x)
    lam = np.ones((N, N)) - np.eye(N)
    nx, ny = (133, 1) if lattice == "D1Q3" else (37, 29)
    p = dict(lattice=lattice, nx=nx, ny=ny, ncomp=N, tau=1.0, kT=kT, gamma_mu=0.15, a=a, b=b,
             kappa=np.full((N, N), 0.1), lam=lam)
    sim, orc = make_pair(p)
    rho = lbinputs.uniform_noise_fields(N, ny, nx, 1.3 * x, 1e-2, 2024 + N)
    r_g, j_g, r_o, j_o = run_both(sim, orc, rho, 300)
    # below the critical temperature the mixture phase-separates, which amplifies
    # rounding differences: the bound is 1e-12 or 100 x the trajectory's own growth
    # of a one-ulp perturbation, whichever is larger
    amp = ulp_amplification(orc, rho, 300)
    bound = max(1e-12, 100.0 * amp)
    parity_bound("oracle 1-ulp amplification", amp, 1.0)
    parity_bound("rho rel. max, 300 steps", rel_err(r_g, r_o), bound)
    parity_bound("j / max rho, 300 steps", np.max(np.abs(j_g - j_o)) / np.max(np.abs(r_o)), bound)


def test_fp64_nid_force_and_tau(gpu_lib, parity_bound):
    # "nid" force (Eq. forceMuId), and the "log" force at tau = 0.8, in the one-phase
    # region of the config-2 mixture (no amplification of rounding differences)
    p = lbinputs.base_params("c2")
    kT = 1.1 * lbinputs.one_fluid_critical_kT(p["a"], p["b"], p["x"])
    rho = lbinputs.fields("c2", nx=40, ny=33)
    sim, orc = make_pair(p, force="nid", nx=40, ny=33, tau=0.8, kT=kT)
    r_g, _, r_o, _ = run_both(sim, orc, rho, 500)
    parity_bound("nid: rho rel. max, 500 steps", rel_err(r_g, r_o), 1e-12)
    sim, orc = make_pair(p, nx=40, ny=33, tau=0.8, kT=kT)
    r_g, _, r_o, _ = run_both(sim, orc, rho, 500)
    parity_bound("tau 0.8: rho rel. max, 500 steps", rel_err(r_g, r_o), 1e-12)


def test_fp64_initial_momentum(gpu_lib, parity_bound):
    p = lbinputs.base_params("c2")
    sim, orc = make_pair(p, nx=33, ny=40)
    rho = lbinputs.fields("c2", nx=33, ny=40)
    mom = np.random.default_rng(5).normal(0, 1e-3, (2, 2, 40, 33))
    r_g, j_g, r_o, j_o = run_both(sim, orc, rho, 200, mom=mom)
    parity_bound("rho rel. max, 200 steps", rel_err(r_g, r_o), 1e-12)
    parity_bound("j max abs, 200 steps", np.max(np.abs(j_g - j_o)), 1e-12)


def test_tile_shapes_give_identical_results(gpu_lib):
    # halo or synchronisation errors would make the result depend on the tiling
    p = lbinputs.base_params("c2")
    rho = lbinputs.fields("c2", nx=100, ny=70)
    outs = []
    for tile in [(32, 8), (64, 4), (32, 16)]:
        sim, _ = make_pair(p, tile=tile, nx=100, ny=70)
        sim.init(rho)
        sim.step(100)
        outs.append(sim.moments()[0])
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    p1 = lbinputs.base_params("c1")
    rho1 = lbinputs.fields("c1")
    o1 = []
    for tile in [(128, 1), (256, 1)]:
        sim, _ = make_pair(p1, tile=tile)
        sim.init(rho1)
        sim.step(100)
        o1.append(sim.moments()[0])
    assert np.array_equal(o1[0], o1[1])


def test_fp64_full_size_config2_sampled_one_step(gpu_lib, parity_bound):
    # 1024 x 1024, the benchmark's launch configuration: one step on the GPU, and the
    # oracle's step on 9 x 9 periodic windows around sampled nodes (the step's
    # dependency radius is 3, so the window centre is exact).
    p = lbinputs.base_params("c2")
    sim, _ = make_pair(p)
    rho = lbinputs.fields("c2")
    sim.init(rho)
    sim.step(1)
    r_g, j_g = sim.moments()
    r = np.random.default_rng(77)
    kw = lbinputs.lib_kwargs(p)
    win = oracle.Lattice("D2Q9", 9, 9, 2, kw["tau"], kw["kT"], kw["gamma_mu"], kw["a"], kw["kappa"],
                         kw["lam"], kw["b"])
    pts = [(0, 0), (1023, 1023), (512, 0), (0, 777)] + [tuple(r.integers(0, 1024, 2)) for _ in range(40)]
    worst = 0.0
    for (y, x) in pts:
        ys = (np.arange(-4, 5) + y) % 1024
        xs = (np.arange(-4, 5) + x) % 1024
        sub = rho[:, ys][:, :, xs]
        ro, jo = win.moments(win.run(win.equilibrium(sub), 1))
        worst = max(worst, np.max(np.abs(r_g[:, y, x] - ro[:, 4, 4])), np.max(np.abs(j_g[:, :, y, x] - jo[:, :, 4, 4])))
    parity_bound("first step, rho and j", worst, 1e-13)


@pytest.mark.parametrize("config,precision,bar", [("c2", "fp32_dfmu", 2e-6), ("c4", "fp32_dfmu", 2e-6)])
def test_fp32_full_size_sampled_one_step(gpu_lib, parity_bound, config, precision, bar):
    # the benchmark's FP32 launch configurations at full size (1024^2 two components,
    # 2048^2 four components, 32x8 tiles in lane pairs): one GPU step against the FP64
    # oracle's step on 9 x 9 periodic windows around sampled nodes.  The GPU starts from
    # FP32-stored deviations and steps in FP32, so the bar is FP32 rounding, not 1e-13.
    p = lbinputs.base_params(config)
    sim, _ = make_pair(p, precision=precision)
    assert sim.kernel == ("tiles", (32, 8))
    rho = lbinputs.fields(config)
    N, ny, nx = rho.shape
    sim.init(rho)
    sim.step(1)
    r_g, j_g = sim.moments()
    r = np.random.default_rng(78)
    kw = lbinputs.lib_kwargs(p)
    win = oracle.Lattice("D2Q9", 9, 9, N, kw["tau"], kw["kT"], kw["gamma_mu"], kw["a"], kw["kappa"],
                         kw["lam"], kw["b"])
    pts = [(0, 0), (ny - 1, nx - 1), (ny // 2, 0), (0, nx - 7)]
    pts += [(int(r.integers(0, ny)), int(r.integers(0, nx))) for _ in range(30)]
    worst = 0.0
    for (y, x) in pts:
        ys = (np.arange(-4, 5) + y) % ny
        xs = (np.arange(-4, 5) + x) % nx
        ro, jo = win.moments(win.run(win.equilibrium(rho[:, ys][:, :, xs]), 1))
        worst = max(worst, np.max(np.abs(r_g[:, y, x] - ro[:, 4, 4])), np.max(np.abs(j_g[:, :, y, x] - jo[:, :, 4, 4])))
    parity_bound("first step, rho and j", worst, bar)


D2Q9_W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def test_fp32_full_size_chained_steps_restart_against_oracle(gpu_lib, parity_bound):
    # the headline's launch configuration: 1024^2, two components, FP32 deviation storage
    # with double-float mu, consecutive steps of one lb_step call (chained launches: the
    # first CTA rows wait on neighbouring tiles' flags, the others on the whole previous
    # grid).  At steps 0 and 300 of the GPU's own chained trajectory, two chained GPU steps
    # against two FP64 oracle steps restarted from the GPU's state (f = g + w_i rho_ref) at
    # sampled nodes.  The GPU steps in FP32: the bar is FP32 rounding.
    p = lbinputs.base_params("c2")
    rho = lbinputs.fields("c2")
    rref = np.array([float(np.float32(rho[c].mean())) for c in range(2)])
    sim, _ = make_pair(p, precision="fp32_dfmu", rho_ref=rref)
    assert sim.kernel == ("tiles", (32, 8)) and sim.chain_rows > 0
    kw = lbinputs.lib_kwargs(p)
    win9 = oracle.Lattice("D2Q9", 9, 9, 2, kw["tau"], kw["kT"], kw["gamma_mu"], kw["a"], kw["kappa"],
                          kw["lam"], kw["b"])
    fshape = (2, 9, 1024, 1024)
    r = np.random.default_rng(81)
    sim.init(rho)
    done = 0
    for t in (0, 300):
        sim.step(t - done)
        g = gpu_populations(sim, fshape, dtype=np.float32)
        f_t = g.astype(np.float64) + D2Q9_W[None, :, None, None] * rref[:, None, None, None]
        sim.step(2)
        done = t + 2
        r_g, j_g = sim.moments()
        pts = [(0, 0), (1023, 1023), (512, 0), (0, 777), (7, 31), (8, 32), (215, 500)]
        pts += [tuple(int(v) for v in r.integers(0, 1024, 2)) for _ in range(25)]
        worst = 0.0
        for (y, x) in pts:
            ro, jo = oracle_two_steps_at(win9, f_t, y, x)
            worst = max(worst, float(np.max(np.abs(r_g[:, y, x] - ro))), float(np.max(np.abs(j_g[:, :, y, x] - jo))))
        parity_bound(f"two chained steps at {t}, rho and j", worst, 1e-6)


def test_free_energy_diagnostic_matches_oracle(gpu_lib):
    p = lbinputs.base_params("c2")
    sim, orc = make_pair(p, nx=64, ny=50)
    rho = lbinputs.fields("c2", nx=64, ny=50)
    sim.init(rho)
    sim.step(50)
    r_g, j_g = sim.moments()
    F, mass, mom = sim.free_energy()
    F_o, mass_o = orc.free_energy(r_g)
    assert abs(F - F_o) < 1e-12 * abs(F_o)
    assert np.max(np.abs(mass - mass_o)) < 1e-12 * np.max(mass_o)
    assert np.max(np.abs(mom - j_g.sum(axis=(0, 2, 3)))) < 1e-12
    # bitwise reproducible reduction order
    assert sim.free_energy()[0] == F


def test_save_load_resume_is_bitwise(gpu_lib):
    p = lbinputs.base_params("c2")
    rho = lbinputs.fields("c2", nx=48, ny=40)
    sim, _ = make_pair(p, nx=48, ny=40)
    sim.init(rho)
    sim.step(200)
    want = sim.moments()[0]
    sim2, _ = make_pair(p, nx=48, ny=40)
    sim2.init(rho)
    sim2.step(100)
    buf = sim2.save_state()
    sim3, _ = make_pair(p, nx=48, ny=40)
    sim3.init(rho)
    sim3.load_state(buf)
    assert sim3.steps == 100
    sim3.step(100)
    assert np.array_equal(sim3.moments()[0], want)


def test_domain_errors_poison_and_recover(gpu_lib):
    from paper_1805_07251_gb300 import capi

    p = lbinputs.base_params("c2")
    sim, _ = make_pair(p, nx=32, ny=32)
    bad = lbinputs.fields("c2", nx=32, ny=32)
    bad[0, 3, 4] = -0.1
    with pytest.raises(capi.LBError) as e:
        sim.init(bad)
    assert e.value.status == capi.LB_E_DOMAIN
    # a state that leaves the domain during the steps: gamma_mu far above the stable range
    sim2, _ = make_pair(p, nx=32, ny=32, gamma_mu=50.0)
    sim2.init(lbinputs.fields("c2", nx=32, ny=32))
    sim2.step(200)
    with pytest.raises(capi.LBError) as e:
        sim2.moments()
    assert e.value.status == capi.LB_E_DOMAIN
    with pytest.raises(capi.LBError) as e:
        sim2.step(1)
    assert e.value.status == capi.LB_E_STATE
    sim2.init(lbinputs.fields("c2", nx=32, ny=32))   # setting the fields clears the poison
    sim2.step(1)
    sim2.moments()


def test_device_pointer_entry_points(gpu_lib):
    import torch

    p = lbinputs.base_params("c2")
    sim, orc = make_pair(p, nx=40, ny=36)
    rho = lbinputs.fields("c2", nx=40, ny=36)
    rho_t = torch.from_numpy(rho).cuda()
    sim.init_dev(rho_t.data_ptr())
    sim.step(100)
    out_r = torch.empty_like(rho_t)
    out_j = torch.empty((2, 2, 36, 40), dtype=torch.float64, device="cuda")
    sim.moments_dev(out_r.data_ptr(), out_j.data_ptr())
    torch.cuda.synchronize()
    r_o, j_o = orc.moments(orc.run(orc.equilibrium(rho), 100))
    assert rel_err(out_r.cpu().numpy(), r_o) < 1e-12
    assert np.max(np.abs(out_j.cpu().numpy() - j_o)) < 1e-12


# ------------------------------------------------------------------ FP32 storage

W_D2Q9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W_D1Q3 = np.array([2 / 3, 1 / 6, 1 / 6])


def gpu_populations_f32(sim, fshape, rho0):
    """Stored FP32 deviations -> populations f = g + w_i rho_ref (rho_ref = float(mean rho0))."""
    g = gpu_populations(sim, fshape, dtype=np.float32).astype(np.float64)
    N, Q = fshape[0], fshape[1]
    w = W_D1Q3 if Q == 3 else W_D2Q9
    ref = np.float32(rho0.reshape(N, -1).mean(axis=1)).astype(np.float64)
    return g + w.reshape(1, Q, 1, 1) * ref.reshape(N, 1, 1, 1)


def test_chemical_potential_logarithms(gpu_lib):
    # the table-driven FP64 log and the double-float log against CUDA's log
    from paper_1805_07251_gb300 import capi

    r = np.random.default_rng(3)
    x = np.concatenate([np.exp(r.uniform(-12, 6, 20000)), 1 + r.uniform(-1e-3, 1e-3, 5000),
                        r.uniform(0.05, 4.0, 20000), [1.0, 2.0, 0.5, 1 - 2 ** -52, 1 + 2 ** -52]])
    tbl, dfl, ref = capi.lb_selftest_log(0, x)
    scale = np.maximum(1.0, np.abs(ref))
    assert np.max(np.abs(tbl - ref) / scale) < 4 * 2.0 ** -53
    assert np.max(np.abs(dfl - ref) / scale) < 2.0 ** -43


def test_double_float_reciprocal(gpu_lib):
    # 1/eta of the double-float chemical potential (MUFU seed, one Newton step, exact FMA
    # residual, second-order correction) against the FP64 quotient: relative error at the
    # df precision, over eta's range (0, 1] and beyond
    from paper_1805_07251_gb300 import capi

    r = np.random.default_rng(5)
    x = np.concatenate([r.uniform(1e-3, 1.0, 40000), np.exp(r.uniform(-20, 20, 20000)),
                        [1.0, 0.5, 2.0, 1 - 2.0 ** -24, 1 + 2.0 ** -23, 0.75, 1.0 / 3.0]])
    inv = capi.lb_selftest_recip(0, x)
    assert np.max(np.abs(inv * x - 1.0)) < 2.0 ** -44


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32_dfmu", "fp32"])
def test_fp32_one_phase_within_1e5_of_fp64_oracle(gpu_lib, parity_bound, precision):
    p = lbinputs.base_params("c2")
    kT = 1.1 * lbinputs.one_fluid_critical_kT(p["a"], p["b"], p["x"])
    sim, orc = make_pair(p, precision=precision, nx=70, ny=45, kT=kT)
    rho = lbinputs.fields("c2", nx=70, ny=45)
    r_g, _, r_o, _ = run_both(sim, orc, rho, 1000)
    parity_bound("rho max abs, 1000 steps", np.max(np.abs(r_g - r_o)), 1e-5)
    m0 = rho.reshape(2, -1).sum(axis=1)
    _, mass, _ = sim.free_energy()
    parity_bound("mass drift", np.max(np.abs(mass - m0) / m0), 1e-6)


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32_dfmu", "fp32"])
def test_fp32_spinodal_step_and_trajectory(gpu_lib, parity_bound, precision):
    # one step from the GPU's own state agrees with the FP64 oracle to FP32 rounding;
    # the 1000-step trajectory is bounded by 1e-5 or by 10x the spread that FP32-size
    # noise produces on the oracle's own trajectory (spinodal growth amplifies it)
    p = lbinputs.base_params("c2")
    sim, orc = make_pair(p, precision=precision, nx=70, ny=45)
    rho = lbinputs.fields("c2", nx=70, ny=45)
    fshape = orc.fshape()
    sim.init(rho)
    for t in range(3):
        f_t = gpu_populations_f32(sim, fshape, rho)
        sim.step(1)
        f_next = gpu_populations_f32(sim, fshape, rho)
        parity_bound(f"one step at {401 * t}", np.max(np.abs(f_next - orc.run(f_t, 1))), 2e-6)
        sim.step(400)
    sim.init(rho)
    sim.step(1000)
    r_g, _ = sim.moments()
    r_o, _ = orc.moments(orc.run(orc.equilibrium(rho), 1000))
    spread = fp32_noise_spread(orc, rho, 1000)
    parity_bound("oracle FP32-noise spread", spread, 1.0)
    parity_bound("rho max abs, 1000 steps", np.max(np.abs(r_g - r_o)), max(1e-5, 10.0 * spread))


def fp32_noise_spread(orc, rho, steps, seed=0):
    """Spread of oracle trajectories when every population is perturbed at every step by
    relative noise of 2^-22 (a few FP32 ulps: the storage rounding plus the FP32
    arithmetic of the step): the deviation FP32 alone produces on this trajectory."""
    r0, _ = orc.moments(orc.run(orc.equilibrium(rho), steps))
    rng = np.random.default_rng(seed)
    f = orc.equilibrium(rho)
    for _ in range(steps):
        f = orc.run(f * (1 + 2.0 ** -22 * rng.uniform(-1, 1, f.shape)), 1)
    r1, _ = orc.moments(f)
    return float(np.max(np.abs(r1 - r0)))


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32_dfmu", "fp32"])
def test_fp32_d1q3_config1(gpu_lib, parity_bound, precision):
    # config 1 (slab with noise) amplifies rounding: one step from the GPU state agrees
    # with the oracle to FP32 rounding; the trajectory bar is 1e-5 or 10x the spread that
    # FP32-size noise produces on the oracle's own trajectory, whichever is larger
    p = lbinputs.base_params("c1")
    sim, orc = make_pair(p, precision=precision)
    rho = lbinputs.fields("c1")
    sim.init(rho)
    sim.step(500)
    f_t = gpu_populations_f32(sim, orc.fshape(), rho)
    sim.step(1)
    parity_bound("one step at 500", np.max(np.abs(gpu_populations_f32(sim, orc.fshape(), rho) - orc.run(f_t, 1))),
                 2e-6)
    r_g, _, r_o, _ = run_both(sim, orc, rho, 1000)
    spread = fp32_noise_spread(orc, rho, 1000)
    parity_bound("oracle FP32-noise spread", spread, 1.0)
    parity_bound("rho max abs, 1000 steps", np.max(np.abs(r_g - r_o)), max(1e-5, 10.0 * spread))


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32_dfmu", "fp32"])
def test_fp32_equilibrium_coexistence_within_1e4(gpu_lib, parity_bound, precision):
    # config 1 (D1Q3 slab) run to equilibrium in FP32 storage and in the FP64 oracle:
    # coexisting bulk densities (averaged over the two sublattices) agree to 1e-4
    p = lbinputs.base_params("c1")
    sim, orc = make_pair(p, precision=precision)
    rho = lbinputs.fields("c1")
    r_g, _, r_o, _ = run_both(sim, orc, rho, 20000)
    for x in (0, 128):
        parity_bound(f"bulk rho at x = {x}, 20k steps",
                     np.max(np.abs(r_g[:, 0, x:x + 2].mean(axis=1) - r_o[:, 0, x:x + 2].mean(axis=1))), 1e-4)


def test_fp32_tile_shapes_identical(gpu_lib):
    p = lbinputs.base_params("c2")
    rho = lbinputs.fields("c2", nx=130, ny=70)
    for precision in ("fp32_mixed", "fp32_dfmu"):
        outs = []
        for tile in [(32, 8), (64, 4), (32, 16), (64, 8)]:
            sim, _ = make_pair(p, precision=precision, tile=tile, nx=130, ny=70)
            sim.init(rho)
            sim.step(50)
            outs.append(sim.moments()[0])
        for o in outs[1:]:
            assert np.array_equal(outs[0], o)


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed", "fp32_dfmu"])
def test_four_component_mixture(gpu_lib, parity_bound, precision):
    # config-4 mixture (random symmetric a_ij, four components) on a small ragged lattice:
    # one step from the GPU state against the oracle, and the 500-step trajectory bounded
    # by 1e-12 (FP64) / 1e-5 (FP32) or the conditioning of the trajectory
    p = lbinputs.base_params("c4")
    nx, ny = 40, 30
    sim, orc = make_pair(p, precision=precision, nx=nx, ny=ny)
    rho = lbinputs.fields("c4", nx=nx, ny=ny)
    fshape = orc.fshape()
    sim.init(rho)
    sim.step(100)
    if precision == "fp64":
        f_t = gpu_populations(sim, fshape)
        sim.step(1)
        parity_bound("one step at 100", np.max(np.abs(gpu_populations(sim, fshape) - orc.run(f_t, 1))), 1e-14)
    else:
        f_t = gpu_populations_f32(sim, fshape, rho)
        sim.step(1)
        parity_bound("one step at 100", np.max(np.abs(gpu_populations_f32(sim, fshape, rho) - orc.run(f_t, 1))),
                     2e-6)
    r_g, _, r_o, _ = run_both(sim, orc, rho, 500)
    if precision == "fp64":
        amp = ulp_amplification(orc, rho, 500)
        parity_bound("oracle 1-ulp amplification", amp, 1.0)
        parity_bound("rho rel. max, 500 steps", rel_err(r_g, r_o), max(1e-12, 100.0 * amp))
    else:
        spread = fp32_noise_spread(orc, rho, 500)
        parity_bound("oracle FP32-noise spread", spread, 1.0)
        parity_bound("rho max abs, 500 steps", np.max(np.abs(r_g - r_o)), max(1e-5, 10.0 * spread))
    m0 = rho.reshape(4, -1).sum(axis=1)
    _, mass, _ = sim.free_energy()
    parity_bound("mass drift", np.max(np.abs(mass - m0) / m0), 1e-13 if precision == "fp64" else 1e-6)


# ------------------------------------------------------------------ kernel organisations

def strip_case(p, N, nx, ny, precision, force="log", segments=0, steps=40):
    from paper_1805_07251_gb300 import Simulation

    kw = lbinputs.lib_kwargs(p, nx=nx, ny=ny)
    if N != kw["ncomp"]:
        # the first N components of the mixture, above their critical temperature
        kw.update(ncomp=N, a=kw["a"][:N, :N], kappa=kw["kappa"][:N, :N], lam=kw["lam"][:N, :N], b=kw["b"][:N],
                  kT=1.1 * lbinputs.one_fluid_critical_kT(kw["a"][:N, :N], kw["b"][:N], np.full(N, 1.0 / N)))
    rho = lbinputs.fields(p["name"], nx=nx, ny=ny)[:N]
    outs = []
    for kernel in ("tiles", "strips"):
        sim = Simulation(precision=precision, force=force, kernel=kernel, segments=segments, **kw)
        assert sim.kernel[0] == kernel
        sim.init(rho)
        sim.step(steps)
        outs.append(sim.moments())
        sim.close()
    return outs


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32_dfmu", "fp32"])
@pytest.mark.parametrize("N,nx,ny", [(1, 64, 48), (2, 32, 8), (2, 96, 40), (3, 64, 36), (4, 32, 4), (4, 96, 20)])
def test_strip_kernel_is_bitwise_equal_to_tiles(gpu_lib, precision, N, nx, ny):
    # the streaming-strip organisation computes every node with the same arithmetic in
    # the same order as the tile kernel (which the rest of this file checks against the
    # oracle): single strips, single row blocks, wrap-around halos in x and y
    p = lbinputs.base_params("c4" if N > 2 else "c2")
    (r_t, j_t), (r_s, j_s) = strip_case(p, N, nx, ny, precision)
    assert np.array_equal(r_t, r_s) and np.array_equal(j_t, j_s)


@pytest.mark.parametrize("segments", [1, 2, 5, 64])
def test_strip_kernel_segments_and_nid_force(gpu_lib, segments):
    # any split of the strips into row segments (more segments than row blocks is
    # clamped), and the "nid" force
    p = lbinputs.base_params("c2")
    for force in ("log", "nid"):
        (r_t, j_t), (r_s, j_s) = strip_case(p, 2, 64, 64, "fp32_dfmu", force=force, segments=segments)
        assert np.array_equal(r_t, r_s) and np.array_equal(j_t, j_s)


def test_strip_kernel_full_size_matches_tiles(gpu_lib):
    # workload c2 at 1024^2 (the benchmark's launch configuration), 20 steps
    p = lbinputs.base_params("c2")
    (r_t, j_t), (r_s, j_s) = strip_case(p, 2, p["nx"], p["ny"], "fp32_dfmu", steps=20)
    assert np.array_equal(r_t, r_s) and np.array_equal(j_t, j_s)


def ws_case(p, nx, ny, precision, force="log", steps=40, **extra):
    from paper_1805_07251_gb300 import Simulation

    kw = lbinputs.lib_kwargs(p, nx=nx, ny=ny)
    kw.update(extra)
    rho = lbinputs.fields(p["name"], nx=nx, ny=ny)
    outs = []
    for kernel in ("tiles", "ws"):
        sim = Simulation(precision=precision, force=force, kernel=kernel, **kw)
        assert sim.kernel[0] == kernel
        sim.init(rho)
        sim.step(steps)
        outs.append(sim.moments())
        sim.close()
    return outs


@pytest.mark.parametrize("precision", ["fp32_dfmu", "fp32"])
@pytest.mark.parametrize("nx,ny", [(32, 8), (70, 45), (100, 70), (33, 9), (256, 200)])
def test_ws_kernel_is_bitwise_equal_to_tiles(gpu_lib, precision, nx, ny):
    # the warp-specialised persistent tiles compute every node with the arithmetic of the
    # tile kernel: single tiles, ragged edges, more tiles than resident CTAs
    p = lbinputs.base_params("c2")
    (r_t, j_t), (r_w, j_w) = ws_case(p, nx, ny, precision)
    assert np.array_equal(r_t, r_w) and np.array_equal(j_t, j_w)


def test_ws_kernel_nid_force_and_moment_collision(gpu_lib):
    p = lbinputs.base_params("c2")
    (r_t, j_t), (r_w, j_w) = ws_case(p, 96, 40, "fp32_dfmu", force="nid")
    assert np.array_equal(r_t, r_w) and np.array_equal(j_t, j_w)
    (r_t, j_t), (r_w, j_w) = ws_case(p, 96, 40, "fp32_dfmu", tau_shear=0.7, tau_ghost=0.9)
    assert np.array_equal(r_t, r_w) and np.array_equal(j_t, j_w)


def test_ws_kernel_full_size_matches_tiles(gpu_lib):
    # workload c2 at 1024^2 (the benchmark's lattice), 20 steps
    p = lbinputs.base_params("c2")
    (r_t, j_t), (r_w, j_w) = ws_case(p, p["nx"], p["ny"], "fp32_dfmu", steps=20)
    assert np.array_equal(r_t, r_w) and np.array_equal(j_t, j_w)


@pytest.mark.parametrize("precision", ["fp64", "fp32_dfmu"])
@pytest.mark.parametrize("lattice,nx,ny", [("D2Q9", 2, 2), ("D2Q9", 3, 2), ("D2Q9", 2, 5), ("D2Q9", 5, 3),
                                           ("D2Q9", 7, 9), ("D2Q9", 33, 3), ("D2Q9", 31, 17),
                                           ("D1Q3", 2, 1), ("D1Q3", 3, 1), ("D1Q3", 5, 1), ("D1Q3", 127, 1)])
def test_degenerate_lattices_match_oracle(gpu_lib, parity_bound, precision, lattice, nx, ny):
    # lattices narrower than a tile and its ring (the periodic wrap reaches a node more than
    # once, down to 2 nodes), one tile with a ragged edge, and lb_step(0): the one-phase
    # config-2 mixture, so 50 steps agree to the FP64 bar, or to FP32 rounding
    p = lbinputs.base_params("c2")
    kT = 1.1 * lbinputs.one_fluid_critical_kT(p["a"], p["b"], p["x"])
    sim, orc = make_pair(p, precision=precision, nx=nx, ny=ny, kT=kT, lattice=lattice)
    rho = lbinputs.uniform_noise_fields(2, ny, nx, 1.2 * p["x"], 1e-2, 3000 + nx * 100 + ny)
    sim.init(rho)
    r0, j0 = sim.moments()
    sim.step(0)
    r1, j1 = sim.moments()
    assert np.array_equal(r0, r1) and np.array_equal(j0, j1)
    sim.step(50)
    r_g, j_g = sim.moments()
    f = orc.run(orc.equilibrium(rho), 50)
    r_o, j_o = orc.moments(f)
    bound = 1e-12 if precision == "fp64" else 1e-5
    parity_bound(f"{lattice} {nx}x{ny}: rho rel. max, 50 steps", rel_err(r_g, r_o), bound)
    parity_bound(f"{lattice} {nx}x{ny}: j / max rho", np.max(np.abs(j_g - j_o)) / np.max(np.abs(r_o)), bound)
    sim.close()
