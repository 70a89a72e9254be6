"""GPU parity of the fused CUDA timestep against the CPU oracle, through the C ABI.

Bars: FP64 densities within 1e-12 relative (max norm) after 1000 steps and mass
conserved to 1e-13; FP32-mixed densities within 1e-5 of the FP64 oracle after
1000 steps.  Inputs are the seeded synthetic fields of ``lbinputs``."""
import numpy as np
import pytest

import lbinputs
import oracle

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

def test_fp64_d2q9_two_components_1000_steps(gpu_lib):
    # config-2 mixture (spinodal decomposition), ragged lattice spanning several tiles
    p = lbinputs.base_params("c2")
    sim, orc = make_pair(p, nx=70, ny=45)
    rho = lbinputs.fields("c2", nx=70, ny=45)
    r_g, j_g, r_o, j_o = run_both(sim, orc, rho, 1000)
    assert rel_err(r_g, r_o) < 1e-12
    assert np.max(np.abs(j_g - j_o)) < 1e-12 * np.max(np.abs(r_o))
    m0 = rho.reshape(2, -1).sum(axis=1)
    F, mass, _ = sim.free_energy()
    assert np.max(np.abs(mass - m0) / m0) < 1e-13


def test_fp64_d1q3_config1_full_size(gpu_lib):
    p = lbinputs.base_params("c1")
    sim, orc = make_pair(p)
    rho = lbinputs.fields("c1")
    r_g, j_g, r_o, j_o = run_both(sim, orc, rho, 1000)
    assert rel_err(r_g, r_o) < 1e-12
    m0 = rho.reshape(2, -1).sum(axis=1)
    _, mass, _ = sim.free_energy()
    assert np.max(np.abs(mass - m0) / m0) < 1e-13


@pytest.mark.parametrize("N", [1, 3, 4])
@pytest.mark.parametrize("lattice", ["D1Q3", "D2Q9"])
def test_fp64_component_counts(gpu_lib, N, lattice):
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
    assert rel_err(r_g, r_o) < 1e-12
    assert np.max(np.abs(j_g - j_o)) < 1e-12 * np.max(np.abs(r_o))


def test_fp64_nid_force_and_tau(gpu_lib):
    # "nid" force (Eq. forceMuId) in the one-phase region (it is unstable in the
    # spinodal case), and the "log" force at tau = 0.8
    p = lbinputs.base_params("c2")
    kT = 1.1 * lbinputs.one_fluid_critical_kT(p["a"], p["b"], p["x"])
    rho = lbinputs.fields("c2", nx=40, ny=33)
    sim, orc = make_pair(p, force="nid", nx=40, ny=33, tau=0.8, kT=kT)
    r_g, _, r_o, _ = run_both(sim, orc, rho, 500)
    assert rel_err(r_g, r_o) < 1e-12
    sim, orc = make_pair(p, nx=40, ny=33, tau=0.8)
    r_g, _, r_o, _ = run_both(sim, orc, rho, 500)
    assert rel_err(r_g, r_o) < 1e-12


def test_fp64_initial_momentum(gpu_lib):
    p = lbinputs.base_params("c2")
    sim, orc = make_pair(p, nx=33, ny=40)
    rho = lbinputs.fields("c2", nx=33, ny=40)
    mom = np.random.default_rng(5).normal(0, 1e-3, (2, 2, 40, 33))
    r_g, j_g, r_o, j_o = run_both(sim, orc, rho, 200, mom=mom)
    assert rel_err(r_g, r_o) < 1e-12
    assert np.max(np.abs(j_g - j_o)) < 1e-12


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


def test_fp64_full_size_config2_sampled_one_step(gpu_lib):
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
    for (y, x) in pts:
        ys = (np.arange(-4, 5) + y) % 1024
        xs = (np.arange(-4, 5) + x) % 1024
        sub = rho[:, ys][:, :, xs]
        ro, jo = win.moments(win.run(win.equilibrium(sub), 1))
        assert np.max(np.abs(r_g[:, y, x] - ro[:, 4, 4])) < 1e-13
        assert np.max(np.abs(j_g[:, :, y, x] - jo[:, :, 4, 4])) < 1e-13


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


# ------------------------------------------------------------------ FP32-mixed

def test_fp32_mixed_d2q9_within_1e5_of_fp64_oracle(gpu_lib):
    p = lbinputs.base_params("c2")
    sim, orc = make_pair(p, precision="fp32_mixed", nx=70, ny=45)
    rho = lbinputs.fields("c2", nx=70, ny=45)
    r_g, _, r_o, _ = run_both(sim, orc, rho, 1000)
    assert np.max(np.abs(r_g - r_o)) < 1e-5
    m0 = rho.reshape(2, -1).sum(axis=1)
    _, mass, _ = sim.free_energy()
    assert np.max(np.abs(mass - m0) / m0) < 1e-6


def test_fp32_mixed_d1q3_config1(gpu_lib):
    p = lbinputs.base_params("c1")
    sim, orc = make_pair(p, precision="fp32_mixed")
    rho = lbinputs.fields("c1")
    r_g, _, r_o, _ = run_both(sim, orc, rho, 1000)
    assert np.max(np.abs(r_g - r_o)) < 1e-5
