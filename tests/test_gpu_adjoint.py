"""GPU tests of the adjoint rollout: the hand-written transpose of the fused FP64 step
against central finite differences (h = 1e-4) of the GPU forward and of the CPU oracle,
checkpoint invariance, and the torch.autograd.Function wrapper; the FP32 rollouts (FP32
storage, FP64 or double-float mu in the forward; FP32 adjoint with FP64 mu) against the
one-step dot-product identity and against the FP64 gradients."""
import numpy as np
import pytest

import lbinputs
import oracle

pytestmark = pytest.mark.gpu


def spec_small(lattice, steps):
    p = lbinputs.base_params("c5")
    nx, ny = (64, 1) if lattice == "D1Q3" else (24, 20)
    return dict(lattice=lattice, nx=nx, ny=ny, ncomp=2, tau=1.0, kT=p["kT"], gamma_mu=p["gamma_mu"],
                a=p["a"], b=p["b"], kappa=0.1, lam=p["lam"], steps=steps)


def fields(spec):
    return lbinputs.fields("c5", nx=spec["nx"], ny=spec["ny"])


def target(spec):
    r = np.random.default_rng(99)
    return fields(spec) + r.normal(0, 1e-2, (2, spec["ny"], spec["nx"]))


def gpu_loss(spec, a12, kappa, b, rho0, tgt):
    from paper_1805_07251_gb300 import Simulation

    a = np.array(spec["a"], float).copy()
    a[0, 1] = a[1, 0] = a12
    sim = Simulation(lattice=spec["lattice"], nx=spec["nx"], ny=spec["ny"], ncomp=2, tau=spec["tau"],
                     kT=spec["kT"], gamma_mu=spec["gamma_mu"], a=a, kappa=np.full((2, 2), kappa), lam=spec["lam"],
                     b=b, precision="fp64")
    sim.init(rho0)
    sim.step(spec["steps"])
    r, _ = sim.moments()
    sim.close()
    return float(np.sum((r - tgt) ** 2))


def oracle_loss(spec, a12, kappa, b, rho0, tgt):
    a = np.array(spec["a"], float).copy()
    a[0, 1] = a[1, 0] = a12
    L = oracle.Lattice(spec["lattice"], spec["nx"], spec["ny"], 2, spec["tau"], spec["kT"], spec["gamma_mu"], a,
                       np.full((2, 2), kappa), spec["lam"], b)
    r, _ = L.moments(L.run(L.equilibrium(rho0), spec["steps"]))
    return float(np.sum((r - tgt) ** 2))


def adjoint_grads(spec, rho0, tgt, ckpt, precision="fp64"):
    from paper_1805_07251_gb300 import Simulation, capi

    sim = Simulation(lattice=spec["lattice"], nx=spec["nx"], ny=spec["ny"], ncomp=2, tau=spec["tau"],
                     kT=spec["kT"], gamma_mu=spec["gamma_mu"], a=spec["a"], kappa=np.full((2, 2), spec["kappa"]),
                     lam=spec["lam"], b=spec["b"], precision=precision)
    sim.init(rho0)
    capi.lb_rollout_forward(sim.ctx, spec["steps"], ckpt)
    r, _ = sim.moments()
    rb0, g = capi.lb_rollout_backward(sim.ctx, 2.0 * (r - tgt), 2)
    sim.close()
    return rb0, g[0:4].reshape(2, 2), g[4:8].reshape(2, 2), g[8:10]


def central(fun, x0, h):
    """Central difference with step h, Richardson-extrapolated with h/2 so that its own
    truncation error (O(h^2) through tens of nonlinear steps) stays below the 1e-6 bar."""
    d1 = (fun(x0 + h) - fun(x0 - h)) / (2 * h)
    d2 = (fun(x0 + h / 2) - fun(x0 - h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("lattice", ["D1Q3", "D2Q9"])
def test_adjoint_matches_finite_differences(gpu_lib, lattice):
    spec = spec_small(lattice, 60)
    rho0, tgt = fields(spec), target(spec)
    a12, kap, b = spec["a"][0, 1], spec["kappa"], np.array(spec["b"], float)
    rb0, ga, gk, gb = adjoint_grads(spec, rho0, tgt, ckpt=25)
    h = 1e-4
    fd_a = central(lambda v: gpu_loss(spec, v, kap, b, rho0, tgt), a12, h)
    assert abs((ga[0, 1] + ga[1, 0]) - fd_a) <= 1e-6 * abs(fd_a)
    fd_k = central(lambda v: gpu_loss(spec, a12, v, b, rho0, tgt), kap, h)
    assert abs(gk.sum() - fd_k) <= 1e-6 * abs(fd_k)
    for c in range(2):
        e = np.zeros(2); e[c] = 1.0
        fd_b = central(lambda v: gpu_loss(spec, a12, kap, b + v * e, rho0, tgt), 0.0, h)
        assert abs(gb[c] - fd_b) <= 1e-6 * abs(fd_b)
    v = 1e-2 * np.random.default_rng(5).normal(0, 1, rho0.shape)
    fd_r = central(lambda t: gpu_loss(spec, a12, kap, b, rho0 + t * v, tgt), 0.0, h)
    assert abs(np.sum(rb0 * v) - fd_r) <= 1e-6 * abs(fd_r)


@pytest.mark.parametrize("lattice", ["D1Q3", "D2Q9"])
def test_adjoint_matches_oracle_finite_differences(gpu_lib, lattice):
    spec = spec_small(lattice, 40)
    rho0, tgt = fields(spec), target(spec)
    a12, kap, b = spec["a"][0, 1], spec["kappa"], np.array(spec["b"], float)
    rb0, ga, gk, _ = adjoint_grads(spec, rho0, tgt, ckpt=40)
    h = 1e-4
    fd_a = central(lambda v: oracle_loss(spec, v, kap, b, rho0, tgt), a12, h)
    assert abs((ga[0, 1] + ga[1, 0]) - fd_a) <= 1e-6 * abs(fd_a)
    fd_k = central(lambda v: oracle_loss(spec, a12, v, b, rho0, tgt), kap, h)
    assert abs(gk.sum() - fd_k) <= 1e-6 * abs(fd_k)
    v = 1e-2 * np.random.default_rng(6).normal(0, 1, rho0.shape)
    fd_r = central(lambda t: oracle_loss(spec, a12, kap, b, rho0 + t * v, tgt), 0.0, h)
    assert abs(np.sum(rb0 * v) - fd_r) <= 1e-6 * abs(fd_r)


def final_density(spec, a12, rho0, precision="fp64"):
    from paper_1805_07251_gb300 import Simulation

    a = np.array(spec["a"], float).copy()
    a[0, 1] = a[1, 0] = a12
    sim = Simulation(lattice=spec["lattice"], nx=spec["nx"], ny=spec["ny"], ncomp=2, tau=spec["tau"],
                     kT=spec["kT"], gamma_mu=spec["gamma_mu"], a=a, kappa=np.full((2, 2), spec["kappa"]),
                     lam=spec["lam"], b=spec["b"], precision=precision)
    sim.init(rho0)
    sim.step(spec["steps"])
    r, _ = sim.moments()
    sim.close()
    return r


@pytest.mark.parametrize("lattice", ["D1Q3", "D2Q9"])
def test_one_step_dot_product(gpu_lib, lattice):
    # <J v, w> = <v, J^T w> for one step (J = d rho_1 / d (rho_0, a12)), with J v from a
    # Richardson-extrapolated central difference: over one step its truncation and rounding
    # errors are far below the bar, so this checks the transpose itself
    from paper_1805_07251_gb300 import Simulation, capi

    spec = spec_small(lattice, 1)
    rho0 = fields(spec)
    rng = np.random.default_rng(11)
    v = 1e-2 * rng.normal(0, 1, rho0.shape)
    w = rng.normal(0, 1, rho0.shape)
    sim = Simulation(lattice=spec["lattice"], nx=spec["nx"], ny=spec["ny"], ncomp=2, tau=spec["tau"],
                     kT=spec["kT"], gamma_mu=spec["gamma_mu"], a=spec["a"], kappa=np.full((2, 2), spec["kappa"]),
                     lam=spec["lam"], b=spec["b"], precision="fp64")
    sim.init(rho0)
    capi.lb_rollout_forward(sim.ctx, 1, 1)
    rb0, g = capi.lb_rollout_backward(sim.ctx, w, 2)
    sim.close()
    a12 = spec["a"][0, 1]
    jv = central(lambda t: float(np.sum(final_density(spec, a12, rho0 + t * v) * w)), 0.0, 1e-4)
    assert abs(np.sum(rb0 * v) - jv) <= 1e-8 * abs(jv)
    # a12 moves rho_1 only weakly (d<rho_1, w>/d a12 ~ 1e-3): a wider step keeps the
    # quotient's rounding error (~1e-16 |<rho_1, w>| / h) below the bar
    ja = central(lambda t: float(np.sum(final_density(spec, t, rho0) * w)), a12, 1e-3)
    assert abs((g[1] + g[2]) - ja) <= 1e-8 * abs(ja)


def test_checkpoint_interval_does_not_change_gradients(gpu_lib):
    spec = spec_small("D2Q9", 50)
    rho0, tgt = fields(spec), target(spec)
    r1 = adjoint_grads(spec, rho0, tgt, ckpt=50)
    r2 = adjoint_grads(spec, rho0, tgt, ckpt=7)
    for u, w in zip(r1, r2):
        assert np.array_equal(u, w)


def test_autograd_function(gpu_lib):
    import torch

    from paper_1805_07251_gb300.adjoint import rollout

    spec = spec_small("D2Q9", 30)
    spec["ckpt_every"] = 10
    rho0 = torch.tensor(fields(spec), dtype=torch.float64, requires_grad=True)
    a12 = torch.tensor(spec["a"][0, 1], dtype=torch.float64, requires_grad=True)
    kap = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    b = torch.tensor(np.array(spec["b"], float), requires_grad=True)
    tgt = torch.tensor(target(spec))
    loss = ((rollout(a12, kap, b, rho0, spec) - tgt) ** 2).sum()
    loss.backward()
    rb0, ga, gk, gb = adjoint_grads(spec, fields(spec), target(spec), ckpt=10)
    assert abs(a12.grad.item() - (ga[0, 1] + ga[1, 0])) <= 1e-12 * abs(a12.grad.item())
    assert abs(kap.grad.item() - gk.sum()) <= 1e-12 * abs(kap.grad.item())
    assert np.allclose(rho0.grad.numpy(), rb0, rtol=1e-12, atol=0)


# ------------------------------------------------------------------ FP32 rollouts

@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32_dfmu"])
@pytest.mark.parametrize("lattice", ["D1Q3", "D2Q9"])
def test_fp32_one_step_dot_product(gpu_lib, parity_bound, lattice, precision):
    # <J v, w> = <v, J^T w> for one step of an FP32-storage context, J^T w from the FP32
    # adjoint (FP64 mu).  J v comes from Richardson-extrapolated central differences of the
    # FP64 forward from the same initial densities: the two linearisation points differ by
    # the FP32 rounding of the stored state, so agreement is bounded by FP32 precision.
    from paper_1805_07251_gb300 import Simulation, capi

    spec = spec_small(lattice, 1)
    rho0 = fields(spec)
    rng = np.random.default_rng(11)
    v = 1e-2 * rng.normal(0, 1, rho0.shape)
    w = rng.normal(0, 1, rho0.shape)
    sim = Simulation(lattice=spec["lattice"], nx=spec["nx"], ny=spec["ny"], ncomp=2, tau=spec["tau"],
                     kT=spec["kT"], gamma_mu=spec["gamma_mu"], a=spec["a"], kappa=np.full((2, 2), spec["kappa"]),
                     lam=spec["lam"], b=spec["b"], precision=precision)
    sim.init(rho0)
    capi.lb_rollout_forward(sim.ctx, 1, 1)
    rb0, g = capi.lb_rollout_backward(sim.ctx, w, 2)
    sim.close()
    a12 = spec["a"][0, 1]
    jv = central(lambda t: float(np.sum(final_density(spec, a12, rho0 + t * v) * w)), 0.0, 1e-4)
    parity_bound("<v, J^T w> vs <J v, w> (rel.)", abs(np.sum(rb0 * v) - jv) / abs(jv), 1e-5)
    ja = central(lambda t: float(np.sum(final_density(spec, t, rho0) * w)), a12, 1e-3)
    parity_bound("d<rho_1, w>/d a12 (rel.)", abs((g[1] + g[2]) - ja) / abs(ja), 1e-4)


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32_dfmu"])
@pytest.mark.parametrize("lattice", ["D1Q3", "D2Q9"])
def test_fp32_gradients_against_fp64(gpu_lib, parity_bound, lattice, precision):
    # the FP32 rollout's gradients (FP32 forward and adjoint, FP64 mu) against the FP64
    # rollout's on the same loss: they differ by the FP32 forward trajectory's distance
    # from the FP64 one and the FP32 arithmetic of the adjoint; checkpointing must not
    # change them (the recompute is bitwise the forward)
    spec = spec_small(lattice, 60)
    rho0, tgt = fields(spec), target(spec)
    r64 = adjoint_grads(spec, rho0, tgt, ckpt=25)
    r32 = adjoint_grads(spec, rho0, tgt, ckpt=25, precision=precision)
    r32b = adjoint_grads(spec, rho0, tgt, ckpt=7, precision=precision)
    for u, w in zip(r32, r32b):
        assert np.array_equal(u, w)
    rb64, ga64, gk64, gb64 = r64
    rb32, ga32, gk32, gb32 = r32
    da = abs((ga32[0, 1] + ga32[1, 0]) - (ga64[0, 1] + ga64[1, 0])) / abs(ga64[0, 1] + ga64[1, 0])
    dk = abs(gk32.sum() - gk64.sum()) / abs(gk64.sum())
    db = np.max(np.abs(gb32 - gb64)) / np.max(np.abs(gb64))
    dr = np.max(np.abs(rb32 - rb64)) / np.max(np.abs(rb64))
    parity_bound("dL/da12 vs FP64 adjoint (rel.)", da, 1e-3)
    parity_bound("dL/dkappa vs FP64 adjoint (rel.)", dk, 1e-3)
    parity_bound("dL/db vs FP64 adjoint (rel. max)", db, 1e-3)
    parity_bound("dL/drho0 vs FP64 adjoint (rel. max)", dr, 1e-3)


@pytest.mark.parametrize("N,precision", [(3, "fp64"), (4, "fp64"), (4, "fp32_dfmu")])
def test_adjoint_more_components(gpu_lib, parity_bound, N, precision):
    # the adjoint kernels for N = 3, 4 (the forward's general N-component friction solve;
    # for FP32 storage and four components the forward runs as two lane pairs): dL/da_12
    # and dL/dkappa against Richardson-extrapolated central differences of the FP64 forward
    from paper_1805_07251_gb300 import Simulation, capi

    r = np.random.default_rng(300 + N)
    a = r.uniform(0.5, 1.2, (N, N)); a = 0.5 * (a + a.T); np.fill_diagonal(a, 1.0)
    b = r.uniform(0.2, 0.35, N)
    x = np.full(N, 1.0 / N)
    kT = 1.05 * lbinputs.one_fluid_critical_kT(a, b, x)
    lam = np.ones((N, N)) - np.eye(N)
    nx, ny, steps = 24, 20, 40
    rho0 = lbinputs.uniform_noise_fields(N, ny, nx, 1.3 * x, 1e-2, 4000 + N)
    tgt = rho0 + np.random.default_rng(5).normal(0, 1e-2, rho0.shape)

    def make(aa, kap, prec):
        return Simulation(lattice="D2Q9", nx=nx, ny=ny, ncomp=N, tau=1.0, kT=kT, gamma_mu=0.1, a=aa,
                          kappa=np.full((N, N), kap), lam=lam, b=b, precision=prec)

    def loss(a12, kap):
        aa = a.copy(); aa[0, 1] = aa[1, 0] = a12
        s = make(aa, kap, "fp64")
        s.init(rho0)
        s.step(steps)
        rr, _ = s.moments()
        s.close()
        return float(np.sum((rr - tgt) ** 2))

    s = make(a, 0.1, precision)
    s.init(rho0)
    capi.lb_rollout_forward(s.ctx, steps, 16)
    rr, _ = s.moments()
    _, g = capi.lb_rollout_backward(s.ctx, 2.0 * (rr - tgt), N)
    s.close()
    ga = g[1] + g[N]
    gk = g[N * N: 2 * N * N].sum()
    fa = central(lambda v: loss(v, 0.1), a[0, 1], 1e-4)
    fk = central(lambda v: loss(a[0, 1], v), 0.1, 1e-4)
    bar = 1e-6 if precision == "fp64" else 1e-3
    parity_bound("dL/da12 vs FD (rel.)", abs(ga - fa) / abs(fa), bar)
    parity_bound("dL/dkappa vs FD (rel.)", abs(gk - fk) / abs(fk), bar)
