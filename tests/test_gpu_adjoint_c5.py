"""The adjoint rollout at the full size of workload c5: D2Q9, two components, 512 x 512,
the config-2 mixture with a12 = 0.75, 2000 steps checkpointed every 100; loss = sum of
(rho_T - rho_target)^2 with the target from the FP64 forward at a12 = 0.8.

The FP64 rollout's gradients in a12, kappa and one random direction of the initial
densities are compared with central differences of the FP64 forward (h = 1e-4, h/2, h/4,
Richardson-extrapolated to O(h^6)) at the 1e-6 relative bar; the FP32-storage rollout
(double-float mu forward, FP32 adjoint with FP64 mu) with the FP64 adjoint at 1e-3, the
distance between the FP32 and FP64 spinodal trajectories over 2000 steps."""
import numpy as np
import pytest

import lbinputs

pytestmark = pytest.mark.gpu


def richardson(fun, x0, h):
    d = [(fun(x0 + s) - fun(x0 - s)) / (2 * s) for s in (h, h / 2, h / 4)]
    r1 = (4 * d[1] - d[0]) / 3
    r2 = (4 * d[2] - d[1]) / 3
    return (16 * r2 - r1) / 15


def test_c5_full_size_gradients(gpu_lib, parity_bound):
    from paper_1805_07251_gb300 import Simulation, capi

    p = lbinputs.base_params("c5")
    n, steps = p["nx"], p["steps"]
    assert (n, steps) == (512, 2000)
    rho0 = lbinputs.fields("c5")

    def make(a12, kap, precision="fp64"):
        a = p["a"].copy()
        a[0, 1] = a[1, 0] = a12
        return Simulation(lattice="D2Q9", nx=n, ny=n, ncomp=2, tau=1.0, kT=p["kT"], gamma_mu=p["gamma_mu"], a=a,
                          kappa=np.full((2, 2), kap), lam=p["lam"], b=p["b"], precision=precision, device=0)

    def final(a12, kap, r0):
        s = make(a12, kap)
        s.init(r0)
        s.step(steps)
        r, _ = s.moments()
        s.close()
        return r

    tgt = final(0.8, 0.1, rho0)
    v = 1e-2 * np.random.default_rng(5).normal(0, 1, rho0.shape)

    def loss(a12, kap, r0=rho0):
        return float(np.sum((final(a12, kap, r0) - tgt) ** 2))

    def gradient(precision):
        s = make(0.75, 0.1, precision)
        s.init(rho0)
        capi.lb_rollout_forward(s.ctx, steps, 100)
        r, _ = s.moments()
        rb0, g = capi.lb_rollout_backward(s.ctx, 2.0 * (r - tgt), 2)
        s.close()
        return g[1] + g[2], g[4:8].sum(), float(np.sum(rb0 * v))

    ga, gk, gr = gradient("fp64")
    fa = richardson(lambda x: loss(x, 0.1), 0.75, 1e-4)
    fk = richardson(lambda x: loss(0.75, x), 0.1, 1e-4)
    fr = richardson(lambda t: loss(0.75, 0.1, rho0 + t * v), 0.0, 1e-4)
    parity_bound("FP64 dL/da12 vs FD (rel.)", abs(ga - fa) / abs(fa), 1e-6)
    parity_bound("FP64 dL/dkappa vs FD (rel.)", abs(gk - fk) / abs(fk), 1e-6)
    parity_bound("FP64 dL/drho0 . v vs FD (rel.)", abs(gr - fr) / abs(fr), 1e-6)

    qa, qk, qr = gradient("fp32_dfmu")
    parity_bound("FP32 dL/da12 vs FP64 adjoint (rel.)", abs(qa - ga) / abs(ga), 1e-3)
    parity_bound("FP32 dL/dkappa vs FP64 adjoint (rel.)", abs(qk - gk) / abs(gk), 1e-3)
    parity_bound("FP32 dL/drho0 . v vs FP64 adjoint (rel.)", abs(qr - gr) / abs(gr), 1e-3)
