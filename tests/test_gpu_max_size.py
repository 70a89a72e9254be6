"""GPU parity at the largest lattices the FP32 and FP64 storages address.

FP32 storage addresses a component's Q planes with unsigned 32-bit element offsets from a
per-component base pointer, so Q nx ny must stay below 2^32 (checked by lb_create); the
FP64 path uses 64-bit offsets.  These tests step lattices whose element offsets pass 2^31
(FP64) and come within 1 % of 2^32 (FP32, 21760^2 nodes, two components: 4.26e9 elements
per component) and compare sampled nodes, including those at the highest offsets, with the
oracle's step on 9 x 9 periodic windows (the step's dependency radius is 3, so a window's
centre is exact).  The chained steps of lb_step(n) must give the bits of one launch per step
at that size too.  They hold ~130 GB (FP32) and ~110 GB (FP64) of device memory."""
import numpy as np
import pytest

import lbinputs
import oracle

pytestmark = pytest.mark.gpu


def _free_bytes():
    import torch

    return torch.cuda.mem_get_info(0)[0]


def _windows(rho_dev, pts):
    """9 x 9 periodic windows of the device densities around the sampled nodes (host copies)."""
    import torch

    N, ny, nx = rho_dev.shape
    out = []
    for (y, x) in pts:
        ys = torch.tensor((np.arange(-4, 5) + y) % ny, device=rho_dev.device)
        xs = torch.tensor((np.arange(-4, 5) + x) % nx, device=rho_dev.device)
        out.append(rho_dev[:, ys][:, :, xs].cpu().numpy())
    return out


def _samples(ny, nx, seed):
    r = np.random.default_rng(seed)
    pts = [(0, 0), (ny - 1, nx - 1), (ny - 1, 0), (0, nx - 1), (ny - 2, nx - 33), (ny // 2, nx // 2)]
    pts += [(int(r.integers(ny - 64, ny)), int(r.integers(0, nx))) for _ in range(6)]  # highest offsets
    pts += [(int(r.integers(0, ny)), int(r.integers(0, nx))) for _ in range(12)]
    return pts


def _moments_at(sim, N, ny, nx, pts):
    import torch

    rho = torch.empty((N, ny, nx), dtype=torch.float64, device="cuda:0")
    mom = torch.empty((N, 2, ny, nx), dtype=torch.float64, device="cuda:0")
    sim.moments_dev(rho.data_ptr(), mom.data_ptr())
    torch.cuda.synchronize()
    ys = torch.tensor([p[0] for p in pts], device="cuda:0")
    xs = torch.tensor([p[1] for p in pts], device="cuda:0")
    r_s = rho[:, ys, xs].cpu().numpy()
    j_s = mom[:, :, ys, xs].cpu().numpy()
    return rho, mom, r_s, j_s


def _oracle_step(kw, N, wins):
    win = oracle.Lattice("D2Q9", 9, 9, N, kw["tau"], kw["kT"], kw["gamma_mu"], kw["a"], kw["kappa"], kw["lam"],
                         kw["b"])
    res = []
    for w in wins:
        ro, jo = win.moments(win.run(win.equilibrium(w), 1))
        res.append((ro[:, 4, 4], jo[:, :, 4, 4]))
    return res


def test_fp32_near_maximum_lattice_one_step_and_chain(gpu_lib, parity_bound):
    # 21760^2 nodes: 9 nx ny = 4.261e9 of the 4.295e9 elements a component's 32-bit offsets
    # reach.  One step against the oracle at sampled nodes (FP32 rounding bar, as at 1024^2),
    # then three chained steps (one lb_step(3) call) against three single launches, bitwise.
    import torch
    from paper_1805_07251_gb300 import Simulation

    n = 21760
    assert 9 * n * n < 1 << 32 and 9 * n * n > 0.99 * (1 << 32)
    if _free_bytes() < 140e9:
        pytest.skip("needs ~140 GB of free device memory")
    p = lbinputs.base_params("c2")
    kw = lbinputs.lib_kwargs(p, nx=n, ny=n)
    N = kw["ncomp"]
    rho0 = lbinputs.fields_on_device("c2", n, n, "cuda:0", 1805072517)
    pts = _samples(n, n, 91)
    wins = _windows(rho0, pts)
    sim = Simulation(precision="fp32_dfmu", device=0, **kw)
    try:
        assert sim.kernel == ("tiles", (32, 8)) and sim.chain_rows > 0
        sim.init_dev(rho0.data_ptr())
        sim.step(1)
        rho, mom, r_s, j_s = _moments_at(sim, N, n, n, pts)
        del mom
        worst = 0.0
        for k, (ro, jo) in enumerate(_oracle_step(kw, N, wins)):
            worst = max(worst, float(np.max(np.abs(r_s[:, k] - ro))), float(np.max(np.abs(j_s[:, :, k] - jo))))
        parity_bound("first step at 21760^2, rho and j", worst, 2e-6)
        # chained steps against single launches, from the same initial state
        sim.step(3)
        rho_chain = torch.empty_like(rho)
        sim.moments_dev(rho_chain.data_ptr(), None)
        sim.init_dev(rho0.data_ptr())
        for _ in range(4):
            sim.step(1)
        sim.moments_dev(rho.data_ptr(), None)
        torch.cuda.synchronize()
        assert torch.equal(rho_chain, rho), "chained steps differ from single launches at 21760^2"
    finally:
        sim.close()
        del rho0
        torch.cuda.empty_cache()


def test_fp64_lattice_with_offsets_beyond_2e31(gpu_lib, parity_bound):
    # FP64 at 16384^2: 9 nx ny = 2.4e9 elements per component, past 2^31 (64-bit offsets).
    # One step against the oracle at sampled nodes, FP64 bar.
    import torch
    from paper_1805_07251_gb300 import Simulation

    n = 16384
    assert 9 * n * n > 1 << 31
    if _free_bytes() < 120e9:
        pytest.skip("needs ~120 GB of free device memory")
    p = lbinputs.base_params("c2")
    kw = lbinputs.lib_kwargs(p, nx=n, ny=n)
    N = kw["ncomp"]
    rho0 = lbinputs.fields_on_device("c2", n, n, "cuda:0", 1805072518)
    pts = _samples(n, n, 92)
    wins = _windows(rho0, pts)
    sim = Simulation(precision="fp64", device=0, **kw)
    try:
        sim.init_dev(rho0.data_ptr())
        sim.step(1)
        _, _, r_s, j_s = _moments_at(sim, N, n, n, pts)
        worst = 0.0
        for k, (ro, jo) in enumerate(_oracle_step(kw, N, wins)):
            worst = max(worst, float(np.max(np.abs(r_s[:, k] - ro))), float(np.max(np.abs(j_s[:, :, k] - jo))))
        parity_bound("first step at 16384^2 (FP64), rho and j", worst, 1e-13)
    finally:
        sim.close()
        del rho0
        torch.cuda.empty_cache()
