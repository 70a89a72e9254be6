"""GPU test of lb_free_energy_noalloc, the diagnostics entry point that allocates
nothing.  It serves callers that cannot allocate device memory where they need the
numbers: code inside another framework's memory pool or under a fixed memory budget,
tools handed a bare device pointer to a state, and code that must not trigger an
allocation (and the synchronisation it can bring) in the middle of its own stream work.

Each case is checked through the C ABI, on two calls in a row (the shared static scratch
keeps the previous call's contents, so the second call must not depend on them):
  * against the context-based lb_free_energy on the same state, and
  * against the oracle's free energy and masses of the densities the GPU state holds
    (Eq. discreteFreeEnergy of the paper, computed on the CPU from lb_read_moments).
The cases cover D1Q3 (no y momentum), two and four components, every storage precision,
and a lattice of more nodes (576 x 576) than the reduction's 1024 partial sums x 256
threads cover in one pass.  This file is named to be collected last."""
import numpy as np
import pytest

import lbinputs
import oracle

pytestmark = pytest.mark.gpu

CASES = [
    # (workload recipe, nx, ny, precision)
    ("c2", 96, 80, "fp64"),
    ("c2", 96, 80, "fp32_dfmu"),
    ("c2", 96, 80, "fp32_mixed"),
    ("c2", 96, 80, "fp32"),
    ("c1", 300, 1, "fp64"),
    ("c1", 300, 1, "fp32_dfmu"),
    ("c4", 64, 64, "fp64"),
    ("c4", 64, 64, "fp32_dfmu"),
    ("c2", 576, 576, "fp32_dfmu"),
]


def _state(name, nx, ny, precision):
    from paper_1805_07251_gb300 import Simulation

    p = lbinputs.base_params(name)
    kw = lbinputs.lib_kwargs(p)
    kw["nx"], kw["ny"] = nx, ny
    rho = lbinputs.fields(name, nx=nx, ny=ny)
    N = kw["ncomp"]
    rho_ref = None
    if precision != "fp64":
        # the reference densities are passed explicitly, so the context and the
        # no-allocation call subtract the same w_i rho_ref^c
        rho_ref = [float(np.float32(v)) for v in rho.reshape(N, -1).mean(axis=1)]
    sim = Simulation(precision=precision, rho_ref=rho_ref, **kw)
    sim.init(rho)
    sim.step(40)
    orc = oracle.Lattice(kw["lattice"], nx, ny, N, kw["tau"], kw["kT"], kw["gamma_mu"], kw["a"], kw["kappa"],
                         kw["lam"], kw["b"])
    return sim, orc


@pytest.mark.parametrize("name,nx,ny,precision", CASES)
def test_noalloc_matches_context_and_oracle(gpu_lib, name, nx, ny, precision):
    import torch

    from paper_1805_07251_gb300 import capi

    sim, orc = _state(name, nx, ny, precision)
    N = sim.ncomp
    F, mass, mom = sim.free_energy()
    rho_gpu, j_gpu = sim.moments()
    F_orc, mass_orc = orc.free_energy(rho_gpu)
    mom_orc = j_gpu.sum(axis=(0, 2, 3))
    buf = sim.save_state()
    dtype = np.float64 if precision == "fp64" else np.float32
    f_host = np.frombuffer(buf[64:].tobytes(), dtype=dtype).copy()
    f_dev = torch.from_numpy(f_host).cuda()
    p = sim.params
    p.stream = torch.cuda.current_stream().cuda_stream
    dev_before = torch.cuda.current_device()
    scale_F = max(abs(F_orc), float(np.sum(mass_orc)))
    for _ in range(2):
        out = torch.full((N + 4,), float("nan"), dtype=torch.float64, device="cuda")
        capi.lb_free_energy_noalloc(p, f_dev.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        assert torch.cuda.current_device() == dev_before
        o = out.cpu().numpy()
        assert o[N + 3] == 0.0
        # against the context's reduction (same kernels, same order)
        assert np.max(np.abs(o[:N] - mass) / mass) < 1e-12
        assert abs(o[N] - F) <= 1e-12 * abs(F)
        assert np.max(np.abs(o[N + 1:N + 3] - mom)) < 1e-12
        # against the oracle on the same densities (different summation order)
        assert np.max(np.abs(o[:N] - mass_orc) / mass_orc) < 1e-12
        assert abs(o[N] - F_orc) <= 1e-12 * scale_F
        assert np.max(np.abs(o[N + 1:N + 1 + sim.d] - mom_orc[:sim.d])) < 1e-10 * float(np.sum(mass_orc))
    sim.close()


def test_noalloc_rejects_states_beyond_its_scratch(gpu_lib):
    import torch

    from paper_1805_07251_gb300 import capi, make_params

    p = lbinputs.base_params("c2")
    kw = lbinputs.lib_kwargs(p)
    kw["nx"], kw["ny"] = 1024, 1024          # 2 * 3 * 2^20 doubles > 2^21
    prm = make_params(**kw)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.LBError) as e:
        capi.lb_free_energy_noalloc(prm, dummy.data_ptr(), out.data_ptr())
    assert e.value.status == capi.LB_E_INVALID
