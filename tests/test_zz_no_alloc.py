"""GPU test of lb_free_energy_noalloc, the diagnostics entry point that allocates
nothing (for callers that cannot allocate device memory where they need the numbers,
e.g. inside another framework's memory pool or under a fixed memory budget).

It is checked through the C ABI against the context-based lb_free_energy on the same
state, on two calls in a row (the shared static scratch keeps the previous call's
contents, so the second call must not depend on them).  This file is named to be
collected last."""
import numpy as np
import pytest

import lbinputs

pytestmark = pytest.mark.gpu


def _state(precision, nx, ny):
    from paper_1805_07251_gb300 import Simulation

    p = lbinputs.base_params("c2")
    kw = lbinputs.lib_kwargs(p)
    kw["nx"], kw["ny"] = nx, ny
    rho = lbinputs.fields("c2", nx=nx, ny=ny)
    sim = Simulation(precision=precision, **kw)
    sim.init(rho)
    sim.step(40)
    return sim, rho


@pytest.mark.parametrize("precision", ["fp64", "fp32_dfmu"])
def test_noalloc_matches_context_diagnostics(gpu_lib, precision):
    import torch

    from paper_1805_07251_gb300 import capi

    sim, rho = _state(precision, 96, 80)
    F, mass, mom = sim.free_energy()
    buf = sim.save_state()
    dtype = np.float64 if precision == "fp64" else np.float32
    f_host = np.frombuffer(buf[64:].tobytes(), dtype=dtype).copy()
    f_dev = torch.from_numpy(f_host).cuda()
    p = sim.params
    if precision != "fp64":
        ref = np.float32(rho.reshape(2, -1).mean(axis=1))
        for c in range(2):
            p.rho_ref[c] = float(ref[c])
    p.stream = torch.cuda.current_stream().cuda_stream
    N = 2
    for _ in range(2):
        out = torch.full((N + 4,), float("nan"), dtype=torch.float64, device="cuda")
        capi.lb_free_energy_noalloc(p, f_dev.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert o[N + 3] == 0.0
        assert np.max(np.abs(o[:N] - mass) / mass) < 1e-12
        assert abs(o[N] - F) <= 1e-12 * abs(F)
        assert np.max(np.abs(o[N + 1:N + 3] - mom)) < 1e-12
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
