"""Chained steps (lb_step with two or more steps on D2Q9, two FP32 components, 32 x 8
tiles): step s + 1 launches while step s finishes, and its first tiles wait on the
completion flags of the 3 x 3 tiles around them.  The arithmetic of a tile is unchanged,
so n chained steps must be bitwise equal to n single-step calls (one plain launch each):
on lattices of many tile rows (flags on the first rows only), of fewer rows than one wave
(every row sets flags), with ragged tiles, with the "nid" force, the moment-space
collision, FP32 mu, and chains cut by check_every; with the evict-first L2 policy of the
input (every lattice of the first test) and without it (4096^2 in the long-chain test)."""
import numpy as np
import pytest

import lbinputs

pytestmark = pytest.mark.gpu


def _pair(nx, ny, precision="fp32_dfmu", **over):
    from paper_1805_07251_gb300 import Simulation

    p = lbinputs.base_params("c2")
    kw = lbinputs.lib_kwargs(p, nx=nx, ny=ny)
    kw.update(over)
    rho = lbinputs.fields("c2", nx, ny)
    sims = [Simulation(precision=precision, device=0, **kw) for _ in range(2)]
    for s in sims:
        s.init(rho)
    return sims


@pytest.mark.parametrize("nx,ny,steps,over", [
    (1024, 1024, 20, {}),
    (2048, 512, 9, {}),
    (1000, 1000, 13, {}),
    (96, 64, 12, {}),
    (70, 45, 11, {}),
    (200, 40, 7, {"precision": "fp32"}),
    (256, 256, 10, {"force": "nid"}),
    (256, 192, 10, {"tau_shear": 0.8, "tau_ghost": 1.0}),
    (512, 256, 23, {"check_every": 5}),
])
def test_chained_steps_bitwise_equal_single_steps(gpu_lib, nx, ny, steps, over):
    over = dict(over)
    precision = over.pop("precision", "fp32_dfmu")
    a, b = _pair(nx, ny, precision, **over)
    try:
        assert a.chain_rows > 0 and b.chain_rows == a.chain_rows
        assert a.chain_rows <= (ny + 7) // 8
        a.step(steps)
        for _ in range(steps):
            b.step(1)
        assert a.steps == b.steps == steps
        sa, sb = a.save_state(), b.save_state()
        assert np.array_equal(sa, sb)
        # and the moments read back from both agree (the chain leaves the right buffer current)
        ra, _ = a.moments()
        rb, _ = b.moments()
        assert np.array_equal(ra, rb)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("nx,ny,over", [
    (66, 64, {}),                      # a ragged tile column 2 nodes wide: not chained
    (64, 66, {}),                      # a ragged tile row 2 nodes high: not chained
    (256, 256, {"precision": "fp32_mixed"}),
    (256, 256, {"ncomp4": True}),
])
def test_unchained_configurations_step_plainly(gpu_lib, nx, ny, over):
    from paper_1805_07251_gb300 import Simulation

    over = dict(over)
    precision = over.pop("precision", "fp32_dfmu")
    if over.pop("ncomp4", False):
        p = lbinputs.base_params("c4")
        kw = lbinputs.lib_kwargs(p, nx=nx, ny=ny)
        rho = lbinputs.fields("c4", nx, ny)
    else:
        p = lbinputs.base_params("c2")
        kw = lbinputs.lib_kwargs(p, nx=nx, ny=ny)
        rho = lbinputs.fields("c2", nx, ny)
    a, b = (Simulation(precision=precision, device=0, **kw) for _ in range(2))
    try:
        assert a.chain_rows == 0
        a.init(rho)
        b.init(rho)
        a.step(6)
        for _ in range(6):
            b.step(1)
        assert np.array_equal(a.save_state(), b.save_state())
    finally:
        a.close()
        b.close()


def test_chains_continue_across_calls_and_reinitialisation(gpu_lib):
    """Flags carry the chain step number; a new call, a new state or a reload starts a
    fresh chain whose first step waits on nothing, so stale flags never release a tile."""
    a, b = _pair(512, 512)
    try:
        rho = lbinputs.fields("c2", 512, 512)
        for n in (3, 2, 5):
            a.step(n)
            for _ in range(n):
                b.step(1)
        assert np.array_equal(a.save_state(), b.save_state())
        snap = a.save_state()
        a.init(rho)
        b.init(rho)
        a.step(4)
        for _ in range(4):
            b.step(1)
        assert np.array_equal(a.save_state(), b.save_state())
        a.load_state(snap)
        b.load_state(snap)
        a.step(6)
        for _ in range(6):
            b.step(1)
        assert np.array_equal(a.save_state(), b.save_state())
    finally:
        a.close()
        b.close()


def test_steps_captured_in_a_cuda_graph_replay_like_single_steps(gpu_lib):
    """lb_step enqueued while its stream is captured into a CUDA graph uses plain launches
    (a replayed chain would reuse its captured step numbers); three replays of a captured
    call of 4 steps equal 12 single steps."""
    import torch

    from paper_1805_07251_gb300 import Simulation

    p = lbinputs.base_params("c2")
    kw = lbinputs.lib_kwargs(p, nx=256, ny=256)
    rho = lbinputs.fields("c2", 256, 256)
    s = torch.cuda.Stream()
    a = Simulation(precision="fp32_dfmu", device=0, stream=s.cuda_stream, **kw)
    b = Simulation(precision="fp32_dfmu", device=0, **kw)
    try:
        assert a.chain_rows > 0
        a.init(rho)
        b.init(rho)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            a.step(4)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        for _ in range(12):
            b.step(1)
        # populations only: the saved header holds the host's step count, which graph
        # replays do not advance (4 against 12)
        assert np.array_equal(a.save_state()[64:], b.save_state()[64:])
        assert a.steps == 4 and b.steps == 12
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("n,evict_first", [(1024, True), (1536, False), (4096, False)])
def test_l2_policy_of_the_chain_follows_the_buffer_size(gpu_lib, n, evict_first):
    # the chained steps mark their input evict-first in the L2 where one population buffer
    # (72 B per node for two FP32 components) takes at most 60 % of the L2: 75.5 MB at
    # 1024^2 (of GB300's ~126 MB), not 170 MB at 1536^2; single steps never do
    from paper_1805_07251_gb300 import Simulation

    p = lbinputs.base_params("c2")
    s = Simulation(precision="fp32_dfmu", device=0, **lbinputs.lib_kwargs(p, nx=n, ny=n))
    try:
        assert s.chain_rows > 0 and s.chain_evict_first == evict_first
    finally:
        s.close()
    s = Simulation(precision="fp64", device=0, **lbinputs.lib_kwargs(p, nx=256, ny=256))
    try:
        assert s.chain_rows == 0 and not s.chain_evict_first
    finally:
        s.close()


@pytest.mark.parametrize("n,steps", [(1024, 3000), (4096, 120)])
def test_long_chains_bitwise_equal_single_steps(gpu_lib, n, steps):
    """Long chains at the headline size (3000 steps in one call, the flag hand-off repeated
    about 100,000 times) and on a lattice of 512 tile rows (9 of them handing over by flags),
    bitwise against one plain launch per step: an ordering fault in the hand-off between
    overlapping grids would show up as a difference here."""
    a, b = _pair(n, n)
    try:
        assert a.chain_rows > 0
        a.step(steps)
        for _ in range(steps):
            b.step(1)
        assert np.array_equal(a.save_state()[64:], b.save_state()[64:])
    finally:
        a.close()
        b.close()
