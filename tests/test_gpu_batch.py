"""GPU tests of batched independent runs (lb_batch_*): every run of a batch equals the
same run advanced alone (bitwise), per-run error flags isolate a failing run, the tile
autotuner returns a compiled tile, and a batch run matches the FP64 oracle."""
import numpy as np
import pytest

import lbinputs
import oracle

pytestmark = pytest.mark.gpu


def small_sweep(n1=3, n2=3):
    runs = lbinputs.sweep_runs()
    d1 = [r for r in runs[:256] if r["nx"] <= 1500][:n1]
    d2 = [r for r in runs[256:] if r["nx"] <= 130][:n2]
    return d1 + d2


def make_batch(recs, precision, tile=None):
    from paper_1805_07251_gb300.batch import Batch

    p = lbinputs.base_params("c1")
    return Batch(recs, p["a"], p["b"], p["kappa"], p["lam"], 2, precision=precision, tile=tile)


def single(rec, precision, steps):
    from paper_1805_07251_gb300 import Simulation

    p = lbinputs.base_params("c1")
    sim = Simulation(lattice=rec["lattice"], nx=rec["nx"], ny=rec["ny"], ncomp=2, tau=1.0, kT=rec["kT"],
                     gamma_mu=rec["gamma_mu"], a=p["a"], kappa=p["kappa"], lam=p["lam"], b=p["b"],
                     precision=precision)
    sim.init(lbinputs.sweep_fields(rec))
    sim.step(steps)
    out = sim.moments()
    sim.close()
    return out


@pytest.mark.parametrize("precision", ["fp32_dfmu", "fp32_mixed", "fp64"])
def test_batch_runs_equal_single_runs(gpu_lib, precision):
    recs = small_sweep()
    b = make_batch(recs, precision)
    fields = [lbinputs.sweep_fields(r) for r in recs]
    b.init(fields)
    b.step(100)          # 3 graph chunks of 32 and a remainder of 4: both parities
    for k, rec in enumerate(recs):
        rb, jb = b.read(k)
        rs, js = single(rec, precision, 100)
        assert np.array_equal(rb, rs), (k, rec["lattice"], float(np.max(np.abs(rb - rs))))
        assert np.array_equal(jb, js)
    b.step(37)
    rb, _ = b.read(0)
    rs, _ = single(recs[0], precision, 137)
    assert np.array_equal(rb, rs)
    assert not b.errors().any()
    b.close()


def test_batch_error_flag_isolates_a_failing_run(gpu_lib):
    recs = small_sweep(2, 2)
    recs[1] = dict(recs[1], gamma_mu=50.0)     # far above the stable range
    b = make_batch(recs, "fp32_dfmu")
    b.init([lbinputs.sweep_fields(r) for r in recs])
    b.step(300)
    err = b.errors()
    assert err[1] != 0 and err[0] == 0 and err[2] == 0 and err[3] == 0
    rb, _ = b.read(2)
    rs, _ = single(recs[2], "fp32_dfmu", 300)
    assert np.array_equal(rb, rs)
    b.close()


def test_batch_autotune_picks_a_compiled_tile(gpu_lib, tmp_path):
    from paper_1805_07251_gb300.batch import TILES, autotune

    recs = small_sweep(1, 4)
    fields = [lbinputs.sweep_fields(r) for r in recs]
    b = make_batch(recs, "fp32_dfmu")
    b.init(fields)
    tile, times = autotune(b, fields, "fp32_dfmu", steps=16, cache_path=str(tmp_path / "tune.json"))
    assert tuple(tile) in TILES and len(times) == len(TILES)
    tile2, _ = autotune(b, fields, "fp32_dfmu", cache_path=str(tmp_path / "tune.json"))
    assert tuple(tile2) == tuple(tile)
    # the autotuned batch still reproduces the single runs (results do not depend on the
    # tile); a run that left the domain in the batch does so alone too
    from paper_1805_07251_gb300 import capi

    b.step(40)
    err = b.errors()
    for k, rec in enumerate(recs):
        if err[k]:
            with pytest.raises(capi.LBError):
                single(rec, "fp32_dfmu", 40)
            continue
        rb, _ = b.read(k)
        rs, _ = single(rec, "fp32_dfmu", 40)
        assert np.array_equal(rb, rs)
    b.close()


def test_batch_fp64_runs_match_oracle(gpu_lib):
    recs = small_sweep(1, 1)
    b = make_batch(recs, "fp64")
    b.init([lbinputs.sweep_fields(r) for r in recs])
    b.step(200)
    p = lbinputs.base_params("c1")
    for k, rec in enumerate(recs):
        rb, _ = b.read(k)
        orc = oracle.Lattice(rec["lattice"], rec["nx"], rec["ny"], 2, 1.0, rec["kT"], rec["gamma_mu"], p["a"],
                             p["kappa"], p["lam"], p["b"])
        ro, _ = orc.moments(orc.run(orc.equilibrium(lbinputs.sweep_fields(rec)), 200))
        assert np.max(np.abs(rb - ro)) / np.max(np.abs(ro)) < 1e-12
    b.close()
