#!/usr/bin/env python
"""Benchmark of the fused multicomponent van der Waals lattice Boltzmann step.

Workload (default): D2Q9, 2 components, 1024 x 1024 periodic, the asymmetric
mixture a = [[1, .9], [.9, .6]], b = (.25, .3), kappa = .1, kT = 0.85 of the
one-fluid critical temperature, uniform density 1.2 at mole fraction 0.4 plus
seeded Gaussian noise (sigma 1e-2): spinodal decomposition.  One benchmark step
is one lattice Boltzmann timestep (one fused kernel launch) of the whole
lattice.  The K timed steps run back to back in one lb_step call between two
CUDA events, as in a run of the workload (the library chains consecutive
launches of the two-component FP32 paths); the state, two population buffers
of 151 MB, is larger than the 129 MB L2.  Each path is also timed with one
launch per step and the L2 flushed (256 MB write) before each, outside the
events (``flushed`` in the line).

Metric: component-MLUPS = ncomp * nodes * steps / s / 1e6.  Three paths are
timed in the same run: FP32 storage with the chemical potential in
double-float arithmetic (headline ``value``), FP32 storage with the chemical
potential in FP64 (``fp32_fp64mu``) and the plain FP64 path (``fp64``), each
with the roofline fraction of its step kernel against the measured HBM copy
bandwidth.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With torchrun (N > 1) every rank runs an independent replica of the workload
(the path has no exchange between independent runs); the timed region is
bracketed by barriers and the maximum over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "component-MLUPS and % of HBM roofline: batched FP32 vs plain FP64 at stated error"
UNIT = "component-MLUPS"
WORKLOAD = "c2"
FLUSH_BYTES = 256 << 20
DTYPES = {"fp32_dfmu": "f32 (populations and step), double-float mu",
          "fp32_mixed": "f32 (populations and step), f64 mu", "fp32": "f32 (populations, step and mu)",
          "fp64": "f64"}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--tile", default=None, help="D2Q9 tile as TXxTY (default: the library's)")
    ap.add_argument("--kernel", choices=["auto", "tiles", "strips", "ws"], default="auto",
                    help="organisation of the step kernel (default: the library's choice)")
    ap.add_argument("--segments", type=int, default=0, help="strips: row segments per strip (0 = library's)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the batched-sweep measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-rollout measurement")
    ap.add_argument("--no-c4", action="store_true", help="skip the four-component measurement")
    ap.add_argument("--adjoint-steps", type=int, default=0,
                    help="adjoint rollouts: steps of the rollout (0: the workload's 2000)")
    ap.add_argument("--no-fd", action="store_true",
                    help="adjoint rollouts: skip the finite-difference checks (profiling runs)")
    ap.add_argument("--only", choices=["fp32_dfmu", "fp32_mixed", "fp32", "fp64", "sweep", "c4", "adjoint", "c1",
                                       "sizes"],
                    default=None,
                    help="time one path only (profiling runs): no e2e, no cpu baseline; 'sizes': the headline "
                         "path on lattices of 512^2 to 4096^2 of the same recipe")
    return ap.parse_args(argv)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the headline
# step kernel (the chained step), from an ncu capture of this script (the profile file
# named beside it).  The value holds for the kernel sources whose digest is recorded with
# it and is reported as null once they change.
KERNEL_SOURCES = ("lb_kernels.cuh", "lb_chain.cuh", "lb_lane.cuh", "lb_mu.cuh", "lb_tu.cuh", "lb_launch.cuh",
                  "lb_d2q9_df.cu")
TRAFFIC = {"fp32_dfmu": {"digest": "7beb09f974cde77630c9b30434b768a5bf723b374759841067535a37725fe51c",
                         "bytes": 76000512 + 17210880, "warp_instructions": 29754080, "issue_active": 0.595,
                         "fma_pipe_active": 0.520,
                         "stalls_per_issue": {"barrier": 2.90, "long_scoreboard": 2.49, "not_selected": 2.52,
                                              "math_pipe_throttle": 2.14, "wait": 1.23},
                         "profile": "profiles/lb_chain_kernel_fp32_dfmu_c2_1024.md"}}
# FP64-pipe utilisation of the two FP64-bound paths (sm__pipe_fp64_cycles_active of one
# launch, the profile named beside it), valid for the kernel sources of the same digest
FP64_PIPE = {"digest": "7beb09f974cde77630c9b30434b768a5bf723b374759841067535a37725fe51c",
             "fp32_mixed": 0.840, "fp64": 0.851, "profile": "profiles/lb_step_kernel_fp64_c2_1024.md"}
# nominal HBM3e bandwidth of the GPU (GB/s), reported beside the measured copy peak
HBM_NOMINAL_GBS = 7900.0
# instruction issue peak of the GPU: 152 SMs x 4 schedulers x 2.07 GHz (one warp instruction
# per scheduler per cycle)
ISSUE_PEAK = 152 * 4 * 2.07e9


def kernel_digest():
    import hashlib

    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1805_07251_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_of(precision):
    rec = TRAFFIC.get(precision)
    if rec and rec["digest"] == kernel_digest():
        return rec["bytes"], rec["profile"]
    return None, None


def limiter_of(precision, alg_bytes, peak_gbs):
    """What bounds the step kernel, from the same ncu capture: how busy instruction issue
    and the FMA pipe are, the largest warp stall reasons, and the HBM fraction the launch's
    warp instructions would allow at the GPU's peak issue rate."""
    rec = TRAFFIC.get(precision)
    if not rec or rec["digest"] != kernel_digest():
        return None
    t_issue = rec["warp_instructions"] / ISSUE_PEAK
    return {"kind": "latency (barriers between the phases, global-load waits, FMA-pipe bursts)",
            "warp_instructions_per_launch": rec["warp_instructions"], "issue_active": rec["issue_active"],
            "fma_pipe_active": rec["fma_pipe_active"], "stalls_per_issue": rec["stalls_per_issue"],
            "launch_time_at_peak_issue_us": t_issue * 1e6,
            "hbm_frac_at_peak_issue": alg_bytes / t_issue / 1e9 / peak_gbs, "profile": rec["profile"]}


def max_over_ranks(dist, value, device):
    """The largest of the ranks' values (a job lasts as long as its slowest replica);
    the value itself on a single process."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Whole-job throughput in millions of units per second: every rank processes the same
    number of units (independent replicas, weak scaling) in at most `seconds`."""
    return world * units_per_rank / seconds / 1e6


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        with open(self.tmp.name) as fh:
            rows = [r.strip().split(",") for r in fh if r.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model():
    """The host CPU's model name (lscpu), for the CPU-baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform

    return platform.processor() or platform.machine()


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def cpu_baseline_oracle(kw, nx, steps, threads):
    """Time the CPU oracle (as it stands, OpenMP over rows with ``threads`` threads) on an
    nx x nx sample of the same recipe; returns (component-MLUPS, seconds, threads used)."""
    import lbinputs
    import oracle

    used = oracle.set_threads(threads)
    rho = lbinputs.fields(WORKLOAD, nx=nx, ny=nx)
    L = oracle.Lattice(kw["lattice"], nx, nx, kw["ncomp"], kw["tau"], kw["kT"], kw["gamma_mu"], kw["a"],
                       kw["kappa"], kw["lam"], kw["b"])
    f = L.equilibrium(rho)
    t0 = time.perf_counter()
    L.run(f, steps)
    dt = time.perf_counter() - t0
    return kw["ncomp"] * nx * nx * steps / dt / 1e6, dt, used


def run_reference(args):
    """Reference arm: the CPU oracle on the same workload, one oracle timestep of the
    full 1024 x 1024 lattice per benchmark step."""
    import lbinputs
    import oracle

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p = lbinputs.base_params(WORKLOAD)
    kw = lbinputs.lib_kwargs(p)
    rho = lbinputs.fields(WORKLOAD)
    threads = oracle.set_threads(host_cores())
    L = oracle.Lattice(kw["lattice"], kw["nx"], kw["ny"], kw["ncomp"], kw["tau"], kw["kT"], kw["gamma_mu"], kw["a"],
                       kw["kappa"], kw["lam"], kw["b"])
    f = L.equilibrium(rho)
    f = L.run(f, args.warmup)
    t0 = time.perf_counter()
    L.run(f, args.steps)
    dt = time.perf_counter() - t0
    nodes = kw["nx"] * kw["ny"]
    value = kw["ncomp"] * nodes * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "D2Q9, 2 components, 1024x1024 periodic, spinodal mixture (c2)",
                   "nodes": nodes, "ncomp": kw["ncomp"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu": cpu_model(),
                         "sample": f"full 1024x1024 lattice, {args.steps} oracle timesteps after {args.warmup} "
                                   f"warm-up, OpenMP over rows with {threads} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def time_sweep(torch, dev, precision, steps, warmup, dist):
    """Batched sweep (workload c3): 256 D1Q3 + 128 D2Q9 independent runs advanced together
    by CUDA-graph replays; D2Q9 tile from the autotuner.  The state (1.8 GB per step)
    exceeds the L2, so no flush is needed between steps.  Before timing, the campaign's
    pre-scan (3000 steps) re-tunes runs that leave the density domain (wider interfaces,
    lower gamma_mu), as the paper's campaigns did."""
    import lbinputs
    from paper_1805_07251_gb300.batch import Batch, autotune, prescan

    p = lbinputs.base_params("c1")
    recs, scan_fail = prescan(lbinputs.sweep_runs(), lbinputs.sweep_fields, p["a"], p["b"], p["kappa"], p["lam"], 2,
                              precision=precision, device=dev, stream=torch.cuda.current_stream(dev).cuda_stream)
    fields = [lbinputs.sweep_fields(r) for r in recs]
    b = Batch(recs, p["a"], p["b"], p["kappa"], p["lam"], 2, precision=precision, device=dev,
              stream=torch.cuda.current_stream(dev).cuda_stream)
    b.init(fields)
    tile, _ = autotune(b, fields, precision, steps=16)
    b.step(warmup)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    l0 = b.launches
    ms = max_over_ranks(dist, b.time_steps(steps), dev)
    launches = b.launches - l0
    unstable = int((b.errors() != 0).sum())
    cn = b.total_component_nodes()
    world = dist.get_world_size() if dist is not None else 1
    out = {"value": job_throughput(world, cn * steps, ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
           "runs": len(recs), "d1q3_runs": sum(r["lattice"] == "D1Q3" for r in recs),
           "d2q9_runs": sum(r["lattice"] == "D2Q9" for r in recs), "component_nodes": cn,
           "tile": "x".join(map(str, tile)) if tile else None, "unstable_runs_after_warmup_and_timed": unstable,
           "retuned_runs": sum(1 for r in recs if r.get("retuned")), "prescan_failures": scan_fail,
           "dtype": DTYPES[precision], "gpu_launches": launches,
           "note": "one CUDA-graph replay per 32 timesteps: D1Q3 runs resident in shared memory, "
                   "D2Q9 runs as one tile-list launch per timestep"}
    b.close()
    return out


def time_c4(torch, dev, precision, steps, warmup):
    """Workload c4: D2Q9, 4 components, 2048 x 2048 (604 MB of FP32 populations per
    buffer, larger than the L2), seeded random symmetric mixture, kT = 0.8 of the
    one-fluid critical temperature.  Times `steps` timesteps, then runs on towards the
    configuration's 5000 steps in chunks of 50, reporting the per-component mass drift at
    the last chunk that ended inside the density domain and the step at which the run left
    it.  This deep quench drives some node's density to zero after a number of steps
    proportional to 1/gamma_mu for every gamma_mu tried, in FP64 as in FP32: the mean's
    unstable direction has every component of one sign, so total-density waves grow
    until a gas node empties.  The same run re-tuned as the sweep's campaign re-tunes its
    failing runs (kappa x 4, gamma_mu / 4: wider interfaces) then runs the configured 5000
    steps, and its mass drift over them is reported."""
    import numpy as np

    import lbinputs
    from paper_1805_07251_gb300 import Simulation, capi

    p = lbinputs.base_params("c4")
    kw = lbinputs.lib_kwargs(p)
    rho = lbinputs.fields("c4")
    m0 = rho.reshape(p["ncomp"], -1).sum(axis=1)
    stream = torch.cuda.current_stream(dev)
    sim = Simulation(precision=precision, device=dev, stream=stream.cuda_stream, **kw)
    sim.init(rho)
    sim.step(warmup)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = sim.launches
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    launches = sim.launches - l0
    done, drift, left = warmup + steps, None, None
    try:
        _, mass, _ = sim.free_energy()
        drift = (done, float(np.max(np.abs(mass - m0) / m0)))
        while done < p["steps"]:
            sim.step(50)
            _, mass, _ = sim.free_energy()
            done += 50
            drift = (done, float(np.max(np.abs(mass - m0) / m0)))
    except capi.LBError:
        left = done + 50 if drift is not None else done
    sim.close()
    # the campaign's re-tuning of a run that leaves the density domain (the sweep's rule,
    # batch.retune): kappa x 4 and gamma_mu / 4; the run then completes its configured steps
    from paper_1805_07251_gb300.batch import KAPPA_STEP

    kw2 = dict(kw, kappa=np.asarray(kw["kappa"]) * KAPPA_STEP, gamma_mu=kw["gamma_mu"] / KAPPA_STEP)
    sim = Simulation(precision=precision, device=dev, stream=stream.cuda_stream, **kw2)
    sim.init(rho)
    retuned = {"kappa_scale": KAPPA_STEP, "gamma_mu": kw2["gamma_mu"]}
    try:
        sim.step(p["steps"])
        _, mass, _ = sim.free_energy()
        retuned.update(steps_in_domain=p["steps"], mass_drift_max_rel=float(np.max(np.abs(mass - m0) / m0)))
    except capi.LBError as e:
        retuned.update(error=str(e)[:160])
    sim.close()
    nodes = p["nx"] * p["ny"]
    N = p["ncomp"]
    return {"workload": "D2Q9, 4 components, 2048x2048, seeded mixture, kT = 0.8 theta_cr^mix",
            "value": N * nodes / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms,
            "roofline_hbm": {"achieved": N * nodes * 9 * 2 * 4 / (ms * 1e-3) / 1e9},
            "timed_steps_in_domain": drift is not None,
            "mass_drift_max_rel": drift[1] if drift else None, "mass_drift_after_steps": drift[0] if drift else None,
            "left_density_domain_by_step": left, "steps_configured": p["steps"], "retuned_run": retuned,
            "dtype": DTYPES[precision], "gpu_launches": launches, "l2": "state larger than L2, no flush"}


def time_c1(torch, dev, steps):
    """Workload c1: D1Q3, 2 components, 256 nodes, FP64, the config's 10,000 steps.  So small
    a lattice is bound by launches, not by the GPU: timed as a single run (one lb_step
    launch per step) and as a one-run batch (the run resident in shared memory, 32 steps
    per launch, replayed CUDA graphs), both with CUDA events; mass drift of each."""
    import numpy as np

    import lbinputs
    from paper_1805_07251_gb300 import Simulation
    from paper_1805_07251_gb300.batch import Batch

    p = lbinputs.base_params("c1")
    kw = lbinputs.lib_kwargs(p)
    rho = lbinputs.fields("c1")
    m0 = rho.reshape(2, -1).sum(axis=1)
    stream = torch.cuda.current_stream(dev)
    sim = Simulation(precision="fp64", device=dev, stream=stream.cuda_stream, **kw)
    sim.init(rho)
    sim.step(100)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    single_s = e0.elapsed_time(e1) * 1e-3
    _, mass, _ = sim.free_energy()
    single_drift = float(np.max(np.abs(mass - m0) / m0))
    sim.close()
    rec = dict(lattice="D1Q3", nx=p["nx"], ny=1, kT=p["kT"], gamma_mu=p["gamma_mu"])
    b = Batch([rec], p["a"], p["b"], p["kappa"], p["lam"], 2, tau=p["tau"], precision="fp64", device=dev,
              stream=stream.cuda_stream)
    b.init([rho])
    b.step(96)
    batch_s = b.time_steps(steps) * 1e-3
    r, _ = b.read(0)
    batch_drift = float(np.max(np.abs(r.reshape(2, -1).sum(axis=1) - m0) / m0))
    b.close()
    cu = 2 * p["nx"] * steps
    return {"workload": "D1Q3, 2 components, 256 nodes, FP64, slab (c1)", "steps": steps,
            "single_run": {"steps_per_s": steps / single_s, "value": cu / single_s / 1e6, "unit": UNIT,
                           "mass_drift_max_rel": single_drift},
            "resident_batch_of_one": {"steps_per_s": steps / batch_s, "value": cu / batch_s / 1e6, "unit": UNIT,
                                      "mass_drift_max_rel": batch_drift}}


def richardson(fun, x0, h):
    """Central difference with step h, extrapolated twice (h, h/2, h/4): O(h^6)."""
    d = [(fun(x0 + s) - fun(x0 - s)) / (2 * s) for s in (h, h / 2, h / 4)]
    r1 = (4 * d[1] - d[0]) / 3
    r2 = (4 * d[2] - d[1]) / 3
    return (16 * r2 - r1) / 15, d[0]


class MemPeak:
    """Lowest free device memory seen while a call runs (polled from a host thread every
    5 ms through cudaMemGetInfo): the call's peak device memory is the drop from before."""

    def __init__(self, torch, dev):
        import threading

        self.torch, self.dev = torch, dev
        self.free0 = torch.cuda.mem_get_info(dev)[0]
        self.low = self.free0
        self.stop_ev = threading.Event()
        self.th = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self.stop_ev.is_set():
            self.low = min(self.low, self.torch.cuda.mem_get_info(self.dev)[0])
            time.sleep(0.005)

    def __enter__(self):
        self.th.start()
        return self

    def __exit__(self, *exc):
        self.stop_ev.set()
        self.th.join()

    @property
    def peak_bytes(self):
        return self.free0 - self.low


def time_adjoint(torch, dev, steps_override=0, fd=True):
    """Workload c5: D2Q9, 2 components, 512^2, config-2 mixture and temperature with
    a12 = 0.75, 2000 steps checkpointed every 100; loss = sum (rho_T - rho_target)^2 with
    the target from the FP64 forward at a12 = 0.8.  Times one gradient (forward with
    checkpoints + backward) of the FP64 rollout and of the two FP32-storage rollouts (FP32
    adjoint, FP64 mu), and checks each against central finite differences of the FP64
    forward (h = 1e-4: plain and Richardson-extrapolated) and the FP32 ones against the
    FP64 adjoint.  Peak device memory of each rollout (checkpoints + backward) is polled."""
    import numpy as np

    import lbinputs
    from paper_1805_07251_gb300 import Simulation, capi

    p = lbinputs.base_params("c5")
    n, steps = p["nx"], (steps_override or p["steps"])
    ckpt = min(100, steps)
    rho0 = lbinputs.fields("c5")
    st = torch.cuda.current_stream(dev).cuda_stream

    def make(a12, kap, precision="fp64"):
        a = p["a"].copy()
        a[0, 1] = a[1, 0] = a12
        return Simulation(lattice="D2Q9", nx=n, ny=n, ncomp=2, tau=1.0, kT=p["kT"], gamma_mu=p["gamma_mu"], a=a,
                          kappa=np.full((2, 2), kap), lam=p["lam"], b=p["b"], precision=precision, device=dev,
                          stream=st)

    def final(a12, kap, r0):
        s = make(a12, kap)
        s.init(r0)
        s.step(steps)
        r, _ = s.moments()
        s.close()
        return r

    tgt = final(0.8, 0.1, rho0)

    def loss(a12, kap, r0=rho0):
        return float(np.sum((final(a12, kap, r0) - tgt) ** 2))

    v = 1e-2 * np.random.default_rng(5).normal(0, 1, rho0.shape)

    def gradient(precision):
        torch.cuda.synchronize(dev)
        with MemPeak(torch, dev) as mp:
            t0 = time.perf_counter()
            s = make(0.75, 0.1, precision)
            s.init(rho0)
            capi.lb_rollout_forward(s.ctx, steps, ckpt)
            r, _ = s.moments()
            t1 = time.perf_counter()
            rb0, g = capi.lb_rollout_backward(s.ctx, 2.0 * (r - tgt), 2)
            t2 = time.perf_counter()
            s.close()
        return dict(ga=g[1] + g[2], gk=g[4:8].sum(), gr=float(np.sum(rb0 * v)), total=t2 - t0, fwd=t1 - t0,
                    bwd=t2 - t1, mem=mp.peak_bytes)

    g64 = gradient("fp64")
    if not fd:
        out = {"steps": steps, "s_per_gradient": g64["total"], "backward_s": g64["bwd"],
               "peak_device_bytes": g64["mem"]}
        for precision in ("fp32_mixed", "fp32_dfmu"):
            g = gradient(precision)
            out[precision] = {"s_per_gradient": g["total"], "backward_s": g["bwd"], "peak_device_bytes": g["mem"]}
        return out
    fa, fa0 = richardson(lambda x: loss(x, 0.1), 0.75, 1e-4)
    fk, fk0 = richardson(lambda x: loss(0.75, x), 0.1, 1e-4)
    fr, fr0 = richardson(lambda t: loss(0.75, 0.1, rho0 + t * v), 0.0, 1e-4)
    out = {"workload": "D2Q9, 2 components, %dx%d, a12 = 0.75, gamma_mu = %.4g, %d steps, checkpoint every %d"
                       % (n, n, p["gamma_mu"], steps, ckpt),
           "s_per_gradient": g64["total"], "forward_s": g64["fwd"], "backward_s": g64["bwd"],
           "peak_device_bytes": g64["mem"],
           "grad_a12": g64["ga"], "fd_a12": fa, "rel_err_a12": abs(g64["ga"] - fa) / abs(fa),
           "grad_kappa": g64["gk"], "fd_kappa": fk, "rel_err_kappa": abs(g64["gk"] - fk) / abs(fk),
           "grad_rho0_dir": g64["gr"], "fd_rho0_dir": fr, "rel_err_rho0_dir": abs(g64["gr"] - fr) / abs(fr),
           "fd_plain_h1e-4": {"a12": fa0, "kappa": fk0, "rho0_dir": fr0},
           "rel_err_vs_plain_fd": {"a12": abs(g64["ga"] - fa0) / abs(fa0), "kappa": abs(g64["gk"] - fk0) / abs(fk0),
                                   "rho0_dir": abs(g64["gr"] - fr0) / abs(fr0)},
           "dtype": "f64 (forward and adjoint)"}
    for precision, key in (("fp32_mixed", "fp32_fp64mu"), ("fp32_dfmu", "fp32_dfmu")):
        g = gradient(precision)
        out[key] = {
            "dtype": "f32 storage and adjoint, %s mu in the forward, f64 mu in the adjoint"
                     % ("f64" if precision == "fp32_mixed" else "double-float"),
            "s_per_gradient": g["total"], "forward_s": g["fwd"], "backward_s": g["bwd"],
            "peak_device_bytes": g["mem"],
            "grad_a12": g["ga"], "grad_kappa": g["gk"], "grad_rho0_dir": g["gr"],
            "rel_diff_vs_fp64_adjoint": {"a12": abs(g["ga"] - g64["ga"]) / abs(g64["ga"]),
                                         "kappa": abs(g["gk"] - g64["gk"]) / abs(g64["gk"]),
                                         "rho0_dir": abs(g["gr"] - g64["gr"]) / abs(g64["gr"])},
            "rel_err_vs_fd_richardson": {"a12": abs(g["ga"] - fa) / abs(fa), "kappa": abs(g["gk"] - fk) / abs(fk),
                                         "rho0_dir": abs(g["gr"] - fr) / abs(fr)},
            "rel_err_vs_fd_plain_h1e-4": {"a12": abs(g["ga"] - fa0) / abs(fa0), "kappa": abs(g["gk"] - fk0) / abs(fk0),
                                          "rho0_dir": abs(g["gr"] - fr0) / abs(fr0)}}
    return out


def time_path(torch, Simulation, kw, rho, precision, steps, warmup, flush, dev):
    """A context of the precision, warmed up (single steps with the L2 flushed before each,
    then one call of `warmup` steps), and one pair of CUDA events per timed step."""
    stream = torch.cuda.current_stream(dev)
    sim = Simulation(precision=precision, device=dev, stream=stream.cuda_stream, tile=TILE,
                     kernel=kernel_for(precision), segments=SEGMENTS, **kw)
    sim.init(rho)
    for _ in range(warmup):
        flush.zero_()
        sim.step(1)
    sim.step(warmup)  # the chained launches too, untimed
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = sim.launches
    return sim, ev, launches0, stream


def time_sizes(torch, Simulation, dev, steps, warmup, flush):
    """The headline path (FP32 storage, double-float mu) on square lattices of the c2 recipe
    from 512^2 to 4096^2: K steps back to back in one lb_step call, and one launch per step
    with the L2 flushed before each.  What does not scale with the lattice (launch, the
    first wave of CTAs, the last) shows as the difference between the sizes."""
    import lbinputs

    p = lbinputs.base_params(WORKLOAD)
    peak_gbs, _ = read_peaks()
    out = {}
    for n in (512, 1024, 2048, 4096):
        kw = lbinputs.lib_kwargs(p, nx=n, ny=n)
        rho = lbinputs.fields(WORKLOAD, n, n)
        sim, ev, _, stream = time_path(torch, Simulation, kw, rho, "fp32_dfmu", steps, warmup, flush, dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        job = e0.elapsed_time(e1) / steps * 1e-3
        fl = sum(a.elapsed_time(b) for a, b in ev) / steps * 1e-3
        alg = 2 * n * n * 9 * 2 * 4
        out[str(n)] = {"nodes": n * n, "chain_rows": sim.chain_rows,
                       "job_us_per_step": job * 1e6, "job_frac": alg / job / 1e9 / peak_gbs,
                       "flushed_us_per_step": fl * 1e6, "flushed_frac": alg / fl / 1e9 / peak_gbs}
        sim.close()
    return {"sizes": out, "peak_gbs": peak_gbs, "steps": steps}


def kernel_for(precision):
    """The requested kernel organisation where it applies to the precision, else the
    library's choice (strips: FP32 storage; warp-specialised tiles: FP32-class mu)."""
    if precision == "fp64" or (KERNEL == "ws" and precision == "fp32_mixed"):
        return "auto"
    return KERNEL


TILE = None
KERNEL = "auto"
SEGMENTS = 0


def main():
    global TILE, KERNEL, SEGMENTS
    args = parse()
    if args.tile:
        TILE = tuple(int(v) for v in args.tile.lower().split("x"))
    KERNEL, SEGMENTS = args.kernel, args.segments
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3:
        args.warmup = 3

    import numpy as np
    import torch

    import lbinputs
    from paper_1805_07251_gb300 import Simulation, build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = local
    torch.cuda.set_device(dev)
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    build.build()

    p = lbinputs.base_params(WORKLOAD)
    kw = lbinputs.lib_kwargs(p)
    rho = lbinputs.fields(WORKLOAD)
    N, nodes = kw["ncomp"], kw["nx"] * kw["ny"]
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    peak_gbs, peak_kind = read_peaks()

    results = {}
    clocks = None
    if args.only in ("sweep", "c4", "adjoint", "c1", "sizes"):
        # profiling runs of one secondary workload: its JSON object alone
        if args.only == "sizes":
            out = time_sizes(torch, Simulation, dev, args.steps, args.warmup, flush)
        elif args.only == "sweep":
            out = time_sweep(torch, dev, "fp32_dfmu", args.steps, args.warmup, dist)
        elif args.only == "c4":
            out = time_c4(torch, dev, "fp32_dfmu", args.steps, args.warmup)
        elif args.only == "c1":
            out = time_c1(torch, dev, 10000)
        else:
            out = time_adjoint(torch, dev, args.adjoint_steps, fd=not args.no_fd)
        if rank == 0:
            print(json.dumps({"only": args.only, **out}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return 0
    HEAD = args.only or "fp32_dfmu"
    paths = [HEAD, "fp32_mixed", "fp32"] if args.no_fp64 else [HEAD, "fp32_mixed", "fp32", "fp64"]
    if args.only:
        paths = [args.only]
    for precision in paths:
        sim, ev, l0, stream = time_path(torch, Simulation, kw, rho, precision, args.steps, args.warmup, flush, dev)
        sampler = ClockSampler(dev) if precision == HEAD else None
        if sampler:
            sampler.start()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        # the job: K steps back to back in one lb_step call (chained launches where the
        # configuration chains); the state (both population buffers) exceeds the L2
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        job_ms = max_over_ranks(dist, e0.elapsed_time(e1), dev)
        # one plain launch per step, the L2 flushed before each, outside the events
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        if sampler:
            clocks = sampler.stop()
        launches = sim.launches - l0
        per = [a.elapsed_time(b) for a, b in ev]
        fl_ms = max_over_ranks(dist, float(sum(per)), dev) / args.steps
        kind, tile = sim.kernel
        ms = job_ms / args.steps
        elem = 8 if precision == "fp64" else 4
        alg_bytes = N * nodes * 9 * 2 * elem
        results[precision] = dict(
            value=job_throughput(world, N * nodes * args.steps, job_ms * 1e-3), ms=ms, launches=launches,
            alg_bytes=alg_bytes, achieved=alg_bytes / (ms * 1e-3) / 1e9, chained=sim.chain_rows > 0,
            evict_first=sim.chain_evict_first,
            kernel="%s %dx%d" % (kind, tile[0], tile[1]),
            flushed={"value": job_throughput(world, N * nodes, fl_ms * 1e-3), "unit": UNIT, "ms_per_step": fl_ms,
                     "achieved_gbs": alg_bytes / (fl_ms * 1e-3) / 1e9,
                     "frac": alg_bytes / (fl_ms * 1e-3) / 1e9 / peak_gbs})
        sim.close()

    sweep = None
    if not args.only and not args.no_sweep:
        sweep = time_sweep(torch, dev, HEAD, args.steps, args.warmup, dist)
    c1 = time_c1(torch, dev, 10000) if not args.only and rank == 0 else None
    c4 = None
    if not args.only and not args.no_c4:
        c4 = time_c4(torch, dev, HEAD, args.steps, args.warmup)
    adjoint = None
    if not args.only and not args.no_adjoint and rank == 0:
        from paper_1805_07251_gb300 import capi as _capi

        try:
            adjoint = time_adjoint(torch, dev)
        except _capi.LBError as e:  # a run of the gradient check left the domain
            adjoint = {"error": str(e)}
    e2e = None
    if not args.only:
        # end to end through the C ABI with host buffers: pinned host densities in,
        # K timesteps, densities and momenta back to pinned host memory
        sim = Simulation(precision=HEAD, device=dev, stream=torch.cuda.current_stream(dev).cuda_stream, **kw)
        h_rho = torch.from_numpy(rho).pin_memory().numpy()
        o_rho = torch.empty(rho.shape, dtype=torch.float64).pin_memory().numpy()
        o_mom = torch.empty((N, 2) + rho.shape[1:], dtype=torch.float64).pin_memory().numpy()
        from paper_1805_07251_gb300 import capi

        sim.init(h_rho)
        sim.step(args.warmup)
        capi.lb_read_moments(sim.ctx, o_rho, o_mom)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        capi.lb_init_fields(sim.ctx, h_rho)
        sim.step(args.steps)
        capi.lb_read_moments(sim.ctx, o_rho, o_mom)
        e2e_s = max_over_ranks(dist, time.perf_counter() - t0, dev)
        sim.close()
        e2e = {"value": job_throughput(world, N * nodes * args.steps, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(rho.nbytes // args.steps),
               "d2h_bytes_per_step": int((o_rho.nbytes + o_mom.nbytes) // args.steps),
               "note": "per-step bytes amortise one host->device field upload and one device->host "
                       "read of densities and momenta over the K timesteps of the job"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    head = results[HEAD]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[HEAD], "data": "synthetic",
        "config": {"workload": "D2Q9, 2 components, 1024x1024 periodic, spinodal mixture (c2), " + HEAD,
                   "nodes": nodes, "ncomp": N, "kernel": head["kernel"] + (", chained" if head["chained"] else "")
                   + (", input evict-first in the L2" if head["evict_first"] else ""),
                   "l2": "no flush: the job's state (two population buffers, %.0f MB) is larger than the 129 MB "
                         "L2; the K timed steps run back to back in one lb_step call between two CUDA events. "
                         "One launch per step with a 256 MB L2 flush before each: 'flushed'"
                         % (head["alg_bytes"] / 1e6),
                   "parallelism": "independent replica per GPU" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": head["achieved"], "peak": peak_gbs, "unit": "GB/s",
                     "frac": head["achieved"] / peak_gbs, "traffic": traffic_of(HEAD)[0],
                     "traffic_profile": traffic_of(HEAD)[1], "peak_kind": peak_kind,
                     "kernel": "%s<D2Q9, N=2, %s, %s>" % (
                         "lb_chain_kernel" if head["chained"] else
                         {"strips": "lb_strip_kernel", "ws": "lb_step_ws_kernel"}.get(head["kernel"].split()[0],
                                                                                      "lb_step_kernel"),
                         head["kernel"].split()[1], HEAD),
                     "alg_bytes_per_launch": head["alg_bytes"],
                     "frac_of_nominal": head["achieved"] / HBM_NOMINAL_GBS, "nominal_gbs": HBM_NOMINAL_GBS,
                     "duration": "K launches between two CUDA events / K",
                     "limiter": limiter_of(HEAD, head["alg_bytes"], peak_gbs)},
        "gpu_launches": head["launches"],
        "flushed": dict(head["flushed"], kernel="lb_step_kernel",
                        note="one lb_step(1) per timed step (a plain launch) between its own CUDA events, a 256 MB "
                             "L2 flush before each outside them (writes of a step drain during the next flush)"),
    }
    if "fp32_mixed" in results:
        fm = results["fp32_mixed"]
        line["config"]["fp64_mu_path"] = (
            "FP32 storage with mu in FP64 (the precision split of the method's FP32 variant taken "
            "literally): %.0f component-MLUPS, %.1f %% of the HBM peak; the headline replaces the FP64 "
            "mu by double-float (~44-bit) mu on the FP32 pipe" % (fm["value"], 100 * fm["achieved"] / peak_gbs))
    if e2e is not None:
        line["e2e"] = e2e
    if adjoint is not None:
        line["adjoint_rollout"] = adjoint
    if c1 is not None:
        line["c1_small_lattice"] = c1
    if c4 is not None:
        c4["roofline_hbm"].update({"peak": peak_gbs, "unit": "GB/s", "frac": c4["roofline_hbm"]["achieved"] / peak_gbs})
        line["four_components"] = c4
        line["gpu_launches"] += c4["gpu_launches"]
    if sweep is not None:
        if "fp64" in results:
            sweep["vs_fp64_single_run"] = sweep["value"] / results["fp64"]["value"]
        line["batched_sweep"] = sweep
        line["gpu_launches"] += sweep["gpu_launches"]
    for key, name in (("fp32_mixed", "fp32_fp64mu"), ("fp32", "fp32_fp32mu"), ("fp64", "fp64")):
        if key not in results or key == HEAD:
            continue
        rr = results[key]
        line[name] = {"value": rr["value"], "unit": UNIT, "ms_per_step": rr["ms"], "dtype": DTYPES[key],
                      "kernel": rr["kernel"] + (", chained" if rr["chained"] else ""),
                      "roofline_hbm": {"achieved": rr["achieved"], "peak": peak_gbs, "unit": "GB/s",
                                       "frac": rr["achieved"] / peak_gbs},
                      "flushed": rr["flushed"]}
        if key in FP64_PIPE and FP64_PIPE["digest"] == kernel_digest():
            line[name]["fp64_pipe_active"] = FP64_PIPE[key]
            line[name]["fp64_pipe_profile"] = FP64_PIPE["profile"]
        line["gpu_launches"] += rr["launches"]
    if clocks:
        line["clocks"] = clocks
    if world == 1 and not args.no_cpu_baseline and not args.only:
        # the oracle as it stands: OpenMP over rows on every host core (the headline CPU
        # figure), and one thread on a smaller sample
        cores = host_cores()
        va, dta, used = cpu_baseline_oracle(kw, 1024, 10, cores)
        v1, dt1, _ = cpu_baseline_oracle(kw, 256, 100, 1)
        line["cpu_baseline"] = {
            "value": va, "unit": UNIT, "cores": used, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"full 1024x1024 lattice of the same recipe, 10 oracle timesteps ({dta:.1f} s, "
                      f"OpenMP over rows, {used} threads)",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"256x256 lattice of the same recipe, 100 oracle timesteps ({dt1:.1f} s)"}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    del np
    return 0


if __name__ == "__main__":
    sys.exit(main())
