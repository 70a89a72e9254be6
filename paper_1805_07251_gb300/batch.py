"""Batched independent runs (phase-diagram sweeps) and the D2Q9 tile autotuner.

``Batch`` wraps the ``lb_batch_*`` C ABI: runs share the mixture, tau, the number of
components and the precision, and differ in lattice, size, kT and gamma_mu.  The
autotuner times each D2Q9 tile shape the library compiles on the batch itself, keeps
the fastest and caches the choice in a JSON file keyed by GPU name, precision,
component count and the batch's D2Q9 size profile (``LBVDW_AUTOTUNE_CACHE`` overrides
the file location).
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import capi
from . import make_params

TILES = [(32, 8), (64, 4), (32, 16), (64, 8)]
_DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")


class Batch:
    """Independent runs advanced together on one GPU (owns an ``lb_batch``)."""

    def __init__(self, runs, a, b, kappa, lam, ncomp, tau=1.0, precision="fp32_dfmu", force="log",
                 device=0, stream=None, tile=None):
        """runs: list of dicts with lattice ("D1Q3"/"D2Q9"), nx, ny, kT, gamma_mu and an
        optional kappa_scale (this run's kappa = kappa_scale * kappa; default 1)."""
        self.shared = make_params("D2Q9", 2, 2, ncomp, tau, 1.0, 1.0, a, kappa, lam, b, precision=precision,
                                  force=force, device=device, stream=stream, tile=tile)
        self.ncomp = ncomp
        self.runs = [dict(r) for r in runs]
        lat = {"D1Q3": capi.LB_D1Q3, "D2Q9": capi.LB_D2Q9}
        self.b = capi.lb_batch_create(self.shared, [(lat[r["lattice"]], r["nx"], r["ny"], r["kT"], r["gamma_mu"],
                                                      r.get("kappa_scale", 0.0)) for r in self.runs])

    def nodes(self, k):
        return self.runs[k]["nx"] * self.runs[k]["ny"]

    def total_component_nodes(self):
        return self.ncomp * sum(self.nodes(k) for k in range(len(self.runs)))

    def init(self, rho_list):
        flat = np.concatenate([np.ascontiguousarray(r, dtype=np.float64).ravel() for r in rho_list])
        capi.lb_batch_init(self.b, flat)

    def step(self, n):
        capi.lb_batch_step(self.b, n)

    def read(self, k):
        r = self.runs[k]
        d = 1 if r["lattice"] == "D1Q3" else 2
        rho = np.empty((self.ncomp, r["ny"], r["nx"]))
        mom = np.empty((self.ncomp, d, r["ny"], r["nx"]))
        capi.lb_batch_read(self.b, k, rho, mom)
        return rho, mom

    def errors(self):
        return capi.lb_batch_errors(self.b, len(self.runs))

    def set_tile(self, tx, ty):
        capi.lb_batch_set_tile(self.b, tx, ty)

    def time_steps(self, n):
        return capi.lb_batch_time_steps(self.b, n)

    @property
    def launches(self):
        return capi.lb_batch_launch_count(self.b)

    def close(self):
        if self.b is not None:
            capi.lb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# The campaign's automatic re-tuning of a run that leaves the density domain (Sec. VI: deep
# quenches were stabilised by widening interfaces -- larger kappa, which the bulk phases do
# not depend on -- and lowering gamma_mu): each retry multiplies kappa by KAPPA_STEP,
# divides gamma_mu by the same factor (the interface relation gamma_0 = 1 / (6 kappa rho_l))
# and widens the initial tanh profile by sqrt(KAPPA_STEP) (the interface width grows as
# sqrt(kappa)).
KAPPA_STEP = 4.0


def retune(rec):
    """A run record with the next stabilisation step applied."""
    r = dict(rec)
    r["kappa_scale"] = r.get("kappa_scale", 1.0) * KAPPA_STEP
    r["gamma_mu"] = r["gamma_mu"] / KAPPA_STEP
    r["width"] = r.get("width", 2.0) * KAPPA_STEP ** 0.5
    r["retuned"] = r.get("retuned", 0) + 1
    return r


def prescan(runs, fields_of, a, b, kappa, lam, ncomp, steps=3000, rounds=2, **batch_kw):
    """Scan every run for ``steps`` timesteps in one batch; runs that leave the density
    domain are re-tuned (``retune``) and scanned again, up to ``rounds`` times.  Returns
    the run records to use and the number of runs still failing the scan.  ``fields_of``
    maps a run record to its initial densities."""
    recs = [dict(r) for r in runs]
    todo = list(range(len(recs)))
    for rnd in range(rounds + 1):
        if not todo:
            break
        sub = [recs[k] for k in todo]
        bt = Batch(sub, a, b, kappa, lam, ncomp, **batch_kw)
        bt.init([fields_of(r) for r in sub])
        bt.step(steps)
        err = bt.errors()
        bt.close()
        failed = [k for k, e in zip(todo, err) if e]
        if rnd == rounds:
            return recs, len(failed)
        for k in failed:
            recs[k] = retune(recs[k])
        todo = failed
    return recs, 0


def _gpu_name(device):
    try:
        import torch

        return torch.cuda.get_device_name(device)
    except Exception:  # pragma: no cover
        return "unknown"


def autotune_key(batch, precision):
    sizes = sorted(r["nx"] * r["ny"] for r in batch.runs if r["lattice"] == "D2Q9")
    if not sizes:
        return None
    q = np.quantile(sizes, [0.1, 0.5, 0.9]).astype(int).tolist()
    return f"{_gpu_name(batch.shared.device)}|{precision}|N{batch.ncomp}|D2Q9x{len(sizes)}|{q}"


def autotune(batch, rho_list, precision, steps=64, cache_path=None, use_cache=True):
    """Pick the fastest D2Q9 tile for this batch; leaves the batch re-initialised with
    rho_list and the chosen tile.  Returns (tile, {tile: ms})."""
    cache_path = cache_path or os.environ.get("LBVDW_AUTOTUNE_CACHE", _DEFAULT_CACHE)
    key = autotune_key(batch, precision)
    if key is None:
        return None, {}
    cache = {}
    if os.path.exists(cache_path):
        try:
            with open(cache_path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        tile = tuple(cache[key]["tile"])
        batch.set_tile(*tile)
        batch.init(rho_list)
        return tile, cache[key].get("ms", {})
    times = {}
    for t in TILES:
        batch.set_tile(*t)
        batch.init(rho_list)
        batch.time_steps(8)                      # warm-up (graph capture, caches)
        times["x".join(map(str, t))] = batch.time_steps(steps)
    best = min(times, key=times.get)
    tile = tuple(int(v) for v in best.split("x"))
    batch.set_tile(*tile)
    batch.init(rho_list)
    cache[key] = {"tile": list(tile), "ms": times, "steps": steps}
    try:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        with open(cache_path, "w") as fh:
            json.dump(cache, fh, indent=1)
    except OSError:
        pass
    return tile, times
