"""ctypes binding of the C ABI in include/lbvdw.h (argument marshalling only).

Every function keeps the C name and signature; arrays are passed as NumPy
host arrays (``lb_init_fields``, ``lb_read_moments`` ...) or as raw device
addresses (``*_dev``), e.g. ``torch.Tensor.data_ptr()``.  The library is the
in-tree ``_lib/liblbvdw.so`` built by ``build.py``; loading fails loudly if it
is missing -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "liblbvdw.so")

LBVDW_ABI = 3
LB_OK, LB_E_INVALID, LB_E_NOMEM, LB_E_CUDA, LB_E_DOMAIN, LB_E_TIMEOUT, LB_E_STATE = range(7)
LB_D1Q3, LB_D2Q9 = 1, 2
LB_FP64, LB_FP32_MIXED, LB_FP32_DFMU, LB_FP32 = 0, 1, 2, 3
LB_FORCE_LOG, LB_FORCE_NID = 0, 1
LB_KERNEL_AUTO, LB_KERNEL_TILES, LB_KERNEL_STRIPS, LB_KERNEL_WS = 0, 1, 2, 3


class lb_run_desc(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32),
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("kT", ctypes.c_double),
        ("gamma_mu", ctypes.c_double),
        ("kappa_scale", ctypes.c_double),
    ]


class lb_params(ctypes.Structure):
    _fields_ = [
        ("abi", ctypes.c_uint32),
        ("lattice", ctypes.c_int32),
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("ncomp", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("force_method", ctypes.c_int32),
        ("check_every", ctypes.c_int32),
        ("tau", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("gamma_mu", ctypes.c_double),
        ("a", ctypes.c_double * 16),
        ("kappa", ctypes.c_double * 16),
        ("lambda_", ctypes.c_double * 16),
        ("b", ctypes.c_double * 4),
        ("rho_ref", ctypes.c_double * 4),
        ("device", ctypes.c_int32),
        ("tile_x", ctypes.c_int32),
        ("tile_y", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("segments", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("tau_shear", ctypes.c_double),
        ("tau_ghost", ctypes.c_double),
    ]


_lib = None
_DP = ctypes.POINTER(ctypes.c_double)


class LBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_str(status)}: {msg}")
        self.status = status


def load():
    """Load liblbvdw.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run paper_1805_07251_gb300.build.build())")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER(lb_params)
    C = ctypes.c_void_p
    sig = {
        "lb_default_params": (None, [P]),
        "lb_create": (ctypes.c_int, [P, ctypes.POINTER(C)]),
        "lb_init_fields": (ctypes.c_int, [C, _DP, _DP]),
        "lb_init_fields_dev": (ctypes.c_int, [C, C, C]),
        "lb_step": (ctypes.c_int, [C, ctypes.c_int64]),
        "lb_read_moments": (ctypes.c_int, [C, _DP, _DP]),
        "lb_read_moments_dev": (ctypes.c_int, [C, C, C]),
        "lb_free_energy": (ctypes.c_int, [C, _DP, _DP, _DP]),
        "lb_state_bytes": (ctypes.c_size_t, [C]),
        "lb_save_state": (ctypes.c_int, [C, C, ctypes.c_size_t]),
        "lb_load_state": (ctypes.c_int, [C, C, ctypes.c_size_t]),
        "lb_step_count": (ctypes.c_int64, [C]),
        "lb_launch_count": (ctypes.c_int64, [C]),
        "lb_chain_rows": (ctypes.c_int32, [C]),
        "lb_chain_evict_first": (ctypes.c_int32, [C]),
        "lb_get_params": (ctypes.c_int, [C, ctypes.POINTER(lb_params)]),
        "lb_destroy": (ctypes.c_int, [C]),
        "lb_status_str": (ctypes.c_char_p, [ctypes.c_int]),
        "lb_last_error": (ctypes.c_char_p, [C]),
        "lb_selftest_log": (ctypes.c_int, [ctypes.c_int32, _DP, ctypes.c_int64, _DP, _DP, _DP]),
        "lb_selftest_recip": (ctypes.c_int, [ctypes.c_int32, _DP, ctypes.c_int64, _DP]),
        "lb_selftest_wait": (ctypes.c_int, [ctypes.c_int32, ctypes.c_uint32, ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_uint32)]),
        "lb_selftest_flag_wait": (ctypes.c_int, [ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32,
                                                 ctypes.POINTER(ctypes.c_uint32)]),
        "lb_free_energy_noalloc": (ctypes.c_int, [P, C, C]),
        "lb_batch_create": (ctypes.c_int, [P, ctypes.POINTER(lb_run_desc), ctypes.c_int32, ctypes.POINTER(C)]),
        "lb_batch_init": (ctypes.c_int, [C, _DP]),
        "lb_batch_step": (ctypes.c_int, [C, ctypes.c_int64]),
        "lb_batch_read": (ctypes.c_int, [C, ctypes.c_int32, _DP, _DP]),
        "lb_batch_errors": (ctypes.c_int, [C, ctypes.POINTER(ctypes.c_uint32)]),
        "lb_batch_set_tile": (ctypes.c_int, [C, ctypes.c_int32, ctypes.c_int32]),
        "lb_batch_time_steps": (ctypes.c_int, [C, ctypes.c_int32, _DP]),
        "lb_batch_step_count": (ctypes.c_int64, [C]),
        "lb_batch_launch_count": (ctypes.c_int64, [C]),
        "lb_batch_last_error": (ctypes.c_char_p, [C]),
        "lb_batch_destroy": (ctypes.c_int, [C]),
        "lb_rollout_forward": (ctypes.c_int, [C, ctypes.c_int64, ctypes.c_int32]),
        "lb_rollout_backward": (ctypes.c_int, [C, _DP, _DP, _DP]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_str(s):
    return load().lb_status_str(int(s)).decode()


def _dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


def _check(ctx, rc, what):
    if rc != LB_OK:
        msg = load().lb_last_error(ctx).decode() if ctx else ""
        raise LBError(rc, f"{what}: {msg}")


# --- thin wrappers with the C names -----------------------------------------

def lb_default_params():
    p = lb_params()
    load().lb_default_params(ctypes.byref(p))
    return p


def lb_create(p):
    out = ctypes.c_void_p()
    rc = load().lb_create(ctypes.byref(p), ctypes.byref(out))
    if rc != LB_OK:
        raise LBError(rc, "lb_create rejected the parameters")
    return out


def lb_init_fields(ctx, rho, mom=None):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    mom = None if mom is None else np.ascontiguousarray(mom, dtype=np.float64)
    _check(ctx, load().lb_init_fields(ctx, _dp(rho), _dp(mom)), "lb_init_fields")


def lb_init_fields_dev(ctx, rho_ptr, mom_ptr=None):
    _check(ctx, load().lb_init_fields_dev(ctx, ctypes.c_void_p(rho_ptr),
                                          ctypes.c_void_p(mom_ptr) if mom_ptr else None),
           "lb_init_fields_dev")


def lb_step(ctx, nsteps):
    _check(ctx, load().lb_step(ctx, int(nsteps)), "lb_step")


def lb_read_moments(ctx, rho_out, mom_out=None):
    _check(ctx, load().lb_read_moments(ctx, _dp(rho_out), _dp(mom_out)), "lb_read_moments")


def lb_read_moments_dev(ctx, rho_ptr, mom_ptr=None):
    _check(ctx, load().lb_read_moments_dev(ctx, ctypes.c_void_p(rho_ptr),
                                           ctypes.c_void_p(mom_ptr) if mom_ptr else None),
           "lb_read_moments_dev")


def lb_free_energy(ctx, ncomp):
    F = np.zeros(1)
    mass = np.zeros(ncomp)
    mom = np.zeros(2)
    _check(ctx, load().lb_free_energy(ctx, _dp(F), _dp(mass), _dp(mom)), "lb_free_energy")
    return float(F[0]), mass, mom


def lb_state_bytes(ctx):
    return int(load().lb_state_bytes(ctx))


def lb_save_state(ctx):
    buf = np.empty(lb_state_bytes(ctx), dtype=np.uint8)
    _check(ctx, load().lb_save_state(ctx, buf.ctypes.data, buf.nbytes), "lb_save_state")
    return buf


def lb_load_state(ctx, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(ctx, load().lb_load_state(ctx, buf.ctypes.data, buf.nbytes), "lb_load_state")


def lb_step_count(ctx):
    return int(load().lb_step_count(ctx))


def lb_launch_count(ctx):
    return int(load().lb_launch_count(ctx))


def lb_chain_rows(ctx):
    return int(load().lb_chain_rows(ctx))


def lb_chain_evict_first(ctx):
    return int(load().lb_chain_evict_first(ctx))


def lb_get_params(ctx):
    p = lb_params()
    _check(ctx, load().lb_get_params(ctx, ctypes.byref(p)), "lb_get_params")
    return p


def lb_destroy(ctx):
    load().lb_destroy(ctx)


def lb_last_error(ctx):
    return load().lb_last_error(ctx).decode()


def lb_selftest_wait(device, polls, arrive):
    flag = ctypes.c_uint32(0)
    rc = load().lb_selftest_wait(int(device), int(polls), int(arrive), ctypes.byref(flag))
    if rc != LB_OK:
        raise LBError(rc, "lb_selftest_wait")
    return int(flag.value)


def lb_selftest_flag_wait(device, wait_ns, set_flag):
    flag = ctypes.c_uint32(0)
    rc = load().lb_selftest_flag_wait(int(device), int(wait_ns), int(set_flag), ctypes.byref(flag))
    if rc != LB_OK:
        raise LBError(rc, "lb_selftest_flag_wait")
    return int(flag.value)


def lb_selftest_log(device, x):
    """Table-driven FP64 log, double-float log and CUDA's log of x on the device."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    o = [np.empty_like(x) for _ in range(3)]
    rc = load().lb_selftest_log(int(device), _dp(x), x.size, _dp(o[0]), _dp(o[1]), _dp(o[2]))
    if rc != LB_OK:
        raise LBError(rc, "lb_selftest_log")
    return o


def lb_selftest_recip(device, x):
    """The double-float reciprocal of the chemical potential (1/eta) of x on the device."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    o = np.empty_like(x)
    rc = load().lb_selftest_recip(int(device), _dp(x), x.size, _dp(o))
    if rc != LB_OK:
        raise LBError(rc, "lb_selftest_recip")
    return o


def lb_free_energy_noalloc(p, f_ptr, out_ptr):
    """Enqueue the no-allocation diagnostics on p.stream (device pointers in and out)."""
    rc = load().lb_free_energy_noalloc(ctypes.byref(p), ctypes.c_void_p(f_ptr), ctypes.c_void_p(out_ptr))
    if rc != LB_OK:
        raise LBError(rc, "lb_free_energy_noalloc")


# --- batched runs -------------------------------------------------------------

def _bcheck(b, rc, what):
    if rc != LB_OK:
        msg = load().lb_batch_last_error(b).decode() if b else ""
        raise LBError(rc, f"{what}: {msg}")


def lb_batch_create(shared, runs):
    """runs: sequence of (lattice, nx, ny, kT, gamma_mu[, kappa_scale])."""
    arr = (lb_run_desc * len(runs))()
    for k, run in enumerate(runs):
        lat, nx, ny, kT, g = run[:5]
        arr[k].lattice, arr[k].nx, arr[k].ny, arr[k].kT, arr[k].gamma_mu = int(lat), int(nx), int(ny), kT, g
        arr[k].kappa_scale = float(run[5]) if len(run) > 5 else 0.0
    out = ctypes.c_void_p()
    rc = load().lb_batch_create(ctypes.byref(shared), arr, len(runs), ctypes.byref(out))
    if rc != LB_OK:
        raise LBError(rc, "lb_batch_create rejected the runs")
    return out


def lb_batch_init(b, rho_all):
    rho_all = np.ascontiguousarray(rho_all, dtype=np.float64)
    _bcheck(b, load().lb_batch_init(b, _dp(rho_all)), "lb_batch_init")


def lb_batch_step(b, nsteps):
    _bcheck(b, load().lb_batch_step(b, int(nsteps)), "lb_batch_step")


def lb_batch_read(b, run, rho_out, mom_out=None):
    _bcheck(b, load().lb_batch_read(b, int(run), _dp(rho_out), _dp(mom_out)), "lb_batch_read")


def lb_batch_errors(b, nruns):
    flags = (ctypes.c_uint32 * nruns)()
    _bcheck(b, load().lb_batch_errors(b, flags), "lb_batch_errors")
    return np.array(flags[:], dtype=np.uint32)


def lb_batch_set_tile(b, tx, ty):
    _bcheck(b, load().lb_batch_set_tile(b, int(tx), int(ty)), "lb_batch_set_tile")


def lb_batch_time_steps(b, nsteps):
    ms = np.zeros(1)
    _bcheck(b, load().lb_batch_time_steps(b, int(nsteps), _dp(ms)), "lb_batch_time_steps")
    return float(ms[0])


def lb_batch_step_count(b):
    return int(load().lb_batch_step_count(b))


def lb_batch_launch_count(b):
    return int(load().lb_batch_launch_count(b))


def lb_batch_destroy(b):
    load().lb_batch_destroy(b)


# --- adjoint rollout ----------------------------------------------------------

def lb_rollout_forward(ctx, nsteps, ckpt_every):
    _check(ctx, load().lb_rollout_forward(ctx, int(nsteps), int(ckpt_every)), "lb_rollout_forward")


def lb_rollout_backward(ctx, rho_bar_T, ncomp):
    """Returns (rho_bar_0, grad) with grad = [dL/da (N*N), dL/dkappa (N*N), dL/db (N)]."""
    rho_bar_T = np.ascontiguousarray(rho_bar_T, dtype=np.float64)
    rb0 = np.empty_like(rho_bar_T)
    grad = np.empty(2 * ncomp * ncomp + ncomp)
    _check(ctx, load().lb_rollout_backward(ctx, _dp(rho_bar_T), _dp(rb0), _dp(grad)), "lb_rollout_backward")
    return rb0, grad
