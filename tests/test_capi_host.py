"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function that include/lbvdw.h declares, and the pure-host entry
points behave as documented."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = "".join(open(os.path.join(ROOT, "include", h)).read()
                  for h in sorted(os.listdir(os.path.join(ROOT, "include"))) if h.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(lb_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_07251_gb300 import build, capi

    build.build()
    return capi.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lb_create", "lb_init_fields", "lb_step", "lb_read_moments", "lb_free_energy",
                     "lb_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1805_07251_gb300 import capi

    out = subprocess.run(["nm", "-D", "--defined-only", capi.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(lb_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_status_strings_and_defaults(lib):
    from paper_1805_07251_gb300 import capi

    assert capi.status_str(capi.LB_OK) == "LB_OK"
    assert capi.status_str(capi.LB_E_DOMAIN) == "LB_E_DOMAIN"
    assert capi.status_str(99) == "LB_E_UNKNOWN"
    p = capi.lb_default_params()
    assert p.abi == capi.LBVDW_ABI and p.tau == 1.0 and p.ncomp == 2 and p.lattice == capi.LB_D2Q9
    assert ctypes.sizeof(capi.lb_params) == 8 * 4 + 8 * 3 + 8 * (16 * 3 + 8) + 4 * 6 + 8 + 8 * 2
    assert p.tau_shear == 0.0 and p.tau_ghost == 0.0


def test_null_arguments_are_rejected_without_cuda(lib):
    from paper_1805_07251_gb300 import capi

    assert lib.lb_create(None, None) == capi.LB_E_INVALID
    assert lib.lb_step(None, 1) == capi.LB_E_INVALID
    assert lib.lb_destroy(None) == capi.LB_OK
    assert lib.lb_last_error(None) == b"NULL context"
    # invalid parameter sets fail validation before any CUDA call
    p = capi.lb_default_params()
    out = ctypes.c_void_p()
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID  # b = 0
    p.b[0] = p.b[1] = 0.3
    p.a[1], p.a[4] = 0.5, 0.4                                                  # a not symmetric
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    p.a[4] = 0.5
    p.tau = 0.5
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    p.tau = 1.0
    p.ncomp = 5
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    p.ncomp = 2
    p.lattice = capi.LB_D1Q3  # ny must be 1
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    # streaming strips: D2Q9 with FP32 storage, nx % 32 == 0, ny % 8 == 0 (1-2 components)
    p.lattice = capi.LB_D2Q9
    p.kernel = 3
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    p.kernel = capi.LB_KERNEL_STRIPS                     # FP64 storage has no strips
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    p.precision = capi.LB_FP32_DFMU
    p.nx = 40
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    p.nx, p.ny = 64, 60
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    p.ny = 64
    p.tile_x, p.tile_y = 64, 4
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    p.tile_x, p.tile_y = 32, 8
    p.segments = -1
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID


def test_batches_reject_the_fp32_mu_precision_without_cuda(lib):
    # LB_FP32 (FP32 mu) serves single runs only; a batch asking for it is refused
    # before any CUDA call
    from paper_1805_07251_gb300 import capi

    p = capi.lb_default_params()
    p.b[0] = p.b[1] = 0.3
    p.precision = capi.LB_FP32
    runs = (capi.lb_run_desc * 1)()
    runs[0].lattice, runs[0].nx, runs[0].ny, runs[0].kT, runs[0].gamma_mu = capi.LB_D2Q9, 64, 64, 1.0 / 3.0, 0.1
    out = ctypes.c_void_p()
    assert lib.lb_batch_create(ctypes.byref(p), runs, 1, ctypes.byref(out)) == capi.LB_E_INVALID
    assert lib.lb_batch_create(None, runs, 1, ctypes.byref(out)) == capi.LB_E_INVALID


def test_relaxation_times_are_validated_without_cuda(lib):
    # the moment-space collision: 1/2 < tau_shear <= tau, tau_ghost > 1/2, D2Q9 tiles of
    # 32 x 8 only; batches run BGK.  Each case fails validation before any CUDA call.
    from paper_1805_07251_gb300 import capi

    def base():
        p = capi.lb_default_params()
        p.b[0] = p.b[1] = 0.3
        p.tau = 1.0
        return p

    out = ctypes.c_void_p()
    for ts, tg in ((1.2, 0.0), (0.5, 0.0), (0.0, 0.5), (float("nan"), 0.0), (0.7, float("inf"))):
        p = base()
        p.tau_shear, p.tau_ghost = ts, tg
        assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    p = base()
    p.tau_shear = 0.7
    p.lattice, p.ny = capi.LB_D1Q3, 1                    # no shear moments in D1Q3
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    p = base()
    p.tau_ghost = 0.8
    p.tile_x, p.tile_y = 64, 4
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    p = base()
    p.tau_shear = 0.7
    p.precision, p.kernel = capi.LB_FP32_DFMU, capi.LB_KERNEL_STRIPS
    assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID
    p = base()
    p.tau_shear = 0.7
    runs = (capi.lb_run_desc * 1)()
    runs[0].lattice, runs[0].nx, runs[0].ny, runs[0].kT, runs[0].gamma_mu = capi.LB_D2Q9, 64, 64, 1.0 / 3.0, 0.1
    assert lib.lb_batch_create(ctypes.byref(p), runs, 1, ctypes.byref(out)) == capi.LB_E_INVALID


def test_warp_specialised_kernel_is_validated_without_cuda(lib):
    # LB_KERNEL_WS: D2Q9, two components, FP32 storage with an FP32-class mu, 32 x 8 tiles
    from paper_1805_07251_gb300 import capi

    out = ctypes.c_void_p()
    for change in ({"ncomp": 3}, {"precision": capi.LB_FP64}, {"precision": capi.LB_FP32_MIXED},
                   {"tile_x": 64, "tile_y": 4}, {"lattice": capi.LB_D1Q3, "ny": 1}):
        p = capi.lb_default_params()
        p.b[0] = p.b[1] = p.b[2] = 0.3
        p.precision, p.kernel = capi.LB_FP32_DFMU, capi.LB_KERNEL_WS
        for k, v in change.items():
            setattr(p, k, v)
        assert lib.lb_create(ctypes.byref(p), ctypes.byref(out)) == capi.LB_E_INVALID, change


def test_lattice_size_limits_are_validated_without_cuda(lib):
    # FP32 storage addresses a component's Q planes with 32-bit element offsets, so
    # Q nx ny must stay below 2^32; every precision needs nx ny <= 2^31.  A size at the
    # limit fails validation (LB_E_INVALID) before any CUDA call; one node row below it
    # passes validation (on a host without a GPU it then fails at the first CUDA call; where
    # a GPU has the memory the context is created, and destroyed again here).
    from paper_1805_07251_gb300 import capi

    out = ctypes.c_void_p()

    def create(precision, lattice, nx, ny):
        p = capi.lb_default_params()
        p.b[0] = p.b[1] = 0.3
        p.precision, p.lattice, p.nx, p.ny = precision, lattice, nx, ny
        st = lib.lb_create(ctypes.byref(p), ctypes.byref(out))
        if st == capi.LB_OK:
            lib.lb_destroy(out)
        return st

    nx = 32768  # 9 nx ny = 2^32 at ny = 2^32 / (9 nx), which is not an integer
    ny_lim = -(-(1 << 32) // (9 * nx))  # smallest ny with 9 nx ny >= 2^32
    assert 9 * nx * ny_lim >= 1 << 32 > 9 * nx * (ny_lim - 1)
    for prec in (capi.LB_FP32_DFMU, capi.LB_FP32_MIXED, capi.LB_FP32):
        assert create(prec, capi.LB_D2Q9, nx, ny_lim) == capi.LB_E_INVALID
    assert create(capi.LB_FP32_DFMU, capi.LB_D2Q9, nx, ny_lim - 1) != capi.LB_E_INVALID
    nx3 = -(-(1 << 32) // 3)  # D1Q3: 3 nx >= 2^32
    assert create(capi.LB_FP32_DFMU, capi.LB_D1Q3, nx3, 1) == capi.LB_E_INVALID
    # FP64: 64-bit offsets, nx ny <= 2^31 only (2^31 FP64 nodes exceed any GPU's memory)
    assert create(capi.LB_FP64, capi.LB_D2Q9, 1 << 16, (1 << 15) + 1) == capi.LB_E_INVALID
    assert create(capi.LB_FP64, capi.LB_D2Q9, 1 << 16, 1 << 15) not in (capi.LB_E_INVALID, capi.LB_OK)
