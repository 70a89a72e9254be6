"""GB300 lattice Boltzmann for N-component van der Waals mixtures.

The compute path is the CUDA library ``_lib/liblbvdw.so`` behind the C ABI of
``include/lbvdw.h`` (fused timestep of Ridl & Wagner, arXiv:1805.07251,
Sec. III and V).  This package holds the ctypes binding (``capi``), a small
object wrapper (``Simulation``) and the build step (``build``).  PyTorch, when
present, only supplies the CUDA stream; every step of the method runs in the
library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import capi

__all__ = ["capi", "Simulation", "make_params"]

_LATTICES = {"D1Q3": capi.LB_D1Q3, "D2Q9": capi.LB_D2Q9}
_PRECISIONS = {"fp64": capi.LB_FP64, "fp32_mixed": capi.LB_FP32_MIXED, "fp32_dfmu": capi.LB_FP32_DFMU, "fp32": capi.LB_FP32}
_FORCES = {"log": capi.LB_FORCE_LOG, "nid": capi.LB_FORCE_NID}
_KERNELS = {"auto": capi.LB_KERNEL_AUTO, "tiles": capi.LB_KERNEL_TILES, "strips": capi.LB_KERNEL_STRIPS,
            "ws": capi.LB_KERNEL_WS}


def _current_stream(device):
    try:
        import torch
    except ImportError:  # pragma: no cover - torch is part of the runtime image
        return None
    if not torch.cuda.is_available():
        return None
    return torch.cuda.current_stream(device).cuda_stream


def make_params(lattice, nx, ny, ncomp, tau, kT, gamma_mu, a, kappa, lam, b,
                precision="fp64", force="log", device=0, stream=None, tile=None,
                rho_ref=None, check_every=0, kernel="auto", segments=0, tau_shear=0.0, tau_ghost=0.0):
    """Fill an ``lb_params`` struct from Python values (matrices as N x N).  ``kernel``:
    "auto", "tiles" or "strips" (organisation of the step kernel, see lb_kernel_kind).
    ``tau_shear`` / ``tau_ghost``: relaxation times of the shear and ghost moments (D2Q9;
    0 = tau, the BGK collision)."""
    p = capi.lb_default_params()
    p.lattice = _LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    p.nx, p.ny, p.ncomp = int(nx), int(ny), int(ncomp)
    p.precision = _PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.force_method = _FORCES[force] if isinstance(force, str) else int(force)
    p.check_every = int(check_every)
    p.tau, p.kT, p.gamma_mu = float(tau), float(kT), float(gamma_mu)
    N = int(ncomp)
    A = np.asarray(a, dtype=np.float64).reshape(N, N)
    K = np.asarray(kappa, dtype=np.float64).reshape(N, N)
    Lm = np.asarray(lam, dtype=np.float64).reshape(N, N)
    B = np.asarray(b, dtype=np.float64).reshape(N)
    for c in range(N):
        p.b[c] = B[c]
        if rho_ref is not None:
            p.rho_ref[c] = float(rho_ref[c])
        for cc in range(N):
            p.a[c * 4 + cc] = A[c, cc]
            p.kappa[c * 4 + cc] = K[c, cc]
            p.lambda_[c * 4 + cc] = Lm[c, cc]
    p.device = int(device)
    if tile is not None:
        p.tile_x, p.tile_y = int(tile[0]), int(tile[1])
    p.kernel = _KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    p.segments = int(segments)
    p.tau_shear, p.tau_ghost = float(tau_shear), float(tau_ghost)
    if stream is None:
        stream = _current_stream(device)
    p.stream = stream
    return p


class Simulation:
    """One lattice Boltzmann run on one GPU (owns an ``lb_ctx``)."""

    def __init__(self, **kw):
        self.params = make_params(**kw)
        self.lattice = self.params.lattice
        self.ncomp = self.params.ncomp
        self.nx, self.ny = self.params.nx, self.params.ny
        self.q = 3 if self.lattice == capi.LB_D1Q3 else 9
        self.d = 1 if self.lattice == capi.LB_D1Q3 else 2
        self.ctx = capi.lb_create(self.params)

    # shapes
    def rshape(self):
        return (self.ncomp, self.ny, self.nx)

    def mshape(self):
        return (self.ncomp, self.d, self.ny, self.nx)

    def init(self, rho, mom=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.rshape())
        if mom is not None:
            mom = np.ascontiguousarray(mom, dtype=np.float64).reshape(self.mshape())
        capi.lb_init_fields(self.ctx, rho, mom)

    def init_dev(self, rho_ptr, mom_ptr=None):
        capi.lb_init_fields_dev(self.ctx, rho_ptr, mom_ptr)

    def step(self, n=1):
        capi.lb_step(self.ctx, n)

    def moments(self):
        rho = np.empty(self.rshape())
        mom = np.empty(self.mshape())
        capi.lb_read_moments(self.ctx, rho, mom)
        return rho, mom

    def moments_dev(self, rho_ptr, mom_ptr=None):
        capi.lb_read_moments_dev(self.ctx, rho_ptr, mom_ptr)

    def free_energy(self):
        return capi.lb_free_energy(self.ctx, self.ncomp)

    def save_state(self):
        return capi.lb_save_state(self.ctx)

    def load_state(self, buf):
        capi.lb_load_state(self.ctx, buf)

    @property
    def steps(self):
        return capi.lb_step_count(self.ctx)

    @property
    def launches(self):
        return capi.lb_launch_count(self.ctx)

    @property
    def chain_rows(self):
        """Tile rows of a chained step that set flags (0: lb_step does not chain)."""
        return capi.lb_chain_rows(self.ctx)

    @property
    def chain_evict_first(self):
        """Whether the chained steps mark their input evict-first in the L2 (lb_chain_evict_first)."""
        return bool(capi.lb_chain_evict_first(self.ctx))

    @property
    def kernel(self):
        """Organisation of the step kernel chosen by lb_create: ("tiles" or "strips", tile)."""
        p = capi.lb_get_params(self.ctx)
        kind = {capi.LB_KERNEL_TILES: "tiles", capi.LB_KERNEL_STRIPS: "strips", capi.LB_KERNEL_WS: "ws"}[p.kernel]
        return kind, (p.tile_x, p.tile_y)

    def close(self):
        if self.ctx is not None:
            capi.lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
