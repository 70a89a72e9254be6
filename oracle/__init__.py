"""CPU oracle for the multicomponent van der Waals lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this package; the library under
``paper_1805_07251_gb300`` never imports it, and it never imports that
library.  ``lbvdw_oracle.c`` holds the lattice Boltzmann timestep (plain FP64
loops in the order of Ridl & Wagner, Sec. III and Sec. V); ``thermo.py`` holds
the bulk thermodynamics (Sec. II) and the coexistence solvers the step is
pinned against.

The ctypes wrapper below compiles ``lbvdw_oracle.c`` with plain ``gcc -O2``
(no fast-math, no FMA contraction, OpenMP over rows when the compiler has it) on
first use, or uses the copy that ``__graft_entry__.build()`` compiled.  The
number of threads never changes a result (``set_threads``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbvdw_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liblbvdw_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_E_INVALID, ORC_E_NOMEM, ORC_E_DOMAIN = 0, 1, 2, 4


class OracleError(RuntimeError):
    pass


class OracleDomainError(OracleError):
    """rho^c <= 0 or eta = 1 - sum b rho <= 0 met during a step."""


class _Params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("ncomp", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("gamma_mu", ctypes.c_double),
        ("a", ctypes.c_double * 16),
        ("kappa", ctypes.c_double * 16),
        ("lam", ctypes.c_double * 16),
        ("b", ctypes.c_double * 4),
        ("force_method", ctypes.c_int),
        ("psi_sign", ctypes.c_double),
        ("mrt", ctypes.c_int),
        ("tau_s", ctypes.c_double),
        ("tau_g", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True, text=True)
        if r.returncode != 0:            # no OpenMP runtime: the same code, one thread
            subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.orc_run.argtypes = [P, dp, ctypes.c_long]
            lib.orc_moments.argtypes = [P, dp, dp, dp]
            lib.orc_mu.argtypes = [P, dp, dp]
            lib.orc_forces.argtypes = [P, dp, dp, dp]
            lib.orc_equilibrium.argtypes = [P, dp, dp, dp]
            lib.orc_free_energy.argtypes = [P, dp, dp, dp]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            for fn in (lib.orc_run, lib.orc_moments, lib.orc_mu, lib.orc_forces,
                       lib.orc_equilibrium, lib.orc_free_energy, lib.orc_set_threads):
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads the oracle's stages use (n < 1: leave unchanged); returns the number in
    effect (1 when built without OpenMP)."""
    return int(_load().orc_set_threads(int(n)))


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc == ORC_OK:
        return
    if rc == ORC_E_DOMAIN:
        raise OracleDomainError(f"{what}: density or eta left its domain")
    raise OracleError(f"{what}: error {rc}")


class Lattice:
    """Plain parameter record for the oracle (no arithmetic of the method)."""

    def __init__(self, lattice, nx, ny, ncomp, tau, kT, gamma_mu, a, kappa, lam, b,
                 force_method=0, psi_sign=-1.0, tau_s=None, tau_g=None):
        self.lattice = {"D1Q3": 1, "D2Q9": 2}.get(lattice, lattice)
        self.nx, self.ny, self.ncomp = int(nx), int(ny), int(ncomp)
        self.q = 3 if self.lattice == 1 else 9
        self.d = 1 if self.lattice == 1 else 2
        self.tau, self.kT, self.gamma_mu = float(tau), float(kT), float(gamma_mu)
        self.a = np.asarray(a, dtype=np.float64).reshape(ncomp, ncomp)
        self.kappa = np.asarray(kappa, dtype=np.float64).reshape(ncomp, ncomp)
        self.lam = np.asarray(lam, dtype=np.float64).reshape(ncomp, ncomp)
        self.b = np.asarray(b, dtype=np.float64).reshape(ncomp)
        self.force_method = int(force_method)
        self.psi_sign = float(psi_sign)
        # distinct relaxation times of the shear and ghost moments (D2Q9): None = tau (BGK)
        self.mrt = int(tau_s is not None or tau_g is not None)
        self.tau_s = float(tau if tau_s is None else tau_s)
        self.tau_g = float(tau if tau_g is None else tau_g)

    def _c(self):
        p = _Params()
        p.lattice, p.nx, p.ny, p.ncomp = self.lattice, self.nx, self.ny, self.ncomp
        p.tau, p.kT, p.gamma_mu = self.tau, self.kT, self.gamma_mu
        N = self.ncomp
        for c in range(N):
            p.b[c] = self.b[c]
            for cc in range(N):
                p.a[c * 4 + cc] = self.a[c, cc]
                p.kappa[c * 4 + cc] = self.kappa[c, cc]
                p.lam[c * 4 + cc] = self.lam[c, cc]
        p.force_method = self.force_method
        p.psi_sign = self.psi_sign
        p.mrt, p.tau_s, p.tau_g = self.mrt, self.tau_s, self.tau_g
        return p

    # shapes -------------------------------------------------------------
    @property
    def nodes(self):
        return self.nx * self.ny

    def fshape(self):
        return (self.ncomp, self.q, self.ny, self.nx)

    def rshape(self):
        return (self.ncomp, self.ny, self.nx)

    def mshape(self):
        return (self.ncomp, self.d, self.ny, self.nx)

    # calls --------------------------------------------------------------
    def equilibrium(self, rho, mom=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.rshape())
        if mom is not None:
            mom = np.ascontiguousarray(mom, dtype=np.float64).reshape(self.mshape())
        f = np.empty(self.fshape(), dtype=np.float64)
        p = self._c()
        _check(_load().orc_equilibrium(ctypes.byref(p), _dptr(rho), _dptr(mom), _dptr(f)),
               "equilibrium")
        return f

    def run(self, f, nsteps):
        """Advance a copy of f by nsteps timesteps and return it."""
        f = np.array(f, dtype=np.float64, order="C", copy=True).reshape(self.fshape())
        p = self._c()
        _check(_load().orc_run(ctypes.byref(p), _dptr(f), int(nsteps)), "run")
        return f

    def moments(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.fshape())
        rho = np.empty(self.rshape())
        mom = np.empty(self.mshape())
        p = self._c()
        _check(_load().orc_moments(ctypes.byref(p), _dptr(f), _dptr(rho), _dptr(mom)), "moments")
        return rho, mom

    def mu(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.rshape())
        mu = np.empty(self.rshape())
        p = self._c()
        _check(_load().orc_mu(ctypes.byref(p), _dptr(rho), _dptr(mu)), "mu")
        return mu

    def forces(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.fshape())
        G = np.empty(self.mshape())
        Gmu = np.empty(self.mshape())
        p = self._c()
        _check(_load().orc_forces(ctypes.byref(p), _dptr(f), _dptr(G), _dptr(Gmu)), "forces")
        return G, Gmu

    def free_energy(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.rshape())
        F = np.zeros(1)
        mass = np.zeros(4)
        p = self._c()
        _check(_load().orc_free_energy(ctypes.byref(p), _dptr(rho), _dptr(F), _dptr(mass)),
               "free_energy")
        return float(F[0]), mass[: self.ncomp].copy()
