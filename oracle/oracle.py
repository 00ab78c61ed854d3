"""ctypes wrapper around the FP64 CPU oracle (``les_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is the correctness reference for the CUDA
library.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module; the library never does.

Parity status of each routine (see the pins in ``tests/test_oracle_*.py``):
  * press (rhs, red-black SOR, residual, gauge) -- pinned: textbook Laplacian
    and graph-Laplacian matrices, dense direct solve, manufactured solutions
    with 2nd-order convergence, colour order, matrix-form SOR.
  * velnw (projection) -- pinned: discrete divergence equals dt * residual,
    |div u| <= 1e-10 after a converged solve, closed faces exactly zero.
  * velfg / les / adam / feedbf / bondv1 -- the paper prints only the
    u-component of velfg; the remaining discretisation is a stated reading,
    pinned by polynomial exactness, Taylor-Green decay, mirror symmetry,
    dissipation sign and mass-flux balance (partially pinned: a reading that
    satisfies every invariant but differs from the original Fortran cannot
    be excluded).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "les_oracle.c")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "liblesoracle.so")

# array ids (must follow the enum in les_oracle.c)
A_U, A_V, A_W, A_P, A_RHS, A_NUT, A_US, A_VS, A_WS, A_FU, A_FV, A_FW = range(12)


class OrcParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32), ("bc_z", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dt", ctypes.c_double), ("cs", ctypes.c_double), ("nu", ctypes.c_double),
                ("omega", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_sweeps", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("fixed_sweeps", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("turb", ctypes.c_double), ("seed", ctypes.c_uint64)]


class OrcStats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("rhs_norm", ctypes.c_double),
                ("rhs_mean", ctypes.c_double), ("mass_factor", ctypes.c_double),
                ("p_mean", ctypes.c_double), ("q_in", ctypes.c_double),
                ("q_out", ctypes.c_double)]


LIB_OMP = os.path.join(LIBDIR, "liblesoracle_omp.so")


def _compile(out: str, extra) -> None:
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared"] + list(extra) + ["-o", tmp, SRC, "-lm"]
    try:
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    finally:
        if os.path.exists(tmp):
            os.remove(tmp)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction),
    once sequential and once with -fopenmp (same source, bit-identical results;
    the threaded build times the CPU baseline on every host core)."""
    os.makedirs(LIBDIR, exist_ok=True)
    for out, extra in ((LIB, []), (LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
            _compile(out, extra)
    return LIB


_libs = {}


def lib(omp: bool = False):
    """The sequential oracle library, or the OpenMP build with omp=True."""
    if omp not in _libs:
        build()
        L = ctypes.CDLL(LIB_OMP if omp else LIB)
        vp = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_create.restype = vp
        L.orc_create.argtypes = [ctypes.POINTER(OrcParams), dp, ctypes.c_void_p, dp]
        L.orc_destroy.argtypes = [vp]
        L.orc_get.argtypes = [vp, ctypes.c_int, dp]
        L.orc_set.argtypes = [vp, ctypes.c_int, dp]
        L.orc_raw.restype = dp
        L.orc_raw.argtypes = [vp, ctypes.c_int]
        L.orc_dims.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
        L.orc_stats_get.argtypes = [vp, ctypes.POINTER(OrcStats)]
        L.orc_step_index.restype = ctypes.c_int64
        L.orc_step_index.argtypes = [vp]
        L.orc_set_step_index.argtypes = [vp, ctypes.c_int64]
        for name in ("orc_bc_fill", "orc_les_nut", "orc_momentum", "orc_outflow_fix",
                     "orc_make_rhs", "orc_sor_solve", "orc_gauge", "orc_project"):
            getattr(L, name).argtypes = [vp]
        L.orc_sor_half.argtypes = [vp, ctypes.c_int]
        L.orc_sor_sweeps.argtypes = [vp, ctypes.c_int]
        L.orc_twin_sweeps.argtypes = [vp, ctypes.c_int, ctypes.c_double]
        L.orc_twin_sweeps.restype = ctypes.c_int
        L.orc_residual.restype = ctypes.c_double
        L.orc_residual.argtypes = [vp]
        L.orc_tendency.argtypes = [vp, ctypes.c_int]
        L.orc_apply_A.argtypes = [vp, dp, dp]
        L.orc_divergence.argtypes = [vp, dp]
        L.orc_pressure_solve.argtypes = [vp, dp]
        L.orc_step.argtypes = [vp, ctypes.c_int]
        L.orc_gauss.restype = ctypes.c_double
        L.orc_gauss.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_set_inflow_series.restype = ctypes.c_int
        L.orc_set_inflow_series.argtypes = [vp, ctypes.c_int, dp, dp]
        L.orc_inflow_profile.argtypes = [vp, dp]
        L.orc_threads.restype = ctypes.c_int
        L.orc_threads.argtypes = []
        L.orc_set_threads.argtypes = [ctypes.c_int]
        _libs[omp] = L
    return _libs[omp]


def threads(omp: bool = True) -> int:
    """Threads the oracle build uses (1 for the sequential build)."""
    return lib(omp).orc_threads()


def set_threads(n: int) -> None:
    """Thread count of the OpenMP build."""
    lib(True).orc_set_threads(int(n))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One FP64 LES domain on the CPU."""

    def __init__(self, sc, omp=False, **override):
        self.L = L = lib(omp)
        prm = sc.params()
        prm.update(override)
        self.nx, self.ny, self.nz = prm["nx"], prm["ny"], prm["nz"]
        self.bc = (prm["bc_x"], prm["bc_y"], prm["bc_z"])
        P = OrcParams(nx=prm["nx"], ny=prm["ny"], nz=prm["nz"], bc_x=prm["bc_x"],
                      bc_y=prm["bc_y"], bc_z=prm["bc_z"], dx=prm["dx"], dy=prm["dy"],
                      dt=prm["dt"], cs=prm["cs"], nu=prm["nu"], omega=prm["omega"],
                      tol=prm["tol"], max_sweeps=prm["max_sweeps"],
                      check_every=prm["check_every"], fixed_sweeps=prm["fixed_sweeps"],
                      pad_=0, turb=prm["turb"], seed=prm["seed"])
        self._dz = np.ascontiguousarray(sc.dz, dtype=np.float64)
        self._solid = np.ascontiguousarray(sc.solid, dtype=np.uint8)
        self._inflow = np.ascontiguousarray(sc.inflow_u, dtype=np.float64)
        h = L.orc_create(ctypes.byref(P), _dp(self._dz), self._solid.ctypes.data, _dp(self._inflow))
        if not h:
            raise ValueError("oracle: invalid grid")
        self.h = h
        if sc.u0 is not None:
            self.set_fields(sc.u0, sc.v0, sc.w0, sc.p0)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.orc_destroy(h)
            self.h = None

    # shapes in I/O layout
    def shape(self, which):
        nx, ny, nz = self.nx, self.ny, self.nz
        if which in (A_U, A_US, A_FU):
            return (nz, ny, nx + 1)
        if which in (A_V, A_VS, A_FV):
            return (nz, ny + 1, nx)
        if which in (A_W, A_WS, A_FW):
            return (nz + 1, ny, nx)
        return (nz, ny, nx)

    def get(self, which) -> np.ndarray:
        out = np.empty(self.shape(which), dtype=np.float64)
        self.L.orc_get(self.h, which, _dp(out))
        return out

    def set(self, which, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.shape == self.shape(which), (a.shape, self.shape(which))
        self.L.orc_set(self.h, which, _dp(a))

    def raw(self, which) -> np.ndarray:
        """Writable view of a padded array, shape (nz+2, ny+2, nx+2), index [k, j, i]."""
        d = (ctypes.c_int32 * 3)()
        self.L.orc_dims(self.h, d)
        sx, sy, sz = d[0], d[1], d[2]
        ptr = self.L.orc_raw(self.h, which)
        return np.ctypeslib.as_array(ptr, shape=(sz, sy, sx))

    def set_fields(self, u, v, w, p):
        self.set(A_U, u)
        self.set(A_V, v)
        self.set(A_W, w)
        self.set(A_P, p)

    def fields(self):
        return self.get(A_U), self.get(A_V), self.get(A_W), self.get(A_P)

    def stats(self) -> dict:
        s = OrcStats()
        self.L.orc_stats_get(self.h, ctypes.byref(s))
        return {f: getattr(s, f) for f, _ in OrcStats._fields_}

    @property
    def step_index(self) -> int:
        return self.L.orc_step_index(self.h)

    @step_index.setter
    def step_index(self, s):
        self.L.orc_set_step_index(self.h, s)

    def step(self, n=1):
        self.L.orc_step(self.h, n)

    # phases
    def bc_fill(self): self.L.orc_bc_fill(self.h)
    def les_nut(self): self.L.orc_les_nut(self.h)
    def momentum(self): self.L.orc_momentum(self.h)
    def outflow_fix(self): self.L.orc_outflow_fix(self.h)
    def make_rhs(self): self.L.orc_make_rhs(self.h)
    def sor_half(self, nrd): self.L.orc_sor_half(self.h, nrd)
    def sor_sweeps(self, n): self.L.orc_sor_sweeps(self.h, n)
    def twin_sweeps(self, n, omega):
        """n sweeps of the twinned double buffer (Sec. 2.6) with relaxation omega."""
        if self.L.orc_twin_sweeps(self.h, n, omega) != 0:
            raise MemoryError("orc_twin_sweeps")
    def residual(self) -> float: return self.L.orc_residual(self.h)
    def sor_solve(self): self.L.orc_sor_solve(self.h)
    def gauge(self): self.L.orc_gauge(self.h)
    def project(self): self.L.orc_project(self.h)
    def tendency(self, with_sgs=True): self.L.orc_tendency(self.h, 1 if with_sgs else 0)

    def set_inflow_series(self, times, profiles):
        """Inflow profiles [n][nz] at increasing times [n] (n = 0: the fixed profile)."""
        self._st = np.ascontiguousarray(times, dtype=np.float64)
        self._sp = np.ascontiguousarray(profiles, dtype=np.float64)
        n = len(self._st)
        if self.L.orc_set_inflow_series(self.h, n, _dp(self._st) if n else None, _dp(self._sp) if n else None):
            raise ValueError("inflow series: times must increase")

    def inflow_profile(self) -> np.ndarray:
        out = np.empty(self.nz)
        self.L.orc_inflow_profile(self.h, _dp(out))
        return out

    def apply_A(self, p) -> np.ndarray:
        p = np.ascontiguousarray(p, dtype=np.float64)
        out = np.empty_like(p)
        self.L.orc_apply_A(self.h, _dp(p), _dp(out))
        return out

    def divergence(self) -> np.ndarray:
        out = np.empty((self.nz, self.ny, self.nx))
        self.L.orc_divergence(self.h, _dp(out))
        return out

    def pressure_solve(self, rhs=None):
        if rhs is None:
            self.L.orc_pressure_solve(self.h, None)
        else:
            r = np.ascontiguousarray(rhs, dtype=np.float64)
            self.L.orc_pressure_solve(self.h, _dp(r))


def gauss(seed: int, ctr: int) -> float:
    return lib().orc_gauss(seed, ctr)


def splitmix64(seed: int, ctr: int) -> int:
    return lib().orc_splitmix64(seed, ctr)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
