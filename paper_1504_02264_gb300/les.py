"""Thin ctypes binding of the C ABI in ``include/les.h`` (argument marshalling only).

Every function keeps the C name and signature; host arrays are numpy arrays in
the I/O layout of the header.  All computation happens in the CUDA library:
if ``lib/libles.so`` is missing this module raises instead of falling back.
``Domain`` is a small convenience wrapper over the same calls.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LES_OK, LES_ENOCONV = 0, 1
LES_EINVAL, LES_ENOMEM, LES_ECUDA, LES_ETIMEOUT, LES_ENONFINITE, LES_ESTATE = -1, -2, -3, -4, -5, -6
LES_BC_INOUT, LES_BC_FREESLIP, LES_BC_WALL, LES_BC_PERIODIC = 0, 1, 2, 3
LES_FP32, LES_FP64 = 0, 1
(LES_AUX_NUT, LES_AUX_RHS, LES_AUX_USTAR, LES_AUX_VSTAR, LES_AUX_WSTAR,
 LES_AUX_FU, LES_AUX_FV, LES_AUX_FW, LES_AUX_R0, LES_AUX_DELTA, LES_AUX_MASK,
 LES_AUX_NET_IN, LES_AUX_NET_Q) = range(13)
LES_WARM_PREV, LES_WARM_NET, LES_WARM_ZERO = 0, 1, 2
LES_SOR_REDBLACK, LES_SOR_TWINNED = 0, 1
LES_SOR_NTILES = 35                 # sweep tile indices 0 .. LES_SOR_NTILES - 1 (les_set_sor_config)
LES_NET_MMA_SYNC, LES_NET_TCGEN05, LES_NET_TCGEN05_GMEM_SPLIT = 0, 1, 2
LES_NET_KERNELS_FOLDED, LES_NET_KERNELS_PERSISTENT, LES_NET_KERNELS_LAYERS = 0, 1, 2
LES_NET_KERNELS_OWN_POOL = 4     # or-ed into a layout: the network's own pooling kernel


class les_grid_t(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32), ("bc_z", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.POINTER(ctypes.c_double)),
                ("dt", ctypes.c_double), ("cs", ctypes.c_double), ("nu", ctypes.c_double),
                ("omega", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_sweeps", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("fixed_sweeps", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("turb", ctypes.c_double), ("seed", ctypes.c_uint64)]


class les_stats_t(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("rhs_norm", ctypes.c_double),
                ("rhs_mean", ctypes.c_double), ("mass_factor", ctypes.c_double),
                ("q_in", ctypes.c_double), ("q_out", ctypes.c_double),
                ("p_mean", ctypes.c_double), ("step", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("graph", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class les_timing_t(ctypes.Structure):
    _fields_ = [("ms_momentum", ctypes.c_double), ("ms_sor", ctypes.c_double),
                ("ms_residual", ctypes.c_double), ("ms_project", ctypes.c_double),
                ("steps", ctypes.c_int64), ("sor_sweeps", ctypes.c_int64),
                ("sor_launches", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("ms_net", ctypes.c_double), ("net_cycles", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """Load ``libles.so``; raises if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"LES CUDA library not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.les_version.restype = ctypes.c_char_p
        L.les_last_error.restype = ctypes.c_char_p
        L.les_last_error.argtypes = [vp]
        L.les_create.argtypes = [ctypes.POINTER(les_grid_t), vp, vp, vp, ctypes.POINTER(vp)]
        L.les_destroy.argtypes = [vp]
        L.les_destroy.restype = None
        L.les_set_fields.argtypes = [vp, vp, vp, vp, vp]
        L.les_get_fields.argtypes = [vp, vp, vp, vp, vp]
        L.les_set_inflow.argtypes = [vp, vp, ctypes.c_double, ctypes.c_uint64]
        L.les_step.argtypes = [vp, i32, ctypes.POINTER(les_stats_t)]
        L.les_pressure_solve.argtypes = [vp, vp, ctypes.POINTER(les_stats_t)]
        L.les_get_aux.argtypes = [vp, i32, vp]
        L.les_get_state.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
        L.les_set_state.argtypes = [vp, vp, ctypes.c_size_t]
        L.les_profiler_range.argtypes = [i32]
        L.les_residual_noalloc.argtypes = [ctypes.POINTER(les_grid_t), vp, vp, vp, vp, vp, vp]
        L.les_ensemble_create.argtypes = [i32, vp, vp, vp, vp, ctypes.POINTER(vp)]
        L.les_ensemble_destroy.argtypes = [vp]
        L.les_ensemble_destroy.restype = None
        L.les_ensemble_last_error.argtypes = [vp]
        L.les_ensemble_last_error.restype = ctypes.c_char_p
        L.les_ensemble_size.argtypes = [vp, ctypes.POINTER(i32)]
        L.les_ensemble_member.argtypes = [vp, i32, ctypes.POINTER(vp)]
        L.les_ensemble_step.argtypes = [vp, i32, vp]
        L.les_ensemble_set_graph.argtypes = [vp, i32]
        L.les_ensemble_set_tile.argtypes = [vp, i32, i32]
        L.les_ensemble_get_tile.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.les_ensemble_autotune.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double)]
        L.les_ensemble_launches.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        L.les_ensemble_set_persistent.argtypes = [vp, i32]
        L.les_ensemble_set_warmstart.argtypes = [vp, vp, i32]
        L.les_selftest_wait_timeout.argtypes = [ctypes.c_int64, vp]
        L.les_time_sor.argtypes = [vp, i32, i32, i32, ctypes.POINTER(ctypes.c_double)]
        L.les_sor_compare.argtypes = [vp, i32, ctypes.c_double, i32, vp, vp, vp, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
        L.les_set_record.argtypes = [vp, i32]
        L.les_set_record_at.argtypes = [vp, i32]
        L.les_set_net_kernels.argtypes = [vp, i32]
        L.les_set_net_async.argtypes = [vp, i32]
        L.les_set_net_start.argtypes = [vp, i32]
        L.les_set_inflow_series.argtypes = [vp, i32, vp, vp]
        L.les_set_net_schedule.argtypes = [vp, i32]
        L.les_set_warmstart.argtypes = [vp, i32, vp]
        L.les_net_create.argtypes = [ctypes.c_uint64, vp, ctypes.POINTER(vp)]
        L.les_net_destroy.argtypes = [vp]
        L.les_net_destroy.restype = None
        L.les_net_last_error.argtypes = [vp]
        L.les_net_last_error.restype = ctypes.c_char_p
        L.les_net_num_params.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        L.les_net_set_stride.argtypes = [vp, i32]
        L.les_net_get_stride.argtypes = [vp, ctypes.POINTER(i32)]
        L.les_net_set_engine.argtypes = [vp, i32]
        L.les_net_get_engine.argtypes = [vp, ctypes.POINTER(i32)]
        L.les_net_get_params.argtypes = [vp, vp]
        L.les_net_set_params.argtypes = [vp, vp]
        L.les_net_forward.argtypes = [vp, vp, vp, vp, i32, i32, i32]
        L.les_net_gradient.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, vp, ctypes.POINTER(ctypes.c_double)]
        L.les_net_train_step.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, ctypes.c_float,
                                         ctypes.POINTER(ctypes.c_double)]
        L.les_set_graph.argtypes = [vp, i32]
        L.les_set_sor_config.argtypes = [vp, i32, i32]
        L.les_get_sor_config.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.les_sor_tile.argtypes = [i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.les_autotune_sor.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double)]
        L.les_set_timing.argtypes = [vp, i32]
        L.les_get_timing.argtypes = [vp, ctypes.POINTER(les_timing_t)]
        for name in ("les_ensemble_create", "les_ensemble_size", "les_ensemble_member", "les_ensemble_step",
                     "les_ensemble_set_graph", "les_ensemble_set_tile", "les_ensemble_get_tile",
                     "les_ensemble_autotune", "les_ensemble_launches", "les_ensemble_set_persistent", "les_ensemble_set_warmstart", "les_selftest_wait_timeout", "les_time_sor", "les_set_net_kernels", "les_set_net_async", "les_set_net_start", "les_set_inflow_series", "les_set_record", "les_set_record_at", "les_set_net_schedule", "les_set_warmstart",
                     "les_net_create", "les_net_num_params", "les_net_set_stride", "les_net_get_stride",
                     "les_net_set_engine", "les_net_get_engine",
                     "les_net_get_params", "les_net_set_params", "les_net_forward", "les_net_gradient",
                     "les_net_train_step", "les_residual_noalloc", "les_profiler_range", "les_set_graph",
                     "les_set_sor_config", "les_get_sor_config", "les_sor_tile", "les_autotune_sor",
                     "les_set_timing", "les_get_timing", "les_create", "les_set_fields", "les_get_fields",
                     "les_set_inflow", "les_step", "les_pressure_solve", "les_get_aux", "les_get_state",
                     "les_set_state"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


class LesError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _check(rc, h=None):
    if rc < 0:
        msg = lib().les_last_error(h)
        raise LesError(rc, msg.decode() if msg else "")
    return rc


def _ptr(a):
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------------------
# C-named functions

def les_version() -> str:
    return lib().les_version().decode()


def les_create(grid: les_grid_t, solid: np.ndarray, inflow_u: np.ndarray, stream=None) -> int:
    h = ctypes.c_void_p()
    rc = lib().les_create(ctypes.byref(grid), _ptr(solid), _ptr(inflow_u), stream, ctypes.byref(h))
    _check(rc)
    return h.value


def les_destroy(h):
    lib().les_destroy(h)


def les_set_fields(h, u, v, w, p):
    return _check(lib().les_set_fields(h, _ptr(u), _ptr(v), _ptr(w), _ptr(p)), h)


def les_get_fields(h, u, v, w, p):
    return _check(lib().les_get_fields(h, _ptr(u), _ptr(v), _ptr(w), _ptr(p)), h)


def les_set_inflow(h, inflow_u, turb, seed):
    return _check(lib().les_set_inflow(h, _ptr(inflow_u), float(turb), int(seed)), h)


def les_step(h, nsteps, stats: les_stats_t | None = None):
    return _check(lib().les_step(h, nsteps, ctypes.byref(stats) if stats is not None else None), h)


def les_pressure_solve(h, rhs, stats: les_stats_t | None = None):
    return _check(lib().les_pressure_solve(h, _ptr(rhs), ctypes.byref(stats) if stats is not None else None), h)


def les_get_aux(h, which, out):
    return _check(lib().les_get_aux(h, which, _ptr(out)), h)


def les_get_state(h, buf, length: ctypes.c_size_t):
    return _check(lib().les_get_state(h, buf, ctypes.byref(length)), h)


def les_set_state(h, buf, length):
    return _check(lib().les_set_state(h, buf, length), h)


def les_set_timing(h, enable):
    return _check(lib().les_set_timing(h, 1 if enable else 0), h)


def les_get_timing(h, t: les_timing_t):
    return _check(lib().les_get_timing(h, ctypes.byref(t)), h)


def les_residual_noalloc(grid: les_grid_t, d_p, d_rhs, d_solid, d_dz, d_out, stream=None):
    """Device pointers (ints) in, device pointer out; allocates nothing."""
    return _check(lib().les_residual_noalloc(ctypes.byref(grid), d_p, d_rhs, d_solid, d_dz, d_out, stream))


def les_set_record(h, enable):
    return _check(lib().les_set_record(h, 1 if enable else 0), h)


def les_set_record_at(h, after_sweeps):
    return _check(lib().les_set_record_at(h, after_sweeps), h)


def les_set_net_schedule(h, every_sweeps):
    return _check(lib().les_set_net_schedule(h, every_sweeps), h)


def les_set_warmstart(h, mode, net):
    return _check(lib().les_set_warmstart(h, mode, net), h)


def _ncheck(rc, n):
    if rc < 0:
        m = lib().les_net_last_error(n)
        raise LesError(rc, m.decode() if m else "")
    return rc


def les_net_create(seed, stream=None):
    h = ctypes.c_void_p()
    rc = lib().les_net_create(seed, stream, ctypes.byref(h))
    if rc < 0:
        raise LesError(rc, "les_net_create failed")
    return h.value


def les_net_destroy(n):
    lib().les_net_destroy(n)


def les_net_num_params(n):
    c = ctypes.c_int64()
    _ncheck(lib().les_net_num_params(n, ctypes.byref(c)), n)
    return c.value


def les_net_set_stride(n, stride):
    return _ncheck(lib().les_net_set_stride(n, stride), n)


def les_net_get_stride(n):
    s = ctypes.c_int32()
    _ncheck(lib().les_net_get_stride(n, ctypes.byref(s)), n)
    return s.value


def les_net_set_engine(n, engine):
    return _ncheck(lib().les_net_set_engine(n, engine), n)


def les_net_get_engine(n):
    e = ctypes.c_int32()
    _ncheck(lib().les_net_get_engine(n, ctypes.byref(e)), n)
    return e.value


def les_net_get_params(n, out):
    return _ncheck(lib().les_net_get_params(n, _ptr(out)), n)


def les_net_set_params(n, params):
    return _ncheck(lib().les_net_set_params(n, _ptr(params)), n)


def les_net_forward(n, d_r, d_mask, d_y, nx, ny, nz):
    return _ncheck(lib().les_net_forward(n, d_r, d_mask, d_y, nx, ny, nz), n)


def les_net_gradient(n, d_r, d_mask, d_t, batch, nx, ny, nz, d_grad):
    loss = ctypes.c_double()
    _ncheck(lib().les_net_gradient(n, d_r, d_mask, d_t, batch, nx, ny, nz, d_grad, ctypes.byref(loss)), n)
    return loss.value


def les_net_train_step(n, d_r, d_mask, d_t, batch, nx, ny, nz, lr):
    loss = ctypes.c_double()
    _ncheck(lib().les_net_train_step(n, d_r, d_mask, d_t, batch, nx, ny, nz, lr, ctypes.byref(loss)), n)
    return loss.value


class Net:
    """The warm-start network (device weights owned by the library)."""

    def __init__(self, seed=0, stream="torch", stride=1):
        st = current_stream() if stream == "torch" else stream
        self.h = les_net_create(seed, st)
        self.nparam = les_net_num_params(self.h)
        les_net_set_stride(self.h, stride)

    @property
    def stride(self):
        return les_net_get_stride(self.h)

    @stride.setter
    def stride(self, s):
        les_net_set_stride(self.h, s)

    @property
    def engine(self):
        """LES_NET_TCGEN05 (default) or LES_NET_MMA_SYNC: the forward convolutions' tensor-core path."""
        return les_net_get_engine(self.h)

    @engine.setter
    def engine(self, e):
        les_net_set_engine(self.h, e)

    def close(self):
        if getattr(self, "h", None):
            les_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(self.nparam, np.float32)
        les_net_get_params(self.h, out)
        return out

    def set_params(self, p):
        les_net_set_params(self.h, np.ascontiguousarray(p, np.float32))


def _echeck(rc, e):
    if rc < 0:
        m = lib().les_ensemble_last_error(e)
        raise LesError(rc, m.decode() if m else "")
    return rc


class Ensemble:
    """Uneven domains stepped together (batched SOR launches over all members)."""

    def __init__(self, scenes, stream="torch"):
        n = len(scenes)
        grids = (les_grid_t * n)()
        self._keep = []
        solid_p = (ctypes.c_void_p * n)()
        inflow_p = (ctypes.c_void_p * n)()
        for i, sc in enumerate(scenes):
            g, dz, solid, inflow = grid_of(sc, LES_FP32)
            grids[i] = g
            self._keep += [dz, solid, inflow]
            solid_p[i] = solid.ctypes.data
            inflow_p[i] = inflow.ctypes.data
        st = current_stream() if stream == "torch" else stream
        h = ctypes.c_void_p()
        rc = lib().les_ensemble_create(n, grids, solid_p, inflow_p, st, ctypes.byref(h))
        if rc < 0:
            raise LesError(rc, "les_ensemble_create failed")
        self.h = h.value
        self.n = n
        self.members = []
        for i, sc in enumerate(scenes):
            mh = ctypes.c_void_p()
            _echeck(lib().les_ensemble_member(self.h, i, ctypes.byref(mh)), self.h)
            d = Domain(sc, handle=mh.value)
            if sc.u0 is not None:
                d.set_fields(sc.u0, sc.v0, sc.w0, sc.p0)
            self.members.append(d)

    def close(self):
        if getattr(self, "h", None):
            for d in self.members:
                d.close()
            lib().les_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        st = (les_stats_t * self.n)()
        rc = _echeck(lib().les_ensemble_step(self.h, n, st), self.h)
        out = []
        for i in range(self.n):
            d = {f: getattr(st[i], f) for f, _ in les_stats_t._fields_}
            d["rc"] = rc
            out.append(d)
        return out

    def set_graph(self, enable=True):
        _echeck(lib().les_ensemble_set_graph(self.h, 1 if enable else 0), self.h)

    def set_tile(self, tile, ctas_per_sm=4):
        _echeck(lib().les_ensemble_set_tile(self.h, tile, ctas_per_sm), self.h)

    def tile(self):
        t, c = ctypes.c_int32(), ctypes.c_int32()
        _echeck(lib().les_ensemble_get_tile(self.h, ctypes.byref(t), ctypes.byref(c)), self.h)
        return t.value, c.value

    def autotune(self, sweeps=10):
        ms = ctypes.c_double()
        _echeck(lib().les_ensemble_autotune(self.h, sweeps, ctypes.byref(ms)), self.h)
        return self.tile(), ms.value

    def launches(self):
        v = ctypes.c_int64()
        _echeck(lib().les_ensemble_launches(self.h, ctypes.byref(v)), self.h)
        return v.value

    def set_persistent(self, enable=True):
        """Plain-SOR steps: the whole solve as one persistent cooperative launch per step."""
        _echeck(lib().les_ensemble_set_persistent(self.h, 1 if enable else 0), self.h)

    def set_warmstart(self, net=None, every_sweeps=10):
        """Learned correction in every member's solve (net None: previous-step start)."""
        _echeck(lib().les_ensemble_set_warmstart(self.h, net.h if net is not None else None, every_sweeps),
                self.h)
        self._net = net


def les_selftest_wait_timeout(limit_ns, stream=None):
    """Returns the C status (LES_ETIMEOUT expected) without raising on it."""
    rc = lib().les_selftest_wait_timeout(int(limit_ns), stream)
    if rc < 0 and rc != LES_ETIMEOUT:
        raise LesError(rc, lib().les_last_error(None).decode())
    return rc


def les_profiler_range(start):
    return _check(lib().les_profiler_range(1 if start else 0))


def les_set_graph(h, enable):
    return _check(lib().les_set_graph(h, 1 if enable else 0), h)


def les_set_sor_config(h, tile, kc):
    return _check(lib().les_set_sor_config(h, tile, kc), h)


def les_get_sor_config(h):
    t, k = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().les_get_sor_config(h, ctypes.byref(t), ctypes.byref(k)), h)
    return t.value, k.value


def les_sor_tile(tile):
    tx, ty, tz = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().les_sor_tile(tile, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(tz)))
    return tx.value, ty.value, tz.value


def les_autotune_sor(h, sweeps):
    ms = ctypes.c_double()
    _check(lib().les_autotune_sor(h, sweeps, ctypes.byref(ms)), h)
    return ms.value


def les_last_error(h) -> str:
    m = lib().les_last_error(h)
    return m.decode() if m else ""


# ---------------------------------------------------------------------------
# convenience wrapper

def current_stream():
    """The current torch CUDA stream handle (torch supplies streams only)."""
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def grid_of(sc, precision=LES_FP32, **override):
    """The les_grid_t of a scene (the returned dz array backs its dz pointer)."""
    prm = sc.params()
    prm.update(override)
    dz = np.ascontiguousarray(sc.dz, dtype=np.float64)
    g = les_grid_t(nx=prm["nx"], ny=prm["ny"], nz=prm["nz"], bc_x=prm["bc_x"], bc_y=prm["bc_y"],
                   bc_z=prm["bc_z"], dx=prm["dx"], dy=prm["dy"],
                   dz=dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                   dt=prm["dt"], cs=prm["cs"], nu=prm["nu"], omega=prm["omega"], tol=prm["tol"],
                   max_sweeps=prm["max_sweeps"], check_every=prm["check_every"],
                   fixed_sweeps=prm["fixed_sweeps"], precision=precision, turb=prm["turb"],
                   seed=prm["seed"])
    solid = np.ascontiguousarray(sc.solid, dtype=np.uint8)
    inflow = np.ascontiguousarray(sc.inflow_u, dtype=np.float64)
    return g, dz, solid, inflow


class Domain:
    """One LES domain on the GPU, built from a ``scene.Scene``."""

    def __init__(self, sc, precision=LES_FP32, stream="torch", handle=None, **override):
        g, self._dz, solid, inflow = grid_of(sc, precision, **override)
        self.nx, self.ny, self.nz = g.nx, g.ny, g.nz
        self.dtype = np.float64 if precision == LES_FP64 else np.float32
        self._owned = handle is None
        if handle is None:
            st = current_stream() if stream == "torch" else stream
            self.h = les_create(g, solid, inflow, st)
        else:
            self.h = handle
        if sc.u0 is not None and handle is None:
            self.set_fields(sc.u0, sc.v0, sc.w0, sc.p0)

    def close(self):
        if getattr(self, "h", None):
            if self._owned:
                les_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shapes(self):
        nx, ny, nz = self.nx, self.ny, self.nz
        return (nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx), (nz, ny, nx)

    def _c(self, a):
        return None if a is None else np.ascontiguousarray(a, dtype=self.dtype)

    def set_fields(self, u=None, v=None, w=None, p=None):
        les_set_fields(self.h, self._c(u), self._c(v), self._c(w), self._c(p))

    def fields(self):
        out = [np.empty(s, dtype=self.dtype) for s in self.shapes()]
        les_get_fields(self.h, *out)
        return out

    def step(self, n=1) -> dict:
        st = les_stats_t()
        rc = les_step(self.h, n, st)
        d = {f: getattr(st, f) for f, _ in les_stats_t._fields_}
        d["rc"] = rc
        return d

    def pressure_solve(self, rhs=None) -> dict:
        st = les_stats_t()
        rc = les_pressure_solve(self.h, self._c(rhs), st)
        d = {f: getattr(st, f) for f, _ in les_stats_t._fields_}
        d["rc"] = rc
        return d

    def aux(self, which) -> np.ndarray:
        nx, ny, nz = self.nx, self.ny, self.nz
        shape = {LES_AUX_NUT: (nz, ny, nx), LES_AUX_RHS: (nz, ny, nx), LES_AUX_R0: (nz, ny, nx),
                 LES_AUX_DELTA: (nz, ny, nx), LES_AUX_MASK: (nz, ny, nx), LES_AUX_NET_IN: (nz, ny, nx),
                 LES_AUX_NET_Q: (nz, ny, nx),
                 LES_AUX_USTAR: (nz, ny, nx + 1), LES_AUX_FU: (nz, ny, nx + 1),
                 LES_AUX_VSTAR: (nz, ny + 1, nx), LES_AUX_FV: (nz, ny + 1, nx),
                 LES_AUX_WSTAR: (nz + 1, ny, nx), LES_AUX_FW: (nz + 1, ny, nx)}[which]
        out = np.empty(shape, dtype=np.float32 if which == LES_AUX_NET_Q else self.dtype)
        les_get_aux(self.h, which, out)
        return out

    def get_state(self) -> bytes:
        n = ctypes.c_size_t(0)
        les_get_state(self.h, None, n)
        buf = ctypes.create_string_buffer(n.value)
        les_get_state(self.h, buf, n)
        return buf.raw

    def set_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        les_set_state(self.h, buf, len(blob))

    def set_record(self, enable=True, after_sweeps=0):
        les_set_record(self.h, enable)
        les_set_record_at(self.h, after_sweeps)

    def set_net_schedule(self, every_sweeps):
        les_set_net_schedule(self.h, every_sweeps)

    def set_inflow_series(self, times, profiles):
        """Inflow profiles [n][nz] at increasing times [n] (n = 0: the fixed profile)."""
        t = np.ascontiguousarray(times, dtype=np.float64)
        p = np.ascontiguousarray(profiles, dtype=np.float64)
        _check(lib().les_set_inflow_series(self.h, len(t), _ptr(t) if len(t) else None,
                                           _ptr(p) if len(t) else None), self.h)

    def set_net_start(self, enable=True):
        _check(lib().les_set_net_start(self.h, 1 if enable else 0), self.h)

    def set_net_async(self, enable=True):
        _check(lib().les_set_net_async(self.h, 1 if enable else 0), self.h)

    def set_net_kernels(self, persistent=True):
        """True: the persistent network launch; False: per-layer launches with
        the folded packing, head and prolongation (default); or one of the
        LES_NET_KERNELS_* layouts."""
        mode = persistent if not isinstance(persistent, bool) else (
            LES_NET_KERNELS_PERSISTENT if persistent else LES_NET_KERNELS_FOLDED)
        _check(lib().les_set_net_kernels(self.h, int(mode)), self.h)

    def set_warmstart(self, net=None, mode=None):
        """net given: learned warm start; else mode LES_WARM_PREV (default) or LES_WARM_ZERO."""
        if net is not None:
            les_set_warmstart(self.h, LES_WARM_NET, net.h)
        else:
            les_set_warmstart(self.h, LES_WARM_PREV if mode is None else mode, None)
        self._net = net          # keep the network alive while the handle uses it

    def set_graph(self, enable=True):
        les_set_graph(self.h, enable)

    def set_sor_config(self, tile, kc=0):
        les_set_sor_config(self.h, tile, kc)

    def sor_config(self):
        return les_get_sor_config(self.h)

    def sor_compare(self, variant, omega, sweeps, rhs, p0):
        """les_sor_compare: (p0 + d after `sweeps` sweeps of the variant, ms per
        sweep, FP64 relative residual).  rhs, p0: (nz, ny, nx) float64."""
        nx, ny, nz = self.nx, self.ny, self.nz
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        p0 = np.ascontiguousarray(p0, dtype=np.float64)
        if rhs.shape != (nz, ny, nx) or p0.shape != (nz, ny, nx):
            raise ValueError("rhs and p0 must be (nz, ny, nx)")
        out = np.empty((nz, ny, nx), dtype=np.float64)
        ms, rel = ctypes.c_double(), ctypes.c_double()
        _check(lib().les_sor_compare(self.h, variant, float(omega), int(sweeps), rhs.ctypes.data,
                                     p0.ctypes.data, out.ctypes.data, ctypes.byref(ms), ctypes.byref(rel)), self.h)
        return out, ms.value, rel.value

    def time_sor(self, tile, kc=0, sweeps=20):
        ms = ctypes.c_double()
        _check(lib().les_time_sor(self.h, tile, kc, sweeps, ctypes.byref(ms)), self.h)
        return ms.value

    def autotune_sor(self, sweeps=20):
        ms = les_autotune_sor(self.h, sweeps)
        return self.sor_config(), ms

    def set_timing(self, enable=True):
        les_set_timing(self.h, enable)

    def timing(self) -> dict:
        t = les_timing_t()
        les_get_timing(self.h, t)
        return {f: getattr(t, f) for f, _ in les_timing_t._fields_}

    def set_inflow(self, inflow_u, turb, seed):
        les_set_inflow(self.h, np.ascontiguousarray(inflow_u, dtype=np.float64), turb, seed)
