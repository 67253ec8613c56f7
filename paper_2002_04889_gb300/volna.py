"""Python binding of the volna_gb C ABI (include/volna_gb.h).

Argument marshalling only: every step of the solver runs in the CUDA library
``_build/libvolna_gb.so``.  There is no fallback: if the library cannot be
loaded, importing the solver raises.

The functions ``vg_*`` mirror the C entry points one to one (same names,
same arguments, status codes turned into ``VolnaError``).  ``Solver`` wraps a
context for convenience and accepts numpy arrays (host) or CUDA torch tensors
(device, read on the context's stream).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

VG_OK = 0
VG_EINVAL = -1
VG_ENOMEM = -2
VG_ECUDA = -3
VG_ENONFINITE = -4
VG_ENEGDEPTH = -5
VG_ETIMEOUT = -6
VG_ESTATE = -7

RENUMBER = {"none": 0, "morton": 1, "rcm": 2, "hilbert": 3}
BOUNDARY = {"wall": 1, "open": 2, "absorbing": 3}


class VolnaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class vg_params(C.Structure):
    _fields_ = [("g", C.c_double), ("cfl", C.c_double), ("h_threshold", C.c_double),
                ("dt_fixed", C.c_double), ("dt_max", C.c_double), ("t_end", C.c_double),
                ("order", C.c_int32), ("gauge_every", C.c_int32),
                ("strict_positivity", C.c_int32), ("block_cells", C.c_int32),
                ("block_threads", C.c_int32), ("fp64_literal", C.c_int32),
                ("rk_unfused", C.c_int32)]


class vg_diag(C.Structure):
    _fields_ = [("t", C.c_double), ("last_dt", C.c_double), ("mass", C.c_double),
                ("min_H", C.c_double), ("steps", C.c_int64), ("neg_count", C.c_int64),
                ("dry_count", C.c_int64), ("launches", C.c_int64), ("n_records", C.c_int64)]


_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_V = C.c_void_p
_lib = None

_SIGNATURES = {
    "vg_version": ([], C.c_int),
    "vg_strerror": ([C.c_int], C.c_char_p),
    "vg_default_params": ([C.POINTER(vg_params)], C.c_int),
    "vg_create": ([C.POINTER(_V), C.c_int, C.c_int, _V], C.c_int),
    "vg_destroy": ([_V], None),
    "vg_last_error": ([_V], C.c_char_p),
    "vg_mesh_upload": ([_V, C.c_int64, _D, C.c_int64, _I32, _D, C.c_int], C.c_int),
    "vg_get_permutation": ([_V, _I32], C.c_int),
    "vg_get_flipped": ([_V, _I64], C.c_int),
    "vg_set_params": ([_V, C.POINTER(vg_params)], C.c_int),
    "vg_get_params": ([_V, C.POINTER(vg_params)], C.c_int),
    "vg_set_state": ([_V, _D, _D, _D, C.c_double], C.c_int),
    "vg_set_state_dev": ([_V, _V, _V, _V, C.c_double], C.c_int),
    "vg_get_state": ([_V, _D, _D, _D, _D], C.c_int),
    "vg_set_state_f32": ([_V, _F, _F, _F, C.c_double], C.c_int),
    "vg_get_state_f32": ([_V, _F, _F, _F, _D], C.c_int),
    "vg_get_state_dev": ([_V, _V, _V, _V], C.c_int),
    "vg_set_gauges": ([_V, C.c_int32, _D], C.c_int),
    "vg_get_gauge_cells": ([_V, _I32], C.c_int),
    "vg_step": ([_V, C.c_int64], C.c_int),
    "vg_advance_to": ([_V, C.c_double], C.c_int),
    "vg_get_gauges": ([_V, _D, _D, C.c_int64, _I64], C.c_int),
    "vg_get_diagnostics": ([_V, C.POINTER(vg_diag)], C.c_int),
    "vg_profile": ([_V, C.c_int], C.c_int),
    "vg_get_profile": ([_V, C.c_int32, C.POINTER(C.c_char_p), _I64, _D, _I32], C.c_int),
    "vg_device_bytes": ([_V, _I64], C.c_int),
    "vg_step_noalloc": ([_V, _V, _V, C.c_double, _D], C.c_int),
    "vg_set_depth": ([_V, _D], C.c_int),
    "vg_set_bed_motion": ([_V, _D, _D, C.c_double], C.c_int),
    "vg_adj_bed_gradient": ([_V, _D, _D], C.c_int),
    "vg_set_open_boundary": ([_V, C.c_int64, _I32], C.c_int),
    "vg_set_boundary": ([_V, C.c_int64, _I32, _I32], C.c_int),
    "vg_adj_forward": ([_V, C.c_int64, C.c_double, C.c_int64], C.c_int),
    "vg_adj_forward_binomial": ([_V, C.c_int64, C.c_double, C.c_int32], C.c_int),
    "vg_adj_backward": ([_V, _D, _D, _D, _D, _D, _D], C.c_int),
    "vg_batch_create": ([C.POINTER(_V), C.c_int, C.c_int, _V], C.c_int),
    "vg_batch_destroy": ([_V], None),
    "vg_batch_last_error": ([_V], C.c_char_p),
    "vg_batch_set_params": ([_V, C.POINTER(vg_params)], C.c_int),
    "vg_batch_add_mesh": ([_V, C.c_int64, _D, C.c_int64, _I32, _D, C.c_int, C.c_int32,
                           C.POINTER(C.c_int32)], C.c_int),
    "vg_batch_set_state": ([_V, C.c_int32, C.c_int32, _D, _D, _D, C.c_double], C.c_int),
    "vg_batch_get_state": ([_V, C.c_int32, C.c_int32, _D, _D, _D, _D, _I64], C.c_int),
    "vg_batch_step": ([_V, C.c_int64], C.c_int),
    "vg_batch_run": ([_V, C.c_double, C.c_int64, _I64], C.c_int),
    "vg_batch_autotune": ([_V, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), _D], C.c_int),
    "vg_batch_info": ([_V, C.POINTER(C.c_int32), C.POINTER(C.c_int32), _I64, _I64], C.c_int),
    "vg_batch_set_gauges": ([_V, C.c_int32, C.c_int32, _D], C.c_int),
    "vg_batch_set_open_boundary": ([_V, C.c_int32, C.c_int64, _I32], C.c_int),
    "vg_batch_set_boundary": ([_V, C.c_int32, C.c_int64, _I32, _I32], C.c_int),
    "vg_batch_get_gauges": ([_V, C.c_int32, C.c_int32, _D, _D, C.c_int64, _I64], C.c_int),
}

VG_NOALLOC_MAX_CELLS = 262144


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libvolna_gb.so (building it first if it is missing); raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"volna_gb CUDA library not built: {path}")
        _build.build()
    lib = C.CDLL(path)
    for name, (args, res) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(ctx, rc: int) -> None:
    if rc != VG_OK:
        lib = load()
        msg = lib.vg_last_error(ctx).decode() if ctx else lib.vg_strerror(rc).decode()
        raise VolnaError(rc, msg or lib.vg_strerror(rc).decode())


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _fp(a: np.ndarray):
    return a.ctypes.data_as(_F)


# ---------------------------------------------------------------- one-to-one entry points


def vg_version() -> int:
    return load().vg_version()


def vg_strerror(code: int) -> str:
    return load().vg_strerror(code).decode()


def vg_default_params() -> vg_params:
    p = vg_params()
    _check(None, load().vg_default_params(C.byref(p)))
    return p


def vg_create(precision: int = 64, device: int = 0, stream: int | None = None):
    h = _V()
    rc = load().vg_create(C.byref(h), int(precision), int(device), _V(stream) if stream else None)
    if rc != VG_OK:
        raise VolnaError(rc, f"vg_create failed: {vg_strerror(rc)}")
    return h


def vg_destroy(ctx) -> None:
    load().vg_destroy(ctx)


def vg_last_error(ctx) -> str:
    return load().vg_last_error(ctx).decode()


def vg_mesh_upload(ctx, xy, tri, depth_v, renumber="hilbert") -> None:
    xy = _f64(xy).reshape(-1, 2)
    tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
    depth_v = _f64(depth_v)
    if isinstance(renumber, str):
        renumber = RENUMBER[renumber]
    _check(ctx, load().vg_mesh_upload(ctx, xy.shape[0], _dp(xy), tri.shape[0],
                                      tri.ctypes.data_as(_I32), _dp(depth_v), int(renumber)))


def vg_get_permutation(ctx, nc: int) -> np.ndarray:
    out = np.empty(nc, dtype=np.int32)
    _check(ctx, load().vg_get_permutation(ctx, out.ctypes.data_as(_I32)))
    return out


def vg_get_flipped(ctx) -> int:
    n = C.c_int64()
    _check(ctx, load().vg_get_flipped(ctx, C.byref(n)))
    return n.value


def vg_set_params(ctx, p: vg_params) -> None:
    _check(ctx, load().vg_set_params(ctx, C.byref(p)))


def vg_get_params(ctx) -> vg_params:
    p = vg_params()
    _check(ctx, load().vg_get_params(ctx, C.byref(p)))
    return p


def vg_set_state(ctx, H, Hu, Hv, t=0.0) -> None:
    H, Hu, Hv = _f64(H), _f64(Hu), _f64(Hv)
    _check(ctx, load().vg_set_state(ctx, _dp(H), _dp(Hu), _dp(Hv), float(t)))


def vg_set_state_dev(ctx, H_ptr: int, Hu_ptr: int, Hv_ptr: int, t=0.0) -> None:
    _check(ctx, load().vg_set_state_dev(ctx, _V(H_ptr), _V(Hu_ptr), _V(Hv_ptr), float(t)))


def vg_get_state(ctx, nc: int, out=None):
    if out is None:
        out = (np.empty(nc), np.empty(nc), np.empty(nc))
    if any(o.dtype != np.float64 or not o.flags.c_contiguous or o.size != nc for o in out):
        raise ValueError("out must be three contiguous float64 arrays of nc values")
    t = C.c_double()
    _check(ctx, load().vg_get_state(ctx, _dp(out[0]), _dp(out[1]), _dp(out[2]), C.byref(t)))
    return out[0], out[1], out[2], t.value


def vg_set_state_f32(ctx, H, Hu, Hv, t=0.0) -> None:
    H, Hu, Hv = _f32(H), _f32(Hu), _f32(Hv)
    _check(ctx, load().vg_set_state_f32(ctx, _fp(H), _fp(Hu), _fp(Hv), float(t)))


def vg_get_state_f32(ctx, nc: int, out=None):
    if out is None:
        out = tuple(np.empty(nc, dtype=np.float32) for _ in range(3))
    if any(o.dtype != np.float32 or not o.flags.c_contiguous or o.size != nc for o in out):
        raise ValueError("out must be three contiguous float32 arrays of nc values")
    t = C.c_double()
    _check(ctx, load().vg_get_state_f32(ctx, _fp(out[0]), _fp(out[1]), _fp(out[2]), C.byref(t)))
    return out[0], out[1], out[2], t.value


def vg_get_state_dev(ctx, H_ptr: int, Hu_ptr: int, Hv_ptr: int) -> None:
    _check(ctx, load().vg_get_state_dev(ctx, _V(H_ptr), _V(Hu_ptr), _V(Hv_ptr)))


def vg_set_gauges(ctx, xy) -> None:
    xy = _f64(xy).reshape(-1, 2)
    _check(ctx, load().vg_set_gauges(ctx, xy.shape[0], _dp(xy) if xy.shape[0] else None))


def vg_get_gauge_cells(ctx, n: int) -> np.ndarray:
    out = np.empty(max(n, 1), dtype=np.int32)
    _check(ctx, load().vg_get_gauge_cells(ctx, out.ctypes.data_as(_I32)))
    return out[:n]


def vg_step(ctx, n_steps: int) -> None:
    _check(ctx, load().vg_step(ctx, int(n_steps)))


def vg_advance_to(ctx, t: float) -> None:
    _check(ctx, load().vg_advance_to(ctx, float(t)))


def vg_get_gauges(ctx, n_gauges: int):
    n = C.c_int64()
    _check(ctx, load().vg_get_gauges(ctx, None, None, 0, C.byref(n)))
    t = np.empty(max(n.value, 1))
    eta = np.empty((max(n.value, 1), max(n_gauges, 1)))
    _check(ctx, load().vg_get_gauges(ctx, _dp(t), _dp(eta), n.value, C.byref(n)))
    return t[:n.value], eta[:n.value, :n_gauges]


def vg_get_diagnostics(ctx) -> dict:
    d = vg_diag()
    _check(ctx, load().vg_get_diagnostics(ctx, C.byref(d)))
    return {k: getattr(d, k) for k, _ in vg_diag._fields_}


def vg_profile(ctx, enable: bool) -> None:
    _check(ctx, load().vg_profile(ctx, 1 if enable else 0))


def vg_get_profile(ctx) -> dict:
    n = 16
    names = (C.c_char_p * n)()
    launches = np.zeros(n, dtype=np.int64)
    ms = np.zeros(n)
    n_out = C.c_int32()
    _check(ctx, load().vg_get_profile(ctx, n, names, launches.ctypes.data_as(_I64), _dp(ms),
                                      C.byref(n_out)))
    return {names[k].decode(): (int(launches[k]), float(ms[k])) for k in range(n_out.value)}


def vg_device_bytes(ctx) -> int:
    b = C.c_int64()
    _check(ctx, load().vg_device_bytes(ctx, C.byref(b)))
    return b.value


def vg_step_noalloc(ctx, w_in_ptr: int, w_out_ptr: int, t: float) -> float:
    """One step on caller-owned device states ([3][nc], internal cell order) that
    allocates no device memory; returns the step's dt."""
    dt = C.c_double()
    _check(ctx, load().vg_step_noalloc(ctx, _V(w_in_ptr), _V(w_out_ptr), float(t), C.byref(dt)))
    return dt.value


def vg_set_depth(ctx, depth_v) -> None:
    d = _f64(depth_v)
    _check(ctx, load().vg_set_depth(ctx, _dp(d)))


def _boundary_arrays(edges, kinds):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    if isinstance(kinds, str):
        kinds = [kinds] * e.shape[0]
    k = np.ascontiguousarray([BOUNDARY[x] if isinstance(x, str) else int(x) for x in kinds], dtype=np.int32)
    if k.shape[0] != e.shape[0]:
        raise ValueError("one boundary kind per edge")
    return e, k


def vg_adj_forward(ctx, n_steps: int, dt: float, checkpoint_every: int = 0) -> None:
    _check(ctx, load().vg_adj_forward(ctx, int(n_steps), float(dt), int(checkpoint_every)))


def vg_adj_backward(ctx, dJ_deta, nc: int, nv: int) -> dict:
    w = _f64(dJ_deta)
    out = {k: np.empty(nc) for k in ("H0", "Hu0", "Hv0", "z")}
    out["depth"] = np.empty(nv)
    _check(ctx, load().vg_adj_backward(ctx, _dp(w), _dp(out["H0"]), _dp(out["Hu0"]), _dp(out["Hv0"]),
                                       _dp(out["z"]), _dp(out["depth"])))
    return out


# ---------------------------------------------------------------- convenience wrapper


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)          # torch.cuda.Stream


class Solver:
    """One context: a mesh, parameters, a state and gauges on one GPU."""

    def __init__(self, precision: int = 64, device: int = 0, stream=None):
        self.precision = precision
        self.ctx = vg_create(precision, device, _stream_handle(stream))
        self.nc = 0
        self.n_gauges = 0

    def close(self) -> None:
        if getattr(self, "ctx", None):
            vg_destroy(self.ctx)
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

    # mesh / parameters
    def upload_mesh(self, mesh=None, xy=None, tri=None, depth=None, renumber="hilbert") -> None:
        if mesh is not None:
            xy, tri, depth = mesh.xy, mesh.tri, mesh.depth
        vg_mesh_upload(self.ctx, xy, tri, depth, renumber)
        self.nc = int(np.asarray(tri).reshape(-1, 3).shape[0])
        self.n_gauges = 0

    def set_params(self, **kw) -> vg_params:
        p = vg_get_params(self.ctx)
        for k, v in kw.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        vg_set_params(self.ctx, p)
        return p

    @property
    def params(self) -> dict:
        p = vg_get_params(self.ctx)
        return {k: getattr(p, k) for k, _ in vg_params._fields_}

    def permutation(self) -> np.ndarray:
        return vg_get_permutation(self.ctx, self.nc)

    # state
    def set_state(self, H, Hu, Hv, t: float = 0.0) -> None:
        if hasattr(H, "is_cuda") and H.is_cuda:
            import torch
            dt = torch.float64 if self.precision == 64 else torch.float32
            H, Hu, Hv = (x.to(dt).contiguous() for x in (H, Hu, Hv))
            vg_set_state_dev(self.ctx, H.data_ptr(), Hu.data_ptr(), Hv.data_ptr(), t)
            self._keep = (H, Hu, Hv)
        elif all(getattr(x, "dtype", None) == np.float32 for x in (H, Hu, Hv)):
            vg_set_state_f32(self.ctx, H, Hu, Hv, t)
        else:
            vg_set_state(self.ctx, H, Hu, Hv, t)

    def get_state(self, dtype=np.float64, out=None):
        """(H, Hu, Hv, t) as numpy arrays (float64, or float32 through the FP32
        host interface) in the original cell order."""
        if np.dtype(dtype) == np.float32:
            return vg_get_state_f32(self.ctx, self.nc, out)
        return vg_get_state(self.ctx, self.nc, out)

    def get_state_dev(self, out=None):
        import torch
        dt = torch.float64 if self.precision == 64 else torch.float32
        if out is None:
            out = tuple(torch.empty(self.nc, dtype=dt, device="cuda") for _ in range(3))
        vg_get_state_dev(self.ctx, out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
        return out

    # gauges and stepping
    def set_gauges(self, xy) -> np.ndarray:
        xy = _f64(xy).reshape(-1, 2)
        vg_set_gauges(self.ctx, xy)
        self.n_gauges = xy.shape[0]
        return vg_get_gauge_cells(self.ctx, self.n_gauges)

    def step(self, n: int = 1) -> None:
        vg_step(self.ctx, n)

    def advance_to(self, t: float) -> None:
        vg_advance_to(self.ctx, t)

    def gauges(self):
        return vg_get_gauges(self.ctx, self.n_gauges)

    def diagnostics(self) -> dict:
        return vg_get_diagnostics(self.ctx)

    def profile(self, enable: bool = True) -> None:
        vg_profile(self.ctx, enable)

    def get_profile(self) -> dict:
        return vg_get_profile(self.ctx)

    def device_bytes(self) -> int:
        return vg_device_bytes(self.ctx)

    def set_depth(self, depth_v) -> None:
        vg_set_depth(self.ctx, depth_v)

    def set_open_boundary(self, edges) -> None:
        """Open (transmissive) boundary edges [(a, b), ...] (vg_set_open_boundary)."""
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        _check(self.ctx, load().vg_set_open_boundary(self.ctx, e.shape[0], e.ctypes.data_as(_I32)))

    def set_boundary(self, edges, kinds) -> None:
        """Boundary kinds per edge [(a, b), ...]: "wall", "open" or "absorbing" (or
        1, 2, 3); every other boundary face a wall (vg_set_boundary)."""
        e, k = _boundary_arrays(edges, kinds)
        _check(self.ctx, load().vg_set_boundary(self.ctx, e.shape[0], e.ctypes.data_as(_I32), k.ctypes.data_as(_I32)))

    def set_bed_motion(self, uplift_v, onset_v=None, rise: float = 0.0) -> None:
        """Moving bed (vg_set_bed_motion); uplift_v None removes it."""
        if uplift_v is None:
            _check(self.ctx, load().vg_set_bed_motion(self.ctx, None, None, 0.0))
            return
        up, on = _f64(uplift_v), _f64(onset_v)
        _check(self.ctx, load().vg_set_bed_motion(self.ctx, _dp(up), _dp(on), float(rise)))

    def adj_forward(self, n_steps: int, dt: float = 0.0, checkpoint_every: int = 0):
        """Run keeping checkpoints, with the fixed step dt or (dt = 0) the CFL
        step of every step; returns the gauge records (t, eta)."""
        vg_adj_forward(self.ctx, n_steps, dt, checkpoint_every)
        return self.gauges()

    def adj_forward_binomial(self, n_steps: int, dt: float = 0.0, slots: int = 8):
        """adj_forward for binomial checkpointing with `slots` state buffers."""
        _check(self.ctx, load().vg_adj_forward_binomial(self.ctx, int(n_steps), float(dt), int(slots)))
        return self.gauges()

    def adj_backward(self, dJ_deta, nv: int) -> dict:
        return vg_adj_backward(self.ctx, dJ_deta, self.nc, nv)

    def adj_bed_gradient(self, nv: int):
        """(dJ/duplift_v, dJ/donset_v) after adj_backward of a run with a moving bed."""
        gu, go = np.empty(nv), np.empty(nv)
        _check(self.ctx, load().vg_adj_bed_gradient(self.ctx, _dp(gu), _dp(go)))
        return gu, go


# ---------------------------------------------------------------- batched ensembles


def _bcheck(b, rc: int) -> None:
    if rc != VG_OK:
        lib = load()
        msg = lib.vg_batch_last_error(b).decode() if b else ""
        raise VolnaError(rc, msg or lib.vg_strerror(rc).decode())


class Batch:
    """Many scenarios on several meshes advanced together (vg_batch_*)."""

    def __init__(self, precision: int = 32, device: int = 0, stream=None):
        h = _V()
        rc = load().vg_batch_create(C.byref(h), int(precision), int(device),
                                    _V(_stream_handle(stream)) if stream is not None else None)
        if rc != VG_OK:
            raise VolnaError(rc, f"vg_batch_create failed: {vg_strerror(rc)}")
        self.h = h
        self.precision = precision
        self.nc = []
        self.n_gauges = {}

    def close(self) -> None:
        if getattr(self, "h", None):
            load().vg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, **kw) -> None:
        p = vg_default_params()
        for k, v in kw.items():
            setattr(p, k, v)
        _bcheck(self.h, load().vg_batch_set_params(self.h, C.byref(p)))

    def add_mesh(self, mesh, n_scenarios: int, renumber="hilbert") -> int:
        xy = _f64(mesh.xy).reshape(-1, 2)
        tri = np.ascontiguousarray(mesh.tri, dtype=np.int32).reshape(-1, 3)
        depth = _f64(mesh.depth)
        mid = C.c_int32()
        r = RENUMBER[renumber] if isinstance(renumber, str) else int(renumber)
        _bcheck(self.h, load().vg_batch_add_mesh(self.h, xy.shape[0], _dp(xy), tri.shape[0],
                                                 tri.ctypes.data_as(_I32), _dp(depth), r,
                                                 int(n_scenarios), C.byref(mid)))
        self.nc.append(tri.shape[0])
        return mid.value

    def set_state(self, mesh_id: int, scen: int, H, Hu, Hv, t: float = 0.0) -> None:
        H, Hu, Hv = _f64(H), _f64(Hu), _f64(Hv)
        _bcheck(self.h, load().vg_batch_set_state(self.h, mesh_id, scen, _dp(H), _dp(Hu), _dp(Hv),
                                                  float(t)))

    def get_state(self, mesh_id: int, scen: int):
        n = self.nc[mesh_id]
        H, Hu, Hv = np.empty(n), np.empty(n), np.empty(n)
        t = C.c_double()
        steps = C.c_int64()
        _bcheck(self.h, load().vg_batch_get_state(self.h, mesh_id, scen, _dp(H), _dp(Hu), _dp(Hv),
                                                  C.byref(t), C.byref(steps)))
        return H, Hu, Hv, t.value, steps.value

    def step(self, n: int) -> None:
        _bcheck(self.h, load().vg_batch_step(self.h, int(n)))

    def run(self, t_end: float, max_steps: int = 10 ** 9) -> int:
        taken = C.c_int64()
        _bcheck(self.h, load().vg_batch_run(self.h, float(t_end), int(max_steps), C.byref(taken)))
        return taken.value

    def autotune(self, n_steps: int = 4):
        """(block cells, ms per step, CTAs per SM or 0 for as many as fit) of the
        fastest launch shape (vg_batch_autotune)."""
        blk, ctas = C.c_int32(), C.c_int32()
        ms = C.c_double()
        _bcheck(self.h, load().vg_batch_autotune(self.h, int(n_steps), C.byref(blk), C.byref(ctas), C.byref(ms)))
        return blk.value, ms.value, ctas.value

    def set_gauges(self, mesh_id: int, xy) -> None:
        xy = _f64(xy).reshape(-1, 2)
        _bcheck(self.h, load().vg_batch_set_gauges(self.h, int(mesh_id), xy.shape[0],
                                                   _dp(xy) if xy.shape[0] else None))
        self.n_gauges[mesh_id] = xy.shape[0]

    def set_open_boundary(self, mesh_id: int, edges) -> None:
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        _bcheck(self.h, load().vg_batch_set_open_boundary(self.h, int(mesh_id), e.shape[0],
                                                          e.ctypes.data_as(_I32)))

    def set_boundary(self, mesh_id: int, edges, kinds) -> None:
        e, k = _boundary_arrays(edges, kinds)
        _bcheck(self.h, load().vg_batch_set_boundary(self.h, int(mesh_id), e.shape[0], e.ctypes.data_as(_I32),
                                                     k.ctypes.data_as(_I32)))

    def gauges(self, mesh_id: int, scen: int):
        """Gauge records (t [n], eta [n, G]) of one scenario."""
        n = C.c_int64()
        _bcheck(self.h, load().vg_batch_get_gauges(self.h, int(mesh_id), int(scen), None, None, 0, C.byref(n)))
        G = self.n_gauges.get(mesh_id, 0)
        t, eta = np.empty(n.value), np.empty((n.value, G))
        if n.value:
            _bcheck(self.h, load().vg_batch_get_gauges(self.h, int(mesh_id), int(scen), _dp(t), _dp(eta),
                                                       n.value, C.byref(n)))
        return t, eta

    def info(self) -> dict:
        nm, ns = C.c_int32(), C.c_int32()
        cells, launches = C.c_int64(), C.c_int64()
        _bcheck(self.h, load().vg_batch_info(self.h, C.byref(nm), C.byref(ns), C.byref(cells),
                                             C.byref(launches)))
        return dict(meshes=nm.value, scenarios=ns.value, cells=cells.value, launches=launches.value)
