"""Plain FP64 CPU oracle of the finite-volume shallow-water step (ctypes binding).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  It shares no
code with the CUDA library in ``paper_2002_04889_gb300`` and never calls it.

The arithmetic lives in ``volna_oracle.c`` (built by ``oracle.build``); this
module only marshals numpy arrays.  Every function cites the section of
Giles et al., "Performance analysis of Volna-OP2", that it follows.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import library_path, build as _build

_lib = None
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)


class Params(C.Structure):
    """Scheme parameters: g (9.81), CFL, H_threshold (Sec. 2.4), fixed / max dt,
    end time, order (1 first order, 2 MUSCL reconstruction of Sec. 2.4) and
    limiter (1 Barth-Jespersen; 0 none, only for the convergence pins)."""
    _fields_ = [("g", C.c_double), ("cfl", C.c_double), ("h_threshold", C.c_double),
                ("dt_fixed", C.c_double), ("dt_max", C.c_double), ("t_end", C.c_double),
                ("order", C.c_int32), ("limiter", C.c_int32)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        _build()
    lib = C.CDLL(path)
    lib.vo_mesh_build.argtypes = [C.c_int64, _D, C.c_int64, _I32, _D, C.POINTER(C.c_void_p)]
    lib.vo_mesh_build.restype = C.c_int
    lib.vo_mesh_free.argtypes = [C.c_void_p]
    lib.vo_default_params.argtypes = [C.POINTER(Params)]
    lib.vo_hll_normal.argtypes = [C.c_double] * 7 + [_D, _D]
    lib.vo_hll_speeds.argtypes = [C.c_double] * 5 + [_D]
    lib.vo_face_flux.argtypes = ([C.c_double] * 10 + [C.c_double, C.c_double, C.c_int]
                                 + [_D, _D, _D, _D])
    lib.vo_reconstruct_cell.argtypes = [C.c_void_p, C.POINTER(Params), _D, _D, _D, C.c_int64,
                                        _D, _D, _D, _D]
    lib.vo_reconstruct_cell.restype = C.c_int
    lib.vo_residual.argtypes = [C.c_void_p, C.POINTER(Params), _D, _D, _D, _D, _D, _D, _D]
    lib.vo_time_step.argtypes = [C.c_void_p, C.POINTER(Params), _D, C.c_double]
    lib.vo_time_step.restype = C.c_double
    lib.vo_step.argtypes = [C.c_void_p, C.POINTER(Params), _D, _D, _D, _D, _D, _I64]
    lib.vo_run.argtypes = [C.c_void_p, C.POINTER(Params), _D, _D, _D, _D, C.c_int64, _D, _I64,
                           C.c_int32, _I32, _D]
    lib.vo_run.restype = C.c_int64
    lib.vo_run_bed.argtypes = [C.c_void_p, C.POINTER(Params), _D, _D, _D, _D, C.c_int64, _D, _I64,
                               C.c_int32, _I32, _D, _D, _D, _D, C.c_double]
    lib.vo_run_bed.restype = C.c_int64
    lib.vo_bed_at.argtypes = [C.c_void_p, _D, _D, _D, C.c_double, C.c_double]
    lib.vo_set_open.argtypes = [C.c_void_p, C.c_int64, _I32]
    lib.vo_set_open.restype = C.c_int
    lib.vo_set_boundary.argtypes = [C.c_void_p, C.c_int64, _I32, _I32]
    lib.vo_set_boundary.restype = C.c_int
    lib.vo_locate.argtypes = [C.c_void_p, _D, C.c_int32, _D, _I32]
    lib.vo_mesh_get.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
    lib.vo_mesh_get.restype = C.c_int
    lib.vo_mesh_n_flipped.argtypes = [C.c_void_p]
    lib.vo_mesh_n_flipped.restype = C.c_int64
    lib.vo_set_threads.argtypes = [C.c_int]
    lib.vo_max_threads.restype = C.c_int
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    """OpenMP threads for the cell and edge loops (results do not depend on it)."""
    _load().vo_set_threads(int(n))


def max_threads() -> int:
    return int(_load().vo_max_threads())


def params(g=9.81, cfl=0.9, h_threshold=1e-5, dt_fixed=0.0, dt_max=0.0, t_end=0.0,
           order=2, limiter=1) -> Params:
    return Params(g, cfl, h_threshold, dt_fixed, dt_max, t_end, order, limiter)


def hll_normal(g, HL, unL, utL, HR, unR, utR):
    """HLL flux in the normal frame with the Sec. 2.2 wave speeds; returns (F[3], a)."""
    F = np.zeros(3)
    a = C.c_double()
    _load().vo_hll_normal(g, HL, unL, utL, HR, unR, utR, _dp(F), C.byref(a))
    return F, a.value


def hll_speeds(g, HL, unL, HR, unR):
    """(s_L, s_R) of Sec. 2.2 (dry-bed speeds when one side is dry)."""
    s = np.zeros(2)
    _load().vo_hll_speeds(g, HL, unL, HR, unR, _dp(s))
    return float(s[0]), float(s[1])


def face_flux(g, hthr, left, zL, right, zR, n, wall=False):
    """Flux through a face seen from the left cell (hydrostatic reconstruction +
    HLL, Sec. 2.2; wall ghost of Sec. 2.5; wall="open" for the transmissive
    ghost of vo_set_open, wall="absorbing" for the characteristic ghost of
    vo_set_boundary).  left/right = (H_f, Hu_f, Hv_f).
    Returns (Phi[3], P_L, P_R, a)."""
    Phi = np.zeros(3)
    PL, PR, a = C.c_double(), C.c_double(), C.c_double()
    r = right if right is not None else (0.0, 0.0, 0.0)
    _load().vo_face_flux(g, hthr, left[0], left[1], left[2], zL, r[0], r[1], r[2], zR,
                         n[0], n[1], {"open": 2, "absorbing": 3}.get(wall, 1 if wall else 0), _dp(Phi), C.byref(PL), C.byref(PR),
                         C.byref(a))
    return Phi, PL.value, PR.value, a.value


class OracleMesh:
    """Mesh with geometry, adjacency and bed of Sec. 2 (see volna_oracle.c)."""

    _FIELDS = {"vtx": (0, np.int32, 3), "nbr": (1, np.int32, 3), "nbr_face": (2, np.int32, 3),
               "z": (3, np.float64, 1), "area": (4, np.float64, 1), "cx": (5, np.float64, 1),
               "cy": (6, np.float64, 1), "nx": (7, np.float64, 3), "ny": (8, np.float64, 3),
               "len": (9, np.float64, 3), "fx": (10, np.float64, 3), "fy": (11, np.float64, 3),
               "wx": (12, np.float64, 3), "wy": (13, np.float64, 3), "dx": (14, np.float64, 3),
               "dy": (15, np.float64, 3), "zf": (16, np.float64, 3)}

    def __init__(self, xy, tri, depth):
        lib = _load()
        self.xy = _f64(xy).reshape(-1, 2)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
        self.depth = _f64(depth)
        h = C.c_void_p()
        rc = lib.vo_mesh_build(self.xy.shape[0], _dp(self.xy), self.tri.shape[0],
                               self.tri.ctypes.data_as(_I32), _dp(self.depth), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle mesh rejected (code {rc})")
        self._h = h
        self.nc = self.tri.shape[0]

    @classmethod
    def from_mesh(cls, mesh):
        return cls(mesh.xy, mesh.tri, mesh.depth)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.vo_mesh_free(self._h)
            self._h = None

    def get(self, name):
        what, dt, k = self._FIELDS[name]
        out = np.empty(self.nc * k, dtype=dt)
        _load().vo_mesh_get(self._h, what, out.ctypes.data_as(C.c_void_p))
        return out.reshape(self.nc, 3) if k == 3 else out

    @property
    def n_flipped(self):
        return int(_load().vo_mesh_n_flipped(self._h))

    def reconstruct_cell(self, prm, H, Hu, Hv, K, with_bed=False):
        """Face values (H_f, Hu_f, Hv_f) of cell K (Sec. 2.4); with_bed: also the
        bed under each face value and whether the cell reconstructed."""
        H, Hu, Hv = _f64(H), _f64(Hu), _f64(Hv)
        o = [np.zeros(3) for _ in range(4)]
        rec = _load().vo_reconstruct_cell(self._h, C.byref(prm), _dp(H), _dp(Hu), _dp(Hv), int(K),
                                          _dp(o[0]), _dp(o[1]), _dp(o[2]), _dp(o[3]))
        return (o[0], o[1], o[2], o[3], bool(rec)) if with_bed else o[:3]

    def residual(self, prm, H, Hu, Hv):
        """L(w) and per-cell max l_f a_f (Sec. 2.2)."""
        H, Hu, Hv = _f64(H), _f64(Hu), _f64(Hv)
        R = [np.zeros(self.nc) for _ in range(3)]
        am = np.zeros(self.nc)
        _load().vo_residual(self._h, C.byref(prm), _dp(H), _dp(Hu), _dp(Hv),
                            _dp(R[0]), _dp(R[1]), _dp(R[2]), _dp(am))
        return R, am

    def time_step(self, prm, amax, t):
        return float(_load().vo_time_step(self._h, C.byref(prm), _dp(_f64(amax)), float(t)))

    def locate(self, pts):
        pts = _f64(pts).reshape(-1, 2)
        out = np.zeros(pts.shape[0], dtype=np.int32)
        _load().vo_locate(self._h, _dp(self.xy), pts.shape[0], _dp(pts), out.ctypes.data_as(_I32))
        return out

    def run(self, prm, state, n_steps, gauge_cells=None, bed_motion=None):
        """n SSP-RK(2,2) steps (Sec. 2.3) from state (H, Hu, Hv, t), on copies.
        bed_motion = (depth0_v, uplift_v, onset_v, rise): the moving bed of
        vo_bed_at (time-dependent depth, Sec. 2.1); the mesh keeps the bed of
        the final time afterwards.
        Returns dict(H, Hu, Hv, t, dts, neg_count, gauges[n_steps, G])."""
        H, Hu, Hv = _f64(state[0]).copy(), _f64(state[1]).copy(), _f64(state[2]).copy()
        t = C.c_double(float(state[3]) if len(state) > 3 else 0.0)
        dts = np.zeros(max(int(n_steps), 1))
        neg = C.c_int64(0)
        gc = ge = None
        if gauge_cells is not None and len(gauge_cells):
            gc = np.ascontiguousarray(gauge_cells, dtype=np.int32)
            ge = np.zeros((max(int(n_steps), 1), gc.shape[0]))
        g_args = (gc.shape[0], gc.ctypes.data_as(_I32), _dp(ge)) if gc is not None else (0, None, None)
        if bed_motion is None:
            _load().vo_run(self._h, C.byref(prm), _dp(H), _dp(Hu), _dp(Hv), C.byref(t),
                           int(n_steps), _dp(dts), C.byref(neg), *g_args)
        else:
            d0, up, on = (_f64(a) for a in bed_motion[:3])
            _load().vo_run_bed(self._h, C.byref(prm), _dp(H), _dp(Hu), _dp(Hv), C.byref(t),
                               int(n_steps), _dp(dts), C.byref(neg), *g_args,
                               _dp(d0), _dp(up), _dp(on), float(bed_motion[3]))
        return dict(H=H, Hu=Hu, Hv=Hv, t=t.value, dts=dts[:n_steps], neg_count=neg.value,
                    gauges=None if ge is None else ge[:n_steps])

    def set_open(self, edges):
        """Marks the boundary edges [(a, b), ...] (vertex ids) open, every other
        boundary face a wall (vo_set_open, transmissive ghost)."""
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        rc = _load().vo_set_open(self._h, e.shape[0], e.ctypes.data_as(_I32))
        if rc != 0:
            raise ValueError("an edge is not a boundary face of the mesh")

    def set_boundary(self, edges, kinds):
        """Boundary kinds per edge [(a, b), ...]: 1 wall, 2 open, 3 absorbing (the
        characteristic ghost of a sea at rest beyond the boundary); every other
        boundary face a wall (vo_set_boundary)."""
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        k = np.ascontiguousarray(np.asarray(kinds, dtype=np.int32).reshape(-1))
        if k.shape[0] != e.shape[0]:
            raise ValueError("one kind per edge")
        rc = _load().vo_set_boundary(self._h, e.shape[0], e.ctypes.data_as(_I32), k.ctypes.data_as(_I32))
        if rc != 0:
            raise ValueError("an edge is not a boundary face of the mesh, or an unknown kind")

    def bed_at(self, depth0, uplift, onset, rise, t):
        """Sets the cell beds to the moving bed at time t (vo_bed_at) and returns them."""
        _load().vo_bed_at(self._h, _dp(_f64(depth0)), _dp(_f64(uplift)), _dp(_f64(onset)),
                          float(rise), float(t))
        return self.get("z")

    def mass(self, H):
        """Discrete mass sum_K |K| H_K."""
        return float(np.sum(self.get("area") * _f64(H)))


_ad = None


def _load_ad():
    global _ad
    if _ad is not None:
        return _ad
    from .build import ad_library_path, build_ad
    path = ad_library_path()
    build_ad()
    lib = C.CDLL(path)
    lib.vo_ad_gauge_gradient.argtypes = [C.c_int64, _D, C.c_int64, _I32, _D, _D, _D, _D, C.c_double,
                                         C.c_double, C.c_int, C.c_double, C.c_double, C.c_int64, C.c_int32,
                                         _I32, _D, _D, _D, _D, _D, _D, _D, _D]
    lib.vo_ad_gauge_gradient.restype = C.c_int
    lib.vo_ad_gauge_gradient_bed.argtypes = [C.c_int64, _D, C.c_int64, _I32, _D, _D, _D, _D, C.c_double,
                                             C.c_double, C.c_int, C.c_double, C.c_double, C.c_int64, C.c_int32,
                                             _I32, _D, _D, _D, C.c_double, _D, _D, _D, _D, _D, _D, _D, _D, _D]
    lib.vo_ad_gauge_gradient_bed.restype = C.c_int
    lib.vo_ad_set_open.argtypes = [C.c_int64, _I32]
    lib.vo_ad_set_open.restype = C.c_int
    lib.vo_ad_set_boundary.argtypes = [C.c_int64, _I32, _I32]
    lib.vo_ad_set_boundary.restype = C.c_int
    _ad = lib
    return lib


def ad_gauge_gradient(mesh, state, dt, n_steps, gauge_cells, weights, g=9.81, h_threshold=1e-5,
                      order=2, cfl=0.9, bed_motion=None, open_edges=None, boundary_kinds=None):
    """The oracle's discrete adjoint (tape AD of the oracle's own arithmetic) of
    J = sum_{n,g} weights[n, g] * eta_g(t_n), n = 0..n_steps (Sec. 2.3 steps), with
    the fixed time step dt, or for dt = 0 / None the CFL step of each step,
    differentiated through its minimum.  bed_motion = (uplift_v, onset_v, rise):
    the moving bed of vo_bed_at over the mesh's depths, also differentiated.
    open_edges: boundary edges [(a, b), ...] made open (vo_set_open), or of the
    kinds boundary_kinds [n] (1 wall, 2 open, 3 absorbing: vo_set_boundary).
    Returns dict(J, eta[n+1, G], dts[n], dH0, dHu0, dHv0, ddepth[, duplift, donset])."""
    oe = np.ascontiguousarray(np.asarray(open_edges if open_edges is not None else [], dtype=np.int32).reshape(-1, 2))
    bk = None
    if boundary_kinds is not None:
        bk = np.ascontiguousarray(np.broadcast_to(np.asarray(boundary_kinds, dtype=np.int32), (oe.shape[0],)))
    _load_ad().vo_ad_set_boundary(oe.shape[0], oe.ctypes.data_as(_I32), None if bk is None else bk.ctypes.data_as(_I32))
    xy = _f64(mesh.xy).reshape(-1, 2)
    tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
    depth = _f64(mesh.depth)
    H0, Hu0, Hv0 = (_f64(a) for a in state[:3])
    gc = np.ascontiguousarray(gauge_cells, dtype=np.int32)
    w = _f64(weights).reshape(n_steps + 1, gc.shape[0])
    nc, nv = tri.shape[0], xy.shape[0]
    eta = np.zeros((n_steps + 1, gc.shape[0]))
    dts = np.zeros(max(int(n_steps), 1))
    J = C.c_double()
    out = [np.zeros(nc) for _ in range(3)] + [np.zeros(nv)]
    if bed_motion is None:
        rc = _load_ad().vo_ad_gauge_gradient(nv, _dp(xy), nc, tri.ctypes.data_as(_I32), _dp(depth),
                                             _dp(H0), _dp(Hu0), _dp(Hv0), g, h_threshold, order, float(cfl),
                                             float(dt or 0.0), int(n_steps), gc.shape[0], gc.ctypes.data_as(_I32),
                                             _dp(w), _dp(eta), _dp(dts), C.byref(J), *(_dp(o) for o in out))
    else:
        up, on = _f64(bed_motion[0]), _f64(bed_motion[1])
        out += [np.zeros(nv), np.zeros(nv)]
        rc = _load_ad().vo_ad_gauge_gradient_bed(nv, _dp(xy), nc, tri.ctypes.data_as(_I32), _dp(depth),
                                                 _dp(H0), _dp(Hu0), _dp(Hv0), g, h_threshold, order, float(cfl),
                                                 float(dt or 0.0), int(n_steps), gc.shape[0],
                                                 gc.ctypes.data_as(_I32), _dp(w), _dp(up), _dp(on),
                                                 float(bed_motion[2]), _dp(eta), _dp(dts), C.byref(J),
                                                 *(_dp(o) for o in out))
    _load_ad().vo_ad_set_boundary(0, None, None)
    if rc != 0:
        raise ValueError(f"oracle mesh rejected (code {rc})")
    r = dict(J=J.value, eta=eta, dts=dts[:n_steps], dH0=out[0], dHu0=out[1], dHv0=out[2], ddepth=out[3])
    if bed_motion is not None:
        r["duplift"], r["donset"] = out[4], out[5]
    return r


_count = None


def count_step_ops(mesh, state, g=9.81, h_threshold=1e-5, cfl=0.9) -> dict:
    """Floating-point operations of one adaptive SSP-RK(2,2) step (Sec. 2.3) of
    the oracle's arithmetic from `state`, counted by the oracle compiled with an
    operation-counting scalar (op_count.hpp): add, sub, mul, div, sqrt, minmax
    (min/max/abs), and the step dt."""
    global _count
    from .build import build_count
    if _count is None:
        lib = C.CDLL(build_count())
        lib.vo_count_step.argtypes = [C.c_int64, _D, C.c_int64, _I32, _D, _D, _D, _D, C.c_double,
                                      C.c_double, C.c_double, _I64, _D]
        lib.vo_count_step.restype = C.c_int
        _count = lib
    xy = _f64(mesh.xy).reshape(-1, 2)
    tri = np.ascontiguousarray(mesh.tri, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(6, dtype=np.int64)
    dt = C.c_double()
    rc = _count.vo_count_step(xy.shape[0], _dp(xy), tri.shape[0], tri.ctypes.data_as(_I32), _dp(_f64(mesh.depth)),
                              _dp(_f64(state[0])), _dp(_f64(state[1])), _dp(_f64(state[2])), float(g),
                              float(h_threshold), float(cfl), out.ctypes.data_as(_I64), C.byref(dt))
    if rc != 0:
        raise ValueError(f"vo_count_step failed ({rc})")
    keys = ("add", "sub", "mul", "div", "sqrt", "minmax")
    r = {k: int(v) for k, v in zip(keys, out)}
    r["dt"] = dt.value
    return r
