"""Helpers of the GPU tests: run the CUDA path and the oracle on the same seeded
inputs, compare field by field, and cut oracle-sized patches out of big meshes."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2002_04889_gb300 import inputs as I
from paper_2002_04889_gb300 import volna

FIELDS = ("H", "Hu", "Hv")


def rel_l2(a, b) -> float:
    nb = float(np.linalg.norm(b))
    na = float(np.linalg.norm(np.asarray(a) - np.asarray(b)))
    if nb == 0.0:
        return na
    return na / nb


def gpu_run(mesh, state, n_steps, precision=64, renumber="morton", gauges=None, **params):
    with volna.Solver(precision=precision, device=0) as sv:
        sv.set_params(**params)
        sv.upload_mesh(mesh, renumber=renumber)
        if gauges is not None:
            sv.set_gauges(gauges)
        sv.set_state(state.H, state.Hu, state.Hv, state.t)
        sv.step(n_steps)
        H, Hu, Hv, t = sv.get_state()
        out = dict(H=H, Hu=Hu, Hv=Hv, t=t, diag=sv.diagnostics())
        if gauges is not None:
            out["gauge_t"], out["gauge_eta"] = sv.gauges()
        return out


def oracle_params(**params):
    keys = ("g", "cfl", "h_threshold", "dt_fixed", "dt_max", "t_end", "order")
    return O.params(**{k: v for k, v in params.items() if k in keys})


def oracle_run(mesh, state, n_steps, gauges=None, **params):
    om = O.OracleMesh.from_mesh(mesh)
    cells = om.locate(gauges) if gauges is not None else None
    r = om.run(oracle_params(**params), (state.H, state.Hu, state.Hv, state.t), n_steps,
               gauge_cells=cells)
    r["z"] = om.get("z")
    r["gauge_cells"] = cells
    return r


class VertexAdjacency:
    """Cells around each vertex (CSR), built once for a mesh."""

    def __init__(self, tri: np.ndarray, nv: int):
        self.tri = tri
        flat = tri.ravel().astype(np.int64)
        order = np.argsort(flat, kind="stable")
        counts = np.bincount(flat, minlength=nv)
        self.start = np.concatenate([[0], np.cumsum(counts)])
        self.cell_of = (order // 3).astype(np.int64)

    def rings(self, seeds, rings: int) -> np.ndarray:
        """Cells within `rings` vertex-adjacency steps of the seed cells (a superset
        of their face-adjacency rings), as sorted original ids."""
        found = set(int(c) for c in np.atleast_1d(seeds))
        frontier = np.asarray(sorted(found), dtype=np.int64)
        for _ in range(rings):
            verts = np.unique(self.tri[frontier].ravel())
            new = np.unique(np.concatenate([self.cell_of[self.start[v]:self.start[v + 1]] for v in verts]))
            new = np.array([c for c in new if int(c) not in found], dtype=np.int64)
            found.update(int(c) for c in new)
            frontier = new
            if frontier.size == 0:
                break
        return np.array(sorted(found), dtype=np.int64)


def patch_mesh(mesh, cells: np.ndarray):
    """Sub-mesh of the given cells with vertices renumbered in increasing order (so
    the smallest-vertex-id rule picks the same local face order)."""
    sub = mesh.tri[cells]
    verts, inv = np.unique(sub.ravel(), return_inverse=True)
    return I.Mesh(mesh.xy[verts], inv.reshape(-1, 3).astype(np.int32), mesh.depth[verts])
