"""Seeded synthetic inputs: meshes, bathymetry, initial states and gauge positions.

This module is shared by the CUDA path, the CPU oracle, the tests and the
benchmark.  It holds none of the finite-volume method's arithmetic (no cell
geometry, no reconstruction, no flux, no time stepping): it only builds the
inputs that the paper's workloads are shaped like.

* Thacker's periodic paraboloid basin (Sec. 3): a jittered structured grid of
  squares, each split along a seeded diagonal, over a parabolic bowl; the
  initial state is the closed-form solution at t = 0.
* A synthetic ocean-to-coast basin standing in for the Rockall Bank real case
  (Sec. 5, 800 x 1000 km domain, 450-2050 m resolutions), which needs
  bathymetry and a landslide source that are not available here: a conformal
  log-polar sector graded 20:1 towards the coast, a depth profile from a
  4000 m abyssal plain over a 200 m shelf to dry land, a seeded Gaussian
  random field perturbation, and an elliptical N-wave seafloor uplift.

All random numbers come from a counter-based splitmix64 generator written out
here, so the same seed gives the same inputs on every machine and numpy version.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function (Steele, Lea, Flood 2014) on a uint64 array."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from the splitmix64 counter sequence of (seed, stream)."""
    key = _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
    with np.errstate(over="ignore"):
        key = _mix64(key ^ np.uint64(stream & 0xFFFFFFFFFFFFFFFF))[0]
        idx = np.arange(offset, offset + n, dtype=np.uint64)
        z = _mix64(key + (idx + np.uint64(1)) * _GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Mesh:
    """An unstructured triangular mesh with per-vertex depth (positive down)."""
    xy: np.ndarray          # [nv, 2] float64 vertex coordinates
    tri: np.ndarray         # [nc, 3] int32 vertex ids, counter-clockwise
    depth: np.ndarray       # [nv] float64 bathymetry depth h (z = -h)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.xy.shape[0])

    @property
    def nc(self) -> int:
        return int(self.tri.shape[0])

    def vertex_mean(self, values: np.ndarray) -> np.ndarray:
        """Mean of a per-vertex field over each triangle's three vertices."""
        t = self.tri
        return (values[t[:, 0]] + values[t[:, 1]] + values[t[:, 2]]) / 3.0

    def cell_points(self) -> np.ndarray:
        """Vertex-mean point of each triangle, where cell initial data are sampled."""
        return np.stack([self.vertex_mean(self.xy[:, 0]), self.vertex_mean(self.xy[:, 1])], axis=1)


@dataclass
class State:
    H: np.ndarray
    Hu: np.ndarray
    Hv: np.ndarray
    t: float = 0.0


# ----------------------------------------------------------------------------
# Jittered structured grid (Thacker basin and its larger variants)
# ----------------------------------------------------------------------------

def _scatter_permutation(n: int, seed: int) -> np.ndarray:
    """A seeded permutation of range(n) that scatters neighbours far apart:
    k -> (a k + b) mod n with a coprime to n (no sort needed at 40M cells)."""
    u = uniform(seed, 4, 2)
    a = int(n * (0.5 + 0.3 * u[0])) | 1
    while math.gcd(a, n) != 1:
        a += 2
    b = int(n * u[1])
    k = np.arange(n, dtype=np.int64)
    return (a * k + b) % n


def jittered_grid(n: int, half_width: float, seed: int = 0, jitter: float = 0.2,
                  shuffle_cells: bool = False, ny: int | None = None,
                  half_height: float | None = None) -> tuple[np.ndarray, np.ndarray]:
    """n x ny squares on [-half_width, half_width] x [-half_height, half_height].

    Each square is split into two counter-clockwise triangles along a diagonal
    picked by a seeded coin flip; every interior vertex moves uniformly inside a
    disk of radius jitter * dx.  With shuffle_cells the triangles are emitted in
    a seeded random order (the library's renumbering restores locality).
    """
    ny = n if ny is None else ny
    half_height = half_width if half_height is None else half_height
    xs = -half_width + (2.0 * half_width) * np.arange(n + 1, dtype=np.float64) / n
    ys = -half_height + (2.0 * half_height) * np.arange(ny + 1, dtype=np.float64) / ny
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    X = X.ravel()
    Y = Y.ravel()
    nv = (n + 1) * (ny + 1)
    ii = np.tile(np.arange(n + 1), ny + 1)
    jj = np.repeat(np.arange(ny + 1), n + 1)
    interior = (ii > 0) & (ii < n) & (jj > 0) & (jj < ny)
    dx = min(2.0 * half_width / n, 2.0 * half_height / ny)
    rad = jitter * dx * np.sqrt(uniform(seed, 1, nv))
    ang = 2.0 * math.pi * uniform(seed, 2, nv)
    X = np.where(interior, X + rad * np.cos(ang), X)
    Y = np.where(interior, Y + rad * np.sin(ang), Y)
    xy = np.stack([X, Y], axis=1)

    nsq = n * ny
    sq = np.arange(nsq, dtype=np.int64)
    v00 = (sq // n) * (n + 1) + (sq % n)
    v10 = v00 + 1
    v01 = v00 + (n + 1)
    v11 = v01 + 1
    flip = uniform(seed, 3, nsq) < 0.5
    tri = np.empty((2 * nsq, 3), dtype=np.int32)
    # unflipped square: (v00, v10, v11) and (v00, v11, v01); flipped: (v00, v10, v01), (v10, v11, v01)
    tri[0::2, 0] = v00
    tri[0::2, 1] = v10
    tri[0::2, 2] = np.where(flip, v01, v11)
    tri[1::2, 0] = np.where(flip, v10, v00)
    tri[1::2, 1] = np.where(flip, v11, v11)
    tri[1::2, 2] = v01
    if shuffle_cells:
        tri = tri[_scatter_permutation(tri.shape[0], seed)]
    return xy, tri


def thacker_bowl_depth(xy: np.ndarray, h0: float, alpha: float) -> np.ndarray:
    """Depth h = h0 (1 - r^2 / alpha^2) of the paraboloid z(r) = -h (Sec. 3)."""
    r2 = xy[:, 0] ** 2 + xy[:, 1] ** 2
    return h0 * (1.0 - r2 / (alpha * alpha))


def thacker_mesh(n: int = 100, half_width: float = 2.0, seed: int = 0, h0: float = 0.1,
                 alpha: float = 1.0, r0: float = 0.8, shuffle_cells: bool = False) -> Mesh:
    """Thacker's paraboloid basin on a jittered n x n grid (Sec. 3 parameters by default:
    alpha = 1 m, r0 = 0.8 m, h0 = 0.1 m, domain [-2, 2]^2)."""
    xy, tri = jittered_grid(n, half_width, seed=seed, shuffle_cells=shuffle_cells)
    depth = thacker_bowl_depth(xy, h0, alpha)
    return Mesh(xy, tri, depth, name=f"thacker_{n}x{n}",
                meta=dict(h0=h0, alpha=alpha, r0=r0, half_width=half_width, n=n, seed=seed,
                          dx=2.0 * half_width / n))


def thacker_large_mesh(n: int = 4472, dx: float = 0.04, seed: int = 0,
                       shuffle_cells: bool = True) -> Mesh:
    """The Thacker generator on a wider domain at the same dx, with the bowl scaled
    up to the domain (alpha = half width, h0 = 0.1 alpha, r0 = 0.8 alpha)."""
    half = 0.5 * n * dx
    return thacker_mesh(n=n, half_width=half, seed=seed, h0=0.1 * half, alpha=half,
                        r0=0.8 * half, shuffle_cells=shuffle_cells)


def thacker_initial_state(mesh: Mesh, g: float = 9.81) -> State:
    """Thacker's solution at t = 0 sampled at each cell's vertex-mean point:
    H = max(0, eta0 - z_cell) with z_cell the vertex-mean bed, at rest."""
    h0 = mesh.meta["h0"]
    alpha = mesh.meta["alpha"]
    r0 = mesh.meta["r0"]
    A = (alpha * alpha - r0 * r0) / (alpha * alpha + r0 * r0)
    p = mesh.cell_points()
    r2 = p[:, 0] ** 2 + p[:, 1] ** 2
    k = (1.0 + A) / (1.0 - A)
    eta0 = h0 * (math.sqrt(k) - 1.0 - (r2 / (alpha * alpha)) * (k - 1.0))
    z = -mesh.vertex_mean(mesh.depth)
    H = np.maximum(0.0, eta0 - z)
    zero = np.zeros_like(H)
    return State(H, zero.copy(), zero.copy(), 0.0)


def thacker_free_surface(x, y, t: float, h0: float = 0.1, alpha: float = 1.0, r0: float = 0.8,
                         g: float = 9.81):
    """Free-surface elevation of Thacker's periodic paraboloid at time t (Sec. 3;
    the printed h(r, t) minus the bed), before clipping by the bed."""
    omega = math.sqrt(8.0 * g * h0) / alpha
    A = (alpha * alpha - r0 * r0) / (alpha * alpha + r0 * r0)
    c = 1.0 - A * math.cos(omega * t)
    r2 = np.asarray(x) ** 2 + np.asarray(y) ** 2
    return h0 * (math.sqrt(1.0 - A * A) / c - 1.0 - (r2 / (alpha * alpha)) * ((1.0 - A * A) / (c * c) - 1.0))


def lake_at_rest_state(mesh: Mesh, eta: float) -> State:
    """Still water at level eta over the mesh's bed (dry where the bed is above eta)."""
    z = -mesh.vertex_mean(mesh.depth)
    H = np.maximum(0.0, eta - z)
    zero = np.zeros_like(H)
    return State(H, zero.copy(), zero.copy(), 0.0)


def gaussian_hump_state(mesh: Mesh, eta0: float, amp: float, x0: float, y0: float,
                        width: float) -> State:
    """Still water at level eta0 plus a Gaussian hump of the free surface, at rest."""
    z = -mesh.vertex_mean(mesh.depth)
    p = mesh.cell_points()
    r2 = (p[:, 0] - x0) ** 2 + (p[:, 1] - y0) ** 2
    H = np.maximum(0.0, eta0 + amp * np.exp(-r2 / (width * width)) - z)
    zero = np.zeros_like(H)
    return State(H, zero.copy(), zero.copy(), 0.0)


def flat_basin_mesh(n: int, half_width: float, depth: float, seed: int = 0,
                    shuffle_cells: bool = False) -> Mesh:
    """All-wet control: the jittered grid over a flat bed of constant depth."""
    xy, tri = jittered_grid(n, half_width, seed=seed, shuffle_cells=shuffle_cells)
    return Mesh(xy, tri, np.full(xy.shape[0], float(depth)), name=f"flat_{n}x{n}",
                meta=dict(half_width=half_width, n=n, seed=seed, dx=2.0 * half_width / n))


def strip_mesh(nx: int, length: float, width_cells: int = 2, seed: int = 0) -> Mesh:
    """A y-invariant strip [-length/2, length/2] x [-w/2, w/2] with no jitter, flat bed 0."""
    dx = length / nx
    xy, tri = jittered_grid(nx, 0.5 * length, seed=seed, jitter=0.0, ny=width_cells,
                            half_height=0.5 * width_cells * dx)
    return Mesh(xy, tri, np.zeros(xy.shape[0]), name=f"strip_{nx}",
                meta=dict(dx=dx, length=length))


def dam_break_state(mesh: Mesh, h_left: float) -> State:
    """Water of depth h_left for x < 0, dry bed for x > 0, at rest (Ritter's problem)."""
    p = mesh.cell_points()
    H = np.where(p[:, 0] < 0.0, h_left, 0.0)
    zero = np.zeros_like(H)
    return State(H, zero.copy(), zero.copy(), 0.0)


def boundary_edges(mesh: Mesh, where=None) -> np.ndarray:
    """Boundary edges (in one triangle only) as vertex pairs [n, 2], optionally
    only those whose midpoint m satisfies where(m) (m: [n, 2] array -> bool)."""
    t = mesh.tri.astype(np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    key = np.sort(e, axis=1)
    uniq, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    b = uniq[cnt == 1]
    if where is not None and len(b):
        mid = 0.5 * (mesh.xy[b[:, 0]] + mesh.xy[b[:, 1]])
        b = b[np.asarray(where(mid), dtype=bool)]
    return b.astype(np.int32)


def radial_rupture(xy: np.ndarray, amplitude: float, x0: float, y0: float, width: float,
                   v_rupture: float, start: float = 0.0):
    """A moving-bed source at the vertices: Gaussian uplift amplitude exp(-r^2 /
    width^2) around (x0, y0) whose onset spreads outward from the centre at
    v_rupture (onset = start + r / v_rupture).  Returns (uplift_v, onset_v)."""
    r = np.hypot(xy[:, 0] - x0, xy[:, 1] - y0)
    return amplitude * np.exp(-(r / width) ** 2), start + r / v_rupture


# ----------------------------------------------------------------------------
# Synthetic ocean-to-coast basin (stand-in for the paper's Sec. 5 real case)
# ----------------------------------------------------------------------------

COAST_R_MIN = 50_000.0       # inner (land) boundary radius, m
COAST_R_MAX = 1_000_000.0    # outer (ocean) boundary radius, m
COAST_R_SHORE = 70_000.0     # shoreline radius, m


def coast_depth_profile(r: np.ndarray) -> np.ndarray:
    """Depth by radius: +50 m land at the inner boundary, shoreline at 70 km, a 200 m
    shelf from 120 to 250 km, a continental slope to a 4000 m abyssal plain at 350 km."""
    r = np.asarray(r, dtype=np.float64)
    d = np.empty_like(r)
    land = r < COAST_R_SHORE
    d[land] = -50.0 * (COAST_R_SHORE - r[land]) / (COAST_R_SHORE - COAST_R_MIN)
    ramp = (~land) & (r < 120_000.0)
    d[ramp] = 200.0 * (r[ramp] - COAST_R_SHORE) / (120_000.0 - COAST_R_SHORE)
    shelf = (r >= 120_000.0) & (r < 250_000.0)
    d[shelf] = 200.0
    slope = (r >= 250_000.0) & (r < 350_000.0)
    s = (r[slope] - 250_000.0) / 100_000.0
    d[slope] = 200.0 + 3800.0 * (s * s * (3.0 - 2.0 * s))
    d[r >= 350_000.0] = 4000.0
    return d


def gaussian_random_field(xy: np.ndarray, seed: int, n_modes: int = 256,
                          corr_len: float = 20_000.0, chunk: int = 1 << 18) -> np.ndarray:
    """Unit-variance stationary field: a sum of n_modes random-phase cosines with
    wavenumbers drawn around 1 / corr_len in uniformly random directions."""
    u = uniform(seed, 101, 3 * n_modes).reshape(3, n_modes)
    kmag = (0.5 + u[0]) / corr_len
    theta = 2.0 * math.pi * u[1]
    phase = 2.0 * math.pi * u[2]
    kx = kmag * np.cos(theta)
    ky = kmag * np.sin(theta)
    out = np.empty(xy.shape[0])
    amp = math.sqrt(2.0 / n_modes)
    for s in range(0, xy.shape[0], chunk):
        p = xy[s:s + chunk]
        arg = p[:, 0:1] * kx[None, :] + p[:, 1:2] * ky[None, :] + phase[None, :]
        out[s:s + chunk] = amp * np.cos(arg).sum(axis=1)
    return out


def coast_mesh(n_theta: int = 913, n_xi: int | None = None, seed: int = 0,
               jitter: float = 0.2, grf: bool = True) -> Mesh:
    """Conformal log-polar sector r in [50, 1000] km, theta in [0, 1] rad, with
    d(ln r) = d(theta): square cells of side r dtheta, about 55 m at the coast and
    1.1 km offshore (20:1 grading).  Defaults give 2 x 2735 x 913 ~ 5.0M triangles."""
    dth = 1.0 / n_theta
    xi_max = math.log(COAST_R_MAX / COAST_R_MIN)
    if n_xi is None:
        n_xi = int(round(xi_max / dth))
    # Grid in (xi, theta) space, jittered like the Thacker grid, then mapped.
    xy_l, tri = jittered_grid(n_xi, 0.5, seed=seed, jitter=jitter, ny=n_theta, half_height=0.5)
    # Map [-0.5, 0.5]^2 to xi in [0, xi_max], theta in [0, 1].  The jitter is
    # relative to the grid spacing, which after the map is isotropic.
    xi = (xy_l[:, 0] + 0.5) * xi_max
    th = (xy_l[:, 1] + 0.5) * 1.0
    r = COAST_R_MIN * np.exp(xi)
    xy = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    depth = coast_depth_profile(r)
    if grf:
        G = gaussian_random_field(xy, seed)
        depth = depth + 0.05 * np.maximum(np.abs(depth), 20.0) * G
    return Mesh(xy, tri, depth, name=f"coast_{n_xi}x{n_theta}",
                meta=dict(n_theta=n_theta, n_xi=n_xi, seed=seed))


def coast_mesh_with_cells(n_cells: int, seed: int) -> Mesh:
    """A coast basin with about n_cells triangles (same 3:1 grid aspect)."""
    xi_max = math.log(COAST_R_MAX / COAST_R_MIN)
    n_theta = max(2, int(round(math.sqrt(n_cells / (2.0 * xi_max)))))
    n_xi = max(2, int(round(n_cells / (2.0 * n_theta))))
    return coast_mesh(n_theta=n_theta, n_xi=n_xi, seed=seed)


def nwave_uplift(p: np.ndarray, amplitude: float = 3.0, center=(300_000.0 * math.cos(0.5),
                 300_000.0 * math.sin(0.5)), semi_axes=(75_000.0, 25_000.0),
                 angle_deg: float = 30.0) -> np.ndarray:
    """Elliptical N-wave seafloor uplift xi = A 2 sqrt(e) s exp(-2 rho^2), with s the
    along-axis coordinate over its semi-axis and rho^2 the elliptical radius squared;
    its crest is A at s = 1/2 and its trough -A at s = -1/2."""
    a = math.radians(angle_deg)
    dx = p[:, 0] - center[0]
    dy = p[:, 1] - center[1]
    s = (math.cos(a) * dx + math.sin(a) * dy) / semi_axes[0]
    q = (-math.sin(a) * dx + math.cos(a) * dy) / semi_axes[1]
    rho2 = s * s + q * q
    return amplitude * 2.0 * math.sqrt(math.e) * s * np.exp(-2.0 * rho2)


def coast_rupture(mesh: Mesh, amplitude: float = 3.0, angle_deg: float = 30.0,
                  v_rupture: float = 2_000.0):
    """Kinematic version of the N-wave source at the mesh vertices: the same
    uplift, released along the long axis from its far end at v_rupture (onset =
    along-axis distance from the end / v_rupture).  Returns (uplift_v, onset_v)."""
    up = nwave_uplift(mesh.xy, amplitude=amplitude, angle_deg=angle_deg)
    a = math.radians(angle_deg)
    c = (300_000.0 * math.cos(0.5), 300_000.0 * math.sin(0.5))
    s = math.cos(a) * (mesh.xy[:, 0] - c[0]) + math.sin(a) * (mesh.xy[:, 1] - c[1])
    return up, np.maximum(0.0, s + 75_000.0) / v_rupture


def coast_initial_state(mesh: Mesh, amplitude: float = 3.0, angle_deg: float = 30.0) -> State:
    """Sea at rest at level 0 plus an instantaneous free-surface offset equal to the
    seafloor uplift, applied where the sea is (H = max(0, h_cell + xi) with h_cell the
    vertex-mean depth, xi only where h_cell > 0)."""
    h = mesh.vertex_mean(mesh.depth)
    xi = nwave_uplift(mesh.cell_points(), amplitude=amplitude, angle_deg=angle_deg)
    H = np.where(h > 0.0, np.maximum(0.0, h + xi), 0.0)
    zero = np.zeros_like(H)
    return State(H, zero.copy(), zero.copy(), 0.0)


def coast_gauges(n: int = 16, radius: float = 85_000.0) -> np.ndarray:
    """n gauges on an arc just offshore of the 70 km shoreline."""
    th = np.linspace(0.05, 0.95, n)
    return np.stack([radius * np.cos(th), radius * np.sin(th)], axis=1)


THACKER_GAUGES = np.array([[0.0, 0.0], [0.5, 0.0], [1.0, 0.0]])   # Sec. 3 gauge positions


def ensemble_meshes(n_meshes: int = 8, smallest: int = 50_000, ratio: float = 40.0) -> list[int]:
    """Cell counts of the batched-ensemble meshes, geometric from smallest to ratio x smallest."""
    return [int(round(smallest * ratio ** (i / (n_meshes - 1)))) for i in range(n_meshes)]


def ensemble_sources(mesh_index: int, n_scen: int = 32) -> list[tuple[float, float]]:
    """(amplitude in [1, 5] m, orientation in [0, 180) deg) for each scenario of a mesh."""
    u = uniform(1000 + mesh_index, 7, 2 * n_scen).reshape(2, n_scen)
    return [(1.0 + 4.0 * u[0, k], 180.0 * u[1, k]) for k in range(n_scen)]
