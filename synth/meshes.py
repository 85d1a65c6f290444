"""Mesh, grid and field generators (seeded, numpy only).

Conventions used by every consumer:

* Coordinates are float64, row-major ``(n_nodes, dim)``; connectivity is int32,
  row-major ``(n_elems, dim+1)``.
* A grid is described by its *base* (pressure) cells: ``ncell[k]`` cells of
  width ``h[k]`` starting at ``origin[k]``.  With ``staggered=False`` one nodal
  Q1 grid sits on the base grid nodes ``origin + i*h``.  With
  ``staggered=True`` there is one velocity grid per axis ``g``: its nodes sit at
  ``origin[g] + i*h[g]`` along axis ``g`` and at cell centres
  ``origin[k] + (j+1/2)*h[k]`` along the other axes (the staggered arrangement
  of Sec. 2.2, "Spatial Discretization").
* Node ``(i0, i1, i2)`` of a grid with ``nn`` nodes per axis has linear index
  ``i0 + nn0*(i1 + nn1*i2)`` (x fastest).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Grid:
    dim: int
    ncell: tuple
    h: tuple
    origin: tuple
    staggered: bool
    # stretched (rectilinear) grids: per axis the ncell[k] + 1 base-node
    # coordinates, strictly increasing; None = uniform (origin + i * h)
    axis: tuple | None = None

    @property
    def n_grids(self) -> int:
        return self.dim if self.staggered else 1

    def sub_ncell(self, g: int) -> tuple:
        """Q1 cells per axis of velocity grid ``g``."""
        if not self.staggered:
            return tuple(self.ncell)
        return tuple(self.ncell[k] if k == g else self.ncell[k] - 1 for k in range(self.dim))

    def sub_nnode(self, g: int) -> tuple:
        return tuple(c + 1 for c in self.sub_ncell(g))

    def sub_origin(self, g: int) -> tuple:
        if not self.staggered:
            return tuple(self.origin)
        return tuple(self.origin[k] if k == g else self.origin[k] + 0.5 * self.h[k]
                     for k in range(self.dim))

    def n_fluid_nodes(self, g: int) -> int:
        return int(np.prod(self.sub_nnode(g)))

    def base_axis(self, k: int) -> np.ndarray:
        """Base-grid node coordinates along axis k."""
        if self.axis is not None:
            return np.asarray(self.axis[k], dtype=np.float64)
        return self.origin[k] + np.arange(self.ncell[k] + 1, dtype=np.float64) * self.h[k]

    def sub_axis(self, g: int, k: int) -> np.ndarray:
        """Node coordinates of velocity grid g along axis k: the base nodes along
        axis g (and on a non-staggered grid), the base cell centres otherwise."""
        if self.axis is None:
            return self.sub_origin(g)[k] + np.arange(self.sub_nnode(g)[k], dtype=np.float64) * self.h[k]
        x = self.base_axis(k)
        if not self.staggered or k == g:
            return x
        return 0.5 * (x[:-1] + x[1:])


def stretched_axis(n: int, lo: float = 0.0, hi: float = 1.0, amp: float = 0.5) -> np.ndarray:
    """n + 1 nodes on [lo, hi] from x = xi + amp sin(2 pi xi) / (2 pi), xi uniform:
    strictly increasing for amp < 1, spacing (1 - amp)/n at the centre and
    (1 + amp)/n at the ends (points concentrated around the middle, where the
    bodies sit)."""
    xi = np.arange(n + 1, dtype=np.float64) / n
    x = xi + amp * np.sin(2.0 * np.pi * xi) / (2.0 * np.pi)
    x[0], x[-1] = 0.0, 1.0
    return lo + (hi - lo) * x


def stretched_grid(dim: int, n: int, amp: float = 0.5, staggered: bool = True) -> "Grid":
    """Stretched grid on [0,1]^dim with n cells per axis (same stretching on every axis)."""
    ax = tuple(stretched_axis(n, 0.0, 1.0, amp) for _ in range(dim))
    return Grid(dim, (n,) * dim, (1.0 / n,) * dim, (0.0,) * dim, staggered, ax)


def grid_node_coords(grid: Grid, g: int) -> np.ndarray:
    """Coordinates (n_nodes, dim) of the nodes of velocity grid ``g``, x fastest."""
    axes = [grid.sub_axis(g, k) for k in range(grid.dim)]
    mesh = np.meshgrid(*axes, indexing="ij")
    # ravel in Fortran order so that axis 0 runs fastest
    return np.stack([m.ravel(order="F") for m in mesh], axis=1)


# ----------------------------------------------------------------------------- meshes

def disk_mesh(n_rings: int = 9, radius: float = 0.2, center=(0.5, 0.5), jitter: float = 0.1,
              seed: int = 0):
    """Concentric-ring triangulation of a disk: ring k has 6k nodes.

    ``1 + 3K(K+1)`` nodes and ``6K^2`` triangles (K=9: 271 nodes, 486 triangles).
    Interior nodes (not the centre, not the outer ring) are jittered by
    ``U(-jitter*hr, jitter*hr)`` per coordinate, ``hr = radius / K``.
    """
    rng = np.random.default_rng(seed)
    K = n_rings
    hr = radius / K
    pts = [(0.0, 0.0)]
    ring_start = [0]
    for k in range(1, K + 1):
        ring_start.append(len(pts))
        for s in range(6 * k):
            a = 2.0 * np.pi * s / (6 * k)
            pts.append((k * hr * np.cos(a), k * hr * np.sin(a)))
    X = np.array(pts, dtype=np.float64)
    tris = []
    # ring 0 -> ring 1
    for s in range(6):
        tris.append((0, ring_start[1] + s, ring_start[1] + (s + 1) % 6))
    for k in range(2, K + 1):
        inner0, outer0 = ring_start[k - 1], ring_start[k]
        ni, no = 6 * (k - 1), 6 * k
        # walk both rings by angle; each hex sector has (k-1) inner, k outer segments
        i = o = 0
        while i < ni or o < no:
            ai = (i + 0.5) / ni if i < ni else 2.0
            ao = (o + 0.5) / no if o < no else 2.0
            if ao <= ai:
                tris.append((inner0 + i % ni, outer0 + o % no, outer0 + (o + 1) % no))
                o += 1
            else:
                tris.append((inner0 + i % ni, outer0 + (o % no), inner0 + (i + 1) % ni))
                i += 1
    E = np.array(tris, dtype=np.int32)
    if jitter > 0:
        interior = np.arange(1, ring_start[K])
        X[interior] += rng.uniform(-jitter * hr, jitter * hr, size=(interior.size, 2))
    X += np.asarray(center, dtype=np.float64)
    return X, E


def _kuhn_tets(nx: int, ny: int, nz: int):
    """Six Kuhn tetrahedra per hexahedron of an nx*ny*nz block (conforming)."""
    def nid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    base = np.stack([ii.ravel(order="F"), jj.ravel(order="F"), kk.ravel(order="F")], axis=1)
    tets = []
    for p in perms:
        c0 = base.copy()
        c1 = c0.copy(); c1[:, p[0]] += 1
        c2 = c1.copy(); c2[:, p[1]] += 1
        c3 = c0 + 1
        tets.append(np.stack([nid(*c.T) for c in (c0, c1, c2, c3)], axis=1))
    T = np.stack(tets, axis=1).reshape(-1, 4)
    return T.astype(np.int32)


def _block_nodes(nx, ny, nz, size):
    xs = [np.linspace(-0.5 * size[a], 0.5 * size[a], n + 1) for a, n in enumerate((nx, ny, nz))]
    gx, gy, gz = np.meshgrid(*xs, indexing="ij")
    return np.stack([gx.ravel(order="F"), gy.ravel(order="F"), gz.ravel(order="F")], axis=1)


def block_face_mask(nx: int, ny: int, nz: int, axis: int = 2) -> np.ndarray:
    """Nodes of a block mesh (``beam_mesh`` numbering) on its two faces normal to
    ``axis``: the top and bottom faces of a beam or plate for axis 2."""
    i = np.arange((nx + 1) * (ny + 1) * (nz + 1))
    idx = [i % (nx + 1), (i // (nx + 1)) % (ny + 1), i // ((nx + 1) * (ny + 1))]
    n = (nx, ny, nz)[axis]
    return (idx[axis] == 0) | (idx[axis] == n)


BEAM_HEXES = {"beam128": (80, 20, 5), "beam64": (40, 10, 3), "beam32": (20, 5, 2), "beam16": (8, 2, 1)}


def beam_mesh(nx: int = 80, ny: int = 20, nz: int = 5, size=(0.4, 0.1, 0.02)):
    """Box beam centred at the origin, nx*ny*nz hexahedra x 6 Kuhn tetrahedra."""
    X = _block_nodes(nx, ny, nz, size)
    return X.astype(np.float64), _kuhn_tets(nx, ny, nz)


def leaflet_mesh(n: int = 230, nt: int = 3, size=(0.3, 0.3, 0.01), cap_radius: float = 0.5):
    """Thin square shell bent onto a spherical cap of the given radius, centred at the origin."""
    X, E = beam_mesh(n, n, nt, size)
    R = cap_radius
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    # map the flat plate onto a sphere of radius R + z (arc-length preserving in x,y)
    r = np.hypot(x, y)
    theta = r / R
    scale = np.where(r > 0, np.sin(theta) / np.where(r > 0, theta, 1.0), 1.0)
    rr = R + z
    Xn = np.stack([x * scale * rr / R, y * scale * rr / R, rr * np.cos(theta) - R], axis=1)
    # re-centre the cap's bounding box at the origin
    Xn -= 0.5 * (Xn.min(axis=0) + Xn.max(axis=0))
    return Xn, E


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def place_body(X: np.ndarray, R: np.ndarray, centre) -> np.ndarray:
    return X @ R.T + np.asarray(centre, dtype=np.float64)


def _signed_volumes(X, E):
    a = X[E[:, 1]] - X[E[:, 0]]
    b = X[E[:, 2]] - X[E[:, 0]]
    c = X[E[:, 3]] - X[E[:, 0]]
    return np.einsum("ij,ij->i", a, np.cross(b, c))


def deformed_beam_mesh(nx=320, ny=80, nz=26, size=(0.4, 0.1, 0.02), sigma_rel=0.02,
                       sweeps=10, seed=0, max_tries=8):
    """Beam with node displacements N(0, sigma_rel * thickness), then smoothed.

    The beam's smallest dimension (its thickness, 0.02) is read as the "width"
    the displacement amplitude is relative to; relative to the 0.1 side the
    unsmoothed noise would be larger than the elements.  Smoothing replaces each
    node's displacement by the mean of its 6 lattice neighbours ``sweeps`` times.
    A sample whose tetrahedra change orientation is rejected and redrawn.
    """
    rng = np.random.default_rng(seed)
    X0, E = beam_mesh(nx, ny, nz, size)
    sign0 = np.sign(_signed_volumes(X0, E))
    sigma = sigma_rel * min(size)
    shape = (nx + 1, ny + 1, nz + 1)
    for _ in range(max_tries):
        D = rng.normal(0.0, sigma, size=X0.shape).reshape(shape[2], shape[1], shape[0], 3)
        for _s in range(sweeps):
            P = np.pad(D, ((1, 1), (1, 1), (1, 1), (0, 0)), mode="edge")
            D = (P[1:-1, 1:-1, 1:-1] * 0.0 + P[2:, 1:-1, 1:-1] + P[:-2, 1:-1, 1:-1]
                 + P[1:-1, 2:, 1:-1] + P[1:-1, :-2, 1:-1] + P[1:-1, 1:-1, 2:] + P[1:-1, 1:-1, :-2]) / 6.0
        X = X0 + D.reshape(-1, 3)
        if np.all(np.sign(_signed_volumes(X, E)) == sign0):
            return X, E
    raise RuntimeError("deformed_beam_mesh: could not draw a non-inverting sample")


# ----------------------------------------------------------------------------- fields

def sin_cos_2d(P: np.ndarray) -> np.ndarray:
    return np.sin(2 * np.pi * P[:, 0]) * np.cos(3 * np.pi * P[:, 1])


def taylor_green(P: np.ndarray, g: int) -> np.ndarray:
    """Divergence-free Taylor-Green-type velocity component ``g`` at points P."""
    x, y, z = (2 * np.pi * P[:, k] for k in range(3))
    if g == 0:
        return np.sin(x) * np.cos(y) * np.cos(z)
    if g == 1:
        return -np.cos(x) * np.sin(y) * np.cos(z)
    return np.zeros(P.shape[0])


# ----------------------------------------------------------------------------- workloads

@dataclass
class Workload:
    name: str
    grid: Grid
    coords: np.ndarray
    elems: np.ndarray
    fields: list = field(default_factory=list)   # one array per velocity grid
    force: np.ndarray | None = None               # (n_nodes, n_grids) nodal force

    @property
    def dim(self):
        return self.grid.dim


def _fields_for(grid: Grid, kind: str, dtype=np.float64):
    out = []
    for g in range(grid.n_grids):
        P = grid_node_coords(grid, g)
        if kind == "sincos":
            out.append(sin_cos_2d(P).astype(dtype))
        elif kind == "tg":
            out.append(taylor_green(P, g).astype(dtype))
        else:
            raise ValueError(kind)
    return out


def workload(name: str, seed: int = 0, field_dtype=np.float64) -> Workload:
    """Named synthetic workloads, shaped like the paper's beam and plate problems.

    * ``disk2d``       : 64x64 nodal grid on [0,1]^2, jittered 486-triangle disk (r=0.2).
    * ``beam128``      : 128^3 staggered grids, rotated 48k-tet beam 0.4x0.1x0.02.
    * ``leaflet256``   : 256^3 staggered grids, 952k-tet curved leaflet 0.3x0.3x0.01.
    * ``leaflet32``    : 32^3 staggered grids, 2352-tet leaflet (finite-difference sub-instance).
    * ``beam512``      : 512x512x256 staggered grids on [0,1]^2x[0,0.5], 4.0M-tet deformed beam.
    * ``beam16`` / ``beam32``: small rotated beams for tests (16^3 / 32^3 grids).
    * ``disk2d_small`` : 16x16 grid, 2-ring disk.
    * ``disk2d_s``, ``beam16s``, ``beam32s``, ``beam64s``: the same bodies on stretched
      grids (``stretched_axis`` with amp 0.5: cells at the centre half as wide as a
      uniform grid's of the same count; beam64s has beam128's resolution at the body).
    """
    rng = np.random.default_rng(seed)
    if name in ("disk2d", "disk2d_small", "disk2d_s"):
        n, K = (16, 3) if name == "disk2d_small" else (64, 9)
        grid = (stretched_grid(2, n, 0.5, staggered=False) if name == "disk2d_s"
                else Grid(2, (n, n), (1.0 / n, 1.0 / n), (0.0, 0.0), False))
        X, E = disk_mesh(K, 0.2, (0.5, 0.5), 0.1, seed)
        wl = Workload(name, grid, X, E, _fields_for(grid, "sincos", field_dtype))
        wl.force = rng.standard_normal((X.shape[0], 1))
        return wl
    if name in ("beam128", "beam16", "beam32", "beam64", "beam16s", "beam32s", "beam64s"):
        base = name.rstrip("s")
        n = {"beam128": 128, "beam64": 64, "beam32": 32, "beam16": 16}[base]
        hexes = BEAM_HEXES[base] if name != "beam64s" else BEAM_HEXES["beam128"]
        grid = (stretched_grid(3, n, 0.5) if name.endswith("s")
                else Grid(3, (n, n, n), (1.0 / n,) * 3, (0.0, 0.0, 0.0), True))
        X, E = beam_mesh(*hexes)
        X = place_body(X, random_rotation(rng), (0.5, 0.5, 0.5))
        wl = Workload(name, grid, X, E, _fields_for(grid, "tg", field_dtype))
        wl.force = rng.standard_normal((X.shape[0], 3))
        return wl
    if name in ("leaflet256", "leaflet32"):
        n, (m, nt) = {"leaflet256": (256, (230, 3)), "leaflet32": (32, (14, 2))}[name]
        grid = Grid(3, (n, n, n), (1.0 / n,) * 3, (0.0, 0.0, 0.0), True)
        X, E = leaflet_mesh(m, nt)
        X = place_body(X, random_rotation(rng), (0.5, 0.5, 0.5))
        wl = Workload(name, grid, X, E, _fields_for(grid, "tg", field_dtype))
        wl.force = rng.standard_normal((X.shape[0], 3))
        return wl
    if name == "beam512":
        grid = Grid(3, (512, 512, 256), (1.0 / 512,) * 3, (0.0, 0.0, 0.0), True)
        X, E = deformed_beam_mesh(seed=seed)
        X = X + np.array([0.5, 0.5, 0.25])
        wl = Workload(name, grid, X, E, _fields_for(grid, "tg", field_dtype))
        wl.force = rng.standard_normal((X.shape[0], 3))
        return wl
    raise ValueError(f"unknown workload {name!r}")


def batch_bodies(n_bodies=64, min_tets=1000, max_tets=200000, seed=0):
    """Reference-configuration bodies with log-uniform tetrahedron counts (beams and disks)."""
    rng = np.random.default_rng(seed)
    bodies = []
    for b in range(n_bodies):
        target = float(np.exp(rng.uniform(np.log(min_tets), np.log(max_tets))))
        if b % 2 == 0:   # beam with aspect 20:5:1 scaled to the target count
            s = (target / (6 * 100.0)) ** (1.0 / 3.0)
            nx, ny, nz = max(2, round(20 * s)), max(1, round(5 * s)), max(1, round(s))
            X, E = beam_mesh(nx, ny, nz, (0.12, 0.03, 0.006))
        else:            # thin disk-like plate, square footprint
            s = (target / (6 * 2.0)) ** 0.5
            n = max(2, round(s))
            X, E = beam_mesh(n, n, 2, (0.08, 0.08, 0.008))
        R = random_rotation(rng)
        c = rng.uniform(0.2, 0.8, size=3)
        bodies.append(dict(X0=X, E=E, R=R, centre=c,
                           wave=rng.uniform(0.0, 2 * np.pi), amp=0.002))
    return bodies


def body_motion(body: dict, step: int, n_steps: int) -> np.ndarray:
    """Current configuration of a body at a time step: rigid motion plus a travelling wave."""
    t = step / max(1, n_steps)
    ang = 0.5 * t
    c, s = np.cos(ang), np.sin(ang)
    Rz = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    X0 = body["X0"]
    wave = body["amp"] * np.sin(40.0 * X0[:, 0] + body["wave"] + 2 * np.pi * t)
    Xw = X0 + np.stack([np.zeros_like(wave), np.zeros_like(wave), wave], axis=1)
    drift = 0.02 * np.array([np.sin(2 * np.pi * t), np.cos(2 * np.pi * t), 0.0])
    return place_body(Xw, body["R"] @ Rz, body["centre"] + drift)


def combine_bodies(parts):
    """One mesh made of several bodies: list of (X, E) -> (X, E, node_ranges, elem_ranges)."""
    Xs, Es, nr, er = [], [], [], []
    n0 = e0 = 0
    for X, E in parts:
        Xs.append(X)
        Es.append(E + n0)
        nr.append((n0, n0 + X.shape[0]))
        er.append((e0, e0 + E.shape[0]))
        n0 += X.shape[0]
        e0 += E.shape[0]
    return np.concatenate(Xs), np.concatenate(Es).astype(np.int32), nr, er


def batch_workload(n_bodies=64, n_cells=256, min_tets=1000, max_tets=200000, seed=0):
    """Moving bodies on a staggered n_cells^3 grid: (grid, bodies, E, node_ranges, elem_ranges);
    positions at step t come from ``batch_coords(bodies, t, n_steps)``."""
    bodies = batch_bodies(n_bodies, min_tets, max_tets, seed)
    grid = Grid(3, (n_cells,) * 3, (1.0 / n_cells,) * 3, (0.0, 0.0, 0.0), True)
    X, E, nr, er = combine_bodies([(b["X0"], b["E"]) for b in bodies])
    return grid, bodies, E, nr, er


def batch_coords(bodies, step, n_steps):
    return np.concatenate([body_motion(b, step, n_steps) for b in bodies])
