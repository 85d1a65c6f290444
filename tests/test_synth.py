"""The seeded synthetic inputs (``synth/``) against the recipe they state: mesh
sizes, valid elements, every node used, the distance from the walls that the
out-of-grid reading needs (every element inside the cells of every velocity
grid, kept at least two cells away), motion without inverted elements, and
determinism per seed with independent problems per rank."""
import numpy as np
import pytest

import synth


def _signed_volumes(X, E):
    d = X.shape[1]
    J = np.stack([X[E[:, a]] - X[E[:, 0]] for a in range(1, d + 1)], axis=1)
    return np.linalg.det(J)


def _check_mesh(X, E):
    assert E.dtype == np.int32 and X.dtype == np.float64
    assert E.min() >= 0 and E.max() < X.shape[0]
    assert np.unique(E).size == X.shape[0]                  # every node belongs to an element
    v = np.abs(_signed_volumes(X, E))
    assert v.min() > 1e-3 * v.mean()                         # no degenerate element


def _wall_margin_in_cells(grid, X):
    """Smallest distance from the mesh to the edge of the region covered by the
    cells of any velocity grid, in cell widths at that edge."""
    worst = np.inf
    for g in range(grid.n_grids):
        for k in range(grid.dim):
            ax = grid.sub_axis(g, k)
            lo, hi = X[:, k].min(), X[:, k].max()
            worst = min(worst, (lo - ax[0]) / (ax[1] - ax[0]), (ax[-1] - hi) / (ax[-1] - ax[-2]))
    return worst


# name -> (nodes, elements)
SIZES = {
    "disk2d": (271, 486),
    "beam128": (10206, 48000),
    "beam16": (3 * 9 * 2, 6 * 8 * 2 * 1),
    "beam32": (21 * 6 * 3, 6 * 20 * 5 * 2),
    "leaflet32": (675, 2352),
    "beam64s": (10206, 48000),
}


@pytest.mark.parametrize("name", sorted(SIZES))
def test_named_workloads_follow_their_recipe(name):
    w = synth.workload(name)
    n, m = SIZES[name]
    assert w.coords.shape == (n, w.dim) and w.elems.shape == (m, w.dim + 1)
    _check_mesh(w.coords, w.elems)
    assert _wall_margin_in_cells(w.grid, w.coords) >= 2.0
    assert len(w.fields) == w.grid.n_grids
    for g, f in enumerate(w.fields):
        assert f.shape == (w.grid.n_fluid_nodes(g),) and np.all(np.isfinite(f))
    assert w.force.shape == (n, w.grid.n_grids)


def test_large_meshes_follow_their_recipe():
    """The 952 200-tet leaflet (230 x 230 x 3 hexahedra) and the 3 993 600-tet
    deformed beam (320 x 80 x 26), whose noise must not invert any tetrahedron."""
    X, E = synth.leaflet_mesh(230, 3)
    assert E.shape == (6 * 230 * 230 * 3, 4) and X.shape == (231 * 231 * 4, 3)
    _check_mesh(X, E)
    X, E = synth.deformed_beam_mesh(seed=0)
    assert E.shape == (6 * 320 * 80 * 26, 4) and X.shape == (321 * 81 * 27, 3)
    _check_mesh(X, E)
    X0, _ = synth.beam_mesh(320, 80, 26)
    assert np.array_equal(np.sign(_signed_volumes(X, E)), np.sign(_signed_volumes(X0, E)))
    assert np.abs(X - X0).max() > 0.0                        # the noise was applied
    grid = synth.Grid(3, (512, 512, 256), (1.0 / 512,) * 3, (0.0, 0.0, 0.0), True)
    assert _wall_margin_in_cells(grid, X + np.array([0.5, 0.5, 0.25])) >= 2.0


def test_batch_of_moving_bodies_follows_its_recipe():
    """64 bodies, 2 234 256 tetrahedra and 535 718 nodes; over the eight replayed
    configurations of the 200-step motion every body stays two cells inside the
    grids and no tetrahedron inverts."""
    grid, bodies, E, nr, er = synth.batch_workload(64, 256, 1000, 200000, seed=0)
    assert len(bodies) == 64 and E.shape == (2234256, 4) and nr[-1][1] == 535718
    sizes = [b["E"].shape[0] for b in bodies]
    assert min(sizes) >= 1000 * 0.5 and max(sizes) <= 200000 * 1.5   # log-uniform counts, rounded shapes
    X0 = synth.batch_coords(bodies, 0, 200)
    _check_mesh(X0, E)
    s0 = np.sign(_signed_volumes(X0, E))
    prev = X0
    for k in range(1, 8):
        X = synth.batch_coords(bodies, k * 25, 200)
        assert _wall_margin_in_cells(grid, X) >= 2.0
        assert np.array_equal(np.sign(_signed_volumes(X, E)), s0)
        assert np.abs(X - prev).max() > 0.0                  # the bodies move
        prev = X
    for (n0, n1), (e0, e1) in zip(nr, er):                   # bodies are disjoint node sets
        assert E[e0:e1].min() >= n0 and E[e0:e1].max() < n1


def test_inputs_are_seeded_and_ranks_draw_their_own():
    a, b = synth.workload("beam32", 0), synth.workload("beam32", 0)
    assert np.array_equal(a.coords, b.coords) and np.array_equal(a.force, b.force)
    c = synth.workload("beam32", 1)                          # another rank's rotation
    assert not np.allclose(a.coords, c.coords)
    assert np.array_equal(a.elems, c.elems)
    g0 = synth.batch_workload(8, 64, 300, 3000, seed=0)
    g1 = synth.batch_workload(8, 64, 300, 3000, seed=1)
    assert not np.allclose(g0[1][0]["centre"], g1[1][0]["centre"])


def test_taylor_green_field_is_divergence_free_on_the_staggered_cells():
    """The velocity field sampled on the staggered grids is the Taylor-Green
    vortex (u, v, w) = (sin x cos y cos z, -cos x sin y cos z, 0) at 2 pi scale.
    On the staggered (MAC) cells its discrete divergence cancels exactly: the
    two difference quotients are both (2/h) sin(pi h) cos cos cos at the cell
    centre, with opposite signs."""
    n = 32
    grid = synth.Grid(3, (n,) * 3, (1.0 / n,) * 3, (0.0,) * 3, True)
    f = [synth.taylor_green(synth.grid_node_coords(grid, g), g).reshape(grid.sub_nnode(g), order="F")
         for g in range(3)]
    h = 1.0 / n
    du = np.diff(f[0], axis=0) / h            # u on x-faces: (n, n, n) cell values
    dv = np.diff(f[1], axis=1) / h            # v on y-faces
    assert du.shape == dv.shape == (n, n, n)
    assert np.abs(du).max() > 1.0             # the field is not trivially zero
    assert np.abs(du + dv).max() <= 1e-11
    assert np.abs(f[2]).max() == 0.0
