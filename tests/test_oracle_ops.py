"""Pins of the oracle's operation tallies (the algorithmic work behind the
benchmark's roofline of the clipping step) against counts derived by hand from
the clipping recipe of steps (II)-(III) of Sec. 2.3: split the simplex against
the 2d half-spaces of the cell in the order x >= lo, x <= hi, y >= lo, ...;
one side value per simplex vertex and half-space; one cut point per edge that
crosses a plane; one determinant per sub-simplex of the result.
"""
import numpy as np

import oracle
import synth

# operations of one tally, by the statements they stand for (3-D; 2-D in brackets)
SIDE = 1                      # one subtraction
CUT3, CUT2 = 2 + 3 * 3, 2 + 3 * 2   # t = sp / (sp - sq), then p + t (q - p) per axis
DET3, DET2 = 9 + 14, 4 + 3    # edge vectors and the determinant
FRAME3, FRAME2 = 2 * 3 + 3 * 4, 2 * 2 + 2 * 3   # cell corner per axis, vertices minus corner
# Gauss-Jordan inverse of the (d+1)x(d+1) barycentric system, with its identity block
BARY3, BARY2 = 4 * (2 * 4 + 3 * 4 * 4), 3 * (2 * 3 + 2 * 4 * 3)
# per quadrature point: weight 2, Jacobian 3 (2-D 1), point 6/axis, lambda 2d per
# vertex, t 2/axis, f and vol 2, psi (d + d/2 per corner), block 3 per entry
QPT3 = 2 + 3 + 18 + 4 * 6 + 6 + 2 + 8 * 3 + 8 * 3 // 2 + 3 * 4 * 8
QPT2 = 2 + 1 + 12 + 3 * 4 + 4 + 2 + 4 * 2 + 4 * 2 // 2 + 3 * 3 * 4


def _counts(grid, X, E):
    sg = oracle.subgrid(grid, 0)
    pe, pc = oracle.candidate_pairs(sg, X, E)
    ops = {}
    oracle.pair_blocks(sg, X, E, pe, pc, nthreads=1, ops=ops)
    return len(pe), ops


def test_tallies_tet_inside_one_cell():
    """No plane cuts: 6 half-spaces x 4 vertices side values, one sub-simplex,
    a 4x4x4-point rule on it."""
    grid = synth.Grid(3, (4, 4, 4), (0.25,) * 3, (0.0,) * 3, False)
    X = np.array([[0.3, 0.3, 0.3], [0.4, 0.3, 0.3], [0.3, 0.4, 0.3], [0.3, 0.3, 0.4]])
    E = np.array([[0, 1, 2, 3]], dtype=np.int32)
    n, ops = _counts(grid, X, E)
    assert n == 1
    assert ops == {"frame": FRAME3, "clip": 6 * 4 * SIDE, "volume": DET3, "bary": BARY3, "quad": 64 * QPT3}


def test_tallies_tet_across_one_plane():
    """Vertex D beyond x = 0.5, the others before it: two candidate cells.
    Cell [0.25, 0.5]: the x <= hi split of the whole tet (4 side values, 3 cut
    points) leaves a prism of 3 tets, which the four y/z half-spaces then test
    vertex by vertex.  Cell [0.5, 0.75]: the x >= lo split keeps the corner tet
    at D (3 cut points), which five more half-spaces test."""
    grid = synth.Grid(3, (4, 4, 4), (0.25,) * 3, (0.0,) * 3, False)
    X = np.array([[0.40, 0.30, 0.30], [0.45, 0.40, 0.30], [0.45, 0.30, 0.40], [0.55, 0.35, 0.35]])
    E = np.array([[0, 1, 2, 3]], dtype=np.int32)
    n, ops = _counts(grid, X, E)
    assert n == 2
    clip_a = 4 * SIDE + (4 * SIDE + 3 * CUT3) + 4 * (3 * 4 * SIDE)
    clip_b = (4 * SIDE + 3 * CUT3) + 5 * (4 * SIDE)
    assert ops["clip"] == clip_a + clip_b
    assert ops["volume"] == (3 + 1) * DET3
    assert ops["frame"] == 2 * FRAME3
    assert ops["bary"] == 2 * BARY3
    assert ops["quad"] == (3 + 1) * 64 * QPT3


def test_tallies_triangle_inside_one_cell():
    grid = synth.Grid(2, (4, 4), (0.25,) * 2, (0.0,) * 2, False)
    X = np.array([[0.3, 0.3], [0.4, 0.3], [0.3, 0.4]])
    E = np.array([[0, 1, 2]], dtype=np.int32)
    n, ops = _counts(grid, X, E)
    assert n == 1
    assert ops == {"frame": FRAME2, "clip": 4 * 3 * SIDE, "volume": DET2, "bary": BARY2, "quad": 9 * QPT2}


def test_tallies_triangle_across_one_line():
    """Vertex c beyond x = 0.5: cell [0.25, 0.5] keeps a quadrilateral (2 cut
    points, split into 2 triangles), cell [0.5, 0.75] a triangle (2 cut points)."""
    grid = synth.Grid(2, (4, 4), (0.25,) * 2, (0.0,) * 2, False)
    X = np.array([[0.40, 0.30], [0.45, 0.40], [0.55, 0.35]])
    E = np.array([[0, 1, 2]], dtype=np.int32)
    n, ops = _counts(grid, X, E)
    assert n == 2
    clip_a = 3 * SIDE + (3 * SIDE + 2 * CUT2) + 2 * (2 * 3 * SIDE)
    clip_b = (3 * SIDE + 2 * CUT2) + 3 * (3 * SIDE)
    assert ops["clip"] == clip_a + clip_b
    assert ops["volume"] == (2 + 1) * DET2
    assert ops["quad"] == (2 + 1) * 9 * QPT2


def test_tallies_add_over_threads():
    """The per-thread tallies sum to the same totals on 1 and 4 threads."""
    w = synth.workload("beam16")
    sg = oracle.subgrid(w.grid, 1)
    pe, pc = oracle.candidate_pairs(sg, w.coords, w.elems)
    o1, o4 = {}, {}
    oracle.pair_blocks(sg, w.coords, w.elems, pe, pc, nthreads=1, ops=o1)
    oracle.pair_blocks(sg, w.coords, w.elems, pe, pc, nthreads=4, ops=o4)
    assert o1 == o4 and o1["clip"] > 0
