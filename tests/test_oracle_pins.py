"""Pins of the FP64 oracle against facts fixed by the method and by mathematics.

Each test names the property it checks; a plausible mistake in the oracle
(dropped term, wrong sign or index, transposed operand) breaks at least one.
Mortar integrals and the algebraic transfer: Sec. 2.3, "Variational Transfer".
"""
import itertools
import math
import random
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import synth
from oracle import exact


def _phi_integrals(X, E):
    d = X.shape[1]
    vol = oracle.element_volumes(X, E)
    phi = np.zeros(X.shape[0])
    np.add.at(phi, E.ravel(), np.repeat(vol / (d + 1), d + 1))
    return phi, vol


def _cell_lo(sg, c):
    d = sg.dim
    ci = [c % sg.ncell[0], (c // sg.ncell[0]) % sg.ncell[1]]
    if d == 3:
        ci.append(c // (sg.ncell[0] * sg.ncell[1]))
    return [sg.origin[k] + ci[k] * sg.h[k] for k in range(d)]


# --------------------------------------------------------------- quadrature pins

@pytest.mark.parametrize("n,s", [(2, 1), (3, 2)])
def test_gm_rule_exact_on_monomials(n, s):
    """Grundmann-Moeller mean-value rule reproduces the Dirichlet moments
    E[mu^alpha] = n! alpha! / (n + |alpha|)! for every |alpha| <= 2s+1."""
    rule = exact.gm_rule(n, s)
    for deg in range(2 * s + 2):
        for alpha in itertools.product(range(deg + 1), repeat=n + 1):
            if sum(alpha) != deg:
                continue
            q = sum(w * math.prod(mu[j] ** alpha[j] for j in range(n + 1)) for w, mu in rule)
            ref = Fr(math.factorial(n) * math.prod(math.factorial(a) for a in alpha),
                     math.factorial(n + deg))
            assert q == ref, (alpha, q, ref)


# --------------------------------------------------------------- (I) candidate pairs

def _bruteforce_pairs(sg, X, E):
    """Every cell whose open box meets the open bounding box of the element
    (exact rational arithmetic); element-major, x fastest."""
    d = sg.dim
    out = []
    for e in range(E.shape[0]):
        P = [[Fr(X[v, k]) for k in range(d)] for v in E[e]]
        lo = [min(p[k] for p in P) for k in range(d)]
        hi = [max(p[k] for p in P) for k in range(d)]
        ranges = []
        for k in range(d):
            o, h = Fr(sg.origin[k]), Fr(sg.h[k])
            ranges.append([i for i in range(int(sg.ncell[k]))
                           if o + i * h < hi[k] and o + (i + 1) * h > lo[k]])
        if d == 2:
            cells = [(i, j, 0) for j in ranges[1] for i in ranges[0]]
        else:
            cells = [(i, j, k) for k in ranges[2] for j in ranges[1] for i in ranges[0]]
        for (i, j, k) in cells:
            out.append((e, i + int(sg.ncell[0]) * (j + int(sg.ncell[1]) * k)))
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_candidate_pairs_match_bruteforce_on_dyadic_input(dim):
    """With dyadic coordinates (exact division) the floor/ceil index rule must
    give exactly the cells whose interior meets the element's bounding box,
    including vertices lying exactly on grid lines."""
    rng = np.random.default_rng(3)
    n = 8
    grid = synth.Grid(dim, (n,) * dim, (1.0 / n,) * dim, (0.0,) * dim, dim == 3)
    m = 30
    # vertices on a 1/64 lattice, many exactly on grid lines (multiples of 1/8)
    X = rng.integers(12, 52, size=(m * (dim + 1), dim)).astype(np.float64) / 64.0
    E = np.arange(m * (dim + 1), dtype=np.int32).reshape(m, dim + 1)
    for g in range(oracle.n_grids(grid)):
        sg = oracle.subgrid(grid, g)
        keep = oracle.element_volumes(X, E) > 0
        pe, pc = oracle.candidate_pairs(sg, X, E[keep])
        ref = _bruteforce_pairs(sg, X, E[keep])
        assert list(zip(pe.tolist(), pc.tolist())) == ref


def test_out_of_grid_is_reported():
    grid = synth.Grid(2, (4, 4), (0.25, 0.25), (0.0, 0.0), False)
    X = np.array([[0.1, 0.1], [1.2, 0.1], [0.1, 0.5]])
    E = np.array([[0, 1, 2]], dtype=np.int32)
    with pytest.raises(oracle.OracleError):
        oracle.candidate_pairs(oracle.subgrid(grid, 0), X, E)


# --------------------------------------------------------------- (II)+(III) exact rational brute force

@pytest.mark.parametrize("name,stride", [("disk2d_small", 5), ("beam16", 23)])
def test_pair_blocks_match_exact_rational(name, stride):
    """P8: clipping + quadrature agree with exact rational vertex enumeration and
    Grundmann-Moeller integration to 1e-14 of the element volume."""
    w = synth.workload(name)
    d = w.dim
    vol_e = oracle.element_volumes(w.coords, w.elems)
    for g in range(oracle.n_grids(w.grid)):
        sg = oracle.subgrid(w.grid, g)
        pe, pc = oracle.candidate_pairs(sg, w.coords, w.elems)
        blocks, vols = oracle.pair_blocks(sg, w.coords, w.elems, pe, pc)
        for p in range(g, len(pe), stride):
            e, c = int(pe[p]), int(pc[p])
            blk, vol = exact.pair_block_exact(d, w.coords[w.elems[e]], _cell_lo(sg, c), sg.h[:d])
            ex = np.array([[float(x) for x in row] for row in blk])
            scale = vol_e[e]
            assert abs(float(vol) - vols[p]) <= 1e-14 * scale
            assert np.abs(ex - blocks[p]).max() <= 1e-14 * scale, (p, ex, blocks[p])


def test_golden_2d_exact_block():
    """Stored exact rational B of a two-triangle mesh on a 4x4 grid (written by
    tests/golden/make_golden.py from the exact rational reference)."""
    import json, os
    path = os.path.join(os.path.dirname(__file__), "golden", "two_triangles_4x4.json")
    with open(path) as f:
        gold = json.load(f)
    X = np.array(gold["coords"], dtype=np.float64)
    E = np.array(gold["elems"], dtype=np.int32)
    grid = synth.Grid(2, tuple(gold["ncell"]), tuple(gold["h"]), tuple(gold["origin"]), False)
    B = oracle.assemble_B(oracle.subgrid(grid, 0), X, E).tocoo()
    got = {(int(r), int(c)): v for r, c, v in zip(B.row, B.col, B.data)}
    ref = {(int(r), int(c)): float(Fr(s)) for r, c, s in gold["B"]}
    assert set(got) == set(ref)
    for k in ref:
        assert abs(got[k] - ref[k]) <= 1e-15 * max(abs(v) for v in ref.values())


def test_golden_file_is_what_its_script_writes():
    """The stored fixture is exactly the output of tests/golden/make_golden.py,
    which calls only the exact rational reference (oracle/exact.py)."""
    import importlib.util, json, os
    here = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(here, "two_triangles_4x4.json")) as f:
        assert json.load(f) == json.loads(json.dumps(mod.build()))


# --------------------------------------------------------------- invariants

@pytest.mark.parametrize("name", ["disk2d", "beam16", "leaflet32"])
def test_row_sums_and_total_volume(name):
    """P1/P2: the Q1 basis is a partition of unity on every cell, so
    sum_j B_ij = int phi_i = sum_{E ∋ i} |E|/(d+1), and the pair volumes add up
    to the solid volume on every grid."""
    w = synth.workload(name)
    phi, vol = _phi_integrals(w.coords, w.elems)
    C = oracle.Coupling(w.grid, w.coords, w.elems, nthreads=4)
    for g, B in enumerate(C.B):
        rs = np.asarray(B.sum(axis=1)).ravel()
        assert np.abs(rs - phi).max() <= 1e-14 * phi.max()
        assert abs(C.pairs[g][3].sum() - vol.sum()) <= 1e-14 * vol.sum()
        assert abs(B.sum() - vol.sum()) <= 1e-14 * vol.sum()


def _block_solid(n_grid, lo, hi, nh):
    """Kuhn-tetrahedral (3-D) box [lo, hi]^3 with nh hexahedra per side."""
    X, E = synth.beam_mesh(nh, nh, nh, (hi - lo,) * 3)
    X = X + 0.5 * (lo + hi)
    grid = synth.Grid(3, (n_grid,) * 3, (1.0 / n_grid,) * 3, (0.0,) * 3, True)
    return grid, X, E


def test_column_sums_of_covered_fluid_nodes():
    """P3: sum_i B_ij = int psi_j; it equals h^3 for fluid nodes whose whole
    support lies inside the solid (a rotated-free cube of tetrahedra)."""
    grid, X, E = _block_solid(8, 0.21, 0.79, 5)
    C = oracle.Coupling(grid, X, E)
    for g in range(3):
        sg = oracle.subgrid(grid, g)
        P = synth.grid_node_coords(grid, g)
        h = sg.h[0]
        inside = np.all((P - h >= 0.21) & (P + h <= 0.79), axis=1)
        assert inside.sum() > 0
        cs = np.asarray(C.B[g].sum(axis=0)).ravel()
        assert np.abs(cs[inside] - h ** 3).max() <= 1e-14 * h ** 3


@pytest.mark.parametrize("name", ["disk2d", "beam16", "leaflet32"])
def test_affine_fields_are_reproduced(name):
    """P4: Q1 and P1 both contain the affine functions, so the L2 projection of
    an affine fluid field is the same affine function at the solid nodes."""
    w = synth.workload(name)
    d = w.dim
    C = oracle.Coupling(w.grid, w.coords, w.elems)
    coef = np.array([0.3, 1.5, -0.7, 2.0])[: d + 1]
    fields = []
    for g in range(oracle.n_grids(w.grid)):
        P = synth.grid_node_coords(w.grid, g)
        fields.append(coef[0] + P @ coef[1:] + g)
    W = C.transfer_velocity(fields)
    ex = np.stack([coef[0] + w.coords @ coef[1:] + g for g in range(len(fields))], axis=1)
    assert np.abs(W - ex).max() <= 1e-13 * np.abs(ex).max()


def test_mass_matrix_matches_exact_quadrature():
    """P5: the closed-form P1 mass matrix equals exact Grundmann-Moeller
    quadrature of phi_a phi_b on every element, and 1^T M 1 = |Omega_s|."""
    w = synth.workload("beam16")
    M = oracle.mass_matrix(w.coords, w.elems).toarray()
    _, vol = _phi_integrals(w.coords, w.elems)
    assert abs(M.sum() - vol.sum()) <= 1e-15 * vol.sum() * 10
    Mref = np.zeros_like(M)
    for e in range(0, w.elems.shape[0], 5):
        V = [[Fr(x) for x in w.coords[v]] for v in w.elems[e]]

        def f(x, V=V):
            # barycentric coordinates of x by exact solve
            A = [[V[j][r] for j in range(4)] for r in range(3)] + [[Fr(1)] * 4]
            lam = exact._solve(A, list(x) + [Fr(1)])
            return [lam[a] * lam[b] for a in range(4) for b in range(4)]
        r, _ = exact.simplex_integral(V, f, 1)
        Mloc = np.array([float(x) for x in r]).reshape(4, 4)
        single = oracle.mass_matrix(w.coords, w.elems[e:e + 1]).toarray()
        idx = w.elems[e]
        assert np.abs(single[np.ix_(idx, idx)] - Mloc).max() <= 1e-15 * np.abs(Mloc).max() * 10


@pytest.mark.parametrize("method", ["dense", "lu", "cg"])
def test_mass_solves_satisfy_the_defining_equation(method):
    """Every branch of the oracle's solve with S = M_s (the equation S w = B v of
    the algebraic transfer, Sec. 2.3) returns W with M W = Y to rounding, for
    several right-hand sides at once and for one."""
    w = synth.workload("beam16")
    M = oracle.mass_matrix(w.coords, w.elems)
    rng = np.random.default_rng(9)
    Y = rng.standard_normal((M.shape[0], 3))
    W = oracle.solve_mass(M, Y, method=method)
    assert np.abs(M @ W - Y).max() <= 1e-13 * np.abs(Y).max()
    w1 = oracle.solve_mass(M, Y[:, 1], method=method)
    assert w1.shape == (M.shape[0],)
    assert np.abs(w1 - W[:, 1]).max() <= 1e-12 * np.abs(W).max()


@pytest.mark.parametrize("name", ["disk2d", "beam16"])
def test_force_transfer_is_the_adjoint(name):
    """P6: f . (T u) = (T^T f) . u with T u from the velocity transfer and T^T f
    from the dual force transfer; f . (B u) = (B^T f) . u for the nodal one."""
    w = synth.workload(name)
    rng = np.random.default_rng(7)
    C = oracle.Coupling(w.grid, w.coords, w.elems)
    ng = oracle.n_grids(w.grid)
    U = [rng.standard_normal(C.sub[g].n_nodes) for g in range(ng)]
    F = rng.standard_normal((w.coords.shape[0], ng))
    TU = C.transfer_velocity(U)
    TtF = C.transfer_force(F, mode="dual", scale=1.0)
    BtF = C.transfer_force(F, mode="nodal", scale=2.5)
    for g in range(ng):
        lhs, rhs = F[:, g] @ TU[:, g], TtF[g] @ U[g]
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(F[:, g]).sum())
        BU = C.B[g] @ U[g]
        assert abs(2.5 * (F[:, g] @ BU) - BtF[g] @ U[g]) <= 1e-12 * np.abs(BtF[g]).sum()


def _dirichlet_product_integral(V, funcs):
    """Exact int_T prod_j l_j for affine l_j over a simplex with vertices V:
    |T| * n!/(n+k)! * sum over k-tuples of vertices of alpha! prod_j l_j(v_{i_j})."""
    n = len(V) - 1
    k = len(funcs)
    rows = [[V[i + 1][c] - V[0][c] for c in range(n)] for i in range(n)]
    volT = abs(exact._det(rows)) / math.factorial(n)
    vals = [[f(v) for v in V] for f in funcs]
    tot = Fr(0)
    for tup in itertools.product(range(n + 1), repeat=k):
        mult = [tup.count(i) for i in range(n + 1)]
        tot += math.prod(math.factorial(m) for m in mult) * math.prod(vals[j][tup[j]] for j in range(k))
    return volT * Fr(math.factorial(n), math.factorial(n + k)) * tot


@pytest.mark.parametrize("dim", [2, 3])
def test_element_inside_one_cell_is_textbook(dim):
    """P7: an element strictly inside one cell is not clipped, and its block is
    the textbook integral of the product of d+1 affine functions over a simplex."""
    rng = np.random.default_rng(11)
    n = 4
    h = 1.0 / n
    grid = synth.Grid(dim, (n,) * dim, (h,) * dim, (0.0,) * dim, False)
    sg = oracle.subgrid(grid, 0)
    lo = np.array([1.0 * h] * dim)
    V = lo + h * (0.1 + 0.8 * rng.random((dim + 1, dim)))
    E = np.arange(dim + 1, dtype=np.int32)[None]
    pe, pc = oracle.candidate_pairs(sg, V, E)
    assert len(pe) == 1
    blocks, vols = oracle.pair_blocks(sg, V, E, pe, pc)
    Vf = [[Fr(x) for x in v] for v in V]
    A = [[Vf[j][r] for j in range(dim + 1)] for r in range(dim)] + [[Fr(1)] * (dim + 1)]
    for a in range(dim + 1):
        for b in range(1 << dim):
            def lam(x, a=a):
                return exact._solve(A, list(x) + [Fr(1)])[a]
            fs = [lam]
            for k in range(dim):
                if (b >> k) & 1:
                    fs.append(lambda x, k=k: (x[k] - Fr(lo[k])) / Fr(h))
                else:
                    fs.append(lambda x, k=k: 1 - (x[k] - Fr(lo[k])) / Fr(h))
            ref = float(_dirichlet_product_integral(Vf, fs))
            # scale: the element volume (= sum of the whole block)
            assert abs(blocks[0, a, b] - ref) <= 1e-14 * vols[0]


def test_mirror_symmetry():
    """P11: mirroring mesh and grid in x (h a power of two, grid lines exact)
    mirrors B: B'[i, mirror(j)] = B[i, j]."""
    w = synth.workload("disk2d")
    grid = w.grid
    X2 = w.coords.copy()
    X2[:, 0] = 1.0 - X2[:, 0]
    B1 = oracle.Coupling(grid, w.coords, w.elems).B[0].toarray()
    B2 = oracle.Coupling(grid, X2, w.elems).B[0].toarray()
    nn = grid.ncell[0] + 1
    j = np.arange(B1.shape[1])
    mj = (nn - 1 - j % nn) + nn * (j // nn)
    assert np.abs(B2[:, mj] - B1).max() <= 1e-15 * np.abs(B1).max() * 10


def test_subcell_sampling_converges():
    """P9 (sanity): midpoint sampling of lambda_a psi_j on a fine lattice
    approaches the exact B to about the lattice spacing."""
    w = synth.workload("disk2d_small")
    sg = oracle.subgrid(w.grid, 0)
    B = oracle.assemble_B(sg, w.coords, w.elems).toarray()
    X, E = w.coords, w.elems
    nsub = 128
    h = sg.h[0]
    dx = h / nsub
    nn = int(sg.ncell[0]) + 1
    Bs = np.zeros_like(B)
    for e in range(E.shape[0]):
        V = X[E[e]]
        lo = np.floor(V.min(axis=0) / dx).astype(int)
        hi = np.ceil(V.max(axis=0) / dx).astype(int)
        PX, PY = np.meshgrid((np.arange(lo[0], hi[0]) + 0.5) * dx, (np.arange(lo[1], hi[1]) + 0.5) * dx,
                             indexing="ij")
        pts = np.stack([PX.ravel(), PY.ravel()], axis=1)
        T = np.array([[V[0, 0], V[1, 0], V[2, 0]], [V[0, 1], V[1, 1], V[2, 1]], [1, 1, 1]])
        lam = np.linalg.solve(T, np.vstack([pts.T, np.ones(len(pts))]))
        inside = np.all(lam >= 0, axis=0)
        pts, lam = pts[inside], lam[:, inside]
        ij = np.floor(pts / h).astype(int)
        t = pts / h - ij
        for b in range(4):
            bx, by = b & 1, b >> 1
            psi = (t[:, 0] if bx else 1 - t[:, 0]) * (t[:, 1] if by else 1 - t[:, 1])
            col = (ij[:, 0] + bx) + nn * (ij[:, 1] + by)
            for a in range(3):
                Bs[E[e, a]] += np.bincount(col, weights=lam[a] * psi * dx * dx, minlength=B.shape[1])
    assert np.abs(Bs - B).max() <= 2e-3 * np.abs(B).max()


# --------------------------------------------------------------- dual multiplier basis ("pseudo" L2 projection)

@pytest.mark.parametrize("dim", [2, 3])
def test_dual_basis_is_biorthogonal(dim):
    """Eq. (biorth) on one element: the element dual function (d+2) lambda_a - 1
    satisfies int_E mu_a lambda_b = delta_ab int_E mu_a, and int_E mu_a = |E|/(d+1)
    (exact rational integration of products of affine functions)."""
    rng = np.random.default_rng(5)
    V = [[Fr(float(x)) for x in row] for row in rng.random((dim + 1, dim))]
    A = [[V[j][r] for j in range(dim + 1)] for r in range(dim)] + [[Fr(1)] * (dim + 1)]

    def lam(x, a):
        return exact._solve(A, list(x) + [Fr(1)])[a]

    rows = [[V[i + 1][c] - V[0][c] for c in range(dim)] for i in range(dim)]
    volE = abs(exact._det(rows)) / math.factorial(dim)
    for a in range(dim + 1):
        def mu(x, a=a):
            return (dim + 2) * lam(x, a) - 1
        mass = _dirichlet_product_integral(V, [mu])
        assert mass == volE / (dim + 1)
        for b in range(dim + 1):
            got = _dirichlet_product_integral(V, [mu, lambda x, b=b: lam(x, b)])
            assert got == (mass if a == b else 0)


@pytest.mark.parametrize("name,stride", [("disk2d_small", 5), ("beam16", 23)])
def test_dual_blocks_match_exact_rational(name, stride):
    """The dual weights of the oracle (from the lambda blocks and the partition of
    unity of the barycentrics) equal exact rational integration of
    ((d+2) lambda_a - 1) psi_b over E cap C."""
    w = synth.workload(name)
    d = w.dim
    vol_e = oracle.element_volumes(w.coords, w.elems)
    for g in range(oracle.n_grids(w.grid)):
        sg = oracle.subgrid(w.grid, g)
        pe, pc = oracle.candidate_pairs(sg, w.coords, w.elems)
        blocks, _ = oracle.pair_blocks(sg, w.coords, w.elems, pe, pc)
        dual = oracle.dual_blocks(blocks)
        for p in range(g, len(pe), stride):
            e, c = int(pe[p]), int(pc[p])
            blk, _ = exact.pair_block_exact(d, w.coords[w.elems[e]], _cell_lo(sg, c), sg.h[:d], dual=True)
            ex = np.array([[float(x) for x in row] for row in blk])
            assert np.abs(ex - dual[p]).max() <= 1e-14 * (d + 2) * vol_e[e], (p, ex, dual[p])


@pytest.mark.parametrize("name", ["disk2d", "beam16"])
def test_dual_rows_sum_to_the_lumped_mass(name):
    """sum_j B_ij = int mu_i = int phi_i = S_ii for the dual basis (Q1 partition
    of unity), so S^{-1} B maps constants to constants; S = diag(int phi_i)."""
    w = synth.workload(name)
    phi, vol = _phi_integrals(w.coords, w.elems)
    C = oracle.Coupling(w.grid, w.coords, w.elems, multiplier="dual")
    S = C.M.toarray()
    assert np.abs(S - np.diag(phi)).max() <= 1e-15 * phi.max() * 4
    for B in C.B:
        rs = np.asarray(B.sum(axis=1)).ravel()
        assert np.abs(rs - phi).max() <= 1e-13 * phi.max()
        assert abs(B.sum() - vol.sum()) <= 1e-13 * vol.sum()


@pytest.mark.parametrize("name", ["disk2d", "beam16", "leaflet32"])
def test_dual_projection_reproduces_affine_fields(name):
    """The pseudo L2 projection is exact on P1: an affine fluid field is returned
    at the solid nodes, without any iterative solve."""
    w = synth.workload(name)
    d = w.dim
    C = oracle.Coupling(w.grid, w.coords, w.elems, multiplier="dual")
    coef = np.array([-0.4, 0.9, 1.7, -1.1])[: d + 1]
    fields = [coef[0] + synth.grid_node_coords(w.grid, g) @ coef[1:] - g
              for g in range(oracle.n_grids(w.grid))]
    W = C.transfer_velocity(fields)
    ex = np.stack([coef[0] + w.coords @ coef[1:] - g for g in range(len(fields))], axis=1)
    assert np.abs(W - ex).max() <= 1e-13 * np.abs(ex).max()


def test_dual_force_transfer_is_the_adjoint():
    """f . (T u) = (T^T f) . u for T = S^{-1} B of the dual basis."""
    w = synth.workload("beam16")
    rng = np.random.default_rng(9)
    C = oracle.Coupling(w.grid, w.coords, w.elems, multiplier="dual")
    U = [rng.standard_normal(C.sub[g].n_nodes) for g in range(3)]
    F = rng.standard_normal((w.coords.shape[0], 3))
    TU = C.transfer_velocity(U)
    TtF = C.transfer_force(F, mode="dual", scale=1.0)
    for g in range(3):
        lhs, rhs = F[:, g] @ TU[:, g], TtF[g] @ U[g]
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(F[:, g]).sum())


def test_dual_and_standard_projections_differ_off_p1():
    """On a field that is not P1 on the solid the two multiplier spaces give
    different (both consistent) transfers: the dual one is a local
    approximation, not the L2 projection; the L2 projection minimises the L2
    error over V_s, so its error is not larger (checked through B of the
    standard space: (M w - B v) = 0 only for the standard w)."""
    w = synth.workload("disk2d")
    Cs = oracle.Coupling(w.grid, w.coords, w.elems)
    Cd = oracle.Coupling(w.grid, w.coords, w.elems, multiplier="dual")
    v = [synth.sin_cos_2d(synth.grid_node_coords(w.grid, 0))]
    ws = Cs.transfer_velocity(v)[:, 0]
    wd = Cd.transfer_velocity(v)[:, 0]
    assert np.abs(ws - wd).max() > 1e-6
    r_std = Cs.M @ ws - Cs.B[0] @ v[0]
    r_dual = Cs.M @ wd - Cs.B[0] @ v[0]
    assert np.abs(r_std).max() <= 1e-13 * np.abs(Cs.B[0] @ v[0]).max()
    assert np.abs(r_dual).max() > 1e-9
    # L2 error against v restricted to the solid: (w - v)^T M (w - v) minimal for ws
    # expressed with the Galerkin identity ||v - w||^2 = ||v||^2 - 2 w.Bv + w.Mw
    def err(wv):
        return -2 * wv @ (Cs.B[0] @ v[0]) + wv @ (Cs.M @ wv)
    assert err(ws) <= err(wd)


# --------------------------------------------------------------- Picard iteration (Sec. 3, Steps 1-6)

def test_picard_norms_and_criteria_closed_form():
    """Infinity norms of a hand-made example and the two criteria (AC), (RC)."""
    fn = [np.array([1.0, -4.0, 2.0]), np.array([0.5, 0.0, -3.5])]
    fp = [np.array([1.5, -4.0, 2.0]), np.array([0.5, 1.25, -3.5])]
    assert oracle.picard_norms(fn, fp) == (1.25, 4.0)
    assert oracle.picard_converged(1.25, 2.0, 0.0, 4.0)          # (AC)
    assert oracle.picard_converged(1.25, 1.0, 0.5, 4.0)          # (RC): 1.25/4 < 0.5
    assert not oracle.picard_converged(1.25, 1.0, 0.3, 4.0)
    assert not oracle.picard_converged(1.25, 1.0, 0.5, 0.0)      # no reference norm: (AC) only
    assert not oracle.picard_converged(float("nan"), 1.0, 0.5, 4.0)
    # both criteria are strict inequalities in Eqs. (AC) and (RC)
    assert not oracle.picard_converged(1.25, 1.25, 0.0, 4.0)
    assert not oracle.picard_converged(1.25, 1.0, 1.25 / 4.0, 4.0)


def test_picard_loop_reaches_the_fixed_point_of_a_linear_model():
    """With a linear solid (f = -k (w - w_target)) and fluid (v = v0 + beta f~)
    the Picard map is an affine contraction; its limit solves
    (I + beta k T^T T) v = v0 + beta k T^T w_target, computed directly."""
    w_ = synth.workload("disk2d_small")
    C = oracle.Coupling(w_.grid, w_.coords, w_.elems)
    T = C.dense_T(0)
    rng = np.random.default_rng(3)
    v0 = rng.standard_normal(T.shape[1])
    wt = rng.standard_normal(T.shape[0])
    lam = np.linalg.norm(T, 2) ** 2
    k, beta = 1.0, 0.8 / lam
    solid = lambda w: (-k * (w[:, 0] - wt))[:, None]
    fluid = lambda ft: [v0 + beta * ft[0]]
    v, w, f, it, hist = oracle.picard_time_step(C, [v0], solid, fluid, eps_abs=1e-13, eps_rel=1e-14, max_iter=400)
    assert it < 400
    A = np.eye(T.shape[1]) + beta * k * T.T @ T
    v_star = np.linalg.solve(A, v0 + beta * k * T.T @ wt)
    assert np.abs(v[0] - v_star).max() <= 1e-10 * np.abs(v_star).max()
    # the force differences die out (a contraction in this model)
    d = [h[0] for h in hist[1:]]
    assert d[-1] <= 1e-9 * d[0]


# --------------------------------------------------------------- interface-restricted force transfer

@pytest.mark.parametrize("multiplier", ["standard", "dual"])
def test_masked_force_transfer_conserves_force_and_moment(multiplier):
    """With the input restricted to the top and bottom faces Gamma of the beam,
    the fluid force keeps the total force and the first moment of the solid
    force on Gamma: sum_j f~_j = s sum_{i in Gamma} r_i and sum_j x_j f~_j =
    s sum_{i in Gamma} X_i r_i (DUAL mode: Q1 and P1 reproduce 1 and x, and
    B 1 = S 1 for either basis); NODAL mode: sum_j f~_j = s sum_{i in Gamma}
    f_i int phi_i."""
    w = synth.workload("beam32")
    mask = synth.block_face_mask(*synth.BEAM_HEXES["beam32"], axis=2)
    assert 0 < mask.sum() < mask.size
    C = oracle.Coupling(w.grid, w.coords, w.elems, multiplier=multiplier)
    rng = np.random.default_rng(13)
    R = rng.standard_normal((w.coords.shape[0], 3))
    s = 0.7
    ft = C.transfer_force(R, mode="dual", scale=s, mask=mask)
    fn = C.transfer_force(R, mode="nodal", scale=s, mask=mask)
    phi, _ = _phi_integrals(w.coords, w.elems)
    for g in range(3):
        P = synth.grid_node_coords(w.grid, g)
        r = np.where(mask, R[:, g], 0.0)
        assert abs(ft[g].sum() - s * r.sum()) <= 1e-12 * np.abs(r).sum()
        mom = P.T @ ft[g]
        ref = s * (w.coords.T @ r)
        assert np.abs(mom - ref).max() <= 1e-12 * np.abs(r).sum()
        assert abs(fn[g].sum() - s * (phi * r).sum()) <= 1e-12 * (phi * np.abs(r)).sum()
    # nodes outside Gamma do not contribute
    R2 = R.copy()
    R2[~mask] = 1e3 * rng.standard_normal((int((~mask).sum()), 3))
    ft2 = C.transfer_force(R2, mode="dual", scale=s, mask=mask)
    for g in range(3):
        assert np.array_equal(ft2[g], ft[g])


# --------------------------------------------------------------- stretched (rectilinear) grids

def _cell_box(sg, c):
    d = sg.dim
    ci = [c % sg.ncell[0], (c // sg.ncell[0]) % sg.ncell[1]]
    if d == 3:
        ci.append(c // (sg.ncell[0] * sg.ncell[1]))
    lo = [float(sg.axis[k][ci[k]]) for k in range(d)]
    hi = [float(sg.axis[k][ci[k] + 1]) for k in range(d)]
    return lo, hi


@pytest.mark.parametrize("name,stride", [("disk2d_s", 7), ("beam16s", 17)])
def test_stretched_pair_blocks_match_exact_rational(name, stride):
    """On a stretched grid every cell has its own widths; the blocks agree with
    exact rational integration over the exact cell [x_i, x_{i+1}] to 1e-14 |E|."""
    w = synth.workload(name)
    d = w.dim
    vol_e = oracle.element_volumes(w.coords, w.elems)
    for g in range(oracle.n_grids(w.grid)):
        sg = oracle.subgrid(w.grid, g)
        assert sg.axis is not None
        pe, pc = oracle.candidate_pairs(sg, w.coords, w.elems)
        blocks, vols = oracle.pair_blocks(sg, w.coords, w.elems, pe, pc)
        for p in range(g, len(pe), stride):
            e, c = int(pe[p]), int(pc[p])
            lo, hi = _cell_box(sg, c)
            blk, vol = exact.pair_block_exact(d, w.coords[w.elems[e]], lo, None, cell_hi=hi)
            ex = np.array([[float(x) for x in row] for row in blk])
            assert abs(float(vol) - vols[p]) <= 1e-14 * vol_e[e]
            assert np.abs(ex - blocks[p]).max() <= 1e-14 * vol_e[e], (p, ex, blocks[p])


@pytest.mark.parametrize("dim", [2, 3])
def test_stretched_candidate_pairs_match_bruteforce(dim):
    """Candidate cells on stretched axes are exactly the half-open cells
    [x_i, x_{i+1}) with x_{i+1} > lo and x_i < hi, including vertices placed
    exactly on nodes; elements leaving the grid are reported."""
    rng = np.random.default_rng(17 + dim)
    n = 12
    grid = synth.stretched_grid(dim, n, 0.6, staggered=(dim == 3))
    for g in range(oracle.n_grids(grid)):
        sg = oracle.subgrid(grid, g)
        ax = sg.axis
        m = 60
        lo_b = np.array([ax[k][1] for k in range(dim)])
        hi_b = np.array([ax[k][-2] for k in range(dim)])
        X = lo_b + (hi_b - lo_b) * rng.random((m * (dim + 1), dim))
        # a third of the coordinates exactly on a node
        on = rng.random(X.shape) < 0.33
        for k in range(dim):
            idx = rng.integers(1, len(ax[k]) - 1, size=X.shape[0])
            X[on[:, k], k] = ax[k][idx[on[:, k]]]
        E = np.arange(m * (dim + 1), dtype=np.int32).reshape(m, dim + 1)
        pe, pc = oracle.candidate_pairs(sg, X, E)
        got = set(zip(pe.tolist(), pc.tolist()))
        ref = set()
        nc = sg.ncell
        for e in range(m):
            V = X[E[e]]
            lo, hi = V.min(axis=0), V.max(axis=0)
            ranges = []
            for k in range(dim):
                cells = [i for i in range(nc[k]) if ax[k][i + 1] > lo[k] and ax[k][i] < hi[k]]
                if not cells:  # zero extent exactly on a node: the cell that starts there
                    cells = [int(np.searchsorted(ax[k], lo[k], side="right")) - 1]
                ranges.append(cells)
            for cz in (ranges[2] if dim == 3 else [0]):
                for cy in ranges[1]:
                    for cx in ranges[0]:
                        ref.add((e, cx + nc[0] * (cy + nc[1] * cz)))
        assert got == ref
    # leaving the grid is reported
    sg = oracle.subgrid(grid, 0)
    Xb = np.zeros((dim + 1, dim)) + 0.5
    Xb[0, 0] = -1e-3
    with pytest.raises(oracle.OracleError):
        oracle.candidate_pairs(sg, Xb, np.arange(dim + 1, dtype=np.int32)[None])


@pytest.mark.parametrize("name", ["disk2d_s", "beam16s", "beam32s"])
def test_stretched_row_sums_and_affine_reproduction(name):
    """P1 row sums, the total volume and affine reproduction hold on stretched
    grids (Q1 on a rectilinear cell contains the affine functions)."""
    w = synth.workload(name)
    d = w.dim
    phi, vol = _phi_integrals(w.coords, w.elems)
    C = oracle.Coupling(w.grid, w.coords, w.elems, nthreads=4)
    for g, B in enumerate(C.B):
        rs = np.asarray(B.sum(axis=1)).ravel()
        assert np.abs(rs - phi).max() <= 1e-14 * phi.max()
        assert abs(C.pairs[g][3].sum() - vol.sum()) <= 1e-14 * vol.sum()
    coef = np.array([0.3, 1.5, -0.7, 2.0])[: d + 1]
    fields = [coef[0] + synth.grid_node_coords(w.grid, g) @ coef[1:] + g for g in range(oracle.n_grids(w.grid))]
    W = C.transfer_velocity(fields)
    ex = np.stack([coef[0] + w.coords @ coef[1:] + g for g in range(len(fields))], axis=1)
    assert np.abs(W - ex).max() <= 1e-13 * np.abs(ex).max()


def test_uniform_grid_given_as_node_arrays_matches_the_uniform_path():
    """A uniform grid passed as explicit node arrays (dyadic spacing: the nodes
    are exact) gives the same pairs and the same blocks as the uniform path."""
    w = synth.workload("beam16")
    n = w.grid.ncell[0]
    ax = tuple(np.arange(n + 1, dtype=np.float64) / n for _ in range(3))
    grid_s = synth.Grid(3, w.grid.ncell, w.grid.h, w.grid.origin, True, ax)
    for g in range(3):
        su, ss = oracle.subgrid(w.grid, g), oracle.subgrid(grid_s, g)
        pu = oracle.candidate_pairs(su, w.coords, w.elems)
        ps = oracle.candidate_pairs(ss, w.coords, w.elems)
        assert np.array_equal(pu[0], ps[0]) and np.array_equal(pu[1], ps[1])
        bu, vu = oracle.pair_blocks(su, w.coords, w.elems, *pu)
        bs, vs = oracle.pair_blocks(ss, w.coords, w.elems, *ps)
        assert np.abs(bu - bs).max() <= 1e-16 and np.abs(vu - vs).max() <= 1e-16
