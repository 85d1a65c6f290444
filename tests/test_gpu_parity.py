"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Pairs must match bit for bit; B, M_s and the transferred fields within 1e-12
relative in FP64 (plain and fused paths) and 1e-6 in the mixed FP32/FP64 form.
Mortar integrals and transfer: Sec. 2.3 "Variational Transfer"; assembly steps
(I)-(IV) there.
"""
import numpy as np
import pytest

import oracle
import synth
from _helpers import (csr_from_gpu, gpu_coupling, max_row_rel, oracle_coupling, rel_fro, rel_l2, workload)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL_MIXED = 1e-6

SMALL = ["disk2d", "disk2d_small", "beam16", "beam32", "leaflet32"]


def _l2x():
    import paper_1810_13046_gb300 as l2x
    return l2x


def _fields(w, dtype):
    return [torch.from_numpy(f.astype(dtype)).cuda() for f in w.fields]


@pytest.mark.parametrize("name", SMALL + ["beam128"])
@pytest.mark.parametrize("path", ["fused", "plain"])
def test_candidate_pairs_bit_exact(name, path):
    l2x = _l2x()
    w = workload(name)
    c = gpu_coupling(w, path=l2x.FUSED if path == "fused" else l2x.PLAIN)
    oc = oracle_coupling(name)
    for g in range(oracle.n_grids(w.grid)):
        e, cell = c.export_pairs(g)
        pe, pc = oc.pairs[g][0], oc.pairs[g][1]
        assert np.array_equal(e.cpu().numpy(), pe)
        assert np.array_equal(cell.cpu().numpy().astype(np.int64), pc)


@pytest.mark.parametrize("name", SMALL + ["beam128"])
@pytest.mark.parametrize("path,precision", [("fused", "fp64"), ("plain", "fp64"), ("fused", "mixed")])
def test_pair_blocks(name, path, precision):
    """Local blocks int_{E∩C} lambda_a psi_b and |E∩C| against the oracle, pair by
    pair, scaled by the element volume."""
    l2x = _l2x()
    w = workload(name)
    c = gpu_coupling(w, path=l2x.FUSED if path == "fused" else l2x.PLAIN,
                     precision=l2x.MIXED if precision == "mixed" else l2x.FP64)
    oc = oracle_coupling(name)
    vol_e = oracle.element_volumes(w.coords, w.elems)
    tol = TOL_MIXED if precision == "mixed" else TOL64
    for g in range(oracle.n_grids(w.grid)):
        b, v = c.export_pair_blocks(g)
        b, v = b.cpu().numpy(), v.cpu().numpy()
        ob, ov = oc.pairs[g][2], oc.pairs[g][3]
        scale = vol_e[oc.pairs[g][0]]
        # intersection volumes: FP64-level in every form (the mixed form keeps them
        # in double-float), so that no sliver is lost to FP32 rounding
        assert (np.abs(v - ov) <= TOL64 * scale + 1e-300).all()
        err = np.abs(b - ob).max(axis=(1, 2)) / scale
        assert err.max() <= tol, (int(err.argmax()), float(err.max()))


@pytest.mark.parametrize("name", SMALL + ["beam128"])
@pytest.mark.parametrize("path,precision", [("fused", "fp64"), ("plain", "fp64"), ("fused", "mixed")])
def test_coupling_and_mass_matrices(name, path, precision):
    l2x = _l2x()
    w = workload(name)
    c = gpu_coupling(w, path=l2x.FUSED if path == "fused" else l2x.PLAIN,
                     precision=l2x.MIXED if precision == "mixed" else l2x.FP64)
    oc = oracle_coupling(name)
    tol = TOL_MIXED if precision == "mixed" else TOL64
    for g, B in enumerate(oc.B):
        Bg = csr_from_gpu(c, g, B.shape[1])
        assert rel_fro(Bg, B) <= tol
        assert max_row_rel(Bg, B) <= 10 * tol
        # sparsity: the GPU pattern may differ from the oracle's only in entries
        # that are negligible on both sides (pairs whose volume rounds to zero)
        if precision == "fp64":
            diff = (Bg != 0).astype(np.int8) - (B != 0).astype(np.int8)
            if diff.nnz:
                D = abs(Bg - B)
                assert D.max() <= 1e-13 * abs(B).max()
    M = csr_from_gpu(c, 3, c.n_nodes)
    assert rel_fro(M, oc.M) <= 1e-14
    assert (M != 0).nnz == oc.M.nnz


def _affine_fields(w, dtype):
    d = w.dim
    coef = np.array([0.3, 1.5, -0.7, 2.0])[: d + 1]
    fields = []
    for g in range(oracle.n_grids(w.grid)):
        P = synth.grid_node_coords(w.grid, g)
        fields.append(coef[0] + P @ coef[1:] + g)
    exact = np.stack([coef[0] + w.coords @ coef[1:] + g for g in range(len(fields))], axis=1)
    return fields, exact


@pytest.mark.parametrize("name", SMALL + ["beam128"])
@pytest.mark.parametrize("path,precision", [("fused", "fp64"), ("plain", "fp64"), ("fused", "mixed")])
def test_velocity_transfer(name, path, precision):
    """u_s = M^-1 B u_f on the workload's field and on an affine field (which the
    projection reproduces exactly, Q1 and P1 both containing the affine functions)."""
    l2x = _l2x()
    w = workload(name)
    mixed = precision == "mixed"
    c = gpu_coupling(w, path=l2x.FUSED if path == "fused" else l2x.PLAIN,
                     precision=l2x.MIXED if mixed else l2x.FP64, cg_rtol=1e-9 if mixed else 1e-14)
    oc = oracle_coupling(name)
    dt = np.float32 if mixed else np.float64
    tol = TOL_MIXED if mixed else TOL64
    for fields in (w.fields, _affine_fields(w, dt)[0]):
        f_in = [f.astype(dt) for f in fields]
        u_s = c.transfer_velocity([torch.from_numpy(f).cuda() for f in f_in])
        ref = oc.transfer_velocity([f.astype(np.float64) for f in f_in])
        got = np.stack([u.cpu().numpy() for u in u_s], axis=1)
        assert rel_l2(got, ref) <= tol
        info = c.info()
        assert info["cg_residual"] <= (1e-9 if mixed else 1e-14)


@pytest.mark.parametrize("name", SMALL + ["beam128"])
@pytest.mark.parametrize("mode", ["dual", "nodal"])
@pytest.mark.parametrize("path,precision", [("fused", "fp64"), ("plain", "fp64"), ("fused", "mixed")])
def test_force_transfer(name, mode, path, precision):
    """f_f += s B^T M^-1 r (dual) or s B^T f (nodal), accumulated into the fluid arrays."""
    l2x = _l2x()
    w = workload(name)
    mixed = precision == "mixed"
    scale = 0.75
    c = gpu_coupling(w, path=l2x.FUSED if path == "fused" else l2x.PLAIN,
                     precision=l2x.MIXED if mixed else l2x.FP64, cg_rtol=1e-9 if mixed else 1e-14,
                     force_mode=l2x.DUAL if mode == "dual" else l2x.NODAL, force_scale=scale)
    oc = oracle_coupling(name)
    dt = np.float32 if mixed else np.float64
    F = w.force.astype(dt)
    ref = oc.transfer_force(F.astype(np.float64), mode=mode, scale=scale)
    f_s = [torch.from_numpy(np.ascontiguousarray(F[:, g])).cuda() for g in range(F.shape[1])]
    tol = TOL_MIXED if mixed else TOL64
    # the value, into zeroed fluid arrays
    f_f = c.transfer_force(f_s)
    for g in range(len(ref)):
        assert rel_l2(f_f[g].cpu().numpy(), ref[g]) <= tol
    # the call accumulates: from a non-zero array of the result's magnitude the
    # result is base + value, up to the roundings of the sums in the field type
    rng = np.random.default_rng(4)
    base = [(0.5 * np.abs(r).max() * rng.random(r.shape[0])).astype(dt) for r in ref]
    f_acc = [torch.from_numpy(b.copy()).cuda() for b in base]
    c.transfer_force(f_s, f_acc)
    eps = np.finfo(dt).eps
    for g in range(len(ref)):
        b64, v64 = base[g].astype(np.float64), f_f[g].cpu().numpy().astype(np.float64)
        # roundings of the sums in the field type (the plain path adds term by term)
        bound = 64 * eps * (np.linalg.norm(b64) + np.linalg.norm(v64))
        assert np.linalg.norm(f_acc[g].cpu().numpy() - (b64 + v64)) <= bound


def test_fused_build_is_deterministic():
    l2x = _l2x()
    w = workload("beam32")
    c1 = gpu_coupling(w)
    c2 = gpu_coupling(w)
    for which in (0, 1, 2, 3):
        a = c1.export_csr(which)
        b = c2.export_csr(which)
        for x, y in zip(a, b):
            assert torch.equal(x, y)


def test_update_geometry_matches_fresh_oracle():
    l2x = _l2x()
    w = workload("beam32")
    c = gpu_coupling(w)
    rng = np.random.default_rng(5)
    X2 = w.coords + np.array([0.013, -0.021, 0.008]) + rng.uniform(-1e-3, 1e-3, size=w.coords.shape)
    c.update_geometry(torch.from_numpy(X2).cuda())
    oc = oracle.Coupling(w.grid, X2, w.elems, nthreads=8)
    for g, B in enumerate(oc.B):
        e, cell = c.export_pairs(g)
        assert np.array_equal(e.cpu().numpy(), oc.pairs[g][0])
        assert np.array_equal(cell.cpu().numpy().astype(np.int64), oc.pairs[g][1])
        assert rel_fro(csr_from_gpu(c, g, B.shape[1]), B) <= TOL64
    assert rel_fro(csr_from_gpu(c, 3, c.n_nodes), oc.M) <= 1e-14


# ---------------------------------------------------------------- edge cases

def _one_element(dim, verts, n=8, staggered=None):
    grid = synth.Grid(dim, (n,) * dim, (1.0 / n,) * dim, (0.0,) * dim, dim == 3 if staggered is None else staggered)
    X = np.asarray(verts, dtype=np.float64)
    E = np.arange(dim + 1, dtype=np.int32)[None]
    w = synth.meshes.Workload("one", grid, X, E, [])
    return w


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("case", ["inside_one_cell", "on_grid_lines", "spans_many_cells"])
def test_single_element_cases(dim, case):
    """Degenerate and extreme geometry: an element strictly inside one cell (no
    clipping), vertices exactly on grid lines (ties of the index rule), and one
    element spanning ~20 cells per axis (every cell plane cuts it; row boxes larger
    than the shared-memory tile)."""
    l2x = _l2x()
    rng = np.random.default_rng(2)
    n = 32
    h = 1.0 / n
    if case == "inside_one_cell":
        V = (5 + 0.15 + 0.7 * rng.random((dim + 1, dim))) * h
    elif case == "on_grid_lines":
        V = np.array([[5, 5, 5], [9, 6, 5], [6, 10, 7], [7, 6, 11]][: dim + 1], dtype=np.float64)[:, :dim] * h
    else:
        V = np.array([[3.3, 4.1, 3.7], [27.2, 5.6, 4.4], [5.1, 28.3, 6.2], [6.4, 5.5, 27.9]][: dim + 1])[:, :dim] * h
    w = _one_element(dim, V, n)
    oc = oracle.Coupling(w.grid, w.coords, w.elems)
    for path in (l2x.FUSED, l2x.PLAIN):
        c = gpu_coupling(w, path=path)
        for g, B in enumerate(oc.B):
            e, cell = c.export_pairs(g)
            assert np.array_equal(cell.cpu().numpy().astype(np.int64), oc.pairs[g][1])
            assert rel_fro(csr_from_gpu(c, g, B.shape[1]), B) <= TOL64


@pytest.mark.parametrize("bad", ["outside", "degenerate", "nan", "bad_index"])
def test_errors_are_reported_not_trapped(bad):
    l2x = _l2x()
    w = workload("beam16")
    X = w.coords.copy()
    E = w.elems.copy()
    expect = {"outside": 4, "degenerate": 5, "nan": 9, "bad_index": 1}[bad]
    if bad == "outside":
        X[:, 0] += 0.45
    elif bad == "degenerate":
        X[E[3, 1]] = X[E[3, 0]]
    elif bad == "nan":
        X[7, 1] = np.nan
    else:
        E[2, 2] = X.shape[0] + 5
    ww = synth.meshes.Workload("bad", w.grid, X, E, [])
    with pytest.raises(l2x.L2XError) as ei:
        gpu_coupling(ww)
    assert ei.value.status == expect
    # the context is still usable afterwards
    c = gpu_coupling(w)
    assert c.info()["n_pairs_total"] > 0


# ---------------------------------------------------------------- autograd

def test_autograd_velocity_and_force_transfer():
    """Hand-written backward = exact adjoint: against the oracle's dense T^T and
    FP64 central finite differences (step 1e-6) on the 32^3 / 2352-tet leaflet."""
    l2x = _l2x()
    w = workload("leaflet32")
    oc = oracle_coupling("leaflet32")
    c = gpu_coupling(w, cg_rtol=1e-14)
    rng = np.random.default_rng(9)
    u = [torch.from_numpy(rng.standard_normal(n)).cuda().requires_grad_(True) for n in c.fluid_sizes()]
    out = l2x.VelocityTransfer.apply(c, *u)
    gw = [torch.from_numpy(rng.standard_normal(c.n_nodes)).cuda() for _ in out]
    loss = sum((o * g).sum() for o, g in zip(out, gw))
    loss.backward()
    for g in range(3):
        T = oc.dense_T(g)
        ref = T.T @ gw[g].cpu().numpy()
        assert rel_l2(u[g].grad.cpu().numpy(), ref) <= 1e-11
    # central differences along a random direction of grid 1
    v = rng.standard_normal(c.fluid_sizes()[1])
    eps = 1e-6
    up = [x.detach().clone() for x in u]
    um = [x.detach().clone() for x in u]
    up[1] += eps * torch.from_numpy(v).cuda()
    um[1] -= eps * torch.from_numpy(v).cuda()
    fd = (c.transfer_velocity(up)[1] - c.transfer_velocity(um)[1]).cpu().numpy() / (2 * eps)
    assert rel_l2(fd, oc.dense_T(1) @ v) <= 1e-8
    # force transfer (dual): backward = s M^-1 B
    f = [torch.from_numpy(rng.standard_normal(c.n_nodes)).cuda().requires_grad_(True) for _ in range(3)]
    ff = l2x.ForceTransfer.apply(c, *f)
    gf = [torch.from_numpy(rng.standard_normal(n)).cuda() for n in c.fluid_sizes()]
    sum((a * b).sum() for a, b in zip(ff, gf)).backward()
    for g in range(3):
        ref = oc.dense_T(g) @ gf[g].cpu().numpy()
        assert rel_l2(f[g].grad.cpu().numpy(), ref) <= 1e-11


def test_autotune_keeps_results():
    """The autotuner only changes work-chunk sizes: pair blocks are identical and
    the transfers agree to solver tolerance after tuning."""
    l2x = _l2x()
    w = workload("beam32")
    c = gpu_coupling(w, cg_rtol=1e-14)
    u = [torch.from_numpy(f).cuda() for f in w.fields]
    before = torch.stack(c.transfer_velocity(u)).cpu().numpy()
    b0 = c.export_pair_blocks(0)[0].clone()
    choice = c.autotune()
    assert choice["clip_block"] in (64, 128, 256) and choice["pcg_rows_per_block"] in (32, 64, 128, 256, 512, 1024)
    assert choice["pcg_cluster"] in (0, 8, 16)
    c.update_geometry(torch.from_numpy(w.coords).cuda())
    assert torch.equal(c.export_pair_blocks(0)[0], b0)
    after = torch.stack(c.transfer_velocity(u)).cpu().numpy()
    assert rel_l2(after, before) <= 1e-13
