"""Parity of the dual multiplier basis ("pseudo" L2 projection, Eq. (biorth) in
Sec. 2.3) on the CUDA path against the FP64 oracle.

With the dual basis, B is assembled from the weights (d+2) lambda_a - 1 and S is
diagonal, so the velocity transfer is one sparse product and a division (no CG)
and the force transfer a division and one product with B^T.  The bars are those
of the standard space: 1e-12 relative in FP64, 1e-6 in the mixed form.
"""
import numpy as np
import pytest

import oracle
import synth
from _helpers import NTHREADS, csr_from_gpu, gpu_coupling, max_row_rel, rel_fro, rel_l2, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL_MIXED = 1e-6
CASES = ["disk2d", "disk2d_small", "beam16", "beam32", "leaflet32", "beam128"]
FORMS = [("fused", "fp64"), ("plain", "fp64"), ("fused", "mixed")]
_ORACLE = {}


def _l2x():
    import paper_1810_13046_gb300 as l2x
    return l2x


def _oracle(name):
    if name not in _ORACLE:
        w = workload(name)
        _ORACLE[name] = oracle.Coupling(w.grid, w.coords, w.elems, nthreads=NTHREADS, multiplier="dual")
    return _ORACLE[name]


def _coupling(w, path, precision, **kw):
    l2x = _l2x()
    return gpu_coupling(w, path=l2x.FUSED if path == "fused" else l2x.PLAIN,
                        precision=l2x.MIXED if precision == "mixed" else l2x.FP64,
                        multiplier=l2x.DUAL_BASIS, **kw)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("path,precision", FORMS)
def test_dual_matrices(name, path, precision):
    """B of the dual basis entry by entry; S = diag(int phi_i) with one entry per row."""
    w = workload(name)
    c = _coupling(w, path, precision)
    oc = _oracle(name)
    tol = TOL_MIXED if precision == "mixed" else TOL64
    assert c.info()["multiplier"] == 1
    for g, B in enumerate(oc.B):
        Bg = csr_from_gpu(c, g, B.shape[1])
        assert rel_fro(Bg, B) <= tol
        assert max_row_rel(Bg, B) <= 10 * tol
    S = csr_from_gpu(c, 3, c.n_nodes)
    assert S.nnz == c.n_nodes
    assert np.array_equal(S.indices, np.arange(c.n_nodes))
    assert rel_fro(S, oc.M) <= 1e-14


def _affine(w, coef):
    d = w.dim
    coef = np.asarray(coef)[: d + 1]
    fields = [coef[0] + synth.grid_node_coords(w.grid, g) @ coef[1:] + g for g in range(oracle.n_grids(w.grid))]
    exact = np.stack([coef[0] + w.coords @ coef[1:] + g for g in range(len(fields))], axis=1)
    return fields, exact


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("path,precision", FORMS)
def test_dual_velocity_transfer(name, path, precision):
    """u_s = S^-1 B u_f on the workload field; affine fields come back exactly
    (to rounding), with no iterations."""
    w = workload(name)
    mixed = precision == "mixed"
    c = _coupling(w, path, precision)
    oc = _oracle(name)
    dt = np.float32 if mixed else np.float64
    tol = TOL_MIXED if mixed else TOL64
    aff, exact = _affine(w, [0.3, -1.2, 0.8, 1.9])
    for fields in (w.fields, aff):
        f_in = [f.astype(dt) for f in fields]
        u_s = c.transfer_velocity([torch.from_numpy(f).cuda() for f in f_in])
        ref = oc.transfer_velocity([f.astype(np.float64) for f in f_in])
        got = np.stack([u.cpu().numpy() for u in u_s], axis=1)
        assert rel_l2(got, ref) <= tol
        assert c.info()["cg_iters"] == 0
    if not mixed:
        assert np.abs(got - exact).max() <= 1e-12 * np.abs(exact).max()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("mode", ["dual", "nodal"])
@pytest.mark.parametrize("path,precision", FORMS)
def test_dual_force_transfer(name, mode, path, precision):
    """f_f += s B^T S^-1 r (dual force mode) or s B^T f (nodal), accumulated."""
    l2x = _l2x()
    w = workload(name)
    mixed = precision == "mixed"
    scale = 1.25
    c = _coupling(w, path, precision, force_mode=l2x.DUAL if mode == "dual" else l2x.NODAL, force_scale=scale)
    oc = _oracle(name)
    dt = np.float32 if mixed else np.float64
    F = w.force.astype(dt)
    ref = oc.transfer_force(F.astype(np.float64), mode=mode, scale=scale)
    f_s = [torch.from_numpy(np.ascontiguousarray(F[:, g])).cuda() for g in range(F.shape[1])]
    tol = TOL_MIXED if mixed else TOL64
    f_f = c.transfer_force(f_s)
    for g in range(len(ref)):
        assert rel_l2(f_f[g].cpu().numpy(), ref[g]) <= tol
    # accumulation: base + value up to the roundings of the sums
    rng = np.random.default_rng(6)
    base = [(0.5 * np.abs(r).max() * rng.random(r.shape[0])).astype(dt) for r in ref]
    f_acc = [torch.from_numpy(b.copy()).cuda() for b in base]
    c.transfer_force(f_s, f_acc)
    eps = np.finfo(dt).eps
    for g in range(len(ref)):
        b64, v64 = base[g].astype(np.float64), f_f[g].cpu().numpy().astype(np.float64)
        # roundings of the sums in the field type (the plain path adds term by term)
        bound = 64 * eps * (np.linalg.norm(b64) + np.linalg.norm(v64))
        assert np.linalg.norm(f_acc[g].cpu().numpy() - (b64 + v64)) <= bound


def test_dual_autograd_is_the_adjoint():
    """Backward of the dual velocity transfer = T^T with T = S^-1 B (dense oracle)."""
    l2x = _l2x()
    w = workload("leaflet32")
    oc = _oracle("leaflet32")
    c = _coupling(w, "fused", "fp64")
    rng = np.random.default_rng(12)
    u = [torch.from_numpy(rng.standard_normal(n)).cuda().requires_grad_(True) for n in c.fluid_sizes()]
    out = l2x.VelocityTransfer.apply(c, *u)
    gw = [torch.from_numpy(rng.standard_normal(c.n_nodes)).cuda() for _ in out]
    sum((o * g).sum() for o, g in zip(out, gw)).backward()
    for g in range(3):
        ref = oc.dense_T(g).T @ gw[g].cpu().numpy()
        assert rel_l2(u[g].grad.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dual_step_graph_matches_fresh_assembly(precision):
    """A captured time step with the dual basis equals a fresh per-call assembly
    on the same moved positions, and the oracle on one body."""
    l2x = _l2x()
    grid, bodies, E, nr, er = synth.batch_workload(5, 64, 300, 5000, 8)
    fields = [synth.taylor_green(synth.grid_node_coords(grid, g), g) for g in range(3)]
    mixed = precision == "mixed"
    dt = torch.float32 if mixed else torch.float64
    X0 = synth.batch_coords(bodies, 0, 10)
    mk = lambda X: l2x.Coupling(grid, torch.from_numpy(X).cuda(), torch.from_numpy(E).cuda(),
                                precision=l2x.MIXED if mixed else l2x.FP64, multiplier=l2x.DUAL_BASIS)
    c = mk(X0)
    n = X0.shape[0]
    F = np.random.default_rng(2).standard_normal((n, 3))
    u_f = [torch.from_numpy(f).cuda().to(dt) for f in fields]
    f_s = [torch.from_numpy(np.ascontiguousarray(F[:, g])).cuda().to(dt) for g in range(3)]
    u_s = [torch.zeros(n, dtype=dt, device="cuda") for _ in range(3)]
    f_f = [torch.zeros(m, dtype=dt, device="cuda") for m in c.fluid_sizes()]
    src = torch.from_numpy(X0).cuda()
    graph = c.capture_step(src, u_f, u_s, f_s, f_f, margin=1.5)
    tol = TOL_MIXED if mixed else TOL64
    for step in (1, 4):
        Xt = synth.batch_coords(bodies, step, 10)
        src.copy_(torch.from_numpy(Xt).cuda())
        graph.launch()
        graph.status()
        ref = mk(Xt)
        ur = ref.transfer_velocity(u_f)
        fr = ref.transfer_force(f_s)
        assert rel_l2(torch.stack(u_s).cpu().numpy(), torch.stack(ur).cpu().numpy()) <= tol
        for a, b in zip(f_f, fr):
            assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= tol
    # every body against the oracle on that body alone (its rows of B and S
    # involve only its own elements)
    src_fields = [f.astype(np.float32).astype(np.float64) if mixed else f for f in fields]
    got_all = torch.stack(u_s).cpu().numpy().T
    for k in range(len(bodies)):
        n0, n1 = nr[k]
        e0, e1 = er[k]
        ok = oracle.Coupling(grid, Xt[n0:n1], E[e0:e1] - n0, nthreads=NTHREADS, multiplier="dual")
        assert rel_l2(got_all[n0:n1], ok.transfer_velocity(src_fields)) <= tol, k
