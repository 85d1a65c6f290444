"""Stretched (rectilinear) grids on the CUDA path against the oracle: the
candidate pairs bit for bit (comparisons only on stretched axes), the blocks,
B and S, and both transfers, on the plain, fused FP64 and mixed forms, the
dual basis and a captured step.  The paper's fluid grids are all stretched to
concentrate points around the structure (Sec. 4)."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import NTHREADS, csr_from_gpu, gpu_coupling, max_row_rel, oracle_coupling, rel_fro, rel_l2, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = ["disk2d_s", "beam16s", "beam32s", "beam64s"]
FORMS = [("fused", "fp64"), ("plain", "fp64"), ("fused", "mixed")]


def _l2x():
    import paper_1810_13046_gb300 as l2x
    return l2x


def _coupling(w, path, precision, **kw):
    l2x = _l2x()
    mixed = precision == "mixed"
    return gpu_coupling(w, path=l2x.FUSED if path == "fused" else l2x.PLAIN,
                        precision=l2x.MIXED if mixed else l2x.FP64, cg_rtol=1e-9 if mixed else 1e-14, **kw)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("path", ["fused", "plain"])
def test_stretched_pairs_bit_exact(name, path):
    w = workload(name)
    c = _coupling(w, path, "fp64")
    oc = oracle_coupling(name)
    for g in range(oracle.n_grids(w.grid)):
        e, cell = c.export_pairs(g)
        assert np.array_equal(e.cpu().numpy(), oc.pairs[g][0])
        assert np.array_equal(cell.cpu().numpy().astype(np.int64), oc.pairs[g][1])


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("path,precision", FORMS)
def test_stretched_blocks_matrices_and_transfers(name, path, precision):
    w = workload(name)
    mixed = precision == "mixed"
    c = _coupling(w, path, precision)
    oc = oracle_coupling(name)
    tol = 1e-6 if mixed else 1e-12
    vol_e = oracle.element_volumes(w.coords, w.elems)
    for g, B in enumerate(oc.B):
        if path == "fused":
            b, v = c.export_pair_blocks(g)
            scale = vol_e[oc.pairs[g][0]]
            err = np.abs(b.cpu().numpy() - oc.pairs[g][2]).max(axis=(1, 2)) / scale
            assert err.max() <= tol
        Bg = csr_from_gpu(c, g, B.shape[1])
        assert rel_fro(Bg, B) <= tol
        assert max_row_rel(Bg, B) <= 10 * tol
    M = csr_from_gpu(c, 3, c.n_nodes)
    assert rel_fro(M, oc.M) <= 1e-14
    dt = np.float32 if mixed else np.float64
    u_s = c.transfer_velocity([torch.from_numpy(f.astype(dt)).cuda() for f in w.fields])
    ref = oc.transfer_velocity([f.astype(dt).astype(np.float64) for f in w.fields])
    assert rel_l2(np.stack([u.cpu().numpy() for u in u_s], axis=1), ref) <= tol
    F = w.force.astype(dt)
    f_f = c.transfer_force([torch.from_numpy(np.ascontiguousarray(F[:, g])).cuda() for g in range(F.shape[1])])
    fref = oc.transfer_force(F.astype(np.float64), mode="dual")
    for g in range(len(fref)):
        assert rel_l2(f_f[g].cpu().numpy(), fref[g]) <= tol


def test_stretched_affine_reproduction_and_dual_basis():
    """Affine fields come back exactly on a stretched grid, for the standard and
    the dual multiplier basis (which needs no solve)."""
    l2x = _l2x()
    w = workload("beam32s")
    coef = np.array([0.2, -1.1, 0.7, 1.3])
    fields = [coef[0] + synth.grid_node_coords(w.grid, g) @ coef[1:] + g for g in range(3)]
    ex = np.stack([coef[0] + w.coords @ coef[1:] + g for g in range(3)], axis=1)
    for mult in (l2x.STANDARD_BASIS, l2x.DUAL_BASIS):
        c = gpu_coupling(w, cg_rtol=1e-14, multiplier=mult)
        u = np.stack([x.cpu().numpy() for x in c.transfer_velocity([torch.from_numpy(f).cuda() for f in fields])],
                     axis=1)
        assert np.abs(u - ex).max() <= 1e-12 * np.abs(ex).max()
    od = oracle.Coupling(w.grid, w.coords, w.elems, nthreads=NTHREADS, multiplier="dual")
    c = gpu_coupling(w, multiplier=l2x.DUAL_BASIS)
    for g in range(3):
        assert rel_fro(csr_from_gpu(c, g, od.B[g].shape[1]), od.B[g]) <= 1e-12


def test_stretched_step_graph():
    """A captured step re-assembles on a stretched grid like a fresh build."""
    l2x = _l2x()
    w = workload("beam32s")
    c = gpu_coupling(w, precision=l2x.MIXED, cg_rtol=1e-9)
    u_f = [torch.from_numpy(f.astype(np.float32)).cuda() for f in w.fields]
    f_s = [torch.from_numpy(np.ascontiguousarray(w.force[:, g].astype(np.float32))).cuda() for g in range(3)]
    u_s = [torch.zeros(c.n_nodes, dtype=torch.float32, device="cuda") for _ in range(3)]
    f_f = [torch.zeros(n, dtype=torch.float32, device="cuda") for n in c.fluid_sizes()]
    # move the beam a little so the replay re-assembles a new configuration
    X1 = w.coords + np.array([0.0071, -0.0043, 0.0029])
    src = torch.from_numpy(w.coords).cuda()
    g = c.capture_step(src, u_f, u_s, f_s, f_f, margin=1.5)
    src.copy_(torch.from_numpy(X1).cuda())
    g.launch()
    g.status()
    oc = oracle.Coupling(w.grid, X1, w.elems, nthreads=NTHREADS)
    ref = oc.transfer_velocity([f.astype(np.float32).astype(np.float64) for f in w.fields])
    assert rel_l2(torch.stack(u_s).cpu().numpy().T, ref) <= 1e-6
