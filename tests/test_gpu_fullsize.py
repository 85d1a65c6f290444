"""Parity at the full sizes of the larger workloads, on sampled outputs the
oracle computes one by one and on properties that hold at any size.

* 952,200-tet curved leaflet on 256^3 staggered grids (differentiable-transfer
  workload) and 3,993,600-tet deformed beam on 512x512x256 grids (mixed-precision
  workload), in the launch configuration bench.py uses (fused path).
* Sampled: candidate pairs (bit-exact), local blocks and intersection volumes of
  several element ranges spread over the mesh, against the FP64 oracle.
* At any size: partition-of-unity row sums of every B_g, reproduction of an affine
  field by the velocity transfer, FP64 vs mixed agreement of the transfers.
* Whole leaflet: the chosen mixed form's transfers (velocity, dual and nodal
  force) against the oracle's, node by node, to 1e-6.
"""
import numpy as np
import pytest

import oracle
from _helpers import oracle_coupling, rel_l2, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [("leaflet256", "fp64"), ("leaflet256", "mixed"), ("beam512", "mixed"), ("beam512", "fp64")]


def _coupling(w, precision):
    import paper_1810_13046_gb300 as l2x
    X = torch.from_numpy(w.coords).cuda()
    E = torch.from_numpy(w.elems).cuda()
    prec = l2x.MIXED if precision == "mixed" else l2x.FP64
    return l2x.Coupling(w.grid, X, E, path=l2x.FUSED, precision=prec,
                        cg_rtol=1e-9 if precision == "mixed" else 1e-13)


@pytest.mark.parametrize("name,precision", CASES)
def test_sampled_pairs_and_blocks(name, precision):
    w = workload(name)
    c = _coupling(w, precision)
    m = w.elems.shape[0]
    tol = 1e-6 if precision == "mixed" else 1e-12
    rng = np.random.default_rng(1)
    starts = sorted(rng.integers(0, m - 64, size=5).tolist()) + [0, m - 64]
    vol_e = oracle.element_volumes(w.coords, w.elems)
    for g in range(3):
        sg = oracle.subgrid(w.grid, g)
        for e0 in starts:
            E_sub = w.elems[e0:e0 + 64]
            pe, pc = oracle.candidate_pairs(sg, w.coords, E_sub)
            ob, ov = oracle.pair_blocks(sg, w.coords, E_sub, pe, pc)
            e, cell, b, v = c.export_pair_range(g, e0, 64)
            assert np.array_equal(e.cpu().numpy(), pe + e0)
            assert np.array_equal(cell.cpu().numpy().astype(np.int64), pc)
            scale = vol_e[pe + e0]
            err = np.abs(b.cpu().numpy() - ob).max(axis=(1, 2)) / scale
            assert err.max() <= tol, (g, e0, float(err.max()))
            # volumes at FP64 level in both forms
            assert (np.abs(v.cpu().numpy() - ov) <= 1e-12 * scale).all()


@pytest.mark.parametrize("name,precision", CASES)
def test_row_sums_and_affine_reproduction(name, precision):
    """Sum_j B_ij = int phi_i (the Q1 functions sum to one on every cell), and the
    L2 projection reproduces affine fields."""
    import scipy.sparse as sp
    w = workload(name)
    c = _coupling(w, precision)
    d = 3
    vol = oracle.element_volumes(w.coords, w.elems)
    phi = np.zeros(w.coords.shape[0])
    np.add.at(phi, w.elems.ravel(), np.repeat(vol / (d + 1), d + 1))
    for g in range(3):
        rp, cols, vals = c.export_csr(g)
        rs = np.add.reduceat(vals.cpu().numpy(), rp.cpu().numpy()[:-1]) if vals.numel() else np.zeros(c.n_nodes)
        empty = np.diff(rp.cpu().numpy()) == 0
        rs[empty] = 0.0
        assert np.abs(rs - phi).max() <= (1e-6 if precision == "mixed" else 1e-13) * phi.max()
    import synth
    coef = np.array([0.3, 1.5, -0.7, 2.0])
    dt = np.float32 if precision == "mixed" else np.float64
    fields = [(coef[0] + synth.grid_node_coords(w.grid, g) @ coef[1:] + g).astype(dt) for g in range(3)]
    u_s = c.transfer_velocity([torch.from_numpy(f).cuda() for f in fields])
    got = np.stack([u.cpu().numpy() for u in u_s], axis=1)
    ex = np.stack([coef[0] + w.coords @ coef[1:] + g for g in range(3)], axis=1)
    assert rel_l2(got, ex) <= (1e-6 if precision == "mixed" else 1e-12)


@pytest.mark.parametrize("name", ["leaflet256", "beam512"])
def test_mixed_form_agrees_with_fp64(name):
    """The chosen FP32/FP64 form against the all-FP64 GPU path on the workload's
    Taylor-Green field and nodal forces (both transfers), to 1e-6."""
    w = workload(name)
    c64 = _coupling(w, "fp64")
    c32 = _coupling(w, "mixed")
    u64 = c64.transfer_velocity([torch.from_numpy(f).cuda() for f in w.fields])
    u32 = c32.transfer_velocity([torch.from_numpy(f.astype(np.float32)).cuda() for f in w.fields])
    # compare all components together (the Taylor-Green w component is zero)
    assert rel_l2(np.stack([a.cpu().numpy() for a in u32]), np.stack([b.cpu().numpy() for b in u64])) <= 1e-6
    F = w.force
    f64 = c64.transfer_force([torch.from_numpy(np.ascontiguousarray(F[:, g])).cuda() for g in range(3)])
    f32 = c32.transfer_force([torch.from_numpy(np.ascontiguousarray(F[:, g]).astype(np.float32)).cuda()
                              for g in range(3)])
    for a, b in zip(f32, f64):
        assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= 1e-6  # N(0,1) forces: no zero component


def test_leaflet256_mixed_transfers_against_oracle():
    """The chosen form (fused, FP64 geometry, FP32 fields) on the whole
    952,200-tet leaflet: u_s of the Taylor-Green field and f_f of N(0,1) nodal
    forces in both force modes, against the FP64 oracle's, to 1e-6."""
    import paper_1810_13046_gb300 as l2x
    w = workload("leaflet256")
    oc = oracle_coupling("leaflet256")
    X = torch.from_numpy(w.coords).cuda()
    E = torch.from_numpy(w.elems).cuda()
    fields32 = [f.astype(np.float32) for f in w.fields]
    F32 = w.force.astype(np.float32)
    f_s = [torch.from_numpy(np.ascontiguousarray(F32[:, g])).cuda() for g in range(3)]
    c = l2x.Coupling(w.grid, X, E, path=l2x.FUSED, precision=l2x.MIXED, cg_rtol=1e-9)
    u_s = c.transfer_velocity([torch.from_numpy(f).cuda() for f in fields32])
    ref = oc.transfer_velocity([f.astype(np.float64) for f in fields32])
    got = np.stack([u.cpu().numpy() for u in u_s], axis=1)
    assert rel_l2(got, ref) <= 1e-6
    for mode, fm in (("dual", l2x.DUAL), ("nodal", l2x.NODAL)):
        cm = c if fm == l2x.DUAL else l2x.Coupling(w.grid, X, E, path=l2x.FUSED, precision=l2x.MIXED,
                                                   cg_rtol=1e-9, force_mode=fm)
        f_f = cm.transfer_force(f_s)
        fref = oc.transfer_force(F32.astype(np.float64), mode=mode)
        for g in range(3):
            assert rel_l2(f_f[g].cpu().numpy(), fref[g]) <= 1e-6, (mode, g)
