"""Interface-restricted force transfer on the CUDA path against the oracle: the
force input is masked to the top and bottom faces of the beam (the plate of
Sec. 4 passes only the forces of its top and bottom edges)."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import NTHREADS, gpu_coupling, rel_l2, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _l2x():
    import paper_1810_13046_gb300 as l2x
    return l2x


@pytest.mark.parametrize("name", ["beam32", "beam128"])
@pytest.mark.parametrize("multiplier", ["standard", "dual"])
@pytest.mark.parametrize("mode", ["dual", "nodal"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_masked_force_transfer(name, multiplier, mode, precision):
    l2x = _l2x()
    w = workload(name)
    mixed = precision == "mixed"
    mask = synth.block_face_mask(*synth.BEAM_HEXES[name], axis=2)
    c = gpu_coupling(w, precision=l2x.MIXED if mixed else l2x.FP64, cg_rtol=1e-9 if mixed else 1e-14,
                     force_mode=l2x.DUAL if mode == "dual" else l2x.NODAL, force_scale=0.6,
                     multiplier=l2x.DUAL_BASIS if multiplier == "dual" else l2x.STANDARD_BASIS)
    c.set_force_mask(torch.from_numpy(mask).cuda())
    oc = oracle.Coupling(w.grid, w.coords, w.elems, nthreads=NTHREADS, multiplier=multiplier)
    dt = np.float32 if mixed else np.float64
    F = w.force.astype(dt)
    ref = oc.transfer_force(F.astype(np.float64), mode=mode, scale=0.6, mask=mask)
    f_s = [torch.from_numpy(np.ascontiguousarray(F[:, g])).cuda() for g in range(3)]
    got = c.transfer_force(f_s)
    tol = 1e-6 if mixed else 1e-12
    for g in range(3):
        assert rel_l2(got[g].cpu().numpy(), ref[g]) <= tol
    # the enqueue-only form applies the same mask
    ff = [torch.zeros_like(x) for x in got]
    c.transfer_force_async(f_s, ff)
    c.sync_status()
    for a, b in zip(ff, got):
        assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= tol
    # removing the mask restores the unrestricted transfer
    c.set_force_mask(None)
    full = c.transfer_force(f_s)
    ref_full = oc.transfer_force(F.astype(np.float64), mode=mode, scale=0.6)
    for g in range(3):
        assert rel_l2(full[g].cpu().numpy(), ref_full[g]) <= tol


def test_masked_force_autograd_and_step_graph():
    """The backward of the restricted force transfer is s m ⊙ S^-1 B (dense
    oracle), and a step graph captured with the mask set applies it."""
    l2x = _l2x()
    w = workload("beam32")
    mask = synth.block_face_mask(*synth.BEAM_HEXES["beam32"], axis=2)
    c = gpu_coupling(w, cg_rtol=1e-14, force_scale=1.5)
    c.set_force_mask(torch.from_numpy(mask).cuda())
    oc = oracle.Coupling(w.grid, w.coords, w.elems, nthreads=NTHREADS)
    rng = np.random.default_rng(21)
    f = [torch.from_numpy(rng.standard_normal(c.n_nodes)).cuda().requires_grad_(True) for _ in range(3)]
    out = l2x.ForceTransfer.apply(c, *f)
    gf = [torch.from_numpy(rng.standard_normal(n)).cuda() for n in c.fluid_sizes()]
    sum((a * b).sum() for a, b in zip(out, gf)).backward()
    for g in range(3):
        ref = 1.5 * mask * (oc.dense_T(g) @ gf[g].cpu().numpy())
        assert rel_l2(f[g].grad.cpu().numpy(), ref) <= 1e-11
    # captured step with the mask
    X = torch.from_numpy(w.coords).cuda()
    u_f = [torch.from_numpy(x).cuda() for x in w.fields]
    f_s = [torch.from_numpy(np.ascontiguousarray(w.force[:, g])).cuda() for g in range(3)]
    u_s = [torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda") for _ in range(3)]
    f_f = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in c.fluid_sizes()]
    graph = c.capture_step(X.clone(), u_f, u_s, f_s, f_f, margin=1.2)
    graph.launch()
    graph.status()
    ref = oc.transfer_force(w.force, mode="dual", scale=1.5, mask=mask)
    for g in range(3):
        assert rel_l2(f_f[g].cpu().numpy(), ref[g]) <= 1e-12
