"""The single-cluster Jacobi-PCG (search direction in distributed shared memory,
cluster barriers) against the oracle, forced through l2x_set_work_shape: the
velocity and dual force transfers at every cluster size, in both precisions,
per call and inside a captured step."""
import numpy as np
import pytest

from _helpers import gpu_coupling, oracle_coupling, rel_l2, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _l2x():
    import paper_1810_13046_gb300 as l2x
    return l2x


@pytest.mark.parametrize("name", ["disk2d", "beam32", "beam128"])
@pytest.mark.parametrize("cluster", [4, 8, 16])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cluster_pcg_transfers(name, cluster, precision):
    l2x = _l2x()
    w = workload(name)
    mixed = precision == "mixed"
    c = gpu_coupling(w, precision=l2x.MIXED if mixed else l2x.FP64, cg_rtol=1e-9 if mixed else 1e-14)
    c.set_work_shape(128, 64, cluster)
    assert c.info()["pcg_cluster"] == cluster
    oc = oracle_coupling(name)
    dt = np.float32 if mixed else np.float64
    tol = 1e-6 if mixed else 1e-12
    u_s = c.transfer_velocity([torch.from_numpy(f.astype(dt)).cuda() for f in w.fields])
    ref = oc.transfer_velocity([f.astype(dt).astype(np.float64) for f in w.fields])
    assert rel_l2(np.stack([u.cpu().numpy() for u in u_s], axis=1), ref) <= tol
    assert c.info()["cg_residual"] <= (1e-9 if mixed else 1e-14)
    F = w.force.astype(dt)
    f_f = c.transfer_force([torch.from_numpy(np.ascontiguousarray(F[:, g])).cuda() for g in range(F.shape[1])])
    fref = oc.transfer_force(F.astype(np.float64), mode="dual")
    for g in range(len(fref)):
        assert rel_l2(f_f[g].cpu().numpy(), fref[g]) <= tol
    # the enqueue-only form and a captured step use the same solver
    us2 = [torch.zeros_like(u) for u in u_s]
    c.transfer_velocity_async([torch.from_numpy(f.astype(dt)).cuda() for f in w.fields], us2)
    c.sync_status()
    assert rel_l2(torch.stack(us2).cpu().numpy(), torch.stack(u_s).cpu().numpy()) <= tol


def test_cluster_pcg_in_a_step_graph_matches_grid_pcg():
    l2x = _l2x()
    w = workload("beam128")
    res = {}
    for shape in [(128, 64, 0), (128, 64, 16)]:
        c = gpu_coupling(w, precision=l2x.MIXED, cg_rtol=1e-9)
        c.set_work_shape(*shape)
        u_f = [torch.from_numpy(f.astype(np.float32)).cuda() for f in w.fields]
        f_s = [torch.from_numpy(np.ascontiguousarray(w.force[:, g].astype(np.float32))).cuda() for g in range(3)]
        u_s = [torch.zeros(c.n_nodes, dtype=torch.float32, device="cuda") for _ in range(3)]
        f_f = [torch.zeros(n, dtype=torch.float32, device="cuda") for n in c.fluid_sizes()]
        X = torch.from_numpy(w.coords).cuda()
        g = c.capture_step(X, u_f, u_s, f_s, f_f, margin=1.2)
        for _ in range(3):
            g.launch()
        g.status()
        res[shape[2]] = (torch.stack(u_s).cpu().numpy(), [x.cpu().numpy() for x in f_f])
    assert rel_l2(res[16][0], res[0][0]) <= 1e-6
    for a, b in zip(res[16][1], res[0][1]):
        assert rel_l2(a, b) <= 1e-6


def test_work_shape_is_validated():
    l2x = _l2x()
    w = workload("beam16")
    c = gpu_coupling(w)
    with pytest.raises(l2x.L2XError):
        c.set_work_shape(100, 64, 0)
    with pytest.raises(l2x.L2XError):
        c.set_work_shape(128, 0, 0)
    with pytest.raises(l2x.L2XError):
        c.set_work_shape(128, 64, 17)
    with pytest.raises(l2x.L2XError):
        c.set_work_shape(128, 64, 0, 0)
    with pytest.raises(l2x.L2XError):
        c.set_work_shape(128, 64, 0, 8192)


def test_step_work_shape_is_honoured_and_does_not_change_the_result():
    """The combined solve of a captured step at 32 and at 1024 rows per block
    (set apart from the per-call solve's 64) gives the same transfers."""
    l2x = _l2x()
    w = workload("beam32")
    res = {}
    for rpbs in (32, 1024):
        c = gpu_coupling(w, precision=l2x.MIXED, cg_rtol=1e-9)
        c.set_work_shape(128, 64, 0, rpbs)
        i = c.info()
        assert (i["pcg_rows_per_block"], i["pcg_rows_per_block_step"]) == (64, rpbs)
        u_f = [torch.from_numpy(f.astype(np.float32)).cuda() for f in w.fields]
        f_s = [torch.from_numpy(np.ascontiguousarray(w.force[:, g].astype(np.float32))).cuda() for g in range(3)]
        u_s = [torch.zeros(c.n_nodes, dtype=torch.float32, device="cuda") for _ in range(3)]
        f_f = [torch.zeros(n, dtype=torch.float32, device="cuda") for n in c.fluid_sizes()]
        g = c.capture_step(torch.from_numpy(w.coords).cuda(), u_f, u_s, f_s, f_f, margin=1.2)
        g.launch()
        g.status()
        res[rpbs] = (torch.stack(u_s).cpu().numpy(), [x.cpu().numpy() for x in f_f])
    assert rel_l2(res[32][0], res[1024][0]) <= 1e-6
    for a, b in zip(res[32][1], res[1024][1]):
        assert rel_l2(a, b) <= 1e-6
