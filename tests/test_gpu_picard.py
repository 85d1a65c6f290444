"""Picard iterations on one assembled coupling (Sec. 3, Steps 1-6) on the CUDA path.

The enqueue-only transfers and the device infinity norms of Step 6 are checked
against the oracle: the norms exactly (maxima are order independent), a whole
Picard time step with a linear model of the solid and fluid solvers against
the oracle's loop (same iteration count, same limit), and the same iteration
captured into a CUDA graph and replayed.
"""
import numpy as np
import pytest

import oracle
from _helpers import NTHREADS, gpu_coupling, rel_l2, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _l2x():
    import paper_1810_13046_gb300 as l2x
    return l2x


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_picard_norms_match_numpy(precision):
    l2x = _l2x()
    w = workload("beam16")
    c = gpu_coupling(w, precision=l2x.MIXED if precision == "mixed" else l2x.FP64)
    dt = torch.float32 if precision == "mixed" else torch.float64
    rng = np.random.default_rng(1)
    n = c.n_nodes
    fn = [rng.standard_normal(n) for _ in range(3)]
    fp = [x + 1e-3 * rng.standard_normal(n) for x in fn]
    fn[2][n // 3] = -7.5            # planted maxima
    fp[1][n - 1] = fn[1][n - 1] + 0.25
    fn_t = [torch.from_numpy(x).to(dt).cuda() for x in fn]
    fp_t = [torch.from_numpy(x).to(dt).cuda() for x in fp]
    ref = oracle.picard_norms([x.cpu().numpy() for x in fn_t], [x.cpu().numpy() for x in fp_t])
    norms = c.picard_norms(fn_t, fp_t, copy=True)
    got = norms.cpu().numpy()
    assert got[0] == ref[0] and got[1] == ref[1]
    for a, b in zip(fn_t, fp_t):
        assert torch.equal(a, b)              # copied
    assert c.picard_norms(fn_t, fp_t, copy=False).cpu().numpy()[0] == 0.0
    conv, hn = l2x.Coupling.picard_converged(norms, 1.01 * ref[0], 0.0, 0.0)      # (AC) holds
    assert conv and hn == (ref[0], ref[1])
    assert not l2x.Coupling.picard_converged(norms, ref[0], 0.0, 0.0)[0]          # strict <
    conv, _ = l2x.Coupling.picard_converged(norms, 0.1, 0.01, ref[1])
    assert conv == oracle.picard_converged(ref[0], 0.1, 0.01, ref[1])
    # NaN makes the norm NaN and the test fail
    fn_t[0][5] = float("nan")
    nn = c.picard_norms(fn_t, fp_t, copy=False)
    assert np.isnan(nn.cpu().numpy()[0])
    assert not l2x.Coupling.picard_converged(nn, 1e30, 1e30, 1.0)[0]


def _linear_model(T_norm2, v0, wt, dt):
    k = 1.0
    beta = 0.8 / T_norm2

    def solid(w):          # Steps 2-3: reaction force of a linear spring to w_target
        return [-k * (wi - ti) for wi, ti in zip(w, wt)]

    def fluid(ft):         # Step 5: a linear "fluid solve"
        return [a + beta * b for a, b in zip(v0, ft)]
    return solid, fluid, k, beta


@pytest.mark.parametrize("multiplier", ["standard", "dual"])
def test_picard_time_step_matches_the_oracle(multiplier):
    """Eager loop: async transfers + device norms, against oracle.picard_time_step."""
    l2x = _l2x()
    w = workload("disk2d_small")
    mult = l2x.DUAL_BASIS if multiplier == "dual" else l2x.STANDARD_BASIS
    c = gpu_coupling(w, cg_rtol=1e-14, multiplier=mult)
    oc = oracle.Coupling(w.grid, w.coords, w.elems, nthreads=NTHREADS, multiplier=multiplier)
    T = oc.dense_T(0)
    lam = np.linalg.norm(T, 2) ** 2
    rng = np.random.default_rng(2)
    v0 = rng.standard_normal(T.shape[1])
    wt = rng.standard_normal(T.shape[0])
    eps_a, eps_r = 1e-12, 1e-13
    # oracle
    solid_o = lambda ws: (-(ws[:, 0] - wt))[:, None]
    fluid_o = lambda ft: [v0 + 0.8 / lam * ft[0]]
    v_ref, w_ref, f_ref, it_ref, hist = oracle.picard_time_step(oc, [v0], solid_o, fluid_o, eps_a, eps_r, 200)
    # GPU
    v0_t, wt_t = [torch.from_numpy(v0).cuda()], [torch.from_numpy(wt).cuda()]
    solid, fluid, _, _ = _linear_model(lam, v0_t, wt_t, torch.float64)
    v = [x.clone() for x in v0_t]
    ws = [torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda")]
    f_prev = [torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda")]
    ff = [torch.zeros(c.fluid_sizes()[0], dtype=torch.float64, device="cuda")]
    f0 = None
    it = 0
    for it in range(1, 201):
        c.transfer_velocity_async(v, ws)                      # Step 1
        f = solid(ws)                                         # Steps 2-3
        for z in ff:
            z.zero_()
        c.transfer_force_async(f, ff)                         # Step 4
        v = fluid(ff)                                         # Step 5
        norms = c.picard_norms(f, f_prev, copy=True)          # Step 6
        conv, (dn, fn) = l2x.Coupling.picard_converged(norms, eps_a, eps_r, f0 if f0 is not None else 0.0)
        if f0 is None:
            f0 = fn
        if it > 1 and conv:
            break
    c.sync_status()
    # both loops stop once the force change is below 1e-12; rounding (and the CG
    # tolerance of the standard space) may move that by one iteration
    assert abs(it - it_ref) <= 1 and it < 200
    assert rel_l2(v[0].cpu().numpy(), v_ref[0]) <= 1e-10
    assert rel_l2(ws[0].cpu().numpy(), w_ref[:, 0]) <= 1e-10


def test_picard_iteration_captured_in_a_cuda_graph():
    """One Picard iteration (both transfers, the linear model, the norms) captured
    with torch.cuda.graph and replayed until Step 6 accepts; the result equals the
    eager loop's (beam16, 3 grids, mixed precision)."""
    l2x = _l2x()
    w = workload("beam16")
    c = gpu_coupling(w, precision=l2x.MIXED, cg_rtol=1e-9)
    dt = torch.float32
    rng = np.random.default_rng(4)
    n, nf = c.n_nodes, c.fluid_sizes()
    v0 = [torch.from_numpy(rng.standard_normal(m)).to(dt).cuda() for m in nf]
    wt = [torch.from_numpy(rng.standard_normal(n)).to(dt).cuda() for _ in range(3)]
    # a safe step: ||T||^2 bounded through the power method on T^T T in FP64 on the oracle
    oc = oracle.Coupling(w.grid, w.coords, w.elems, nthreads=NTHREADS)
    lam = max(np.linalg.norm(oc.dense_T(g), 2) ** 2 for g in range(3))
    beta = 0.5 / lam

    def run(capture):
        v = [x.clone() for x in v0]
        ws = [torch.zeros(n, dtype=dt, device="cuda") for _ in range(3)]
        f = [torch.zeros(n, dtype=dt, device="cuda") for _ in range(3)]
        f_prev = [torch.zeros(n, dtype=dt, device="cuda") for _ in range(3)]
        ff = [torch.zeros(m, dtype=dt, device="cuda") for m in nf]
        norms = torch.zeros(2, dtype=torch.float64, device="cuda")

        def iteration():
            c.transfer_velocity_async(v, ws)
            for a, wi, ti in zip(f, ws, wt):
                torch.sub(wi, ti, out=a)
                a.neg_()
            for z in ff:
                z.zero_()
            c.transfer_force_async(f, ff)
            for vi, v0i, fi in zip(v, v0, ff):
                torch.add(v0i, fi, alpha=beta, out=vi)
            c.picard_norms(f, f_prev, copy=True, out=norms)

        if capture:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                iteration()                      # warm-up outside the graph
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            for x, y in zip(v, v0):
                x.copy_(y)
            for x in f_prev:
                x.zero_()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                iteration()
            step = g.replay
        else:
            step = iteration
        f0 = 0.0
        for it in range(1, 100):
            step()
            conv, (dn, fn) = l2x.Coupling.picard_converged(norms, 1e-5, 1e-6, f0)
            if it == 1:
                f0 = fn
            elif conv:
                break
        c.sync_status()
        return it, torch.stack(v).cpu().numpy(), torch.stack(ws).cpu().numpy()

    it_e, v_e, w_e = run(False)
    it_g, v_g, w_g = run(True)
    assert it_e == it_g and it_e > 2
    assert rel_l2(v_g, v_e) <= 1e-6 and rel_l2(w_g, w_e) <= 1e-6
