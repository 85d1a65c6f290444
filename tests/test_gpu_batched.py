"""Batched moving bodies: one mesh made of many bodies of uneven size, re-assembled
and transferred every time step by one replay of a captured CUDA graph.

The graph's results must equal a fresh assembly on the same positions (same
kernels: to 1e-12 in FP64, 1e-6 in the mixed form), the oracle on every body and
on the whole mesh,
and overflowing the captured capacities must be reported, not faulted."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(n_bodies=6, n_cells=64, seed=3, n_steps=10):
    grid, bodies, E, nr, er = synth.batch_workload(n_bodies, n_cells, 300, 6000, seed)
    fields = [synth.taylor_green(synth.grid_node_coords(grid, g), g) for g in range(3)]
    return grid, bodies, E, nr, er, fields, n_steps


def _coupling(grid, X, E, precision):
    import paper_1810_13046_gb300 as l2x
    prec = l2x.MIXED if precision == "mixed" else l2x.FP64
    return l2x.Coupling(grid, torch.from_numpy(X).cuda(), torch.from_numpy(E).cuda(), path=l2x.FUSED,
                        precision=prec, cg_rtol=1e-9 if precision == "mixed" else 1e-14)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_graph_matches_fresh_assembly_and_oracle(precision):
    grid, bodies, E, nr, er, fields, n_steps = _setup()
    dt = torch.float32 if precision == "mixed" else torch.float64
    X0 = synth.batch_coords(bodies, 0, n_steps)
    c = _coupling(grid, X0, E, precision)
    n = X0.shape[0]
    rng = np.random.default_rng(5)
    F = rng.standard_normal((n, 3))
    u_f = [torch.from_numpy(f).cuda().to(dt) for f in fields]
    f_s = [torch.from_numpy(np.ascontiguousarray(F[:, g])).cuda().to(dt) for g in range(3)]
    u_s = [torch.zeros(n, dtype=dt, device="cuda") for _ in range(3)]
    f_f = [torch.zeros(m, dtype=dt, device="cuda") for m in c.fluid_sizes()]
    src = torch.from_numpy(X0).cuda()
    graph = c.capture_step(src, u_f, u_s, f_s, f_f, margin=1.5)
    tol = 1e-6 if precision == "mixed" else 1e-12
    for step in (1, 2, 3):
        Xt = synth.batch_coords(bodies, step, n_steps)
        src.copy_(torch.from_numpy(Xt).cuda())
        graph.launch()
        graph.status()
        ref = _coupling(grid, Xt, E, precision)
        ur = ref.transfer_velocity(u_f)
        fr = ref.transfer_force(f_s)
        assert rel_l2(torch.stack(u_s).cpu().numpy(), torch.stack(ur).cpu().numpy()) <= tol
        for a, b in zip(f_f, fr):
            assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= tol
    # the oracle: every body alone (its rows of B and M_s involve only its own
    # elements) for u_s, and the whole mesh for the fluid forces, where bodies
    # that share fluid nodes add up
    src = [f.astype(np.float32 if precision == "mixed" else np.float64).astype(np.float64) for f in fields]
    got = torch.stack(u_s).cpu().numpy().T
    for k in range(len(bodies)):
        n0, n1 = nr[k]
        e0, e1 = er[k]
        ok = oracle.Coupling(grid, Xt[n0:n1], E[e0:e1] - n0, nthreads=8)
        assert rel_l2(got[n0:n1], ok.transfer_velocity(src)) <= tol, k
    oall = oracle.Coupling(grid, Xt, E, nthreads=8)
    Fin = F.astype(np.float32).astype(np.float64) if precision == "mixed" else F
    fref = oall.transfer_force(Fin, mode="dual")
    for g in range(3):
        assert rel_l2(f_f[g].cpu().numpy(), fref[g]) <= tol


def test_step_graph_reports_capacity_overflow():
    import paper_1810_13046_gb300 as l2x
    grid, bodies, E, nr, er, fields, n_steps = _setup()
    X0 = synth.batch_coords(bodies, 0, n_steps)
    c = _coupling(grid, X0, E, "fp64")
    n = X0.shape[0]
    u_f = [torch.from_numpy(f).cuda() for f in fields]
    f_s = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(3)]
    u_s = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(3)]
    f_f = [torch.zeros(m, dtype=torch.float64, device="cuda") for m in c.fluid_sizes()]
    src = torch.from_numpy(X0).cuda()
    graph = c.capture_step(src, u_f, u_s, f_s, f_f, margin=1.0)
    # enlarge every body by 60 % about its centre: many more candidate pairs
    Xb = X0.copy()
    for (a, b) in nr:
        ctr = Xb[a:b].mean(axis=0)
        Xb[a:b] = ctr + 1.6 * (Xb[a:b] - ctr)
    src.copy_(torch.from_numpy(Xb).cuda())
    graph.launch()
    with pytest.raises(l2x.L2XError) as ei:
        graph.status()
    assert ei.value.status == 3  # L2X_ECAPACITY
    # the original positions still replay fine
    src.copy_(torch.from_numpy(X0).cuda())
    graph.launch()
    graph.status()


def test_step_graph_reports_a_mesh_leaving_its_node_box():
    """The B^T rows of a captured step cover the touched fluid nodes at capture,
    padded by the capacity margin: a translated mesh that leaves that box is
    reported as L2X_ECAPACITY, and the captured positions replay fine again."""
    import paper_1810_13046_gb300 as l2x
    import synth as sy
    w = sy.workload("beam32")
    c = l2x.Coupling(w.grid, torch.from_numpy(w.coords).cuda(), torch.from_numpy(w.elems).cuda())
    n = w.coords.shape[0]
    u_f = [torch.from_numpy(f).cuda() for f in w.fields]
    f_s = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(3)]
    u_s = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(3)]
    f_f = [torch.zeros(m, dtype=torch.float64, device="cuda") for m in c.fluid_sizes()]
    src = torch.from_numpy(w.coords).cuda()
    n_pairs0 = c.info()["n_pairs_total"]
    graph = c.capture_step(src, u_f, u_s, f_s, f_f, margin=1.3)
    # a shift of 0.25 (8 cells on the 32^3 grid; the box is padded by about 6
    # nodes) keeps the beam inside the grid and within the pair capacity, but
    # moves it out of the padded box
    src.copy_(torch.from_numpy(w.coords + np.array([0.25, 0.0, 0.0])).cuda())
    graph.launch()
    with pytest.raises(l2x.L2XError) as ei:
        graph.status()
    assert ei.value.status == 3
    assert c.info()["n_pairs_total"] <= 1.3 * n_pairs0   # the pairs fitted: the box was the limit
    src.copy_(torch.from_numpy(w.coords).cuda())
    graph.launch()
    graph.status()
    ref = c.transfer_velocity(u_f)
    assert rel_l2(torch.stack(u_s).cpu().numpy(), torch.stack(ref).cpu().numpy()) <= 1e-12


def test_older_graph_is_refused_after_a_new_capture_or_a_rebuild():
    """A second capture or an update_geometry may move the buffers a captured step
    uses: launching the older graph then fails on the host (L2X_EINVAL), and the
    newest graph replays correctly."""
    import paper_1810_13046_gb300 as l2x
    import synth as sy
    w = sy.workload("beam16")
    c = l2x.Coupling(w.grid, torch.from_numpy(w.coords).cuda(), torch.from_numpy(w.elems).cuda())
    n = w.coords.shape[0]
    u_f = [torch.from_numpy(f).cuda() for f in w.fields]
    f_s = [torch.from_numpy(np.ascontiguousarray(w.force[:, g])).cuda() for g in range(3)]
    u_s = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(3)]
    f_f = [torch.zeros(m, dtype=torch.float64, device="cuda") for m in c.fluid_sizes()]
    src = torch.from_numpy(w.coords).cuda()
    g1 = c.capture_step(src, u_f, u_s, f_s, f_f, margin=1.2)
    g1.launch()
    g1.status()
    g2 = c.capture_step(src, u_f, u_s, f_s, f_f, margin=2.0)
    with pytest.raises(l2x.L2XError) as ei:
        g1.launch()
    assert ei.value.status == 1
    for x in u_s:
        x.zero_()
    g2.launch()
    g2.status()
    ref = l2x.Coupling(w.grid, src, torch.from_numpy(w.elems).cuda()).transfer_velocity(u_f)
    assert rel_l2(torch.stack(u_s).cpu().numpy(), torch.stack(ref).cpu().numpy()) <= 1e-12
    c.update_geometry(src)
    with pytest.raises(l2x.L2XError) as ei:
        g2.launch()
    assert ei.value.status == 1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_graph_in_2d_matches_fresh_assembly(precision):
    """A captured step on the 2-D disk (one nodal grid: one transpose, on the
    main branch of the graph) equals a fresh assembly at moved positions."""
    import paper_1810_13046_gb300 as l2x
    import synth as sy
    w = sy.workload("disk2d")
    mixed = precision == "mixed"
    dt = torch.float32 if mixed else torch.float64
    kw = dict(precision=l2x.MIXED if mixed else l2x.FP64, cg_rtol=1e-9 if mixed else 1e-13)
    E = torch.from_numpy(w.elems).cuda()
    c = l2x.Coupling(w.grid, torch.from_numpy(w.coords).cuda(), E, **kw)
    n = w.coords.shape[0]
    u_f = [torch.from_numpy(w.fields[0]).cuda().to(dt)]
    f_s = [torch.from_numpy(np.ascontiguousarray(w.force[:, 0])).cuda().to(dt)]
    u_s = [torch.zeros(n, dtype=dt, device="cuda")]
    f_f = [torch.zeros(c.fluid_sizes()[0], dtype=dt, device="cuda")]
    src = torch.from_numpy(w.coords).cuda()
    graph = c.capture_step(src, u_f, u_s, f_s, f_f, margin=1.5)
    X1 = w.coords + np.array([0.013, -0.007])
    src.copy_(torch.from_numpy(X1).cuda())
    graph.launch()
    graph.status()
    ref = l2x.Coupling(w.grid, torch.from_numpy(X1).cuda(), E, **kw)
    ur = ref.transfer_velocity(u_f)
    fr = ref.transfer_force(f_s)
    tol = 1e-6 if mixed else 1e-12
    assert rel_l2(u_s[0].cpu().numpy(), ur[0].cpu().numpy()) <= tol
    assert rel_l2(f_f[0].cpu().numpy(), fr[0].cpu().numpy()) <= tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_host_buffer_graph_matches_the_device_buffer_graph(precision):
    """l2x_graph_create_host: the same step with page-locked host arrays in and
    out (the copies are graph nodes) gives the results of the device-array graph
    on the same positions, step after step."""
    grid, bodies, E, nr, er, fields, n_steps = _setup(n_bodies=4, seed=8)
    dt = torch.float32 if precision == "mixed" else torch.float64
    X0 = synth.batch_coords(bodies, 0, n_steps)
    cd = _coupling(grid, X0, E, precision)
    ch = _coupling(grid, X0, E, precision)
    n = X0.shape[0]
    rng = np.random.default_rng(9)
    F = rng.standard_normal((n, 3))
    u_f = [torch.from_numpy(f).to(dt) for f in fields]
    f_s = [torch.from_numpy(np.ascontiguousarray(F[:, g])).to(dt) for g in range(3)]
    # device-array graph
    src = torch.from_numpy(X0).cuda()
    du_f = [u.cuda() for u in u_f]
    df_s = [f.cuda() for f in f_s]
    du_s = [torch.zeros(n, dtype=dt, device="cuda") for _ in range(3)]
    df_f = [torch.zeros(m, dtype=dt, device="cuda") for m in cd.fluid_sizes()]
    gd = cd.capture_step(src, du_f, du_s, df_s, df_f, margin=1.5)
    # host-array graph
    hsrc = torch.from_numpy(X0.copy()).pin_memory()
    hu_f = [u.pin_memory() for u in u_f]
    hf_s = [f.pin_memory() for f in f_s]
    hu_s = [torch.full((n,), float("nan"), dtype=dt).pin_memory() for _ in range(3)]
    hf_f = [torch.full((m,), float("nan"), dtype=dt).pin_memory() for m in ch.fluid_sizes()]
    gh = ch.capture_step_host(hsrc, hu_f, hu_s, hf_s, hf_f, margin=1.5)
    tol = 1e-6 if precision == "mixed" else 1e-12
    for step in (1, 2, 3):
        Xt = synth.batch_coords(bodies, step, n_steps)
        src.copy_(torch.from_numpy(Xt).cuda())
        hsrc.copy_(torch.from_numpy(Xt))
        gd.launch()
        gd.status()
        gh.launch()
        gh.status()
        # norm-wise (u_s of the third grid is zero: the flow has no z-component);
        # every value was copied back (the host arrays started as NaN)
        for a, b in list(zip(hu_s, du_s)) + list(zip(hf_f, df_f)):
            a, b = a.numpy(), b.cpu().numpy()
            assert np.all(np.isfinite(a)), step
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), step


def test_host_buffer_graph_refuses_pageable_memory():
    import ctypes

    import paper_1810_13046_gb300 as l2x
    grid, bodies, E, nr, er, fields, n_steps = _setup(n_bodies=2, seed=4)
    X0 = synth.batch_coords(bodies, 0, n_steps)
    c = _coupling(grid, X0, E, "fp64")
    n = X0.shape[0]
    pageable = torch.from_numpy(X0.copy())  # not page-locked
    pin_n = [torch.zeros(n, dtype=torch.float64).pin_memory() for _ in range(3)]
    pin_f = [torch.zeros(m, dtype=torch.float64).pin_memory() for m in c.fluid_sizes()]
    lib = l2x.load_library()
    g = ctypes.c_void_p()
    stream = torch.cuda.Stream()
    st = lib.l2x_graph_create_host(c._h, ctypes.c_void_p(pageable.data_ptr()), l2x._ptrs(pin_f), l2x._ptrs(pin_n),
                                   l2x._ptrs(pin_n), l2x._ptrs(pin_f), 1.5, 1, ctypes.c_void_p(stream.cuda_stream),
                                   ctypes.byref(g))
    assert st == 1 and not g.value  # L2X_EINVAL
    assert b"page-locked" in lib.l2x_last_error()
    with pytest.raises(ValueError):
        c.capture_step_host(pageable, pin_f, pin_n, pin_n, pin_f)


def test_host_buffer_graph_accumulates_into_the_host_forces():
    """zero_force off: f_f_host += s B^T ... (the box of touched fluid nodes is
    copied in, added to and copied back), equal to the device-array graph started
    from the same forces; the bytes a replay copies are those of the boxes."""
    grid, bodies, E, nr, er, fields, n_steps = _setup(n_bodies=3, seed=10)
    dt = torch.float64
    X0 = synth.batch_coords(bodies, 0, n_steps)
    cd = _coupling(grid, X0, E, "fp64")
    ch = _coupling(grid, X0, E, "fp64")
    n = X0.shape[0]
    rng = np.random.default_rng(12)
    F = rng.standard_normal((n, 3))
    base = [rng.standard_normal(m) for m in cd.fluid_sizes()]
    src = torch.from_numpy(X0).cuda()
    du_f = [torch.from_numpy(f).cuda() for f in fields]
    df_s = [torch.from_numpy(np.ascontiguousarray(F[:, g])).cuda() for g in range(3)]
    du_s = [torch.zeros(n, dtype=dt, device="cuda") for _ in range(3)]
    df_f = [torch.from_numpy(b.copy()).cuda() for b in base]
    gd = cd.capture_step(src, du_f, du_s, df_s, df_f, margin=1.5, zero_force=False)
    hsrc = torch.from_numpy(X0.copy()).pin_memory()
    hu_f = [torch.from_numpy(f).pin_memory() for f in fields]
    hf_s = [torch.from_numpy(np.ascontiguousarray(F[:, g])).pin_memory() for g in range(3)]
    hu_s = [torch.zeros(n, dtype=dt).pin_memory() for _ in range(3)]
    hf_f = [torch.from_numpy(b.copy()).pin_memory() for b in base]
    gh = ch.capture_step_host(hsrc, hu_f, hu_s, hf_s, hf_f, margin=1.5, zero_force=False)
    for step in (1, 2):
        Xt = synth.batch_coords(bodies, step, n_steps)
        src.copy_(torch.from_numpy(Xt).cuda())
        hsrc.copy_(torch.from_numpy(Xt))
        gd.launch()
        gd.status()
        gh.launch()
        gh.status()
        for a, b in list(zip(hu_s, du_s)) + list(zip(hf_f, df_f)):
            a, b = a.numpy(), b.cpu().numpy()
            assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b), step
    h2d, d2h = gh.io_bytes()
    full = sum(8 * m for m in ch.fluid_sizes())
    assert 0 < d2h - 8 * 3 * n < full  # u_s, then the f_f boxes only
    assert h2d > d2h
    assert gd.io_bytes() == (0, 0)
