"""Numerical building blocks of the CUDA path, through the C ABI:

* the clipping kernel's arithmetic helpers against the CUDA operations they
  stand in for (quotient, double -> float conversion, double-float split);
* intersection volumes of sliver pairs (vertices 1e-9 h from cell planes) in
  every form, against the FP64 oracle, with no positive-volume pair dropped;
* the failure status of a mass-matrix solve that misses its tolerance, on the
  per-call, enqueue-only and captured forms;
* the adjoint of the force transfer (the backward of the differentiable force
  transfer) against the oracle and the transpose identity;
* the FMA throughput probe behind the ALU roofline.
Mortar integrals and the algebraic transfer: Sec. 2.3 "Variational Transfer".
"""
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


# ---------------------------------------------------------------- arithmetic helpers

def _ulp(x):
    return np.spacing(np.abs(x))


def test_quotient_matches_division():
    """Two Newton-Raphson steps on an FP32 reciprocal seed, then a * r: within two
    ulps of CUDA's correctly rounded division on random operands with a / b in
    [0, 1] (the clipping kernel's use), exact for a = 0, and the hardware
    division for operands outside the refined range."""
    l2x = _l2x()
    rng = np.random.default_rng(11)
    n = 1 << 20
    b = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-30, 30, n)
    t = rng.random(n)
    t[:64] = 0.0
    t[64:128] = 1.0
    a = t * b
    # outside the refined exponent range: the hardware division
    b[-64:] = 10.0 ** rng.uniform(40, 60, 64)
    a[-64:] = b[-64:] * rng.random(64)
    A, Bt = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    q = l2x.fp_selftest(0, A, Bt).cpu().numpy()
    ref = l2x.fp_selftest(1, A, Bt).cpu().numpy()
    diff = np.abs(q - ref)
    assert np.all(diff <= 2 * _ulp(ref)), float((diff / np.maximum(_ulp(ref), 1e-300)).max())
    assert np.mean(q == ref) >= 0.5
    assert np.array_equal(q[:64], ref[:64]) and np.array_equal(q[-64:], ref[-64:])
    assert np.all(np.abs(q[64:128] - 1.0) <= 2 * np.spacing(1.0))


def test_fast_quotient_of_the_mixed_form():
    """The mixed precision form's crossing parameter: an FP32 quotient and one
    FP64 correction, within 2^-44 of the correctly rounded a / b on operands with
    a / b in [-1, 1] (both crossing formulas), exact for a = 0, to 2^-44 of 1 for a = b; the
    hardware division outside the refined range."""
    l2x = _l2x()
    rng = np.random.default_rng(13)
    n = 1 << 20
    b = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-30, 30, n)
    t = rng.uniform(-1.0, 1.0, n)
    t[:64] = 0.0
    t[64:128] = 1.0
    a = t * b
    b[-64:] = 10.0 ** rng.uniform(40, 60, 64)
    a[-64:] = b[-64:] * rng.random(64)
    A, Bt = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    q = l2x.fp_selftest(6, A, Bt).cpu().numpy()
    ref = l2x.fp_selftest(1, A, Bt).cpu().numpy()
    rel = np.abs(q - ref) / np.maximum(np.abs(ref), 1e-300)
    assert np.all(rel[128:-64] <= 2.0 ** -44), float(rel[128:-64].max())
    assert np.array_equal(q[:64], ref[:64]) and np.array_equal(q[-64:], ref[-64:])
    assert np.all(np.abs(q[64:128] - 1.0) <= 2.0 ** -44)


def test_double_to_float_conversion():
    """Integer-instruction conversion: equal to __double2float_rn away from ties;
    on an exact tie it rounds away from zero; below 2^-126 it gives zero."""
    l2x = _l2x()
    rng = np.random.default_rng(12)
    n = 1 << 20
    x = rng.choice([-1.0, 1.0], n) * rng.uniform(1.0, 2.0, n) * 2.0 ** rng.integers(-120, 120, n)
    low = x.view(np.uint64) & np.uint64(0x1FFFFFFF)
    x = x[low != np.uint64(0x10000000)]  # exact ties are checked below
    X = torch.from_numpy(x).cuda()
    ours = l2x.fp_selftest(2, X).cpu().numpy()
    rn = l2x.fp_selftest(3, X).cpu().numpy()
    assert np.array_equal(ours, rn)
    # exact ties: f + half an ulp of f (f a float), both signs
    f = (rng.uniform(1.0, 2.0, 4096) * 2.0 ** rng.integers(-100, 100, 4096)).astype(np.float32)
    f = f * rng.choice([-1.0, 1.0], 4096).astype(np.float32)
    up = np.nextafter(f, np.where(f > 0, np.float32(np.inf), np.float32(-np.inf)))
    tie = f.astype(np.float64) + 0.5 * (up.astype(np.float64) - f.astype(np.float64))
    got = l2x.fp_selftest(2, torch.from_numpy(tie).cuda()).cpu().numpy()
    assert np.array_equal(got, up.astype(np.float64))
    tiny = np.array([2.0 ** -127, -(2.0 ** -130), 1e-45, 0.0, -0.0])
    got = l2x.fp_selftest(2, torch.from_numpy(tiny).cuda()).cpu().numpy()
    assert np.all(got == 0.0)
    # float -> double by integer instructions is exact
    back = l2x.fp_selftest(5, X).cpu().numpy()
    assert np.array_equal(back, rn)


def test_double_float_split():
    """hi + lo of the split reproduces x to 2^-46 |x| (47 or more bits), with hi
    the rounded float of x."""
    l2x = _l2x()
    rng = np.random.default_rng(13)
    n = 1 << 20
    x = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-25, 5, n)
    x[:8] = [1.0, -1.0, 0.5, 3.0, 1.0 + 2.0 ** -30, 1.0 - 2.0 ** -40, 0.0, 2.0 ** -90]
    X = torch.from_numpy(x).cuda()
    hi = l2x.fp_selftest(2, X).cpu().numpy()
    lo = l2x.fp_selftest(4, X).cpu().numpy()
    assert np.all(np.abs(lo) <= _ulp(hi.astype(np.float32)).astype(np.float64) + 1e-300)
    assert np.all(np.abs((hi + lo) - x) <= 2.0 ** -46 * np.abs(x))


# ---------------------------------------------------------------- sliver pairs

def _sliver_mesh(h, rng):
    """Kuhn tetrahedra of a lattice of spacing h/2 whose nodes sit on the base and
    staggered cell planes, each coordinate then moved by +-(0.5..1) 1e-9 h: every
    element reaches across some cell plane of every velocity grid by 1e-9 h."""
    X, E = synth.beam_mesh(8, 8, 4, (4 * h, 4 * h, 2 * h))
    X = X + 0.5
    X = X + rng.choice([-1.0, 1.0], X.shape) * rng.uniform(0.5, 1.0, X.shape) * 1e-9 * h
    return X, E


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sliver_volumes_match_oracle(precision):
    """|E ∩ C| of every candidate pair to 1e-12 |E| in both forms (the mixed form
    keeps the volumes in double-float); every pair whose oracle volume exceeds
    that bound has a positive volume, so its entries stay in B."""
    l2x = _l2x()
    n = 16
    h = 1.0 / n
    grid = synth.Grid(3, (n, n, n), (h,) * 3, (0.0,) * 3, True)
    X, E = _sliver_mesh(h, np.random.default_rng(14))
    c = l2x.Coupling(grid, torch.from_numpy(X).cuda(), torch.from_numpy(E).cuda(), path=l2x.FUSED,
                     precision=l2x.MIXED if precision == "mixed" else l2x.FP64)
    oc = oracle.Coupling(grid, X, E, nthreads=NTHREADS)
    vol_e = oracle.element_volumes(X, E)
    n_sliver = 0
    for g in range(3):
        e, cell = c.export_pairs(g)
        assert np.array_equal(e.cpu().numpy(), oc.pairs[g][0])
        assert np.array_equal(cell.cpu().numpy().astype(np.int64), oc.pairs[g][1])
        _, v = c.export_pair_blocks(g)
        v = v.cpu().numpy()
        ov = oc.pairs[g][3]
        scale = vol_e[oc.pairs[g][0]]
        assert np.all(np.abs(v - ov) <= 1e-12 * scale)
        kept = ov > 1e-12 * scale
        assert np.all(v[kept] > 0.0)
        n_sliver += int(np.sum(kept & (ov < 1e-6 * scale)))
    assert n_sliver > 100  # the mesh does produce slivers


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_faces_within_ulps_of_cell_planes_match_oracle(precision):
    """Nodes on the base and staggered cell planes, each coordinate then moved by
    -4..4 ulps: element faces lie within rounding of cell faces, where the
    computed inside flags of a cut can split into several runs (repaired by the
    clipping; see the clip kernel).  Pair lists equal the oracle's, volumes
    within 1e-12 |E|, blocks within 1e-12 |E| (FP64) or 1e-6 |E| (mixed)."""
    l2x = _l2x()
    n = 16
    h = 1.0 / n
    grid = synth.Grid(3, (n, n, n), (h,) * 3, (0.0,) * 3, True)
    rng = np.random.default_rng(15)
    X, E = synth.beam_mesh(8, 8, 4, (4 * h, 4 * h, 2 * h))
    X = X + 0.5
    X = X + rng.integers(-4, 5, X.shape) * np.spacing(X)
    c = l2x.Coupling(grid, torch.from_numpy(X).cuda(), torch.from_numpy(E).cuda(), path=l2x.FUSED,
                     precision=l2x.MIXED if precision == "mixed" else l2x.FP64)
    oc = oracle.Coupling(grid, X, E, nthreads=NTHREADS)
    vol_e = oracle.element_volumes(X, E)
    tol_b = 1e-6 if precision == "mixed" else 1e-12
    for g in range(3):
        e, cell = c.export_pairs(g)
        assert np.array_equal(e.cpu().numpy(), oc.pairs[g][0])
        assert np.array_equal(cell.cpu().numpy().astype(np.int64), oc.pairs[g][1])
        b, v = c.export_pair_blocks(g)
        b, v = b.cpu().numpy(), v.cpu().numpy()
        scale = vol_e[oc.pairs[g][0]]
        assert np.all(np.isfinite(b)) and np.all(np.isfinite(v))
        assert np.all(np.abs(v - oc.pairs[g][3]) <= 1e-12 * scale)
        ob = np.asarray(oc.pairs[g][2]).reshape(b.shape)
        assert np.all(np.abs(b - ob) <= tol_b * scale[:, None, None])


# ---------------------------------------------------------------- solver status

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_not_converged_is_reported(precision):
    """A mass-matrix solve capped at one CG iteration misses its tolerance: the
    per-call transfer returns L2X_ENOTCONVERGED, and so do the status reads after
    the enqueue-only transfer and after a captured step."""
    l2x = _l2x()
    w = workload("beam16")
    mixed = precision == "mixed"
    dt = torch.float32 if mixed else torch.float64
    c = gpu_coupling(w, precision=l2x.MIXED if mixed else l2x.FP64, cg_rtol=1e-9 if mixed else 1e-13,
                     cg_max_iter=1)
    u_f = [torch.from_numpy(f).cuda().to(dt) for f in w.fields]
    with pytest.raises(l2x.L2XError) as ei:
        c.transfer_velocity(u_f)
    assert ei.value.status == 6
    u_s = [torch.zeros(c.n_nodes, dtype=dt, device="cuda") for _ in range(3)]
    c.transfer_velocity_async(u_f, u_s)
    with pytest.raises(l2x.L2XError) as ei:
        c.sync_status()
    assert ei.value.status == 6
    c.sync_status()  # the status was cleared by the read
    f_s = [torch.from_numpy(np.ascontiguousarray(w.force[:, g])).cuda().to(dt) for g in range(3)]
    f_f = [torch.zeros(m, dtype=dt, device="cuda") for m in c.fluid_sizes()]
    graph = c.capture_step(torch.from_numpy(w.coords).cuda(), u_f, u_s, f_s, f_f, margin=1.2)
    graph.launch()
    with pytest.raises(l2x.L2XError) as ei:
        graph.status()
    assert ei.value.status == 6
    del graph
    # with enough iterations the same handle converges
    c2 = gpu_coupling(w, precision=l2x.MIXED if mixed else l2x.FP64, cg_rtol=1e-9 if mixed else 1e-13)
    c2.transfer_velocity(u_f)


# ---------------------------------------------------------------- adjoint of the force transfer

@pytest.mark.parametrize("mode", ["dual", "nodal"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("masked", [False, True])
def test_force_adjoint(mode, precision, masked):
    """g_s = s m ⊙ S^-1 B g_f (dual) or s m ⊙ B g_f (nodal) against the oracle,
    and <g_f, F f> = <g_s, f> for the force transfer F."""
    l2x = _l2x()
    w = workload("beam32")
    mixed = precision == "mixed"
    dt = np.float32 if mixed else np.float64
    tol = 1e-6 if mixed else 1e-12
    s = 0.7
    c = gpu_coupling(w, precision=l2x.MIXED if mixed else l2x.FP64, cg_rtol=1e-9 if mixed else 1e-14,
                     force_mode=l2x.DUAL if mode == "dual" else l2x.NODAL, force_scale=s)
    mask = synth.block_face_mask(*synth.BEAM_HEXES["beam32"], axis=2) if masked else None
    if masked:
        c.set_force_mask(torch.from_numpy(mask).cuda())
    oc = oracle.Coupling(w.grid, w.coords, w.elems, nthreads=NTHREADS)
    rng = np.random.default_rng(15)
    g_f = [rng.standard_normal(m).astype(dt) for m in c.fluid_sizes()]
    g_s = c.transfer_force_adjoint([torch.from_numpy(x).cuda() for x in g_f])
    m = mask.astype(np.float64) if masked else 1.0
    for g in range(3):
        y = oc.B[g] @ g_f[g].astype(np.float64)
        ref = s * m * (oc.solve_S(y) if mode == "dual" else y)
        assert rel_l2(g_s[g].cpu().numpy(), ref) <= tol
    f = rng.standard_normal((c.n_nodes, 3)).astype(dt)
    Ff = c.transfer_force([torch.from_numpy(np.ascontiguousarray(f[:, g])).cuda() for g in range(3)])
    lhs = sum(float(np.dot(g_f[g].astype(np.float64), Ff[g].cpu().numpy().astype(np.float64))) for g in range(3))
    rhs = sum(float(np.dot(g_s[g].cpu().numpy().astype(np.float64), f[:, g].astype(np.float64))) for g in range(3))
    scale = sum(np.linalg.norm(g_f[g]) * np.linalg.norm(Ff[g].cpu().numpy()) for g in range(3))
    assert abs(lhs - rhs) <= 10 * tol * scale


# ---------------------------------------------------------------- FMA probe

def test_fma_probe_runs_and_is_deterministic():
    l2x = _l2x()
    for prec, dt in ((l2x.FP64, torch.float64), (l2x.MIXED, torch.float32)):
        sink = torch.zeros(4 * 256, dtype=dt, device="cuda")
        flops = l2x.fma_probe(prec, 4, 100, sink)
        assert flops == 2 * 8 * 256 * 4 * 100
        a = sink.clone()
        l2x.fma_probe(prec, 4, 100, sink)
        assert torch.isfinite(sink).all() and torch.equal(a, sink)
    with pytest.raises(l2x.L2XError):  # an unknown precision is refused by the library
        l2x.fma_probe(7, 4, 100, torch.zeros(4 * 256, dtype=torch.float32, device="cuda"))


# ---------------------------------------------------------------- single-pass scan

@pytest.mark.parametrize("n", [1, 7, 4096, 4097, 3 * 4096 + 5, (1 << 20) + 3])
def test_scan_matches_cumsum(n):
    """The single-pass decoupled look-back scan (pair offsets, CSR row pointers):
    exclusive prefix sums and the total, twice in a row on one workspace
    (each launch leaves it zeroed for the next)."""
    l2x = _l2x()
    rng = np.random.default_rng(n)
    x = rng.integers(0, 1000, n).astype(np.int64)
    want = np.concatenate([[0], np.cumsum(x)])
    for _ in range(2):
        st, out = l2x.scan_selftest(torch.from_numpy(x).cuda())
        assert st == 0
        assert np.array_equal(out.cpu().numpy(), want)


def test_scan_bounded_wait_reports_timeout():
    """A tile whose predecessor never publishes gives up after its poll limit:
    the call returns L2X_ETIMEOUT instead of hanging, and the device and the
    scan keep working afterwards."""
    l2x = _l2x()
    x = torch.ones(3 * 4096 + 5, dtype=torch.int64, device="cuda")
    st, _ = l2x.scan_selftest(x, missing_first=True, spin_limit=20000)
    assert st == 7  # L2X_ETIMEOUT
    st, out = l2x.scan_selftest(x)
    assert st == 0 and int(out[-1]) == x.numel()
