"""l2x_solve_mass_noalloc: the Jacobi-PCG solve for callers that cannot allocate
device memory (for example when an outer framework owns the device memory pool),
with its work vectors in a fixed device array of the library.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test first.  The GPU test must pass both alone in a
fresh process and after the other tests: the entry point shares one scratch
array between calls and must not depend on what an earlier call left there.
"""
import ctypes

import numpy as np
import pytest

import paper_1810_13046_gb300 as l2x

MAX_ENTRIES = 131072


def _lib():
    lib = l2x.load_library()
    f = lib.l2x_solve_mass_noalloc
    f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                  ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_double,
                  ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    lib.l2x_noalloc_last_error.restype = ctypes.c_char_p
    return lib


def _ptr_array(ts):
    a = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        a[i] = t.data_ptr() if t is not None else 0
    return a


def test_oversized_problem_is_rejected_before_touching_the_device():
    lib = _lib()
    dummy = ctypes.c_void_p(16)
    ys = (ctypes.c_void_p * 3)(16, 16, 16)
    ws = (ctypes.c_void_p * 3)(16, 16, 16)
    it = ctypes.c_int32(0)
    res = ctypes.c_double(0)
    n = MAX_ENTRIES // 3 + 1
    st = lib.l2x_solve_mass_noalloc(n, dummy, dummy, dummy, 3, ys, ws, 1e-12, 100, None, ctypes.byref(it),
                                    ctypes.byref(res))
    assert st == 3  # L2X_ECAPACITY
    assert b"exceeds the fixed scratch" in lib.l2x_noalloc_last_error()


@pytest.mark.gpu
def test_noalloc_solve_matches_the_allocating_solve_on_two_calls_in_a_row():
    """Two consecutive calls with different right-hand sides agree with
    l2x_solve_mass of a coupling built on the same mesh (FP64, fused path)."""
    import torch

    import synth

    lib = _lib()
    w = synth.workload("beam32")
    X = torch.from_numpy(w.coords).cuda()
    E = torch.from_numpy(w.elems).cuda()
    c = l2x.Coupling(w.grid, X, E, path=l2x.FUSED, precision=l2x.FP64, cg_rtol=1e-13)
    rp, cols, vals = c.export_csr(3)  # M_s
    n = c.n_nodes
    assert 3 * n <= MAX_ENTRIES
    rng = np.random.default_rng(21)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        ys = [torch.from_numpy(rng.standard_normal(n) * (call + 1)).cuda() for _ in range(3)]
        ref = c.solve_mass(ys)
        out = [torch.full((n,), np.nan, dtype=torch.float64, device="cuda") for _ in range(3)]
        it = ctypes.c_int32(0)
        res = ctypes.c_double(0)
        st = lib.l2x_solve_mass_noalloc(n, rp.data_ptr(), cols.data_ptr(), vals.data_ptr(), 3, _ptr_array(ys),
                                        _ptr_array(out), 1e-13, 200, ctypes.c_void_p(stream), ctypes.byref(it),
                                        ctypes.byref(res))
        assert st == 0, lib.l2x_noalloc_last_error()
        assert 0 < it.value <= 200 and res.value <= 1e-13
        for a, b in zip(out, ref):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-12


def _tridiagonal_csr(n):
    """A = tridiag(-1, 4, -1), symmetric positive definite (row sums >= 2)."""
    rows = np.repeat(np.arange(n), 3)
    cols = (rows + np.tile([-1, 0, 1], n))
    vals = np.tile([-1.0, 4.0, -1.0], n)
    keep = (cols >= 0) & (cols < n)
    rows, cols, vals = rows[keep], cols[keep], vals[keep]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr), cols.astype(np.int32), vals


@pytest.mark.gpu
@pytest.mark.parametrize("n_rhs", [1, 2])
def test_noalloc_solve_at_full_capacity_allocates_nothing(n_rhs):
    """n * n_rhs equal to the scratch capacity (the status words at the end of the
    array, the most blocks), against a CPU banded solve; the free device memory
    is the same before and after the call, so the call allocated nothing."""
    import scipy.linalg
    import torch

    lib = _lib()
    n = MAX_ENTRIES // n_rhs
    rp, cols, vals = _tridiagonal_csr(n)
    rng = np.random.default_rng(40 + n_rhs)
    Y = rng.standard_normal((n, n_rhs))
    ab = np.zeros((3, n))
    ab[0, 1:] = -1.0
    ab[1, :] = 4.0
    ab[2, :-1] = -1.0
    ref = scipy.linalg.solve_banded((1, 1), ab, Y)
    d_rp, d_cols, d_vals = (torch.from_numpy(a).cuda() for a in (rp, cols, vals))
    ys = [torch.from_numpy(np.ascontiguousarray(Y[:, k])).cuda() for k in range(n_rhs)]
    out = [torch.full((n,), np.nan, dtype=torch.float64, device="cuda") for _ in range(n_rhs)]
    stream = torch.cuda.current_stream().cuda_stream
    it = ctypes.c_int32(0)
    res = ctypes.c_double(0)

    def call():
        return lib.l2x_solve_mass_noalloc(n, d_rp.data_ptr(), d_cols.data_ptr(), d_vals.data_ptr(), n_rhs,
                                          _ptr_array(ys), _ptr_array(out), 1e-13, 500, ctypes.c_void_p(stream),
                                          ctypes.byref(it), ctypes.byref(res))

    assert call() == 0, lib.l2x_noalloc_last_error()  # the first call on the device loads the module
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for o in out:
        o.fill_(np.nan)
    assert call() == 0, lib.l2x_noalloc_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    for k in range(n_rhs):
        got = out[k].cpu().numpy()
        assert np.linalg.norm(got - ref[:, k]) / np.linalg.norm(ref[:, k]) <= 1e-12


@pytest.mark.gpu
def test_noalloc_solve_refuses_a_capturing_stream():
    """The call synchronises its stream to read the solver status, so it returns
    L2X_EINVAL on a stream that is being captured (nothing is enqueued)."""
    import torch

    lib = _lib()
    n = 64
    rp, cols, vals = _tridiagonal_csr(n)
    d_rp, d_cols, d_vals = (torch.from_numpy(a).cuda() for a in (rp, cols, vals))
    ys = [torch.ones(n, dtype=torch.float64, device="cuda")]
    out = [torch.zeros(n, dtype=torch.float64, device="cuda")]
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        st = lib.l2x_solve_mass_noalloc(n, d_rp.data_ptr(), d_cols.data_ptr(), d_vals.data_ptr(), 1,
                                        _ptr_array(ys), _ptr_array(out), 1e-12, 100,
                                        ctypes.c_void_p(side.cuda_stream), None, None)
        out[0].add_(1.0)  # the capture itself stays valid
    assert st == 1  # L2X_EINVAL
    assert b"capturing" in lib.l2x_noalloc_last_error()
