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
