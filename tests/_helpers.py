"""Shared helpers for the GPU parity tests (oracle side on the CPU, library side on cuda:0)."""
import functools
import os

import numpy as np
import scipy.sparse as sp

import oracle
import synth

NTHREADS = max(1, min(16, os.cpu_count() or 1))


@functools.lru_cache(maxsize=None)
def workload(name, seed=0):
    return synth.workload(name, seed)


@functools.lru_cache(maxsize=None)
def oracle_coupling(name, seed=0):
    w = workload(name, seed)
    return oracle.Coupling(w.grid, w.coords, w.elems, nthreads=NTHREADS)


def gpu_coupling(w, **kw):
    import torch
    import paper_1810_13046_gb300 as l2x
    X = torch.from_numpy(np.ascontiguousarray(w.coords)).cuda()
    E = torch.from_numpy(np.ascontiguousarray(w.elems)).cuda()
    return l2x.Coupling(w.grid, X, E, **kw)


def csr_from_gpu(c, which, n_cols):
    rp, cols, vals = c.export_csr(which)
    return sp.csr_matrix((vals.cpu().numpy(), cols.cpu().numpy().astype(np.int64), rp.cpu().numpy()),
                         shape=(c.n_nodes, n_cols))


def rel_fro(A, B):
    """||A - B||_F / ||B||_F for sparse or dense matrices (missing entries count as 0)."""
    D = A - B
    if sp.issparse(D):
        num = sp.linalg.norm(D)
        den = sp.linalg.norm(B)
    else:
        num = np.linalg.norm(D)
        den = np.linalg.norm(B)
    return num / den


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def max_row_rel(A, B):
    """max_i max_j |A_ij - B_ij| / max_j |B_ij|  (rows of B that are empty are skipped)."""
    D = (A - B).tocsr()
    B = B.tocsr()
    Dm = np.asarray(abs(D).max(axis=1).todense()).ravel()
    Bm = np.asarray(abs(B).max(axis=1).todense()).ravel()
    keep = Bm > 0
    return float((Dm[keep] / Bm[keep]).max()) if keep.any() else 0.0
