"""Plain FP64 CPU oracle of the L2-projection fluid <-> solid transfer (Sec. 2.3).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  It shares no code with the
CUDA path.

* ``l2x_oracle.c`` (compiled by :func:`build`) does steps (I)-(III) of the
  assembly recipe of Sec. 2.3: candidate pairs, clipping, quadrature.
* This module does step (IV) (sparse assembly by summing duplicate entries), the
  P1 mass matrix (the "S = M_s" case of the mortar integrals, with the P1 mass
  matrix of Sec. 2.1 "Spatial Discretization"), the solve ``S w = B v`` of the
  algebraic transfer and the transpose force transfer ``f = s * T^T r``.
* With ``multiplier="dual"`` the multiplier space is spanned by the dual basis
  of Eq. (biorth) (the "pseudo" L2-projection of Sec. 2.3): B is assembled from
  the dual weights and S is diagonal.

Readings of the paper taken here (each is a stated choice, not paper text):
* one Q1 space per staggered velocity grid; grid g has nodes at ``o_g + i*h``
  along axis g and at cell centres along the other axes;
* the force input of the DUAL mode is an integrated residual r, so
  ``T^T r = B^T M^{-1} r``; the NODAL mode takes nodal force coefficients and
  returns ``B^T f``;
* a solid element must lie inside the cells covered by every Q1 grid;
* the dual basis is built element by element: on element E the function dual
  to the hat function of its vertex a is mu_a = (d+2) lambda_a - 1, and the
  global dual function of node i is the sum of these over the elements around
  i.  Then int_E mu_a lambda_b = delta_ab |E|/(d+1), which is Eq. (biorth) with
  (mu_i, 1) = sum_{E ni i} |E|/(d+1), so S = diag(int phi_i).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lib = None

EOUTOFGRID = 4
EDEGENERATE = 5


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (no contraction into FMA)."""
    src = os.path.join(_HERE, "l2x_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.orc_count_pairs.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_int64, P, P, P, P]
        lib.orc_count_pairs.restype = ctypes.c_int
        lib.orc_emit_pairs.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_int64, P, P, P, P, P]
        lib.orc_emit_pairs.restype = None
        lib.orc_pair_blocks.argtypes = [ctypes.c_int, P, P, P, P, P, P, ctypes.c_int64, P, P, P, P,
                                        ctypes.c_int]
        lib.orc_pair_blocks.restype = ctypes.c_int
        lib.orc_pair_blocks_counted.argtypes = lib.orc_pair_blocks.argtypes + [P]
        lib.orc_pair_blocks_counted.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------- grids

@dataclass
class SubGrid:
    """One Q1 grid: ``ncell`` cells of width ``h`` from ``origin`` or, on a
    stretched grid, cells between the node coordinates ``axis[k]``."""
    dim: int
    ncell: np.ndarray   # int64[3]
    origin: np.ndarray  # float64[3]
    h: np.ndarray       # float64[3]
    axis: list | None = None  # stretched: per axis the ncell[k] + 1 node coordinates

    @property
    def nnode(self):
        return self.ncell[: self.dim] + 1

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.nnode))

    def cell_frame(self, k: int, i: int):
        """(lower corner, width) of cell i along axis k."""
        if self.axis is not None:
            return float(self.axis[k][i]), float(self.axis[k][i + 1] - self.axis[k][i])
        return float(self.origin[k] + i * self.h[k]), float(self.h[k])

    def _axis_ptrs(self):
        if self.axis is None:
            return None, None
        keep = [np.ascontiguousarray(a, dtype=np.float64) for a in self.axis]
        arr = (ctypes.c_void_p * 3)()
        for k, a in enumerate(keep):
            arr[k] = a.ctypes.data
        keep.append(arr)
        return ctypes.cast(arr, ctypes.c_void_p), keep


def subgrid(grid, g: int) -> SubGrid:
    """Velocity grid g of a base grid (attributes dim, ncell, h, origin, staggered,
    and ``axis`` for a stretched grid).

    Staggered: along axis g the nodes are the base grid nodes, along the other
    axes they are the base cell centres (midpoints of consecutive base nodes on a
    stretched grid), so those axes have one cell fewer.
    """
    d = grid.dim
    nc = np.ones(3, dtype=np.int64)
    o = np.zeros(3)
    h = np.ones(3)
    base_axis = getattr(grid, "axis", None)
    axis = [] if base_axis is not None else None
    for k in range(d):
        h[k] = grid.h[k]
        shifted = grid.staggered and k != g
        if shifted:
            nc[k] = grid.ncell[k] - 1
            o[k] = grid.origin[k] + 0.5 * grid.h[k]
        else:
            nc[k] = grid.ncell[k]
            o[k] = grid.origin[k]
        if axis is not None:
            x = np.asarray(base_axis[k], dtype=np.float64)
            if x.shape != (grid.ncell[k] + 1,) or not np.all(np.diff(x) > 0):
                raise OracleError("a stretched axis needs ncell+1 strictly increasing node coordinates")
            axis.append(0.5 * (x[:-1] + x[1:]) if shifted else x.copy())
            o[k] = axis[k][0]
    return SubGrid(d, nc, o, h, axis)


def n_grids(grid) -> int:
    return grid.dim if grid.staggered else 1


# ----------------------------------------------------------------------------- (I)

def candidate_pairs(sg: SubGrid, X: np.ndarray, E: np.ndarray):
    """Candidate (element, cell) pairs in element-major, cell-lexicographic order."""
    lib = _load()
    d = sg.dim
    X = np.ascontiguousarray(X, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.int32)
    m = E.shape[0]
    counts = np.zeros(m, dtype=np.int64)
    bad = np.zeros(1, dtype=np.int64)
    ax, keep = sg._axis_ptrs()
    st = lib.orc_count_pairs(d, _ptr(sg.ncell), _ptr(sg.origin), _ptr(sg.h), ax, m, _ptr(X), _ptr(E),
                             _ptr(counts), _ptr(bad))
    if st == EOUTOFGRID:
        raise OracleError(f"element {int(bad[0])} leaves the grid")
    offsets = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    n = int(offsets[-1])
    pe = np.zeros(n, dtype=np.int32)
    pc = np.zeros(n, dtype=np.int64)
    lib.orc_emit_pairs(d, _ptr(sg.ncell), _ptr(sg.origin), _ptr(sg.h), ax, m, _ptr(X), _ptr(E),
                       _ptr(offsets), _ptr(pe), _ptr(pc))
    return pe, pc


# ----------------------------------------------------------------------------- (II)+(III)

# categories of the operation tallies of steps (II)-(III), in the order of the C code
OP_CATEGORIES = ("frame", "clip", "volume", "bary", "quad")


def pair_blocks(sg: SubGrid, X, E, pe, pc, nthreads: int = 1, ops: dict | None = None):
    """Local blocks B^loc[p, a, b] = int_{E cap C} lambda_a psi_b and vol(E cap C).

    With a dict ``ops``, the floating-point operations the C code executed for
    these pairs are added into it by category (:data:`OP_CATEGORIES`)."""
    lib = _load()
    d = sg.dim
    X = np.ascontiguousarray(X, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.int32)
    pe = np.ascontiguousarray(pe, dtype=np.int32)
    pc = np.ascontiguousarray(pc, dtype=np.int64)
    n = pe.shape[0]
    blocks = np.zeros((n, d + 1, 1 << d))
    vols = np.zeros(n)
    ax, keep = sg._axis_ptrs()
    tally = np.zeros(len(OP_CATEGORIES), dtype=np.uint64)
    st = lib.orc_pair_blocks_counted(d, _ptr(sg.ncell), _ptr(sg.origin), _ptr(sg.h), ax, _ptr(X), _ptr(E), n,
                                     _ptr(pe), _ptr(pc), _ptr(blocks), _ptr(vols), int(nthreads), _ptr(tally))
    if ops is not None:
        for name, v in zip(OP_CATEGORIES, tally):
            ops[name] = ops.get(name, 0) + int(v)
    if st == EDEGENERATE:
        raise OracleError("degenerate element")
    if st != 0:
        raise OracleError(f"oracle status {st}")
    return blocks, vols


def corner_nodes(sg: SubGrid, pc: np.ndarray) -> np.ndarray:
    """Fluid node index of every corner b of every cell: (n_pairs, 2^d)."""
    d = sg.dim
    nc, nn = sg.ncell, sg.nnode
    ci = [pc % nc[0], (pc // nc[0]) % nc[1]]
    if d == 3:
        ci.append(pc // (nc[0] * nc[1]))
    out = np.zeros((pc.shape[0], 1 << d), dtype=np.int64)
    for b in range(1 << d):
        idx = [ci[k] + ((b >> k) & 1) for k in range(d)]
        if d == 2:
            out[:, b] = idx[0] + nn[0] * idx[1]
        else:
            out[:, b] = idx[0] + nn[0] * (idx[1] + nn[1] * idx[2])
    return out


# ----------------------------------------------------------------------------- (IV)

def dual_blocks(blocks: np.ndarray) -> np.ndarray:
    """int_{E cap C} mu_a psi_b for the element dual basis mu_a = (d+2) lambda_a - 1.

    The barycentrics sum to one, so int_{E cap C} psi_b = sum_a' int lambda_a' psi_b
    and the dual integral is (d+2) * block[a][b] - sum_a' block[a'][b].
    """
    d = blocks.shape[1] - 1
    return (d + 2) * blocks - blocks.sum(axis=1, keepdims=True)


def assemble_B(sg: SubGrid, X, E, nthreads: int = 1, return_pairs: bool = False,
               multiplier: str = "standard", ops: dict | None = None):
    """Mixed coupling matrix B (n_solid x n_fluid) of one Q1 grid, Eq. of the mortar integrals.

    B_ij = int N_fsi,i psi_j with N_fsi,i = phi_i (``multiplier="standard"``) or
    the dual function of node i (``"dual"``).  Entries of pairs whose
    intersection volume is exactly zero are left out.
    """
    if multiplier not in ("standard", "dual"):
        raise ValueError(multiplier)
    pe, pc = candidate_pairs(sg, X, E)
    blocks, vols = pair_blocks(sg, X, E, pe, pc, nthreads, ops)
    d = sg.dim
    keep = vols > 0.0
    w = dual_blocks(blocks[keep]) if multiplier == "dual" else blocks[keep]
    rows = np.repeat(E[pe[keep]].astype(np.int64)[:, :, None], 1 << d, axis=2)
    cols = np.repeat(corner_nodes(sg, pc[keep])[:, None, :], d + 1, axis=1)
    B = sp.coo_matrix((w.ravel(), (rows.ravel(), cols.ravel())),
                      shape=(X.shape[0], sg.n_nodes)).tocsr()
    B.sum_duplicates()
    B.sort_indices()
    if return_pairs:
        return B, (pe, pc, blocks, vols)
    return B


def element_volumes(X, E) -> np.ndarray:
    d = X.shape[1]
    J = np.stack([X[E[:, a]] - X[E[:, 0]] for a in range(1, d + 1)], axis=1)
    return np.abs(np.linalg.det(J)) / (2.0 if d == 2 else 6.0)


def mass_matrix(X, E):
    """P1 mass matrix M_ij = int phi_i phi_j: element block |E|(1+delta_ab)/((d+1)(d+2))."""
    d = X.shape[1]
    vol = element_volumes(X, E)
    if np.any(vol == 0.0):
        raise OracleError("degenerate element")
    na = d + 1
    loc = (np.ones((na, na)) + np.eye(na)) / ((d + 1) * (d + 2))
    vals = vol[:, None, None] * loc[None]
    rows = np.repeat(E[:, :, None], na, axis=2)
    cols = np.repeat(E[:, None, :], na, axis=1)
    M = sp.coo_matrix((vals.ravel(), (rows.ravel().astype(np.int64), cols.ravel().astype(np.int64))),
                      shape=(X.shape[0], X.shape[0])).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return M


def lumped_mass(X, E):
    """S of the dual multiplier space: diag(int phi_i) = diag(sum_{E ni i} |E|/(d+1))."""
    d = X.shape[1]
    vol = element_volumes(X, E)
    if np.any(vol == 0.0):
        raise OracleError("degenerate element")
    diag = np.zeros(X.shape[0])
    for a in range(d + 1):
        np.add.at(diag, E[:, a], vol / (d + 1))
    return sp.diags(diag, format="csr")


def solve_mass(M, Y: np.ndarray, rtol: float = 1e-15, max_iter: int = 10000, method: str = "auto"):
    """Solve M W = Y column by column.

    Direct methods where they are cheap (dense Cholesky for n <= 4000, sparse LU
    for n <= 300000); plain conjugate gradients without preconditioning to
    ||r|| <= rtol ||b|| beyond that (P1 mass matrices are well conditioned).
    ``method`` ("dense", "lu" or "cg") forces one of the three.
    """
    if method not in ("auto", "dense", "lu", "cg"):
        raise ValueError(method)
    Y = np.asarray(Y, dtype=np.float64)
    one = Y.ndim == 1
    Y2 = Y[:, None] if one else Y
    n = M.shape[0]
    if method == "auto":
        method = "dense" if n <= 4000 else ("lu" if n <= 300000 else "cg")
    if method == "dense":
        c = scipy.linalg.cho_factor(M.toarray())
        W = scipy.linalg.cho_solve(c, Y2)
    elif method == "lu":
        lu = scipy.sparse.linalg.splu(M.tocsc())
        W = lu.solve(np.ascontiguousarray(Y2))
    else:
        W = np.zeros_like(Y2)
        for j in range(Y2.shape[1]):
            b = Y2[:, j]
            x = np.zeros(n)
            r = b.copy()
            p = r.copy()
            rr = r @ r
            bn = np.sqrt(b @ b)
            for _ in range(max_iter):
                if np.sqrt(rr) <= rtol * bn:
                    break
                q = M @ p
                alpha = rr / (p @ q)
                x += alpha * p
                r -= alpha * q
                rr_new = r @ r
                p = r + (rr_new / rr) * p
                rr = rr_new
            W[:, j] = x
    return W[:, 0] if one else W


class Coupling:
    """B_g for every velocity grid and S for one mesh in its current configuration.

    ``multiplier="standard"``: S = M_s (multipliers in V_s); ``"dual"``: the dual
    basis of Eq. (biorth), S = diag(int phi_i).  ``self.M`` holds S.
    ``self.ops`` holds the operation tallies of steps (II)-(III) over all grids.
    """

    def __init__(self, grid, X, E, nthreads: int = 1, multiplier: str = "standard"):
        self.ops = {}
        self.grid = grid
        self.multiplier = multiplier
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.E = np.ascontiguousarray(E, dtype=np.int32)
        self.sub = [subgrid(grid, g) for g in range(n_grids(grid))]
        self.B = []
        self.pairs = []
        for sg in self.sub:
            B, pr = assemble_B(sg, self.X, self.E, nthreads, return_pairs=True, multiplier=multiplier,
                               ops=self.ops)
            self.B.append(B)
            self.pairs.append(pr)
        self.M = lumped_mass(self.X, self.E) if multiplier == "dual" else mass_matrix(self.X, self.E)

    def solve_S(self, Y):
        """S^{-1} Y: a division by the diagonal for the dual basis, else :func:`solve_mass`."""
        if self.multiplier == "dual":
            Y = np.asarray(Y, dtype=np.float64)
            dg = self.M.diagonal()
            return Y / (dg if Y.ndim == 1 else dg[:, None])
        return solve_mass(self.M, Y)

    def transfer_velocity(self, fields):
        """w_g = S^{-1} B_g v_g for every grid g  ->  (n_solid, n_grids)."""
        Y = np.stack([self.B[g] @ np.asarray(fields[g], dtype=np.float64)
                      for g in range(len(self.B))], axis=1)
        return self.solve_S(Y)

    def transfer_force(self, F, mode: str = "nodal", scale: float = 1.0, mask=None):
        """Fluid force per grid: s * B_g^T S^{-1} r_g (dual) or s * B_g^T f_g (nodal).

        ``mask`` (one flag per solid node) restricts the input to the interface:
        entries of nodes outside it count as zero (Sec. 4's plate passes only the
        forces of its top and bottom edges)."""
        F = np.asarray(F, dtype=np.float64)
        if F.ndim == 1:
            F = F[:, None]
        if mask is not None:
            F = np.where(np.asarray(mask, dtype=bool)[:, None], F, 0.0)
        Z = self.solve_S(F) if mode == "dual" else F
        return [scale * (self.B[g].T @ Z[:, g]) for g in range(len(self.B))]

    def dense_T(self, g: int):
        """Dense transfer operator T_g = S^{-1} B_g (small instances only)."""
        return self.solve_S(self.B[g].toarray())


# ----------------------------------------------------------------------------- Picard iteration (Sec. 3)

def picard_norms(f_new, f_prev):
    """Step 6: (max |f_new - f_prev|, max |f_new|) over all components and nodes."""
    a = np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in f_new])
    b = np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in f_prev])
    return float(np.max(np.abs(a - b))), float(np.max(np.abs(a)))


def picard_converged(d_norm: float, eps_abs: float, eps_rel: float, f0_norm: float) -> bool:
    """Eq. (AC) or Eq. (RC); the norm of the first iteration's force is f0_norm
    (infinity norm, a reading: the paper leaves that norm unnamed)."""
    return d_norm < eps_abs or (f0_norm > 0.0 and d_norm / f0_norm < eps_rel)


def picard_time_step(C: "Coupling", v_f0, solid, fluid, eps_abs: float, eps_rel: float, max_iter: int = 50,
                     scale: float = 1.0):
    """One time step of the segregated FSI algorithm of Sec. 3 on a fixed T.

    Step 1 w = T v (velocity transfer); Steps 2-3 ``f = solid(w)`` (the caller's
    solid solve, returning the reaction force); Step 4 f~ = s T^T f; Step 5
    ``v = fluid(f~)`` (the caller's fluid solve); Step 6 the infinity-norm tests.
    Returns (v, w, f, iterations, history of (||f_l - f_{l-1}||, ||f_l||)).
    The force before the first iteration is taken as zero (a reading).
    """
    v = [np.asarray(x, dtype=np.float64) for x in v_f0]
    f_prev = None
    f0 = None
    hist = []
    for it in range(1, max_iter + 1):
        w = C.transfer_velocity(v)
        f = np.asarray(solid(w), dtype=np.float64)
        ft = C.transfer_force(f, mode="dual", scale=scale)
        v = [np.asarray(x, dtype=np.float64) for x in fluid(ft)]
        cur = [f[:, g] for g in range(f.shape[1])]
        prev = f_prev if f_prev is not None else [np.zeros_like(c) for c in cur]
        dn, fn = picard_norms(cur, prev)
        hist.append((dn, fn))
        if f0 is None:
            f0 = fn
        f_prev = cur
        if it > 1 and picard_converged(dn, eps_abs, eps_rel, f0):
            return v, w, f, it, hist
    return v, w, f, max_iter, hist
