"""GB300 L2-projection transfer between a staggered Q1 fluid grid and a P1 solid mesh.

A thin ctypes binding of ``libl2xfer.so`` (C ABI declared in ``include/l2xfer.h``):
argument marshalling only, every step of the transfer runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current CUDA stream.

The method is the variational transfer of Sec. 2.3 of the paper (mortar
integrals ``B_ij = ∫ psi_j N_i``, ``S_ij = ∫ phi_j N_i`` with N_i = phi_i
(``S = M_s``) or the dual basis of Eq. (biorth) (S diagonal),
``w_s = S^-1 B v_f``, forces by ``T^T``), assembled by the four steps given
there, plus the Picard-iteration helpers of Sec. 3 (enqueue-only transfers and
the infinity norms of Step 6) and an interface mask on the force input.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

__all__ = ["kernel_launch_count", "PHASES", "StepGraph", "Coupling", "Grid", "VelocityTransfer", "ForceTransfer", "L2XError", "library_path", "load_library",
           "PLAIN", "FUSED", "FP64", "MIXED", "NODAL", "DUAL", "STANDARD_BASIS", "DUAL_BASIS"]

PLAIN, FUSED = 0, 1
FP64, MIXED = 0, 1
NODAL, DUAL = 0, 1
STANDARD_BASIS, DUAL_BASIS = 0, 1   # multiplier space: S = M_s, or the dual basis of Eq. (biorth)
MAT_M = 3


class L2XError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"l2xfer status {status}: {msg}")
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("staggered", ctypes.c_int32), ("ncell", ctypes.c_int32 * 3),
                ("origin", ctypes.c_double * 3), ("h", ctypes.c_double * 3), ("axis", ctypes.c_void_p * 3)]


class _Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n_nodes", ctypes.c_int64),
                ("n_elems", ctypes.c_int64), ("coords", ctypes.c_void_p), ("elems", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("precision", ctypes.c_int32), ("cg_rtol", ctypes.c_double),
                ("cg_max_iter", ctypes.c_int32), ("force_mode", ctypes.c_int32), ("force_scale", ctypes.c_double),
                ("multiplier", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _Info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_grids", ctypes.c_int32), ("path", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("n_nodes", ctypes.c_int64), ("n_elems", ctypes.c_int64),
                ("n_pairs", ctypes.c_int64 * 3), ("n_pairs_total", ctypes.c_int64), ("nnz_B", ctypes.c_int64 * 3),
                ("nnz_M", ctypes.c_int64), ("n_fluid", ctypes.c_int64 * 3), ("nnode", (ctypes.c_int32 * 3) * 3),
                ("cg_iters", ctypes.c_int32), ("reserved", ctypes.c_int32), ("cg_residual", ctypes.c_double),
                ("phase_ms", ctypes.c_double * 8), ("phase_calls", ctypes.c_int64 * 8),
                ("clip_block", ctypes.c_int32), ("pcg_rows_per_block", ctypes.c_int32),
                ("multiplier", ctypes.c_int32), ("pcg_cluster", ctypes.c_int32),
                ("tuned_clip_ms", ctypes.c_double), ("tuned_solve_ms", ctypes.c_double),
                ("pcg_rows_per_block_step", ctypes.c_int32), ("clip_chunk", ctypes.c_int32)]


PHASES = ["pairs", "clip", "rows", "transpose", "mass", "spmv_B", "pcg", "spmv_BT"]


_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libl2xfer.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libl2xfer.so not found at {_build.LIB}; run paper_1810_13046_gb300.build.build()")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "l2x_default_opts": ([ctypes.POINTER(_Opts)], None),
        "l2x_build_coupling": ([ctypes.POINTER(_Grid), ctypes.POINTER(_Mesh), ctypes.POINTER(_Opts), P,
                                ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "l2x_update_geometry": ([P, P, P], ctypes.c_int),
        "l2x_transfer_velocity": ([P, PP, PP, P], ctypes.c_int),
        "l2x_transfer_force": ([P, PP, PP, P], ctypes.c_int),
        "l2x_apply_B": ([P, PP, PP, P], ctypes.c_int),
        "l2x_transfer_force_adjoint": ([P, PP, PP, P], ctypes.c_int),
        "l2x_fma_probe": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P], ctypes.c_int),
        "l2x_fp_selftest": ([ctypes.c_int32, ctypes.c_int64, P, P, P, P], ctypes.c_int),
        "l2x_scan_selftest": ([ctypes.c_int64, P, P, ctypes.c_int32, ctypes.c_int64, P], ctypes.c_int),
        "l2x_transfer_velocity_async": ([P, PP, PP, P], ctypes.c_int),
        "l2x_set_force_mask": ([P, P, P], ctypes.c_int),
        "l2x_transfer_force_async": ([P, PP, PP, P], ctypes.c_int),
        "l2x_sync_status": ([P, P], ctypes.c_int),
        "l2x_picard_norms": ([P, PP, PP, ctypes.c_int32, P, P], ctypes.c_int),
        "l2x_picard_converged": ([P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double), P], ctypes.c_int),
        "l2x_apply_BT": ([P, PP, PP, ctypes.c_double, P], ctypes.c_int),
        "l2x_solve_mass": ([P, PP, PP, P], ctypes.c_int),
        "l2x_query": ([P, ctypes.POINTER(_Info)], ctypes.c_int),
        "l2x_export_pairs": ([P, ctypes.c_int32, P, P, P], ctypes.c_int),
        "l2x_export_pair_blocks": ([P, ctypes.c_int32, P, P, P], ctypes.c_int),
        "l2x_export_csr": ([P, ctypes.c_int32, P, P, P, P], ctypes.c_int),
        "l2x_export_pair_range": ([P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64), P, P, P, P, P], ctypes.c_int),
        "l2x_destroy": ([P], ctypes.c_int),
        "l2x_set_timing": ([P, ctypes.c_int32], ctypes.c_int),
        "l2x_autotune": ([P, P], ctypes.c_int),
        "l2x_set_work_shape": ([P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
        "l2x_set_step_work_shape": ([P, ctypes.c_int32], ctypes.c_int),
        "l2x_set_clip_chunk": ([P, ctypes.c_int32], ctypes.c_int),
        "l2x_graph_create": ([P, P, PP, PP, PP, PP, ctypes.c_double, ctypes.c_int32, P,
                              ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "l2x_graph_create_host": ([P, P, PP, PP, PP, PP, ctypes.c_double, ctypes.c_int32, P,
                                   ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "l2x_graph_io_bytes": ([P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "l2x_graph_launch": ([P, P], ctypes.c_int),
        "l2x_graph_sync_status": ([P, P], ctypes.c_int),
        "l2x_graph_destroy": ([P], ctypes.c_int),
        "l2x_kernel_launch_count": ([], ctypes.c_int64),
        "l2x_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "l2x_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def fma_probe(precision: int, n_blocks: int, iters: int, sink: torch.Tensor):
    """Enqueues the FMA-pipe throughput probe (FP64 for ``FP64``, FP32 for
    ``MIXED``) on the current stream; returns its floating-point operations.
    ``sink``: a CUDA tensor of n_blocks * 256 doubles (or floats)."""
    dt = torch.float64 if precision == FP64 else torch.float32
    if sink.dtype != dt or not sink.is_cuda or sink.numel() < n_blocks * 256:
        raise ValueError("sink must be a CUDA tensor of n_blocks * 256 entries of the probe's type")
    with torch.cuda.device(sink.device):
        _check(load_library().l2x_fma_probe(int(precision), int(n_blocks), int(iters),
                                            ctypes.c_void_p(sink.data_ptr()), _stream_ptr(sink.device)))
    return 2 * 8 * 256 * int(n_blocks) * int(iters)


def fp_selftest(op: int, a: torch.Tensor, b: torch.Tensor | None = None) -> torch.Tensor:
    """Runs one of the clipping kernel's arithmetic helpers (or the CUDA operation
    it stands in for) elementwise on CUDA float64 tensors; see l2x_fp_selftest."""
    a = a.to(torch.float64).contiguous()
    b = (a if b is None else b.to(torch.float64)).contiguous()
    out = torch.empty_like(a)
    with torch.cuda.device(a.device):
        _check(load_library().l2x_fp_selftest(int(op), a.numel(), ctypes.c_void_p(a.data_ptr()),
                                              ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                              _stream_ptr(a.device)))
    return out


def scan_selftest(x: torch.Tensor, missing_first: bool = False, spin_limit: int = 1 << 22):
    """The library's single-pass prefix sum on a CUDA int64 tensor: returns
    (status, out) with out[i] = sum(x[:i]) for i <= len(x); see l2x_scan_selftest."""
    x = x.to(torch.int64).contiguous()
    out = torch.full((x.numel() + 1,), -1, dtype=torch.int64, device=x.device)
    with torch.cuda.device(x.device):
        st = load_library().l2x_scan_selftest(x.numel(), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                              int(bool(missing_first)), int(spin_limit), _stream_ptr(x.device))
    return int(st), out


def kernel_launch_count() -> int:
    """Kernels launched by libl2xfer in this process so far."""
    return int(load_library().l2x_kernel_launch_count())


def _check(status: int):
    if status != 0:
        lib = load_library()
        msg = lib.l2x_last_error().decode() or lib.l2x_status_string(status).decode()
        raise L2XError(status, msg)


def _stream_ptr(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptrs(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = t.data_ptr()
    return arr


@dataclass
class Grid:
    """Base (pressure) grid: ``ncell`` cells of width ``h`` from ``origin``.

    ``staggered=True`` gives one Q1 velocity grid per axis (Sec. 2.2's staggered
    arrangement); ``False`` gives one nodal Q1 grid.  ``axis``: a stretched grid's
    base-node coordinates per axis (ncell[k] + 1 increasing values), or None."""
    dim: int
    ncell: tuple
    h: tuple
    origin: tuple
    staggered: bool
    axis: tuple | None = None


def _as_cgrid(grid):
    """The C struct, and the host arrays its axis pointers refer to (keep both
    alive for the duration of the call)."""
    import numpy as np
    g = _Grid()
    g.dim = int(grid.dim)
    g.staggered = int(bool(grid.staggered))
    keep = []
    axis = getattr(grid, "axis", None)
    for k in range(3):
        g.ncell[k] = int(grid.ncell[k]) if k < grid.dim else 1
        g.origin[k] = float(grid.origin[k]) if k < grid.dim else 0.0
        g.h[k] = float(grid.h[k]) if k < grid.dim else 1.0
        g.axis[k] = None
        if axis is not None and k < grid.dim:
            a = np.ascontiguousarray(axis[k], dtype=np.float64)
            if a.shape != (int(grid.ncell[k]) + 1,):
                raise ValueError("a stretched axis needs ncell[k] + 1 node coordinates")
            keep.append(a)
            g.axis[k] = a.ctypes.data
    return g, keep


class Coupling:
    """B_g (one per velocity grid) and M_s of a P1 mesh in its current configuration.

    ``coords``: (n_nodes, dim) float64 CUDA tensor; ``elems``: (n_elems, dim+1)
    int32 CUDA tensor.  Fields are float64 tensors (``precision=FP64``) or float32
    tensors (``precision=MIXED``)."""

    def __init__(self, grid, coords: torch.Tensor, elems: torch.Tensor, path: int = FUSED,
                 precision: int = FP64, cg_rtol: float | None = None, cg_max_iter: int = 200,
                 force_mode: int = DUAL, force_scale: float = 1.0, multiplier: int = STANDARD_BASIS):
        lib = load_library()
        if not coords.is_cuda or not elems.is_cuda:
            raise ValueError("coords and elems must be CUDA tensors")
        self.device = coords.device
        self.coords = coords.to(torch.float64).contiguous()
        self.elems = elems.to(torch.int32).contiguous()
        self.grid = grid
        self.dim = int(grid.dim)
        self.n_grids = self.dim if grid.staggered else 1
        self.precision = precision
        self.dtype = torch.float32 if precision == MIXED else torch.float64
        opts = _Opts()
        lib.l2x_default_opts(ctypes.byref(opts))
        opts.path = path
        opts.precision = precision
        opts.cg_rtol = cg_rtol if cg_rtol is not None else (1e-13 if precision == FP64 else 1e-9)
        opts.cg_max_iter = cg_max_iter
        opts.force_mode = force_mode
        opts.force_scale = force_scale
        opts.multiplier = multiplier
        self.multiplier = multiplier
        self.force_mask = None
        self.force_mode = force_mode
        self.force_scale = force_scale
        mesh = _Mesh()
        mesh.dim = self.dim
        mesh.n_nodes = self.coords.shape[0]
        mesh.n_elems = self.elems.shape[0]
        mesh.coords = self.coords.data_ptr()
        mesh.elems = self.elems.data_ptr()
        self._grid_c, axis_arrays = _as_cgrid(grid)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.l2x_build_coupling(ctypes.byref(self._grid_c), ctypes.byref(mesh), ctypes.byref(opts),
                                          _stream_ptr(self.device), ctypes.byref(h)))
        self._h = h
        self.n_nodes = int(mesh.n_nodes)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.l2x_destroy(h)
            self._h = None

    # ------------------------------------------------------------------ info
    def info(self) -> dict:
        inf = _Info()
        _check(load_library().l2x_query(self._h, ctypes.byref(inf)))
        G = inf.n_grids
        return dict(dim=inf.dim, n_grids=G, n_nodes=inf.n_nodes, n_elems=inf.n_elems,
                    n_pairs=[inf.n_pairs[g] for g in range(G)], n_pairs_total=inf.n_pairs_total,
                    nnz_B=[inf.nnz_B[g] for g in range(G)], nnz_M=inf.nnz_M,
                    n_fluid=[inf.n_fluid[g] for g in range(G)],
                    nnode=[tuple(inf.nnode[g][k] for k in range(3)) for g in range(G)],
                    cg_iters=inf.cg_iters, cg_residual=inf.cg_residual,
                    phase_ms={p: inf.phase_ms[i] for i, p in enumerate(PHASES)},
                    phase_calls={p: inf.phase_calls[i] for i, p in enumerate(PHASES)},
                    clip_block=inf.clip_block, pcg_rows_per_block=inf.pcg_rows_per_block,
                    multiplier=inf.multiplier, pcg_cluster=inf.pcg_cluster, tuned_clip_ms=inf.tuned_clip_ms,
                    tuned_solve_ms=inf.tuned_solve_ms, pcg_rows_per_block_step=inf.pcg_rows_per_block_step,
                    clip_chunk=inf.clip_chunk)

    def autotune(self):
        """Pick work-chunk sizes by timing candidates on this coupling."""
        with torch.cuda.device(self.device):
            _check(load_library().l2x_autotune(self._h, _stream_ptr(self.device)))
        i = self.info()
        return dict(clip_block=i["clip_block"], clip_chunk=i["clip_chunk"], pcg_rows_per_block=i["pcg_rows_per_block"],
                    pcg_cluster=i["pcg_cluster"], pcg_rows_per_block_step=i["pcg_rows_per_block_step"],
                    clip_ms=i["tuned_clip_ms"], solve_ms=i["tuned_solve_ms"])

    def set_work_shape(self, clip_block: int = 128, pcg_rows_per_block: int = 64, pcg_cluster: int = 0,
                       pcg_rows_per_block_step: int | None = None, clip_chunk: int | None = None):
        """Set the work shape explicitly (what :meth:`autotune` picks).  The combined
        solve of captured steps takes ``pcg_rows_per_block_step``, or
        ``pcg_rows_per_block`` when it is None; ``clip_chunk`` (blocks' worth of
        pairs per work-queue fetch of the clip kernel) is left as it is when None."""
        lib = load_library()
        _check(lib.l2x_set_work_shape(self._h, int(clip_block), int(pcg_rows_per_block), int(pcg_cluster)))
        if pcg_rows_per_block_step is not None:
            _check(lib.l2x_set_step_work_shape(self._h, int(pcg_rows_per_block_step)))
        if clip_chunk is not None:
            _check(lib.l2x_set_clip_chunk(self._h, int(clip_chunk)))

    def set_timing(self, enable: bool = True):
        """CUDA-event timing of the library's phases (totals in info()['phase_ms'])."""
        _check(load_library().l2x_set_timing(self._h, int(bool(enable))))

    def fluid_sizes(self):
        return self.info()["n_fluid"]

    # ------------------------------------------------------------------ geometry
    def update_geometry(self, coords: torch.Tensor):
        c = coords.to(device=self.device, dtype=torch.float64).contiguous()
        if c.shape != self.coords.shape:
            raise ValueError("update_geometry needs the same number of nodes")
        with torch.cuda.device(self.device):
            _check(load_library().l2x_update_geometry(self._h, ctypes.c_void_p(c.data_ptr()),
                                                      _stream_ptr(self.device)))
        self.coords = c

    # ------------------------------------------------------------------ apply
    def _solid(self):
        return [torch.empty(self.n_nodes, dtype=self.dtype, device=self.device) for _ in range(self.n_grids)]

    def _fields(self, xs, n):
        xs = list(xs)
        if len(xs) != self.n_grids:
            raise ValueError(f"expected {self.n_grids} arrays")
        out = []
        for x, m in zip(xs, n):
            if x.dtype != self.dtype or not x.is_cuda or x.numel() != m:
                raise ValueError(f"field must be a CUDA {self.dtype} tensor with {m} entries")
            out.append(x.contiguous())
        return out

    def transfer_velocity(self, u_f, out=None):
        """u_s[g] = S^-1 B_g u_f[g] for every velocity grid g (S = M_s, or diagonal
        for the dual multiplier basis)."""
        u_f = self._fields(u_f, self.fluid_sizes())
        u_s = out if out is not None else self._solid()
        with torch.cuda.device(self.device):
            _check(load_library().l2x_transfer_velocity(self._h, _ptrs(u_f), _ptrs(u_s), _stream_ptr(self.device)))
        return u_s

    def transfer_force(self, f_s, f_f=None):
        """f_f[g] += s B_g^T S^-1 f_s[g] (DUAL) or s B_g^T f_s[g] (NODAL); returns f_f."""
        f_s = self._fields(f_s, [self.n_nodes] * self.n_grids)
        if f_f is None:
            f_f = [torch.zeros(n, dtype=self.dtype, device=self.device) for n in self.fluid_sizes()]
        with torch.cuda.device(self.device):
            _check(load_library().l2x_transfer_force(self._h, _ptrs(f_s), _ptrs(f_f), _stream_ptr(self.device)))
        return f_f

    def apply_B(self, x_f, out=None):
        x_f = self._fields(x_f, self.fluid_sizes())
        y = out if out is not None else self._solid()
        with torch.cuda.device(self.device):
            _check(load_library().l2x_apply_B(self._h, _ptrs(x_f), _ptrs(y), _stream_ptr(self.device)))
        return y

    def apply_BT(self, z_s, f_f=None, scale: float = 1.0):
        z_s = self._fields(z_s, [self.n_nodes] * self.n_grids)
        if f_f is None:
            f_f = [torch.zeros(n, dtype=self.dtype, device=self.device) for n in self.fluid_sizes()]
        with torch.cuda.device(self.device):
            _check(load_library().l2x_apply_BT(self._h, _ptrs(z_s), _ptrs(f_f), float(scale), _stream_ptr(self.device)))
        return f_f

    def transfer_force_adjoint(self, g_f, out=None):
        """g_s[g] = s m ⊙ S^-1 B_g g_f[g] (DUAL) or s m ⊙ B_g g_f[g] (NODAL): the
        transpose of :meth:`transfer_force` (m the interface mask, s the scale)."""
        g_f = self._fields(g_f, self.fluid_sizes())
        g_s = out if out is not None else self._solid()
        with torch.cuda.device(self.device):
            _check(load_library().l2x_transfer_force_adjoint(self._h, _ptrs(g_f), _ptrs(g_s),
                                                             _stream_ptr(self.device)))
        return g_s

    def solve_mass(self, y_s, out=None):
        y_s = self._fields(y_s, [self.n_nodes] * self.n_grids)
        w = out if out is not None else self._solid()
        with torch.cuda.device(self.device):
            _check(load_library().l2x_solve_mass(self._h, _ptrs(y_s), _ptrs(w), _stream_ptr(self.device)))
        return w

    # ------------------------------------------------------------------ interface restriction
    def set_force_mask(self, mask):
        """Restrict the force input to the nodes where ``mask`` (bool/uint8 tensor of
        n_nodes) is set; ``None`` removes the restriction."""
        if mask is None:
            self.force_mask = None
            ptr = None
        else:
            m = mask.to(device=self.device, dtype=torch.uint8).contiguous()
            if m.numel() != self.n_nodes:
                raise ValueError("mask needs one entry per solid node")
            self.force_mask = m
            ptr = ctypes.c_void_p(m.data_ptr())
        with torch.cuda.device(self.device):
            _check(load_library().l2x_set_force_mask(self._h, ptr, _stream_ptr(self.device)))

    # ------------------------------------------------------------------ Picard iterations
    def transfer_velocity_async(self, u_f, u_s):
        """Enqueue-only velocity transfer (no host synchronisation; capturable).
        Solver status is read by :meth:`sync_status`."""
        with torch.cuda.device(self.device):
            _check(load_library().l2x_transfer_velocity_async(self._h, _ptrs(u_f), _ptrs(u_s),
                                                              _stream_ptr(self.device)))
        return u_s

    def transfer_force_async(self, f_s, f_f):
        """Enqueue-only force transfer (accumulates into f_f)."""
        with torch.cuda.device(self.device):
            _check(load_library().l2x_transfer_force_async(self._h, _ptrs(f_s), _ptrs(f_f),
                                                           _stream_ptr(self.device)))
        return f_f

    def sync_status(self):
        """Wait for the stream and raise on a recorded error of enqueued calls."""
        with torch.cuda.device(self.device):
            _check(load_library().l2x_sync_status(self._h, _stream_ptr(self.device)))

    def picard_norms(self, f_new, f_prev, copy: bool = True, out=None):
        """Device tensor [max|f_new - f_prev|, max|f_new|] over all components
        (Step 6's infinity norms); f_prev <- f_new when ``copy``."""
        norms = out if out is not None else torch.empty(2, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _check(load_library().l2x_picard_norms(self._h, _ptrs(f_new), _ptrs(f_prev), int(bool(copy)),
                                                   ctypes.c_void_p(norms.data_ptr()), _stream_ptr(self.device)))
        return norms

    @staticmethod
    def picard_converged(norms, eps_abs: float, eps_rel: float, f0_norm: float):
        """Eqs. (AC)/(RC) on device norms: returns (converged, (norm_diff, norm_new))."""
        conv = ctypes.c_int32()
        hn = (ctypes.c_double * 2)()
        with torch.cuda.device(norms.device):
            _check(load_library().l2x_picard_converged(ctypes.c_void_p(norms.data_ptr()), float(eps_abs),
                                                       float(eps_rel), float(f0_norm), ctypes.byref(conv), hn,
                                                       _stream_ptr(norms.device)))
        return bool(conv.value), (hn[0], hn[1])

    # ------------------------------------------------------------------ captured steps
    def capture_step(self, coords_src, u_f, u_s, f_s, f_f, margin: float = 1.5, zero_force: bool = True,
                     stream=None):
        """A CUDA graph that re-assembles the coupling for the positions in
        ``coords_src`` and runs both transfers; see :class:`StepGraph`."""
        return StepGraph(self, coords_src, u_f, u_s, f_s, f_f, margin, zero_force, stream)

    def capture_step_host(self, coords_h, u_f, u_s, f_s, f_f, margin: float = 1.5, zero_force: bool = True,
                          stream=None):
        """The captured step with page-locked CPU tensors as its inputs and outputs
        (``coords_h`` float64 n_nodes x dim; u_f, f_f per grid over its fluid nodes;
        u_s, f_s per grid over the solid nodes; fields in the coupling's dtype): every
        launch copies them in and out as part of the graph, of u_f and f_f the box of
        fluid nodes the mesh can touch (see l2x_graph_create_host: with zero_force, f_f
        outside the box is zeroed once, here)."""
        fl = self.fluid_sizes()
        want = [(coords_h, torch.float64, self.n_nodes * self.dim, "coords_h")]
        for g in range(self.n_grids):
            want += [(u_f[g], self.dtype, fl[g], "u_f"), (f_f[g], self.dtype, fl[g], "f_f"),
                     (u_s[g], self.dtype, self.n_nodes, "u_s"), (f_s[g], self.dtype, self.n_nodes, "f_s")]
        for t, dt, numel, what in want:
            if t.device.type != "cpu" or not t.is_pinned() or not t.is_contiguous() or t.dtype != dt \
                    or t.numel() != numel:
                raise ValueError(f"{what}: expected a contiguous page-locked CPU tensor of {numel} {dt}")
        return StepGraph(self, coords_h, u_f, u_s, f_s, f_f, margin, zero_force, stream, host=True)

    # ------------------------------------------------------------------ exports (tests)
    def export_pairs(self, g: int):
        n = self.info()["n_pairs"][g]
        e = torch.empty(n, dtype=torch.int32, device=self.device)
        c = torch.empty(n, dtype=torch.int32, device=self.device)
        _check(load_library().l2x_export_pairs(self._h, g, ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                               _stream_ptr(self.device)))
        return e, c

    def export_pair_blocks(self, g: int):
        n = self.info()["n_pairs"][g]
        d = self.dim
        b = torch.empty((n, d + 1, 1 << d), dtype=torch.float64, device=self.device)
        v = torch.empty(n, dtype=torch.float64, device=self.device)
        _check(load_library().l2x_export_pair_blocks(self._h, g, ctypes.c_void_p(b.data_ptr()),
                                                     ctypes.c_void_p(v.data_ptr()), _stream_ptr(self.device)))
        return b, v

    def export_pair_range(self, g: int, e_first: int, n_elems: int):
        """Pairs, blocks and volumes of the elements [e_first, e_first + n_elems) on grid g."""
        lib = load_library()
        p0, npairs = ctypes.c_int64(0), ctypes.c_int64(0)
        st = _stream_ptr(self.device)
        _check(lib.l2x_export_pair_range(self._h, g, e_first, n_elems, ctypes.byref(p0), ctypes.byref(npairs),
                                         None, None, None, None, st))
        n = npairs.value
        d = self.dim
        e = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        c = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        b = torch.empty((max(n, 1), d + 1, 1 << d), dtype=torch.float64, device=self.device)
        v = torch.empty(max(n, 1), dtype=torch.float64, device=self.device)
        _check(lib.l2x_export_pair_range(self._h, g, e_first, n_elems, None, None, ctypes.c_void_p(e.data_ptr()),
                                         ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                         ctypes.c_void_p(v.data_ptr()), st))
        return e[:n], c[:n], b[:n], v[:n]

    def export_csr(self, which: int):
        """(row_ptr int64, cols int32, vals float64) of B_which (0..n_grids-1) or M_s (which=3)."""
        inf = self.info()
        nnz = inf["nnz_M"] if which == MAT_M else inf["nnz_B"][which]
        rp = torch.empty(self.n_nodes + 1, dtype=torch.int64, device=self.device)
        cols = torch.empty(max(nnz, 1), dtype=torch.int32, device=self.device)
        vals = torch.empty(max(nnz, 1), dtype=torch.float64, device=self.device)
        _check(load_library().l2x_export_csr(self._h, which, ctypes.c_void_p(rp.data_ptr()),
                                             ctypes.c_void_p(cols.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                             _stream_ptr(self.device)))
        return rp, cols[:nnz], vals[:nnz]


class StepGraph:
    """One time step of a (multi-body) coupling captured as a CUDA graph.

    Every :meth:`launch` copies the node positions from ``coords_src``, rebuilds
    B_g, B_g^T and M_s and runs the velocity and force transfers into the arrays
    given at capture time, without host synchronisation.  :meth:`status` waits
    and raises :class:`L2XError` if the last replay overflowed the capacities
    (create a new graph with a larger margin) or CG did not converge."""

    def __init__(self, c: Coupling, coords_src, u_f, u_s, f_s, f_f, margin, zero_force, stream, host=False):
        lib = load_library()
        self.c = c
        self.stream = stream if stream is not None else torch.cuda.Stream(device=c.device)
        # keep the buffers alive as long as the graph
        self.buffers = (coords_src, list(u_f), list(u_s), list(f_s), list(f_f))
        g = ctypes.c_void_p()
        torch.cuda.current_stream(c.device).synchronize()
        create = lib.l2x_graph_create_host if host else lib.l2x_graph_create
        with torch.cuda.device(c.device):
            _check(create(c._h, ctypes.c_void_p(coords_src.data_ptr()), _ptrs(u_f), _ptrs(u_s),
                          _ptrs(f_s), _ptrs(f_f), float(margin), int(bool(zero_force)),
                          ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(g)))
        self._g = g

    def launch(self):
        """Replay one step, ordered after the work already queued on the current
        stream (e.g. the copy of new positions into coords_src) and before
        anything queued on it afterwards."""
        cur = torch.cuda.current_stream(self.c.device)
        self.stream.wait_stream(cur)
        _check(load_library().l2x_graph_launch(self._g, ctypes.c_void_p(self.stream.cuda_stream)))
        cur.wait_stream(self.stream)

    def status(self):
        _check(load_library().l2x_graph_sync_status(self._g, ctypes.c_void_p(self.stream.cuda_stream)))

    def io_bytes(self):
        """(bytes copied host to device, device to host) per replay of a host-array graph."""
        h2d, d2h = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(load_library().l2x_graph_io_bytes(self._g, ctypes.byref(h2d), ctypes.byref(d2h)))
        return h2d.value, d2h.value

    def __del__(self):
        g = getattr(self, "_g", None)
        if g is not None and g.value and _lib is not None:
            _lib.l2x_graph_destroy(g)
            self._g = None


# ---------------------------------------------------------------------- autograd

class VelocityTransfer(torch.autograd.Function):
    """u_s = S^-1 B u_f per grid; backward: grad_u_f = B^T S^-1 grad_u_s (the exact adjoint)."""

    @staticmethod
    def forward(ctx, coupling: Coupling, *u_f):
        ctx.coupling = coupling
        return tuple(coupling.transfer_velocity([u.detach() for u in u_f]))

    @staticmethod
    def backward(ctx, *grad_u_s):
        c = ctx.coupling
        gs = [(g if g is not None else torch.zeros(c.n_nodes, dtype=c.dtype, device=c.device)).contiguous()
              for g in grad_u_s]
        z = c.solve_mass(gs)
        gf = c.apply_BT(z, scale=1.0)
        return (None, *gf)


class ForceTransfer(torch.autograd.Function):
    """f_f = s B^T S^-1 (m ⊙ f_s) (DUAL) or s B^T (m ⊙ f_s) (NODAL) per grid, m the
    interface mask (all ones unless set); backward applies the adjoint
    s m ⊙ S^-1 B (DUAL) or s m ⊙ B (NODAL) to grad_f_f."""

    @staticmethod
    def forward(ctx, coupling: Coupling, *f_s):
        ctx.coupling = coupling
        return tuple(coupling.transfer_force([f.detach() for f in f_s]))

    @staticmethod
    def backward(ctx, *grad_f_f):
        c = ctx.coupling
        gf = [(g if g is not None else torch.zeros(n, dtype=c.dtype, device=c.device)).contiguous()
              for g, n in zip(grad_f_f, c.fluid_sizes())]
        return (None, *c.transfer_force_adjoint(gf))
