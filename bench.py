#!/usr/bin/env python
"""Benchmark of the L2-projection fluid <-> solid transfer on GB300.

One step = the whole hot path of Sec. 2.3 on the current configuration of the
solid: assembly of B_g (3 staggered Q1 grids) and M_s from scratch (candidate
pairs, clipping + quadrature, CSR), the velocity transfer u_s = M_s^-1 B u_f
(3 components) and the dual force transfer f_f = B^T M_s^-1 r (3 components).
The chosen form runs a step as one replay of a captured CUDA graph (new node
positions copied in, no host synchronisation); the per-call form (one library
call per operation) is timed beside it with per-phase CUDA events.

Workload (default, the largest single-GPU configuration): 512 x 512 x 256-cell
staggered grids on [0,1]^2 x [0,0.5] (h = 1/512), a 0.4 x 0.1 x 0.02 beam of
3,993,600 P1 tetrahedra with smoothed random node displacements, a
Taylor-Green velocity field (float32) and N(0,1) nodal forces; synthetic data.
The 48k-tet beam on 128^3 grids, the 952k-tet leaflet on 256^3 grids (with the
differentiable transfer) and the 64 moving bodies on 256^3 grids are reported
as extra keys of the same line.  Each rank (torchrun, N > 1) transfers its own
body: weak scaling, no collective on the data path.

value = candidate pairs per second over whole steps (summed over ranks);
assembly pairs/s and apply ms are reported beside it, together with the plain
FP64 GPU path.  Inputs are resident in HBM; L2 is flushed (256 MB write) before
every timed step.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "L2-transfer assembly pairs/s & apply ms, 1 GB300, fused vs plain at rel≤1e-6"
UNIT = "pairs/s"
WORKLOAD = "beam512"
EXTRA_WORKLOADS = ("beam128", "leaflet256", "batch64")
WORKLOAD_DESCS = {
    "beam128": ("3-D staggered Q1 grids 128^3 cells (h=1/128) on [0,1]^3; rotated beam 0.4x0.1x0.02, "
                "48,000 P1 tets / 10,206 nodes; Taylor-Green u_f (f32); N(0,1) nodal forces"),
    "leaflet256": ("3-D staggered Q1 grids 256^3 cells (h=1/256) on [0,1]^3; rotated spherical-cap leaflet "
                   "0.3x0.3x0.01, 952,200 P1 tets / 213,444 nodes; Taylor-Green u_f (f32); N(0,1) nodal forces"),
    "beam512": ("3-D staggered Q1 grids 512x512x256 cells (h=1/512) on [0,1]^2x[0,0.5]; deformed beam "
                "0.4x0.1x0.02, 3,993,600 P1 tets / 702,027 nodes; Taylor-Green u_f (f32); N(0,1) nodal forces"),
    "beam64s": ("3-D staggered Q1 grids 64^3 cells on [0,1]^3, stretched x = xi + 0.5 sin(2 pi xi)/(2 pi) per axis "
                "(cells 1/128 wide at the body, 3/128 at the walls); the rotated 48,000-tet beam of beam128; "
                "Taylor-Green u_f (f32); N(0,1) nodal forces"),
    "batch64": ("3-D staggered Q1 grids 256^3 cells (h=1/256); 64 moving bodies (beams and plates, seeded poses, "
                "log-uniform 1k-200k tets; 2,234,256 tets / 535,718 nodes in all), rigid motion plus a travelling "
                "wave, 8 configurations of a 200-step motion replayed in turn; B_g, M_s rebuilt every step"),
}
# Elements of the CPU oracle's sample: the slab of tetrahedra nearest one end of
# the body along x, taken as a mesh of its own (about 10 s of single-thread work
# on the 4M-tet beam).
CPU_SAMPLE_ELEMS = 30000
# Elements of the smaller samples whose operation tallies give the extra
# workloads' algorithmic work per pair.
TALLY_SAMPLE_ELEMS = 4000
# DRAM bytes per candidate pair of the clipping kernel (read + write) from one
# capture of its first launch on the 48k-tet beam (716,130 pairs; ncu --metrics
# dram__bytes_read.sum,dram__bytes_write.sum -k regex:clip_fused_kernel -c 1):
# 24.9 MB read + 201.7 MB written.  The traffic grows with the pairs (each pair
# writes its block and volume once), so it scales to a launch by the pair count.
CLIP_DRAM_BYTES_PER_PAIR = 316.4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--plain-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extras", default=",".join(EXTRA_WORKLOADS),
                    help="comma-separated extra workloads reported as keys of the same line ('none': no extras)")
    ap.add_argument("--extra-steps", type=int, default=10)
    ap.add_argument("--work-shape", default=None, metavar="CB,RPB,CL,RPBS[,CC]",
                    help="fix the fused forms' work shape (clip block, PCG rows per block, PCG cluster, rows "
                         "per block of the captured step's combined solve, optionally the clip kernel's "
                         "work-queue chunk) instead of autotuning it; for profiler runs, where the autotuner's "
                         "timings are distorted")
    args = ap.parse_args()
    if args.work_shape is not None:
        try:
            args.work_shape = tuple(int(x) for x in args.work_shape.split(","))
        except ValueError:
            ap.error("--work-shape takes four or five integers")
        if len(args.work_shape) not in (4, 5):
            ap.error("--work-shape takes four or five integers")
    args.extras = [] if args.extras in ("", "none") else args.extras.split(",")
    for x in args.extras:
        if x not in WORKLOAD_DESCS:
            ap.error(f"unknown extra workload {x!r}")
    return args


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device="cuda"):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device="cuda"):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate(step_ms: float, pairs: int, world: int, device="cuda"):
    """Whole-job throughput: every rank transfers its own body (weak scaling, no
    data-path collective); the job's step time is the slowest rank's."""
    t = max_over_ranks(step_ms, world, device)
    total = sum_over_ranks(float(pairs), world, device)
    return t, total, total / (t * 1e-3)


def workload_seed(rank: int) -> int:
    """Each rank draws its own rotation of the beam."""
    return rank


def shard_bodies(sizes, world: int):
    """Greedy balanced partition of bodies (by tetrahedron count) over ranks:
    largest first onto the least-loaded rank.  Returns a list of index lists."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------- oracle legs

def spmv_bytes(c, torch):
    """Algorithmic bytes of one y = B u_f and one f_f += s B^T z over all grids in
    the mixed form (FP32 values, int32 columns, int64 row pointers): every
    matrix entry once, every touched vector entry once, results written once."""
    bB = bT = 0
    n = c.n_nodes
    for g in range(c.n_grids):
        rp, cols, _ = c.export_csr(g)
        nnz = int(cols.numel())
        touched = int(torch.unique(cols).numel())
        bB += (n + 1) * 8 + nnz * 8 + touched * 4 + n * 4
        bT += (touched + 1) * 8 + nnz * 8 + n * 4 + touched * 8
    return bB, bT


def pcg_bytes(c, iters: int, n_rhs: int):
    """Algorithmic bytes of a Jacobi-PCG solve in the mixed form: per iteration
    one product with M_s (FP32 values, int32 columns, int64 row pointers) and the
    vector passes of the Chronopoulos-Gear recurrences (u, w, r, p, s, x, m read
    or written once per right-hand side, FP32)."""
    n, nnz = c.n_nodes, c.info()["nnz_M"]
    return iters * ((n + 1) * 8 + nnz * 8 + 7 * n * n_rhs * 4)


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json copy bandwidth)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def cpu_model():
    """CPU model name from lscpu (Arm hosts have no 'model name' in /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.TimeoutExpired):
        pass
    import platform
    return platform.processor() or platform.machine()


def slab_sample(coords, elems, n_max: int):
    """The n_max elements with the lowest centroid x (a slab at one end of the
    body), or all of them."""
    if elems.shape[0] <= n_max:
        return elems, "the whole mesh"
    cx = coords[elems].mean(axis=1)[:, 0]
    keep = np.sort(np.argpartition(cx, n_max)[:n_max])
    return elems[keep], f"the {n_max} of {elems.shape[0]} tetrahedra with the lowest centroid x (a slab at one end), as a mesh of its own"


def oracle_step(grid, coords, elems, force, nthreads, fields=None):
    """One step of the plain FP64 CPU oracle (assembly + both transfers) on the
    mesh made of ``elems``: the nodes it uses, renumbered (nodes outside it would
    give empty rows of M_s).  Returns the oracle's coupling, u_s, f_f, pairs,
    the assembly and apply seconds, and the operation tallies."""
    import oracle
    used = np.unique(elems)
    if used.size == coords.shape[0]:
        X, E, F = coords, elems, force
    else:
        remap = np.full(coords.shape[0], -1, dtype=np.int64)
        remap[used] = np.arange(used.size)
        X, E, F = coords[used], remap[elems].astype(np.int32), force[used]
    t0 = time.perf_counter()
    oc = oracle.Coupling(grid, X, E, nthreads=nthreads)
    t1 = time.perf_counter()
    us = ff = None
    if fields is not None:
        us = oc.transfer_velocity([f.astype(np.float32).astype(np.float64) for f in fields])
        ff = oc.transfer_force(F.astype(np.float32).astype(np.float64), mode="dual")
    t2 = time.perf_counter()
    npairs = sum(len(p[0]) for p in oc.pairs)
    return oc, us, ff, npairs, t1 - t0, t2 - t1, dict(oc.ops)


def fp64_flops_per_pair(ops: dict, npairs: int):
    """Algorithmic FP64 work of the clipping step per candidate pair: the
    oracle's tallies of the cell frame, the plane-side values and cut points and
    the sub-simplex volumes (the geometry the method keeps in FP64)."""
    return (ops["frame"] + ops["clip"] + ops["volume"]) / max(1, npairs)


def cpu_baseline_leg(grid, coords, elems, force, fields, n_max=CPU_SAMPLE_ELEMS, single=True):
    """The oracle as it stands on a bounded sample of the workload: one step on
    all host cores and, with ``single``, one on a single thread; its operation
    tallies give the algorithmic FP64 work per pair."""
    cores = os.cpu_count() or 1
    sub, what = slab_sample(coords, elems, n_max)
    _, _, _, npairs, tb, ta, ops = oracle_step(grid, coords, sub, force, cores, fields)
    out = {"value": npairs / (tb + ta), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"one full step (assembly + velocity + dual force transfer) on {what}; {npairs} candidate pairs",
           "assembly_s": tb, "apply_s": ta, "nproc": cores, "cpu_model": cpu_model(),
           "fp64_flops_per_pair": fp64_flops_per_pair(ops, npairs),
           "op_tallies_per_pair": {k: v / max(1, npairs) for k, v in ops.items()}}
    if single:
        _, _, _, n1, tb1, ta1, _ = oracle_step(grid, coords, sub, force, 1, fields)
        out["single_thread"] = {"value": n1 / (tb1 + ta1), "unit": UNIT, "cores": 1, "assembly_s": tb1,
                                "apply_s": ta1}
    return out


def reference_arm(args, rank, world):
    """The oracle as it stands, on the host cores: each step the same bounded
    sample of the workload as the CPU baseline (a slab of the body)."""
    if rank != 0:
        return 0
    import synth
    w = synth.workload(args.workload, 0)
    cores = os.cpu_count() or 1
    sub, what = slab_sample(w.coords, w.elems, CPU_SAMPLE_ELEMS)
    for _ in range(args.warmup):
        oracle_step(w.grid, w.coords, sub, w.force, cores, w.fields)
    times, pairs = [], 0
    for _ in range(args.steps):
        _, _, _, npairs, tb, ta, _ = oracle_step(w.grid, w.coords, sub, w.force, cores, w.fields)
        times.append(tb + ta)
        pairs = npairs
    total = sum(times)
    value = pairs * len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload,
                                            "desc": WORKLOAD_DESCS.get(args.workload, args.workload),
                                            "sample": f"{what} per step ({pairs} candidate pairs)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{what} per step, {args.steps} steps", "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def fma_peaks(torch, l2x, dev):
    """FP64 and FP32 FMA-pipe throughput of this GPU (the library's probe kernel,
    CUDA events, best of three launches of about 20 ms), in TFLOP/s."""
    out = {}
    n_blocks = 152 * 8
    stream = torch.cuda.current_stream(dev)
    for name, prec, iters in (("fp64", l2x.FP64, 5000), ("fp32", l2x.MIXED, 300000)):
        sink = torch.empty(n_blocks * 256, dtype=torch.float64 if prec == l2x.FP64 else torch.float32, device=dev)
        l2x.fma_probe(prec, n_blocks, max(1, iters // 10), sink)
        best = 0.0
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flops = l2x.fma_probe(prec, n_blocks, iters, sink)
            e1.record(stream)
            e1.synchronize()
            best = max(best, flops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        out[name + "_tflops"] = best
    out["how"] = ("library FMA probe: 1216 blocks x 256 threads x 8 independent FMA chains, best of 3 "
                  "CUDA-event-timed launches (burst, kernel timed alone)")
    return out


# ----------------------------------------------------------------------------- our arm

class Arm:
    """Timing of one coupling form on one rank's inputs (positions resident in HBM)."""

    def __init__(self, torch, l2x, grid, positions, E, u32, f32, dev, world, flush, work_shape=None):
        self.torch, self.l2x, self.grid, self.positions, self.E = torch, l2x, grid, positions, E
        self.u32, self.f32, self.dev, self.world, self.flush = u32, f32, dev, world, flush
        self.work_shape = work_shape

    def coupling(self, path, precision, X=None, multiplier=0):
        """A coupling on the first configuration; fused forms pick their work-chunk
        sizes with the library's autotuner."""
        l2x = self.l2x
        c = l2x.Coupling(self.grid, self.positions[0] if X is None else X, self.E, path=path,
                         precision=precision, cg_rtol=1e-9 if precision == l2x.MIXED else 1e-13,
                         multiplier=multiplier)
        if path == l2x.FUSED and self.work_shape is not None:
            cb, rpb, cl, rpbs = self.work_shape[:4]
            cc = self.work_shape[4] if len(self.work_shape) > 4 else None
            c.set_work_shape(cb, rpb, cl, rpbs, clip_chunk=cc)
            self.tuned = dict(clip_block=cb, clip_chunk=c.info()["clip_chunk"], pcg_rows_per_block=rpb,
                              pcg_cluster=cl, pcg_rows_per_block_step=rpbs, fixed=True)
        elif path == l2x.FUSED:
            self.tuned = c.autotune()
        return c

    def per_call(self, path, precision, steps, warmup, timing=False, multiplier=0):
        """One library call per operation: update_geometry, transfer_velocity, transfer_force."""
        torch, l2x = self.torch, self.l2x
        dt = torch.float32 if precision == l2x.MIXED else torch.float64
        c = self.coupling(path, precision, multiplier=multiplier)
        uf = [u.to(dt) for u in self.u32]
        fs = [f.to(dt) for f in self.f32]
        ff = [torch.zeros(n, dtype=dt, device=self.dev) for n in c.fluid_sizes()]
        stream = torch.cuda.current_stream(self.dev)
        P = self.positions

        def step(i, ev=None):
            if ev is not None:
                ev[0].record(stream)
            c.update_geometry(P[i % len(P)])
            if ev is not None:
                ev[1].record(stream)
            c.transfer_velocity(uf)
            for z in ff:
                z.zero_()
            c.transfer_force(fs, ff)
            if ev is not None:
                ev[2].record(stream)

        for i in range(warmup):
            step(i)
        torch.cuda.synchronize()
        if timing:
            c.set_timing(True)
        barrier(self.world)
        n0 = l2x.kernel_launch_count()
        tb = ta = 0.0
        pairs = 0
        for i in range(steps):
            self.flush.fill_(1.0)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            step(i, ev)
            ev[2].synchronize()
            tb += ev[0].elapsed_time(ev[1])
            ta += ev[1].elapsed_time(ev[2])
            pairs += c.info()["n_pairs_total"] if len(P) > 1 or i == 0 else 0
        barrier(self.world)
        launches = l2x.kernel_launch_count() - n0
        info = c.info()
        pairs_per_step = pairs / steps if len(P) > 1 else info["n_pairs_total"]
        return dict(c=c, info=info, build_ms=tb / steps, apply_ms=ta / steps, launches=launches,
                    pairs=pairs_per_step, uf=uf, fs=fs)

    def picard(self, c, uf, fs, iters):
        """Picard iterations on one assembled coupling (Sec. 3): per iteration the
        enqueue-only velocity and force transfers and the Step-6 infinity norms
        (the caller's solid and fluid solves are not part of the library)."""
        torch = self.torch
        dt = uf[0].dtype
        us = [torch.zeros(c.n_nodes, dtype=dt, device=self.dev) for _ in range(3)]
        ff = [torch.zeros(n, dtype=dt, device=self.dev) for n in c.fluid_sizes()]
        fprev = [torch.zeros(c.n_nodes, dtype=dt, device=self.dev) for _ in range(3)]
        norms = torch.zeros(2, dtype=torch.float64, device=self.dev)
        stream = torch.cuda.current_stream(self.dev)

        def it():
            c.transfer_velocity_async(uf, us)
            for z in ff:
                z.zero_()
            c.transfer_force_async(fs, ff)
            c.picard_norms(fs, fprev, copy=True, out=norms)

        for _ in range(3):
            it()
        c.sync_status()
        self.flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(iters):
            it()
        e1.record(stream)
        e1.synchronize()
        c.sync_status()
        return e0.elapsed_time(e1) / iters

    def graph(self, precision, steps, warmup, multiplier=0):
        """The whole step captured as one CUDA graph and replayed."""
        torch, l2x = self.torch, self.l2x
        dt = torch.float32 if precision == l2x.MIXED else torch.float64
        c = self.coupling(l2x.FUSED, precision, multiplier=multiplier)
        uf = [u.to(dt) for u in self.u32]
        fs = [f.to(dt) for f in self.f32]
        us = [torch.zeros(c.n_nodes, dtype=dt, device=self.dev) for _ in range(3)]
        ff = [torch.zeros(n, dtype=dt, device=self.dev) for n in c.fluid_sizes()]
        P = self.positions
        src = P[0].clone()
        k0 = l2x.kernel_launch_count()
        g = c.capture_step(src, uf, us, fs, ff, margin=1.3)
        # the library counts each kernel it launches, including those recorded
        # into the graph: this is the number of kernel nodes every replay runs
        kernels_per_step = l2x.kernel_launch_count() - k0
        pairs_at = []
        for i in range(len(P)):
            src.copy_(P[i])
            g.launch()
            g.status()
            pairs_at.append(c.info()["n_pairs_total"])
        for i in range(warmup):
            src.copy_(P[i % len(P)])
            g.launch()
        g.status()
        barrier(self.world)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream(self.dev)
        tot = 0.0
        pairs = 0
        for i in range(steps):
            self.flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            src.copy_(P[i % len(P)])
            g.launch()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
            pairs += pairs_at[i % len(P)]
        g.status()
        barrier(self.world)
        return dict(c=c, g=g, step_ms=tot / steps, pairs=pairs / steps, pairs_at=pairs_at,
                    buffers=(src, uf, us, fs, ff), kernels_per_step=kernels_per_step)


def load_workload(name, rank, dev, torch):
    """Host inputs and device tensors of one rank's workload."""
    import synth
    batch = name == "batch64"
    if batch:
        grid, bodies, Eh, nr, er = synth.batch_workload(64, 256, 1000, 200000, seed=workload_seed(rank))
        n_steps, n_conf = 200, 8
        coords = [synth.batch_coords(bodies, k * (n_steps // n_conf), n_steps) for k in range(n_conf)]
        fields = [synth.taylor_green(synth.grid_node_coords(grid, g), g) for g in range(3)]
        rng = np.random.default_rng(100 + rank)
        F = rng.standard_normal((coords[0].shape[0], 3))
    else:
        w = synth.workload(name, seed=workload_seed(rank))
        grid, Eh, fields, F = w.grid, w.elems, w.fields, w.force
        coords = [w.coords]
    positions = [torch.from_numpy(c).to(dev) for c in coords]
    E = torch.from_numpy(Eh).to(dev)
    u32 = [torch.from_numpy(f.astype(np.float32)).to(dev) for f in fields]
    F32 = F.astype(np.float32)
    f32 = [torch.from_numpy(np.ascontiguousarray(F32[:, g])).to(dev) for g in range(3)]
    return dict(name=name, batch=batch, grid=grid, coords=coords, Eh=Eh, fields=fields, F=F,
                positions=positions, E=E, u32=u32, f32=f32)


def clip_roofline(ph, calls, pairs_per_step, n_steps, flops_per_pair, peak, peak_source):
    """ALU roofline of the clipping kernel from per-call phase times: the oracle's
    algorithmic FP64 operations per pair x pairs per launch / launch time."""
    launch_ms = ph["clip"] / max(1, calls["clip"])
    pairs_per_launch = pairs_per_step / max(1, calls["clip"] // n_steps)
    achieved = flops_per_pair * pairs_per_launch / (launch_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "kernel": "clip_fused_kernel<3,float> (FP64 pipe)", "launch_ms": launch_ms,
            "pairs_per_launch": pairs_per_launch, "flops_per_pair": flops_per_pair,
            "flops_per_pair_source": "oracle operation tallies (cell frame, plane-side values, cut points, "
                                     "sub-simplex volumes) on the CPU sample of this workload",
            "peak_source": peak_source,
            "traffic": (CLIP_DRAM_BYTES_PER_PAIR * pairs_per_launch if CLIP_DRAM_BYTES_PER_PAIR is not None
                        else None)}


def apply_roofline(pc, ph, calls, torch, peak_hbm, peak_src):
    """HBM rooflines of the sparse products and the mass-matrix solve of the apply
    (per-call phase times, mixed form)."""
    c = pc["c"]
    bB, bT = spmv_bytes(c, torch)
    tB = ph["spmv_B"] / max(1, calls["spmv_B"])
    tT = ph["spmv_BT"] / max(1, calls["spmv_BT"])
    tP = ph["pcg"] / max(1, calls["pcg"])
    iters = pc["info"]["cg_iters"]
    bP = pcg_bytes(c, iters, c.n_grids)

    def entry(b, t):
        return {"bytes": b, "ms": t, "achieved": b / (t * 1e-3) / 1e9, "frac": b / (t * 1e-3) / 1e9 / peak_hbm}
    return {"bound": "hbm", "unit": "GB/s", "peak": peak_hbm, "peak_source": peak_src,
            "spmv_B": entry(bB, tB), "spmv_BT": entry(bT, tT),
            "pcg": dict(entry(bP, tP), iters_per_solve=iters,
                        note="one 3-component solve; bytes: per iteration the M_s product and 7 vector passes"),
            "pcg_ms_per_solve": tP}


def autograd_ms(l2x, torch, cg, uf, dev, n=10):
    """Forward + hand-written backward of the differentiable velocity transfer."""
    ua = [u.clone().requires_grad_(True) for u in uf]
    gw = [torch.ones(cg.n_nodes, dtype=ua[0].dtype, device=dev) for _ in ua]
    for _ in range(3):
        out = l2x.VelocityTransfer.apply(cg, *ua)
        torch.autograd.backward(out, gw)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(torch.cuda.current_stream(dev))
    for _ in range(n):
        out = l2x.VelocityTransfer.apply(cg, *ua)
        torch.autograd.backward(out, gw)
    a1.record(torch.cuda.current_stream(dev))
    a1.synchronize()
    return {"forward_backward_ms": a0.elapsed_time(a1) / n,
            "form": "VelocityTransfer forward (B, S^-1) + backward (S^-1, B^T), mixed precision"}


def sample_vs_oracle(l2x, torch, wl, dev, cpu):
    """The chosen (mixed) form on the CPU baseline's sample mesh, against the
    oracle's results on it: relative L2 error per result."""
    sub, _ = slab_sample(wl["coords"][0], wl["Eh"], CPU_SAMPLE_ELEMS)
    used = np.unique(sub)
    remap = np.full(wl["coords"][0].shape[0], -1, dtype=np.int64)
    remap[used] = np.arange(used.size)
    X, E, F = wl["coords"][0][used], remap[sub].astype(np.int32), wl["F"][used]
    c = l2x.Coupling(wl["grid"], torch.from_numpy(X).to(dev), torch.from_numpy(E).to(dev), path=l2x.FUSED,
                     precision=l2x.MIXED, cg_rtol=1e-9)
    uf = [torch.from_numpy(f.astype(np.float32)).to(dev) for f in wl["fields"]]
    us = c.transfer_velocity(uf)
    fs = [torch.from_numpy(np.ascontiguousarray(F[:, g].astype(np.float32))).to(dev) for g in range(3)]
    ff = c.transfer_force(fs)
    ref_us, ref_ff = cpu.pop("_us"), cpu.pop("_ff")
    got = np.stack([u.double().cpu().numpy() for u in us], axis=1)
    err_u = float(np.linalg.norm(got - ref_us) / np.linalg.norm(ref_us))
    err_f = max(float(np.linalg.norm(ff[k].double().cpu().numpy() - ref_ff[k]) / np.linalg.norm(ref_ff[k]))
                for k in range(3))
    del c
    return err_u, err_f


def run_workload(args, name, rank, world, local, dev, torch, l2x, flush, steps, warmup, headline, peaks):
    """Times one workload; ``headline`` adds the plain/FP64/dual/Picard/e2e arms
    and the full CPU baseline."""
    wl = load_workload(name, rank, dev, torch)
    batch = wl["batch"]
    arm = Arm(torch, l2x, wl["grid"], wl["positions"], wl["E"], wl["u32"], wl["f32"], dev, world, flush,
              args.work_shape)
    res = {}
    with ClockSampler(local) as clocks:
        gr = arm.graph(l2x.MIXED, steps, warmup)
    res["clocks"] = clocks.summary()
    res["autotuned"] = dict(arm.tuned)
    step_ms, total_pairs, value = aggregate(gr["step_ms"], gr["pairs"], world)
    res.update(value=value, ms_per_step=step_ms, pairs_per_step=gr["pairs"], steps=steps,
               kernels_per_step=gr["kernels_per_step"])

    # per-call form of the same precision, with per-phase timing
    n_pc = max(3, steps // 4)
    pc = arm.per_call(l2x.FUSED, l2x.MIXED, n_pc, 3, timing=True)
    ph, calls = pc["info"]["phase_ms"], pc["info"]["phase_calls"]
    res["per_call_mixed"] = {"build_ms": pc["build_ms"], "apply_ms": pc["apply_ms"],
                             "pairs_per_s": pc["pairs"] / ((pc["build_ms"] + pc["apply_ms"]) * 1e-3),
                             "assembly_pairs_per_s": pc["pairs"] / (pc["build_ms"] * 1e-3),
                             "phase_ms_per_step": {k: v / n_pc for k, v in ph.items()},
                             "cg_iters": pc["info"]["cg_iters"]}
    peak_hbm, peak_src = hbm_peak()
    res["apply_roofline"] = apply_roofline(pc, ph, calls, torch, peak_hbm, peak_src)

    # the oracle on a bounded sample: CPU baseline and algorithmic work per pair
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        coords0 = wl["coords"][0]
        if headline:
            cpu = cpu_baseline_leg(wl["grid"], coords0, wl["Eh"], wl["F"], wl["fields"])
            # results of the sample for the accuracy check below
            sub, _ = slab_sample(coords0, wl["Eh"], CPU_SAMPLE_ELEMS)
            _, us_o, ff_o, _, _, _, _ = oracle_step(wl["grid"], coords0, sub, wl["F"], os.cpu_count() or 1,
                                                    wl["fields"])
            cpu["_us"], cpu["_ff"] = us_o, ff_o
            eu, ef = sample_vs_oracle(l2x, torch, wl, dev, cpu)
            cpu["rel_err_u_s"], cpu["rel_err_f_f"] = eu, ef
            cpu["rel_err_note"] = "chosen mixed form on the sample mesh vs the oracle's FP64 results on it"
        else:
            cpu = cpu_baseline_leg(wl["grid"], coords0, wl["Eh"], wl["F"], wl["fields"], n_max=TALLY_SAMPLE_ELEMS,
                                   single=False)
        res["roofline"] = clip_roofline(ph, calls, pc["pairs"], n_pc, cpu["fp64_flops_per_pair"],
                                        peaks["fp64_tflops"], "measured: library FMA probe, FP64, burst")
        fp32_flops = cpu["op_tallies_per_pair"]["quad"]
        res["roofline"]["oracle_quadrature_flops_per_pair"] = fp32_flops
    res["cpu_baseline"] = cpu

    if name == "leaflet256" or headline:
        res["autograd"] = autograd_ms(l2x, torch, pc["c"], pc["uf"], dev)

    if headline:
        picard_ms = arm.picard(pc["c"], pc["uf"], pc["fs"], 20)
        res["picard"] = {"iteration_ms": picard_ms, "iterations_per_time_step": 3,
                         "time_step_ms": pc["build_ms"] + 3 * picard_ms,
                         "pairs_per_s": pc["pairs"] / ((pc["build_ms"] + 3 * picard_ms) * 1e-3),
                         "form": "per-call assembly, then 3 x (enqueue-only velocity + force transfer + Step-6 "
                                 "norms), mixed precision, standard multipliers"}

        def results(r):
            c = r["c"]
            c.update_geometry(wl["positions"][0])
            u = c.transfer_velocity(r["uf"])
            f = c.transfer_force(r["fs"])
            return [x.double() for x in u], [x.double() for x in f]

        def rel(a, b):
            nb = float(torch.linalg.norm(b))
            return float(torch.linalg.norm(a - b)) / nb if nb > 0 else None  # None: a zero reference component

        um, fm = results(pc)
        del pc
        gc.collect()
        f64 = arm.per_call(l2x.FUSED, l2x.FP64, args.plain_steps, 2)
        u64, f64r = results(f64)
        res["mixed_vs_fp64"] = {"u_s": [rel(a, b) for a, b in zip(um, u64)],
                                "f_f": [rel(a, b) for a, b in zip(fm, f64r)],
                                "u_s_all": rel(torch.cat(um), torch.cat(u64)),
                                "f_f_all": rel(torch.cat(fm), torch.cat(f64r)),
                                "against": "fused FP64 GPU path on the same configuration (which matches the FP64 "
                                           "oracle to 1e-12)"}
        del um, fm, u64, f64r
        res["fused_fp64"] = {"assembly_ms": f64["build_ms"], "apply_ms": f64["apply_ms"],
                             "pairs_per_s": f64["pairs"] / ((f64["build_ms"] + f64["apply_ms"]) * 1e-3),
                             "assembly_pairs_per_s": f64["pairs"] / (f64["build_ms"] * 1e-3),
                             "cg_iters": f64["info"]["cg_iters"]}
        del f64
        gc.collect()
        plain = arm.per_call(l2x.PLAIN, l2x.FP64, args.plain_steps, 2)
        res["plain_fp64"] = {"assembly_ms": plain["build_ms"], "apply_ms": plain["apply_ms"],
                             "pairs_per_s": plain["pairs"] / ((plain["build_ms"] + plain["apply_ms"]) * 1e-3),
                             "assembly_pairs_per_s": plain["pairs"] / (plain["build_ms"] * 1e-3),
                             "cg_iters": plain["info"]["cg_iters"]}
        del plain
        gc.collect()

        # the dual multiplier basis (pseudo L2 projection, S diagonal: no CG), same step
        n_dual = max(3, steps // 4)
        dgr = arm.graph(l2x.MIXED, n_dual, 3, multiplier=l2x.DUAL_BASIS)
        d_ms, d_pairs, d_value = aggregate(dgr["step_ms"], dgr["pairs"], world)
        del dgr
        gc.collect()
        res["pseudo_l2_dual"] = {"form": "fused, captured step graph, mixed precision, dual multiplier basis",
                                 "value": d_value, "unit": UNIT, "ms_per_step": d_ms, "steps": n_dual}

        # end to end through the public API with host buffers: the captured step of
        # l2x_graph_create_host, whose replay copies the positions, u_f and f_s in from
        # page-locked host arrays and u_s and f_f back (graph nodes, inside the timed
        # region); a caller with a host-side fluid solver makes this call
        c = gr["c"]
        src, uf, us, fs, ff = gr["buffers"]
        dt = uf[0].dtype
        gr["g"] = None  # the new capture retires the device-array graph
        Ph = [p.cpu() for p in wl["positions"]]
        coords_h = torch.empty_like(Ph[0]).pin_memory()
        uh = [u.cpu().pin_memory() for u in uf]
        fh = [f.cpu().pin_memory() for f in fs]
        us_h = [torch.empty(c.n_nodes, dtype=dt).pin_memory() for _ in range(3)]
        ff_h = [torch.empty(n, dtype=dt).pin_memory() for n in c.fluid_sizes()]
        coords_h.copy_(Ph[0])
        gh = c.capture_step_host(coords_h, uh, us_h, fh, ff_h, margin=1.3)
        stream = torch.cuda.current_stream(dev)

        def e2e_step(i):
            coords_h.copy_(Ph[i % len(Ph)])  # the caller's new positions (host memory, before the launch)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gh.launch()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1)

        for i in range(2):
            e2e_step(i)
        gh.status()
        barrier(world)
        e_ms = 0.0
        n_e2e = max(3, steps // 4)
        e2e_pairs = 0
        for i in range(n_e2e):
            flush.fill_(1.0)
            e_ms += e2e_step(i)
            e2e_pairs += gr["pairs_at"][i % len(gr["pairs_at"])]
        gh.status()
        e_ms = e_ms / n_e2e
        e_step_ms, e_total, e_value = aggregate(e_ms, e2e_pairs / n_e2e, world)
        h2d, d2h = gh.io_bytes()  # counted by the library from the copies the graph holds
        res["e2e"] = {"value": e_value, "unit": UNIT, "ms_per_step": e_step_ms,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "form": "l2x_graph_create_host: copies in and out are nodes of the step graph "
                              "(positions, f_s and the touched-node box of u_f in beside the assembly; u_s out "
                              "beside the force transfer; the box of f_f out last)"}
        del gh, Ph, uh, fh, us_h, ff_h, coords_h
    else:
        del pc
    del gr, arm, wl
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    import torch
    import paper_1810_13046_gb300 as l2x

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks = fma_peaks(torch, l2x, dev)

    # the chosen form on the headline workload: captured step graph, fused, FP64
    # geometry + FP32 fields/SpMV/CG with compensated dots and FP64 refinement
    h = run_workload(args, args.workload, rank, world, local, dev, torch, l2x, flush, args.steps, args.warmup,
                     True, peaks)
    extras = {}
    if world == 1:
        for name in args.extras:
            if name == args.workload:
                continue
            r = run_workload(args, name, rank, world, local, dev, torch, l2x, flush, args.extra_steps,
                             max(3, args.warmup // 2), False, peaks)
            r["desc"] = WORKLOAD_DESCS[name]
            r["gpu_launches_per_step"] = r.pop("kernels_per_step")
            extras[name] = r

    if rank == 0:
        pcm = h["per_call_mixed"]
        line = {
            "metric": METRIC, "value": h["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOAD_DESCS.get(args.workload, args.workload),
                       "form": "fused, captured step graph; FP64 geometry, FP32 fields/SpMV/CG with compensated "
                               "dots and FP64 refinement", "pairs_per_step": h["pairs_per_step"],
                       "l2": "flushed (256 MB write) before every timed step"},
            "assembly_pairs_per_s": pcm["assembly_pairs_per_s"], "apply_ms": pcm["apply_ms"],
            "per_call_mixed": pcm,
            "plain_fp64": h["plain_fp64"],
            "fused_fp64": h["fused_fp64"],
            "e2e": h["e2e"],
            "autotuned": h["autotuned"],
            "pseudo_l2_dual": h["pseudo_l2_dual"],
            "picard": h["picard"],
            "gpu_launches": int(h["kernels_per_step"] * args.steps),
            "gpu_launches_note": f"{h['kernels_per_step']} kernel nodes per captured step (counted by the "
                                 f"library as they were recorded) x {args.steps} timed replays",
            "roofline": h.get("roofline"),
            "apply_roofline": h["apply_roofline"],
            "peaks_measured": peaks,
            "mixed_vs_fp64": h["mixed_vs_fp64"],
            "autograd": h["autograd"],
            "cpu_baseline": h["cpu_baseline"],
            "clocks": h["clocks"],
            "workloads": extras,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
