"""Benchmark: P1 stiffness S + weighted mass M^[w] assembly on one GB300 (per GPU for N > 1).

Workload: the jittered, node-permuted unit-square mesh with 2048 x 2048 cells (nq = 4,198,401,
nme = 8,388,608), w = 1 + 0.5 sin(2 pi x) cos(2 pi y) + U(0, 0.1), FP64 throughout. One step
is one pass of the whole path over resident device inputs, as one sparse() call of the paper
would do it: mesh validation (fe_mesh_create), the structural pattern (fe_pattern_build) and
the values of S and M^[w] (fe_assemble_stiff_wmass). The value is triangles per second over
the timed steps. Also reported:
  - assemble_only: the values with the pattern built once beforehand (repeated assembly), L2
    flushed between calls, and warm (back to back, the time-stepping use);
  - batched: 256 uneven meshes (N log-uniform in [16, 512]) in one graph-replayed persistent
    launch vs 256 plain launches;
  - e2e: the same step from pinned host arrays to host CSR arrays through the public API (mean,
    median, p90 and max of the steps);
  - arith: the arithmetic of the element stage (the default row-owner variant computes in
    double-float on the FP32 pipes), and fp64_variants: the same step by the two variants whose
    element arithmetic is plain FP64 (staged gather, FP64 atomics);
  - per-kernel shares of the step, each with its algorithmic bytes and HBM fraction;
  - unstructured: the same step on the random-diagonal 2048 x 2048 square (valences 4 to 8), and
    disk: on a Delaunay mesh of the unit disk from 2^20 random points (valences 3 to about 20);
  - partition: the same mesh split into 2, 4 and 8 row ranges (halo triangles, no exchange of
    values), each rank's step timed in turn on this GPU;
  - roofline of the dominant kernel, timed live with the library's own CUDA events;
  - the other legs: plane elasticity, the adjoint, zero dropping, tetrahedra, 3-D elasticity on
    tetrahedra, P2 and P3 triangles, each with both scatter variants where it has them;
  - cpu_baseline: the FP64 CPU oracle on a bounded sample of the same workload, single-threaded,
    on all host cores (one process per core), and beside every other leg.
Between timed steps L2 is flushed by writing a 512 MB buffer (outside the timed intervals).
Python's collector is off inside the timed regions.

Multi-GPU (torchrun): every rank assembles its own replica of the workload (no collective;
weak scaling); value = all ranks' triangles / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "P1 assembly Melements/s and HBM GB/s (% peak), FP64, batched vs plain launches"
UNIT = "Melem/s"
N_CELLS = 2048
SEED = 13053122 + 2


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ algorithmic bytes
#
# Bytes a kernel's role must move, per launch, for a mesh with nq vertices, nme triangles and
# nnz stored entries per scalar matrix (int32 indices, FP64 values). The assembly figure is the
# method's compulsory traffic (me, q, w read once; both value arrays written once).

def algorithmic_bytes(name: str, nq: int, nme: int, nnz: int) -> int | None:
    table = {
        "k_scalar_atomic": 12 * nme + 16 * nq + 8 * nq + 16 * nnz,
        "k_scalar_stage": 12 * nme + 16 * nq + 8 * nq + 2 * 72 * nme,
        "k_seg_gather": 4 * (nnz + 1) + 36 * nme + 2 * 72 * nme + 16 * nnz,
        "k_fan_scalar": 12 * nme + 16 * nq + 8 * nq + 16 * nnz,
        "k_pack_vrec": 16 * nq + 8 * nq + 32 * nq,
        "k_validate": 12 * nme + 16 * nq + 4 * nq,             # me, q; valence counts written
        "k_pack_coords": 32 * nq,
        "k_fill_adj": 12 * nme + 8 * nq + 24 * nme,             # me, cursors; bucket records
        "k_row_analyse": 8 * nq + 24 * nme + 24 * nme + 8 * nq,  # offsets, buckets; fan records, headers
        "k_col_fill": 12 * nq + 24 * nme + 4 * nnz,             # offsets, fan records; col_idx
        "k_build_map": 12 * nme + 4 * nq + 4 * nnz + 36 * nme,
        "k_tile_sums": 4 * nq,
        "k_tile_scan": 8 * nq,
    }
    return table.get(name)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0: float | None = None, t1: float | None = None) -> dict:
        """Median SM clock etc. over the samples taken between host times t0 and t1 (the timed
        region; a 0.25 s margin on each side covers the sampler's own period)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if t0 is not None and not (t0 - 0.25 <= ts <= t1 + 0.25):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle leg

def cpu_oracle_sample(target_s: float = 10.0, n_cells: int = 512) -> dict:
    """The oracle (single-threaded C, FP64) on a bounded sample: one 512 x 512-cell mesh of the
    same recipe, S + M^[w] assembled repeatedly for about target_s seconds."""
    import oracle
    from paper_1305_3122_gb300 import meshgen

    m = meshgen.square_mesh(n_cells, SEED)
    w = meshgen.vertex_weights(m, SEED)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.assemble(oracle.STIFF, m.q, m.me)
        oracle.assemble(oracle.WMASS, m.q, m.me, w)
        reps += 1
        el = time.perf_counter() - t0
        if el >= target_s:
            break
    return {"value": round(reps * m.nme / el / 1e6, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} x (S + M^[w]) on the {n_cells}x{n_cells}-cell mesh of the same recipe "
                      f"(nme={m.nme}), {el:.1f} s, single-threaded C oracle"}


def _oracle_worker(job: tuple[int, float, int]) -> tuple[int, float]:
    """One process of the all-cores oracle timing: S + M^[w] on its own copy of the sample mesh for
    about target_s seconds; returns (elements assembled, seconds)."""
    n_cells, target_s, seed = job
    import oracle
    from paper_1305_3122_gb300 import meshgen

    m = meshgen.square_mesh(n_cells, seed)
    w = meshgen.vertex_weights(m, seed)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.assemble(oracle.STIFF, m.q, m.me)
        oracle.assemble(oracle.WMASS, m.q, m.me, w)
        reps += 1
        el = time.perf_counter() - t0
        if el >= target_s:
            return reps * m.nme, el


def cpu_oracle_all_cores(target_s: float = 8.0, n_cells: int = 512) -> dict:
    """The unmodified single-threaded oracle run as one process per host core, each on its own
    sample of the workload (independent meshes: the all-cores throughput of the CPU program).
    Processes are spawned, not forked, since the GPU is already in use."""
    import multiprocessing as mp

    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_worker, [(n_cells, target_s, SEED)] * n)
    elems = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return {"value": round(elems / el / 1e6, 4), "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} processes of the single-threaded C oracle, each S + M^[w] on its own {n_cells}x{n_cells}-cell "
                      f"mesh of the same recipe for about {target_s:.0f} s ({elems} elements in {el:.1f} s)"}


def _oracle_rate(fn, units: float, target_s: float) -> tuple[float, int, float]:
    """Repeat fn() for about target_s seconds; units processed per second, repetitions, seconds."""
    reps, t0 = 0, time.perf_counter()
    while True:
        fn()
        reps += 1
        el = time.perf_counter() - t0
        if el >= target_s:
            return reps * units / el, reps, el


def cpu_oracle_legs(legs, target_s: float = 2.0) -> dict:
    """The oracle beside each other leg: each leg's computation by the single-threaded C oracle on
    a bounded sample of that leg's workload (same recipe, smaller size), in the leg's own unit."""
    import oracle
    from paper_1305_3122_gb300 import meshgen

    out = {}

    def entry(rate, unit, reps, el, what):
        return {"value": round(rate, 4), "unit": unit, "cores": 1, "kind": "oracle",
                "sample": f"{reps} x {what}, {el:.1f} s"}

    if "elasticity" in legs:
        m = meshgen.square_mesh(256, 13053122 + 3)
        r = _oracle_rate(lambda: oracle.assemble(oracle.ELAS, m.q, m.me, lam=1.0, mu=0.5), m.nme / 1e6, target_s)
        out["elasticity"] = entry(*r[:1], "Melem/s", r[1], r[2], f"K (lambda 1, mu 0.5) on the 256x256-cell mesh (nme={m.nme})")
    if "adjoint" in legs:
        seed = 13053122 + 5
        m = meshgen.square_mesh(256, seed)
        w = meshgen.vertex_weights(m, seed)
        rp, ci, _ = oracle.assemble(oracle.STIFF, m.q, m.me)
        GS, GM = meshgen.upstream_gradients(seed, len(ci))

        def adj():
            dq, dw = oracle.adjoint(oracle.STIFF, m.q, m.me, rp, ci, GS, w)
            oracle.adjoint(oracle.WMASS, m.q, m.me, rp, ci, GM, w, dq, dw)
        r = _oracle_rate(adj, m.nme / 1e6, target_s)
        out["adjoint"] = entry(r[0], "Melem/s", r[1], r[2], f"dL/dq, dL/dw of <G_S, S> + <G_M, M^[w]> on the 256x256-cell mesh (nme={m.nme})")
    if "drop_zeros" in legs:
        m = meshgen.square_mesh(512, SEED)
        rp, ci, va = oracle.assemble(oracle.STIFF, m.q, m.me)
        r = _oracle_rate(lambda: oracle.drop_zeros(rp, ci, va), len(va) / 1e9, target_s)
        out["drop_zeros"] = entry(r[0], "Gentries/s", r[1], r[2], f"zero dropping of S on the 512x512-cell mesh (nnz={len(va)})")
    if "tetrahedra" in legs:
        m = meshgen.cube_mesh(24, 13053122 + 6)
        r = _oracle_rate(lambda: oracle.tet_assemble(oracle.STIFF, m.q, m.me), m.nme / 1e6, target_s)
        out["tetrahedra"] = entry(r[0], "Melem/s", r[1], r[2], f"S on the 24^3-cell cube (nme={m.nme})")
    if "tet_elasticity" in legs:
        m = meshgen.cube_mesh(12, 13053122 + 9)
        r = _oracle_rate(lambda: oracle.tet_elas_assemble(m.q, m.me, 1.25, 0.4), m.nme / 1e6, target_s)
        out["tet_elasticity"] = entry(r[0], "Melem/s", r[1], r[2], f"3-D K (lambda 1.25, mu 0.4) on the 12^3-cell cube (nme={m.nme})")
    if "p2" in legs:
        m = meshgen.square_mesh(48, 13053122 + 7)
        r = _oracle_rate(lambda: oracle.p2_assemble(oracle.STIFF, m.q, m.me), m.nme / 1e6, target_s)
        out["p2"] = entry(r[0], "Melem/s", r[1], r[2], f"P2 S on the 48x48-cell square (nme={m.nme})")
    if "p3" in legs:
        m = meshgen.square_mesh(32, 13053122 + 8)
        r = _oracle_rate(lambda: oracle.p3_assemble(oracle.STIFF, m.q, m.me), m.nme / 1e6, target_s)
        out["p3"] = entry(r[0], "Melem/s", r[1], r[2], f"P3 S on the 32x32-cell square (nme={m.nme})")
    if "batched" in legs:
        ms = meshgen.batch_meshes(13053122 + 4, count=8)
        n = sum(x.nme for x in ms)

        def batch():
            for x in ms:
                oracle.assemble(oracle.STIFF, x.q, x.me)
                oracle.assemble(oracle.MASS, x.q, x.me)
        r = _oracle_rate(batch, n / 1e6, target_s)
        out["batched"] = entry(r[0], "Melem/s", r[1], r[2], f"S + M of the batch recipe's first 8 meshes (nme={n})")
    return out


def run_reference(args) -> int:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_1305_3122_gb300 import meshgen

    # each step is a bounded sample of the workload: a mesh of the same recipe sized so that the
    # whole warm-up + timed run takes about a minute at the oracle's ~0.85 Melem/s
    per_step_s = 60.0 / max(args.steps + args.warmup, 1)
    n_cells = int(math.sqrt(0.85e6 * per_step_s / 2.0)) // 16 * 16
    n_cells = max(32, min(512, n_cells))
    m = meshgen.square_mesh(n_cells, SEED)
    w = meshgen.vertex_weights(m, SEED)

    def step():
        oracle.assemble(oracle.STIFF, m.q, m.me)
        oracle.assemble(oracle.WMASS, m.q, m.me, w)

    for _ in range(args.warmup):
        step()
    gc.collect()
    gc.disable()                         # as in the GPU arm's timed regions
    try:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        el = time.perf_counter() - t0
    finally:
        gc.enable()
    value = args.steps * m.nme / el / 1e6
    sample = (f"each step: S + M^[w] by the single-threaded FP64 C oracle (triplets + sparse) on the "
              f"{n_cells}x{n_cells}-cell mesh of the same recipe (nme={m.nme}), a bounded sample of the "
              f"2048x2048 workload")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * el / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "arith": "fp64",
            "data": "synthetic",
            "config": _config({"sample_of": _config()["workload"],
                               "step": "S + M^[w] by the CPU oracle (triplets, stable sort, ordered sums) on the "
                                       "sample mesh; its sort builds the structure, as sparse() does"},
                              cells=n_cells, nq=m.nq, nme=m.nme, nnz=_nnz_grid(n_cells)),
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _nnz_grid(n: int) -> int:
    """Stored entries per scalar matrix of the n x n-cell grid: one per vertex, two per edge."""
    return (n + 1) ** 2 + 2 * (3 * n * n + 2 * n)


def _config(extra: dict | None = None, cells: int = N_CELLS, nq: int = 4198401, nme: int = 8388608,
            nnz: int = 29372417) -> dict:
    c = {"workload": f"P1 stiffness S + weighted mass M^[w], FP64, jittered node-permuted unit-square mesh "
                     f"{cells}x{cells} cells (nq={nq}, nme={nme}, nnz={nnz} per matrix)",
         "step": "mesh validation + pattern build + S and M^[w] values (one sparse()-equivalent call)",
         "l2": "flushed between timed steps (512 MB write); inputs+outputs (~0.67 GB) exceed L2 too"}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------------ whole-job aggregation

def rank_seed(rank: int) -> int:
    """Each rank assembles its own mesh of the same recipe (replicas, weak scaling)."""
    return SEED + 1000 * rank


def max_over_ranks(x: float, device) -> float:
    """The slowest rank's figure: the whole job ends when its last rank does."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job throughput in millions of units per second: all ranks' units over the max time."""
    return world * units_per_rank / (ms_max / 1e3) / 1e6


# ------------------------------------------------------------------ GPU arm

def run_ours(args) -> int:
    import torch
    import torch.distributed as dist

    from paper_1305_3122_gb300 import feasm, meshgen

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    variant = {"atomic": feasm.ATOMIC, "gather": feasm.GATHER, "row": feasm.ROW}[args.variant]

    m = meshgen.square_mesh(args.cells, rank_seed(rank))
    w = meshgen.vertex_weights(m, rank_seed(rank))
    q_d = torch.tensor(m.q, device=dev)
    me_d = torch.tensor(m.me, device=dev)
    w_d = torch.tensor(w, device=dev)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    gather = variant == feasm.GATHER
    use_map = variant == feasm.ATOMIC
    mesh0 = feasm.Mesh(q_d, me_d)
    pat0 = feasm.Pattern(mesh0, gather=gather, map=use_map)
    nnz = pat0.nnz
    S = pat0.new_values()
    M = pat0.new_values()

    def step():
        # create, build, assemble and release: every allocation and free is inside the step; the
        # device-resident connectivity is used in place (FE_PTR_DEVICE_BORROW)
        mesh = feasm.Mesh(q_d, me_d, borrow=True)
        pat = feasm.Pattern(mesh, gather=gather, map=use_map)
        feasm.assemble_stiff_wmass(mesh, pat, w_d, variant, S, M)
        pat.close()
        mesh.close()

    for _ in range(args.warmup):
        step()
        flush.fill_(1)
    def timed_steps():
        # the collector is off while timing (as timeit does): a full collection of this process's
        # objects takes tens of milliseconds and would stall the host between launches
        times = []
        gc.collect()
        gc.disable()
        try:
            for _ in range(args.steps):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        finally:
            gc.enable()
        torch.cuda.synchronize()
        return times

    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # the headline timed region: the library's per-kernel events are off (they cost ~4% of a step)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)                      # let the sampler start before the timed region
    t_begin = time.time()
    times = timed_steps()
    t_end = time.time()
    clk = clocks.stop(t_begin, t_end)
    # the same steps again with the library's per-kernel CUDA events (recorded on each kernel's
    # launch stream): kernel durations for the roofline and the breakdown
    feasm.profile_reset()
    feasm.profile_enable(True)
    times_prof = timed_steps()
    feasm.profile_enable(False)
    prof = feasm.profile_read()
    if world > 1:
        dist.barrier()
    ms = sum(times) / len(times)
    ms_max = max_over_ranks(ms, dev)
    value = job_value(m.nme, world, ms_max)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    hbm, peak_kind = _peaks()
    # dominant kernel of the step and its roofline
    launches = sum(c for _, c in prof.values())
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    dom_bytes = algorithmic_bytes(dom, m.nq, m.nme, nnz)
    roof = _roofline(dom, dom_bytes, dom_ms, hbm, peak_kind, args.traffic, args.cells)

    # assembly with a prebuilt pattern
    asm = assemble_only(feasm, torch, mesh0, pat0, w_d, variant, S, M, flush, stream, args, m, nnz, hbm, peak_kind)
    kern = {}
    tot = sum(x[0] for x in prof.values())
    for k, v in sorted(prof.items()):
        kern[k] = {"ms_per_launch": round(v[0] / v[1], 5), "launches": int(v[1]), "share": round(v[0] / tot, 4)}
        kb = algorithmic_bytes(k, m.nq, m.nme, nnz)
        if kb:
            kern[k]["algorithmic_bytes"] = kb
            kern[k]["hbm_frac"] = round(kb / (v[0] / v[1] / 1e3) / 1e9 / hbm, 4)
    line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "arith": ARITH[args.variant], "data": "synthetic",
            "config": _config({"variant": args.variant, "parallelism": f"replicas{world}" if world > 1 else "single"},
                              cells=args.cells, nq=m.nq, nme=m.nme, nnz=nnz),
            "roofline": roof, "gpu_launches": int(launches), "clocks": clk,
            "ms_per_step_with_kernel_events": round(sum(times_prof) / len(times_prof), 4),
            "kernels": kern,
            "assemble_only": asm}
    # end to end through the host-buffer call, right after the device-resident step (before the
    # other legs fill the device memory pools)
    if not args.no_e2e:
        line["e2e"] = e2e(feasm, torch, m, w, args)
    if not args.no_fp64_variants and args.variant == "row":
        line["fp64_variants"] = fp64_variants(feasm, torch, q_d, me_d, w_d, flush, stream, m)
    if not args.no_other and args.variant == "row" and args.cells == N_CELLS:
        line["unstructured"] = unstructured(feasm, meshgen, torch, flush, stream)
        line["disk"] = disk(feasm, meshgen, torch, flush, stream)
        line["partition"] = partition(feasm, meshgen, torch, flush)
    if not args.no_batched:
        line["batched"] = batched(feasm, meshgen, torch, args, hbm, peak_kind)
    if not args.no_other:
        line["elasticity"] = elasticity(feasm, meshgen, torch, flush, hbm, peak_kind)
        line["adjoint"] = adjoint(feasm, meshgen, torch, flush, hbm, peak_kind)
        line["drop_zeros"] = drop_zeros(feasm, torch, pat0, S, flush, hbm, peak_kind, cells=args.cells)
        line["tetrahedra"] = tetrahedra(feasm, meshgen, torch, flush, hbm, peak_kind)
        line["tet_elasticity"] = tet_elasticity(feasm, meshgen, torch, flush, hbm, peak_kind)
        line["p2"] = p2(feasm, meshgen, torch, flush, hbm, peak_kind)
        line["p3"] = p3(feasm, meshgen, torch, flush, hbm, peak_kind)
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_oracle_sample()
        line["cpu_baseline"]["all_cores"] = cpu_oracle_all_cores()
        legs = [k for k in ("batched", "elasticity", "adjoint", "drop_zeros", "tetrahedra", "tet_elasticity", "p2", "p3")
                if k in line]
        if legs:
            line["cpu_baseline"]["legs"] = cpu_oracle_legs(legs)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# The arithmetic each variant's element stage computes in (inputs and outputs are FP64 in all).
ARITH = {"row": "double-float (pairs of FP32, about 48-bit significands) element arithmetic on the FP32 pipes; "
                "FP64 inputs, coordinate differences and outputs",
         "gather": "fp64", "atomic": "fp64"}


def mesh_step(feasm, torch, flush, stream, m, w, reps: int = 20) -> dict:
    """The headline step (mesh, pattern, S + M^[w] by row owners) on another mesh: its time (first
    half of the steps, without the per-kernel events) and its kernels' times (second half)."""
    q_d, me_d, w_d = (torch.tensor(a, device="cuda") for a in (m.q, m.me, w))
    pat0 = feasm.Pattern(feasm.Mesh(q_d, me_d, borrow=True), map=False)
    S, M = pat0.new_values(), pat0.new_values()
    nnz = pat0.nnz
    pat0.close()

    def step():
        mesh = feasm.Mesh(q_d, me_d, borrow=True)
        pat = feasm.Pattern(mesh, map=False)
        feasm.assemble_stiff_wmass(mesh, pat, w_d, feasm.ROW, S, M)
        pat.close()
        mesh.close()

    for _ in range(3):
        step()
    feasm.profile_reset()
    ts = []
    for i in range(2 * reps):
        if i == reps:                                  # the second half with the per-kernel events
            feasm.profile_enable(True)
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        if i < reps:
            ts.append(e0.elapsed_time(e1))
    feasm.profile_enable(False)
    prof = feasm.profile_read()
    ms = sum(ts) / len(ts)
    val = np.bincount(m.me.ravel(), minlength=m.nq)
    return {"nnz": nnz, "ms_per_step": round(ms, 4), "value": round(m.nme / ms / 1e3, 3), "unit": UNIT,
            "rows_over_8_triangles": round(float(np.mean(val > 8)), 5),
            "kernels_ms": {k: round(v[0] / v[1], 4) for k, v in sorted(prof.items())}}


def unstructured(feasm, meshgen, torch, flush, stream, reps: int = 20) -> dict:
    """The headline step on the 2048 x 2048-cell square with random cell diagonals: interior
    vertices in 4 to 8 triangles, as in unstructured meshes."""
    m = meshgen.square_mesh(N_CELLS, SEED, random_diagonals=True)
    r = mesh_step(feasm, torch, flush, stream, m, meshgen.vertex_weights(m, SEED), reps)
    return {"workload": f"S + M^[w], random-diagonal {N_CELLS}x{N_CELLS}-cell square (nq={m.nq}, nme={m.nme}, "
                        f"nnz={r.pop('nnz')} per matrix)", **r}


def disk(feasm, meshgen, torch, flush, stream, n: int = 1 << 20, reps: int = 20) -> dict:
    """The headline step on a Delaunay mesh of the unit disk, the paper's domain, from random
    points (valences 3 to about 20; about 4% of the rows are longer than 8 triangles and go to the
    general-row kernel; thin slivers take the FP64 fan terms)."""
    seed = SEED + 20
    m = meshgen.disk_mesh(n, seed, points="poisson")
    r = mesh_step(feasm, torch, flush, stream, m, meshgen.vertex_weights(m, seed), reps)
    return {"workload": f"S + M^[w], Delaunay mesh of the unit disk from random points (nq={m.nq}, nme={m.nme}, "
                        f"nnz={r.pop('nnz')} per matrix)", **r}


def fp64_variants(feasm, torch, q_d, me_d, w_d, flush, stream, m, reps: int = 10) -> dict:
    """The same step (mesh, pattern, S + M^[w]) by the two variants whose element arithmetic is
    plain FP64: the deterministic staged gather and the FP64 atomics."""
    out = {}
    for name, variant in (("gather", feasm.GATHER), ("atomic", feasm.ATOMIC)):
        gather, use_map = variant == feasm.GATHER, variant == feasm.ATOMIC
        pat0 = feasm.Pattern(feasm.Mesh(q_d, me_d, borrow=True), gather=gather, map=use_map)
        S, M = pat0.new_values(), pat0.new_values()
        pat0.close()

        def step():
            mesh = feasm.Mesh(q_d, me_d, borrow=True)
            pat = feasm.Pattern(mesh, gather=gather, map=use_map)
            feasm.assemble_stiff_wmass(mesh, pat, w_d, variant, S, M)
            pat.close()
            mesh.close()

        for _ in range(3):
            step()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = sum(ts) / len(ts)
        out[name] = {"ms_per_step": round(ms, 4), "value": round(m.nme / ms / 1e3, 3), "unit": UNIT, "arith": "fp64",
                     "steps": reps}
        del S, M
    return out


# Source files whose change invalidates a recorded DRAM-traffic figure of a kernel.
KERNEL_SOURCES = {"k_fan_scalar": ["rowasm.cu", "ff.cuh"]}


def kernel_source_hash(name: str) -> str | None:
    files = KERNEL_SOURCES.get(name)
    if not files:
        return None
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1305_3122_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_counters(name: str, cells: int, traffic_path: str | None) -> dict:
    """ncu counters of one launch of this kernel on this mesh size (DRAM bytes, and warp
    instructions where recorded), or {} when none were recorded or the kernel's source changed
    since."""
    if not traffic_path or not os.path.exists(traffic_path):
        return {}
    with open(traffic_path) as f:
        rec = json.load(f).get(name)
    if not isinstance(rec, dict) or rec.get("cells") != cells or rec.get("source") != kernel_source_hash(name):
        return {}
    return rec


def recorded_traffic(name: str, cells: int, traffic_path: str | None):
    """DRAM bytes per launch from an ncu capture of this kernel on this mesh size, or None."""
    return recorded_counters(name, cells, traffic_path).get("bytes")


# Issue roof: 4 warp instructions per SM per clock (one per scheduler), 152 SMs, 2.07 GHz.
ISSUE_PEAK = 4 * 152 * 2.07e9


# What limits a kernel below its HBM roof, from its ncu captures (profiles/).
LIMITS = {
    "k_fan_scalar": "instruction issue and load latency: 80.6 M warp instructions at 1024^2 issued on 65.8% of cycles "
                    "(FP32 FMA pipe 42%, integer ALU 38%, FP64 pipe 48%: double-float arithmetic in place of FP64, "
                    "with FP64 for the coordinate differences and the output sums), the rest waiting on the dependent "
                    "fan-record and vertex-record loads (2.9 long-scoreboard stalls per issue, 20 warps per SM at 86 "
                    "registers; ncu at 1024^2); at 2048^2 the random vertex-record gathers also miss "
                    "L2 (traffic above). Locality orders, shared-memory staging and cp.async gathers measured slower",
}


def _roofline(name, nbytes, ms, hbm, peak_kind, traffic_path, cells=N_CELLS):
    achieved = nbytes / (ms / 1e3) / 1e9 if nbytes else None
    traffic = recorded_traffic(name, cells, traffic_path)
    out = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1) if achieved else None,
           "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4) if achieved else None,
           "traffic": traffic, "algorithmic_bytes": nbytes, "ms_per_launch": round(ms, 5),
           "peak_source": f"{peak_kind} HBM copy bandwidth"}
    if name in LIMITS:
        out["limit"] = LIMITS[name]
    inst = recorded_counters(name, cells, traffic_path).get("inst_executed")
    if inst:
        # the kernel's own bound: warp instructions per launch (ncu, same source and mesh size)
        # over the launch time measured here, against the issue roof
        rate = inst / (ms / 1e3)
        out["issue"] = {"inst_per_launch": int(inst), "achieved": round(rate / 1e9, 1), "peak": round(ISSUE_PEAK / 1e9, 1),
                        "unit": "G warp instr/s", "frac": round(rate / ISSUE_PEAK, 4),
                        "peak_source": "4 warp instructions per SM per clock x 152 SMs x 2.07 GHz (maximum SM clock)"}
    return out


def assemble_only(feasm, torch, mesh, pat, w_d, variant, S, M, flush, stream, args, m, nnz, hbm, peak_kind):
    for _ in range(3):
        feasm.assemble_stiff_wmass(mesh, pat, w_d, variant, S, M)
    feasm.profile_reset()
    feasm.profile_enable(True)
    times = []
    reps = max(args.steps, 10)
    for _ in range(reps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        feasm.assemble_stiff_wmass(mesh, pat, w_d, variant, S, M)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    feasm.profile_enable(False)
    prof = feasm.profile_read()
    ms = sum(times) / len(times)
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    roof = _roofline(dom, algorithmic_bytes(dom, m.nq, m.nme, nnz), dom_ms, hbm, peak_kind, args.traffic, args.cells)
    # warm: back-to-back calls without the flush (time stepping: same mesh, new values each step)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        feasm.assemble_stiff_wmass(mesh, pat, w_d, variant, S, M)
    e1.record(stream)
    e1.synchronize()
    ms_warm = e0.elapsed_time(e1) / reps
    return {"value": round(m.nme / (ms / 1e3) / 1e6, 3), "unit": UNIT, "ms": round(ms, 4), "reps": reps,
            "warm": {"value": round(m.nme / (ms_warm / 1e3) / 1e6, 3), "unit": UNIT, "ms": round(ms_warm, 4),
                     "what": "the same calls back to back without the L2 flush (the time-stepping use case)"},
            "kernels": {k: round(v[0] / v[1], 5) for k, v in prof.items()}, "roofline": roof}


def _time_calls(torch, fn, flush, reps=20):
    """Median device time (ms) of fn() between L2 flushes, CUDA events on the current stream."""
    for _ in range(3):
        fn()
    ts = []
    for _ in range(reps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts.sort()
    return ts[len(ts) // 2]


def partition(feasm, meshgen, torch, flush, worlds=(2, 4, 8), reps: int = 5) -> dict:
    """The row partition of the headline mesh over `world` ranks (fe_mesh_create_part,
    fe_pattern_build_part, the row owners on the rank's window): each rank's whole step (its halo
    mesh from the global arrays, its rows' pattern, S + M^[w] of its rows, release) timed in turn on
    this GPU, L2 flushed before each. The ranks exchange no values, so each rank's step on its
    own GPU is this step; projected = all triangles / the slowest rank's step.
    The mesh is the headline recipe with its nodes numbered row by row (permute=False), as a
    partitioner would number them: an owned id range is then a band of the square and the halo is
    one row of cells per cut. (With the headline's random numbering an id range is scattered over
    the whole square, and each of two ranks holds about 87% of the triangles.)"""
    from paper_1305_3122_gb300 import partition as part_rows
    m = meshgen.square_mesh(N_CELLS, SEED, permute=False)
    w = meshgen.vertex_weights(m, SEED)
    q_d, me_d, w_d = (torch.tensor(a, device="cuda") for a in (m.q, m.me, w))
    nq, nme = m.nq, m.nme
    whole = _time_calls(torch, lambda: _whole_step(feasm, q_d, me_d, w_d), flush, reps=reps)
    out = {}
    for world in worlds:
        ranks = []
        halo = 0
        for r0, r1 in part_rows.row_ranges(nq, world):
            def step():
                mesh = feasm.Mesh.part(q_d, me_d, r0, r1)
                pat = feasm.Pattern(mesh, rows=(r0, r1), map=False)
                feasm.assemble_stiff_wmass(mesh, pat, w_d, feasm.ROW)
                pat.close()
                mesh.close()
            ranks.append(_time_calls(torch, step, flush, reps=reps))
            probe = feasm.Mesh.part(q_d, me_d, r0, r1)
            halo += probe.nme
            probe.close()
        worst = max(ranks)
        out[str(world)] = {"rank_ms": [round(t, 4) for t in ranks], "rank_ms_max": round(worst, 4),
                           "triangles_held_over_nme": round(halo / nme, 4),
                           "projected_value": round(nme / worst / 1e3, 1), "unit": UNIT}
    # where the time of rank 0's step goes at the largest world: the library's kernel events
    world = max(worlds)
    r0, r1 = part_rows.row_ranges(nq, world)[0]
    feasm.profile_reset()
    feasm.profile_enable(True)
    for _ in range(reps):
        mesh = feasm.Mesh.part(q_d, me_d, r0, r1)
        pat = feasm.Pattern(mesh, rows=(r0, r1), map=False)
        feasm.assemble_stiff_wmass(mesh, pat, w_d, feasm.ROW)
        pat.close()
        mesh.close()
    torch.cuda.synchronize()
    feasm.profile_enable(False)
    prof = feasm.profile_read()
    kernels = {k: round(v[0] / reps, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}
    return {"workload": f"row partition of the {N_CELLS}x{N_CELLS}-cell headline mesh, nodes numbered row by row, "
                        "S + M^[w] by row owners",
            "how": f"each rank's step timed in turn on one GPU (median of {reps} between L2 flushes); the ranks "
                   "exchange no values, so the projection for `world` GPUs is nme / the slowest rank's step",
            "whole_ms": round(whole, 4), "worlds": out,
            "rank0_kernels_ms": {"world": world, "kernel_sum_ms": round(sum(kernels.values()), 4),
                                 "what": "rank 0's step with the library's kernel events (ms per step, L2 not flushed)",
                                 "kernels": kernels}}


def _whole_step(feasm, q_d, me_d, w_d):
    mesh = feasm.Mesh(q_d, me_d, borrow=True)
    pat = feasm.Pattern(mesh, map=False)
    feasm.assemble_stiff_wmass(mesh, pat, w_d, feasm.ROW)
    pat.close()
    mesh.close()


def elasticity(feasm, meshgen, torch, flush, hbm, peak_kind) -> dict:
    """Plane-elasticity K (Section 7) on the 1024 x 1024-cell mesh, lambda = 1, mu = 0.5, row owners,
    pattern prebuilt (2 dofs per vertex)."""
    m = meshgen.square_mesh(1024, 13053122 + 3)
    mesh = feasm.Mesh(torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"))
    pat = feasm.Pattern(mesh, dofs=2, map=False)
    K = pat.new_values()
    feasm.profile_reset()
    feasm.profile_enable(True)
    ms = _time_calls(torch, lambda: feasm.assemble_elas(mesh, pat, 1.0, 0.5, feasm.ROW, K), flush)
    feasm.profile_enable(False)
    prof = feasm.profile_read()
    k_ms = prof["k_fan_elas"][0] / prof["k_fan_elas"][1]
    nbytes = 12 * m.nme + 16 * m.nq + 8 * pat.nnz            # me, q, K values
    return {"workload": f"K, 1024x1024-cell mesh (nq={m.nq}, nme={m.nme}, nnz={pat.nnz})", "ms": round(ms, 4),
            "melem_s": round(m.nme / ms / 1e3, 2), "k_fan_elas_ms": round(k_ms, 4),
            "roofline": {"kernel": "k_fan_elas", "bound": "hbm", "algorithmic_bytes": nbytes,
                         "achieved": round(nbytes / k_ms / 1e6, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(nbytes / k_ms / 1e6 / hbm, 4), "peak_source": f"{peak_kind} HBM copy bandwidth"}}


def drop_zeros(feasm, torch, pat, S, flush, hbm, peak_kind, cells: int = N_CELLS) -> dict:
    """Matlab's value-dependent sparse() result from the structural one: fe_csr_drop_zeros on the
    step's S (2048 x 2048 cells unless --cells says otherwise). The jittered mesh has no exact zero,
    so every entry is kept and every byte moves; the call includes its one synchronisation (the
    kept count)."""
    feasm.profile_reset()
    feasm.profile_enable(True)
    kept = []
    ms = _time_calls(torch, lambda: kept.append(feasm.drop_zeros(pat.row_ptr, pat.col_idx, S)[1].numel()), flush)
    feasm.profile_enable(False)
    prof = feasm.profile_read()
    k_ms = prof["k_compact_rows"][0] / prof["k_compact_rows"][1]
    c_ms = prof["k_row_nonzeros"][0] / prof["k_row_nonzeros"][1]
    n, nnz, out = pat.n_rows, pat.nnz, kept[-1]
    nbytes = 4 * (n + 1) + 12 * nnz + 4 * (n + 1) + 12 * out     # read CSR once, write the kept CSR
    kbytes = 8 * (n + 1) + 12 * nnz + 12 * out                   # k_compact_rows: both row_ptr, entries in and out
    return {"workload": f"S of the {cells}x{cells}-cell mesh (n_rows={n}, nnz={nnz}, kept={out})", "ms": round(ms, 4),
            "gentries_s": round(nnz / ms / 1e6, 2), "algorithmic_bytes": nbytes,
            "k_row_nonzeros_ms": round(c_ms, 4), "k_compact_rows_ms": round(k_ms, 4),
            "roofline": {"kernel": "k_compact_rows", "bound": "hbm", "algorithmic_bytes": kbytes,
                         "achieved": round(kbytes / k_ms / 1e6, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(kbytes / k_ms / 1e6 / hbm, 4), "peak_source": f"{peak_kind} HBM copy bandwidth"}}


# FP64 instructions of one stiffness element in k_tet_atomic / k_tet_stage: 9 edge differences,
# 3 cross products (18), the determinant (3), g_0 (6) and the 10 additions that convert the
# double-float entries back; 1/(6 det), the 10 dot products and their scaling run on the FP32 pipes.
TET_STIFF_FP64_OPS = 46
# FP64 issue rate of GB300: 2 instructions per SM per clock (measured about 0.6 T DFMA/s).
FP64_PEAK_G = 152 * 2 * 2.07


def tetrahedra(feasm, meshgen, torch, flush, hbm, peak_kind, cells: int = 128) -> dict:
    """P1 tetrahedra (the 3-D extension), 128^3-cell cube (jittered, node-permuted): mesh, pattern,
    and S / M^w / M values by FP64 atomics and by the deterministic gather."""
    seed = 13053122 + 6
    m = meshgen.cube_mesh(cells, seed)
    w = torch.tensor(meshgen.vertex_weights3(m, seed), device="cuda")
    q = torch.tensor(m.q, device="cuda")
    me = torch.tensor(m.me, device="cuda")
    ms_mesh = _time_calls(torch, lambda: feasm.TetMesh(q, me, borrow=True).close(), flush, reps=5)
    mesh = feasm.TetMesh(q, me, borrow=True)
    ms_pat = _time_calls(torch, lambda: feasm.TetPattern(mesh).close(), flush, reps=5)
    ms_pat_g = _time_calls(torch, lambda: feasm.TetPattern(mesh, gather=True).close(), flush, reps=5)
    pat = feasm.TetPattern(mesh, gather=True)
    out = pat.new_values()
    res = {}
    for kn, k in (("S", feasm.TET_STIFF), ("Mw", feasm.TET_WMASS), ("M", feasm.TET_MASS)):
        for vn, v in (("atomic", feasm.ATOMIC), ("gather", feasm.GATHER)):
            res[f"{kn}_{vn}_ms"] = round(_time_calls(torch, lambda: feasm.tet_assemble(mesh, pat, k, w, v, out), flush), 4)
    feasm.profile_reset()
    feasm.profile_enable(True)
    _time_calls(torch, lambda: feasm.tet_assemble(mesh, pat, feasm.TET_STIFF, None, feasm.ATOMIC, out), flush)
    feasm.profile_enable(False)
    prof = feasm.profile_read()
    k_ms = prof["k_tet_atomic"][0] / prof["k_tet_atomic"][1]
    ops = TET_STIFF_FP64_OPS * m.nme
    nbytes = 16 * m.nme + 32 * m.nq + 64 * m.nme + 8 * pat.nnz     # me, vertex records, map, values
    fp64_g = feasm.measure_fp64_rate() / 1e9                        # measured FP64 issue rate
    return {"workload": f"S, M^w, M of the {cells}^3-cell cube (nq={m.nq}, nme={m.nme} tetrahedra, nnz={pat.nnz})",
            "mesh_ms": round(ms_mesh, 4), "pattern_ms": round(ms_pat, 4), "pattern_gather_ms": round(ms_pat_g, 4),
            **res, "S_atomic_melem_s": round(m.nme / res["S_atomic_ms"] / 1e3, 1),
            "roofline": {"kernel": "k_tet_atomic<S>", "bound": "hbm", "algorithmic_bytes": nbytes,
                         "achieved": round(nbytes / k_ms / 1e6, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(nbytes / k_ms / 1e6 / hbm, 4), "peak_source": f"{peak_kind} HBM copy bandwidth",
                         "limit": "L2 FP64 atomics (16 per tetrahedron): M, which has no arithmetic, takes as long as S",
                         "fp64": {"algorithmic_ops": ops, "achieved": round(ops / k_ms / 1e6, 1), "peak": round(fp64_g, 1),
                                  "unit": "G FP64 instr/s", "frac": round(ops / k_ms / 1e6 / fp64_g, 4),
                                  "peak_source": "measured: independent FP64 fused multiply-add chains on every SM "
                                                 "(fe_measure_fp64_rate)",
                                  "nominal_peak": round(FP64_PEAK_G, 1),
                                  "nominal_peak_source": "2 FP64 instructions per SM per clock x 152 SMs x 2.07 GHz"}}}


def tet_elasticity(feasm, meshgen, torch, flush, hbm, peak_kind, cells: int = 64) -> dict:
    """3-D linear elasticity (lambda 1.25, mu 0.4) on the 64^3-cell cube (jittered, node-permuted):
    the pattern with the elasticity structure (with and without the ordered variant's lists), and
    K by FP64 atomics and by staged element matrices summed row by row, with the roofline of each."""
    seed = 13053122 + 9
    lam, mu = 1.25, 0.4
    m = meshgen.cube_mesh(cells, seed)
    mesh = feasm.TetMesh(torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"))
    ms_pat = _time_calls(torch, lambda: feasm.TetPattern(mesh, elas=True).close(), flush, reps=5)
    ms_pat_g = _time_calls(torch, lambda: feasm.TetPattern(mesh, gather=True, elas=True).close(), flush, reps=5)
    pat = feasm.TetPattern(mesh, gather=True, elas=True)
    out = torch.empty(pat.elas_nnz, dtype=torch.float64, device="cuda")
    ms = {}
    kern = {}
    for vn, v in (("atomic", feasm.ATOMIC), ("gather", feasm.GATHER)):
        ms[vn] = _time_calls(torch, lambda: feasm.tet_assemble_elas(mesh, pat, lam, mu, v, out), flush)
        feasm.profile_reset()
        feasm.profile_enable(True)
        _time_calls(torch, lambda: feasm.tet_assemble_elas(mesh, pat, lam, mu, v, out), flush)
        feasm.profile_enable(False)
        kern[vn] = {k: round(t / c, 4) for k, (t, c) in feasm.profile_read().items()}
    nnz3 = pat.elas_nnz
    # compulsory bytes: me, the vertex records, the scalar map and row_ptr read once, K written once
    b_atomic = 16 * m.nme + 32 * m.nq + 64 * m.nme + 4 * (m.nq + 1) + 8 * nnz3
    # the ordered variant: me and the vertex records read, the 1152-byte element matrices written
    # and read back once, the incidence lists (12 bytes per incidence) read, K written once
    b_gather = 16 * m.nme + 32 * m.nq + 2 * 1152 * m.nme + 48 * m.nme + 8 * nnz3
    k_at = kern["atomic"]["k_tet_elas_atomic"]
    k_g = sum(kern["gather"].values())

    def roof(name, nbytes, t_ms, limit):
        return {"kernel": name, "bound": "hbm", "algorithmic_bytes": int(nbytes), "achieved": round(nbytes / t_ms / 1e6, 1),
                "peak": hbm, "unit": "GB/s", "frac": round(nbytes / t_ms / 1e6 / hbm, 4),
                "peak_source": f"{peak_kind} HBM copy bandwidth", "limit": limit}
    return {"workload": f"3-D elasticity K of the {cells}^3-cell cube (nq={m.nq}, nme={m.nme} tetrahedra, "
                        f"{3 * m.nq} dofs, nnz={nnz3})",
            "pattern_ms": round(ms_pat, 4), "pattern_gather_ms": round(ms_pat_g, 4),
            "atomic_ms": round(ms["atomic"], 4), "gather_ms": round(ms["gather"], 4),
            "atomic_melem_s": round(m.nme / ms["atomic"] / 1e3, 1), "gather_melem_s": round(m.nme / ms["gather"] / 1e3, 1),
            "kernels_ms": kern,
            "roofline": roof("k_tet_elas_atomic", b_atomic, k_at,
                             "144 FP64 atomics per tetrahedron into values zeroed first, and FP64 element arithmetic"),
            "roofline_gather": roof("k_tet_elas_stage + k_tet_elas_rowsum", b_gather, k_g,
                                    "FP64 element arithmetic in the stage; random 96-byte element rows in the row sums")}


def p2(feasm, meshgen, torch, flush, hbm, peak_kind, cells: int = 1024) -> dict:
    """P2 (quadratic) triangles on the 1024 x 1024-cell square (jittered, node-permuted): the P2
    pattern from the scalar one (with and without the ordered variant's row lists), and the mass
    and stiffness by FP64 atomics and by ordered row sums."""
    seed = 13053122 + 7
    m = meshgen.square_mesh(cells, seed)
    mesh = feasm.Mesh(torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"))
    pat = feasm.Pattern(mesh, map=False)
    ms_pat = _time_calls(torch, lambda: feasm.P2Pattern(mesh, pat).close(), flush, reps=5)
    ms_pat_g = _time_calls(torch, lambda: feasm.P2Pattern(mesh, pat, gather=True).close(), flush, reps=5)
    p2p = feasm.P2Pattern(mesh, pat, gather=True)
    out = p2p.new_values()
    ms_m = _time_calls(torch, lambda: feasm.p2_assemble(mesh, p2p, feasm.P2_MASS, out), flush)
    ms_s = _time_calls(torch, lambda: feasm.p2_assemble(mesh, p2p, feasm.P2_STIFF, out), flush)
    ms_mg = _time_calls(torch, lambda: feasm.p2_assemble(mesh, p2p, feasm.P2_MASS, out, variant=feasm.GATHER), flush)
    ms_sg = _time_calls(torch, lambda: feasm.p2_assemble(mesh, p2p, feasm.P2_STIFF, out, variant=feasm.GATHER), flush)
    feasm.profile_reset()
    feasm.profile_enable(True)
    _time_calls(torch, lambda: feasm.p2_assemble(mesh, p2p, feasm.P2_STIFF, out), flush)
    feasm.profile_enable(False)
    prof = feasm.profile_read()
    k_ms = prof["k_p2_atomic"][0] / prof["k_p2_atomic"][1]
    nbytes = 12 * m.nme + 16 * m.nq + 144 * m.nme + 8 * p2p.nnz          # me, q, map, values
    return {"workload": f"P2 M and S of the {cells}x{cells}-cell square (nq={m.nq}, edges={p2p.n_edges}, "
                        f"dofs={p2p.n_rows}, nme={m.nme}, nnz={p2p.nnz})",
            "pattern_ms": round(ms_pat, 4), "pattern_gather_ms": round(ms_pat_g, 4), "M_ms": round(ms_m, 4),
            "S_ms": round(ms_s, 4), "M_gather_ms": round(ms_mg, 4), "S_gather_ms": round(ms_sg, 4),
            "S_melem_s": round(m.nme / ms_s / 1e3, 1), "k_p2_atomic_S_ms": round(k_ms, 4),
            "roofline": {"kernel": "k_p2_atomic<S>", "bound": "hbm", "algorithmic_bytes": nbytes,
                         "achieved": round(nbytes / k_ms / 1e6, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(nbytes / k_ms / 1e6 / hbm, 4), "peak_source": f"{peak_kind} HBM copy bandwidth",
                         "note": "36 FP64 atomics per element into values zeroed first; the atomics, not DRAM, set the time"}}


def p3(feasm, meshgen, torch, flush, hbm, peak_kind, cells: int = 1024) -> dict:
    """P3 (cubic) triangles on the 1024 x 1024-cell square (jittered, node-permuted): the P3 pattern
    from the scalar one (with and without the ordered variant's row lists), and the mass and
    stiffness by FP64 atomics and by ordered row sums."""
    seed = 13053122 + 8
    m = meshgen.square_mesh(cells, seed)
    mesh = feasm.Mesh(torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"))
    pat = feasm.Pattern(mesh, map=False)
    ms_pat = _time_calls(torch, lambda: feasm.P3Pattern(mesh, pat).close(), flush, reps=5)
    ms_pat_g = _time_calls(torch, lambda: feasm.P3Pattern(mesh, pat, gather=True).close(), flush, reps=5)
    p3p = feasm.P3Pattern(mesh, pat, gather=True)
    out = p3p.new_values()
    res = {}
    for kn, k in (("M", feasm.P3_MASS), ("S", feasm.P3_STIFF)):
        for vn, v in (("atomic", feasm.ATOMIC), ("gather", feasm.GATHER)):
            res[f"{kn}_{vn}_ms"] = round(_time_calls(torch, lambda: feasm.p3_assemble(mesh, p3p, k, out, variant=v), flush), 4)
    feasm.profile_reset()
    feasm.profile_enable(True)
    _time_calls(torch, lambda: feasm.p3_assemble(mesh, p3p, feasm.P3_STIFF, out), flush)
    feasm.profile_enable(False)
    prof = feasm.profile_read()
    k_ms = prof["k_p3_atomic"][0] / prof["k_p3_atomic"][1]
    nbytes = 12 * m.nme + 16 * m.nq + 400 * m.nme + 8 * p3p.nnz          # me, q, map, values
    return {"workload": f"P3 M and S of the {cells}x{cells}-cell square (nq={m.nq}, edges={p3p.n_edges}, "
                        f"dofs={p3p.n_rows}, nme={m.nme}, nnz={p3p.nnz})",
            "pattern_ms": round(ms_pat, 4), "pattern_gather_ms": round(ms_pat_g, 4), **res,
            "S_melem_s": round(m.nme / res["S_atomic_ms"] / 1e3, 1), "k_p3_atomic_S_ms": round(k_ms, 4),
            "roofline": {"kernel": "k_p3_atomic<S>", "bound": "hbm", "algorithmic_bytes": nbytes,
                         "achieved": round(nbytes / k_ms / 1e6, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(nbytes / k_ms / 1e6 / hbm, 4), "peak_source": f"{peak_kind} HBM copy bandwidth",
                         "note": "100 FP64 atomics per element into values zeroed first"}}


def adjoint(feasm, meshgen, torch, flush, hbm, peak_kind) -> dict:
    """dL/dq, dL/dw of L = <G_S, S> + <G_M, M^[w]> on the 1024 x 1024-cell mesh (deterministic gather)."""
    seed = 13053122 + 5
    m = meshgen.square_mesh(1024, seed)
    w = torch.tensor(meshgen.vertex_weights(m, seed), device="cuda")
    mesh = feasm.Mesh(torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"))
    pat = feasm.Pattern(mesh, gather=True)
    GS, GM = (torch.tensor(g, device="cuda") for g in meshgen.upstream_gradients(seed, pat.nnz))
    ms_g = _time_calls(torch, lambda: feasm.adjoint_stiff_wmass(mesh, pat, w, GS, GM, feasm.GATHER), flush)
    ms_a = _time_calls(torch, lambda: feasm.adjoint_stiff_wmass(mesh, pat, w, GS, GM, feasm.ATOMIC), flush)
    ms_f = _time_calls(torch, lambda: feasm.assemble_stiff_wmass(mesh, pat, w, feasm.ROW), flush)
    # compulsory bytes of the backward pass: both upstream arrays, me, q and w read once; dL/dq and
    # dL/dw written once (the element-to-nnz map is the design's, not the method's)
    nbytes = 16 * pat.nnz + 12 * m.nme + 16 * m.nq + 8 * m.nq + 16 * m.nq + 8 * m.nq
    ms_b = min(ms_g, ms_a)
    return {"workload": f"S + M^[w] and adjoint, 1024x1024-cell mesh (nq={m.nq}, nme={m.nme}, nnz={pat.nnz})",
            "forward_ms": round(ms_f, 4), "adjoint_gather_ms": round(ms_g, 4), "adjoint_atomic_ms": round(ms_a, 4),
            "adjoint_melem_s": round(m.nme / ms_b / 1e3, 2),
            "roofline": {"scope": "whole adjoint call (its kernels together), faster variant", "bound": "hbm",
                         "algorithmic_bytes": nbytes, "achieved": round(nbytes / ms_b / 1e6, 1), "peak": hbm,
                         "unit": "GB/s", "frac": round(nbytes / ms_b / 1e6 / hbm, 4),
                         "peak_source": f"{peak_kind} HBM copy bandwidth"}}


def batched(feasm, meshgen, torch, args, hbm, peak_kind) -> dict:
    seed = 13053122 + 4
    meshes = meshgen.batch_meshes(seed)
    fm = [feasm.Mesh(x.q, x.me) for x in meshes]
    fp = [feasm.Pattern(x) for x in fm]
    b = feasm.Batch(fm, fp)
    b.tune()
    variant, block, tile = b.config()
    nme = sum(x.nme for x in meshes)

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_g = timed(b.assemble)
    ms_p = timed(b.assemble_plain)
    # compulsory bytes: me and q read once, S and M values written once, per mesh
    nbytes = sum(12 * x.nme + 16 * x.nq + 16 * p.nnz for x, p in zip(meshes, fp))
    return {"meshes": len(meshes), "nme": nme, "graph_ms": round(ms_g, 4), "plain_ms": round(ms_p, 4),
            "roofline": {"scope": "one graph replay (the persistent launch)", "bound": "hbm", "algorithmic_bytes": nbytes,
                         "achieved": round(nbytes / ms_g / 1e6, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(nbytes / ms_g / 1e6 / hbm, 4), "peak_source": f"{peak_kind} HBM copy bandwidth",
                         "l2": "not flushed between the back-to-back replays; the batch's inputs and outputs (~1.5 GB) "
                               "exceed L2"},
            "graph_melem_s": round(nme / ms_g / 1e3, 2), "plain_melem_s": round(nme / ms_p / 1e3, 2),
            "speedup": round(ms_p / ms_g, 3),
            "tuned": {"variant": {feasm.ROW: "row", feasm.ATOMIC: "atomic"}[variant], "block": block, "tile": tile,
                      "units_per_thread": tile / block,
                      "unit": "rows" if variant == feasm.ROW else "triangles"},
            "what": "S + M (Eq. 1, Eq. 3) of 256 meshes, one graph-replayed persistent launch vs 256 plain "
                    "launches of the same scheme; scheme, block and tile picked by fe_batch_tune"}


def e2e(feasm, torch, m, w, args) -> dict:
    """Same step from pinned host inputs to pinned host CSR outputs through feasm.assemble_host."""
    q_h = torch.tensor(m.q).pin_memory()
    me_h = torch.tensor(m.me).pin_memory()
    w_h = torch.tensor(w).pin_memory()
    pinned = {}
    variant = {"atomic": feasm.ATOMIC, "gather": feasm.GATHER, "row": feasm.ROW}[args.variant]

    def step():
        return feasm.assemble_host("stiff_wmass", q_h.numpy(), me_h.numpy(), w_h.numpy(), variant=variant,
                                   pinned_out=pinned)

    out = step()                         # allocates the pinned outputs, kept in `pinned`
    # at least 10 untimed calls: the library's memory pool reaches its steady size for this call
    # (the device-resident steps before it left blocks of other sizes)
    for _ in range(max(args.warmup - 1, 10)):
        step()
    t = []
    gc.collect()
    gc.disable()                         # no collector pauses inside the timed steps (as timeit)
    try:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            out = step()
            t.append(time.perf_counter() - t0)
    finally:
        gc.enable()
    el = sum(t) / len(t)
    ts = sorted(t)
    h2d = q_h.numel() * 8 + me_h.numel() * 4 + w_h.numel() * 8
    d2h = sum(v.numel() * v.element_size() for k, v in out.items() if k != "nnz")
    return {"value": round(m.nme / el / 1e6, 3), "unit": UNIT, "ms_per_step": round(el * 1e3, 3),
            "median_ms": round(ts[len(ts) // 2] * 1e3, 3), "p90_ms": round(ts[int(0.9 * (len(ts) - 1))] * 1e3, 3),
            "max_ms": round(ts[-1] * 1e3, 3),
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "api": ("feasm.assemble_host('stiff_wmass', ...) from pinned host arrays to pinned host CSR arrays: one "
                    "fe_assemble_stiff_wmass_host call (uploads, validation, pattern, assembly, downloads overlapped "
                    "with the assembly of later row blocks)") if variant == feasm.ROW else
                   ("feasm.assemble_host('stiff_wmass', ...) from pinned host arrays to pinned host CSR arrays: "
                    "mesh, pattern and assembly calls, then the downloads")}


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--variant", choices=["atomic", "gather", "row"], default="row")
    ap.add_argument("--cells", type=int, default=N_CELLS,
                    help="cells per side of the mesh (the workload is 2048; smaller values are for profiling)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-fp64-variants", action="store_true", help="skip the step timed by the FP64 variants")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-other", action="store_true", help="skip the elasticity, adjoint, zero-dropping, tetrahedra and P2 legs")
    ap.add_argument("--traffic", default=os.path.join(ROOT, "profiles", "traffic.json"),
                    help="per-kernel DRAM bytes per launch from an ncu capture (JSON)")
    ap.add_argument("--only", choices=["elasticity", "adjoint", "drop_zeros", "tetrahedra", "p2", "p3", "partition"],
                    help="run this one leg alone and print its object (for profiling; no headline step)")
    ap.add_argument("--tet-cells", type=int, default=128, help="cells per side of the tetrahedra leg's cube")
    ap.add_argument("--p2-cells", type=int, default=1024, help="cells per side of the P2 leg's square")
    ap.add_argument("--part-worlds", default="2,4,8", help="rank counts of the partition leg (comma-separated)")
    ap.add_argument("--part-reps", type=int, default=5, help="timed repetitions of each rank's step in the partition leg")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)    # at least 3 untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_leg(args)
    return run_ours(args)


def run_leg(args) -> int:
    """One extra leg alone, on its own inputs, printed as {"leg": name, ...}."""
    import torch
    from paper_1305_3122_gb300 import feasm, meshgen
    hbm, peak_kind = _peaks()
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.int32, device="cuda")
    if args.only == "elasticity":
        out = elasticity(feasm, meshgen, torch, flush, hbm, peak_kind)
    elif args.only == "adjoint":
        out = adjoint(feasm, meshgen, torch, flush, hbm, peak_kind)
    elif args.only == "tetrahedra":
        out = tetrahedra(feasm, meshgen, torch, flush, hbm, peak_kind, cells=args.tet_cells)
    elif args.only == "p2":
        out = p2(feasm, meshgen, torch, flush, hbm, peak_kind, cells=args.p2_cells)
    elif args.only == "p3":
        out = p3(feasm, meshgen, torch, flush, hbm, peak_kind, cells=args.p2_cells)
    elif args.only == "partition":
        worlds = tuple(int(x) for x in args.part_worlds.split(","))
        out = partition(feasm, meshgen, torch, flush, worlds=worlds, reps=max(args.part_reps, 1))
    else:
        m = meshgen.square_mesh(args.cells, 13053122 + 2)
        mesh = feasm.Mesh(torch.tensor(m.q, device="cuda"), torch.tensor(m.me, device="cuda"))
        pat = feasm.Pattern(mesh, map=False)
        S = feasm.assemble_stiff(mesh, pat, feasm.ROW)
        out = drop_zeros(feasm, torch, pat, S, flush, hbm, peak_kind, cells=args.cells)
    print(json.dumps({"leg": args.only, **out}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
