#!/usr/bin/env python3
"""Benchmark of the NTVS hot path: histories/s per DROP+TVS iteration.

Workload (default): CTP404-like phantom on a 200x200x16 grid of 1x1x2.5 mm voxels,
10M bent proton histories over 360 angles (CSR, int32 columns, FP32 lengths, ~260
entries per row), 20 DROP blocks, N=3 TV steps, alpha=0.75, lambda=2e-4, no TV check.
One step = one NTVS cycle: N TV perturbation steps, a DROP sweep over all 20 blocks and
the FP64 TV of the result.  value = histories / second of one cycle, whole job.

The system (~21 GB) is far larger than L2 (129 MB), so every timed cycle streams it from
HBM; no L2 flush is needed.  Device timing: CUDA events on the stream the library
launches on.  `e2e` times the public C-ABI path from pinned host buffers: load the
system, set the image, run 12 cycles, read the image back.

--impl reference times the FP64 CPU oracle (plain C, one thread) on a bounded sample of
the same workload (its first rows), per step one cycle.

Multi-GPU (torchrun): every rank runs an independent replica of the reconstruction
(reconstructions share nothing); value = all ranks' histories / max rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "histories/s per DROP+TVS iteration"
UNIT = "histories/s"
PARAMS = dict(lam=2e-4, N=3, alpha=0.75, seed=2)
E2E_CYCLES = 12
L2_NOTE = "inputs larger than L2: the system streamed every cycle is ~21 GB vs 129 MB L2"


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ntvs", "reference"], default="ntvs")
    ap.add_argument("--workload", choices=["ctp404_full", "slice2d"], default="ctp404_full")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mixed", type=int, default=1, help="also time BF16 lengths + DELTA16 columns (0: skip)")
    ap.add_argument("--fp64-arith", type=int, default=1,
                    help="also time FP64 arithmetic on the FP32-stored system (0: skip)")
    ap.add_argument("--batched", type=int, default=1, help="also time the batched parameter sweep (0: skip)")
    ap.add_argument("--batch-members", type=int, default=64)
    ap.add_argument("--batch-scale", type=float, default=1.0)
    ap.add_argument("--onthefly", type=int, default=1, help="also time on-the-fly rows on the 256x256x64 grid")
    ap.add_argument("--otf-histories", type=int, default=60_000_000)
    ap.add_argument("--fbp", type=int, default=1,
                    help="also time the initial iterate (FBP + median r=2 + hull) on the workload's histories")
    ap.add_argument("--tile", default="4x4", help="internal voxel tile of the FP32 path (1x1: canonical order)")
    ap.add_argument("--canonical", type=int, default=1,
                    help="also time the canonical voxel order on the same workload (0: skip)")
    ap.add_argument("--check", type=int, default=1,
                    help="also time N = 6 and the TV-reduction check on (N in {3, 6}) (0: skip)")
    ap.add_argument("--cpu-rows", type=int, default=3_000_000,
                    help="single-threaded oracle sample: first rows of the workload")
    ap.add_argument("--cpu-omp-rows", type=int, default=10_000_000,
                    help="OpenMP oracle sample: first rows of the workload (default: all)")
    ap.add_argument("--ref-rows", type=int, default=2_000_000, help="reference arm: rows per step")
    ap.add_argument("--schedule", choices=["auto", "plain", "window", "pipeline"], default="auto",
                    help="DROP kernel schedule (auto picks the windowed one for slice-ordered rows)")
    ap.add_argument("--rows", type=int, default=0,
                    help="profiling case: only the first ROWS histories, in blocks of the full workload's size")
    ap.add_argument("--shard", action="store_true",
                    help="one reconstruction with the rows of every block split over the ranks (strong scaling; "
                         "delta summed per block by an NCCL all-reduce) instead of one replica per rank")
    return ap.parse_args(argv)


def workload_spec(name):
    import synth
    if name == "slice2d":
        return synth.spec_slice_2d(), np.float64
    return synth.spec_ctp404_3d(), np.float32


# ------------------------------------------------------------------ distributed helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """MAX of a float over ranks (identity when world == 1)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 100 ms while the timed region runs; start() returns once the
    first sample is written, so the samples cover the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        self.index = ids[local_rank] if local_rank < len(ids) and ids[local_rank].strip().isdigit() else str(local_rank)
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ntvs_bench_clocks_rank{local_rank}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 3.0 and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ roofline inputs
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def drop_kernel_hash():
    h = hashlib.sha256()
    for f in ("kernels_drop.cuh", "kernels_drop.cu", "kernels_drop_tma.cu", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1803_01112_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def ncu_traffic_per_launch(config, dtype):
    """dram bytes per DROP launch from the committed ncu summary, if it was taken on the
    current kernel source and scaled to this line's workload and configuration; else None."""
    p = os.path.join(ROOT, "profiles", "drop_block_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_src_sha256") != drop_kernel_hash():
        return None
    want = d.get("applies_to") or {}
    have = dict(config, dtype=dtype)
    if not want or any(have.get(k) != v for k, v in want.items()):
        return None
    return d.get("dram_bytes_per_full_launch")


def algorithmic_drop_bytes(s, val_itemsize, b_itemsize, index_bytes=4, extra_row_bytes=0):
    """HBM bytes a DROP block launch must move, per block: each entry's value and column
    once, plus row_ptr (8 B), b and 1/||a||^2 per row (and, for DELTA16, the row's base
    column and exception offset).  x and delta stay in L2."""
    bp = s.block_ptr()
    out = []
    for t in range(len(bp) - 1):
        r0, r1 = int(bp[t]), int(bp[t + 1])
        nnz = int(s.row_ptr[r1] - s.row_ptr[r0])
        out.append(nnz * (val_itemsize + index_bytes) + (r1 - r0) * (8 + 2 * b_itemsize + extra_row_bytes))
    return out


# ------------------------------------------------------------------ CPU oracle timing
def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return os.cpu_count() or 1, model


def time_oracle(spec, vdt, rows, K=1, omp=False):
    """Oracle cycles on the first `rows` histories of the workload (blocks of the same
    size as the workload's), with the single-threaded checker or its OpenMP timing build
    (all host cores).  Returns (seconds per cycle, rows, blocks)."""
    import oracle
    import synth
    rows = min(rows, spec.n_hist)
    s = synth.generate(spec, vdt, rows=(0, rows))
    per = -(-spec.n_hist // spec.n_blocks)
    B = max(1, -(-rows // per))
    bp = np.minimum(np.arange(B + 1, dtype=np.int64) * per, rows)
    val = s.val.astype(np.float64)
    b = s.b.astype(vdt).astype(np.float64)
    shape = (spec.nx, spec.ny, spec.nz)
    prm = oracle.Params(lam=PARAMS["lam"], N=PARAMS["N"], alpha=PARAMS["alpha"], seed=PARAMS["seed"])
    oracle.build(omp=omp)
    t0 = time.perf_counter()
    oracle.ntvs(s.row_ptr, s.col, val, b, bp, shape, prm, K, s.xbar, omp=omp)
    return (time.perf_counter() - t0) / K, rows, B


# ------------------------------------------------------------------ arms
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    spec, vdt = workload_spec(args.workload)
    rows = min(args.ref_rows, spec.n_hist)
    import oracle
    import synth
    s = synth.generate(spec, vdt, rows=(0, rows))
    per = -(-spec.n_hist // spec.n_blocks)
    B = max(1, -(-rows // per))
    bp = np.minimum(np.arange(B + 1, dtype=np.int64) * per, rows)
    val = s.val.astype(np.float64)
    b = s.b.astype(vdt).astype(np.float64)
    shape = (spec.nx, spec.ny, spec.nz)
    prm = oracle.Params(lam=PARAMS["lam"], N=PARAMS["N"], alpha=PARAMS["alpha"], seed=PARAMS["seed"])
    ncores, model = host_cpu()
    oracle.build(omp=True)
    x = s.xbar.copy()
    ell = 0
    for k in range(args.warmup):
        res = oracle.ntvs(s.row_ptr, s.col, val, b, bp, shape, prm, 1, x, k0=k, ell_prev=ell, omp=True)
        x, ell = res.x, res.ell_prev
    t0 = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        res = oracle.ntvs(s.row_ptr, s.col, val, b, bp, shape, prm, 1, x, k0=k, ell_prev=ell, omp=True)
        x, ell = res.x, res.ell_prev
    dt = (time.perf_counter() - t0) / args.steps
    value = rows / dt
    sample = (f"first {rows} of {spec.n_hist} histories ({B} blocks of {per} rows), one NTVS cycle per step, "
              f"FP64 C oracle built with OpenMP on {ncores} threads ({model})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": spec.name, "n_blocks": spec.n_blocks, **PARAMS, "tv_check": False},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle", "sample": sample,
                             "cpu_model": model},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def batch_members(n_members, seed=4, scale=1.0):
    """Members of the batched sweep: grids nx = ny in {64..128} (step 8), nz in {8..16},
    histories U(0.5, 4) * 1e6 * scale (bent paths over 90 angles, 4-8 random inserts,
    20 blocks), and (N, alpha, lambda) drawn from {1..6} x {0.5, 0.6, 0.75, 0.9} x
    {1e-4, 2e-4, 5e-4} without repetition."""
    import synth
    rng = np.random.default_rng(seed)
    combos = [(N, a, l) for N in range(1, 7) for a in (0.5, 0.6, 0.75, 0.9) for l in (1e-4, 2e-4, 5e-4)]
    pick = rng.choice(len(combos), size=n_members, replace=n_members > len(combos))
    out = []
    for k in range(n_members):
        n = int(rng.integers(8, 17)) * 8
        nz = int(rng.integers(8, 17))
        m = max(1000, int(rng.uniform(0.5, 4.0) * 1e6 * scale))
        N, a, l = combos[pick[k]]
        out.append((synth.spec_batch_member(1000 + k, n, n, nz, m), dict(lam=l, N=N, alpha=a, seed=2000 + k)))
    return out


def batch_cycle_bytes(members):
    """Algorithmic HBM bytes of one batched cycle: per member each stored entry's value
    and column once, 16 B per row (row_ptr, b, 1/||a||^2), and per voxel 44 B per TV step
    (gradient: x split read, g written; step: x, g read, x and its three FP32 copies
    written), 32 B per DROP block (x, delta, 1/s read; x, its copy, delta written) and 8 B
    for phi."""
    return sum(8.0 * nnz + 16.0 * M + V * (44.0 * N + 32.0 * B + 8.0) for (nnz, M, V, N, B) in members)


def run_batched_variant(args, ntvs, local, stream, world, device):
    """The batched parameter sweep at its stated size.  Members are generated as path
    records on the host; on the device b = (A x*)(1 + 0.01 z) is formed by projecting the
    phantom through the traced paths, and ntvs_batch_add_paths traces and stores the rows.
    The same members run once without and once with the TV check."""
    import time

    import torch

    import synth
    members = batch_members(args.batch_members, scale=args.batch_scale)
    t_gen = t_load = 0.0
    dev = []   # (spec, params, paths on the device, b on the device, xbar)
    for sp, prm in members:
        t0 = time.perf_counter()
        P = synth.generate_paths(sp, with_rhs=False)
        t1 = time.perf_counter()
        pd = torch.from_numpy(P.paths).to(device)
        shape, voxel = (sp.nx, sp.ny, sp.nz), (sp.dx, sp.dy, sp.dz)
        r = ntvs.Reconstructor(local, stream.cuda_stream)
        r.load_paths(shape, voxel, pd, torch.zeros(sp.n_hist, dtype=torch.float32, device=device),
                     n_blocks=sp.n_blocks, n_seg=sp.n_seg, min_len=sp.min_len)
        bclean = torch.empty(sp.n_hist, dtype=torch.float32, device=device)
        r.forward_project(P.xstar, out=bclean)
        r.close()
        gen = torch.Generator(device=device).manual_seed(sp.seed)
        b = bclean * (1.0 + sp.noise_sigma * torch.randn(sp.n_hist, generator=gen, device=device))
        del bclean
        torch.cuda.synchronize(device)
        t_gen += t1 - t0
        t_load += time.perf_counter() - t1
        dev.append((sp, prm, pd, b, P.xbar))
    lines = []
    for check in (False, True):
        bt = ntvs.Batch(local, stream.cuda_stream)
        t0 = time.perf_counter()
        for sp, prm, pd, b, xbar in dev:
            bt.add_paths((sp.nx, sp.ny, sp.nz), (sp.dx, sp.dy, sp.dz), pd, b, sp.n_blocks,
                         ntvs.Params(tv_check=check, **prm), xbar, n_seg=sp.n_seg, min_len=sp.min_len)
        t_add = time.perf_counter() - t0
        t0 = time.perf_counter()
        bt.finalize(max_cycles=args.warmup + args.steps + 1)
        t_fin = time.perf_counter() - t0
        bt.run(args.warmup)
        bt.sync()
        barrier(world, device)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        bt.run(args.steps)
        g1.record(stream)
        bt.sync()
        ms_b = max_over_ranks(g0.elapsed_time(g1), world, device)
        bst = bt.stats()
        tuning = bt.tuning()
        mems = [bt.member(i) for i in range(len(dev))]
        sizes = [(bt.sizes(i)[1], sp.n_hist, sp.V, prm["N"], sp.n_blocks)
                 for i, (sp, prm, _, _, _) in enumerate(dev)]
        total_rows = sum(sp.n_hist for sp, *_ in dev)
        cyc_bytes = batch_cycle_bytes(sizes)
        ms_cycle = ms_b / args.steps
        peak, peak_src = measured_peaks()
        ach = cyc_bytes / (ms_cycle / 1e3) / 1e9
        seq = None
        if not check:
            seq = sequential_sample(args, ntvs, local, stream, world, device, bt, dev, min(4, len(dev)))
        bt.close()
        line = {"name": f"batched sweep of {len(dev)} members" + (", TV-reduction check on" if check else ""),
                "value": world * total_rows * args.steps / (ms_b / 1e3), "unit": UNIT, "ms_per_step": ms_cycle,
                "members": len(dev), "total_histories": int(total_rows), "total_nnz": int(bst["total_nnz"]),
                "kernels_per_cycle": int(bst["kernels_per_cycle"]),
                "gpu_launches_per_step": bst["n_launches"] / max(bst["cycles"], 1),
                "schedule": {"rows_per_item": bst["rows_per_item"], "window_floats": bst["window_floats"],
                             "ctas": bst["ctas"], "ctas_per_sm": bst["ctas_per_sm"],
                             "lanes_per_row": [bst["lanes_per_row_min"], bst["lanes_per_row"]],
                             "lanes_per_row_all": bst["lanes_per_row_all"],
                             "tuning_ms": [[r, w, c, l, round(ms, 3)] for r, w, c, l, ms in tuning]},
                "tries_per_step": sum(m["n_tries"] for m in mems) / max(sum(m["n_steps"] for m in mems), 1),
                "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                             "algorithmic_bytes_per_cycle": cyc_bytes, "peak_source": peak_src,
                             "kernel": "batch_cycle_kernel (the whole cycle is one launch)"},
                "load_seconds": {"host_path_generation": t_gen, "device_b_projection": t_load,
                                 "add_paths_tracing_and_prep": t_add, "finalize_and_tuning": t_fin},
                "recipe": "nx=ny in {64..128}, nz in {8..16}, 0.5-4M bent histories each (x batch_scale), 4-8 "
                          "random inserts, 20 blocks, (N, alpha, lambda) from the 72-combination sweep; rows traced "
                          "on the device from path records"}
        if seq is not None:
            line.update(seq)
        lines.append(line)
    return lines


def sequential_sample(args, ntvs, local, stream, world, device, bt, dev, n):
    """The first n members one after another through single FP32 contexts loaded with the
    batch's stored rows: time per cycle, scaled to all members by their histories."""
    import torch
    seq_ms, rows_n = 0.0, 0
    for i in range(n):
        sp, prm, pd, b, xbar = dev[i]
        rp, col, val = bt.rows(i)
        r = ntvs.Reconstructor(local, stream.cuda_stream)
        r.load((sp.nx, sp.ny, sp.nz), rp, col, val, b.cpu().numpy(), n_blocks=sp.n_blocks)
        r.set_params(**prm)
        r.set_image(xbar)
        r.run(1)
        r.sync()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        r.run(args.steps)
        h1.record(stream)
        torch.cuda.synchronize(device)
        seq_ms += h0.elapsed_time(h1)
        rows_n += sp.n_hist
        r.close()
    total = sum(d[0].n_hist for d in dev)
    seq_all = max_over_ranks(seq_ms * total / rows_n, world, device)
    return {"sequential_value": world * total * args.steps / (seq_all / 1e3),
            "sequential_sample": f"first {n} members through single contexts, scaled by histories"}


def otf_kernel_hash():
    h = hashlib.sha256()
    for f in ("kernels_onthefly.cu", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1803_01112_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def otf_profile_fractions():
    """SM and L2 throughput (% of peak) of the on-the-fly DROP kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "otf_drop_kernel_fractions.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_src_sha256") != otf_kernel_hash():
        return None
    return {k: d[k] for k in ("sm_throughput_pct", "l2_throughput_pct", "dram_throughput_pct", "source")}


def run_onthefly_variant(args, ntvs, local, stream, world, device):
    """256x256x64 grid (0.8x0.8x1.25 mm), bent paths over 720 angles, 40 blocks, N = 4,
    rows traced in every sweep from 44-byte history records (10 path floats + b).  The
    path records come from the generator; b = (A x*)(1 + sigma z) is formed on the device by
    projecting the phantom through the same traced paths (ntvs_forward_project) with the
    generator's 1 % Gaussian noise from a seeded device generator."""
    import torch

    import synth
    spec = synth.spec_large_onthefly(n_hist=args.otf_histories)
    pr = synth.generate_paths(spec, with_rhs=False)
    paths = torch.from_numpy(pr.paths).to(device)
    shape, voxel = (spec.nx, spec.ny, spec.nz), (spec.dx, spec.dy, spec.dz)
    kw = dict(n_blocks=spec.n_blocks, n_seg=spec.n_seg, min_len=spec.min_len)
    r = ntvs.Reconstructor(local, stream.cuda_stream)
    r.load_paths(shape, voxel, paths, torch.zeros(spec.n_hist, dtype=torch.float32, device=device), **kw)
    bclean = torch.empty(spec.n_hist, dtype=torch.float32, device=device)
    r.forward_project(pr.xstar, out=bclean)
    gen = torch.Generator(device=device).manual_seed(spec.seed)
    b = bclean * (1.0 + spec.noise_sigma * torch.randn(spec.n_hist, generator=gen, device=device))
    del bclean
    r.load_paths(shape, voxel, paths, b, **kw)
    r.set_params(lam=2e-4, N=4, alpha=0.75, seed=5)
    r.set_image(pr.xbar)
    r.run(1)
    r.sync()
    steps = max(1, min(args.steps, 5))
    barrier(world, device)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r.run(steps)
    e1.record(stream)
    torch.cuda.synchronize(device)
    ms = max_over_ranks(e0.elapsed_time(e1), world, device)
    r.set_profiling(True)
    r.run(1)
    prof = r.profile()
    r.close()
    avg = prof["drop_block_ms"] / max(prof["drop_block_launches"], 1)
    hbm_bytes = 44.0 * spec.n_hist / spec.n_blocks + 16.0 * spec.n_hist / spec.n_blocks   # records + 1/||a||^2 etc.
    return {"name": "on-the-fly rows, 256x256x64, 720 angles, 40 blocks, N=4",
            "value": world * spec.n_hist * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "histories": spec.n_hist, "drop_launch_ms": avg,
            "kernel_ms_per_step": {k: prof[k] for k in ("drop_block_ms", "drop_apply_ms", "tv_ms")},
            "tv_share": prof["tv_ms"] / max(prof["drop_block_ms"] + prof["drop_apply_ms"] + prof["tv_ms"], 1e-12),
            "hbm_gb_s_per_drop_launch": hbm_bytes / (avg / 1e3) / 1e9,
            "bound": "alu + L2 atomics (path tracing; 60 B of HBM per history and launch)",
            "ncu_fractions": otf_profile_fractions(),
            "note": "b = (A x*)(1 + 0.01 z) formed on the device through the traced paths"}


def run_fbp_variant(args, ntvs, stream, world, device, spec, b):
    """The initial iterate x-bar of the workload's own histories: chord binning into 180
    angle bins centred on whole degrees x 160 lateral bins of 1 mm x the workload's
    slices, Ram-Lak filter, back-projection onto its grid, median filter r = 2 per slice,
    threshold hull at 0.3 (include/ntvs_fbp.h).  Timed with CUDA events on the stream,
    whole chain and stage by stage."""
    import math

    import torch

    import synth
    pr = synth.generate_paths(spec, with_rhs=False)
    paths = torch.from_numpy(pr.paths).to(device)
    wepl = torch.from_numpy(np.ascontiguousarray(b, np.float64)).to(device)
    del pr
    g = ntvs.fbp_geom(spec.nx, spec.ny, spec.nz, spec.dx, spec.dy, spec.dz, 180, 160, 1.0, theta0=-math.pi / 360)
    S, V = spec.nz * 180 * 160, spec.V
    out = torch.empty(V, dtype=torch.float64, device=device)
    ws = torch.empty(ntvs.ntvs_fbp_workspace_bytes(g), dtype=torch.uint8, device=device)
    sino = torch.empty(S, dtype=torch.float64, device=device)
    cnt = torch.empty(S, dtype=torch.int32, device=device)
    q = torch.empty(S, dtype=torch.float64, device=device)
    img = torch.empty(V, dtype=torch.float64, device=device)
    cs = stream.cuda_stream

    def chain():
        ntvs.ntvs_initial_iterate(g, paths, wepl, out, median_radius=2, use_hull=True, tau=0.3, workspace=ws,
                                  stream=cs)

    stages = [("bin", lambda: ntvs.ntvs_fbp_bin(g, paths, wepl, sino, cnt, stream=cs)),
              ("filter", lambda: ntvs.ntvs_fbp_filter(g, sino, q, stream=cs)),
              ("backproject", lambda: ntvs.ntvs_fbp_backproject(g, q, img, stream=cs)),
              ("median_hull", lambda: ntvs.ntvs_median_filter(img, out, (spec.nx, spec.ny, spec.nz), 2,
                                                              use_hull=True, tau=0.3, stream=cs))]
    for _ in range(3):
        chain()
    reps = 10
    torch.cuda.synchronize(device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 + 2 * len(stages))]
    ev[0].record(stream)
    for _ in range(reps):
        chain()
    ev[1].record(stream)
    stage_ms = {}
    for i, (name, fn) in enumerate(stages):
        ev[2 + 2 * i].record(stream)
        for _ in range(reps):
            fn()
        ev[3 + 2 * i].record(stream)
    torch.cuda.synchronize(device)
    ms = max_over_ranks(ev[0].elapsed_time(ev[1]) / reps, world, device)
    for i, (name, _) in enumerate(stages):
        stage_ms[name] = ev[2 + 2 * i].elapsed_time(ev[3 + 2 * i]) / reps
    # back-projection: per (voxel, angle) 12 FP64 operations (two products and sums for t,
    # one FMA for u, floor, three for the weights, two products and two sums)
    bp_flops = 12.0 * V * 180
    res = {"name": "initial iterate: FBP + median r=2 + hull, " + spec.name, "value": world * spec.n_hist / (ms / 1e3),
           "unit": "histories/s", "ms_per_call": ms, "histories": spec.n_hist, "bins": [spec.nz, 180, 160],
           "stage_ms": stage_ms, "gpu_launches_per_call": 7,
           "backproject_fp64_gflops": bp_flops / (stage_ms["backproject"] / 1e3) / 1e9,
           "arithmetic": "f64"}
    del paths, wepl, out, ws, sino, cnt, q, img
    return res


def shard_system(spec, vdt, rank, world):
    """This rank's rows of the workload: block t's rows cut into `world` contiguous runs,
    run `rank` of each, generated run by run (no rank builds the whole system)."""
    import synth
    per = -(-spec.n_hist // spec.n_blocks)
    parts, bp = [], [0]
    for t in range(spec.n_blocks):
        b0, b1 = min(t * per, spec.n_hist), min((t + 1) * per, spec.n_hist)
        lo, hi = b0 + (b1 - b0) * rank // world, b0 + (b1 - b0) * (rank + 1) // world
        parts.append(synth.generate(spec, vdt, rows=(lo, hi)) if hi > lo else None)
        bp.append(bp[-1] + hi - lo)
    live = [q for q in parts if q is not None]
    rp = [np.zeros(1, np.int64)]
    off = 0
    for q in live:
        rp.append(q.row_ptr[1:] + off)
        off += int(q.row_ptr[-1])
    col = np.concatenate([q.col for q in live])
    val = np.concatenate([q.val for q in live])
    b = np.concatenate([q.b for q in live]).astype(vdt)
    return np.concatenate(rp), col, val, b, np.asarray(bp, np.int64), live[0].xbar


def run_sharded(args):
    """One reconstruction of the workload row-sharded over the ranks: every rank holds its
    runs of every block's rows, the TV steps run on every rank on identical images, and
    each DROP block's delta (and residual) is summed over the ranks by an NCCL all-reduce
    on the library's stream before it is applied with the global hit counts.  Strong
    scaling: value = the workload's histories per cycle / max rank time.  With one rank
    the collective is the identity."""
    import torch

    import paper_1803_01112_gb300 as ntvs
    from paper_1803_01112_gb300 import _ffi
    rank, world, local = dist_env()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    ntvs.lib()
    spec, vdt = workload_spec(args.workload)
    rp, col, val, b, sbp, xbar = shard_system(spec, vdt, rank, world)
    stream = torch.cuda.Stream(device)
    tile = tuple(int(v) for v in args.tile.lower().split("x"))
    r = ntvs.Reconstructor(local, stream.cuda_stream).set_voxel_tile(*tile)
    r.load((spec.nx, spec.ny, spec.nz), rp, col, val, b, n_blocks=len(sbp) - 1, block_ptr=sbp)
    fn = ntvs.torch_allreduce(device=local) if world > 1 else _ffi.ALLREDUCE_FN(lambda *a: 0)
    r.set_allreduce(fn)
    r.set_params(**PARAMS)
    r.set_image(xbar.astype(vdt))
    r.run(args.warmup)
    r.sync()
    barrier(world, device)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        r.run(1)
    e1.record(stream)
    torch.cuda.synchronize(device)
    ms = max_over_ranks(e0.elapsed_time(e1), world, device)
    launches = r.stats()["n_launches"]
    r.close()
    if rank == 0:
        line = {"metric": METRIC, "value": spec.n_hist * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f32" if vdt == np.float32 else "f64", "data": "synthetic",
                "config": {"workload": spec.name, "histories": spec.n_hist, "n_blocks": spec.n_blocks, **PARAMS,
                           "tv_check": False, "l2": L2_NOTE,
                           "parallelism": f"row-sharded DROP over {world} GPU(s): NCCL all-reduce of delta per block"},
                "gpu_launches": launches,
                "note": "measured only with one GPU here (identity collective); multi-GPU runs unmeasured on hardware"}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_ntvs(args):
    import torch

    import synth
    import paper_1803_01112_gb300 as ntvs

    rank, world, local = dist_env()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    ntvs.lib()
    spec, vdt = workload_spec(args.workload)

    def pinned(shape, dt):
        t = torch.empty(int(np.prod(shape)), dtype=getattr(torch, np.dtype(dt).name), pin_memory=True)
        return t.numpy()

    n_blocks = spec.n_blocks
    if args.rows:
        per = -(-spec.n_hist // spec.n_blocks)
        s = synth.generate(spec, vdt, alloc=pinned, rows=(0, min(args.rows, spec.n_hist)))
        n_blocks = max(1, -(-s.M // per))
        spec = spec.replace(n_hist=s.M, n_blocks=n_blocks, name=f"{spec.name}_first{s.M}rows")
        s.spec = spec
    else:
        s = synth.generate(spec, vdt, alloc=pinned)
    b = pinned((s.M,), vdt)
    b[:] = s.b.astype(vdt)
    x0 = pinned((spec.V,), vdt)
    x0[:] = s.xbar.astype(vdt)
    shape = (spec.nx, spec.ny, spec.nz)
    stream = torch.cuda.Stream(device)   # the library launches on this stream; events are recorded on it

    tile = tuple(int(v) for v in args.tile.lower().split("x"))
    r = ntvs.Reconstructor(local, stream.cuda_stream).set_voxel_tile(*tile)
    sched = {"auto": 0, "plain": 1, "window": 2, "pipeline": 3}[args.schedule]
    r.load(shape, s.row_ptr, s.col, s.val, b, n_blocks=spec.n_blocks, schedule=sched)
    r.set_params(**PARAMS)
    r.set_image(x0)
    st0 = r.stats()
    r.run(args.warmup)
    r.sync()
    torch.cuda.synchronize(device)

    # ---- timed region: K cycles, events on the launching stream (no per-launch events here:
    # an event recorded around each of the ~47 launches of a cycle costs ~2.5 % of it)
    clocks = ClockSampler(local)
    barrier(world, device)
    torch.cuda.synchronize(device)
    launches0 = r.stats()["n_launches"]
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        r.run(1)
    e1.record(stream)
    torch.cuda.synchronize(device)
    ms_local = e0.elapsed_time(e1)
    clk = clocks.stop()
    barrier(world, device)
    launches = r.stats()["n_launches"] - launches0
    ms = max_over_ranks(ms_local, world, device)
    ms_step = ms / args.steps
    value = world * spec.n_hist * args.steps / (ms / 1e3)

    # ---- second timed pass of K cycles with CUDA events around every launch on the same
    # stream: per-kernel device time, and the DROP kernel's average launch for the roofline
    barrier(world, device)
    torch.cuda.synchronize(device)
    r.set_profiling(True)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        r.run(1)
    p1.record(stream)
    torch.cuda.synchronize(device)
    ms_prof_pass = p0.elapsed_time(p1)
    prof = r.profile()
    r.set_profiling(False)

    # ---- roofline of the dominant kernel (DROP gather + scatter)
    vsz = np.dtype(vdt).itemsize
    blk_bytes = algorithmic_drop_bytes(s, vsz, vsz)
    avg_bytes = float(np.mean(blk_bytes))
    avg_ms = prof["drop_block_ms"] / max(prof["drop_block_launches"], 1)
    achieved = avg_bytes / (avg_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    kname = {2: "drop_block_window_kernel", 3: "drop_pipe_kernel"}.get(st0["drop_schedule"], "drop_block_kernel")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": ncu_traffic_per_launch(
                    {"workload": spec.name, "storage": "csr32",
                     "drop_schedule": {1: "plain", 2: "window", 3: "pipeline"}.get(st0["drop_schedule"]),
                     "voxel_tile": f"{st0['voxel_tile_x']}x{st0['voxel_tile_y']}"},
                    "f32" if vdt == np.float32 else "f64"),
                "kernel": kname,
                "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch": avg_bytes,
                "avg_launch_ms": avg_ms,
                "timing": f"CUDA events around every launch in a second timed pass of {args.steps} cycles "
                          f"({ms_prof_pass / args.steps:.3f} ms per cycle with the events)"}
    kernel_ms = {k: prof[k] / args.steps for k in ("drop_block_ms", "drop_apply_ms", "tv_ms")}

    # ---- end to end through the C ABI from pinned host buffers; measured before the variant
    # legs, whose many device allocations and frees slow later multi-GB allocations down
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        h2d = s.row_ptr.nbytes + s.col.nbytes + s.val.nbytes + b.nbytes + x0.nbytes
        out = pinned((spec.V,), vdt)
        times, split = [], []
        for _ in range(args.e2e_steps):
            barrier(world, device)
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            re = ntvs.Reconstructor(local, stream.cuda_stream).set_voxel_tile(*tile)
            re.load(shape, s.row_ptr, s.col, s.val, b, n_blocks=spec.n_blocks, schedule=sched)
            t_l = time.perf_counter()
            re.set_params(**PARAMS)
            re.set_image(x0)
            re.run(E2E_CYCLES)
            ntvs.ntvs_get_image(re.handle, out)
            t1 = time.perf_counter()
            re.close()
            times.append(max_over_ranks(t1 - t0, world, device))
            split.append((t_l - t0, t1 - t_l))
        t_e2e = statistics.mean(times)
        # the floor under the load: a plain copy of the same column and value bytes from the
        # same pinned host buffers into device memory on two streams (what the loader
        # overlaps its device work with)
        floor = None
        try:
            cs = [torch.cuda.Stream(device), torch.cuda.Stream(device)]
            srcs = [torch.from_numpy(a.reshape(-1).view(np.uint8)) for a in (s.col, s.val)]
            dsts = [torch.empty(t.numel(), dtype=torch.uint8, device=device) for t in srcs]
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            for k, (dst_t, src_t) in enumerate(zip(dsts, srcs)):
                with torch.cuda.stream(cs[k]):
                    dst_t.copy_(src_t, non_blocking=True)
            torch.cuda.synchronize(device)
            floor = time.perf_counter() - t0
            del dsts
        except RuntimeError:   # not enough device memory beside the context's
            floor = None
        torch.cuda.empty_cache()   # the library allocates with cudaMalloc, not from torch's cache
        e2e = {"value": world * spec.n_hist * E2E_CYCLES / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(out.nbytes), "cycles_per_step": E2E_CYCLES,
               "seconds_per_step": t_e2e, "load_seconds": statistics.mean(x for x, _ in split),
               "run_and_readback_seconds": statistics.mean(y for _, y in split),
               "load_seconds_each": [round(x, 4) for x, _ in split],
               "h2d_copy_floor_seconds": floor}

    # ---- variants on the same workload: canonical voxel order, N = 6 and the TV-reduction
    # check (the 2 x 2 of N in {3, 6} x check off/on), FP64 arithmetic on the FP32-stored
    # system, and mixed precision (FP32 arithmetic): BF16 lengths with int32 or DELTA16 columns
    variants = []
    cases = []

    def case(name, **kw):
        c = dict(name=name, vals=s.val, storage=ntvs.NTVS_CSR32, vb=vsz, ib=4, tile=tile, prm=PARAMS,
                 compute=ntvs.NTVS_F32)
        c.update(kw)
        cases.append(c)

    if vdt == np.float32:
        if args.canonical and tile != (1, 1):
            case("fp32, canonical voxel order", tile=(1, 1))
        if args.check:
            case("fp32, TV-reduction check on", prm=dict(PARAMS, tv_check=True))
            case("fp32, N=6", prm=dict(PARAMS, N=6))
            case("fp32, N=6, TV-reduction check on", prm=dict(PARAMS, N=6, tv_check=True))
        if args.fp64_arith:
            case("fp64 arithmetic on fp32 storage", compute=ntvs.NTVS_F64)
        if args.mixed:
            import torch as _t
            vbf = _t.from_numpy(s.val).to(_t.bfloat16)
            case("bf16 lengths + int32 columns", vals=vbf, vb=2)
            case("bf16 lengths + delta16 columns", vals=vbf, vb=2, ib=2.125, storage=ntvs.NTVS_DELTA16)
    for c in cases:
        rm = ntvs.Reconstructor(local, stream.cuda_stream).set_voxel_tile(*c["tile"])
        rm.set_compute_dtype(c["compute"])
        rm.load(shape, s.row_ptr, s.col, c["vals"], b, n_blocks=spec.n_blocks, storage=c["storage"], schedule=sched)
        rm.set_params(**c["prm"])
        rm.set_image(x0)
        stm = rm.stats()
        rm.run(args.warmup)
        rm.sync()
        barrier(world, device)
        torch.cuda.synchronize(device)
        rm.set_profiling(True)
        n0 = rm.stats()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            rm.run(1)
        f1.record(stream)
        torch.cuda.synchronize(device)
        msm = max_over_ranks(f0.elapsed_time(f1), world, device)
        pm = rm.profile()
        stf = rm.stats()
        rm.close()
        b_item = 8 if stm["compute_dtype"] == ntvs.NTVS_F64 else 4   # b and 1/||a||^2 per row
        # DELTA16: 2-byte offsets plus a 4-byte base per 32 entries, 128 bytes per escaped chunk
        bytes_m = float(np.mean(algorithmic_drop_bytes(s, c["vb"], b_item, index_bytes=c["ib"]))) + \
            128.0 * stm["n_escaped"] / spec.n_blocks
        avg_m = pm["drop_block_ms"] / max(pm["drop_block_launches"], 1)
        ach = bytes_m / (avg_m / 1e3) / 1e9
        steps_done = max(stf["n_steps"] - n0["n_steps"], 1)
        variants.append({"name": c["name"], "value": world * spec.n_hist * args.steps / (msm / 1e3), "unit": UNIT,
                         "ms_per_step": msm / args.steps, "vs_headline": ms / msm,
                         "N": c["prm"]["N"], "tv_check": bool(c["prm"].get("tv_check", False)),
                         "compute_dtype": "f64" if stm["compute_dtype"] == ntvs.NTVS_F64 else "f32",
                         "voxel_tile": f"{stm['voxel_tile_x']}x{stm['voxel_tile_y']}",
                         "tries_per_step": (stf["n_tries"] - n0["n_tries"]) / steps_done,
                         "drop_schedule": {1: "plain", 2: "window", 3: "pipeline"}.get(stm["drop_schedule"]),
                         "gpu_launches_per_step": (stf["n_launches"] - n0["n_launches"]) / args.steps,
                         "kernel_ms_per_step": {k: pm[k] / args.steps for k in ("drop_block_ms", "drop_apply_ms",
                                                                                "tv_ms")},
                         "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                      "frac": ach / peak, "algorithmic_bytes_per_launch": bytes_m,
                                      "avg_launch_ms": avg_m}})
    cases = vbf = None

    # ---- batched reconstructions: a parameter sweep over members of uneven size
    if args.batched:
        variants.extend(run_batched_variant(args, ntvs, local, stream, world, device))

    # ---- on-the-fly rows on the large grid
    if args.onthefly:
        variants.append(run_onthefly_variant(args, ntvs, local, stream, world, device))

    # ---- the initial iterate from the same histories
    if args.fbp:
        variants.append(run_fbp_variant(args, ntvs, stream, world, device, spec, s.b))

    # ---- CPU oracle baseline (rank 0, one GPU only): the OpenMP timing build of the oracle on
    # all host cores over the whole workload, and the single-threaded checker on a sample
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ncores, model = host_cpu()
        sec, rows, B = time_oracle(spec, vdt, args.cpu_omp_rows, omp=True)
        sec1, rows1, B1 = time_oracle(spec, vdt, args.cpu_rows)
        cpu = {"value": rows / sec, "unit": UNIT, "cores": ncores, "kind": "oracle", "cpu_model": model,
               "sample": f"first {rows} of {spec.n_hist} histories ({B} blocks), one NTVS cycle, FP64 C oracle "
                         f"built with OpenMP on {ncores} threads (same source as the checker)",
               "single_thread": {"value": rows1 / sec1, "cores": 1,
                                 "sample": f"first {rows1} histories ({B1} blocks), one cycle, the checker build"}}

    r.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if vdt == np.float32 else "f64", "data": "synthetic",
                "config": {"workload": spec.name, "grid": [spec.nx, spec.ny, spec.nz], "histories": spec.n_hist,
                           "nnz": s.nnz, "n_blocks": spec.n_blocks, **PARAMS, "tv_check": False,
                           "storage": "csr32", "l2": L2_NOTE,
                           "drop_schedule": {1: "plain", 2: "window", 3: "pipeline"}.get(st0["drop_schedule"]),
                           "lanes_per_row": st0["lanes_per_row"],
                           "voxel_tile": f"{st0['voxel_tile_x']}x{st0['voxel_tile_y']}",
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "kernel_ms_per_step": kernel_ms, "clocks": clk, "variants": variants}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.shard:
        return run_sharded(args)
    return run_ntvs(args)


if __name__ == "__main__":
    sys.exit(main())
