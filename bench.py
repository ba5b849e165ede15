#!/usr/bin/env python3
"""Benchmark of the hot path: Y = mask(P) * (H P), P^T Y and P^T P.

One step = fe_apply_H_gram (apply, P^T Y, P^T P) on the paper-scale p=2
workload (64x40x40 Q2 cells, 846,369 DoFs x 320 orbitals in 38 column
blocks, ~20% block fill), FP32 cell arithmetic with FP64 Gram accumulation;
the FP64 path is timed beside it.  Inputs are resident in HBM when the timed
region starts; P and Y (215 MB each in FP32) are larger than L2, so no flush
is needed between steps.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H·P DoF·columns/s + Gram GFLOP/s, FP32-mixed vs FP64 at tol; p50/p99"
UNIT = "DoF*columns/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="p2")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-p4", action="store_true", help="skip the p = 4 workload beside p = 2")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--serving", type=int, default=2000, help="requests per load point of the serving run (0: skip)")
    ap.add_argument("--serving-pool", type=int, default=6, help="distinct workloads in the serving mix")
    ap.add_argument("--serving-small", dest="serving_full", action="store_false",
                    help="draw serving meshes from the two smaller sizes and 32-320 orbitals only")
    ap.add_argument("--serving-loads", type=lambda s: [float(x) for x in s.split(",")], default=[0.5, 0.8, 1.2, 2.0],
                    help="offered loads, as multiples of the one-at-a-time rate (comma-separated)")
    ap.add_argument("--cpu-blocks", type=int, default=1000,
                    help="column blocks in the CPU oracle sample (default: all of them)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: no data-path collective)
# ---------------------------------------------------------------------------
def dist_init(n, backend=None):
    """Rank, world size and local rank from the torchrun environment; with
    more than one rank, a process group (NCCL when CUDA is present, else
    gloo) used only for the timing barrier and the max over ranks."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(n_dofs, n_cols, ms_step, world):
    """Weak scaling over replicas: every rank processes the same workload, so
    the job processes world * N * M DoF-columns per (max over ranks) step."""
    return world * n_dofs * n_cols / (ms_step * 1e-3)


# ---------------------------------------------------------------------------
# SM clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="fe_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def _oracle_worker(cfg_name, pick, fp32, conn):
    """One CPU worker of the oracle team: sets up the FP64 oracle (assembled
    operator on the rows of its column blocks' pattern, the orbitals of its
    column blocks) once, then on each "go" times Y = mask(P) (H P), P^T Y and
    P^T P for its columns and sends the seconds back."""
    import numpy as np
    from oracle import fe_oracle as O
    from synth import inputs
    cfg = inputs.get_config(cfg_name)
    mesh = O.BoxMesh.from_config(cfg)
    blk = O.Blocking(mesh)
    centres = inputs.orbital_centres(cfg)
    perm, ptr = O.column_blocks(blk, centres, cfg.n_col_blocks)
    orbs = {int(perm[j]) for c in pick for j in range(ptr[c], ptr[c + 1])}
    mv = O.build_orbitals(mesh, cfg, centres, round_fp32=fp32, orbitals=orbs)
    pat = O.block_pattern(blk, mv, perm, ptr)
    cb_of_orb = O.entry_mask(blk, pat, perm, ptr)
    rows = np.nonzero(pat[:, pick].any(1))[0]
    keys = np.nonzero(np.isin(blk.owner_rank(np.arange(mesh.n_nodes)), rows))[0]
    cells = O.mesh_cells_touching(mesh, keys)
    t0 = time.perf_counter()
    H = O.assemble(mesh, O.potential_fn(cfg, fp32), cells=cells)
    t_asm = time.perf_counter() - t0
    Psp = O.sparse_multivector(mesh, mv)
    conn.send(("ready", len(orbs), t_asm, len(cells), int(mesh.n_nodes), len(ptr) - 1, len(perm)))
    while conn.recv() == "go":
        t0 = time.perf_counter()
        Y = O.apply_masked(H, Psp, blk, pat, cb_of_orb)
        O.gram(Psp, Y)
        O.gram(Psp, Psp)
        conn.send(time.perf_counter() - t0)


class OracleTeam:
    """The FP64 oracle as it stands, run on the host cores: one spawned
    worker process per core in the affinity mask (at most one per column
    block), each with a contiguous share of the sampled column blocks.  A
    step sends "go" to every worker and waits for all of them, so the
    workers run concurrently and the step's wall time covers all sampled
    columns.  Assembly is done once per worker at start-up and timed apart."""

    def __init__(self, cfg, blocks, workers=None, fp32=True):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        n = max(1, min(workers or cores, len(blocks)))
        self.cores_available = cores
        shares = [blocks[i * len(blocks) // n:(i + 1) * len(blocks) // n] for i in range(n)]
        self.conns, self.procs = [], []
        t0 = time.perf_counter()
        for share in shares:
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(cfg.name, share, fp32, b), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        info = [c.recv() for c in self.conns]
        self.setup_s = time.perf_counter() - t0
        self.cols = [x[1] for x in info]
        self.assembly_s = max(x[2] for x in info)
        self.n_nodes = info[0][4]
        self.n_blocks_total, self.n_cols_total = info[0][5], info[0][6]
        self.blocks = blocks
        self.workers = n

    def step(self, only=None):
        """Seconds of one step of all workers (or of worker `only` alone)."""
        sel = range(self.workers) if only is None else [only]
        t0 = time.perf_counter()
        for i in sel:
            self.conns[i].send("go")
        for i in sel:
            self.conns[i].recv()
        return time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            c.send("stop")
        for p in self.procs:
            p.join(timeout=30)

    def sample_text(self):
        nb = len(self.blocks)
        scope = ("all" if nb == self.n_blocks_total else f"{nb} of") + f" {self.n_blocks_total} column blocks"
        return (f"{scope} ({sum(self.cols)} of {self.n_cols_total} columns), all their pattern rows, "
                f"split over {self.workers} worker processes; FP64 scipy SpMM + P^T Y + P^T P per "
                f"worker's columns; assembly of the needed rows timed apart ({self.assembly_s:.1f} s)")


def cpu_baseline(cfg, n_blocks, reps=5):
    """The oracle on all host cores (median of `reps` steps) and, beside it,
    one worker's share alone (single core)."""
    team = OracleTeam(cfg, list(range(min(n_blocks, cfg.n_col_blocks))))
    try:
        team.step()                                        # warm caches
        t_all = statistics.median(team.step() for _ in range(reps))
        t_one = statistics.median(team.step(only=0) for _ in range(reps))
        cols = sum(team.cols)
        return {"value": team.n_nodes * cols / t_all, "unit": UNIT, "cores": team.workers, "kind": "oracle",
                "sample": team.sample_text(), "seconds_median_of": reps, "seconds": t_all,
                "cores_in_affinity_mask": team.cores_available,
                "single_core": {"value": team.n_nodes * team.cols[0] / t_one, "seconds": t_one,
                                "columns": team.cols[0]},
                "setup_s": team.setup_s}
    finally:
        team.close()


def run_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:      # rank 0 alone runs the oracle; others exit
        return
    from synth import inputs
    cfg = inputs.get_config(args.config)
    team = OracleTeam(cfg, list(range(min(args.cpu_blocks, cfg.n_col_blocks))))
    try:
        for _ in range(args.warmup):
            team.step()
        times = [team.step() for _ in range(args.steps)]
    finally:
        team.close()
    t = statistics.median(times)
    v = team.n_nodes * sum(team.cols) / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_name(cfg)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": team.workers, "kind": "oracle",
                             "sample": team.sample_text()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _workload_name(cfg):
    n = (cfg.p * cfg.nx + 1) * (cfg.p * cfg.ny + 1) * (cfg.p * cfg.nz + 1)
    fill = f", ~{int(round(100 * cfg.target_fill))}% block fill" if cfg.target_fill else ", clustered centres"
    return (f"{cfg.name}: {cfg.nx}x{cfg.ny}x{cfg.nz} Q{cfg.p} cells, {n:,} DoFs x {cfg.n_orb} orbitals "
            f"in {cfg.n_col_blocks} column blocks{fill}")


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def load_bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)).get("bf16_tflops", 1900.0) * 1e12
    return 1900.0e12


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the FP32 p2 workload (profiles/*_p2_f32.md), with the SHA-256
# of the kernel's source files at capture time; reported only while those
# sources are unchanged.
_SRC_GRAM = ("gram_tc.cu", "tc_common.cuh")
_SRC_APPLY = ("apply_unit.cu", "unit_common.cuh")
_SRC_MMULT = ("mmult_tc.cu", "tc_common.cuh")
NCU_TRAFFIC = {
    # P^T Y (symmetric form) and P^T P (diagonal + off-diagonal tiles)
    "gram_py": (_SRC_GRAM, "38f8f61988a3352f5b41e75a079c54aa342cc7618ddff5dd06381a995fbb7a45", 513261312),
    "gram_pp": (_SRC_GRAM, "38f8f61988a3352f5b41e75a079c54aa342cc7618ddff5dd06381a995fbb7a45", 277447680),
    # post-multiplication with beta = 1 (the second OM call: A and C read, C written)
    "mmult": (_SRC_MMULT, "7d3ba5b905daeb249bc2c98c043408c2e09233844b13a47f2fed7b0ae2c1faa9", 712096512),
    "apply": (_SRC_APPLY, "dcc43559e402f7a95e266b012ea5ce4ed2b7bb1a70b25ce53a6455d603070966", 730593536),
}


def ncu_traffic(kernel, config_name):
    import hashlib
    if config_name != "p2" or kernel not in NCU_TRAFFIC:
        return None
    files, sha, nbytes = NCU_TRAFFIC[kernel]
    h = hashlib.sha256()
    for fname in files:
        h.update(open(os.path.join(ROOT, "paper_1907_01005_gb300", "csrc", fname), "rb").read())
    return nbytes if h.hexdigest() == sha else None


def probe_alu(dtype):
    import ctypes as C
    from paper_1907_01005_gb300 import _capi
    f = C.c_double()
    _capi.check(_capi.fe_probe_fma(dtype, 200 if dtype == 2 else 4000, C.byref(f), C.c_void_p(0)))
    return f.value


def time_path(pb, steps, warmup):
    """CUDA-event times (ms) on the current stream: `steps` whole steps through
    fe_apply_H_gram (P^T P overlapped with the apply), then `steps` runs of the
    three calls one after another for the per-kernel breakdown."""
    import torch
    from paper_1907_01005_gb300 import apply_H, apply_H_gram, gram_PtP, gram_PtY, gram_PtY_sym
    # the step forms P^T Y in its symmetric form on a closed pattern (upper
    # blocks, mirrored); the breakdown times the same form
    pty = gram_PtY_sym if pb.P.get_closed() else gram_PtY
    d = pb.dev
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        apply_H_gram(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"], s)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(s)
    for k in range(steps):
        apply_H_gram(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"], s)
        ev[k + 1].record(s)
    torch.cuda.synchronize()
    total = ev[0].elapsed_time(ev[-1])
    per = {"step": [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]}
    eb = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for k in range(steps):
        e = eb[k]
        e[0].record(s)
        apply_H(pb.mesh, pb.P, pb.Y, s)
        e[1].record(s)
        pty(pb.P, pb.Y, d["G_PY"], s)
        e[2].record(s)
        gram_PtP(pb.P, d["G_PP"], s)
        e[3].record(s)
    torch.cuda.synchronize()
    per["apply"] = [e[0].elapsed_time(e[1]) for e in eb]
    per["gram_py"] = [e[1].elapsed_time(e[2]) for e in eb]
    per["gram_pp"] = [e[2].elapsed_time(e[3]) for e in eb]
    per["sequential"] = [e[0].elapsed_time(e[3]) for e in eb]
    return total, per


def kernel_rooflines(cfg, pb, per, ms_step, hbm_peak, peak_src, fp32_peak):
    """Per-kernel medians, rooflines and the dominant kernel's roofline from the
    breakdown timings `per` of one workload."""
    info = pb.P.info
    # algorithmic work per launch (stored entries, not the 16-byte row padding):
    # apply reads P and V_q and writes Y; P^T Y reads P and Y; P^T P reads P
    s = 4
    n_q = int(pb.mesh.info.n_q)
    nnz = int(info.stored_entries)
    apply_bytes = 2 * nnz * s + n_q * s
    py_bytes = 2 * nnz * s
    pp_bytes = nnz * s
    n = cfg.p + 1
    apply_flops = info.active_cell_cols * (18 * n ** 4 + 3 * n ** 3)
    # sliced Gram: 6 bf16 slice products for P^T Y (3 x 3 slices, s+t <= 4)
    # and 15 for P^T P (5 x 5 slices, s+t <= 6), both on half the output
    # blocks (symmetric forms: P^T Y on a closed pattern, P^T P)
    py_tc = (3.0 if pb.P.get_closed() else 6.0) * info.gram_flops
    pp_tc = 7.5 * info.gram_flops
    bf16_peak = load_bf16_peak()
    t_apply = statistics.median(per["apply"]) * 1e-3
    t_py = statistics.median(per["gram_py"]) * 1e-3
    t_pp = statistics.median(per["gram_pp"]) * 1e-3

    def bound(t, nbytes, work, peak, unit_name):
        """roofline of one kernel: the resource whose ideal time is longest"""
        t_mem = nbytes / (hbm_peak * 1e9)
        t_cmp = work / peak
        if t_mem >= t_cmp:
            return {"bound": "hbm", "achieved": nbytes / t / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": nbytes / t / 1e9 / hbm_peak}
        return {"bound": unit_name, "achieved": work / t / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": work / t / peak}

    kernels = {
        "apply": {"ms_p50": 1e3 * t_apply, "ms_p99": pct(per["apply"], 0.99), "bytes": apply_bytes,
                  "flops": apply_flops, "gbs": apply_bytes / t_apply / 1e9,
                  "hbm_frac": apply_bytes / t_apply / 1e9 / hbm_peak,
                  "gflops": apply_flops / t_apply / 1e9, "fp32_frac": apply_flops / t_apply / fp32_peak,
                  **{"roof_" + k: v for k, v in bound(t_apply, apply_bytes, apply_flops, fp32_peak, "alu").items()}},
        "gram_py": {"ms_p50": 1e3 * t_py, "ms_p99": pct(per["gram_py"], 0.99), "bytes": py_bytes,
                    "gflops": info.gram_flops / t_py / 1e9, "tc_tflops": py_tc / t_py / 1e12,
                    "gbs": py_bytes / t_py / 1e9,
                    **{"roof_" + k: v for k, v in bound(t_py, py_bytes, py_tc, bf16_peak, "tensor").items()}},
        "gram_pp": {"ms_p50": 1e3 * t_pp, "ms_p99": pct(per["gram_pp"], 0.99), "bytes": pp_bytes,
                    "gflops": info.gram_flops / t_pp / 1e9, "tc_tflops": pp_tc / t_pp / 1e12,
                    "gbs": pp_bytes / t_pp / 1e9,
                    **{"roof_" + k: v for k, v in bound(t_pp, pp_bytes, pp_tc, bf16_peak, "tensor").items()}},
    }
    dom = max(("apply", t_apply), ("gram_py", t_py), ("gram_pp", t_pp), key=lambda x: x[1])[0]
    kd = kernels[dom]
    roof = {"kernel": dom, "bound": kd["roof_bound"], "achieved": kd["roof_achieved"], "peak": kd["roof_peak"],
            "unit": kd["roof_unit"], "frac": kd["roof_frac"],
            "traffic": ncu_traffic(dom, cfg.name),
            "peak_source": (f"{peak_src} hbm_gbs" if kd["roof_bound"] == "hbm" else
                            "measured fp32 FMA probe" if kd["roof_bound"] == "alu" else "measured bf16_tflops"),
            "per_launch": {"hbm": "achieved = algorithmic bytes of one launch / its CUDA-event median",
                           "alu": "achieved = algorithmic flops of one launch (active cell-columns x "
                                  "(18 n^4 + 3 n^3)) / its CUDA-event median",
                           "tensor": "achieved = bf16 slice-product flops of one launch / its CUDA-event median"
                           }[kd["roof_bound"]]}
    step_bytes = apply_bytes + py_bytes + pp_bytes
    step_roof = {"bytes": step_bytes, "ideal_ms": step_bytes / (hbm_peak * 1e9) * 1e3,
                 "frac": step_bytes / (ms_step * 1e-3) / 1e9 / hbm_peak}

    return t_apply, t_py, t_pp, kernels, roof, step_roof


def measure_second(cfg_name, args, world, hbm_peak, peak_src, fp32_peak):
    """The same step on a second workload (the p = 4 paper-scale mesh beside
    p = 2): step time, per-kernel breakdown and rooflines, value."""
    import torch
    from paper_1907_01005_gb300 import FE_F32, harness
    from synth import inputs
    cfg = inputs.get_config(cfg_name)
    pb = harness.build_problem(cfg, FE_F32)
    harness.to_device(pb)
    if not args.no_tune:
        from paper_1907_01005_gb300 import autotune
        autotune(pb.mesh, pb.P, pb.Y)
    steps = max(20, args.steps // 4)
    barrier(world)
    total_ms, per = time_path(pb, steps, max(3, args.warmup // 2))
    barrier(world)
    if pb.mesh.check_device() != 0:
        raise RuntimeError("device status word set during the timed region")
    ms_step = max_over_ranks(total_ms / steps, world)
    N, M = pb.mesh.n_dofs, pb.n_cols
    t_apply, t_py, t_pp, kernels, roof, step_roof = kernel_rooflines(cfg, pb, per, ms_step, hbm_peak, peak_src,
                                                                     fp32_peak)
    out = {"workload": _workload_name(cfg), "steps": steps, "ms_per_step": ms_step,
           "value": whole_job_value(N, M, ms_step, world), "unit": UNIT,
           "p50_ms": pct(per["step"], 0.5), "p99_ms": pct(per["step"], 0.99),
           "sequential_ms_per_step": statistics.median(per["sequential"]),
           "kernels": kernels, "roofline": roof, "step_hbm_roofline": step_roof,
           "launch": dict(zip(("persistent", "ctas_per_sm", "cells_per_round"), pb.P.get_launch()))}
    del pb
    torch.cuda.empty_cache()
    return out


def time_graph(pb, steps, warmup):
    """ms per step of the CUDA graph of the whole step (one graph launch per step)."""
    import torch
    from paper_1907_01005_gb300 import StepGraph
    d = pb.dev
    s = torch.cuda.current_stream()
    g = StepGraph(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"], s)
    for _ in range(warmup):
        g.launch(s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(steps):
        g.launch(s)
    e1.record(s)
    torch.cuda.synchronize()
    del g
    return e0.elapsed_time(e1) / steps


def time_cellmat(pb, steps):
    """Medians (ms) of fe_apply_H and fe_apply_M in the cell-matrix form (FP32,
    p <= 2, element matrices on the tensor cores), the form restored after."""
    import torch
    from paper_1907_01005_gb300 import FORM_CELLMAT, FORM_SUMFAC, apply_H, apply_M
    s = torch.cuda.current_stream()
    pb.P.set_form(FORM_CELLMAT)
    out = {}
    try:
        for name, f in (("apply_H", apply_H), ("apply_M", apply_M)):
            for _ in range(3):
                f(pb.mesh, pb.P, pb.Y, s)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
            ev[0].record(s)
            for k in range(steps):
                f(pb.mesh, pb.P, pb.Y, s)
                ev[k + 1].record(s)
            torch.cuda.synchronize()
            out[name] = statistics.median(ev[k].elapsed_time(ev[k + 1]) for k in range(steps))
        if pb.mesh.check_device() != 0:
            raise RuntimeError("device status word set by the cell-matrix kernel")
    finally:
        pb.P.set_form(FORM_SUMFAC)
    return out


def time_om(pb, steps):
    """The rest of an orbital-minimisation gradient evaluation on the step's
    workload (Sec. 2): Phi_M = M P, Mbar = P^T Phi_M, the two post-
    multiplications of the gradient and tr(D^T G); CUDA-event medians (ms)."""
    import torch
    from paper_1907_01005_gb300 import BCSR, apply_M, gram_PtY_sym, mmult, trace_dot
    d = pb.dev
    M = pb.n_cols

    def like():
        B = BCSR(pb.mesh, pb.cbp, pb.row_ptr, pb.col_idx, pb.dtype)
        v, t = B.alloc()
        B.bind(v, t)
        return B
    YM, G, D = like(), like(), like()
    D.values.normal_()
    Mb = torch.zeros((M, M), dtype=torch.float64, device="cuda")
    g = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    names = ("apply_M", "gram_M", "mmult_1", "mmult_2", "trace")
    calls = (lambda: apply_M(pb.mesh, pb.P, YM, s), lambda: gram_PtY_sym(pb.P, YM, Mb, s),
             lambda: mmult(pb.Y, Mb, G, -2.0, -2.0, 0.0, s), lambda: mmult(YM, d["G_PY"], G, -2.0, 0.0, 1.0, s),
             lambda: trace_dot(D, G, g, s))
    for _ in range(3):
        for f in calls:
            f()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)] for _ in range(steps)]
    for k in range(steps):
        ev[k][0].record(s)
        for i, f in enumerate(calls):
            f()
            ev[k][i + 1].record(s)
    torch.cuda.synchronize()
    out = {n: statistics.median(e[i].elapsed_time(e[i + 1]) for e in ev) for i, n in enumerate(names)}
    out["total_ms"] = sum(out.values())
    return out


SIZE_CLASSES = {"small": (0.0, 1e7), "medium": (1e7, 1e8), "large": (1e8, float("inf"))}


def serving_run(args, dtype=1, loads=None, n_requests=None):
    """Poisson streams of apply_H + Gram requests through the continuous-batching
    server: a pool of distinct workloads drawn from the serving mix (meshes
    taken in turn), arrivals at multiples of the rate one request at a time
    sustains; p50/p99 overall and per size class (DoF x columns) beside each
    class's one-at-a-time latency."""
    from paper_1907_01005_gb300 import harness
    from paper_1907_01005_gb300.serving import Server, latency_stats
    from synth import inputs
    meshes = inputs.SERVING_MESHES if args.serving_full else inputs.SERVING_MESHES[:2]
    orbs = (32, 640) if args.serving_full else (32, 320)
    loads = loads or args.serving_loads
    n_requests = n_requests or args.serving
    t0 = time.perf_counter()
    probs = []
    for cfg in inputs.serving_mix(args.serving_pool, meshes=meshes, orb_range=orbs):
        try:
            probs.append(harness.build_problem(cfg, dtype))
        except Exception as e:           # a drawn pattern the library refuses (reported, not served)
            print(f"serving: skipped {cfg.name}: {e}", file=sys.stderr)
    setup_s = time.perf_counter() - t0
    srv = Server(slots=4)
    pids = [srv.register(pb) for pb in probs]
    dofs_cols = {pid: srv.payloads[pid].dofs_cols for pid in pids}
    for pid in pids:                      # residency and one warm call each
        srv.submit(pid)
        srv.drain()
    alone_ms = {}
    for pid in pids:                      # one at a time: the service time of each payload
        ts = []
        for _ in range(3):
            r = srv.submit(pid)
            srv.drain()
            ts.append(r.latency)
        alone_ms[pid] = 1e3 * statistics.median(ts)
    serial = sum(alone_ms.values()) / len(pids) * 1e-3
    # offered load swept in multiples of the rate one request at a time
    # sustains; the main figures are those at 0.8 of it
    sweep = []
    st = None
    for li, load in enumerate(loads):
        rate = load / serial
        rng = np.random.default_rng(190701005 + li)
        arr = inputs.poisson_arrivals(n_requests, rate, seed=190701005 + li)
        trace = [(float(arr[i]), int(pids[rng.integers(len(pids))])) for i in range(n_requests)]
        srv.finished.clear()
        reqs = srv.run_trace(trace)
        s = latency_stats(reqs, dofs_cols, SIZE_CLASSES, alone_ms)
        sweep.append({"load": load, "offered_rate_per_s": rate, "p50_ms": s["p50_ms"], "p99_ms": s["p99_ms"],
                      "dof_cols_per_s": s["dof_cols_per_s"], "achieved_rate_per_s": len(reqs) / s["span_s"],
                      "classes": s.get("classes", {})})
        if st is None or abs(load - 0.8) < 1e-9:
            st = dict(s, offered_rate_per_s=rate)
    st.update({"sweep": sweep, "serial_ms": 1e3 * serial, "slots": srv.slots, "pool": len(pids),
               "pool_dofs": [int(srv.payloads[p].problem.mesh.n_dofs) for p in pids],
               "pool_columns": [int(srv.payloads[p].problem.n_cols) for p in pids],
               "pool_degree": [int(srv.payloads[p].problem.cfg.p) for p in pids],
               "alone_ms": [alone_ms[p] for p in pids],
               "evictions": srv.evictions, "host_setup_s": setup_s, "dtype": "f32" if dtype == 1 else "f64",
               "serving_config": (f"{n_requests} Poisson requests per load point at {', '.join(f'{x:g}' for x in loads)}"
                                  f" x the one-at-a-time rate, drawn from a pool of {len(pids)} workloads "
                                  f"(meshes {', '.join('x'.join(map(str, m)) for m in meshes)} cells in turn, "
                                  f"p in {{2, 4}}, {orbs[0]}-{orbs[1]} orbitals log-uniform, fill 10-30%); "
                                  f"4 stream slots; admission by device-memory footprint, shortest predicted "
                                  f"first with an age bound, last slot kept for small requests")})
    return st


def pct(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    from paper_1907_01005_gb300 import FE_F32, FE_F64, apply_H_gram_host, harness
    from synth import inputs
    cfg = inputs.get_config(args.config)

    pb = harness.build_problem(cfg, FE_F32)
    harness.to_device(pb)
    N, M = pb.mesh.n_dofs, pb.n_cols
    info = pb.P.info
    hbm_peak, peak_src = load_peaks()
    fp32_peak = max(probe_alu(1), probe_alu(3))   # scalar FFMA or packed FP32x2, whichever is faster
    fp64_peak = probe_alu(2)
    tune_ms = None
    if not args.no_tune:
        from paper_1907_01005_gb300 import autotune
        tune_ms = autotune(pb.mesh, pb.P, pb.Y)
    knobs = pb.P.get_launch()

    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    total_ms, per = time_path(pb, args.steps, args.warmup)
    clk = clocks.stop()
    barrier(world)
    if pb.mesh.check_device() != 0:
        raise RuntimeError("device status word set during the timed region")
    graph_ms = time_graph(pb, args.steps, args.warmup)
    ms_step = max_over_ranks(total_ms / args.steps, world)
    value = whole_job_value(N, M, ms_step, world)

    t_apply, t_py, t_pp, kernels, roof, step_roof = kernel_rooflines(cfg, pb, per, ms_step, hbm_peak, peak_src,
                                                                     fp32_peak)
    s = 4
    nnz = int(info.stored_entries)
    apply_bytes = kernels["apply"]["bytes"]
    bf16_peak = load_bf16_peak()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": _workload_name(cfg), "dofs": N, "columns": M,
                       "col_blocks": cfg.n_col_blocks, "block_fill": info.nnz_blocks / (pb.mesh.n_row_blocks * cfg.n_col_blocks),
                       "stored_values": int(info.stored_entries), "tiles": int(info.n_tiles),
                       "gram_accumulate": "f64", "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (P and Y %.0f MB each)" % (info.n_values * 4 / 1e6)},
            "launch": {"persistent": knobs[0], "ctas_per_sm": knobs[1], "cells_per_round": knobs[2],
                       "autotune_apply_ms": tune_ms},
            "graph_ms_per_step": graph_ms,
            "p50_ms": pct(per["step"], 0.5), "p99_ms": pct(per["step"], 0.99),
            "sequential_ms_per_step": statistics.median(per["sequential"]),
            "apply_dof_cols_per_s": N * M / t_apply,
            "gram_gflops": {"PtY": info.gram_flops / t_py / 1e9, "PtP": info.gram_flops / t_pp / 1e9},
            "kernels": kernels, "roofline": roof, "step_hbm_roofline": step_roof,
            "alu_peaks_tflops": {"fp32": probe_alu(1) / 1e12, "fp32x2": probe_alu(3) / 1e12,
                                 "fp64": fp64_peak / 1e12},
            # per step: the apply; P^T P's exponent pass and Gram kernel for the
            # diagonal and for the off-diagonal tiles, and its mirror; the
            # symmetric P^T Y's exponent pass, Gram kernel and mirror
            "gpu_launches": 9 * args.steps, "clocks": clk}

    # the p = 4 paper-scale workload beside p = 2 (same DoFs and orbitals)
    if args.config == "p2" and not args.no_p4:
        line["p4"] = measure_second("p4", args, world, hbm_peak, peak_src, fp32_peak)

    # the rest of an orbital-minimisation gradient evaluation (NEXT rows f1, f3)
    om = time_om(pb, max(10, args.steps // 10))
    t_mm = om["mmult_1"] * 1e-3
    t_mm2 = om["mmult_2"] * 1e-3
    # the tensor-core post-multiplication is bound by HBM: A read and C written
    # (beta = 0), plus C read (beta = 1); its 3-term TF32 products take less
    # time at the tensor peak than those bytes at the HBM peak
    om["mmult_roofline"] = {"bound": "hbm", "achieved": 2 * nnz * s / t_mm / 1e9, "peak": hbm_peak,
                            "unit": "GB/s", "frac": 2 * nnz * s / t_mm / 1e9 / hbm_peak,
                            "gflops": info.gram_flops / t_mm / 1e9,
                            "traffic_beta1": ncu_traffic("mmult", cfg.name),
                            "hbm_frac_beta1": 3 * nnz * s / t_mm2 / 1e9 / hbm_peak}
    om["gradient_ms"] = ms_step + om["total_ms"]      # H P, Hbar, P^T P (the step) plus the above
    line["om"] = om

    # cell-matrix form of the apply (NEXT row f2): element matrices as dense
    # TF32 tensor-core products with a 3-term split; work per active
    # cell-column: 3 splits x 2 (n^3)^2 flops for each of K_L, S3, Sb3 (H) or
    # M_c (M)
    if cfg.p <= 2:
        cm = time_cellmat(pb, max(10, args.steps // 4))
        n3 = (cfg.p + 1) ** 3
        tf32_peak = bf16_peak * 1.1 / 2.25         # measured bf16 x nominal TF32/bf16 ratio
        wH = info.active_cell_cols * 3 * 3 * 2 * n3 * n3
        wM = info.active_cell_cols * 3 * 2 * n3 * n3
        tH = cm["apply_H"] * 1e-3
        line["cellmat"] = {
            "apply_H_ms": cm["apply_H"], "apply_M_ms": cm["apply_M"],
            "vs_sumfac_apply": cm["apply_H"] / (1e3 * t_apply),
            "tf32_tflops_H": wH / tH / 1e12, "tf32_tflops_M": wM / (cm["apply_M"] * 1e-3) / 1e12,
            "roofline": {"bound": "tensor", "achieved": wH / tH / 1e12, "peak": tf32_peak / 1e12,
                         "unit": "TFLOP/s", "frac": wH / tH / tf32_peak,
                         "peak_source": "measured bf16_tflops x 1.1/2.25 (nominal TF32/bf16)",
                         "hbm_frac": apply_bytes / tH / 1e9 / hbm_peak}}

    # FP64 path on the same workload
    if not args.no_fp64:
        pb64 = harness.build_problem(cfg, FE_F64)
        harness.to_device(pb64)
        k64 = max(3, args.steps // 5)
        tot64, per64 = time_path(pb64, k64, max(3, args.warmup // 2))
        ms64 = max_over_ranks(tot64 / k64, world)
        a64, py64, pp64 = (statistics.median(per64[k]) for k in ("apply", "gram_py", "gram_pp"))
        line["fp64"] = {"ms_per_step": ms64, "value": world * N * M / (ms64 * 1e-3),
                        "p50_ms": pct(per64["step"], 0.5), "p99_ms": pct(per64["step"], 0.99),
                        "apply_ms": a64, "gram_py_ms": py64, "gram_pp_ms": pp64,
                        "apply_dof_cols_per_s": N * M / (a64 * 1e-3),
                        "gram_gflops": {"PtY": info.gram_flops / (py64 * 1e-3) / 1e9,
                                        "PtP": info.gram_flops / (pp64 * 1e-3) / 1e9},
                        "mixed_speedup": ms64 / ms_step}
        del pb64
        torch.cuda.empty_cache()

    # end to end through the host-buffer entry point (pinned buffers)
    if not args.no_e2e:
        d = pb.dev
        Ph = torch.from_numpy(pb.P_host).pin_memory()
        Yh = torch.empty_like(Ph).pin_memory()
        Gh1 = torch.empty((M, M), dtype=torch.float64).pin_memory()
        Gh2 = torch.empty((M, M), dtype=torch.float64).pin_memory()
        s = torch.cuda.current_stream()
        for _ in range(2):
            apply_H_gram_host(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"], Ph, Yh, Gh1, Gh2, s)
        k = max(3, args.steps // 3)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(k):
            apply_H_gram_host(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"], Ph, Yh, Gh1, Gh2, s)
        t_e2e = max_over_ranks((time.perf_counter() - t0) / k, world)
        line["e2e"] = {"value": world * N * M / t_e2e, "unit": UNIT,
                       "h2d_bytes_per_step": int(info.value_bytes),
                       "d2h_bytes_per_step": int(info.value_bytes + 2 * M * M * 8),
                       "ms_per_step": 1e3 * t_e2e}

    if args.serving > 0 and world == 1:
        pb = d = None                      # release the benchmark workload's device buffers
        torch.cuda.empty_cache()
        line["serving"] = serving_run(args, 1)
        if not args.no_fp64:
            torch.cuda.empty_cache()
            line["serving_fp64"] = serving_run(args, 2, loads=[0.8], n_requests=max(1, args.serving // 4))

    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(cfg, args.cpu_blocks)
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
