#!/usr/bin/env python
"""Benchmark of the FeLoG walk + SGNS hot path on one B300.

Workload (N=1): R-MAT scale 20 (1,048,576 nodes), edge factor 16,
(a, b, c, d) = (0.57, 0.19, 0.19, 0.05), symmetrised, deduplicated, 10 % of
the edges held out for link prediction; walks of 80 nodes, 10 walks per node
(one per round, 10 rounds), window 10, 5 negatives, d = 128 float tables,
lock-free (Hogwild) SGNS.

One step = one round of Algorithm 1 over the whole graph: compact V_a, walk
(corpus counts fused), build the unigram^0.75 alias table, train SGNS,
compute Psi and the next active set.  The plain form (feedback off) keeps
every non-isolated node active, so every step does the same work.  The
tables (2 x 512 MiB) exceed the 126 MB L2, so no L2 flush is needed between
steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walk steps/s + SGNS tokens/s at fixed AUC, chosen vs plain form; p50/p99 latency"
SCALE, EDGE_FACTOR, GRAPH_SEED, SPLIT_SEED = 20, 16, 1, 7
L, WPR, ROUNDS, WINDOW, NEG, DIM, LR0 = 80, 1, 10, 10, 5, 128, 0.025
MU, KS = 0.65, 8
SEED = 2026


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--scale", type=int, default=SCALE, help="R-MAT scale (20 = the benchmark workload)")
    p.add_argument("--no-quality", action="store_true", help="skip the full-run AUC comparison")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--form", type=int, default=0, choices=[0, 1, 2, 3, 4, 5],
                   help="Hogwild kernel form: 0 automatic, 1 full warp per pair, 2 half warp per pair, "
                        "3 half warp with the window's phi_in increments staged in shared memory, "
                        "4 half warp with the next step's rows prefetched to shared memory")
    p.add_argument("--stage-flush", type=int, default=0,
                   help="form 3: staged increments reach memory every this many centers (0: on leaving the window)")
    p.add_argument("--mode", default="round", choices=["round", "tile", "batch", "serve", "mu"],
                   help="round: one round of Algorithm 1 on R-MAT 20 (default); tile: rounds with the "
                        "shared-negatives tile trainer; batch: the 512-graph "
                        "batching form; serve: the request loop with Poisson arrivals; mu: the "
                        "feedback-threshold sweep on homophilic / heterophilic / R-MAT graphs")
    p.add_argument("--jobs", type=int, default=512, help="batch mode: number of graphs")
    p.add_argument("--rate", type=float, default=20.0, help="serve mode: arrivals per second")
    p.add_argument("--duration", type=float, default=20.0, help="serve mode: seconds of arrivals")
    p.add_argument("--max-nodes", type=int, default=1 << 16, help="serve mode: largest job in nodes")
    p.add_argument("--no-forms", action="store_true", help="round mode: skip the small batch/serve runs")
    p.add_argument("--no-persistent", action="store_true",
                   help="batch mode: time only the CUDA-graph launch form, not the persistent kernel")
    p.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                   help="table precision of the timed rounds (fp32 = the plain form)")
    return p.parse_args()


def _workload(scale, rank=0):
    from paper_2606_22180_b300 import inputs

    g = inputs.workload_rmat(scale, GRAPH_SEED + 1000 * rank, EDGE_FACTOR)
    split = inputs.link_split(g, 0.1, SPLIT_SEED + rank)
    return split


def _workload_name(scale, precision="fp32"):
    return (f"rmat{scale}-ef{EDGE_FACTOR} (a,b,c,d)=(0.57,0.19,0.19,0.05), 10% edges held out; "
            f"L={L}, {ROUNDS} walks/node, window {WINDOW}, {NEG} negatives, d={DIM} {precision}, hogwild")


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(device_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower() in ("active", "1"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def _kernel_source_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _profile_traffic(kernel_srcs, name="sgns_hogwild_rmat20_fp32.md"):
    """DRAM bytes per launch of the SGNS kernel from the committed ncu
    summary `name`, or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(path).read()
    except OSError:
        return None
    src_hash = _kernel_source_hash(kernel_srcs)
    vals = {}
    for line in txt.splitlines():
        if ": " in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(": ", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("sgns.cu + sgns_core.cuh sha256[:16]") != src_hash:
        return None
    try:
        return float(vals["dram_bytes_per_full_launch"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# one round of Algorithm 1 through the C ABI, buffers preallocated
# ---------------------------------------------------------------------------
class RoundRunner:
    KERNELS_PER_ROUND = 13  # compact 3, walk 1, noise table 6, train 2, feedback 1

    def __init__(self, fl, dg, tp, fp, seed):
        import torch

        self.fl, self.dg, self.tp, self.fp, self.seed = fl, dg, tp, fp, seed
        self.lib = fl.load()
        n = dg.n
        dev = dg.offsets.device
        self.n = n
        dt = fl.table_dtype(tp.precision)
        self.phi_in = torch.empty((n, tp.dim), dtype=dt, device=dev)
        self.phi_out = torch.empty((n, tp.dim), dtype=dt, device=dev)
        self.active = [torch.empty(n, dtype=torch.uint8, device=dev) for _ in range(2)]
        self.starts = torch.empty(n, dtype=torch.int32, device=dev)
        self.n_active_d = torch.zeros(1, dtype=torch.int32, device=dev)
        self.n_next_d = torch.zeros(1, dtype=torch.int32, device=dev)
        self.walks = torch.empty(n * WPR * L, dtype=torch.int32, device=dev)
        self.counts = torch.empty(n, dtype=torch.int32, device=dev)
        self.thr = torch.empty(n, dtype=torch.int64, device=dev)
        self.alias = torch.empty(n, dtype=torch.int32, device=dev)
        self.S = torch.empty(1, dtype=torch.int64, device=dev)
        self.loss = torch.empty(1, dtype=torch.float64, device=dev)
        self.n_active_h = torch.zeros(1, dtype=torch.int32).pin_memory()
        self.loss_h = torch.zeros(1, dtype=torch.float64).pin_memory()
        P = ctypes.c_void_p
        self.cws = torch.empty(self.lib.felog_compact_workspace_bytes(n), dtype=torch.uint8, device=dev)
        self.nws = torch.empty(self.lib.felog_noise_workspace_bytes(n), dtype=torch.uint8, device=dev)
        tb = self.lib.felog_train_workspace_bytes(n * WPR, L, n, ctypes.byref(tp))
        self.tws = torch.empty(max(tb, 256), dtype=torch.uint8, device=dev)
        self.csr = fl._Csr(dg.offsets.data_ptr(), dg.cols.data_ptr(), n, dg.nnz)
        self.wp = fl._WalkParams(L, WPR)
        self.P = P
        self.cur = 0
        self.clock = 0
        self.ev = None

    def reset(self):
        import torch

        fl = self.fl
        fl._check(self.lib.felog_init_tables(self.n, self.tp.dim, self.tp.precision, self.seed,
                                             self.P(self.phi_in.data_ptr()), self.P(self.phi_out.data_ptr()),
                                             fl._stream()), "init")
        deg = self.dg.offsets[1:] - self.dg.offsets[:-1]
        self.active[0].copy_((deg > 0).to(torch.uint8))
        self.n_live = int((deg > 0).sum().item())
        self.cur = 0
        self.clock = 0

    def run(self, r, events=None):
        """One round; returns (n_active, tokens).  events: 5 CUDA events for phase times."""
        fl, lib, P = self.fl, self.lib, self.P
        s = fl._stream()
        a_in, a_out = self.active[self.cur], self.active[self.cur ^ 1]
        fl._check(lib.felog_compact_active(P(a_in.data_ptr()), self.n, P(self.starts.data_ptr()),
                                           P(self.n_active_d.data_ptr()), P(self.cws.data_ptr()),
                                           self.cws.numel(), s), "compact")
        self.n_active_h.copy_(self.n_active_d, non_blocking=True)
        import torch

        torch.cuda.current_stream().synchronize()
        na = int(self.n_active_h.item())
        if na == 0:
            return 0, 0
        n_walks = na * WPR
        if events:
            events[0].record()
        self.counts.zero_()
        fl._check(lib.felog_walk(ctypes.byref(self.csr), P(self.starts.data_ptr()), na, ctypes.byref(self.wp),
                                 self.seed, r, P(self.walks.data_ptr()), P(self.counts.data_ptr()), s), "walk")
        if events:
            events[1].record()
        fl._check(lib.felog_noise_table(P(self.counts.data_ptr()), self.n, P(self.thr.data_ptr()),
                                        P(self.alias.data_ptr()), P(self.S.data_ptr()), P(self.nws.data_ptr()),
                                        self.nws.numel(), s), "noise")
        if events:
            events[2].record()
        fl._check(lib.felog_train(P(self.walks.data_ptr()), n_walks, L, self.n, ctypes.byref(self.tp),
                                  P(self.thr.data_ptr()), P(self.alias.data_ptr()), P(self.S.data_ptr()),
                                  self.seed, r, self.clock, P(self.phi_in.data_ptr()), P(self.phi_out.data_ptr()),
                                  P(self.loss.data_ptr()), P(self.tws.data_ptr()), self.tws.numel(), s), "train")
        if events:
            events[3].record()
        fl._check(lib.felog_feedback(ctypes.byref(self.csr), P(self.phi_in.data_ptr()), self.tp.dim,
                                     self.tp.precision, ctypes.byref(self.fp), self.seed, r, P(a_in.data_ptr()),
                                     P(a_out.data_ptr()), None, P(self.n_next_d.data_ptr()), s), "feedback")
        if events:
            events[4].record()
        self.clock += n_walks * L
        self.cur ^= 1
        return na, n_walks * L


def _sgns_kernel_name(form, precision):
    t = "float" if precision == "fp32" else "bf16"
    if form == 1:
        return f"k_sgns_hogwild<128,{t},8,5>"
    if form == 4 or (form == 0 and t == "bf16"):  # the automatic form for bf16 tables of dim 128
        return f"k_sgns_hogwild_pf<128,{t},5>"
    if form == 5 and t == "float":
        return "k_sgns_hogwild_bulk<128,5>"
    staged = form == 3
    return f"k_sgns_hogwild_hw<128,{t},5,{'true' if staged else 'false'}>"


def _e2e_job(fl, g, tp, fp, seed, world, barrier):
    """One embedding job end to end through felog_embed: the CSR from pinned
    host memory to the device, every round of Algorithm 1, the embedding
    phi_in back to pinned host memory.  Buffers and the workspace are
    allocated before the timed region."""
    import torch

    off_h = torch.from_numpy(g.offsets).pin_memory()
    col_h = torch.from_numpy(g.cols).pin_memory()
    dgj = fl.DeviceGraph(torch.empty_like(off_h, device="cuda"), torch.empty_like(col_h, device="cuda"))
    dt = fl.table_dtype(tp.precision)
    phi_in = torch.empty((g.n, tp.dim), dtype=dt, device="cuda")
    phi_out = torch.empty_like(phi_in)
    out_h = torch.empty((g.n, tp.dim), dtype=dt).pin_memory()
    wp = fl._WalkParams(L, WPR)
    ws = torch.empty(fl.load().felog_embed_workspace_bytes(g.n, ctypes.byref(wp), ctypes.byref(tp)),
                     dtype=torch.uint8, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record()
    dgj.offsets.copy_(off_h, non_blocking=True)
    dgj.cols.copy_(col_h, non_blocking=True)
    _, _, st = fl.felog_embed(dgj, L, WPR, tp, fp, seed, phi_in=phi_in, phi_out=phi_out, workspace=ws)
    out_h.copy_(phi_in, non_blocking=True)
    e1.record()
    barrier()
    ms = e0.elapsed_time(e1)
    tokens = float(sum(x["tokens"] for x in st))
    if world > 1:
        ms, tokens = reduce_over_ranks(ms, tokens, "cuda")
    del phi_in, phi_out, ws, dgj
    return {"value": tokens / (ms / 1e3), "unit": "tokens/s",
            "h2d_bytes_per_step": int(g.offsets.nbytes + g.cols.nbytes),
            "d2h_bytes_per_step": int(out_h.numel() * out_h.element_size()),
            "step": f"one whole felog_embed job ({len(st)} rounds): CSR in from pinned host memory, "
                    "phi_in out to pinned host memory", "ms": ms, "tokens": tokens}


def _ripp(fl, evaluate, dg, split, n_live):
    """The round-interleaved pipeline (Section 5.3) on the round workload with
    the chosen form's feedback (mu = 0.65, bf16-SR): felog_embed_pipelined with
    feedback_lag 0 (Algorithm 1 as printed: the streams alternate) and 1 (Psi on
    the snapshot as training starts: sampling runs under training); wall time,
    stream busy times and overlap from CUDA events, link AUC."""
    import torch

    T = ROUNDS * WPR * n_live * L
    tp = fl.train_params(DIM, WINDOW, NEG, LR0, T, fl.FELOG_SGNS_HOGWILD, 4096, fl.FELOG_BF16_SR)
    fp = fl.feedback_params(True, MU, KS, ROUNDS, False)
    out = {"workload": _workload_name(SCALE, "bf16-SR") + f", feedback mu={MU}"}
    for lag in (0, 1):
        torch.cuda.synchronize()
        pi, _, st, ps = fl.felog_embed_pipelined(dg, L, WPR, tp, fp, SEED, feedback_lag=lag)
        torch.cuda.synchronize()
        tokens = sum(x["tokens"] for x in st)
        out[f"lag{lag}"] = {"wall_ms": ps["wall_ms"], "train_busy_ms": ps["train_busy_ms"],
                            "sample_busy_ms": ps["sample_busy_ms"], "overlap_ms": ps["overlap_ms"],
                            "train_stream_busy_frac": ps["train_busy_ms"] / ps["wall_ms"],
                            "rounds": ps["rounds"], "tokens": tokens, "tokens_per_s": tokens / (ps["wall_ms"] / 1e3),
                            "active_per_round": [x["n_active"] for x in st],
                            "auc": evaluate.link_auc(pi, split.pos, split.neg)}
        del pi
    return out


def _bf16_rounds(fl, dg, T, args):
    """The precision form's rounds on the round workload's graph (bf16 tables,
    stochastic rounding), timed like the plain rounds."""
    import torch

    tp = fl.train_params(DIM, WINDOW, NEG, LR0, T, fl.FELOG_SGNS_HOGWILD, 4096, fl.FELOG_BF16_SR, 0, args.form)
    runner = RoundRunner(fl, dg, tp, fl.feedback_params(False, MU, KS, ROUNDS, False), SEED)
    runner.reset()
    for w in range(args.warmup):
        runner.run(w)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    tokens = 0
    for k in range(args.steps):
        tokens += runner.run(args.warmup + k, events=ev[k])[1]
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    phase = {name: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in ev)
             for i, name in enumerate(["walk", "noise", "train", "feedback"])}
    del runner
    # roofline of the bf16 SGNS launch: 256-byte rows; DRAM traffic from the
    # committed capture of the automatic bf16 kernel while its source matches
    n_live = T // (ROUNDS * WPR * L)
    alg_bytes = DIM * 2 * (4 * n_live * WPR * L + 2 * NEG * n_live * WPR * _pairs_per_walk())
    peak, _ = _peaks()
    csrc = os.path.join(ROOT, "paper_2606_22180_b300", "csrc")
    traffic = None
    if args.form in (0, 4):
        traffic = _profile_traffic([os.path.join(csrc, "sgns.cu"), os.path.join(csrc, "sgns_core.cuh")],
                                   "sgns_hogwild_pf_bf16_rmat18.md")
    train_s = phase["train"] / 1e3
    return {"workload": _workload_name(SCALE, "bf16-SR"), "tokens_per_s": tokens / (ms / 1e3),
            "ms_per_step": ms / args.steps, "phase_ms": phase,
            "kernel": _sgns_kernel_name(args.form, "bf16"), "steps": args.steps,
            "roofline": {"bound": "hbm", "achieved": alg_bytes / train_s / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg_bytes / train_s / 1e9 / peak, "bytes_per_launch": alg_bytes,
                         "traffic": traffic,
                         "dram_frac": traffic / train_s / 1e9 / peak if traffic else None,
                         "note": "algorithmic row bytes (256-byte bf16 rows) per launch / CUDA-event time; "
                                 "the launch is bound by instruction issue (ncu: 66 % issue active), "
                                 "not by DRAM or the L2 request path"}}


def reduce_over_ranks(ms: float, tokens: float, device) -> tuple[float, float]:
    """Whole-job aggregation of independent replicas: the slowest rank's time
    and the tokens of all ranks (no collective on the data path; this is the
    only exchange)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    k = torch.tensor([tokens], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(k, op=dist.ReduceOp.SUM)
    return float(t.item()), float(k.item())


def _pairs_per_walk():
    return sum(min(p, WINDOW) + min(L - 1 - p, WINDOW) for p in range(L))


def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_2606_22180_b300 import build, evaluate, felog as fl

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    fl.load()

    split = _workload(args.scale, rank)
    g = split.train
    dg = fl.DeviceGraph.from_host(g)
    n_live = int((g.degrees() > 0).sum())
    T = ROUNDS * WPR * n_live * L
    prec = fl.FELOG_FP32 if args.precision == "fp32" else fl.FELOG_BF16_SR
    tp = fl.train_params(DIM, WINDOW, NEG, LR0, T, fl.FELOG_SGNS_HOGWILD, 4096, prec, 0, args.form,
                         stage_flush=args.stage_flush)
    fp_plain = fl.feedback_params(False, MU, KS, ROUNDS, False)
    runner = RoundRunner(fl, dg, tp, fp_plain, SEED + rank)
    runner.reset()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for w in range(args.warmup):
        runner.run(w)
    # timed region: K plain rounds
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    barrier()
    start.record()
    tokens = 0
    for k in range(args.steps):
        _, tok = runner.run(args.warmup + k, events=ev[k])
        tokens += tok
    stop.record()
    barrier()
    clocks = sampler.stop()
    ms = start.elapsed_time(stop)
    if world > 1:
        ms, tokens_all = reduce_over_ranks(ms, tokens, "cuda")
    else:
        tokens_all = float(tokens)
    phase = {name: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in ev)
             for i, name in enumerate(["walk", "noise", "train", "feedback"])}
    steps_per_round = n_live * WPR * (L - 1)
    value = tokens_all / (ms / 1e3)

    # roofline of the dominant kernel (SGNS): algorithmic bytes per launch
    row = DIM * (4 if args.precision == "fp32" else 2)
    pairs = n_live * WPR * _pairs_per_walk()
    alg_bytes = row * (4 * n_live * WPR * L + 2 * NEG * pairs)
    achieved = alg_bytes / (phase["train"] / 1e3) / 1e9
    peak, peak_kind = _peaks()
    csrc = os.path.join(ROOT, "paper_2606_22180_b300", "csrc")
    traffic = _profile_traffic([os.path.join(csrc, "sgns.cu"), os.path.join(csrc, "sgns_core.cuh")])
    if args.precision != "fp32" or args.scale != SCALE or args.form not in (0, 2):
        traffic = None  # the committed capture is of the automatic fp32 launch at scale 20

    # end to end through the public call a user makes: one whole embedding
    # job (felog_embed, all rounds) with the CSR copied in from pinned host
    # memory and the embedding phi_in copied back to pinned host memory
    e2e = _e2e_job(fl, g, tp, fp_plain, SEED + rank, world, barrier)
    result = {
        "metric": METRIC,
        "value": value,
        "unit": "tokens/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "bf16 tables, f32 math",
        "data": "synthetic (seeded R-MAT graph; no dataset)",
        "config": {
            "workload": _workload_name(args.scale, args.precision),
            "nodes": g.n, "directed_csr_entries": g.nnz, "non_isolated": n_live,
            "step": "one plain round of Algorithm 1 (walk, counts, alias table, SGNS, Psi, V_a)",
            "l2": "inputs larger than L2 (tables 2 x 512 MiB), no flush",
            "parallelism": "replicas" if world > 1 else "single GPU",
        },
        "walk_steps_per_s": steps_per_round * world / (phase["walk"] / 1e3),
        "tokens_per_s_sgns_kernel": n_live * WPR * L * world / (phase["train"] / 1e3),
        "phase_ms": phase,
        "gpu_launches": RoundRunner.KERNELS_PER_ROUND * args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "dram_frac": (traffic / (phase["train"] / 1e3) / 1e9 / peak) if traffic else None,
                     "bytes_per_launch": alg_bytes,
                     "note": "achieved/frac: algorithmic row bytes (4 rows per token, 2K per pair, window "
                             "truncated at walk ends) per launch / CUDA-event time; rows of hot negatives hit "
                             "in L2, so DRAM traffic (ncu, per launch) is below them and dram_frac is the "
                             "HBM fraction; the launch is bound by the L1-to-L2 request path and L2 "
                             "reductions, not by DRAM",
                     "kernel": _sgns_kernel_name(args.form, args.precision),
                     "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"},
        "e2e": e2e,
        "clocks": clocks,
    }

    # the quality runs, the other forms and the CPU baseline belong to the
    # single-GPU line; under torchrun (N > 1) only the replicated rounds run,
    # so the N GPUs are not held while rank 0 runs them
    single = world == 1
    if not args.no_quality and single:
        result["quality"] = _quality(fl, evaluate, dg, split, n_live, args.form, args.stage_flush)
        q = result["quality"]
        result["chosen_vs_plain"] = {
            "auc_plain": q["plain"]["auc"], "auc_chosen": q["chosen"]["auc"],
            "auc_delta": q["chosen"]["auc"] - q["plain"]["auc"],
            "time_plain_s": q["plain"]["seconds"], "time_chosen_s": q["chosen"]["seconds"],
            "speedup_time_to_result": q["plain"]["seconds"] / q["chosen"]["seconds"],
            "tokens_plain": q["plain"]["tokens"], "tokens_chosen": q["chosen"]["tokens"],
            "chosen": "feedback mu=0.65 + bf16-SR tables, same graph and split",
        }
    if not args.no_forms and single:
        na = int(runner.n_active_h.item())
        result["fabc"] = _fabc_form(fl, runner.walks[: na * WPR * L].view(-1, L), runner.counts)
        result["node2vec"] = _node2vec_form(fl, dg, runner.starts[:na], runner.walks, runner.counts)
        del runner
        torch.cuda.empty_cache()
        # the precision form on the same graph: bf16 tables, stochastic rounding
        result["bf16_round"] = _bf16_rounds(fl, dg, T, args)
        torch.cuda.empty_cache()
        result["tile_form"] = _tile_form(fl, dg, n_live, T)
        torch.cuda.empty_cache()
        del dg
        torch.cuda.empty_cache()
        result["batching"] = run_batch(fl, jobs=512, n_hi=200000, warmup=1, steps=1, autotune=True)
        torch.cuda.empty_cache()
        cap = result["bf16_round"]["tokens_per_s"]
        result["serving"] = run_serve(fl, rate=20.0, duration=20.0, max_nodes=1 << 16, sustainable=True)
        result["serving_large"] = run_serve_large(fl, capacity_tokens_per_s=cap)
        dg = fl.DeviceGraph.from_host(g)
        result["ripp"] = _ripp(fl, evaluate, dg, split, n_live)
        del dg
    if not args.no_cpu and single:
        result["cpu_baseline"] = _cpu_baseline(split, n_live)
        result["vs_cpu_baseline"] = value / result["cpu_baseline"]["value"]
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# batching form: many graphs, one captured launch per run
# ---------------------------------------------------------------------------
BATCH_L, BATCH_W, BATCH_K, BATCH_ROUNDS = 40, 5, 5, 10


def run_batch(fl, jobs=512, n_hi=200000, warmup=1, steps=1, autotune=True, seed=3, persistent=True):
    """The batching workload: `jobs` graphs (half planted partitions with
    4..32 communities, half R-MAT), node counts log-uniform in [1e3, n_hi],
    average degree 8..32, d in {64, 128}, bf16 tables, 10 walks per node of
    length 40, window 5, 5 negatives; all rounds of all graphs in one
    captured CUDA graph.  A step is one launch of that graph."""
    import torch

    from paper_2606_22180_b300 import inputs

    t0 = time.perf_counter()
    mix = inputs.graph_mix(jobs, seed, 1000, n_hi, workers=_gen_workers())
    gen_s = time.perf_counter() - t0
    dgs = [fl.DeviceGraph.from_host(g) for g, _ in mix]
    dims = [d for _, d in mix]
    tp = fl.train_params(128, BATCH_W, BATCH_K, LR0, 0, fl.FELOG_SGNS_HOGWILD, 4096, fl.FELOG_BF16_SR)
    fp = fl.feedback_params(False, MU, KS, BATCH_ROUNDS, False)
    b = fl.Batch(dgs, dims, [SEED + i for i in range(jobs)], BATCH_L, 1, tp, fp)
    os.makedirs(os.path.join(ROOT, "_build"), exist_ok=True)
    tuning = b.autotune(os.path.join(ROOT, "_build", "felog_tune.txt")) if autotune else None
    stream = torch.cuda.Stream()

    def timed(persistent):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                b.run(use_graph=True, persistent=persistent)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                b.run(use_graph=True, persistent=persistent)
            e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / steps
        stats, _, _ = b.read()
        return ms, sum(s["tokens"] for s in stats)

    ms, tokens = timed(False)
    out = {"workload": f"{jobs} graphs (SBM/R-MAT), |V| log-uniform [1e3, {n_hi}], deg 8-32, d 64/128 bf16, "
                       f"L={BATCH_L}, {BATCH_ROUNDS} rounds, w={BATCH_W}, K={BATCH_K}",
           "nodes": int(sum(g.n for g, _ in mix)), "tokens_per_run": int(tokens),
           "ms_per_run": ms, "tokens_per_s": tokens / (ms / 1e3), "launch": "one CUDA graph per run",
           "warmup_runs": warmup, "timed_runs": steps, "tuning": tuning, "graph_gen_s": gen_s,
           "device_bytes": b.device_bytes()}
    if persistent:
        pms, ptok = timed(True)
        out["persistent"] = {"launch": "one persistent kernel per run (all rounds, grid-wide barriers)",
                             "ms_per_run": pms, "tokens_per_run": int(ptok), "tokens_per_s": ptok / (pms / 1e3)}
    b.close()
    return out


# ---------------------------------------------------------------------------
# serving form: Poisson arrivals into the continuous-batching server
# ---------------------------------------------------------------------------
def run_serve(fl, rate=20.0, duration=20.0, max_nodes=1 << 16, pool_size=48, budget=150 << 30, seed=4,
              sustainable=True, pool=None):
    """Requests arrive as a Poisson process at `rate` per second for
    `duration` seconds; each is a graph drawn from a pool (half SBM, half
    R-MAT, node counts log-uniform in [1e3, max_nodes]) with its own seed,
    trained with the round workload's walk/SGNS parameters, d = 128, bf16
    tables, feedback mu = 0.65.  Reports latency percentiles over completed
    requests and offered vs completed load."""
    from paper_2606_22180_b300 import inputs

    if pool is None:
        pool = inputs.graph_mix(pool_size, seed, 1000, max_nodes, dims=(128,), workers=_gen_workers())
    pool_size = len(pool)
    max_nodes = max(g.n for g, _ in pool)
    tp = fl.train_params(DIM, WINDOW, NEG, LR0, 0, fl.FELOG_SGNS_HOGWILD, 4096, fl.FELOG_BF16_SR)
    fp = fl.feedback_params(True, MU, KS, ROUNDS, False)

    def one(rate_):
        rng = np.random.default_rng(seed)
        sv = fl.Server(budget, L, WPR, tp, fp)
        t_arr, ids, offered_tokens = 0.0, [], 0
        start = time.perf_counter()
        while True:
            t_arr += rng.exponential(1.0 / rate_)
            if t_arr > duration:
                break
            g, _ = pool[int(rng.integers(0, pool_size))]
            while time.perf_counter() - start < t_arr:
                time.sleep(0.0005)
            ids.append(sv.submit(g, DIM, int(rng.integers(1 << 62))))
            offered_tokens += int((g.degrees() > 0).sum()) * L * ROUNDS
        sv.drain(3600)
        wall = time.perf_counter() - start
        res = [sv.wait(r, 60) for r in ids]
        st = sv.stats()
        sv.close()
        done = [r for r in res if r["state"] == fl.JOB_DONE]
        lat = np.array([r["t_done"] - r["t_submit"] for r in done])
        tokens = sum(r["tokens"] for r in done)
        return {"rate_per_s": rate_, "requests": len(ids), "completed": len(done),
                "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
                "offered_tokens_per_s_full_schedule": offered_tokens / duration,
                "completed_tokens_per_s": tokens / wall, "wall_s": wall,
                "peak_resident_jobs": st["peak_resident_jobs"], "steps": st["steps"],
                "peak_resident_gib": st["peak_resident_bytes"] / 2 ** 30,
                "busy_s": st["busy_seconds"],
                "busy_tokens_per_s": tokens / st["busy_seconds"] if st["busy_seconds"] else None}

    lo_nodes = min(g.n for g, _ in pool)
    out = {"workload": f"Poisson {rate:.4g}/s for {duration}s over a pool of {pool_size} SBM/R-MAT graphs "
                       f"(|V| drawn log-uniform; the pool spans {lo_nodes}..{max_nodes} nodes), "
                       f"L={L}, w={WINDOW}, K={NEG}, d={DIM} bf16, "
                       f"feedback mu={MU}, budget {budget >> 30} GiB",
           "stated": one(rate)}
    if sustainable:
        # capacity: tokens per second of server busy time at the stated rate
        cap = out["stated"]["busy_tokens_per_s"] or out["stated"]["completed_tokens_per_s"]
        mean_tokens = np.mean([int((g.degrees() > 0).sum()) * L * ROUNDS for g, _ in pool])
        out["sustainable"] = one(max(0.5, 0.7 * cap / mean_tokens))
    return out


def _gen_workers():
    return max(1, min(32, (os.cpu_count() or 1) - 1))


def run_serve_large(fl, capacity_tokens_per_s, duration=60.0, n_lo=1 << 15, n_hi=1 << 22, pool_size=12,
                    budget=150 << 30, seed=5):
    """Serving with large jobs: requests on graphs with |V| log-uniform in
    [2^15, 2^22] (up to about 6 GB of device memory each), the round
    workload's parameters, d = 128 bf16, feedback mu = 0.65, arriving as a
    Poisson process at 0.7 x the measured capacity (capacity_tokens_per_s /
    mean tokens per job) for `duration` seconds."""
    from paper_2606_22180_b300 import inputs

    pool = inputs.graph_mix(pool_size, seed, n_lo, n_hi, dims=(128,), workers=_gen_workers())
    mean_tokens = float(np.mean([int((g.degrees() > 0).sum()) * L * ROUNDS for g, _ in pool]))
    rate = 0.7 * capacity_tokens_per_s / mean_tokens
    out = run_serve(fl, rate=rate, duration=duration, budget=budget, seed=seed, sustainable=False,
                    pool=pool)
    out["rate_rule"] = (f"0.7 x measured capacity {capacity_tokens_per_s:.3g} tokens/s (bf16 round) / "
                        f"{mean_tokens:.3g} tokens per job (feedback off; mu = 0.65 trains fewer)")
    out["job_nodes"] = f"log-uniform [{n_lo}, {n_hi}]"
    out["largest_job_nodes"] = int(max(g.n for g, _ in pool))
    return out


TILE_NS = 512


MU_GRID = (0.5, 0.6, 0.65, 0.7, 0.8, 0.9)


def run_mu_sweep(fl, evaluate, seed=5):
    """Feedback threshold mu (Eq. 5) on synthetic graphs of three kinds:
    homophilic planted partition (20 communities, p_in / p_out = 20),
    heterophilic planted partition (2 communities, p_in / p_out = 1/20: most
    edges cross, close to bipartite) and R-MAT scale 16.  Edges: 10 % test,
    then 10 % of the rest validation.  For each mu (and feedback off, and
    mu = 0.65 with reactivation) one run of Algorithm 1: trained tokens, wall
    time, validation and test AUC.  The validation-calibrated mu is the one
    with the fewest tokens whose validation AUC is within 0.005 of feedback
    off; its test AUC and token saving are reported."""
    import torch

    from paper_2606_22180_b300 import inputs

    graphs = {
        "sbm_homophilic": inputs.sbm_degree(20000, 20, 16, seed, ratio=20.0),
        "sbm_heterophilic": inputs.sbm_degree(20000, 2, 16, seed, ratio=0.05),
        "rmat16": inputs.rmat(16, 16, seed=seed),
    }
    Lm, R = 40, 10
    out = {"workload": f"L={Lm}, {R} rounds, w=5, K=5, d=64 fp32 Hogwild; 10 % test, 10 % validation edges",
           "graphs": {}}
    for name, g in graphs.items():
        test = inputs.link_split(g, 0.1, seed)
        val = inputs.link_split(test.train, 0.1, seed + 1)
        dg = fl.DeviceGraph.from_host(val.train)
        n_live = int((val.train.degrees() > 0).sum())
        T = R * n_live * Lm
        runs = {}
        settings = [("off", False, 0.65, False)] + [(f"mu={m}", True, m, False) for m in MU_GRID] + \
                   [("mu=0.65 reactivate", True, 0.65, True)]
        for label, enabled, mu, react in settings:
            tp = fl.train_params(64, 5, 5, LR0, T, fl.FELOG_SGNS_HOGWILD, 4096, fl.FELOG_FP32)
            fp = fl.feedback_params(enabled, mu, KS, R, react)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pi, _, st = fl.felog_embed(dg, Lm, 1, tp, fp, seed)
            torch.cuda.synchronize()
            runs[label] = {"tokens": int(sum(x["tokens"] for x in st)), "rounds": len(st),
                           "seconds": time.perf_counter() - t0,
                           "active_per_round": [x["n_active"] for x in st],
                           "auc_val": evaluate.link_auc(pi, val.pos, val.neg),
                           "auc_test": evaluate.link_auc(pi, test.pos, test.neg)}
            del pi
        base = runs["off"]
        ok = [k for k in runs if k.startswith("mu=") and runs[k]["auc_val"] >= base["auc_val"] - 0.005]
        pick = min(ok, key=lambda k: runs[k]["tokens"]) if ok else "off"
        out["graphs"][name] = {
            "nodes": g.n, "runs": runs, "calibrated": pick,
            "calibrated_auc_test_delta": runs[pick]["auc_test"] - base["auc_test"],
            "calibrated_token_fraction": runs[pick]["tokens"] / base["tokens"],
        }
    return out


def _node2vec_form(fl, dg, starts, walks, counts, reps=3, p=0.5, q=2.0):
    """node2vec walks (Sample variant) over the same starts as a round: walk
    steps per second (CUDA events), next to the uniform walk kernel's."""
    import torch

    n = starts.numel()
    out = walks[: n * WPR * L].view(-1, L)
    fl.felog_walk_node2vec(dg, starts, n, L, WPR, p, q, SEED, 0, counts=counts, out=out)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for r in range(reps):
        counts.zero_()
        fl.felog_walk_node2vec(dg, starts, n, L, WPR, p, q, SEED, r + 1, counts=counts, out=out)
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    steps = n * WPR * (L - 1)
    return {"workload": f"{n} starts x {WPR} walks x {L} nodes on the round graph, p={p}, q={q}",
            "ms_per_launch": ms, "walk_steps_per_s": steps / (ms / 1e3)}


def _fabc_form(fl, walks, counts, reps=5):
    """FaBC (Section 5.2.2) on the last round's corpus: the Eq. 8 selection
    and, for it and for a forced top-2, the encoded size against the raw
    4 N L bytes (Eq. 7) and the encode / decode rates (CUDA events; bytes =
    the walks read plus the encoded bytes written, or the reverse)."""
    import torch

    N, Lw = walks.shape
    ids, F = fl.felog_fabc_select(counts, Lw, 32)
    peak, _ = _peaks()
    out = {"workload": f"one plain round of the round workload: {N} walks x {Lw}",
           "eq8": {"k": len(ids), "F_k": F, "g_k": 1 - F + len(ids) / Lw + len(ids) / 32}}
    top2 = torch.topk(counts.long(), 2).indices.tolist()
    ws = fl.fabc_workspace(N, walks.device)
    for name, sel in (("eq8", ids), ("top2", top2)):
        ids_d = torch.tensor(sel, dtype=torch.int32, device=walks.device)
        k = len(sel)
        buf, tail = fl.felog_fabc_encode(walks, ids_d, workspace=ws)
        size = fl.fabc_encoded_bytes(N, Lw, k, int(tail.item()))
        back = fl.felog_fabc_decode(buf[:size], N, Lw, k, workspace=ws)
        ok = bool(torch.equal(back, walks))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        for _ in range(reps):  # output, tail count and workspace reused, as a caller streaming rounds would
            fl.felog_fabc_encode(walks, ids_d, workspace=ws, out=buf, tail=tail)
        ev[1].record()
        for _ in range(reps):
            fl.felog_fabc_decode(buf[:size], N, Lw, k, walks=back, workspace=ws)
        ev[2].record()
        torch.cuda.synchronize()
        t_enc = ev[0].elapsed_time(ev[1]) / reps / 1e3
        t_dec = ev[1].elapsed_time(ev[2]) / reps / 1e3
        raw = 4 * N * Lw
        out[name] = {"k": k, "ratio": size / raw, "round_trip_exact": ok,
                     "encode_ms": t_enc * 1e3, "decode_ms": t_dec * 1e3,
                     "encode_gbs": (raw + size) / t_enc / 1e9, "decode_gbs": (raw + size) / t_dec / 1e9,
                     "encode_frac_hbm": (raw + size) / t_enc / 1e9 / peak}
    return out


def _tile_flops(n_tiles, dim, ns):
    """Tensor-core FLOPs of the tile trainer: per tile and per 128-column
    block (positions, then Ns / 128 blocks of negatives) S_b = X Y_b^T,
    dX += G_b Y_b and dY_b = G_b^T X, each 128 x 128 x dim."""
    blocks = 1 + ns // 128
    return n_tiles * blocks * 3 * 2 * 128 * 128 * dim


def _tile_form(fl, dg, n_live, T, steps=3, warmup=2, scale=SCALE, full=True):
    """The shared-negatives tile trainer (TILE mode, bf16 tables) on the same
    graph: plain rounds timed with CUDA events per phase; its tensor FLOP/s
    against the measured bf16 peak and its gathered/added row bytes against
    HBM bandwidth.  The automatic concurrency cap is the quality-preserving
    setting; `full` adds the same measurement with one tile per SM (the
    kernel's speed; lower AUC)."""
    out = _tile_rounds(fl, dg, T, steps, warmup, scale, 0)
    if full:
        full_ctas = _sm_count()
        out["one_tile_per_sm"] = _tile_rounds(fl, dg, T, steps, warmup, scale, full_ctas)
    return out


def _sm_count():
    import torch

    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def _tile_rounds(fl, dg, T, steps, warmup, scale, ctas):
    import torch

    tp = fl.train_params(DIM, WINDOW, NEG, LR0, T, fl.FELOG_SGNS_TILE, 1, fl.FELOG_BF16_SR,
                         tile_negatives=TILE_NS, tile_ctas=ctas)
    runner = RoundRunner(fl, dg, tp, fl.feedback_params(False, MU, KS, ROUNDS, False), SEED)
    runner.reset()
    for w in range(warmup):
        runner.run(w)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tokens = 0
    for k in range(steps):
        _, tok = runner.run(warmup + k, events=ev[k])
        tokens += tok
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    train_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in ev)
    tok_round = tokens / steps
    tc = 128 - 2 * WINDOW
    n_tiles = -(-tok_round // tc)
    flops = _tile_flops(n_tiles, DIM, TILE_NS)
    row = DIM * 2
    alg_bytes = n_tiles * 2 * (128 + tc + TILE_NS) * row
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    bf16_peak = float(peaks.get("bf16_tflops_sustained", 1400.0))
    hbm_peak, _ = _peaks()
    tflops = flops / (train_ms / 1e3) / 1e12
    gbs = alg_bytes / (train_ms / 1e3) / 1e9
    out = {
        "workload": f"{_workload_name(scale, 'bf16')}, TILE mode, Ns={TILE_NS} shared negatives per tile of {tc} centers",
        "concurrent_tiles": ctas if ctas else f"automatic: min(SMs, n / 28000) = {min(_sm_count(), max(1, dg.n // 28000))}",
        "tokens_per_round": tok_round,
        "round_tokens_per_s": tokens / sec,
        "train_ms": train_ms,
        "tokens_per_s_train_kernel": tok_round / (train_ms / 1e3),
        "tiles_per_launch": n_tiles,
        "tensor": {"achieved": tflops, "peak": bf16_peak, "unit": "TFLOP/s", "frac": tflops / bf16_peak,
                   "flops_per_launch": flops, "peak_source": "measured bf16 sustained (cuBLAS)"},
        "rows": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                 "bytes_per_launch": alg_bytes},
        "kernel": "k_sgns_tile<128,bf16>",
    }
    del runner
    return out


def _quality(fl, evaluate, dg, split, n_live, form=0, stage_flush=0):
    """Full runs of Algorithm 1: plain (feedback off, fp32, the timed rounds'
    Hogwild form), plain_bf16 (the same in bf16 with stochastic rounding) and
    chosen (feedback mu = 0.65, bf16 with stochastic rounding, the automatic
    form); AUC on the held-out edges, wall time of the felog_embed call."""
    import torch

    out = {}
    T = ROUNDS * WPR * n_live * L
    forms = {
        "plain": (fl.train_params(DIM, WINDOW, NEG, LR0, T, fl.FELOG_SGNS_HOGWILD, 4096, fl.FELOG_FP32,
                                  0, form, stage_flush=stage_flush),
                  fl.feedback_params(False, MU, KS, ROUNDS, False)),
        "plain_bf16": (fl.train_params(DIM, WINDOW, NEG, LR0, T, fl.FELOG_SGNS_HOGWILD, 4096, fl.FELOG_BF16_SR,
                                       0, form, stage_flush=stage_flush),
                       fl.feedback_params(False, MU, KS, ROUNDS, False)),
        "chosen": (fl.train_params(DIM, WINDOW, NEG, LR0, T, fl.FELOG_SGNS_HOGWILD, 4096, fl.FELOG_BF16_SR),
                   fl.feedback_params(True, MU, KS, ROUNDS, False)),
        "tile": (fl.train_params(DIM, WINDOW, NEG, LR0, T, fl.FELOG_SGNS_TILE, 1, fl.FELOG_BF16_SR,
                                 tile_negatives=TILE_NS),
                 fl.feedback_params(False, MU, KS, ROUNDS, False)),
        "tile_one_per_sm": (fl.train_params(DIM, WINDOW, NEG, LR0, T, fl.FELOG_SGNS_TILE, 1, fl.FELOG_BF16_SR,
                                            tile_negatives=TILE_NS, tile_ctas=_sm_count()),
                            fl.feedback_params(False, MU, KS, ROUNDS, False)),
    }
    for name, (tp, fp) in forms.items():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pi, po, st = fl.felog_embed(dg, L, WPR, tp, fp, SEED)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        tokens = sum(s["tokens"] for s in st)
        out[name] = {
            "auc": evaluate.link_auc(pi, split.pos, split.neg),
            "rounds": len(st),
            "active_per_round": [s["n_active"] for s in st],
            "tokens": tokens,
            "seconds": sec,
            "tokens_per_s": tokens / sec,
            "loss_per_round": [s["loss"] for s in st],
        }
        del pi, po
    return out


def _cpu_round(g, n_live, seed, rnd, pi, po, sgns_walks, psi_nodes, T):
    """One round of the round workload by the oracle's routines on every host
    core (oracle/felog_cpu_baseline.c): all walks (OpenMP), corpus counts and
    the alias table (serial oracle), Hogwild SGNS in binary64 over the first
    `sgns_walks` walks, Psi of the first `psi_nodes` nodes.  Returns the
    measured seconds of each part and the sizes behind them."""
    import oracle

    starts = np.nonzero(g.degrees() > 0)[0].astype(np.int32)
    t0 = time.perf_counter()
    W = oracle.baseline_walk(g.offsets, g.cols, starts, L, seed, rnd)
    t1 = time.perf_counter()
    _, thr, alias, S = oracle.noise_table(oracle.counts(W, g.n))
    t2 = time.perf_counter()
    Ws = W[:sgns_walks]
    oracle.baseline_sgns_hogwild(Ws, g.n, DIM, WINDOW, NEG, LR0, T, thr, alias, S, seed, rnd, 0, pi, po)
    t3 = time.perf_counter()
    oracle.baseline_psi(g.offsets, g.cols, pi, KS, seed, rnd, starts[:psi_nodes])
    t4 = time.perf_counter()
    return {"walk_s": t1 - t0, "noise_s": t2 - t1, "sgns_s": t3 - t2, "psi_s": t4 - t3,
            "walks": int(W.shape[0]), "sgns_tokens": int(Ws.size), "psi_nodes": int(min(psi_nodes, starts.shape[0]))}


def _cpu_round_rate(r, n_live):
    """Tokens per second of a whole round, the sampled parts scaled to the
    round: walks, counts and table measured whole; SGNS and Psi per sampled
    token and node."""
    tokens = n_live * WPR * L
    sec = (r["walk_s"] + r["noise_s"] + r["sgns_s"] * tokens / r["sgns_tokens"]
           + r["psi_s"] * n_live / r["psi_nodes"])
    return tokens / sec, sec


def _cpu_baseline(split, n_live):
    """The oracle on every host core (threads reported): a whole round's walks
    and alias table, Hogwild SGNS on a sample of about 3,000 walks per thread
    (some 10-30 s of binary64 work), Psi on 5,000 nodes per thread; the
    sampled parts are scaled to the round."""
    import oracle

    g = split.train
    threads = oracle.baseline_threads()
    pi, po = oracle.init_tables(g.n, DIM, SEED)
    T = ROUNDS * WPR * n_live * L
    r = _cpu_round(g, n_live, SEED, 0, pi, po, sgns_walks=3000 * threads, psi_nodes=5000 * threads, T=T)
    value, sec = _cpu_round_rate(r, n_live)
    return {"value": value, "unit": "tokens/s", "cores": threads, "host_cpus": os.cpu_count(),
            "kind": "oracle",
            "sample": f"one round of the round workload: all {r['walks']} walks (OpenMP) and the alias table "
                      f"measured whole; binary64 Hogwild SGNS on the first {r['sgns_tokens']} tokens and Psi "
                      f"on {r['psi_nodes']} nodes, scaled to the round's {n_live * WPR * L} tokens",
            "walk_steps_per_s": r["walks"] * (L - 1) / r["walk_s"],
            "sgns_tokens_per_s": r["sgns_tokens"] / r["sgns_s"],
            "round_seconds_estimated": sec, "measured": r}


def run_reference(args):
    """The oracle, as it stands, on every host core: each step one round of
    the round workload with SGNS and Psi on a bounded sample (see
    _cpu_round), reported as whole-round tokens/s.  Under torchrun only rank
    0 runs."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    split = _workload(args.scale)
    g = split.train
    n_live = int((g.degrees() > 0).sum())
    threads = oracle.baseline_threads()
    pi, po = oracle.init_tables(g.n, DIM, SEED)
    T = ROUNDS * WPR * n_live * L
    sw, pn = 256 * threads, 2000 * threads

    rates, secs = [], []
    for k in range(args.warmup + args.steps):
        r = _cpu_round(g, n_live, SEED, k % 65536, pi, po, sgns_walks=sw, psi_nodes=pn, T=T)
        if k >= args.warmup:
            v, _ = _cpu_round_rate(r, n_live)
            rates.append(v)
            secs.append(r["walk_s"] + r["noise_s"] + r["sgns_s"] + r["psi_s"])  # measured wall of the step
    v = float(np.mean(rates))
    sample = (f"each step one round of the round workload on {threads} threads: all walks (OpenMP) and the alias "
              f"table whole, binary64 Hogwild SGNS on {sw} walks and Psi on {pn} nodes, scaled to the round")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "tokens/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded R-MAT graph; no dataset)",
        "config": {"workload": _workload_name(args.scale)},
        "cpu_baseline": {"value": v, "unit": "tokens/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "tokens/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_form(args):
    """--mode tile / batch / serve / mu: one JSON line for that form."""
    import torch

    from paper_2606_22180_b300 import build, felog as fl

    build.build()
    fl.load()
    torch.cuda.set_device(0)
    if args.mode == "mu":
        from paper_2606_22180_b300 import evaluate

        r = run_mu_sweep(fl, evaluate)
        line = {"metric": "trained tokens and link AUC per feedback threshold mu", "value": None,
                "unit": "tokens", "n_gpus": 1, "higher_is_better": False, "dtype": "f32",
                "data": "synthetic (seeded SBM and R-MAT graphs)", "config": {"workload": r["workload"]},
                "mu_sweep": r}
    elif args.mode == "tile":
        split = _workload(args.scale)
        dg = fl.DeviceGraph.from_host(split.train)
        n_live = int((split.train.degrees() > 0).sum())
        r = _tile_form(fl, dg, n_live, ROUNDS * WPR * n_live * L, steps=args.steps, warmup=args.warmup,
                       scale=args.scale)
        line = {"metric": "SGNS tokens/s, shared-negatives tile form", "value": r["round_tokens_per_s"],
                "unit": "tokens/s", "n_gpus": 1, "higher_is_better": True, "dtype": "bf16 tables, f32 math",
                "data": "synthetic (seeded R-MAT graph; no dataset)", "config": {"workload": r["workload"]},
                "tile_form": r}
    elif args.mode == "batch":
        r = run_batch(fl, jobs=args.jobs, warmup=1, steps=1, persistent=not args.no_persistent)
        line = {"metric": "SGNS tokens/s, batching form", "value": r["tokens_per_s"], "unit": "tokens/s",
                "n_gpus": 1, "higher_is_better": True, "dtype": "bf16 tables, f32 math",
                "data": "synthetic (seeded SBM/R-MAT mix)", "config": {"workload": r["workload"]}, "batching": r}
    else:
        r = run_serve(fl, rate=args.rate, duration=args.duration, max_nodes=args.max_nodes)
        line = {"metric": "p50/p99 latency and completed tokens/s, serving form",
                "value": r["stated"]["completed_tokens_per_s"], "unit": "tokens/s", "n_gpus": 1,
                "higher_is_better": True, "dtype": "bf16 tables, f32 math",
                "data": "synthetic (seeded SBM/R-MAT pool)", "config": {"workload": r["workload"]}, "serving": r}
    print(json.dumps(line))


if __name__ == "__main__":
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.mode != "round":
        run_form(a)
    else:
        run_native(a)
