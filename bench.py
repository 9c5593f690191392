#!/usr/bin/env python3
"""Benchmark: Parallel CFR iterations per second on GB300.

Default workload (one "step"): batched serving of 256 independent river subgames of uneven
size in one handle -- seeded 5-card boards, 1081 two-card hands per player with seeded
integer showdown strengths in [0, 2000), Dirichlet(1) ranges, 1-4 pot-fraction bet sizes
plus all-in, stacks 100-1000, 21-315 public nodes each -- solved together by DCFR (alpha
1.5, beta 0, gamma 2) from scratch: reset, 500 alternating iterations of every subgame
(every stage of the paper's pipeline, Section 4.1), then the best-response exploitability
pass of every subgame.  `value` is subgame-iterations per second of device time over the K
timed steps (the state of all subgames, about 2.5 GB, is larger than L2, and L2 is also
flushed between steps with a 256 MB write outside the timed events).  The launch tiling is
autotuned before the timed region.

Under torchrun each rank solves its own batch (seeds offset by rank) with no collective:
weak scaling, value = all ranks' subgame-iterations / the slowest rank's time.

`--impl reference` times the FP64 CPU oracle (the paper publishes no code, so the oracle is
the reference implementation) on a bounded sample of the same workload instead, on the
host cores.

Other workloads (`--workload`): `river` (one 1081-hand river subgame, pot 100, stacks 400,
bet sizes {0.5, 1.0 pot, all-in}, at most 3 bets or raises, 1000 iterations per step),
`leaf` and `flop` (depth-limited turn and flop subgames with the BF16 leaf network, against
the exact subgames), `gemm` (the network's layers).
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CFR iters/sec (ms/iter) per GB300 at fixed exploitability vs plain exact form; HBM GB/s"
BB_CHIPS = 100.0  # big blind used for mbb/hand (the pot is 100 chips)
L2_FLUSH_BYTES = 256 << 20
SCHEDULE_NAMES = {1: "level", 2: "stream", 3: "wide", 4: "resident"}  # cfr_schedule's values (include/pcfr.h)


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["river", "batch", "leaf", "flop", "gemm"], default="batch",
                    help="batch (default): 256 uneven river subgames in one handle; river: one 1081-hand river "
                         "subgame; "
                         "leaf: depth-limited turn subgame with the BF16 leaf network, against the exact turn; "
                         "flop: depth-limited flop subgame (leaves at the river card), against the exact flop; "
                         "gemm: the leaf network's dense layers alone")
    ap.add_argument("--batch-size", type=int, default=256)
    ap.add_argument("--iters-per-step", type=int, default=None, help="default 1000 (river) or 500 (batch)")
    ap.add_argument("--precision", choices=["pairs", "single"], default=None,
                    help="values as FP32 pairs or plain FP32 (R and S are FP64 either way); default FP32, "
                         "the precision the method's values are specified in")
    ap.add_argument("--chunk-hands", type=int, default=0)
    ap.add_argument("--schedule", choices=["auto", "level", "stream", "wide", "resident"], default="auto")
    ap.add_argument("--warp-hands", type=int, choices=[0, 32, 64], default=0,
                    help="stream schedule: hands per warp (0 = automatic)")
    ap.add_argument("--term-nodes", type=int, choices=range(0, 9), default=0,
                    help="terminal nodes per block of the terminal launch (0 = automatic)")
    ap.add_argument("--runout-tables", choices=["on", "off"], default="on",
                    help="flop: evaluate the all-in run-outs by win-minus-loss tables (wide schedule) or board "
                         "by board")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-autotune", action="store_true",
                    help="batch: keep the automatic layout instead of running the launch-tiling autotuner")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ distributed plumbing

def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def dist_init(world: int, use_cuda: bool):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group("nccl" if use_cuda else "gloo")
    return dist


def max_over_ranks(x: float, dist, device=None) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist, device=None):
    if dist is not None:
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def aggregate(iters_local: int, seconds_local: float, world: int, dist, device=None) -> tuple[float, float]:
    """Whole-job throughput: all ranks' iterations / the slowest rank's time."""
    t = max_over_ranks(seconds_local, dist, device)
    return iters_local * world / t, t


# ------------------------------------------------------------------ workload

def workload_spec(rank: int = 0):
    from paper_2605_19928_gb300 import synth
    return synth.river_subgame(seed=0 + 1000 * rank, range_seed=1 + 1000 * rank)


def workload_specs(args, rank: int = 0):
    from paper_2605_19928_gb300 import synth
    if args.workload == "batch":
        return synth.batch_rivers(args.batch_size, seed=rank)
    return [workload_spec(rank)]


def workload_config(args, spec, n_nodes):
    return {"workload": "river subgame, exact (no depth limit)", "board_cards": 5, "hands": spec.n_hands,
            "public_nodes": n_nodes, "pot": spec.pot, "stack": spec.stack, "bet_sizes": "0.5,1.0 pot,all-in",
            "max_raises": spec.max_raises, "variant": "DCFR(1.5,0,2) alternating",
            "iters_per_step": args.iters_per_step, "step": "reset + iterations + exploitability",
            "values": "fp32 pairs" if args.precision == "pairs" else "fp32",
            "l2": "flushed between steps (256 MB write, outside the timed events)",
            "seeds": spec.seeds}


def batch_config(args, specs, shapes):
    nodes = [sh["nodes"] for sh in shapes]
    return {"workload": f"batched serving: {len(specs)} uneven river subgames in one handle, exact",
            "subgames": len(specs), "hands": specs[0].n_hands, "public_nodes_min_median_max":
                [min(nodes), sorted(nodes)[len(nodes) // 2], max(nodes)], "public_nodes_total": sum(nodes),
            "pot": 100.0, "stacks": "100-1000", "bet_sizes": "1-4 pot fractions + all-in", "max_raises": "2-3",
            "variant": "DCFR(1.5,0,2) alternating", "iters_per_step": args.iters_per_step,
            "step": "reset + iterations + exploitability, all subgames together",
            "values": "fp32 pairs" if args.precision == "pairs" else "fp32",
            "l2": "inputs larger than L2 (state of all subgames) and 256 MB flush between steps",
            "seeds": {"batch": "synth.batch_rivers(seed=rank)", "boards_strengths": "1000+k", "ranges": "5000+k"}}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0, period_ms: int = 100):
        self.index, self.period_ms = index, period_ms
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", f"-lms={self.period_ms}",
                                          f"--filename={self.path}"],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(self.period_ms / 1000.0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if _num(r[3]))}


def _num(x):
    try:
        float(x)
        return True
    except ValueError:
        return False


# ------------------------------------------------------------------ roofline

def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def bf16_peak(sustained: bool = False):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
        if key in d:
            return float(d[key]), "measured " + key
    return (1700.0 if sustained else 1900.0), "fallback"


def tree_shape(capi, tree, game: int = 0):
    n_nodes, n_hands, _ = capi.cfr_tree_info(tree, game)
    rows = [0, 0]
    ends = 0
    for n in range(n_nodes):
        info = capi.cfr_node_info(tree, n, game)
        if info["type"] == capi.CFR_NODE_DECISION:
            rows[info["player"]] += info["n_actions"]
        elif info["type"] in (capi.CFR_NODE_FOLD, capi.CFR_NODE_SHOWDOWN, capi.CFR_NODE_LEAF):
            ends += 1
    return {"nodes": n_nodes, "hands": n_hands, "rows": rows, "terminals": ends}


def algorithmic_bytes(shape, stage: str, value_bytes: int = 4) -> float:
    """Algorithmic bytes of one launch, from the per-unit figures of the traversal:
    per (decision row, hand) and iteration R and S read + written (32 B) and the strategy
    written once and read by the two traversals (3 V); per (node, hand) and traversal the
    reach written + read and the value written + read (4 V).  With V = 4 (FP32 values) that
    is 44 B per row-hand and 32 B per node-hand per iteration.  An update launch (one
    player) owns its player's rows and one traversal's inner nodes, a terminal launch one
    traversal's terminal nodes; the figures are the mean over the two players' launches."""
    H, V = shape["hands"], value_bytes
    rows = 0.5 * (shape["rows"][0] + shape["rows"][1])
    inner = shape["nodes"] - shape["terminals"]
    if stage == "update":
        return H * (rows * (32 + 3 * V) + inner * 4 * V)
    if stage == "terminal":
        return H * shape["terminals"] * 4 * V
    raise ValueError(stage)


def without_sections(text: str, names) -> str:
    """kernels.cu without the named sections: a section runs from its header line
    ('// ----- name') to the next header."""
    out, skip = [], False
    for line in text.splitlines(keepends=True):
        m = re.match(r"// -{10,} (.+)$", line.rstrip("\n"))
        if m:
            skip = m.group(1).strip() in names
        if not skip:
            out.append(line)
    return "".join(out)


def kernels_digest(exclude=()) -> str:
    """First 16 hex digits of the sha256 of the kernel sources (kernels.cu, then
    pcfr_internal.h), leaving out the sections of kernels.cu named in `exclude`: the digest
    of a profiled kernel that uses none of them stays the same when only they change."""
    h = hashlib.sha256()
    for name in ("kernels.cu", "pcfr_internal.h"):
        with open(os.path.join(ROOT, "paper_2605_19928_gb300", "csrc", name), "rb") as f:
            data = f.read()
        if name == "kernels.cu" and exclude:
            data = without_sections(data.decode(), set(exclude)).encode()
        h.update(data)
    return h.hexdigest()[:16]


def profiled_traffic(stage: str, workload: str = "river1081"):
    """DRAM bytes per launch from the committed ncu summary, if it matches these kernels
    (its digest, over the sources without the sections it names as unused by its kernel)."""
    path = os.path.join(ROOT, "profiles", f"{stage}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"kernels_digest:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    x = re.search(r"kernels_digest_excludes:\s*(.+)", text)
    exclude = tuple(n.strip() for n in x.group(1).split(",")) if x else ()
    if not m or not t or m.group(1) != kernels_digest(exclude):
        return None
    return float(t.group(1))


# ------------------------------------------------------------------ oracle (CPU) timing

def oracle_sample(spec, seconds: float, threads: int | None = None):
    """Time the FP64 oracle as it stands on this host: iterations of the same solve until
    the budget is spent, then one exploitability pass."""
    from oracle.oracle import Oracle
    orc = Oracle(spec, variant="dcfr", alternating=True, threads=threads)
    t0 = time.perf_counter()
    n = 0
    while True:
        orc.iterate(1)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    t_iter = time.perf_counter() - t0
    e = orc.exploitability()[0]
    t_all = time.perf_counter() - t0
    return {"iters": n, "seconds": t_all, "iter_seconds": t_iter, "threads": orc.threads, "expl": e}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    batch = args.workload == "batch"
    specs = workload_specs(args, 0)
    picks = sorted(set(int(k * len(specs) / 4) for k in range(4))) if batch else [0]
    budget = max(1.0, args.cpu_seconds / 4)
    for k in range(args.warmup):
        oracle_sample(specs[picks[k % len(picks)]], budget / 4)
    total_iters, total_s, threads = 0, 0.0, 1
    for k in range(args.steps):
        r = oracle_sample(specs[picks[k % len(picks)]], budget)
        total_iters += r["iters"]
        total_s += r["seconds"]
        threads = r["threads"]
    value = total_iters / total_s
    unit = "subgame iter/s" if batch else "iter/s"
    what = f"subgames {picks} of the {len(specs)}-subgame batch in turn" if batch else "the 1081-hand river subgame"
    from oracle.oracle import Oracle
    nodes = [Oracle(s, variant="dcfr", threads=1).n_nodes for s in specs]  # the oracle's own trees
    config = (batch_config(args, specs, [{"nodes": n} for n in nodes]) if batch
              else workload_config(args, specs[0], nodes[0]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "kind": "oracle",
                             "sample": f"{total_iters} DCFR iterations of {what} over {args.steps} steps "
                                       f"of {budget:.1f} s, each followed by one exploitability pass"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm

def time_to_target(capi, tree, n_games, max_iters, every, target_mbb):
    """Iterations each subgame needs until its exploitability is at most target_mbb
    (checked every `every` iterations; None if not reached within max_iters)."""
    capi.cfr_reset(tree)
    need = [None] * n_games
    done = 0
    while done < max_iters and any(x is None for x in need):
        capi.cfr_iterate(tree, every)
        done += every
        expl, _ = capi.cfr_exploitability(tree, n_games)
        for g in range(n_games):
            if need[g] is None and 1000.0 * float(expl[g]) / BB_CHIPS <= target_mbb:
                need[g] = done
    return need


def pinned_copy(torch, spec):
    out = {}
    for name in ("hands", "ranges", "strength", "board"):
        a = getattr(spec, name)
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        out[name] = t
    return type(spec)(**{**spec.__dict__, **{k: v.numpy() for k, v in out.items()}}), out


def run_ours(args):
    import numpy as np
    import torch

    from paper_2605_19928_gb300 import capi

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device: the CUDA path has no CPU fallback"}))
        return 2
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    dist = dist_init(world, True)
    capi.load()
    capi.use_torch_allocator()
    stream = torch.cuda.current_stream(device)
    batch = args.workload == "batch"
    specs = workload_specs(args, rank)
    G = len(specs)
    opts = capi.make_opts("dcfr", 1.5, 0.0, 2.0, alternating=True, chunk_hands=args.chunk_hands,
                          precision=args.precision, schedule=args.schedule, warp_hands=args.warp_hands,
                          term_nodes=args.term_nodes)
    tuned = None
    if (not args.no_autotune and args.schedule == "auto" and args.chunk_hands == 0 and args.warp_hands == 0
            and args.term_nodes == 0):
        # launch tiling (schedule, hands per block, terminal nodes per block), outside the timed region
        opts, ms_tuned = capi.cfr_autotune(specs, opts, iters=20, stream=stream.cuda_stream)
        tuned = {"schedule": SCHEDULE_NAMES[opts.schedule], "chunk_hands": opts.chunk_hands, "term_nodes": opts.term_nodes,
                 "warp_hands": opts.warp_hands,
                 "ms_per_iter_while_tuning": ms_tuned}

    def create(sp):
        if batch:
            return capi.cfr_batch_create(sp, opts, stream=stream.cuda_stream)
        return capi.cfr_tree_create(sp[0], opts, stream=stream.cuda_stream)

    tree = create(specs)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    ips = args.iters_per_step

    def step():
        capi.cfr_reset(tree)
        capi.cfr_iterate(tree, ips)
        capi.cfr_exploitability_async(tree)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize(device)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = capi.cfr_counters(tree)["kernel_launches"]
    clocks = ClockSampler(device.index)
    barrier(dist, device)
    torch.cuda.synchronize(device)
    clocks.start()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize(device)
    clock_info = clocks.stop()
    barrier(dist, device)
    gpu_launches = capi.cfr_counters(tree)["kernel_launches"] - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    local_s = sum(step_ms) / 1000.0
    value, t_max = aggregate(args.steps * ips * G, local_s, world, dist, device)
    expl, br = capi.cfr_exploitability_result(tree, G)
    ms_per_iter = 1000.0 * t_max / (args.steps * ips)

    # per-kernel device time (un-graphed, CUDA events between launches) for the roofline
    shapes = [tree_shape(capi, tree, g) for g in range(G)]
    capi.cfr_reset(tree)
    stages = capi.cfr_stage_times(tree, min(ips, 200 if not batch else 20))
    vbytes = 8 if args.precision == "pairs" else 4  # bytes of one stored value
    per_step = {k: stages[k][0] * (2 * ips if k in ("terminal", "update") else 1) for k in stages}
    dom = max(("update", "terminal"), key=lambda k: per_step[k])
    peak, peak_kind = peaks()
    schedule = SCHEDULE_NAMES[capi.cfr_schedule(tree)]
    if schedule == "resident":
        # one launch runs whole iterations: per iteration both players' terminal and update
        # launches' algorithmic bytes, over the launch's own device time (20 iterations, the
        # launch the committed ncu summary captures)
        n_res = min(ips, 20)
        capi.cfr_reset(tree)
        torch.cuda.synchronize(device)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        capi.cfr_iterate(tree, n_res)
        r1.record(stream)
        torch.cuda.synchronize(device)
        launch_ms = r0.elapsed_time(r1)
        per_iter = lambda v: sum(2 * (algorithmic_bytes(sh, "update", v) + algorithmic_bytes(sh, "terminal", v))
                                 for sh in shapes)
        alg = n_res * per_iter(4)
        roofline = {"bound": "hbm", "kernel": "k_resident", "achieved": alg / (launch_ms * 1e-3) / 1e9,
                    "peak": peak, "unit": "GB/s", "frac": alg / (launch_ms * 1e-3) / 1e9 / peak,
                    "peak_source": f"{peak_kind} hbm_gbs", "traffic": profiled_traffic("resident", "river1081"),
                    "algorithmic_bytes_per_launch": alg, "value_bytes_in_model": 4, "launch_ms": launch_ms,
                    "iterations_per_launch": n_res,
                    "stage_ms_level_kernels": {k: v[0] for k, v in stages.items()}}
        if vbytes != 4:
            roofline["algorithmic_bytes_per_launch_pair_storage"] = n_res * per_iter(vbytes)
    else:
        # the roofline model counts 4-byte values whatever the storage precision
        alg = sum(algorithmic_bytes(sh, dom, 4) for sh in shapes)
        achieved = alg / (stages[dom][0] * 1e-3) / 1e9
        upd_kernel = "k_stream_update" if schedule == "stream" else "k_hand<update>"
        roofline = {"bound": "hbm", "kernel": upd_kernel if dom == "update" else "k_terminal",
                    "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": f"{peak_kind} hbm_gbs",
                    "traffic": profiled_traffic(dom, "batch256" if batch else "river1081"),
                    "algorithmic_bytes_per_launch": alg, "value_bytes_in_model": 4, "launch_ms": stages[dom][0],
                    "stage_ms": {k: v[0] for k, v in stages.items()}}
        if vbytes != 4:  # the same model with the stored pair values, for comparison only
            roofline["algorithmic_bytes_per_launch_pair_storage"] = sum(algorithmic_bytes(sh, dom, vbytes)
                                                                        for sh in shapes)

    target = None
    if not batch:  # the single subgame: iterations (and device time) to 1 mbb/hand
        need = time_to_target(capi, tree, 1, max_iters=ips, every=10, target_mbb=1.0)[0]
        target = {"target_mbb_per_hand": 1.0, "checked_every_iters": 10, "iters": need,
                  "ms": None if need is None else need * ms_per_iter}
    if batch:
        limit = 4 * ips
        need = time_to_target(capi, tree, G, max_iters=limit, every=10, target_mbb=1.0)
        ranked = sorted(x if x is not None else float("inf") for x in need)
        pct = (lambda q: ranked[min(G - 1, int(q * G))])
        fmt = (lambda x: None if x == float("inf") else x)
        target = {"target_mbb_per_hand": 1.0, "reached": sum(x is not None for x in need), "of": G,
                  "checked_every_iters": 10, "limit_iters": limit,
                  "iters_p50": fmt(pct(0.50)), "iters_p99": fmt(pct(0.99)),
                  "ms_p50": None if fmt(pct(0.50)) is None else pct(0.50) * ms_per_iter,
                  "ms_p99": None if fmt(pct(0.99)) is None else pct(0.99) * ms_per_iter,
                  "note": "iterations of the whole batch (all subgames advance together) times the "
                          "measured ms per batch iteration; null = not reached within limit_iters"}

    # end to end through the C ABI with host buffers: inputs from pinned host memory,
    # create + solve + exploitability + read of each root's average strategy, every step
    e2e = None
    if args.e2e_steps > 0:
        pspecs = [pinned_copy(torch, sp)[0] for sp in specs]
        roots = []
        times, h2d, d2h = [], 0, 0
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            tr = create(pspecs)
            capi.cfr_iterate(tr, ips)
            ex, _ = capi.cfr_exploitability(tr, G)
            nbytes = 16 * G
            for g in range(G):
                a = capi.cfr_node_info(tr, 0, g)["n_actions"]
                roots.append(capi.cfr_strategy(tr, 0, average=True, game=g))
                nbytes += a * specs[g].n_hands * vbytes
            t1 = time.perf_counter()
            if k > 0:
                times.append(t1 - t0)
                h2d = capi.cfr_counters(tr)["h2d_bytes"]
                d2h = nbytes
            capi.cfr_tree_destroy(tr)
            roots.clear()
        e2e_val, _ = aggregate(ips * G * len(times), sum(times), world, dist, device)
        e2e = {"value": e2e_val, "unit": "subgame iter/s" if batch else "iter/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "step": f"create from pinned host inputs + {ips} iterations + exploitability + root average "
                       "strateg" + ("ies of every subgame" if batch else "y") + " to host"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(specs, args.cpu_seconds, batch)
    capi.cfr_tree_destroy(tree)
    if rank == 0:
        if batch:
            config = {**batch_config(args, specs, shapes), "schedule": schedule}
            if tuned is not None:
                config["autotune"] = tuned
            e_mbb = sorted(1000.0 * float(x) / BB_CHIPS for x in expl)
            quality = {"exploitability_mbb_median": e_mbb[G // 2], "exploitability_mbb_max": e_mbb[-1],
                       "time_to_1mbb": target}
        else:
            config = {**workload_config(args, specs[0], shapes[0]["nodes"]), "schedule": schedule}
            if tuned is not None:
                config["autotune"] = tuned
            quality = {"exploitability_mbb": 1000.0 * float(expl[0]) / BB_CHIPS, "time_to_1mbb": target,
                       "exploitability_pct_pot": 100.0 * float(expl[0]) / specs[0].pot}
        line = {"metric": METRIC, "value": value, "unit": "subgame iter/s" if batch else "iter/s",
                "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps,
                "ms_per_step_std": float(np.std(step_ms)), "ms_per_iter": ms_per_iter,
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32x2 values, f64 R/S" if args.precision == "pairs" else
                "f32 values, f64 R/S", "data": "synthetic", "config": config, **quality,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(gpu_launches),
                "clocks": clock_info}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def cpu_baseline(specs, seconds, batch):
    """The oracle as it stands on the host cores, on a bounded sample of the workload."""
    if not batch:
        r = oracle_sample(specs[0], seconds)
        one = oracle_sample(specs[0], seconds / 3, threads=1)  # the same oracle on one core
        return {"value": r["iters"] / r["seconds"], "unit": "iter/s", "cores": r["threads"], "kind": "oracle",
                "sample": f"{r['iters']} DCFR iterations of the same 1081-hand river subgame plus one "
                          f"exploitability pass ({r['seconds']:.1f} s, FP64, walks every history)",
                "single_thread": {"value": one["iters"] / one["seconds"], "unit": "iter/s", "cores": 1,
                                  "sample": f"{one['iters']} iterations plus one exploitability pass "
                                            f"({one['seconds']:.1f} s)"}}
    picks = sorted(set(int(k * len(specs) / 4) for k in range(4)))
    sec_per_iter, iters, total, threads = [], 0, 0.0, 1
    for g in picks:
        r = oracle_sample(specs[g], seconds / len(picks))
        sec_per_iter.append(r["seconds"] / r["iters"])
        iters += r["iters"]
        total += r["seconds"]
        threads = r["threads"]
    value = 1.0 / (sum(sec_per_iter) / len(sec_per_iter))
    return {"value": value, "unit": "subgame iter/s", "cores": threads, "kind": "oracle",
            "sample": f"{iters} DCFR iterations (+ one exploitability pass each) of subgames {picks} of the "
                      f"batch ({total:.1f} s); value = 1 / mean seconds per subgame iteration"}


def node_paths(capi, tree, game: int = 0) -> dict:
    """Action path from the root (tuple of child indices) -> node id."""
    n_nodes = capi.cfr_tree_info(tree, game)[0]
    paths = {0: ()}
    for n in range(1, n_nodes):
        info = capi.cfr_node_info(tree, n, game)
        paths[n] = paths[info["parent"]] + (info["action"],)
    return {p: n for n, p in paths.items()}


def gemm_throughput(capi, torch, device, M=16384, reps=20):
    """TFLOP/s of the leaf network's layers on the tensor cores (inputs in HBM), each as the
    network runs it: the hidden layers with GELU and BF16 output, the output layer linear
    with FP32 output."""
    out = {}
    for name, (N, K, act, dtype) in (("layer1", (512, 2752, True, torch.bfloat16)),
                                     ("layer2", (512, 512, True, torch.bfloat16)),
                                     ("layer4", (2688, 512, False, torch.float32))):
        A = torch.randn(M, K, device=device).to(torch.bfloat16)
        B = (torch.randn(N, K, device=device) / K ** 0.5).to(torch.bfloat16)
        bias = torch.zeros(N, device=device)
        C = torch.empty(M, N, device=device, dtype=dtype)
        err = torch.zeros(1, dtype=torch.int32, device=device)
        for _ in range(3):
            capi.cfr_gemm_bf16(A, B, bias, C, act, err)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(device)
        s.record()
        for _ in range(reps):
            capi.cfr_gemm_bf16(A, B, bias, C, act, err)
        e.record()
        torch.cuda.synchronize(device)
        ms = s.elapsed_time(e) / reps
        out[name] = {"M": M, "N": N, "K": K, "gelu": act, "out": str(dtype).replace("torch.", ""), "ms": ms,
                     "tflops": 2.0 * M * N * K / (ms * 1e-3) / 1e12,
                     "out_gbs": M * N * C.element_size() / (ms * 1e-3) / 1e9, "wait_errors": int(err.item())}
    return out


def run_gemm(args):
    """Only the leaf network's dense layers on the tensor cores (for profiling)."""
    import torch

    from paper_2605_19928_gb300 import capi
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    capi.load()
    g = gemm_throughput(capi, torch, device, reps=max(1, args.steps))
    peak, kind = bf16_peak()
    print(json.dumps({"workload": "leaf network layers, M = 16384 rows", "layers": g, "peak_tflops": peak,
                      "peak_source": kind}))
    return 0


def run_leaf(args):
    """Depth-limited subgame with the learned leaf network vs the exact subgame: the turn
    (workload leaf) or the flop (workload flop, turn card dealt by chance inside the tree)."""
    import numpy as np
    import torch

    from paper_2605_19928_gb300 import capi, leafnet_train, serve, synth

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device: the CUDA path has no CPU fallback"}))
        return 2
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    dist = dist_init(world, True)
    capi.load()
    capi.use_torch_allocator()
    stream = torch.cuda.current_stream(device)
    kw = dict(seed=0 + 1000 * rank, range_seed=1 + 1000 * rank)
    flop = args.workload == "flop"
    make = synth.ranked_flop_subgame if flop else synth.ranked_turn_subgame
    spec_leaf = make(depth_limit=1, **kw)
    spec_exact = make(depth_limit=0, **kw)
    tables = flop and args.runout_tables == "on" and args.precision == "single"  # (FP32 values only)
    opts = capi.make_opts("dcfr", 1.5, 0.0, 2.0, alternating=True, precision=args.precision,
                          schedule="wide" if tables else "auto", runout_tables=tables)
    W, b = leafnet_train.load_weights()
    meta = np.load(os.path.join(ROOT, "paper_2605_19928_gb300", "leafnet_weights.npz"))["meta"]
    L = capi.cfr_tree_create(spec_leaf, opts, stream=stream.cuda_stream)
    E = capi.cfr_tree_create(spec_exact, opts, stream=stream.cuda_stream)
    capi.cfr_set_leaf_net(L, W, b)
    ips = args.iters_per_step
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def timed(tree, steps, warmup):
        for _ in range(warmup):
            flush.zero_()
            capi.cfr_reset(tree)
            capi.cfr_iterate(tree, ips)
            capi.cfr_exploitability_async(tree)
        torch.cuda.synchronize(device)
        st = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            st[k].record(stream)
            capi.cfr_reset(tree)
            capi.cfr_iterate(tree, ips)
            capi.cfr_exploitability_async(tree)
            en[k].record(stream)
        torch.cuda.synchronize(device)
        return sum(a.elapsed_time(c) for a, c in zip(st, en)) / 1000.0

    launches0 = capi.cfr_counters(L)["kernel_launches"]
    clocks = ClockSampler(device.index)
    barrier(dist, device)
    clocks.start()
    t_leaf = timed(L, args.steps, args.warmup)
    clock_info = clocks.stop()
    gpu_launches = capi.cfr_counters(L)["kernel_launches"] - launches0
    value, t_max = aggregate(args.steps * ips, t_leaf, world, dist, device)
    e_leaf_own, _ = capi.cfr_exploitability_result(L)
    # the served form: the network judged on its own leaf rows (per leaf: 4 rows of each turn
    # leaf, 1 of each flop leaf) against exact river solves of their continuations; the
    # leaves above the tolerance are solved exactly beside the network leaves of the rest
    per_leaf = 1 if flop else 4
    judge = serve.judge_leaves(L, spec_leaf, n_rows=64, iters=300, seed=rank, stream=stream.cuda_stream,
                               evaluated=True, per_leaf=per_leaf)
    n_leaves_total = len(capi.cfr_leaf_info(L))
    exact_leaves = serve.fallback_leaves(judge.leaf_errors, serve.DEFAULT_TOL)
    exact_steps = 1 if flop else max(1, args.steps // 4)
    t_exact = timed(E, exact_steps, 1)
    e_exact, _ = capi.cfr_exploitability_result(E)
    exact_ips = exact_steps * ips / t_exact
    # the learned turn strategy in the exact game: E's river play, L's turn play
    pe, pl = node_paths(capi, E), node_paths(capi, L)
    for path, nl in pl.items():
        if capi.cfr_node_info(L, nl)["type"] == capi.CFR_NODE_DECISION:
            capi.cfr_write_values(E, capi.CFR_READ_AVG_SUM, pe[path], capi.cfr_read_values(L, capi.CFR_READ_AVG_SUM, nl))
    e_hybrid, _ = capi.cfr_exploitability(E)
    # the network against exact river solving at every leaf: give the depth-limited handle
    # the exact handle's turn strategy, evaluate the network there, and compare with the
    # values the exact handle's next player-0 traversal finds at the same river-card nodes
    snap = {}
    for path, nl in pl.items():
        if capi.cfr_node_info(L, nl)["type"] == capi.CFR_NODE_DECISION:
            snap[path] = capi.cfr_read_values(E, capi.CFR_READ_REGRET, pe[path])
    for path, nl in pl.items():
        if path in snap:
            capi.cfr_write_values(L, capi.CFR_READ_REGRET, nl, snap[path])
    capi.cfr_eval_leaves(L)
    capi.cfr_iterate(E, 1)
    rel, abs_err = [], 0.0
    lp = {n: p for p, n in pl.items()}
    for _, nl, _ in capi.cfr_leaf_info(L):
        path = lp[nl]
        v_net = capi.cfr_read_values(L, capi.CFR_READ_CFV, nl, player=0)
        v_ex = capi.cfr_read_values(E, capi.CFR_READ_CFV, pe[path], player=0)
        rel.append(float(np.abs(v_net - v_ex).sum() / max(np.abs(v_ex).sum(), 1e-30)))
        abs_err += float(np.abs(v_net - v_ex).sum())
    leaf_check = {"relative_l1_mean": float(np.mean(rel)), "relative_l1_max": float(np.max(rel)),
                  "leaves": len(rel),
                  "note": "player 0's leaf values from the network vs from the exact river subtrees, same turn "
                          "strategy (the exact solve's current one); sum over hands of |difference| / sum |exact|"}
    # per-stage times of the learned form (launch by launch)
    capi.cfr_reset(L)
    stages = capi.cfr_stage_times(L, min(ips, 100))
    leaves = capi.cfr_leaf_info(L)
    rows = len(leaves) * capi.LEAF_CARDS
    flops = 2.0 * rows * (capi.LEAF_IN * capi.LEAF_HIDDEN + 2 * capi.LEAF_HIDDEN ** 2 + capi.LEAF_HIDDEN * capi.LEAF_OUT)
    gemm = gemm_throughput(capi, torch, device)
    peak, peak_kind = bf16_peak()
    best = max(gemm.values(), key=lambda g: g["tflops"])
    roofline = {"bound": "tensor", "kernel": "k_gemm_bf16 (leaf network layers, M = 16384 rows)",
                "achieved": best["tflops"], "peak": peak, "unit": "TFLOP/s", "frac": best["tflops"] / peak,
                "peak_source": peak_kind, "traffic": None, "layers": gemm,
                "leaf_stage": {"rows_per_evaluation": rows, "flops_per_evaluation": flops,
                               "ms": stages["leaf"][0],
                               "tflops_incl_input_and_value_kernels": flops / (stages["leaf"][0] * 1e-3) / 1e12},
                "stage_ms": {k: v[0] for k, v in stages.items()}}
    mbb = lambda e: 1000.0 * float(e) / BB_CHIPS
    ms_leaf_step, ms_exact_step = 1000.0 * t_leaf / args.steps, 1000.0 * t_exact / exact_steps
    if not exact_leaves:
        form, e_served, ms_fallback = "learned", e_hybrid[0], 0.0
    elif len(exact_leaves) == n_leaves_total:
        form, e_served, ms_fallback = "exact (every leaf failed)", e_exact[0], ms_exact_step
    else:  # one handle: exact river subtrees at the failed leaves, the network at the rest
        Mx = capi.cfr_tree_create(dataclasses.replace(spec_leaf, exact_leaves=tuple(exact_leaves)), opts,
                                  stream=stream.cuda_stream)
        try:
            capi.cfr_set_leaf_net(Mx, W, b)
            ms_fallback = 1000.0 * timed(Mx, 1, 1)
            pm = node_paths(capi, Mx)
            for path, nm in pm.items():  # its strategy in the exact game, E's river play elsewhere
                if capi.cfr_node_info(Mx, nm)["type"] == capi.CFR_NODE_DECISION:
                    capi.cfr_write_values(E, capi.CFR_READ_AVG_SUM, pe[path],
                                          capi.cfr_read_values(Mx, capi.CFR_READ_AVG_SUM, nm))
            e_served = capi.cfr_exploitability(E)[0][0]
        finally:
            capi.cfr_tree_destroy(Mx)
        form = "mixed"
    served = {"form": form, "tol_pot": serve.DEFAULT_TOL,
              "leaves": n_leaves_total, "exact_leaves": len(exact_leaves), "judged_rows_per_leaf": per_leaf,
              "judge": {"rows": judge.rows, "candidates": judge.candidates,
                        "mean_abs_error_pot": judge.mean_abs_error,
                        "reach_weighted_error_pot": judge.reach_weighted_error,
                        "max_row_error_pot": judge.max_row_error,
                        "continuation_exploitability_mbb": judge.continuation_exploitability_mbb,
                        "ms": judge.ms, "continuation_iters": 300},
              "exploitability_in_exact_game_mbb": mbb(e_served),
              "ms_per_solve": ms_leaf_step + judge.ms + ms_fallback,
              "note": "one solve = the depth-limited solve (one step), the judge (host wall time, "
                      "continuation solves included) and, where leaves failed, the solve with those "
                      "leaves exact (one step; the whole exact subgame when all failed)"}
    n_exact = capi.cfr_tree_info(E)[0]
    n_leaf_nodes = capi.cfr_tree_info(L)[0]
    sched = {capi.CFR_SCHEDULE_LEVEL: "level", capi.CFR_SCHEDULE_STREAM: "stream",
             capi.CFR_SCHEDULE_WIDE: "wide"}
    schedules = {"learned": sched[capi.cfr_schedule(L)], "exact": sched[capi.cfr_schedule(E)]}
    capi.cfr_tree_destroy(L)
    capi.cfr_tree_destroy(E)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps,
                "ms_per_iter": 1000.0 * t_max / (args.steps * ips), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": ("f32x2" if args.precision == "pairs" else "f32") + " values, f64 R/S, bf16 network",
                "data": "synthetic (rank-based showdowns; network trained on %dk self-generated river solves%s)"
                        % (int(meta[0]) // 1000, " and the river-card nodes of %d exact turn solves" % int(meta[6])
                           if len(meta) > 6 and meta[6] > 0 else ""),
                "config": {"workload": ("depth-limited flop subgame (turn card by chance), leaf network at the "
                                        "river card" if flop else
                                        "depth-limited turn subgame, leaf network at the river card"),
                           "board_cards": len(spec_leaf.board), "hands": spec_leaf.n_hands, "leaves": len(leaves),
                           "nodes": n_leaf_nodes, "schedules": schedules, "runout_tables": tables,
                           "network": "2752-512-512-512-2688 BF16, GELU", "pot": spec_leaf.pot,
                           "stack": spec_leaf.stack,
                           "bet_sizes": ",".join("all-in" if x <= 0 else "%g" % x for x in spec_leaf.bet_sizes)
                                        + " (pot fractions)",
                           "max_raises": spec_leaf.max_raises,
                           "variant": "DCFR(1.5,0,2) alternating", "iters_per_step": ips,
                           "step": "reset + iterations + exploitability (network leaves)",
                           "l2": "flushed between steps (256 MB write, outside the timed events)",
                           "seeds": spec_leaf.seeds},
                "exact_form": {"iter_per_s": exact_ips, "ms_per_iter": 1000.0 / exact_ips, "nodes": n_exact,
                               "exploitability_mbb": mbb(e_exact[0])},
                "learned_form": {"exploitability_in_exact_game_mbb": mbb(e_hybrid[0]),
                                 "exploitability_with_network_leaves_mbb": mbb(e_leaf_own[0]),
                                 "note_network_leaves": "best responses with the network's values at the "
                                                        "leaves; the two players' outputs are not zero-sum, "
                                                        "so this can fall below 0",
                                 "gap_to_exact_mbb": mbb(e_hybrid[0]) - mbb(e_exact[0]),
                                 "note": "strategy of the depth-limited solve above the leaves, river play of "
                                         "the exact solve, best responses in the exact game"},
                "leaf_values_vs_exact_river": leaf_check,
                "served": served,
                "network": {"training_solves": int(meta[0]), "solve_iters": int(meta[1]), "epochs": int(meta[2]),
                            "median_solve_exploitability_mbb": float(meta[4]),
                            "validation_mean_abs_error_pot": float(meta[5]),
                            "turn_solves": int(meta[6]) if len(meta) > 6 else 0,
                            "turn_leaf_examples": int(meta[7]) if len(meta) > 7 else 0},
                "speedup_vs_exact": value / exact_ips,
                "roofline": roofline, "cpu_baseline": None, "e2e": None, "gpu_launches": int(gpu_launches),
                "clocks": clock_info}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.iters_per_step is None:
        args.iters_per_step = {"batch": 500, "leaf": 300, "flop": 300}.get(args.workload, 1000)
    if args.precision is None:
        args.precision = "single"
    if args.workload in ("leaf", "flop") and args.impl == "ours":
        return run_leaf(args)
    if args.workload == "gemm" and args.impl == "ours":
        return run_gemm(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
