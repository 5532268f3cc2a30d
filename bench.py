#!/usr/bin/env python3
"""Benchmark of the GB300 interaction-net evaluator.

One step = one whole reduction to normal form (the int/com loop of Sec. 3.6)
of one batch of synthetic nets.  Default workload: 2048 independent nets
Mul(S^m Z, S^n Z), m, n ~ U{0..64} (seed 14040076 + 1), reduced by the
batched persistent kernel; 47 391 647 interactions per step.

  python bench.py [--gpus N --steps K --warmup W] [--workload W] [--mode M]
  python bench.py --impl reference ...   # the CPU oracle on the host cores

Prints one JSON line (rank 0).  `value` = interactions per second of device
time, inputs resident in HBM (nets loaded and staged before the timed
region, L2 flushed between steps); `e2e` = the same through the public API
from host text to host results, copies included.
"""
from __future__ import annotations

import argparse
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

import workloads as W  # noqa: E402
from paper_1404_0076_gb300.shard import combine, rank_seed  # noqa: E402

METRIC = "interactions/sec and HBM-roofline fraction (batched vs plain); p50/p99 latency"
UNIT = "interactions/s"


def workload(name: str, rank: int = 0):
    """(nets, description, capacities) of a named workload.  Under N ranks
    each rank reduces its own batch (seed offset by rank): weak scaling."""
    if name == "mul2048":
        w = W.config1(seed=rank_seed(W.SEED_BASE + 1, rank))
        desc = "2048 nets Mul(S^m Z, S^n Z), m,n ~ U{0..64}, seed 14040076+1"
        caps = dict(max_agents=1 << 24, max_vars=1 << 24, max_pairs=1 << 20, max_nets=4096)
    elif name == "add4096":
        w = W.config0(seed=rank_seed(W.SEED_BASE + 0, rank))
        desc = "4096 nets Add(S^m Z, S^n Z), m,n ~ U{0..256}, seed 14040076"
        caps = dict(max_agents=1 << 22, max_vars=1 << 22, max_pairs=1 << 20, max_nets=8192)
    elif name == "ack3":
        w = W.config2()
        desc = "5 nets A(S^3 Z, S^b Z), b = 4..8"
        caps = dict(max_agents=1 << 22, max_vars=1 << 22, max_pairs=1 << 20, max_nets=64)
    elif name == "fib":
        w = W.config3()
        desc = "6 nets Fib(S^n Z), n = 20..25"
        caps = dict(max_agents=1 << 23, max_vars=1 << 23, max_pairs=1 << 20, max_nets=64)
    elif name == "lsys27":
        w = W.config5()
        desc = "one net SymA(r) = S^27 Z: the L-System A -> AB, B -> A after 27 steps (514229 symbols)"
        caps = dict(max_agents=1 << 22, max_vars=1 << 22, max_pairs=1 << 21, max_nets=16)
    elif name == "chain20k":
        w = W.Workload("chain20k", W.ARITH_RULES, [W.add_net(20000, 0)], [(20000, 0)])
        desc = "one net Add(Z, r) = S^20000 Z: a chain of 20001 dependent interactions"
        caps = dict(max_agents=1 << 20, max_vars=1 << 20, max_pairs=1 << 16, max_nets=16)
    elif name == "fib25x64":
        w = W.replicated(W.config3(ns=(25,)), 64)
        desc = "64 copies of Fib(S^25 Z)"
        caps = dict(max_agents=1 << 25, max_vars=1 << 25, max_pairs=1 << 23, max_nets=128)
    else:
        raise SystemExit(f"unknown workload {name}")
    return w.nets, desc, caps, w.rules


# --- algorithmic bytes per interaction ---------------------------------------------
# B_r = 8 (pair) + 8 (two labels) + 4 (ar_alpha + ar_beta) (auxiliary words read)
#     + sum over new agents 4 (1 + ar) (records written) + 4 fresh names
#     + 8 per equation linked (exchange or pair push) + 4 |new agents - 2|
#     + 8 when batched (net id with the pair read and with the pair pushed).
def bytes_per_rule(rules: list[dict], batched: bool) -> list[int]:
    out = []
    for r in rules:
        b = 8 + 8 + 4 * (r["arity_alpha"] + r["arity_beta"]) + 4 * (r["n_new"] + r["new_ports"])
        b += 4 * r["n_fresh"] + 8 * r["n_link"] + 4 * abs(r["n_new"] - 2)
        if batched:
            b += 8
        out.append(b)
    return out


# DRAM bytes per launch from ncu captures (profiles/), valid only for the
# kernel sources they were taken on (sha1 prefix over csrc/inet_kernels.cuh
# and csrc/inet_async.cuh) and for the kernel they were taken of (the last
# key: the asynchronous kernel compiled for the rule set, or the general one).
NCU_TRAFFIC = {("mul2048", "async", "21bd99a5a4f1", True): 6_204_672 + 11_322_624}


def kernel_source_hash() -> str:
    """sha1 prefix of the kernel sources' code (comments and blank lines
    left out, so a comment edit keeps the key of measured traffic)."""
    import hashlib
    import re
    h = hashlib.sha1()
    for name in ("inet_kernels.cuh", "inet_async.cuh"):
        with open(os.path.join(ROOT, "paper_1404_0076_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()[:12]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --- clocks during the timed region ---------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --- the CPU oracle (cpu_baseline and the reference arm) -----------------------------
def oracle_binary() -> str:
    exe = os.path.join(ROOT, "oracle", "inet_oracle")
    src = os.path.join(ROOT, "oracle", "inet_oracle.cpp")
    if not os.path.exists(exe) or os.path.getmtime(exe) < os.path.getmtime(src):
        subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", src, "-o", exe], check=True)
    return exe


def run_oracle(nets, threads: int, rules: str = W.ARITH_RULES):
    """Times the oracle on the host; returns (interactions, seconds)."""
    import tempfile
    exe = oracle_binary()
    with tempfile.TemporaryDirectory() as d:
        rp, np_ = os.path.join(d, "r.txt"), os.path.join(d, "n.txt")
        with open(rp, "w") as f:
            f.write(rules)
        with open(np_, "w") as f:
            f.write("\n".join(nets) + "\n")
        p = subprocess.run([exe, rp, np_, "--quiet", "--threads", str(threads)], capture_output=True, text=True)
    tail = json.loads(p.stderr.strip().splitlines()[-1])
    return tail["interactions"], tail["seconds"]


def reference_arm(args, rank, world):
    if rank != 0:
        return
    nets, desc, _, rules = workload(args.workload)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        run_oracle(nets, cores, rules)
    tot_i, tot_s = 0, 0.0
    for _ in range(args.steps):
        i, s = run_oracle(nets, cores, rules)
        tot_i += i
        tot_s += s
    value = tot_i / tot_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": desc, "nets": len(nets)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"whole workload per step ({len(nets)} nets), {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --- serving ----------------------------------------------------------------------
def expected_value(r) -> int:
    """The numeral a serving request reduces to (closed forms)."""
    if r.family == "add":
        return r.params[0] + r.params[1]
    if r.family == "mul":
        return r.params[0] * r.params[1]
    if r.family == "ack":
        return W._ack(*r.params)
    return W._fib_values(r.params[0] + 1)[r.params[0]]


def serving_leg(args, local: int) -> dict:
    """Continuous batching on the serving mix: the 100k-request Poisson
    stream (--serve-requests takes its first requests only).  First every
    request arrives at once (saturated): the serving capacity C is the rate
    of interactions the device performs while admission still has a
    backlog (the queue of arrived requests never empties in that window),
    not the wall time of the whole run, which the longest request's chain of
    dependent interactions sets.  Then the stream is replayed on the wall
    clock at load rho of C (arrival rate rho * C / mean request size) for
    each rho of --serve-rhos.  Every result is checked against its closed
    form (value and exact interaction count)."""
    import dataclasses

    from paper_1404_0076_gb300.serve import Server, summarize
    reqs = W.config4()[: args.serve_requests]
    expect = [expected_value(r) for r in reqs]
    mean_size = sum(r.size for r in reqs) / len(reqs)
    budget = args.serve_budget_gb << 30
    srv = Server(W.ARITH_RULES, device=local, budget_bytes=budget, epoch_us=args.serve_epoch_us, max_pairs=1 << 23)
    out = {"workload": "serving mix: Poisson arrivals, one net each from add/mul/ack/fib, sizes lognormal "
                       "(median 1e3 interactions, sigma 2.16, clipped to 1e7), seed 14040076+4",
           "requests": len(reqs), "mean_request_interactions": mean_size, "budget_bytes": budget, "arenas": 1,
           "largest_request_interactions": max(r.size for r in reqs),
           "epoch_us": args.serve_epoch_us,
           "sample": "the whole 100000-request stream" if len(reqs) == 100000
           else f"first {len(reqs)} of the 100000-request stream"}

    def run(scale: float, sample=None) -> dict:
        rr = reqs if sample is None else reqs[:sample]
        e0, s0, n0, p0 = srv.epochs, srv.frees, srv.freed, srv.performed
        h0 = dict(srv.host_s)
        win = {}

        def queue_empty(t, done_so_far):
            win["t"] = t
            win["performed"] = srv.performed - p0
            win["completed"] = len(done_so_far)

        t0 = time.perf_counter()
        done = srv.serve(rr, time_scale=scale, on_queue_empty=queue_empty)
        wall = time.perf_counter() - t0
        rec = summarize(done, wall)
        rec.update(wall_s=wall, epochs=srv.epochs - e0, free_calls=srv.frees - s0, nets_freed=srv.freed - n0,
                   device_interactions=srv.performed - p0,
                   host_s={k: round(v - h0.get(k, 0.0), 3) for k, v in srv.host_s.items()},
                   largest_served=max((rr[d.rid].size for d in done if d.status == "OK"), default=0),
                   wrong=sum(1 for d in done if d.status != "OK"
                             or (d.value, d.interactions) != (expect[d.rid], rr[d.rid].size)))
        if win:
            rec["backlog_window_s"] = win["t"]
            rec["backlog_interactions"] = win["performed"]
            rec["backlog_completed"] = win["completed"]
        return rec

    try:
        srv.serve([dataclasses.replace(r, arrival_s=0.0) for r in reqs[:256]])  # warm-up
        sat = run(0.0)
        out["saturated"] = sat
        # capacity: interactions performed per second while arrived requests
        # were still waiting for admission (at least 0.5 s of backlog); else
        # the whole run
        if sat.get("backlog_window_s", 0) >= 0.5:
            cap = sat["backlog_interactions"] / sat["backlog_window_s"]
            out["capacity_how"] = "device interactions per second while the admission queue was non-empty " \
                                  f"({sat['backlog_window_s']:.2f} s backlog of the saturated run)"
        else:
            cap = sat["device_interactions"] / sat["wall_s"]
            out["capacity_how"] = "device interactions per second over the whole saturated run (no backlog)"
        out["capacity_interactions_per_s"] = cap
        rate0 = len(reqs) / reqs[-1].arrival_s          # the stream's own rate
        for rho in args.serve_rhos:
            lam = rho * cap / mean_size                   # requests per second
            rec = run(rate0 / lam, args.serve_rho_sample)
            rec["rho"], rec["requests_per_s"] = rho, lam
            out[f"rho_{rho}"] = rec
    finally:
        srv.close()
    return out


def narrow_leg(args, local: int, name: str) -> dict:
    """A narrow-frontier workload (the paper's Fig. 2 regime): timed like
    the headline, over --narrow-steps steps, in the form and launch shape
    the autotuner picks, with its critical-path depth (steps of the
    maximally parallel loop) and time per level."""
    import torch

    from paper_1404_0076_gb300 import Evaluator
    from paper_1404_0076_gb300.autotune import Autotuner
    nets, desc, caps, rules_text = workload(name)
    ev = Evaluator(device=local, **caps)
    ev.load_rules(rules_text)
    props = torch.cuda.get_device_properties(local)
    tuned = Autotuner().tune(ev, rules_text, nets, "auto", gpu=props.name, num_sms=props.multi_processor_count)
    opts = dict(mode="async", block=0, grid=0, solo_max=0)
    opts.update(tuned)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")

    def prepared():
        ev.reset()
        ev.stage(ev.load_nets(nets))
        flush.fill_(1)
        torch.cuda.synchronize()

    for _ in range(3):
        prepared()
        ev.reduce([], **opts)
    ms, ints = [], 0
    for _ in range(args.narrow_steps):
        prepared()
        st = ev.reduce([], **opts)
        ms.append(st["device_ms"])
        ints += st["interactions"]
    prepared()
    depth = ev.reduce([], mode="persistent")["steps"]
    ev.close()
    step_ms = sum(ms) / len(ms)
    return {"workload": desc, "interactions_per_step": ints // args.narrow_steps,
            "interactions_per_s": ints / (sum(ms) / 1e3), "ms_per_step": step_ms, "steps": args.narrow_steps,
            "depth_levels": depth, "ns_per_level": 1e6 * step_ms / max(1, depth),
            "mode": opts["mode"], "block": opts["block"] or 256, "grid": opts["grid"] or "auto",
            "launch_shape": "autotuned"}


# --- our arm ------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mul2048")
    ap.add_argument("--mode", default="auto", choices=["auto", "async", "persistent", "graph", "plain"],
                    help="loop form; auto: the autotuner picks async or persistent for the workload")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--grid", type=int, default=0)
    ap.add_argument("--solo-max", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--no-control", action="store_true", help="skip the sort-based linker control")
    ap.add_argument("--serve-requests", type=int, default=100000)
    ap.add_argument("--serve-rhos", type=float, nargs="*", default=[0.5, 0.8, 0.95])
    ap.add_argument("--serve-rho-sample", type=int, default=None,
                    help="requests of the stream replayed at each rho (default: all)")
    ap.add_argument("--no-narrow", action="store_true", help="skip the Ackermann and Fibonacci keys")
    ap.add_argument("--narrow-steps", type=int, default=5)
    ap.add_argument("--plain-sample", type=int, default=128,
                    help="nets of the batch (every k-th) reduced one per launch by the host-driven loop")
    ap.add_argument("--serve-epoch-us", type=int, default=250)
    ap.add_argument("--serve-budget-gb", type=int, default=64)
    ap.add_argument("--no-jit", action="store_true",
                    help="asynchronous mode on the general kernel, not the one compiled for the rule set")
    args = ap.parse_args()
    if args.no_jit:
        os.environ["INET_JIT"] = "0"  # read by every context this process creates
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    from paper_1404_0076_gb300 import Evaluator

    nets, desc, caps, rules_text = workload(args.workload, rank)
    ev = Evaluator(device=local, **caps)
    ev.load_rules(rules_text)
    rules = ev.rules()
    bpr = bytes_per_rule(rules, batched=len(nets) > 1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")  # > 129 MB L2
    opts = dict(mode=args.mode, block=args.block, grid=args.grid, solo_max=args.solo_max)
    tuned = None
    if args.mode == "auto" and (args.no_tune or args.block or args.grid or args.solo_max):
        opts["mode"] = "async"
    if not args.no_tune and not (args.block or args.grid or args.solo_max):
        # launch shape from the autotuner (timed runs outside the measured steps)
        from paper_1404_0076_gb300.autotune import Autotuner
        props = torch.cuda.get_device_properties(local)
        tuned = Autotuner().tune(
            ev, rules_text, nets, args.mode, gpu=props.name, num_sms=props.multi_processor_count)
        opts.update(tuned)

    def prepared():
        ev.reset()
        ids = ev.load_nets(nets)
        ev.stage(ids)
        flush.fill_(1)
        torch.cuda.synchronize()
        return ids

    for _ in range(args.warmup):
        prepared()
        ev.reduce([], **opts)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    dev_ms, ints, launches, alg_bytes = [], 0, 0, 0.0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            prepared()
            st = ev.reduce([], **opts)
            dev_ms.append(st["device_ms"])
            ints += st["interactions"]
            launches += st["launches"]
            alg_bytes += sum(c * b for c, b in zip(st["per_rule"], bpr))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_s = sum(dev_ms) / 1e3
    total_s_max, ints_all = combine(total_s, ints, dist)
    value = ints_all / total_s_max

    # roofline of the dominant kernel: one launch of it per step (k_async or
    # k_persistent) or, for the step kernels, per reduction step
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / total_s / 1e9
    ji = ev.jit_info()
    specialised = bool(ji["enabled"] and ji["state"] == 1 and opts["mode"] == "async")
    traffic = NCU_TRAFFIC.get((args.workload, opts["mode"], kernel_source_hash(), specialised))
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind, "bytes_per_interaction": alg_bytes / max(1, ints),
            # the same fraction at the DRAM bytes ncu measured for one launch
            "frac_at_traffic": (traffic / (total_s / args.steps) / 1e9) / peak if traffic else None,
            "kernel": {"async": "k_async" + ("<rule-specialised>" if specialised else ""), "persistent": "k_persistent",
                       "graph": "k_step", "plain": "k_step"}[opts["mode"]],
            "launch_time": "device time of the reduce call (for async: the queue fill, set-up and wind-down "
                           "kernels around k_async add a few microseconds)"}

    # secondary bounds.  Atomic units: every equation linked is at most one
    # exchange on a name slot; measured random exchanges per second, in a
    # slot array that fits L2 and in one that does not.  Critical path: the
    # number of maximally parallel steps (the persistent form's step count)
    # times the time per interaction along one dependency chain.
    from paper_1404_0076_gb300 import capi
    links = [r["n_link"] for r in rules]
    hist_tot = st["per_rule"]
    exch_per_int = sum(c * l for c, l in zip(hist_tot, links)) / max(1, sum(hist_tot))
    ex_l2 = capi.inet_bench_exch(local, 1 << 22, 1 << 28)
    ex_hbm = capi.inet_bench_exch(local, 1 << 30, 1 << 28)
    roof["atomics"] = {"exch_per_s_l2_resident": ex_l2, "exch_per_s_hbm": ex_hbm,
                       "exch_per_interaction_max": exch_per_int,
                       "interactions_per_s_bound": ex_hbm / max(1e-9, exch_per_int),
                       "frac": value / (ex_hbm / max(1e-9, exch_per_int)),
                       "how": "inet_bench_exch: random 32-bit atomicExch returning the old value, 16 MiB and 4 GiB arrays"}
    prepared()
    stp_depth = ev.reduce([], mode="persistent")
    depth = stp_depth["steps"]
    # the latency of one interaction with nothing else running: one warp on
    # one dependent chain of Add interactions (arithmetic rule set only)
    lone = None
    if rules_text == W.ARITH_RULES:
        ev.reset()
        ids_c = ev.load_nets([W.add_net(20000, 0)])
        ev.stage(ids_c)
        torch.cuda.synchronize()
        stc = ev.reduce([], mode="async", block=32, grid=1)
        lone = 1e6 * stc["device_ms"] / max(1, stc["interactions"])
    step_s = total_s / args.steps
    # the hardware floor of one level: one thread's dependent round trips
    # through L2 (16 MiB of records), measured here: a record load; an
    # exchange, then the record it names; a record store, fence, exchange and
    # load (what a level of second arrivals needs at the least)
    floor = {name: capi.inet_bench_chase(local, 1 << 20, 1 << 16, v)
             for v, name in ((0, "load"), (1, "exch_load"), (2, "store_fence_exch_load"))}
    per_level = floor["store_fence_exch_load"]
    roof["critical_path"] = {"depth_steps": depth,
                             "ns_per_level": 1e9 * step_s / max(1, depth),
                             "hw_floor_ns": floor,
                             "bound_ms": depth * per_level * 1e-6,
                             "frac": depth * per_level * 1e-9 / step_s,
                             "lone_chain_ns_per_interaction": lone,
                             "frac_of_lone_chain": depth * lone * 1e-9 / step_s if lone else None,
                             "how": "depth = steps of the maximally parallel loop (persistent form) on the same batch; "
                                    "ns_per_level = timed device time per step / depth; bound = depth x the hardware "
                                    "floor of one level (inet_bench_chase: one thread storing a record, fencing, "
                                    "exchanging a name slot and loading the record the exchange names, 2^16 dependent "
                                    "steps over an L2-resident array of 2^20 16-byte records); lone chain = one warp "
                                    "reducing Add(Z, r) = S^20000 Z with nothing else running, for comparison"}

    # e2e: public API from host text to host results, copies included.  The
    # steps run back to back and are timed together, from the parse of the
    # first step's texts to the numerals (or texts) of the last on the host;
    # each step's texts are parsed on a second thread (inet_parse_nets, which
    # needs no device) while the device reduces the step before, as a user of
    # the API would overlap them, and are then placed and uploaded
    # (inet_load_parsed, the host-to-device copy inside the timed region).
    e2e_int = 0
    ev.reset()
    torch.cuda.synchronize()
    h0, d0 = ev.transfer_bytes()
    t0 = time.perf_counter()
    parsed = ev.parse(nets)
    for k in range(args.e2e_steps):
        if k:
            ev.reset()
        ids = ev.load_parsed(parsed, 0, parsed.n)
        # the next step's parse starts once this step's placement is done:
        # both use the process's pool of host threads, which serves one job
        # at a time (a second job runs on its caller's thread alone)
        ahead, box = None, {}
        if k + 1 < args.e2e_steps:
            ahead = threading.Thread(target=lambda: box.__setitem__("p", ev.parse(nets)))
            ahead.start()
        st = ev.reduce(ids, **opts)
        if rules_text == W.ARITH_RULES:
            vals, per_net = ev.readback_nats(ids)   # the numerals, walked on the device
            assert all(v is not None for v in vals)
        else:
            texts = [ev.readback(i) for i in ids]   # the normal forms (->sub / ->col), rendered on the device
            per_net = [st["interactions"]]          # every net of the batch was reduced by this call
            assert all(texts)
        e2e_int += sum(per_net)
        if ahead is not None:
            ahead.join()
            parsed = box["p"]
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    h1, d1 = ev.transfer_bytes()
    e2e_h2d, e2e_d2h = (h1 - h0) // args.e2e_steps, (d1 - d0) // args.e2e_steps
    e2e_int //= args.e2e_steps
    # whole job: interactions of all ranks over the slowest rank's time
    e2e_s_max, e2e_int_all = combine(e2e_s, e2e_int, dist)
    e2e = {"value": e2e_int_all / e2e_s_max, "unit": UNIT,
           "h2d_bytes_per_step": e2e_h2d, "d2h_bytes_per_step": e2e_d2h,
           "ms_per_step": 1e3 * e2e_s_max, "steps": args.e2e_steps,
           "how": "steps back to back, timed together; each step's texts parsed on a second thread while the "
                  "device reduces the step before (the first step's in line)"}

    # the other loop forms on the same batch (one run each), and the plain
    # host-driven loop with one net per launch sequence
    plain = None
    if not args.no_plain and rank == 0:
        forms = {}
        for m in ("async", "persistent", "graph", "paper"):
            prepared()
            stm = ev.reduce([], mode=m)
            forms[m] = stm["interactions"] / (stm["device_ms"] / 1e3)
        ids = prepared()
        stp = ev.reduce([], mode="plain")
        one = []
        stride = max(1, len(nets) // max(1, args.plain_sample))
        sample = nets[::stride][: args.plain_sample]
        for net in sample:
            ev.reset()
            i = ev.load_net(net)
            ev.stage([i])
            torch.cuda.synchronize()
            s1 = ev.reduce([], mode="plain")
            one.append((s1["interactions"], s1["device_ms"]))
        plain = {"forms": forms, "forms_note": "paper = the loop of Sec. 3.6 with the sort-based communication of "
                                               "Sec. 3.5 (own kernels), for comparison",
                 "batch_plain": stp["interactions"] / (stp["device_ms"] / 1e3),
                 "one_net_per_launch": sum(a for a, _ in one) / (sum(b for _, b in one) / 1e3),
                 "one_net_sample": f"{len(sample)} nets (every {stride}th of the batch), each reduced alone by "
                                   "the host-driven loop",
                 "unit": UNIT}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        ci, cs = run_oracle(nets, cores, rules_text)
        cpu = {"value": ci / cs, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"whole workload once ({len(nets)} nets, {ci} interactions), {cores} threads"}
        # and single-threaded, on a bounded sample of the same nets
        sample = nets[: max(1, min(len(nets), 256))]
        si, ss = run_oracle(sample, 1, rules_text)
        cpu["single_thread"] = {"value": si / ss, "unit": UNIT, "cores": 1,
                                "sample": f"first {len(sample)} nets ({si} interactions), one thread"}

    # control: the paper's sort + merge communication phase (Sec. 3.5) on
    # the GPU against the atomic linker, on one synthetic equation set
    control = None
    if rank == 0 and world == 1 and not args.no_control:
        from paper_1404_0076_gb300 import capi as _capi
        eq, n_vars, expected = W.equation_chains(400000, 0.2, n_free=4000, n_direct=40000)
        best = {}
        for method in (0, 1):
            for _ in range(3):
                pairs, passes, ms = _capi.inet_control_link(local, eq, n_vars, method)
                assert len(pairs) == len(expected)
                if method not in best or ms < best[method][1]:
                    best[method] = (passes, ms)
        control = {"equations": int(len(eq)), "names": n_vars, "pairs": len(expected),
                   "atomic_ms": best[0][1], "sort_merge_ms": best[1][1], "sort_merge_passes": best[1][0],
                   "sort_merge_over_atomic": best[1][1] / max(1e-9, best[0][1]),
                   "how": "inet_control_link: stable LSD radix sort by name + merge of adjacent equations per pass "
                          "until no merge (method 1) vs one launch of atomic exchanges with chain chasing (method 0); "
                          "chains of 1 + Geometric(0.8) - 1 names; best of 3"}

    narrow = None
    if rank == 0 and world == 1 and not args.no_narrow:
        narrow = {name: narrow_leg(args, local, name) for name in ("ack3", "fib")}
        for rec in narrow.values():
            rec["frac_of_hw_floor"] = per_level / rec["ns_per_level"]

    ji = ev.jit_info()
    jit_note = {"rule_specialised": specialised,
                "jit_state": ji["state"], "jit_compile_ms": round(ji["compile_ms"], 1), "jit_source": ji["source"],
                "jit_launches": ji["launches"], "jit_msg": ji["msg"],
                "how": "asynchronous mode compiles k_async for the loaded rule set at its first launch (NVRTC, "
                       "before the timed steps); warps whose lanes all reduce one rule run that rule's code"}
    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        serving = serving_leg(args, local)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total_s_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": desc, "nets_per_rank": len(nets), "interactions_per_step": ints // args.steps,
                           "mode": opts["mode"], "mode_choice": "autotuned" if args.mode == "auto" and tuned else "given",
                           "block": opts["block"] or 256, "grid": opts["grid"] or "auto",
                           "launch_shape": "autotuned" if tuned else "given",
                           "l2": "flushed (256 MiB write) before every timed step",
                           "kernel": jit_note,
                           "parallelism": f"independent batches, {world} rank(s)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(), "plain": plain, "serving": serving, "paper_com_control": control,
                "narrow_frontier": narrow}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    ev.close()


if __name__ == "__main__":
    main()
