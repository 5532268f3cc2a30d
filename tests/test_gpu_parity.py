"""GPU parity: the CUDA evaluator against the CPU oracle, element by element.

Everything is integer graph rewriting, so the bar is bit-exact: the rendered
normal form, the numeral value, the interaction count (per net and per rule),
the live and residual agents of every net, and the per-step frontier sizes
against the oracle's maximally parallel "rounds" schedule.
"""
import json
import os
import time

import pytest

import workloads as W
from tests import oracle_runner

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
MODES = ["plain", "graph", "persistent"]
R = W.ARITH_RULES


@pytest.fixture(scope="module")
def orc():
    oracle_runner.build()
    return oracle_runner


def make_ev(**kw):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_1404_0076_gb300 import Evaluator
    return Evaluator(device=0, **kw)


def run_gpu(rules, nets, mode, text=True, trace=False, **kw):
    caps = {k: kw.pop(k) for k in ("max_agents", "max_vars", "max_pairs", "max_nets") if k in kw}
    ev = make_ev(**caps)
    ev.load_rules(rules)
    ids = ev.load_nets(nets)
    st = ev.reduce(ids, mode=mode, trace=trace, **kw)
    out = []
    for i in ids:
        info = ev.net_info(i)
        rec = {"info": info}
        if text:
            rec["result"] = ev.readback(i)
        try:
            rec["nat"] = ev.readback_nat(i)[0]
        except Exception:
            rec["nat"] = None
        out.append(rec)
    tr = ev.trace() if trace else None
    ev.close()
    return st, out, tr


def compare(oracle_res, gpu_out, text=True):
    for k, (o, g) in enumerate(zip(oracle_res, gpu_out)):
        assert o["status"] == "ok", o
        gi = g["info"]
        assert gi["status"] == "OK" and gi["reduced"], (k, gi)
        assert gi["interactions"] == o["interactions"], (k, gi, o["interactions"])
        assert gi["live_agents"] == o["live"], (k, gi, o["live"])
        assert gi["residual_agents"] == o["residual_agents"], (k, gi)
        assert g["nat"] == o["nat"], (k, g["nat"], o["nat"])
        if text:
            assert g["result"] == o["result"], (k, g["result"][:200], o["result"][:200])


def summed_rounds(oracle_res):
    L = max((len(o.get("rounds", [])) for o in oracle_res), default=0)
    agg = [0] * L
    for o in oracle_res:
        for i, x in enumerate(o.get("rounds", [])):
            agg[i] += x
    return agg


def golden():
    with open(os.path.join(HERE, "golden", "paper_examples.jsonl")) as f:
        return [json.loads(line) for line in f if line.strip()]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", golden(), ids=lambda c: c["id"])
def test_paper_examples(orc, mode, case):
    o = orc.run(case["rules"], case["net"], mode="rounds")
    st, g, tr = run_gpu(case["rules"], [case["net"]], mode, trace=True)
    compare(o, g)
    assert g[0]["result"] == case["expect"]["result"]
    assert tr[0] == case["expect"]["rounds"]


SMALL = ([W.add_net(m, n) for m, n in [(0, 0), (1, 0), (0, 1), (3, 4), (17, 5), (64, 64)]]
         + [W.mul_net(m, n) for m, n in [(0, 0), (0, 5), (1, 1), (3, 4), (7, 2), (9, 9)]]
         + [W.ack_net(a, b) for a, b in [(0, 0), (1, 3), (2, 2), (3, 1), (3, 3)]]
         + [W.fib_net(n) for n in range(0, 13)]
         + [W.pred_net(n) for n in range(3)]
         + ["< r | Add(y, r) = S(Z), Add(S(Z), y) = Z >", "< a, b | Dup(a, b) = S(S(Z)) >",
            "< | >", "< r, s | r = s >", "< S(Z) | >", "< | x = y, y = x >", "< | x = S(y), y = S(x) >",
            "< r | Add(y, r) = S(S(Z)), y = Add(Z, q), q = Z >"])


@pytest.mark.parametrize("mode", MODES)
def test_small_mixed_batch(orc, mode):
    o = orc.run(R, SMALL, mode="rounds")
    st, g, tr = run_gpu(R, SMALL, mode, trace=True)
    compare(o, g)
    assert tr[0] == summed_rounds(o)
    assert st["interactions"] == sum(x["interactions"] for x in o)
    per_rule = [sum(x["per_rule"][r] for x in o) for r in range(len(o[0]["per_rule"]))]
    assert st["per_rule"] == per_rule


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("block", [64, 256, 512])
def test_several_tiles_and_ragged_tail(orc, mode, block):
    # 1000 Add nets plus a few wide ones: frontiers of 1000+ pairs over
    # blocks of 64..512 threads, never a multiple of the block size.
    nets = [W.add_net((7 * i) % 23, i % 5) for i in range(1000)] + [W.fib_net(11), W.mul_net(6, 5)]
    o = orc.run(R, nets, mode="rounds", quiet=True)
    st, g, tr = run_gpu(R, nets, mode, text=False, trace=True, block=block)
    compare(o, g, text=False)
    assert tr[0] == summed_rounds(o)


@pytest.mark.parametrize("solo_max", [-1, 64, 1024])
def test_persistent_solo_and_wide(orc, solo_max):
    nets = [W.fib_net(14), W.ack_net(3, 2), W.mul_net(8, 8)] + [W.add_net(i, 3) for i in range(300)]
    o = orc.run(R, nets, mode="rounds")
    st, g, tr = run_gpu(R, nets, "persistent", trace=True, solo_max=solo_max)
    compare(o, g)
    assert tr[0] == summed_rounds(o)


def full_config(k):
    w = W.CONFIGS[k]()
    return w.nets


@pytest.mark.parametrize("cfg,mode", [(0, "persistent"), (0, "graph"), (1, "persistent"), (2, "persistent"),
                                      (3, "persistent"), (2, "graph")])
def test_full_size_configs(orc, cfg, mode):
    nets = full_config(cfg)
    o = orc.run(R, nets, mode="rounds", quiet=(cfg == 1), threads=os.cpu_count() or 4)
    st, g, tr = run_gpu(R, nets, mode, text=(cfg != 1), trace=True, max_agents=1 << 24, max_vars=1 << 24,
                        max_pairs=1 << 21)
    compare(o, g, text=(cfg != 1))
    assert tr[0] == summed_rounds(o)
    assert st["interactions"] == sum(x["interactions"] for x in o)


def test_plain_loop_fib_and_ack(orc):
    nets = [W.fib_net(18), W.ack_net(3, 4)]
    o = orc.run(R, nets, mode="rounds")
    st, g, tr = run_gpu(R, nets, "plain", trace=True)
    compare(o, g)
    assert tr[0] == summed_rounds(o)


@pytest.mark.parametrize("mode", MODES)
def test_step_limit_is_resumable(orc, mode):
    net = W.fib_net(13)
    o = orc.run(R, net)[0]
    ev = make_ev()
    ev.load_rules(R)
    i = ev.load_net(net)
    st = ev.reduce([i], mode=mode, max_steps=7, check=False)
    calls = 1
    while st["status"] == "STEP_LIMIT":
        assert st["steps"] == 7
        st = ev.reduce([], mode=mode, max_steps=7, check=False)
        calls += 1
    assert st["status"] == "OK" and calls > 3
    assert ev.readback(i) == o["result"] and ev.net_info(i)["interactions"] == o["interactions"]
    ev.close()


@pytest.mark.parametrize("mode", MODES)
def test_no_rule_stops_only_its_net(orc, mode):
    rules = R + "Foo(x) = Bar -> x = Bar;\n"
    nets = [W.add_net(5, 2), "< r | Foo(r) = Z >", W.fib_net(7)]
    ev = make_ev()
    ev.load_rules(rules)
    ids = ev.load_nets(nets)
    st = ev.reduce(ids, mode=mode, check=False)
    assert st["status"] == "NO_RULE"
    assert ev.net_info(ids[1])["status"] == "NO_RULE"
    o = orc.run(rules, [nets[0], nets[2]])
    assert ev.readback(ids[0]) == o[0]["result"] and ev.readback(ids[2]) == o[1]["result"]
    ev.close()


@pytest.mark.parametrize("mode", MODES)
def test_arena_full_is_reported_and_reset_recovers(orc, mode):
    from paper_1404_0076_gb300 import InetError
    ev = make_ev(max_agents=400, max_vars=400, max_pairs=256)
    ev.load_rules(R)
    i = ev.load_net(W.fib_net(12))
    st = ev.reduce([i], mode=mode, check=False)
    assert st["status"] == "ARENA_FULL"
    with pytest.raises(InetError):
        ev.load_net(W.add_net(1, 1))
    ev.reset()
    j = ev.load_net(W.add_net(4, 4))
    ev.reduce([j], mode=mode)
    assert ev.readback_nat(j) == (8, 5)
    ev.close()


def test_bounded_wait_times_out_cleanly(orc):
    # A 1 ns wait limit makes every grid-barrier wait of the persistent
    # kernel give up: the kernel must return INET_ERR_TIMEOUT, not hang, and
    # the context must work again after a reset.
    ev = make_ev()
    ev.load_rules(R)
    ids = ev.load_nets([W.add_net(200, 1) for _ in range(2000)])
    st = ev.reduce(ids, mode="persistent", solo_max=-1, timeout_s=1e-9, check=False)
    assert st["status"] == "TIMEOUT"
    ev.reset()
    j = ev.load_net(W.mul_net(3, 3))
    ev.reduce([j], mode="persistent")
    assert ev.readback_nat(j)[0] == 9
    ev.close()


def test_incremental_batches_share_the_loop(orc):
    # Nets added to a running context (after a partial reduction) finish
    # with the same results as alone.
    nets_a = [W.fib_net(12), W.mul_net(5, 7)]
    nets_b = [W.ack_net(2, 3), W.add_net(30, 4)]
    o = orc.run(R, nets_a + nets_b)
    ev = make_ev()
    ev.load_rules(R)
    ia = ev.load_nets(nets_a)
    st = ev.reduce(ia, mode="persistent", max_steps=20, check=False)
    assert st["status"] == "STEP_LIMIT"
    ib = ev.load_nets(nets_b)
    ev.reduce(ib, mode="persistent")
    for k, i in enumerate(ia + ib):
        assert ev.readback(i) == o[k]["result"]
        assert ev.net_info(i)["interactions"] == o[k]["interactions"]
    ev.close()


# --- the asynchronous driver (no steps: results and counts, no per-step trace) ---

@pytest.mark.parametrize("block", [32, 128, 256])
def test_async_small_mixed_batch(orc, block):
    o = orc.run(R, SMALL)
    st, g, _ = run_gpu(R, SMALL, "async", block=block)
    compare(o, g)
    assert st["interactions"] == sum(x["interactions"] for x in o)
    per_rule = [sum(x["per_rule"][r] for x in o) for r in range(len(o[0]["per_rule"]))]
    assert st["per_rule"] == per_rule


def test_async_many_nets_and_wide_fanout(orc):
    nets = [W.add_net((7 * i) % 23, i % 5) for i in range(1000)] + [W.fib_net(14), W.mul_net(9, 8), W.ack_net(3, 3)]
    o = orc.run(R, nets, quiet=True)
    st, g, _ = run_gpu(R, nets, "async", text=False)
    compare(o, g, text=False)


@pytest.mark.parametrize("cfg", [0, 1, 2, 3])
def test_async_full_size_configs(orc, cfg):
    nets = full_config(cfg)
    o = orc.run(R, nets, quiet=(cfg == 1), threads=os.cpu_count() or 4)
    st, g, _ = run_gpu(R, nets, "async", text=(cfg != 1), max_agents=1 << 24, max_vars=1 << 24, max_pairs=1 << 21)
    compare(o, g, text=(cfg != 1))
    assert st["interactions"] == sum(x["interactions"] for x in o)


_MUL_ORACLE = {}


@pytest.mark.parametrize("block,grid", [(64, 1216), (128, 608), (256, 304), (256, 152)])
def test_async_mul_batch_in_the_bench_shapes(orc, block, grid):
    # the 2048-net Mul batch in the launch shapes the autotuner picks for the
    # bench (16 warps per SM) and one block per SM, every net against the oracle
    nets = full_config(1)
    if "o" not in _MUL_ORACLE:
        _MUL_ORACLE["o"] = orc.run(R, nets, quiet=True, threads=os.cpu_count() or 4)
    o = _MUL_ORACLE["o"]
    st, g, _ = run_gpu(R, nets, "async", text=False, block=block, grid=grid, max_agents=1 << 24,
                       max_vars=1 << 24, max_pairs=1 << 20, max_nets=4096)
    compare(o, g, text=False)
    assert st["interactions"] == sum(x["interactions"] for x in o) == 47391647


def test_async_slices_are_resumable(orc):
    nets = [W.fib_net(17), W.mul_net(12, 11)]
    o = orc.run(R, nets)
    ev = make_ev()
    ev.load_rules(R)
    ids = ev.load_nets(nets)
    st = ev.reduce(ids, mode="async", slice_us=200, check=False)
    calls = 1
    while st["status"] == "STEP_LIMIT":
        st = ev.reduce([], mode="async", slice_us=200, check=False)
        calls += 1
        assert calls < 10000
    assert st["status"] == "OK"
    for k, i in enumerate(ids):
        assert ev.readback(i) == o[k]["result"]
        assert ev.net_info(i)["interactions"] == o[k]["interactions"]
        assert ev.net_info(i)["live_agents"] == o[k]["live"]
    ev.close()


def test_async_then_steps_continue_the_same_nets(orc):
    # a sliced asynchronous call leaves its pairs in the frontier, which the
    # step kernels can finish (and the reverse)
    nets = [W.fib_net(15), W.ack_net(2, 5)]
    o = orc.run(R, nets)
    ev = make_ev()
    ev.load_rules(R)
    ids = ev.load_nets(nets)
    ev.reduce(ids, mode="persistent", max_steps=30, check=False)
    ev.reduce([], mode="async", slice_us=100, check=False)
    ev.reduce([], mode="graph")
    for k, i in enumerate(ids):
        assert ev.readback(i) == o[k]["result"]
        assert ev.net_info(i)["interactions"] == o[k]["interactions"]
    ev.close()


def test_async_no_rule_and_arena_full(orc):
    rules = R + "Foo(x) = Bar -> x = Bar;\n"
    nets = [W.add_net(5, 2), "< r | Foo(r) = Z >", W.fib_net(7)]
    ev = make_ev()
    ev.load_rules(rules)
    ids = ev.load_nets(nets)
    st = ev.reduce(ids, mode="async", check=False)
    assert st["status"] == "NO_RULE"
    o = orc.run(rules, [nets[0], nets[2]])
    assert ev.readback(ids[0]) == o[0]["result"] and ev.readback(ids[2]) == o[1]["result"]
    ev.close()
    ev = make_ev(max_agents=400, max_vars=400, max_pairs=256)
    ev.load_rules(R)
    i = ev.load_net(W.fib_net(12))
    t0 = time.perf_counter()
    assert ev.reduce([i], mode="async", check=False)["status"] == "ARENA_FULL"
    # the error ends the loop at once, not after a bounded wait runs out
    assert time.perf_counter() - t0 < 2.0
    ev.reset()
    j = ev.load_net(W.add_net(4, 4))
    ev.reduce([j], mode="async")
    assert ev.readback_nat(j) == (8, 5)
    ev.close()


def test_pending_and_batched_nat_readback(orc):
    # inet_net_pending counts a net's unreduced pairs; inet_readback_nats
    # reads many numerals at once and marks an interface that is not S^k(Z)
    nets = [W.fib_net(16), W.add_net(7, 9), W.mul_net(9, 8), "< a, b | Add(a, b) = Z >", W.ack_net(2, 4)]
    o = orc.run(R, nets)
    ev = make_ev()
    ev.load_rules(R)
    ids = ev.load_nets(nets)
    ev.stage(ids)
    assert ev.pending(ids) == [ev.net_info(i)["pending_pairs"] for i in ids]
    st = ev.reduce([], mode="async", slice_us=50, check=False)
    while st["status"] == "STEP_LIMIT":
        pend = ev.pending(ids)
        assert all(p >= 0 for p in pend)
        st = ev.reduce([], mode="async", slice_us=50, check=False)
    assert st["status"] == "OK"
    assert ev.pending(ids) == [0] * len(ids)
    vals, ints = ev.readback_nats(ids)
    assert ints == [x["interactions"] for x in o]
    assert vals == [x["nat"] for x in o]
    assert vals[3] is None
    # the batched walk agrees with the one-net readback, also in another order
    rev = ids[::-1]
    assert ev.readback_nats(rev)[0] == vals[::-1]
    for i, v in zip(ids, vals):
        if v is not None:
            assert ev.readback_nat(i)[0] == v
    assert ev.readback_nats([]) == ([], [])
    ev.close()


@pytest.mark.parametrize("grid,block", [(1, 32), (0, 0)])
def test_async_queue_wraps_near_capacity(orc, grid, block):
    # in-flight pairs hold two live agents each, so with these nets (at
    # most about 900 live agents at once under any schedule) 512 pairs
    # always suffice, while the ticket queue of 512 slots wraps several
    # times; producers then wait for slots of the previous lap
    nets = [W.fib_net(12), W.ack_net(3, 4)]
    o = orc.run(R, nets)
    ev = make_ev(max_pairs=512)
    ev.load_rules(R)
    ids = ev.load_nets(nets)
    t0 = time.perf_counter()
    st = ev.reduce(ids, mode="async", grid=grid, block=block)
    assert time.perf_counter() - t0 < 5.0
    assert st["status"] == "OK"
    for k, i in enumerate(ids):
        assert ev.readback(i) == o[k]["result"]
        assert ev.net_info(i)["interactions"] == o[k]["interactions"]
    ev.close()


def test_async_pair_capacity_is_an_error_not_a_wait(orc):
    # more pairs in flight than the frontier holds ends the loop with
    # ARENA_FULL at once; if this schedule stayed below the capacity the
    # results must be exact
    nets = [W.fib_net(14)]
    ev = make_ev(max_pairs=64)
    ev.load_rules(R)
    ids = ev.load_nets(nets)
    t0 = time.perf_counter()
    st = ev.reduce(ids, mode="async", check=False)
    assert time.perf_counter() - t0 < 2.0
    assert st["status"] in ("ARENA_FULL", "OK")
    if st["status"] == "OK":
        o = orc.run(R, nets)
        assert ev.readback(ids[0]) == o[0]["result"]
    ev.reset()
    j = ev.load_net(W.add_net(3, 4))
    ev.reduce([j], mode="async")
    assert ev.readback_nat(j) == (7, 4)
    ev.close()


def test_batched_nat_readback_leaves_the_trace(orc):
    nets = [W.add_net(20, 5), W.mul_net(6, 7)]
    o = orc.run(R, nets, mode="rounds")
    ev = make_ev()
    ev.load_rules(R)
    ids = ev.load_nets(nets)
    ev.reduce(ids, mode="persistent", trace=True)
    tr = ev.trace()
    assert tr[0] == summed_rounds(o)
    assert ev.readback_nats(ids)[0] == [25, 42]
    assert ev.trace() == tr
    ev.close()


def test_nonblocking_readback_overlaps_reduction(orc):
    # finished nets are read back on the context's second stream while the
    # main stream keeps reducing another net of the same arena
    from paper_1404_0076_gb300.capi import InetError
    first = [W.add_net(3000, 7), W.mul_net(40, 30), W.fib_net(14), "< a, b | Add(a, b) = Z >"]
    o = orc.run(R, first)
    ev = make_ev()
    ev.load_rules(R)
    ids = ev.load_nets(first)
    ev.reduce(ids, mode="async")
    with pytest.raises(InetError):
        ev.readback_nats_end()              # nothing begun
    ev.readback_nats_begin(ids)
    with pytest.raises(InetError):
        ev.readback_nats_begin(ids)         # one batch at a time
    with pytest.raises(InetError):
        ev.readback_nats(ids)               # the blocking form shares its scratch
    late = ev.load_net(W.ack_net(3, 5))
    ev.reduce([late], mode="async")
    r = None
    for _ in range(100000):
        r = ev.readback_nats_end()
        if r is not None:
            break
    assert r is not None
    vals, ints = r
    assert vals == [x["nat"] for x in o] and ints == [x["interactions"] for x in o]
    assert ev.readback_nat(late)[0] == 253
    ev.readback_nats_begin([late])
    assert ev.readback_nats_end(wait=True) == ([253], [ev.net_info(late)["interactions"]])
    ev.readback_nats_begin(ids)
    ev.reset()                              # waits for the walk, drops it
    with pytest.raises(InetError):
        ev.readback_nats_end()
    ev.close()


def long_readback_nets():
    # numerals longer than one thread's walk (list ranking finishes them),
    # walks that end exactly at the budget, a name chain in front of a
    # numeral, a long S chain that ends in a non-numeral agent
    chain = "< r | r = x1, " + ", ".join(f"x{i} = x{i + 1}" for i in range(1, 400)) + f", x400 = {W.numeral(300)} >"
    nonnat = "< r | r = " + "S(" * 300 + "Add(Z, x)" + ")" * 300 + ", x = Z >"
    return [W.add_net(3000, 7), W.mul_net(40, 50), W.add_net(0, 129), W.add_net(128, 0), W.add_net(127, 1),
            W.add_net(63, 1), chain, nonnat, "< a, b | Add(a, b) = Z >", W.add_net(1, 1), W.fib_net(18),
            W.add_net(0, 0), W.add_net(0, 257), W.add_net(256, 0), W.add_net(255, 1), W.add_net(254, 1)]


@pytest.mark.parametrize("mode", ["async", "persistent"])
def test_batched_nat_readback_ranks_long_numerals(orc, mode):
    nets = long_readback_nets()
    o = orc.run(R, nets)
    want = [x["nat"] for x in o]
    assert want[:6] == [3007, 2000, 129, 128, 128, 64] and want[6:8] == [300, None]
    ev = make_ev()
    ev.load_rules(R)
    ids = ev.load_nets(nets)
    ev.reduce(ids, mode=mode)
    vals, ints = ev.readback_nats(ids)
    assert vals == want and ints == [x["interactions"] for x in o]
    for i, v in zip(ids, vals):
        if v is not None:
            assert ev.readback_nat(i)[0] == v
    # subsets and repeats, blocking and non-blocking
    sub = [ids[7], ids[0], ids[0], ids[9], ids[1]]
    assert ev.readback_nats(sub)[0] == [want[7], want[0], want[0], want[9], want[1]]
    ev.readback_nats_begin(ids[::-1])
    assert ev.readback_nats_end(wait=True)[0] == want[::-1]
    # the arena grows: the ranking scratch grows with it
    more = ev.load_nets([W.mul_net(64, 64), W.add_net(5000, 5000)])
    ev.reduce(more, mode=mode)
    assert ev.readback_nats(more + ids[:2])[0] == [4096, 10000, 3007, 2000]
    ev.close()


def test_batched_nat_readback_of_the_full_mul_batch():
    # all 2048 numerals of the Mul batch (results up to 4096 S agents)
    w = W.config1()
    ev = make_ev(max_agents=1 << 24, max_vars=1 << 24, max_pairs=1 << 20, max_nets=4096)
    ev.load_rules(w.rules)
    ids = ev.load_nets(w.nets)
    ev.reduce(ids, mode="async")
    vals, _ = ev.readback_nats(ids)
    assert vals == [m * n for m, n in w.params]
    ev.readback_nats_begin(ids)
    assert ev.readback_nats_end(wait=True)[0] == vals
    ev.close()


# --- the L-System benchmark (Sec. 5) ---------------------------------------------

@pytest.mark.parametrize("mode", MODES + ["async"])
def test_lsystem_small(orc, mode):
    nets = [W.lsys_net(n) for n in (0, 1, 5, 10, 14)]
    o = orc.run(W.LSYS_RULES, nets, mode="rounds")
    st, g, tr = run_gpu(W.LSYS_RULES, nets, mode, trace=(mode != "async"))
    compare(o, g)
    if mode != "async":
        assert tr[0] == summed_rounds(o)
    per_rule = [sum(x["per_rule"][r] for x in o) for r in range(len(o[0]["per_rule"]))]
    assert st["per_rule"] == per_rule


@pytest.mark.parametrize("mode", ["async", "persistent"])
def test_lsystem_27_full_size(mode):
    # 514 229 symbols, 2 692 506 interactions: checked against the closed
    # forms and the word obtained by rewriting the string
    from tests.test_oracle import leaves, lsys_counts, lsys_word
    ev = make_ev(max_agents=1 << 22, max_vars=1 << 22, max_pairs=1 << 21)
    ev.load_rules(W.LSYS_RULES)
    i = ev.load_net(W.lsys_net(27))
    st = ev.reduce([i], mode=mode)
    ints, per_rule = lsys_counts(27)
    assert st["interactions"] == ints and st["per_rule"] == per_rule
    info = ev.net_info(i)
    assert info["interactions"] == ints and info["live_agents"] == 2 * 514229 - 1
    assert leaves(ev.readback(i)) == lsys_word(27)
    ev.close()


def test_finished_nets_are_reported_once(orc):
    # inet_net_finished reports every net once its pending pairs reach zero:
    # normal forms, nets with no pair at all, and nets stopped by NO_RULE
    rules = R + "Foo(x) = Bar -> x = Bar;\n"
    nets = [W.fib_net(15), W.add_net(5, 2), "< r | r = Z >", "< r | Foo(r) = Z >", W.mul_net(20, 30)]
    ev = make_ev()
    ev.load_rules(rules)
    ids = ev.load_nets(nets)
    ev.stage(ids)
    seen = []
    for _ in range(100000):
        # a slice that met the missing rule returns NO_RULE, not STEP_LIMIT,
        # while other nets may still be reducing
        st = ev.reduce([], mode="async", slice_us=50, check=False)
        assert st["status"] in ("OK", "STEP_LIMIT", "NO_RULE")
        seen += ev.finished()
        if not any(ev.pending(ids)):
            break
    seen += ev.finished()
    assert sorted(seen) == sorted(ids)               # each exactly once
    assert ev.finished() == []
    assert ev.pending(ids) == [0] * len(ids)
    o = orc.run(rules, [nets[0], nets[1], nets[4]])
    assert [ev.net_info(ids[i])["interactions"] for i in (0, 1, 4)] == [x["interactions"] for x in o]
    assert ev.net_info(ids[3])["status"] == "NO_RULE"
    # a net loaded later is reported after it finishes, not before
    late = ev.load_net(W.add_net(3, 3))
    assert ev.finished() == []
    ev.reduce([late], mode="async")
    assert ev.finished() == [late]
    ev.close()


# --- randomized batches against the oracle (the lock-free queue under stress) -----

def random_batch(rng, n):
    nets = []
    for _ in range(n):
        f = rng.randrange(5)
        if f == 0:
            nets.append(W.add_net(rng.randrange(0, 400), rng.randrange(0, 50)))
        elif f == 1:
            nets.append(W.mul_net(rng.randrange(0, 25), rng.randrange(0, 25)))
        elif f == 2:
            nets.append(W.ack_net(rng.choice([1, 2, 3]), rng.randrange(0, 5)))
        elif f == 3:
            nets.append(W.fib_net(rng.randrange(0, 17)))
        else:
            nets.append(W.pred_net(rng.randrange(0, 30)))
    return nets


@pytest.mark.parametrize("seed", range(6))
def test_async_random_batches_and_launch_shapes(orc, seed):
    import random
    rng = random.Random(14040076 + 100 + seed)
    nets = random_batch(rng, rng.randrange(1, 400))
    o = orc.run(R, nets, quiet=True)
    block = rng.choice([32, 64, 128, 256])
    grid = rng.choice([1, 2, 7, 0, 152, 600])
    slice_us = rng.choice([0, 0, 100, 1000])
    # pairs in flight never exceed half the live agents, plus one per lane
    # between consuming a pair and counting it out, so this capacity always
    # suffices while the ticket ring still wraps
    need = sum(x["peak_live"] for x in o) // 2 + 80000
    max_pairs = need * rng.choice([1, 2, 4])
    ev = make_ev(max_pairs=max_pairs)
    ev.load_rules(R)
    ids = ev.load_nets(nets)
    ev.stage(ids)
    for _ in range(100000):
        st = ev.reduce([], mode="async", block=block, grid=grid, slice_us=slice_us, check=False)
        assert st["status"] in ("OK", "STEP_LIMIT"), (st["status"], block, grid, slice_us, max_pairs)
        if st["status"] == "OK":
            break
    vals, ints = ev.readback_nats(ids)
    assert ints == [x["interactions"] for x in o], (block, grid, slice_us, max_pairs)
    assert vals == [x["nat"] for x in o], (block, grid, slice_us, max_pairs)
    for i, x in zip(ids, o):
        assert ev.net_info(i)["live_agents"] == x["live"]
    assert sorted(ev.finished()) == sorted(ids)
    ev.close()


def test_async_random_serving_arenas_in_sequence(orc):
    # several batches through one context with resets in between: queue
    # cells, stacks and counters start over each time
    import random
    rng = random.Random(14040076 + 200)
    batches = [random_batch(rng, rng.randrange(10, 200)) for _ in range(5)]
    results = [orc.run(R, nets, quiet=True) for nets in batches]
    need = max(sum(x["peak_live"] for x in o) for o in results) // 2 + 80000
    ev = make_ev(max_pairs=need)
    ev.load_rules(R)
    for rnd, (nets, o) in enumerate(zip(batches, results)):
        ids = ev.load_nets(nets)
        ev.reduce(ids, mode="async", block=rng.choice([64, 256]), grid=rng.choice([0, 304]))
        vals, ints = ev.readback_nats(ids)
        assert (vals, ints) == ([x["nat"] for x in o], [x["interactions"] for x in o]), rnd
        ev.reset()
    ev.close()


def test_package_docstring_example():
    ev = make_ev()
    with ev:
        ev.load_rules("Add(y, r) = Z -> r = y;\n"
                      "Add(y, r) = S(x) -> Add(y, w) = x, r = S(w);\n")
        ids = ev.load_nets(["< r | Add(S(Z), r) = S(S(Z)) >"])
        ev.reduce(ids, mode="async")
        assert ev.readback(ids[0]) == "S(S(S(Z)))"
        assert ev.readback_nats(ids) == ([3], [3])


# --- the paper's own loop form (Sec. 3.5-3.6) -------------------------------------

@pytest.mark.parametrize("case", golden(), ids=lambda c: c["id"])
def test_paper_form_examples(orc, case):
    st, g, _ = run_gpu(case["rules"], [case["net"]], "paper")
    o = orc.run(case["rules"], [case["net"]])
    compare(o, g)


def test_paper_form_mixed_batch_and_tiles(orc):
    nets = SMALL + [W.add_net(i % 37, i % 11) for i in range(1002)]
    o = orc.run(R, nets)
    st, g, _ = run_gpu(R, nets, "paper", text=True, block=128)
    compare(o, g)
    assert st["interactions"] == sum(x["interactions"] for x in o)


def test_paper_form_full_add_batch_and_lsystem(orc):
    nets = W.config0().nets
    o = orc.run(R, nets, quiet=True)
    st, g, _ = run_gpu(R, nets, "paper", text=False)
    compare(o, g, text=False)
    from tests.test_oracle import leaves, lsys_counts, lsys_word
    ev = make_ev()
    ev.load_rules(W.LSYS_RULES)
    i = ev.load_net(W.lsys_net(16))
    st = ev.reduce([i], mode="paper")
    assert (st["interactions"], st["per_rule"]) == lsys_counts(16)
    assert leaves(ev.readback(i)) == lsys_word(16)
    ev.close()


def test_paper_form_continues_what_another_form_left(orc):
    # name slots bound by a sliced asynchronous run become equations of the
    # paper's form, and what the paper's form leaves is read back as usual
    nets = [W.fib_net(14), W.mul_net(12, 9), W.ack_net(2, 3)]
    o = orc.run(R, nets)
    ev = make_ev()
    ev.load_rules(R)
    ids = ev.load_nets(nets)
    ev.reduce(ids, mode="async", slice_us=30, check=False)
    ev.reduce([], mode="paper")
    for k, i in enumerate(ids):
        assert ev.readback(i) == o[k]["result"]
        assert ev.net_info(i)["interactions"] == o[k]["interactions"]
        assert ev.net_info(i)["live_agents"] == o[k]["live"]
    ev.close()
