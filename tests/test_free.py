"""Per-net reclamation (inet_free_nets) and placement of new nets into the
freed slots, on the GPU, against the oracle.

Nets are independent configurations (Sec. 2.2), so a finished net's slots can
be handed to later nets; every result must stay what the oracle computes for
the net alone, and memory must be reused instead of the bump pointers
growing.
"""
import pytest

import workloads as W
from tests import oracle_runner

pytestmark = pytest.mark.gpu
R = W.ARITH_RULES

# non-numeral normal forms (two interface terms, a residual-free pair of
# numerals) and degenerate nets next to arithmetic
MIXED = [W.add_net(5, 3), W.mul_net(4, 6), "< a, b | Dup(a, b) = S(S(S(Z))) >", W.ack_net(2, 2), W.fib_net(9),
         "< r | r = Z >", "< r, s | Add(s, r) = Z >", W.mul_net(0, 7)]


@pytest.fixture(scope="module")
def orc():
    oracle_runner.build()
    return oracle_runner


def make_ev(**kw):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_1404_0076_gb300 import Evaluator
    return Evaluator(device=0, free_nets=True, **kw)


def check_against(ev, ids, expect, text=True):
    for i, o in zip(ids, expect):
        info = ev.net_info(i)
        assert info["status"] == "OK" and info["reduced"], (i, info)
        assert info["interactions"] == o["interactions"], (i, info, o["interactions"])
        assert info["live_agents"] == o["live"], (i, info, o["live"])
        if text:
            assert ev.readback(i) == o["result"], (i, o["result"])


@pytest.mark.parametrize("mode", ["persistent", "async", "plain"])
def test_freed_slots_are_reused_and_results_stay_exact(orc, mode):
    nets = MIXED * 8 + W.config1(count=64).nets
    expect = orc.run(R, nets)
    ev = make_ev(max_agents=1 << 21, max_vars=1 << 21, max_pairs=1 << 18, max_nets=2048)
    ev.load_rules(R)
    first = None
    id_sets = []
    for rnd in range(4):
        ids = ev.load_nets(nets)
        id_sets.append(set(ids))
        ev.reduce(ids, mode=mode)
        check_against(ev, ids, expect)
        use = ev.arena_usage()
        slack = 4 if mode == "async" else 16     # the async driver's allocation order varies most
        if first is None:
            first = use
        else:
            # the round before left every slot in the rings; the bump
            # pointers grow by at most a small share (how many slots each
            # step takes from the rings before freed ones are published varies
            # with the order pairs are handed out), never by a round's worth
            assert use["agent_slots"] <= first["agent_slots"] + first["agent_slots"] // slack + 64, (rnd, use, first)
            assert use["name_slots"] <= first["name_slots"] + first["name_slots"] // slack + 64, (rnd, use, first)
        assert use["live_agents"] == sum(o["live"] for o in expect)
        ev.free(ids)
        use = ev.arena_usage()
        # nothing leaks: every slot below the bump pointers is back in a ring
        assert use["live_agents"] == 0 and use["nets"] == 0, use
        assert use["free_agent_slots"] == use["agent_slots"] and use["free_name_slots"] == use["name_slots"], use
    # every round reused the ids the previous one released
    assert all(s == id_sets[0] for s in id_sets)
    ev.close()


def test_free_while_other_nets_reduce(orc):
    """Short nets arrive, finish, are read back and freed in epochs while two
    long nets keep reducing; later arrivals land in the freed slots."""
    longs = [W.fib_net(15), W.mul_net(30, 30)]
    shorts = [W.add_net(17 * k % 200, 31 * k % 150) for k in range(40)] + \
             [W.mul_net(k % 9, (5 * k) % 11) for k in range(40)] + [W.fib_net(k % 10) for k in range(20)]
    exp_long = orc.run(R, longs)
    exp_short = orc.run(R, shorts)
    ev = make_ev(max_agents=1 << 21, max_vars=1 << 21, max_pairs=1 << 18, max_nets=4096)
    ev.load_rules(R)
    lid = ev.load_nets(longs)
    ev.stage(lid)
    live_short = {}   # net id -> index into shorts
    usage = []
    batches = 0
    for _ in range(100000):
        if batches < 12:
            ids = ev.load_nets(shorts)
            ev.stage(ids)
            live_short.update({i: k for k, i in enumerate(ids)})
            batches += 1
        st = ev.reduce([], mode="async", slice_us=300, check=False)
        assert st["status"] in ("OK", "STEP_LIMIT"), st
        fin = [i for i in ev.finished() if i in live_short]
        if fin:
            vals, ints = ev.readback_nats(fin)
            for i, v, n in zip(fin, vals, ints):
                o = exp_short[live_short[i]]
                assert (v, n) == (o["nat"], o["interactions"]), (i, v, n, o)
            ev.free(fin)
            for i in fin:
                del live_short[i]
            usage.append(ev.arena_usage()["agent_slots"])
        if st["status"] == "OK" and not live_short and batches >= 12:
            break
    else:
        raise AssertionError("the loop did not finish")
    check_against(ev, lid, exp_long, text=False)
    vals, _ = ev.readback_nats(lid)
    assert vals == [o["nat"] for o in exp_long]
    # twelve batches of short nets passed through; the arena did not grow by
    # twelve batches' worth (every batch after the first reuses freed slots)
    from paper_1404_0076_gb300 import capi
    h = capi.inet_create(-1)
    capi.inet_load_rules(h, R)
    capi.inet_load_nets(h, shorts)
    one_batch = capi.inet_arena_usage(h)["agent_slots"]
    capi.inet_destroy(h)
    assert len(usage) >= 2
    assert usage[-1] <= usage[0] + 5 * one_batch, (usage, one_batch)
    ev.free(lid)
    use = ev.arena_usage()
    assert use["live_agents"] == 0 and use["nets"] == 0, use
    assert use["free_agent_slots"] == use["agent_slots"] and use["free_name_slots"] == use["name_slots"], use
    ev.close()


def test_free_errors_leave_everything_in_place(orc):
    ev = make_ev(max_agents=1 << 20, max_vars=1 << 20, max_pairs=1 << 16, max_nets=64)
    ev.load_rules(R)
    from paper_1404_0076_gb300 import InetError
    a, b = ev.load_nets([W.fib_net(14), W.add_net(40, 2)])
    c = ev.load_net(W.add_net(3, 3))             # loaded, never staged
    ev.reduce([a, b], mode="async", slice_us=50, check=False)
    pend = ev.pending([a, b])
    if pend[0]:
        with pytest.raises(InetError) as e:      # a net with active pairs left
            ev.free([a, b])
        assert e.value.name == "STATE"
    with pytest.raises(InetError) as e:
        ev.free([c])
    assert e.value.name == "STATE"
    ev.reduce([], mode="async")                  # finish both
    with pytest.raises(InetError) as e:
        ev.free([b, b])
    assert e.value.name == "INVALID_ARG"
    # a net whose readback is in flight is not freed
    ev.readback_nats_begin([a])
    with pytest.raises(InetError) as e:
        ev.free([a])
    assert e.value.name == "STATE"
    vals, _ = ev.readback_nats_end(wait=True)
    exp = orc.run(R, [W.fib_net(14), W.add_net(40, 2), W.add_net(3, 3)])
    assert vals == [exp[0]["nat"]]
    ev.free([a, b])
    with pytest.raises(InetError) as e:          # freed ids are unknown
        ev.readback(a)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(InetError):
        ev.free([a])
    # the released ids come back, and the net that waited reduces correctly
    d, f = ev.load_nets([W.fib_net(14), W.add_net(40, 2)])
    assert {d, f} == {a, b}
    ev.reduce([c, d, f], mode="persistent")
    assert ev.readback(c) == exp[2]["result"]
    assert ev.readback(d) == exp[0]["result"] and ev.readback(f) == exp[1]["result"]
    ev.close()


def test_quota_stops_one_net_only(orc):
    nets = [W.fib_net(18), W.mul_net(9, 11), W.add_net(50, 7)]
    exp = orc.run(R, nets)
    ev = make_ev(max_agents=1 << 20, max_vars=1 << 20, max_pairs=1 << 16, max_nets=64)
    ev.load_rules(R)
    ids = ev.load_nets(nets)
    # Fibonacci(18) peaks far above 500 live agents; the others far below
    # their quotas
    ev.set_quotas(ids, [500, 1 << 20, 0])
    ev.stage(ids)
    for _ in range(1000):
        st = ev.reduce([], mode="async", slice_us=100, check=False)
        if st["status"] == "OK" or ids[0] in ev.finished():
            break
    ev.reduce([], mode="async")
    assert ev.status(ids) == ["ARENA_FULL", "OK", "OK"]
    assert ev.pending(ids) == [0, 0, 0]
    check_against(ev, ids[1:], exp[1:])
    ev.free(ids)
    use = ev.arena_usage()
    assert use["live_agents"] == 0 and use["free_agent_slots"] == use["agent_slots"]
    # the context goes on: the same net without a quota reduces correctly
    i = ev.load_net(nets[0])
    ev.reduce([i], mode="async")
    check_against(ev, [i], exp[:1])
    ev.close()


def test_free_needs_owner_tracking(orc):
    from paper_1404_0076_gb300 import Evaluator, InetError
    with Evaluator(device=0, max_agents=1 << 16, max_vars=1 << 16, max_pairs=1 << 12, max_nets=16) as ev:
        ev.load_rules(R)
        ids = ev.load_nets([W.add_net(3, 4)])
        ev.reduce(ids, mode="async")
        with pytest.raises(InetError) as e:
            ev.free(ids)
        assert e.value.name == "STATE"
        assert ev.readback(ids[0]) == "S(S(S(S(S(S(S(Z)))))))"


def test_placement_rewrites_pairs_of_nets_staged_later(orc):
    """Nets uploaded together into freed slots but staged in two calls: the
    second call's initial pairs were rewritten on the host."""
    nets = [W.mul_net(6, 5), W.add_net(9, 4), "< a, b | Dup(a, b) = S(Z) >", W.ack_net(2, 1)]
    exp = orc.run(R, nets)
    ev = make_ev(max_agents=1 << 18, max_vars=1 << 18, max_pairs=1 << 14, max_nets=64)
    ev.load_rules(R)
    warm = ev.load_nets(nets * 4)
    ev.reduce(warm, mode="async")
    ev.free(warm)
    u0 = ev.arena_usage()
    ids = ev.load_nets(nets)
    ev.stage(ids[:2])                            # uploads all four, places them, stages two
    u1 = ev.arena_usage()                        # all of them went into freed slots
    assert (u1["agent_slots"], u1["name_slots"]) == (u0["agent_slots"], u0["name_slots"]), (u0, u1)
    ev.reduce(ids[2:], mode="async")             # the other two join, with rewritten pairs
    check_against(ev, ids, exp)
    ev.close()
