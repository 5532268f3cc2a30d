"""Text readback on the device (->col / ->sub, Theorem 1, and the rendering
of the interface) against the oracle, byte for byte.

Every inet_readback of the other GPU tests goes through the same path; here
the device side is checked to have done the work (no fallback to the host
walk), on the L-System's 514 229-symbol word, on names numbered past 9, on
interfaces that are names, and on nets that share an arena with many others.
"""
import pytest

import workloads as W
from tests import oracle_runner

pytestmark = pytest.mark.gpu
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


def names_net(k: int) -> str:
    """< Dup(a0, a1), Dup(a2, a3), .., a_p(0), a_p(1), .. >: k names (k even),
    each once inside a Dup and once as a root, the roots in a scrambled
    order, so the canonical numbers run past 9 and follow first occurrence."""
    dups = [f"Dup(a{2 * i}, a{2 * i + 1})" for i in range(k // 2)]
    perm = [(7 * i + 3) % k for i in range(k)]
    return "< " + ", ".join(dups + [f"a{p}" for p in perm]) + " | >"


def test_lsystem_27_text_on_the_device():
    from tests.test_oracle import leaves, lsys_word
    ev = make_ev(max_agents=1 << 22, max_vars=1 << 22, max_pairs=1 << 21)
    ev.load_rules(W.LSYS_RULES)
    i = ev.load_net(W.lsys_net(27))
    ev.reduce([i], mode="persistent")
    text = ev.readback(i)
    assert ev.readback_counts() == (1, 0)
    assert leaves(text) == lsys_word(27)
    # the oracle's text, byte for byte (the oracle prints the first million
    # characters of a text this long and marks it truncated)
    o = oracle_runner.run(W.LSYS_RULES, [W.lsys_net(27)], timeout=300)[0]
    assert text == o["result"] or (o["truncated"] and len(o["result"]) > 1000000 and text.startswith(o["result"]))
    # the render counted the net's agents: net_info takes them from it
    info = ev.net_info(i)
    assert info["live_agents"] == 2 * 514229 - 1 == o["live"] and info["residual_agents"] == 0
    ev.close()


def test_mixed_texts_and_counts_on_the_device(orc):
    nets = [W.add_net(5, 3), W.mul_net(4, 6), "< a, b | Dup(a, b) = S(S(S(Z))) >", W.ack_net(2, 2),
            W.fib_net(9), "< r | r = Z >", "< r, s | Add(s, r) = Z >", W.mul_net(0, 7), names_net(6),
            names_net(40), "< | x = S(y), y = S(x) >", "< r, s | r = s >", "< a, b, c | Dup(a, b) = c >",
            "< r | r = x, x = y, y = S(Z) >", "< q | Add(S(Z), q) = S(S(Z)), Era = Z >"]
    exp = orc.run(R, nets)
    ev = make_ev(max_agents=1 << 20, max_vars=1 << 20, max_pairs=1 << 16, max_nets=64)
    ev.load_rules(R)
    ids = ev.load_nets(nets)
    ev.reduce(ids, mode="async")
    for i, o in zip(ids, exp):
        assert o["status"] == "ok", o
        assert ev.readback(i) == o["result"], (i, o["result"])
        info = ev.net_info(i)     # after the render: live and residual from the device
        assert (info["live_agents"], info["residual_agents"]) == (o["live"], o["residual_agents"]), (i, info, o)
        assert info["interactions"] == o["interactions"]
    assert ev.readback_counts() == (len(nets), 0)
    ev.close()


def test_one_net_among_many_in_a_large_arena(orc):
    # the render works on the net's own agents, whatever else the arena holds
    batch = W.config1(count=512).nets
    pick = [3, 100, 511]
    exp = orc.run(R, [batch[k] for k in pick])
    ev = make_ev(max_agents=1 << 22, max_vars=1 << 22, max_pairs=1 << 20, max_nets=1024)
    ev.load_rules(R)
    ids = ev.load_nets(batch)
    ev.reduce(ids, mode="async")
    for k, o in zip(pick, exp):
        assert ev.readback(ids[k]) == o["result"]
    assert ev.readback_counts() == (len(pick), 0)
    ev.close()
