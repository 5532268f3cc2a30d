"""CPU check of the library's net parser against the oracle's own parser:
seeded random edits of valid nets (a character dropped, inserted or two
swapped) must be accepted or rejected alike, with the same error class
(PARSE or LINEARITY).  The two parsers share no code."""
import random

import pytest

import workloads as W
from tests import oracle_runner

BASE = [W.add_net(3, 2), W.mul_net(2, 3), W.fib_net(4), "< a, b | Dup(a, b) = S(Z) >",
        "< r | Add(y, r) = S(Z), y = Z >", "< | >", "< r, s | r = s >", "< | x = y, y = x >", "< S(Z), Z() | >",
        "< r | T(r) = S(S(Z)) >"]


def mutated(n: int, seed: int) -> list[str]:
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        t = rng.choice(BASE)
        op = rng.randrange(4)
        j = rng.randrange(len(t) + 1)
        if op == 0 and len(t) > 1:
            t = t[:j] + t[j + 1:]
        elif op == 1:
            t = t[:j] + rng.choice("(),=|<>;xyzSZ -") + t[j:]
        elif op == 2 and len(t) > 2:
            k = rng.randrange(len(t) - 1)
            t = t[:k] + t[k + 1] + t[k] + t[k + 2:]
        out.append(t)
    return out


@pytest.fixture(scope="module")
def capi():
    from paper_1404_0076_gb300 import build
    build.build()
    from paper_1404_0076_gb300 import capi as c
    return c


def test_mutated_nets_are_accepted_or_rejected_like_the_oracle(capi):
    oracle_runner.build()
    ctx = capi.inet_create(-1, None, None)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    accepted = 0
    for t in mutated(300, 14040076):
        r = oracle_runner.run(W.ARITH_RULES, [t], quiet=True)
        want = r[0]["status"] if r and "status" in r[0] else (r[0].get("nets") if r else None)
        try:
            capi.inet_load_net(ctx, t)
            got = "ok"
        except capi.InetError as e:
            got = e.name
        assert got == want, (t, got, want)
        accepted += got == "ok"
    assert 100 < accepted < 280  # both kinds of text were drawn
    capi.inet_destroy(ctx)
