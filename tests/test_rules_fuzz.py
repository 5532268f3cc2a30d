"""CPU check of the rule compiler against the oracle's own rule parser:
seeded random edits inside one rule of the arithmetic and L-System rule
sets must be accepted or rejected alike.  A text can then hold two errors
(say a broken name and a stray character after the rule); the two checkers
may report different ones of them, so the error class must agree on almost
every rejected text, not on all."""
import random

import pytest

import workloads as W
from tests import oracle_runner


def edited(n: int, seed: int) -> list[str]:
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        lines = rng.choice([W.ARITH_RULES, W.LSYS_RULES]).splitlines(keepends=True)
        k = rng.choice([i for i, l in enumerate(lines) if l.strip() and not l.lstrip().startswith("#")])
        l = lines[k]
        op = rng.randrange(3)
        j = rng.randrange(len(l))
        if op == 0 and len(l) > 2:
            l = l[:j] + l[j + 1:]
        elif op == 1:
            l = l[:j] + rng.choice("(),=;xyzSZ -") + l[j:]
        elif len(l) > 3:
            j = rng.randrange(len(l) - 2)
            l = l[:j] + l[j + 1] + l[j] + l[j + 2:]
        lines[k] = l
        out.append("".join(lines))
    return out


@pytest.fixture(scope="module")
def capi():
    from paper_1404_0076_gb300 import build
    build.build()
    from paper_1404_0076_gb300 import capi as c
    return c


def test_edited_rule_sets_are_accepted_or_rejected_like_the_oracle(capi):
    oracle_runner.build()
    accepted = rejected = same_class = 0
    for text in edited(200, 14040076):
        r = oracle_runner.run(text, "< | >", quiet=True)
        want = r[0].get("rules", "ok") if r else None
        ctx = capi.inet_create(-1, None, None)
        try:
            capi.inet_load_rules(ctx, text)
            got = "ok"
        except capi.InetError as e:
            got = e.name
        capi.inet_destroy(ctx)
        assert (got == "ok") == (want == "ok"), (text, got, want)
        if got == "ok":
            accepted += 1
        else:
            rejected += 1
            same_class += got == want
    assert accepted > 30 and rejected > 60
    assert same_class >= 0.95 * rejected, (same_class, rejected)
