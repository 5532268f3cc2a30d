"""Plants mistakes in a copy of the oracle's source (CPU only) and checks
that the pins of test_oracle.py catch every one of them.  The oracle itself
carries no hooks: each mutant is a textual edit of one statement, applied to
a temporary copy, and the edit must find its statement exactly once (so a
change to the oracle cannot silently leave a mutant untested).

Mutants: 1 transposed argument binding, 2 an interaction with an empty
right-hand side left uncounted, 3 bound names not kept apart, 4 rule
orientation ignored, 5 a wrong substitution in ->col/->sub, 6 live-agent
count off by one, 7 ->com drops a side.
"""
import os
import tempfile
import types

import pytest

from tests import oracle_runner
from tests import test_oracle as pins

# (statement in the oracle, what the mutant puts in its place)
MUTANTS = {
    1: ("bind[(size_t)rule.a_vars[i]] = l->arg[i];",
        "bind[(size_t)rule.a_vars[i]] = l->arg[rule.a_vars.size() - 1 - i];"),
    2: ("    interactions++;\n    per_rule[(size_t)ridx]++;",
        "    if (!rule.rhs.empty()) interactions++;\n    per_rule[(size_t)ridx]++;"),
    3: ("if (!rule.is_lhs[(size_t)v]) fresh[(size_t)v] = fresh_name();",
        "if (!rule.is_lhs[(size_t)v]) { int64_t s = -1; for (int u = 0; u < v; u++) "
        "if (fresh[(size_t)u] >= 0) { s = fresh[(size_t)u]; break; } fresh[(size_t)v] = s >= 0 ? s : fresh_name(); }"),
    4: ("if (it->second & 1) std::swap(l, r);", "if (false) std::swap(l, r);"),
    5: ("      free_names.push_back(x);\n      *slot = t;",
        "      free_names.push_back(x);\n      if (!is_name(t) && rs.sym.arity[(size_t)t->sym] > 0) t = t->arg[0];\n"
        "      *slot = t;"),
    6: ("live += rule.rhs_agents - 2;", "live += rule.rhs_agents - 2 + (rule.rhs_agents > 2 ? 1 : 0);"),
    7: ("    free_names.push_back(x);\n    add_eq(t, u);",
        "    free_names.push_back(x);\n    if (!is_name(u) && !is_name(t)) { add_eq(t, t); return true; }\n"
        "    add_eq(t, u);"),
}

CHECKS = [
    lambda o: [pins.test_paper_examples(o, c) for c in pins.golden()],
    pins.test_add_values_and_counts,
    pins.test_mul_values_counts_and_histogram,
    pins.test_ackermann_values_and_counts,
    pins.test_fibonacci_values_and_counts,
    lambda o: [pins.test_bruteforce_all_orders(o, n) for n in pins.BRUTE[:6]],
]


def mutant_source(k: int) -> str:
    with open(oracle_runner.SRC) as f:
        src = f.read()
    old, new = MUTANTS[k]
    assert src.count(old) == 1, f"mutant {k}: its statement occurs {src.count(old)} times in the oracle"
    return src.replace(old, new)


def test_every_mutant_finds_its_statement():
    for k in MUTANTS:
        assert mutant_source(k) != open(oracle_runner.SRC).read()


@pytest.mark.slow
@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant):
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, f"mutant{mutant}.cpp")
        with open(src, "w") as f:
            f.write(mutant_source(mutant))
        exe = oracle_runner.compile_oracle(os.path.join(d, f"mutant{mutant}"), src=src)

        def run(*a, **k):
            k["binary"] = exe
            k.setdefault("timeout", 60)
            return oracle_runner.run(*a, **k)

        o = types.SimpleNamespace(run=run)
        caught = []
        for check in CHECKS:
            try:
                check(o)
            except Exception as ex:  # an assertion, a crash or a bad status all count
                caught.append(type(ex).__name__)
        assert caught, f"mutant {mutant} passed every pin"
