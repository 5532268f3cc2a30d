"""Plants mistakes in the oracle (compile-time hooks, CPU only) and checks
that the pins of test_oracle.py catch every one of them.

Mutants: 1 transposed argument binding, 2 an interaction left uncounted,
3 bound names not kept apart, 4 rule orientation ignored, 5 a wrong
substitution in ->col/->sub, 6 live-agent count off by one, 7 ->com drops a
side.
"""
import os
import tempfile
import types

import pytest

from tests import oracle_runner
from tests import test_oracle as pins

CHECKS = [
    lambda o: [pins.test_paper_examples(o, c) for c in pins.golden()],
    pins.test_add_values_and_counts,
    pins.test_mul_values_counts_and_histogram,
    pins.test_ackermann_values_and_counts,
    pins.test_fibonacci_values_and_counts,
    lambda o: [pins.test_bruteforce_all_orders(o, n) for n in pins.BRUTE[:6]],
]


@pytest.mark.slow
@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7])
def test_pins_catch_planted_mistake(mutant):
    with tempfile.TemporaryDirectory() as d:
        exe = oracle_runner.compile_oracle(os.path.join(d, f"mutant{mutant}"), {"ORACLE_MUTANT": mutant})

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
