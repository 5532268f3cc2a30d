"""Pins for the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: the paper's worked examples
(tests/golden), closed-form values and interaction counts derived by hand
from the rules, an independent brute-force enumeration of every reduction
order (tests/bruteforce.py), and the invariants of Sec. 2.1 / Sec. 2.2.
"""
import json
import os

import pytest

import workloads as W
from tests import bruteforce

HERE = os.path.dirname(os.path.abspath(__file__))
R = W.ARITH_RULES
RULE = {name: i for i, name in enumerate(W.ARITH_RULE_NAMES)}


def golden():
    with open(os.path.join(HERE, "golden", "paper_examples.jsonl")) as f:
        return [json.loads(line) for line in f if line.strip()]


# --- closed forms, written from the rules by hand ---------------------------

def fib(n):
    a, b = 0, 1
    for _ in range(n):
        a, b = b, a + b
    return a


def ack(m, n):
    # Textbook closed forms for m <= 3 (checked against the recursive
    # definition on small arguments in test_ack_closed_forms).
    return [n + 1, n + 2, 2 * n + 3, 2 ** (n + 3) - 3][m]


def ack_rec(m, n):
    if m == 0:
        return n + 1
    if n == 0:
        return ack_rec(m - 1, 1)
    return ack_rec(m - 1, ack_rec(m, n - 1))


def count_mul(m, n):
    # Mul><Z once, Era over the copy of n (n+1), and per Mul><S step k
    # (k = 0..m-1): itself, Dup over n (n+1), and Add over k*n (k*n+1).
    return 1 + (n + 1) + sum(1 + (n + 1) + (k * n + 1) for k in range(m))


def count_ack(m, n):
    # A><Z: 1.  A><S then A2><Z: 2 + C(m-1, 1).  A><S then A2><S:
    # 2 + the Dup of m-1 (m steps) + C(m, n-1) + C(m-1, ack(m, n-1)).
    # Tables are filled bottom-up (the recursion is too deep for Python).
    tab = {0: None}

    def c(mm, nn):
        if mm == 0:
            return 1
        row = tab.setdefault(mm, [])
        while len(row) <= nn:
            k = len(row)
            if k == 0:
                row.append(2 + c(mm - 1, 1))
            else:
                row.append(2 + mm + row[k - 1] + c(mm - 1, ack(mm, k - 1)))
        return row[nn]

    return c(m, n)


def count_fib(n):
    # Fib><Z: 1.  Fib><S + Fib2><Z: 2.  Fib><S + Fib2><S: 2 + Dup of k=n-2
    # (k+1) + fib(k+1) and fib(k) subcomputations + Add over fib(k+1).
    c = [1, 2]
    for k in range(0, n - 1):
        c.append(2 + (k + 1) + c[k + 1] + c[k] + fib(k + 1) + 1)
    return c[n]


# --- the paper's worked examples ---------------------------------------------

@pytest.mark.parametrize("case", golden(), ids=lambda c: c["id"])
def test_paper_examples(oracle, case):
    e = case["expect"]
    r = oracle.run(case["rules"], case["net"])[0]
    assert r["status"] == "ok", r
    assert r["result"] == e["result"]
    assert r["interactions"] == e["interactions"]
    if "nat" in e:
        assert r["nat"] == e["nat"]
    if "live" in e:
        assert r["live"] == e["live"]
    rr = oracle.run(case["rules"], case["net"], mode="rounds")[0]
    assert rr.get("rounds", []) == e["rounds"]


# --- closed forms --------------------------------------------------------------

def test_add_values_and_counts(oracle):
    cases = [(m, n) for m in range(0, 9) for n in range(0, 9)] + [(256, 0), (0, 256), (200, 57)]
    res = oracle.run(R, [W.add_net(m, n) for m, n in cases], quiet=True)
    for (m, n), r in zip(cases, res):
        assert r["status"] == "ok"
        assert r["nat"] == m + n
        assert r["interactions"] == m + 1
        assert r["per_rule"][RULE["Add><S"]] == m
        assert r["per_rule"][RULE["Add><Z"]] == 1
        assert r["live"] == m + n + 1          # garbage-free: exactly S^(m+n) Z remains


def test_mul_values_counts_and_histogram(oracle):
    cases = [(m, n) for m in range(0, 7) for n in range(0, 7)] + [(12, 9), (64, 64)]
    res = oracle.run(R, [W.mul_net(m, n) for m, n in cases], quiet=True)
    for (m, n), r in zip(cases, res):
        assert r["status"] == "ok"
        assert r["nat"] == m * n
        assert r["interactions"] == count_mul(m, n)
        h = r["per_rule"]
        assert h[RULE["Mul><S"]] == m and h[RULE["Mul><Z"]] == 1
        assert h[RULE["Dup><S"]] == m * n and h[RULE["Dup><Z"]] == m
        assert h[RULE["Era><S"]] == n and h[RULE["Era><Z"]] == 1
        assert h[RULE["Add><S"]] == n * m * (m - 1) // 2 and h[RULE["Add><Z"]] == m
        assert r["live"] == m * n + 1


def test_ackermann_values_and_counts(oracle):
    cases = [(a, b) for a in range(0, 3) for b in range(0, 6)] + [(3, b) for b in range(0, 6)]
    res = oracle.run(R, [W.ack_net(a, b) for a, b in cases], quiet=True)
    for (a, b), r in zip(cases, res):
        assert r["status"] == "ok"
        assert r["nat"] == ack(a, b)
        assert r["interactions"] == count_ack(a, b)
        assert r["live"] == ack(a, b) + 1
    assert count_ack(3, 7) == 1388937 and ack(3, 8) == 2045


def test_ack_closed_forms():
    for m in range(4):
        for n in range(5 if m == 3 else 12):
            assert ack(m, n) == ack_rec(m, n)


def test_fibonacci_values_and_counts(oracle):
    ns = list(range(0, 18))
    res = oracle.run(R, [W.fib_net(n) for n in ns], quiet=True)
    for n, r in zip(ns, res):
        assert r["status"] == "ok"
        assert r["nat"] == fib(n)
        assert r["interactions"] == count_fib(n)
        assert r["live"] == fib(n) + 1
    assert fib(20) == 6765 and count_fib(20) == 138336


def test_pred(oracle):
    res = oracle.run(R, [W.pred_net(n) for n in range(5)])
    for n, r in enumerate(res):
        assert r["nat"] == max(0, n - 1) and r["interactions"] == 1


# --- invariants: uniform confluence (Sec. 2.1) and Theorem 1 (Sec. 2.2) -------

SMALL = [W.add_net(5, 3), W.mul_net(4, 3), W.ack_net(2, 2), W.ack_net(3, 1), W.fib_net(9),
         "< r | Add(y, r) = S(Z), Add(S(Z), y) = Z >",
         "< a, b | Dup(a, b) = S(S(Z)) >"]


def test_every_schedule_gives_the_same_result(oracle):
    ref = oracle.run(R, SMALL)
    for mode, seed in [("fifo", 1), ("rounds", 1), ("random", 1), ("random", 7), ("random", 12345)]:
        got = oracle.run(R, SMALL, mode=mode, seed=seed)
        for a, b in zip(ref, got):
            assert (a["result"], a["interactions"], a["per_rule"], a["live"]) == \
                   (b["result"], b["interactions"], b["per_rule"], b["live"]), mode


def test_deferring_sub_and_col_changes_nothing(oracle):
    # Theorem 1: int/com first, sub/col at the end == interleaving them.
    ref = oracle.run(R, SMALL)
    eager = oracle.run(R, SMALL, eager=True)
    for a, b in zip(ref, eager):
        assert (a["result"], a["interactions"]) == (b["result"], b["interactions"])


def test_rounds_profile_sums_to_interactions(oracle):
    res = oracle.run(R, [W.fib_net(12), W.ack_net(3, 3), W.mul_net(9, 7)], mode="rounds")
    for r in res:
        assert sum(r["rounds"]) == r["interactions"]
        assert len(r["live_rounds"]) == len(r["rounds"])
        assert max(r["live_rounds"]) <= r["peak_live"]
    # Add is sequential: one active pair per round.
    r = oracle.run(R, W.add_net(20, 5), mode="rounds")[0]
    assert r["rounds"] == [1] * 21


def test_peak_live_of_addition(oracle):
    # Add(y, r) = S(x) keeps two agents for two; Add(y, r) = Z removes both:
    # the most agents alive is what the net starts with, Add and the numerals
    # S^m Z and S^n Z, in every order: m + n + 3
    for m, n in ((0, 0), (1, 0), (7, 3), (40, 200)):
        for mode in ("lifo", "fifo", "rounds"):
            r = oracle.run(R, W.add_net(m, n), mode=mode)[0]
            assert r["peak_live"] == m + n + 3 and r["live"] == m + n + 1


BRUTE = [W.add_net(2, 1), W.mul_net(1, 2), W.mul_net(2, 2), W.ack_net(1, 1), W.ack_net(2, 1),
         W.fib_net(3), W.fib_net(4), "< a, b | Dup(a, b) = S(S(Z)) >",
         "< r | Add(y, r) = S(Z), Add(S(Z), y) = Z >"]


@pytest.mark.parametrize("net", BRUTE)
def test_bruteforce_all_orders(oracle, net):
    bf = bruteforce.explore(R, net)
    assert bf["consistent"], "two maximal reduction paths of different length"
    assert bf["min"] == bf["max"]
    assert len(bf["finals"]) == 1, bf["finals"]
    (text, residual), = bf["finals"]
    r = oracle.run(R, net)[0]
    assert r["result"] == text and r["residual_eqs"] == residual
    assert r["interactions"] == bf["min"]
    # the oracle's peak of live agents is that of one reduction path, in
    # every schedule it offers
    for mode in ("lifo", "fifo", "random", "rounds"):
        p = oracle.run(R, net, mode=mode)[0]["peak_live"]
        assert bf["peak_min"] <= p <= bf["peak_max"], (mode, p, bf["peak_min"], bf["peak_max"])


# --- the linker cases of Sec. 3.6 and degenerate nets ---------------------------

def test_chain_of_names_resolves_to_one_pair(oracle):
    rules = "Alpha = Beta -> ;\n"
    for k in range(0, 6):
        chain = ", ".join([f"x{i} = x{i + 1}" for i in range(k)])
        net = f"< | Alpha = x0{', ' + chain if chain else ''}, x{k} = Beta >"
        r = oracle.run(rules, net, mode="rounds")[0]
        assert r["interactions"] == 1 and r["rounds"] == [1] and r["live"] == 0


def test_vicious_circles(oracle):
    r = oracle.run(R, "< | x = y, y = x >")[0]
    assert r["status"] == "ok" and r["interactions"] == 0 and r["residual_eqs"] == 1
    r = oracle.run(R, "< | x = S(y), y = S(x) >")[0]
    assert r["residual_eqs"] == 1 and r["residual_agents"] == 2


def test_empty_and_trivial_nets(oracle):
    assert oracle.run(R, "< | >")[0]["result"] == ""
    r = oracle.run(R, "< r, s | r = s >")[0]
    assert r["result"] == "x0, x0" and r["interactions"] == 0
    r = oracle.run(R, "< S(Z) | >")[0]
    assert r["nat"] == 1


# --- errors ---------------------------------------------------------------------

def test_errors(oracle):
    foo = "Foo(x) = Bar -> x = Bar;\n"
    assert oracle.run(foo, "< r | Foo(r) = Baz >")[0]["status"] == "PARSE"
    assert oracle.run(foo + "Baz = Bar -> ;\n", "< r | Foo(r) = Baz >")[0]["status"] == "NO_RULE"
    assert oracle.run("Foo(x) = Bar -> ;\n", "< | >")[0].get("rules") == "LINEARITY"
    assert oracle.run(R, "< r | Add(x, r) = S(x), x = Z >")[0]["status"] == "LINEARITY"
    bad = oracle.run("Foo(x) = Bar -> x = y;\n", "< | >")[0]
    assert bad.get("rules") == "LINEARITY"
    assert oracle.run(R, W.fib_net(10), max_interactions=100)[0]["status"] == "STEP_LIMIT"


# --- the L-System benchmark (Sec. 5: A -> AB, B -> A) -----------------------------

def lsys_word(n: int) -> str:
    """The L-System word after n steps from A, by plain string rewriting."""
    w = "A"
    for _ in range(n):
        w = "".join("AB" if ch == "A" else "A" for ch in w)
    return w


def fibs(k: int) -> list[int]:
    f = [0, 1]
    while len(f) <= k:
        f.append(f[-1] + f[-2])
    return f


def lsys_counts(n: int) -> tuple[int, list[int]]:
    """Interactions and per-rule counts of lsys_net(n), derived by hand from
    the six rules: a symbol with count m > 0 applies its S rule once; SymA
    also duplicates S^(m-1) Z (m - 1 Dup><S and one Dup><Z) and spawns SymA
    and SymB with m - 1; SymB becomes SymA with m - 1; at m = 0 a symbol
    becomes a leaf (one Z rule)."""
    f = fibs(n + 3)
    a_expand = f[n + 2] - 1                 # A-symbols over steps 0..n-1: sum fib(i+1)
    b_expand = f[n + 1] - 1                 # B-symbols over steps 0..n-1: sum fib(i)
    dup_s = sum(f[i + 1] * (n - i - 1) for i in range(n))
    per_rule = [f[n + 1], a_expand, f[n], b_expand, a_expand, dup_s]
    ia, ib = [1], [1]                       # the recursion over the count, as a cross-check
    for m in range(1, n + 1):
        ia.append(1 + m + ia[m - 1] + ib[m - 1])
        ib.append(1 + ia[m - 1])
    assert ia[n] == sum(per_rule)
    return ia[n], per_rule


def leaves(text: str) -> str:
    return "".join("A" if t == "LeafA" else "B" for t in text.replace("(", " ").replace(")", " ")
                   .replace(",", " ").split() if t in ("LeafA", "LeafB"))


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 8, 12, 16])
def test_lsystem_word_counts_and_histogram(oracle, n):
    r = oracle.run(W.LSYS_RULES, [W.lsys_net(n)])[0]
    assert r["status"] == "ok"
    assert leaves(r["result"]) == lsys_word(n)
    ints, per_rule = lsys_counts(n)
    assert r["interactions"] == ints and r["per_rule"] == per_rule
    f = fibs(n + 2)
    assert r["live"] == 2 * f[n + 2] - 1        # leaves plus the Cat nodes over them
    assert r["result"].count("Cat(") == f[n + 2] - 1


def test_lsystem_grows_in_parallel(oracle):
    # the rounds schedule: depth linear in n, width exponential (Sec. 5
    # reports several hundred thousand parallel interactions at n = 27)
    r = oracle.run(W.LSYS_RULES, [W.lsys_net(20)], mode="rounds", quiet=True)[0]
    assert sum(r["rounds"]) == lsys_counts(20)[0]
    assert len(r["rounds"]) <= 3 * 20
    assert max(r["rounds"]) > 10000


@pytest.mark.parametrize("n", [1, 2, 3])
def test_lsystem_bruteforce_all_orders(oracle, n):
    net = W.lsys_net(n)
    bf = bruteforce.explore(W.LSYS_RULES, net)
    assert bf["consistent"] and bf["min"] == bf["max"] and len(bf["finals"]) == 1
    (text, _), = bf["finals"]
    r = oracle.run(W.LSYS_RULES, [net])[0]
    assert r["result"] == text and r["interactions"] == bf["min"] == lsys_counts(n)[0]


# --- binary trees (a second rule set with arity-two constructors) -----------
# Closed forms from the rules: a walker meets every constructor of the tree
# once (nodes + leaves interactions); Leaves also adds, at each node, the
# left subtree's count into the right's (Add consumes its S^k Z: k + 1
# interactions); Left drops the right subtree; Swap touches the root only.

def t_nodes(t):
    return 0 if t is None else 1 + t_nodes(t[0]) + t_nodes(t[1])


def t_leaves(t):
    return 1 if t is None else t_leaves(t[0]) + t_leaves(t[1])


def t_mirror(t):
    return None if t is None else (t_mirror(t[1]), t_mirror(t[0]))


def t_add_cost(t):
    return 0 if t is None else t_leaves(t[0]) + 1 + t_add_cost(t[0]) + t_add_cost(t[1])


def tree_cases(seed=20240607, count=40, depth=6):
    import random
    rng = random.Random(seed)
    trees = [None, (None, None), ((None, None), None)]
    while len(trees) < count:
        trees.append(W.random_tree(rng, depth))
    return trees


def test_tree_walkers_values_and_counts(oracle):
    trees = tree_cases()
    nets, want = [], []
    for t in trees:
        tt, agents = W.tree_text(t), t_nodes(t) + t_leaves(t)
        nets.append(f"< r | Mirror(r) = {tt} >")
        want.append((W.tree_text(t_mirror(t)), agents))
        nets.append(f"< r | Leaves(r) = {tt} >")
        want.append((W.numeral(t_leaves(t)), agents + t_add_cost(t)))
        nets.append(f"< p, q | Copy(p, q) = {tt} >")
        want.append((tt + ", " + tt, agents))
        nets.append(f"< | Drop = {tt} >")
        want.append(("", agents))
        nets.append(f"< r | Left(r) = {tt} >")
        want.append(("Leaf" if t is None else W.tree_text(t[0]),
                     1 if t is None else 1 + t_nodes(t[1]) + t_leaves(t[1])))
        nets.append(f"< r | Swap(r) = {tt} >")
        want.append(("Leaf" if t is None else W.tree_text((t[1], t[0])), 1))
        nets.append(f"< r | Mirror(r) = x, Mirror(x) = {tt} >")
        want.append((tt, 2 * agents))
    res = oracle.run(W.TREE_RULES, nets)
    for net, r, (text, n) in zip(nets, res, want):
        assert r["status"] == "ok", net
        assert (r["result"], r["interactions"]) == (text, n), net
        assert r["residual_agents"] == 0


@pytest.mark.parametrize("net", ["< r | Leaves(r) = Node(Node(Leaf, Leaf), Leaf) >",
                                 "< p, q | Copy(p, q) = Node(Leaf, Node(Leaf, Leaf)) >",
                                 "< r | Swap(r) = x, Mirror(x) = Node(Node(Leaf, Leaf), Leaf) >"])
def test_tree_bruteforce_all_orders(oracle, net):
    bf = bruteforce.explore(W.TREE_RULES, net)
    assert bf["consistent"] and bf["min"] == bf["max"] and len(bf["finals"]) == 1
    (text, _), = bf["finals"]
    r = oracle.run(W.TREE_RULES, [net])[0]
    assert r["result"] == text and r["interactions"] == bf["min"]
