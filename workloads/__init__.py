"""Seeded synthetic inputs for the interaction-net evaluator and its oracle.

This module only writes text: the rule set (in the lightweight-calculus
syntax of Sec. 2.2, one rule ``alpha(x..) = beta(y..) -> Theta;`` per line)
and configurations ``< t.. | Delta >`` built from unary numerals.  It holds
none of the method's arithmetic: no reduction, no linking, no counting.  Both
the CUDA path and the CPU oracle parse the same text with their own parsers.

Rule set (Sec. 2.2, Eq. 1-2 for addition; the others are our own encodings of
the textbook recurrences, since the paper prints no rules for its other
benchmarks):

  Add   add(0,y)=y ; add(S x,y)=S add(x,y)                (Eq. 2, Eq. 1)
  Dup   copies a numeral ; Era erases one
  Mul   mul(0,y)=0 ; mul(S x,y)=add(mul(x,y), y)
  A/A2  ack(0,n)=n+1 ; ack(m+1,0)=ack(m,1) ; ack(m+1,n+1)=ack(m,ack(m+1,n))
  Pred  pred(0)=0 ; pred(S x)=x
  Fib/Fib2  fib(0)=0 ; fib(1)=1 ; fib(k+2)=fib(k+1)+fib(k)

The principal port of every function agent faces the argument it matches on;
the auxiliary ports are listed in the order written, the last one being the
result.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Seeds: 14040076 + configuration index (numpy PCG64 via default_rng).
SEED_BASE = 14040076

ARITH_RULES = """\
# Addition: Sec. 2.2, Eq. (2) and Eq. (1).
Add(y, r) = Z -> r = y;
Add(y, r) = S(x) -> Add(y, w) = x, r = S(w);
# Duplication and erasure of numerals.
Dup(a, b) = Z -> a = Z, b = Z;
Dup(a, b) = S(x) -> Dup(p, q) = x, a = S(p), b = S(q);
Era = Z -> ;
Era = S(x) -> Era = x;
# Multiplication: mul(0, y) = 0 ; mul(S x, y) = add(mul(x, y), y).
Mul(y, r) = Z -> Era = y, r = Z;
Mul(y, r) = S(x) -> Dup(y1, y2) = y, Mul(y1, w) = x, Add(y2, r) = w;
# Ackermann: A(n, r) = m computes r = ack(m, n).
A(n, r) = Z -> r = S(n);
A(n, r) = S(m) -> A2(m, r) = n;
A2(m, r) = Z -> A(S(Z), r) = m;
A2(m, r) = S(n) -> Dup(m1, m2) = m, A(n, w) = S(m2), A(w, r) = m1;
# Predecessor.
Pred(r) = Z -> r = Z;
Pred(r) = S(x) -> r = x;
# Fibonacci: Fib(r) = k computes r = fib(k).
Fib(r) = Z -> r = Z;
Fib(r) = S(x) -> Fib2(r) = x;
Fib2(r) = Z -> r = S(Z);
Fib2(r) = S(x) -> Dup(a, b) = x, Fib(w1) = S(a), Fib(w2) = b, Add(w2, r) = w1;
"""

# Algae L-System, A -> AB and B -> A (the paper's third benchmark, Sec. 5;
# the paper prints no rules, so the encoding is ours).  A symbol agent meets
# the number of iterations still to apply: at zero it becomes a leaf of the
# result; SymA splits into a concatenation of SymA and SymB, each with its
# own copy of the remaining count (duplicated by Dup on every step, the
# drops in parallelism Sec. 5 mentions); SymB becomes SymA.
LSYS_RULES = """\
SymA(r) = Z -> r = LeafA;
SymA(r) = S(k) -> Dup(k1, k2) = k, SymA(x) = k1, SymB(y) = k2, r = Cat(x, y);
SymB(r) = Z -> r = LeafB;
SymB(r) = S(k) -> SymA(r) = k;
Dup(a, b) = Z -> a = Z, b = Z;
Dup(a, b) = S(x) -> Dup(p, q) = x, a = S(p), b = S(q);
"""

LSYS_RULE_NAMES = ["SymA><Z", "SymA><S", "SymB><Z", "SymB><S", "Dup><Z", "Dup><S"]

# Binary trees (Leaf, Node(a, b)) walked by agents that mirror, count the
# leaves of, copy, drop, take the left subtree of, or swap the children of a
# tree: a second rule set, with arity-two constructors, for the kernel
# compiled per rule set (the paper's examples are numerals; these rules are
# ours).  Every rule consumes one constructor, so every net terminates.
TREE_RULES = """\
Mirror(r) = Leaf -> r = Leaf;
Mirror(r) = Node(a, b) -> r = Node(y, x), Mirror(x) = a, Mirror(y) = b;
Leaves(r) = Leaf -> r = S(Z);
Leaves(r) = Node(a, b) -> Leaves(x) = a, Leaves(y) = b, Add(y, r) = x;
Drop = Leaf -> ;
Drop = Node(a, b) -> Drop = a, Drop = b;
Copy(p, q) = Leaf -> p = Leaf, q = Leaf;
Copy(p, q) = Node(a, b) -> Copy(a1, a2) = a, Copy(b1, b2) = b, p = Node(a1, b1), q = Node(a2, b2);
Left(r) = Leaf -> r = Leaf;
Left(r) = Node(a, b) -> r = a, Drop = b;
Swap(r) = Leaf -> r = Leaf;
Swap(r) = Node(a, b) -> r = Node(b, a);
Add(y, r) = Z -> r = y;
Add(y, r) = S(x) -> Add(y, w) = x, r = S(w);
"""


def random_tree(rng, depth: int):
    """A random binary tree of at most `depth` levels: None is a leaf, a
    pair (left, right) a node."""
    if depth == 0 or rng.random() < 0.3:
        return None
    return (random_tree(rng, depth - 1), random_tree(rng, depth - 1))


def tree_text(t) -> str:
    if t is None:
        return "Leaf"
    return f"Node({tree_text(t[0])}, {tree_text(t[1])})"

# Rule names in file order (R1..R18), for per-rule histograms.
ARITH_RULE_NAMES = [
    "Add><Z", "Add><S", "Dup><Z", "Dup><S", "Era><Z", "Era><S",
    "Mul><Z", "Mul><S", "A><Z", "A><S", "A2><Z", "A2><S",
    "Pred><Z", "Pred><S", "Fib><Z", "Fib><S", "Fib2><Z", "Fib2><S",
]


def numeral(k: int) -> str:
    """S^k(Z) as a nested term."""
    if k < 0:
        raise ValueError("numerals are non-negative")
    return "S(" * k + "Z" + ")" * k


def add_net(m: int, n: int) -> str:
    """< r | Add(S^n Z, r) = S^m Z > : r = m + n (principal port on m)."""
    return f"< r | Add({numeral(n)}, r) = {numeral(m)} >"


def mul_net(m: int, n: int) -> str:
    """< r | Mul(S^n Z, r) = S^m Z > : r = m * n."""
    return f"< r | Mul({numeral(n)}, r) = {numeral(m)} >"


def ack_net(a: int, b: int) -> str:
    """< r | A(S^b Z, r) = S^a Z > : r = ack(a, b)."""
    return f"< r | A({numeral(b)}, r) = {numeral(a)} >"


def fib_net(n: int) -> str:
    """< r | Fib(r) = S^n Z > : r = fib(n)."""
    return f"< r | Fib(r) = {numeral(n)} >"


def pred_net(n: int) -> str:
    return f"< r | Pred(r) = {numeral(n)} >"


@dataclass
class Workload:
    """A named batch of nets over one rule set."""
    name: str
    rules: str
    nets: list[str]
    params: list[tuple] = field(default_factory=list)
    family: list[str] = field(default_factory=list)


def config0(seed: int = SEED_BASE + 0, count: int = 4096, hi: int = 256) -> Workload:
    """4096 nets Add(S^m Z, S^n Z), m, n ~ U{0..256} i.i.d."""
    rng = np.random.default_rng(seed)
    mn = rng.integers(0, hi + 1, size=(count, 2))
    params = [(int(m), int(n)) for m, n in mn]
    return Workload("add4096", ARITH_RULES, [add_net(m, n) for m, n in params],
                    params, ["add"] * count)


def config1(seed: int = SEED_BASE + 1, count: int = 2048, hi: int = 64) -> Workload:
    """2048 nets Mul(S^m Z, S^n Z), m, n ~ U{0..64} i.i.d."""
    rng = np.random.default_rng(seed)
    mn = rng.integers(0, hi + 1, size=(count, 2))
    params = [(int(m), int(n)) for m, n in mn]
    return Workload("mul2048", ARITH_RULES, [mul_net(m, n) for m, n in params],
                    params, ["mul"] * count)


def config2(bs=(4, 5, 6, 7, 8)) -> Workload:
    """Single nets A(S^3 Z, S^b Z) for b = 4..8 (no randomness)."""
    params = [(3, b) for b in bs]
    return Workload("ack3", ARITH_RULES, [ack_net(a, b) for a, b in params],
                    params, ["ack"] * len(params))


def config3(ns=(20, 21, 22, 23, 24, 25)) -> Workload:
    """Single nets Fib(S^n Z) for n = 20..25 (no randomness)."""
    params = [(n,) for n in ns]
    return Workload("fib", ARITH_RULES, [fib_net(n) for n in ns],
                    params, ["fib"] * len(params))


def replicated(w: Workload, times: int) -> Workload:
    return Workload(f"{w.name}x{times}", w.rules, w.nets * times, w.params * times,
                    w.family * times)


# ---------------------------------------------------------------------------
# Serving mix.  Request sizes are drawn in interactions; each family's
# parameter is picked so its interaction count is close to the draw.  The
# size model below is only used to size requests, never to check a result.

def _fib_values(n):
    f = [0, 1]
    while len(f) <= n + 1:
        f.append(f[-1] + f[-2])
    return f


def _size_add(m, n):
    return m + 1


def _size_mul(m, n):
    return n + 2 + m * (n + 3) + n * m * (m - 1) // 2


def _ack(m, n):
    if m == 0:
        return n + 1
    if m == 1:
        return n + 2
    if m == 2:
        return 2 * n + 3
    return 2 ** (n + 3) - 3


def _size_ack_table(max_a=3, max_b=12):
    # Interaction counts of A(S^b Z, r) = S^a Z under the rules above, by
    # the recursion of the rules (used only for request sizing).
    memo = {}

    def c(m, n):
        key = (m, n)
        if key in memo:
            return memo[key]
        if m == 0:
            v = 1
        elif n == 0:
            v = 2 + c(m - 1, 1)
        else:
            v = 2 + m + c(m, n - 1) + c(m - 1, _ack(m, n - 1))
        memo[key] = v
        return v

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(100000)
    try:
        out = {}
        for a in range(max_a + 1):
            for b in range(max_b + 1):
                v = c(a, b)
                if v > 2e7:
                    break
                out[(a, b)] = v
        return out
    finally:
        sys.setrecursionlimit(old)


def _size_fib_table(max_n=30):
    f = _fib_values(max_n + 2)
    a = [1, 2]
    for k in range(0, max_n - 1):
        a.append(2 + (k + 1) + a[k + 1] + a[k] + f[k + 1] + 1)
    return {n: a[n] for n in range(max_n + 1)}


_NET_BUILDERS = {"add": add_net, "mul": mul_net, "ack": ack_net, "fib": fib_net}


@dataclass
class Request:
    arrival_s: float
    family: str
    params: tuple
    size: int

    @property
    def net(self) -> str:
        """Net text, built on demand (large requests are tens of MB)."""
        return _NET_BUILDERS[self.family](*self.params)


def config4(seed: int = SEED_BASE + 4, count: int = 100_000, rate_per_s: float = 1000.0,
            median: float = 1e3, sigma: float = 2.16, cap: float = 1e7) -> list[Request]:
    """Serving mix: Poisson arrivals at ``rate_per_s``; each request picks a
    family uniformly from {add, mul, ack, fib} and a target size
    T ~ LogNormal(ln median, sigma) clipped to [1, cap] interactions."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    arrivals = np.cumsum(gaps)
    fams = rng.integers(0, 4, size=count)
    targets = np.clip(rng.lognormal(math.log(median), sigma, size=count), 1, cap)
    ack_tab = sorted(_size_ack_table().items(), key=lambda kv: kv[1])
    fib_tab = sorted(_size_fib_table().items(), key=lambda kv: kv[1])
    mul_tab = sorted((((m, n), _size_mul(m, n)) for m in range(0, 401) for n in range(0, 401)),
                     key=lambda kv: kv[1])
    mul_sizes = np.array([s for _, s in mul_tab])
    out = []
    for i in range(count):
        t = float(targets[i])
        f = int(fams[i])
        if f == 0:
            m = max(0, int(round(t)) - 1)
            n = int(rng.integers(0, 65))
            out.append(Request(float(arrivals[i]), "add", (m, n), _size_add(m, n)))
        elif f == 1:
            j = int(np.clip(np.searchsorted(mul_sizes, t), 0, len(mul_tab) - 1))
            (m, n), s = mul_tab[j]
            out.append(Request(float(arrivals[i]), "mul", (m, n), s))
        elif f == 2:
            (a, b), s = min(ack_tab, key=lambda kv: abs(math.log(kv[1]) - math.log(t)))
            out.append(Request(float(arrivals[i]), "ack", (a, b), s))
        else:
            n, s = min(fib_tab, key=lambda kv: abs(math.log(kv[1]) - math.log(t)))
            out.append(Request(float(arrivals[i]), "fib", (n,), s))
    return out


def lsys_net(n: int) -> str:
    """< r | SymA(r) = S^n Z > : r = the L-System word after n steps from A,
    as a tree of Cat nodes over LeafA / LeafB."""
    return f"< r | SymA(r) = {numeral(n)} >"


def config5(ns=(27,)) -> Workload:
    """The L-System benchmark: single nets of n = 27 steps (514 229 symbols)."""
    return Workload("lsys", LSYS_RULES, [lsys_net(n) for n in ns], [(n,) for n in ns], ["lsys"] * len(ns))


def equation_chains(n_pairs: int, p_more: float = 0.2, n_free: int = 0, n_direct: int = 0,
                    seed: int = SEED_BASE + 6):
    """A set of equations as one linking step leaves it, for the linker
    control: n_pairs pairs of agents, each joined through a chain of
    1 + Geometric(1 - p_more) - 1 names (A = x1, x1 = x2, .., xk = B),
    n_direct agent pairs written directly (A = B), and n_free chains from an
    agent to a name that occurs once (no pair).  Names are numbered at
    random, every equation is oriented at random and the list is shuffled.
    Returns (eq, n_vars, expected): eq a uint64 array of t | u << 32 over
    term words (agent i: 4i + 1, name v: 4v + 2), expected the sorted list
    of (min, max) agent pairs that linking must produce."""
    rng = np.random.default_rng(seed)
    A = lambda i: (i << 2) | 1          # noqa: E731
    V = lambda v: (v << 2) | 2          # noqa: E731
    lens = rng.geometric(1.0 - p_more, size=n_pairs)            # >= 1 names per chain
    flen = rng.geometric(0.5, size=n_free)                      # >= 1 names per free chain
    n_vars = int(lens.sum() + flen.sum())
    perm = rng.permutation(n_vars)
    eqs, expected = [], []
    nv = agent = 0
    for k in lens:
        a, b = agent, agent + 1
        agent += 2
        vs = perm[nv:nv + k]
        nv += int(k)
        eqs.append((A(a), V(int(vs[0]))))
        eqs.extend((V(int(vs[j])), V(int(vs[j + 1]))) for j in range(k - 1))
        eqs.append((V(int(vs[-1])), A(b)))
        expected.append((a, b))
    for _ in range(n_direct):
        eqs.append((A(agent), A(agent + 1)))
        expected.append((agent, agent + 1))
        agent += 2
    for k in flen:
        vs = perm[nv:nv + k]
        nv += int(k)
        eqs.append((A(agent), V(int(vs[0]))))
        eqs.extend((V(int(vs[j])), V(int(vs[j + 1]))) for j in range(k - 1))
        agent += 1
    arr = np.array(eqs, dtype=np.uint64).reshape(-1, 2)
    flip = rng.random(len(arr)) < 0.5
    arr[flip] = arr[flip][:, ::-1]
    arr = arr[rng.permutation(len(arr))]
    eq = np.ascontiguousarray(arr[:, 0] | (arr[:, 1] << np.uint64(32)))
    return eq, n_vars, sorted(expected)


CONFIGS = {0: config0, 1: config1, 2: config2, 3: config3}
