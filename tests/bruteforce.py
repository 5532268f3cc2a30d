"""Brute force over every reduction order of tiny nets (test infrastructure).

A second, independent and deliberately naive implementation of the
lightweight calculus (Sec. 2.2) in pure Python, used to pin the C++ oracle:
from a configuration it tries every ->int step on every active equation,
applies ->com until it no longer applies, and recurses, memoising states up to
renaming (a canonical walk of the port graph from the interface).  At the end
it applies ->col and ->sub literally, by search and replace.  Uniform
confluence (Sec. 2.1) predicts one terminal state and equal path lengths from
every state; the tests check both, and that the terminal state equals the
oracle's.
"""
from __future__ import annotations

import sys
from collections import defaultdict

# Terms: ("n", name) | ("a", symbol, (args...))


class Parser:
    def __init__(self, text: str):
        lines = [ln.split("#", 1)[0] for ln in text.splitlines()]
        self.s = "\n".join(lines)
        self.i = 0

    def ws(self):
        while self.i < len(self.s) and self.s[self.i].isspace():
            self.i += 1

    def eat(self, tok: str) -> bool:
        self.ws()
        if self.s.startswith(tok, self.i):
            self.i += len(tok)
            return True
        return False

    def need(self, tok: str):
        if not self.eat(tok):
            raise ValueError(f"expected {tok!r} at {self.i}: {self.s[self.i:self.i + 20]!r}")

    def ident(self) -> str:
        self.ws()
        j = self.i
        while j < len(self.s) and (self.s[j].isalnum() or self.s[j] in "_'"):
            j += 1
        if j == self.i:
            raise ValueError(f"identifier expected at {self.i}")
        tok = self.s[self.i:j]
        self.i = j
        return tok

    def term(self):
        name = self.ident()
        if name[0].islower():
            return ("n", name)
        args = []
        if self.eat("("):
            if not self.eat(")"):
                while True:
                    args.append(self.term())
                    if self.eat(")"):
                        break
                    self.need(",")
        return ("a", name, tuple(args))

    def done(self) -> bool:
        self.ws()
        return self.i >= len(self.s)


def parse_rules(text: str):
    p = Parser(text)
    rules = {}
    order = []
    while not p.done():
        lhs_a = p.term()
        p.need("=")
        lhs_b = p.term()
        p.need("->")
        rhs = []
        if not p.eat(";"):
            while True:
                t = p.term()
                p.need("=")
                u = p.term()
                rhs.append((t, u))
                if p.eat(";"):
                    break
                p.need(",")
        idx = len(order)
        order.append((lhs_a[1], lhs_b[1]))
        rules[(lhs_a[1], lhs_b[1])] = (idx, lhs_a, lhs_b, rhs, False)
        rules[(lhs_b[1], lhs_a[1])] = (idx, lhs_b, lhs_a, rhs, True)
    return rules, order


def parse_net(text: str):
    p = Parser(text)
    p.need("<")
    iface = []
    if not p.eat("|"):
        while True:
            iface.append(p.term())
            if p.eat("|"):
                break
            p.need(",")
    eqs = []
    if not p.eat(">"):
        while True:
            t = p.term()
            p.need("=")
            u = p.term()
            eqs.append((t, u))
            if p.eat(">"):
                break
            p.need(",")
    return iface, eqs


def is_name(t):
    return t[0] == "n"


def names_in(t, acc):
    if is_name(t):
        acc.append(t[1])
    else:
        for a in t[2]:
            names_in(a, acc)
    return acc


def replace(t, x, s):
    if is_name(t):
        return s if t[1] == x else t
    return ("a", t[1], tuple(replace(a, x, s) for a in t[2]))


class Fresh:
    def __init__(self):
        self.n = 0

    def __call__(self):
        self.n += 1
        return f"_f{self.n}"


def interact(eqs, i, rules, fresh):
    """->int on equation i (Sec. 2.2): Theta with bound names fresh and the
    LHS names replaced by the actual arguments."""
    t, u = eqs[i]
    key = (t[1], u[1])
    if key not in rules:
        raise KeyError(f"no rule for {key}")
    idx, la, lb, rhs, _flip = rules[key]
    sub = {}
    for x, arg in zip(la[2], t[2]):
        sub[x[1]] = arg
    for y, arg in zip(lb[2], u[2]):
        sub[y[1]] = arg

    def inst(r):
        if is_name(r):
            if r[1] not in sub:
                sub[r[1]] = ("n", fresh())
            return sub[r[1]]
        return ("a", r[1], tuple(inst(a) for a in r[2]))

    new = [(inst(a), inst(b)) for a, b in rhs]
    return eqs[:i] + eqs[i + 1:] + new, idx


def com_fixpoint(eqs):
    """->com until it no longer applies: x = t, x = u  becomes  t = u."""
    eqs = list(eqs)
    while True:
        top = defaultdict(list)
        for k, (t, u) in enumerate(eqs):
            if is_name(t):
                top[t[1]].append(k)
            if is_name(u):
                top[u[1]].append(k)
        hit = None
        for x, ks in top.items():
            if len(ks) == 2 and ks[0] != ks[1]:
                hit = (x, ks[0], ks[1])
                break
        if hit is None:
            return eqs
        x, k1, k2 = hit
        t1, u1 = eqs[k1]
        t2, u2 = eqs[k2]
        a = u1 if (is_name(t1) and t1[1] == x) else t1
        b = u2 if (is_name(t2) and t2[1] == x) else t2
        eqs = [e for k, e in enumerate(eqs) if k not in (k1, k2)] + [(a, b)]


def sub_col(iface, eqs):
    """->col and ->sub (Sec. 2.2) by literal search until neither applies."""
    iface = list(iface)
    eqs = list(eqs)
    changed = True
    while changed:
        changed = False
        for k, (t, u) in enumerate(eqs):
            for x, s in ((t, u), (u, t)):
                if not is_name(x):
                    continue
                name = x[1]
                if name in names_in(s, []):
                    continue
                if any(name in names_in(it, []) for it in iface):          # col
                    iface = [replace(it, name, s) for it in iface]
                    eqs.pop(k)
                    changed = True
                    break
                for j, (a, b) in enumerate(eqs):                          # sub
                    if j == k:
                        continue
                    if not is_name(a) and name in names_in(a, []):
                        eqs[j] = (replace(a, name, s), b)
                    elif not is_name(b) and name in names_in(b, []):
                        eqs[j] = (a, replace(b, name, s))
                    else:
                        continue
                    eqs.pop(k)
                    changed = True
                    break
                if changed:
                    break
            if changed:
                break
    return iface, eqs


def render(iface) -> str:
    canon = {}

    def r(t):
        if is_name(t):
            if t[1] not in canon:
                canon[t[1]] = len(canon)
            return f"x{canon[t[1]]}"
        if not t[2]:
            return t[1]
        return t[1] + "(" + ", ".join(r(a) for a in t[2]) + ")"

    return ", ".join(r(t) for t in iface)


def canon_key(iface, eqs) -> str:
    """Canonical form of the port graph up to renaming of names."""
    adj = {}
    occ = defaultdict(list)
    syms = []
    counter = [0]

    def link(a, b):
        adj[a] = b
        adj[b] = a

    def root(t):
        if is_name(t):
            counter[0] += 1
            e = ("N", counter[0])
            occ[t[1]].append(e)
            return e
        aid = len(syms)
        syms.append((t[1], len(t[2])))
        for j, a in enumerate(t[2]):
            link(("P", aid, j + 1), root(a))
        return ("P", aid, 0)

    for i, t in enumerate(iface):
        link(("I", i), root(t))
    for t, u in eqs:
        link(root(t), root(u))
    through = {}
    for x, es in occ.items():
        if len(es) == 2:
            through[es[0]] = es[1]
            through[es[1]] = es[0]

    def resolve(p):
        q = adj[p]
        steps = 0
        while q[0] == "N":
            if q not in through:
                return ("FREE",)
            q = adj[through[q]]
            steps += 1
            if steps > 10 * len(adj) + 10:
                return ("LOOP",)
        return q

    order = {}
    queue = []

    def describe(q):
        if q[0] == "P":
            if q[1] not in order:
                order[q[1]] = len(order)
                queue.append(q[1])
            return f"{order[q[1]]}.{q[2]}"
        if q[0] == "I":
            return f"I{q[1]}"
        return q[0]

    out = [describe(resolve(("I", i))) for i in range(len(iface))]
    k = 0
    while k < len(queue):
        a = queue[k]
        k += 1
        sym, ar = syms[a]
        out.append(sym + "[" + ",".join(describe(resolve(("P", a, p))) for p in range(ar + 1)) + "]")
    unreached = len(syms) - len(order)
    return "|".join(out) + f"#{unreached}"


def agents_in(t) -> int:
    return 0 if is_name(t) else 1 + sum(agents_in(a) for a in t[2])


def explore(rules_text: str, net_text: str, limit_states: int = 200000):
    """All reduction orders from the net.  Returns a dict: states, min / max
    path length (->int steps), finals (the set of rendered normal forms),
    consistent (every state's paths have one length), and peak_min /
    peak_max: over all paths, the least and the greatest largest number of
    live agents (agents anywhere in the interface and the equations) that a
    path passes through."""
    rules, _ = parse_rules(rules_text)
    iface, eqs = parse_net(net_text)
    fresh = Fresh()
    memo = {}
    consistent = [True]
    sys.setrecursionlimit(max(10000, sys.getrecursionlimit()))

    iface_agents = sum(agents_in(t) for t in iface)

    def go(eqs):
        key = canon_key(iface, eqs)
        if key in memo:
            return memo[key]
        if len(memo) > limit_states:
            raise RuntimeError("state space too large")
        live = iface_agents + sum(agents_in(t) + agents_in(u) for t, u in eqs)
        active = [k for k, (t, u) in enumerate(eqs) if not is_name(t) and not is_name(u)]
        if not active:
            fi, fe = sub_col(iface, eqs)
            res = (0, 0, frozenset([(render(fi), len(fe))]), live, live)
        else:
            lo, hi, fin, plo, phi = None, None, set(), None, None
            for k in active:
                new, _ = interact(eqs, k, rules, fresh)
                a, b, f, pa, pb = go(com_fixpoint(new))
                lo = a + 1 if lo is None else min(lo, a + 1)
                hi = b + 1 if hi is None else max(hi, b + 1)
                plo = pa if plo is None else min(plo, pa)
                phi = pb if phi is None else max(phi, pb)
                fin |= f
            if lo != hi:
                consistent[0] = False
            res = (lo, hi, frozenset(fin), max(live, plo), max(live, phi))
        memo[key] = res
        return res

    lo, hi, fin, plo, phi = go(com_fixpoint(eqs))
    return {"states": len(memo), "min": lo, "max": hi, "finals": fin, "consistent": consistent[0],
            "peak_min": plo, "peak_max": phi}
