"""CPU-only checks of the boundary: the library loads, exports every symbol
include/inet.h declares, and its host logic (parser, linearity checks, rule
compiler, net flattener, initial ->com) behaves, through host-only contexts
that make no CUDA call."""
import os
import re

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_1404_0076_gb300 import build
    build.build()
    from paper_1404_0076_gb300 import capi as c
    return c


def declared_functions():
    text = open(os.path.join(ROOT, "include", "inet.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(inet_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(capi):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(capi.LIB, n), n
    assert sorted(capi.EXPORTED) == names


def test_owner_tracking_is_a_flag(capi):
    base = capi.inet_arena_cfg(1 << 16, 1 << 16, 1 << 10, 64, 0)
    kept = capi.inet_arena_cfg(1 << 16, 1 << 16, 1 << 10, 64, capi.INET_ARENA_FREE_NETS)
    # 4 bytes per name slot for the owners (256-byte rounding aside)
    assert capi.inet_workspace_bytes(kept) - capi.inet_workspace_bytes(base) >= 4 * (1 << 16)
    with pytest.raises(capi.InetError):
        capi.inet_workspace_bytes(capi.inet_arena_cfg(1 << 16, 1 << 16, 1 << 10, 64, 2))


def test_workspace_size_grows_with_capacity(capi):
    small = capi.inet_workspace_bytes(capi.inet_arena_cfg(1000, 1000, 1000, 10, 0))
    big = capi.inet_workspace_bytes(capi.inet_arena_cfg(10 ** 6, 10 ** 6, 10 ** 5, 1000, 0))
    assert big - small >= 16 * (10 ** 6 - 1000)


def host_ctx(capi):
    return capi.inet_create(-1, None, None)


def test_rule_compiler_shapes(capi):
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    assert capi.inet_rule_count(ctx) == 18
    info = {capi.inet_rule_info(ctx, i)["name"]: capi.inet_rule_info(ctx, i) for i in range(18)}
    # Eq. (1): +(y,r) = S(x) -> +(y,w) = x, r = S(w): two agents, the name w
    # joins two auxiliary ports, two equations to link.
    assert info["Add><S"] == {"name": "Add><S", "arity_alpha": 2, "arity_beta": 1, "n_new": 2,
                              "new_ports": 3, "n_fresh": 1, "n_link": 2}
    # Eq. (2): +(y,r) = Z -> r = y: no agent, one equation.
    assert info["Add><Z"]["n_new"] == 0 and info["Add><Z"]["n_link"] == 1
    # Fib2><S: Dup, Fib, S, Fib, Add; Fib(w1) = S(a) is itself an active pair.
    f = info["Fib2><S"]
    assert (f["n_new"], f["n_fresh"], f["n_link"]) == (5, 2, 2)
    m = info["Mul><S"]
    assert (m["n_new"], m["n_fresh"], m["n_link"]) == (3, 2, 2)
    assert info["Era><Z"]["n_new"] == 0 and info["Era><Z"]["n_link"] == 0
    capi.inet_destroy(ctx)


@pytest.mark.parametrize("text,status", [
    ("Foo(x) = Bar -> ;", "LINEARITY"),
    ("Foo(x) = Bar -> x = y;", "LINEARITY"),
    ("Foo(x, x) = Bar -> x = Bar;", "LINEARITY"),
    ("Foo(x) = Bar -> x = Bar", "PARSE"),
    ("Foo(x) = Foo(y) -> x = y;", "PARSE"),
    ("Foo(x) = Bar -> x = Bar; Foo(y) = Bar -> y = Bar;", "PARSE"),
    ("Foo(a, b, c, d) = Bar -> a = b, c = d;", "PARSE"),
    ("Foo(x) = Bar -> x = Bar(Z);", "PARSE"),
    ("Foo(x) = Bar -> x = $;", "PARSE"),
])
def test_rule_errors(capi, text, status):
    ctx = host_ctx(capi)
    with pytest.raises(capi.InetError) as e:
        capi.inet_load_rules(ctx, text)
    assert e.value.name == status
    capi.inet_destroy(ctx)


@pytest.mark.parametrize("text,status", [
    ("< r | Add(x, r) = S(x), x = Z >", "LINEARITY"),
    ("< r | Foo(r) = Z >", "PARSE"),
    ("< r | Add(r) = Z >", "PARSE"),
    ("< r | Add(y r) = Z >", "PARSE"),
    ("< r | Add(y, r) = Z", "PARSE"),
    ("< r | Add(y, r) = Z > junk", "PARSE"),
    ("< r | S(r >", "PARSE"),
    ("< r | S(r)) = Z >", "PARSE"),
    ("< r | S(Z, Z) = r >", "PARSE"),
    ("< r | S = r >", "PARSE"),
    ("< r | S() = r >", "PARSE"),
    ("< r | r = Z > $", "PARSE"),
    ("< r | r = Z $ >", "PARSE"),
    ("< r | r -> Z >", "PARSE"),
    ("< r | r(x) = Z, x = Z >", "PARSE"),
    ("< r | r = Z, >", "PARSE"),
    ("", "PARSE"),
    ("r = Z", "PARSE"),
    ("< x, x, x | >", "LINEARITY"),
])
def test_net_errors(capi, text, status):
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    with pytest.raises(capi.InetError) as e:
        capi.inet_load_net(ctx, text)
    assert e.value.name == status
    capi.inet_destroy(ctx)


@pytest.mark.parametrize("text,pairs", [
    ("<r|Add(y,r)=S(Z),y=Z>", 1),
    ("< r | # a comment to the end of the line\n  Add(y, r) = S(Z()) , y = Z() >", 1),
    ("< | >", 0),
    ("< r, s | r = s >", 0),
    ("< S(Z), Z | >", 0),
    ("< r | Add(y, r) = x, x = S(Z), y = Z >", 1),
    ("< r | x = S(Z), Add(y, r) = x, y = Z >", 1),
])
def test_net_syntax_accepted(capi, text, pairs):
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    i = capi.inet_load_net(ctx, text)
    assert capi.inet_net_info(ctx, i)["pending_pairs"] == pairs
    capi.inet_destroy(ctx)


def test_initial_com_finds_active_pairs(capi):
    # Sec. 3.6: {A = x, x = y, y = B} must yield exactly one active pair at
    # load time; a chain ending in a name yields none.
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, "Alpha = Beta -> ;\n")
    chain = capi.inet_load_net(ctx, "< | Alpha = x, x = y, y = Beta >")
    rev = capi.inet_load_net(ctx, "< | y = Beta, x = y, Alpha = x >")
    open_ = capi.inet_load_net(ctx, "< y | Alpha = x1, x1 = x2, x2 = y >")
    assert capi.inet_net_info(ctx, chain)["pending_pairs"] == 1
    assert capi.inet_net_info(ctx, rev)["pending_pairs"] == 1
    assert capi.inet_net_info(ctx, open_)["pending_pairs"] == 0
    capi.inet_destroy(ctx)


def test_config_nets_load_with_one_pair_each(capi):
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    for k in (0, 1, 2, 3):
        for net in W.CONFIGS[k]().nets[:50]:
            i = capi.inet_load_net(ctx, net)
            assert capi.inet_net_info(ctx, i)["pending_pairs"] == 1
    capi.inet_destroy(ctx)


def test_deep_numeral_parses_iteratively(capi):
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    i = capi.inet_load_net(ctx, W.add_net(200000, 3))
    assert capi.inet_net_info(ctx, i)["pending_pairs"] == 1
    capi.inet_destroy(ctx)


def test_host_only_context_refuses_device_work(capi):
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    i = capi.inet_load_net(ctx, W.add_net(2, 2))
    with pytest.raises(capi.InetError) as e:
        capi.inet_reduce(ctx, [i])
    assert e.value.name == "NO_DEVICE"
    with pytest.raises(capi.InetError):
        capi.inet_readback(ctx, i)
    capi.inet_destroy(ctx)


def test_rules_cannot_change_with_nets_loaded(capi):
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    capi.inet_load_net(ctx, W.add_net(1, 1))
    with pytest.raises(capi.InetError) as e:
        capi.inet_load_rules(ctx, W.ARITH_RULES)
    assert e.value.name == "STATE"
    capi.inet_reset(ctx)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    capi.inet_destroy(ctx)


def test_batch_load_matches_one_by_one(capi):
    nets = W.config1(count=300).nets + [W.fib_net(7)] + \
        ["< a, b | Dup(a, b) = S(S(Z)) >", "< r | r = Z >"]
    one, many = host_ctx(capi), host_ctx(capi)
    for c in (one, many):
        capi.inet_load_rules(c, W.ARITH_RULES)
    ids1 = [capi.inet_load_net(one, t) for t in nets]
    ids2 = capi.inet_load_nets(many, nets)
    assert ids1 == ids2 == list(range(len(nets)))
    for i in ids1:
        assert capi.inet_net_info(one, i)["pending_pairs"] == capi.inet_net_info(many, i)["pending_pairs"]
    assert capi.inet_load_nets(many, []) == []
    # staged sizes agree: both contexts need the same workspace for the next net
    a = capi.inet_load_net(one, W.add_net(3, 3))
    b = capi.inet_load_nets(many, [W.add_net(3, 3)])[0]
    assert a == b


def test_parsed_batches_load_like_load_nets(capi):
    import threading
    nets = W.config1(count=200).nets + [W.fib_net(7), "< a, b | Dup(a, b) = S(S(Z)) >", "< r | r = Z >"]
    one, two = host_ctx(capi), host_ctx(capi)
    for c in (one, two):
        capi.inet_load_rules(c, W.ARITH_RULES)
    ids1 = capi.inet_load_nets(one, nets)
    # parsed on another thread, loaded in three slices
    box = {}
    th = threading.Thread(target=lambda: box.setdefault("p", capi.inet_parse_nets(two, nets)))
    th.start()
    th.join()
    p = box["p"]
    assert capi.inet_parsed_info(p)[0] == len(nets)
    ids2 = capi.inet_load_parsed(two, p, 0, 50) + capi.inet_load_parsed(two, p, 50, 100) + \
        capi.inet_load_parsed(two, p, 150, len(nets) - 150)
    assert ids1 == ids2
    assert capi.inet_arena_usage(one) == capi.inet_arena_usage(two)
    for i in ids1:
        assert capi.inet_net_info(one, i)["pending_pairs"] == capi.inet_net_info(two, i)["pending_pairs"]
    with pytest.raises(capi.InetError) as e:      # each net of a batch loads once
        capi.inet_load_parsed(two, p, 10, 1)
    assert e.value.name == "INVALID_ARG"
    capi.inet_parsed_free(p)
    # a parse error surfaces when the net is loaded; the nets before it load
    q = capi.inet_parse_nets(one, [W.add_net(1, 1), "< r | Nope(r) = Z >", W.add_net(2, 2)])
    with pytest.raises(capi.InetError) as e:
        capi.inet_load_parsed(one, q, 0, 3)
    assert e.value.name == "PARSE"
    # a batch parsed under another rule set is refused
    capi.inet_reset(one)
    capi.inet_load_rules(one, W.ARITH_RULES)
    with pytest.raises(capi.InetError) as e:
        capi.inet_load_parsed(one, q, 2, 1)
    assert e.value.name == "STATE"
    capi.inet_parsed_free(q)


def test_batch_load_stops_at_the_first_bad_net(capi):
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    nets = [W.add_net(1, 1)] * 100 + ["< r | Nope(r) = Z >"] + [W.add_net(2, 2)] * 100
    with pytest.raises(capi.InetError) as e:
        capi.inet_load_nets(ctx, nets)
    assert e.value.name == "PARSE"
    # the 100 nets before it are loaded; the next id continues after them
    assert capi.inet_load_net(ctx, W.add_net(0, 0)) == 100


def test_argument_errors_are_reported_not_crashed(capi):
    import ctypes as C
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    L = capi.LIB
    ids = (C.c_int32 * 4)()
    n = C.c_int32()
    # offsets that go backwards, and a null output for a non-empty batch
    offs = (C.c_uint64 * 3)(0, 10, 5)
    assert L.inet_load_nets(ctx, b"x" * 10, offs, 2, ids, C.byref(n)) == capi.INET_ERR_INVALID_ARG
    assert L.inet_load_nets(ctx, b"", offs, 2, None, C.byref(n)) == capi.INET_ERR_INVALID_ARG
    assert L.inet_load_nets(ctx, None, None, 0, None, C.byref(n)) == capi.INET_OK and n.value == 0
    # pending and finished on unknown nets / host-only contexts
    bad = (C.c_int32 * 1)(7)
    out = (C.c_uint64 * 1)()
    assert L.inet_net_pending(ctx, bad, 1, out) == capi.INET_ERR_INVALID_ARG
    assert L.inet_net_finished(ctx, ids, 4, C.byref(n)) == capi.INET_ERR_NO_DEVICE
    assert L.inet_net_finished(ctx, ids, -1, C.byref(n)) == capi.INET_ERR_INVALID_ARG
    assert L.inet_readback_nats_begin(ctx, bad, 1) == capi.INET_ERR_NO_DEVICE
    assert L.inet_readback_nats_begin(ctx, bad, 70000) == capi.INET_ERR_INVALID_ARG
    # freeing nets: bad arguments first, then host-only contexts cannot
    assert L.inet_free_nets(ctx, None, 1) == capi.INET_ERR_INVALID_ARG
    assert L.inet_free_nets(ctx, bad, -1) == capi.INET_ERR_INVALID_ARG
    assert L.inet_free_nets(ctx, bad, 70000) == capi.INET_ERR_INVALID_ARG
    assert L.inet_free_nets(None, bad, 1) == capi.INET_ERR_INVALID_ARG
    assert L.inet_free_nets(ctx, bad, 0) == capi.INET_ERR_NO_DEVICE
    assert L.inet_free_net(ctx, 7) == capi.INET_ERR_NO_DEVICE
    assert L.inet_arena_usage(None, None) == capi.INET_ERR_INVALID_ARG
    assert L.inet_arena_usage(ctx, None) == capi.INET_ERR_INVALID_ARG
    assert L.inet_control_link(0, None, 0, 0, 7, None, 0, out, None, None) == capi.INET_ERR_INVALID_ARG
    assert L.inet_bench_exch(0, 0, 0, None) == capi.INET_ERR_INVALID_ARG
    ns = C.c_double()
    assert L.inet_bench_chase(0, 1 << 10, 1 << 10, 0, C.byref(ns)) == capi.INET_ERR_INVALID_ARG  # hops > n - 1
    assert L.inet_bench_chase(0, 1 << 10, 100, 3, C.byref(ns)) == capi.INET_ERR_INVALID_ARG
    assert L.inet_bench_chase(0, 1 << 10, 100, 0, None) == capi.INET_ERR_INVALID_ARG


def test_arena_usage_counts_loaded_nets(capi):
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    zero = {"agent_slots": 0, "name_slots": 0, "free_agent_slots": 0, "free_name_slots": 0, "live_agents": 0,
            "nets": 0, "free_net_ids": 0}
    assert capi.inet_arena_usage(ctx) == zero
    capi.inet_load_net(ctx, W.add_net(3, 2))        # Add, S^3 Z, S^2 Z: 8 agents; the name r
    capi.inet_load_nets(ctx, [W.add_net(0, 0)] * 2)
    assert capi.inet_arena_usage(ctx) == dict(zero, agent_slots=8 + 2 * 3, name_slots=3, live_agents=14, nets=3)


def test_reduce_refuses_bad_modes_and_shapes(capi):
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    i = capi.inet_load_net(ctx, W.add_net(2, 2))
    for mode, block in ((9, 256), (capi.INET_MODE_ASYNC, 512), (capi.INET_MODE_PAPER, 16)):
        st, _ = capi.inet_reduce(ctx, [i], capi.inet_reduce_opts(mode, block, 0, 0, 0, 0, 0, 0), check=False)
        assert st in (capi.INET_ERR_INVALID_ARG, capi.INET_ERR_NO_DEVICE)


def _loaded_pairs(capi, ctx, ids):
    return [capi.inet_net_info(ctx, i)["pending_pairs"] for i in ids]


def test_batch_loads_from_several_threads_at_once(capi):
    # the host pool runs one job at a time; a second caller parses on its
    # own thread, and every context gets the same nets as a lone load
    import threading
    nets = W.config1(count=700).nets
    ref = host_ctx(capi)
    capi.inet_load_rules(ref, W.ARITH_RULES)
    want = _loaded_pairs(capi, ref, capi.inet_load_nets(ref, nets))
    ctxs = [host_ctx(capi) for _ in range(4)]
    out = [None] * len(ctxs)

    def work(k):
        capi.inet_load_rules(ctxs[k], W.ARITH_RULES)
        for _ in range(3):
            capi.inet_reset(ctxs[k])
            ids = capi.inet_load_nets(ctxs[k], nets)
        out[k] = _loaded_pairs(capi, ctxs[k], ids)

    th = [threading.Thread(target=work, args=(k,)) for k in range(len(ctxs))]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=120)
    assert all(o == want for o in out)
    for c in ctxs + [ref]:
        capi.inet_destroy(c)


@pytest.mark.filterwarnings("ignore::DeprecationWarning")  # forking a threaded process is the point
def test_batch_load_in_a_forked_child(capi):
    # a process forked after the pool started has no pool threads: the
    # child must load on its own thread instead of waiting for them
    import time
    nets = W.config1(count=300).nets
    ctx = host_ctx(capi)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    capi.inet_load_nets(ctx, nets)  # the pool is running now
    pid = os.fork()
    if pid == 0:
        code = 1
        try:
            c2 = host_ctx(capi)
            capi.inet_load_rules(c2, W.ARITH_RULES)
            ids = capi.inet_load_nets(c2, nets)
            code = 0 if len(ids) == len(nets) else 2
        finally:
            os._exit(code)
    deadline = time.time() + 60
    status = None
    while time.time() < deadline:
        done, st = os.waitpid(pid, os.WNOHANG)
        if done:
            status = st
            break
        time.sleep(0.05)
    if status is None:
        os.kill(pid, 9)
        os.waitpid(pid, 0)
    capi.inet_destroy(ctx)
    assert status is not None, "the forked child did not finish its load"
    assert os.WIFEXITED(status) and os.WEXITSTATUS(status) == 0
