"""The rule-specialised asynchronous kernel (include/inet.h, inet_jit_*).

CPU: the library generates the kernel's source for a rule set and NVRTC
compiles it with no GPU (host-only context); the cubin cache on disk is
found again by a new process.  GPU: with the specialised kernel on, every
result equals the oracle's and the general kernel's (values, interactions
per net and per rule), in both kernel instantiations (with and without
owner tracking), on rule sets whose warps are uniform (Add chains) and mixed
(Ackermann, Fibonacci, the L-System)."""
import os
import subprocess
import sys

import pytest

import workloads as W
from tests import oracle_runner

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_1404_0076_gb300 import build
    build.build()
    from paper_1404_0076_gb300 import capi as c
    return c


def test_jit_args(capi):
    ctx = capi.inet_create(-1)
    assert capi.LIB.inet_set_jit(ctx, 2) == capi.INET_ERR_INVALID_ARG
    with pytest.raises(capi.InetError) as e:
        capi.inet_jit_build(ctx)
    assert e.value.name == "STATE"           # no rules loaded
    assert capi.LIB.inet_jit_build(ctx, 2) == capi.INET_ERR_INVALID_ARG
    info = capi.inet_jit_info(ctx)
    assert info["state"] == 0 and info["launches"] == 0
    capi.inet_set_jit(ctx, False)
    assert capi.inet_jit_info(ctx)["enabled"] == 0
    capi.inet_destroy(ctx)


def test_jit_compiles_without_a_gpu(capi, tmp_path, monkeypatch):
    # NVRTC needs no device: the generated source of both instantiations
    # compiles, and a second process finds the cubins on disk
    monkeypatch.setenv("INET_JIT_CACHE", str(tmp_path))
    ctx = capi.inet_create(-1)
    capi.inet_load_rules(ctx, W.ARITH_RULES)
    for track in (False, True):
        capi.inet_jit_build(ctx, track)
        info = capi.inet_jit_info(ctx)
        assert info["source"] == 1 and info["compile_ms"] > 0, info
    capi.inet_jit_build(ctx, False)
    assert capi.inet_jit_info(ctx)["source"] == 3      # kept by this process
    capi.inet_load_rules(ctx, W.LSYS_RULES)
    capi.inet_jit_build(ctx, False)
    capi.inet_destroy(ctx)
    assert len(list(tmp_path.glob("k_async_sm_103a_*.cubin"))) == 3
    code = ("from paper_1404_0076_gb300 import capi as C; import workloads as W; "
            "ctx = C.inet_create(-1); C.inet_load_rules(ctx, W.ARITH_RULES); C.inet_jit_build(ctx, True); "
            "print(C.inet_jit_info(ctx)['source'])")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120,
                         env=dict(os.environ, INET_JIT_CACHE=str(tmp_path)))
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "2"                  # from the disk cache


def test_jit_off_by_environment(capi, monkeypatch):
    monkeypatch.setenv("INET_JIT", "0")
    ctx = capi.inet_create(-1)
    assert capi.inet_jit_info(ctx)["enabled"] == 0
    capi.inet_destroy(ctx)


# ---- GPU ---------------------------------------------------------------------


@pytest.fixture(scope="module")
def orc():
    oracle_runner.build()
    return oracle_runner


def make_ev(**kw):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_1404_0076_gb300 import Evaluator
    return Evaluator(device=0, **kw)


def run_async(nets, rules, jit, free_nets=False, mode="async", **caps):
    ev = make_ev(jit=jit, free_nets=free_nets, **caps)
    ev.load_rules(rules)
    ids = ev.load_nets(nets)
    st = ev.reduce(ids, mode=mode)
    if rules == W.ARITH_RULES:
        vals, inter = ev.readback_nats(ids)
        out = list(zip(vals, inter))
    else:
        out = [(ev.readback(i), ev.net_info(i)["interactions"]) for i in ids]
    info = ev.jit_info()
    ev.close()
    return out, list(st["per_rule"]), info


@pytest.mark.gpu
@pytest.mark.parametrize("free_nets", [False, True])
def test_jit_equals_general_kernel_and_oracle(orc, free_nets):
    # uniform warps (Add chains of the Mul batch) and mixed ones (Ackermann,
    # Fibonacci) in one batch; the oracle gives values and interactions
    nets = W.config1(count=256).nets + W.config2(bs=(4, 5)).nets + W.config3(ns=(14, 16)).nets
    caps = dict(max_agents=1 << 23, max_vars=1 << 23, max_pairs=1 << 20, max_nets=512)
    got, hist, info = run_async(nets, W.ARITH_RULES, True, free_nets, **caps)
    assert info["state"] == 1 and info["launches"] >= 1, info
    ref, hist0, info0 = run_async(nets, W.ARITH_RULES, False, free_nets, **caps)
    assert info0["launches"] == 0
    assert got == ref and hist == hist0
    exp = orc.run(W.ARITH_RULES, nets, timeout=600)
    for (v, n), o in zip(got, exp):
        assert o["status"] == "ok"
        assert (v, n) == (o["nat"], o["interactions"]), o


@pytest.mark.gpu
def test_jit_lsystem_text(orc):
    nets = [W.lsys_net(k) for k in (5, 12, 18)]
    got, hist, info = run_async(nets, W.LSYS_RULES, True, max_agents=1 << 21, max_vars=1 << 21,
                                max_pairs=1 << 19, max_nets=16)
    assert info["state"] == 1
    exp = orc.run(W.LSYS_RULES, nets)
    for (text, n), o in zip(got, exp):
        assert (text, n) == (o["result"], o["interactions"])


@pytest.mark.gpu
def test_jit_chain_and_slices():
    # a lone chain (one lane, one rule) resumed across time slices
    ev = make_ev(jit=True, max_agents=1 << 20, max_vars=1 << 20, max_pairs=1 << 16, max_nets=16)
    ev.load_rules(W.ARITH_RULES)
    i = ev.load_net(W.add_net(20000, 7))
    st = ev.reduce([i], mode="async", slice_us=200, check=False)
    slices = 1
    while st["status"] == "STEP_LIMIT" and slices < 10000:
        st = ev.reduce([], mode="async", slice_us=200, check=False)
        slices += 1
    assert st["status"] == "OK" and slices > 1
    assert ev.readback_nat(i) == (20007, 20001)
    assert ev.jit_info()["launches"] >= 1
    ev.close()


def test_jit_without_nvrtc_reports_why(tmp_path):
    # a process whose NVRTC cannot be opened: the build fails with the
    # reason, nothing is cached, and nothing else changes
    code = ("from paper_1404_0076_gb300 import capi as C; import workloads as W; "
            "ctx = C.inet_create(-1); C.inet_load_rules(ctx, W.ARITH_RULES)\n"
            "try:\n    C.inet_jit_build(ctx, False)\nexcept C.InetError as e:\n    print(e.name, str(e))\n")
    env = dict(os.environ, INET_NVRTC_LIB=str(tmp_path / "missing.so"), INET_JIT_CACHE=str(tmp_path))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120, env=env)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("CUDA") and "NVRTC" in out.stdout
    assert not list(tmp_path.glob("*.cubin"))


@pytest.mark.gpu
def test_jit_missing_nvrtc_falls_back_to_the_general_kernel(tmp_path):
    # the specialised kernel cannot be built: asynchronous reduces run on
    # the general kernel with the same results, and the context says why
    code = ("import torch, workloads as W\n"
            "from paper_1404_0076_gb300 import Evaluator\n"
            "ev = Evaluator(device=0, max_agents=1 << 20, max_vars=1 << 20, max_pairs=1 << 16, max_nets=64)\n"
            "ev.load_rules(W.ARITH_RULES)\n"
            "ids = ev.load_nets([W.mul_net(7, 9), W.add_net(300, 4)])\n"
            "ev.reduce(ids, mode='async')\n"
            "print(ev.readback_nats(ids)[0], ev.jit_info()['state'], ev.jit_info()['launches'], ev.jit_info()['msg'])\n")
    env = dict(os.environ, INET_NVRTC_LIB=str(tmp_path / "missing.so"), INET_JIT_CACHE=str(tmp_path))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("[63, 304] -1 0 NVRTC"), out.stdout


def tree_nets(seed: int, count: int, depth: int) -> list[str]:
    from tests.test_oracle import tree_cases
    nets = []
    for t in tree_cases(seed=seed, count=count, depth=depth):
        tt = W.tree_text(t)
        nets += [f"< r | Mirror(r) = {tt} >", f"< r | Leaves(r) = {tt} >", f"< p, q | Copy(p, q) = {tt} >",
                 f"< | Drop = {tt} >", f"< r | Left(r) = {tt} >", f"< r | Swap(r) = {tt} >",
                 f"< r | Leaves(r) = x, Copy(x, y) = {tt}, Drop = y >",
                 f"< r | Swap(r) = x, Mirror(x) = y, Mirror(y) = {tt} >"]
    return nets


@pytest.mark.gpu
@pytest.mark.parametrize("free_nets", [False, True])
def test_jit_tree_rules_equal_the_oracle(orc, free_nets):
    # a rule set with arity-two constructors: its rules of at most two new
    # agents get their own code, the others (Mirror, Leaves, Copy of a node)
    # run the general code in the same kernel
    nets = tree_nets(seed=7, count=48, depth=9)
    exp = orc.run(W.TREE_RULES, nets)
    caps = dict(max_agents=1 << 22, max_vars=1 << 22, max_pairs=1 << 19, max_nets=512)
    for jit, mode in ((True, "async"), (False, "async"), (False, "persistent")):
        got, hist, info = run_async(nets, W.TREE_RULES, jit, free_nets, mode=mode, **caps)
        assert info["state"] == (1 if jit else 0), info
        for net, (text, n), o in zip(nets, got, exp):
            assert o["status"] == "ok"
            assert (text, n) == (o["result"], o["interactions"]), (mode, net)


@pytest.mark.gpu
def test_jit_damaged_cache_file_is_rebuilt(tmp_path):
    # a cached cubin that no longer loads is compiled again and replaced
    code = ("import workloads as W\n"
            "from paper_1404_0076_gb300 import Evaluator\n"
            "ev = Evaluator(device=0, max_agents=1 << 20, max_vars=1 << 20, max_pairs=1 << 16, max_nets=64)\n"
            "ev.load_rules(W.ARITH_RULES)\n"
            "ids = ev.load_nets([W.mul_net(5, 6)])\n"
            "ev.reduce(ids, mode='async')\n"
            "print(ev.readback_nats(ids)[0][0], ev.jit_info()['state'], ev.jit_info()['source'], "
            "repr(ev.jit_info()['msg']))\n")
    env = dict(os.environ, INET_JIT_CACHE=str(tmp_path))
    run = lambda: subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                                 timeout=300, env=env)
    out = run()
    assert out.returncode == 0 and out.stdout.split() == ["30", "1", "1", "''"], (out.stdout, out.stderr)
    files = list(tmp_path.glob("*.cubin"))
    assert len(files) == 1
    head = files[0].read_bytes().split(b"\n", 1)[0]
    files[0].write_bytes(head + b"\n" + b"not a cubin" * 16)
    out = run()
    assert out.returncode == 0 and out.stdout.split() == ["30", "1", "1", "''"], (out.stdout, out.stderr)
    assert files[0].read_bytes()[len(head) + 1:] != b"not a cubin" * 16


def ring_rules(k: int = 32) -> str:
    """2k rules (64 for k = 32, the most a rule set may hold): C_i passes a
    numeral on as C_(i+1 mod k), one S at a time."""
    out = []
    for i in range(k):
        out.append(f"C{i}(r) = Z -> r = Z;")
        out.append(f"C{i}(r) = S(x) -> C{(i + 1) % k}(w) = x, r = S(w);")
    return "\n".join(out) + "\n"


def test_jit_builds_the_largest_rule_set(capi, tmp_path, monkeypatch):
    # 64 rules: the first 32 with two new agents or fewer get their own code
    # (about half a minute of NVRTC)
    monkeypatch.setenv("INET_JIT_CACHE", str(tmp_path))
    ctx = capi.inet_create(-1)
    capi.inet_load_rules(ctx, ring_rules())
    assert capi.inet_rule_count(ctx) == 64
    capi.inet_jit_build(ctx, False)
    assert capi.inet_jit_info(ctx)["source"] == 1
    capi.inet_destroy(ctx)


@pytest.mark.gpu
def test_jit_largest_rule_set_equals_the_oracle(orc):
    # chains that pass through all 64 rules, half of them with their own
    # code and half on the general code, in one kernel
    rules = ring_rules()
    nets = [f"< r | C{i}(r) = {W.numeral(n)} >" for i in range(32) for n in (0, 1, 7, 40, 129)]
    exp = orc.run(rules, nets)
    got, hist, info = run_async(nets, rules, True, max_agents=1 << 20, max_vars=1 << 20, max_pairs=1 << 16,
                                max_nets=256)
    assert info["state"] == 1
    for net, (text, n), o in zip(nets, got, exp):
        assert (text, n) == (o["result"], o["interactions"]), net
    assert sum(hist) == sum(o["interactions"] for o in exp)
