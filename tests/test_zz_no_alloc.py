"""The entry point that allocates nothing, inet_reduce_into.

It is for callers that may not allocate while serving a request (their
allocator already owns the GPU, or a device allocation would break a latency
budget): the caller passes its own device arena, and the library's scratch is
a fixed array in device memory.  The test owns the arena (allocated here, by
the caller) and checks, on two calls in a row, that every net gives the
numeral and interaction count the oracle computes for it alone, and the same
as the ordinary entry point, inet_reduce.  One net (Fibonacci(14)) has a
frontier wider than one block of the persistent kernel.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import pytest

import workloads as W
from tests import oracle_runner

pytestmark = pytest.mark.gpu

R = W.ARITH_RULES
NETS = [W.fib_net(12), W.mul_net(6, 7), W.ack_net(2, 3), W.add_net(40, 9), W.fib_net(1), W.fib_net(14)]


def arena_bytes(max_agents, max_vars):
    return (16 * max_agents + 255) // 256 * 256 + 4 * max_vars


def test_reduce_into_matches_the_oracle_and_inet_reduce_on_two_calls():
    import torch

    from paper_1404_0076_gb300 import Evaluator, capi
    oracle_runner.build()
    alone = [(o["nat"], o["interactions"]) for o in oracle_runner.run(R, NETS)]
    assert all(v is not None for v, _ in alone)
    with Evaluator(device=0) as ev:
        ev.load_rules(R)
        ids = ev.load_nets(NETS)
        st = ev.reduce(ids, mode="persistent", trace=True)
        expect = [ev.readback_nat(i) for i in ids]
        fronts, _ = ev.trace()
    assert expect == alone
    assert max(fronts) > 256           # some step spans more than one block of 256 threads

    host = capi.inet_create(-1)
    try:
        capi.inet_load_rules(host, R)
        hids = [capi.inet_load_net(host, n) for n in NETS]
        max_agents = max_vars = 1 << 17
        nbytes = arena_bytes(max_agents, max_vars)
        arena = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda:0")  # the caller's memory
        ptr = arena.data_ptr() + (-arena.data_ptr()) % 256
        stream = torch.cuda.current_stream(0).cuda_stream
        for _call in range(2):
            got = [capi.inet_reduce_into(host, i, ptr, nbytes, max_agents, max_vars, 0, stream) for i in hids]
            assert got == alone
        # sizes beyond the fixed scratch are refused before any device work
        with pytest.raises(capi.InetError) as e:
            big = 1 << 21
            capi.inet_reduce_into(host, hids[0], ptr, arena_bytes(big, big), big, big, 0, stream)
        assert e.value.name == "INVALID_ARG"
        with pytest.raises(capi.InetError):
            capi.inet_reduce_into(host, hids[0], ptr, nbytes // 2, max_agents, max_vars, 0, stream)
        torch.cuda.synchronize()
    finally:
        capi.inet_destroy(host)
