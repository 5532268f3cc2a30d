"""The continuous-batching request loop (paper_1404_0076_gb300/serve.py).

CPU: the admission and freeing logic against a fake evaluator.
GPU: a stream of mixed requests whose results, computed while they overlap
on the device, must equal each request reduced alone (the oracle).
"""
import random
from dataclasses import dataclass

import pytest

import workloads as W
from paper_1404_0076_gb300.serve import Server, default_footprint, summarize


@dataclass
class Req:
    arrival_s: float
    net: str
    size: int


class FakeEvaluator:
    """Completes each net after `size` epochs; reuses freed ids like the
    library; counts resets and the most nets held at once."""

    def __init__(self):
        self.left = {}
        self.value = {}
        self.next_id = 0
        self.free_ids = []
        self.resets = 0
        self.staged = set()
        self.batch = None
        self.reported = set()
        self.held_max = 0

    def load_rules(self, text):
        pass

    def load_net(self, text):
        if self.free_ids:
            i = self.free_ids.pop()
        else:
            i = self.next_id
            self.next_id += 1
        size = int(text.split(":")[1])
        self.left[i] = size
        self.value[i] = size * 10
        self.held_max = max(self.held_max, len(self.left))
        return i

    def load_nets(self, texts):
        return [self.load_net(t) for t in texts]

    def parse(self, texts):
        return list(texts)

    def load_parsed(self, parsed, first, n):
        return [self.load_net(t) for t in parsed[first:first + n]]

    def set_quotas(self, ids, quotas):
        pass

    def status(self, ids):
        return ["OK"] * len(ids)

    def free(self, ids):
        for i in ids:
            assert self.left[i] == 0 and i not in (self.batch or [])
            del self.left[i], self.value[i]
            self.staged.discard(i)
            self.reported.discard(i)
            self.free_ids.append(i)

    def stage(self, ids):
        self.staged.update(ids)

    def reduce(self, ids, mode, slice_us, block, grid, check):
        for i in list(self.staged):
            if self.left[i] > 0:
                self.left[i] -= 1
        return {"status": "OK" if all(v == 0 for v in self.left.values()) else "STEP_LIMIT"}

    def pending(self, ids):
        return [self.left[i] for i in ids]

    def finished(self):
        out = [i for i, v in self.left.items() if v == 0 and i not in self.reported]
        self.reported.update(out)
        return out

    def readback_nats(self, ids):
        return [self.value[i] for i in ids], [self.value[i] // 10 for i in ids]

    def readback_nats_begin(self, ids):
        assert self.batch is None
        assert all(self.left[i] == 0 for i in ids)
        self.batch = list(ids)
        self.polls = 0

    def readback_nats_end(self, wait=False):
        assert self.batch is not None
        self.polls += 1
        if not wait and self.polls < 2:   # done at the second poll
            return None
        r = self.readback_nats(self.batch)
        self.batch = None
        return r

    def reset(self):
        self.resets += 1
        self.left.clear()
        self.value.clear()
        self.staged.clear()
        self.next_id = 0
        self.batch = None
        self.reported.clear()

    def close(self):
        pass


def test_admission_and_freeing_on_cpu():
    fakes = []

    def make():
        f = FakeEvaluator()
        fakes.append(f)
        return f

    srv = Server("", budget_bytes=64 << 20, max_pairs=1 << 10, make_evaluator=make,
                 footprint=lambda text, size: 10_000)
    cap = srv.max_agents // 10_000          # requests the arena admits at once
    assert cap >= 2
    reqs = [Req(0.0, f"net:{1 + (i % 5)}", 1 + (i % 5)) for i in range(4 * cap + 3)]
    done = srv.serve(reqs)
    assert len(done) == len(reqs)
    assert sorted(d.rid for d in done) == list(range(len(reqs)))
    for d in done:
        size = 1 + (d.rid % 5)
        assert d.value == 10 * size and d.interactions == size
        assert d.finished >= d.admitted >= d.arrival >= 0
    # one arena, never reset: finished nets were freed and their ids reused
    assert len(fakes) == 1 and fakes[0].resets == 0
    assert srv.frees >= 2 and srv.freed == len(reqs)
    assert fakes[0].held_max <= cap and fakes[0].next_id <= cap
    assert srv.used == 0 and not fakes[0].left
    s = summarize(done, 1.0)
    assert s["requests"] == len(reqs) and s["p99_ms"] >= s["p50_ms"]


def test_oversized_request_is_refused_on_cpu():
    srv = Server("", budget_bytes=64 << 20, max_pairs=1 << 10, make_evaluator=FakeEvaluator,
                 footprint=lambda text, size: 1 << 40)
    with pytest.raises(ValueError):
        srv.serve([Req(0.0, "net:1", 1)])


def mixed_requests(n, seed=14040076 + 4):
    rng = random.Random(seed)
    out = []
    t = 0.0
    for _ in range(n):
        t += rng.expovariate(20000.0)
        f = rng.randrange(4)
        if f == 0:
            m, k = rng.randrange(0, 300), rng.randrange(0, 50)
            out.append(Req(t, W.add_net(m, k), m + 1))
        elif f == 1:
            m, k = rng.randrange(0, 20), rng.randrange(0, 20)
            out.append(Req(t, W.mul_net(m, k), 2 + m * (k + 3) + k * m * m // 2))
        elif f == 2:
            a, b = rng.choice([(1, 5), (2, 3), (2, 6), (3, 2), (3, 4)])
            out.append(Req(t, W.ack_net(a, b), 25000))
        else:
            k = rng.randrange(0, 16)
            out.append(Req(t, W.fib_net(k), 3000))
    return out


@pytest.mark.gpu
def test_results_in_the_mix_equal_results_alone(oracle):
    reqs = mixed_requests(600)
    # an arena holding about a quarter of the stream's estimated footprint
    # makes requests wait for the memory of finished ones, which is freed
    # while others are in flight
    total = sum(default_footprint(r.net, r.size) for r in reqs)
    max_pairs = 1 << 16
    per_arena = max(total // 4, 4 * max(default_footprint(r.net, r.size) for r in reqs))
    budget = per_arena * 80 // 3 + 24 * max_pairs
    srv = Server(W.ARITH_RULES, budget_bytes=budget, epoch_us=300, max_pairs=max_pairs)
    assert srv.max_agents < total // 2
    try:
        done = srv.serve(reqs)
        use = srv.ev.arena_usage()
    finally:
        srv.close()
    assert srv.frees >= 2 and srv.resets == 0
    # the arena's bump pointer never passed its capacity: freed slots were reused
    assert use["agent_slots"] <= srv.max_agents and use["live_agents"] == 0
    assert len(done) == len(reqs)
    alone = oracle.run(W.ARITH_RULES, [r.net for r in reqs], quiet=True, threads=8)
    for d in sorted(done, key=lambda d: d.rid):
        o = alone[d.rid]
        assert d.status == "OK"
        assert (d.value, d.interactions) == (o["nat"], o["interactions"]), d.rid
    # requests overlapped on the device: some request was admitted while
    # another one was still in flight
    spans = sorted((d.admitted, d.finished) for d in done)
    assert any(b[0] < a[1] for a, b in zip(spans, spans[1:]))


@pytest.mark.gpu
def test_an_underestimated_request_fails_alone(oracle):
    """One request claims a footprint far below what it builds: it stops with
    ARENA_FULL at an epoch boundary (its quota), and every other request in
    the mix completes exactly as alone; the arena is never poisoned."""
    reqs = mixed_requests(300, seed=14040076 + 6)
    bad = len(reqs) // 3
    reqs[bad] = Req(reqs[bad].arrival_s, W.fib_net(19), 3000)   # peaks near 20 000 live agents

    def footprint(text, size):
        return 40 if text == reqs[bad].net else default_footprint(text, size)
    srv = Server(W.ARITH_RULES, budget_bytes=256 << 20, epoch_us=300, max_pairs=1 << 16, footprint=footprint)
    try:
        done = srv.serve(reqs)
    finally:
        srv.close()
    assert sorted(d.rid for d in done) == list(range(len(reqs)))
    assert srv.resets == 0
    alone = oracle.run(W.ARITH_RULES, [r.net for r in reqs], quiet=True, threads=8)
    for d in done:
        if d.rid == bad:
            assert d.status == "ARENA_FULL", d
            continue
        assert d.status == "OK", d
        assert (d.value, d.interactions) == (alone[d.rid]["nat"], alone[d.rid]["interactions"]), d.rid


def test_summary_percentiles_on_cpu():
    from paper_1404_0076_gb300.serve import Finished
    done = [Finished(i, 0.0, 0.001 * i, 0.01 * (i + 1), i, i) for i in range(100)]
    s = summarize(done, 2.0)
    assert s["p50_ms"] == 500.0 and s["p99_ms"] == 990.0
    assert s["admission_wait_p50_ms"] == 49.0
    assert abs(s["service_p50_ms"] - 451.0) < 1e-9
    assert s["interactions_per_s"] == sum(range(100)) / 2.0
    assert summarize([], 1.0)["p50_ms"] is None


def test_requests_shard_over_devices_on_cpu():
    from paper_1404_0076_gb300.serve import MultiServer

    def make(dev):
        return Server("", budget_bytes=64 << 20, max_pairs=1 << 10, make_evaluator=FakeEvaluator,
                      footprint=lambda text, size: 1000)
    ms = MultiServer("", devices=[0, 1, 2], make_server=make)
    reqs = [Req(0.0001 * i, f"net:{1 + (i % 7)}", 1 + (i % 7)) for i in range(300)]
    done = ms.serve(reqs)
    assert sorted(d.rid for d in done) == list(range(300))
    for d in done:
        size = 1 + (d.rid % 7)
        assert d.value == 10 * size and d.interactions == size
    # every device got work (how much depends on how fast each serving
    # thread reports completions), and every request's load was returned
    assert all(n > 0 for n in ms.routed) and sum(ms.routed) == 300
    assert ms.load == [0, 0, 0]
    # the routing itself: an arrival goes to the least loaded device
    ms.load = [50, 7, 20]
    assert ms.route("net:5", 5) == 1 and ms.load == [50, 12, 20]
    assert ms.route("net:9", 9) == 1 and ms.route("net:1", 1) == 2
    ms.close()


@pytest.mark.gpu
def test_two_servers_share_the_stream_and_agree_with_the_oracle(oracle):
    # both on device 0 here (one GPU per box); each has its own contexts and
    # streams, and their kernels never wait on one another
    from paper_1404_0076_gb300.serve import MultiServer
    reqs = mixed_requests(300, seed=14040076 + 5)
    ms = MultiServer(W.ARITH_RULES, devices=[0, 0], budget_bytes=256 << 20, epoch_us=300, max_pairs=1 << 16)
    try:
        done = ms.serve(reqs)
    finally:
        ms.close()
    assert sorted(d.rid for d in done) == list(range(len(reqs)))
    alone = oracle.run(W.ARITH_RULES, [r.net for r in reqs], quiet=True, threads=8)
    for d in done:
        assert d.status == "OK"
        assert (d.value, d.interactions) == (alone[d.rid]["nat"], alone[d.rid]["interactions"]), d.rid
    assert all(n > 0 for n in ms.routed)
