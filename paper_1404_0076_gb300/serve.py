"""Continuous-batching request loop over the evaluator's C ABI.

Requests (one net each) are admitted as they arrive, while the arena has
room for them by an estimate of their footprint; every admitted net joins
the frontier of the nets already in flight (inet_stage), and the device runs
the asynchronous loop in bounded epochs (slice_us), between which finished
nets are found (inet_net_finished, a device scan that reports each net once)
and new ones admitted.  The results of finished nets are read back on a
second stream (inet_readback_nats_begin / _end) while the device keeps
reducing the others, so a long readback walk never stalls the loop.
Requests therefore overlap on the device with whatever is in flight; each
result is independent of the mix because nets share no agent and
interactions are local (Sec. 2.1).

Memory: one arena.  A request's net is freed once its result has been read
back (inet_free_nets returns its agent and name slots and its id), and later
requests are placed into the freed slots, so a long request holds only its
own memory.  Frees are batched (one scan of the arena frees many nets): when
the nets waiting to be freed hold a sixteenth of the arena, when net ids run
short, or when a request does not fit.  Each admitted net gets its footprint
estimate as its quota (inet_set_quotas): a request that outgrows its
estimate stops alone with ARENA_FULL at the next epoch boundary, and the
others, whose estimates admission reserved, are untouched.
"""
from __future__ import annotations

import collections
import itertools
import math
import time
from dataclasses import dataclass


@dataclass
class Finished:
    rid: int
    arrival: float      # seconds, on the server clock
    admitted: float
    finished: float
    value: int | None   # numeral result, None if the interface is not S^k(Z)
    interactions: int
    status: str = "OK"
    detected: float = 0.0  # when the device scan reported the net finished (before its readback)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def default_footprint(text: str, size: int) -> int:
    """Estimated peak agent slots of a request, without scanning its text:
    every agent symbol takes at least two characters of the text ("S(",
    "Z,"), so len(text) is at least twice the net's agents; plus a share
    per expected interaction (numerals built by the net stay alive)."""
    return len(text) + size + 64


class Server:
    def __init__(self, rules: str, device: int = 0, budget_bytes: int = 2 << 30, epoch_us: int = 1000,
                 max_nets: int = 1 << 15, max_pairs: int = 1 << 22, block: int = 0, grid: int = 0,
                 footprint=default_footprint, make_evaluator=None, quotas: bool = True):
        # per agent slot: 16-byte record + 4-byte ring entry; per name slot:
        # 4 (slot) + 4 (ring entry) + 4 (owner); per pair: 2 x 8 frontier + 8 sequence
        rest = max(budget_bytes - 24 * max_pairs, 1 << 20)
        self.max_agents = int(min(rest * 3 // 4 // 20, (1 << 30) - 1))
        self.max_vars = int(min(rest // 4 // 12, (1 << 30) - 1))
        if make_evaluator is None:
            from . import Evaluator

            def make_evaluator():
                return Evaluator(device, max_agents=self.max_agents, max_vars=self.max_vars,
                                 max_pairs=max_pairs, max_nets=max_nets, free_nets=True)
        self.ev = make_evaluator()
        self.ev.load_rules(rules)
        # the asynchronous kernel for these rules is compiled now, not in the
        # first epoch a request waits for (without NVRTC the general kernel
        # serves, and the build's error says why)
        if hasattr(self.ev, "build_jit"):
            from .capi import InetError
            try:
                self.ev.build_jit()
            except InetError:
                pass
        self.max_nets = max_nets
        self.epoch_us = epoch_us
        self.block, self.grid = block, grid
        self.footprint = footprint
        self.quotas = quotas        # each net may hold at most its footprint estimate
        self.used = 0               # estimated agent slots of admitted nets not freed yet
        self.inflight = {}          # net id -> (rid, arrival, admitted, need)
        self.unstaged = []          # admitted nets not yet handed to the device
        self.running = 0            # admitted nets not finished yet
        self.ready = []             # finished, readback not yet begun
        self.detected = {}          # net id -> when the device scan reported it finished
        self.rb_batch = None        # nets of the readback in flight
        self.to_free = []           # read back, waiting to be freed
        self.free_need = 0          # their estimated slots
        self.epochs = 0
        self.frees = 0              # inet_free_nets calls
        self.freed = 0              # nets freed
        self.resets = 0             # fatal errors (the arena is reset)
        self.performed = 0          # interactions the device performed (all epochs)
        self.host_s = collections.Counter()   # wall time by phase: load, stage, reduce, finished, harvest, free

    def close(self):
        self.ev.close()

    # -- admission -------------------------------------------------------
    def _room(self, need: int) -> bool:
        return self.used + need <= self.max_agents and len(self.inflight) + len(self.to_free) < self.max_nets

    def _free(self):
        """Frees every net read back so far (one scan of the arena per call)."""
        t0 = time.perf_counter()
        while self.to_free:
            batch, self.to_free = self.to_free[:65536], self.to_free[65536:]
            self.ev.free(batch)
            self.frees += 1
            self.freed += len(batch)
        self.used -= self.free_need
        self.free_need = 0
        self.host_s["free"] += time.perf_counter() - t0

    def try_admit(self, rid: int, text: str, size: int, arrival: float, now: float) -> bool:
        return self.admit_many([(rid, text, size, arrival)], now) == 1

    def admit_many(self, reqs, now: float) -> int:
        """Admits requests (rid, text, size, arrival) in order while they
        fit; their texts are parsed together (inet_load_nets, on the host
        thread pool).  Returns how many were admitted."""
        take, needs = [], []
        extra = 0

        def fits(need):
            return (self.used + extra + need <= self.max_agents and
                    len(self.inflight) + len(self.to_free) + len(take) < self.max_nets)
        for rid, text, size, arrival in reqs:
            need = self.footprint(text, size)
            if need > self.max_agents:
                raise ValueError(f"request {rid} needs about {need} agent slots; the arena holds {self.max_agents}")
            if not fits(need) and self.to_free:
                self._free()
            if not fits(need):
                break                             # wait for running requests to finish
            take.append((rid, text, size, arrival))
            needs.append(need)
            extra += need
        if not take:
            return 0
        t0 = time.perf_counter()
        nids = self.ev.load_nets([t for _, t, _, _ in take])
        if self.quotas:
            self.ev.set_quotas(nids, needs)
        self.host_s["load"] += time.perf_counter() - t0
        for (rid, _, _, arrival), need, nid in zip(take, needs, nids):
            self.unstaged.append(nid)
            self.used += need
            self.inflight[nid] = (rid, arrival, now, need)
            self.running += 1
        return len(take)

    # -- device epochs and harvest ------------------------------------------
    def epoch(self, now_fn) -> list[Finished]:
        done = []
        ev = self.ev
        clk = time.perf_counter
        t0 = clk()
        if self.unstaged:
            ev.stage(self.unstaged)   # one upload for every net admitted since
            self.unstaged = []
        t1 = clk()
        self.host_s["stage"] += t1 - t0
        reduced = False
        if self.running:
            st = ev.reduce([], mode="async", slice_us=self.epoch_us, block=self.block, grid=self.grid,
                           check=False)
            t2 = clk()
            self.host_s["reduce"] += t2 - t1
            self.performed += st.get("interactions", 0)
            self.epochs += 1
            reduced = True
            if st["status"] not in ("OK", "STEP_LIMIT", "NO_RULE"):
                # a fatal error poisons the arena: every request in it fails
                t = now_fn()
                for nid, (rid, arr, adm, _) in self.inflight.items():
                    done.append(Finished(rid, arr, adm, t, None, 0, st["status"]))
                self._reset()
                return done
            fin = [nid for nid in ev.finished() if nid in self.inflight]
            self.running -= len(fin)
            self.ready.extend(fin)
            if fin:
                td = now_fn()
                for nid in fin:
                    self.detected[nid] = td
            self.host_s["finished"] += clk() - t2
        t3 = clk()
        done.extend(self._harvest(now_fn, wait=False))
        self.host_s["harvest"] += clk() - t3
        if self.to_free and (self.free_need * 16 >= self.max_agents or len(self.to_free) * 4 >= self.max_nets):
            self._free()
        if not reduced and self.rb_batch is not None:
            time.sleep(50e-6)   # only a readback in flight: poll gently
        return done

    def _reset(self):
        if self.rb_batch is not None:
            self.ev.readback_nats_end(True)
        self.ev.reset()
        self.resets += 1
        self.used = 0
        self.inflight = {}
        self.unstaged = []
        self.running = 0
        self.ready = []
        self.rb_batch = None
        self.to_free = []
        self.free_need = 0
        self.detected = {}

    def _harvest(self, now_fn, wait: bool) -> list[Finished]:
        """Completes the readback in flight (if done) and begins the next."""
        out = []
        ev = self.ev
        if self.rb_batch is not None:
            r = ev.readback_nats_end(wait)
            if r is None:
                return out
            vals, ints = r
            t = now_fn()
            stats = ev.status(self.rb_batch) if self.quotas else ["OK"] * len(self.rb_batch)
            for nid, v, n, stt in zip(self.rb_batch, vals, ints, stats):
                rid, arr, adm, need = self.inflight.pop(nid)
                self.to_free.append(nid)
                self.free_need += need
                out.append(Finished(rid, arr, adm, t, v, n, stt, self.detected.pop(nid, t)))
            self.rb_batch = None
        if self.ready:
            batch, self.ready = self.ready[:65536], self.ready[65536:]
            ev.readback_nats_begin(batch)
            self.rb_batch = batch
        return out

    def busy(self) -> bool:
        return bool(self.inflight)

    def _admit_parsed(self, chunk, now: float) -> int:
        """Admits requests of a parsed chunk from chunk["next"] on, in order,
        while they fit.  Returns how many."""
        take, needs = 0, []
        extra = 0
        reqs = chunk["reqs"]
        while chunk["next"] + take < len(reqs):
            rid, text, size, arrival = reqs[chunk["next"] + take]
            need = self.footprint(text, size)
            if need > self.max_agents:
                raise ValueError(f"request {rid} needs about {need} agent slots; the arena holds {self.max_agents}")
            fits = (self.used + extra + need <= self.max_agents and
                    len(self.inflight) + len(self.to_free) + take < self.max_nets)
            if not fits and self.to_free:
                self._free()
                fits = (self.used + extra + need <= self.max_agents and
                        len(self.inflight) + len(self.to_free) + take < self.max_nets)
            if not fits:
                break
            needs.append(need)
            extra += need
            take += 1
        if not take:
            return 0
        t0 = time.perf_counter()
        nids = self.ev.load_parsed(chunk["parsed"], chunk["next"], take)
        if self.quotas:
            self.ev.set_quotas(nids, needs)
        self.host_s["load"] += time.perf_counter() - t0
        for (rid, _, _, arrival), need, nid in zip(reqs[chunk["next"]:chunk["next"] + take], needs, nids):
            self.unstaged.append(nid)
            self.used += need
            self.inflight[nid] = (rid, arrival, now, need)
            self.running += 1
        chunk["next"] += take
        return take

    def serve(self, requests, time_scale: float = 1.0, max_wall_s: float = math.inf,
              on_queue_empty=None) -> list[Finished]:
        """Runs `requests` (objects with .arrival_s, .net, .size) to the end.
        Arrivals are replayed on the wall clock, scaled by time_scale.
        on_queue_empty(t, done), if given, is called once, the first time
        every request has arrived and been admitted.

        The texts of arrived requests are built and parsed on a second host
        thread (inet_parse_nets reads only the rule set), in chunks, while
        this thread runs the device epochs; admission then only places
        parsed nets (inet_load_parsed)."""
        import threading
        reqs = sorted(enumerate(requests), key=lambda ir: ir[1].arrival_s)
        pending = collections.deque(reqs)
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        out: list[Finished] = []
        to_parse = collections.deque()   # (rid, request) arrived, not yet parsed
        parsed = collections.deque()     # chunks: {"reqs": [(rid, text, size, arrival)], "parsed", "next"}
        lock = threading.Lock()
        wake = threading.Event()
        stop = threading.Event()
        err = []
        ahead = [0]                      # requests parsed and not yet admitted

        def parser():
            try:
                while not stop.is_set():
                    with lock:
                        room = ahead[0] < 65536
                        batch, nbytes = [], 0
                        while room and to_parse and len(batch) < 2048 and nbytes < (8 << 20):
                            rid, r = to_parse.popleft()
                            batch.append((rid, r))
                            nbytes += r.size
                    if not batch:
                        wake.wait(0.0005)
                        wake.clear()
                        continue
                    rows = [(rid, r.net, r.size, r.arrival_s * time_scale) for rid, r in batch]
                    p = self.ev.parse([t for _, t, _, _ in rows])
                    with lock:
                        parsed.append({"reqs": rows, "parsed": p, "next": 0})
                        ahead[0] += len(rows)
            except BaseException as e:  # surfaced on the serving thread
                err.append(e)

        th = threading.Thread(target=parser, daemon=True)
        th.start()
        try:
            while pending or to_parse or parsed or ahead[0] or self.busy():
                if err:
                    raise err[0]
                t = now()
                if t > max_wall_s:
                    break
                arrived = False
                while pending and pending[0][1].arrival_s * time_scale <= t:
                    with lock:
                        to_parse.append(pending.popleft())
                    arrived = True
                if arrived:
                    wake.set()
                while True:
                    with lock:
                        chunk = parsed[0] if parsed else None
                    if chunk is None:
                        break
                    k = self._admit_parsed(chunk, now())
                    with lock:
                        ahead[0] -= k
                        if chunk["next"] == len(chunk["reqs"]):
                            parsed.popleft()
                    if chunk["next"] < len(chunk["reqs"]):
                        break                    # the next request does not fit yet
                    wake.set()
                if on_queue_empty is not None and not pending:
                    with lock:
                        empty = not to_parse and not parsed and ahead[0] == 0
                    if empty:
                        on_queue_empty(now(), list(out))
                        on_queue_empty = None
                if self.busy():
                    out.extend(self.epoch(now))
                elif pending and not to_parse and not parsed:
                    time.sleep(max(0.0, min(0.001, pending[0][1].arrival_s * time_scale - now())))
                else:
                    time.sleep(50e-6)            # arrivals are being parsed
        finally:
            stop.set()
            wake.set()
            th.join()
        if self.to_free:
            self._free()
        return out


def _pct(xs: list[float], p: float):
    """The p-th percentile (nearest rank) of sorted xs, or None."""
    if not xs:
        return None
    return xs[min(len(xs) - 1, max(0, int(math.ceil(p / 100.0 * len(xs))) - 1))]


def summarize(done: list[Finished], wall_s: float) -> dict:
    """Latency percentiles (arrival to result on the host), split into the
    wait for admission and the time from admission to result."""
    lat = sorted(f.latency for f in done)
    wait = sorted(f.admitted - f.arrival for f in done)
    serv = sorted(f.finished - f.admitted for f in done)
    comp = sorted(f.detected - f.admitted for f in done if f.detected)
    rdbk = sorted(f.finished - f.detected for f in done if f.detected)

    def ms(x):
        return None if x is None else 1e3 * x

    ints = sum(f.interactions for f in done)
    return {"requests": len(done), "p50_ms": ms(_pct(lat, 50)), "p99_ms": ms(_pct(lat, 99)),
            "mean_ms": ms(sum(lat) / len(lat)) if lat else None,
            "admission_wait_p50_ms": ms(_pct(wait, 50)), "admission_wait_p99_ms": ms(_pct(wait, 99)),
            "service_p50_ms": ms(_pct(serv, 50)), "service_p99_ms": ms(_pct(serv, 99)),
            # service = reduction (admitted to reported finished) + readback
            "reduce_p50_ms": ms(_pct(comp, 50)), "reduce_p99_ms": ms(_pct(comp, 99)),
            "readback_p50_ms": ms(_pct(rdbk, 50)), "readback_p99_ms": ms(_pct(rdbk, 99)),
            "interactions": ints, "interactions_per_s": ints / wall_s if wall_s > 0 else None,
            "failed": sum(1 for f in done if f.status != "OK")}


class MultiServer:
    """Requests sharded over several devices: one Server per device, each
    driven by its own host thread, every arrival routed to the device with
    the least outstanding estimated work.  Requests are independent nets
    (Sec. 2.1), so no data crosses devices."""

    def __init__(self, rules: str, devices, footprint=default_footprint, make_server=None, **server_kw):
        import threading
        if make_server is None:
            def make_server(dev):
                return Server(rules, device=dev, footprint=footprint, **server_kw)
        self.servers = [make_server(dev) for dev in devices]
        self.footprint = footprint
        self.lock = threading.Lock()
        self.load = [0] * len(self.servers)       # estimated work admitted and not finished
        self.routed = [0] * len(self.servers)

    def close(self):
        for s in self.servers:
            s.close()

    def route(self, text: str, size: int) -> int:
        with self.lock:
            k = min(range(len(self.servers)), key=lambda i: self.load[i])
            self.load[k] += size
            self.routed[k] += 1
            return k

    def serve(self, requests, time_scale: float = 1.0) -> list[Finished]:
        """Replays `requests` on the wall clock across the devices."""
        import threading
        reqs = sorted(enumerate(requests), key=lambda ir: ir[1].arrival_s)
        inbox = [collections.deque() for _ in self.servers]
        done: list[Finished] = []
        arrived = threading.Event()
        stop = threading.Event()
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        def worker(k: int):
            srv = self.servers[k]
            waiting = collections.deque()
            while True:
                while inbox[k]:
                    waiting.append(inbox[k].popleft())
                while waiting:
                    rid, r = waiting[0]
                    if not srv.try_admit(rid, r.net, r.size, r.arrival_s * time_scale, now()):
                        break
                    waiting.popleft()
                if srv.busy():
                    fin = srv.epoch(now)
                    if fin:
                        with self.lock:
                            for f in fin:
                                self.load[k] -= requests[f.rid].size
                            done.extend(fin)
                elif stop.is_set() and not waiting and not inbox[k]:
                    return
                else:
                    arrived.wait(0.0005)

        threads = [threading.Thread(target=worker, args=(k,), daemon=True) for k in range(len(self.servers))]
        for th in threads:
            th.start()
        try:
            for rid, r in reqs:
                delay = r.arrival_s * time_scale - now()
                if delay > 0:
                    time.sleep(delay)
                inbox[self.route(r.net, r.size)].append((rid, r))
                arrived.set()
                arrived.clear()
        finally:
            stop.set()
            for th in threads:
                th.join()
        return done
