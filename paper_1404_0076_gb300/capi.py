"""ctypes binding of the evaluator's C ABI (include/inet.h).

Every C entry point has a Python function of the same name here; they only
marshal arguments and turn a negative status into InetError.  All of the
reduction runs in the CUDA library; if the library is missing this module
raises at import time instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import itertools
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libinet.so")

INET_OK = 0
INET_ERR_INVALID_ARG = -1
INET_ERR_PARSE = -2
INET_ERR_LINEARITY = -3
INET_ERR_NO_RULE = -4
INET_ERR_ARENA_FULL = -5
INET_ERR_STEP_LIMIT = -6
INET_ERR_TIMEOUT = -7
INET_ERR_CUDA = -8
INET_ERR_NO_DEVICE = -9
INET_ERR_STATE = -10

STATUS_NAMES = {
    0: "OK", -1: "INVALID_ARG", -2: "PARSE", -3: "LINEARITY", -4: "NO_RULE", -5: "ARENA_FULL",
    -6: "STEP_LIMIT", -7: "TIMEOUT", -8: "CUDA", -9: "NO_DEVICE", -10: "STATE",
}

INET_MODE_PLAIN = 0
INET_MODE_GRAPH = 1
INET_MODE_PERSISTENT = 2
INET_MODE_ASYNC = 3
INET_MODE_PAPER = 4
INET_MAX_RULES = 64
INET_ARENA_FREE_NETS = 1

EXPORTED = [
    "inet_workspace_bytes", "inet_create", "inet_attach_workspace", "inet_destroy",
    "inet_load_rules", "inet_rule_count", "inet_rule_info", "inet_load_net", "inet_reduce",
    "inet_stage", "inet_transfer_bytes", "inet_readback", "inet_readback_nat", "inet_net_info",
    "inet_trace", "inet_reset", "inet_last_error", "inet_reduce_into", "inet_net_pending",
    "inet_readback_nats", "inet_readback_nats_begin", "inet_readback_nats_end", "inet_bench_exch",
    "inet_control_link", "inet_control_segsum", "inet_net_finished", "inet_load_nets",
    "inet_free_nets", "inet_free_net", "inet_arena_usage", "inet_bench_chase", "inet_readback_counts",
    "inet_set_quotas", "inet_net_status", "inet_parse_nets", "inet_parsed_info", "inet_load_parsed",
    "inet_parsed_free", "inet_set_jit", "inet_jit_info", "inet_jit_build",
]

READ_CHUNK = 65536  # nets per non-blocking readback batch


class inet_arena_cfg(C.Structure):
    _fields_ = [("max_agents", C.c_uint64), ("max_vars", C.c_uint64), ("max_pairs", C.c_uint64),
                ("max_nets", C.c_uint32), ("flags", C.c_uint32)]


class inet_reduce_opts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("block", C.c_int32), ("grid", C.c_int32), ("solo_max", C.c_int32),
                ("max_steps", C.c_uint64), ("timeout_ns", C.c_uint64), ("trace", C.c_int32),
                ("slice_us", C.c_int32)]


class inet_reduce_stats(C.Structure):
    _fields_ = [("interactions", C.c_uint64), ("steps", C.c_uint64), ("max_frontier", C.c_uint64),
                ("live_agents", C.c_int64), ("peak_live_agents", C.c_int64), ("pending_pairs", C.c_uint64),
                ("device_ms", C.c_double), ("n_rules", C.c_uint32), ("launches", C.c_uint32),
                ("per_rule", C.c_uint64 * INET_MAX_RULES)]


class inet_net_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("reduced", C.c_int32), ("interactions", C.c_uint64),
                ("pending_pairs", C.c_uint64), ("live_agents", C.c_int64), ("residual_agents", C.c_int64)]


class inet_rule_desc(C.Structure):
    _fields_ = [("name", C.c_char * 64), ("arity_alpha", C.c_int32), ("arity_beta", C.c_int32),
                ("n_new", C.c_int32), ("new_ports", C.c_int32), ("n_fresh", C.c_int32), ("n_link", C.c_int32)]


class inet_arena_usage_t(C.Structure):
    _fields_ = [("agent_slots", C.c_uint64), ("name_slots", C.c_uint64), ("free_agent_slots", C.c_uint64),
                ("free_name_slots", C.c_uint64), ("live_agents", C.c_int64), ("nets", C.c_uint32),
                ("free_net_ids", C.c_uint32)]


class inet_jit_info_t(C.Structure):
    _fields_ = [("enabled", C.c_int32), ("state", C.c_int32), ("source", C.c_int32), ("pad", C.c_int32),
                ("compile_ms", C.c_double), ("launches", C.c_uint64), ("msg", C.c_char * 256)]


class InetError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with python -m paper_1404_0076_gb300.build")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sig = {
        "inet_workspace_bytes": ([C.POINTER(inet_arena_cfg), C.POINTER(C.c_size_t)], C.c_int32),
        "inet_create": ([C.POINTER(P), C.c_int, P, C.POINTER(inet_arena_cfg)], C.c_int32),
        "inet_attach_workspace": ([P, P, C.c_size_t], C.c_int32),
        "inet_destroy": ([P], None),
        "inet_load_rules": ([P, C.c_char_p, C.c_size_t], C.c_int32),
        "inet_rule_count": ([P, C.POINTER(C.c_int32)], C.c_int32),
        "inet_rule_info": ([P, C.c_int32, C.POINTER(inet_rule_desc)], C.c_int32),
        "inet_load_net": ([P, C.c_char_p, C.c_size_t, C.POINTER(C.c_int32)], C.c_int32),
        "inet_reduce": ([P, C.POINTER(C.c_int32), C.c_int32, C.POINTER(inet_reduce_opts),
                         C.POINTER(inet_reduce_stats)], C.c_int32),
        "inet_stage": ([P, C.POINTER(C.c_int32), C.c_int32], C.c_int32),
        "inet_free_nets": ([P, C.POINTER(C.c_int32), C.c_int32], C.c_int32),
        "inet_free_net": ([P, C.c_int32], C.c_int32),
        "inet_set_quotas": ([P, C.POINTER(C.c_int32), C.POINTER(C.c_uint64), C.c_int32], C.c_int32),
        "inet_parse_nets": ([P, C.c_char_p, C.POINTER(C.c_uint64), C.c_int32, C.POINTER(P)], C.c_int32),
        "inet_parsed_info": ([P, C.POINTER(C.c_int32), C.POINTER(C.c_uint64)], C.c_int32),
        "inet_load_parsed": ([P, P, C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)], C.c_int32),
        "inet_parsed_free": ([P], None),
        "inet_net_status": ([P, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32)], C.c_int32),
        "inet_readback_counts": ([P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)], C.c_int32),
        "inet_arena_usage": ([P, C.POINTER(inet_arena_usage_t)], C.c_int32),
        "inet_set_jit": ([P, C.c_int32], C.c_int32),
        "inet_jit_info": ([P, C.POINTER(inet_jit_info_t)], C.c_int32),
        "inet_jit_build": ([P, C.c_int32], C.c_int32),
        "inet_transfer_bytes": ([P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)], C.c_int32),
        "inet_readback": ([P, C.c_int32, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)], C.c_int32),
        "inet_readback_nat": ([P, C.c_int32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)], C.c_int32),
        "inet_net_info": ([P, C.c_int32, C.POINTER(inet_net_stats)], C.c_int32),
        "inet_net_pending": ([P, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_uint64)], C.c_int32),
        "inet_net_finished": ([P, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32)], C.c_int32),
        "inet_load_nets": ([P, C.c_char_p, C.POINTER(C.c_uint64), C.c_int32, C.POINTER(C.c_int32),
                            C.POINTER(C.c_int32)], C.c_int32),
        "inet_readback_nats": ([P, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_uint64),
                                C.POINTER(C.c_uint64)], C.c_int32),
        "inet_readback_nats_begin": ([P, C.POINTER(C.c_int32), C.c_int32], C.c_int32),
        "inet_bench_exch": ([C.c_int, C.c_uint64, C.c_uint64, C.POINTER(C.c_double)], C.c_int32),
        "inet_bench_chase": ([C.c_int, C.c_uint64, C.c_uint64, C.c_int32, C.POINTER(C.c_double)], C.c_int32),
        "inet_control_link": ([C.c_int, C.POINTER(C.c_uint64), C.c_uint64, C.c_uint32, C.c_int32,
                               C.POINTER(C.c_uint32), C.c_uint64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32),
                               C.POINTER(C.c_double)], C.c_int32),
        "inet_control_segsum": ([C.c_int, C.POINTER(C.c_int32), C.c_uint64, C.POINTER(C.c_int32),
                                 C.POINTER(C.c_uint64)], C.c_int32),
        "inet_readback_nats_end": ([P, C.c_int32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.c_int32,
                                    C.POINTER(C.c_int32)], C.c_int32),
        "inet_trace": ([P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_size_t, C.POINTER(C.c_size_t)],
                       C.c_int32),
        "inet_reset": ([P], C.c_int32),
        "inet_last_error": ([P], C.c_char_p),
        "inet_reduce_into": ([P, C.c_int32, P, C.c_size_t, C.c_uint64, C.c_uint64, C.c_int, P,
                              C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)], C.c_int32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


LIB = _load()


def _check(ctx, status: int) -> int:
    if status != INET_OK:
        msg = LIB.inet_last_error(ctx).decode(errors="replace") if ctx else ""
        raise InetError(status, msg)
    return status


# --- one Python function per C entry point ------------------------------------

def inet_workspace_bytes(cfg: inet_arena_cfg | None = None) -> int:
    n = C.c_size_t()
    _check(None, LIB.inet_workspace_bytes(C.byref(cfg) if cfg else None, C.byref(n)))
    return n.value


def inet_create(device: int, stream: int | None = None, cfg: inet_arena_cfg | None = None) -> C.c_void_p:
    ctx = C.c_void_p()
    st = LIB.inet_create(C.byref(ctx), device, C.c_void_p(stream) if stream else None,
                         C.byref(cfg) if cfg else None)
    if st != INET_OK:
        raise InetError(st, "inet_create failed")
    return ctx


def inet_attach_workspace(ctx, dptr: int, nbytes: int) -> None:
    _check(ctx, LIB.inet_attach_workspace(ctx, C.c_void_p(dptr), nbytes))


def inet_destroy(ctx) -> None:
    LIB.inet_destroy(ctx)


def inet_load_rules(ctx, text: str) -> None:
    b = text.encode()
    _check(ctx, LIB.inet_load_rules(ctx, b, len(b)))


def inet_rule_count(ctx) -> int:
    n = C.c_int32()
    _check(ctx, LIB.inet_rule_count(ctx, C.byref(n)))
    return n.value


def inet_rule_info(ctx, rule: int) -> dict:
    d = inet_rule_desc()
    _check(ctx, LIB.inet_rule_info(ctx, rule, C.byref(d)))
    return {"name": d.name.decode(), "arity_alpha": d.arity_alpha, "arity_beta": d.arity_beta,
            "n_new": d.n_new, "new_ports": d.new_ports, "n_fresh": d.n_fresh, "n_link": d.n_link}


def inet_load_nets(ctx, texts) -> list[int]:
    """Loads many nets in one call (parsed on several host threads)."""
    enc = [t.encode() for t in texts]
    n = len(enc)
    offs = (C.c_uint64 * (n + 1))(0, *itertools.accumulate(map(len, enc)))
    ids = (C.c_int32 * max(1, n))()
    done = C.c_int32()
    _check(ctx, LIB.inet_load_nets(ctx, b"".join(enc), offs, n, ids, C.byref(done)))
    return list(ids[:n])


def inet_parse_nets(ctx, texts) -> C.c_void_p:
    """Parses nets apart from the context (may run on another thread); the
    batch is freed with inet_parsed_free."""
    enc = [t.encode() for t in texts]
    n = len(enc)
    offs = (C.c_uint64 * (n + 1))(0, *itertools.accumulate(map(len, enc)))
    out = C.c_void_p()
    _check(None, LIB.inet_parse_nets(ctx, b"".join(enc), offs, n, C.byref(out)))
    return out


def inet_parsed_info(p) -> tuple[int, int]:
    n, a = C.c_int32(), C.c_uint64()
    _check(None, LIB.inet_parsed_info(p, C.byref(n), C.byref(a)))
    return n.value, a.value


def inet_load_parsed(ctx, p, first: int, n: int) -> list[int]:
    ids = (C.c_int32 * max(1, n))()
    done = C.c_int32()
    _check(ctx, LIB.inet_load_parsed(ctx, p, first, n, ids, C.byref(done)))
    return list(ids[:n])


def inet_parsed_free(p) -> None:
    LIB.inet_parsed_free(p)


def inet_load_net(ctx, text: str) -> int:
    b = text.encode()
    nid = C.c_int32()
    _check(ctx, LIB.inet_load_net(ctx, b, len(b), C.byref(nid)))
    return nid.value


def inet_reduce(ctx, net_ids, opts: inet_reduce_opts | None = None, check: bool = True):
    """Returns (status, inet_reduce_stats).  With check=True a non-OK status
    raises InetError (carrying the stats as .stats)."""
    ids = (C.c_int32 * len(net_ids))(*net_ids)
    st = inet_reduce_stats()
    rc = LIB.inet_reduce(ctx, ids, len(net_ids), C.byref(opts) if opts else None, C.byref(st))
    if check and rc != INET_OK:
        err = InetError(rc, LIB.inet_last_error(ctx).decode(errors="replace"))
        err.stats = st
        raise err
    return rc, st


def inet_stage(ctx, net_ids) -> None:
    ids = (C.c_int32 * len(net_ids))(*net_ids)
    _check(ctx, LIB.inet_stage(ctx, ids, len(net_ids)))


def inet_free_nets(ctx, net_ids) -> None:
    ids = (C.c_int32 * len(net_ids))(*net_ids)
    _check(ctx, LIB.inet_free_nets(ctx, ids, len(net_ids)))


def inet_free_net(ctx, net_id: int) -> None:
    _check(ctx, LIB.inet_free_net(ctx, net_id))


def inet_set_quotas(ctx, net_ids, quotas) -> None:
    ids = (C.c_int32 * len(net_ids))(*net_ids)
    q = (C.c_uint64 * len(quotas))(*quotas)
    _check(ctx, LIB.inet_set_quotas(ctx, ids, q, len(net_ids)))


def inet_net_status(ctx, net_ids) -> list[str]:
    ids = (C.c_int32 * len(net_ids))(*net_ids)
    out = (C.c_int32 * max(1, len(net_ids)))()
    _check(ctx, LIB.inet_net_status(ctx, ids, len(net_ids), out))
    return [STATUS_NAMES.get(out[i], out[i]) for i in range(len(net_ids))]


def inet_readback_counts(ctx) -> tuple[int, int]:
    a, b = C.c_uint64(), C.c_uint64()
    _check(ctx, LIB.inet_readback_counts(ctx, C.byref(a), C.byref(b)))
    return a.value, b.value


def inet_arena_usage(ctx) -> dict:
    u = inet_arena_usage_t()
    _check(ctx, LIB.inet_arena_usage(ctx, C.byref(u)))
    return {k: getattr(u, k) for k, _ in u._fields_}


def inet_set_jit(ctx, enable: bool) -> None:
    _check(ctx, LIB.inet_set_jit(ctx, 1 if enable else 0))


def inet_jit_info(ctx) -> dict:
    u = inet_jit_info_t()
    _check(ctx, LIB.inet_jit_info(ctx, C.byref(u)))
    d = {k: getattr(u, k) for k, _ in u._fields_ if k not in ("pad", "msg")}
    d["msg"] = u.msg.decode(errors="replace")
    return d


def inet_jit_build(ctx, track: bool | None = False) -> None:
    """track None: the instantiation the context launches."""
    _check(ctx, LIB.inet_jit_build(ctx, -1 if track is None else (1 if track else 0)))


def inet_transfer_bytes(ctx) -> tuple[int, int]:
    a = C.c_uint64()
    b = C.c_uint64()
    _check(ctx, LIB.inet_transfer_bytes(ctx, C.byref(a), C.byref(b)))
    return a.value, b.value


def inet_readback(ctx, net_id: int) -> str:
    need = C.c_size_t()
    rc = LIB.inet_readback(ctx, net_id, None, 0, C.byref(need))
    if rc not in (INET_OK, INET_ERR_INVALID_ARG) or need.value == 0:
        _check(ctx, rc)
    buf = C.create_string_buffer(need.value)
    _check(ctx, LIB.inet_readback(ctx, net_id, buf, need.value, C.byref(need)))
    return buf.value.decode()


def inet_readback_nat(ctx, net_id: int) -> tuple[int, int]:
    v = C.c_uint64()
    n = C.c_uint64()
    _check(ctx, LIB.inet_readback_nat(ctx, net_id, C.byref(v), C.byref(n)))
    return v.value, n.value


def inet_net_info(ctx, net_id: int) -> dict:
    s = inet_net_stats()
    _check(ctx, LIB.inet_net_info(ctx, net_id, C.byref(s)))
    return {"status": STATUS_NAMES.get(s.status, s.status), "reduced": bool(s.reduced),
            "interactions": s.interactions, "pending_pairs": s.pending_pairs,
            "live_agents": s.live_agents, "residual_agents": s.residual_agents}


def inet_net_pending(ctx, net_ids) -> list[int]:
    ids = (C.c_int32 * len(net_ids))(*net_ids)
    out = (C.c_uint64 * max(1, len(net_ids)))()
    _check(ctx, LIB.inet_net_pending(ctx, ids, len(net_ids), out))
    return list(out[:len(net_ids)])


def inet_net_finished(ctx, cap: int = READ_CHUNK) -> list[int]:
    """Ids of nets finished since the last call (any order)."""
    out = (C.c_int32 * max(1, cap))()
    n = C.c_int32()
    _check(ctx, LIB.inet_net_finished(ctx, out, cap, C.byref(n)))
    return list(out[:n.value])


def inet_readback_nats(ctx, net_ids) -> tuple[list[int | None], list[int]]:
    """(values, interactions); a value is None when the interface is not a numeral."""
    ids = (C.c_int32 * len(net_ids))(*net_ids)
    vals = (C.c_uint64 * max(1, len(net_ids)))()
    ints = (C.c_uint64 * max(1, len(net_ids)))()
    _check(ctx, LIB.inet_readback_nats(ctx, ids, len(net_ids), vals, ints))
    none = (1 << 64) - 1
    return [None if v == none else v for v in vals[:len(net_ids)]], list(ints[:len(net_ids)])


def inet_readback_nats_begin(ctx, net_ids) -> None:
    ids = (C.c_int32 * max(1, len(net_ids)))(*net_ids)
    _check(ctx, LIB.inet_readback_nats_begin(ctx, ids, len(net_ids)))


def inet_bench_exch(device: int, n_slots: int, n_ops: int) -> float:
    """Random atomic exchanges per second over n_slots 32-bit slots."""
    out = C.c_double()
    st = LIB.inet_bench_exch(device, n_slots, n_ops, C.byref(out))
    if st != INET_OK:
        raise InetError(st, "inet_bench_exch failed")
    return out.value


def inet_bench_chase(device: int, n_slots: int, hops: int, variant: int) -> float:
    ns = C.c_double()
    _check(None, LIB.inet_bench_chase(device, n_slots, hops, variant, C.byref(ns)))
    return ns.value


def inet_control_link(device: int, eq, n_vars: int, method: int):
    """(pairs as a list of (a, b), passes, ms).  eq: sequence of 64-bit
    equation words t | u << 32; method 0 = atomic linker, 1 = sort + merge."""
    n = len(eq)
    if hasattr(eq, "ctypes"):   # a contiguous numpy uint64 array
        arr = eq.ctypes.data_as(C.POINTER(C.c_uint64))
    else:
        arr = (C.c_uint64 * max(1, n))(*eq)
    pairs = (C.c_uint32 * max(2, 2 * n))()
    npairs, passes, ms = C.c_uint64(), C.c_uint32(), C.c_double()
    st = LIB.inet_control_link(device, arr, n, n_vars, method, pairs, n, C.byref(npairs), C.byref(passes), C.byref(ms))
    if st != INET_OK:
        raise InetError(st, "inet_control_link failed")
    k = npairs.value
    return [(pairs[2 * i], pairs[2 * i + 1]) for i in range(k)], passes.value, ms.value


def inet_control_segsum(device: int, values) -> list[int]:
    n = len(values)
    arr = (C.c_int32 * max(1, n))(*values)
    out = (C.c_int32 * max(1, n))()
    m = C.c_uint64()
    st = LIB.inet_control_segsum(device, arr, n, out, C.byref(m))
    if st != INET_OK:
        raise InetError(st, "inet_control_segsum failed")
    return list(out[:m.value])


def readback_buffers():
    """Output arrays for inet_readback_nats_end (one pair per context)."""
    return (C.c_uint64 * READ_CHUNK)(), (C.c_uint64 * READ_CHUNK)()


def inet_readback_nats_end(ctx, wait: bool, bufs=None):
    """(values, interactions) of the batch begun last, or None while it runs."""
    vals, ints = bufs if bufs is not None else readback_buffers()
    n = C.c_int32()
    _check(ctx, LIB.inet_readback_nats_end(ctx, 1 if wait else 0, vals, ints, READ_CHUNK, C.byref(n)))
    if n.value < 0:
        return None
    none = (1 << 64) - 1
    return [None if v == none else v for v in vals[:n.value]], list(ints[:n.value])


def inet_trace(ctx) -> tuple[list[int], list[int]]:
    n = C.c_size_t()
    _check(ctx, LIB.inet_trace(ctx, None, None, 0, C.byref(n)))
    fr = (C.c_int64 * max(1, n.value))()
    lv = (C.c_int64 * max(1, n.value))()
    _check(ctx, LIB.inet_trace(ctx, fr, lv, n.value, C.byref(n)))
    return list(fr[:n.value]), list(lv[:n.value])


def inet_reset(ctx) -> None:
    _check(ctx, LIB.inet_reset(ctx))


def inet_reduce_into(host_ctx, net_id: int, arena_ptr: int, arena_bytes: int, max_agents: int,
                     max_vars: int, device: int, stream: int | None = None) -> tuple[int, int]:
    """Reduces a net of a host-only context inside caller-owned device memory
    without allocating anything; returns (numeral value, interactions)."""
    v = C.c_uint64()
    n = C.c_uint64()
    _check(host_ctx, LIB.inet_reduce_into(host_ctx, net_id, C.c_void_p(arena_ptr), arena_bytes, max_agents,
                                          max_vars, device, C.c_void_p(stream) if stream else None,
                                          C.byref(v), C.byref(n)))
    return v.value, n.value


def inet_last_error(ctx) -> str:
    return LIB.inet_last_error(ctx).decode(errors="replace")
