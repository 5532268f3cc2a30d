"""GB300 evaluator for interaction nets (the data-parallel reduction loop of
the lightweight interaction calculus, Sec. 3 of Jiresch, "Towards a
GPU-based implementation of interaction nets").

`capi` mirrors the C ABI one function per entry point; `Evaluator` wraps a
context whose device workspace and stream come from PyTorch.

    from paper_1404_0076_gb300 import Evaluator
    with Evaluator(device=0) as ev:
        ev.load_rules("Add(y, r) = Z -> r = y;\n"
                      "Add(y, r) = S(x) -> Add(y, w) = x, r = S(w);\n")
        ids = ev.load_nets(["< r | Add(S(Z), r) = S(S(Z)) >"])
        st = ev.reduce(ids, mode="async")      # or "persistent", "graph", "plain"
        ev.readback(ids[0])                    # 'S(S(S(Z)))'
        ev.readback_nats(ids)                  # ([3], [3]): value, interactions

Other modules: `serve` (continuous batching of requests over two arenas),
`autotune` (launch shape and loop form per batch), `shard` (N ranks),
`build` (compiles the library for sm_103a).
"""
from __future__ import annotations

import importlib

# The CUDA library is loaded on first use of `capi` (or anything that needs
# it), so `paper_1404_0076_gb300.build` can be imported before it exists;
# using the evaluator without the library raises ImportError.
MODES = {"plain": 0, "graph": 1, "persistent": 2, "async": 3, "paper": 4}


def __getattr__(name):
    if name == "capi":
        return importlib.import_module(".capi", __name__)
    if name == "InetError":
        return importlib.import_module(".capi", __name__).InetError
    raise AttributeError(name)


class _Lazy:
    def __getattr__(self, name):
        return getattr(importlib.import_module(".capi", __name__), name)


capi_lazy = _Lazy()


class Parsed:
    """A batch of nets parsed by Evaluator.parse; freed when dropped."""

    def __init__(self, handle):
        # Bound now: a batch dropped at interpreter exit cannot import.
        self._free = capi_lazy.inet_parsed_free
        self.handle = handle
        self.n = capi_lazy.inet_parsed_info(handle)[0]

    def __del__(self):
        if getattr(self, "handle", None):
            self._free(self.handle)
            self.handle = None


class Evaluator:
    """One evaluation context on one GPU (device < 0: host-only, for parsing
    and loading without a GPU).

    The workspace is one uint8 tensor from PyTorch's caching allocator and
    the context runs on PyTorch's current stream of that device.
    free_nets=True keeps the owner of every name slot, so that finished nets
    can be freed (free()); it costs one store per name a reduction creates.
    jit=False keeps the asynchronous mode on the general kernel instead of
    the one compiled for the loaded rules (None: the library's default)."""

    def __init__(self, device: int = 0, max_agents: int = 0, max_vars: int = 0, max_pairs: int = 0,
                 max_nets: int = 0, use_torch: bool = True, free_nets: bool = False, jit: bool | None = None):
        from . import capi
        self.cfg = capi.inet_arena_cfg(max_agents, max_vars, max_pairs, max_nets,
                                       capi.INET_ARENA_FREE_NETS if free_nets else 0)
        self.device = device
        self._ws = None
        stream = None
        if device >= 0 and use_torch:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self.ctx = capi.inet_create(device, stream, self.cfg)
        if jit is not None:
            capi.inet_set_jit(self.ctx, jit)
        if device >= 0 and use_torch:
            import torch
            nbytes = capi.inet_workspace_bytes(self.cfg)
            ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=f"cuda:{device}")
            off = (-ws.data_ptr()) % 256
            self._ws = ws
            capi.inet_attach_workspace(self.ctx, ws.data_ptr() + off, nbytes)

    # -- lifecycle
    def close(self):
        from . import capi
        if getattr(self, "ctx", None):
            capi.inet_destroy(self.ctx)
            self.ctx = None
        self._ws = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API
    def load_rules(self, text: str) -> None:
        capi_lazy.inet_load_rules(self.ctx, text)

    def rules(self) -> list[dict]:
        return [capi_lazy.inet_rule_info(self.ctx, i) for i in range(capi_lazy.inet_rule_count(self.ctx))]

    def load_net(self, text: str) -> int:
        return capi_lazy.inet_load_net(self.ctx, text)

    def parse(self, texts) -> "Parsed":
        """Parses nets apart from the context (inet_parse_nets): another
        thread may do this while the context reduces."""
        return Parsed(capi_lazy.inet_parse_nets(self.ctx, list(texts)))

    def load_parsed(self, parsed: "Parsed", first: int, n: int) -> list[int]:
        """Places nets [first, first + n) of a parsed batch (inet_load_parsed)."""
        return capi_lazy.inet_load_parsed(self.ctx, parsed.handle, first, n)

    def load_nets(self, texts) -> list[int]:
        return capi_lazy.inet_load_nets(self.ctx, list(texts))

    def reduce(self, net_ids, mode: str = "persistent", block: int = 0, grid: int = 0, solo_max: int = 0,
               max_steps: int = 0, timeout_s: float = 0.0, trace: bool = False, check: bool = True,
               slice_us: int = 0) -> dict:
        o = capi_lazy.inet_reduce_opts(MODES[mode], block, grid, solo_max, max_steps, int(timeout_s * 1e9),
                                       1 if trace else 0, slice_us)
        rc, st = capi_lazy.inet_reduce(self.ctx, list(net_ids), o, check=check)
        return {"status": capi_lazy.STATUS_NAMES.get(rc, rc), "interactions": st.interactions, "steps": st.steps,
                "max_frontier": st.max_frontier, "live_agents": st.live_agents,
                "peak_live_agents": st.peak_live_agents, "pending_pairs": st.pending_pairs,
                "device_ms": st.device_ms, "launches": st.launches,
                "per_rule": list(st.per_rule[:st.n_rules])}

    def stage(self, net_ids) -> None:
        capi_lazy.inet_stage(self.ctx, list(net_ids))

    def transfer_bytes(self) -> tuple[int, int]:
        return capi_lazy.inet_transfer_bytes(self.ctx)

    def readback(self, net_id: int) -> str:
        return capi_lazy.inet_readback(self.ctx, net_id)

    def readback_nat(self, net_id: int) -> tuple[int, int]:
        return capi_lazy.inet_readback_nat(self.ctx, net_id)

    def pending(self, net_ids) -> list[int]:
        return capi_lazy.inet_net_pending(self.ctx, list(net_ids))

    def finished(self) -> list[int]:
        """Nets finished since the last call (device scan of the counters)."""
        return capi_lazy.inet_net_finished(self.ctx)

    def readback_nats(self, net_ids):
        return capi_lazy.inet_readback_nats(self.ctx, list(net_ids))

    def readback_nats_begin(self, net_ids) -> None:
        """Starts a batched numeral readback that overlaps later reductions."""
        capi_lazy.inet_readback_nats_begin(self.ctx, list(net_ids))

    def readback_nats_end(self, wait: bool = False):
        """(values, interactions) of the batch begun last, or None while it runs."""
        if getattr(self, "_rb_bufs", None) is None:
            self._rb_bufs = capi_lazy.readback_buffers()
        return capi_lazy.inet_readback_nats_end(self.ctx, wait, self._rb_bufs)

    def free(self, net_ids) -> None:
        """Returns the slots and ids of finished nets for reuse (inet_free_nets)."""
        capi_lazy.inet_free_nets(self.ctx, list(net_ids))

    def set_quotas(self, net_ids, quotas) -> None:
        """Most live agents each net may hold (inet_set_quotas)."""
        capi_lazy.inet_set_quotas(self.ctx, list(net_ids), list(quotas))

    def status(self, net_ids) -> list[str]:
        """Each net's status name: OK, NO_RULE or ARENA_FULL (over its quota)."""
        return capi_lazy.inet_net_status(self.ctx, list(net_ids))

    def readback_counts(self) -> tuple[int, int]:
        """Texts inet_readback rendered on the device and on the host."""
        return capi_lazy.inet_readback_counts(self.ctx)

    def jit_info(self) -> dict:
        """State of the rule-specialised asynchronous kernel (inet_jit_info)."""
        return capi_lazy.inet_jit_info(self.ctx)

    def build_jit(self, track: bool | None = None) -> None:
        """Builds the rule-specialised kernel now (inet_jit_build); by
        default the instantiation this context launches."""
        capi_lazy.inet_jit_build(self.ctx, track)

    def arena_usage(self) -> dict:
        """Bump pointers (agent and name slots handed out) and live agents."""
        return capi_lazy.inet_arena_usage(self.ctx)

    def net_info(self, net_id: int) -> dict:
        return capi_lazy.inet_net_info(self.ctx, net_id)

    def trace(self):
        return capi_lazy.inet_trace(self.ctx)

    def reset(self) -> None:
        capi_lazy.inet_reset(self.ctx)


__all__ = ["Evaluator", "InetError", "capi", "MODES"]
