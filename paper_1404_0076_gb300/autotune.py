"""Launch-shape autotuner for the reduction loop.

For a batch of nets and a loop form (or "auto": the two whole-loop forms)
it times a small set of launch shapes
on the device and keeps the fastest: threads per block, blocks in the grid
(grid x block against the frontier sets how many pairs each thread takes per
step in the step forms; in the asynchronous form every lane holds one pair,
so it sets how many lanes poll for work), and for the persistent form the
frontier size below which one block runs the steps alone (solo_max).  Every
candidate must reach the same interaction count: reduction is uniformly
confluent, so the count is a property of the nets and not of the launch
(Sec. 2.1), and a candidate that disagrees is an error, not a winner.

Results are cached in a JSON file keyed by the GPU, the rule set, the loop
form and a coarse signature of the batch (log2 buckets of its size), so a
serving process or a benchmark tunes once per kind of batch.
"""
from __future__ import annotations

import hashlib
import json
import math
import os
from dataclasses import dataclass


def default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "paper_1404_0076_gb300", "autotune.json")


def candidates(mode: str, num_sms: int) -> list[dict]:
    """Launch shapes tried for one loop form (grid 0 = the form's default).
    "auto" tries the two whole-loop forms and lets the batch decide: the
    asynchronous loop wins on deep dependency chains, the persistent step
    loop on very wide frontiers."""
    if mode == "auto":
        return ([dict(mode="async", **s) for s in candidates("async", num_sms)] +
                [dict(mode="persistent", **s) for s in candidates("persistent", num_sms)])
    if mode == "async":
        return [dict(block=b, grid=g) for b in (64, 128, 256)
                for g in (num_sms // 2, num_sms, 2 * num_sms, 4 * num_sms, 8 * num_sms)]
    if mode == "persistent":
        return [dict(block=b, grid=0, solo_max=s) for b in (128, 256, 512) for s in (0, 1024, -1)]
    if mode in ("graph", "plain"):
        return [dict(block=b, grid=0) for b in (128, 256, 512)]
    raise ValueError(f"unknown loop form {mode}")


def _bucket(x: float) -> int:
    return int(math.floor(math.log2(max(1.0, x))))


def signature(nets: list[str]) -> str:
    """Coarse shape of a batch: log2 buckets of the net count and of the
    mean and largest text size (agents scale with text)."""
    sizes = [len(t) for t in nets] or [0]
    return f"n{_bucket(len(nets))}-mean{_bucket(sum(sizes) / len(sizes))}-max{_bucket(max(sizes))}"


@dataclass
class Trial:
    shape: dict
    ms: float
    interactions: int


class Autotuner:
    def __init__(self, cache_path: str | None = None, reps: int = 2):
        self.cache_path = cache_path or default_cache_path()
        self.reps = reps
        self.cache = self._load()
        self.trials: list[Trial] = []

    def _load(self) -> dict:
        try:
            with open(self.cache_path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}

    def _save(self) -> None:
        d = os.path.dirname(self.cache_path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    @staticmethod
    def key(gpu: str, rules: str, mode: str, nets: list[str]) -> str:
        h = hashlib.sha256(rules.encode()).hexdigest()[:12]
        return f"{gpu}|{h}|{mode}|{signature(nets)}"

    def tune(self, ev, rules: str, nets: list[str], mode: str = "async", gpu: str = "", num_sms: int = 0,
             shapes: list[dict] | None = None, force: bool = False) -> dict:
        """The fastest launch shape for `nets` under `mode` on evaluator `ev`
        (rules already loaded); cached unless `force`."""
        k = self.key(gpu, rules, mode, nets)
        if not force and k in self.cache:
            return dict(self.cache[k]["shape"])
        shapes = shapes or candidates(mode, num_sms)
        self.trials = []
        counts = set()
        for shape in shapes:
            best = math.inf
            try:
                for _ in range(self.reps):
                    ev.reset()
                    ids = ev.load_nets(nets)
                    ev.stage(ids)
                    st = ev.reduce([], **({"mode": mode} | shape))
                    best = min(best, st["device_ms"])
                    counts.add(st["interactions"])
            except RuntimeError as e:
                if getattr(e, "name", "") == "INVALID_ARG":
                    continue        # a shape this device or form does not take
                raise
            self.trials.append(Trial(dict(shape), best, st["interactions"]))
        if not self.trials:
            raise RuntimeError("no launch shape was accepted")
        if len(counts) != 1:
            raise RuntimeError(f"launch shapes disagree on the interaction count: {sorted(counts)}")
        win = min(self.trials, key=lambda t: t.ms)
        self.cache[k] = {"shape": win.shape, "ms": win.ms,
                         "tried": [{"shape": t.shape, "ms": t.ms} for t in self.trials]}
        self._save()
        return dict(win.shape)
