"""The launch-shape autotuner (paper_1404_0076_gb300/autotune.py): choice,
cache and the interaction-count check against a fake evaluator on CPU; one
real tuning run on the GPU."""
import json

import pytest

import workloads as W
from paper_1404_0076_gb300.autotune import Autotuner, candidates, signature


class FakeEv:
    """Device time depends on the shape; the count is fixed unless `bad`."""

    def __init__(self, bad=None):
        self.bad = bad
        self.calls = 0

    def reset(self):
        pass

    def load_nets(self, nets):
        return list(range(len(nets)))

    def stage(self, ids):
        pass

    def reduce(self, ids, mode, block=0, grid=0, solo_max=0):
        self.calls += 1
        ms = abs(block - 128) / 10 + abs(grid - 304) / 100 + (0.5 if solo_max == -1 else 0)
        n = 1000 + (1 if self.bad == (block, grid) else 0)
        return {"device_ms": 1 + ms, "interactions": n}


def test_candidates_cover_each_form():
    for mode in ("async", "persistent", "graph", "plain"):
        c = candidates(mode, 152)
        assert c and all(s["block"] % 32 == 0 for s in c)
    assert {s["grid"] for s in candidates("async", 152)} == {76, 152, 304, 608, 1216}
    with pytest.raises(ValueError):
        candidates("warp", 152)


def test_picks_the_fastest_and_caches(tmp_path):
    path = str(tmp_path / "cache.json")
    nets = ["< r | Add(Z, r) = Z >"] * 10
    ev = FakeEv()
    best = Autotuner(path, reps=1).tune(ev, "rules", nets, "async", gpu="GB300", num_sms=152)
    assert best == {"block": 128, "grid": 304}
    n = ev.calls
    assert n == len(candidates("async", 152))
    again = Autotuner(path, reps=1).tune(ev, "rules", nets, "async", gpu="GB300", num_sms=152)
    assert again == best and ev.calls == n            # from the cache
    data = json.load(open(path))
    (entry,) = data.values()
    assert len(entry["tried"]) == n
    # another rule set, form or batch shape is another key
    Autotuner(path, reps=1).tune(ev, "other rules", nets, "async", gpu="GB300", num_sms=152)
    Autotuner(path, reps=1).tune(ev, "rules", nets, "persistent", gpu="GB300", num_sms=152)
    Autotuner(path, reps=1).tune(ev, "rules", nets * 100, "async", gpu="GB300", num_sms=152)
    assert len(json.load(open(path))) == 4


def test_shapes_that_disagree_on_the_count_are_an_error(tmp_path):
    with pytest.raises(RuntimeError):
        Autotuner(str(tmp_path / "c.json"), reps=1).tune(FakeEv(bad=(256, 152)), "r", ["x"], "async",
                                                         num_sms=152)


def test_auto_chooses_the_loop_form(tmp_path):
    class TwoForms(FakeEv):
        def reduce(self, ids, mode, block=0, grid=0, solo_max=0):
            r = super().reduce(ids, mode, block, grid, solo_max)
            if mode == "persistent":
                r["device_ms"] = 0.5 + abs(block - 128) / 10   # the step loop is faster here
            return r
    best = Autotuner(str(tmp_path / "c.json"), reps=1).tune(TwoForms(), "r", ["x"], "auto", num_sms=152)
    assert best["mode"] == "persistent" and best["block"] == 128
    shapes = candidates("auto", 152)
    assert {s["mode"] for s in shapes} == {"async", "persistent"}


def test_signature_buckets():
    assert signature(["ab"] * 3) == signature(["abc"] * 3)
    assert signature(["ab"] * 3) != signature(["ab"] * 300)


@pytest.mark.gpu
def test_tuning_a_small_batch_on_the_device(tmp_path):
    import torch
    from paper_1404_0076_gb300 import Evaluator
    nets = W.config1(count=128).nets
    ev = Evaluator(0, max_agents=1 << 22, max_vars=1 << 22)
    ev.load_rules(W.ARITH_RULES)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tuner = Autotuner(str(tmp_path / "c.json"), reps=1)
    best = tuner.tune(ev, W.ARITH_RULES, nets, "async", gpu=torch.cuda.get_device_name(0), num_sms=sms)
    assert best in candidates("async", sms)
    assert len({t.interactions for t in tuner.trials}) == 1
    ev.reset()
    ids = ev.load_nets(nets)
    ev.reduce(ids, mode="async", **best)
    vals, _ = ev.readback_nats(ids)
    assert vals == [m * n for m, n in W.config1(count=128).params]
    ev.close()


def test_shapes_the_device_refuses_are_skipped(tmp_path):
    class Refusing(FakeEv):
        def reduce(self, ids, mode, block=0, grid=0, solo_max=0):
            if block == 512:
                e = RuntimeError("INVALID_ARG: too much shared memory")
                e.name = "INVALID_ARG"
                raise e
            return super().reduce(ids, mode, block, grid, solo_max)
    best = Autotuner(str(tmp_path / "c.json"), reps=1).tune(Refusing(), "r", ["x"], "persistent", num_sms=152)
    assert best["block"] == 128 and best["solo_max"] != -1
