"""The ensemble autotuner's host logic on CPU: candidate order, selection, cache round trip and
invalidation, and the reset after its trials (a fake batch and a fake timer stand in for the GPU)."""
import json

import pytest

from paper_2606_28534_gb300 import autotune, pic
from paper_2606_28534_gb300 import workloads as W

VARIANTS = ["tpb256_minb3_stages2", "tpb128_minb6_stages2", "tpb256_minb2_stages3"]
OCC = [3, 6, 2]  # CTAs per SM that fit, per shape


def _invalid():
    # the binding's error for PIC_EINVAL, made without the library (its message is not needed)
    e = pic.PicError.__new__(pic.PicError)
    RuntimeError.__init__(e, "PIC_EINVAL")
    e.status = 1
    return e


class Batch:
    """Stands in for pic.Batch: records calls; CTA counts beyond OCC are refused as the library
    refuses them."""

    def __init__(self, params, times):
        self.params = params
        self.times = times  # (variant, ctas, use_graph) -> ms per step
        self.tuning = None
        self.calls = []

    def set_tuning(self, variant, ctas_per_sm, use_graph):
        if ctas_per_sm > OCC[variant]:
            raise _invalid()
        self.tuning = (variant, ctas_per_sm, use_graph)
        self.calls.append(("set", self.tuning))

    def step(self, n):
        self.calls.append(("step", n))

    def sync(self):
        pass

    def reset(self):
        self.calls.append(("reset",))


def _timer(batch, steps):
    v, c, g = batch.tuning
    return batch.times(v, c, g) * steps


def _times(v, c, g):
    # shape 1 is fastest; 4 CTAs per SM beat 6 for it; graph replay saves a little
    t = {0: 10.0, 1: 9.0, 2: 9.5}[v]
    if v == 1 and c == 4:
        t -= 0.5
    if not g:
        t += 0.25
    return t


def test_tuner_picks_the_fastest_and_resets(tmp_path):
    runs = W.small_ensemble()
    b = Batch(runs, _times)
    path = str(tmp_path / "t.json")
    r = autotune.tune(b, cache_path=path, timer=_timer, device=("GB300", 152), variants=VARIANTS)
    assert not r["cached"]
    assert r["tuning"] == {"variant": 1, "ctas_per_sm": 4, "use_graph": True}
    assert r["ms_per_step"] == pytest.approx(9.0 - 0.5)
    assert b.tuning == (1, 4, True)
    # the winner is set, then the batch goes back to its initial state
    assert b.calls[-2][0] == "set" and b.calls[-1] == ("reset",)
    # every trial runs whole cycles of 2 * sort_interval steps
    assert all(c[1] == 2 * runs[0]["sort_interval"] for c in b.calls if c[0] == "step")
    # shapes first, then CTA counts (only those that fit), then graphs off
    tried = [t["tuning"] for t in r["trials"]]
    assert [t["variant"] for t in tried[:3]] == [0, 1, 2]
    assert [t["ctas_per_sm"] for t in tried[3:3 + OCC[1]]] == list(range(1, OCC[1] + 1))
    cache = json.load(open(path))
    assert list(cache.values())[0]["variant_name"] == VARIANTS[1]


def test_cache_hit_sets_without_trials_and_key_separates_shapes(tmp_path):
    runs = W.small_ensemble()
    path = str(tmp_path / "t.json")
    autotune.tune(Batch(runs, _times), cache_path=path, timer=_timer, device=("GB300", 152), variants=VARIANTS)
    b2 = Batch(runs, _times)
    r = autotune.tune(b2, cache_path=path, timer=_timer, device=("GB300", 152), variants=VARIANTS)
    assert r["cached"] and r["trials"] == []
    assert [c[0] for c in b2.calls] == ["set"]
    assert b2.tuning == (1, 4, True)
    # another GPU, another ensemble, or another set of compiled shapes: no hit
    k = autotune.shape_key(runs, "GB300", 152, VARIANTS)
    assert k != autotune.shape_key(runs, "GB300", 148, VARIANTS)
    assert k != autotune.shape_key(runs[:-1], "GB300", 152, VARIANTS)
    assert k != autotune.shape_key(runs, "GB300", 152, VARIANTS[:2])
    bigger = [W.variant(p, ppc=(4 * p["ppc"][0], 4 * p["ppc"][1])) for p in runs]
    assert k != autotune.shape_key(bigger, "GB300", 152, VARIANTS)
    # force re-tunes
    r3 = autotune.tune(Batch(runs, _times), cache_path=path, timer=_timer, device=("GB300", 152),
                       variants=VARIANTS, force=True)
    assert not r3["cached"]


def test_corrupt_or_stale_cache_entries_are_ignored(tmp_path):
    runs = W.small_ensemble()
    path = tmp_path / "t.json"
    key = autotune.shape_key(runs, "GB300", 152, VARIANTS)
    path.write_text(json.dumps({key: {"tuning": {"variant": 7, "ctas_per_sm": 0, "use_graph": True},
                                      "ms_per_step": 1.0}}))
    r = autotune.tune(Batch(runs, _times), cache_path=str(path), timer=_timer, device=("GB300", 152),
                      variants=VARIANTS)
    assert not r["cached"]
    path.write_text("not json")
    r = autotune.tune(Batch(runs, _times), cache_path=str(path), timer=_timer, device=("GB300", 152),
                      variants=VARIANTS)
    assert not r["cached"]
    assert json.loads(path.read_text())[key]["tuning"]["variant"] == 1
