"""The launch tuner's search and storage (CPU; the objective is a stand-in)."""
import pytest

from paper_1903_03406_gb300 import autotune


def test_coordinate_search_finds_the_best_setting():
    target = {"fused_max": 64, "grow1_blocks_per_sm": 4, "tier2_warps": 1216}
    calls = []

    def measure(s):
        calls.append(dict(s))
        return (sum(abs(autotune.SPACE[k].index(s[k]) - autotune.SPACE[k].index(target[k]))
                    for k in target) + 1.0)

    best, t, trials = autotune.search(measure)
    assert best == target and t == 1.0
    assert len(trials) == len(calls) and trials[0][0] == autotune.DEFAULTS


def test_search_keeps_the_start_when_nothing_is_faster():
    best, t, trials = autotune.search(lambda s: 1.0 if s == autotune.DEFAULTS else 2.0)
    assert best == autotune.DEFAULTS and t == 1.0
    # one pass over every other value, then stop
    assert len(trials) == 1 + sum(len(v) - 1 for v in autotune.SPACE.values())


def test_save_load_apply(tmp_path):
    p = tmp_path / "t.json"
    assert autotune.load(str(p)) is None
    s = {"fused_max": 32, "grow1_blocks_per_sm": 8, "tier2_warps": 608}
    autotune.save(s, {"note": "x"}, str(p))
    assert autotune.load(str(p)) == s

    class Obj:
        def tune(self, **kw):
            self.kw = kw

    o = Obj()
    autotune.apply(o, s)
    assert o.kw == s
    autotune.apply(o, None)  # nothing stored: nothing applied
    assert o.kw == s
