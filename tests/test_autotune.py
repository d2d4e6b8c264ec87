"""The launch tuner's search and storage (CPU; the objective is a stand-in)."""
import pytest

from paper_1903_03406_gb300 import autotune


def test_coordinate_search_finds_the_best_setting():
    target = {"fused_max": 64, "grow1_blocks_per_sm": 4, "tier2_warps": 1216,
              "tier1_cavity": 32, "tier1_boundary": 72}
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


def test_a_win_inside_the_noise_is_not_taken():
    """Repeated timings: a setting 1% faster on the median but with a 5% spread
    does not replace the incumbent; one faster by more than the spread does."""
    def noisy(base):
        return [base * 0.975, base, base * 1.025]

    fast = dict(autotune.DEFAULTS, grow1_blocks_per_sm=16)

    def measure(s):
        return noisy(0.99 if s == fast else 1.0)

    best, _, _ = autotune.search(measure)
    assert best == autotune.DEFAULTS

    def measure2(s):
        return noisy(0.9 if s == fast else 1.0)

    best, t, trials = autotune.search(measure2)
    assert best == fast and abs(t - 0.9) < 1e-12
    assert all(len(x) == 3 for x in trials)  # setting, median, spread


def test_save_load_apply(tmp_path):
    p = tmp_path / "t.json"
    assert autotune.load(str(p)) is None
    s = {"fused_max": 32, "grow1_blocks_per_sm": 8, "tier2_warps": 608, "tier1_cavity": 32,
         "tier1_boundary": 96}
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


def test_settings_are_kept_per_kind(tmp_path):
    """Batches and single meshes keep separate settings; a file in the older
    one-setting form reads as the batched setting."""
    p = str(tmp_path / "t.json")
    a = dict(autotune.DEFAULTS, tier1_cavity=32)
    b = dict(autotune.DEFAULTS, grow1_blocks_per_sm=16)
    autotune.save(a, {"w": "batched"}, p, kind="batched")
    autotune.save(b, {"w": "plain"}, p, kind="plain")
    assert autotune.load(p, kind="batched") == a and autotune.load(p, kind="plain") == b
    import json
    with open(p, "w") as f:
        json.dump({"setting": a, "info": {}}, f)
    assert autotune.load(p) == a and autotune.load(p, kind="plain") is None
    autotune.save(b, None, p, kind="plain")
    assert autotune.load(p) == a and autotune.load(p, kind="plain") == b

