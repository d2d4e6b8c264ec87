"""Host logic of the serving loop (admission by memory budget, continuous
batching, retirement, latency), run against a stand-in batch on the CPU."""
import numpy as np
import pytest

from paper_1903_03406_gb300 import serve


class FakeBatch:
    """Instances finish after a number of rounds fixed by their size; slots of
    removed instances are reused, as in the library."""

    def __init__(self):
        self.left, self.free, self.log = {}, [], []
        self.n = 0

    def add(self, B, xyz, *rest):
        slot = self.free.pop() if self.free else self.n
        if slot == self.n:
            self.n += 1
        self.left[slot] = max(1, len(xyz) // 100)
        self.log.append(("add", slot, len(xyz)))
        return slot

    def round(self):
        active = 0
        for k in self.left:
            if self.left[k] > 0:
                self.left[k] -= 1
                active += 1
        return active

    def finished(self):
        return [k for k, v in self.left.items() if v == 0]

    def stats(self, slot):
        return {"state": "done" if self.left[slot] == 0 else "refining", "steiner_inserted": 1}

    def export(self, slot):
        return {"slot": slot}

    def sizes(self, slot):
        return {}

    def remove(self, slot):
        del self.left[slot]
        self.free.append(slot)
        self.log.append(("remove", slot))


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


def _mesh(n):
    return dict(xyz=np.zeros((n, 3)), tets=None, segs=None, seg_id=None, tris=None, facet_id=None,
                nfacets=6)


def test_estimate_grows_with_size_and_quality():
    assert serve.growth(1.4) > serve.growth(1.6) > serve.growth(2.0) > 1.0
    assert serve.estimate_bytes(2000, 1.4) > serve.estimate_bytes(1000, 1.4)
    assert abs(serve.growth(1.5) - np.interp(1 / 1.5, [1 / 1.6, 1 / 1.4],
                                             [serve.growth(1.6), serve.growth(1.4)])) < 1e-12


def test_admission_respects_the_budget_and_arrival_order():
    b = FakeBatch()
    per = serve.estimate_bytes(1000, 1.6)
    srv = serve.Server(b, budget_bytes=int(2.5 * per), clock=Clock())
    for i in range(6):
        srv.submit(serve.Request(i, arrival=0.0, B=1.6, mesh=_mesh(1000)))
    srv.admit(1.0)
    assert len(srv.running) == 2 and srv.used_bytes == 2 * per
    res = srv.run()
    assert [r.rid for r in sorted(res, key=lambda r: r.rid)] == list(range(6))
    assert srv.used_bytes == 0 and not srv.running
    # never more than two instances on the device at once
    live, peak = 0, 0
    for ev in b.log:
        live += 1 if ev[0] == "add" else -1
        peak = max(peak, live)
    assert peak == 2
    # admission in arrival order: request i is admitted no later than i+1
    adm = {r.rid: r.admitted for r in res}
    assert all(adm[i] <= adm[i + 1] for i in range(5))


def test_continuous_batching_overlaps_requests():
    b = FakeBatch()
    srv = serve.Server(b, budget_bytes=10 ** 12, clock=Clock())
    srv.submit(serve.Request(0, 0.0, 1.4, _mesh(3000)))  # 30 rounds
    srv.submit(serve.Request(1, 0.0, 1.4, _mesh(500)))   # 5 rounds
    res = srv.run()
    by = {r.rid: r for r in res}
    assert by[1].done < by[0].done          # the short one leaves first
    assert srv.rounds == 30                 # they shared rounds
    s = serve.latency_summary(res)
    assert s["n"] == 2 and s["p99_s"] >= s["p50_s"] > 0


def test_oversized_request_is_refused():
    srv = serve.Server(FakeBatch(), budget_bytes=1000)
    with pytest.raises(ValueError):
        srv.submit(serve.Request(0, 0.0, 1.4, _mesh(10 ** 6)))


def test_calibrate_takes_the_largest_ratio_with_margin():
    t = serve.calibrate([(1000, 1.4, 4000), (2000, 1.4, 9000), (1000, 2.0, 1500)], margin=1.0)
    assert t == {1.4: 4.5, 2.0: 1.5}
    assert serve.calibrate([(10, 1.6, 30)])[1.6] == pytest.approx(3.3)


def test_poisson_arrivals():
    t = serve.poisson_arrivals(20000, rate=50.0, seed=3)
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 50.0) < 2.0


class _Oom(RuntimeError):
    status = serve.CDR_ERR_OOM


class OomOnceBatch(FakeBatch):
    """The device refuses one admission for lack of memory."""

    def __init__(self, fail_at):
        super().__init__()
        self.calls = 0
        self.fail_at = fail_at

    def add(self, B, xyz, *rest):
        self.calls += 1
        if self.calls == self.fail_at:
            raise _Oom("out of device memory")
        return super().add(B, xyz, *rest)


def test_out_of_memory_admission_waits_and_loses_nothing():
    b = OomOnceBatch(fail_at=2)
    srv = serve.Server(b, budget_bytes=10 ** 12, clock=Clock())
    for i in range(4):
        srv.submit(serve.Request(i, arrival=0.0, B=1.6, mesh=_mesh(300 + 100 * i)))
    srv.admit(1.0)
    # the second request met the refusal: it still waits, and its bytes are not counted
    assert len(srv.running) == 1 and len(srv.waiting) == 3 and srv.oom_deferrals == 1
    assert srv.used_bytes == srv.running[0][0].est_bytes
    res = srv.run()
    assert sorted(r.rid for r in res) == [0, 1, 2, 3]
    assert srv.used_bytes == 0


def test_out_of_memory_with_nothing_running_is_raised():
    srv = serve.Server(OomOnceBatch(fail_at=1), budget_bytes=10 ** 12, clock=Clock())
    srv.submit(serve.Request(0, arrival=0.0, B=1.6, mesh=_mesh(300)))
    with pytest.raises(_Oom):
        srv.admit(1.0)
    assert len(srv.waiting) == 1


def test_other_admission_errors_are_raised():
    class Broken(FakeBatch):
        def add(self, *a):
            raise ValueError("malformed mesh")

    srv = serve.Server(Broken(), budget_bytes=10 ** 12, clock=Clock())
    srv.submit(serve.Request(0, arrival=0.0, B=1.6, mesh=_mesh(300)))
    with pytest.raises(ValueError):
        srv.admit(1.0)


def test_cancel_frees_the_slot_and_budget():
    b = FakeBatch()
    per = serve.estimate_bytes(1000, 1.6)
    srv = serve.Server(b, budget_bytes=int(2.5 * per), clock=Clock())
    for i in range(4):
        srv.submit(serve.Request(i, arrival=0.0, B=1.6, mesh=_mesh(1000)))
    srv.step()                       # requests 0 and 1 run, 2 and 3 wait
    assert sorted(r.rid for r, _ in srv.running.values()) == [0, 1]
    slot1 = next(k for k, (r, _) in srv.running.items() if r.rid == 1)
    assert srv.cancel(1)             # mid-flight: removed from the batch
    assert ("remove", slot1) in b.log and srv.used_bytes == per
    assert srv.cancel(3)             # still waiting: leaves the queue
    assert not srv.cancel(3) and not srv.cancel(99)
    srv.step()                       # request 2 takes the freed slot
    assert any(ev == ("add", slot1, 1000) for ev in b.log[-3:])
    res = srv.run()
    assert sorted(r.rid for r in res) == [0, 2]
    assert srv.cancelled == [1, 3] and srv.used_bytes == 0 and srv.idle()
