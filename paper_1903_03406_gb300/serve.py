"""Serving: refinement requests admitted into one device-resident batch.

Requests (a CDT with labels and a bound B) arrive over time. The server keeps
one batch (cdr_batch_*) on the GPU. Between rounds it:

* admits waiting requests, in arrival order, while the estimated device memory
  of everything admitted stays within the budget (continuous batching: a
  request joins the running batch at once, and its rounds overlap with those of
  requests admitted earlier);
* runs one batch round, in which every instance serves its own class;
* exports every instance that has finished, records its latency (arrival to
  export complete) and removes it, freeing its slot and memory for the next
  admissions.

An instance's result does not depend on what else is in the batch (the batch
gives each instance the mesh it gets alone), so serving changes latency and
throughput only.

The memory estimate of a request is its final size predicted from its input
size and B: final vertices = V0 * growth(B), at `bytes_per_vertex` device
bytes each. `calibrate` fits the growth table from refined samples (input
vertices, B, final vertices); the defaults are a conservative table for
unit-cube inputs with 1% constraints.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np

# final vertices / input vertices for unit-cube inputs with 1% constraints, by B
DEFAULT_GROWTH = {1.4: 4.6, 1.6: 2.7, 2.0: 1.6}
# device bytes per final vertex: ~6.3 tets of 32+16+8+8+4+1 B, the vertex (32+4 B),
# subfaces and subsegments, the per-round candidate slabs, and headroom for the
# batch's 1.5x capacity growth
DEFAULT_BYTES_PER_VERTEX = 1400
# status of a failed device allocation (CDR_ERR_OOM in include/cdr.h)
CDR_ERR_OOM = -2


@dataclass
class Request:
    rid: int
    arrival: float          # seconds, on the server's clock
    B: float
    mesh: dict              # xyz, tets, segs, seg_id, tris, facet_id, nfacets
    est_bytes: int = 0


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    done: float
    stats: dict
    mesh: dict | None = None

    @property
    def latency(self):
        return self.done - self.arrival


def growth(B, table=None):
    """Final / input vertex ratio for bound B (interpolated in 1/B)."""
    t = sorted((table or DEFAULT_GROWTH).items())
    xs = np.array([1.0 / b for b, _ in t])[::-1]
    ys = np.array([g for _, g in t])[::-1]
    return float(np.interp(1.0 / B, xs, ys))


def estimate_bytes(n_verts, B, table=None, bytes_per_vertex=DEFAULT_BYTES_PER_VERTEX):
    return int(n_verts * growth(B, table) * bytes_per_vertex)


def calibrate(samples, margin=1.1):
    """Growth table {B: ratio} from (input vertices, B, final vertices) samples:
    the largest observed ratio per B, times a safety margin."""
    table = {}
    for n0, B, n1 in samples:
        table[float(B)] = max(table.get(float(B), 0.0), n1 / float(n0))
    return {B: g * margin for B, g in table.items()}


@dataclass
class Server:
    """Continuous-batching server over a batch object with the cdr.Batch API
    (add, round, finished, stats, export, remove)."""

    batch: object
    budget_bytes: int
    keep_meshes: bool = False
    growth_table: dict | None = None
    bytes_per_vertex: int = DEFAULT_BYTES_PER_VERTEX
    clock: object = time.perf_counter
    waiting: list = field(default_factory=list)      # heap of (arrival, rid, Request)
    running: dict = field(default_factory=dict)      # slot -> (Request, admitted time)
    results: list = field(default_factory=list)
    used_bytes: int = 0
    rounds: int = 0
    oom_deferrals: int = 0
    cancelled: list = field(default_factory=list)

    def submit(self, req: Request):
        n = len(req.mesh["xyz"])
        req.est_bytes = estimate_bytes(n, req.B, self.growth_table, self.bytes_per_vertex)
        if req.est_bytes > self.budget_bytes:
            raise ValueError("request %d needs ~%d bytes, more than the whole budget (%d)"
                             % (req.rid, req.est_bytes, self.budget_bytes))
        heapq.heappush(self.waiting, (req.arrival, req.rid, req))

    def admit(self, now):
        """Admit arrived requests in arrival order while the budget allows.

        A request leaves the queue only once the batch has taken it. If the
        device runs out of memory although the estimate fit the budget
        (status CDR_ERR_OOM), admission stops for this step and the request
        waits for running instances to retire; with nothing running, nothing
        would free memory, so the error is raised."""
        admitted = 0
        while self.waiting and self.waiting[0][0] <= now:
            req = self.waiting[0][2]
            if self.used_bytes + req.est_bytes > self.budget_bytes:
                break
            m = req.mesh
            try:
                slot = self.batch.add(req.B, m["xyz"], m["tets"], m["segs"], m["seg_id"],
                                      m["tris"], m["facet_id"], m["nfacets"])
            except Exception as exc:
                if getattr(exc, "status", None) != CDR_ERR_OOM or not self.running:
                    raise
                self.oom_deferrals += 1
                break
            heapq.heappop(self.waiting)
            self.running[slot] = (req, self.clock())
            self.used_bytes += req.est_bytes
            admitted += 1
        return admitted

    def retire(self):
        """Export and remove every finished instance."""
        done = []
        for slot in self.batch.finished():
            if slot not in self.running:
                continue
            req, t_adm = self.running[slot]
            st = self.batch.stats(slot)
            mesh = self.batch.export(slot)  # the result reaches the host
            self.batch.remove(slot)
            self.used_bytes -= req.est_bytes
            del self.running[slot]
            r = Result(req.rid, req.arrival, t_adm, self.clock(), st,
                       mesh if self.keep_meshes else None)
            self.results.append(r)
            done.append(r)
        return done

    def cancel(self, rid):
        """Withdraw request `rid`. A waiting request leaves the queue. A running
        one is removed from the batch between rounds (cdr_batch_remove), which
        frees its slot and its share of the budget for the next admissions; its
        partial mesh is dropped. Returns False if the request is unknown or has
        already finished."""
        for i, (_, r_id, _req) in enumerate(self.waiting):
            if r_id == rid:
                self.waiting.pop(i)
                heapq.heapify(self.waiting)
                self.cancelled.append(rid)
                return True
        for slot, (req, _t) in list(self.running.items()):
            if req.rid == rid:
                self.batch.remove(slot)
                self.used_bytes -= req.est_bytes
                del self.running[slot]
                self.cancelled.append(rid)
                return True
        return False

    def step(self):
        """One scheduling step: admit, one round, retire. Returns the number of
        instances that had work in the round."""
        self.admit(self.clock())
        active = 0
        if self.running:
            active = self.batch.round()
            self.rounds += 1
        self.retire()
        return active

    def idle(self):
        return not self.running and not self.waiting

    def run(self, until_empty=True, max_steps=1 << 40):
        steps = 0
        while steps < max_steps:
            if self.idle() and until_empty:
                break
            if not self.running and self.waiting:
                wait = self.waiting[0][0] - self.clock()
                if wait > 0:
                    time.sleep(min(wait, 0.01))
            self.step()
            steps += 1
        return self.results


def poisson_arrivals(n, rate, seed, t0=0.0):
    """n arrival times of a Poisson process of the given rate (per second)."""
    rng = np.random.default_rng(seed)
    return t0 + np.cumsum(rng.exponential(1.0 / rate, size=n))


def latency_summary(results):
    lat = np.array([r.latency for r in results])
    if len(lat) == 0:
        return {}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "n": int(len(lat))}
