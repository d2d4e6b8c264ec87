"""Benchmark: Steiner points inserted per second by the refinement rounds on GB300.

One step = the whole refinement (every round, every kernel of the hot path) of
one instance of the workload, from its initial constrained Delaunay mesh (kept
on the device and restored at the start of the step) to the end.

Workload (default, the largest single-GPU configuration): 500,000 points drawn
from a mixture of 3 isotropic Gaussians (sigma 50) in [0,1000]^3 plus the 8 box
corners, 5,000 segments between nearby points and 5,000 triangles inside the
box (seed 2), B = 1.4, subsegments and subfaces split in the same rounds. The
segments that are not Delaunay edges are recovered by midpoints and the
triangles drawn among the recovered mesh's faces; the initial Delaunay meshes
are built on the GPU by the library's point-insertion rounds (untimed set-up).
`--workload uniform100k` runs the 100,000-point uniform configuration instead,
`--workload table1` a sweep shaped like the paper's Table 1, and
`--workload handoff` the gQM3D+ hand-off (a CPU stage for the first k
insertions, then the GPU rounds) against the GPU rounds from the start.

The line also carries:
* quality_band: the final Steiner count and fraction of bad tetrahedra against
  the oracle's sequential refinement of the same input run to the end (stored
  by tests/golden/make_oracle_counts.py), with the ratios;
* batched: a batch of unit-cube PLCs (1k-50k interior points, log-uniform; 1%
  segments and 1% triangles; B = 1.6) refined one after another (create,
  refine, export each) and as one batch: meshes/s of both;
* served: a Poisson stream of requests (unit-cube PLCs with 2k-200k points, B
  drawn from {1.4, 1.6, 2.0}) served by continuous batching under a 120 GB
  budget: meshes/s of a closed-loop run (all requests at once), then p50 / p99
  latency (arrival to export) and meshes/s of a Poisson stream at 0.8x that
  rate, next to the same requests refined one after another.
Their instance and request counts are bounded samples of the 256-instance and
2,000-request streams (--batched / --served set them; 0 leaves the part out).
`--workload batched64` / `served40` print those parts as lines of their own.

--impl reference times the CPU oracle (sequential refinement) on the same
workload, a bounded number of insertions per step, on the host cores.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1903_03406_gb300.inputs import CONFIGS as WORKLOADS  # noqa: E402
METRIC = "Steiner pts inserted/s on 1 GB300"
UNIT = "Steiner points/s"


def log(*a):
    print("[bench %.1fs]" % (time.perf_counter() - T0), *a, file=sys.stderr, flush=True)


T0 = time.perf_counter()
MAX_ROUNDS = 200000


GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_counts.json")


def oracle_counts(name):
    """The oracle's sequential refinement of `name` run to the end (stored)."""
    try:
        with open(GOLDEN) as f:
            return json.load(f).get(name)
    except (OSError, ValueError):
        return None


def quality_band(name, steiner, bad, tets):
    """Steiner count and bad-tetrahedron fraction against the stored oracle run."""
    o = oracle_counts(name)
    if not o:
        return None
    frac = bad / tets if tets else 0.0
    rs = steiner / o["steiner"] if o["steiner"] else None
    rb = frac / o["bad_frac"] if o["bad_frac"] else (1.0 if frac == 0 else None)
    return {"reference": "oracle sequential refinement to the end (mode S)",
            "oracle_steiner": o["steiner"], "oracle_bad_left": o["bad_left"],
            "oracle_tets": o["tets"], "oracle_bad_frac": o["bad_frac"],
            "steiner": int(steiner), "bad_left": int(bad), "tets": int(tets),
            "bad_frac": frac, "steiner_ratio": rs, "bad_frac_ratio": rb,
            "band": 1.15,
            "within_band": bool(rs is not None and rb is not None and rs <= 1.15 and rb <= 1.15)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- workload
def make_workload(name, rank, cdr, stream):
    """Points, the GPU-built initial Delaunay mesh and constraint labels."""
    from paper_1903_03406_gb300 import inputs
    w = WORKLOADS[name]
    from paper_1903_03406_gb300 import replicas
    seed = replicas.instance_seed(w["seed"], rank)
    pts, _, _ = inputs.box_points(w["kind"], w["n"], seed)
    if w["recipe"] == "recovered":
        from paper_1903_03406_gb300 import recover
        segs = inputs.free_segments(pts, w["n_seg"], seed)
        log("recovering %d segments on the GPU (%d points)" % (len(segs), len(pts)))
        xyz, tets, chains, passes = recover.recover_segments(pts, segs, cdr, stream=stream)
        log("recovery: %d passes, %d midpoints" % (passes, len(xyz) - len(pts)))
        ex = {"xyz": xyz, "tets": tets, "recovery_passes": passes,
              "midpoints": len(xyz) - len(pts)}
        plc = inputs.plc_with_chains(xyz, tets, chains, len(pts), w["n_tri"], seed)
        return pts, ex, plc
    log("building the initial Delaunay mesh on the GPU (%d points)" % len(pts))
    dt = cdr.Handle.delaunay_box(pts, stream=stream)
    log("delaunay: %d rounds, %d skipped" % (dt.dt_rounds, dt.skipped))
    ex = dt.export()
    dt.close()
    plc = inputs.plc_from_delaunay(pts, ex["tets"], w["n_seg"], w["n_tri"], seed)
    return pts, ex, plc


def kernel_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "predicates.cuh", "mesh.cuh"):
        with open(os.path.join(ROOT, "paper_1903_03406_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, alg_bytes_per_launch):
    """DRAM bytes per average launch, from the committed ncu record of one launch
    taken on the current kernels (else None): the captured launch's DRAM bytes,
    scaled by the ratio of algorithmic bytes (traffic taken to grow in proportion
    to the work)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d.get(kernel)
        if e and e.get("kernels_sha") == kernel_hash():
            dram = float(e["dram_bytes_read"]) + float(e["dram_bytes_write"])
            return dram * alg_bytes_per_launch / float(e["algorithmic_bytes"])
    except Exception:
        pass
    return None


# Algorithmic bytes of the region-growth kernel, from its device counters:
#  * each neighbour tetrahedron tested: its 32 B record and the one vertex
#    across the shared face (24 B of coordinates);
#  * each cavity tetrahedron: its 32 B record, an 8 B priority mark read and
#    written (atomicMin), a 4 B id written to the slab;
#  * each boundary face: the shell tetrahedron's 8 B mark read and written and
#    12 B of face vertex ids plus 8 B of face links written to the slab.
def grow_bytes(ctr):
    return ctr["tested"] * (32 + 24) + ctr["cavity"] * (32 + 16 + 4) + ctr["boundary"] * (16 + 20)


# -------------------------------------------------------------------- GPU arm
def gpu_arm(args, rank, world):
    import torch
    from paper_1903_03406_gb300 import autotune, cdr

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cdr.lib()
    tuning = autotune.load(kind="plain")  # the tuner's single-mesh setting, if any
    stream = torch.cuda.current_stream()
    w = WORKLOADS[args.workload]
    B = w["B"]
    pts, ex, plc = make_workload(args.workload, rank, cdr, stream)
    log("workload ready: %d points, %d tets, %d subfaces, %d subsegments" %
        (len(ex["xyz"]), len(ex["tets"]), len(plc["tris"]), len(plc["segs"])))
    al = cdr.TorchAllocator()
    h = cdr.Handle.create(ex["xyz"], ex["tets"], plc["segs"], plc["seg_id"], plc["tris"],
                          plc["facet_id"], plc["nfacets"], mixed_rounds=args.mixed,
                          allocator=al, stream=stream)
    autotune.apply(h, tuning)
    h.checkpoint()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for k in range(args.warmup):
        h.restore()
        t0 = time.perf_counter()
        st = h.refine(B, MAX_ROUNDS)
        log("warmup %d: %.3fs rounds %d inserted %d status %d" %
            (k, time.perf_counter() - t0, st["rounds"], st["steiner_inserted"], st["status"]))
    torch.cuda.synchronize()

    clocks = ClockSampler(dev)
    clocks.start()
    h.profile(enable=2, reset=True)  # events around the region-growth launches only
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")
    total_ms = 0.0
    inserted = 0
    last = None
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 flush between timed steps, outside the events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.restore()
        last = h.refine(B, MAX_ROUNDS)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        inserted += last["steiner_inserted"]
        log("step %d: %.3f ms, %d inserted" % (k, e0.elapsed_time(e1), last["steiner_inserted"]))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier()
    t_wall = time.perf_counter() - t_wall0
    prof = h.profile(enable=0)
    clk = clocks.stop()
    # one more step, untimed, with events around every kernel group
    h.restore()
    h.profile(enable=1, reset=True)
    h.refine(B, MAX_ROUNDS)
    torch.cuda.synchronize()
    breakdown = h.profile(enable=0)["ms"]

    # end to end through the C-ABI with host buffers: create (host -> device),
    # refine, export (device -> host), every step
    n_e2e = max(1, min(args.steps, 3))
    h2d = sum(a.nbytes for a in (ex["xyz"], ex["tets"], plc["segs"], plc["seg_id"], plc["tris"],
                                 plc["facet_id"]))
    d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ins_e2e = 0
    for _ in range(n_e2e):
        he = cdr.Handle.create(ex["xyz"], ex["tets"], plc["segs"], plc["seg_id"], plc["tris"],
                               plc["facet_id"], plc["nfacets"], mixed_rounds=args.mixed,
                               allocator=al, stream=stream)
        autotune.apply(he, tuning)
        st = he.refine(B, MAX_ROUNDS)
        out = he.export()
        torch.cuda.synchronize()
        ins_e2e += st["steiner_inserted"]
        d2h = sum(v.nbytes for v in out.values())
        he.close()
    t_e2e = time.perf_counter() - t0
    # quality of the last exported mesh (host report, outside every timed region)
    from paper_1903_03406_gb300 import quality
    try:
        qual = quality.report(out["xyz"], out["tets"], B)
    except Exception as e:  # a report, not a measurement: never lose the line over it
        qual = {"error": repr(e)}

    # max over ranks of the time, sum of the work (independent instances)
    from paper_1903_03406_gb300 import replicas
    (total_ms_max, e2e_max), (ins_sum, e2e_ins) = replicas.reduce_measurement(
        [total_ms, t_e2e], [inserted, ins_e2e], world, device="cuda")
    if rank != 0:
        return None

    peak, peak_kind = load_peaks()
    ms = prof["ms"]
    dom = max(breakdown, key=lambda g: breakdown[g])
    calls = prof["calls"]
    gb = grow_bytes(prof["counters"]) / 1e9
    grow_ms = ms["grow1"]
    achieved = gb / (grow_ms / 1e3) if grow_ms > 0 else 0.0
    per_launch_traffic = ncu_traffic("k_grow1", gb * 1e9 / max(calls["grow1"], 1))
    launches = prof["counters"].get("launches", None)
    value = ins_sum / (total_ms_max / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(workload_config(args, world), l2="flushed between steps (256 MB write)",
                       initial_mesh=({"segment_recovery_passes": ex["recovery_passes"],
                                      "midpoints": ex["midpoints"],
                                      "built": "on the GPU, untimed"}
                                     if "recovery_passes" in ex else "GPU Delaunay, untimed"),
                       tuning=tuning or "defaults",
                       steiner_per_step=last["steiner_inserted"], rounds_per_step=last["rounds"],
                       rounds_by_class=last.get("rounds_by_class"),
                       final_tets=last["n_tets"], bad_left=last["n_bad_left"], wall_s=t_wall),
        "e2e": {"value": e2e_ins / e2e_max, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "roofline": {"kernel": "k_grow1 (region growth, tier 1)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None,
                     "peak_source": peak_kind,
                     "traffic": per_launch_traffic,
                     "algorithmic_bytes_per_launch": gb * 1e9 / max(calls["grow1"], 1),
                     "avg_launch_ms": grow_ms / max(calls["grow1"], 1),
                     "dominant_group": dom,
                     "group_ms_per_step_untimed_profile": {g: v for g, v in breakdown.items()
                                                           if v > 0}},
        "gpu_launches": launches,
        "quality": qual,
        "quality_band": quality_band(args.workload, last["steiner_inserted"],
                                     last["n_bad_left"], last["n_tets"]),
        "clocks": clk,
    }
    return line


# ------------------------------------------------- batched and served arms
def _margs(m):
    return (m["xyz"], m["tets"], m["segs"], m["seg_id"], m["tris"], m["facet_id"], m["nfacets"])


def multi_arm(args, rank, world, name=None, count=None, cpu=True):
    """The batched or served workload `name` (default: args.workload), with
    `count` instances / requests (default: the workload's own)."""
    import torch
    from paper_1903_03406_gb300 import autotune, cdr, replicas, serve, workloads
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cdr.lib()
    stream = torch.cuda.current_stream()
    name = name or args.workload
    spec = dict(workloads.MULTI[name])
    full = workloads.FULL_COUNT[name]
    if count:
        spec["count"] = int(count)
    tuning = autotune.load()  # the tuner's stored launch setting, if any
    t0 = time.perf_counter()
    insts = workloads.multi_instances(spec, rank, cdr, stream)
    log("%d instances ready in %.1fs (%d points)" % (len(insts), time.perf_counter() - t0,
                                                     sum(x["n"] for x in insts)))
    al = cdr.TorchAllocator()
    clocks = ClockSampler(dev)
    if name.startswith("batched"):
        # warm-up: one small batch and one small instance alone
        for _ in range(max(1, args.warmup)):
            b = cdr.Batch(allocator=al, stream=stream)
            b.add(insts[0]["B"], *_margs(insts[0]["mesh"]))
            b.refine()
            b.close()
        torch.cuda.synchronize()
        clocks.start()
        t0 = time.perf_counter()
        serial_ins = []
        for x in insts:
            h = cdr.Handle.create(*_margs(x["mesh"]), allocator=al, stream=stream)
            autotune.apply(h, tuning)
            st = h.refine(x["B"])
            h.export()
            serial_ins.append(st["steiner_inserted"])
            h.close()
        torch.cuda.synchronize()
        t_serial = time.perf_counter() - t0
        t0 = time.perf_counter()
        b = cdr.Batch(allocator=al, stream=stream)
        autotune.apply(b, tuning)
        slots = [b.add(x["B"], *_margs(x["mesh"])) for x in insts]
        rounds = b.refine()
        batch_ins = []
        for k in slots:
            batch_ins.append(b.stats(k)["steiner_inserted"])
            b.export(k)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        b.close()
        clk = clocks.stop()
        (t_s, t_b), (ins_s, ins_b) = replicas.reduce_measurement(
            [t_serial, t_batch], [sum(serial_ins), sum(batch_ins)], world, device="cuda")
        if rank != 0:
            return None
        n_all = len(insts) * world
        cpu = None
        if world == 1 and cpu and not args.no_cpu_baseline:
            log("cpu baseline: the oracle on all host cores")
            cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else \
                (os.cpu_count() or 1)
            cpu = oracle_all_cores(workloads.multi_specs(spec, rank), cores)
        return {
            "metric": "batched vs serial meshes/s", "value": n_all / t_b, "unit": "meshes/s",
            "serial": {"value": n_all / t_s, "unit": "meshes/s", "steiner_per_s": ins_s / t_s},
            "batched": {"value": n_all / t_b, "unit": "meshes/s", "steiner_per_s": ins_b / t_b,
                        "rounds": rounds},
            "same_counts": serial_ins == batch_ins, "n_gpus": world, "steps": 1,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "instances": len(insts),
                       "points": [x["n"] for x in insts][:8] + ["..."],
                       "points_total": sum(x["n"] for x in insts), "B": spec["B"],
                       "constraints": "1% segments + 1% triangles",
                       "timed": "create/add + refine + export of every instance",
                       "tuning": tuning or "defaults",
                       "sample": "%d of the %d-instance batched workload" % (len(insts), full)},
            "clocks": clk,
            "cpu_baseline": cpu,
        }
    # served: a closed-loop run of every request (all arrived at once: the
    # server's capacity), then a Poisson stream of them at 0.8x that rate
    budget = 120 * 10 ** 9
    reqs = [serve.Request(i, 0.0, x["B"], x["mesh"]) for i, x in enumerate(insts)]
    nw = len(reqs)
    b = cdr.Batch(allocator=al, stream=stream)
    autotune.apply(b, tuning)
    srv = serve.Server(b, budget_bytes=budget)
    t0 = time.perf_counter()
    for r in reqs[:nw]:
        srv.submit(serve.Request(r.rid, t0, r.B, r.mesh))
    srv.run()
    torch.cuda.synchronize()
    closed = nw / (time.perf_counter() - t0)
    b.close()
    rate = 0.8 * closed
    b = cdr.Batch(allocator=al, stream=stream)
    autotune.apply(b, tuning)
    srv = serve.Server(b, budget_bytes=budget)
    clocks.start()
    t0 = time.perf_counter()
    arr = serve.poisson_arrivals(len(reqs), rate, seed=spec["seed"] + rank, t0=t0)
    for r, a in zip(reqs, arr):
        srv.submit(serve.Request(r.rid, float(a), r.B, r.mesh))
    res = srv.run()
    torch.cuda.synchronize()
    t_end = time.perf_counter()
    clk = clocks.stop()
    b.close()
    lat = serve.latency_summary(res)
    span = max(r.done for r in res) - t0
    # the plain per-mesh path on the same requests, one after another
    t0 = time.perf_counter()
    serial_ins = []
    for r in reqs:
        h = cdr.Handle.create(*_margs(r.mesh), allocator=al, stream=stream)
        autotune.apply(h, tuning)
        serial_ins.append(h.refine(r.B)["steiner_inserted"])
        h.export()
        h.close()
    torch.cuda.synchronize()
    t_serial = time.perf_counter() - t0
    served_ins = {r.rid: r.stats["steiner_inserted"] for r in res}
    if rank != 0:
        return None
    return {
        "metric": "served meshes/s; p50/p99 latency", "value": len(res) / span,
        "unit": "meshes/s", "latency": lat, "arrival_rate": rate,
        "closed_loop": {"value": closed, "unit": "meshes/s", "requests": nw},
        "serial": {"value": len(reqs) / t_serial, "unit": "meshes/s",
                   "steiner_per_s": sum(serial_ins) / t_serial,
                   "timed": "create + refine + export of each request, one after another"},
        "same_counts": [served_ins.get(r.rid) for r in reqs] == serial_ins,
        "steiner_per_s": sum(r.stats["steiner_inserted"] for r in res) / span,
        "rounds": srv.rounds, "n_gpus": world, "steps": 1, "warmup": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": name, "requests": len(reqs),
                   "points_total": sum(x["n"] for x in insts), "B": spec["B"],
                   "hbm_budget_gb": budget / 1e9, "arrival": "Poisson, 0.8x closed-loop",
                   "tuning": tuning or "defaults",
                   "sample": "%d of the %d-request served stream" % (len(reqs), full)},
        "clocks": clk,
    }


def workload_config(args, world):
    """The workload named in both arms' JSON lines."""
    w = WORKLOADS[args.workload]
    return {"workload": args.workload, "points": w["n"] + 8, "segments": w["n_seg"],
            "triangles": w["n_tri"], "B": w["B"],
            "constraints": {"recovered": "free segments between nearby points, recovered by "
                                         "midpoints; triangles (some in edge-sharing pairs) "
                                         "among the recovered mesh's faces",
                            "delaunay": "among the Delaunay edges and faces"}[w["recipe"]],
            "parallelism": "independent instances x%d (replicas)" % world,
            "rounds": {0: "one class per round",
                       1: "mixed: every class each round, class-first priority",
                       2: "mixed: subsegments and subfaces together, class-first priority"}[
                           getattr(args, "mixed", 0)]}


# ---------------------------------------------------------- CPU (oracle) arm
def _oracle_instance_job(x):
    """One instance of a multi-instance workload refined by the oracle's
    sequential refinement, in a worker process: its Delaunay mesh and
    constraints are built untimed, the refinement is timed."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    from paper_1903_03406_gb300 import inputs, workloads
    pts, _, _ = inputs.box_points("cube", x["n"], x["seed"])
    om = oracle.Mesh.box_delaunay(pts)
    e = om.export()
    plc = workloads.instance_plc(pts, e["tets"], x["n"], x["seed"])
    om.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"], plc["nfacets"])
    t0 = time.perf_counter()
    st = om.refine_S(x["B"])
    return time.perf_counter() - t0, st["inserted"]


def oracle_all_cores(specs, cores):
    """The oracle on all host cores: `cores` processes (spawned, so safe after
    CUDA is initialised) refine the first `cores` instances, one each. A core
    that refines meshes back to back finishes one per mean refinement time, so
    the host's rate is cores / mean time. Initial Delaunay meshes excluded."""
    import multiprocessing as mp
    sample = specs[:cores]
    with mp.get_context("spawn").Pool(len(sample)) as pool:
        res = pool.map(_oracle_instance_job, sample, chunksize=1)
    mean_t = sum(t for t, _ in res) / len(res)
    ins = sum(i for _, i in res)
    return {"value": len(sample) / mean_t, "unit": "meshes/s", "cores": len(sample),
            "kind": "oracle",
            "sample": "the first %d instances (%d to %d points), one per core, sequential "
                      "refinement, %d insertions, mean %.2f s per mesh" %
                      (len(sample), min(x["n"] for x in sample), max(x["n"] for x in sample),
                       ins, mean_t)}


def oracle_workload(name):
    import oracle
    from paper_1903_03406_gb300 import inputs
    w = WORKLOADS[name]
    pts, _, _ = inputs.box_points(w["kind"], w["n"], w["seed"])
    if w["recipe"] == "recovered":
        from oracle.recover import recover_segments
        segs = inputs.free_segments(pts, w["n_seg"], w["seed"])
        om, xyz, chains, _ = recover_segments(pts, segs)
        e = om.export()
        plc = inputs.plc_with_chains(xyz, e["tets"], chains, len(pts), w["n_tri"], w["seed"])
    else:
        om = oracle.Mesh.box_delaunay(pts)
        e = om.export()
        plc = inputs.plc_from_delaunay(pts, e["tets"], w["n_seg"], w["n_tri"], w["seed"])
    om.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"], plc["nfacets"])
    return om, e, plc


def cpu_sample(om, B, seconds):
    """Sequential refinement for about `seconds` of CPU time, in chunks."""
    ins, t = 0, 0.0
    chunk = 2000
    while t < seconds:
        t0 = time.perf_counter()
        st = om.refine_S(B, chunk)
        t += time.perf_counter() - t0
        ins += st["inserted"]
        if st["steps"] < chunk:
            break
    return ins, t


def reference_arm(args, rank, world):
    if rank != 0:
        return None
    if args.workload not in WORKLOADS:
        return {"impl": "reference", "unavailable": "the reference arm times single-mesh "
                "workloads only; %s is not one" % args.workload}
    w = WORKLOADS[args.workload]
    om, e, plc = oracle_workload(args.workload)
    import oracle
    ins, t = 0, 0.0
    for k in range(args.warmup + args.steps):
        i, dt = cpu_sample(om, w["B"], args.ref_seconds)
        if i == 0:  # refinement finished: start a fresh instance
            om = oracle.Mesh.create(e["xyz"], e["tets"])
            om.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"],
                               plc["nfacets"])
            i, dt = cpu_sample(om, w["B"], args.ref_seconds)
        if k >= args.warmup:
            ins += i
            t += dt
    v = ins / t
    o = oracle_counts(args.workload)
    cover = ""
    if o and o.get("steiner"):
        cover = (", each step continuing the refinement from where the last stopped "
                 "(%d of the %d insertions made to the end were timed)" % (ins, o["steiner"]))
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args, world),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "sequential refinement, %g s of insertions per step%s" %
                                   (args.ref_seconds, cover)},
        "oracle_to_the_end": o,
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def profile_run(args):
    """One refinement of the plain workload for a profiler to capture, round by
    round: a first pass finds the round with the most candidates, then the same
    refinement is replayed from a checkpoint inside an NVTX range named
    "replay", with that round inside a range named "largest" (for example
    ncu --nvtx --nvtx-include "replay/largest/")."""
    import torch
    from paper_1903_03406_gb300 import autotune, cdr
    torch.cuda.set_device(0)
    cdr.lib()
    stream = torch.cuda.current_stream()
    w = WORKLOADS[args.workload]
    pts, ex, plc = make_workload(args.workload, 0, cdr, stream)
    h = cdr.Handle.create(ex["xyz"], ex["tets"], plc["segs"], plc["seg_id"], plc["tris"],
                          plc["facet_id"], plc["nfacets"], mixed_rounds=args.mixed,
                          allocator=cdr.TorchAllocator(), stream=stream)
    autotune.apply(h, autotune.load(kind="plain"))
    h.checkpoint()
    cands = []
    while len(cands) < MAX_ROUNDS:
        r = h.round(w["B"])
        if r["cls"] < 0:
            break
        cands.append(r["candidates"])
    big = max(range(len(cands)), key=lambda k: cands[k])
    h.restore()
    h.profile(enable=0, reset=True)
    ins = 0
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("replay")  # the whole second refinement
    c0 = c1 = None
    for k in range(len(cands)):
        if k == big:
            c0 = h.profile()["counters"]
            torch.cuda.nvtx.range_push("largest")
        ins += h.round(w["B"])["steiner_inserted"]
        if k == big:
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            c1 = h.profile()["counters"]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    delta = {c: c1[c] - c0[c] for c in ("tested", "cavity", "boundary")}
    print(json.dumps({"profile_run": args.workload, "rounds": len(cands), "steiner": ins,
                      "largest_round": big, "largest_candidates": cands[big],
                      "largest_round_growth": delta,
                      "largest_round_algorithmic_bytes": grow_bytes(delta),
                      "kernels_sha": kernel_hash(),
                      "counters": h.profile()["counters"]}), flush=True)
    h.close()


# ----------------------------------------------------------- Table-1-like sweep
TABLE1 = os.path.join(ROOT, "tests", "golden", "paper_table1.json")


def table1_arm(args, rank, world):
    """A Table-1-like sweep (paper Table 1: 25K points of a ball distribution
    plus gamma x 25K polygons, mainly rectangles, for several B): 25,000
    points uniform in a ball, gamma x 25,000 axis-parallel rectangles as facets
    (their corners added as points), each (gamma, B) refined once on the GPU.
    Points, tetrahedra, bad tetrahedra left, time and the dihedral-angle
    histogram are reported beside the paper's gQM3D figures, as context."""
    import torch
    from paper_1903_03406_gb300 import autotune, cdr, inputs, quality
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cdr.lib()
    stream = torch.cuda.current_stream()
    with open(TABLE1) as f:
        paper = {(r["B"], r["gamma"]): r for r in json.load(f)["rows"]}
    tuning = autotune.load(kind="plain")
    pts, _, _ = inputs.box_points("ball", 25000, 7 + rank)
    rows = []
    for g in args.gammas:
        rect = inputs.rectangles(pts, int(round(g * 25000)), 7 + rank)
        xyz = np.ascontiguousarray(np.concatenate([pts, rect.reshape(-1, 3)]))
        dt = cdr.Handle.delaunay_box(xyz, stream=stream)
        ex = dt.export()
        dt.close()
        plc = inputs.plc_rectangles(ex["xyz"], ex["tets"], len(pts), len(rect))
        h = cdr.Handle.create(ex["xyz"], ex["tets"], plc["segs"], plc["seg_id"], plc["tris"],
                              plc["facet_id"], plc["nfacets"], mixed_rounds=args.mixed,
                              allocator=cdr.TorchAllocator(), stream=stream)
        autotune.apply(h, tuning)
        h.checkpoint()
        for B in args.Bs:
            h.restore()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = h.refine(B, MAX_ROUNDS)
            torch.cuda.synchronize()
            dt_s = time.perf_counter() - t0
            out = h.export()
            q = quality.report(out["xyz"], out["tets"], B)
            p = paper.get((B, g))
            rows.append({
                "gamma": g, "B": B, "input_points": int(len(xyz)), "rectangles": int(len(rect)),
                "points_M": st["n_verts"] / 1e6, "tets_M": st["n_tets"] / 1e6,
                "bad_tets": st["n_bad_left"], "seconds": dt_s, "rounds": st["rounds"],
                "steiner_per_s": st["steiner_inserted"] / dt_s,
                "dihedral_hist": q.get("dihedral_hist"), "dihedral_min_deg": q.get("dihedral_min_deg"),
                "paper_gQM3D": ({"points_M": p["points_M"]["gQM3D"], "tets_M": p["tets_M"]["gQM3D"],
                                 "bad_tets": p["bad_tets"]["gQM3D"], "minutes": p["minutes"]["gQM3D"]}
                                if p else None)})
            log("table1 gamma %.2f B %.1f: %.2fM points, %.2fM tets, %d bad, %.2fs" %
                (g, B, st["n_verts"] / 1e6, st["n_tets"] / 1e6, st["n_bad_left"], dt_s))
        h.close()
    if rank != 0:
        return None
    return {"metric": "Table-1-like sweep (context: the paper's gQM3D figures beside)",
            "value": sum(r["steiner_per_s"] for r in rows) / len(rows), "unit": "Steiner points/s",
            "n_gpus": world, "steps": 1, "warmup": 0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "table1", "points": 25000, "distribution": "uniform in a ball",
                       "polygons": "axis-parallel rectangles, gamma x 25,000",
                       "tuning": tuning or "defaults"},
            "rows": rows}


# ------------------------------------------------- gQM3D+ hand-off (Sec. 3)
def handoff_labels(e):
    """cdr_create arguments from an exported oracle mesh: its subsegments and
    subfaces become the constraint labels, its per-facet reference points the
    facet references (so the GPU continues with the same in-facet predicate)."""
    ss, sf = np.asarray(e["ss"]), np.asarray(e["sf"])
    return dict(xyz=np.ascontiguousarray(e["xyz"]), tets=np.ascontiguousarray(e["tets"]),
                segs=np.ascontiguousarray(ss[:, :2]), seg_id=np.ascontiguousarray(ss[:, 2]),
                tris=np.ascontiguousarray(sf[:, :3]), facet_id=np.ascontiguousarray(sf[:, 3]),
                nfacets=int(len(e["facetq"])), facet_ref=np.ascontiguousarray(e["facetq"]))


def _handoff_cpu_job(name, ks, seconds):
    """The CPU stage of the hand-off, in a spawned process: the oracle's
    sequential refinement of the workload, snapshotted (exported) after k
    insertions for every k in ks it reaches within `seconds` of refinement.
    Returns [(k, cumulative refinement seconds, labels)], k = 0 first."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    om, _, _ = oracle_workload(name)
    B = WORKLOADS[name]["B"]
    out = [(0, 0.0, handoff_labels(om.export()))]
    done, t, ended = 0, 0.0, False
    for k in sorted(ks):
        if ended or t >= seconds:
            break
        while done < k:  # a step may refuse its point instead of inserting it
            t0 = time.perf_counter()
            st = om.refine_S(B, k - done)
            t += time.perf_counter() - t0
            done += st["inserted"]
            if st["steps"] < k - done + st["inserted"]:
                ended = True  # the refinement finished first
                break
        if not ended:
            out.append((done, t, handoff_labels(om.export())))
    return out


def handoff_arm(args, rank, world):
    """gQM3D+ (Sec. 3) replaces the initial part of the computation with a CPU
    program. Measured here: a sequential CPU refiner (the oracle's sequential
    refinement stands in for it) makes the first k insertions, the mesh is
    handed to the library through cdr_create, and the GPU rounds finish it;
    against the GPU rounds from the start. Also the GPU's own time for its
    first k insertions (round by round), beside the CPU's."""
    if rank != 0:
        return None
    import multiprocessing as mp
    import torch
    from paper_1903_03406_gb300 import autotune, cdr
    name = args.handoff_of
    w = WORKLOADS[name]
    B = w["B"]
    log("hand-off: the CPU stage (sequential refinement of %s, up to %.0f s)" %
        (name, args.cpu_seconds))
    with mp.get_context("spawn").Pool(1) as pool:
        snaps = pool.apply(_handoff_cpu_job, (name, args.handoff_k, args.cpu_seconds))
    torch.cuda.set_device(0)
    cdr.lib()
    stream = torch.cuda.current_stream()
    tuning = autotune.load(kind="plain")
    al = cdr.TorchAllocator()

    def create(lab):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = cdr.Handle.create(lab["xyz"], lab["tets"], lab["segs"], lab["seg_id"], lab["tris"],
                              lab["facet_id"], lab["nfacets"], facet_ref=lab["facet_ref"],
                              mixed_rounds=args.mixed, allocator=al, stream=stream)
        autotune.apply(h, tuning)
        torch.cuda.synchronize()
        return h, time.perf_counter() - t0

    # the GPU from the start: whole refinements, then one round by round
    h, t_create0 = create(snaps[0][2])
    h.checkpoint()
    for _ in range(args.warmup):
        h.restore()
        h.refine(B, MAX_ROUNDS)
    times = []
    for _ in range(args.steps):
        h.restore()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st0 = h.refine(B, MAX_ROUNDS)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    t_gpu_all = statistics.median(times)
    h.restore()
    torch.cuda.synchronize()
    timeline = []  # (cumulative insertions, cumulative seconds) after each round
    ins, t = 0, 0.0
    by = {}  # (class, candidate bucket) -> [rounds, seconds, insertions]
    while len(timeline) < MAX_ROUNDS:
        t0 = time.perf_counter()
        r = h.round(B)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        t += dt
        if r["cls"] < 0:
            break
        ins += r["steiner_inserted"]
        timeline.append((ins, t))
        c = r["candidates"]
        bucket = next(b for b in (128, 1000, 10000, 100000, 1 << 62) if c <= b)
        acc = by.setdefault((r["cls"], bucket), [0, 0.0, 0])
        acc[0] += 1
        acc[1] += dt
        acc[2] += r["steiner_inserted"]
    # a second pass with CUDA events around every kernel group (untimed):
    # device time per group, summed over the rounds of each class
    h.restore()
    h.profile(enable=1, reset=True)
    groups = {}
    prev = h.profile()["ms"]
    while True:
        r = h.round(B)
        if r["cls"] < 0:
            break
        cur = h.profile()["ms"]
        acc = groups.setdefault(r["cls"], {})
        for g, v in cur.items():
            if v > prev[g]:
                acc[g] = acc.get(g, 0.0) + v - prev[g]
        prev = cur
    h.profile(enable=0)
    h.close()
    cls_name = {0: "subsegments", 1: "subfaces", 2: "tetrahedra", 3: "mixed"}
    round_profile = [{"class": cls_name.get(c, str(c)), "candidates_up_to": b, "rounds": v[0],
                      "seconds": v[1], "inserted": v[2]} for (c, b), v in sorted(by.items())]

    def gpu_first(k):
        for n, s in timeline:
            if n >= k:
                return s
        return None

    rows = []
    for k, t_cpu, lab in snaps:
        if k == 0:
            rows.append({"k": 0, "cpu_s": 0.0, "handoff_s": t_create0, "gpu_rest_s": t_gpu_all,
                         "total_s": t_create0 + t_gpu_all, "steiner": st0["steiner_inserted"],
                         "bad_left": st0["n_bad_left"], "tets": st0["n_tets"]})
            continue
        hk, t_create = create(lab)
        hk.checkpoint()
        rest = []
        for j in range(max(1, min(args.steps, 3))):
            hk.restore()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = hk.refine(B, MAX_ROUNDS)
            torch.cuda.synchronize()
            rest.append(time.perf_counter() - t0)
        hk.close()
        g = gpu_first(k)
        rows.append({"k": k, "cpu_s": t_cpu, "cpu_rate": k / t_cpu if t_cpu > 0 else None,
                     "gpu_first_k_s": g, "gpu_first_k_rate": k / g if g else None,
                     "handoff_s": t_create, "gpu_rest_s": statistics.median(rest),
                     "total_s": t_cpu + t_create + statistics.median(rest),
                     "steiner": k + st["steiner_inserted"], "bad_left": st["n_bad_left"],
                     "tets": st["n_tets"]})
        log("hand-off k=%d: CPU %.2f s, create %.3f s, GPU rest %.3f s (GPU alone: first k "
            "in %s s)" % (k, t_cpu, t_create, statistics.median(rest),
                          "%.3f" % g if g else "-"))
    base = rows[0]["total_s"]
    better = [r["k"] for r in rows[1:] if r["total_s"] < base]
    return {"metric": "gQM3D+ hand-off: CPU refinement of the first k insertions, then the GPU "
                      "rounds (Sec. 3)",
            "value": base, "unit": "s (GPU rounds from the start, create included)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(argparse.Namespace(workload=name, mixed=args.mixed),
                                           1),
                           cpu_stage="the oracle's sequential refinement, one host core",
                           initial_mesh="the oracle's Delaunay mesh and segment recovery",
                           tuning=tuning or "defaults"),
            "rows": rows, "gpu_rounds": len(timeline),
            "gpu_round_profile": {"timing": "host clock around each cdr_round (one "
                                            "synchronisation per round)",
                                  "seconds": t, "by_class_and_size": round_profile,
                                  "group_ms_by_class": {cls_name.get(c, str(c)): v for c, v in
                                                        sorted(groups.items())}},
            "crossover_k": min(better) if better else None,
            "crossover": ("the hand-off is faster from k = %d" % min(better)) if better else
                         "none: at every k measured the GPU rounds from the start finish first"}


def _cpu_baseline_job(name, seconds):
    """The plain workload's CPU baseline, in a spawned process: the oracle's
    sequential refinement of the same input for about `seconds`; its initial
    Delaunay mesh is built untimed."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    t0 = time.perf_counter()
    om, _, _ = oracle_workload(name)
    setup = time.perf_counter() - t0
    ins, t = cpu_sample(om, WORKLOADS[name]["B"], seconds)
    return ins, t, setup


def cpu_baseline_line(name, ins, t):
    o = oracle_counts(name)
    cover = ""
    if o and o.get("steiner"):
        cover = ("; %d of the %d insertions it makes to the end (%.1f%%), the first part of "
                 "the refinement" % (ins, o["steiner"], 100.0 * ins / o["steiner"]))
    return {"value": ins / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "sequential refinement of the same workload for %.1f s (%d insertions, "
                      "initial Delaunay excluded%s)" % (t, ins, cover)}


def _nested(line):
    """A batched / served line folded into the main line."""
    if line is None:
        return None
    drop = {"n_gpus", "steps", "warmup", "higher_is_better", "scaling", "vs_baseline", "dtype",
            "data"}
    return {k: v for k, v in line.items() if k not in drop}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    from paper_1903_03406_gb300 import workloads
    ap.add_argument("--workload", default="clustered500k",
                    choices=sorted(WORKLOADS) + sorted(workloads.MULTI) + ["table1", "handoff"])
    ap.add_argument("--gammas", type=float, nargs="+", default=[0.05, 0.10, 0.15, 0.20, 0.25],
                    help="table1: polygons per input point")
    ap.add_argument("--Bs", type=float, nargs="+", default=[1.4, 1.6, 1.8, 2.0],
                    help="table1: radius-edge bounds")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--handoff-of", default="clustered500k", choices=sorted(WORKLOADS),
                    help="handoff: the single-mesh workload refined")
    ap.add_argument("--handoff-k", type=int, nargs="+", default=[500, 2000, 8000],
                    help="handoff: insertions made by the CPU stage before the hand-off")
    ap.add_argument("--ref-seconds", type=float, default=5.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", type=int, default=128,
                    help="instances of the batched part of the line (0: leave it out)")
    ap.add_argument("--served", type=int, default=40,
                    help="requests of the served part of the line (0: leave it out)")
    ap.add_argument("--mixed", type=int, default=2, choices=[0, 1, 2],
                    help="round kind: 0 one class per round, 1 every class, "
                         "2 subsegments and subfaces together")
    ap.add_argument("--profile-run", action="store_true",
                    help="for profilers: build the workload and refine it once, untimed "
                         "(no warm-up, no other part); prints its counts, not a bench line")
    args = ap.parse_args()
    if args.profile_run:
        profile_run(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        # the oracle on the host cores: rank 0 alone runs it, the others exit
        line = reference_arm(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    plain = args.workload not in workloads.MULTI
    if args.workload in ("table1", "handoff"):
        line = (table1_arm if args.workload == "table1" else handoff_arm)(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if not plain:
        line = multi_arm(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return
    line = gpu_arm(args, rank, world)
    batched = served = None
    if args.batched > 0:
        log("batched part: %d instances" % args.batched)
        batched = multi_arm(args, rank, world, name="batched64", count=args.batched, cpu=False)
    if args.served > 0:
        log("served part: %d requests" % args.served)
        served = multi_arm(args, rank, world, name="served40", count=args.served)
    if line is not None and world == 1 and not args.no_cpu_baseline:
        # after every GPU-timed region, so that the host stays quiet while they run
        log("cpu baseline: the oracle's sequential refinement (one core)")
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(1) as pool:
            ins, t, setup = pool.apply(_cpu_baseline_job, (args.workload, args.cpu_seconds))
        line["cpu_baseline"] = cpu_baseline_line(args.workload, ins, t)
    if batched is not None and world == 1 and not args.no_cpu_baseline:
        log("batched part: the oracle on all host cores")
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else \
            (os.cpu_count() or 1)
        spec = dict(workloads.MULTI["batched64"], count=args.batched)
        batched["cpu_baseline"] = oracle_all_cores(workloads.multi_specs(spec, rank), cores)
    if line is not None:
        if batched is not None:
            line["batched"] = _nested(batched)
        if served is not None:
            line["served"] = _nested(served)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
