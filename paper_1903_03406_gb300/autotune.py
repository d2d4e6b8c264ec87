"""Launch tuning: search the settings `cdr_set_tuning` takes, for a workload.

A setting changes speed only (every setting gives the same meshes), so the tuner
times a callable that refines a sample workload under each candidate setting.
The settings are the launch shape (fused small rounds, growth grid, tier-2
warps) and the region-growth buffers: how many cavity tetrahedra and boundary
faces a tier-1 (shared-memory) workspace holds before a region moves to tier 2.
The search is coordinate descent: one parameter at a time over its candidate
values, starting from the defaults, repeated while a pass improves. Every
setting is timed several times; a candidate replaces the incumbent only if its
median is faster by more than the spread (max - min) of either one's trials, so
that the choice is not made inside the run-to-run noise. The chosen setting is
stored as JSON beside this module (`tuning.json`) and applied with `apply`.

    python -m paper_1903_03406_gb300.autotune [--instances 16] [--out PATH]
    python -m paper_1903_03406_gb300.autotune --plain clustered500k

The first tunes on a sample of the batched workload (unit-cube PLCs, 1k-50k
points) and stores the setting of batches and serving ("batched"); the second
times whole refinements of a single-mesh workload and stores the setting of
single meshes ("plain"). Each kind keeps its own entry in the file.
"""
from __future__ import annotations

import argparse
import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_PATH = os.path.join(HERE, "tuning.json")

DEFAULTS = {"fused_max": 128, "grow1_blocks_per_sm": 8, "tier2_warps": 608,
            "tier1_cavity": 64, "tier1_boundary": 96}
SPACE = {
    "fused_max": [-1, 16, 32, 64, 128, 256, 512],
    "grow1_blocks_per_sm": [2, 4, 8, 16],
    "tier2_warps": [152, 304, 608, 1216],
    "tier1_cavity": [16, 32, 64],
    "tier1_boundary": [48, 72, 96],
}
REPEAT = 3  # timings per setting


def _stats(times):
    ts = sorted(float(t) for t in (times if isinstance(times, (list, tuple)) else [times]))
    n = len(ts)
    med = ts[n // 2] if n % 2 else 0.5 * (ts[n // 2 - 1] + ts[n // 2])
    return med, ts[-1] - ts[0]


def beats(cand_times, best_times):
    """True if the candidate's median is faster than the incumbent's by more
    than the spread of either one's timings."""
    mc, sc = _stats(cand_times)
    mb, sb = _stats(best_times)
    return mc < mb - max(sc, sb)


def search(measure, space=None, start=None, passes=2):
    """measure(setting) -> seconds, or a list of seconds (one per timing).
    Returns (best setting, its median time, every trial as (setting, median,
    spread))."""
    space = SPACE if space is None else space
    best = dict(DEFAULTS if start is None else start)
    best_ts = measure(best)
    trials = [(dict(best),) + _stats(best_ts)]
    for _ in range(passes):
        improved = False
        for key, values in space.items():
            for v in values:
                if v == best[key]:
                    continue
                cand = dict(best)
                cand[key] = v
                ts = measure(cand)
                trials.append((dict(cand),) + _stats(ts))
                if beats(ts, best_ts):
                    best, best_ts, improved = cand, ts, True
        if not improved:
            break
    return best, _stats(best_ts)[0], trials


KINDS = ("batched", "plain")


def _read(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(setting, info=None, path=DEFAULT_PATH, kind="batched"):
    """Store the setting of one kind (batched or plain), keeping the other's."""
    d = _read(path)
    settings = d.get("settings", {})
    infos = d.get("info", {})
    if "setting" in d:  # a file written before settings were kept per kind
        settings.setdefault("batched", d["setting"])
        infos = {"batched": infos}
    settings[kind] = setting
    infos[kind] = info or {}
    with open(path, "w") as f:
        json.dump({"settings": settings, "info": infos}, f, indent=1)


def load(path=DEFAULT_PATH, kind="batched"):
    """The stored setting of a kind (batched: batches and serving; plain: one
    mesh), or None."""
    d = _read(path)
    if "settings" in d:
        return d["settings"].get(kind)
    if kind == "batched":
        return d.get("setting")
    return None


def apply(obj, setting):
    """Apply a setting to a cdr.Handle or cdr.Batch."""
    if setting:
        obj.tune(**setting)


def _batch_measure(cdr, insts, allocator, stream, repeat=REPEAT):
    import torch

    def measure(setting):
        times = []
        for _ in range(repeat):
            b = cdr.Batch(allocator=allocator, stream=stream)
            apply(b, setting)
            for x in insts:
                m = x["mesh"]
                b.add(x["B"], m["xyz"], m["tets"], m["segs"], m["seg_id"], m["tris"],
                      m["facet_id"], m["nfacets"])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.refine()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            b.close()
        return times
    return measure


def _plain_measure(cdr, name, stream, repeat=REPEAT, mixed=2):
    """Whole refinements of the single-mesh workload `name` (its initial mesh
    built once, restored before each refinement)."""
    import torch
    from paper_1903_03406_gb300 import inputs, recover
    w = inputs.CONFIGS[name]
    pts, _, _ = inputs.box_points(w["kind"], w["n"], w["seed"])
    if w["recipe"] == "recovered":
        segs = inputs.free_segments(pts, w["n_seg"], w["seed"])
        xyz, tets, chains, _ = recover.recover_segments(pts, segs, cdr, stream=stream)
        plc = inputs.plc_with_chains(xyz, tets, chains, len(pts), w["n_tri"], w["seed"])
    else:
        dt = cdr.Handle.delaunay_box(pts, stream=stream)
        ex = dt.export()
        dt.close()
        xyz, tets = ex["xyz"], ex["tets"]
        plc = inputs.plc_from_delaunay(pts, tets, w["n_seg"], w["n_tri"], w["seed"])
    h = cdr.Handle.create(xyz, tets, plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"],
                          plc["nfacets"], mixed_rounds=mixed, allocator=cdr.TorchAllocator(),
                          stream=stream)
    h.checkpoint()

    def measure(setting):
        apply(h, dict(DEFAULTS, **(setting or {})))
        times = []
        for _ in range(repeat):
            h.restore()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.refine(w["B"])
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        return times
    return measure


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--instances", type=int, default=16)
    ap.add_argument("--seed", type=int, default=4242)
    ap.add_argument("--out", default=DEFAULT_PATH)
    ap.add_argument("--plain", default=None,
                    help="tune single-mesh refinement on this workload (e.g. clustered500k)")
    args = ap.parse_args()
    import torch
    from paper_1903_03406_gb300 import cdr, workloads
    if args.plain:
        cdr.lib()
        stream = torch.cuda.current_stream()
        measure = _plain_measure(cdr, args.plain, stream)
        measure(DEFAULTS)  # warm-up
        best, t, trials = search(measure)
        save(best, {"workload": args.plain + " (whole refinements, boundary-mixed rounds)",
                    "seconds": t, "timings_per_setting": REPEAT,
                    "trials": [[s_, med, spread] for s_, med, spread in trials]},
             args.out, kind="plain")
        print(json.dumps({"kind": "plain", "setting": best, "seconds": t, "trials": len(trials)}))
        return
    cdr.lib()
    stream = torch.cuda.current_stream()
    spec = dict(workloads.MULTI["batched64"], count=args.instances, seed=args.seed)
    insts = workloads.multi_instances(spec, 0, cdr, stream)
    measure = _batch_measure(cdr, insts, cdr.TorchAllocator(), stream)
    measure(DEFAULTS)  # warm-up
    best, t, trials = search(measure)
    save(best, {"workload": "batched sample of %d instances (seed %d)" % (args.instances, args.seed),
                "seconds": t, "timings_per_setting": REPEAT,
                "trials": [[s, med, spread] for s, med, spread in trials]}, args.out,
         kind="batched")
    print(json.dumps({"setting": best, "seconds": t, "trials": len(trials)}))


if __name__ == "__main__":
    main()
