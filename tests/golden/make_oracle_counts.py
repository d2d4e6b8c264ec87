"""Writes tests/golden/oracle_counts.json: the oracle's sequential refinement
(mode S: one point at a time, subsegments before subfaces before bad
tetrahedra, Sec. 2's order) run to the end on the single-mesh workloads, with
its final Steiner count, tetrahedron count and bad tetrahedra left.

These are the reference figures of the quality band: the refinement rounds
must end within 1.15x of the sequential refinement's Steiner count and
fraction of bad tetrahedra left. The script calls only the oracle and the
seeded input generators; nothing here comes from the CUDA path.

    python tests/golden/make_oracle_counts.py [workload ...]
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "oracle_counts.json")


def run(name):
    import oracle
    from paper_1903_03406_gb300 import inputs
    w = inputs.CONFIGS[name]
    pts, _, _ = inputs.box_points(w["kind"], w["n"], w["seed"])
    t0 = time.perf_counter()
    if w["recipe"] == "recovered":
        from oracle.recover import recover_segments
        segs = inputs.free_segments(pts, w["n_seg"], w["seed"])
        om, xyz, chains, passes = recover_segments(pts, segs)
        e = om.export()
        plc = inputs.plc_with_chains(xyz, e["tets"], chains, len(pts), w["n_tri"], w["seed"])
    else:
        om = oracle.Mesh.box_delaunay(pts)
        e = om.export()
        plc = inputs.plc_from_delaunay(pts, e["tets"], w["n_seg"], w["n_tri"], w["seed"])
    assert om.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"],
                              plc["nfacets"]) == 0
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    st = om.refine_S(w["B"])
    t_ref = time.perf_counter() - t0
    c = om.check(w["B"])
    bad = int(c["bad_tets"] + c["bad_tets_unspl"])
    return {
        "B": w["B"], "points_in": int(len(pts)), "mesh_verts_in": int(len(e["xyz"])),
        "recipe": w["recipe"], "steiner": int(st["inserted"]),
        "evaluated": int(st["evaluated"]), "tets": int(c["tets"]), "bad_left": bad,
        "bad_frac": bad / c["tets"], "contract_ok": bool(
            c["bad_orient"] == 0 and c["nonlocal_delaunay"] == 0 and c["euler"] == 1
            and c["enc_subsegs"] == 0 and c["enc_subfaces"] == 0 and c["bad_tets"] == 0),
        "refine_s": round(t_ref, 1), "setup_s": round(t_setup, 1),
        "host": platform.machine(),
    }


def main():
    names = sys.argv[1:] or ["cube2k", "uniform100k", "clustered500k"]
    try:
        with open(OUT) as f:
            data = json.load(f)
    except FileNotFoundError:
        data = {}
    for n in names:
        print("mode S on", n, flush=True)
        data[n] = run(n)
        print(n, data[n], flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main()
