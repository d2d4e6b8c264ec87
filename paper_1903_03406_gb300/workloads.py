"""Multi-instance workloads (batched and served): seeded unit-cube PLCs with
log-uniform sizes, 1% segments and 1% triangles, and their initial Delaunay
meshes built on the GPU (cdr_delaunay_box)."""
from __future__ import annotations

import numpy as np

MULTI = {
    "batched64": dict(count=64, nmin=1000, nmax=50000, B=(1.6,), seed=1000),
    "served40": dict(count=40, nmin=2000, nmax=200000, B=(1.4, 1.6, 2.0), seed=10 ** 6),
}
# instances / requests of the whole workloads these are samples of
FULL_COUNT = {"batched64": 256, "served40": 2000}


def multi_specs(spec, rank):
    """Per-instance (n interior points, B, seed) of a multi-instance workload:
    log-uniform sizes and B drawn from the spec's set, seeded per rank."""
    from paper_1903_03406_gb300 import replicas
    seed = replicas.instance_seed(spec["seed"], rank)
    rng = np.random.default_rng(seed)
    out = []
    for i in range(spec["count"]):
        n = int(round(np.exp(rng.uniform(np.log(spec["nmin"]), np.log(spec["nmax"])))))
        B = float(spec["B"][rng.integers(len(spec["B"]))])
        out.append(dict(n=n, B=B, seed=seed * 1000 + i))
    return out


def instance_plc(pts, tets, n, seed):
    """The constraints of one instance: 1% segments and 1% triangles chosen
    among the edges and faces of its Delaunay mesh."""
    from paper_1903_03406_gb300 import inputs
    k = max(1, n // 100)
    return inputs.plc_from_delaunay(pts, tets, k, k, seed)


def multi_instances(spec, rank, cdr, stream):
    """Seeded unit-cube PLCs with log-uniform sizes; initial meshes built on the GPU."""
    from paper_1903_03406_gb300 import inputs
    out = []
    for x in multi_specs(spec, rank):
        n, B = x["n"], x["B"]
        pts, _, _ = inputs.box_points("cube", n, x["seed"])
        dt = cdr.Handle.delaunay_box(pts, stream=stream)
        ex = dt.export()
        dt.close()
        plc = instance_plc(pts, ex["tets"], n, x["seed"])
        out.append(dict(B=B, n=n, mesh=dict(xyz=ex["xyz"], tets=ex["tets"], segs=plc["segs"],
                                            seg_id=plc["seg_id"], tris=plc["tris"],
                                            facet_id=plc["facet_id"], nfacets=plc["nfacets"])))
    return out
