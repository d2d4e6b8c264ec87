"""Multi-instance workloads (batched and served): seeded unit-cube PLCs with
log-uniform sizes, 1% segments and 1% triangles, and their initial Delaunay
meshes built on the GPU (cdr_delaunay_box)."""
from __future__ import annotations

import numpy as np

MULTI = {
    "batched64": dict(count=64, nmin=1000, nmax=50000, B=(1.6,), seed=1000),
    "served40": dict(count=40, nmin=2000, nmax=200000, B=(1.4, 1.6, 2.0), seed=10 ** 6),
}


def multi_instances(spec, rank, cdr, stream):
    """Seeded unit-cube PLCs with log-uniform sizes; initial meshes built on the GPU."""
    from paper_1903_03406_gb300 import inputs, replicas
    seed = replicas.instance_seed(spec["seed"], rank)
    rng = np.random.default_rng(seed)
    out = []
    for i in range(spec["count"]):
        n = int(round(np.exp(rng.uniform(np.log(spec["nmin"]), np.log(spec["nmax"])))))
        B = float(spec["B"][rng.integers(len(spec["B"]))])
        pts, _, _ = inputs.box_points("cube", n, seed * 1000 + i)
        dt = cdr.Handle.delaunay_box(pts, stream=stream)
        ex = dt.export()
        dt.close()
        k = max(1, n // 100)
        plc = inputs.plc_from_delaunay(pts, ex["tets"], k, k, seed * 1000 + i)
        out.append(dict(B=B, n=n, mesh=dict(xyz=ex["xyz"], tets=ex["tets"], segs=plc["segs"],
                                            seg_id=plc["seg_id"], tris=plc["tris"],
                                            facet_id=plc["facet_id"], nfacets=plc["nfacets"])))
    return out
