"""Multi-instance workloads on the CPU: the instance list is a function of the
spec and the rank, instances built through a stand-in for the library's
Delaunay call carry valid constraint labels, and the benchmark's all-cores
oracle leg refines a sample in spawned processes."""
import os
import sys

import numpy as np

import oracle
from paper_1903_03406_gb300 import replicas, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = dict(count=5, nmin=60, nmax=400, B=(1.6, 2.0), seed=77)


def test_specs_are_seeded_log_uniform_and_distinct_per_rank():
    a = workloads.multi_specs(SMALL, 0)
    assert a == workloads.multi_specs(SMALL, 0)
    assert len(a) == 5
    assert all(60 <= x["n"] <= 400 and x["B"] in (1.6, 2.0) for x in a)
    assert len({x["seed"] for x in a}) == 5
    b = workloads.multi_specs(SMALL, 1)
    assert b[0]["seed"] == replicas.instance_seed(77, 1) * 1000
    assert [x["n"] for x in a] != [x["n"] for x in b]


class _DelaunayStandIn:
    """cdr.Handle.delaunay_box served by the oracle's Delaunay builder."""

    class Handle:
        def __init__(self, m):
            self.m = m

        @classmethod
        def delaunay_box(cls, pts, stream=None):
            return cls(oracle.Mesh.box_delaunay(pts))

        def export(self):
            return self.m.export()

        def close(self):
            pass


def test_instances_carry_valid_constraints():
    insts = workloads.multi_instances(SMALL, 0, _DelaunayStandIn, None)
    specs = workloads.multi_specs(SMALL, 0)
    assert [x["n"] for x in insts] == [x["n"] for x in specs]
    for x in insts:
        m = x["mesh"]
        assert len(m["xyz"]) == x["n"] + 8
        k = max(1, x["n"] // 100)
        # 12 box edges, k free segments, 3 per triangle; 12 box triangles + k
        assert len(m["segs"]) == 12 + k + 3 * k and len(m["tris"]) == 12 + k
        om = oracle.Mesh.create(m["xyz"], m["tets"])
        assert om.set_constraints(m["segs"], m["seg_id"], m["tris"], m["facet_id"],
                                  m["nfacets"]) == 0


def test_all_cores_oracle_leg():
    sys.path.insert(0, ROOT)
    import bench
    specs = workloads.multi_specs(SMALL, 0)
    r = bench.oracle_all_cores(specs, 2)
    assert r["kind"] == "oracle" and r["unit"] == "meshes/s" and r["cores"] == 2
    assert r["value"] > 0 and np.isfinite(r["value"])
    assert "first 2 instances" in r["sample"]
