"""Serving (continuous batching over cdr_batch_*) on the GPU: requests that
arrive while others refine are admitted as memory frees up, and each result is
the mesh the request gets alone and the mesh of the oracle's round-by-round
refinement (mode R) of the same input (needs a GPU)."""
import numpy as np
import pytest

from _meshes import assert_same_mesh, oracle_case

pytestmark = pytest.mark.gpu

CASES = [("uniform", 350, 3, 3, 21, 1.6), ("cube", 200, 0, 0, 22, 2.0),
         ("uniform", 500, 4, 4, 23, 1.4), ("clustered", 300, 3, 2, 24, 1.6),
         ("uniform", 250, 2, 2, 25, 2.0), ("cube", 400, 0, 0, 26, 1.6)]


@pytest.fixture(scope="module")
def cdr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03406_gb300 import cdr as c
    c.lib()
    return c


class StepClock:
    """Advances by one unit per reading: arrivals are spread over rounds."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1.0
        return self.t


def test_served_results_equal_alone(cdr):
    from paper_1903_03406_gb300 import serve
    reqs, alone, orc = [], [], []
    for i, (kind, n, ns, nt, seed, B) in enumerate(CASES):
        om, e, plc = oracle_case(kind, n, ns, nt, seed)
        mesh = dict(xyz=e["xyz"], tets=e["tets"], segs=plc["segs"], seg_id=plc["seg_id"],
                    tris=plc["tris"], facet_id=plc["facet_id"], nfacets=plc["nfacets"])
        h = cdr.Handle.create(mesh["xyz"], mesh["tets"], mesh["segs"], mesh["seg_id"],
                              mesh["tris"], mesh["facet_id"], mesh["nfacets"])
        st = h.refine(B)
        alone.append((h.export(), st))
        h.close()
        so = om.refine_R(B)
        orc.append((om.export(), so))
        reqs.append(serve.Request(i, arrival=float(6 * i), B=B, mesh=mesh))
    b = cdr.Batch()
    # room for about two requests at a time: later ones queue, then join the
    # running batch as earlier ones finish
    budget = 2 * max(serve.estimate_bytes(len(r.mesh["xyz"]), r.B) for r in reqs) + 1
    srv = serve.Server(b, budget_bytes=budget, keep_meshes=True, clock=StepClock())
    for r in reqs:
        srv.submit(r)
    res = srv.run()
    assert sorted(r.rid for r in res) == list(range(len(CASES)))
    for r in res:
        ex, st = alone[r.rid]
        assert_same_mesh(r.mesh, ex, "request %d" % r.rid)
        assert_same_mesh(r.mesh, orc[r.rid][0], "request %d against the oracle" % r.rid)
        assert r.stats["steiner_inserted"] == st["steiner_inserted"] == orc[r.rid][1]["inserted"]
        assert r.done > r.admitted >= r.arrival
    # requests overlapped on the device: fewer rounds than run one after another
    assert srv.rounds < sum(st["rounds"] for _, st in alone)
    b.close()
