"""Several GPUs run independent instances (replicas); the only cross-rank step
is the reduction of the measurement. Checked here with world_size-2 gloo ranks on
the CPU, each refining its own small instance with the oracle."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1903_03406_gb300 import inputs, replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _instance(rank):
    """A small constrained instance of rank `rank` (base seed 7), refined by the
    oracle in rounds; returns (points, Steiner points inserted)."""
    import oracle
    seed = replicas.instance_seed(7, rank)
    pts, _, _ = inputs.box_points("uniform", 120, seed)
    om = oracle.Mesh.box_delaunay(pts)
    e = om.export()
    plc = inputs.plc_from_delaunay(pts, e["tets"], 6, 6, seed)
    assert om.set_constraints(plc["segs"], plc["seg_id"], plc["tris"], plc["facet_id"],
                              plc["nfacets"]) == 0
    st = om.refine_R(1.6)
    return pts, int(st["inserted"])


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pts, ins = _instance(rank)
        t = 10.0 + rank  # a stand-in step time: rank 1 is the slower one
        (t_max, ), (ins_sum, ) = replicas.reduce_measurement([t], [ins], world)
        np.savez(os.path.join(out_dir, "r%d.npz" % rank), pts=pts, ins=ins, t_max=t_max,
                 ins_sum=ins_sum)
    finally:
        dist.destroy_process_group()


def test_seeds_are_distinct_per_rank():
    seeds = [replicas.instance_seed(5, r) for r in range(8)]
    assert len(set(seeds)) == 8 and seeds[0] == 5


def test_single_rank_reduction_is_identity():
    assert replicas.reduce_measurement([1.5, 2.0], [3, 4], 1) == ([1.5, 2.0], [3.0, 4.0])


def test_two_gloo_ranks_reduce_time_by_max_and_work_by_sum(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r = [np.load(tmp_path / ("r%d.npz" % k)) for k in range(world)]
    # every rank refined its own instance: different points, its own count
    assert not np.array_equal(r[0]["pts"], r[1]["pts"])
    own = [int(x["ins"]) for x in r]
    assert all(n > 0 for n in own)
    for x in r:
        assert float(x["t_max"]) == 11.0
        assert int(x["ins_sum"]) == sum(own)
    # the reduced work equals what each instance gives when refined alone
    assert _instance(0)[1] == own[0] and _instance(1)[1] == own[1]
