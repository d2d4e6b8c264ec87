"""Host-side pieces of bench.py, on the CPU: the clock record taken during the
timed region (parsed from nvidia-smi's CSV lines), the roofline peak and the
algorithmic-bytes model of region growth."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_takes_median_max_and_active_reasons():
    c = bench.ClockSampler(0)
    c.proc = _Done()
    c.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1965, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    r = c.stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}


def test_clock_record_is_none_without_samples():
    c = bench.ClockSampler(0)
    assert c.stop() is None
    c.proc = _Done()
    assert c.stop() is None


def test_peak_comes_from_the_measured_file_when_present():
    peak, kind = bench.load_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            assert (peak, kind) == (float(json.load(f)["hbm_gbs"]), "measured")
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_growth_bytes_model():
    # 56 B per neighbour tested, 52 B per cavity tetrahedron, 36 B per boundary face
    assert bench.grow_bytes({"tested": 1, "cavity": 0, "boundary": 0}) == 56
    assert bench.grow_bytes({"tested": 0, "cavity": 1, "boundary": 0}) == 52
    assert bench.grow_bytes({"tested": 0, "cavity": 0, "boundary": 1}) == 36
    assert bench.grow_bytes({"tested": 2727545, "cavity": 1958595, "boundary": 816510}) == \
        283983820  # the largest round's figure in profiles/ncu_traffic.json


def test_traffic_record_scales_or_is_withheld():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)["k_grow1"]
    t = bench.ncu_traffic("k_grow1", rec["algorithmic_bytes"] / 10)
    if rec["kernels_sha"] == bench.kernel_hash():
        # taken on the current kernels: traffic scales with the algorithmic bytes
        dram = rec["dram_bytes_read"] + rec["dram_bytes_write"]
        assert abs(t - dram / 10) < 1e-6 * dram
    else:
        # the kernels changed since the capture: no traffic figure is reported
        assert t is None
    assert bench.ncu_traffic("no_such_kernel", 1.0) is None


def test_quality_band_against_the_stored_oracle_run():
    """The band object compares the GPU's final counts with the stored oracle
    run: ratios of the Steiner count and of the bad-tetrahedron fraction."""
    o = bench.oracle_counts("clustered500k")
    assert o and o["steiner"] > 0 and o["contract_ok"]
    b = bench.quality_band("clustered500k", o["steiner"], o["bad_left"], o["tets"])
    assert b["steiner_ratio"] == 1.0 and abs(b["bad_frac_ratio"] - 1.0) < 1e-12
    assert b["within_band"]
    b = bench.quality_band("clustered500k", int(o["steiner"] * 1.2), o["bad_left"], o["tets"])
    assert not b["within_band"]
    # a workload with no bad tetrahedra left on either side is in the band
    c = bench.oracle_counts("cube2k")
    b = bench.quality_band("cube2k", c["steiner"], 0, c["tets"])
    assert c["bad_left"] == 0 and b["bad_frac_ratio"] == 1.0 and b["within_band"]
    assert bench.quality_band("no_such_workload", 1, 0, 1) is None


def test_cpu_baseline_states_its_coverage():
    o = bench.oracle_counts("clustered500k")
    line = bench.cpu_baseline_line("clustered500k", 50000, 15.0)
    assert line["value"] == 50000 / 15.0 and line["cores"] == 1 and line["kind"] == "oracle"
    assert "of the %d insertions" % o["steiner"] in line["sample"]


def test_handoff_cpu_stage_snapshots_are_valid_cdts():
    """The hand-off's CPU stage stops after exactly k insertions and exports a
    mesh whose labels, loaded the way cdr_create takes them, form a CDT of the
    PLC that refines on to the end."""
    import oracle
    snaps = bench._handoff_cpu_job("cube2k", [40, 150], 60.0)
    assert [k for k, _, _ in snaps] == [0, 40, 150]
    assert snaps[0][1] == 0.0 and 0.0 < snaps[1][1] <= snaps[2][1]
    B = bench.WORKLOADS["cube2k"]["B"]
    n0 = len(snaps[0][2]["xyz"])
    for k, _, lab in snaps:
        assert len(lab["xyz"]) == n0 + k
        assert lab["segs"].shape[1] == 2 and len(lab["seg_id"]) == len(lab["segs"])
        assert lab["tris"].shape[1] == 3 and len(lab["facet_id"]) == len(lab["tris"])
        assert lab["facet_ref"].shape == (lab["nfacets"], 3)
        om = oracle.Mesh.create(lab["xyz"], lab["tets"])
        assert om.set_constraints(lab["segs"], lab["seg_id"], lab["tris"], lab["facet_id"],
                                  lab["nfacets"], facetq=lab["facet_ref"]) == 0
        c = om.check(B)
        assert c["bad_orient"] == 0 and c["nonlocal_delaunay"] == 0
        assert c["sf_not_face"] == 0 and c["ss_not_edge"] == 0 and c["seg_chain_bad"] == 0
        om.refine_S(B)
        c = om.check(B)
        assert c["nonlocal_delaunay"] == 0 and c["enc_subsegs"] == 0 and c["enc_subfaces"] == 0
