"""Host logic of bench.py's recorded ncu counters (CPU, no GPU).

bench.py reports a kernel's DRAM traffic, and the FP64 sweep's flops per node, from
profiles/ncu_traffic.json only while the digest of the kernel sources matches the one stored
with the counters; any other state reads as "not measured" (None).  The fingering-grid workload
is the full M x Ca x theta grid of 2000 x 102 channels.
"""
import json

import bench
from paper_1707_00198_gb300 import inputs as I


def test_recorded_counters_follow_the_source_digest(tmp_path, monkeypatch):
    d = bench.kernel_source_digest()
    rec = {"k_a": {"src_digest": d, "dram_bytes_per_fluid_node": 146.5, "fp64_flops_per_fluid_node": 400.0},
           "k_old": {"src_digest": "0" * 16, "dram_bytes_per_fluid_node": 150.0},
           "k_flops_only": {"src_digest": d, "fp64_flops_per_fluid_node": 412.0}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: d)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("k_a", 10) == 1465.0
    assert bench.recorded_counter("k_a", "fp64_flops_per_fluid_node") == 400.0
    assert bench.recorded_traffic("k_old", 10) is None             # taken from other sources
    assert bench.recorded_traffic("k_flops_only", 10) is None      # no DRAM figure recorded
    assert bench.recorded_counter("k_flops_only", "fp64_flops_per_fluid_node") == 412.0
    assert bench.recorded_traffic("k_missing", 10) is None
    assert bench.recorded_counter("k_a", "no_such_key") is None
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "nowhere"))
    assert bench.recorded_traffic("k_a", 10) is None               # no file


def test_committed_records_match_the_current_sources():
    rec = json.load(open(f"{bench.ROOT}/profiles/ncu_traffic.json"))
    for name, r in rec.items():
        assert r["src_digest"] == bench.kernel_source_digest(), name
    assert 144.0 <= rec["k_sweepf<fp32>"]["dram_bytes_per_fluid_node"] <= 160.0


def test_fingering_grid_is_the_full_parameter_grid():
    geoms, prms = I.fingering_grid()
    assert len(geoms) == len(I.M_GRID) * len(I.CA_GRID) * len(I.THETA_GRID) == 75
    assert all(g.nx == 2000 and g.ny == 102 for g in geoms)
    pts = {(round(p.nu_R / p.nu_B, 9), round(p.nu_R * p.u_in / p.sigma, 9), round(p.theta, 9)) for p in prms}
    assert len(pts) == 75
