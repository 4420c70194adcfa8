"""Host logic of bench.py that its JSON line depends on, without a GPU: the
oracle solve-time model behind `cpu_baseline` and the reference arm, and the
source-region hash that keeps `roofline.traffic` tied to the captured
kernels."""
import json
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_modelled_solve_time_counts_cycles_and_parts():
    # t(n) = a n + b n (n-1)/2 per restart cycle, plus residuals and assemblies
    pt = dict(res=0.5, tan=3.0, a=0.1, b=0.01)
    work = dict(nit=2, assemblies=1, lit_hist=[0, 120, 30])
    t = bench.modelled_solve_s(pt, work, restart=50)
    cycles = [50, 50, 20, 30]
    expect = 3 * 0.5 + 3.0 + sum(0.1 * c + 0.01 * c * (c - 1) / 2 for c in cycles)
    assert abs(t - expect) < 1e-12


def test_recorded_oracle_structure_is_consistent():
    rec = bench.oracle_work("cook_p2_64x64x8", "iB", 50)
    assert rec is not None and rec["status"] == 0
    assert sum(rec["lit_hist"][1:rec["nit"] + 1]) == rec["lit_total"]
    assert rec["assemblies"] == 1


def test_traffic_records_follow_the_captured_kernels():
    # a record scales to the run's bytes while the captured kernels' source
    # region is unchanged, and gives null (no traffic claim) once it changed
    path = os.path.join(ROOT, "profiles", "traffic.json")
    recs = json.load(open(path))
    for cls, rec in recs.items():
        src = os.path.join(ROOT, rec["source"])
        assert 0.9 < rec["traffic_over_algorithmic"] < 1.2, cls
        if bench.source_sha(src, rec.get("region")) == rec["source_sha"]:
            assert bench.traffic_record(cls, 1e8) == round(rec["traffic_over_algorithmic"] * 1e8)
        else:
            assert bench.traffic_record(cls, 1e8) is None


def test_source_region_hash_ignores_edits_outside(tmp_path):
    f = tmp_path / "k.cu"
    f.write_text("head\n// A\nkernel body\n// B\ntail\n")
    h = bench.source_sha(str(f), ["// A", "// B"])
    f.write_text("changed head\n// A\nkernel body\n// B\nchanged tail\n")
    assert bench.source_sha(str(f), ["// A", "// B"]) == h
    f.write_text("head\n// A\nkernel body changed\n// B\ntail\n")
    assert bench.source_sha(str(f), ["// A", "// B"]) != h
