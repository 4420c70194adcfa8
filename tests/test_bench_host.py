"""Host logic of bench.py that its JSON line depends on, without a GPU: the
oracle solve-time model behind `cpu_baseline` and the reference arm (and the
reference arm's line itself), the source-region hash that keeps
`roofline.traffic` tied to the captured kernels, the kernel count of a
V-cycle graph behind `gpu_launches`, and the serving sample's requests."""
import json
import os
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_scaled_solve_time_from_the_first_iterations():
    # the first iteration (tangent, preconditioner setup, first step) plus the
    # second iteration's cost per Krylov iteration for all later ones
    assert bench.scaled_solve_s([0.1, 30.0, 42.5], [0, 33, 10], 133) == 30.0 + 12.5 * 10


def test_recorded_oracle_structure_is_consistent():
    rec = bench.oracle_work("cook_p2_64x64x8", "iB", 50, "amg")
    assert rec is not None and rec["status"] == 0
    assert sum(rec["lit_hist"][1:rec["nit"] + 1]) == rec["lit_total"]
    assert rec["assemblies"] == 1
    th = rec["time_hist"]
    # the scaled estimate from the recorded first iterations against the recorded full solve
    est = bench.scaled_solve_s(th, rec["lit_hist"], rec["lit_total"])
    assert abs(est - th[rec["nit"]]) <= 0.1 * th[rec["nit"]], (est, th[rec["nit"]])


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


def test_vcycle_kernel_count():
    # one V-cycle graph: k_vc_init0, 2 steps + restriction per level above the
    # bottom, the bottom block or the coarsest solve, prolongation + 2 steps
    # per level above it again
    assert bench.vcycle_kernels([282897, 3799, 41, 2]) == 14  # levels 2-3 in one block
    assert bench.vcycle_kernels([9801, 147, 4]) == 8          # levels 1-2 in one block
    assert bench.vcycle_kernels([243, 13]) == 8               # level 1 is the coarsest: no bottom block
    assert bench.vcycle_kernels([21609, 323, 7]) == 14        # level 1 too large for the block
    assert bench.vcycle_kernels([12]) == 2                    # one level: conversion and dense solve


def test_serving_sample_requests_snap_to_their_sizes():
    # the bench line's serving sample: each request of the seeded stream is
    # built at the structured resolution nearest its (capped) size and solved
    # by iNK from rest
    import oracle as O
    import workloads as W
    for r in W.serving_stream(nreq=32):
        w, meth, load, tm, name = bench.serving_workload(r, 4e3)
        target = min(r["dofs"], 4e3)
        ndof = O.Mesh(w).ndof
        assert meth == "iNK" and name.split("_")[0] in ("cook", "twist", "heart")
        assert 0.7 * target <= ndof <= 1.3 * target, (name, ndof, target)
        assert (load, tm) == tuple(w["steps"][0])


def test_reference_arm_line(monkeypatch, capsys):
    # the reference arm on a small Cook P2 mesh with a stand-in solve record:
    # ms_per_step is the measured wall time of one sample, value the solve
    # rate scaled with the record's iteration structure
    rec = dict(workload="cook_p2_4x4x2", method="iB", ksp_restart=50, pc="amg", status=0, nit=6,
               assemblies=1, lit_total=60, wall_s=1.0, host=dict(machine="test"))
    monkeypatch.setattr(bench, "oracle_work", lambda *a: rec)
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()
    args.impl, args.mesh, args.steps, args.warmup = "reference", "4,4,2", 2, 0
    bench.run_reference(args)
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert out["impl"] == "reference" and out["unit"] == "solves/s" and out["steps"] == 2
    assert out["value"] > 0 and out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"] == dict(value=out["value"], unit="solves/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0)
    # a sample is one residual and REF_KRYLOV_ITS Krylov iterations; the scaled
    # solve adds the setup, nit + 1 residuals and lit_total iterations
    # the same `config` as the GPU arm's line for these arguments
    w, name = bench.workload(args)
    assert out["config"] == bench.line_config(args, w, name, out["config"]["dofs"], out["config"]["blocks"],
                                              ["iB"], 1)
    assert name == "cook_p2_4x4x2" and out["config"]["dofs"] == 3 * 9 * 9 * 5 and out["solver"]["precision"] == "fp64"
    assert 1.0 / out["value"] > out["ms_per_step"] / 1e3 > 0
    assert abs(1.0 / out["value"] - out["scaled_solve_s"]) <= 0.05 + 1e-6  # scaled_solve_s is rounded to 0.1 s
