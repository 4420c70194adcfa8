"""Benchmark of the nonlinear-solve hot path on GB300.

One step = one quasi-static load step of Cook's membrane, P2 tetrahedra,
64x64x8 hexes (196,608 tets, 848,691 DoF, 7,773,249 3x3 blocks), solved from
rest to ||R||/||R0|| < 1e-8 by each of the methods in --methods (default iB,
inexact BFGS, which runs every part of the hot path: residual and tangent
assembly, GMRES with block-CSR SpMV, block-Jacobi and MGS Arnoldi, the L-BFGS
two-loop and secant update, the basic line search and the residual test).
The metric is nonlinear solves per second (one nl_solve = one load step).

Inputs are synthetic (deterministic mesh generator); the mesh, pattern and
workspace are resident in HBM before the timed region; the timed working set
(tangent 280-560 MB, Krylov basis 3.4 GB) is far larger than L2, so no flush
is needed between steps.

After the timed region the line adds, measured outside it: each method in
FP64 and mixed precision with its error against the FP64 oracle's solution,
the other configurations (Cook P1, the twist, the cardiac shell quasi-static
and as an elastodynamic heartbeat) and a bounded sample of the serving mix
(--serve-sample requests up to --serve-sample-max-dofs unknowns); --serve N
prints the serving mix alone as the line.

Multi-GPU: replicas only -- every rank solves its own copy of the workload on
its own GPU, no data-path collective; value = solves of all ranks / max time.

--impl reference times the CPU oracle (plain single-threaded FP64 C) on a
bounded sample of the same workload, on rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "nonlinear solves/sec & time-to-||R||/||R0||<1e-8, NK/iNK/B/iB; p50/p99; HBM %"
TOL = 1e-8
FP64_PEAK_TFLOPS = 1.25


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--methods", default="iB")
    p.add_argument("--restart", type=int, default=50)
    p.add_argument("--orthog", type=int, default=2, choices=[0, 1, 2],
                   help="Arnoldi: 0 sequential MGS sweep (paper), 1 low-synchronisation MGS, "
                        "2 blocked MGS (8 basis vectors per grid reduction)")
    p.add_argument("--precision", default="mixed_fp32", choices=["fp64", "mixed_fp32", "mixed_bf16"])
    p.add_argument("--ib-adaptive", type=int, default=0, choices=[0, 1],
                   help="iB: Eisenstat-Walker type adaptive H0 tolerance (an extension; 0 = the paper's fixed 1e-2)")
    p.add_argument("--pc", default="amg", choices=["bj", "amg", "amg_bf16"],
                   help="displacement-block preconditioner: nodal block-Jacobi or the AMG V-cycle")
    p.add_argument("--nu", type=float, default=0.3)
    p.add_argument("--traction", type=float, default=1.0)
    p.add_argument("--mesh", default="64,64,8")
    p.add_argument("--workload", default="cook", choices=["cook", "cook1", "twist", "heart"],
                   help="cook: Cook P2 (--mesh hexes); cook1: Cook P1 8x8x2; twist: Taylor-Hood cube 32^3; "
                        "heart: prolate shell, 149,760 P1 tets")
    p.add_argument("--twist-material", default="neo_hookean", choices=["neo_hookean", "polyconvex"],
                   help="twist: Taylor-Hood neo-Hookean stand-in, or the paper's polyconvex potential")
    p.add_argument("--twist-pressure", default="P1", choices=["P1", "P0"],
                   help="twist pressure space: P1 (Taylor-Hood) or P0 (the paper's P2-P0 pair)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--no-matrix", action="store_true",
                   help="skip the methods x precisions matrix measured after the timed region")
    p.add_argument("--serve", type=int, default=0,
                   help="serving mix: number of requests of the seeded Poisson stream (0 = off)")
    p.add_argument("--serve-max-dofs", type=float, default=5e4)
    p.add_argument("--serve-slots", type=int, default=64)
    p.add_argument("--serve-batch-dofs", type=float, default=1e3,
                   help="serving: requests up to this size run in shared launches (0: never)")
    p.add_argument("--serve-rate", type=float, default=4.0,
                   help="offered load: arrival rate as a multiple of the measured one-at-a-time capacity "
                        "(above 1 the queue fills and the served rate is the server's capacity)")
    p.add_argument("--serve-precision", default="mixed_fp32", choices=["fp64", "mixed_fp32"])
    p.add_argument("--serve-sample", type=int, default=32,
                   help="requests of the serving mix measured after the timed region of the default line "
                        "(sizes up to --serve-sample-max-dofs; 0 = off)")
    p.add_argument("--serve-sample-max-dofs", type=float, default=4e3)
    return p.parse_args()


def workload(args):
    """The synthetic workload of the run and its name (sizes in the name)."""
    import workloads as W
    if args.workload == "cook1":
        return W.cook(8, 8, 2, order=1, nu=args.nu, traction_scale=args.traction), "cook_p1_8x8x2"
    if args.workload == "twist":
        w = W.twist(32, order=2, material=args.twist_material, pressure=args.twist_pressure)
        return w, w["name"] + ("_polyconvex" if args.twist_material == "polyconvex" else "")
    if args.workload == "heart":
        return W.heart(), "heart_p1_4x80x78"
    nx, ny, nz = (int(v) for v in args.mesh.split(","))
    w = W.cook(nx, ny, nz, order=2, nu=args.nu, traction_scale=args.traction)
    return w, f"cook_p2_{nx}x{ny}x{nz}"


PC_NAMES = {"bj": "nodal block-Jacobi", "amg": "AMG V-cycle", "amg_bf16": "AMG V-cycle, BF16 fine-level smoother"}
ORTHOG_NAMES = ["mgs", "mgs_lowsync", "mgs_blocked"]


def line_config(args, w, name, dofs, blocks, methods, world):
    """`config` of both arms' lines: the workload and the solve it asks for
    (how an arm computes it -- precision, orthogonalisation -- is its
    `solver`)."""
    return dict(workload=name, dofs=int(dofs), blocks=int(blocks), nu=args.nu, traction=args.traction,
                load_step=f"step 1 of {len(w['steps'])} from rest", methods=list(methods), tol=TOL,
                ksp_restart=args.restart, preconditioner=PC_NAMES[args.pc],
                ib_h0_tolerance="adaptive (extension)" if args.ib_adaptive else "fixed",
                l2="working set > L2 (tangent and Krylov basis), no flush", parallelism=f"replicas x{world}")


def world_reduce(x, dist=None, device="cpu", op="max"):
    """x reduced over the ranks of the job (max or sum); x itself without a
    process group.  The timed region's duration is the max over ranks and
    the solves are summed, so `value` is whole-job throughput."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(converged_local, ms_local, dist=None, device="cpu"):
    """(solves of all ranks, max duration over ranks in ms, solves/s)."""
    ms = world_reduce(ms_local, dist, device, "max")
    solves = world_reduce(converged_local, dist, device, "sum")
    return solves, ms, solves / (ms / 1e3)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def traffic_record(kernel_class, algorithmic_bytes_per_launch):
    """DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
    the ncu capture recorded in profiles/traffic.json, as the measured
    traffic/algorithmic-bytes ratio of the captured launch times this run's
    average algorithmic bytes per launch (traffic grows in proportion to the
    basis vectors a step reads).  None once the kernels' source has changed
    since the capture (sha256 of their source region recorded with it)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel_class)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    try:
        h = source_sha(os.path.join(ROOT, rec["source"]), rec.get("region"))
    except (OSError, ValueError):
        return None
    if h != rec.get("source_sha"):
        return None
    return round(rec["traffic_over_algorithmic"] * algorithmic_bytes_per_launch)


def source_sha(path, region=None):
    """sha256 (16 hex digits) of a source file, or of the part of it from the
    line region[0] up to the line region[1] (the kernels of one class and
    their device helpers), so edits elsewhere in the file keep the record."""
    text = open(path, "rb").read()
    if region:
        a = text.index(region[0].encode())
        text = text[a:text.index(region[1].encode(), a)]
    return hashlib.sha256(text).hexdigest()[:16]


ORACLE_WORK = os.path.join(ROOT, "tests", "golden", "oracle_solve_work.json")
ORACLE_SOLUTION = os.path.join(ROOT, "tests", "golden", "cook_p2_64x64x8_step1.npz")
SAMPLE_ITS = 2  # nonlinear iterations of the oracle's timed sample


def oracle_pc(pc):
    """The oracle's preconditioner for a GPU preconditioner choice: its AMG
    is FP64 throughout, the counterpart of both GPU AMG variants."""
    return "amg" if pc == "amg_bf16" else pc


def oracle_work(name, method, restart, pc):
    """The oracle's own full solve of this workload (written by
    tests/golden/oracle_solve_work.py, which calls only the oracle): its
    iteration structure, per-iteration times and wall time, or None when not
    recorded for this workload, method, restart and preconditioner."""
    try:
        rec = json.load(open(ORACLE_WORK))
    except (OSError, ValueError):
        return None
    if (rec.get("workload") != name or rec.get("method") != method or rec.get("ksp_restart") != restart
            or rec.get("pc") != oracle_pc(pc) or rec.get("status") != 0):
        return None
    return rec


def scaled_solve_s(time_hist, lit_hist, lit_total):
    """Full-solve time from the timed first two iterations of the same
    solve: the first iteration (which also assembles the tangent and sets up
    the preconditioner) plus the second iteration's cost per Krylov
    iteration times the Krylov iterations of all later iterations (the cost
    of an iteration follows its Krylov iterations; lit_hist and lit_total
    from the oracle's own full solve)."""
    t1, t2 = float(time_hist[1]), float(time_hist[2])
    return t1 + (t2 - t1) * (lit_total - lit_hist[1]) / max(lit_hist[2], 1)


def oracle_sample(w, method, restart, pc):
    """The oracle's solve of the workload, stopped after its first
    SAMPLE_ITS nonlinear iterations: per-iteration times (time_hist)."""
    import numpy as np
    import oracle as O
    m = O.Mesh(w)
    load, tm = w["steps"][0]
    m.set_load(load, tm)
    t0 = time.perf_counter()
    _, st = m.solve(method, np.zeros(m.ndof), tol=TOL, max_it=SAMPLE_ITS,
                    opts=dict(ksp_restart=restart, pc_type={"bj": 0, "amg": 1}[oracle_pc(pc)]))
    return dict(time_hist=[float(x) for x in st["time_hist"]], lit=int(st["lit_total"]), nit=int(st["nit"]),
                wall_s=time.perf_counter() - t0)


def cpu_baseline_from(sample, rec, name, method, pc):
    """cpu_baseline of the JSON line: the timed sample scaled to solves/s
    with the oracle's own iteration count, and its measured full solve."""
    nit = rec["nit"]
    t_full = scaled_solve_s(sample["time_hist"], rec["lit_hist"], rec["lit_total"])
    th = sample["time_hist"]
    return dict(value=round(1.0 / t_full, 6), unit="solves/s", cores=1, kind="oracle",
                sample=(f"oracle (plain FP64 C, 1 thread) {method} with the {oracle_pc(pc).upper()} preconditioner on {name}, "
                        f"stopped after its first {SAMPLE_ITS} nonlinear iterations ({th[1]:.1f} s and "
                        f"{th[2]:.1f} s from the start; the first includes the tangent and the preconditioner "
                        f"setup), scaled to a full solve by Krylov work (the oracle's own full solve: {nit} "
                        f"nonlinear, {rec['lit_total']} Krylov iterations): {t_full:.1f} s per solve"),
                scaled_solve_s=round(t_full, 1),
                measured_full_solve=dict(wall_s=rec["wall_s"], nit=nit, lit=rec["lit_total"], host=rec.get("host"),
                                         note="the oracle's full solve recorded by tests/golden/oracle_solve_work.py"))


def run_oracle_sample(args):
    """--oracle-sample: print the oracle's timed sample as one JSON line."""
    w, name = workload(args)
    method = [m.strip() for m in args.methods.split(",") if m.strip()][0]
    print(json.dumps(dict(name=name, method=method, **oracle_sample(w, method, args.restart, args.pc))), flush=True)


def start_oracle_sample(args):
    """The CPU baseline runs beside the GPU work in a process of its own
    (started before the first CUDA call)."""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--methods", args.methods, "--restart",
           str(args.restart), "--pc", args.pc, "--mesh", args.mesh, "--nu", str(args.nu), "--traction",
           str(args.traction), "--workload", args.workload]
    return subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)


REF_KRYLOV_ITS = 10  # Krylov iterations timed per reference step


def run_reference(args):
    """The oracle as the reference arm.  Its full solve of this workload
    takes minutes (single-threaded FP64), so every step times a bounded
    sample of it -- one residual evaluation and REF_KRYLOV_ITS iterations of
    the preconditioned GMRES on the tangent of d_0 -- and the step's solve
    time is these per-part times combined with the iteration structure of
    the oracle's own full solve (nonlinear iterations, Krylov iterations),
    plus the tangent assembly and preconditioner setup timed once before the
    steps.  ms_per_step is the measured wall time of one sample, value the
    scaled solve rate.  Warm-up steps run the small Cook P1 8x8x2 solve (CPU
    code needs no warming)."""
    world, rank, local = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle as O
    import workloads as W
    w, name = workload(args)
    method = [m.strip() for m in args.methods.split(",") if m.strip()][0]
    rec = oracle_work(name, method, args.restart, args.pc)
    if rec is None:
        print(json.dumps(dict(impl="reference", unavailable=f"no recorded oracle solve of {name} {method} "
                                                            f"restart {args.restart} pc {args.pc}")), flush=True)
        return
    for _ in range(args.warmup):
        wc = W.cook(8, 8, 2, order=1, nu=args.nu)
        mc = O.Mesh(wc)
        mc.set_load(wc["steps"][0][0])
        mc.solve(method, np.zeros(mc.ndof), opts=dict(pc_type={"bj": 0, "amg": 1}[oracle_pc(args.pc)]))
    m = O.Mesh(w)
    load, tm = w["steps"][0]
    m.set_load(load, tm)
    d = m.apply_dirichlet(np.zeros(m.ndof))
    r, _ = m.residual(d)
    m.set_pc(oracle_pc(args.pc))
    t0 = time.perf_counter()
    m.tangent(d)
    t_setup = time.perf_counter() - t0
    t_model, t_wall = 0.0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        m.residual(d)
        t_res = time.perf_counter() - t0
        t0 = time.perf_counter()
        m.gmres(-r, rtol=0.0, atol=0.0, restart=args.restart, max_it=REF_KRYLOV_ITS)
        t_kry = (time.perf_counter() - t0) / REF_KRYLOV_ITS
        t_wall += t_res + t_kry * REF_KRYLOV_ITS
        t_model += rec["assemblies"] * t_setup + (rec["nit"] + 1) * t_res + rec["lit_total"] * t_kry
    value = args.steps / t_model
    sample = (f"each step: oracle (plain FP64 C, 1 thread) residual and {REF_KRYLOV_ITS} {oracle_pc(args.pc).upper()}-"
              f"preconditioned GMRES iterations on {name}; solve time = tangent + preconditioner setup "
              f"({t_setup:.1f} s, timed once) + {rec['nit'] + 1} residuals + {rec['lit_total']} Krylov iterations "
              f"(the oracle's own full {method} solve), scaled from these per-part times; the oracle's measured "
              f"full solve took {rec['wall_s']} s on {rec.get('host', {}).get('machine', '?')}")
    # ms_per_step is the wall time of one timed sample (what the run spent per
    # step); value is the solve rate scaled from the samples' per-part times
    out = dict(impl="reference", metric=METRIC, value=round(value, 6), unit="solves/s", n_gpus=args.gpus,
               steps=args.steps, warmup=args.warmup, ms_per_step=round(1e3 * t_wall / args.steps, 1),
               step=(f"one bounded sample of the solve: 1 residual and {REF_KRYLOV_ITS} Krylov iterations "
                     f"(value scales it to a full solve)"),
               scaled_solve_s=round(t_model / args.steps, 1),
               higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
               config=line_config(args, w, name, m.ndof, m.nnzb, [method], world),
               solver=dict(precision="fp64", orthog="mgs",
                           preconditioner=f"{oracle_pc(args.pc).upper()} (FP64 throughout)"),
               cpu_baseline=dict(kind="oracle", cores=1, value=round(value, 6), unit="solves/s", sample=sample,
                                 scaled_solve_s=round(t_model / args.steps, 1),
                                 measured_full_solve=dict(wall_s=rec["wall_s"], host=rec.get("host"))),
               e2e=dict(value=round(value, 6), unit="solves/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(out), flush=True)


def serving_workload(req, max_dofs):
    """Request of the seeded stream -> (workload, method, load, time, name).

    Sizes are log-uniform in [1e3, max_dofs] DoF, snapped to the nearest
    structured resolution of the family; every request is solved by iNK (the
    method that converges on all three families from rest at the stream's
    load scales: inexact BFGS diverges on Cook beyond about 2x the traction
    and on the incompressible twist, as in the paper).  Cook and twist solve
    their first load step, the cardiac shell its first time step."""
    import workloads as W
    target = min(req["dofs"], max_dofs)
    fam = req["family"]
    if fam == 0:
        best = min(range(2, 90), key=lambda n: abs(3 * (2 * n + 1) ** 2 * (2 * max(1, n // 8) + 1) - target))
        w = W.cook(best, best, max(1, best // 8), order=2, nu=req["nu"], traction_scale=req["load"])
        return w, "iNK", w["steps"][0][0], 0.0, f"cook_p2_{best}"
    if fam == 1:
        best = min(range(2, 40), key=lambda n: abs(3 * (2 * n + 1) ** 3 + (n + 1) ** 3 - target))
        w = W.twist(best, order=2)
        return w, "iNK", w["steps"][0][0], 0.0, f"twist_{best}"
    def hdofs(f):
        return 3 * (max(2, round(4 * f)) + 1) * max(8, round(80 * f)) * (max(6, round(78 * f)) + 1)
    best = min((s / 32 for s in range(2, 320)), key=lambda f: abs(hdofs(f) - target))
    nr, nc, nl = max(2, round(4 * best)), max(8, round(80 * best)), max(6, round(78 * best))
    w = W.heart(nr=nr, nc=nc, nl=nl)
    load, tm = w["steps"][0]
    return w, "iNK", load, tm, f"heart_{nr}x{nc}x{nl}"


def run_serving(args):
    """--serve N: the serving mix as the JSON line (see serve_mix)."""
    out = serve_mix(args.serve, args.serve_max_dofs, args.serve_slots, args.serve_batch_dofs, args.serve_rate,
                    args.serve_precision, args.restart, args.orthog, per_request=True)
    print(json.dumps(out), flush=True)


def serve_mix(nreq, max_dofs, slots, batch_dofs, rate, precision, restart, orthog, per_request=False):
    """Serving mix: the seeded Poisson stream served with continuous batching
    in the mixed form (small requests in shared launches, the rest on their
    own streams), against the plain FP64 solve of each request one at a time;
    arrivals at `rate` times the one-at-a-time capacity.  Both forms solve to
    the same relative residual; each served result's difference from the
    FP64 solution is reported (per request on stderr with per_request)."""
    import numpy as np
    import torch
    import paper_2203_05610_gb300 as fe
    import workloads as W
    reqs = W.serving_stream(nreq=nreq)
    jobs = [serving_workload(r, max_dofs) for r in reqs]
    base = dict(ksp_restart=restart, orthog=orthog)
    bopts = dict(base, precision="fp64")
    sopts = dict(base, precision=precision)
    # plain FP64 one at a time (also warms up the library)
    t_solo, solo_st, solo_x = [], [], []
    for w, meth, load, tm, _ in jobs:
        m = fe.Mesh(w)
        m.set_load(load, tm)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d, st = m.solve(meth, m.zeros(), tol=TOL, opts=bopts)
        torch.cuda.synchronize()
        t_solo.append(time.perf_counter() - t0)
        solo_st.append(st["status"])
        solo_x.append(d.cpu().numpy())
        m.close()
    solo_ok = sum(1 for x in solo_st if x == 0)
    cap = solo_ok / sum(t_solo)
    # arrivals: the stream's exponential gaps rescaled to rate x capacity
    arr = np.array([r["arrival"] for r in reqs])
    arr = (arr - arr[0]) / (arr[-1] - arr[0] + 1e-12) * (len(jobs) / (rate * cap))
    srv = fe.Server(max_active=slots, batch_max_dofs=int(batch_dofs) if batch_dofs else -1)
    t0 = srv.clock()
    ids = []
    for (w, meth, load, tm, _), a in zip(jobs, arr):
        while srv.clock() - t0 < a:
            time.sleep(min(0.002, max(0.0, a - (srv.clock() - t0))))
        ids.append(srv.submit(w, meth, tol=TOL, opts=sopts, load=load, time=tm))
    res = [srv.poll(i, wait=True) for i in ids]
    tune = srv.tuning()
    srv.close()
    done = [r for r in res if r["state"] == "done" and r["result"] == 0]
    span = max(r["t_end"] for r in res) - t0
    lat = np.sort([r["t_end"] - r["t_submit"] for r in done])
    solo = np.sort(t_solo)
    diffs = []
    for (w, meth, load, tm, name), ts, ss, xs, r in zip(jobs, t_solo, solo_st, solo_x, res):
        rd = None
        if r["state"] == "done" and r["result"] == 0 and ss == 0:
            rd = float(np.linalg.norm(r["d"] - xs) / max(np.linalg.norm(xs), 1e-300))
            diffs.append(rd)
        if not per_request:
            continue
        print(json.dumps(dict(request=name, ndof=r["ndof"], solo_fp64_s=round(ts, 4), solo_status=int(ss),
                              served_state=r["state"], served_result=r["result"],
                              served_run_s=round(r["t_end"] - r["t_start"], 4),
                              latency_s=round(r["t_end"] - r["t_submit"], 4), rel_diff_vs_fp64=rd)),
              file=sys.stderr)
    eligible = sum(1 for w, *_ in jobs if w["pressure_order"] == 0) if batch_dofs else 0
    out = dict(metric=METRIC, value=round(len(done) / span, 4), unit="solves/s", n_gpus=1, steps=len(jobs),
               warmup=0, ms_per_step=round(1e3 * span / len(jobs), 3), higher_is_better=True, scaling="weak",
               vs_baseline=None, dtype="f32+f64" if precision == "mixed_fp32" else "f64",
               data="synthetic",
               config=dict(workload="serving_mix", requests=len(jobs), seed=20220311,
                           dofs_range=[1e3, max_dofs], slots=slots,
                           batch_max_dofs=batch_dofs, ksp_restart=restart,
                           orthog=["mgs", "mgs_lowsync", "mgs_blocked"][orthog], method="iNK",
                           preconditioner="nodal block-Jacobi", tol=TOL,
                           arrival_rate_x_capacity=rate, precision=precision,
                           families={n: sum(1 for j in jobs if j[4].startswith(n)) for n in ("cook", "twist", "heart")},
                           displacement_form_requests=eligible),
               p50_latency_s=round(float(np.percentile(lat, 50)), 4) if len(lat) else None,
               p99_latency_s=round(float(np.percentile(lat, 99)), 4) if len(lat) else None,
               failed=len(res) - len(done),
               accuracy=dict(note="relative difference of each served solution from the plain FP64 solution, "
                                  "both at ||R||/||R0|| <= %g" % TOL,
                             median=float(np.median(diffs)) if diffs else None,
                             max=float(np.max(diffs)) if diffs else None),
               autotuner=tune,
               baseline_fp64_one_at_a_time=dict(value=round(cap, 4), unit="solves/s", failed=len(jobs) - solo_ok,
                                                 p50_solve_s=round(float(np.percentile(solo, 50)), 4),
                                                 p99_solve_s=round(float(np.percentile(solo, 99)), 4)))
    return out


VC_BOTTOM_MAXN = 256  # nodes per level that the one-block bottom of the V-cycle takes


def vcycle_kernels(sizes):
    """Kernels in one launch of the V-cycle's CUDA graph for AMG levels of
    `sizes` nodes (the composition built by vcycle_launches in fe_amg.cu):
    k_vc_init0; per level above the bottom two Chebyshev steps and a
    restriction; the one-block bottom (the levels of at most VC_BOTTOM_MAXN
    nodes below level 0, when one of them is smoothed) or the coarsest
    solve; per level above the bottom a prolongation and two Chebyshev
    steps.  One level: a conversion and the dense solve."""
    L = len(sizes)
    if L <= 1:
        return 2
    q0 = L - 1
    while q0 > 1 and sizes[q0 - 1] <= VC_BOTTOM_MAXN:
        q0 -= 1
    qf = q0 if q0 <= L - 2 else L - 1
    return 2 + 6 * qf


def oracle_solution(name):
    """The oracle's converged solution of the benchmark workload (written by
    tests/golden/oracle_reference_solution.py), or None."""
    if name != "cook_p2_64x64x8":
        return None
    try:
        import numpy as np
        return np.load(ORACLE_SOLUTION)["d"]
    except (OSError, KeyError, ValueError):
        return None


def method_matrix(m, dev, opts_base, ref, methods=("NK", "iNK", "B", "iB"), precisions=("mixed_fp32", "fp64")):
    """Each method in each precision (with the run's preconditioner), solved
    once after a warm-up solve, outside the timed region: status, nonlinear
    and Krylov iterations, time to tolerance and the relative error against
    the FP64 oracle's solution."""
    import numpy as np
    import torch
    out = {}
    d = torch.zeros(m.ndof, dtype=torch.float64, device=dev)
    for prec in precisions:
        for meth in methods:
            o = dict(opts_base, precision=prec)
            rec = None
            for rep in range(2):
                d.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, st = m.solve(meth, d, tol=TOL, opts=o)
                torch.cuda.synchronize()
                rec = dict(status=st["status"], nit=st["nit"], lit=st["lit_total"], assemblies=st["assemblies"],
                           time_to_tol_s=round(time.perf_counter() - t0, 4), rrel=st["rfinal"] / st["r0"])
            if ref is not None and rec["status"] == 0:
                x = d.cpu().numpy()
                rec["err_vs_oracle"] = float(np.linalg.norm(x - ref) / np.linalg.norm(ref))
            out[f"{meth}/{prec}"] = rec
    return out


def other_configs(dev, opts_base):
    """The other workloads of the metric, each method timed on its last of
    `reps` solves (the twist: its only solve, which includes building the
    AMG structure), outside the timed region: Cook P1 8x8x2 (FP64, all four
    methods), the Taylor-Hood twist P2-P1 32^3 (step 1 of 10, iNK and iB)
    and the cardiac shell 4x80x78 (time step 1 of 100, all four methods),
    the last two in the run's precision and preconditioner."""
    import torch
    import paper_2203_05610_gb300 as fe
    import workloads as W
    runs = [("cook_p1_8x8x2", W.cook(8, 8, 2, order=1), ("NK", "iNK", "B", "iB"), dict(opts_base, precision="fp64"), 2),
            ("twist_p2p1_32", W.twist(32, order=2), ("iNK", "iB"), opts_base, 1),
            ("heart_p1_4x80x78", W.heart(), ("NK", "iNK", "B", "iB"), opts_base, 2)]
    out = {}
    for name, w, methods, o, reps in runs:
        m = fe.Mesh(w, device=dev.index or 0)
        load, tm = w["steps"][0]
        m.set_load(load, tm)
        d = torch.zeros(m.ndof, dtype=torch.float64, device=dev)
        res = dict(dofs=m.ndof, solves_per_method=reps)
        for meth in methods:
            for rep in range(reps):
                d.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, st = m.solve(meth, d, tol=TOL, opts=o)
                torch.cuda.synchronize()
                t = time.perf_counter() - t0
            res[meth] = dict(status=st["status"], nit=st["nit"], lit=st["lit_total"], time_to_tol_s=round(t, 4),
                             rrel=st["rfinal"] / st["r0"] if st["r0"] > 0 else 0.0)
        out[name] = res
        m.close()
    return out


def dynamic_cardiac(dev, opts_base, nsteps=10, methods=("NK", "iNK", "B", "iB")):
    """The cardiac configuration (4 x 80 x 78 hexes, 149,760 P1 tets) as an
    elastodynamic heartbeat: inertia, epicardial dashpots and the follower
    endocardial pressure, nsteps Newmark steps from rest, each step
    warm-started from the last; per method the median step time, the
    nonlinear and Krylov iterations, and the final relative residuals.
    Outside the timed region of the headline line."""
    import torch
    import paper_2203_05610_gb300 as fe
    import workloads as W
    w = W.heart(dynamics=True, follower=True)
    m = fe.Mesh(w, device=dev.index or 0)
    out = dict(workload=w["name"], dofs=m.ndof, rho=w["rho"], dt=w["dt"], steps=nsteps)
    for meth in methods:
        m.set_dynamics(w["rho"], w["dt"])
        d = torch.zeros(m.ndof, dtype=torch.float64, device=dev)
        times, nits, lits, worst = [], [], [], 0.0
        ok = True
        for s in range(nsteps):
            load, tm = w["steps"][s]
            m.set_load(load, tm)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = m.solve(meth, d, tol=TOL, opts=opts_base)
            m.dynamics_advance(d)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            nits.append(st["nit"])
            lits.append(st["lit_total"])
            ok = ok and st["status"] == 0
            if st["r0"] > 0:
                worst = max(worst, st["rfinal"] / st["r0"])
        srt = sorted(times)
        out[meth] = dict(converged_all=ok, step_s_median=round(srt[len(srt) // 2], 4),
                         steps_per_s=round(nsteps / sum(times), 3), nit=nits, lit=lits, worst_rrel=worst)
    m.close()
    return out


def main():
    args = parse()
    if args.oracle_sample:
        run_oracle_sample(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.serve:
        run_serving(args)
        return
    world, rank, local = dist_env()
    cpu_proc = None
    if world == 1 and not args.no_cpu_baseline:
        cpu_proc = start_oracle_sample(args)  # a process of its own, before any CUDA call
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
    import paper_2203_05610_gb300 as fe
    w, name = workload(args)
    methods = [m.strip() for m in args.methods.split(",") if m.strip()]
    m = fe.Mesh(w, device=local)
    load, tm = w["steps"][0]
    m.set_load(load, tm)
    opts = dict(precision=args.precision, ksp_restart=args.restart, orthog=args.orthog, ib_adaptive=args.ib_adaptive,
                pc_type=args.pc)
    dev = torch.device("cuda", local)
    d = torch.zeros(m.ndof, dtype=torch.float64, device=dev)
    stats = {}

    def step(collect=False):
        for meth in methods:
            d.zero_()
            _, st = m.solve(meth, d, tol=TOL, opts=opts)
            if collect:
                stats.setdefault(meth, []).append(st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    m.profile_reset(timing=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.steps):
        step(collect=True)
    ev1.record()
    torch.cuda.synchronize()
    prof = m.profile_read()
    clocks = sampler.stop()
    # kernels per preconditioner launch: a V-cycle is one graph launch of
    # several kernels (displacement form; the u-p form's class mixes in its
    # Schur kernels)
    pc_kernels = 1
    if args.pc in ("amg", "amg_bf16") and w["pressure_order"] == 0:
        try:
            pc_kernels = vcycle_kernels(m.amg_sizes())
        except Exception:  # a count only: never fail the run over it
            pc_kernels = 1
    # only converged solves count (a solve that stops at max_it or diverges is
    # reported per method with its status)
    converged = sum(1 for meth in methods for st in stats[meth] if st["status"] == 0)
    solves, ms, value = job_throughput(converged, ev0.elapsed_time(ev1), dist, dev)
    if dist:
        dist.barrier()
    m.profile_reset(timing=False)

    # end to end through the C ABI with host buffers: pinned initial guess in,
    # solution out, every step
    h_in = torch.zeros(m.ndof, dtype=torch.float64).pin_memory()
    h_out = torch.empty(m.ndof, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for meth in methods:
            d.copy_(h_in, non_blocking=True)
            m.solve(meth, d, tol=TOL, opts=opts)
            h_out.copy_(d, non_blocking=True)
            torch.cuda.synchronize()
    e2e_s = world_reduce(time.perf_counter() - t0, dist, dev, "max")

    if rank == 0:
        import numpy as np
        ref = oracle_solution(name)
        err_headline = None
        if ref is not None:
            err_headline = float(np.linalg.norm(h_out.numpy() - ref) / np.linalg.norm(ref))
        matrix = None
        if not args.no_matrix and args.workload == "cook":
            base = dict(ksp_restart=args.restart, orthog=args.orthog, pc_type=args.pc)
            matrix = method_matrix(m, dev, base, ref)
            if args.pc == "amg":  # nodal block-Jacobi (the simpler preconditioner), for comparison
                matrix.update({k + "/block_jacobi": v for k, v in
                               method_matrix(m, dev, dict(base, pc_type="bj"), ref, methods=("iB",),
                                             precisions=("mixed_fp32",)).items()})
        dyn = others = None
        if not args.no_matrix and args.workload == "cook":
            ob = dict(ksp_restart=args.restart, orthog=args.orthog, pc_type=args.pc, precision=args.precision)
            dyn = dynamic_cardiac(dev, ob)
            others = other_configs(dev, ob)
        serving = None
        if not args.no_matrix and args.workload == "cook" and world == 1 and args.serve_sample > 0:
            srv = serve_mix(args.serve_sample, args.serve_sample_max_dofs, args.serve_slots, args.serve_batch_dofs,
                            args.serve_rate, args.serve_precision, args.restart, args.orthog)
            serving = {k: v for k, v in srv.items() if k not in ("metric", "n_gpus", "steps", "warmup",
                                                                  "higher_is_better", "scaling", "vs_baseline", "data")}
        pk, src = peaks()
        timed = {k: v for k, v in prof.items() if v["timed"] > 0}
        dom = max(timed, key=lambda k: timed[k]["ms"])
        tot_ms = sum(v["ms"] for v in timed.values())

        def hbm_line(cls):
            v = timed[cls]
            achieved = v["bytes"] / (v["ms"] / 1e3) / 1e9
            tr = traffic_record(cls, v["bytes"] / v["timed"])
            return dict(kernel=cls, bound="hbm", achieved=round(achieved, 1), peak=pk["hbm_gbs"], unit="GB/s",
                        frac=round(achieved / pk["hbm_gbs"], 4), traffic=tr,
                        peak_source=f"{src} STREAM-style copy (MEASURED_PEAKS.json)",
                        avg_launch_us=round(1e3 * v["ms"] / v["timed"], 2),
                        share_of_kernel_time=round(v["ms"] / tot_ms, 3),
                        algorithmic_bytes_per_launch=round(v["bytes"] / v["timed"]))

        def alu_line(cls):
            # FP64 dot/axpy sweeps: bound by the FP64 FMA rate (2 FMA per entry
            # per inner product), not by HBM; peak: GB300 FP64 1.25 TFLOP/s
            v = timed[cls]
            achieved = v["flops"] / (v["ms"] / 1e3) / 1e12
            line = hbm_line(cls)
            return dict(kernel=cls, bound="alu", achieved=round(achieved, 4), peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                        frac=round(achieved / FP64_PEAK_TFLOPS, 4), traffic=line["traffic"],
                        peak_source="FP64 FMA: nominal GB300 1.25 TFLOP/s (an FMA-chain probe measured 1.19)",
                        avg_launch_us=line["avg_launch_us"], share_of_kernel_time=line["share_of_kernel_time"],
                        algorithmic_bytes_per_launch=line["algorithmic_bytes_per_launch"],
                        algorithmic_flops_per_launch=round(v["flops"] / v["timed"]),
                        hbm_view=dict(achieved=line["achieved"], peak=line["peak"], unit="GB/s", frac=line["frac"]))

        roof = alu_line(dom) if dom in ("arnoldi", "twoloop") else hbm_line(dom)
        per_method = {}
        for meth in methods:
            sts = stats[meth]
            per_method[meth] = dict(status=sts[-1]["status"], converged=sum(1 for x in sts if x["status"] == 0),
                                    nit=sts[-1]["nit"], lit=sts[-1]["lit_total"],
                                    assemblies=sts[-1]["assemblies"],
                                    time_to_tol_s=sorted(s_["time_s"] for s_ in sts)[len(sts) // 2],
                                    rrel=sts[-1]["rfinal"] / sts[-1]["r0"])
            if err_headline is not None and meth == methods[-1]:
                per_method[meth]["err_vs_oracle"] = err_headline
        launches = sum(v["launches"] for v in prof.values()) + (pc_kernels - 1) * prof["pc"]["launches"]
        out = dict(metric=METRIC, value=round(value, 4), unit="solves/s", n_gpus=world, steps=args.steps,
                   warmup=args.warmup, ms_per_step=round(ms / args.steps, 3), higher_is_better=True,
                   scaling="weak", vs_baseline=None,
                   dtype="f64" if args.precision == "fp64" else ("f32+f64" if args.precision == "mixed_fp32"
                                                                 else "bf16+f32+f64"),
                   data="synthetic",
                   config=line_config(args, w, name, m.ndof, m.nnzb, methods, world),
                   solver=dict(precision=args.precision, orthog=ORTHOG_NAMES[args.orthog]),
                   methods=per_method, roofline=roof,
                   roofline_spmv=hbm_line("spmv") if "spmv" in timed else None,
                   roofline_arnoldi=alu_line("arnoldi") if "arnoldi" in timed else None,
                   kernels={k: dict(launches=v["launches"], ms=round(v["ms"], 3),
                                    gbs=round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1)) for k, v in prof.items()},
                   gpu_launches=launches, clocks=clocks,
                   e2e=dict(value=round(solves / e2e_s, 4) if converged else 0.0, unit="solves/s",
                            h2d_bytes_per_step=8 * m.ndof * len(methods),
                            d2h_bytes_per_step=8 * m.ndof * len(methods)))
        if matrix is not None:
            out["method_matrix"] = dict(note="each method in each precision solved once after a warm-up solve, "
                                             "outside the timed region; err_vs_oracle against the FP64 oracle's "
                                             "solution (tests/golden/cook_p2_64x64x8_step1.npz)", results=matrix)
        if dyn is not None:
            out["dynamic_cardiac"] = dyn
        if others is not None:
            out["other_configs"] = others
        if serving is not None:
            out["serving_mix"] = dict(note="a bounded sample (see config) of the seeded Poisson stream of Cook, "
                                           "twist and cardiac requests, "
                                           "served in the mixed form with continuous batching against the plain "
                                           "FP64 solve of each request one at a time; outside the timed region",
                                      **serving)
        if cpu_proc is not None:
            try:
                line = cpu_proc.communicate(timeout=900)[0].strip().splitlines()[-1]
                smp = json.loads(line)
                rec = oracle_work(name, smp["method"], args.restart, args.pc)
                if rec is not None:
                    out["cpu_baseline"] = cpu_baseline_from(smp, rec, name, smp["method"], args.pc)
            except (subprocess.TimeoutExpired, IndexError, ValueError) as e:
                cpu_proc.kill()
                out["cpu_baseline"] = dict(unavailable=f"oracle sample did not finish: {type(e).__name__}")
        print(json.dumps(out), flush=True)
    elif cpu_proc is not None:
        cpu_proc.kill()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
