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


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--methods", default="iB")
    p.add_argument("--restart", type=int, default=50)
    p.add_argument("--precision", default="mixed_fp32", choices=["fp64", "mixed_fp32", "mixed_bf16"])
    p.add_argument("--nu", type=float, default=0.3)
    p.add_argument("--traction", type=float, default=1.0)
    p.add_argument("--mesh", default="64,64,8")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-iters", type=int, default=20)
    return p.parse_args()


def workload(args):
    import workloads as W
    nx, ny, nz = (int(v) for v in args.mesh.split(","))
    w = W.cook(nx, ny, nz, order=2, nu=args.nu, traction_scale=args.traction)
    return w, f"cook_p2_{nx}x{ny}x{nz}"


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


def traffic_record(kernel_class):
    """ncu DRAM traffic per launch recorded in profiles/traffic.json, valid only
    while the kernel source it was taken on is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel_class)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return rec if h == rec.get("source_sha") else None


def cpu_baseline_sample(w, args, gpu_stats, method_list):
    """Time the oracle on a bounded sample of the same workload and express it
    in solves/s using the GPU run's own iteration structure (nit, Krylov
    iterations per GMRES solve).  Sample: one residual assembly, one tangent
    assembly and one GMRES cycle of cpu_sample_iters iterations."""
    import numpy as np
    import oracle as O
    m = O.Mesh(w)
    load = w["steps"][0][0]
    m.set_load(load)
    d = np.zeros(m.ndof)
    m.apply_dirichlet(d)
    t0 = time.perf_counter()
    r, _ = m.residual(d)
    t_res = time.perf_counter() - t0
    t0 = time.perf_counter()
    m.tangent(d)
    t_tan = time.perf_counter() - t0
    its = args.cpu_sample_iters
    t0 = time.perf_counter()
    m.gmres(-r, rtol=0.0, atol=0.0, restart=500, max_it=its)
    t_gm = time.perf_counter() - t0
    t0 = time.perf_counter()
    m.gmres(-r, rtol=0.0, atol=0.0, restart=500, max_it=max(its // 4, 1))
    t_gm4 = time.perf_counter() - t0
    # per-iteration cost a + b*j from the two samples (j = Arnoldi step index)
    n1, n2 = max(its // 4, 1), its
    s1, s2 = n1 * (n1 - 1) / 2, n2 * (n2 - 1) / 2
    # t(n) = a*n + b*n(n-1)/2 through both samples: a = SpMV + preconditioner
    # + vector work per iteration, b = one MGS dot/axpy pair
    A = np.array([[n1, s1], [n2, s2]])
    a_, b_ = np.linalg.solve(A, np.array([t_gm4, t_gm]))
    a_, b_ = max(a_, 0.0), max(b_, 0.0)
    total = 0.0
    for meth in method_list:
        st = gpu_stats[meth]
        nit = st["nit"]
        t = (nit + 1) * t_res + st["assemblies"] * t_tan
        for L in st["lit_hist"][1:nit + 1]:
            L = int(L)
            while L > 0:  # restart cycles of at most args.restart iterations
                c = min(L, args.restart)
                t += a_ * c + b_ * c * (c - 1) / 2
                L -= c
        total += t
    value = len(method_list) / total
    sample = (f"oracle on the same Cook P2 workload: 1 residual ({t_res:.2f} s), 1 tangent ({t_tan:.2f} s), "
              f"GMRES cycles of {n1} and {n2} iterations ({t_gm4:.2f} s, {t_gm:.2f} s); solves/s from these "
              f"per-part times and the GPU run's nit / Krylov iterations per solve")
    return dict(value=value, unit="solves/s", cores=1, kind="oracle", sample=sample,
                modelled_solve_s=total / len(method_list))


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    w, name = workload(args)
    import numpy as np
    import oracle as O
    m = O.Mesh(w)
    load = w["steps"][0][0]
    m.set_load(load)
    its = args.cpu_sample_iters

    def step():
        d = np.zeros(m.ndof)
        m.apply_dirichlet(d)
        r, _ = m.residual(d)
        m.tangent(d)
        m.gmres(-r, rtol=0.0, atol=0.0, restart=500, max_it=its)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    # one sample step = one Newton iteration's assembly plus `its` Krylov
    # iterations; expressed as solves/s of a solve that needed exactly that work
    value = args.steps / el
    out = dict(impl="reference", metric=METRIC, value=value, unit="solves/s", n_gpus=args.gpus,
               steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * el / args.steps,
               higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
               config=dict(workload=name, nu=args.nu, traction=args.traction, load_step="1/5",
                           sample=f"residual + tangent + {its} GMRES iterations per step"),
               cpu_baseline=dict(kind="oracle", cores=1, value=value,
                                 sample=f"each step: 1 residual, 1 tangent, {its} GMRES iterations (one Newton "
                                        f"iteration of a truncated solve)"),
               e2e=dict(value=value, unit="solves/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    world, rank, local = dist_env()
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
    load = w["steps"][0][0]
    m.set_load(load)
    opts = dict(precision=args.precision, ksp_restart=args.restart)
    dev = torch.device("cuda", local)
    d = torch.zeros(m.ndof, dtype=torch.float64, device=dev)
    stats = {}

    def step(collect=False):
        for meth in methods:
            d.zero_()
            _, st = m.solve(meth, d, tol=TOL, opts=opts)
            if st["status"] != 0:
                raise RuntimeError(f"{meth} did not converge: status {st['status']} after {st['nit']} its")
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
    ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    solves = args.steps * len(methods) * world
    value = solves / (ms / 1e3)

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
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    if rank == 0:
        pk, src = peaks()
        timed = {k: v for k, v in prof.items() if v["timed"] > 0}
        dom = max(timed, key=lambda k: timed[k]["ms"])
        tot_ms = sum(v["ms"] for v in timed.values())
        dv = timed[dom]
        achieved = dv["bytes"] / (dv["ms"] / 1e3) / 1e9
        tr = traffic_record(dom)
        roof = dict(kernel=dom, bound="hbm", achieved=round(achieved, 1), peak=pk["hbm_gbs"], unit="GB/s",
                    frac=round(achieved / pk["hbm_gbs"], 4),
                    traffic=None if tr is None else tr["bytes_per_launch"],
                    peak_source=f"{src} STREAM-style copy",
                    avg_launch_us=round(1e3 * dv["ms"] / dv["timed"], 2),
                    share_of_kernel_time=round(dv["ms"] / tot_ms, 3),
                    algorithmic_bytes_per_launch=round(dv["bytes"] / dv["timed"]))
        per_method = {}
        for meth in methods:
            sts = stats[meth]
            per_method[meth] = dict(nit=sts[-1]["nit"], lit=sts[-1]["lit_total"],
                                    assemblies=sts[-1]["assemblies"],
                                    time_to_tol_s=sorted(s["time_s"] for s in sts)[len(sts) // 2],
                                    rrel=sts[-1]["rfinal"] / sts[-1]["r0"])
        launches = sum(v["launches"] for v in prof.values())
        out = dict(metric=METRIC, value=round(value, 4), unit="solves/s", n_gpus=world, steps=args.steps,
                   warmup=args.warmup, ms_per_step=round(ms / args.steps, 3), higher_is_better=True,
                   scaling="weak", vs_baseline=None,
                   dtype="f64" if args.precision == "fp64" else ("f32+f64" if args.precision == "mixed_fp32"
                                                                 else "bf16+f32+f64"),
                   data="synthetic",
                   config=dict(workload=name, dofs=m.ndof, blocks=m.nnzb, nu=args.nu, traction=args.traction,
                               load_step="1/5 from rest", methods=methods, precision=args.precision, tol=TOL,
                               ksp_restart=args.restart,
                               l2="working set > L2 (tangent and Krylov basis), no flush",
                               parallelism=f"replicas x{world}"),
                   methods=per_method, roofline=roof,
                   kernels={k: dict(launches=v["launches"], ms=round(v["ms"], 3),
                                    gbs=round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1)) for k, v in prof.items()},
                   gpu_launches=launches, clocks=clocks,
                   e2e=dict(value=round(solves / e2e_s, 4), unit="solves/s", h2d_bytes_per_step=8 * m.ndof * len(methods),
                            d2h_bytes_per_step=8 * m.ndof * len(methods)))
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_sample(w, args, {k: v[-1] for k, v in stats.items()}, methods)
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
