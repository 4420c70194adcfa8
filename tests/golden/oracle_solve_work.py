"""Record the oracle's own full solve of the benchmark workload -- Cook P2
64x64x8, nu = 0.3, load step 1 of 5 from rest, inexact BFGS with the AMG
preconditioner, GMRES restart 50, ||R||/||R0|| < 1e-8 -- into
oracle_solve_work.json: its iteration structure (nonlinear iterations,
tangent assemblies, Krylov iterations per GMRES solve), the time at the end
of every nonlinear iteration, the wall time and the host it ran on.

Calls only the CPU oracle.  bench.py scales its timed sample of the same
solve (its first two nonlinear iterations) to a full solve with the
recorded iteration count, and states this record's measured full-solve time
beside it.  Single-threaded FP64: minutes.
"""
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def main(method="iB", restart=50, pc="amg"):
    w = W.cook(64, 64, 8, order=2, nu=0.3)
    m = O.Mesh(w)
    load, tm = w["steps"][0]
    m.set_load(load, tm)
    t0 = time.time()
    d, st = m.solve(method, np.zeros(m.ndof), tol=1e-8,
                    opts=dict(ksp_restart=restart, pc_type={"bj": 0, "amg": 1}[pc]))
    out = dict(workload="cook_p2_64x64x8", nu=0.3, load_step="1 of 5", method=method, pc=pc, ksp_restart=restart,
               tol=1e-8, status=int(st["status"]), nit=int(st["nit"]), assemblies=int(st["assemblies"]),
               lit_total=int(st["lit_total"]), lit_hist=[int(x) for x in st["lit_hist"]],
               res_hist=[float(x) for x in st["res_hist"]],
               time_hist=[round(float(x), 3) for x in st["time_hist"]], wall_s=round(time.time() - t0, 1),
               host=dict(machine=platform.machine(), cores=os.cpu_count(), threads_used=1))
    with open(os.path.join(HERE, "oracle_solve_work.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k not in ("lit_hist", "res_hist", "time_hist")}))


if __name__ == "__main__":
    main()
