"""Write the oracle's converged solution of the benchmark workload -- Cook's
membrane P2 64x64x8 (848,691 DoF), nu = 0.3, load step 1 of 5 from rest --
to cook_p2_64x64x8_step1.npz, for the error against the FP64 oracle that the
benchmark reports for each method and precision.

Calls only the CPU oracle: Newton-Krylov with the AMG-preconditioned GMRES
at ksp_rtol 1e-8 (each Newton step then cuts the residual by about 1e-8 on
top of the quadratic term) to ||R||/||R0|| <= 1e-11, just above the FP64
residual floor of these meshes (near 2e-12) and far below the benchmark's
1e-8.  The solution of R(d) = 0 on this
load path does not depend on the method, so every method's result is
compared with it.  Single-threaded FP64: minutes.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "cook_p2_64x64x8_step1.npz")


def main():
    w = W.cook(64, 64, 8, order=2, nu=0.3)
    m = O.Mesh(w)
    load, tm = w["steps"][0]
    m.set_load(load, tm)
    t0 = time.time()
    d, st = m.solve("NK", np.zeros(m.ndof), tol=1e-11, max_it=20,
                    opts=dict(ksp_rtol=1e-8, ksp_atol=0.0, ksp_restart=100, ksp_max_it=3000, pc_type=1))
    meta = dict(workload="cook_p2_64x64x8", nu=0.3, load_step="1 of 5", method="NK", pc="amg", ksp_rtol=1e-8,
                tol=1e-11, status=int(st["status"]), nit=int(st["nit"]), lit_total=int(st["lit_total"]),
                res_hist=[float(x) for x in st["res_hist"]], wall_s=round(time.time() - t0, 1))
    np.savez_compressed(OUT, d=d, meta=json.dumps(meta))
    print(json.dumps({k: v for k, v in meta.items() if k != "res_hist"}), meta["res_hist"])


if __name__ == "__main__":
    main()
