"""ctypes binding of the plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The oracle (``oracle.c``) shares no code
with the CUDA library; see the header of ``oracle.c`` for what it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None
HIST = 1024

METHODS = {"NK": 0, "iNK": 1, "B": 2, "iB": 3}


def build(force=False):
    """Compile oracle.c into _lib/liboracle.so with gcc (plain IEEE FP64)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src),
                                             os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c99",
           "-D_DEFAULT_SOURCE", "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            D = ctypes.c_double
            I = ctypes.c_int
            L.om_create.restype = P
            L.om_create.argtypes = [I, I, I, I, P, P, P, I, P, I, P, P, P, P, P]
            L.om_destroy.argtypes = [P]
            L.om_info.argtypes = [P, P]
            L.om_topology.argtypes = [P, P, P, P, P, P]
            L.om_set_load.argtypes = [P, D, D]
            L.om_apply_dirichlet.argtypes = [P, P]
            L.om_residual.restype = D
            L.om_residual.argtypes = [P, P, P]
            L.om_energy.restype = D
            L.om_energy.argtypes = [P, P]
            L.om_tangent.argtypes = [P, P]
            L.om_tangent_copy.argtypes = [P, P, P, P]
            L.om_spmv.argtypes = [P, P, P]
            L.om_pc.argtypes = [P, P, P]
            L.om_gmres.restype = I
            L.om_gmres.argtypes = [P, P, P, D, D, I, I, P]
            L.om_solve.restype = I
            L.om_solve.argtypes = [P, I, D, I, P, P, P]
            L.om_lbfgs_apply.argtypes = [P, P, P, P, I, P, P, I]
            L.om_material.argtypes = [P, P, P, D, D, P, P, P, P]
            L.om_tet_rule.restype = I
            L.om_tet_rule.argtypes = [I, P, P]
            L.om_tri_rule.restype = I
            L.om_tri_rule.argtypes = [P, P]
            L.om_set_pc.argtypes = [P, I]
            L.om_set_dynamics.argtypes = [P, D, D]
            L.om_dynamics_set.argtypes = [P, P, P, P]
            L.om_dynamics_advance.argtypes = [P, P]
            L.om_dynamics_get.argtypes = [P, P, P]
            L.om_amg_levels.restype = I
            L.om_amg_levels.argtypes = [P]
            L.om_amg_level_info.argtypes = [P, I, P]
            L.om_amg_copy.argtypes = [P, I, P, P, P, P, P, P, P, P, P, P, P, P]
            L.om_amg_smooth.argtypes = [P, I, P, P, I]
            L.om_amg_vcycle.argtypes = [P, P, P]
            L.om_splitmix64.restype = ctypes.c_ulonglong
            L.om_splitmix64.argtypes = [ctypes.c_ulonglong]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def matp(material):
    """Material dict (workloads) -> the oracle's parameter array."""
    m = material
    a = np.zeros(15)
    a[0] = m["kind"]
    a[1] = m.get("vol_literal", 0)
    a[2] = m.get("E", 0.0)
    a[3] = m.get("nu", 0.0)
    a[4] = m.get("mu", 0.0)
    a[5] = m.get("C", 0.0)
    a[6] = m.get("bf", 0.0)
    a[7] = m.get("bt", 0.0)
    a[8] = m.get("bfs", 0.0)
    a[9] = m.get("kappa", 0.0)
    a[10] = m.get("Ta_peak", 0.0)
    a[11] = m.get("period", 1.0)
    a[12] = m.get("alpha_p", 0.0)
    a[13] = m.get("beta_p", 0.0)
    a[14] = m.get("c_log", 0.0)
    return a


def material_point(material, F, fib=None, gamma=0.0, p=0.0):
    """psi, P (3x3), A (9x9, A[3i+J, 3k+L]) and dP/dp at one point."""
    L = lib()
    mp = matp(material)
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(9)
    fb = None if fib is None else np.ascontiguousarray(fib, dtype=np.float64).reshape(9)
    psi = np.zeros(1)
    P = np.zeros(9)
    A = np.zeros(81)
    dPdp = np.zeros(9)
    L.om_material(_p(mp), _p(F), _p(fb), gamma, p, _p(psi), _p(P), _p(A), _p(dPdp))
    return psi[0], P.reshape(3, 3), A.reshape(9, 9), dPdp.reshape(3, 3)


def tet_rule(order):
    lam = np.zeros(16)
    w = np.zeros(4)
    n = lib().om_tet_rule(order, _p(lam), _p(w))
    return lam[: 4 * n].reshape(n, 4), w[:n]


def tri_rule():
    lam = np.zeros(18)
    w = np.zeros(6)
    n = lib().om_tri_rule(_p(lam), _p(w))
    return lam.reshape(n, 3), w


def splitmix64(x):
    return int(lib().om_splitmix64(int(x)))


def default_opts(method):
    """Appendix A defaults, with the readings: restart 500, m = 50."""
    o = np.zeros(14)
    o[0] = 0
    o[1] = {0: 1e-6, 1: 1e-2, 2: 0.0, 3: 1e-2}[method]
    o[2] = {0: 1e-10, 1: 1e-14, 2: 0.0, 3: 1e-14}[method]
    o[3] = 0.1
    o[4] = 0.1
    o[5] = 500
    o[6] = 10000
    o[7] = 50
    o[8] = 1e4
    o[9] = 1
    o[10] = 1  # jac_lag
    o[11] = 0  # hess_reassemble
    o[12] = 0  # ib_adaptive
    o[13] = 0  # pc_type: 0 block-Jacobi, 1 AMG
    return o


class Mesh:
    """Oracle mesh built from a workloads dict."""

    def __init__(self, w):
        L = lib()
        self._keep = []
        groups = np.zeros((max(len(w["groups"]), 1), 8))
        for g, G in enumerate(w["groups"]):
            groups[g] = [G["mask"], *G["center"], G["angle"], *G["translation"]]
        self._mp = matp(w["material"])
        arrs = [w["coords"], w["tets"], w["dir_group"], groups, w["faces"], w["face_kind"],
                w["face_data"], self._mp, w["fibers"]]
        self._keep = arrs
        nf = int(w["faces"].shape[0])
        self.h = L.om_create(w["order"], w["pressure_order"], w["coords"].shape[0],
                             w["tets"].shape[0], _p(w["coords"]), _p(w["tets"]),
                             _p(w["dir_group"]), len(w["groups"]), _p(groups), nf,
                             _p(w["faces"]), _p(w["face_kind"]), _p(w["face_data"]),
                             _p(self._mp), _p(w["fibers"]))
        info = np.zeros(7, dtype=np.int64)
        L.om_info(self.h, _p(info))
        self.nn, self.np_, self.ndof, self.nnzb, self.nnz_up, self.ncolors, self.nen = map(int, info)
        self.ne = int(w["tets"].shape[0])
        self.nv = int(w["coords"].shape[0])

    def close(self):
        if self.h:
            lib().om_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def topology(self):
        conn = np.zeros((self.ne, self.nen), dtype=np.int32)
        colors = np.zeros(self.ne, dtype=np.int32)
        rp = np.zeros(self.nn + 1, dtype=np.int32)
        col = np.zeros(self.nnzb, dtype=np.int32)
        X = np.zeros((self.nn, 3))
        lib().om_topology(self.h, _p(conn), _p(colors), _p(rp), _p(col), _p(X))
        return dict(conn=conn, colors=colors, row_ptr=rp, col=col, X=X)

    def set_load(self, load, time=0.0):
        lib().om_set_load(self.h, float(load), float(time))

    def apply_dirichlet(self, d):
        lib().om_apply_dirichlet(self.h, _p(d))
        return d

    def residual(self, d):
        d = np.ascontiguousarray(d, dtype=np.float64)
        r = np.zeros(self.ndof)
        nrm = lib().om_residual(self.h, _p(d), _p(r))
        return r, nrm

    def energy(self, d):
        d = np.ascontiguousarray(d, dtype=np.float64)
        return lib().om_energy(self.h, _p(d))

    def tangent(self, d):
        d = np.ascontiguousarray(d, dtype=np.float64)
        lib().om_tangent(self.h, _p(d))

    def tangent_copy(self):
        val = np.zeros((self.nnzb, 3, 3))
        bup = np.zeros((max(self.nnz_up, 1), 3))
        dinv = np.zeros((self.nn, 3, 3))
        lib().om_tangent_copy(self.h, _p(val), _p(bup), _p(dinv))
        return val, bup[: self.nnz_up], dinv

    def spmv(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.ndof)
        lib().om_spmv(self.h, _p(x), _p(y))
        return y

    def pc(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.ndof)
        lib().om_pc(self.h, _p(x), _p(y))
        return y

    def gmres(self, b, x0=None, rtol=1e-6, atol=1e-10, restart=500, max_it=10000):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.ndof) if x0 is None else np.array(x0, dtype=np.float64)
        res = np.zeros(1)
        it = lib().om_gmres(self.h, _p(b), _p(x), rtol, atol, restart, max_it, _p(res))
        return x, it, res[0]

    def set_pc(self, pc_type):
        """Preconditioner of the displacement block: 0 / "bj" nodal
        block-Jacobi, 1 / "amg" the AMG V-cycle (set up by tangent())."""
        lib().om_set_pc(self.h, {"bj": 0, "amg": 1}.get(pc_type, pc_type))

    def set_dynamics(self, rho, dt):
        """Newmark elastodynamics with density rho and time step dt (rho <= 0: off)."""
        lib().om_set_dynamics(self.h, float(rho), float(dt))

    def dynamics_set(self, d=None, v=None, a=None):
        n3 = 3 * self.nn
        arrs = [None if x is None else np.ascontiguousarray(x[:n3], dtype=np.float64) for x in (d, v, a)]
        lib().om_dynamics_set(self.h, *[_p(x) for x in arrs])

    def dynamics_advance(self, d):
        lib().om_dynamics_advance(self.h, _p(np.ascontiguousarray(d, dtype=np.float64)))

    def dynamics_get(self):
        v = np.zeros(3 * self.nn)
        a = np.zeros(3 * self.nn)
        lib().om_dynamics_get(self.h, _p(v), _p(a))
        return v, a

    def amg_levels(self):
        """The AMG hierarchy of the last tangent: one dict per level (A_l,
        absent components, near null space, aggregates, P and T, rho; the
        coarsest level's dense inverse)."""
        L = lib()
        out = []
        nlev = L.om_amg_levels(self.h)
        for lv in range(nlev):
            info = np.zeros(5, dtype=np.int64)
            L.om_amg_level_info(self.h, lv, _p(info))
            n, b, nnz, nc, nnzp = map(int, info)
            d = dict(n=n, b=b, ptr=np.zeros(n + 1, dtype=np.int32), col=np.zeros(nnz, dtype=np.int32),
                     val=np.zeros((nnz, b, b)), absent=np.zeros(n, dtype=np.uint8), ns=np.zeros((n * b, 6)), nc=nc)
            rho = np.zeros(1)
            if nnzp:
                d.update(agg=np.zeros(n, dtype=np.int32), pptr=np.zeros(n + 1, dtype=np.int32),
                         pcol=np.zeros(nnzp, dtype=np.int32), pval=np.zeros((nnzp, b, 6)),
                         tval=np.zeros((nnzp, b, 6)))
            if lv == nlev - 1:
                d["inv"] = np.zeros((n * b, n * b))
            L.om_amg_copy(self.h, lv, _p(d["ptr"]), _p(d["col"]), _p(d["val"]), _p(d["absent"]), _p(d["ns"]),
                          _p(d.get("agg")), _p(d.get("pptr")), _p(d.get("pcol")), _p(d.get("pval")),
                          _p(d.get("tval")), _p(rho), _p(d.get("inv")))
            d["rho"] = float(rho[0])
            out.append(d)
        return out

    def amg_smooth(self, level, b, x, deg=2):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.array(x, dtype=np.float64)
        lib().om_amg_smooth(self.h, int(level), _p(b), _p(x), int(deg))
        return x

    def amg_vcycle(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(3 * self.nn)
        lib().om_amg_vcycle(self.h, _p(b), _p(x))
        return x

    def lbfgs_apply(self, S, Y, rho, q, h0=0):
        S = np.ascontiguousarray(S, dtype=np.float64)
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float64)
        z = np.zeros(self.ndof)
        lib().om_lbfgs_apply(self.h, _p(S), _p(Y), _p(rho), int(len(rho)), _p(q), _p(z), h0)
        return z

    def solve(self, method, d, tol=1e-8, max_it=None, opts=None):
        mth = METHODS[method] if isinstance(method, str) else int(method)
        if max_it is None:
            max_it = 50 if mth < 2 else 1000
        o = default_opts(mth)
        if opts:
            keys = ["precision", "ksp_rtol", "ksp_atol", "ew_rtol0", "ew_rtolmax", "ksp_restart",
                    "ksp_max_it", "lbfgs_m", "dtol", "apply_dirichlet", "jac_lag", "hess_reassemble",
                    "ib_adaptive", "pc_type"]
            for k, v in opts.items():
                o[keys.index(k)] = v
        d = np.ascontiguousarray(d, dtype=np.float64)
        st = np.zeros(6 + 5 * HIST)
        status = lib().om_solve(self.h, mth, tol, max_it, _p(d), _p(o), _p(st))
        nit = int(st[1])
        stats = dict(status=status, nit=nit, lit_total=int(st[2]), assemblies=int(st[3]),
                     r0=st[4], rfinal=st[5], res_hist=st[6:6 + nit + 1].copy(),
                     lit_hist=st[6 + HIST:6 + HIST + nit + 1].astype(int),
                     eta_hist=st[6 + 2 * HIST:6 + 2 * HIST + nit + 1].copy(),
                     lres_hist=st[6 + 3 * HIST:6 + 3 * HIST + nit + 1].copy(),
                     time_hist=st[6 + 4 * HIST:6 + 4 * HIST + nit + 1].copy())
        return d, stats
