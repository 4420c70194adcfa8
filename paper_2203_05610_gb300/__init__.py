"""Python binding of libfe.so: the GB300 nonlinear-elasticity solver library.

Argument marshalling only: every step of the solver path runs in the CUDA
kernels behind the C ABI of ``include/fe.h``.  PyTorch supplies device
memory (CUDA tensors) and nothing else.  There is no CPU fallback: when the
library is missing or no GPU is present the calls raise.

Names follow the C ABI: ``fe_mesh_create`` -> :class:`Mesh`,
``fe_assemble_residual`` -> :meth:`Mesh.residual`, ``fe_assemble_tangent`` ->
:meth:`Mesh.tangent`, ``nl_solve`` -> :meth:`Mesh.solve`, and so on.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_lib", "libfe.so")
# FE_LIB_VARIANT=debug_bounds loads the index-checking build (build(debug_bounds=True))
if os.environ.get("FE_LIB_VARIANT") == "debug_bounds":
    SO_PATH = os.path.join(_HERE, "_lib", "dbg", "libfe_dbg.so")

FE_OK = 0
NL_DIVERGED, NL_MAX_IT, NL_NONFINITE, KSP_BREAKDOWN = 1, 2, 3, 4
METHODS = {"NK": 0, "iNK": 1, "B": 2, "iB": 3}
PRECISIONS = {"fp64": 0, "mixed_fp32": 1, "mixed_bf16": 2}
PC_TYPES = {"bj": 0, "amg": 1, "amg_bf16": 2}
NL_HIST = 1024


class FEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libfe error {code}: {msg}")
        self.code = code


class fe_material(C.Structure):
    _fields_ = [("kind", C.c_int32), ("vol_literal", C.c_int32), ("E", C.c_double), ("nu", C.c_double),
                ("mu", C.c_double), ("C", C.c_double), ("bf", C.c_double), ("bt", C.c_double),
                ("bfs", C.c_double), ("kappa", C.c_double), ("Ta_peak", C.c_double), ("period", C.c_double),
                ("alpha_p", C.c_double), ("beta_p", C.c_double), ("c_log", C.c_double)]


class fe_dirichlet_group(C.Structure):
    _fields_ = [("comp_mask", C.c_uint32), ("center", C.c_double * 3), ("angle", C.c_double),
                ("translation", C.c_double * 3)]


class fe_mesh_desc(C.Structure):
    _fields_ = [("order", C.c_int32), ("pressure_order", C.c_int32), ("nv", C.c_int32), ("ne", C.c_int32),
                ("coords", C.c_void_p), ("tets", C.c_void_p), ("dir_group", C.c_void_p), ("ngroups", C.c_int32),
                ("groups", C.c_void_p), ("nf", C.c_int32), ("faces", C.c_void_p), ("face_kind", C.c_void_p),
                ("face_data", C.c_void_p), ("material", fe_material), ("fibers", C.c_void_p),
                ("device", C.c_int32), ("stream", C.c_void_p)]


class fe_mesh_info(C.Structure):
    _fields_ = [("order", C.c_int32), ("pressure_order", C.c_int32), ("nv", C.c_int32), ("ne", C.c_int32),
                ("nn", C.c_int32), ("np", C.c_int32), ("ndof", C.c_int64), ("nen", C.c_int32),
                ("nnzb", C.c_int64), ("nnz_up", C.c_int64), ("ncolors", C.c_int32), ("device_bytes", C.c_int64)]


class nl_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("ksp_rtol", C.c_double), ("ksp_atol", C.c_double),
                ("ew_rtol0", C.c_double), ("ew_rtolmax", C.c_double), ("ksp_restart", C.c_int32),
                ("ksp_max_it", C.c_int32), ("lbfgs_m", C.c_int32), ("dtol", C.c_double),
                ("apply_dirichlet", C.c_int32), ("orthog", C.c_int32), ("jac_lag", C.c_int32),
                ("hess_reassemble", C.c_int32), ("ib_adaptive", C.c_int32), ("pc_type", C.c_int32)]


class nl_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("nit", C.c_int32), ("lit_total", C.c_int64), ("assemblies", C.c_int32),
                ("r0", C.c_double), ("rfinal", C.c_double), ("time_s", C.c_double), ("hist_len", C.c_int32),
                ("res_hist", C.c_double * NL_HIST), ("lit_hist", C.c_int32 * NL_HIST),
                ("eta_hist", C.c_double * NL_HIST), ("lres_hist", C.c_double * NL_HIST)]


BATCH_HIST = 64  # FE_BATCH_HIST of include/fe_batch.h


class fe_batch_out(C.Structure):
    _fields_ = [("status", C.c_int32), ("nit", C.c_int32), ("assemblies", C.c_int32), ("hist_len", C.c_int32),
                ("lit_total", C.c_int64), ("r0", C.c_double), ("rfinal", C.c_double),
                ("res_hist", C.c_double * BATCH_HIST), ("lit_hist", C.c_int32 * BATCH_HIST),
                ("eta_hist", C.c_double * BATCH_HIST)]


PROF_CLASSES = ["residual", "tangent", "spmv", "pc", "arnoldi", "twoloop", "vector", "other"]


class fe_profile_info(C.Structure):
    _fields_ = [("launches", C.c_int64 * 8), ("timed", C.c_int64 * 8), ("ms", C.c_double * 8),
                ("bytes", C.c_double * 8), ("flops", C.c_double * 8)]


class fe_server_opts(C.Structure):
    _fields_ = [("device", C.c_int32), ("hbm_budget", C.c_int64), ("max_active", C.c_int32),
                ("batch_max_dofs", C.c_int64), ("mesh_cache", C.c_int32)]


class fe_tuning_entry(C.Structure):
    _fields_ = [("order", C.c_int32), ("precision", C.c_int32), ("size_class", C.c_int32), ("threads", C.c_int32),
                ("batches", C.c_int32 * 2), ("cost", C.c_double * 2)]


class fe_request(C.Structure):
    _fields_ = [("mesh", C.POINTER(fe_mesh_desc)), ("method", C.c_int32), ("tol", C.c_double),
                ("max_it", C.c_int32), ("opts", C.POINTER(nl_opts)), ("load", C.c_double), ("time", C.c_double),
                ("d0", C.c_void_p)]


class fe_request_status(C.Structure):
    _fields_ = [("state", C.c_int32), ("result", C.c_int32), ("ndof", C.c_int64), ("footprint", C.c_int64),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_end", C.c_double), ("stats", nl_stats),
                ("mesh_reused", C.c_int32)]


REQ_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}

_lib = None
_lock = threading.Lock()

# exported symbols and their signatures (checked by the CPU tests against include/fe.h)
_P, _I, _D = C.c_void_p, C.c_int, C.c_double
SIGNATURES = {
    "fe_mesh_create": (_I, [C.POINTER(fe_mesh_desc), C.POINTER(C.c_void_p)]),
    "fe_mesh_destroy": (_I, [_P]),
    "fe_mesh_get_info": (_I, [_P, C.POINTER(fe_mesh_info)]),
    "fe_mesh_get_topology": (_I, [_P, _P, _P, _P, _P, _P]),
    "fe_set_load": (_I, [_P, _D, _D]),
    "fe_apply_dirichlet": (_I, [_P, _P]),
    "fe_assemble_residual": (_I, [_P, _P, _P, C.POINTER(C.c_double)]),
    "fe_energy": (_I, [_P, _P, C.POINTER(C.c_double)]),
    "fe_assemble_tangent": (_I, [_P, _P, _I]),
    "fe_tangent_copy": (_I, [_P, _P, _P, _P]),
    "fe_spmv": (_I, [_P, _P, _P]),
    "fe_pc_apply": (_I, [_P, _P, _P]),
    "fe_spmv_noalloc": (_I, [_P, _P, _P]),
    "nl_opts_default": (_I, [_I, C.POINTER(nl_opts)]),
    "nl_solve": (_I, [_P, _I, _D, _I, _P, C.POINTER(nl_opts), C.POINTER(nl_stats)]),
    "fe_gmres": (_I, [_P, _P, _P, _D, _D, _I, _I, _I, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "fe_lbfgs_apply": (_I, [_P, _P, _P, _P, _I, _P, _P, _I]),
    "fe_profile_reset": (_I, [_P, _I]),
    "fe_profile_read": (_I, [_P, C.POINTER(fe_profile_info)]),
    "serve_create": (_I, [C.POINTER(fe_server_opts), C.POINTER(C.c_void_p)]),
    "serve_submit": (_I, [_P, C.POINTER(fe_request), C.POINTER(C.c_int64)]),
    "serve_poll": (_I, [_P, C.c_int64, _I, C.POINTER(fe_request_status), _P]),
    "serve_clock": (_D, [_P]),
    "serve_tuning": (_I, [_P, _P, _I]),
    "serve_destroy": (_I, [_P]),
    "fe_set_pc": (_I, [_P, _I]),
    "fe_amg_levels": (_I, [_P]),
    "fe_amg_get_level": (_I, [_P, _I, _P, C.POINTER(C.c_double), _P, _P, _P, _P, _P, _P, _P, _P]),
    "fe_set_wait_limit": (_I, [_P, C.c_int64]),
    "fe_batch_supported": (_I, [_P, _I, C.POINTER(nl_opts)]),
    "fe_batch_solve": (_I, [_I, _P, _P, _P, _P, _P, _P, _I, _P]),
    "fe_set_dynamics": (_I, [_P, _D, _D]),
    "fe_dynamics_set": (_I, [_P, _P, _P, _P]),
    "fe_dynamics_advance": (_I, [_P, _P]),
    "fe_dynamics_get": (_I, [_P, _P, _P]),
    "fe_last_error": (C.c_char_p, []),
}


def lib():
    """Load libfe.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO_PATH):
                raise ImportError(f"{SO_PATH} is not built; run __graft_entry__.build() first")
            L = C.CDLL(SO_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc):
    if rc < 0:
        raise FEError(rc, lib().fe_last_error().decode())
    return rc


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dev_ptr(t, n, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} entries, expected {n}")
    return C.c_void_p(t.data_ptr())


def material_struct(m):
    s = fe_material()
    s.kind = int(m["kind"])
    s.vol_literal = int(m.get("vol_literal", 0))
    for k in ("E", "nu", "mu", "C", "bf", "bt", "bfs", "kappa", "Ta_peak", "period", "alpha_p", "beta_p", "c_log"):
        setattr(s, k, float(m.get(k, 0.0)))
    if s.period == 0.0:
        s.period = 1.0
    return s


def make_desc(w, device=0):
    """fe_mesh_desc for a workload dict, with the arrays it points to."""
    groups = (fe_dirichlet_group * max(len(w["groups"]), 1))()
    for g, G in enumerate(w["groups"]):
        groups[g].comp_mask = int(G["mask"])
        groups[g].center[:] = [float(x) for x in G["center"]]
        groups[g].angle = float(G["angle"])
        groups[g].translation[:] = [float(x) for x in G["translation"]]
    d = fe_mesh_desc()
    d.order = int(w["order"])
    d.pressure_order = int(w["pressure_order"])
    d.nv = int(w["coords"].shape[0])
    d.ne = int(w["tets"].shape[0])
    keep = [np.ascontiguousarray(w["coords"], dtype=np.float64),
            np.ascontiguousarray(w["tets"], dtype=np.int32),
            np.ascontiguousarray(w["dir_group"], dtype=np.uint8),
            np.ascontiguousarray(w["faces"], dtype=np.int32).reshape(-1, 3),
            np.ascontiguousarray(w["face_kind"], dtype=np.int32).reshape(-1),
            np.ascontiguousarray(w["face_data"], dtype=np.float64).reshape(-1, 3),
            None if w["fibers"] is None else np.ascontiguousarray(w["fibers"], dtype=np.float64),
            groups]
    d.coords = _np_ptr(keep[0])
    d.tets = _np_ptr(keep[1])
    d.dir_group = _np_ptr(keep[2])
    d.ngroups = len(w["groups"])
    d.groups = C.cast(groups, C.c_void_p)
    d.nf = int(keep[3].shape[0])
    d.faces = _np_ptr(keep[3])
    d.face_kind = _np_ptr(keep[4])
    d.face_data = _np_ptr(keep[5])
    d.material = material_struct(w["material"])
    d.fibers = _np_ptr(keep[6])
    d.device = int(device)
    d.stream = None
    return d, keep


def _opts_struct(method, opts):
    o = nl_opts()
    _check(lib().nl_opts_default(method, C.byref(o)))
    for k, v in (opts or {}).items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "pc_type" and isinstance(v, str):
            v = PC_TYPES[v]
        setattr(o, k, v)
    return o


class Mesh:
    """A mesh (and its solver state) resident on one GPU.

    ``w`` is a workload dict from :mod:`workloads` (vertex coordinates, P1
    tets, Dirichlet groups, loaded faces, material, fibres).
    """

    def __init__(self, w, device=0):
        import torch
        L = lib()
        self.device = torch.device("cuda", device)
        d, self._keep = make_desc(w, device)
        torch.cuda.init()
        h = C.c_void_p()
        _check(L.fe_mesh_create(C.byref(d), C.byref(h)))
        self.h = h
        info = fe_mesh_info()
        _check(L.fe_mesh_get_info(self.h, C.byref(info)))
        self.info = info
        self.nn, self.np_, self.ndof, self.nnzb = info.nn, info.np, int(info.ndof), int(info.nnzb)
        self.nnz_up, self.ncolors, self.nen, self.ne = int(info.nnz_up), info.ncolors, info.nen, info.ne

    def close(self):
        if getattr(self, "h", None):
            lib().fe_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- helpers
    def zeros(self):
        import torch
        return torch.zeros(self.ndof, dtype=torch.float64, device=self.device)

    def _vec(self, t, name="x"):
        return _dev_ptr(t, self.ndof, name)

    # -------------------------------------------------------------- C ABI calls
    def topology(self):
        conn = np.zeros((self.ne, self.nen), dtype=np.int32)
        colors = np.zeros(self.ne, dtype=np.int32)
        rp = np.zeros(self.nn + 1, dtype=np.int32)
        col = np.zeros(self.nnzb, dtype=np.int32)
        X = np.zeros((self.nn, 3))
        _check(lib().fe_mesh_get_topology(self.h, _np_ptr(conn), _np_ptr(colors), _np_ptr(rp), _np_ptr(col),
                                          _np_ptr(X)))
        return dict(conn=conn, colors=colors, row_ptr=rp, col=col, X=X)

    def set_load(self, load, time=0.0):
        _check(lib().fe_set_load(self.h, float(load), float(time)))

    def apply_dirichlet(self, d):
        _check(lib().fe_apply_dirichlet(self.h, self._vec(d, "d")))
        return d

    def residual(self, d, r=None):
        r = self.zeros() if r is None else r
        nrm = C.c_double()
        _check(lib().fe_assemble_residual(self.h, self._vec(d, "d"), self._vec(r, "r"), C.byref(nrm)))
        return r, nrm.value

    def energy(self, d):
        out = C.c_double()
        _check(lib().fe_energy(self.h, self._vec(d, "d"), C.byref(out)))
        return out.value

    def tangent(self, d, precision="fp64"):
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(lib().fe_assemble_tangent(self.h, self._vec(d, "d"), p))

    def tangent_copy(self):
        val = np.zeros((self.nnzb, 3, 3))
        bup = np.zeros((max(self.nnz_up, 1), 3))
        dinv = np.zeros((self.nn, 3, 3))
        _check(lib().fe_tangent_copy(self.h, _np_ptr(val), _np_ptr(bup), _np_ptr(dinv)))
        return val, bup[: self.nnz_up], dinv

    def spmv(self, x, y=None):
        y = self.zeros() if y is None else y
        _check(lib().fe_spmv(self.h, self._vec(x), self._vec(y, "y")))
        return y

    def pc(self, x, y=None):
        y = self.zeros() if y is None else y
        _check(lib().fe_pc_apply(self.h, self._vec(x), self._vec(y, "y")))
        return y

    def gmres(self, b, x=None, rtol=1e-6, atol=1e-10, restart=500, max_it=10000, orthog=0):
        x = self.zeros() if x is None else x
        it = C.c_int()
        res = C.c_double()
        _check(lib().fe_gmres(self.h, self._vec(b, "b"), self._vec(x), float(rtol), float(atol), int(restart),
                              int(max_it), int(orthog), C.byref(it), C.byref(res)))
        return x, it.value, res.value

    def lbfgs_apply(self, S, Y, rho, q, h0=0):
        import torch
        k = int(rho.numel())
        z = self.zeros()
        for t, nm in ((S, "S"), (Y, "Y")):
            if t.numel() != k * self.ndof or not t.is_contiguous() or t.dtype != torch.float64:
                raise ValueError(f"{nm} must be a contiguous float64 [k][ndof] CUDA tensor")
        _check(lib().fe_lbfgs_apply(self.h, C.c_void_p(S.data_ptr()), C.c_void_p(Y.data_ptr()),
                                    C.c_void_p(rho.data_ptr()), k, self._vec(q, "q"), self._vec(z, "z"), int(h0)))
        return z

    def set_pc(self, pc_type):
        """Displacement-block preconditioner: "bj" (nodal block-Jacobi) or "amg"."""
        _check(lib().fe_set_pc(self.h, PC_TYPES.get(pc_type, pc_type)))

    def amg_sizes(self):
        """Block rows (nodes) of each AMG level of the last assembly."""
        out = []
        for lv in range(lib().fe_amg_levels(self.h)):
            info = np.zeros(5, dtype=np.int64)
            rho = C.c_double()
            _check(lib().fe_amg_get_level(self.h, lv, _np_ptr(info), C.byref(rho), None, None, None, None, None,
                                          None, None, None))
            out.append(int(info[0]))
        return out

    def amg_levels(self):
        """The AMG hierarchy of the last assembly (fe_amg_get_level), one dict per level."""
        out = []
        for lv in range(lib().fe_amg_levels(self.h)):
            info = np.zeros(5, dtype=np.int64)
            rho = C.c_double()
            _check(lib().fe_amg_get_level(self.h, lv, _np_ptr(info), C.byref(rho), None, None, None, None, None,
                                          None, None, None))
            n, b, nnz, nc, nnzp = map(int, info)
            d = dict(n=n, b=b, nc=nc, rho=rho.value, absent=np.zeros(n, dtype=np.uint8))
            if lv > 0:
                d.update(ptr=np.zeros(n + 1, dtype=np.int32), col=np.zeros(nnz, dtype=np.int32),
                         val=np.zeros((nnz, b, b)))
            if nnzp:
                d.update(agg=np.zeros(n, dtype=np.int32), pptr=np.zeros(n + 1, dtype=np.int32),
                         pcol=np.zeros(nnzp, dtype=np.int32), pval=np.zeros((nnzp, b, 6)))
            _check(lib().fe_amg_get_level(self.h, lv, None, None, _np_ptr(d.get("ptr")), _np_ptr(d.get("col")),
                                          _np_ptr(d.get("val")), _np_ptr(d["absent"]), _np_ptr(d.get("agg")),
                                          _np_ptr(d.get("pptr")), _np_ptr(d.get("pcol")), _np_ptr(d.get("pval"))))
            out.append(d)
        return out

    def set_dynamics(self, rho, dt):
        """Newmark elastodynamics with density rho and step dt, state at rest
        (rho <= 0: static again)."""
        _check(lib().fe_set_dynamics(self.h, float(rho), float(dt)))

    def dynamics_set(self, d=None, v=None, a=None):
        """State d_n, v_n, a_n: CUDA float64 tensors of 3 nn entries (None: zero)."""
        ptrs = [None if t is None else _dev_ptr(t, 3 * self.nn, nm) for t, nm in ((d, "d"), (v, "v"), (a, "a"))]
        _check(lib().fe_dynamics_set(self.h, *ptrs))

    def dynamics_advance(self, d):
        """Move the state to the converged step solution d ([ndof])."""
        _check(lib().fe_dynamics_advance(self.h, self._vec(d, "d")))

    def dynamics_get(self):
        """(v_n, a_n) as CUDA float64 tensors of 3 nn entries."""
        import torch
        v = torch.zeros(3 * self.nn, dtype=torch.float64, device=self.device)
        a = torch.zeros_like(v)
        _check(lib().fe_dynamics_get(self.h, _dev_ptr(v, 3 * self.nn, "v"), _dev_ptr(a, 3 * self.nn, "a")))
        return v, a

    def set_wait_limit(self, polls=-1):
        """Polls before a bounded device wait gives up (< 0: the default)."""
        _check(lib().fe_set_wait_limit(self.h, int(polls)))

    def profile_reset(self, timing=False):
        _check(lib().fe_profile_reset(self.h, 1 if timing else 0))

    def profile_read(self):
        p = fe_profile_info()
        _check(lib().fe_profile_read(self.h, C.byref(p)))
        return {name: dict(launches=int(p.launches[i]), timed=int(p.timed[i]), ms=float(p.ms[i]),
                           bytes=float(p.bytes[i]), flops=float(p.flops[i])) for i, name in enumerate(PROF_CLASSES)}

    def solve(self, method, d, tol=1e-8, max_it=None, opts=None):
        mth = METHODS[method] if isinstance(method, str) else int(method)
        if max_it is None:
            max_it = 50 if mth < 2 else 1000
        o = _opts_struct(mth, opts)
        st = nl_stats()
        rc = _check(lib().nl_solve(self.h, mth, float(tol), int(max_it), self._vec(d, "d"), C.byref(o),
                                   C.byref(st)))
        n = st.hist_len
        stats = dict(status=rc, nit=st.nit, lit_total=int(st.lit_total), assemblies=st.assemblies, r0=st.r0,
                     rfinal=st.rfinal, time_s=st.time_s, res_hist=np.array(st.res_hist[:n]),
                     lit_hist=np.array(st.lit_hist[:n]), eta_hist=np.array(st.eta_hist[:n]),
                lres_hist=np.array(st.lres_hist[:n]))
        return d, stats


def batch_supported(mesh, method, opts):
    """True when the request can run in fe_batch_solve."""
    mth = METHODS[method] if isinstance(method, str) else int(method)
    o = _opts_struct(mth, opts)
    return bool(lib().fe_batch_supported(mesh.h, mth, C.byref(o)))


def batch_solve(meshes, methods, ds, tols, max_its=None, opts=None, threads=256):
    """Solve len(meshes) requests in one launch (include/fe_batch.h), one
    CTA per request.  ds: CUDA float64 tensors [ndof], overwritten by the
    solutions.  opts: one dict (all requests) or a list of dicts.  Returns
    one stats dict per request."""
    n = len(meshes)
    mths = [METHODS[x] if isinstance(x, str) else int(x) for x in methods]
    if max_its is None:
        max_its = [50 if x < 2 else 1000 for x in mths]
    olist = opts if isinstance(opts, (list, tuple)) else [opts] * n
    O = (nl_opts * n)(*[_opts_struct(mths[i], olist[i]) for i in range(n)])
    H = (C.c_void_p * n)(*[m.h.value if isinstance(m.h, C.c_void_p) else m.h for m in meshes])
    D = (C.c_void_p * n)(*[_dev_ptr(ds[i], meshes[i].ndof, "d").value for i in range(n)])
    M = (C.c_int * n)(*mths)
    T = (C.c_double * n)(*[float(t) for t in tols])
    I = (C.c_int * n)(*[int(x) for x in max_its])
    out = (fe_batch_out * n)()
    _check(lib().fe_batch_solve(n, H, M, T, I, O, D, int(threads), out))
    res = []
    for st in out:
        k = st.hist_len
        res.append(dict(status=st.status, nit=st.nit, lit_total=int(st.lit_total), assemblies=st.assemblies,
                        r0=st.r0, rfinal=st.rfinal, res_hist=np.array(st.res_hist[:k]),
                        lit_hist=np.array(st.lit_hist[:k]), eta_hist=np.array(st.eta_hist[:k])))
    return res


def _stats_dict(st):
    n = st.hist_len
    return dict(status=st.status, nit=st.nit, lit_total=int(st.lit_total), assemblies=st.assemblies, r0=st.r0,
                rfinal=st.rfinal, time_s=st.time_s, res_hist=np.array(st.res_hist[:n]),
                lit_hist=np.array(st.lit_hist[:n]), eta_hist=np.array(st.eta_hist[:n]),
                lres_hist=np.array(st.lres_hist[:n]))


class Server:
    """Continuous-batching request loop on one GPU (include/fe_serve.h)."""

    def __init__(self, device=0, hbm_budget=0, max_active=8, batch_max_dofs=0, mesh_cache=True):
        import torch
        torch.cuda.init()
        o = fe_server_opts(device=int(device), hbm_budget=int(hbm_budget), max_active=int(max_active),
                           batch_max_dofs=int(batch_max_dofs), mesh_cache=0 if mesh_cache else -1)
        h = C.c_void_p()
        _check(lib().serve_create(C.byref(o), C.byref(h)))
        self.h = h
        self._ndof = {}

    def tuning(self):
        """The batched path's autotuner table (fe_tuning_entry), one dict per size class."""
        n = lib().serve_tuning(self.h, None, 0)
        arr = (fe_tuning_entry * max(n, 1))()
        n = _check(lib().serve_tuning(self.h, arr, n))
        return [dict(order=e.order, precision=e.precision, size_class=e.size_class, threads=e.threads,
                     batches=list(e.batches), cost=list(e.cost)) for e in arr[:n]]

    def submit(self, w, method, tol=1e-8, max_it=None, opts=None, load=1.0, time=0.0, d0=None):
        mth = METHODS[method] if isinstance(method, str) else int(method)
        if max_it is None:
            max_it = 50 if mth < 2 else 1000
        d, keep = make_desc(w)
        o = _opts_struct(mth, opts)
        d0a = None if d0 is None else np.ascontiguousarray(d0, dtype=np.float64)
        q = fe_request(mesh=C.pointer(d), method=mth, tol=float(tol), max_it=int(max_it), opts=C.pointer(o),
                       load=float(load), time=float(time), d0=_np_ptr(d0a))
        rid = C.c_int64()
        _check(lib().serve_submit(self.h, C.byref(q), C.byref(rid)))
        del keep
        return int(rid.value)

    def poll(self, rid, wait=False):
        st = fe_request_status()
        _check(lib().serve_poll(self.h, int(rid), 1 if wait else 0, C.byref(st), None))
        out = dict(state=REQ_STATES[st.state], result=st.result, ndof=int(st.ndof), footprint=int(st.footprint),
                   t_submit=st.t_submit, t_start=st.t_start, t_end=st.t_end, mesh_reused=bool(st.mesh_reused))
        if st.state == 2:
            x = np.zeros(int(st.ndof))
            _check(lib().serve_poll(self.h, int(rid), 0, C.byref(st), _np_ptr(x)))
            out["d"] = x
            out["stats"] = _stats_dict(st.stats)
        elif st.state == 3:
            out["error"] = lib().fe_last_error().decode()
        return out

    def clock(self):
        return float(lib().serve_clock(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
