"""Pins of the oracle's algebraic multigrid preconditioner (smoothed
aggregation on nodal blocks, the class of the paper's BoomerAMG with block
size 3, Section "Test problems and solvers details" and Appendix A).

Each property is checked against brute force or a closed form computed here
from the exported hierarchy: the aggregation rules, the near null space kept
exactly by the prolongators (rigid motions of a free body), the prolongator
smoothing and the Galerkin products as dense matrix products, the
Chebyshev smoother as its residual polynomial, the coarsest solve, the
V-cycle as the dense two-grid operator, and the solver's iteration counts
under mesh refinement.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle_helpers import strip_bc


def _setup(w, load=None, d=None):
    m = O.Mesh(w)
    m.set_load(w["steps"][0][0] if load is None else load)
    if d is None:
        d = m.apply_dirichlet(np.zeros(m.ndof))
    m.set_pc("amg")
    m.tangent(d)
    return m, m.amg_levels()


def _dense(L, key="val", ptr="ptr", col="col", ncols=None, bc=None):
    b = L["b"]
    bc = b if bc is None else bc
    n = L["n"]
    ncols = n if ncols is None else ncols
    M = np.zeros((n * b, ncols * bc))
    p, c, v = L[ptr], L[col], L[key]
    for a in range(n):
        for k in range(p[a], p[a + 1]):
            M[a * b:(a + 1) * b, c[k] * bc:(c[k] + 1) * bc] = v[k]
    return M


def _graph(L):
    """Neighbour sets of the nodes that are not wholly absent."""
    full = (1 << L["b"]) - 1
    keep = L["absent"] != full
    nb = {}
    for a in range(L["n"]):
        if keep[a]:
            nb[a] = {int(j) for j in L["col"][L["ptr"][a]:L["ptr"][a + 1]] if keep[j] and j != a}
    return nb


@pytest.mark.parametrize("order", [1, 2])
def test_aggregation_rules_brute_force(order):
    w = W.cook(6, 5, 2, order=order, nu=0.3)
    m, levs = _setup(w)
    for L in levs[:-1]:
        nb = _graph(L)
        agg = L["agg"]
        n = L["n"]
        pri = {a: O.splitmix64(a) for a in nb}
        # roots: the greedy distance-2 independent set in priority order
        order_ = sorted(nb, key=lambda a: (-pri[a], a))
        blocked, roots = set(), []
        for a in order_:
            if a in blocked:
                continue
            roots.append(a)
            ring = {a} | nb[a]
            for j in nb[a]:
                ring |= nb[j]
            blocked |= ring
        roots.sort()
        assert L["nc"] == len(roots)
        rid = {r: k for k, r in enumerate(roots)}
        phase1 = {}
        for r in roots:
            for j in {r} | nb[r]:
                assert j not in phase1  # roots are at distance >= 3
                phase1[j] = rid[r]
        for a in range(n):
            if a not in nb:
                assert agg[a] == -1
            elif a in phase1:
                assert agg[a] == phase1[a]
            else:
                first = min(j for j in nb[a] if j in phase1)
                assert agg[a] == phase1[first]


def _free_body(order):
    w = strip_bc(W.cook(4, 3, 2, order=order, nu=0.3))
    # a 0-load stress-free state: K(0) annihilates the six rigid motions
    return _setup(w, load=0.0)


@pytest.mark.parametrize("order", [1, 2])
def test_rigid_motions_kept_by_every_level(order):
    m, levs = _free_body(order)
    assert len(levs) >= 2
    for l, L in enumerate(levs[:-1]):
        C = levs[l + 1]
        A = _dense(L)
        B = L["ns"]
        if l == 0:
            assert np.abs(A @ B).max() <= 1e-10 * np.abs(A).max() * np.abs(B).max()
        T = _dense(L, "tval", "pptr", "pcol", C["n"], 6)
        P = _dense(L, "pval", "pptr", "pcol", C["n"], 6)
        Bc = C["ns"]
        # T R = B (the tentative prolongator reproduces the near null space),
        # and T has orthonormal columns on each aggregate's present components
        assert np.abs(T @ Bc - B).max() <= 1e-12 * np.abs(B).max()
        present = np.array([not (C["absent"][a] >> c) & 1 for a in range(C["n"]) for c in range(6)])
        G = T.T @ T
        assert np.abs(G - np.diag(present.astype(float))).max() <= 1e-12
        # smoothing keeps it: P Bc = B - omega D^-1 A B = B for a free body
        assert np.abs(P @ Bc - B).max() <= 1e-9 * np.abs(B).max()
        # the coarse operator annihilates the coarse rigid motions
        Ac = _dense(C)
        assert np.abs(Ac @ Bc).max() <= 1e-9 * np.abs(Ac).max() * np.abs(Bc).max()


@pytest.mark.parametrize("case", ["cook_p1", "cook_p2"])
def test_prolongator_smoothing_and_galerkin_products(case):
    w = W.cook(5, 4, 2, order=1 if case == "cook_p1" else 2, nu=0.3)
    m, levs = _setup(w)
    for l, L in enumerate(levs[:-1]):
        C = levs[l + 1]
        A = _dense(L)
        T = _dense(L, "tval", "pptr", "pcol", C["n"], 6)
        P = _dense(L, "pval", "pptr", "pcol", C["n"], 6)
        b = L["b"]
        D = np.zeros_like(A)
        for a in range(L["n"]):
            D[a * b:(a + 1) * b, a * b:(a + 1) * b] = A[a * b:(a + 1) * b, a * b:(a + 1) * b]
        DinvA = np.linalg.solve(D, A)
        # rho: 15 power steps stay below the spectral radius and come close to it
        rho_true = np.abs(np.linalg.eigvals(DinvA)).max()
        assert 0.9 * rho_true <= L["rho"] <= rho_true * (1 + 1e-12)
        omega = 4.0 / (3.0 * L["rho"])
        assert np.abs(P - (T - omega * DinvA @ T)).max() <= 1e-12 * np.abs(P).max()
        Ac = P.T @ A @ P
        for a in range(C["n"]):
            for c in range(6):
                if (C["absent"][a] >> c) & 1:
                    Ac[6 * a + c, 6 * a + c] = 1.0
        assert np.abs(_dense(C) - Ac).max() <= 1e-12 * np.abs(Ac).max()


def _cheb_poly(M, lo, hi, deg):
    """Residual polynomial of Chebyshev smoothing: T_deg((theta - M)/delta) / T_deg(theta/delta)."""
    th, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
    Y = (th * np.eye(M.shape[0]) - M) / de
    T0, T1 = np.eye(M.shape[0]), Y
    t0, t1 = 1.0, th / de
    for _ in range(deg - 1):
        T0, T1 = T1, 2 * Y @ T1 - T0
        t0, t1 = t1, 2 * (th / de) * t1 - t0
    return T1 / t1


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_chebyshev_smoother_is_its_residual_polynomial(deg):
    w = W.cook(5, 4, 2, order=2, nu=0.3)
    m, levs = _setup(w)
    for l, L in enumerate(levs[:-1]):
        A = _dense(L)
        b = L["b"]
        D = np.zeros_like(A)
        for a in range(L["n"]):
            D[a * b:(a + 1) * b, a * b:(a + 1) * b] = A[a * b:(a + 1) * b, a * b:(a + 1) * b]
        M = np.linalg.solve(D, A)
        rng = np.random.default_rng(7 + l)
        rhs = rng.standard_normal(A.shape[0])
        x0 = rng.standard_normal(A.shape[0])
        x = m.amg_smooth(l, rhs, x0, deg)
        # error e = x - A^-1 b evolves by the residual polynomial of D^-1 A
        xs = np.linalg.solve(A, rhs)
        Rp = _cheb_poly(M, L["rho"] / 30.0, 1.1 * L["rho"], deg)
        assert np.abs((x - xs) - Rp @ (x0 - xs)).max() <= 1e-9 * np.abs(x0 - xs).max()


def test_vcycle_is_the_dense_multigrid_operator():
    w = W.cook(5, 4, 2, order=1, nu=0.3)
    m, levs = _setup(w)
    assert len(levs) == 2
    L, C = levs
    A = _dense(L)
    b = 3
    D = np.zeros_like(A)
    for a in range(L["n"]):
        D[a * b:(a + 1) * b, a * b:(a + 1) * b] = A[a * b:(a + 1) * b, a * b:(a + 1) * b]
    M = np.linalg.solve(D, A)
    S = np.eye(A.shape[0]) - _cheb_poly(M, L["rho"] / 30.0, 1.1 * L["rho"], 2)  # x = S A^-1 b from 0
    P = _dense(L, "pval", "pptr", "pcol", C["n"], 6)
    Ac = _dense(C)
    # the coarsest level's inverse is the exact inverse
    assert np.abs(C["inv"] @ Ac - np.eye(Ac.shape[0])).max() <= 1e-10
    Ai = np.linalg.inv(A)
    rng = np.random.default_rng(3)
    rhs = rng.standard_normal(A.shape[0])
    x = S @ Ai @ rhs
    x = x + P @ np.linalg.solve(Ac, P.T @ (rhs - A @ x))
    x = x + S @ Ai @ (rhs - A @ x)
    z = m.amg_vcycle(rhs)
    assert np.abs(z - x).max() <= 1e-9 * np.abs(x).max()
    # a fixed linear operator: M(a u + b v) = a M u + b M v
    v = rng.standard_normal(A.shape[0])
    assert np.abs(m.amg_vcycle(2.0 * rhs - 3.0 * v) - (2.0 * z - 3.0 * m.amg_vcycle(v))).max() <= 1e-10 * np.abs(z).max()


def test_single_level_is_an_exact_solve():
    w = W.cook(2, 1, 1, order=1, nu=0.3)  # 12 nodes: the coarsest level at once
    m, levs = _setup(w)
    assert len(levs) == 1
    A = _dense(levs[0])
    rhs = np.random.default_rng(1).standard_normal(A.shape[0])
    assert np.abs(A @ m.amg_vcycle(rhs) - rhs).max() <= 1e-10 * np.abs(rhs).max()


def _gmres_its(w, rtol, pc):
    m = O.Mesh(w)
    m.set_load(w["steps"][0][0])
    d = m.apply_dirichlet(np.zeros(m.ndof))
    r, _ = m.residual(d)
    m.set_pc(pc)
    m.tangent(d)
    _, it, _ = m.gmres(-r, rtol=rtol, atol=0.0, restart=200, max_it=20000)
    return it


def test_iterations_under_refinement_and_against_block_jacobi():
    # Cook P1 at three refinements (225, 729 and 4,335 unknowns): the
    # AMG-preconditioned iteration count at most doubles while the mesh is
    # refined four times in each direction; block-Jacobi's grows more than
    # tenfold over the same meshes (89 to 2,212 here) and ends far above
    its = [_gmres_its(W.cook(4 * k, 4 * k, k, order=1, nu=0.3), 1e-8, "amg") for k in (1, 2, 4)]
    assert its[2] <= 2 * its[0] and max(its) <= 40, its
    bj = [_gmres_its(W.cook(4 * k, 4 * k, k, order=1, nu=0.3), 1e-8, "bj") for k in (1, 4)]
    assert bj[1] >= 10 * bj[0] and bj[1] >= 20 * its[2], (bj, its)


@pytest.mark.parametrize("order,bound", [(1, 0.9), (2, 0.99)])
def test_vcycle_error_reduction(order, bound):
    # linear elasticity K(0) of Cook (no load): the V-cycle as a stationary
    # iteration converges, its error propagation I - M^-1 A having spectral
    # radius below the bound (0.86 and 0.98 measured; GMRES then removes the
    # few slow modes), and it damps three quarters of the modes by more than
    # half per cycle
    w = W.cook(8, 8, 2, order=1, nu=0.3) if order == 1 else W.cook(4, 4, 2, order=2, nu=0.3)
    m, levs = _setup(w, load=0.0)
    A = _dense(levs[0])
    n = A.shape[0]
    E = np.zeros((n, n))
    for j in range(n):
        E[:, j] = -m.amg_vcycle(A[:, j])
        E[j, j] += 1.0
    ev = np.abs(np.linalg.eigvals(E))
    assert ev.max() < bound and np.mean(ev > 0.5) < 0.3, (ev.max(), np.mean(ev > 0.5))


@pytest.mark.parametrize("case", ["cook_p1", "twist_up", "heart_p1"])
def test_solvers_with_amg_reach_the_block_jacobi_solution(case):
    # the preconditioner changes the Krylov iterates, not the nonlinear
    # solution: every method with the AMG V-cycle (as the GMRES
    # preconditioner, or as H0 for B) reaches NK's block-Jacobi solution
    from oracle_helpers import small_cases
    w = small_cases()[case]
    load, time = {"heart_p1": (0.2, 0.01), "twist_up": (0.3, 0.0)}.get(case, (0.4, 0.0))
    methods = ("NK", "iNK") if case == "twist_up" else ("NK", "iNK", "B", "iB")

    def solve(method, pc):
        m = O.Mesh(w)
        m.set_load(load, time)
        tol = 1e-8 if method == "B" else 1e-11
        d, st = m.solve(method, np.zeros(m.ndof), tol=tol, opts=dict(ksp_atol=0.0, pc_type=pc))
        return d, st

    ref, st = solve("NK", 0)
    assert st["status"] == 0
    for mth in methods:
        d, st = solve(mth, 1)
        assert st["status"] == 0, (mth, st["res_hist"][-3:])
        xtol = 1e-6 if mth == "B" else 1e-9
        assert np.linalg.norm(d - ref) <= xtol * np.linalg.norm(ref), mth
