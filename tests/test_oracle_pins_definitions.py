"""Pins of the oracle's material, boundary and forcing terms against the
paper's definitions, restated here independently of the oracle's code.

- Heartbeat potential (Section "Test problems and solvers details", Guccione
  Psi with Q in the fibre frame and the active stress P_act): the oracle's
  Psi and P against a direct numpy restatement with each weight b_ab named,
  P_act against its printed formula, and the second-order expansion of Psi
  at F = I against the oracle's tangent there.
- Face terms (dead pressure, Robin springs of Eq. "bc epi" without the
  dashpot): totals on a flat face against closed forms (-p A N and
  (K_perp N N^T + K_par (I - N N^T)) t A) and nodal values against the
  exact P1/P2 triangle mass matrices.
- Eisenstat-Walker forcing (Section "Numerical solvers", inexact Newton):
  the linear residual norms the oracle records are recomputed from its
  iterates with a dense tangent, and the whole eta sequence is recomputed
  from those norms by choice 1 with the safeguard and the cap.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle_helpers import oracle_dense_K, strip_bc

GUCC = dict(kind=W.MAT_GUCCIONE, C=0.88, bf=18.5, bt=3.58, bfs=1.63, kappa=1e3, Ta_peak=60.0, period=0.8)


# ---------------------------------------------------------------- Heartbeat potential
def _frame(rng):
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 2] *= -1
    return q.T  # rows f, s, n


def guccione_psi(F, fib, mat, gamma):
    """Psi = C/2 (e^Q - 1) + B/2 (J - 1) ln J + gamma |F f| with
    Q = b_ff E_ff^2 + b_ss E_ss^2 + b_nn E_nn^2 + b_fs (E_fs^2 + E_sf^2)
        + b_fn (E_fn^2 + E_nf^2) + b_sn (E_sn^2 + E_ns^2),
    E = (F^T F - I)/2, E_ab = E a . b; weights of the cardiac workload:
    b_ff = bf, b_ss = b_nn = b_sn = bt, b_fs = b_fn = bfs."""
    f, s, n = fib
    E = 0.5 * (F.T @ F - np.eye(3))

    def comp(a, b):
        return float((E @ a) @ b)

    b_ff, b_ss, b_nn, b_sn = mat["bf"], mat["bt"], mat["bt"], mat["bt"]
    b_fs, b_fn = mat["bfs"], mat["bfs"]
    Q = (b_ff * comp(f, f) ** 2 + b_ss * comp(s, s) ** 2 + b_nn * comp(n, n) ** 2
         + b_fs * (comp(f, s) ** 2 + comp(s, f) ** 2) + b_fn * (comp(f, n) ** 2 + comp(n, f) ** 2)
         + b_sn * (comp(s, n) ** 2 + comp(n, s) ** 2))
    J = np.linalg.det(F)
    return (0.5 * mat["C"] * (math.exp(Q) - 1.0) + 0.5 * mat["kappa"] * (J - 1.0) * math.log(J)
            + gamma * np.linalg.norm(F @ f))


def test_guccione_potential_against_its_definition():
    rng = np.random.default_rng(11)
    for trial in range(6):
        F = np.eye(3) + 0.12 * rng.standard_normal((3, 3))
        fib = _frame(rng)
        gam = 0.0 if trial % 2 == 0 else 9.0
        psi, P, _, _ = O.material_point(GUCC, F, fib, gam, 0.0)
        ref = guccione_psi(F, fib, GUCC, gam)
        assert abs(psi - ref) <= 1e-12 * max(1.0, abs(ref)), trial
        # P = dPsi/dF of the restated potential (central differences)
        h = 1e-6
        Pfd = np.zeros((3, 3))
        for k in range(3):
            for L in range(3):
                D = np.zeros((3, 3))
                D[k, L] = h
                Pfd[k, L] = (guccione_psi(F + D, fib, GUCC, gam) - guccione_psi(F - D, fib, GUCC, gam)) / (2 * h)
        assert np.abs(P - Pfd).max() <= 2e-6 * max(1.0, np.abs(P).max()), trial


def test_guccione_active_stress_is_the_printed_formula():
    # P_act = gamma (F f) x f / |F f|: the difference of P with and without gamma
    rng = np.random.default_rng(12)
    for _ in range(4):
        F = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
        fib = _frame(rng)
        gam = 17.5
        _, P1, _, _ = O.material_point(GUCC, F, fib, gam, 0.0)
        _, P0, _, _ = O.material_point(GUCC, F, fib, 0.0, 0.0)
        a = F @ fib[0]
        expect = gam * np.outer(a, fib[0]) / np.linalg.norm(a)
        assert np.abs((P1 - P0) - expect).max() <= 1e-11 * gam


def test_guccione_second_order_expansion_at_identity():
    # Psi(I + H) = 1/2 H:A(I):H + O(|H|^3) with
    # 1/2 H:A(I):H = C/2 sum_ab b_ab (a . sym H b)^2 + B/2 (tr H)^2
    rng = np.random.default_rng(13)
    fib = _frame(rng)
    _, P, A, _ = O.material_point(GUCC, np.eye(3), fib, 0.0, 0.0)
    assert np.abs(P).max() < 1e-13
    f, s, n = fib
    W_ = {("f", "f"): GUCC["bf"], ("s", "s"): GUCC["bt"], ("n", "n"): GUCC["bt"], ("f", "s"): GUCC["bfs"],
          ("s", "f"): GUCC["bfs"], ("f", "n"): GUCC["bfs"], ("n", "f"): GUCC["bfs"], ("s", "n"): GUCC["bt"],
          ("n", "s"): GUCC["bt"]}
    vec = {"f": f, "s": s, "n": n}
    for _ in range(5):
        H = rng.standard_normal((3, 3))
        Hs = 0.5 * (H + H.T)
        quad = 0.5 * GUCC["C"] * sum(w * float(vec[a] @ Hs @ vec[b]) ** 2 for (a, b), w in W_.items())
        quad += 0.5 * GUCC["kappa"] * np.trace(H) ** 2
        hv = H.reshape(9)
        assert abs(0.5 * hv @ A @ hv - quad) <= 1e-11 * max(1.0, abs(quad))


# ---------------------------------------------------------------- face terms
def _bary_int(powers, area):
    # int over a triangle of l1^a l2^b l3^c = 2 A a! b! c! / (a + b + c + 2)!
    a, b, c = powers
    return 2.0 * area * math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 2)


def _tri_shapes(order):
    """Shape functions on a triangle as polynomials in (l1, l2, l3):
    dict {(a, b, c): coeff} per local node (vertices, then edges 01, 12, 02)."""
    if order == 1:
        return [{(1, 0, 0): 1.0}, {(0, 1, 0): 1.0}, {(0, 0, 1): 1.0}]
    v = [{(2, 0, 0): 2.0, (1, 0, 0): -1.0}, {(0, 2, 0): 2.0, (0, 1, 0): -1.0}, {(0, 0, 2): 2.0, (0, 0, 1): -1.0}]
    e = [{(1, 1, 0): 4.0}, {(0, 1, 1): 4.0}, {(1, 0, 1): 4.0}]
    return v + e


def _poly_mul(p, q):
    out = {}
    for ka, va in p.items():
        for kb, vb in q.items():
            k = tuple(x + y for x, y in zip(ka, kb))
            out[k] = out.get(k, 0.0) + va * vb
    return out


def _exact_mass(order, area):
    # degree-1 monomials like l1 need the homogenised form: l1 = l1 (l1 + l2 + l3)
    def homog(p):
        out = {}
        for k, v in p.items():
            if sum(k) == 1 and order == 2:
                for j in range(3):
                    kk = list(k)
                    kk[j] += 1
                    out[tuple(kk)] = out.get(tuple(kk), 0.0) + v
            else:
                out[k] = out.get(k, 0.0) + v
        return out

    N = [homog(p) for p in _tri_shapes(order)]
    M = np.zeros((len(N), len(N)))
    for a in range(len(N)):
        for b in range(len(N)):
            M[a, b] = sum(v * _bary_int(k, area) for k, v in _poly_mul(N[a], N[b]).items())
    return M


def _face_node_map(m, w):
    """Global node of each local face node (3 vertices, then edge nodes 01, 12, 02)."""
    conn = m.topology()["conn"]
    enode = {}
    if w["order"] == 2:
        loc = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
        for e in range(conn.shape[0]):
            for k, (a, b) in enumerate(loc):
                va, vb = conn[e, a], conn[e, b]
                enode[(min(va, vb), max(va, vb))] = conn[e, 4 + k]
    out = []
    for f in w["faces"]:
        nodes = [int(v) for v in f]
        if w["order"] == 2:
            for a, b in ((0, 1), (1, 2), (0, 2)):
                nodes.append(int(enode[(min(f[a], f[b]), max(f[a], f[b]))]))
        out.append(nodes)
    return out


def _cook_bottom(order, kind, data):
    """Cook mesh with no Dirichlet data whose only loaded faces are the
    bottom surface y = 44 x / 48: a plane of area sqrt(48^2 + 44^2) * 10 and
    outward unit normal (44, -48, 0) / sqrt(48^2 + 44^2)."""
    w = strip_bc(W.cook(4, 3, 2, order=order))
    bf = W.boundary_faces(w["coords"], w["tets"])
    x = w["coords"][bf]
    on_bottom = np.all(np.abs(x[:, :, 1] - 44.0 / 48.0 * x[:, :, 0]) < 1e-9, axis=1)
    w["faces"] = bf[on_bottom]
    w["face_kind"] = np.full(on_bottom.sum(), kind, dtype=np.int32)
    w["face_data"] = np.tile(np.asarray(data, dtype=float), (on_bottom.sum(), 1))
    L = math.hypot(48.0, 44.0)
    return w, L * 10.0, np.array([44.0, -48.0, 0.0]) / L


@pytest.mark.parametrize("order", [1, 2])
def test_dead_pressure_total_and_nodal_forces(order):
    # t = -p N per unit reference area; R = internal - external, so at d = 0
    # the residual sums to +p A N, and node a carries p N int(phi_a)
    p = 2.5
    w, area, N = _cook_bottom(order, W.FACE_PRESSURE, [p, 0.0, 0.0])
    m = O.Mesh(w)
    m.set_load(1.0)
    r, _ = m.residual(np.zeros(m.ndof))
    R = r[: 3 * m.nn].reshape(-1, 3)
    assert np.abs(R.sum(axis=0) - p * area * N).max() <= 1e-12 * p * area
    expect = np.zeros_like(R)
    x = w["coords"][w["faces"]]
    for nodes, xf in zip(_face_node_map(m, w), x):
        A = 0.5 * np.linalg.norm(np.cross(xf[1] - xf[0], xf[2] - xf[0]))
        Mf = _exact_mass(order, A)
        for a, na in enumerate(nodes):
            expect[na] += p * N * Mf[a].sum()
    assert np.abs(R - expect).max() <= 1e-12 * p * area


@pytest.mark.parametrize("order", [1, 2])
def test_robin_springs_total_and_nodal_forces(order):
    # t = -(K_perp N N^T + K_par (I - N N^T)) d on the face; Cook is stress free
    # at F = I, so for a rigid translation the residual is the spring force
    kperp, kpar = 7.0, 0.8
    w, area, N = _cook_bottom(order, W.FACE_ROBIN, [kperp, kpar, 0.0])
    m = O.Mesh(w)
    m.set_load(1.0)
    Ks = kperp * np.outer(N, N) + kpar * (np.eye(3) - np.outer(N, N))
    t = np.array([0.3, -0.2, 0.7])
    d = np.tile(t, m.nn)
    r, _ = m.residual(d)
    R = r.reshape(-1, 3)
    assert np.abs(R.sum(axis=0) - Ks @ t * area).max() <= 1e-12 * area
    # a varying field: the spring part of the tangent (tangent with the faces
    # minus tangent without them) couples nodes a, b by M_ab Ks, M the exact
    # face mass matrix
    m.tangent(np.zeros(m.ndof))
    Kd = oracle_dense_K(m, w)
    w0 = dict(w, faces=np.zeros((0, 3), dtype=np.int32), face_kind=np.zeros(0, dtype=np.int32),
              face_data=np.zeros((0, 3)))
    m0 = O.Mesh(w0)
    m0.tangent(np.zeros(m0.ndof))
    K_springs = Kd - oracle_dense_K(m0, w0)
    expect = np.zeros((m.nn, 3, m.nn, 3))
    x = w["coords"][w["faces"]]
    for nodes, xf in zip(_face_node_map(m, w), x):
        A = 0.5 * np.linalg.norm(np.cross(xf[1] - xf[0], xf[2] - xf[0]))
        Mf = _exact_mass(order, A)
        for a, na in enumerate(nodes):
            for b, nb in enumerate(nodes):
                expect[na, :, nb, :] += Mf[a, b] * Ks
    assert np.abs(K_springs - expect.reshape(3 * m.nn, 3 * m.nn)).max() <= 1e-12 * kperp * area


# ---------------------------------------------------------------- Eisenstat-Walker forcing
def test_ink_eta_sequence_from_recorded_norms():
    # eta_0 = ew_rtol0; eta_k = | ||R_k|| - ||R_{k-1} + K_{k-1} delta_k|| | / ||R_{k-1}||,
    # eta_k <- max(eta_k, eta_{k-1}^phi) when eta_{k-1}^phi > 0.1, phi = (1 + sqrt 5)/2,
    # eta_k <- min(eta_k, ew_rtolmax)
    w = W.cook(3, 3, 1, order=1, nu=0.3)
    load, tol = 0.8, 1e-10
    o = dict(ew_rtol0=0.3, ew_rtolmax=0.5)  # room for the safeguard and the cap to act

    def run(max_it):
        m = O.Mesh(w)
        m.set_load(load)
        d, st = m.solve("iNK", np.zeros(m.ndof), tol=tol, max_it=max_it, opts=o)
        return m, d, st

    m, dfin, st = run(50)
    assert st["status"] == 0
    nit = st["nit"]
    res, lres, eta = st["res_hist"], st["lres_hist"], st["eta_hist"]
    # the recorded linear residuals, recomputed from the iterates with a dense tangent
    prev = m.apply_dirichlet(np.zeros(m.ndof))
    for k in range(1, nit + 1):
        _, dk, _ = run(k)
        mk = O.Mesh(w)
        mk.set_load(load)
        rk1, _ = mk.residual(prev)
        mk.tangent(prev)
        K = oracle_dense_K(mk, w)
        lin = np.linalg.norm(rk1 + K @ (dk - prev))
        assert abs(lin - lres[k]) <= 1e-9 * max(lin, 1e-300) + 1e-14 * res[0], k
        prev = dk
    # the eta sequence from the recorded norms
    phi = 0.5 * (1.0 + math.sqrt(5.0))
    e = o["ew_rtol0"]
    assert eta[1] == e
    acted = set()
    for k in range(1, nit):
        cand = abs(res[k] - lres[k]) / res[k - 1]
        if e ** phi > 0.1:
            if e ** phi > cand:
                acted.add("safeguard")
            cand = max(cand, e ** phi)
        if cand > o["ew_rtolmax"]:
            acted.add("cap")
        e = min(cand, o["ew_rtolmax"])
        assert abs(eta[k + 1] - e) <= 1e-14 * e, k
    assert acted == {"safeguard", "cap"}  # both branches took part
