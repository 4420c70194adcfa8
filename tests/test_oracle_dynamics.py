"""Pins of the oracle's elastodynamics and follower-pressure terms against
closed forms and independent restatements.

- Consistent mass (momentum equation with its inertia term, Section
  "Problem formulation"): on one tet, P1 against rho V/20 (1 + delta_ab)
  and P1/P2 against the test's own collapsed-coordinate Gauss quadrature of
  N_a N_b; on a whole mesh the entries sum to rho times the volume
  (partition of unity).
- Dashpots of the epicardial Robin condition (Eq. "bc epi", the C terms):
  2/dt C against the triangle mass matrix times c_perp N N^T + c_par (I - N N^T).
- Follower pressure: at d = 0 it equals the dead pressure; on a closed
  surface its nodal forces are p times the gradient of the enclosed volume
  and its tangent is p times the Hessian of that volume (the test computes
  the volume of the deformed isoparametric mesh with torch autograd); on an
  open surface the tangent is not symmetric and matches central
  differences of the residual, with inertia and dashpots on.
- Newmark average acceleration (the time integrator read into the paper):
  a single small-amplitude mode oscillates as cos(n Omega dt) with
  tan(Omega dt / 2) = omega dt / 2, the trapezoidal rule's closed-form
  frequency; with dashpots the discrete energy drops by exactly
  dt v_mid^T C v_mid per step (linear regime).
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import torch

import oracle as O
import workloads as W
from oracle_helpers import oracle_dense_K, strip_bc

RHO = 1.3
TET_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
TRI_EDGES = [(0, 1), (1, 2), (0, 2)]


# ---------------------------------------------------------------- independent quadrature and shapes
def tet_quadrature(n=6):
    """Collapsed (Duffy) Gauss-Legendre rule on the reference tet
    {xi, eta, zeta >= 0, xi + eta + zeta <= 1}; weights sum to 1/6."""
    g, gw = np.polynomial.legendre.leggauss(n)
    g = 0.5 * (g + 1.0)
    gw = 0.5 * gw
    pts, wts = [], []
    for u, wu in zip(g, gw):
        for v, wv in zip(g, gw):
            for s, ws in zip(g, gw):
                pts.append((u, v * (1 - u), s * (1 - u) * (1 - v)))
                wts.append(wu * wv * ws * (1 - u) ** 2 * (1 - v))
    return np.array(pts), np.array(wts)


def tri_quadrature(n=6):
    g, gw = np.polynomial.legendre.leggauss(n)
    g = 0.5 * (g + 1.0)
    gw = 0.5 * gw
    pts, wts = [], []
    for u, wu in zip(g, gw):
        for v, wv in zip(g, gw):
            pts.append((u, v * (1 - u)))
            wts.append(wu * wv * (1 - u))
    return np.array(pts), np.array(wts)


def lagrange(order, lam, edges):
    """P1: the barycentrics; P2: vertices l (2 l - 1), then 4 l_i l_j per edge."""
    if order == 1:
        return list(lam)
    return [l * (2 * l - 1) for l in lam] + [4 * lam[i] * lam[j] for i, j in edges]


def lagrange_dlam(order, lam, edges):
    """d N_a / d lambda_c as a list of lists (rows a)."""
    nl = len(lam)
    if order == 1:
        return [[1.0 if c == a else 0.0 for c in range(nl)] for a in range(nl)]
    rows = [[(4 * lam[a] - 1) if c == a else 0.0 for c in range(nl)] for a in range(nl)]
    for i, j in edges:
        r = [0.0] * nl
        r[i] = 4 * lam[j]
        r[j] = 4 * lam[i]
        rows.append(r)
    return rows


def one_tet(order, seed=3):
    rng = np.random.default_rng(seed)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) + 0.2 * rng.standard_normal((4, 3))
    tets = W.orient_positive(X, np.array([[0, 1, 2, 3]], dtype=np.int32))
    return W._workload("one_tet", X, tets, order, 0, np.zeros(4, np.uint8), [], np.zeros((0, 3)),
                       np.zeros(0), np.zeros((0, 3)), dict(kind=W.MAT_COOK_NH, E=1.0, nu=0.3, vol_literal=0),
                       None, [(1.0, 0.0)])


def box(n, order, face_kind=None, face_data=(1.0, 0.0, 0.0), seed=0):
    """Unit cube of n^3 hexes (6 tets each), slightly sheared; faces: all
    boundary triangles with the given kind (None: no faces); no Dirichlet."""
    nv = n + 1
    g = np.linspace(0.0, 1.0, nv)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    coords = np.stack([X.ravel() + 0.1 * Y.ravel(), Y.ravel() + 0.05 * Z.ravel(), Z.ravel()], axis=1)
    tets = W.kuhn_tets(n, n, n, lambda i, j, k: (k * nv + j) * nv + i)
    faces = W.boundary_faces(coords, tets) if face_kind is not None else np.zeros((0, 3), np.int32)
    kinds = np.full(faces.shape[0], face_kind if face_kind is not None else 0, np.int32)
    data = np.tile(np.array(face_data, float), (faces.shape[0], 1))
    return W._workload(f"box{n}", coords, tets, order, 0, np.zeros(coords.shape[0], np.uint8), [], faces,
                       kinds, data, dict(kind=W.MAT_COOK_NH, E=1.0, nu=0.3, vol_literal=0), None, [(1.0, 0.0)])


def dyn_difference(w, dt=2.0, rho=RHO, d=None):
    """Dense tangent with the Newmark terms minus the static one (same d)."""
    m = O.Mesh(w)
    d = np.zeros(m.ndof) if d is None else d
    m.tangent(d)
    K0 = oracle_dense_K(m, w)
    m.set_dynamics(rho, dt)
    m.tangent(d)
    K1 = oracle_dense_K(m, w)
    return m, K1 - K0


# ---------------------------------------------------------------- consistent mass
@pytest.mark.parametrize("order", [1, 2])
def test_consistent_mass_of_one_tet(order):
    w = one_tet(order)
    m, D = dyn_difference(w, dt=2.0)  # 4/dt^2 = 1
    topo = m.topology()
    conn = topo["conn"][0]
    X = w["coords"][w["tets"][0]]
    V = abs(np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]]))) / 6.0
    pts, wts = tet_quadrature()
    nen = 4 if order == 1 else 10
    Mref = np.zeros((nen, nen))
    for (xi, eta, zeta), wq in zip(pts, wts):
        N = np.array(lagrange(order, [1 - xi - eta - zeta, xi, eta, zeta], TET_EDGES))
        Mref += wq * 6.0 * V * RHO * np.outer(N, N)
    if order == 1:
        np.testing.assert_allclose(Mref, RHO * V / 20.0 * (np.ones((4, 4)) + np.eye(4)), rtol=1e-13)
    for a in range(nen):
        for b in range(nen):
            blk = D[3 * conn[a]:3 * conn[a] + 3, 3 * conn[b]:3 * conn[b] + 3]
            np.testing.assert_allclose(blk, Mref[a, b] * np.eye(3), rtol=1e-12, atol=1e-15)


def test_mass_sums_to_density_times_volume():
    w = strip_bc(W.cook(3, 3, 1, order=2))
    m, D = dyn_difference(w, dt=2.0)
    vol = W.signed_volumes(w["coords"], w["tets"]).sum()
    for i in range(3):
        assert D[i::3, i::3].sum() == pytest.approx(RHO * vol, rel=1e-12)
        off = D[i::3, (i + 1) % 3::3]
        assert np.abs(off).max() == 0.0


# ---------------------------------------------------------------- dashpots
@pytest.mark.parametrize("order", [1, 2])
def test_dashpot_matrix_against_the_face_mass(order):
    cperp, cpar, dt = 0.7, 0.2, 0.5
    base = strip_bc(W.cook(2, 2, 1, order=order))
    bf = W.boundary_faces(base["coords"], base["tets"])
    sel = np.all(np.isclose(base["coords"][bf][:, :, 2], 0.0), axis=1)  # bottom face z = 0
    faces = bf[sel]
    wf = dict(base, faces=faces, face_kind=np.full(len(faces), 4, np.int32),
              face_data=np.tile([cperp, cpar, 0.0], (len(faces), 1)))
    mA = O.Mesh(wf)
    mA.set_dynamics(RHO, dt)
    mA.tangent(np.zeros(mA.ndof))
    KA = oracle_dense_K(mA, wf)
    mB = O.Mesh(base)
    mB.set_dynamics(RHO, dt)
    mB.tangent(np.zeros(mB.ndof))
    KB = oracle_dense_K(mB, base)
    C = (KA - KB) * dt / 2.0
    # expected: sum over faces of int N_a N_b da (cperp N N^T + cpar (I - N N^T))
    topo = mA.topology()
    Xn = topo["X"]
    pts, wts = tri_quadrature()
    Cref = np.zeros_like(C)
    for f in faces:
        x = base["coords"][f]
        nrm = np.cross(x[1] - x[0], x[2] - x[0])
        A = 0.5 * np.linalg.norm(nrm)
        Nn = nrm / np.linalg.norm(nrm)
        Cs = cperp * np.outer(Nn, Nn) + cpar * (np.eye(3) - np.outer(Nn, Nn))
        nodes = list(f)
        if order == 2:  # mid-edge nodes of the face, found by position
            for i, j in TRI_EDGES:
                mid = 0.5 * (x[i] + x[j])
                nodes.append(int(np.argmin(np.linalg.norm(Xn - mid, axis=1))))
        mf = np.zeros((len(nodes), len(nodes)))
        for (u, v), wq in zip(pts, wts):
            N = np.array(lagrange(order, [1 - u - v, u, v], TRI_EDGES))
            mf += wq * 2.0 * A * np.outer(N, N)
        if order == 1:
            np.testing.assert_allclose(mf, A / 12.0 * (np.ones((3, 3)) + np.eye(3)), rtol=1e-13)
        for a, na in enumerate(nodes):
            for b, nb in enumerate(nodes):
                Cref[3 * na:3 * na + 3, 3 * nb:3 * nb + 3] += mf[a, b] * Cs
    np.testing.assert_allclose(C, Cref, rtol=1e-10, atol=1e-13)
    assert np.abs(Cref).max() > 0.01


# ---------------------------------------------------------------- follower pressure
def random_field(m, w, amp, seed):
    """Smooth displacement of every node (a low-order polynomial of X)."""
    X = m.topology()["X"]
    rng = np.random.default_rng(seed)
    A = amp * rng.standard_normal((3, 3))
    B = amp * rng.standard_normal((3, 3))
    return (X @ A.T + (X ** 2) @ B.T).ravel()


@pytest.mark.parametrize("order", [1, 2])
def test_follower_pressure_equals_dead_pressure_at_rest(order):
    p = 0.37
    wf = box(2, order, face_kind=3, face_data=(p, 0, 0))
    wd = box(2, order, face_kind=W.FACE_PRESSURE, face_data=(p, 0, 0))
    mf, md = O.Mesh(wf), O.Mesh(wd)
    mf.set_load(1.0)
    md.set_load(1.0)
    z = np.zeros(mf.ndof)
    rf, _ = mf.residual(z)
    rd, _ = md.residual(z)
    np.testing.assert_allclose(rf, rd, rtol=1e-12, atol=1e-15)
    assert np.abs(rd).max() > 1e-3
    d = random_field(mf, wf, 0.05, 1)
    rf1, _ = mf.residual(d)
    rd1, _ = md.residual(d)
    assert np.abs(rf1 - rd1).max() > 1e-3  # a follower load moves with the surface


def enclosed_volume(m, w, order):
    """Volume of the deformed isoparametric mesh, as a torch function of the
    nodal positions x [nn, 3]: sum over tets of int det(dx/dxi)."""
    conn = torch.as_tensor(m.topology()["conn"], dtype=torch.long)
    pts, wts = tet_quadrature(3 if order == 1 else 4)
    G = []  # per quadrature point: dN_a/dxi_j [nen, 3]
    for xi, eta, zeta in pts:
        dl = np.array(lagrange_dlam(order, [1 - xi - eta - zeta, xi, eta, zeta], TET_EDGES))
        G.append(dl[:, 1:] - dl[:, :1])
    G = torch.as_tensor(np.array(G))
    wq = torch.as_tensor(wts)

    def V(x):
        xe = x[conn]  # [ne, nen, 3]
        J = torch.einsum("qaj,eai->eqij", G, xe)
        return (torch.linalg.det(J) * wq).sum()

    return V


@pytest.mark.parametrize("order", [1, 2])
def test_follower_pressure_on_a_closed_surface_is_the_volume_gradient(order):
    p = 0.8
    wf = box(2, order, face_kind=3, face_data=(p, 0, 0))
    w0 = box(2, order)
    mf, m0 = O.Mesh(wf), O.Mesh(w0)
    mf.set_load(1.0)
    d = random_field(mf, wf, 0.08, 2)
    rf, _ = mf.residual(d)
    r0, _ = m0.residual(d)
    force = (rf - r0).reshape(-1, 3)
    X = mf.topology()["X"]
    V = enclosed_volume(mf, wf, order)
    x = torch.tensor(X + d.reshape(-1, 3), requires_grad=True)
    (g,) = torch.autograd.grad(V(x), x)
    np.testing.assert_allclose(force, p * g.numpy(), rtol=1e-10, atol=1e-12)
    assert np.abs(force).max() > 1e-3
    # net force and moment of the follower load vanish on a closed surface
    assert np.abs(force.sum(axis=0)).max() < 1e-12
    assert np.abs(np.cross(X + d.reshape(-1, 3), force).sum(axis=0)).max() < 1e-12
    # its tangent is p times the Hessian of the enclosed volume (symmetric here)
    mf.tangent(d)
    m0.tangent(d)
    Kf = oracle_dense_K(mf, wf) - oracle_dense_K(m0, w0)
    H = torch.autograd.functional.hessian(lambda y: V(y.reshape(-1, 3)), x.detach().reshape(-1)).numpy()
    np.testing.assert_allclose(Kf, p * H, rtol=1e-9, atol=1e-11)
    assert np.abs(Kf).max() > 1e-3


def fd_jacobian(m, d, h=1e-6):
    J = np.zeros((m.ndof, m.ndof))
    for j in range(m.ndof):
        e = np.zeros(m.ndof)
        e[j] = h
        rp, _ = m.residual(d + e)
        rm, _ = m.residual(d - e)
        J[:, j] = (rp - rm) / (2 * h)
    return J


@pytest.mark.parametrize("order", [1, 2])
def test_dynamic_tangent_matches_finite_differences(order):
    """Whole tangent (Guccione, springs, follower pressure, inertia,
    dashpots) and its follower part alone (follower minus dead pressure,
    whose tangent is zero) against central differences of the residual."""
    w = W.heart(nr=1, nc=6, nl=3, order=order, dynamics=True, follower=True)
    wd = W.heart(nr=1, nc=6, nl=3, order=order, dynamics=True, follower=False)
    assert W.FACE_FOLLOWER in set(w["face_kind"]) and W.FACE_DASHPOT in set(w["face_kind"])
    rng = np.random.default_rng(5)
    Ks, Js = [], []
    for wk in (w, wd):
        m = O.Mesh(wk)
        m.set_load(0.7, 0.2)
        m.set_dynamics(wk["rho"], wk["dt"])
        r2 = np.random.default_rng(6)
        n3 = 3 * m.nn
        m.dynamics_set(0.01 * r2.standard_normal(n3), 0.1 * r2.standard_normal(n3), r2.standard_normal(n3))
        d = 0.005 * np.random.default_rng(7).standard_normal(m.ndof)
        m.tangent(d)
        Ks.append(oracle_dense_K(m, wk))
        Js.append(fd_jacobian(m, d))
    K, Kfd = Ks[0], Js[0]
    assert np.abs(K - Kfd).max() < 1e-7 * np.abs(K).max()
    Kf, Kffd = Ks[0] - Ks[1], Js[0] - Js[1]
    fscale = np.abs(Kf).max()
    assert fscale > 0.1
    assert np.abs(Kf - Kffd).max() < 1e-6 * fscale
    # the follower pressure on the open endocardium makes the tangent nonsymmetric
    assert np.abs(K - K.T).max() > 0.05 * fscale
    assert np.abs(Ks[1] - Ks[1].T).max() < 1e-9 * np.abs(Ks[1]).max()
    del rng


# ---------------------------------------------------------------- Newmark average acceleration
def clamped_cook():
    return W.cook(4, 4, 1, order=1)


def free_dofs(m):
    """Components that no Dirichlet group prescribes (the clamp of this
    workload prescribes zeros, so apply_dirichlet zeroes exactly those)."""
    x = np.ones(m.ndof)
    m.apply_dirichlet(x)
    return x != 0.0


def modal_setup(w, dt_omega):
    """Stiffness and mass at rest (no dashpots in w) and the lowest mode of
    K phi = omega^2 M phi on the free components."""
    m = O.Mesh(w)
    m.set_load(0.0)
    z = np.zeros(m.ndof)
    m.tangent(z)
    K = oracle_dense_K(m, w)
    m.set_dynamics(RHO, 2.0)
    m.tangent(z)
    M = oracle_dense_K(m, w) - K  # 4/dt^2 = 1
    free = free_dofs(m)
    lam, phi = sla.eigh(K[np.ix_(free, free)], M[np.ix_(free, free)])
    omega = math.sqrt(lam[0])
    mode = np.zeros(m.ndof)
    mode[free] = phi[:, 0]
    for A in (K, M):
        A[~free, :] = 0.0
        A[:, ~free] = 0.0
    return K, M, free, omega, dt_omega / omega, mode


def newmark_steps(m, d0, v0, a0, nsteps):
    """Newmark steps solved by NK; a step is converged when the residual is
    1e-7 of its initial value or at the absolute floor of the residual's
    rounding (about 1e-12 at these amplitudes)."""
    m.dynamics_set(d0, v0, a0)
    d = d0.copy()
    out = [d.copy()]
    for _ in range(nsteps):
        d, st = m.solve("NK", d, tol=1e-7, max_it=8, opts=dict(ksp_rtol=1e-13, ksp_atol=0.0))
        assert st["status"] == 0 or st["rfinal"] < 1e-10
        m.dynamics_advance(d)
        out.append(d.copy())
    return out


def test_newmark_single_mode_has_the_trapezoidal_frequency():
    w = clamped_cook()
    K, M, free, omega, dt, mode = modal_setup(w, dt_omega=1.0)
    m = O.Mesh(w)
    m.set_load(0.0)
    m.set_dynamics(RHO, dt)
    eps = 1e-4 / np.abs(mode).max()
    d0 = eps * mode
    hist = newmark_steps(m, d0, None, -omega ** 2 * d0, 12)
    Omega = 2.0 * math.atan(0.5 * omega * dt) / dt
    mm = mode @ M @ mode
    for n, d in enumerate(hist):
        q = (mode @ M @ d) / (mm * eps)
        assert q == pytest.approx(math.cos(n * Omega * dt), abs=5e-6)
    # distinct from the continuous frequency (the test discriminates)
    assert abs(math.cos(12 * Omega * dt) - math.cos(12 * omega * dt)) > 0.1


def test_newmark_energy_balance_with_dashpots():
    base = clamped_cook()
    bf = W.boundary_faces(base["coords"], base["tets"])
    top = np.all(np.isclose(base["coords"][bf][:, :, 2], 10.0), axis=1)
    w = dict(base, faces=np.concatenate([base["faces"], bf[top]]),
             face_kind=np.concatenate([base["face_kind"], np.full(top.sum(), W.FACE_DASHPOT, np.int32)]),
             face_data=np.concatenate([base["face_data"], np.tile([0.02, 0.005, 0.0], (top.sum(), 1))]))
    K, M, free, omega, dt, mode = modal_setup(base, dt_omega=0.5)
    m = O.Mesh(w)
    m.set_load(0.0)
    m.set_dynamics(RHO, dt)
    m.tangent(np.zeros(m.ndof))
    mB = O.Mesh(base)
    mB.set_load(0.0)
    mB.set_dynamics(RHO, dt)
    mB.tangent(np.zeros(mB.ndof))
    C = (oracle_dense_K(m, w) - oracle_dense_K(mB, base)) * dt / 2.0
    C[~free, :] = 0.0
    C[:, ~free] = 0.0
    eps = 1e-4 / np.abs(mode).max()
    d0 = eps * mode
    hist = newmark_steps(m, d0, None, -omega ** 2 * d0, 8)
    v = np.zeros(m.ndof)
    E = [0.5 * d0 @ K @ d0]
    drops = []
    for dprev, d in zip(hist[:-1], hist[1:]):
        vn = 2.0 / dt * (d - dprev) - v  # Newmark velocity update
        vm = 0.5 * (v + vn)
        E.append(0.5 * vn @ M @ vn + 0.5 * d @ K @ d)
        drops.append(dt * vm @ C @ vm)
        v = vn
    v_or, _ = m.dynamics_get()
    np.testing.assert_allclose(v_or, v[: 3 * m.nn], rtol=1e-9, atol=1e-9 * np.abs(v).max())
    for k in range(len(drops)):
        assert E[k] - E[k + 1] == pytest.approx(drops[k], rel=1e-4)
    assert sum(drops) > 1e-3 * E[0]  # the dashpots really dissipate


# ---------------------------------------------------------------- traction per unit deformed area
def _one_face_box(order, kind, t):
    """The box with a traction on its x = max face only."""
    w = box(2, order)
    bf = W.boundary_faces(w["coords"], w["tets"])
    c = w["coords"]
    Xref = c[:, 0] - 0.1 * (c[:, 1] - 0.05 * c[:, 2])  # the unit-cube coordinate before the shear
    right = bf[np.all(np.isclose(Xref[bf], 1.0), axis=1)]
    assert len(right) == 8
    return dict(w, faces=right, face_kind=np.full(len(right), kind, np.int32),
                face_data=np.tile(np.array(t, float), (len(right), 1)))


@pytest.mark.parametrize("order", [1, 2])
def test_deformed_area_traction(order):
    """Face kind 5 (traction per unit deformed area): equal to the dead
    traction at d = 0; under an affine map x = F X its total force is t
    times the deformed area A |cof(F) N| (Nanson); its tangent matches
    central differences of the residual and is not symmetric."""
    t = (0.3, -0.2, 0.5)
    w5, w0 = _one_face_box(order, 5, t), _one_face_box(order, W.FACE_TRACTION, t)
    wn = dict(w5, faces=w5["faces"][:0], face_kind=w5["face_kind"][:0], face_data=w5["face_data"][:0])
    m5, m0, mn = O.Mesh(w5), O.Mesh(w0), O.Mesh(wn)
    for mm in (m5, m0, mn):
        mm.set_load(1.0)
    z = np.zeros(m5.ndof)
    np.testing.assert_allclose(m5.residual(z)[0], m0.residual(z)[0], rtol=1e-12, atol=1e-15)
    X = m5.topology()["X"]
    F = np.array([[1.2, 0.1, 0.05], [-0.1, 0.9, 0.2], [0.0, 0.15, 1.1]])
    d = ((X @ F.T) - X).ravel()
    f = (m5.residual(d)[0] - mn.residual(d)[0]).reshape(-1, 3)
    x = w5["coords"][w5["faces"][0]]
    nrm = np.cross(x[1] - x[0], x[2] - x[0])
    N = nrm / np.linalg.norm(nrm)
    A = sum(0.5 * np.linalg.norm(np.cross(*(w5["coords"][fc][1:] - w5["coords"][fc][0]))) for fc in w5["faces"])
    cof = np.linalg.det(F) * np.linalg.inv(F).T
    area = A * np.linalg.norm(cof @ N)
    np.testing.assert_allclose(f.sum(axis=0), -np.array(t) * area, rtol=1e-12)
    # tangent of the traction part against central differences
    d = random_field(m5, w5, 0.05, 9)
    m5.tangent(d)
    mn.tangent(d)
    Kt = oracle_dense_K(m5, w5) - oracle_dense_K(mn, wn)
    Kfd = fd_jacobian(m5, d) - fd_jacobian(mn, d)
    assert np.abs(Kt).max() > 1e-3
    assert np.abs(Kt - Kfd).max() < 1e-7 * np.abs(Kt).max()
    assert np.abs(Kt - Kt.T).max() > 1e-3 * np.abs(Kt).max()
