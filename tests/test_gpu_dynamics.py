"""GPU elastodynamics (Newmark average acceleration, consistent mass, Robin
dashpots) and follower pressure vs the oracle, through the C ABI.

Tolerances as in the static parity tests: assembled FP64 quantities to
1e-12 relative to their largest entry (two summation orders); Newmark steps
solved to ||R||/||R0|| <= 1e-11 agree to 1e-10 on the displacements, and
the velocities and accelerations derived from them, 2/dt (d - dtil) and
4/dt^2 (d - dhat), to 1e-10 and 1e-9 of their own magnitudes (the
differences of nearly equal displacements amplify the displacement gap).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import __graft_entry__ as g
    g.build()
    import paper_2203_05610_gb300 as fe
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return fe


def _cook_dyn():
    w = W.cook(4, 4, 2, order=2)
    bf = W.boundary_faces(w["coords"], w["tets"])
    top = np.all(np.isclose(w["coords"][bf][:, :, 2], 10.0), axis=1)
    return dict(w, faces=np.concatenate([w["faces"], bf[top]]),
                face_kind=np.concatenate([w["face_kind"], np.full(top.sum(), W.FACE_DASHPOT, np.int32)]),
                face_data=np.concatenate([w["face_data"], np.tile([0.3, 0.05, 0.0], (top.sum(), 1))]),
                rho=1.0, dt=2.0)


def _box_follower():
    """Unit cube, every boundary face a follower pressure, no Dirichlet."""
    n = 2
    g = np.linspace(0.0, 1.0, n + 1)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    coords = np.stack([X.ravel() + 0.1 * Y.ravel(), Y.ravel(), Z.ravel()], axis=1)
    tets = W.kuhn_tets(n, n, n, lambda i, j, k: (k * (n + 1) + j) * (n + 1) + i)
    faces = W.boundary_faces(coords, tets)
    return W._workload("box_follower", coords, tets, 2, 0, np.zeros(len(coords), np.uint8), [], faces,
                       np.full(len(faces), W.FACE_FOLLOWER, np.int32), np.tile([0.5, 0, 0], (len(faces), 1)),
                       dict(kind=W.MAT_COOK_NH, E=1.0, nu=0.3, vol_literal=0), None, [(1.0, 0.0)],
                       rho=0.0, dt=0.0)


CASES = {
    "heart_p1_dyn": lambda: W.heart(nr=2, nc=8, nl=6, dynamics=True, follower=True),
    "heart_p2_dyn": lambda: W.heart(nr=2, nc=8, nl=4, order=2, dynamics=True, follower=True),
    "cook_p2_dyn": _cook_dyn,
    "box_follower": _box_follower,
    "cook_p2_deformed_traction": lambda: W.cook(4, 4, 2, order=2, nu=0.3, follower=True),
}


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _pair(fe, w, seed=0, load=0.7, time=0.2):
    """GPU and oracle meshes with dynamics on (when the workload has it) and
    the same random Newmark state."""
    m, om = fe.Mesh(w), O.Mesh(w)
    m.set_load(load, time)
    om.set_load(load, time)
    if w.get("rho", 0.0) > 0.0:
        m.set_dynamics(w["rho"], w["dt"])
        om.set_dynamics(w["rho"], w["dt"])
        rng = np.random.default_rng(100 + seed)
        n3 = 3 * om.nn
        st = [0.01 * rng.standard_normal(n3), 0.1 * rng.standard_normal(n3), rng.standard_normal(n3)]
        om.dynamics_set(*st)
        m.dynamics_set(*[torch.from_numpy(x).cuda() for x in st])
    return m, om


@pytest.mark.parametrize("case", list(CASES))
def test_residual_energy_tangent(fe, case):
    w = CASES[case]()
    m, om = _pair(fe, w)
    rng = np.random.default_rng(7)
    d = 0.01 * rng.standard_normal(om.ndof)
    om.apply_dirichlet(d)
    dg = torch.from_numpy(d).cuda()
    r, n = om.residual(d)
    rg, ng = m.residual(dg)
    assert _rel(rg.cpu().numpy(), r) < 1e-12
    assert abs(ng - n) <= 1e-12 * n
    e = om.energy(d)
    assert abs(m.energy(dg) - e) <= 1e-12 * max(1.0, abs(e))
    om.tangent(d)
    m.tangent(dg, "fp64")
    v, _, di = om.tangent_copy()
    vg, _, dig = m.tangent_copy()
    assert _rel(vg, v) < 1e-12
    assert _rel(dig, di) < 1e-10
    x = rng.standard_normal(om.ndof)
    assert _rel(m.spmv(torch.from_numpy(x).cuda()).cpu().numpy(), om.spmv(x)) < 1e-12
    # FP32 storage of the same tangent: FP32 rounding of each entry
    m.tangent(dg, "mixed_fp32")
    v32, _, _ = m.tangent_copy()
    assert np.abs(v32 - v).max() <= 1e-6 * np.abs(v).max()
    if case.startswith("heart"):  # the follower pressure on the open endocardium
        K = v.reshape(-1, 9)
        assert np.abs(K).max() > 0


def test_follower_forces_on_a_closed_surface_balance(fe):
    """Net force and moment of the follower load vanish on the closed surface
    of the deformed box (both derived from the divergence theorem)."""
    w = _box_follower()
    m = fe.Mesh(w)
    m0 = fe.Mesh(dict(w, faces=w["faces"][:0], face_kind=w["face_kind"][:0], face_data=w["face_data"][:0]))
    m.set_load(1.0)
    m0.set_load(1.0)
    X = m.topology()["X"]
    d = (0.05 * np.sin(3.0 * X) + 0.02 * X[:, [1, 2, 0]] ** 2).ravel()
    dg = torch.from_numpy(d).cuda()
    f = (m.residual(dg)[0] - m0.residual(dg)[0]).cpu().numpy().reshape(-1, 3)
    assert np.abs(f).max() > 1e-3
    assert np.abs(f.sum(axis=0)).max() < 1e-13
    assert np.abs(np.cross(X + d.reshape(-1, 3), f).sum(axis=0)).max() < 1e-13


@pytest.mark.parametrize("case", ["heart_p1_dyn", "heart_p2_dyn", "cook_p2_dyn"])
def test_newmark_steps(fe, case):
    w = CASES[case]()
    m, om = fe.Mesh(w), O.Mesh(w)
    for mm in (m, om):
        mm.set_dynamics(w["rho"], w["dt"])
    opts = dict(ksp_atol=0.0)
    d = np.zeros(om.ndof)
    dg = torch.zeros(om.ndof, dtype=torch.float64, device="cuda")
    nsteps = 4
    # the P2 shell takes smaller load steps from rest (NK diverges at 0.25)
    dload = 0.05 if case == "heart_p2_dyn" else 0.25
    for s in range(1, nsteps + 1):
        load, time = (dload * s, 0.02 * s)
        m.set_load(load, time)
        om.set_load(load, time)
        d, so = om.solve("NK", d, tol=1e-11, max_it=25, opts=opts)
        dg, sg = m.solve("NK", dg, tol=1e-11, max_it=25, opts=opts)
        assert so["status"] == 0 and sg["status"] == 0, (s, so["res_hist"][-3:], sg["res_hist"][-3:])
        assert abs(sg["nit"] - so["nit"]) <= 1
        assert np.linalg.norm(dg.cpu().numpy() - d) <= 1e-10 * np.linalg.norm(d)
        om.dynamics_advance(d)
        m.dynamics_advance(dg)
        v, a = om.dynamics_get()
        vg, ag = m.dynamics_get()
        assert np.linalg.norm(vg.cpu().numpy() - v) <= 1e-10 * np.linalg.norm(v)
        assert np.linalg.norm(ag.cpu().numpy() - a) <= 1e-9 * np.linalg.norm(a)
        # the GPU's state is the Newmark update of its own solution
        dn = dg[: 3 * om.nn].cpu().numpy()
        assert np.linalg.norm(v) > 0 and np.linalg.norm(dn) > 0


@pytest.mark.parametrize("method", ["NK", "iNK", "B", "iB"])
def test_dynamic_heart_methods(fe, method):
    """One Newmark step of the dynamic cardiac stand-in with every method:
    same solution as the oracle, iteration counts within 10%."""
    w = CASES["heart_p1_dyn"]()
    m, om = fe.Mesh(w), O.Mesh(w)
    for mm in (m, om):
        mm.set_dynamics(w["rho"], w["dt"])
        mm.set_load(0.2, 0.05)  # at 0.5 the oracle's iB from rest diverges
    tol, xtol = (1e-8, 1e-6) if method == "B" else (1e-11, 1e-10)
    x, so = om.solve(method, np.zeros(om.ndof), tol=tol, opts=dict(ksp_atol=0.0))
    xg, sg = m.solve(method, torch.zeros(om.ndof, dtype=torch.float64, device="cuda"), tol=tol,
                     opts=dict(ksp_atol=0.0))
    assert so["status"] == 0 and sg["status"] == 0
    assert abs(sg["nit"] - so["nit"]) <= max(1, so["nit"] // 10)
    assert np.linalg.norm(xg.cpu().numpy() - x) <= xtol * np.linalg.norm(x)


@pytest.mark.parametrize("method", ["NK", "iNK"])
def test_deformed_area_traction_solve(fe, method):
    """Cook with its traction per unit deformed area (face kind 5, the load
    "in the deformed configuration"): the static solve matches the oracle."""
    w = W.cook(4, 4, 2, order=1, nu=0.3, follower=True)
    m, om = fe.Mesh(w), O.Mesh(w)
    for mm in (m, om):
        mm.set_load(0.5)
    x, so = om.solve(method, np.zeros(om.ndof), tol=1e-11, opts=dict(ksp_atol=0.0))
    xg, sg = m.solve(method, m.zeros(), tol=1e-11, opts=dict(ksp_atol=0.0))
    assert so["status"] == 0 and sg["status"] == 0
    assert abs(sg["nit"] - so["nit"]) <= 1
    assert np.linalg.norm(xg.cpu().numpy() - x) <= 1e-10 * np.linalg.norm(x)
    # not the dead-traction solution
    wd = W.cook(4, 4, 2, order=1, nu=0.3)
    od = O.Mesh(wd)
    od.set_load(0.5)
    xd, _ = od.solve(method, np.zeros(od.ndof), tol=1e-11, opts=dict(ksp_atol=0.0))
    assert np.linalg.norm(xd - x) > 1e-4 * np.linalg.norm(x)


def test_dynamics_switches_and_errors(fe):
    w = CASES["heart_p1_dyn"]()
    m = fe.Mesh(w)
    ref = fe.Mesh(w)
    m.set_load(0.6, 0.1)
    ref.set_load(0.6, 0.1)
    with pytest.raises(RuntimeError):
        m.dynamics_advance(m.zeros())  # dynamics is off
    with pytest.raises(RuntimeError):
        m.set_dynamics(float("nan"), 0.1)
    d = torch.from_numpy(0.01 * np.random.default_rng(1).standard_normal(m.ndof)).cuda()
    r0 = ref.residual(d)[0].cpu().numpy()
    m.set_dynamics(w["rho"], w["dt"])
    r1 = m.residual(d)[0].cpu().numpy()
    assert np.abs(r1 - r0).max() > 1e-6 * np.abs(r0).max()  # inertia and dashpots act
    m.set_dynamics(0.0, 0.0)  # static again: the dashpots leave the face values
    assert np.array_equal(m.residual(d)[0].cpu().numpy(), r0)
    m.set_dynamics(w["rho"], w["dt"])  # on again, state at rest
    assert np.array_equal(m.residual(d)[0].cpu().numpy(), r1)


def test_dynamic_cardiac_full_size(fe):
    """The cardiac configuration (4 x 80 x 78 hexes, 149,760 P1 tets) with
    inertia, dashpots and the follower endocardial pressure: residual and
    FP64 tangent against the oracle, every entry."""
    w = W.heart(dynamics=True, follower=True)
    m, om = _pair(fe, w, seed=3, load=0.8, time=0.3)
    rng = np.random.default_rng(11)
    d = 0.005 * rng.standard_normal(om.ndof)
    dg = torch.from_numpy(d).cuda()
    r, _ = om.residual(d)
    assert _rel(m.residual(dg)[0].cpu().numpy(), r) < 1e-12
    om.tangent(d)
    m.tangent(dg, "fp64")
    assert _rel(m.tangent_copy()[0], om.tangent_copy()[0]) < 1e-12
