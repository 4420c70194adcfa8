"""Deterministic synthetic inputs shaped like the paper's three test problems.

This module only builds geometry and load data: vertex coordinates, P1
tetrahedra from a Kuhn (Freudenthal) split of structured hexahedra, boundary
faces, Dirichlet vertex groups, fibre frames and load schedules.  It holds none
of the method's arithmetic (no shape functions, quadrature, constitutive law or
solver), so both the CPU oracle and the CUDA library can consume it.

Problems (paper, Section "Test problems and solvers details"):
  * Cook's membrane: trapezoid (0,0),(48,44),(48,60),(0,44) extruded to
    thickness 10, clamped on x=0, dead y-traction on x=48.
  * Twist: unit cube, bottom clamped, top rotated about the vertical axis
    through (0.5, 0.5) with the vertical component left free.
  * Cardiac-like: truncated prolate-ellipsoid shell with a helical fibre
    field, endocardial pressure and epicardial Robin springs.
The paper's own meshes, fibre fields and data files are not available; these
generators are stand-ins with the paper's shapes and sizes.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

# material kinds and face kinds, mirrored from include/fe.h
MAT_COOK_NH = 0
MAT_TH_NH = 1
MAT_GUCCIONE = 2
MAT_POLYCONVEX = 3
FACE_TRACTION = 0
FACE_PRESSURE = 1
FACE_ROBIN = 2
FACE_FOLLOWER = 3
FACE_DASHPOT = 4
FACE_TRACTION_DEFORMED = 5

_PERMS = list(itertools.permutations(range(3)))  # lexicographic order


def _perm_parity(p):
    inv = sum(1 for i in range(3) for j in range(i + 1, 3) if p[i] > p[j])
    return inv % 2


def kuhn_tets(nx, ny, nz, vid):
    """Split every hex of an nx*ny*nz grid into 6 tets.

    Tet p of the hex with lower corner (i,j,k) walks v0 -> +e_{pi1} -> +e_{pi2}
    -> +e_{pi3} for the axis permutation pi number p (lexicographic).  For odd
    permutations local vertices 2 and 3 are swapped so that, on an affine
    image of the unit cube with positive Jacobian, every tet has positive
    orientation.  ``vid(i, j, k)`` maps grid indices (arrays) to vertex ids.
    """
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    # hex order: lexicographic with i fastest
    I = I.transpose(2, 1, 0).ravel()
    J = J.transpose(2, 1, 0).ravel()
    K = K.transpose(2, 1, 0).ravel()
    tets = np.empty((I.size, 6, 4), dtype=np.int64)
    for p, perm in enumerate(_PERMS):
        off = np.zeros(3, dtype=np.int64)
        verts = [vid(I, J, K)]
        for ax in perm:
            off[ax] += 1
            verts.append(vid(I + off[0], J + off[1], K + off[2]))
        if _perm_parity(perm):
            verts[2], verts[3] = verts[3], verts[2]
        for a in range(4):
            tets[:, p, a] = verts[a]
    return tets.reshape(-1, 4).astype(np.int32)


def signed_volumes(coords, tets):
    x = coords[tets]
    d1 = x[:, 1] - x[:, 0]
    d2 = x[:, 2] - x[:, 0]
    d3 = x[:, 3] - x[:, 0]
    return np.einsum("ij,ij->i", d1, np.cross(d2, d3)) / 6.0


def orient_positive(coords, tets):
    """Swap local vertices 2 and 3 of any negatively oriented tet."""
    tets = tets.copy()
    neg = signed_volumes(coords, tets) < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    return tets


def boundary_faces(coords, tets):
    """Faces that belong to exactly one tet, ordered so that
    (x1-x0) x (x2-x0) points out of the tet."""
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    opp = np.array([0, 1, 2, 3])
    f = tets[:, loc].reshape(-1, 3)
    o = np.repeat(np.arange(tets.shape[0]), 4)
    ov = tets[np.arange(tets.shape[0])[:, None], opp[None, :]].reshape(-1)
    key = np.sort(f, axis=1)
    _, idx, cnt = np.unique(key, axis=0, return_index=True, return_counts=True)
    sel = idx[cnt == 1]
    faces = f[sel].copy()
    far = ov[sel]
    x = coords[faces]
    nrm = np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0])
    inward = np.einsum("ij,ij->i", nrm, coords[far] - x[:, 0]) > 0
    faces[inward, 1], faces[inward, 2] = faces[inward, 2].copy(), faces[inward, 1].copy()
    del o
    return faces.astype(np.int32)


def _workload(name, coords, tets, order, pressure_order, dir_group, groups,
              faces, face_kind, face_data, material, fibers, steps, **extra):
    w = dict(name=name, coords=np.ascontiguousarray(coords, dtype=np.float64),
             tets=np.ascontiguousarray(tets, dtype=np.int32), order=int(order),
             pressure_order=int(pressure_order),
             dir_group=np.ascontiguousarray(dir_group, dtype=np.uint8),
             groups=groups,
             faces=np.ascontiguousarray(faces, dtype=np.int32).reshape(-1, 3),
             face_kind=np.ascontiguousarray(face_kind, dtype=np.int32).reshape(-1),
             face_data=np.ascontiguousarray(face_data, dtype=np.float64).reshape(-1, 3),
             material=material,
             fibers=None if fibers is None else np.ascontiguousarray(fibers, dtype=np.float64),
             steps=steps)
    w.update(extra)
    return w


def cook(nx=8, ny=8, nz=2, order=1, E=1.0, nu=0.49, traction_scale=1.0,
         nsteps=5, vol_literal=0, follower=False):
    """Cook's membrane (paper: Cook test; sizes from the workload table).

    Map of the unit cube: x = 48 xi, y = 44 xi + eta (44 - 28 xi), z = 10 zeta.
    Vertex id = (k*(ny+1) + j)*(nx+1) + i.  Clamp on x = 0 (group 1, all
    components).  Dead traction (0, traction_scale/16, 0) per unit reference
    area on x = 48.  Load step s of nsteps scales the traction by s/nsteps.
    follower=True applies the traction per unit deformed area instead (face
    kind 5: the load "in the deformed configuration").
    """
    xi = np.linspace(0.0, 1.0, nx + 1)
    eta = np.linspace(0.0, 1.0, ny + 1)
    zeta = np.linspace(0.0, 1.0, nz + 1)
    Z, Y, X = np.meshgrid(zeta, eta, xi, indexing="ij")
    X = X.ravel(); Y = Y.ravel(); Z = Z.ravel()
    coords = np.stack([48.0 * X, 44.0 * X + Y * (44.0 - 28.0 * X), 10.0 * Z], axis=1)

    def vid(i, j, k):
        return (k * (ny + 1) + j) * (nx + 1) + i

    tets = kuhn_tets(nx, ny, nz, vid)
    ii = np.arange(coords.shape[0]) % (nx + 1)
    dir_group = np.where(ii == 0, 1, 0).astype(np.uint8)
    groups = [dict(mask=7, center=(0.0, 0.0, 0.0), angle=0.0, translation=(0.0, 0.0, 0.0))]
    bf = boundary_faces(coords, tets)
    on_right = np.all(np.isclose(coords[bf][:, :, 0], 48.0), axis=1)
    faces = bf[on_right]
    t = traction_scale / 16.0
    face_kind = np.full(faces.shape[0], FACE_TRACTION_DEFORMED if follower else FACE_TRACTION, dtype=np.int32)
    face_data = np.tile(np.array([0.0, t, 0.0]), (faces.shape[0], 1))
    material = dict(kind=MAT_COOK_NH, E=E, nu=nu, vol_literal=vol_literal)
    steps = [((s + 1) / nsteps, 0.0) for s in range(nsteps)]
    return _workload(f"cook_p{order}_{nx}x{ny}x{nz}" + ("_follower" if follower else ""), coords, tets, order, 0,
                     dir_group,
                     groups, faces, face_kind, face_data, material, None, steps,
                     nx=nx, ny=ny, nz=nz)


def twist(n=32, order=2, mu=1.0, total_angle=math.pi / 2, nsteps=10, pressure=True, material="neo_hookean",
          alpha_p=9000.0, beta_p=9000.0, alpha_s=9000.0, beta_s=9000.0):
    """Twist test stand-in: unit cube n^3 hexes, Taylor-Hood P2-P1 (u, p).

    pressure: True or "P1" (vertex pressures, Taylor-Hood), "P0" (one
    constant pressure per element: the paper's P2-P0 pair), False (none).

    Bottom z = 0 clamped (group 1, all components); top z = 1 (group 2):
    x and y components follow the rotation by load*total_angle about the
    vertical axis through (0.5, 0.5); the z component is free.
    material "neo_hookean": Psi = mu/2 (I1 - 3) - mu ln J - p (J - 1);
    "polyconvex": the paper's twist potential alpha_p (F:F - 3) +
    beta_p (cof F : cof F - 3) - (4 beta_s + 2 alpha_s) ln J - p (J - 1)
    (all four coefficients 9000 in the paper; stress-free at F = I when
    2 alpha_p + 4 beta_p = 4 beta_s + 2 alpha_s).
    """
    t1 = np.linspace(0.0, 1.0, n + 1)
    Z, Y, X = np.meshgrid(t1, t1, t1, indexing="ij")
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def vid(i, j, k):
        return (k * (n + 1) + j) * (n + 1) + i

    tets = kuhn_tets(n, n, n, vid)
    kk = np.arange(coords.shape[0]) // ((n + 1) * (n + 1))
    dir_group = np.zeros(coords.shape[0], dtype=np.uint8)
    dir_group[kk == 0] = 1
    dir_group[kk == n] = 2
    groups = [dict(mask=7, center=(0.0, 0.0, 0.0), angle=0.0, translation=(0.0, 0.0, 0.0)),
              dict(mask=3, center=(0.5, 0.5, 0.0), angle=total_angle,
                   translation=(0.0, 0.0, 0.0))]
    empty = np.zeros((0, 3))
    if material == "polyconvex":
        material = dict(kind=MAT_POLYCONVEX, alpha_p=alpha_p, beta_p=beta_p, c_log=4.0 * beta_s + 2.0 * alpha_s)
    else:
        material = dict(kind=MAT_TH_NH, mu=mu)
    steps = [((s + 1) / nsteps, 0.0) for s in range(nsteps)]
    pspace = {True: 1, "P1": 1, "P0": 2, False: 0, None: 0}[pressure]
    ptag = {0: "", 1: "p1", 2: "p0"}[pspace]
    return _workload(f"twist_p{order}{ptag}_{n}", coords, tets, order, pspace,
                     dir_group, groups, empty.astype(np.int32), np.zeros(0), empty,
                     material, None, steps, n=n)


def heart(nr=4, nc=80, nl=78, order=1, a_endo=2.0, c_endo=5.0, a_epi=3.0, c_epi=6.0,
          z_base=1.0, apex_hole=0.15, C=0.88, bf=18.5, bt=3.58, bfs=1.63, kappa=1.0e3,
          Ta_peak=60.0, period=0.8, p_endo=2.0, k_perp=20.0, k_par=2.0, nsteps=100,
          helix_endo_deg=60.0, helix_epi_deg=-60.0, dynamics=False, follower=False,
          rho=1.0, c_perp=2.0, c_par=0.2):
    """Truncated prolate-ellipsoid shell (cardiac-like test stand-in).

    Index space (i transmural 0..nr, j circumferential 0..nc periodic,
    k longitudinal 0..nl); point at transmural e = i/nr with semi-axes
    a(e), c(e) linear between endo and epi:
        x = a sin(th) cos(ph), y = a sin(th) sin(ph), z = c cos(th),
    with th from the base plane z = z_base (k = 0) to pi - apex_hole (k = nl),
    leaving a small apical opening (the structured grid has no apex point).
    Fibres per element from the hex centre: helix angle alpha(e) linear from
    helix_endo_deg (endo) to helix_epi_deg (epi); f = cos(alpha) e_circ +
    sin(alpha) e_long, s = e_circ x e_long (transmural), n = f x s.
    Loads per time step s (t = s*period/nsteps): endocardial pressure
    p_endo*max(sin(2 pi t/period), 0) as the load factor, activation time t.
    Epicardial Robin springs (k_perp, k_par); base and apex opening are free.

    follower=True makes the endocardial pressure a follower load (face kind
    3) instead of a dead one.  dynamics=True adds the inertia of the
    momentum equation and the dashpots of the epicardial Robin condition:
    duplicate epicardial faces of kind 4 with (c_perp, c_par), and the keys
    rho (density) and dt = period / nsteps of the Newmark steps.  The
    default rho = 1 is the momentum equation as printed (no density
    coefficient); in the units of this shell (cm, s, kPa) a tissue density of
    1050 kg / m^3 is rho = 1.05e-4 kPa s^2 / cm^2.  (k_perp, k_par) = (20, 2)
    kPa / cm, (c_perp, c_par) = (2, 0.2) kPa s / cm.
    """
    def geom(e, ph, tt):
        a = a_endo + e * (a_epi - a_endo)
        c = c_endo + e * (c_epi - c_endo)
        th0 = np.arccos(z_base / c)
        th = th0 + tt * (math.pi - apex_hole - th0)
        return a, c, th

    nvr, nvc, nvl = nr + 1, nc, nl + 1
    I, J, K = np.meshgrid(np.arange(nvr), np.arange(nvc), np.arange(nvl), indexing="ij")
    I = I.transpose(2, 1, 0).ravel(); J = J.transpose(2, 1, 0).ravel(); K = K.transpose(2, 1, 0).ravel()
    e = I / nr
    ph = 2.0 * math.pi * J / nc
    tt = K / nl
    a, c, th = geom(e, ph, tt)
    coords = np.stack([a * np.sin(th) * np.cos(ph), a * np.sin(th) * np.sin(ph), c * np.cos(th)], axis=1)

    def vid(i, j, k):
        return (k * nvc + (j % nc)) * nvr + i

    tets = kuhn_tets(nr, nc, nl, vid)
    tets = orient_positive(coords, tets)
    # fibres from the parameters of each hex centre (6 tets per hex, hex order i fastest)
    hi, hj, hk = np.meshgrid(np.arange(nr), np.arange(nc), np.arange(nl), indexing="ij")
    hi = hi.transpose(2, 1, 0).ravel(); hj = hj.transpose(2, 1, 0).ravel(); hk = hk.transpose(2, 1, 0).ravel()
    ec = (hi + 0.5) / nr
    phc = 2.0 * math.pi * (hj + 0.5) / nc
    tc = (hk + 0.5) / nl
    ac, cc, thc = geom(ec, phc, tc)
    ecirc = np.stack([-np.sin(phc), np.cos(phc), np.zeros_like(phc)], axis=1)
    dl = np.stack([ac * np.cos(thc) * np.cos(phc), ac * np.cos(thc) * np.sin(phc), -cc * np.sin(thc)], axis=1)
    elong = dl / np.linalg.norm(dl, axis=1, keepdims=True)
    s_ = np.cross(ecirc, elong)
    alpha = np.deg2rad(helix_endo_deg + ec * (helix_epi_deg - helix_endo_deg))
    f_ = np.cos(alpha)[:, None] * ecirc + np.sin(alpha)[:, None] * elong
    n_ = np.cross(f_, s_)
    frame = np.stack([f_, s_, n_], axis=1).reshape(-1, 9)
    fibers = np.repeat(frame, 6, axis=0)

    bfaces = boundary_faces(coords, tets)
    iv = np.arange(coords.shape[0]) % nvr
    endo = np.all(iv[bfaces] == 0, axis=1)
    epi = np.all(iv[bfaces] == nr, axis=1)
    faces = np.concatenate([bfaces[endo], bfaces[epi]])
    face_kind = np.concatenate([np.full(endo.sum(), FACE_FOLLOWER if follower else FACE_PRESSURE),
                                np.full(epi.sum(), FACE_ROBIN)]).astype(np.int32)
    face_data = np.concatenate([np.tile([p_endo, 0.0, 0.0], (endo.sum(), 1)),
                                np.tile([k_perp, k_par, 0.0], (epi.sum(), 1))])
    extra = {}
    if dynamics:
        faces = np.concatenate([faces, bfaces[epi]])
        face_kind = np.concatenate([face_kind, np.full(epi.sum(), FACE_DASHPOT, np.int32)])
        face_data = np.concatenate([face_data, np.tile([c_perp, c_par, 0.0], (epi.sum(), 1))])
        extra = dict(rho=float(rho), dt=float(period / nsteps))
    material = dict(kind=MAT_GUCCIONE, C=C, bf=bf, bt=bt, bfs=bfs, kappa=kappa,
                    Ta_peak=Ta_peak, period=period)
    steps = []
    for s in range(1, nsteps + 1):
        t = s * period / nsteps
        steps.append((max(math.sin(2.0 * math.pi * t / period), 0.0), t))
    dir_group = np.zeros(coords.shape[0], dtype=np.uint8)
    tag = ("_dyn" if dynamics else "") + ("_follower" if follower else "")
    return _workload(f"heart_p{order}_{nr}x{nc}x{nl}{tag}", coords, tets, order, 0, dir_group, [],
                     faces, face_kind, face_data, material, fibers, steps, **extra)


def serving_stream(nreq=256, seed=20220311, rate=1.0):
    """Seeded Poisson-arrival request stream for the serving mix.

    Each request: family in {cook, twist, heart}, a target size (log-uniform
    DoF in [1e3, 1e6] snapped to a structured resolution), nu ~ U[0.3,0.4999]
    and load scale ~ U[1, 16], arrival time from exponential gaps of mean
    1/rate.  Only the request descriptors are returned.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=nreq)
    arrivals = np.cumsum(gaps)
    fam = rng.integers(0, 3, size=nreq)
    dofs = np.exp(rng.uniform(math.log(1e3), math.log(1e6), size=nreq))
    nu = rng.uniform(0.3, 0.4999, size=nreq)
    load = rng.uniform(1.0, 16.0, size=nreq)
    reqs = []
    for r in range(nreq):
        reqs.append(dict(id=r, arrival=float(arrivals[r]), family=int(fam[r]),
                         dofs=float(dofs[r]), nu=float(nu[r]), load=float(load[r])))
    return reqs
