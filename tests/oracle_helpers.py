"""Helpers shared by the oracle pin tests and the GPU parity tests."""
import numpy as np

import workloads as W


def strip_bc(w):
    """Copy of a workload with no Dirichlet groups and no loaded faces."""
    w = dict(w)
    w["dir_group"] = np.zeros_like(w["dir_group"])
    w["groups"] = []
    w["faces"] = np.zeros((0, 3), dtype=np.int32)
    w["face_kind"] = np.zeros(0, dtype=np.int32)
    w["face_data"] = np.zeros((0, 3))
    return w


def dense_from_bcsr(nn, row_ptr, col, val, np_=0, up_ptr=None, up_col=None, bup=None):
    n = 3 * nn + np_
    K = np.zeros((n, n))
    for a in range(nn):
        for k in range(row_ptr[a], row_ptr[a + 1]):
            b = col[k]
            K[3 * a:3 * a + 3, 3 * b:3 * b + 3] = val[k]
    if np_ and bup is not None:
        for a in range(nn):
            for k in range(up_ptr[a], up_ptr[a + 1]):
                v = up_col[k]
                K[3 * a:3 * a + 3, 3 * nn + v] = bup[k]
                K[3 * nn + v, 3 * a:3 * a + 3] = bup[k]
    return K


def up_pattern(conn, tets, nn, pressure_order=1):
    """Brute-force pattern of the u-p coupling: u node rows; columns are the
    element's vertices (P1 pressure) or the element itself (P0)."""
    rows = [set() for _ in range(nn)]
    for e in range(conn.shape[0]):
        for a in conn[e]:
            rows[a].update([e] if pressure_order == 2 else [int(v) for v in tets[e]])
    ptr = np.zeros(nn + 1, dtype=np.int64)
    cols = []
    for a in range(nn):
        c = sorted(rows[a])
        cols.extend(c)
        ptr[a + 1] = ptr[a] + len(c)
    return ptr, np.array(cols, dtype=np.int64)


def oracle_dense_K(m, w):
    topo = m.topology()
    val, bup, _ = m.tangent_copy()
    if m.np_:
        up_ptr, up_col = up_pattern(topo["conn"], w["tets"], m.nn, w["pressure_order"])
        return dense_from_bcsr(m.nn, topo["row_ptr"], topo["col"], val, m.np_, up_ptr, up_col, bup)
    return dense_from_bcsr(m.nn, topo["row_ptr"], topo["col"], val)


def rotation(axis, angle):
    axis = np.asarray(axis, dtype=float)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


def small_cases():
    """Tiny meshes of every problem family (seconds on the oracle)."""
    return {
        "cook_p1": W.cook(4, 4, 2, order=1),
        "cook_p2": W.cook(3, 3, 1, order=2),
        "twist_up": W.twist(2, order=2),
        "twist_poly": W.twist(2, order=2, material="polyconvex"),
        "twist_p0": W.twist(2, order=2, pressure="P0", material="polyconvex"),
        "heart_p1": W.heart(nr=2, nc=8, nl=6),
    }
