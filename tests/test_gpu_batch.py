"""Many small solves in one launch (include/fe_batch.h) vs the oracle, and
batch independence.

Bars: FP64 requests solved to ||R||/||R0|| <= 1e-11 agree with the oracle
to 1e-10 on the displacements (the FP64 target of the single-solve path),
with nonlinear iteration counts within one; mixed FP32 requests meet the
same residual target with a displacement error at most the mixed factor
of the single-solve tests times the FP64 bound.  A request gives
bit-identical results alone and inside a batch of other requests.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle_helpers import small_cases
from test_gpu_amg import MIXED_FACTOR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import __graft_entry__ as g
    g.build()
    import paper_2203_05610_gb300 as fe
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return fe


LOADS = {"cook_p1": (0.4, 0.0), "cook_p2": (0.4, 0.0), "heart_p1": (0.2, 0.01)}
OPTS = dict(ksp_atol=0.0, ksp_restart=50)


def _case(c):
    """The small families; the P2 Cook case at nu = 0.3 (at 0.49, GMRES(50)
    with block-Jacobi stagnates and iB from rest diverges in the oracle)."""
    return W.cook(3, 3, 1, order=2, nu=0.3) if c == "cook_p2" else small_cases()[c]


def _requests(fe, cases, prec="fp64"):
    ms, ds = [], []
    for c in cases:
        m = fe.Mesh(_case(c))
        m.set_load(*LOADS[c])
        ms.append(m)
        ds.append(m.zeros())
    return ms, ds


@pytest.mark.parametrize("method", ["NK", "iNK", "B", "iB"])
def test_batch_matches_the_oracle_fp64(fe, method):
    cases = ["cook_p1", "cook_p2", "heart_p1"]
    ms, ds = _requests(fe, cases)
    tol = 1e-8 if method == "B" else 1e-11
    opts = dict(OPTS, precision="fp64")
    for m in ms:
        assert fe.batch_supported(m, method, opts)
    st = fe.batch_solve(ms, [method] * len(ms), ds, [tol] * len(ms), opts=opts)
    for c, m, d, s in zip(cases, ms, ds, st):
        om = O.Mesh(_case(c))
        om.set_load(*LOADS[c])
        x, so = om.solve(method, np.zeros(om.ndof), tol=tol,
                         opts=dict(ksp_atol=0.0, ksp_restart=50))
        assert so["status"] == 0 and s["status"] == 0, (c, so["status"], s["status"], s["res_hist"][-3:])
        assert abs(s["nit"] - so["nit"]) <= max(1, so["nit"] // 10), (c, s["nit"], so["nit"])
        xtol = 1e-6 if method == "B" else 1e-10
        assert np.linalg.norm(d.cpu().numpy() - x) <= xtol * np.linalg.norm(x), c
        assert s["rfinal"] <= tol * s["r0"]


@pytest.mark.parametrize("method", ["iNK", "iB"])
def test_batch_mixed_precision_error(fe, method):
    """The mixed form's error against the oracle is at most MIXED_FACTOR
    times the FP64 form's at the same residual (the single-solve bar)."""
    cases = ["cook_p1", "heart_p1"]
    errs, rrel = {}, {}
    for prec in ("fp64", "mixed_fp32"):
        ms, ds = _requests(fe, cases)
        st = fe.batch_solve(ms, [method] * 2, ds, [1e-11] * 2, opts=dict(OPTS, precision=prec))
        errs[prec], rrel[prec] = [], []
        for c, d, s_ in zip(cases, ds, st):
            om = O.Mesh(_case(c))
            om.set_load(*LOADS[c])
            x, so = om.solve("NK", np.zeros(om.ndof), tol=1e-12, opts=dict(ksp_rtol=1e-12, ksp_atol=0.0))
            assert s_["status"] == 0, (c, prec, s_["res_hist"][-3:])
            errs[prec].append(np.linalg.norm(d.cpu().numpy() - x) / np.linalg.norm(x))
            rrel[prec].append(s_["rfinal"] / s_["r0"])
    for i, c in enumerate(cases):
        bound = MIXED_FACTOR * max(errs["fp64"][i] * max(1.0, rrel["mixed_fp32"][i] / rrel["fp64"][i]), 1e-12)
        assert errs["mixed_fp32"][i] <= bound, (c, errs, rrel)


def test_alone_and_in_a_batch_are_bit_identical(fe):
    cases = ["cook_p1", "heart_p1", "cook_p2", "cook_p1"]
    methods = ["iNK", "iB", "NK", "B"]
    tols = [1e-10, 1e-10, 1e-10, 1e-8]
    opts = dict(OPTS, precision="mixed_fp32")
    ms, ds = _requests(fe, cases)
    st_mix = fe.batch_solve(ms, methods, ds, tols, opts=opts)
    for i in range(len(cases)):
        m1, d1 = _requests(fe, [cases[i]])
        st1 = fe.batch_solve(m1, [methods[i]], d1, [tols[i]], opts=opts)
        assert torch.equal(d1[0], ds[i]), i
        assert st1[0]["nit"] == st_mix[i]["nit"] and st1[0]["lit_total"] == st_mix[i]["lit_total"]
        assert np.array_equal(st1[0]["res_hist"], st_mix[i]["res_hist"])


def test_batch_agrees_with_the_single_solve_path(fe):
    c = "cook_p2"
    ms, ds = _requests(fe, [c])
    st = fe.batch_solve(ms, ["NK"], ds, [1e-11], opts=dict(OPTS, precision="fp64"), threads=128)
    m = fe.Mesh(_case(c))
    m.set_load(*LOADS[c])
    d = m.zeros()
    _, s1 = m.solve("NK", d, tol=1e-11, opts=dict(OPTS, precision="fp64"))
    assert st[0]["status"] == 0 and s1["status"] == 0
    assert abs(st[0]["nit"] - s1["nit"]) <= 1  # tol 1e-11 sits near the FP64 floor
    assert torch.linalg.norm(ds[0] - d) <= 1e-10 * torch.linalg.norm(d)


def test_unsupported_requests_are_rejected(fe):
    m_up = fe.Mesh(small_cases()["twist_up"])
    assert not fe.batch_supported(m_up, "NK", OPTS)
    m = fe.Mesh(small_cases()["cook_p1"])
    assert not fe.batch_supported(m, "NK", dict(ksp_restart=500))  # H would not fit in shared memory
    assert not fe.batch_supported(m, "NK", dict(OPTS, pc_type="amg"))
    with pytest.raises(RuntimeError):
        fe.batch_solve([m_up], ["NK"], [m_up.zeros()], [1e-8], opts=OPTS)


def test_launch_shape_does_not_change_the_result(fe):
    """128 and 256 threads per CTA (the autotuner's two shapes) give
    bit-identical solutions: the CTA reductions use 256 virtual lanes."""
    cases = ["cook_p1", "heart_p1"]
    out = {}
    for nt in (128, 256):
        ms, ds = _requests(fe, cases)
        st = fe.batch_solve(ms, ["iNK", "iB"], ds, [1e-10, 1e-10], opts=dict(OPTS, precision="mixed_fp32"),
                            threads=nt)
        out[nt] = (ds, st)
    for i in range(len(cases)):
        assert torch.equal(out[128][0][i], out[256][0][i]), cases[i]
        assert np.array_equal(out[128][1][i]["res_hist"], out[256][1][i]["res_hist"])
