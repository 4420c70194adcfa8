"""fe_spmv_noalloc, the SpMV entry point that allocates no device memory.

Callers that cannot allocate while they run (a serving loop whose memory
pool already owns the free device memory, or code that must avoid the
device-wide synchronisation an allocation can cause) use it instead of
fe_spmv.  It must give the same product as fe_spmv, call after call, since
both run the same SpMV kernel; only where the converted input is staged
differs (a fixed library array instead of a lazily allocated buffer).
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

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


def _noalloc(fe, m, x):
    y = m.zeros()
    rc = fe.lib().fe_spmv_noalloc(m.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()))
    if rc != 0:
        raise fe.FEError(rc, fe.lib().fe_last_error().decode())
    return y


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_noalloc_spmv_matches_fe_spmv(fe, precision):
    w = W.cook(6, 6, 2, order=2, nu=0.3)
    m = fe.Mesh(w)
    m.set_load(0.5)
    rng = np.random.default_rng(21)
    d = torch.from_numpy(0.05 * rng.standard_normal(m.ndof)).cuda()
    m.apply_dirichlet(d)
    m.tangent(d, precision)
    for call in range(2):  # two calls in a row: the shared array keeps the last input
        x = torch.from_numpy(rng.standard_normal(m.ndof)).cuda()
        y_ref = m.spmv(x).cpu().numpy()
        y = _noalloc(fe, m, x).cpu().numpy()
        assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max(), call


def test_noalloc_spmv_rejects_meshes_beyond_its_array(fe):
    w = W.cook(72, 72, 8, order=2)  # 1,072,275 unknowns > 2^20
    m = fe.Mesh(w)
    assert m.ndof > (1 << 20)
    x = m.zeros()
    with pytest.raises(fe.FEError) as e:
        _noalloc(fe, m, x)
    assert e.value.code == -1 and "at most" in str(e.value)
