"""fe_spmv_noalloc, the SpMV entry point that allocates no device memory.

Callers that cannot allocate while they run (a serving loop whose memory
pool already owns the free device memory, or code that must avoid the
device-wide synchronisation an allocation can cause) use it instead of
fe_spmv.  It must give the same product as fe_spmv, call after call, since
both run the same SpMV kernel; only where the converted input is staged
differs (a fixed library array instead of a lazily allocated buffer).  The
calls are checked first on a fresh mesh, before fe_spmv has allocated its
own buffer, with the free device memory (cudaMemGetInfo) and the mesh's
device byte count unchanged across them.
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


def _noalloc(fe, m, x, y):
    rc = fe.lib().fe_spmv_noalloc(m.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()))
    if rc != 0:
        raise fe.FEError(rc, fe.lib().fe_last_error().decode())
    return y


def _device_bytes(fe, m):
    info = fe.fe_mesh_info()
    assert fe.lib().fe_mesh_get_info(m.h, ctypes.byref(info)) == 0
    return int(info.device_bytes)


CASES = {
    "cook_p2_fp64": (lambda: W.cook(6, 6, 2, order=2, nu=0.3), "fp64"),
    "cook_p2_fp32": (lambda: W.cook(6, 6, 2, order=2, nu=0.3), "mixed_fp32"),
    "cook_p2_bf16": (lambda: W.cook(6, 6, 2, order=2, nu=0.3), "mixed_bf16"),
    "twist_up_fp64": (lambda: W.twist(3, order=2), "fp64"),
    "twist_up_fp32": (lambda: W.twist(3, order=2), "mixed_fp32"),
}


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_spmv_matches_fe_spmv(fe, case):
    make, precision = CASES[case]
    w = make()
    m = fe.Mesh(w)  # fresh mesh: fe_spmv has not allocated its input buffer
    m.set_load(0.3)
    rng = np.random.default_rng(21)
    d = torch.from_numpy(0.05 * rng.standard_normal(m.ndof)).cuda()
    m.apply_dirichlet(d)
    m.tangent(d, precision)
    xs = [torch.from_numpy(rng.standard_normal(m.ndof)).cuda() for _ in range(3)]
    ys = [m.zeros() for _ in range(3)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    bytes0 = _device_bytes(fe, m)
    for x, y in zip(xs, ys):  # calls in a row: the shared array keeps the last input
        _noalloc(fe, m, x, y)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert _device_bytes(fe, m) == bytes0
    for call, (x, y) in enumerate(zip(xs, ys)):
        y_ref = m.spmv(x).cpu().numpy()
        assert np.abs(y.cpu().numpy() - y_ref).max() <= 1e-12 * np.abs(y_ref).max(), call


def test_noalloc_spmv_needs_a_tangent(fe):
    m = fe.Mesh(W.cook(3, 3, 1, order=1))
    x, y = m.zeros(), m.zeros()
    with pytest.raises(fe.FEError) as e:
        _noalloc(fe, m, x, y)
    assert e.value.code == -6


def test_noalloc_spmv_rejects_meshes_beyond_its_array(fe):
    w = W.cook(72, 72, 8, order=2)  # 1,072,275 unknowns > 2^20
    m = fe.Mesh(w)
    assert m.ndof > (1 << 20)
    x = m.zeros()
    with pytest.raises(fe.FEError) as e:
        _noalloc(fe, m, x, m.zeros())
    assert e.value.code == -1 and "at most" in str(e.value)
