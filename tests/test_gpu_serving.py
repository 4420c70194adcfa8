"""Serving loop: continuous batching of nonlinear solves on one GPU.

Each request's result must be the same alone and in the mix (same kernels,
same launch shapes, deterministic reductions: compared at 1e-12 relative);
admitted requests overlap on the device; requests that can never fit the
HBM budget are rejected at admission.
"""
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


def _requests():
    return [
        (W.cook(4, 4, 2, order=1, nu=0.3), "NK", dict(precision="fp64", ksp_atol=0.0), (0.4, 0.0)),
        (W.cook(3, 3, 1, order=2, nu=0.3), "iB", dict(precision="mixed_fp32"), (0.4, 0.0)),
        (W.twist(2, order=2), "iNK", dict(precision="fp64"), (0.3, 0.0)),
        (W.heart(nr=2, nc=8, nl=6), "B", dict(precision="fp64"), (0.2, 0.01)),
        (W.cook(8, 8, 2, order=1, nu=0.49), "iNK", dict(precision="mixed_fp32"), (0.2, 0.0)),
        (W.cook(6, 6, 2, order=2, nu=0.3), "NK", dict(precision="mixed_fp32"), (0.2, 0.0)),
    ]


def test_alone_and_in_the_mix_agree(fe):
    reqs = _requests()
    alone = []
    for w, meth, opts, (load, tm) in reqs:
        m = fe.Mesh(w)
        m.set_load(load, tm)
        d, st = m.solve(meth, m.zeros(), tol=1e-8, opts=opts)
        assert st["status"] == 0, (meth, st["res_hist"][-3:])
        alone.append(d.cpu().numpy())
        m.close()
    srv = fe.Server(max_active=4)
    ids = [srv.submit(w, meth, tol=1e-8, opts=opts, load=load, time=tm) for w, meth, opts, (load, tm) in reqs]
    res = [srv.poll(i, wait=True) for i in ids]
    srv.close()
    for r, a, (w, meth, _, _) in zip(res, alone, reqs):
        assert r["state"] == "done" and r["result"] == 0, (meth, r)
        assert np.abs(r["d"] - a).max() <= 1e-12 * np.abs(a).max(), meth
    # admitted requests overlap on the device: some request started before another ended
    spans = sorted((r["t_start"], r["t_end"]) for r in res)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))


def test_one_slot_runs_requests_one_after_another(fe):
    srv = fe.Server(max_active=1)
    w = W.cook(4, 4, 2, order=1, nu=0.3)
    ids = [srv.submit(w, "NK", load=0.1 * (k + 1)) for k in range(3)]
    res = [srv.poll(i, wait=True) for i in ids]
    srv.close()
    assert all(r["state"] == "done" for r in res)
    for a, b in zip(res, res[1:]):
        assert b["t_start"] >= a["t_end"] - 1e-6


def test_admission_rejects_requests_beyond_the_budget(fe):
    srv = fe.Server(hbm_budget=1 << 20, max_active=2)  # 1 MiB: no mesh fits
    rid = srv.submit(W.cook(4, 4, 2, order=1), "NK", load=0.1)
    r = srv.poll(rid, wait=True)
    srv.close()
    assert r["state"] == "failed" and r["result"] == -2 and "budget" in r["error"]


def _small_requests():
    o64 = dict(precision="fp64", ksp_atol=0.0, ksp_restart=30)
    o32 = dict(precision="mixed_fp32", ksp_restart=30)
    return [
        (W.cook(4, 4, 2, order=1, nu=0.3), "NK", o64, (0.4, 0.0)),
        (W.cook(3, 3, 1, order=2, nu=0.3), "iB", o32, (0.4, 0.0)),
        (W.heart(nr=2, nc=8, nl=6), "iNK", o32, (0.2, 0.01)),
        (W.cook(8, 8, 2, order=1, nu=0.49), "iNK", o32, (0.2, 0.0)),
        (W.cook(6, 6, 2, order=2, nu=0.3), "NK", o32, (0.2, 0.0)),
        (W.twist(2, order=2), "iNK", dict(precision="fp64", ksp_restart=30), (0.3, 0.0)),  # u-p: stream path
    ]


def test_small_requests_are_batched_and_match_alone(fe):
    """Small requests go through shared launches (fe_batch.h); each result is
    bit-identical to the same request solved alone by the batched solver
    (whatever launch shape the autotuner gave its batch), and the u-p
    request, which the batched solver does not take, to its solve alone."""
    reqs = _small_requests() * 3
    alone = []
    for w, meth, opts, (load, tm) in reqs:
        m = fe.Mesh(w)
        m.set_load(load, tm)
        d = m.zeros()
        if fe.batch_supported(m, meth, opts):
            st = fe.batch_solve([m], [meth], [d], [1e-8], opts=opts)[0]
        else:
            _, st = m.solve(meth, d, tol=1e-8, opts=opts)
        assert st["status"] == 0, (meth, st["res_hist"][-3:])
        alone.append(d.cpu().numpy())
        m.close()
    srv = fe.Server(max_active=32, batch_max_dofs=4000)
    ids = [srv.submit(w, meth, tol=1e-8, opts=opts, load=load, time=tm) for w, meth, opts, (load, tm) in reqs]
    res = [srv.poll(i, wait=True) for i in ids]
    tune = srv.tuning()
    srv.close()
    for r, a, (w, meth, _, _) in zip(res, alone, reqs):
        assert r["state"] == "done" and r["result"] == 0, (meth, r)
        if w["pressure_order"] == 0:
            assert np.array_equal(r["d"], a), (w["name"], meth)
        else:
            assert np.abs(r["d"] - a).max() <= 1e-12 * np.abs(a).max()
    assert tune and sum(sum(e["batches"]) for e in tune) >= 2


def test_resident_mesh_is_reused_and_matches_a_fresh_one(fe):
    """A request whose mesh description matches an earlier request's runs on
    that request's resident mesh (pattern, colouring, AMG structure and
    workspace kept); its result is bit-identical to a solve on a freshly
    built mesh, whatever the earlier request's load, method and
    preconditioner were."""
    w = W.cook(6, 6, 2, order=2, nu=0.3)
    amg = dict(precision="mixed_fp32", pc_type="amg", ksp_restart=30)
    bj = dict(precision="fp64", ksp_atol=0.0, ksp_restart=30)
    seq = [("NK", amg, 0.2), ("iB", bj, 0.3), ("NK", amg, 0.2), ("iNK", bj, 0.1)]
    fresh = []
    for meth, opts, load in seq:
        m = fe.Mesh(w)
        m.set_load(load, 0.0)
        d, st = m.solve(meth, m.zeros(), tol=1e-8, opts=opts)
        assert st["status"] == 0, (meth, st["res_hist"][-3:])
        fresh.append(d.cpu().numpy())
        m.close()
    for cache in (True, False):
        srv = fe.Server(max_active=1, batch_max_dofs=-1, mesh_cache=cache)
        res = [srv.poll(srv.submit(w, meth, tol=1e-8, opts=opts, load=load), wait=True) for meth, opts, load in seq]
        srv.close()
        assert [r["mesh_reused"] for r in res] == [False] + [cache] * 3
        for r, a, (meth, _, _) in zip(res, fresh, seq):
            assert r["state"] == "done" and r["result"] == 0, (meth, r)
            assert np.array_equal(r["d"], a), (cache, meth)


def test_resident_meshes_are_evicted_least_recently_used(fe):
    """Resident meshes keep their admission charge; a request that needs the
    room evicts the least recently used idle one."""
    a = W.cook(4, 4, 2, order=1, nu=0.3)
    b = W.cook(5, 5, 2, order=1, nu=0.3)
    srv = fe.Server(max_active=1, batch_max_dofs=-1)
    fa = srv.poll(srv.submit(a, "NK", load=0.1), wait=True)["footprint"]
    fb = srv.poll(srv.submit(b, "NK", load=0.1), wait=True)["footprint"]
    r = srv.poll(srv.submit(a, "NK", load=0.2), wait=True)
    srv.close()
    assert r["state"] == "done" and r["mesh_reused"]  # room for both: a stays resident
    srv = fe.Server(hbm_budget=fa + fb - 1, max_active=1, batch_max_dofs=-1)  # room for one
    res = [srv.poll(srv.submit(x, "NK", load=0.1), wait=True) for x in (a, b, a, a)]
    srv.close()
    assert all(x["state"] == "done" for x in res)
    assert [x["mesh_reused"] for x in res] == [False, False, False, True]
