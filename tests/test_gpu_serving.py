"""The request server (continuous batching over batch plans).

A structure's result must not depend on what it was batched with: the same
structure served alone and inside a burst of other requests gives the same
energies, potentials and forces (FP32 rounding), and both match the O1 oracle
on the routed bucket's grid with that bucket's c_w and P.  Every request of a
burst completes; oversize structures and unplanned exponents are refused."""
import math

import numpy as np
import pytest

from conftest import rel_rms
from gpu_helpers import TOL_FP32
from paper_2606_06617_b300 import workloads as wl

pytestmark = pytest.mark.gpu

R_C = 4.0
BUCKETS = [(16, 8, 512), (24, 8, 2048), (32, 8, 4096)]


def _server(K, use_graphs=True, inflight=2):
    import torch
    from paper_2606_06617_b300 import lr
    return lr.Server(K, (1, 6), R_C, BUCKETS, inflight=inflight, use_graphs=use_graphs, device=torch.device("cuda", 0))


def _random_structs(n_struct, K, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_struct):
        n = int(rng.integers(1, 300))
        box = tuple(float(x) for x in rng.uniform(6.0, 15.5, 3))
        p = int(rng.choice([1, 6]))
        out.append(wl.random_system(n, box, (p,) * K, seed=seed * 1000 + i, neutral=bool(i % 2)))
    return out


def test_server_alone_equals_in_mix_and_matches_oracle():
    from oracle.grid import DiscretePSWF, GridConfig
    K = 2
    srv = _server(K)
    probe = wl.random_system(120, (11.0, 9.5, 12.5), (6, 6), seed=77, neutral=False)
    t = srv.submit(probe.pos, probe.q, probe.box, probe.ps)
    e_a, phi_a, f_a, _ = srv.wait(t)
    others = _random_structs(40, K, seed=5)
    tickets = [srv.submit(s.pos, s.q, s.box, s.ps) for s in others[:20]]
    tp = srv.submit(probe.pos, probe.q, probe.box, probe.ps)
    tickets += [srv.submit(s.pos, s.q, s.box, s.ps) for s in others[20:]]
    e_b, phi_b, f_b, _ = srv.wait(tp)
    res = [srv.wait(x) for x in tickets]
    assert np.allclose(e_a, e_b, rtol=1e-6, atol=1e-12)
    assert rel_rms(phi_b, phi_a) < 1e-6 and rel_rms(f_b, f_a) < 1e-6
    _, info = srv.route(probe.n, probe.box)
    g = tuple(info["grid"])
    o = DiscretePSWF(GridConfig(probe.box, g, info["P"], info["c"], R_C, probe.ps, c_w=info["c_w"])).evaluate(
        probe.pos, probe.q)
    for c in range(K):
        assert abs(e_a[c] - float(o["E_ch"][c])) <= TOL_FP32 * abs(float(o["E_ch"][c]))
    assert rel_rms(phi_a, o["phi"].numpy()) <= TOL_FP32
    assert rel_rms(f_a, o["F"].numpy()) <= TOL_FP32
    # a few of the mix against the oracle too
    for s, (e, phi, f, _) in list(zip(others, res))[:4]:
        _, info = srv.route(s.n, s.box)
        o = DiscretePSWF(GridConfig(s.box, tuple(info["grid"]), info["P"], info["c"], R_C, s.ps,
                                    c_w=info["c_w"])).evaluate(s.pos, s.q)
        assert rel_rms(phi, o["phi"].numpy()) <= TOL_FP32
        if s.n > 1:
            assert rel_rms(f, o["F"].numpy()) <= TOL_FP32
    st = srv.stats()
    assert st["status"] == 0 and st["requests"] == 42
    srv.close()


def test_server_graphs_and_direct_launches_agree():
    K = 8
    structs = _random_structs(12, K, seed=9)
    out = []
    for graphs in (True, False):
        srv = _server(K, use_graphs=graphs, inflight=1)
        tk = [srv.submit(s.pos, s.q, s.box, s.ps) for s in structs]
        out.append([srv.wait(t) for t in tk])
        srv.close()
    for (e1, p1, f1, _), (e2, p2, f2, _) in zip(*out):
        assert np.allclose(e1, e2, rtol=1e-6, atol=1e-12)
        assert rel_rms(p1, p2) < 1e-6


def test_server_burst_of_serving_stream():
    """200 requests of the serving stream (K = 8, 32-2048 atoms) in a burst:
    all complete, counters add up."""
    from paper_2606_06617_b300 import lr
    import torch
    reqs = wl.serving_stream(200, seed=3)
    h_max = 0.5 * math.pi * R_C / math.log(3.0 / 1e-5)
    srv = lr.Server(8, (1, 6), R_C, lr.serving_buckets(8, h_max), device=torch.device("cuda", 0))
    tk = [srv.submit(r.system.pos, r.system.q, r.system.box, r.system.ps) for r in reqs]
    lat = []
    for t, r in zip(tk, reqs):
        e, phi, f, ms = srv.wait(t)
        assert np.all(np.isfinite(e)) and np.all(np.isfinite(f))
        lat.append(ms)
    st = srv.stats()
    assert st["requests"] == 200 and st["atoms"] == sum(r.system.n for r in reqs) and st["status"] == 0
    assert st["batches"] < 200          # requests were batched
    srv.close()


def test_server_submit_many_equals_single_submits():
    """pswf_server_submit_many / pswf_server_wait_many: 64 structures of the
    serving stream handed over in one call give the energies, potentials
    and forces of per-structure submits (the same routes, batch-mates do not
    change a result within FP32 flush order); latencies are returned."""
    from paper_2606_06617_b300 import lr
    import torch
    reqs = wl.serving_stream(64, seed=5)
    h_max = 0.5 * math.pi * R_C / math.log(3.0 / 1e-5)
    srv = lr.Server(8, (1, 6), R_C, lr.serving_buckets(8, h_max), device=torch.device("cuda", 0))
    single = []
    for r in reqs:
        t = srv.submit(r.system.pos, r.system.q, r.system.box, r.system.ps)
        single.append(srv.wait(t))
    for borrow in (False, True):   # inputs copied at submission, or read when staged
        tk, off = srv.submit_many([(r.system.pos, r.system.q, r.system.box, r.system.ps) for r in reqs],
                                  borrow=borrow)
        e, ph, f, lat = srv.wait_many(tk, off, phi=True)
        assert lat.shape == (64,) and np.all(lat > 0)
        for i, (e1, ph1, f1, _) in enumerate(single):
            a, b = off[i], off[i + 1]
            np.testing.assert_allclose(e[i], e1, rtol=1e-6, atol=1e-9 * np.abs(e1).max())
            assert rel_rms(ph[8 * a:8 * b].reshape(8, b - a), ph1) < 1e-6
            assert rel_rms(f[a:b], f1) < 1e-6
    # a bad structure (exponent outside the server's set) stops the call; earlier ones stay submitted
    bad = [(reqs[0].system.pos, reqs[0].system.q, reqs[0].system.box, reqs[0].system.ps),
           (reqs[1].system.pos, reqs[1].system.q, reqs[1].system.box, [3] * 8)]
    with pytest.raises(lr.PswfError):
        srv.submit_many(bad)
    srv.close()


def test_server_refuses_what_it_cannot_hold():
    from paper_2606_06617_b300 import lr
    srv = _server(1)
    s = wl.random_system(10, (40.0, 10.0, 10.0), (1,), seed=1)
    with pytest.raises(lr.PswfError):
        srv.submit(s.pos, s.q, s.box, s.ps)
    s = wl.random_system(10, (10.0, 10.0, 10.0), (4,), seed=1)
    with pytest.raises(lr.PswfError):
        srv.submit(s.pos, s.q, s.box, s.ps)
    srv.close()


def test_wait_with_deadline_while_paused():
    """A paused server holds its requests on the host: a wait with a limit
    returns PSWF_ETIMEOUT and the ticket stays valid; after resuming, the same
    ticket completes with the result the request has unpaused."""
    from paper_2606_06617_b300 import lr
    srv = _server(2)
    try:
        s = _random_structs(1, 2, seed=77)[0]
        t_ref = srv.submit(s.pos, s.q, s.box, s.ps)
        e_ref, phi_ref, f_ref, _ = srv.wait(t_ref, timeout_ms=30000)
        srv.pause(True)
        t = srv.submit(s.pos, s.q, s.box, s.ps)
        with pytest.raises(lr.PswfError) as ei:
            srv.wait(t, timeout_ms=50)
        assert ei.value.status == lr.PSWF_ETIMEOUT
        with pytest.raises(lr.PswfError):
            srv.wait(t, timeout_ms=0)
        srv.pause(False)
        e, phi, f, _ = srv.wait(t, timeout_ms=30000)
        np.testing.assert_allclose(e, e_ref, rtol=1e-6)
        assert rel_rms(f, f_ref) < 1e-6 and rel_rms(phi, phi_ref) < 1e-6
    finally:
        srv.close()


def test_plan_sync_with_deadline():
    """pswf_sync_for: a zero limit while a melt-size evaluation runs gives
    PSWF_ETIMEOUT (the work goes on), a generous one returns normally."""
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.ionic_melt(1242757, 233.3, seed=1)
    plan = lr.Plan(s.box, s.n, s.ps, 7.0, P=7, grid=256, device=dev)
    plan.set_points(torch.tensor(s.pos, device=dev), torch.tensor(s.q, dtype=torch.float32, device=dev))
    plan.sync()
    for _ in range(3):
        plan.execute()
    with pytest.raises(lr.PswfError) as ei:
        plan.sync(timeout_ms=0.0)
    assert ei.value.status == lr.PSWF_ETIMEOUT
    plan.sync(timeout_ms=60000.0)
