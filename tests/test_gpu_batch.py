"""Batch plans: several structures with their own boxes, atoms and exponents
in one call (pswf_batch_plan_create / pswf_batch_set_points).

Each structure must match the O1 oracle of that structure alone on the
plan's grid size with the plan's c_w and P (FP32: 2e-6 relative RMS), and a
single-structure plan with the same parameters to FP32 rounding; empty slots
give zero energy; boxes beyond box_max and unplanned exponents are rejected."""
import math

import numpy as np
import pytest

from conftest import rel_rms
from gpu_helpers import TOL_FP32, TOL_FP64
from paper_2606_06617_b300 import workloads as wl

pytestmark = pytest.mark.gpu

R_C = 4.0
C = math.log(3.0 / 1e-5)


def _structures(seed=0, nstruct=5, K=3):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nstruct):
        n = int(rng.integers(1, 400)) if i else 1
        box = tuple(float(x) for x in rng.uniform(7.0, 14.0, 3))
        p = int(rng.choice([1, 6]))
        s = wl.random_system(n, box, (p,) * K, seed=seed * 100 + i, neutral=bool(i % 2))
        out.append(s)
    return out


def _run_batch(structs, b_max, M, precision=0, P=0):
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    K = structs[0].q.shape[0]
    n_tot = sum(s.n for s in structs)
    plan = lr.BatchPlan((14.0, 14.0, 14.0), b_max, max(n_tot, 1), K, (1, 6), R_C, c=C, grid=M, P=P,
                        precision=precision, device=dev)
    offsets = np.concatenate([[0], np.cumsum([s.n for s in structs])]).astype(np.int64)
    boxes = np.array([s.box for s in structs])
    ps = np.array([s.ps for s in structs], dtype=np.int32)
    pos = torch.tensor(np.concatenate([s.pos for s in structs]), device=dev)
    q = torch.tensor(np.concatenate([s.q for s in structs], axis=1), dtype=plan.dtype, device=dev)
    plan.set_points(boxes, ps, offsets, pos, q)
    e, phi, f = plan.execute()
    plan.sync()
    return plan, offsets, e.cpu().numpy(), phi.cpu().double().numpy(), f.cpu().double().numpy()


def _oracle(s, M, plan):
    from oracle.grid import DiscretePSWF, GridConfig
    info = plan.info
    o = DiscretePSWF(GridConfig(tuple(s.box), tuple(M), info["P"], info["c"], R_C, tuple(s.ps), c_w=info["c_w"]))
    return o.evaluate(s.pos, s.q)


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP32), (1, TOL_FP64)])
def test_batch_matches_oracle_per_structure(precision, tol):
    structs = _structures(seed=1)
    M = (28, 28, 28)
    plan, off, e, phi, f = _run_batch(structs, 8, M, precision=precision)
    for i, s in enumerate(structs):
        o = _oracle(s, M, plan)
        sl = slice(off[i], off[i + 1])
        for c in range(s.q.shape[0]):
            ref = float(o["E_ch"][c])
            assert abs(e[i, c] - ref) <= tol * abs(ref) + 1e-12, (i, c, e[i, c], ref)
        if s.n > 1:
            assert rel_rms(phi[:, sl], o["phi"].numpy()) <= tol, (i, rel_rms(phi[:, sl], o["phi"].numpy()))
            assert rel_rms(f[sl], o["F"].numpy()) <= tol, (i, rel_rms(f[sl], o["F"].numpy()))
    # empty slots
    assert np.all(e[len(structs):] == 0.0)


def test_batch_equals_single_plans():
    """Each structure of a batch gives what a single-structure plan on the same
    grid, c_w and P gives (FP32 rounding only)."""
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    structs = _structures(seed=2, nstruct=4, K=2)
    M = (24, 24, 24)
    plan, off, e, phi, f = _run_batch(structs, 4, M)
    info = plan.info
    for i, s in enumerate(structs):
        sp = lr.Plan(s.box, s.n, s.ps, R_C, c=info["c"], c_w=info["c_w"], P=info["P"], grid=M, device=dev)
        sp.set_points(torch.tensor(s.pos, device=dev), torch.tensor(s.q, dtype=torch.float32, device=dev))
        e1, phi1, f1 = sp.execute()
        sp.sync()
        sl = slice(off[i], off[i + 1])
        assert np.allclose(e[i], e1.cpu().numpy(), rtol=1e-6, atol=1e-9)
        assert rel_rms(phi[:, sl], phi1.cpu().double().numpy()) < 1e-6
        if s.n > 1:
            assert rel_rms(f[sl], f1.cpu().double().numpy()) < 1e-6


def test_batch_recomposition_and_self_energy():
    """A plan reused with a different set of structures (fewer, other boxes)
    gives the new structures' results; self energies per slot."""
    structs = _structures(seed=3, nstruct=6)
    M = (28, 28, 28)
    plan, off, e, phi, f = _run_batch(structs, 6, M)
    import torch
    dev = torch.device("cuda", 0)
    sub = structs[3:5]
    off2 = np.array([0, sub[0].n, sub[0].n + sub[1].n], dtype=np.int64)
    plan.set_points(np.array([s.box for s in sub]), np.array([s.ps for s in sub], dtype=np.int32), off2,
                    torch.tensor(np.concatenate([s.pos for s in sub]), device=dev),
                    torch.tensor(np.concatenate([s.q for s in sub], axis=1), dtype=torch.float32, device=dev))
    e2, phi2, f2 = plan.execute()
    plan.sync()
    e2 = e2.cpu().numpy()
    assert np.allclose(e2[0], e[3], rtol=1e-6, atol=1e-9)
    assert np.allclose(e2[1], e[4], rtol=1e-6, atol=1e-9)
    assert np.all(e2[2:] == 0.0)
    se = plan.self_energy()
    for i, s in enumerate(sub):
        o = _oracle(s, M, plan)
        from oracle.grid import DiscretePSWF, GridConfig
        info = plan.info
        oo = DiscretePSWF(GridConfig(tuple(s.box), M, info["P"], info["c"], R_C, tuple(s.ps), c_w=info["c_w"]))
        ref = oo.self_energy(s.q.astype(np.float32).astype(np.float64))
        assert np.allclose(se[i], ref, rtol=1e-7)
    assert np.all(se[2:] == 0.0)


def test_batch_rejects_bad_inputs():
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    plan = lr.BatchPlan((10.0, 10.0, 10.0), 2, 100, 1, (1,), R_C, grid=(20, 20, 20), device=dev)
    pos = torch.zeros(5, 3, dtype=torch.float64, device=dev)
    q = torch.zeros(1, 5, device=dev)
    with pytest.raises(lr.PswfError) as e:
        plan.set_points(np.array([[11.0, 9.0, 9.0]]), np.array([[1]]), np.array([0, 5]), pos, q)
    assert e.value.status == -1
    with pytest.raises(lr.PswfError) as e:
        plan.set_points(np.array([[9.0, 9.0, 9.0]]), np.array([[6]]), np.array([0, 5]), pos, q)
    assert e.value.status == -1
    with pytest.raises(lr.PswfError):
        plan.set_points(np.array([[9.0, 9.0, 9.0]] * 3), np.array([[1]] * 3), np.array([0, 1, 2, 5]), pos, q)
