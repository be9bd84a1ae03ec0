"""The ionic melt at full size (4,194,304 atoms, L = 350, 384^3, K = 4,
P = 7), in the launch configuration the benchmark times.  The oracle cannot
evaluate this size, so the checks are properties that hold at any size:

* the quadratic-form identity E_c = 1/2 sum_i q_i^c phi_i^c of the discrete
  operator (exact up to rounding, zero-frequency terms included);
* a translation of every atom by one grid spacing maps the problem onto
  itself (the grid values move by one point), so potentials and forces are
  unchanged up to FP32 rounding: each run is within the FP32 budget (2e-6
  relative RMS) of the exact discrete result, so the two differ by at most
  twice that;
* the net force vanishes up to the method's error: the discrete operator
  conserves momentum only to the spreading error, so the mean force per atom
  |sum F| / N must stay below the 1e-5 relative force tolerance times the
  RMS force (the oracle shows a coherent net force that grows like N, about
  1e-7 F_rms per atom at this density);
* the FP32 path is within the FP32 budget (2e-6 relative RMS on potentials
  and forces, relative on each channel energy) of the FP64 path on the same
  inputs and parameters; the FP64 path's own parity with the oracle (2e-9)
  is tested at the sizes the oracle can evaluate, so this bounds the full-size
  FP32 error by the budget plus a negligible term.
"""
import math

import numpy as np
import pytest

from conftest import rel_rms
from paper_2606_06617_b300 import workloads as wl

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_ionic_melt_full_size_properties():
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.ionic_melt(4194304, 350.0, seed=0)
    plan = lr.Plan(s.box, s.n, s.ps, 7.0, tol=1e-5, P=7, grid=384, device=dev)
    pos = torch.tensor(s.pos, device=dev)
    q = torch.tensor(s.q, dtype=torch.float32, device=dev)
    plan.set_points(pos, q)
    e, phi, f = plan.execute()
    plan.sync()
    e = e.cpu().numpy()
    qd = q.double()
    for c in range(4):
        half = 0.5 * float((qd[c] * phi[c].double()).sum())
        assert abs(half - e[c]) <= 1e-5 * abs(e[c]), (c, half, e[c])
    h = 350.0 / 384
    plan.set_points(pos + torch.tensor([h, 0.0, 0.0], device=dev, dtype=torch.float64), q)
    e2, phi2, f2 = plan.execute()
    plan.sync()
    assert rel_rms(phi2.cpu().numpy(), phi.cpu().numpy()) < 4e-6
    assert rel_rms(f2.cpu().numpy(), f.cpu().numpy()) < 4e-6
    assert np.allclose(e2.cpu().numpy(), e, rtol=1e-6)
    F = f.double()
    net = F.sum(0).norm().item()
    rms = F.pow(2).sum(1).mean().sqrt().item()
    assert net / s.n <= 1e-5 * rms, (net, rms)


def test_ionic_melt_full_size_fp32_within_budget_of_fp64():
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.ionic_melt(4194304, 350.0, seed=0)
    pos = torch.tensor(s.pos, device=dev)
    out = {}
    for prec in (0, 1):
        plan = lr.Plan(s.box, s.n, s.ps, 7.0, tol=1e-5, P=7, grid=384, precision=prec, device=dev)
        plan.set_points(pos, torch.tensor(s.q, dtype=plan.dtype, device=dev))
        e, phi, f = plan.execute()
        plan.sync()
        out[prec] = (e.cpu().numpy(), phi.cpu().double().numpy(), f.cpu().double().numpy())
        del plan, e, phi, f
        torch.cuda.empty_cache()
    (e32, p32, f32), (e64, p64, f64) = out[0], out[1]
    for c in range(4):
        assert abs(e32[c] - e64[c]) <= 2e-6 * abs(e64[c]), (c, e32[c], e64[c])
        assert rel_rms(p32[c], p64[c]) <= 2e-6, (c, rel_rms(p32[c], p64[c]))
    assert rel_rms(f32, f64) <= 2e-6, rel_rms(f32, f64)


def test_sheared_melt_full_size_fp32_within_budget_of_fp64():
    """The 4,194,304-atom melt in a sheared cell of the same volume
    (pswf_plan_create_cell, 384^3): FP32 within the FP32 budget of FP64."""
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.ionic_melt(4194304, 350.0, seed=0)
    H = np.array([[350.0, 0.0, 0.0], [60.0, 350.0, 0.0], [-40.0, 50.0, 350.0]])
    pos = torch.tensor((s.pos / 350.0) @ H, device=dev)
    out = {}
    for prec in (0, 1):
        plan = lr.Plan(None, s.n, s.ps, 7.0, tol=1e-5, P=7, grid=384, precision=prec, device=dev, cell=H)
        plan.set_points(pos, torch.tensor(s.q, dtype=plan.dtype, device=dev))
        e, phi, f = plan.execute()
        plan.sync()
        out[prec] = (e.cpu().numpy(), phi.cpu().double().numpy(), f.cpu().double().numpy(), plan.info["transform"])
        del plan, e, phi, f
        torch.cuda.empty_cache()
    (e32, p32, f32, t32), (e64, p64, f64, _) = out[0], out[1]
    assert t32 == lr.PSWF_TRANSFORM_OWN
    for c in range(4):
        assert abs(e32[c] - e64[c]) <= 2e-6 * abs(e64[c]), (c, e32[c], e64[c])
        assert rel_rms(p32[c], p64[c]) <= 2e-6, (c, rel_rms(p32[c], p64[c]))
    assert rel_rms(f32, f64) <= 2e-6, rel_rms(f32, f64)
