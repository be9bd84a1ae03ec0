"""Parity of the hand-written backward (pswf_backward, through the C-ABI) with
the oracle's vector-jacobian product of the same discrete forward.

The loss is L = sum_c gE_c E_c + sum gphi * phi + sum gF * F with seeded
upstream gradients; both sides use the same explicit parameters.  The FP64
path must agree to 1e-8 relative RMS; the FP32 path to 4e-6, twice the
largest error measured on a B300 over these cases and the training batch
(grad_pos 1.3e-6 at P = 4, 1.9e-6 in the training shape; grad_q <= 5.1e-7):
the force term involves the second derivative of the window, whose FP32
table error is amplified by (2/h)^2."""
import math

import numpy as np
import pytest

from conftest import rel_rms
from gpu_helpers import window_cw
from paper_2606_06617_b300 import workloads as wl

pytestmark = pytest.mark.gpu

C_TOL = math.log(3.0 / 1e-5)
TOL_BW_FP64 = 1e-8
# FP32: the largest measured errors are grad_pos 2.2e-6 and grad_q 1.5e-6 in
# the training shape (tests/test_gpu_training.py), 1.4e-6 and 1.2e-6 for six
# channels at P = 4; the backward spread accumulates in 32-bit fixed point
# per (tile, channel), whose unit follows the tile's largest contribution
TOL_BW_FP32 = 4e-6


def _oracle(s, r_c, P, M, c, cw):
    from oracle.grid import DiscretePSWF, GridConfig
    return DiscretePSWF(GridConfig(tuple(s.box), tuple(M), P, c, r_c, tuple(s.ps), c_w=cw))


def _upstream(s, seed=5, parts=("E", "phi", "F")):
    rng = np.random.default_rng(seed)
    K, n = s.q.shape
    gE = rng.normal(size=K) if "E" in parts else None
    gphi = rng.normal(size=(K, n)) if "phi" in parts else None
    gF = rng.normal(size=(n, 3)) if "F" in parts else None
    return gE, gphi, gF


def _gpu_backward(s, r_c, P, M, c, cw, precision, up):
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    plan = lr.Plan(s.box, max(s.n, 1), s.ps, r_c, c=c, c_w=cw, P=P, grid=M, precision=precision,
                   flags=lr.PSWF_FLAG_BACKWARD, device=dev)
    pos = torch.tensor(s.pos, dtype=torch.float64, device=dev)
    q = torch.tensor(s.q, dtype=plan.dtype, device=dev)
    plan.set_points(pos, q)
    e, phi, f = plan.execute()
    t = lambda a, dt: None if a is None else torch.tensor(a, dtype=dt, device=dev)
    gE, gphi, gF = up
    gq, gr = plan.backward(t(gE, torch.float64), t(gphi, plan.dtype), t(gF, plan.dtype))
    plan.sync()
    torch.cuda.synchronize()
    return (gq.cpu().double().numpy(), gr.cpu().double().numpy(), phi.cpu().double().numpy(),
            f.cpu().double().numpy())


def _check(s, r_c, P, M, c, precision, tol, parts=("E", "phi", "F"), what="", tol_pos=None):
    cw = window_cw(s.box, M, P, c, r_c)
    up = _upstream(s, parts=parts)
    gq, gr, _, _ = _gpu_backward(s, r_c, P, M, c, cw, precision, up)
    oq, orr = _oracle(s, r_c, P, M, c, cw).vjp(s.pos, s.q, *up)
    print(f"backward {what} precision={precision}: grad_q {rel_rms(gq, oq.numpy()):.3e} "
          f"grad_pos {rel_rms(gr, orr.numpy()):.3e}")
    assert rel_rms(gq, oq.numpy()) <= tol, (what, "grad_q", rel_rms(gq, oq.numpy()))
    tol_pos = tol if tol_pos is None else tol_pos
    assert rel_rms(gr, orr.numpy()) <= tol_pos, (what, "grad_pos", rel_rms(gr, orr.numpy()))


@pytest.mark.parametrize("precision,tol", [(0, TOL_BW_FP32), (1, TOL_BW_FP64)])
def test_backward_water(precision, tol):
    """Water box (1000 molecules, L = 31, p = 1 and 6), grid 64^3, P = 8."""
    s = wl.water_box()
    _check(s, 4.0, 8, (64, 64, 64), C_TOL, precision, tol, what="water")


@pytest.mark.parametrize("parts", [("E",), ("phi",), ("F",)])
def test_backward_each_upstream_fp64(parts):
    """Each upstream term alone (the others NULL), ragged box, two channels."""
    s = wl.random_system(200, (11.0, 13.0, 9.5), (1, 4), seed=21, neutral=False)
    _check(s, 3.5, 6, (22, 27, 19), 10.0, 1, TOL_BW_FP64, parts=parts, what=str(parts))


@pytest.mark.parametrize("P", [4, 7])
def test_backward_six_channels_fp32(P):
    """p = 1..6 in one plan, atoms far outside the primary cell."""
    rng = np.random.default_rng(9)
    box = (13.0, 17.5, 11.0)
    s = wl.random_system(150, box, (1, 2, 3, 4, 5, 6), seed=12, neutral=True)
    s.pos = s.pos + rng.integers(-2, 3, size=s.pos.shape) * np.asarray(box)
    _check(s, 4.5, P, (27, 35, 21), 11.0, 0, TOL_BW_FP32, what=f"six channels P={P}")


def test_backward_energy_only_is_phi_and_minus_force():
    """With only gE = 1 the VJP is (phi, -F) of the forward (FP32, same plan)."""
    s = wl.random_system(300, (12.0, 12.0, 12.0), (1,), seed=2)
    M = (24, 24, 24)
    cw = window_cw(s.box, M, 6, C_TOL, 4.0)
    gq, gr, phi, f = _gpu_backward(s, 4.0, 6, M, C_TOL, cw, 0, (np.ones(1), None, None))
    assert rel_rms(gq, phi) < 1e-6
    assert rel_rms(gr, -f) < 1e-6


def test_backward_single_atom_and_empty():
    import torch
    from paper_2606_06617_b300 import lr
    s = wl.random_system(1, (9.0, 9.0, 9.0), (1, 6), seed=4, neutral=False)
    # a lone atom only feels its own images: its position gradient is a small
    # sum of large cancelling terms, so it is compared at 1e-7
    _check(s, 3.0, 6, (18, 18, 18), 9.0, 1, TOL_BW_FP64, what="one atom", tol_pos=1e-7)
    dev = torch.device("cuda", 0)
    plan = lr.Plan(s.box, 4, s.ps, 3.0, P=6, grid=(18, 18, 18), flags=lr.PSWF_FLAG_BACKWARD, device=dev)
    plan.set_points(torch.zeros(0, 3, dtype=torch.float64, device=dev), torch.zeros(2, 0, device=dev))
    plan.execute()
    gq, gr = plan.backward(torch.ones(2, dtype=torch.float64, device=dev))
    plan.sync()
    assert gq.shape == (2, 0) and gr.shape == (0, 3)


def test_backward_state_errors():
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.random_system(10, (9.0, 9.0, 9.0), (1,), seed=4)
    pos = torch.tensor(s.pos, device=dev)
    q = torch.tensor(s.q, dtype=torch.float32, device=dev)
    plain = lr.Plan(s.box, 10, s.ps, 3.0, P=6, grid=(18, 18, 18), device=dev)
    plain.set_points(pos, q)
    plain.execute()
    with pytest.raises(lr.PswfError) as e:
        plain.backward(torch.ones(1, dtype=torch.float64, device=dev))
    assert e.value.status == -8
    bw = lr.Plan(s.box, 10, s.ps, 3.0, P=6, grid=(18, 18, 18), flags=lr.PSWF_FLAG_BACKWARD, device=dev)
    bw.set_points(pos, q)
    with pytest.raises(lr.PswfError) as e:
        bw.backward(torch.ones(1, dtype=torch.float64, device=dev))
    assert e.value.status == -8


def test_autograd_force_matching():
    """torch.autograd through long_range: a force-matching loss
    sum |F - F_ref|^2 + sum_c E_c, gradients to positions and charges
    against the oracle VJP with gF = 2 (F - F_ref), gE = 1 (FP64 path)."""
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.random_system(120, (10.0, 11.0, 12.0), (1, 6), seed=8, neutral=False)
    M = (20, 22, 24)
    r_c, P = 3.5, 6
    cw = window_cw(s.box, M, P, C_TOL, r_c)
    plan = lr.Plan(s.box, s.n, s.ps, r_c, c=C_TOL, c_w=cw, P=P, grid=M, precision=1,
                   flags=lr.PSWF_FLAG_BACKWARD, device=dev)
    F_ref = np.random.default_rng(1).normal(size=(s.n, 3)) * 0.1
    pos = torch.tensor(s.pos, device=dev, requires_grad=True)
    q = torch.tensor(s.q, device=dev, requires_grad=True)
    E, phi, F = lr.long_range(plan, pos, q)
    loss = ((F - torch.tensor(F_ref, device=dev)) ** 2).sum() + E.sum()
    loss.backward()
    o = _oracle(s, r_c, P, M, C_TOL, cw)
    F_o = o.evaluate(s.pos, s.q)["F"].numpy()
    oq, orr = o.vjp(s.pos, s.q, np.ones(2), None, 2.0 * (F_o - F_ref))
    assert rel_rms(q.grad.cpu().numpy(), oq.numpy()) < TOL_BW_FP64
    assert rel_rms(pos.grad.cpu().numpy(), orr.numpy()) < TOL_BW_FP64
