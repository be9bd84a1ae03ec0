"""Backward of the real-space complement (pswf_real_space_backward) against
the oracle's VJP (double autograd of the pair energy, pinned by finite
differences): gradients in the charges per channel and in the positions,
for upstream gradients on the energies, potentials and forces.  Cell-list
mode in a box and in a sheared cell, direct (image-sum) mode in a small box;
FP64 and FP32."""
import math

import numpy as np
import pytest

from conftest import rel_rms
from paper_2606_06617_b300 import workloads as wl

pytestmark = pytest.mark.gpu

C = math.log(3.0 / 1e-5)
TOL = {1: 1e-12, 0: 1e-6}   # largest measured: FP64 6.6e-13, FP32 4.5e-7

CASES = [  # (name, box or cell, atoms, exponents, r_c)
    ("box_cells", (22.0, 23.0, 21.0), 900, (1, 6), 4.0),
    ("sheared_cells", ((22.0, 0.0, 0.0), (3.0, 21.0, 0.0), (-2.0, 1.5, 20.0)), 800, (1, 4, 6), 4.0),
    ("small_direct", (9.0, 8.5, 9.5), 60, (1, 2, 6), 4.0),
]


def _oracle(pos, q, cell, ps, r_c, gE, gphi, gF):
    from oracle.realspace import real_space_vjp
    gq = np.zeros_like(q)
    gp = np.zeros_like(pos)
    for c, p in enumerate(ps):
        a, b = real_space_vjp(pos, q[c], cell, p, C, r_c, gE[c], gphi[c], gF)
        gq[c] = a
        gp += b
    return gq, gp


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("name,cell,nat,ps,r_c", CASES, ids=[c[0] for c in CASES])
def test_real_space_backward_matches_oracle(name, cell, nat, ps, r_c, precision):
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    general = np.asarray(cell).ndim == 2
    H = np.asarray(cell, dtype=np.float64) if general else np.diag(cell)
    box = tuple(np.diag(H)) if not general else tuple(np.linalg.norm(H, axis=1))
    s = wl.random_system(nat, (1.0, 1.0, 1.0), ps, seed=90 + nat, neutral=False)
    s.pos = s.pos @ H                                # uniform in the cell
    s.pos[::7] += H[0]                               # some atoms outside the primary cell
    kw = dict(cell=H) if general else {}
    plan = lr.Plan(box if not general else None, s.n, ps, r_c, c=C, P=6, grid=(32, 32, 32), precision=precision,
                   flags=lr.PSWF_FLAG_REAL_SPACE, device=dev, **kw)
    rng = np.random.default_rng(5)
    gE, gphi, gF = rng.normal(size=len(ps)), rng.normal(size=(len(ps), s.n)), rng.normal(size=(s.n, 3))
    pos = torch.tensor(s.pos, device=dev)
    q = torch.tensor(s.q, dtype=plan.dtype, device=dev)
    plan.real_space(pos, q)
    t = lambda a: torch.tensor(a, dtype=plan.dtype, device=dev)
    gq, gr = plan.real_space_backward(pos, q, torch.tensor(gE, device=dev), t(gphi), t(gF))
    plan.sync()
    oq, orr = _oracle(s.pos, s.q, H, ps, r_c, gE, gphi, gF)
    eq, er = rel_rms(gq.cpu().double().numpy(), oq), rel_rms(gr.cpu().double().numpy(), orr)
    print(f"{name} precision={precision}: grad_q {eq:.3e} grad_pos {er:.3e}")
    assert eq <= TOL[precision] and er <= TOL[precision], (eq, er)
    # each upstream alone, and the state rules
    for parts in (("E",), ("phi",), ("F",)):
        ge = torch.tensor(gE, device=dev) if "E" in parts else None
        gp_ = t(gphi) if "phi" in parts else None
        gf = t(gF) if "F" in parts else None
        a, b = plan.real_space_backward(pos, q, ge, gp_, gf)
        plan.sync()
        oa, ob = _oracle(s.pos, s.q, H, ps, r_c, gE if "E" in parts else np.zeros(len(ps)),
                         gphi if "phi" in parts else np.zeros_like(gphi), gF if "F" in parts else np.zeros_like(gF))
        assert rel_rms(a.cpu().double().numpy(), oa) <= TOL[precision], parts
        assert rel_rms(b.cpu().double().numpy(), ob) <= TOL[precision], parts


def test_real_space_backward_needs_forward():
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    plan = lr.Plan((20.0, 20.0, 20.0), 100, (1,), 4.0, P=6, grid=32, flags=lr.PSWF_FLAG_REAL_SPACE, device=dev)
    pos = torch.rand(100, 3, device=dev, dtype=torch.float64) * 20
    q = torch.randn(1, 100, device=dev)
    with pytest.raises(lr.PswfError) as e:
        plan.real_space_backward(pos, q, torch.ones(1, dtype=torch.float64, device=dev))
    assert e.value.status == -8


def test_complete_sum_trains_through_real_space():
    """lr.complete_sum: the complete lattice sum (reciprocal + real space -
    self) with autograd.  A force-matching loss sum_c E_c + |F - F_ref|^2 is
    differentiated to the positions and charges and compared with the
    oracle: O1's VJP of the reciprocal part, the real-space VJP and the self
    term (FP64)."""
    import torch
    from oracle.grid import DiscretePSWF, GridConfig
    from oracle.realspace import pswf_total, real_space_vjp
    from oracle.mollifiers import Mollifier
    from gpu_helpers import window_cw
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.random_system(150, (13.0, 14.0, 12.5), (1, 6), seed=4, neutral=False)
    M, P, r_c = (26, 28, 25), 6, 4.0
    cw = window_cw(s.box, M, P, C, r_c)
    plan = lr.Plan(s.box, s.n, s.ps, r_c, c=C, c_w=cw, P=P, grid=M, precision=1,
                   flags=lr.PSWF_FLAG_BACKWARD | lr.PSWF_FLAG_REAL_SPACE, device=dev)
    F_ref = np.random.default_rng(2).normal(size=(s.n, 3))
    pos = torch.tensor(s.pos, device=dev, requires_grad=True)
    q = torch.tensor(s.q, device=dev, requires_grad=True)
    E, phi, F = lr.complete_sum(plan, pos, q)
    loss = ((F - torch.tensor(F_ref, device=dev)) ** 2).sum() + E.sum()
    loss.backward()
    o1 = DiscretePSWF(GridConfig(tuple(s.box), M, P, C, r_c, tuple(s.ps), c_w=cw))
    r1 = o1.evaluate(s.pos, s.q)
    tot = pswf_total(dict(E_ch=r1["E_ch"].numpy(), phi=r1["phi"].numpy(), f=r1["f"].numpy()),
                     s.pos, s.q, s.box, s.ps, C, r_c)
    np.testing.assert_allclose(E.detach().cpu().numpy(), tot["E_ch"], rtol=1e-9, atol=1e-12)
    assert rel_rms(phi.detach().cpu().numpy(), tot["phi"]) < 1e-9
    assert rel_rms(F.detach().cpu().numpy(), tot["F"]) < 1e-9
    gF = 2.0 * (tot["F"] - F_ref)
    gE = np.ones(len(s.ps))
    oq, orr = o1.vjp(s.pos, s.q, gE, None, gF)
    oq, orr = oq.numpy().copy(), orr.numpy().copy()
    moll = Mollifier(C, r_c)
    for c, p in enumerate(s.ps):
        a, b = real_space_vjp(s.pos, s.q[c], s.box, p, C, r_c, gE[c], None, gF, moll)
        oq[c] += a - 2.0 * moll.self_coef(p) * gE[c] * s.q[c]
        orr += b
    assert rel_rms(q.grad.cpu().numpy(), oq) < 1e-8, rel_rms(q.grad.cpu().numpy(), oq)
    assert rel_rms(pos.grad.cpu().numpy(), orr) < 1e-8, rel_rms(pos.grad.cpu().numpy(), orr)
