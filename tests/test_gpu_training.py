"""The training-step shape: a batch of structures (own cubic boxes, 16
channels with exponents alternating 1, 6) through one batch plan, forward
and hand-written backward.  Per structure, the gradients of a loss touching
energies, potentials and forces must match the oracle's VJP of that
structure alone on the plan's grid with the plan's c_w and P (FP32: 4e-6,
twice the largest measured error, 1.9e-6 on grad_pos)."""
import math

import numpy as np
import pytest

from conftest import rel_rms
from paper_2606_06617_b300 import workloads as wl

pytestmark = pytest.mark.gpu

R_C = 4.0


def test_training_batch_backward_matches_oracle():
    import torch
    from oracle.grid import DiscretePSWF, GridConfig
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    K = 16
    structs = wl.training_batch(n_struct=6, K=K, n_lo=60, n_hi=160, seed=4)
    Lmax = max(s.box[0] for s in structs)
    M = 40
    n_tot = sum(s.n for s in structs)
    plan = lr.BatchPlan((Lmax, Lmax, Lmax), 8, n_tot, K, (1, 6), R_C, grid=M, flags=lr.PSWF_FLAG_BACKWARD,
                        device=dev)
    off = np.concatenate([[0], np.cumsum([s.n for s in structs])]).astype(np.int64)
    pos = torch.tensor(np.concatenate([s.pos for s in structs]), device=dev)
    q = torch.tensor(np.concatenate([s.q for s in structs], axis=1), dtype=torch.float32, device=dev)
    plan.set_points(np.array([s.box for s in structs]), np.array([s.ps for s in structs], dtype=np.int32), off,
                    pos, q)
    e, phi, f = plan.execute()
    rng = np.random.default_rng(2)
    gE = rng.normal(size=(8, K))
    gphi = rng.normal(size=(K, n_tot))
    gF = rng.normal(size=(n_tot, 3))
    gq, gr = plan.backward(torch.tensor(gE.ravel(), dtype=torch.float64, device=dev),
                           torch.tensor(gphi, dtype=torch.float32, device=dev),
                           torch.tensor(gF, dtype=torch.float32, device=dev))
    plan.sync()
    gq = gq.cpu().double().numpy()[:, :n_tot]
    gr = gr.cpu().double().numpy()[:n_tot]
    info = plan.info
    for i, s in enumerate(structs[:3]):
        sl = slice(off[i], off[i + 1])
        o = DiscretePSWF(GridConfig(s.box, (M, M, M), info["P"], info["c"], R_C, s.ps, c_w=info["c_w"]))
        oq, orr = o.vjp(s.pos, s.q, gE[i], gphi[:, sl], gF[sl])
        print(f"training structure {i}: grad_q {rel_rms(gq[:, sl], oq.numpy()):.3e} "
              f"grad_pos {rel_rms(gr[sl], orr.numpy()):.3e}")
        assert rel_rms(gq[:, sl], oq.numpy()) < 4e-6, (i, rel_rms(gq[:, sl], oq.numpy()))
        assert rel_rms(gr[sl], orr.numpy()) < 4e-6, (i, rel_rms(gr[sl], orr.numpy()))
