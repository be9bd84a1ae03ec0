"""Shared helpers of the GPU parity tests: run the CUDA path through the
C-ABI binding and the O1 oracle on the same seeded inputs and parameters."""
from __future__ import annotations

import math

import numpy as np

# FP32 path vs FP64 oracle: relative RMS bound on phi and forces, and the
# relative bound on energies (target of the FP32 path).
TOL_FP32 = 2e-6
# FP64 path: window tables fitted to 1e-15 relative, FFT round-off amplified
# by the force stencil (measured ~3e-10 on the water box).
TOL_FP64 = 2e-9


def window_cw(box, M, P, c, r_c):
    """Window bandwidth used by both sides: c_w = P pi (1 - eta / 2), with
    eta = max_d h_d k_c / pi (the planner's default, passed explicitly)."""
    h = max(float(L) / float(m) for L, m in zip(box, M))
    eta = h * (c / r_c) / math.pi
    return P * math.pi * (1.0 - 0.5 * eta)


def run_gpu(sysm, r_c, P, M, c, c_w, precision=0, pos_dtype="float64", flags=0):
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    plan = lr.Plan(sysm.box, sysm.n, sysm.ps, r_c, c=c, c_w=c_w, P=P, grid=M, precision=precision,
                   flags=flags, device=dev)
    pos = torch.tensor(sysm.pos, dtype=getattr(torch, pos_dtype), device=dev)
    q = torch.tensor(sysm.q, dtype=plan.dtype, device=dev)
    plan.set_points(pos, q)
    e, phi, f = plan.execute()
    plan.sync()
    torch.cuda.synchronize()
    return dict(E_ch=e[:-1].cpu().numpy(), E=float(e[-1]), phi=phi.cpu().numpy().astype(np.float64),
                F=f.cpu().numpy().astype(np.float64), info=plan.info, plan=plan, pos=pos, q=q)


def run_oracle(sysm, r_c, P, M, c, c_w):
    from oracle.grid import DiscretePSWF, GridConfig
    o = DiscretePSWF(GridConfig(tuple(sysm.box), tuple(int(m) for m in M), P, c, r_c, tuple(sysm.ps), c_w=c_w))
    r = o.evaluate(sysm.pos, sysm.q)
    return dict(E_ch=r["E_ch"].numpy(), E=r["E"], phi=r["phi"].numpy(), F=r["F"].numpy(),
                f=r["f"].numpy(), self=o.self_energy(sysm.q), Psi=r["Psi"])
