"""The bounds-checked build (libpswf_lr_checked.so, kernels compiled with
-DPSWF_BOUNDS_CHECK: an index outside its buffer records a status and skips
the access) on valid inputs -- stencils, batches, the real-space cell list
and its backward: every case matches the oracle like the normal build and
no check fails -- pswf_sync would report PSWF_EBOUNDS otherwise.
Runs in a child process that loads the checked library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import math, sys
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
import numpy as np, torch
from paper_2606_06617_b300 import lr
from paper_2606_06617_b300 import workloads as wl
from gpu_helpers import TOL_FP32, run_oracle, window_cw
from conftest import rel_rms
assert lr.LIB_PATH.endswith("libpswf_lr_checked.so"), lr.LIB_PATH
dev = torch.device("cuda", 0)
C = math.log(3.0 / 1e-5)
cases = [  # (box, grid, P, r_c, c, exponents): ragged tiles, own transform with channel quadruples, small grid
    ((13.0, 17.5, 11.0), (27, 35, 21), 7, 4.5, C, (1, 2, 3, 4, 5, 6)),
    ((19.2, 17.6, 19.2), (64, 64, 64), 7, 4.0, C, (1, 2, 4, 6)),
    ((5.0, 5.0, 6.0), (6, 6, 8), 4, 2.5, 6.0, (1, 6)),
]
for i, (box, M, P, r_c, C, ps) in enumerate(cases):
    s = wl.random_system(int(0.1 * np.prod(box)), box, ps, seed=50 + i, neutral=bool(i % 2))
    cw = window_cw(box, M, P, C, r_c)
    plan = lr.Plan(box, s.n, s.ps, r_c, c=C, c_w=cw, P=P, grid=M, device=dev)
    plan.set_points(torch.tensor(s.pos, device=dev), torch.tensor(s.q, dtype=torch.float32, device=dev))
    e, phi, f = plan.execute()
    plan.sync()                     # raises PswfError (PSWF_EBOUNDS) if a check failed
    o = run_oracle(s, r_c, P, M, C, cw)
    assert rel_rms(phi.cpu().double().numpy(), o["phi"]) <= TOL_FP32, i
    assert rel_rms(f.cpu().double().numpy(), o["F"]) <= TOL_FP32, i
# a batch of structures (four-channel chunks, several slots)
structs = [wl.random_system(120 + 30 * k, (9.0 + k, 10.0, 11.0), (1, 6) * 4, seed=70 + k) for k in range(3)]
bp = lr.BatchPlan((12.0, 12.0, 12.0), 4, 1000, 8, (1, 6), 4.0, grid=24, device=dev)
off = np.concatenate([[0], np.cumsum([t.n for t in structs])]).astype(np.int64)
bp.set_points(np.array([t.box for t in structs]), np.array([t.ps for t in structs], dtype=np.int32), off,
              torch.tensor(np.concatenate([t.pos for t in structs]), device=dev),
              torch.tensor(np.concatenate([t.q for t in structs], axis=1), dtype=torch.float32, device=dev))
bp.execute()
bp.sync()
# the real-space cell list (half-shell pairs, accumulator rows) and its backward
from oracle.realspace import real_space
box = (13.0, 14.5, 12.5)
s = wl.random_system(300, box, (1, 2, 3, 4, 5, 6), seed=41, neutral=False)
plan = lr.Plan(box, s.n, s.ps, 4.0, c=C, P=6, grid=(28, 30, 26), flags=lr.PSWF_FLAG_REAL_SPACE, device=dev)
pos_d, q_d = torch.tensor(s.pos, device=dev), torch.tensor(s.q, dtype=torch.float32, device=dev)
e, phi, f = plan.real_space(pos_d, q_d)
gq, gp = plan.real_space_backward(pos_d, q_d, g_energy=torch.ones(len(s.ps), dtype=torch.float64, device=dev),
                                  g_forces=torch.ones_like(f))
plan.sync()
F = np.zeros((s.n, 3))
for c, p in enumerate(s.ps):
    o = real_space(s.pos, s.q[c], box, p, C, 4.0)
    assert rel_rms(phi[c].cpu().double().numpy(), o["phi"]) <= TOL_FP32, c
    F += o["F"]
assert rel_rms(f.cpu().double().numpy(), F) <= TOL_FP32
print("checked build: no failed check")
"""


def test_checked_build_on_valid_inputs():
    from paper_2606_06617_b300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, PSWF_LR_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "no failed check" in r.stdout
