"""Partial outputs of pswf_execute against the O1 oracle.

The energy alone needs only steps (i)-(iv) of "Accelerating atom-grid
spreading with PSWFs" (spread, forward transform, multiplier and the energy
reduction; no inverse transform, no gather).  Potentials alone or forces
alone skip the other output of the gather.  Each branch runs on every
transform path a single plan can take (own passes, cuFFT pruned, cuFFT full)
and is compared with the oracle at the path's tolerance, and with the
full call on the same plan.  Charged p = 3 and p = 5 channels exercise the
zero-frequency terms of "Implementation details" (Eq. Correction3r and the
p > 3 formula) on the device.  Both ways the FP32 sort can place the atoms
(records in the idle grid and an unpack pass, or the direct scatter when
the grid is too small to hold the records) match the oracle."""
import math

import numpy as np
import pytest

from conftest import rel_rms
from gpu_helpers import TOL_FP32, TOL_FP64, run_oracle, window_cw
from paper_2606_06617_b300 import workloads as wl

pytestmark = pytest.mark.gpu

C_TOL = math.log(3.0 / 1e-5)

# (name, box, grid, P, r_c, precision, expected transform)
CASES = [
    ("own", (19.2, 19.2, 19.2), (64, 64, 64), 7, 4.0, 0, 3),
    ("cufft_pruned", (19.2, 19.2, 19.2), (64, 64, 64), 7, 4.0, 1, 1),
    ("cufft_full", (13.0, 17.5, 11.0), (27, 35, 21), 6, 4.5, 0, 0),
]


def _plan(s, box, M, P, r_c, precision):
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    cw = window_cw(box, M, P, C_TOL, r_c)
    plan = lr.Plan(box, s.n, s.ps, r_c, c=C_TOL, c_w=cw, P=P, grid=M, precision=precision, device=dev)
    plan.set_points(torch.tensor(s.pos, device=dev), torch.tensor(s.q, dtype=plan.dtype, device=dev))
    return plan, cw


def _np(t):
    return None if t is None else t.cpu().double().numpy()


@pytest.mark.parametrize("name,box,M,P,r_c,precision,transform", CASES, ids=[c[0] for c in CASES])
def test_partial_outputs(name, box, M, P, r_c, precision, transform):
    nat = int(0.1 * np.prod(box))
    s = wl.random_system(nat, box, (1, 6), seed=21, neutral=False)
    plan, cw = _plan(s, box, M, P, r_c, precision)
    assert plan.info["transform"] == transform, (name, plan.info["transform"])
    tol = TOL_FP32 if precision == 0 else TOL_FP64
    o = run_oracle(s, r_c, P, M, C_TOL, cw)

    def check_energy(e):
        e = e if isinstance(e, np.ndarray) else _np(e)
        for c in range(s.q.shape[0]):
            assert abs(e[c] - o["E_ch"][c]) <= tol * abs(o["E_ch"][c]), (name, c, e[c], o["E_ch"][c])

    full = [_np(x) for x in plan.execute()]
    plan.sync()
    # energy only: no inverse transform, no gather
    e, ph, f = plan.execute(phi=False, forces=False)
    plan.sync()
    assert ph is None and f is None
    check_energy(e)
    # the grid flush adds tiles in arbitrary order: same result to round-off
    np.testing.assert_allclose(_np(e), full[0], rtol=tol / 4, atol=0)
    # potentials only
    e, ph, f = plan.execute(forces=False)
    plan.sync()
    assert f is None
    check_energy(e)
    assert rel_rms(_np(ph), o["phi"]) <= tol, (name, rel_rms(_np(ph), o["phi"]))
    assert rel_rms(_np(ph), full[1]) <= tol / 4
    # forces only, energy not requested
    e, ph, f = plan.execute(energy=False, phi=False)
    plan.sync()
    assert e is None and ph is None
    assert rel_rms(_np(f), o["F"]) <= tol, (name, rel_rms(_np(f), o["F"]))
    assert rel_rms(_np(f), full[2]) <= tol / 4
    # and the full call again, after the partial ones
    again = [_np(x) for x in plan.execute()]
    plan.sync()
    check_energy(again[0])
    assert rel_rms(again[1], o["phi"]) <= tol and rel_rms(again[2], o["F"]) <= tol


@pytest.mark.parametrize("precision", [0, 1])
def test_charged_p3_p5(precision):
    """Non-neutral p = 3 and p = 5 channels: energies (with E^0), potentials
    (with the 2 a_p Q shift) and forces against O1 on a ragged grid."""
    box = (13.0, 17.5, 11.0)
    s = wl.random_system(300, box, (3, 5), seed=31, neutral=False)
    s.q = s.q + 0.3
    M = (27, 35, 21)
    plan, cw = _plan(s, box, M, 6, 4.5, precision)
    e, ph, f = (_np(x) for x in plan.execute())
    plan.sync()
    o = run_oracle(s, 4.5, 6, M, C_TOL, cw)
    tol = TOL_FP32 if precision == 0 else TOL_FP64
    assert np.all(np.abs(o["E_ch"]) > 0)
    for c in range(2):
        assert abs(e[c] - o["E_ch"][c]) <= tol * abs(o["E_ch"][c]), (c, e[c], o["E_ch"][c])
    assert rel_rms(ph, o["phi"]) <= tol
    assert rel_rms(f, o["F"]) <= tol


@pytest.mark.parametrize("ps", [(1, 2, 4, 6), (1, 6, 2, 4, 6, 1, 4, 2)], ids=["K4", "K8"])
def test_own_transform_channel_quadruples(ps):
    """Single FP32 plans on the own transform with K a multiple of four keep
    the potential grid as channel quadruples between the inverse transform
    and the gather: one and two quadruples against O1, all outputs."""
    box = (19.2, 17.6, 19.2)
    M = (64, 64, 64)
    s = wl.random_system(int(0.1 * np.prod(box)), box, ps, seed=41, neutral=False)
    plan, cw = _plan(s, box, M, 7, 4.0, 0)
    assert plan.info["transform"] == 3
    e, ph, f = (_np(x) for x in plan.execute())
    plan.sync()
    o = run_oracle(s, 4.0, 7, M, C_TOL, cw)
    for c in range(len(ps)):
        assert abs(e[c] - o["E_ch"][c]) <= TOL_FP32 * abs(o["E_ch"][c]), (c, e[c], o["E_ch"][c])
    assert rel_rms(ph, o["phi"]) <= TOL_FP32, rel_rms(ph, o["phi"])
    assert rel_rms(f, o["F"]) <= TOL_FP32, rel_rms(f, o["F"])


@pytest.mark.parametrize("natoms", [150, 6000], ids=["records", "direct_scatter"])
def test_sort_paths_small_grid(natoms):
    """A 12^3 grid with one channel holds 1 x 12 x 12 x 14 reals = 8064
    bytes: 150 atoms' records (48 bytes each) fit and take the two-pass
    scatter, 6000 do not and take the direct scatter.  Both against O1."""
    box = (9.0, 9.0, 9.0)
    s = wl.random_system(natoms, box, (1,), seed=31, neutral=True)
    M, P, r_c = (12, 12, 12), 5, 4.0
    plan, cw = _plan(s, box, M, P, r_c, 0)
    e, phi, f = plan.execute()
    plan.sync()
    o = run_oracle(s, r_c, P, M, C_TOL, cw)
    assert rel_rms(phi.cpu().double().numpy(), o["phi"]) <= TOL_FP32
    assert rel_rms(f.cpu().double().numpy(), o["F"]) <= TOL_FP32
