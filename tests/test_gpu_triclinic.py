"""General (triclinic) cells through the C-ABI (pswf_plan_create_cell).

The same sheared cell on every transform path (own passes FP32, pruned
cuFFT FP32 and FP64, full cuFFT transform) against the O1 oracle of that
cell with the same grid, P, c and c_w (FP32 2e-6, FP64 2e-9 relative RMS);
a rotated box against the box (rotation invariance of the GPU path); a
diagonal cell equal to the box plan; the backward against the oracle's VJP
and the virial tensor against the oracle's strain differences in the same
cell."""
import math

import numpy as np
import pytest

from conftest import rel_rms
from gpu_helpers import TOL_FP32, TOL_FP64

pytestmark = pytest.mark.gpu

C = math.log(3.0 / 1e-5)
R_C = 4.0
SHEARED = np.array([[19.2, 0.0, 0.0], [4.5, 18.0, 0.0], [-3.0, 3.5, 17.5]])


def _cw(cell, M, P, c=C):
    h = max(float(np.linalg.norm(a)) / m for a, m in zip(np.asarray(cell, dtype=float), M))
    return P * math.pi * (1.0 - 0.5 * h * (c / R_C) / math.pi)


def _system(cell, n, seed, ps=(1, 6)):
    rng = np.random.default_rng(seed)
    s = rng.uniform(-0.5, 1.5, size=(n, 3))          # images outside the cell too
    pos = s @ np.asarray(cell, dtype=float)
    q = rng.normal(size=(len(ps), n))
    q[0] -= q[0].mean()
    return pos, q


def _run(cell, M, P, cw, pos, q, precision, box=None):
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    plan = lr.Plan(box, len(pos), (1, 6), R_C, c=C, c_w=cw, P=P, grid=M, precision=precision, device=dev,
                   cell=cell)
    plan.set_points(torch.tensor(pos, device=dev), torch.tensor(q, dtype=plan.dtype, device=dev))
    e, phi, f = plan.execute()
    plan.sync()
    return (e.cpu().numpy()[:-1], phi.cpu().double().numpy(), f.cpu().double().numpy(), plan.info)


def _oracle(cell, M, P, cw, pos, q):
    from oracle.grid import DiscretePSWF, GridConfig
    o = DiscretePSWF(GridConfig((0, 0, 0), M, P, C, R_C, (1, 6), c_w=cw, cell=cell)).evaluate(pos, q)
    return o["E_ch"].numpy(), o["phi"].numpy(), o["F"].numpy()


@pytest.mark.parametrize("M,precision,transform", [
    ((64, 64, 64), 0, 3),     # own passes
    ((72, 60, 54), 0, 1),     # pruned, cuFFT (lengths not 32 N1)
    ((64, 64, 64), 1, 1),     # FP64: pruned, cuFFT
    ((40, 36, 30), 0, 0),     # Mx < 64: full 3-D transform
])
def test_sheared_cell_matches_oracle(M, precision, transform):
    P = 6
    cw = _cw(SHEARED, M, P)
    pos, q = _system(SHEARED, 700, 11)
    e, phi, f, info = _run(SHEARED, M, P, cw, pos, q, precision)
    assert info["transform"] == transform, info
    assert np.allclose(np.array(info["cell"]).reshape(3, 3), SHEARED)
    oe, ophi, of = _oracle(SHEARED, M, P, cw, pos, q)
    tol = TOL_FP32 if precision == 0 else TOL_FP64
    for c in range(2):
        assert abs(e[c] - oe[c]) <= tol * abs(oe[c]), (c, e[c], oe[c])
    assert rel_rms(phi, ophi) <= tol, rel_rms(phi, ophi)
    assert rel_rms(f, of) <= tol, rel_rms(f, of)


def test_rotated_box_equals_box():
    box = (17.0, 18.5, 16.0)
    M = (64, 64, 64)
    P = 6
    cw = _cw(np.diag(box), M, P)
    pos, q = _system(np.diag(box), 600, 5)
    th = 0.6
    Rz = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    Ry = np.array([[math.cos(0.3), 0.0, math.sin(0.3)], [0.0, 1.0, 0.0], [-math.sin(0.3), 0.0, math.cos(0.3)]])
    R = Ry @ Rz
    for precision, tol in ((1, 1e-9), (0, TOL_FP32)):
        e0, p0, f0, _ = _run(None, M, P, cw, pos, q, precision, box=box)
        e1, p1, f1, info = _run(np.diag(box) @ R.T, M, P, cw, pos @ R.T, q, precision)
        assert np.allclose(e1, e0, rtol=tol)
        assert rel_rms(p1, p0) <= tol
        assert rel_rms(f1, f0 @ R.T) <= tol


def test_diagonal_cell_is_the_box_plan():
    box = (16.0, 17.0, 15.0)
    M = (64, 60, 48)
    P = 6
    cw = _cw(np.diag(box), M, P)
    pos, q = _system(np.diag(box), 400, 6)
    a = _run(None, M, P, cw, pos, q, 0, box=box)
    b = _run(np.diag(box), M, P, cw, pos, q, 0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def _clear_bandwidth(cell, c0, gap=1.5e-4):
    """The first c = c0 (1 + j / 4000) for which no reciprocal-lattice mode
    has |k| within a relative gap of k_c = c / R_C.  Phi-hat_p drops to zero
    at k_c (psi_0 taken as zero beyond the band), so the energy jumps when a strain moves a mode across
    the band edge; the oracle's central differences (strains up to 1e-4, which
    change |k| by at most that fraction) must not straddle such a jump to
    measure the derivative.  Modes lie about 1.4e-4 apart in |k| / k_c here."""
    from oracle.direct import kvectors
    for j in range(400):
        c = c0 * (1.0 + j / 4000.0)
        _, kk = kvectors(cell, 1.2 * c / R_C)
        if np.min(np.abs(kk / (c / R_C) - 1.0)) > gap:
            return c
    raise AssertionError("no clear band edge")


@pytest.mark.parametrize("M,precision,tol", [
    ((64, 64, 64), 0, 2e-5),   # own transform
    ((64, 64, 64), 1, 1e-7),   # FP64, pruned cuFFT
    ((40, 36, 30), 1, 1e-7),   # full transform
])
def test_sheared_cell_stress_matches_oracle(M, precision, tol):
    """Virial tensor (pswf_stress, xx yy zz xy xz yz) in a sheared cell
    against the oracle's central differences under symmetric strain;
    pswf_virial is its diagonal."""
    import torch
    from oracle.grid import DiscretePSWF, GridConfig
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    P = 6
    c = _clear_bandwidth(SHEARED, C)
    cw = _cw(SHEARED, M, P, c)
    pos, q = _system(SHEARED, 200, 31)
    plan = lr.Plan(None, len(pos), (1, 6), R_C, c=c, c_w=cw, P=P, grid=M, precision=precision,
                   flags=lr.PSWF_FLAG_VIRIAL, device=dev, cell=SHEARED)
    plan.set_points(torch.tensor(pos, device=dev), torch.tensor(q, dtype=plan.dtype, device=dev))
    e, _, _ = plan.execute()
    W6 = plan.stress().cpu().numpy()
    Wd = plan.virial().cpu().numpy()
    plan.sync()
    assert np.array_equal(Wd, W6[:, :3])
    ref = DiscretePSWF(GridConfig((0, 0, 0), M, P, c, R_C, (1, 6), c_w=cw, cell=SHEARED)).stress_fd(pos, q)
    idx = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    E = e.cpu().numpy()
    for c in range(2):
        r6 = np.array([ref[c][a, b] for a, b in idx])
        bound = 3 * tol * max(np.abs(r6).max(), abs(E[c]))
        assert np.abs(W6[c] - r6).max() <= bound, (c, W6[c], r6)


@pytest.mark.parametrize("M,precision,tol", [
    ((64, 64, 64), 0, 2e-5),   # own transform
    ((64, 64, 64), 1, 1e-8),   # FP64, pruned cuFFT
    ((40, 36, 30), 1, 1e-8),   # full transform
])
def test_sheared_cell_backward_matches_oracle_vjp(M, precision, tol):
    """pswf_backward in a sheared cell: L = gE.E + gphi.phi + gF.F with
    seeded upstream gradients against the oracle's reverse-mode VJP of the
    same discrete forward (grid coordinates inside, Cartesian dL/dr out)."""
    import torch
    from oracle.grid import DiscretePSWF, GridConfig
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    P = 6
    cw = _cw(SHEARED, M, P)
    pos, q = _system(SHEARED, 250, 21)
    rng = np.random.default_rng(3)
    gE, gphi, gF = rng.normal(size=2), rng.normal(size=(2, len(pos))), rng.normal(size=(len(pos), 3))
    plan = lr.Plan(None, len(pos), (1, 6), R_C, c=C, c_w=cw, P=P, grid=M, precision=precision,
                   flags=lr.PSWF_FLAG_BACKWARD, device=dev, cell=SHEARED)
    plan.set_points(torch.tensor(pos, device=dev), torch.tensor(q, dtype=plan.dtype, device=dev))
    plan.execute()
    gq, gr = plan.backward(torch.tensor(gE, device=dev), torch.tensor(gphi, dtype=plan.dtype, device=dev),
                           torch.tensor(gF, dtype=plan.dtype, device=dev))
    plan.sync()
    oq, orr = DiscretePSWF(GridConfig((0, 0, 0), M, P, C, R_C, (1, 6), c_w=cw, cell=SHEARED)).vjp(
        pos, q, gE, gphi, gF)
    assert rel_rms(gq.cpu().double().numpy(), oq.numpy()) <= tol
    assert rel_rms(gr.cpu().double().numpy(), orr.numpy()) <= tol
