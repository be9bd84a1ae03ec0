"""Pins of the oracles for general (triclinic) cells.

* O2 depends only on the lattice: a unimodular change of basis (same lattice,
  other cell vectors) must leave energies, potentials and forces unchanged.
* O1 is rotation invariant: an orthorhombic box and the same box rotated
  (cell H R^T, positions r R^T) give the same energies and potentials and the
  rotated forces, to rounding.
* O1 on a sheared cell agrees with O2 within the method error (the grid is
  uniform in fractional coordinates; the window bandwidth at the alias limit
  of the cell's effective spacing |a_d| / M_d).
* O1 forces are -dE/dr by central differences on a sheared cell.
"""
import math

import numpy as np
import pytest

from conftest import rel_rms

C = math.log(3.0 / 1e-5)


def _cw(cell, M, P, c, r_c):
    """c_w = P pi (1 - eta / 2), eta = max_d h_d k_c / pi, h_d = |a_d| / M_d."""
    h = max(float(np.linalg.norm(a)) / m for a, m in zip(np.asarray(cell, dtype=float), M))
    return P * math.pi * (1.0 - 0.5 * h * (c / r_c) / math.pi)


def _system(cell, n, seed, ps=(1, 6)):
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.0, 1.0, size=(n, 3))
    pos = s @ np.asarray(cell, dtype=float)
    q = rng.normal(size=(len(ps), n))
    q[0] -= q[0].mean()
    return pos, q


SHEARED = np.array([[13.0, 0.0, 0.0], [3.5, 12.0, 0.0], [-2.0, 2.5, 11.0]])


def test_o2_is_a_function_of_the_lattice():
    from oracle.direct import structure_factor_sum
    U = np.array([[1, 0, 0], [1, 1, 0], [0, -1, 1]], dtype=float)   # det 1
    other = U @ SHEARED
    pos, q = _system(SHEARED, 40, 1)
    a = structure_factor_sum(pos, q, SHEARED, (1, 6), C, 4.0)
    b = structure_factor_sum(pos, q, other, (1, 6), C, 4.0)
    assert np.allclose(a["E_ch"], b["E_ch"], rtol=1e-11)
    assert rel_rms(a["phi"], b["phi"]) < 1e-11
    assert rel_rms(a["F"], b["F"]) < 1e-11


def test_o1_rotation_invariance():
    from oracle.grid import DiscretePSWF, GridConfig
    box = (11.0, 12.5, 10.0)
    M = (24, 24, 24)
    P = 6
    pos, q = _system(np.diag(box), 50, 2)
    th = 0.7
    Rz = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, math.cos(0.4), -math.sin(0.4)], [0.0, math.sin(0.4), math.cos(0.4)]])
    R = Rx @ Rz
    cw = _cw(np.diag(box), M, P, C, 4.0)
    a = DiscretePSWF(GridConfig(box, M, P, C, 4.0, (1, 6), c_w=cw)).evaluate(pos, q)
    b = DiscretePSWF(GridConfig(box, M, P, C, 4.0, (1, 6), c_w=cw, cell=np.diag(box) @ R.T)).evaluate(pos @ R.T, q)
    assert np.allclose(a["E_ch"].numpy(), b["E_ch"].numpy(), rtol=1e-11)
    assert rel_rms(b["phi"].numpy(), a["phi"].numpy()) < 1e-11
    assert rel_rms(b["F"].numpy(), a["F"].numpy() @ R.T) < 1e-11


@pytest.mark.parametrize("P,tol", [(6, 5e-4), (8, 1e-5)])
def test_o1_sheared_cell_matches_o2(P, tol):
    """The method error on the sheared cell is that of an orthorhombic box
    with the same edge lengths (1.8e-4 at P = 6 and 1.8e-6 at P = 8 for the
    orthorhombic cases of the window reading): within 1.3 times it, and
    within tol."""
    from oracle.direct import structure_factor_sum
    from oracle.grid import DiscretePSWF, GridConfig
    M = (28, 28, 28)

    def errors(cell, box):
        pos, q = _system(cell, 60, 3)
        cw = _cw(cell, M, P, C, 4.0)
        o1 = DiscretePSWF(GridConfig(box, M, P, C, 4.0, (1, 6), c_w=cw, cell=cell)).evaluate(pos, q)
        o2 = structure_factor_sum(pos, q, cell, (1, 6), C, 4.0)
        ef = [rel_rms(o1["f"][c].numpy(), o2["f"][c]) for c in range(2)]
        ee = [abs(float(o1["E_ch"][c]) / o2["E_ch"][c] - 1.0) for c in range(2)]
        return ef, ee, rel_rms(o1["phi"].numpy(), o2["phi"])

    edges = tuple(float(x) for x in np.linalg.norm(SHEARED, axis=1))
    ef, ee, ep = errors(SHEARED, edges)
    ef0, _, _ = errors(np.diag(edges), edges)
    for c in range(2):
        assert ef[c] <= 1.3 * ef0[c] + 1e-7, (c, ef[c], ef0[c])
        assert ef[c] <= tol and ee[c] <= tol, (c, ef[c], ee[c])
    assert ep <= tol


def test_o1_sheared_forces_are_minus_energy_gradient():
    from oracle.grid import DiscretePSWF, GridConfig
    M = (20, 20, 20)
    P = 6
    pos, q = _system(SHEARED, 12, 4)
    o = DiscretePSWF(GridConfig((0, 0, 0), M, P, C, 4.0, (1, 6), c_w=_cw(SHEARED, M, P, C, 4.0), cell=SHEARED))
    F = o.evaluate(pos, q)["F"].numpy()
    eps = 1e-5
    for i in (0, 5):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += eps
            pm[i, d] -= eps
            g = (o.evaluate(pp, q)["E"] - o.evaluate(pm, q)["E"]) / (2 * eps)
            assert abs(-g - F[i, d]) <= 1e-6 * max(1.0, abs(F[i, d])), (i, d, -g, F[i, d])


def test_stress_diagonal_is_the_box_virial():
    """On a box the diagonal of the strain-derivative tensor is the
    independently coded edge-scaling virial (virial_fd)."""
    from oracle.grid import DiscretePSWF, GridConfig
    box = (11.0, 12.0, 10.5)
    M = (20, 22, 20)
    P = 6
    pos, q = _system(np.diag(box), 30, 7, ps=(1, 6))
    o = DiscretePSWF(GridConfig(box, M, P, C, 4.0, (1, 6), c_w=_cw(np.diag(box), M, P, C, 4.0)))
    W = o.stress_fd(pos, q)
    Wd = o.virial_fd(pos, q)
    for c in range(2):
        assert np.allclose(np.diag(W[c]), Wd[c], rtol=1e-6, atol=1e-9 * abs(Wd[c]).max())
        assert np.allclose(W[c], W[c].T)


def test_stress_rotates_with_the_cell():
    """W(R H, R r) = R W(H, r) R^T, the off-diagonal entries included."""
    from oracle.grid import DiscretePSWF, GridConfig
    M = (20, 20, 20)
    P = 6
    pos, q = _system(SHEARED, 24, 8)
    th = 0.5
    R = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    cw = _cw(SHEARED, M, P, C, 4.0)
    W0 = DiscretePSWF(GridConfig((0, 0, 0), M, P, C, 4.0, (1, 6), c_w=cw, cell=SHEARED)).stress_fd(pos, q)
    W1 = DiscretePSWF(GridConfig((0, 0, 0), M, P, C, 4.0, (1, 6), c_w=cw, cell=SHEARED @ R.T)).stress_fd(
        pos @ R.T, q)
    for c in range(2):
        ref = R @ W0[c] @ R.T
        # central differences of FP64 energies: ~1e-12 / eps relative rounding
        assert np.abs(W1[c] - ref).max() <= 1e-5 * np.abs(ref).max(), (c, W1[c], ref)
        assert np.abs(W0[c] - np.diag(np.diag(W0[c]))).max() > 1e-3 * np.abs(W0[c]).max()   # really a tensor
