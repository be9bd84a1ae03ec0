"""Pins of the grid oracle O1 and the direct oracle O2, and of the whole
PSWF-LR decomposition against Ewald (Eq. Fourier + real-space complement -
self energy = the 1/r^p lattice sum)."""
import math

import numpy as np
import pytest
import torch

from conftest import rel_rms
from oracle.direct import structure_factor_sum
from oracle.ewald import ewald
from oracle.grid import DiscretePSWF, GridConfig
from oracle.realspace import pswf_total
from paper_2606_06617_b300 import workloads as wl

C = math.log(3.0 / 1e-5)


def cw_max(box, M, P, c, rc):
    eta = max(L / m for L, m in zip(box, M)) * (c / rc) / math.pi
    return P * math.pi * (1 - eta / 2)


def test_naive_dft_equals_fftn():
    """The transform step of O1 (torch.fft.fftn) equals the DFT written out."""
    s = wl.random_system(5, (4.0, 5.0, 4.5), (1,), seed=0)
    o = DiscretePSWF(GridConfig(s.box, (4, 6, 5), 3, 6.0, 2.0, s.ps))
    rho = o.spread(torch.tensor(s.pos), torch.tensor(s.q))[0]
    assert torch.max(torch.abs(o.naive_dft(rho) - torch.fft.fftn(rho))) < 1e-12


def test_window_partition_of_stencil():
    """Each atom's P stencil weights per dimension are psi_0^{c_w} at the
    P points (i0 + j - u) h / omega, all inside [-1, 1]."""
    s = wl.random_system(50, (7.0, 7.0, 7.0), (1,), seed=4)
    o = DiscretePSWF(GridConfig(s.box, (14, 14, 14), 6, C, 4.0, s.ps))
    idx, W, dW = o.stencil(torch.tensor(s.pos))
    assert torch.all(W > 0)
    assert idx.min() >= 0 and idx.max() < 14


def test_o1_quadratic_form_and_gradient():
    """E = 1/2 sum q phi (with the zero-frequency term) and F = -dE/dr by
    autograd through the discrete operator."""
    s = wl.random_system(40, (8.0, 9.0, 7.5), (1, 6), seed=2, neutral=False)
    M = (16, 18, 15)
    o = DiscretePSWF(GridConfig(s.box, M, 6, C, 3.0, s.ps, c_w=cw_max(s.box, M, 6, C, 3.0)))
    r = o.evaluate(s.pos, s.q)
    assert abs(0.5 * float(torch.sum(torch.tensor(s.q) * r["phi"])) / r["E"] - 1) < 1e-12
    pos = torch.tensor(s.pos, requires_grad=True)
    E = o.evaluate(pos, s.q)["E_tensor"]
    (g,) = torch.autograd.grad(E, pos)
    assert rel_rms(-g.numpy(), r["F"].numpy()) < 1e-12


def test_o2_forces_and_invariances():
    s = wl.random_system(30, (7.0, 7.0, 8.0), (1,), seed=6)
    r = structure_factor_sum(s.pos, s.q, s.box, s.ps, C, 3.0)
    assert np.abs(r["F"].sum(0)).max() < 1e-12 * np.abs(r["F"]).max()
    r2 = structure_factor_sum(s.pos + np.array([0.37, -1.1, 2.3]), s.q, s.box, s.ps, C, 3.0)
    assert abs(r2["E"] / r["E"] - 1) < 1e-12
    h = 1e-5
    pp = s.pos.copy(); pp[4, 1] += h
    pm = s.pos.copy(); pm[4, 1] -= h
    fd = -(structure_factor_sum(pp, s.q, s.box, s.ps, C, 3.0)["E"]
           - structure_factor_sum(pm, s.q, s.box, s.ps, C, 3.0)["E"]) / (2 * h)
    assert abs(fd - r["F"][4, 1]) < 1e-7 * np.abs(r["F"]).max()


def test_o1_converges_to_o2():
    """The grid algorithm approximates the continuous sum; the spreading error
    falls with P at the largest alias-free window bandwidth."""
    s = wl.random_charges()
    o2 = structure_factor_sum(s.pos, s.q, s.box, s.ps, C, 4.0)
    errs = []
    for P in (6, 8, 10):
        M = (24, 24, 24)
        o1 = DiscretePSWF(GridConfig(s.box, M, P, C, 4.0, s.ps, c_w=cw_max(s.box, M, P, C, 4.0))).evaluate(s.pos, s.q)
        errs.append(rel_rms(o1["F"].numpy(), o2["F"]))
        assert rel_rms(o1["phi"].numpy(), o2["phi"]) < 1e-4
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 5e-6 and errs[2] < 1e-7


def test_pswf_total_matches_ewald_random_charges():
    """O2 + real-space complement - self energy against Ewald: the method's
    band-truncation error at c = log(3 / 1e-5), r_c = 4."""
    s = wl.random_charges()
    o2 = structure_factor_sum(s.pos, s.q, s.box, s.ps, C, 4.0)
    tot = pswf_total(o2, s.pos, s.q, s.box, s.ps, C, 4.0)
    ew = ewald(s.pos, s.q[0], s.box, 1)
    assert abs(tot["E"] / ew["E"] - 1) < 5e-6
    assert rel_rms(tot["F"], ew["F"]) < 2e-5
    assert rel_rms(tot["phi"][0], ew["phi"]) < 1e-5


def test_pswf_total_matches_madelung():
    """NaCl (shells at 3.99 and 4.88 A straddle r_c = 4): the total within the
    method's band error at c = log(3 / 1e-5)."""
    s = wl.nacl()
    o2 = structure_factor_sum(s.pos, s.q, s.box, s.ps, C, 4.0)
    tot = pswf_total(o2, s.pos, s.q, s.box, s.ps, C, 4.0)
    assert abs(tot["E"] / (-32 * 1.747564594633182 / 2.82) - 1) < 5e-5


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_pswf_total_charged_channels(p):
    """Non-neutral channels: the zero-frequency terms (p > 3 formula,
    Eq. Correction for p <= 2 with the background-integral reading for p = 1,
    Eq. Correction3r for p = 3) make the PSWF total match Ewald with a
    neutralising background (p <= 2) or the finite-part k = 0 term (p = 3:
    both splittings then give the same total, whatever r_c, c or alpha)."""
    s = wl.random_system(20, (7.0, 7.0, 7.0), (p,), seed=10 + p, neutral=False)
    s.q = s.q + 0.3                                     # clearly charged
    o2 = structure_factor_sum(s.pos, s.q, s.box, s.ps, C, 3.0)
    tot = pswf_total(o2, s.pos, s.q, s.box, s.ps, C, 3.0)
    ew = ewald(s.pos, s.q[0], s.box, p)
    tol = {1: 2e-5, 2: 1e-4, 3: 1e-4, 4: 1e-3, 5: 1e-3, 6: 1e-3}[p]
    assert abs(tot["E"] - ew["E"]) < tol * abs(ew["E_self"])
    assert rel_rms(tot["phi"][0], ew["phi"]) < tol


def test_o1_vjp_matches_finite_differences():
    """The oracle's vector-jacobian product (used as the reference of the
    GPU backward) against central finite differences of evaluate itself, for
    a loss touching the energies, the potentials and the forces.  A dropped
    term of the VJP (the zero-frequency part of phi, the second derivative of
    W in the force term, the grid-mediated part) fails one of the checks."""
    s = wl.random_system(12, (6.0, 6.5, 7.0), (1, 4), seed=11, neutral=False)
    M = (12, 13, 14)
    o = DiscretePSWF(GridConfig(s.box, M, 6, C, 2.5, s.ps, c_w=cw_max(s.box, M, 6, C, 2.5)))
    rng = np.random.default_rng(3)
    gE = rng.normal(size=2)
    gphi = rng.normal(size=(2, 12))
    gF = rng.normal(size=(12, 3))

    def loss(pos, q):
        r = o.evaluate(pos, q)
        return float(np.dot(gE, r["E_ch"].numpy()) + np.sum(gphi * r["phi"].numpy()) + np.sum(gF * r["F"].numpy()))

    gq, gr = o.vjp(s.pos, s.q, gE, gphi, gF)
    eps = 1e-5
    for (c, i) in [(0, 0), (1, 5), (0, 11)]:
        qp, qm = s.q.copy(), s.q.copy()
        qp[c, i] += eps
        qm[c, i] -= eps
        fd = (loss(s.pos, qp) - loss(s.pos, qm)) / (2 * eps)
        assert abs(fd - float(gq[c, i])) < 1e-6 * max(1.0, abs(fd))
    for (i, d) in [(0, 0), (3, 1), (7, 2), (11, 0)]:
        pp, pm = s.pos.copy(), s.pos.copy()
        pp[i, d] += eps
        pm[i, d] -= eps
        fd = (loss(pp, s.q) - loss(pm, s.q)) / (2 * eps)
        assert abs(fd - float(gr[i, d])) < 1e-6 * max(1.0, abs(fd))
    # energy-only upstream: dE/dq = phi and dE/dr = -F
    r = o.evaluate(s.pos, s.q)
    gq1, gr1 = o.vjp(s.pos, s.q, np.ones(2))
    assert rel_rms(gq1.numpy(), r["phi"].numpy()) < 1e-12
    assert rel_rms(gr1.numpy(), -r["F"].numpy()) < 1e-12


def test_o1_virial_homogeneity():
    """The oracle's virial (central differences of E_c under L_d -> L_d (1 +-
    eps), fractional coordinates fixed) plus the real-space complement's
    virial equals p E for the assembled 1/r^p total (a lattice sum of a
    degree -p homogeneous kernel), to the method's accuracy; and the
    difference quotient is converged (two step sizes agree)."""
    from oracle.realspace import real_space
    s = wl.random_system(60, (9.0, 10.0, 11.0), (1,), seed=5, neutral=True)
    M, P, rc = (24, 27, 30), 8, 4.0
    o = DiscretePSWF(GridConfig(s.box, M, P, C, rc, s.ps, c_w=cw_max(s.box, M, P, C, rc)))
    r = o.evaluate(s.pos, s.q)
    W = o.virial_fd(s.pos, s.q)
    W2 = o.virial_fd(s.pos, s.q, eps=1e-4)
    assert np.allclose(W, W2, rtol=1e-7, atol=1e-9)
    eps = 1e-5
    W_real = 0.0
    for d in range(3):
        Es = []
        for sg in (1, -1):
            box = list(s.box)
            box[d] *= 1 + sg * eps
            pp = s.pos.copy()
            pp[:, d] *= 1 + sg * eps
            Es.append(real_space(pp, s.q[0], box, 1, C, rc)["E"])
        W_real += -(Es[0] - Es[1]) / (2 * eps)
    tot = pswf_total({"E_ch": r["E_ch"].numpy(), "phi": r["phi"].numpy(), "f": r["f"].numpy()},
                     s.pos, s.q, s.box, s.ps, C, rc)
    assert abs(W.sum() + W_real - tot["E"]) <= 1e-3 * abs(tot["E"])
