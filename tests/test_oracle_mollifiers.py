"""Pins of the oracle's mollifiers and multipliers (Methods, Eq. G1, G6, G,
PhiH, the window transform, the self-energy and zero-frequency terms)."""
import math

import mpmath
import numpy as np
import pytest

from oracle.mollifiers import Mollifier, window_hat
from oracle.pswf import PSWF, gauss_legendre

C = math.log(3.0 / 1e-5)
RC = 4.0


@pytest.fixture(scope="module")
def moll():
    return Mollifier(C, RC)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_phi_hat_is_fourier_transform_of_G(moll, p):
    """Phi-hat_p of Eq. (PhiH) and G_p of Eq. (G1/G6/G) are written from
    different formulas; the inverse 3-D radial transform of the (band-limited)
    Phi-hat_p must reproduce G_p(r) / r^p inside r_c."""
    k, w = gauss_legendre(0.0, moll.k_c, 3000)
    ph = moll.phi_hat(p, k)
    for r in (0.5, 1.0, 2.0, 3.0, 3.9):
        inv = float(np.dot(w, ph * k * np.sin(k * r))) / (2 * math.pi ** 2 * r)
        ref = float(moll.G(p, r)) / r ** p
        assert abs(inv - ref) < 1e-8 * abs(ref), (p, r, inv, ref)


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_long_range_tail_is_inverse_power(moll, p):
    """lim_{r->inf} G_p(r)/r^p = 1/r^p: beyond r_c the reciprocal kernel is
    1/r^p up to the band-truncation error (grows with the derivative order
    of psi_0 used in G_p)."""
    k, w = gauss_legendre(0.0, moll.k_c, 3000)
    ph = moll.phi_hat(p, k)
    bound = {1: 3e-6, 2: 3e-5, 4: 5e-4, 6: 5e-3}[p]
    for r in (5.0, 7.0, 10.0):
        inv = float(np.dot(w, ph * k * np.sin(k * r))) / (2 * math.pi ** 2 * r)
        assert abs(inv * r ** p - 1.0) < bound, (p, r, inv * r ** p)


def test_small_k_limits(moll):
    """Leading small-k behaviour of Eq. (PhiH): the Fourier transforms of
    1/r^p (4 pi / k^2, 2 pi^2 / k, -4 pi log k, -pi^2 k, pi^2 k^3 / 12)."""
    k = 1e-4
    assert abs(moll.phi_hat(1, k) * k * k / (4 * math.pi) - 1) < 1e-7
    assert abs(moll.phi_hat(2, k) * k / (2 * math.pi ** 2) - 1) < 1e-3
    d3 = moll.phi_hat(3, 1e-4) - moll.phi_hat(3, 1e-3)
    assert abs(d3 / (-4 * math.pi * math.log(1e-4 / 1e-3)) - 1) < 1e-5
    s4 = (moll.phi_hat(4, 2e-4) - moll.phi_hat(4, 1e-4)) / 1e-4
    assert abs(s4 / (-math.pi ** 2) - 1) < 1e-3
    kk = np.linspace(0.0, 0.1, 41)
    A = np.stack([np.ones_like(kk), kk ** 2, kk ** 3, kk ** 4, kk ** 5, kk ** 6], 1)
    coef = np.linalg.lstsq(A, moll.phi_hat(6, kk), rcond=None)[0]
    assert abs(coef[2] / (math.pi ** 2 / 12) - 1) < 1e-5


def test_multiplier_vanishes_at_band_edge(moll):
    """With psi_0(x/c) taken as zero for x > c: Phi-hat_p(k) = 0 for k >= k_c; p = 2..6 reach 0 continuously."""
    for p in (1, 2, 3, 4, 5, 6):
        assert abs(moll.phi_hat(p, moll.k_c * 1.001)) < 1e-12
    for p in (2, 3, 4, 5, 6):
        assert abs(moll.phi_hat(p, moll.k_c * (1 - 1e-9))) < 1e-6 * abs(moll.phi_hat(p, 0.1))


@pytest.mark.parametrize("p", [2, 4, 6])
def test_closed_form_moments_vs_adaptive_quadrature(moll, p):
    for k in (0.3, 1.3, 2.9):
        assert abs(moll.phi_hat(p, k) - moll.phi_hat_quad(p, k)) < 1e-10 * max(1.0, abs(moll.phi_hat(p, k)))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_self_energy_is_half_limit_of_G_over_rp(moll, p):
    """E_self^(p) = s_p Q_self with s_p = 1/2 lim_{r->0} G_p(r)/r^p: the
    printed closed forms (derivatives of psi_0 at 0) against the limit taken
    directly in 80-digit arithmetic on the same psi_0."""
    mpmath.mp.dps = 80
    a = [mpmath.mpf(float(v)) for v in moll.psi._wv]
    b = [mpmath.mpf(float(v)) for v in moll.psi._ct]
    a0 = sum(a)
    a = [ai / a0 for ai in a]                 # psi(0) = 1 exactly in 80 digits
    C0 = sum(ai * mpmath.sin(bi) / bi for ai, bi in zip(a, b))
    psi = lambda x, d=0: sum(ai * bi ** d * mpmath.cos(bi * x + d * mpmath.pi / 2) for ai, bi in zip(a, b))
    I = lambda x: sum(ai * mpmath.sin(bi * x) / bi for ai, bi in zip(a, b))
    G = {1: lambda x: I(x) / C0,
         2: lambda x: 1 - psi(x),
         3: lambda x: (I(x) - x * psi(x)) / C0,
         4: lambda x: 1 - psi(x) + x / 2 * psi(x, 1),
         5: lambda x: (I(x) - x * psi(x) + x * x / 3 * psi(x, 1)) / C0,
         6: lambda x: 1 - psi(x) + 5 * x / 8 * psi(x, 1) - x * x / 8 * psi(x, 2)}[p]
    rc = mpmath.mpf(RC)
    f = lambda r: G(r / rc) / r ** p
    r1, r2 = mpmath.mpf("1e-6"), mpmath.mpf("2e-6")
    lim = (4 * f(r1) - f(r2)) / 3            # Richardson, error O(r^4)
    assert abs(float(lim / 2) / moll.self_coef(p) - 1) < 1e-8


def test_window_transform_matches_quadrature():
    """W-hat_pswf(k) = omega lambda_0 psi_0(omega k / c) against direct
    Gauss-Legendre quadrature of int_{-omega}^{omega} psi_0(a/omega) e^{ika} da."""
    ps = PSWF(14.1)
    omega = 1.5
    a, w = gauss_legendre(-omega, omega, 400)
    for k in np.linspace(0.0, ps.c / omega, 17):
        direct = float(np.dot(w, ps(a / omega) * np.cos(k * a)))
        assert abs(window_hat(ps, omega, k) - direct) < 1e-12 * abs(direct) + 1e-15


def test_zero_frequency_p4_p6_is_phi_hat_at_zero(moll):
    V = 1000.0
    for p in (4, 6):
        assert moll.zero_freq_coef(p, V) == pytest.approx(moll.phi_hat(p, 0.0) / (2 * V), rel=1e-14)
    # Phi-hat_p(0) = 4 pi int_0^inf G_p(r) r^{2-p} dr (direct radial integral),
    # equal up to the band-truncation size.  Below r0 the leading Taylor term
    # of G_p is used (G_4 ~ a_4 x^4, G_6 ~ -a_6 x^6, a_n = psi^(n)(0)/n!), as
    # the closed forms cancel to round-off there.
    r0 = 0.3
    for p in (4, 6):
        r, w = gauss_legendre(r0, RC, 400)
        lead = (float(moll.psi(0.0, 4)) / 24 if p == 4 else -float(moll.psi(0.0, 6)) / 720) / RC ** p
        small = lead * r0 ** 3 / 3
        ref = 4 * math.pi * (float(np.dot(w, moll.G(p, r) * r ** (2 - p))) + small + RC ** (3 - p) / (p - 3))
        assert abs(moll.phi_hat(p, 0.0) / ref - 1) < 1e-3


def test_zero_frequency_p1_reading(moll):
    """The p = 1 background-integral reading: the term -(2 pi Q^2/V) int_0^rc r (1 - G_1) dr
    equals Q^2/(2V) lim_{k->0} (Phi-hat_1(k) - 4 pi / k^2) to O(psi_0(1)); the
    printed 'r psi_0(r/r_c)' integrand does not (it is off by a factor ~20)."""
    V = 1000.0
    a1 = moll.zero_freq_coef(1, V)
    k = 1e-4
    lim = (moll.phi_hat(1, k) - 4 * math.pi / k ** 2) / (2 * V)
    assert abs(a1 / lim - 1) < 1e-3
    printed = -2 * math.pi / V * (RC ** 2 / 2 - RC ** 2 * moll.psi.integral(0.0, 1.0, 1))
    assert abs(printed / a1) > 5


def test_zero_frequency_p3_is_finite_part_at_zero(moll):
    """Eq. (Correction3r): the p = 3 term a_3 Q^2 is Q^2/(2V) times the finite
    part of Phi-hat_3 at k -> 0, i.e. lim (Phi-hat_3(k) + 4 pi log k).  The
    limit is taken on the closed-form multiplier (moments of psi_0) at two
    small k, the coefficient by the quadrature of the printed tail integral;
    a flipped log or tail sign moves it by O(1)."""
    V = 1000.0
    a3 = moll.zero_freq_coef(3, V)
    for k in (1e-5, 1e-6):
        lim = (moll.phi_hat(3, k) + 4 * math.pi * math.log(k)) / (2 * V)
        assert abs(a3 - lim) < 1e-8 * abs(a3) + 1e-12, (k, a3, lim)


def test_zero_frequency_p5_is_phi_hat_at_zero(moll):
    """p = 5: a_5 = Phi-hat_5(0) / (2V), and Phi-hat_5(0) = 4 pi int_0^inf
    G_5(r) r^-3 dr (direct radial integral, up to the band truncation)."""
    V = 1000.0
    assert moll.zero_freq_coef(5, V) == pytest.approx(moll.phi_hat(5, 0.0) / (2 * V), rel=1e-14)
    # below r0, the leading Taylor term of G_5 (G_5 ~ b x^5, b from the r -> 0
    # series of the self-energy: s_5 = b / (2 r_c^5))
    r0 = 0.3
    r, w = gauss_legendre(r0, RC, 400)
    b = 2 * moll.self_coef(5) * RC ** 5
    small = b / RC ** 5 * r0 ** 3 / 3
    ref = 4 * math.pi * (float(np.dot(w, moll.G(5, r) * r ** -3)) + small + RC ** -2 / 2)
    assert abs(moll.phi_hat(5, 0.0) / ref - 1) < 1e-3
