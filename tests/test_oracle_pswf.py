"""Pins of the oracle's psi_0^c (Methods, "Prolate spheroidal wave
functions") against facts that do not come from the oracle itself."""
import numpy as np
import pytest
import scipy.special as sp
from scipy.integrate import quad

from oracle.pswf import PSWF

CS = [1.0, 6.0, 12.024, 12.611537753638338, 20.0]


@pytest.mark.parametrize("c", CS)
def test_eigen_relation(c):
    """lambda_0 psi_0(x) = int_{-1}^{1} psi_0(t) exp(icxt) dt (Eq. psidefinit)
    at 50 random points, with a quadrature rule unrelated to the Nystrom nodes."""
    ps = PSWF(c)
    x = np.random.default_rng(0).uniform(-1, 1, 50)
    res = ps.eigen_residual(x)
    assert np.max(np.abs(res)) < 1e-12 * ps.lam0


@pytest.mark.parametrize("c", [1.0, 6.0, 12.024, 12.611537753638338])
def test_matches_scipy_prolate_angular_function(c):
    """psi_0^c is the prolate angular function S_00(c, x) scaled to 1 at 0
    (scipy.special.pro_ang1, accurate for c <~ 14)."""
    ps = PSWF(c)
    x = np.linspace(-0.98, 0.98, 41)
    S = np.array([sp.pro_ang1(0, 0, c, v)[0] for v in x])
    dS = np.array([sp.pro_ang1(0, 0, c, v)[1] for v in x])
    S0 = sp.pro_ang1(0, 0, c, 0.0)[0]
    assert np.max(np.abs(ps(x) - S / S0)) < 1e-10
    assert np.max(np.abs(ps(x, 1) - dS / S0)) < 1e-9 * max(1.0, c)


@pytest.mark.parametrize("c", CS)
def test_prolate_ode(c):
    """(1 - x^2) psi'' - 2 x psi' + (chi - c^2 x^2) psi = 0 with chi the
    characteristic value of scipy.special.pro_cv (pins psi', psi'')."""
    ps = PSWF(c)
    chi = sp.pro_cv(0, 0, c)
    x = np.linspace(-1, 1, 33)
    r = (1 - x * x) * ps(x, 2) - 2 * x * ps(x, 1) + (chi - c * c * x * x) * ps(x)
    tol = 1e-9 if c <= 14 else 1e-6   # pro_cv itself loses accuracy for large c
    assert np.max(np.abs(r)) < tol * max(1.0, c * c)


@pytest.mark.parametrize("c", CS)
def test_lambda0_equals_twice_C0(c):
    """Setting x = 0 in Eq. (psidefinit) with psi_0(0) = 1: lambda_0 = 2 C_0,
    C_0 = int_0^1 psi_0 by adaptive quadrature."""
    ps = PSWF(c)
    C0 = quad(lambda t: float(ps(t)), 0.0, 1.0, epsabs=1e-15, epsrel=1e-13)[0]
    assert abs(ps(0.0) - 1.0) < 1e-14
    assert abs(ps.lam0 - 2 * C0) < 1e-12
    assert abs(ps.C0 - C0) < 1e-13


def test_small_c_limit():
    """c -> 0: F_c -> integration against 1, psi_0 -> 1 (Legendre P_0), lambda_0 -> 2."""
    ps = PSWF(1e-3)
    x = np.linspace(-1, 1, 21)
    assert np.max(np.abs(ps(x) - 1.0)) < 1e-6
    assert abs(ps.lam0 - 2.0) < 1e-6


@pytest.mark.parametrize("c", CS)
def test_even_positive_decreasing(c):
    ps = PSWF(c)
    x = np.linspace(0, 1, 201)
    v = ps(x)
    assert np.allclose(v, ps(-x), atol=1e-14)
    assert np.all(v > 0) and np.all(np.diff(v) < 0)


def test_band_edge_value_shrinks_with_c():
    """The band-truncation size psi_0^c(1) decays roughly like exp(-c)
    ("Parameter selection": c ~ log(1/eps))."""
    cs = (8.0, 12.0, 16.0, 20.0)
    vals = [float(PSWF(c)(1.0)) for c in cs]
    assert all(a > b for a, b in zip(vals, vals[1:]))
    for c, v in zip(cs, vals):
        assert 1e-2 * np.exp(-c) < v < 1e2 * np.exp(-c)


@pytest.mark.parametrize("m", [0, 1, 3])
def test_moments_against_quadrature(m):
    ps = PSWF(12.6)
    u = np.array([0.0, 0.05, 0.3, 0.77, 1.0])
    ref = [quad(lambda s: s ** m * float(ps(s)), 0, x, epsabs=1e-15, epsrel=1e-13)[0] for x in u]
    assert np.max(np.abs(ps.moment(u, m) - ref)) < 1e-12
    v = np.array([0.02, 0.5, 0.9])
    ref2 = [quad(lambda s: float(ps(s)) / s, x, 1, epsabs=1e-15, epsrel=1e-13)[0] for x in v]
    assert np.max(np.abs(ps.inv_moment(v) - ref2)) < 1e-11
