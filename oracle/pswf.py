"""Order-zero prolate spheroidal wave function psi_0^c (oracle, FP64).

Definition followed (Methods, "Prolate spheroidal wave functions",
Eq. (formula) and Eq. (psidefinit)): psi_0^c is the eigenfunction of
F_c[phi](x) = int_{-1}^{1} phi(t) exp(i c x t) dt belonging to the eigenvalue
of largest modulus, lambda_0, scaled so that psi_0^c(0) = 1.

Method (written for this oracle, independent of the CUDA library's planner,
which expands psi_0 in Legendre polynomials instead): psi_0 is even, so on
even functions F_c has the real symmetric kernel cos(c x t).  A Nystrom
discretisation at n Gauss-Legendre nodes t_j with weights w_j gives the
symmetric matrix sqrt(w_i) cos(c t_i t_j) sqrt(w_j); its top eigenpair gives
lambda_0 and psi_0(t_j).  The eigen-relation itself is then the interpolant:

    psi_0(x) = (1/lambda_0) * sum_j w_j psi_0(t_j) cos(c x t_j),

valid (and entire) for every real x, with derivatives of any order obtained by
differentiating cos.  With psi_0(0) = 1, setting x = 0 in Eq. (psidefinit)
gives lambda_0 = int_{-1}^{1} psi_0 = 2 C_0.
"""
from __future__ import annotations

import numpy as np
import torch


def gauss_legendre(a: float, b: float, n: int = 64):
    """Gauss-Legendre nodes and weights on [a, b] (numpy's leggauss)."""
    x, w = np.polynomial.legendre.leggauss(n)
    half = 0.5 * (b - a)
    return a + half * (x + 1.0), half * w


class PSWF:
    """psi_0^c with psi_0^c(0) = 1, its eigenvalue lambda_0 and C_0.

    Attributes
    ----------
    c : bandwidth parameter of Eq. (formula)
    lam0 : lambda_0 (real and positive for n = 0)
    C0 : int_0^1 psi_0^c(x) dx  (Eq. G1)
    """

    def __init__(self, c: float, n_quad: int | None = None):
        if not c > 0:
            raise ValueError("c must be positive")
        self.c = float(c)
        n = n_quad or int(max(64, 2 * np.ceil(1.5 * c) + 48))
        n += n % 2                      # even order: no node at t = 0
        t, w = np.polynomial.legendre.leggauss(n)
        sw = np.sqrt(w)
        A = sw[:, None] * np.cos(self.c * np.outer(t, t)) * sw[None, :]
        evals, evecs = np.linalg.eigh(A)
        lam = float(evals[-1])
        v = evecs[:, -1] / sw
        self._t = t
        self._ct = self.c * t
        # psi(0) = (1/lam) sum_j w_j v_j  -> rescale so that psi(0) = 1
        psi0 = float(np.dot(w, v)) / lam
        v = v / psi0
        self._wv = w * v / lam          # so that psi(x) = sum_j _wv_j cos(c x t_j)
        self.lam0 = lam
        self.C0 = self.integral(0.0, 1.0)
        self._wv_t = torch.tensor(self._wv, dtype=torch.float64)
        self._ct_t = torch.tensor(self._ct, dtype=torch.float64)

    # ---- evaluation -----------------------------------------------------
    def __call__(self, x, d: int = 0):
        """d-th derivative of psi_0^c at x (numpy, any real x)."""
        x = np.asarray(x, dtype=np.float64)
        ph = np.multiply.outer(x, self._ct) + d * (np.pi / 2)
        return (np.cos(ph) * self._ct ** d) @ self._wv

    def torch(self, x: torch.Tensor, d: int = 0) -> torch.Tensor:
        """Same as __call__ in torch FP64, differentiable in x to any order."""
        ph = x.unsqueeze(-1) * self._ct_t + d * (np.pi / 2)
        return (torch.cos(ph) * self._ct_t ** d) @ self._wv_t

    def antiderivative(self, x):
        """int_0^x psi_0^c(s) ds (numpy), from the interpolant (no t_j is 0)."""
        x = np.asarray(x, dtype=np.float64)
        return (np.sin(np.multiply.outer(x, self._ct)) / self._ct) @ self._wv

    def antiderivative_torch(self, x: torch.Tensor) -> torch.Tensor:
        """int_0^x psi_0^c(s) ds in torch FP64 (differentiable)."""
        return (torch.sin(x.unsqueeze(-1) * self._ct_t) / self._ct_t) @ self._wv_t

    def moment(self, u, m: int):
        """int_0^u s**m psi_0^c(s) ds for m in {0, 1, 3}, vectorised over u.

        Closed form for the interpolant sum_j a_j cos(b_j s): antiderivatives
        of s**m cos(b s) (m = 0: sin(bs)/b; m = 1: cos(bs)/b^2 + s sin(bs)/b;
        m = 3: s^3 sin/b + 3 s^2 cos/b^2 - 6 s sin/b^3 - 6 cos/b^4)."""
        u = np.asarray(u, dtype=np.float64)
        b = self._ct
        bu = np.multiply.outer(u, b)
        su, cu = np.sin(bu), np.cos(bu)
        uu = u[..., None]
        if m == 0:
            F = su / b
        elif m == 1:
            F = cu / b ** 2 + uu * su / b - 1.0 / b ** 2
        elif m == 3:
            F = (uu ** 3 * su / b + 3 * uu ** 2 * cu / b ** 2 - 6 * uu * su / b ** 3
                 - 6 * cu / b ** 4 + 6.0 / b ** 4)
        else:
            raise ValueError("moment order must be 0, 1 or 3")
        return F @ self._wv

    def inv_moment(self, u):
        """int_u^1 psi_0^c(s) / s ds for 0 < u <= 1, vectorised: the
        interpolant gives sum_j a_j (Ci(|b_j|) - Ci(|b_j| u))."""
        from scipy.special import sici
        u = np.asarray(u, dtype=np.float64)
        b = np.abs(self._ct)
        ci1 = sici(b)[1]
        ciu = sici(np.multiply.outer(u, b))[1]
        return (ci1 - ciu) @ self._wv

    # ---- integrals ---------------------------------------------------------
    def integral(self, a: float, b: float, power: int = 0, n: int = 96) -> float:
        """int_a^b s**power * psi_0^c(s) ds by Gauss-Legendre (entire integrand)."""
        if a == b:
            return 0.0
        s, w = gauss_legendre(a, b, n)
        return float(np.dot(w, s ** power * self(s)))

    def eigen_residual(self, x, quad=None) -> np.ndarray:
        """lambda_0 psi_0(x) - int_{-1}^{1} psi_0(t) exp(i c x t) dt, using an
        independent quadrature rule (default: 200-point Gauss-Legendre)."""
        t, w = quad if quad is not None else gauss_legendre(-1.0, 1.0, 200)
        x = np.atleast_1d(np.asarray(x, dtype=np.float64))
        f = self(t)
        integ = (np.exp(1j * self.c * np.multiply.outer(x, t)) * f) @ w
        return self.lam0 * self(x) - integ
