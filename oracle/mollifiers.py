"""PSWF mollifiers, Fourier multipliers, window transform, self-energy and
zero-frequency terms (oracle, FP64).

Every formula is written out from Methods:

* real-space mollifiers G_p(r): Eq. (G1), Eq. (G6) and Eq. (G);
* Fourier multipliers Phi-hat_p(k): Eq. (PhiH), with C-hat_0 defined just
  before it;
* window transform W-hat: the equation following the definition of W_pswf in
  "Accelerating atom-grid spreading with PSWFs";
* self-energy E_self^(p): the equation in "Implementation details";
* zero-frequency term E^{0,(p)}: the p > 3 equation, Eq. (Correction) and
  Eq. (Correction3r).

Readings taken where the paper is silent or inconsistent:

* in Eq. (PhiH) psi_0^c(x/c) is taken as zero for x > c (the PSWF lives
  on [-1, 1] in the Fourier variable); so C-hat_0 = c lambda_0 C_0, every
  "int^infinity" stops at c, and Phi-hat_p(k) = 0 for k >= k_c = c / r_c.
* Phi-hat_1 is used exactly as printed (not re-derived from G_1).
* G_p(r) is its formula for r < r_c and 1 for r >= r_c.
* for p = 1 the zero-frequency term uses the background integral
  int_0^{r_c} r (1 - G_1(r)) dr, i.e. the printed "r psi_0(r/r_c)" is read as
  "r G_1(r)"; E_IB = 0 (tin-foil).  The Ewald oracle decides this reading.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .pswf import PSWF, gauss_legendre


class Mollifier:
    """Mollifier family for a given bandwidth c and cutoff r_c."""

    def __init__(self, c: float, r_c: float, psi: PSWF | None = None):
        self.c = float(c)
        self.r_c = float(r_c)
        self.psi = psi if psi is not None else PSWF(c)
        self.lam0 = self.psi.lam0
        self.C0 = self.psi.C0
        # C-hat_0 = int_0^inf lambda_0 psi_0(x/c) dx = c lambda_0 C_0 (psi_0^c(x/c) taken as zero for x > c)
        self.Chat0 = self.c * self.lam0 * self.C0
        self.k_c = self.c / self.r_c

    # ---- the x-integrals of Eq. (PhiH) ------------------------------------
    # With x = c s and psi_0^c(x/c) taken as zero for x > c:
    #   int_0^{k r_c} lambda_0 psi_0(x/c) dx       = c lambda_0 int_0^u psi_0
    #   int_{k r_c}^inf x^m lambda_0 psi_0(x/c) dx = c^(m+1) lambda_0 int_u^1 s^m psi_0
    #   int_{k r_c}^inf lambda_0 psi_0(x/c) / x dx = lambda_0 int_u^1 psi_0(s)/s ds
    # where u = min(k r_c / c, 1).
    def _head(self, u):
        return self.c * self.lam0 * self.psi.moment(u, 0)

    def _tail(self, u, m: int):
        return self.c ** (m + 1) * self.lam0 * (self.psi.moment(1.0, m) - self.psi.moment(u, m))

    def _tail_over_x(self, u):
        out = np.zeros_like(u)
        inside = u < 1.0
        out[inside] = self.lam0 * self.psi.inv_moment(u[inside])
        return out

    # ---- Phi-hat_p (Eq. PhiH) ---------------------------------------------
    def phi_hat(self, p: int, k):
        """Fourier transform of G_p(r)/r^p at wavenumbers k (Eq. PhiH),
        vectorised over k.  p = 1, 2, 3 are singular at k = 0."""
        k = np.asarray(k, dtype=np.float64)
        scalar = k.ndim == 0
        k = np.atleast_1d(k)
        if p <= 3 and np.any(k == 0.0):
            raise ValueError(f"Phi-hat_{p} is singular at k = 0")
        r_c, Chat0, C0 = self.r_c, self.Chat0, self.C0
        u = np.minimum(k * r_c / self.c, 1.0)
        if p == 1:
            psi_u = self.psi(u)
            out = np.where(k * r_c / self.c <= 1.0,
                           4.0 * math.pi * psi_u / (k * k * float(self.psi(0.0))), 0.0)
        elif p == 2:
            out = 2.0 * math.pi ** 2 / k * (1.0 - self._head(u) / Chat0)
        elif p == 3:
            out = 2.0 * math.pi / C0 * self._tail_over_x(u)
        elif p == 4:
            out = -(math.pi ** 2 / Chat0) * (
                Chat0 * k - k * self._head(u) - self._tail(u, 1) / r_c)
        elif p == 5:
            with np.errstate(invalid="ignore"):
                t1 = np.where(k > 0, k * k * self._tail_over_x(np.maximum(u, 1e-300)), 0.0)
            out = -(math.pi / (3.0 * C0)) * (t1 - self._tail(u, 1) / r_c ** 2)
        elif p == 6:
            out = (math.pi ** 2 / (12.0 * Chat0)) * (
                Chat0 * k ** 3
                - k ** 3 * self._head(u)
                - 1.5 * k * k / r_c * self._tail(u, 1)
                + 0.5 / r_c ** 3 * self._tail(u, 3))
        else:
            raise ValueError(f"p = {p} is not one of 1..6")
        return float(out[0]) if scalar else out

    def phi_hat_quad(self, p: int, k: float) -> float:
        """Scalar Phi-hat_p by adaptive quadrature of the printed x-integrals
        (cross-check of the closed-form moments used by phi_hat)."""
        from scipy.integrate import quad
        lam, c, r_c = self.lam0, self.c, self.r_c
        f = lambda x, m: x ** m * lam * float(self.psi(x / c))
        kr = min(k * r_c, c)
        opt = dict(epsabs=1e-14, epsrel=1e-13, limit=200)
        Chat0 = quad(f, 0.0, c, args=(0,), **opt)[0]
        head = quad(f, 0.0, kr, args=(0,), **opt)[0] if kr > 0 else 0.0
        t1 = quad(f, kr, c, args=(1,), **opt)[0]
        t3 = quad(f, kr, c, args=(3,), **opt)[0]
        if p == 2:
            return 2 * math.pi ** 2 / k * (1 - head / Chat0)
        if p == 4:
            return -(math.pi ** 2 / Chat0) * (Chat0 * k - k * head - t1 / r_c)
        if p == 6:
            return (math.pi ** 2 / (12 * Chat0)) * (Chat0 * k ** 3 - k ** 3 * head
                                                   - 1.5 * k * k / r_c * t1 + 0.5 / r_c ** 3 * t3)
        raise ValueError("quadrature cross-check covers p = 2, 4, 6")

    # ---- real-space mollifiers (Eq. G1, G6, G) ------------------------------
    def G(self, p: int, r):
        """G_p(r) for r < r_c; 1 for r >= r_c (taken so beyond the cutoff).  numpy."""
        r = np.asarray(r, dtype=np.float64)
        x = r / self.r_c
        psi, C0 = self.psi, self.C0
        if p == 1:
            g = psi.antiderivative(x) / C0
        elif p == 2:
            g = 1.0 - psi(x)
        elif p == 3:
            g = (psi.antiderivative(x) - x * psi(x)) / C0
        elif p == 4:
            g = 1.0 - psi(x) + 0.5 * x * psi(x, 1)
        elif p == 5:
            g = (psi.antiderivative(x) - x * psi(x) + x * x / 3.0 * psi(x, 1)) / C0
        elif p == 6:
            g = 1.0 - psi(x) + 0.625 * x * psi(x, 1) - 0.125 * x * x * psi(x, 2)
        else:
            raise ValueError(f"p = {p} is not one of 1..6")
        return np.where(x < 1.0, g, 1.0)

    def G_torch(self, p: int, r: torch.Tensor) -> torch.Tensor:
        """Same as G, differentiable torch FP64."""
        x = r / self.r_c
        psi, C0 = self.psi, self.C0
        if p == 1:
            g = psi.antiderivative_torch(x) / C0
        elif p == 2:
            g = 1.0 - psi.torch(x)
        elif p == 3:
            g = (psi.antiderivative_torch(x) - x * psi.torch(x)) / C0
        elif p == 4:
            g = 1.0 - psi.torch(x) + 0.5 * x * psi.torch(x, 1)
        elif p == 5:
            g = (psi.antiderivative_torch(x) - x * psi.torch(x) + x * x / 3.0 * psi.torch(x, 1)) / C0
        elif p == 6:
            g = 1.0 - psi.torch(x) + 0.625 * x * psi.torch(x, 1) - 0.125 * x * x * psi.torch(x, 2)
        else:
            raise ValueError(f"p = {p} is not one of 1..6")
        return torch.where(x < 1.0, g, torch.ones_like(g))

    # ---- self-energy (Implementation details) -------------------------------
    def self_coef(self, p: int) -> float:
        """s_p with E_self^(p) = s_p * Q_self^(p), Q_self = sum_i |q_i|^2."""
        psi, C0, r_c = self.psi, self.C0, self.r_c
        if p == 1:
            return float(psi(0.0)) / (2.0 * C0 * r_c)
        if p == 2:
            return -float(psi(0.0, 2)) / (4.0 * r_c ** 2)
        if p == 3:
            return -float(psi(0.0, 2)) / (6.0 * C0 * r_c ** 3)
        if p == 4:
            return float(psi(0.0, 4)) / (48.0 * r_c ** 4)
        if p == 5:
            return float(psi(0.0, 4)) / (90.0 * C0 * r_c ** 5)
        if p == 6:
            return -float(psi(0.0, 6)) / (1440.0 * r_c ** 6)
        raise ValueError(f"p = {p} is not one of 1..6")

    # ---- zero-frequency term ----------------------------------------------
    def zero_freq_coef(self, p: int, V: float) -> float:
        """a_p with E^{0,(p)} = a_p * Q_net^2 (so d/dq_i = 2 a_p Q_net).

        p > 3: Phi-hat_p(0) / (2V).  p = 2: Eq. (Correction).  p = 1:
        Eq. (Correction) with the background-integral reading and E_IB = 0.  p = 3:
        Eq. (Correction3r) as printed; it equals Q^2/(2V) times the finite part
        lim_{k->0} (Phi-hat_3(k) + 4 pi log k), the k = 0 convention that makes
        the charged p = 3 total independent of the splitting."""
        r_c = self.r_c
        if p > 3:
            return float(self.phi_hat(p, 0.0)) / (2.0 * V)
        if p == 2:
            # int_0^{r_c} psi_0(r/r_c) dr = r_c C_0
            return -2.0 * math.pi / V * r_c * self.C0
        if p == 1:
            # int_0^{r_c} r (1 - G_1(r)) dr, Gauss-Legendre on [0, r_c]
            r, w = gauss_legendre(0.0, r_c, 96)
            return -2.0 * math.pi / V * float(np.dot(w, r * (1.0 - self.G(1, r))))
        if p == 3:
            s, w = gauss_legendre(0.0, 1.0, 96)
            tail = float(np.dot(w, (self.psi(s) - 1.0) / s))
            return 2.0 * math.pi / V * (math.log(self.c / r_c) + tail)
        raise ValueError(f"p = {p} is not one of 1..6")


def window_hat(psi_w: PSWF, omega: float, k):
    """W-hat_pswf(k) = omega lambda_0 psi_0^{c_w}(omega k / c_w), valid for
    |omega k / c_w| <= 1 (the equation after the definition of W_pswf)."""
    k = np.asarray(k, dtype=np.float64)
    arg = omega * k / psi_w.c
    if np.any(np.abs(arg) > 1.0 + 1e-12):
        raise ValueError("W-hat requested outside the PSWF band")
    return omega * psi_w.lam0 * psi_w(arg)
