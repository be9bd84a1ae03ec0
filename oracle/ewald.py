"""O3: physical lattice sums of q_i q_j / r^p (oracle, FP64).

Classical Ewald splitting with the incomplete-gamma screening of
Eq. (screening): G_p^Ewald(r) = Gamma(p/2, alpha^2 r^2) / Gamma(p/2) (upper,
regularised), whose complement is the lower incomplete gamma.  For
E = 1/2 sum_n sum_ij' q_i q_j / |r_ij + n L|^p (Eq. realLR with G_p = 1):

* real part:        1/2 sum' q_i q_j Gamma(p/2, alpha^2 r^2) / (Gamma(p/2) r^p)
* reciprocal part:  1/(2V) sum_{k != 0} phi-hat(k) |rho(k)|^2 with the Fourier
  transform of the smooth part gamma(p/2, alpha^2 r^2) / (Gamma(p/2) r^p),
  phi-hat(k) = pi^{3/2} (k/2)^{p-3} Gamma((3-p)/2, k^2/(4 alpha^2)) / Gamma(p/2)
  (p = 1 gives 4 pi exp(-k^2/(4 alpha^2)) / k^2);
* self term:        1/2 sum_i q_i^2 alpha^p / Gamma(p/2 + 1);
* k = 0 term:       p > 3: pi^{3/2} 2 alpha^{p-3} / ((p-3) Gamma(p/2)) Q^2/(2V);
                    p = 1: -pi Q^2 / (2 V alpha^2) (neutralising background);
                    p = 2: -pi^{3/2} Q^2 / (alpha V) (same);
                    p = 3: the finite part of phi-hat at k -> 0 times
                    Q^2/(2V): phi-hat = 2 pi E_1(k^2/(4 alpha^2)) =
                    -4 pi log k + 2 pi (log(4 alpha^2) - gamma) + O(k^2),
                    so pi (log(4 alpha^2) - gamma) Q^2 / V (gamma: Euler's
                    constant).  The charged p = 3 sum diverges like log R
                    without a convention; taking the finite part of the
                    kernel transform for the k = 0 term gives the same total
                    for every splitting parameter (tests pin this).

Gamma(s, x) for s <= 0 comes from Gamma(s+1, x) = s Gamma(s, x) + x^s e^{-x}
started at Gamma(1/2, x) = sqrt(pi) erfc(sqrt(x)), Gamma(1, x) = e^{-x} or
Gamma(0, x) = E_1(x).

:func:`image_sum` is the plain absolutely convergent sum for p > 3 (explicit
images inside a sphere of radius R, optionally with a smooth taper, plus the
uniform-density remainder).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc, exp1, gamma, gammaincc

from .direct import kvectors


def upper_gamma(s: float, x):
    """Non-regularised upper incomplete gamma Gamma(s, x) for s in
    {1, 1/2, 0, -1/2, -1, -3/2, ...}, x > 0."""
    x = np.asarray(x, dtype=np.float64)
    if s == 1.0:
        return np.exp(-x)
    if s == 0.5:
        return math.sqrt(math.pi) * erfc(np.sqrt(x))
    if s == 0.0:
        return exp1(x)
    if s < 0:
        return (upper_gamma(s + 1.0, x) - x ** s * np.exp(-x)) / s
    raise ValueError(f"unsupported s = {s}")


def screening(p: int, x):
    """Ewald screening G_p = Gamma(p/2, x^2) / Gamma(p/2), x = alpha r
    (regularised upper incomplete gamma)."""
    return gammaincc(p / 2.0, np.asarray(x, dtype=np.float64) ** 2)


def _images(box, r_cut):
    box = np.asarray(box, dtype=np.float64)
    nmax = np.ceil(r_cut / box).astype(int) + 1
    rng = [np.arange(-m, m + 1) for m in nmax]
    n = np.stack(np.meshgrid(*rng, indexing="ij"), -1).reshape(-1, 3)
    return n * box[None, :], n


def ewald(pos, q, box, p: int, alpha: float | None = None, r_cut: float | None = None,
          k_cut: float | None = None):
    """Returns dict(E, E_real, E_recip, E_self, E0, phi [N], F [N,3]).

    Default alpha puts the real-space cutoff at half the smallest box edge, so
    the minimum-image convention applies; tails are ~exp(-42)."""
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    N = len(q)
    V = float(np.prod(box))
    s = p / 2.0
    if alpha is None:
        alpha = 6.5 / (0.5 * float(box.min()))
    if r_cut is None:
        r_cut = 6.5 / alpha
    if k_cut is None:
        k_cut = 2.0 * alpha * 6.5
    Q = float(q.sum())

    # ---- real space ---------------------------------------------------------
    min_image = r_cut <= 0.5 * float(box.min())
    shifts = np.zeros((1, 3)) if min_image else _images(box, r_cut)[0]
    phi = np.zeros(N)
    F = np.zeros((N, 3))
    B = max(1, int(4e6 // max(1, N * len(shifts))))
    for i0 in range(0, N, B):
        d = pos[i0:i0 + B, None, None, :] - pos[None, None, :, :] + shifts[None, :, None, :]   # [b,S,N,3]
        if min_image:
            d = d - box * np.round(d / box)
        r = np.linalg.norm(d, axis=-1)
        mask = (r < r_cut) & (r > 0)
        rr = np.where(mask, r, 1.0)
        x2 = (alpha * rr) ** 2
        Qg = screening(p, alpha * rr)
        g = np.where(mask, Qg / rr ** p, 0.0)
        phi[i0:i0 + B] += np.einsum("bsn,n->b", g, q)
        # d/dr [Q(s, a^2 r^2) r^-p] = -2 a^p e^{-a^2 r^2} / (Gamma(s) r) - p Q r^{-p-1}
        dg = np.where(mask, -2.0 * alpha ** p * np.exp(-x2) / (gamma(s) * rr) - p * Qg / rr ** (p + 1), 0.0)
        F[i0:i0 + B] -= q[i0:i0 + B, None] * np.einsum("bsn,bsnd->bd", q[None, None, :] * dg / rr, d)
    E_real = 0.5 * float(np.dot(q, phi))

    # ---- reciprocal space (half sphere: k and -k give the same |rho|^2) ----
    kvec, kk = kvectors(box, k_cut)
    half = (kvec[:, 0] > 0) | ((kvec[:, 0] == 0) & ((kvec[:, 1] > 0) | ((kvec[:, 1] == 0) & (kvec[:, 2] > 0))))
    kvec, kk = kvec[half], kk[half]
    phk = 2.0 * math.pi ** 1.5 * (kk / 2.0) ** (p - 3) * upper_gamma((3.0 - p) / 2.0, kk ** 2 / (4 * alpha ** 2)) / gamma(s)
    E_recip = 0.0
    phi_r = np.zeros(N)
    for a in range(0, len(kk), 2048):
        kv, ph = kvec[a:a + 2048], phk[a:a + 2048]
        e = np.exp(1j * pos @ kv.T)
        rho = q @ e
        E_recip += float(np.sum(ph * np.abs(rho) ** 2)) / (2 * V)
        phi_r += (np.conj(e) * rho[None, :]).real @ ph / V
        F += q[:, None] * (((e * np.conj(rho)[None, :]).imag * ph[None, :]) @ kv) / V

    # ---- self and k = 0 -----------------------------------------------------------
    sc = alpha ** p / gamma(s + 1.0)
    E_self = 0.5 * sc * float(np.sum(q ** 2))
    if p > 3:
        a0 = math.pi ** 1.5 * 2.0 * alpha ** (p - 3) / ((p - 3) * gamma(s)) / (2 * V)
    elif p == 1:
        a0 = -math.pi / (2 * V * alpha ** 2)
    elif p == 2:
        a0 = -math.pi ** 1.5 / (alpha * V)
    else:
        a0 = math.pi * (math.log(4.0 * alpha ** 2) - np.euler_gamma) / V
    E0 = a0 * Q * Q
    phi_tot = phi + phi_r - sc * q + 2 * a0 * Q
    E = E_real + E_recip - E_self + E0
    return dict(E=E, E_real=E_real, E_recip=E_recip, E_self=E_self, E0=E0, phi=phi_tot, F=F)


def _taper(x):
    """C^infinity partition: 1 for x <= 1/2, 0 for x >= 1, smooth between."""
    x = np.asarray(x, dtype=np.float64)
    t = np.clip(2.0 * x - 1.0, 0.0, 1.0)
    with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
        a = np.where(t > 0, np.exp(-1.0 / np.where(t > 0, t, 1.0)), 0.0)
        b = np.where(t < 1, np.exp(-1.0 / np.where(t < 1, 1.0 - t, 1.0)), 0.0)
        return np.where(t <= 0, 1.0, np.where(t >= 1, 0.0, b / (a + b)))


def _dtaper(x, eps=1e-6):
    return (_taper(x + eps) - _taper(x - eps)) / (2 * eps)


def image_sum(pos, q, box, p: int, R: float, smooth: bool = False):
    """Plain lattice sum for p > 3 (absolutely convergent):
    E = 1/2 sum' q_i q_j S(r/R) r^-p over explicit images, plus the
    uniform-density remainder 1/2 Q^2 (4 pi / V) int_0^inf r^{2-p} (1 - S) dr.
    S is a sharp cutoff at R (smooth=False) or a C-infinity taper from R/2 to
    R (smooth=True, faster convergence).  Returns (E, F [N,3])."""
    if p <= 3:
        raise ValueError("explicit image sums need p > 3")
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    V = float(np.prod(box))
    shifts, _ = _images(box, R)
    E = 0.0
    F = np.zeros((len(q), 3))
    for i in range(len(q)):
        d = pos[i][None, None, :] - pos[None, :, :] + shifts[:, None, :]
        r = np.linalg.norm(d, axis=-1)
        mask = (r < R) & (r > 0)
        rr = np.where(mask, r, 1.0)
        if smooth:
            S = _taper(rr / R)
            dS = _dtaper(rr / R) / R
        else:
            S = np.ones_like(rr)
            dS = np.zeros_like(rr)
        f = np.where(mask, S / rr ** p, 0.0)
        # -d/dr [S r^-p] = p S r^{-p-1} - S' r^-p
        mdf = np.where(mask, p * S / rr ** (p + 1) - dS / rr ** p, 0.0)
        E += 0.5 * q[i] * float(np.sum(q[None, :] * f))
        F[i] += q[i] * np.sum((q[None, :] * mdf / rr)[..., None] * d, axis=(0, 1))
    Q = float(q.sum())
    if smooth:
        from .pswf import gauss_legendre
        rq, wq = gauss_legendre(R / 2, R, 200)
        rem = float(np.dot(wq, rq ** (2 - p) * (1 - _taper(rq / R)))) + R ** (3 - p) / (p - 3)
    else:
        rem = R ** (3 - p) / (p - 3)
    E += 0.5 * Q * Q * 4 * math.pi / V * rem
    return E, F
