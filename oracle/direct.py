"""O2: the continuous PSWF-LR reciprocal sum by direct structure factors.

Eq. (Fourier) with its latent structure factor
rho^(p)(k) = sum_i q_i^(p) exp(i k . r_i), truncated at the effective cutoff
k_c = c / r_c (Phi-hat_p vanishes beyond it, psi_0(x/c) taken as zero for x > c), without any
grid, window or FFT:

    E_k   = 1/(2V) sum_{0 < |k| < k_c} Phi-hat_p(k) |rho(k)|^2
    phi_i = 1/V    sum_k Phi-hat_p(k) Re[exp(-i k.r_i) rho(k)]      (= dE/dq_i)
    F_i   = q_i/V  sum_k Phi-hat_p(k) k Im[exp(i k.r_i) conj(rho(k))] (= -dE/dr_i)

The zero-frequency term and its potential shift are added as in O1.
Plain numpy, FP64, O(N * number of modes).
"""
from __future__ import annotations

import math

import numpy as np

from .mollifiers import Mollifier


def cell_matrix(box) -> np.ndarray:
    """3 x 3 cell with the lattice vectors as rows: diag(box) for an
    orthorhombic box given as three edge lengths."""
    b = np.asarray(box, dtype=np.float64)
    return np.diag(b) if b.shape == (3,) else b.reshape(3, 3)


def kvectors(box, k_max: float):
    """All k = 2 pi H^-1 m (m integer, the reciprocal lattice of the cell H
    whose rows are the lattice vectors; k = 2 pi m / L for a box) with
    0 < |k| < k_max, full sphere, both signs.  |m_d| <= k_max |a_d| / 2 pi
    because m_d = k . a_d / 2 pi."""
    H = cell_matrix(box)
    mmax = np.floor(k_max * np.linalg.norm(H, axis=1) / (2 * math.pi)).astype(int) + 1
    rng = [np.arange(-m, m + 1) for m in mmax]
    mx, my, mz = np.meshgrid(*rng, indexing="ij")
    m = np.stack([mx.ravel(), my.ravel(), mz.ravel()], 1).astype(np.float64)
    k = 2 * math.pi * m @ np.linalg.inv(H).T
    kk = np.linalg.norm(k, axis=1)
    keep = (kk > 0) & (kk < k_max)
    return k[keep], kk[keep]


def structure_factor_sum(pos, q, box, ps, c, r_c, chunk: int = 2048):
    """box: three edge lengths or a 3 x 3 cell (rows = lattice vectors).
    Returns dict(E, E_ch [K], E_k [K], E0 [K], phi [K,N], F [N,3], f [K,N,3])."""
    pos = np.asarray(pos, dtype=np.float64)
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    V = float(abs(np.linalg.det(cell_matrix(box))))
    moll = Mollifier(c, r_c)
    kvec, kk = kvectors(box, moll.k_c)
    K, N = q.shape
    E_k = np.zeros(K)
    phi = np.zeros((K, N))
    f = np.zeros((K, N, 3))
    for ci, p in enumerate(ps):
        Ph = moll.phi_hat(p, kk)
        for s in range(0, len(kk), chunk):
            kv = kvec[s:s + chunk]
            ph = Ph[s:s + chunk]
            e = np.exp(1j * pos @ kv.T)                      # [N, nk] = exp(i k.r_i)
            rho = q[ci] @ e                                  # [nk]
            E_k[ci] += float(np.sum(ph * np.abs(rho) ** 2)) / (2 * V)
            phi[ci] += (np.conj(e) * rho[None, :]).real @ ph / V
            im = (e * np.conj(rho)[None, :]).imag * ph[None, :]   # [N, nk]
            f[ci] += (im @ kv) / V
    a = np.array([moll.zero_freq_coef(p, V) for p in ps])
    Qnet = q.sum(axis=1)
    E0 = a * Qnet ** 2
    phi += (2 * a * Qnet)[:, None]
    F = np.einsum("kn,knd->nd", q, f)
    return dict(E=float(np.sum(E_k + E0)), E_ch=E_k + E0, E_k=E_k, E0=E0, phi=phi, F=F, f=f)
