"""PSWF real-space complement and the assembled PSWF-LR total (oracle).

Methods, "Implementation details": pairing Eq. (Fourier) with the real-space
term (1 - G_p(r)) / r^p and subtracting E_self^(p) gives the complete
1/r^p lattice energy, which Ewald (O3) computes independently.  Under
G_p taken as 1 for r >= r_c, the real-space term only involves pairs
closer than r_c.  Forces and potentials come from torch autograd in FP64.
"""
from __future__ import annotations

import numpy as np
import torch

from .mollifiers import Mollifier

f64 = torch.float64


def _pair_energy(pos, q, box, p: int, r_c: float, moll: Mollifier):
    """(pos_t, q_t, E): the real-space energy of one channel as a torch FP64
    graph in the (wrapped) positions and the charges, both requiring grad."""
    b = np.asarray(box, dtype=np.float64)
    H = np.diag(b) if b.shape == (3,) else b.reshape(3, 3)
    # The sum runs over every periodic image, so moving an atom by a lattice
    # vector leaves it unchanged; with all atoms in the primary cell (s in
    # [0, 1) in fractional coordinates s = r H^-1) a displacement closer than
    # r_c needs |n_d| <= ceil(r_c / h_d) + 1, h_d = V / |a_e x a_f| the
    # cell's height across the faces spanned by the other two vectors.
    s = np.asarray(pos, dtype=np.float64) @ np.linalg.inv(H)
    pos = (s - np.floor(s)) @ H
    V = abs(np.linalg.det(H))
    heights = [V / np.linalg.norm(np.cross(H[(d + 1) % 3], H[(d + 2) % 3])) for d in range(3)]
    H_t = torch.tensor(H, dtype=f64)
    pos_t = torch.tensor(np.asarray(pos, dtype=np.float64), dtype=f64, requires_grad=True)
    q_t = torch.tensor(np.asarray(q, dtype=np.float64), dtype=f64, requires_grad=True)
    nmax = [int(np.ceil(r_c / hd)) + 1 for hd in heights]
    shifts = torch.stack(torch.meshgrid(*[torch.arange(-m, m + 1, dtype=f64) for m in nmax],
                                        indexing="ij"), -1).reshape(-1, 3) @ H_t
    N = pos_t.shape[0]
    E = torch.zeros((), dtype=f64)
    B = max(1, int(2e6 // max(1, N * shifts.shape[0])))
    for i0 in range(0, N, B):
        with torch.no_grad():
            d0 = pos_t[i0:i0 + B, None, None, :] - pos_t[None, None, :, :] + shifts[None, :, None, :]
            r2 = (d0 * d0).sum(-1)
            mask = (r2 < r_c * r_c) & (r2 > 0)
            ii, ss, jj = torch.nonzero(mask, as_tuple=True)
        if ii.numel() == 0:
            continue
        d = pos_t[i0 + ii] - pos_t[jj] + shifts[ss]
        r = torch.sqrt((d * d).sum(-1))
        g = (1.0 - moll.G_torch(p, r)) / r ** p
        E = E + 0.5 * torch.sum(q_t[i0 + ii] * q_t[jj] * g)
    return pos_t, q_t, E


def real_space(pos, q, box, p: int, c: float, r_c: float, moll: Mollifier | None = None):
    """E_real = 1/2 sum_{|r_ij + n H| < r_c}' q_i q_j (1 - G_p(r)) / r^p over
    the lattice n H (H: the cell's lattice vectors as rows; an orthorhombic
    box given as three edge lengths is diag(box)).  Positions may lie
    outside the cell.  Returns dict(E, phi [N], F [N,3])."""
    moll = moll or Mollifier(c, r_c)
    pos_t, q_t, E = _pair_energy(pos, q, box, p, r_c, moll)
    N = pos_t.shape[0]
    if not E.requires_grad:
        return dict(E=0.0, phi=np.zeros(N), F=np.zeros((N, 3)))
    gpos, gq = torch.autograd.grad(E, (pos_t, q_t), allow_unused=True)
    gpos = torch.zeros_like(pos_t) if gpos is None else gpos
    gq = torch.zeros_like(q_t) if gq is None else gq
    return dict(E=float(E.detach()), phi=gq.numpy(), F=(-gpos).numpy())


def real_space_vjp(pos, q, box, p: int, c: float, r_c: float, gE: float, gphi=None, gF=None,
                   moll: Mollifier | None = None):
    """Vector-Jacobian product of one channel's real-space outputs (E, phi =
    dE/dq, F = -dE/dr): the gradients in q and in the positions of L = gE E
    + sum_i gphi_i phi_i + sum_i gF_i . F_i, by differentiating the FP64
    autograd graph of E twice (phi and F are themselves derivatives of E).
    Returns (grad_q [N], grad_pos [N, 3])."""
    moll = moll or Mollifier(c, r_c)
    pos_t, q_t, E = _pair_energy(pos, q, box, p, r_c, moll)
    N = pos_t.shape[0]
    if not E.requires_grad:
        return np.zeros(N), np.zeros((N, 3))
    phi, gpos = torch.autograd.grad(E, (q_t, pos_t), create_graph=True)
    L = float(gE) * E
    if gphi is not None:
        L = L + torch.sum(torch.as_tensor(np.asarray(gphi, dtype=np.float64)) * phi)
    if gF is not None:
        L = L - torch.sum(torch.as_tensor(np.asarray(gF, dtype=np.float64)) * gpos)
    gq, gp = torch.autograd.grad(L, (q_t, pos_t), allow_unused=True)
    gq = torch.zeros_like(q_t) if gq is None else gq
    gp = torch.zeros_like(pos_t) if gp is None else gp
    return gq.detach().numpy(), gp.detach().numpy()


def real_space_atoms(idx, pos, q, box, p: int, c: float, r_c: float, moll: Mollifier | None = None):
    """Potentials and forces of single atoms, summed directly over their
    neighbours: phi_i = sum_{0 < |r_ij| < r_c} q_j (1 - G_p(r)) / r^p and
    F_i = q_i sum_j q_j f_p'(r) (r_j - r_i) / r, f_p = (1 - G_p) / r^p,
    with r_ij the minimum image (every box edge at least 2 r_c, so it is
    the only image closer than r_c).  f_p' by FP64 autograd of f_p in r.
    For outputs of atoms of a system too large for real_space.
    Returns (phi [len(idx)], F [len(idx), 3])."""
    moll = moll or Mollifier(c, r_c)
    box = np.asarray(box, dtype=np.float64)
    assert np.all(box >= 2.0 * r_c), "minimum image needs every edge >= 2 r_c"
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    phi = np.zeros(len(idx))
    F = np.zeros((len(idx), 3))
    for k, i in enumerate(idx):
        d = pos - pos[i]
        d -= box * np.round(d / box)
        r2 = np.einsum("nd,nd->n", d, d)
        nb = np.nonzero((r2 < r_c * r_c) & (r2 > 0.0))[0]
        r = torch.tensor(np.sqrt(r2[nb]), dtype=f64, requires_grad=True)
        f = (1.0 - moll.G_torch(p, r)) / r ** p
        (fp,) = torch.autograd.grad(f.sum(), r)
        qn = q[nb]
        phi[k] = float(np.sum(qn * f.detach().numpy()))
        F[k] = q[i] * np.sum((qn * fp.numpy() / r.detach().numpy())[:, None] * d[nb], axis=0)
    return phi, F


def pswf_total(recip: dict, pos, q, box, ps, c: float, r_c: float):
    """Assemble E = E_k + E^0 + E_real - E_self per channel from a reciprocal
    result (O1 or O2 dict with E_ch [K], phi [K,N], f [K,N,3]).
    Returns dict(E, E_ch [K], phi [K,N], F [N,3], F_ch [K,N,3])."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    moll = Mollifier(c, r_c)
    E_ch = np.array(recip["E_ch"], dtype=np.float64).copy()
    phi = np.array(recip["phi"], dtype=np.float64).copy()
    F_ch = np.einsum("kn,knd->knd", q, np.asarray(recip["f"], dtype=np.float64))
    for ci, p in enumerate(ps):
        rs = real_space(pos, q[ci], box, p, c, r_c, moll)
        sc = moll.self_coef(p)
        E_ch[ci] += rs["E"] - sc * float(np.sum(q[ci] ** 2))
        phi[ci] += rs["phi"] - 2.0 * sc * q[ci]
        F_ch[ci] += rs["F"]
    return dict(E=float(E_ch.sum()), E_ch=E_ch, phi=phi, F=F_ch.sum(0), F_ch=F_ch)
