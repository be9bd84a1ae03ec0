"""O1: the discrete PSWF-LR algorithm, plain PyTorch FP64 on the CPU.

Follows Methods, "Accelerating atom-grid spreading with PSWFs":

* window W(r) = prod_d W_pswf(r_d), W_pswf(a) = psi_0^{c_w}(a / omega) for
  |a| <= omega, omega = P h / 2;  W-hat_pswf(k) = omega lambda_0
  psi_0^{c_w}(omega k / c_w);
* Eq. (EthetaLR): insert W-hat^-2 W-hat^2 into Eq. (Fourier);
* step (i) spreading rho_grid = sum_j q_j [W(r - r_j)]_*, step (ii) forward
  FFT, step (iii) diagonal scaling by W-hat^-2 Phi-hat_p / (2V), step (iv)
  reduction over modes and channels;
* then (not printed in the paper, but implied by forces from the energy) the
  inverse transform and the gather of potentials and forces.

With rho-hat(m) = sum_g rho_g exp(-i k_m . x_g) and Delta V = V / M the grid
cell volume, Delta V rho-hat approximates sum_j q_j W-hat(k) exp(-i k . r_j),
so the energy is

    E_k = Delta V^2 / (2V) * sum_{m != 0} G(k_m) |rho-hat(m)|^2,
    G(k) = Phi-hat_p(|k|) / W-hat(k)^2,

the grid potential is Psi = (Delta V^2 / V) * IDFT[G rho-hat] (unnormalised
inverse), and for each atom phi_i = sum_g Psi_g W(x_g - r_i) and
F_i = q_i sum_g Psi_g (grad W)(x_g - r_i) = -dE/dr_i.

Stencil: with u = r / h, the P points of each dimension are
i0 .. i0 + P - 1 with i0 = ceil(u - P/2), taken modulo M (an atom on a half-integer
takes the ceiling).  The DFT sign does not matter (G is even and rho is real); m = 0 is excluded.

Cells (general, triclinic): with the lattice vectors a_d as the rows of H,
r = sum_d s_d a_d, the grid is uniform in the fractional coordinates s and
everything above is written in grid units: u_d = M_d s_d, the window per
direction is psi^{c_w}((g_d - u_d) / (P/2)), its transform per grid cell is
W-hat_d(m_d) = (P/2) lambda_0 psi^{c_w}(pi P m_d / (c_w M_d)), the modes are
k_m = 2 pi H^-1 m (the reciprocal vectors b_d = columns of H^-1), and
    E_k = 1/(2V) sum_m Phi-hat_p(|k_m|) |rho-hat(m)|^2 / prod_d W-hat_d^2,
    Psi = 1/V IDFT[...],   F_i = q_i H^-1 diag(M) sum_g Psi_g grad_u W,
with V = |det H|.  For an orthorhombic box (H = diag(L)) this is the formula
above: prod_d (h_d W-hat_d) is the Cartesian window transform and
Delta V^2 = prod h_d^2 cancels.

Nothing here is blocked, fused or reordered: atoms are spread by index_add_,
the transform is torch.fft.fftn over the full (not half) spectrum.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from .mollifiers import Mollifier, window_hat
from .pswf import PSWF

f64 = torch.float64


@dataclass
class GridConfig:
    box: tuple            # (L_x, L_y, L_z) in Angstrom (orthorhombic; ignored when cell is given)
    M: tuple              # grid points per dimension
    P: int                # stencil width
    c: float              # mollifier bandwidth
    r_c: float            # mollifier cutoff
    ps: tuple             # exponent p of each channel
    c_w: float | None = None   # window bandwidth (defaults to c)
    cell: object = None   # 3 x 3, rows = lattice vectors a_d (Angstrom); None: diag(box)


class DiscretePSWF:
    """O1 oracle for one periodic system (orthorhombic box or general cell)."""

    def __init__(self, cfg: GridConfig):
        self.cfg = cfg
        self.H = (np.diag(np.asarray(cfg.box, dtype=np.float64)) if cfg.cell is None
                  else np.asarray(cfg.cell, dtype=np.float64).reshape(3, 3))
        self.Hinv = np.linalg.inv(self.H)
        self.M = np.asarray(cfg.M, dtype=np.int64)
        self.P = int(cfg.P)
        self.V = float(abs(np.linalg.det(self.H)))
        self.dV = self.V / float(np.prod(self.M))
        self.half = self.P / 2.0            # window half-width in grid cells
        self.moll = Mollifier(cfg.c, cfg.r_c)
        c_w = cfg.c if cfg.c_w is None else cfg.c_w
        self.psi_w = self.moll.psi if c_w == cfg.c else PSWF(c_w)
        self._G = {}

    # ---- multiplier over the full spectrum --------------------------------
    def multiplier(self, p: int) -> torch.Tensor:
        """G(k_m) on the full M_x x M_y x M_z spectrum (zero at m = 0 and for
        |k| >= k_c, where Phi-hat_p vanishes: psi_0(x/c) taken as zero for x > c)."""
        if p in self._G:
            return self._G[p]
        ms = [np.fft.fftfreq(int(M), d=1.0 / int(M)) for M in self.M]   # signed mode numbers
        mx, my, mz = np.meshgrid(*ms, indexing="ij")
        B = 2.0 * math.pi * self.Hinv                 # k_m = B m
        kv = [B[d, 0] * mx + B[d, 1] * my + B[d, 2] * mz for d in range(3)]
        kk = np.sqrt(kv[0] ** 2 + kv[1] ** 2 + kv[2] ** 2)
        inside = (kk > 0) & (kk < self.moll.k_c)
        G = np.zeros(kk.shape)
        if np.any(inside):
            uniq, inv = np.unique(kk[inside], return_inverse=True)
            phi = self.moll.phi_hat(p, uniq)[inv]
            # window transform per grid cell at kappa_d = 2 pi m_d / M_d
            what = np.ones(int(np.sum(inside)))
            for d, m in enumerate((mx, my, mz)):
                what = what * window_hat(self.psi_w, self.half, 2.0 * math.pi * m[inside] / float(self.M[d]))
            G[inside] = phi / what ** 2
        self._G[p] = torch.tensor(G, dtype=f64)
        return self._G[p]

    # ---- window ---------------------------------------------------------
    def stencil(self, pos: torch.Tensor):
        """Indices [N,3,P] (mod M), weights W_d and dW_d/d(delta) [N,3,P],
        where delta = g_d - u_d in grid cells, u = M (H^-T r)."""
        Hinv = torch.tensor(self.Hinv, dtype=f64)
        u = (pos @ Hinv) * torch.tensor(self.M, dtype=f64)   # [N,3] grid coordinates
        i0 = torch.ceil(u - self.P / 2.0)                      # [N,3]
        j = torch.arange(self.P, dtype=f64)
        idx = i0.unsqueeze(-1) + j                             # [N,3,P]
        x = (idx - u.unsqueeze(-1)) / self.half
        inside = (x.abs() <= 1.0).to(f64)
        W = self.psi_w.torch(x) * inside
        dW = self.psi_w.torch(x, 1) / self.half * inside
        M = torch.tensor(self.M, dtype=torch.int64).view(1, 3, 1)
        idx = torch.remainder(idx.to(torch.int64), M)
        return idx, W, dW

    def _flat(self, idx):
        My, Mz = int(self.M[1]), int(self.M[2])
        ix, iy, iz = idx[:, 0], idx[:, 1], idx[:, 2]          # [N,P] each
        return (ix[:, :, None, None] * My + iy[:, None, :, None]) * Mz + iz[:, None, None, :]

    # ---- step (i) ---------------------------------------------------------
    def spread(self, pos: torch.Tensor, q: torch.Tensor, chunk: int = 131072) -> torch.Tensor:
        """rho[K, Mx, My, Mz] = sum_j q_j W(x_g - r_j), periodised."""
        K = q.shape[0]
        Mtot = int(np.prod(self.M))
        rho = torch.zeros(K, Mtot, dtype=f64)
        for s in range(0, pos.shape[0], chunk):
            idx, W, _ = self.stencil(pos[s:s + chunk])
            flat = self._flat(idx).reshape(-1)
            w3 = (W[:, 0, :, None, None] * W[:, 1, None, :, None] * W[:, 2, None, None, :])
            for c in range(K):
                vals = (q[c, s:s + chunk, None, None, None] * w3).reshape(-1)
                rho[c] = rho[c].index_add(0, flat, vals)
        return rho.reshape(K, *[int(m) for m in self.M])

    # ---- steps (ii)-(iv) and the inverse transform ------------------------
    def solve(self, rho: torch.Tensor):
        """Returns (E_k per channel [K], Psi [K, Mx, My, Mz])."""
        K = rho.shape[0]
        Mtot = float(np.prod(self.M))
        E = []
        Psi = []
        for c in range(K):
            G = self.multiplier(self.cfg.ps[c])
            rh = torch.fft.fftn(rho[c])
            E.append(1.0 / (2.0 * self.V) * torch.sum(G * (rh.real ** 2 + rh.imag ** 2)))
            Psi.append((1.0 / self.V) * torch.fft.ifftn(G * rh).real * Mtot)
        return torch.stack(E), torch.stack(Psi)

    # ---- gather -----------------------------------------------------------
    def gather(self, Psi: torch.Tensor, pos: torch.Tensor, chunk: int = 131072):
        """phi [K,N] = sum_g Psi_g W(x_g - r_i) and per-unit-charge force
        f [K,N,3] = -d phi / d r_i = H^-1 diag(M) sum_g Psi_g (grad_delta W)."""
        K = Psi.shape[0]
        flatPsi = Psi.reshape(K, -1)
        phis, fs = [], []
        for s in range(0, pos.shape[0], chunk):
            idx, W, dW = self.stencil(pos[s:s + chunk])
            flat = self._flat(idx)
            Wx, Wy, Wz = W[:, 0], W[:, 1], W[:, 2]
            dx, dy, dz = dW[:, 0], dW[:, 1], dW[:, 2]
            ph_c, f_c = [], []
            for c in range(K):
                g = flatPsi[c][flat]                           # [n,P,P,P]
                ph_c.append(torch.einsum("nabc,na,nb,nc->n", g, Wx, Wy, Wz))
                f_c.append(torch.stack([torch.einsum("nabc,na,nb,nc->n", g, dx, Wy, Wz),
                                        torch.einsum("nabc,na,nb,nc->n", g, Wx, dy, Wz),
                                        torch.einsum("nabc,na,nb,nc->n", g, Wx, Wy, dz)], -1))
            phis.append(torch.stack(ph_c))
            # grid-cell derivatives -> Cartesian: f = H^-1 (M * f_u), as rows
            J = torch.tensor(self.Hinv * self.M[None, :].astype(np.float64), dtype=f64)   # H^-1 diag(M)
            fs.append(torch.stack(f_c) @ J.T)
        if not phis:
            return torch.zeros(K, 0, dtype=f64), torch.zeros(K, 0, 3, dtype=f64)
        return torch.cat(phis, 1), torch.cat(fs, 1)

    # ---- the whole forward evaluation ---------------------------------------
    def _forward(self, pos: torch.Tensor, q: torch.Tensor):
        rho = self.spread(pos, q)
        E_k, Psi = self.solve(rho)
        phi, f = self.gather(Psi, pos)
        Qnet = q.sum(dim=1)
        a = torch.tensor([self.moll.zero_freq_coef(p, self.V) for p in self.cfg.ps], dtype=f64)
        E0 = a * Qnet ** 2
        phi = phi + (2.0 * a * Qnet).unsqueeze(1)
        F = torch.einsum("kn,knd->nd", q, f)
        return E_k, E0, phi, F, f, Psi

    def evaluate(self, pos, q):
        """pos [N,3], q [K,N] (array-like or tensors).  Returns a dict with
        E (total), E_ch [K] (E_k + E^0 per channel), E_k [K], E0 [K],
        phi [K,N] (including d E^0 / d q_i), F [N,3], f [K,N,3], Psi."""
        pos = torch.as_tensor(pos, dtype=f64)
        q = torch.as_tensor(q, dtype=f64)
        E_k, E0, phi, F, f, Psi = self._forward(pos, q)
        return dict(E=float((E_k + E0).sum().detach()), E_ch=(E_k + E0).detach(), E_k=E_k.detach(), E0=E0.detach(),
                    phi=phi.detach(), F=F.detach(), f=f.detach(), Psi=Psi.detach(), E_tensor=(E_k + E0).sum())

    def vjp(self, pos, q, g_E=None, g_phi=None, g_F=None):
        """Vector-Jacobian product of evaluate's (E_ch, phi, F): for
        L = sum_c g_E[c] E_c + sum g_phi * phi + sum g_F * F returns
        (dL/dq [K,N], dL/dr [N,3]), by reverse-mode differentiation (torch
        autograd, a library primitive) of exactly the steps of evaluate.
        F = -dE/dr makes the g_F term a second derivative of E: W is
        differentiated twice through psi_w.torch."""
        pos = torch.as_tensor(pos, dtype=f64).clone().requires_grad_(True)
        q = torch.as_tensor(q, dtype=f64).clone().requires_grad_(True)
        E_k, E0, phi, F, _, _ = self._forward(pos, q)
        L = torch.zeros((), dtype=f64)
        if g_E is not None:
            L = L + (torch.as_tensor(g_E, dtype=f64) * (E_k + E0)).sum()
        if g_phi is not None:
            L = L + (torch.as_tensor(g_phi, dtype=f64) * phi).sum()
        if g_F is not None:
            L = L + (torch.as_tensor(g_F, dtype=f64) * F).sum()
        if not L.requires_grad:
            return torch.zeros_like(q).detach(), torch.zeros_like(pos).detach()
        gq, gr = torch.autograd.grad(L, [q, pos], allow_unused=True)
        gq = torch.zeros_like(q) if gq is None else gq
        gr = torch.zeros_like(pos) if gr is None else gr
        return gq.detach(), gr.detach()

    def virial_fd(self, pos, q, eps: float = 5e-5) -> np.ndarray:
        """Diagonal virial W[c, d] = -L_d dE_c/dL_d at fixed fractional
        coordinates, by central differences of evaluate (E_c = E_k + E^0)
        under the scaling L_d -> L_d (1 +- h) of the box and the positions,
        at the same grid size, P, c and c_w; Richardson-extrapolated from
        h = eps and 2 eps (truncation O(eps^4), rounding ~1e-12 / eps)."""
        pos = np.asarray(pos, dtype=np.float64)
        if self.cfg.cell is not None and np.any(self.H != np.diag(np.diag(self.H))):
            raise NotImplementedError("the diagonal virial is defined for orthorhombic boxes")
        K = len(self.cfg.ps)
        c_w = self.cfg.c if self.cfg.c_w is None else self.cfg.c_w

        def central(h):
            W = np.zeros((K, 3))
            for d in range(3):
                Es = []
                for sgn in (1.0, -1.0):
                    f = 1.0 + sgn * h
                    box = list(self.cfg.box)
                    box[d] *= f
                    p2 = pos.copy()
                    p2[:, d] *= f
                    cfg = GridConfig(tuple(box), self.cfg.M, self.cfg.P, self.cfg.c, self.cfg.r_c, self.cfg.ps,
                                     c_w=c_w)
                    Es.append(DiscretePSWF(cfg).evaluate(p2, q)["E_ch"].numpy())
                W[:, d] = -(Es[0] - Es[1]) / (2.0 * h)
            return W

        return (4.0 * central(eps) - central(2.0 * eps)) / 3.0

    def stress_fd(self, pos, q, eps: float = 5e-5) -> np.ndarray:
        """Virial tensor W[c] (3 x 3, symmetric) of any cell: W_ab = -dE_c /
        d epsilon_ab under the homogeneous symmetric strain r -> (1 +
        epsilon) r of the cell vectors and the positions together (fixed
        fractional coordinates), same grid size, P, c and c_w.  Central
        differences: epsilon_aa = +-h, or epsilon_ab = epsilon_ba = +-h/2
        for a != b (so dE = -W_ab h); Richardson-extrapolated from h = eps
        and 2 eps.  For a box the diagonal is virial_fd."""
        pos = np.asarray(pos, dtype=np.float64)
        K = len(self.cfg.ps)
        c_w = self.cfg.c if self.cfg.c_w is None else self.cfg.c_w

        def energy(F):
            cfg = GridConfig(self.cfg.box, self.cfg.M, self.cfg.P, self.cfg.c, self.cfg.r_c, self.cfg.ps,
                             c_w=c_w, cell=self.H @ F.T)
            return DiscretePSWF(cfg).evaluate(pos @ F.T, q)["E_ch"].numpy()

        def central(h):
            W = np.zeros((K, 3, 3))
            for a in range(3):
                for b in range(a, 3):
                    Es = []
                    for sgn in (1.0, -1.0):
                        e = np.zeros((3, 3))
                        if a == b:
                            e[a, a] = sgn * h
                        else:
                            e[a, b] = e[b, a] = sgn * h / 2.0
                        Es.append(energy(np.eye(3) + e))
                    W[:, a, b] = W[:, b, a] = -(Es[0] - Es[1]) / (2.0 * h)
            return W

        return (4.0 * central(eps) - central(2.0 * eps)) / 3.0

    def self_energy(self, q) -> np.ndarray:
        """E_self^(p) per channel (Implementation details)."""
        q = np.asarray(q, dtype=np.float64)
        return np.array([self.moll.self_coef(p) * float(np.sum(q[c] ** 2))
                         for c, p in enumerate(self.cfg.ps)])

    # ---- naive DFT (tiny grids only) ---------------------------------------
    def naive_dft(self, rho: torch.Tensor) -> torch.Tensor:
        """rho-hat(m) = sum_g rho_g exp(-2 pi i m.g / M), written out as an
        explicit O(M^2) sum over grid points (cross-check of fftn usage)."""
        Mx, My, Mz = [int(m) for m in self.M]
        g = [torch.arange(m, dtype=f64) for m in (Mx, My, Mz)]
        ex = torch.exp(-2j * math.pi * torch.outer(g[0], g[0]) / Mx)
        ey = torch.exp(-2j * math.pi * torch.outer(g[1], g[1]) / My)
        ez = torch.exp(-2j * math.pi * torch.outer(g[2], g[2]) / Mz)
        out = torch.zeros(Mx, My, Mz, dtype=torch.complex128)
        r = rho.to(torch.complex128)
        for a in range(Mx):
            for b in range(My):
                for cc in range(Mz):
                    phase = ex[a][:, None, None] * ey[b][None, :, None] * ez[cc][None, None, :]
                    out[a, b, cc] = torch.sum(r * phase)
        return out
