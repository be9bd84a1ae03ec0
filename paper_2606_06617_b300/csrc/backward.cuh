// Backward (vector-Jacobian product) of the forward evaluation.
//
// With W_i(g) = W(x_g - r_i), its gradient D_i(g) = (grad W)(x_g - r_i) (with
// respect to a = x_g - r) and Hessian H_i(g), the forward is
//   phi_i^c = sum_g Psi^c_g W_i(g) + 2 a_c Q_c,   f_i^c = sum_g Psi^c_g D_i(g),
//   F_i = sum_c q_i^c f_i^c,   E_c = E_k^c + a_c Q_c^2,
// Psi^c = A_c rho^c, rho^c = sum_i q_i^c W_i (A_c symmetric: FFT, G_c, IFFT).
// For L = sum_c gE_c E_c + sum gphi . phi + sum gF . F:
//   rhobar^c = sum_i [gphi_i^c W_i + q_i^c gF_i . D_i],  Psibar^c = A_c rhobar^c,
//   dL/dq_i^c = gE_c phi_i^c + 2 a_c sum_j gphi_j^c + gF_i . f_i^c
//               + sum_g Psibar^c_g W_i(g),
//   dL/dr_i   = sum_c [ -(gE_c q_i^c + gphi_i^c) f_i^c
//                       - q_i^c sum_g Psibar^c_g D_i(g)
//                       - q_i^c (sum_g Psi^c_g H_i(g)) gF_i ].
// (Per structure s of a batch plan, with E_c, Q_c, a_c of channel g = s K + c.)
// Kernels here are one thread per (channel, sorted atom), reading and writing
// the grids directly (global atomics for the spread and for dL/dr).
#pragma once

#include "stencil.cuh"

namespace pswf {

// Window values, first and second s-derivatives (Horner).
template <typename R, int P>
__device__ inline void window_weights2(R t, const WinCoef<R>& wc, R (&w)[P], R (&dw)[P], R (&d2w)[P]) {
  constexpr int D = WinCoef<R>::kDeg;
  const R s = R(2) * t - R(1);
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const R* c = wc.c + j * (D + 1);
    R v = c[D], dv = R(0), d2v = R(0);
#pragma unroll
    for (int n = D - 1; n >= 0; --n) {
      d2v = d2v * s + R(2) * dv;
      dv = dv * s + v;
      v = v * s + c[n];
    }
    w[j] = v;
    dw[j] = dv;
    d2w[j] = d2v;
  }
}

// rhobar^c(g) = sum_i gphi_i^c W_i(g) + q_i^c gF_i . D_i(g)  (grid2 zeroed
// before).  One thread per (channel, sorted atom), channel-major.
template <typename R, int P>
__global__ void k_spread_bw(int64_t nmax, Geometry g, const double* __restrict__ smol, const int* __restrict__ soff,
                            const int* __restrict__ tile_start, const R* __restrict__ st,
                            const uint64_t* __restrict__ scell, const R* __restrict__ sq,
                            const int* __restrict__ sperm, WinCoef<R> wc, const R* __restrict__ gphi,
                            const R* __restrict__ gF, R* __restrict__ grid2) {
  const int64_t n = soff[g.B];
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n * g.K; t += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(t / n);
    const int64_t a = t - int64_t(c) * n;
    const int sidx = find_struct(tile_start, g.nts, g.B, a);
    const double* mol = smol + 3 * sidx;
    const R two_h[3] = {R(2.0 * mol[0]), R(2.0 * mol[1]), R(2.0 * mol[2])};
    R wx[P], wy[P], wz[P], dx[P], dy[P], dz[P];
    window_weights<R, P>(st[a], wc, wx, dx);
    window_weights<R, P>(st[nmax + a], wc, wy, dy);
    window_weights<R, P>(st[2 * nmax + a], wc, wz, dz);
#pragma unroll
    for (int i = 0; i < P; ++i) {
      dx[i] *= two_h[0];
      dy[i] *= two_h[1];
      dz[i] *= two_h[2];
    }
    int cx, cy, cz;
    unpack_cell(scell[a], cx, cy, cz);
    const int o = sperm[a];
    const R g0 = gF ? gF[3 * int64_t(o)] : R(0), g1 = gF ? gF[3 * int64_t(o) + 1] : R(0),
            g2 = gF ? gF[3 * int64_t(o) + 2] : R(0);
    const R qc = sq[int64_t(c) * nmax + a];
    const R gp = gphi ? gphi[int64_t(c) * n + o] : R(0);
    const R v0 = qc * g0, v1 = qc * g1, v2 = qc * g2;
    R* gc = grid2 + (int64_t(sidx) * g.K + c) * g.M[2] * g.M[1] * g.Mxp;
    int ix[P];
#pragma unroll
    for (int i = 0; i < P; ++i) ix[i] = wrap_index(cx + i, g.M[0]);
    for (int k = 0; k < P; ++k) {
      const int z = wrap_index(cz + k, g.M[2]);
      for (int j = 0; j < P; ++j) {
        const int y = wrap_index(cy + j, g.M[1]);
        // value(i) = wx[i] * A + dx[i] * B with the (j, k) factors folded in
        const R A = gp * wy[j] * wz[k] + v1 * dy[j] * wz[k] + v2 * wy[j] * dz[k];
        const R B = v0 * wy[j] * wz[k];
        R* row = gc + (int64_t(z) * g.M[1] + y) * g.Mxp;
#pragma unroll
        for (int i = 0; i < P; ++i) atomicAdd(row + ix[i], wx[i] * A + dx[i] * B);
      }
    }
  }
}

// Gather of the backward, one thread per (channel, sorted atom): phi
// (recomputed), f and the Hessian contraction from Psi (grid), W and D
// contractions from Psibar (grid2); writes dL/dq and adds the channel's part
// of dL/dr (grad_r zeroed before) in the original atom order.
template <typename R, int P>
__global__ void k_interp_bw(int64_t nmax, Geometry g, const double* __restrict__ smol, const int* __restrict__ soff,
                            const int* __restrict__ tile_start, const R* __restrict__ st,
                            const uint64_t* __restrict__ scell, const R* __restrict__ sq,
                            const int* __restrict__ sperm, WinCoef<R> wc, const R* __restrict__ grid,
                            const R* __restrict__ grid2, const double* __restrict__ zero_coef,
                            const double* __restrict__ charges, const double* __restrict__ gsum,
                            const double* __restrict__ gE, const R* __restrict__ gphi, const R* __restrict__ gF,
                            R* __restrict__ grad_q, R* __restrict__ grad_r) {
  const int64_t n = soff[g.B];
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n * g.K; t += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(t / n);
    const int64_t a = t - int64_t(c) * n;
    const int sidx = find_struct(tile_start, g.nts, g.B, a);
    const double* mol = smol + 3 * sidx;
    const R th[3] = {R(2.0 * mol[0]), R(2.0 * mol[1]), R(2.0 * mol[2])};
    R wx[P], wy[P], wz[P], dx[P], dy[P], dz[P], hx[P], hy[P], hz[P];
    window_weights2<R, P>(st[a], wc, wx, dx, hx);
    window_weights2<R, P>(st[nmax + a], wc, wy, dy, hy);
    window_weights2<R, P>(st[2 * nmax + a], wc, wz, dz, hz);
#pragma unroll
    for (int i = 0; i < P; ++i) {
      dx[i] *= th[0];
      dy[i] *= th[1];
      dz[i] *= th[2];
      hx[i] *= th[0] * th[0];
      hy[i] *= th[1] * th[1];
      hz[i] *= th[2] * th[2];
    }
    int cx, cy, cz;
    unpack_cell(scell[a], cx, cy, cz);
    const int o = sperm[a];
    const R g0 = gF ? gF[3 * int64_t(o)] : R(0), g1 = gF ? gF[3 * int64_t(o) + 1] : R(0),
            g2 = gF ? gF[3 * int64_t(o) + 2] : R(0);
    int ix[P];
#pragma unroll
    for (int i = 0; i < P; ++i) ix[i] = wrap_index(cx + i, g.M[0]);
    const int gi = sidx * g.K + c;
    const R* pc = grid + int64_t(gi) * g.M[2] * g.M[1] * g.Mxp;
    const R* bc = grid2 + int64_t(gi) * g.M[2] * g.M[1] * g.Mxp;
    R ph = 0, f0 = 0, f1 = 0, f2 = 0, sb = 0, b0 = 0, b1 = 0, b2 = 0;
    R h00 = 0, h11 = 0, h22 = 0, h01 = 0, h02 = 0, h12 = 0;
    for (int k = 0; k < P; ++k) {
      const int z = wrap_index(cz + k, g.M[2]);
      for (int j = 0; j < P; ++j) {
        const int y = wrap_index(cy + j, g.M[1]);
        const R* prow = pc + (int64_t(z) * g.M[1] + y) * g.Mxp;
        const R* brow = bc + (int64_t(z) * g.M[1] + y) * g.Mxp;
        R s_w = 0, s_d = 0, s_h = 0, t_w = 0, t_d = 0;
#pragma unroll
        for (int i = 0; i < P; ++i) {
          const R v = prow[ix[i]], u = brow[ix[i]];
          s_w += v * wx[i];
          s_d += v * dx[i];
          s_h += v * hx[i];
          t_w += u * wx[i];
          t_d += u * dx[i];
        }
        const R yz = wy[j] * wz[k];
        ph += s_w * yz;
        f0 += s_d * yz;
        f1 += s_w * dy[j] * wz[k];
        f2 += s_w * wy[j] * dz[k];
        h00 += s_h * yz;
        h11 += s_w * hy[j] * wz[k];
        h22 += s_w * wy[j] * hz[k];
        h01 += s_d * dy[j] * wz[k];
        h02 += s_d * wy[j] * dz[k];
        h12 += s_w * dy[j] * dz[k];
        sb += t_w * yz;
        b0 += t_d * yz;
        b1 += t_w * dy[j] * wz[k];
        b2 += t_w * wy[j] * dz[k];
      }
    }
    const R qc = sq[int64_t(c) * nmax + a];
    const R ge = gE ? R(gE[gi]) : R(0);
    const R gp = gphi ? gphi[int64_t(c) * n + o] : R(0);
    const R phi_c = ph + R(2.0 * zero_coef[gi] * charges[2 * gi]);
    if (grad_q)
      grad_q[int64_t(c) * n + o] = ge * phi_c + R(2.0 * zero_coef[gi] * gsum[2 * gi]) + g0 * f0 + g1 * f1 + g2 * f2 + sb;
    if (grad_r) {
      const R w = ge * qc + gp;
      atomicAdd(grad_r + 3 * int64_t(o), -(w * f0 + qc * b0 + qc * (h00 * g0 + h01 * g1 + h02 * g2)));
      atomicAdd(grad_r + 3 * int64_t(o) + 1, -(w * f1 + qc * b1 + qc * (h01 * g0 + h11 * g1 + h12 * g2)));
      atomicAdd(grad_r + 3 * int64_t(o) + 2, -(w * f2 + qc * b2 + qc * (h02 * g0 + h12 * g1 + h22 * g2)));
    }
  }
}

}  // namespace pswf
