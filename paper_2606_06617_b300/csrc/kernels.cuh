// Device kernels of the PSWF-LR hot path (sm_103a).
//
// A plan holds B structures (B = 1 for a single system) that share one grid
// size M and K channels; structure s has its own box (tables smol[s][3] =
// M_d / L_d, bmat[s][9] = 2 pi H^-1 with the lattice vectors as the rows of
// H, diagonal for a box, and for a general cell tmat[s][9] = diag(M) H^-T)
// and its atoms are soff[s] .. soff[s+1] - 1 of the caller's arrays.
// Data layout in HBM (one plan):
//   grid   real [B][K][M_z][M_y][M_xp], M_xp = 2 (M_x / 2 + 1): the spread
//          density, overwritten in place by the R2C transform, the multiplier
//          and the C2R transform (the grid potential Psi);
//   sorted atoms (structure, then tile order): st[3][n] real window offsets
//          t_d in [0, 1), scell[n] packed stencil-start cell, sq[K][n] real
//          charges, sperm[n] original index;
//   tile_start[B * nts + 1] int32 offsets of each tile's atoms.
// Tiles are kTile^3 blocks of stencil-start cells, nts per structure.
// Per-(structure, channel) values are indexed g = s * K + c.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bounds.cuh"
#include "planner.hpp"

namespace pswf {

constexpr int kTile = 16;     // tile edge in stencil-start cells

struct Geometry {
  int M[3];          // grid points per dimension
  int Mxp;           // padded row length (real elements)
  int P;             // stencil width
  int ntile[3];      // tiles per dimension (of one structure)
  int nts;           // tiles per structure
  int tric;          // 1: general cell (locate through T = diag(M) H^-T), 0: box
  int K;             // channels
  int B;             // structures
};

// Window pieces as monomials in s = 2t - 1, each padded with zero leading
// coefficients to a fixed degree (14 in FP32, 24 in FP64) so that Horner
// loops unroll and read the coefficients as constant operands.
template <typename R>
struct WinCoef {
  static constexpr int kDeg = sizeof(R) == 4 ? 12 : 24;
  int deg;                          // the planner's degree (<= kDeg)
  R c[kMaxP * (kDeg + 1)];          // piece j, monomial n at [j * (kDeg + 1) + n]
};

struct MultParams {
  double inv_kc;      // 1 / k_c
  int M[3];
  int Mxh;            // M_x / 2 + 1
  int deg;            // multiplier polynomial degree
  int K;
};

template <typename R>
struct Cplx {
  R x, y;
};

__host__ __device__ inline uint64_t pack_cell(int x, int y, int z) {
  return uint64_t(uint32_t(x)) | (uint64_t(uint32_t(y)) << 21) | (uint64_t(uint32_t(z)) << 42);
}
__host__ __device__ inline void unpack_cell(uint64_t c, int& x, int& y, int& z) {
  x = int(c & 0x1FFFFF);
  y = int((c >> 21) & 0x1FFFFF);
  z = int((c >> 42) & 0x1FFFFF);
}

// Stencil start: u = x M / L, i0 = ceil(u - P/2), t = i0 + P/2
// - u in [0, 1]; i0 wrapped into [0, M).  With u = fl + f (fl = floor(u),
// f in [0, 1)): for even P, i0 = fl - P/2 + [f > 0] and t = [f > 0] - f; for
// odd P = 2k + 1, i0 = fl - k + [f > 1/2] and t = [f > 1/2] + 1/2 - f.  The
// FP64 work is one multiply, one floor and one subtraction per direction.
// (t = 1 only when 1 - f rounds up, f tiny: the stencil and t then still
// describe u.)
__device__ inline void locate_u(double u, int M, int P, int& i0w, double& t) {
  const double fl = floor(u);
  const double f = u - fl;
  int64_t i0;
  if ((P & 1) == 0) {
    const int c = f > 0.0 ? 1 : 0;
    i0 = int64_t(fl) - P / 2 + c;
    t = double(c) - f;
  } else {
    const int c = f > 0.5 ? 1 : 0;
    i0 = int64_t(fl) - P / 2 + c;
    t = double(c) + 0.5 - f;
  }
  if (t < 0.0) t = 0.0;
  if (t > 1.0) t = 1.0;
  int64_t r = i0 % M;
  if (r < 0) r += M;
  i0w = int(r);
}

// The same for the FP32 path with a single FP64 instruction (the multiply;
// the FP64 pipe is narrow on this GPU): u is read from its bits as 32.32
// fixed point F = floor(u 2^32) plus a sticky flag for nonzero bits below
// 2^-32, so that fl = F >> 32 and the decisions f > 0, f > 1/2 are exactly
// those of the FP64 rule; t is one integer difference modulo 2^32 converted
// once: 2^32 [f > 0] - f 2^32 (even P), 2^31 + 2^32 [f > 1/2] - f 2^32 (odd
// P), with the bits below 2^-32 dropped (t = 1 where that difference wraps
// to 0).  |u| >= 2^30 takes the FP64 route.
__device__ inline void locate_fx_u(double u, int M, int P, int& i0w, float& t) {
  const long long bits = __double_as_longlong(u);
  const int bexp = int((bits >> 52) & 0x7FF);
  const int ex = bexp - 1075;   // |u| = m 2^ex
  if (ex > -23) {
    double td;
    locate_u(u, M, P, i0w, td);
    t = float(td);
    return;
  }
  const long long m = bexp == 0 ? 0LL : ((bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL);
  const int sh = ex + 32;
  long long F;
  bool sticky;
  if (sh >= 0) {
    F = m << sh;
    sticky = false;
  } else if (sh > -64) {
    F = m >> -sh;
    sticky = (m & ((1LL << -sh) - 1)) != 0;
  } else {
    F = 0;
    sticky = m != 0;
  }
  if (bits < 0) F = -F - (sticky ? 1 : 0);
  const int fl = int(F >> 32);
  const unsigned fq = unsigned(F & 0xFFFFFFFFLL);
  int c;
  unsigned d;
  if ((P & 1) == 0) {
    c = (fq != 0u || sticky) ? 1 : 0;
    d = 0u - fq;
  } else {
    c = (fq > 0x80000000u || (fq == 0x80000000u && sticky)) ? 1 : 0;
    d = 0x80000000u - fq;
  }
  t = (d == 0u && c) ? 1.0f : __uint2float_rn(d) * 2.3283064365386963e-10f;   // 2^-32
  int r = (fl - P / 2 + c) % M;
  if (r < 0) r += M;
  i0w = r;
}

// Structure of an atom: the s with off[s] <= i < off[s + 1] (off has B + 1
// non-decreasing entries read with the given stride).
__device__ inline int find_struct(const int* __restrict__ off, int stride, int B, int64_t i) {
  int lo = 0, hi = B;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (int64_t(off[int64_t(mid) * stride]) <= i)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Window weights W_j(t) and dW_j/ds (s = 2t - 1) for the P pieces (Horner).
template <typename R, int P>
__device__ inline void window_weights(R t, const WinCoef<R>& wc, R (&w)[P], R (&dw)[P]) {
  constexpr int D = WinCoef<R>::kDeg;
  const R s = R(2) * t - R(1);
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const R* c = wc.c + j * (D + 1);
    R v = c[D], dv = R(0);
#pragma unroll
    for (int n = D - 1; n >= 0; --n) {
      dv = dv * s + v;
      v = v * s + c[n];
    }
    w[j] = v;
    dw[j] = dv;
  }
}

template <typename R, int P>
__device__ inline void window_values(R t, const WinCoef<R>& wc, R (&w)[P]) {
  constexpr int D = WinCoef<R>::kDeg;
  const R s = R(2) * t - R(1);
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const R* c = wc.c + j * (D + 1);
    R v = c[D];
#pragma unroll
    for (int n = D - 1; n >= 0; --n) v = v * s + c[n];
    w[j] = v;
  }
}

// ---- binning -----------------------------------------------------------------
// k_bin: locate each atom (original order), count it into its tile and keep
// its rank there, its offsets t and its packed start cell for k_scatter.
// smol[s][d] = M_d / L_d of structure s.
// Stencil start and offset of one coordinate u, stored as R.
template <typename R>
__device__ inline void locate_one(double u, int M, int P, int& i0, R* t_out) {
  if constexpr (sizeof(R) == 4) {
    float t;
    locate_fx_u(u, M, P, i0, t);
    *t_out = t;
  } else {
    double t;
    locate_u(u, M, P, i0, t);
    *t_out = R(t);
  }
}

// tmat[s][9] = T = diag(M) H^-T of structure s (general cells, g.tric):
// u = T r; boxes use u_d = r_d M_d / L_d (smol).
template <typename PosT, typename R>
__global__ void k_bin(const PosT* __restrict__ pos, Geometry g, const double* __restrict__ smol,
                      const double* __restrict__ tmat, const int* __restrict__ soff, int* __restrict__ tile_of,
                      int* __restrict__ rank, int* __restrict__ tile_count, R* __restrict__ tmp_t,
                      uint64_t* __restrict__ tmp_cell, int64_t nmax, int* __restrict__ err) {
  const int64_t n = soff[g.B];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int s = find_struct(soff, 1, g.B, i);
    int i0[3];
    if (!g.tric) {
      // box: u_d = r_d M_d / L_d
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double x = double(pos[3 * i + d]);
        if (((__double_as_longlong(x) >> 52) & 0x7FF) == 0x7FF) {   // inf or nan
          atomicCAS(err, 0, -6);
          x = 0.0;
        }
        locate_one<R>(x * smol[3 * s + d], g.M[d], g.P, i0[d], tmp_t + d * nmax + i);
      }
    } else {
      // general cell: u = T r
      double x[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        x[d] = double(pos[3 * i + d]);
        if (((__double_as_longlong(x[d]) >> 52) & 0x7FF) == 0x7FF) {
          atomicCAS(err, 0, -6);
          x[d] = 0.0;
        }
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double* T = tmat + 9 * s + 3 * d;
        locate_one<R>(fma(T[0], x[0], fma(T[1], x[1], T[2] * x[2])), g.M[d], g.P, i0[d], tmp_t + d * nmax + i);
      }
    }
    const int tile = s * g.nts + ((i0[2] / kTile) * g.ntile[1] + i0[1] / kTile) * g.ntile[0] + i0[0] / kTile;
    tile_of[i] = tile;
    tmp_cell[i] = pack_cell(i0[0], i0[1], i0[2]);
    rank[i] = atomicAdd(tile_count + tile, 1);
  }
}

template <typename R>
__global__ void k_scatter(int64_t nmax, const R* __restrict__ q, Geometry g, const int* __restrict__ soff,
                          const int* __restrict__ tile_of, const int* __restrict__ rank,
                          const int* __restrict__ tile_start, const R* __restrict__ tmp_t,
                          const uint64_t* __restrict__ tmp_cell, R* __restrict__ st, uint64_t* __restrict__ scell,
                          R* __restrict__ sq, int* __restrict__ sperm) {
  const int64_t n = soff[g.B];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t dst = int64_t(tile_start[tile_of[i]]) + rank[i];
    if (!in_bounds(dst, nmax, kBoundsScatter)) continue;
    st[dst] = tmp_t[i];
    st[nmax + dst] = tmp_t[nmax + i];
    st[2 * nmax + dst] = tmp_t[2 * nmax + i];
    scell[dst] = tmp_cell[i];
    for (int c = 0; c < g.K; ++c) sq[c * nmax + dst] = q[c * n + i];
    sperm[dst] = int(i);
  }
}

// Fixed-point unit of the FP32 four-channel spread per (tile, channel): with
// S1 = sum |q| and Mq = max |q| over the tile's atoms, s = min(0.99 2^22 /
// Mq, 0.999 2^31 / (1.0001 S1)) keeps each rounded contribution below 2^22
// and every grid sum of the tile below 2^31 (the window is at most 1; the
// 1.0001 and 0.999 factors cover the rounding of the float sum, whose
// relative error is below (n / 32 + 5) 2^-24 for n atoms); 1 for a channel
// of zeros.  One warp per tile, lanes strided over its atoms.
__global__ void k_tile_scale(int ntl, int K, int64_t nmax, const int* __restrict__ tile_start,
                             const float* __restrict__ sq, float* __restrict__ tscale);

// The single-structure set_points writes its atom count here (soff = {0, n}).
__global__ void k_set_count(int* __restrict__ soff, int n);

// Per-thread sums of q and q^2.  FP32 charges: double-float sums (a float
// sum and its running rounding error by TwoSum; q^2 split exactly into
// v*v and fma(v, v, -v*v)), merged across a warp in the same form and
// converted to FP64 once per warp, so the FP64 pipe (narrow on this GPU)
// only sees the sums across warps.  FP64 charges: FP64 sums.
template <typename R>
struct ChargeAcc {
  double a = 0.0, b = 0.0;
  __device__ void add(R v) {
    const double d = double(v);
    a += d;
    b += d * d;
  }
  __device__ void merge(const ChargeAcc& o) {
    a += o.a;
    b += o.b;
  }
  __device__ void warp_reduce() {
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
  }
  __device__ double sum() const { return a; }
  __device__ double sumsq() const { return b; }
};
template <>
struct ChargeAcc<float> {
  float a = 0.f, ae = 0.f, b = 0.f, be = 0.f;
  __device__ static void two_sum(float& s, float& e, float x) {
    const float t = s + x;
    const float bp = t - s;
    e += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ void add(float v) {
    const float p = v * v;
    be += fmaf(v, v, -p);
    two_sum(a, ae, v);
    two_sum(b, be, p);
  }
  __device__ void merge(const ChargeAcc& o) {
    two_sum(a, ae, o.a);
    ae += o.ae;
    two_sum(b, be, o.b);
    be += o.be;
  }
  // lane 0 ends with the warp's sums
  __device__ void warp_reduce() {
    for (int o = 16; o > 0; o >>= 1) {
      ChargeAcc t;
      t.a = __shfl_down_sync(0xffffffffu, a, o);
      t.ae = __shfl_down_sync(0xffffffffu, ae, o);
      t.b = __shfl_down_sync(0xffffffffu, b, o);
      t.be = __shfl_down_sync(0xffffffffu, be, o);
      merge(t);
    }
  }
  __device__ double sum() const { return double(a) + double(ae); }
  __device__ double sumsq() const { return double(b) + double(be); }
};

// Block sums of the threads' accumulators, written by thread 0: merged
// within each warp in the accumulator's form, then across warps in FP64.
template <typename R>
__device__ inline void charge_block_sums(ChargeAcc<R> acc, double* __restrict__ out) {
  __shared__ double sh[2][32];
  acc.warp_reduce();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = acc.sum();
    sh[1][wid] = acc.sumsq();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      x += sh[0][w];
      y += sh[1][w];
    }
    out[0] = x;
    out[1] = y;
  }
  __syncthreads();
}

// Per-(structure, block) partial sums of q and q^2 per channel over the
// structure's atoms (caller order, q [K][n]): blockIdx.y = structure,
// part[((s * gridDim.x + blk) * K + c) * 2 + {0, 1}].
template <typename R>
__global__ void k_charge_partials_seg(const R* __restrict__ q, int K, int B, const int* __restrict__ soff,
                                      double* __restrict__ part) {
  const int s = blockIdx.y;
  const int64_t n = soff[B], a0 = soff[s], a1 = soff[s + 1];
  const int64_t step = int64_t(gridDim.x) * blockDim.x;
  for (int c = 0; c < K; ++c) {
    // four loads in flight per thread, two interleaved accumulators
    ChargeAcc<R> acc0, acc1;
    const R* qc = q + c * n;
    int64_t i = a0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    for (; i + 3 * step < a1; i += 4 * step) {
      const R v0 = qc[i], v1 = qc[i + step], v2 = qc[i + 2 * step], v3 = qc[i + 3 * step];
      acc0.add(v0);
      acc1.add(v1);
      acc0.add(v2);
      acc1.add(v3);
    }
    for (; i < a1; i += step) acc0.add(qc[i]);
    acc0.merge(acc1);
    charge_block_sums(acc0, part + ((size_t(s) * gridDim.x + blockIdx.x) * K + c) * 2);
  }
}

// Q_net and Q_self of one (structure, channel) per warp, g = s K + c:
// charges[2 g] = sum q, charges[2 g + 1] = sum q^2 over the structure's atoms
// (caller order, q [K][n]).  For batch plans, whose structures are small.
template <typename R>
__global__ void k_charge_sums_warp(const R* __restrict__ q, int K, int B, const int* __restrict__ soff,
                                   double* __restrict__ charges) {
  const int g = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= B * K) return;
  const int s = g / K, c = g - s * K;
  const int64_t n = soff[B], a0 = soff[s], a1 = soff[s + 1];
  ChargeAcc<R> acc;
  for (int64_t i = a0 + lane; i < a1; i += 32) acc.add(q[c * n + i]);
  acc.warp_reduce();
  if (lane == 0) {
    charges[2 * g] = acc.sum();
    charges[2 * g + 1] = acc.sumsq();
  }
}

// Per-block partial sums of q and q^2 per channel: part[(blk * K + c) * 2 + {0,1}].
template <typename R>
__global__ void k_charge_partials(int64_t n, const R* __restrict__ q, int K, double* __restrict__ part) {
  for (int c = 0; c < K; ++c) {
    ChargeAcc<R> acc;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
      acc.add(q[c * n + i]);
    charge_block_sums(acc, part + (size_t(blockIdx.x) * K + c) * 2);
  }
}

// charges[c*2+0] = Q_net, charges[c*2+1] = Q_self; one thread per channel.
__global__ void k_charge_final(int nblk, int K, const double* __restrict__ part, double* __restrict__ charges);

// ---- exclusive scan of tile counts (three passes) -------------------------------
constexpr int kScanBlock = 1024;
__global__ void k_scan_block_sums(int n, const int* __restrict__ in, int* __restrict__ sums, int per_block);
__global__ void k_scan_sums(int nb, int* __restrict__ sums);
__global__ void k_scan_apply(int n, const int* __restrict__ in, const int* __restrict__ sums, int per_block,
                             int* __restrict__ out);
// k_charge_final_seg: charges[g][0] = Q_net, charges[g][1] = Q_self from the
// k_charge_partials_seg partials, one block per (structure, channel).
__global__ void k_charge_final_seg(int nblk, int K, int B, const double* __restrict__ part,
                                   double* __restrict__ charges);
// One block per structure: energy[s][c] = sum of the multiplier partials of
// channel g = s K + c plus zero_coef[g] Q_net^2; energy[s][K] = their total.
// With vpart: virial[g][6] (xx, yy, zz, xy, xz, yz) = energy[s][c] on the
// diagonal plus the sums of the virial partials.
__global__ void k_energy_final(int K, int nblk, const double* __restrict__ part, const double* __restrict__ zero_coef,
                               const double* __restrict__ charges, double* __restrict__ energy,
                               const double* __restrict__ vpart, double* __restrict__ virial);

// ---- multiplier helpers ----------------------------------------------------------
// S_p on one piece by Horner, and dS/ds (runtime degree, coefficients in
// global memory).
template <typename R>
__device__ inline R mult_horner(const R* __restrict__ cs, int deg, R sv) {
  R S = cs[deg];
  for (int nn = deg - 1; nn >= 0; --nn) S = S * sv + cs[nn];
  return S;
}
template <typename R>
__device__ inline R mult_horner_d(const R* __restrict__ cs, int deg, R sv) {
  R dS = R(deg) * cs[deg];
  for (int nn = deg - 1; nn >= 1; --nn) dS = dS * sv + R(nn) * cs[nn];
  return dS;
}

// Per-thread energy accumulator.  FP64 sums are plain; FP32 terms are summed
// with Kahan compensation (error about one FP32 rounding of the total,
// independent of the count) and handed to the FP64 block reduction, which
// keeps FP64 arithmetic, narrow on this GPU, out of the per-mode loop.
template <typename R>
struct EnergyAcc {
  double s = 0.0;
  __device__ void add(double x) { s += x; }
  __device__ double value() const { return s; }
};
template <>
struct EnergyAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ double value() const { return double(s) - double(c); }
};

// Phi-hat_p / scale_p from its smooth part: the singular factor per p.
template <typename R>
__device__ inline R mult_value(int p, R S, R k, R k2, R u) {
  switch (p) {
    case 1: return S / k2;
    case 2: return S / k;
    case 3: return S - log(u);
    case 5: return S - u * u * log(u);
    default: return S;
  }
}

// d ln Phi-hat_p / d ln k = u (d phi / du) / phi, with dSu = dS/du.
template <typename R>
__device__ inline R mult_dlog(int p, R S, R dSu, R u, R phi) {
  if (phi == R(0)) return R(0);
  switch (p) {
    case 1: return u * dSu / S - R(2);
    case 2: return u * dSu / S - R(1);
    case 3: return (u * dSu - R(1)) / phi;
    case 5: return u * (dSu - R(2) * u * log(u) - u) / phi;
    default: return u * dSu / phi;
  }
}

// Block sums of the energy partial (and, with vpart, the six virial
// partials xx, yy, zz, xy, xz, yz) written at index `slot` of part /
// vpart[slot][6].
__device__ inline void block_partials(double e, const double (&v)[6], double* __restrict__ part,
                                      double* __restrict__ vpart, size_t slot) {
  __shared__ double sh[7][32];
  double t7[7] = {e, v[0], v[1], v[2], v[3], v[4], v[5]};
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < 7; ++i) t7[i] += __shfl_down_sync(0xffffffffu, t7[i], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < 7; ++i) sh[i][threadIdx.x >> 5] = t7[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int w = 0; w < int(blockDim.x >> 5); ++w)
#pragma unroll
      for (int i = 0; i < 7; ++i) t[i] += sh[i][w];
    part[slot] = t[0];
    if (vpart)
      for (int i = 0; i < 6; ++i) vpart[6 * slot + i] = t[1 + i];
  }
}

// Virial partial of one mode: v_ab += e_m D k_a k_b / k^2 (dlk = D / k^2).
__device__ inline void virial_add(double (&v)[6], double w, double kx, double ky, double kz) {
  v[0] += w * kx * kx;
  v[1] += w * ky * ky;
  v[2] += w * kz * kz;
  v[3] += w * kx * ky;
  v[4] += w * kx * kz;
  v[5] += w * ky * kz;
}

// ---- multiplier and energy (steps (iii)-(iv)) --------------------------------------
// blockIdx.y = g = s K + c.  For each half-spectrum mode m != 0 with
// u = |k|/k_c < 1 (k from structure s's box):
//   G = scale_g * sing_p(k) * (S_p(u) + log part) * iw2x * iw2y * iw2z  (times dV^2/V,
//   folded into scale_g), energy += w_m G |rho-hat|^2 / 2, rho-hat <- G rho-hat;
// all other modes are set to zero.  Energy partials per block in FP64.
template <typename R>
__global__ void __launch_bounds__(256) k_multiply(Cplx<R>* __restrict__ data, MultParams mp,
                                                  const int* __restrict__ pch, const double* __restrict__ scale,
                                                  const double* __restrict__ bmat, const R* __restrict__ coef,
                                                  const R* __restrict__ iw2, int iw2_stride,
                                                  double* __restrict__ part, int want_energy,
                                                  double* __restrict__ vpart) {
  // Modes outside the band |k| < k_c are zero-filled without being read.
  const int g = blockIdx.y;
  const int s = g / mp.K;
  const int p = pch[g];
  const R sc = R(scale[g]);
  const int nrow = mp.M[1] * mp.M[2];
  Cplx<R>* d = data + int64_t(g) * nrow * mp.Mxh;
  const R* cf = coef + size_t(p - 1) * kMultSeg * (mp.deg + 1);
  const R* iw2x = iw2 + size_t(3 * s) * iw2_stride;
  const R* iw2y = iw2x + iw2_stride;
  const R* iw2z = iw2y + iw2_stride;
  const R kc2 = R(1.0 / (mp.inv_kc * mp.inv_kc));
  const R inv_kc = R(mp.inv_kc);
  R bm[9];   // k = B m, B = 2 pi H^-1 of structure s (diagonal for a box)
#pragma unroll
  for (int i = 0; i < 9; ++i) bm[i] = R(bmat[9 * s + i]);
  const bool even_x = (mp.M[0] % 2) == 0;
  EnergyAcc<R> e;
  double vt[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  // Elements of the half spectrum in storage order, spread over the
  // channel's blocks (rows of small grids are shorter than a block).  The
  // element's (ix, iy, iz) advance by the grid stride's own digits with
  // carries: no divisions in the loop.
  const int64_t nel = int64_t(nrow) * mp.Mxh;
  const int64_t el0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  int ix, iy, iz, sx, sy, sz;
  {
    const int64_t r0 = el0 / mp.Mxh, rs = stride / mp.Mxh;
    ix = int(el0 - r0 * mp.Mxh);
    sx = int(stride - rs * mp.Mxh);
    iz = int(r0 / mp.M[1]);
    iy = int(r0 - int64_t(iz) * mp.M[1]);
    sz = int(rs / mp.M[1]);
    sy = int(rs - int64_t(sz) * mp.M[1]);
  }
  for (int64_t el = el0; el < nel; el += stride) {
    const int my = iy <= mp.M[1] / 2 ? iy : iy - mp.M[1];
    const int mz = iz <= mp.M[2] / 2 ? iz : iz - mp.M[2];
    const R kx = bm[0] * R(ix) + bm[1] * R(my) + bm[2] * R(mz);
    const R ky = bm[3] * R(ix) + bm[4] * R(my) + bm[5] * R(mz);
    const R kz = bm[6] * R(ix) + bm[7] * R(my) + bm[8] * R(mz);
    const R k2 = kx * kx + ky * ky + kz * kz;
    Cplx<R>* dp = d + el;
    if (!(k2 < kc2) || k2 == R(0)) {
      *dp = Cplx<R>{R(0), R(0)};
    } else {
      const int ay = my < 0 ? -my : my, az = mz < 0 ? -mz : mz;
      const R k = sqrt(k2);
      R u = k * inv_kc;
      if (u >= R(1)) u = R(1) - R(1e-7);
      int seg = int(u * R(kMultSeg));
      if (seg > kMultSeg - 1) seg = kMultSeg - 1;
      const R sv = R(2) * (u * R(kMultSeg) - R(seg)) - R(1);
      const R* cs = cf + seg * (mp.deg + 1);
      const R S = mult_horner(cs, mp.deg, sv);
      const R phi = mult_value(p, S, k, k2, u);
      const R G = phi * sc * iw2x[ix] * iw2y[ay] * iw2z[az];
      Cplx<R> v = *dp;
      if (want_energy) {
        const bool edge = (ix == 0) || (even_x && ix == mp.Mxh - 1);
        const R em = (edge ? R(0.5) : R(1)) * G * (v.x * v.x + v.y * v.y);
        e.add(em);
        if (vpart) {
          const R dS = mult_horner_d(cs, mp.deg, sv);
          const double dl = double(mult_dlog(p, S, dS * R(2 * kMultSeg), u, phi)) / double(k2);
          virial_add(vt, double(em) * dl, double(kx), double(ky), double(kz));
        }
      }
      v.x *= G;
      v.y *= G;
      *dp = v;
    }
    ix += sx;
    const int carry = ix >= mp.Mxh;
    if (carry) ix -= mp.Mxh;
    iy += sy + carry;
    if (iy >= mp.M[1]) {
      iy -= mp.M[1];
      ++iz;
    }
    iz += sz;
  }
  if (!want_energy) return;
  block_partials(e.value(), vt, part, vpart, size_t(g) * gridDim.x + blockIdx.x);
}

// The same multiplier for up to kMultGroup channels of one structure per
// work item (blockIdx.y = s nchunk + chunk, chunks of consecutive channels):
// a mode's k, window correction and piece are found once, the smooth part
// S_p and its singular factor once per distinct exponent of the chunk (so
// channels that share an exponent share them), and each channel only scales
// its mode and adds its energy.  Coefficients from shared memory.  No virial
// sums (plans that want them keep k_multiply).  Energy partials at the same
// [g][block] slots as k_multiply.
constexpr int kMultGroup = 8;
template <typename R>
__global__ void __launch_bounds__(256) k_multiply_group(Cplx<R>* __restrict__ data, MultParams mp,
                                                        const int* __restrict__ pch, const double* __restrict__ scale,
                                                        const double* __restrict__ bmat, const R* __restrict__ coef,
                                                        const R* __restrict__ iw2, int iw2_stride,
                                                        double* __restrict__ part, int want_energy) {
  __shared__ R cs_s[6 * kMultSeg * (kMaxMultDeg + 1)];
  __shared__ int pu_s[kMultGroup], cu_s[kMultGroup], nu_s;
  __shared__ double esum[kMultGroup][8];
  const int nchunk = (mp.K + kMultGroup - 1) / kMultGroup;
  const int s = blockIdx.y / nchunk, chunk = blockIdx.y - s * nchunk;
  const int c0 = chunk * kMultGroup, nc = min(kMultGroup, mp.K - c0);
  const int g0 = s * mp.K + c0;
  if (threadIdx.x == 0) {
    // the chunk's distinct exponents in first-seen order, and each channel's index among them
    int nu = 0;
    for (int c = 0; c < nc; ++c) {
      const int p = pch[g0 + c];
      int u = 0;
      while (u < nu && pu_s[u] != p) ++u;
      if (u == nu) pu_s[nu++] = p;
      cu_s[c] = u;
    }
    nu_s = nu;
  }
  for (int t = threadIdx.x; t < 6 * kMultSeg * (mp.deg + 1); t += blockDim.x) cs_s[t] = coef[t];
  __syncthreads();
  const int nu = nu_s;
  R sc[kMultGroup];
  const int nrow = mp.M[1] * mp.M[2];
  const int64_t nel = int64_t(nrow) * mp.Mxh;
  Cplx<R>* const d0 = data + int64_t(g0) * nel;   // channel c0 + c at d0 + c nel
#pragma unroll
  for (int c = 0; c < kMultGroup; ++c) sc[c] = c < nc ? R(scale[g0 + c]) : R(0);
  const R* iw2x = iw2 + size_t(3 * s) * iw2_stride;
  const R* iw2y = iw2x + iw2_stride;
  const R* iw2z = iw2y + iw2_stride;
  const R kc2 = R(1.0 / (mp.inv_kc * mp.inv_kc));
  const R inv_kc = R(mp.inv_kc);
  R bm[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) bm[i] = R(bmat[9 * s + i]);
  const bool even_x = (mp.M[0] % 2) == 0;
  EnergyAcc<R> e[kMultGroup];
  const int64_t el0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  int ix, iy, iz, sx, sy, sz;
  {
    const int64_t r0 = el0 / mp.Mxh, rs = stride / mp.Mxh;
    ix = int(el0 - r0 * mp.Mxh);
    sx = int(stride - rs * mp.Mxh);
    iz = int(r0 / mp.M[1]);
    iy = int(r0 - int64_t(iz) * mp.M[1]);
    sz = int(rs / mp.M[1]);
    sy = int(rs - int64_t(sz) * mp.M[1]);
  }
  for (int64_t el = el0; el < nel; el += stride) {
    const int my = iy <= mp.M[1] / 2 ? iy : iy - mp.M[1];
    const int mz = iz <= mp.M[2] / 2 ? iz : iz - mp.M[2];
    const R kx = bm[0] * R(ix) + bm[1] * R(my) + bm[2] * R(mz);
    const R ky = bm[3] * R(ix) + bm[4] * R(my) + bm[5] * R(mz);
    const R kz = bm[6] * R(ix) + bm[7] * R(my) + bm[8] * R(mz);
    const R k2 = kx * kx + ky * ky + kz * kz;
    if (!(k2 < kc2) || k2 == R(0)) {
#pragma unroll
      for (int c = 0; c < kMultGroup; ++c)
        if (c < nc) d0[c * nel + el] = Cplx<R>{R(0), R(0)};
    } else {
      const int ay = my < 0 ? -my : my, az = mz < 0 ? -mz : mz;
      const R k = sqrt(k2);
      R u = k * inv_kc;
      if (u >= R(1)) u = R(1) - R(1e-7);
      int seg = int(u * R(kMultSeg));
      if (seg > kMultSeg - 1) seg = kMultSeg - 1;
      const R sv = R(2) * (u * R(kMultSeg) - R(seg)) - R(1);
      const R iwp = iw2x[ix] * iw2y[ay] * iw2z[az];
      const bool edge = (ix == 0) || (even_x && ix == mp.Mxh - 1);
      const R wm = edge ? R(0.5) : R(1);
      for (int uu = 0; uu < nu; ++uu) {
        const int p = pu_s[uu];
        const R S = mult_horner(cs_s + ((p - 1) * kMultSeg + seg) * (mp.deg + 1), mp.deg, sv);
        const R phi = mult_value(p, S, k, k2, u) * iwp;
#pragma unroll
        for (int c = 0; c < kMultGroup; ++c) {
          if (c >= nc || cu_s[c] != uu) continue;   // the same for every thread of the block
          const R G = phi * sc[c];
          Cplx<R> v = d0[c * nel + el];
          if (want_energy) e[c].add(wm * G * (v.x * v.x + v.y * v.y));
          v.x *= G;
          v.y *= G;
          d0[c * nel + el] = v;
        }
      }
    }
    ix += sx;
    const int carry = ix >= mp.Mxh;
    if (carry) ix -= mp.Mxh;
    iy += sy + carry;
    if (iy >= mp.M[1]) {
      iy -= mp.M[1];
      ++iz;
    }
    iz += sz;
  }
  if (!want_energy) return;
  // block sums per channel (8 warps of 32): warp shuffles, then one thread per channel
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < kMultGroup; ++c) {
    double t = e[c].value();
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) esum[c][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x < nc) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += esum[threadIdx.x][w];
    part[size_t(g0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
  }
}

// Multiplier on the pruned spectrum of a single structure: layout
// [c][kx][z][y] (kx = 0 .. Mxh-1 allocated; only kx < nkx can be inside the
// band).  One (kx, z) line of y per block iteration; the same G, energy
// weights (kx = 0 counted once) and zeroing as k_multiply.
template <typename R>
__global__ void __launch_bounds__(256) k_multiply_planes(Cplx<R>* __restrict__ data, MultParams mp, int nkx,
                                                         const int* __restrict__ pch,
                                                         const double* __restrict__ scale,
                                                         const double* __restrict__ bmat, const R* __restrict__ coef,
                                                         const R* __restrict__ iw2, int iw2_stride,
                                                         double* __restrict__ part, int want_energy,
                                                         double* __restrict__ vpart) {
  const int c = blockIdx.y;
  const int p = pch[c];
  const R sc = R(scale[c]);
  const int64_t plane = int64_t(mp.M[1]) * mp.M[2];
  Cplx<R>* d = data + int64_t(c) * mp.Mxh * plane;
  const R* cf = coef + size_t(p - 1) * kMultSeg * (mp.deg + 1);
  const R* iw2x = iw2;
  const R* iw2y = iw2x + iw2_stride;
  const R* iw2z = iw2y + iw2_stride;
  const R kc2 = R(1.0 / (mp.inv_kc * mp.inv_kc));
  const R inv_kc = R(mp.inv_kc);
  R bm[9];   // k = B m (B = 2 pi H^-1; diagonal for a box)
#pragma unroll
  for (int i = 0; i < 9; ++i) bm[i] = R(bmat[i]);
  EnergyAcc<R> e;
  double vt[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const int nline = nkx * mp.M[2];
  for (int line = blockIdx.x; line < nline; line += gridDim.x) {
    const int ix = line / mp.M[2], iz = line - ix * mp.M[2];
    const int mz = iz <= mp.M[2] / 2 ? iz : iz - mp.M[2];
    // the line's part of k (kx and kz modes), then + my b_y per element
    const R lx = bm[0] * R(ix) + bm[2] * R(mz), ly = bm[3] * R(ix) + bm[5] * R(mz),
            lz = bm[6] * R(ix) + bm[8] * R(mz);
    // smallest |k|^2 of the line over real my: |l|^2 - (l . b_y)^2 / |b_y|^2
    // (= |l|^2 for a box, where b_y is orthogonal to l)
    const R lb = lx * bm[1] + ly * bm[4] + lz * bm[7];
    const R kxz2 = lx * lx + ly * ly + lz * lz - lb * lb / (bm[1] * bm[1] + bm[4] * bm[4] + bm[7] * bm[7]);
    Cplx<R>* dl = d + (int64_t(ix) * mp.M[2] + iz) * mp.M[1];
    if (!(kxz2 < kc2)) {
      for (int iy = threadIdx.x; iy < mp.M[1]; iy += blockDim.x) dl[iy] = Cplx<R>{R(0), R(0)};
      continue;
    }
    const int az = mz < 0 ? -mz : mz;
    const R wxz = sc * iw2x[ix] * iw2z[az];
    const R wedge = ix == 0 ? R(0.5) : R(1);
    for (int iy = threadIdx.x; iy < mp.M[1]; iy += blockDim.x) {
      const int my = iy <= mp.M[1] / 2 ? iy : iy - mp.M[1];
      const R kx = lx + bm[1] * R(my), ky = ly + bm[4] * R(my), kz = lz + bm[7] * R(my);
      const R k2 = kx * kx + ky * ky + kz * kz;
      if (!(k2 < kc2) || k2 == R(0)) {
        dl[iy] = Cplx<R>{R(0), R(0)};
        continue;
      }
      const R k = sqrt(k2);
      R u = k * inv_kc;
      if (u >= R(1)) u = R(1) - R(1e-7);
      int seg = int(u * R(kMultSeg));
      if (seg > kMultSeg - 1) seg = kMultSeg - 1;
      const R sv = R(2) * (u * R(kMultSeg) - R(seg)) - R(1);
      const R* cs = cf + seg * (mp.deg + 1);
      const R S = mult_horner(cs, mp.deg, sv);
      const R phi = mult_value(p, S, k, k2, u);
      const int ay = my < 0 ? -my : my;
      const R G = phi * wxz * iw2y[ay];
      Cplx<R> v = dl[iy];
      if (want_energy) {
        const R em = wedge * G * (v.x * v.x + v.y * v.y);
        e.add(em);
        if (vpart) {
          const R dS = mult_horner_d(cs, mp.deg, sv);
          const double dlg = double(mult_dlog(p, S, dS * R(2 * kMultSeg), u, phi)) / double(k2);
          virial_add(vt, double(em) * dlg, double(kx), double(ky), double(kz));
        }
      }
      v.x *= G;
      v.y *= G;
      dl[iy] = v;
    }
  }
  if (!want_energy) return;
  block_partials(e.value(), vt, part, vpart, size_t(c) * gridDim.x + blockIdx.x);
}

// ---- general cells: forces from grid-coordinate gradients ---------------------------
// The gathers of a general cell run with unit M/L (derivative scale 2 per
// grid cell), so they leave f_u, the gradient with respect to the grid
// coordinates u = T r; the Cartesian force is F = T^T f_u (T = diag(M) H^-T,
// row-major tmat of the single structure).
template <typename R>
__global__ void k_force_cell(int64_t n, const double* __restrict__ tmat, R* __restrict__ forces) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double f0 = forces[3 * i], f1 = forces[3 * i + 1], f2 = forces[3 * i + 2];
#pragma unroll
    for (int d = 0; d < 3; ++d) forces[3 * i + d] = R(tmat[d] * f0 + tmat[3 + d] * f1 + tmat[6 + d] * f2);
  }
}

// Upstream force gradients of a general cell into grid coordinates,
// g_u = T g (the backward kernels then work as for a box with unit M / L).
template <typename R>
__global__ void k_grad_to_cell(int64_t n, const double* __restrict__ tmat, const R* __restrict__ g,
                               R* __restrict__ gu) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double g0 = g[3 * i], g1 = g[3 * i + 1], g2 = g[3 * i + 2];
#pragma unroll
    for (int d = 0; d < 3; ++d) gu[3 * i + d] = R(tmat[3 * d] * g0 + tmat[3 * d + 1] * g1 + tmat[3 * d + 2] * g2);
  }
}

// ---- interpolation, direct from global memory (fallback kernel) ---------------------
// One thread per sorted atom, for plans whose padded regions do not fit in
// shared memory.  phi_c = sum Psi_c W; F = sum_c q_c sum Psi_c grad W, with
// grad_d W = (2 / h_d) dW/ds.  Writes in the original atom order.
template <typename R, int P>
__global__ void k_interp_direct(int64_t nmax, Geometry g, const double* __restrict__ smol,
                                const int* __restrict__ soff, const int* __restrict__ tile_start,
                                const R* __restrict__ st, const uint64_t* __restrict__ scell,
                                const R* __restrict__ sq, const int* __restrict__ sperm, WinCoef<R> wc,
                                const R* __restrict__ grid, const double* __restrict__ zero_coef,
                                const double* __restrict__ charges, R* __restrict__ phi, R* __restrict__ forces) {
  const int64_t n = soff[g.B];
  const int64_t chan = int64_t(g.M[2]) * g.M[1] * g.Mxp;
  for (int64_t a = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; a < n; a += int64_t(gridDim.x) * blockDim.x) {
    const int sidx = find_struct(tile_start, g.nts, g.B, a);
    const R two_hx = R(2.0 * smol[3 * sidx]), two_hy = R(2.0 * smol[3 * sidx + 1]),
            two_hz = R(2.0 * smol[3 * sidx + 2]);
    R wx[P], wy[P], wz[P], dx[P], dy[P], dz[P];
    window_weights<R, P>(st[a], wc, wx, dx);
    window_weights<R, P>(st[nmax + a], wc, wy, dy);
    window_weights<R, P>(st[2 * nmax + a], wc, wz, dz);
    int cx, cy, cz;
    unpack_cell(scell[a], cx, cy, cz);
    int ix[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      int v = cx + i;
      while (v >= g.M[0]) v -= g.M[0];
      ix[i] = v;
    }
    const int orig = sperm[a];
    R F0 = 0, F1 = 0, F2 = 0;
    for (int c = 0; c < g.K; ++c) {
      const int gc_idx = sidx * g.K + c;
      const R* gc = grid + gc_idx * chan;
      R ph = 0, f0 = 0, f1 = 0, f2 = 0;
      for (int k = 0; k < P; ++k) {
        int z = cz + k;
        while (z >= g.M[2]) z -= g.M[2];
        for (int j = 0; j < P; ++j) {
          int y = cy + j;
          while (y >= g.M[1]) y -= g.M[1];
          const R* row = gc + (int64_t(z) * g.M[1] + y) * g.Mxp;
          R sx = 0, dsx = 0;
#pragma unroll
          for (int i = 0; i < P; ++i) {
            const R v = __ldg(row + ix[i]);
            sx += v * wx[i];
            dsx += v * dx[i];
          }
          const R wyz = wy[j] * wz[k];
          ph += sx * wyz;
          f0 += dsx * wyz;
          f1 += sx * dy[j] * wz[k];
          f2 += sx * wy[j] * dz[k];
        }
      }
      ph += R(2.0 * zero_coef[gc_idx] * charges[2 * gc_idx]);
      if (phi) phi[int64_t(c) * n + orig] = ph;
      const R qc = sq[int64_t(c) * nmax + a];
      F0 += qc * f0;
      F1 += qc * f1;
      F2 += qc * f2;
    }
    if (forces) {
      forces[3 * int64_t(orig) + 0] = F0 * two_hx;
      forces[3 * int64_t(orig) + 1] = F1 * two_hy;
      forces[3 * int64_t(orig) + 2] = F2 * two_hz;
    }
  }
}

}  // namespace pswf
