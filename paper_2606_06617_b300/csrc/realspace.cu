// Real-space complement of PSWF-LR (Methods, "Implementation
// details": the pair term (1 - G_p(r)) / r^p that completes the reciprocal
// sum; G_p = 1 beyond r_c by reading C3, so only pairs closer than r_c count).
//
//   E_c   = 1/2 sum_i sum_{j != i, |r_ij| < r_c} q_i^c q_j^c f_p(r_ij)
//   phi_i^c = sum_j q_j^c f_p(r_ij)                       (= dE_c / dq_i^c)
//   F_i   = sum_c q_i^c sum_j q_j^c f_p'(r_ij) (r_j - r_i) / r_ij
//   f_p(r) = (1 - G_p(r / r_c)) / r^p
//
// with G_p the planner's piecewise polynomial in x = r / r_c (the multiplier's
// piece layout).  Neighbours come from a cell list of its own (cells at least
// r_c wide, at least 3 per axis, so each pair is found once, in one image):
// atoms are counted into cells, scanned, and scattered as cell-local
// coordinates with their charges; one warp per cell takes 32 of its atoms at
// a time and reads the 27 neighbour cells' atoms as broadcast loads.
//
// Cell-local coordinates of FP32 plans are integers in units of w / 2^29:
// a pair's displacement is then an exact integer difference (the neighbour
// cell adds its offset o 2^29) rounded to FP32 once, so its relative error
// is that of one rounding at any distance.  FP32 coordinates and an FP32
// cell offset would carry an absolute error ~1e-7 w, which 1/r^p magnifies
// to p 1e-7 w / r on close pairs (5e-6 of an energy at p = 4 with pairs
// 0.2 A apart in 4 A cells).  FP64 plans keep FP64 coordinates.  Every pair is evaluated from
// both ends (no atomics on per-atom outputs); channel energies are warp sums
// added to FP64 totals.
#include "realspace.hpp"

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "kernels.cuh"

namespace pswf {
namespace {

constexpr int kRsThreads = 256;
constexpr int kFixBits = 29;   // FP32 plans: cell-local unit w / 2^29; |dx| <= 2^30

// cell-local coordinate storage: fixed point for FP32, FP64 for FP64
template <typename R>
struct LocalT {
  using type = double;
};
template <>
struct LocalT<float> {
  using type = int;
};

// cell of a wrapped position and the position relative to the cell's corner
template <typename PosT>
__global__ void k_rs_bin(int64_t n, const PosT* __restrict__ pos, RealSpaceGeom g, int* __restrict__ cell_of,
                         int* __restrict__ rank, int* __restrict__ count, int* __restrict__ err) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    int ci[3];
    for (int d = 0; d < 3; ++d) {
      double x = double(pos[3 * i + d]);
      if (((__double_as_longlong(x) >> 52) & 0x7FF) == 0x7FF) {
        atomicCAS(err, 0, -6);
        x = 0.0;
      }
      const double s = x * g.inv_len[d];          // in boxes
      double fs = s - floor(s);                   // [0, 1]
      int c = int(fs * g.nc[d]);
      ci[d] = c < 0 ? 0 : (c >= g.nc[d] ? g.nc[d] - 1 : c);
    }
    const int cell = (ci[2] * g.nc[1] + ci[1]) * g.nc[0] + ci[0];
    cell_of[i] = cell;
    rank[i] = atomicAdd(count + cell, 1);
  }
}

template <typename PosT, typename R>
__global__ void k_rs_scatter(int64_t n, int64_t nmax, int K, const PosT* __restrict__ pos, const R* __restrict__ q,
                             RealSpaceGeom g, const int* __restrict__ cell_of, const int* __restrict__ rank,
                             const int* __restrict__ cell_start, typename LocalT<R>::type* __restrict__ lpos,
                             R* __restrict__ lq, int* __restrict__ perm) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int cell = cell_of[i];
    const int64_t dst = int64_t(cell_start[cell]) + rank[i];
    int ci[3] = {cell % g.nc[0], (cell / g.nc[0]) % g.nc[1], cell / (g.nc[0] * g.nc[1])};
    for (int d = 0; d < 3; ++d) {
      double x = double(pos[3 * i + d]);
      if (((__double_as_longlong(x) >> 52) & 0x7FF) == 0x7FF) x = 0.0;
      const double s = x * g.inv_len[d];
      const double local = (s - floor(s)) * g.len[d] - ci[d] * g.w[d];   // from the cell corner
      if constexpr (std::is_same<R, float>::value) {
        double u = rint(local * (double(1 << kFixBits) / g.w[d]));
        u = u < 0.0 ? 0.0 : (u > double(1 << kFixBits) ? double(1 << kFixBits) : u);
        lpos[4 * dst + d] = int(u);
      } else {
        lpos[4 * dst + d] = local;
      }
    }
    lpos[4 * dst + 3] = 0;
    for (int c = 0; c < K; ++c) lq[int64_t(c) * nmax + dst] = q[int64_t(c) * n + i];
    perm[dst] = int(i);
  }
}

// f_p(r) and f_p'(r) from G_p(x) (Horner on the piece of x) and r^-p.
template <typename R>
__device__ inline void pair_fn(int p, R r, R inv_r, R inv_rc, const R* __restrict__ cg, int deg, R& f, R& fp) {
  R x = r * inv_rc;
  if (x >= R(1)) x = R(1) - R(1e-7);
  int seg = int(x * R(kMultSeg));
  if (seg > kMultSeg - 1) seg = kMultSeg - 1;
  const R sv = R(2) * (x * R(kMultSeg) - R(seg)) - R(1);
  const R* cs = cg + size_t(p - 1) * kMultSeg * (deg + 1) + seg * (deg + 1);
  R G = cs[deg], dG = R(0);
  for (int k = deg - 1; k >= 0; --k) {
    dG = dG * sv + G;
    G = G * sv + cs[k];
  }
  dG *= R(2 * kMultSeg);                           // dG / dx
  R rp = inv_r;
  for (int k = 1; k < p; ++k) rp *= inv_r;         // r^-p
  const R one_m = R(1) - G;
  f = one_m * rp;
  fp = -dG * inv_rc * rp - R(p) * one_m * rp * inv_r;
}

template <typename R>
__global__ void __launch_bounds__(kRsThreads) k_rs_pairs(int64_t nmax, int K, RealSpaceGeom g,
                                                         const int* __restrict__ cell_start,
                                                         const typename LocalT<R>::type* __restrict__ lpos,
                                                         const R* __restrict__ lq,
                                                         const int* __restrict__ perm, const int* __restrict__ pch,
                                                         const R* __restrict__ coef_g, int deg_g, int64_t n,
                                                         double* __restrict__ energy, R* __restrict__ phi,
                                                         R* __restrict__ forces) {
  const int lane = threadIdx.x & 31;
  const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
  const int cell = blockIdx.x * (kRsThreads / 32) + (threadIdx.x >> 5);
  if (cell >= ncell) return;
  const int cx = cell % g.nc[0], cy = (cell / g.nc[0]) % g.nc[1], cz = cell / (g.nc[0] * g.nc[1]);
  using L = typename LocalT<R>::type;
  const R rc2 = R(g.r_c * g.r_c), inv_rc = R(1.0 / g.r_c);
  R unit[3];   // FP32: length of one fixed-point step per axis
  for (int d = 0; d < 3; ++d) unit[d] = R(g.w[d] / double(1 << kFixBits));
  const int a0 = cell_start[cell], a1 = cell_start[cell + 1];
  for (int base = a0; base < a1; base += 32) {
    const int i = base + lane;
    const bool own = i < a1;
    const int ii = own ? i : a0;
    const L xi = lpos[4 * ii], yi = lpos[4 * ii + 1], zi = lpos[4 * ii + 2];
    R fx = 0, fy = 0, fz = 0;
    R ph[kRsMaxK];
#pragma unroll
    for (int c = 0; c < kRsMaxK; ++c) ph[c] = R(0);
    for (int o = 0; o < 27; ++o) {
      const int od[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
      // cells are equal (width L / n_c), so the neighbour's corner is o w
      // from this cell's corner whether or not its index wraps
      const int c3[3] = {cx, cy, cz};
      int nc3[3];
      L sh[3];
      for (int d = 0; d < 3; ++d) {
        int t = c3[d] + od[d];
        t += t < 0 ? g.nc[d] : (t >= g.nc[d] ? -g.nc[d] : 0);
        nc3[d] = t;
        if constexpr (std::is_same<R, float>::value)
          sh[d] = od[d] * (1 << kFixBits);
        else
          sh[d] = od[d] * g.w[d];
      }
      const int nb = (nc3[2] * g.nc[1] + nc3[1]) * g.nc[0] + nc3[0];
      const int b0 = cell_start[nb], b1 = cell_start[nb + 1];
      for (int j = b0; j < b1; ++j) {
        R dx, dy, dz;
        if constexpr (std::is_same<R, float>::value) {
          dx = __int2float_rn(lpos[4 * j] + sh[0] - xi) * unit[0];
          dy = __int2float_rn(lpos[4 * j + 1] + sh[1] - yi) * unit[1];
          dz = __int2float_rn(lpos[4 * j + 2] + sh[2] - zi) * unit[2];
        } else {
          dx = lpos[4 * j] + sh[0] - xi;
          dy = lpos[4 * j + 1] + sh[1] - yi;
          dz = lpos[4 * j + 2] + sh[2] - zi;
        }
        const R r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < rc2) || (o == 13 && j == ii)) continue;
        const R r = sqrt(r2);
        const R inv_r = R(1) / r;
        R fsum = 0;   // sum_c q_i^c q_j^c f_p'(r)
        for (int c = 0; c < K; ++c) {
          R f, fp;
          pair_fn(pch[c], r, inv_r, inv_rc, coef_g, deg_g, f, fp);
          const R qj = lq[int64_t(c) * nmax + j];
          ph[c] += qj * f;
          fsum += lq[int64_t(c) * nmax + ii] * qj * fp;
        }
        const R s = fsum * inv_r;
        fx += s * dx;
        fy += s * dy;
        fz += s * dz;
      }
    }
    const int orig = own ? perm[i] : 0;
    for (int c = 0; c < K; ++c) {
      const R qi = own ? lq[int64_t(c) * nmax + ii] : R(0);
      double e = own ? 0.5 * double(qi) * double(ph[c]) : 0.0;
      for (int off = 16; off > 0; off >>= 1) e += __shfl_down_sync(0xffffffffu, e, off);
      if (lane == 0 && e != 0.0) atomicAdd(energy + c, e);
      if (own && phi) phi[int64_t(c) * n + orig] = ph[c];
    }
    if (own && forces) {
      forces[3 * int64_t(orig)] = fx;
      forces[3 * int64_t(orig) + 1] = fy;
      forces[3 * int64_t(orig) + 2] = fz;
    }
  }
}

__global__ void k_rs_total(int K, double* __restrict__ energy) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int c = 0; c < K; ++c) t += energy[c];
    energy[K] = t;
  }
}

}  // namespace

bool real_space_geometry(const double box[3], double r_c, RealSpaceGeom& g) {
  for (int d = 0; d < 3; ++d) {
    const int nc = int(box[d] / r_c);
    if (nc < 3) return false;
    g.nc[d] = nc;
    g.len[d] = box[d];
    g.inv_len[d] = 1.0 / box[d];
    g.w[d] = box[d] / nc;
  }
  g.r_c = r_c;
  return true;
}

template <typename R>
cudaError_t real_space_run(const RealSpaceArgs& a, cudaStream_t s, int* nlaunch) {
  const RealSpaceGeom& g = a.geo;
  const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.energy, 0, size_t(a.K + 1) * sizeof(double), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.count, 0, size_t(ncell) * sizeof(int), s)) != cudaSuccess) return e;
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((a.n + kRsThreads - 1) / kRsThreads, 148 * 16)));
  if (a.n > 0) {
    if (a.pos_dtype == 1)
      k_rs_bin<double><<<blocks, kRsThreads, 0, s>>>(a.n, static_cast<const double*>(a.pos), g, a.cell_of, a.rank,
                                                     a.count, a.err);
    else
      k_rs_bin<float><<<blocks, kRsThreads, 0, s>>>(a.n, static_cast<const float*>(a.pos), g, a.cell_of, a.rank,
                                                    a.count, a.err);
    ++*nlaunch;
  }
  const int nsb = (ncell + a.scan_per_block - 1) / a.scan_per_block;
  k_scan_block_sums<<<nsb, kScanBlock, 0, s>>>(ncell, a.count, a.scan_sums, a.scan_per_block);
  k_scan_sums<<<1, 32, 0, s>>>(nsb, a.scan_sums);
  k_scan_apply<<<nsb, kScanBlock, 0, s>>>(ncell, a.count, a.scan_sums, a.scan_per_block, a.cell_start);
  *nlaunch += 3;
  if (a.n > 0) {
    if (a.pos_dtype == 1)
      k_rs_scatter<double, R><<<blocks, kRsThreads, 0, s>>>(a.n, a.nmax, a.K, static_cast<const double*>(a.pos),
                                                            static_cast<const R*>(a.q), g, a.cell_of, a.rank,
                                                            a.cell_start, static_cast<typename LocalT<R>::type*>(a.lpos),
                                                            static_cast<R*>(a.lq), a.perm);
    else
      k_rs_scatter<float, R><<<blocks, kRsThreads, 0, s>>>(a.n, a.nmax, a.K, static_cast<const float*>(a.pos),
                                                           static_cast<const R*>(a.q), g, a.cell_of, a.rank,
                                                           a.cell_start, static_cast<typename LocalT<R>::type*>(a.lpos),
                                                           static_cast<R*>(a.lq), a.perm);
    k_rs_pairs<R><<<(ncell + kRsThreads / 32 - 1) / (kRsThreads / 32), kRsThreads, 0, s>>>(
        a.nmax, a.K, g, a.cell_start, static_cast<const typename LocalT<R>::type*>(a.lpos), static_cast<const R*>(a.lq), a.perm, a.pch,
        static_cast<const R*>(a.coef_g), a.deg_g, a.n, a.energy, static_cast<R*>(a.phi), static_cast<R*>(a.forces));
    *nlaunch += 2;
  }
  k_rs_total<<<1, 32, 0, s>>>(a.K, a.energy);
  ++*nlaunch;
  return cudaGetLastError();
}

template cudaError_t real_space_run<float>(const RealSpaceArgs&, cudaStream_t, int*);
template cudaError_t real_space_run<double>(const RealSpaceArgs&, cudaStream_t, int*);

}  // namespace pswf
