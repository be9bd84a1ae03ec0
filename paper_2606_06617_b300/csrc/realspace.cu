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
// coordinates with their charges.
//
// Pair kernel: persistent blocks of 8 warps, one warp per cell at a time,
// its atoms in chunks of up to 32.  A chunk of m atoms gives each atom
// G = 32 / m lanes (a power of two), which split the 27 neighbour cells'
// candidates, so partial chunks keep the lanes busy.  Each lane tests its
// candidates against r_c (about 15% pass in a liquid) and appends the ones
// inside to its own queue in shared memory; the queues are drained in
// rounds in which every lane evaluates one of its queued pairs, so the
// mollifier polynomials run on dense rounds rather than on the few lanes
// whose candidate happens to pass.  Per-atom sums stay in registers (no
// atomics); the G lanes of an atom are summed with shuffles at the end.
//
// Coordinates: the cutoff test reads cell-local coordinates in the plan's
// precision.  FP32 plans evaluate a queued pair from a second copy held as
// integers in units of w / 2^29: the displacement is an exact integer
// difference (the neighbour cell adds its offset o 2^29) rounded to FP32
// once, so its relative error is that of one rounding at any distance.
// FP32 coordinates and an FP32 cell offset would carry an absolute error
// ~1e-7 w, which 1/r^p magnifies to p 1e-7 w / r on close pairs (5e-6 of an
// energy at p = 4 with pairs 0.2 A apart in 4 A cells).  A pair whose FP32
// test and exact distance straddle r_c differs from the sum by a term with
// 1 - G_p(1) ~ 1e-5, which is negligible.  FP64 plans use one FP64 copy.
#include "realspace.hpp"

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "kernels.cuh"

namespace pswf {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kFixBits = 29;     // FP32 plans: cell-local unit w / 2^29; |dx| <= 2^30
constexpr int kQueueCap = 192;   // queued pairs per lane; drained early only above kQueueCap - 32
constexpr int kCellBits = 11;    // queue entry: (neighbour o << 11) | index within that cell
constexpr int kMaxCellAtoms = 1 << kCellBits;
constexpr int kPswfECell = -9;   // PSWF_ECELL

template <typename R>
__host__ __device__ constexpr size_t warp_smem_bytes() {
  // queue [kQueueCap][32] of 16-bit entries, stage [32][4] R, neighbour
  // starts and ends [2][27] (padded to 224 bytes)
  return size_t(kQueueCap) * 32 * 2 + 32 * 4 * sizeof(R) + 224;
}
static_assert(warp_smem_bytes<float>() % 16 == 0 && warp_smem_bytes<double>() % 16 == 0, "aligned warp regions");

// fixed-point copy of the cell-local coordinates: int for FP32 plans, none
// (the FP64 copy itself) for FP64 plans
template <typename R>
struct LocalT {
  using type = double;
};
template <>
struct LocalT<float> {
  using type = int;
};

template <typename T>
__device__ inline void load3(const T* __restrict__ p, int64_t j, T& x, T& y, T& z) {
  if constexpr (sizeof(T) == 4) {
    using V = typename std::conditional<std::is_same<T, float>::value, float4, int4>::type;
    const V v = reinterpret_cast<const V*>(p)[j];
    x = v.x;
    y = v.y;
    z = v.z;
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[2 * j];
    const double2 b = reinterpret_cast<const double2*>(p)[2 * j + 1];
    x = a.x;
    y = a.y;
    z = b.x;
  }
}

// cell of a wrapped position (count and rank within the cell)
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

// cell-local coordinates (test copy [nmax][4] in R; FP32 plans also the
// fixed-point copy [nmax][4]), charges [K][nmax] and the original index
template <typename PosT, typename R>
__global__ void k_rs_scatter(int64_t n, int64_t nmax, int K, const PosT* __restrict__ pos, const R* __restrict__ q,
                             RealSpaceGeom g, const int* __restrict__ cell_of, const int* __restrict__ rank,
                             const int* __restrict__ cell_start, R* __restrict__ lchk,
                             typename LocalT<R>::type* __restrict__ lfix, R* __restrict__ lq,
                             int* __restrict__ perm) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int cell = cell_of[i];
    const int64_t dst = int64_t(cell_start[cell]) + rank[i];
    int ci[3] = {cell % g.nc[0], (cell / g.nc[0]) % g.nc[1], cell / (g.nc[0] * g.nc[1])};
    for (int d = 0; d < 3; ++d) {
      double x = double(pos[3 * i + d]);
      if (((__double_as_longlong(x) >> 52) & 0x7FF) == 0x7FF) x = 0.0;
      const double s = x * g.inv_len[d];
      const double local = (s - floor(s)) * g.len[d] - ci[d] * g.w[d];   // from the cell corner
      lchk[4 * dst + d] = R(local);
      if constexpr (std::is_same<R, float>::value) {
        double u = rint(local * (double(1 << kFixBits) / g.w[d]));
        u = u < 0.0 ? 0.0 : (u > double(1 << kFixBits) ? double(1 << kFixBits) : u);
        lfix[4 * dst + d] = int(u);
      }
    }
    lchk[4 * dst + 3] = R(0);
    if constexpr (std::is_same<R, float>::value) lfix[4 * dst + 3] = 0;
    for (int c = 0; c < K; ++c) lq[int64_t(c) * nmax + dst] = q[int64_t(c) * n + i];
    perm[dst] = int(i);
  }
}

template <typename R>
struct PairArgs {
  RealSpaceGeom g;
  int64_t nmax, n;
  int K, deg;
  const int* cell_start;
  const R* lchk;
  const typename LocalT<R>::type* lfix;
  const R* lq;
  const int* perm;
  const int* pch;
  const R* coef;     // [6][kMultSeg][deg + 1]
  double* energy;
  R* phi;
  R* forces;
  int* err;
};

template <typename R, int NC>
__device__ inline void load_coefs(const R* __restrict__ cs, R (&c)[NC]) {
  if constexpr (std::is_same<R, float>::value) {
#pragma unroll
    for (int k = 0; k < NC; k += 4) {
      const float4 v = *reinterpret_cast<const float4*>(cs + k);
      c[k] = v.x;
      c[k + 1] = v.y;
      c[k + 2] = v.z;
      c[k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < NC; k += 2) {
      const double2 v = *reinterpret_cast<const double2*>(cs + k);
      c[k] = v.x;
      c[k + 1] = v.y;
    }
  }
}

// 1 / sqrt(r2): the hardware estimate refined by one Newton step
// y <- y (3 - r2 y^2) / 2 (FP32); FP64 divides.
template <typename R>
__device__ inline R inv_sqrt(R r2) {
  if constexpr (std::is_same<R, float>::value) {
    const float y = rsqrtf(r2);
    return y * (1.5f - 0.5f * r2 * y * y);
  } else {
    return 1.0 / sqrt(r2);
  }
}

// KC channels per pair evaluation, fully unrolled (channels past K carry
// zero charges); NC coefficients per mollifier piece (zero-padded).
template <typename R, int NC, int KC>
__global__ void __launch_bounds__(kRsThreads, 2) k_rs_pairs(PairArgs<R> a) {
  using L = typename LocalT<R>::type;
  extern __shared__ __align__(16) unsigned char rs_smem[];
  R* coef = reinterpret_cast<R*>(rs_smem);                       // [6][kMultSeg][NC], zero-padded
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wbase = rs_smem + size_t(6) * kMultSeg * NC * sizeof(R) + size_t(warp) * warp_smem_bytes<R>();
  uint16_t* queue = reinterpret_cast<uint16_t*>(wbase);                     // [kQueueCap][32]
  R* stage = reinterpret_cast<R*>(wbase + kQueueCap * 32 * 2);              // [32][4] candidates
  int* nbs = reinterpret_cast<int*>(stage + 32 * 4);                        // [27] neighbour cell starts
  int* nbe = nbs + 27;                                                      // [27] ends
  for (int t = threadIdx.x; t < 6 * kMultSeg * NC; t += blockDim.x) {
    const int k = t % NC, row = t / NC;
    coef[t] = k <= a.deg ? a.coef[size_t(row) * (a.deg + 1) + k] : R(0);
  }
  __syncthreads();

  const RealSpaceGeom& g = a.g;
  const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
  const R rc2 = R(g.r_c * g.r_c), inv_rc = R(1.0 / g.r_c);
  R unit[3];   // FP32: length of one fixed-point step per axis
  for (int d = 0; d < 3; ++d) unit[d] = R(g.w[d] / double(1 << kFixBits));
  int prow[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) prow[c] = c < a.K ? a.pch[c] - 1 : 0;

  for (int cell = blockIdx.x * kRsWarps + warp; cell < ncell; cell += gridDim.x * kRsWarps) {
    const int c3[3] = {cell % g.nc[0], (cell / g.nc[0]) % g.nc[1], cell / (g.nc[0] * g.nc[1])};
    const int a0 = a.cell_start[cell], a1 = a.cell_start[cell + 1];
    for (int base = a0; base < a1; base += 32) {
      const int m = min(32, a1 - base);
      int G = 1;
      while (m * G * 2 <= 32) G *= 2;
      const int slot = lane / G, sub = lane % G;
      const bool own = slot < m;
      const int i = own ? base + slot : a0;
      R xi, yi, zi;
      load3(a.lchk, i, xi, yi, zi);
      L ix, iy, iz;
      if constexpr (std::is_same<R, float>::value)
        load3(a.lfix, i, ix, iy, iz);
      else
        ix = xi, iy = yi, iz = zi;
      R qi[KC], ph[KC];
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        qi[c] = c < a.K ? a.lq[int64_t(c) * a.nmax + i] : R(0);
        ph[c] = R(0);
      }
      R fx = 0, fy = 0, fz = 0;
      int len = 0;

      // every queued pair of this lane: exact displacement, f_p and f_p'
      auto drain = [&]() {
        const int rounds = __reduce_max_sync(0xffffffffu, len);
        for (int t = 0; t < rounds; ++t) {
          if (t >= len) continue;
          const uint32_t e = queue[t * 32 + lane];
          const int o = int(e >> kCellBits), j = nbs[o] + int(e & (kMaxCellAtoms - 1));
          const int o3 = o / 3;
          const int ox = o - 3 * o3 - 1, oy = o3 - 3 * (o3 / 3) - 1, oz = o3 / 3 - 1;
          L jx, jy, jz;
          load3(a.lfix, j, jx, jy, jz);
          R qj[KC];
#pragma unroll
          for (int c = 0; c < KC; ++c) qj[c] = c < a.K ? a.lq[int64_t(c) * a.nmax + j] : R(0);
          R dx, dy, dz;
          if constexpr (std::is_same<R, float>::value) {
            dx = __int2float_rn(jx + ox * (1 << kFixBits) - ix) * unit[0];
            dy = __int2float_rn(jy + oy * (1 << kFixBits) - iy) * unit[1];
            dz = __int2float_rn(jz + oz * (1 << kFixBits) - iz) * unit[2];
          } else {
            dx = jx + ox * g.w[0] - ix;
            dy = jy + oy * g.w[1] - iy;
            dz = jz + oz * g.w[2] - iz;
          }
          const R r2 = dx * dx + dy * dy + dz * dz;
          const R inv_r = inv_sqrt(r2);
          const R r = r2 * inv_r;
          const R ir2 = inv_r * inv_r, ir4 = ir2 * ir2;
          R x = r * inv_rc;
          if (x >= R(1)) x = R(1) - R(1e-7);
          int seg = int(x * R(kMultSeg));
          if (seg > kMultSeg - 1) seg = kMultSeg - 1;
          const R sv = R(2) * (x * R(kMultSeg) - R(seg)) - R(1);
          R fsum = 0;   // sum_c q_i^c q_j^c f_p'(r)
#pragma unroll
          for (int c = 0; c < KC; ++c) {
            R cf[NC];
            load_coefs<R, NC>(coef + (prow[c] * kMultSeg + seg) * NC, cf);
            R Gv = cf[NC - 1], dG = R(0);
#pragma unroll
            for (int k = NC - 2; k >= 0; --k) {
              dG = dG * sv + Gv;
              Gv = Gv * sv + cf[k];
            }
            dG *= R(2 * kMultSeg);                       // dG / dx
            const int p = prow[c] + 1;                    // r^-p from the bits of p
            const R rp = ((p & 1) ? inv_r : R(1)) * ((p & 2) ? ir2 : R(1)) * ((p & 4) ? ir4 : R(1));
            const R one_m = R(1) - Gv;
            const R f = one_m * rp;
            const R fp = -(dG * inv_rc + R(p) * one_m * inv_r) * rp;
            ph[c] += qj[c] * f;
            fsum += qi[c] * qj[c] * fp;
          }
          const R sc = fsum * inv_r;
          fx += sc * dx;
          fy += sc * dy;
          fz += sc * dz;
        }
        len = 0;
      };

      // the 27 neighbour cells' atom ranges, one lane each
      if (lane < 27) {
        const int od[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
        // cells are equal (width L / n_c), so the neighbour's corner is o w
        // from this cell's corner whether or not its index wraps
        int nc3[3];
        for (int d = 0; d < 3; ++d) {
          int t = c3[d] + od[d];
          t += t < 0 ? g.nc[d] : (t >= g.nc[d] ? -g.nc[d] : 0);
          nc3[d] = t;
        }
        const int nb = (nc3[2] * g.nc[1] + nc3[1]) * g.nc[0] + nc3[0];
        int b0 = a.cell_start[nb], b1 = a.cell_start[nb + 1];
        if (b1 - b0 > kMaxCellAtoms) {   // not encodable: reported, cell left out
          atomicCAS(a.err, 0, kPswfECell);
          b1 = b0;
        }
        nbs[lane] = b0;
        nbe[lane] = b1;
      }
      __syncwarp();
      for (int o = 0; o < 27; ++o) {
        const int od[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
        const R ax = xi - R(od[0] * g.w[0]), ay = yi - R(od[1] * g.w[1]), az = zi - R(od[2] * g.w[2]);
        const int b0 = nbs[o], b1 = nbe[o];
        const uint32_t tag = uint32_t(o) << kCellBits;
        for (int jb = b0; jb < b1; jb += 32) {
          if (__reduce_max_sync(0xffffffffu, len) > kQueueCap - 32) drain();
          const int cnt = min(32, b1 - jb);
          // one coalesced load of up to 32 candidates into the warp's stage
          if (lane < cnt) {
            R sx, sy, sz;
            load3(a.lchk, jb + lane, sx, sy, sz);
            stage[4 * lane] = sx;
            stage[4 * lane + 1] = sy;
            stage[4 * lane + 2] = sz;
          }
          __syncwarp();
          if (own) {
#pragma unroll 4
            for (int jj = sub; jj < cnt; jj += G) {
              R xj, yj, zj;
              if constexpr (std::is_same<R, float>::value) {
                const float4 v = reinterpret_cast<const float4*>(stage)[jj];
                xj = v.x, yj = v.y, zj = v.z;
              } else {
                const double2 v0 = reinterpret_cast<const double2*>(stage)[2 * jj];
                xj = v0.x, yj = v0.y, zj = stage[4 * jj + 2];
              }
              const R dx = xj - ax, dy = yj - ay, dz = zj - az;
              const R r2 = dx * dx + dy * dy + dz * dz;
              // r2 = 0 only for the atom itself (or a coincident atom, which
              // the sum excludes too)
              if (r2 < rc2 && r2 > R(0)) queue[len++ * 32 + lane] = uint16_t(tag | uint32_t(jb - b0 + jj));
            }
          }
          __syncwarp();
        }
      }
      drain();
      __syncwarp();   // nbs / nbe are rewritten for the next chunk

      // the G lanes of an atom hold partial sums over its candidates
      for (int off = G / 2; off > 0; off >>= 1) {
#pragma unroll
        for (int c = 0; c < KC; ++c) ph[c] += __shfl_xor_sync(0xffffffffu, ph[c], off);
        fx += __shfl_xor_sync(0xffffffffu, fx, off);
        fy += __shfl_xor_sync(0xffffffffu, fy, off);
        fz += __shfl_xor_sync(0xffffffffu, fz, off);
      }
      const bool lead = own && sub == 0;
      const int orig = lead ? a.perm[i] : 0;
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        if (c >= a.K) break;
        double e = lead ? 0.5 * double(qi[c]) * double(ph[c]) : 0.0;
        for (int off = 16; off > 0; off >>= 1) e += __shfl_down_sync(0xffffffffu, e, off);
        if (lane == 0 && e != 0.0) atomicAdd(a.energy + c, e);
      }
      if (lead && a.phi) {
#pragma unroll
        for (int c = 0; c < KC; ++c)
          if (c < a.K) a.phi[int64_t(c) * a.n + orig] = ph[c];
      }
      if (lead && a.forces) {
        a.forces[3 * int64_t(orig)] = fx;
        a.forces[3 * int64_t(orig) + 1] = fy;
        a.forces[3 * int64_t(orig) + 2] = fz;
      }
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

template <typename R, int NC, int KC>
cudaError_t launch_pairs_k(const PairArgs<R>& pa, int ncell, cudaStream_t s) {
  const size_t smem = size_t(6) * kMultSeg * NC * sizeof(R) + size_t(kRsWarps) * warp_smem_bytes<R>();
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_rs_pairs<R, NC, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               int(smem));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rs_pairs<R, NC, KC>, kRsThreads, smem);
  const int64_t want = (int64_t(ncell) + kRsWarps - 1) / kRsWarps;
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(std::max(nsm, 1)) * std::max(per_sm, 1))));
  k_rs_pairs<R, NC, KC><<<blocks, kRsThreads, smem, s>>>(pa);
  return cudaGetLastError();
}

template <typename R, int NC>
cudaError_t launch_pairs(const PairArgs<R>& pa, int ncell, cudaStream_t s) {
  if (pa.K <= 1) return launch_pairs_k<R, NC, 1>(pa, ncell, s);
  if (pa.K <= 2) return launch_pairs_k<R, NC, 2>(pa, ncell, s);
  if (pa.K <= 4) return launch_pairs_k<R, NC, 4>(pa, ncell, s);
  if (pa.K <= 8) return launch_pairs_k<R, NC, 8>(pa, ncell, s);
  return launch_pairs_k<R, NC, kRsMaxK>(pa, ncell, s);
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
  if (a.deg_g > kMaxMultDeg) return cudaErrorInvalidValue;
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
    using L = typename LocalT<R>::type;
    R* lchk = static_cast<R*>(a.lpos);
    // FP32: the fixed-point copy follows the test copy; FP64: one copy
    L* lfix = std::is_same<R, float>::value ? reinterpret_cast<L*>(lchk + 4 * a.nmax) : reinterpret_cast<L*>(lchk);
    if (a.pos_dtype == 1)
      k_rs_scatter<double, R><<<blocks, kRsThreads, 0, s>>>(a.n, a.nmax, a.K, static_cast<const double*>(a.pos),
                                                            static_cast<const R*>(a.q), g, a.cell_of, a.rank,
                                                            a.cell_start, lchk, lfix, static_cast<R*>(a.lq), a.perm);
    else
      k_rs_scatter<float, R><<<blocks, kRsThreads, 0, s>>>(a.n, a.nmax, a.K, static_cast<const float*>(a.pos),
                                                           static_cast<const R*>(a.q), g, a.cell_of, a.rank,
                                                           a.cell_start, lchk, lfix, static_cast<R*>(a.lq), a.perm);
    PairArgs<R> pa;
    pa.g = g;
    pa.nmax = a.nmax;
    pa.n = a.n;
    pa.K = a.K;
    pa.deg = a.deg_g;
    pa.cell_start = a.cell_start;
    pa.lchk = lchk;
    pa.lfix = lfix;
    pa.lq = static_cast<const R*>(a.lq);
    pa.perm = a.perm;
    pa.pch = a.pch;
    pa.coef = static_cast<const R*>(a.coef_g);
    pa.energy = a.energy;
    pa.phi = static_cast<R*>(a.phi);
    pa.forces = static_cast<R*>(a.forces);
    pa.err = a.err;
    // coefficient rows padded to whole 16-byte loads (the planner's degree
    // is at most kMaxMultDeg = 16)
    static_assert(kMaxMultDeg + 1 <= 18, "coefficient rows");
    if constexpr (std::is_same<R, float>::value) {
      e = a.deg_g + 1 <= 8 ? launch_pairs<R, 8>(pa, ncell, s) : launch_pairs<R, 20>(pa, ncell, s);
    } else {
      e = launch_pairs<R, 18>(pa, ncell, s);
    }
    if (e != cudaSuccess) return e;
    *nlaunch += 2;
  }
  k_rs_total<<<1, 32, 0, s>>>(a.K, a.energy);
  ++*nlaunch;
  return cudaGetLastError();
}

template cudaError_t real_space_run<float>(const RealSpaceArgs&, cudaStream_t, int*);
template cudaError_t real_space_run<double>(const RealSpaceArgs&, cudaStream_t, int*);

}  // namespace pswf
