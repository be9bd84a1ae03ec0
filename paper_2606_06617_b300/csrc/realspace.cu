// Real-space complement of PSWF-LR (Methods, "Implementation
// details": the pair term (1 - G_p(r)) / r^p that completes the reciprocal
// sum; G_p taken as 1 beyond r_c, so only pairs closer than r_c count).
//
//   E_c   = 1/2 sum_i sum_{j != i, |r_ij| < r_c} q_i^c q_j^c f_p(r_ij)
//   phi_i^c = sum_j q_j^c f_p(r_ij)                       (= dE_c / dq_i^c)
//   F_i   = sum_c q_i^c sum_j q_j^c f_p'(r_ij) (r_j - r_i) / r_ij
//   f_p(r) = (1 - G_p(r / r_c)) / r^p
//
// with G_p the planner's piecewise polynomial in x = r / r_c (the multiplier's
// piece layout).  Neighbours come from a cell list of its own along the
// lattice vectors a_d of the cell H: n_c[d] >= 3 list cells per vector, each
// the parallelepiped spanned by a_d / n_c[d] and at least r_c high across
// every pair of faces, so a pair closer than r_c lies in adjacent list cells
// and is found once, in one image (for a box the list cells are boxes).
// Atoms are counted into list cells (fractional coordinates s = r H^-1),
// scanned, and scattered in cell order with their charges.
//
// Pair kernel: persistent blocks of 8 warps, one warp per list cell at a
// time, its atoms in chunks of up to 32.  Each pair is evaluated once: a
// chunk's atoms i take as candidates the atoms of the half shell, the 13
// neighbour cells o with (oz, oy, ox) lexicographically positive and the
// cell itself with j > i in cell order (the other 13 neighbours pair with
// this cell from their own half shell).  A chunk of m atoms gives each atom
// G = 32 / m lanes (a power of two), which split the candidates, so partial
// chunks keep the lanes busy.  Each lane tests its candidates against r_c
// (about 15% pass in a liquid) and appends the ones inside to its own queue
// in shared memory (16-bit entries: half-shell slot and index in that
// cell).  After the sweep the queues are drained: their entries, taken in
// lane order, are cut into 32 ranges of equal length, so every lane
// evaluates the same number of pairs however the atoms' pair counts differ
// (a half shell's counts depend strongly on where the atom sits in its
// cell).  The i side of a pair stays in registers while a lane's range
// stays in one atom's queue and is then added to the atom's accumulator
// row; the j side (phi_j^c += q_i^c f_p, F_j -= F_ij) is added to j's row
// at once, with 16-byte vector atomics in FP32.  The rows are kept in cell
// order and copied to the caller's layouts by a last kernel, which also
// forms the channel energies 1/2 sum_i q_i^c phi_i^c in FP64.  A lane that
// crosses into another atom's queue reads that atom's record from the
// chunk's records, staged in shared memory at the start of the drain.
//
// Coordinates: the cutoff test reads Cartesian coordinates from the list
// cell's corner in the plan's precision (16 or 32 bytes per atom, streamed
// through a shared-memory stage); a neighbour's corner is o . (a_d / n_c)
// away, from a table the block fills once.  A queued pair is evaluated from
// the neighbour's record: its position in its list cell in units of the
// cell's edges and its K charges side by side (one 32-byte sector for K <= 5
// in FP32), so the scattered reads of the pair rounds touch one record, not
// K + 1 arrays.  FP32 records hold the position as integers in units of
// 2^-29 of an edge: the displacement is an exact integer difference (the
// neighbour cell adds its offset o 2^29) times the edge matrix, so its
// relative error is that of a few roundings at any distance.  FP32
// coordinates and an FP32 cell offset would carry an absolute error ~1e-7 w,
// which 1/r^p magnifies to p 1e-7 w / r on close pairs (5e-6 of an energy at
// p = 4 with pairs 0.2 A apart in 4 A cells).  A pair whose FP32 test and
// exact distance straddle r_c differs from the sum by a term with
// 1 - G_p(1) ~ 1e-5, which is negligible.  FP64 records hold FP64 positions.
#include "realspace.hpp"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "kernels.cuh"
#include "pswf_lr.h"

namespace pswf {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kFixBits = 29;     // FP32 plans: cell-local unit w / 2^29; |dx| <= 2^30
// queued pairs per lane (the backward's larger records leave room for
// fewer); a queue is drained early only above its capacity - 32.  Columns
// of an odd number of words, so the lanes' columns start in distinct banks.
template <bool BW>
__host__ __device__ constexpr int queue_cap() {
  return BW ? 160 : 176;
}
template <bool BW>
__host__ __device__ constexpr int queue_stride() {
  return queue_cap<BW>() + 2;
}
constexpr int kCellBits = 11;    // queue entry: (half-shell slot << 11) | index within that cell
constexpr int kMaxCellAtoms = 1 << kCellBits;
// half shell: neighbour offsets o = (ox + 1) + 3 (oy + 1) + 9 (oz + 1) from
// kSelf (the cell itself, o = (0, 0, 0)) to 26, i.e. (oz, oy, ox)
// lexicographically >= 0: slot s is offset kSelf + s
constexpr int kSelf = 13;
constexpr int kHalf = 14;


// exact cell-local coordinates: fixed-point int for FP32 plans, FP64 for FP64
template <typename R>
struct LocalT {
  using type = double;
};
template <>
struct LocalT<float> {
  using type = int;
};

// 16-byte vector of the plan's real type
template <typename R>
using Vec = typename std::conditional<std::is_same<R, float>::value, float4, double2>::type;
template <typename R>
constexpr int kPerVec = 16 / int(sizeof(R));

// per-atom record: 3 coordinates (FP32: fixed-point integers in float
// bits), KC charges, zero padding to whole 16-byte vectors
template <typename R, int KC>
__host__ __device__ constexpr int rec_words() {
  return (3 + KC + kPerVec<R> - 1) / kPerVec<R> * kPerVec<R>;
}

// accumulator row (cell order): KC potentials, 3 force components, zero
// padding to whole 16-byte vectors.  The backward's rows hold dL/dq (KC)
// and dL/dr (3), and its second record per atom gphi (KC) and gF (3) in the
// same layout.
template <typename R, int KC>
__host__ __device__ constexpr int acc_words() {
  return (KC + 3 + kPerVec<R> - 1) / kPerVec<R> * kPerVec<R>;
}

// stage words per atom: the candidates' test coordinates (4) during the
// sweep, the chunk's own records (RW, and AW upstream words in the
// backward) during a drain
template <typename R, int KC, bool BW>
__host__ __device__ constexpr int stage_words() {
  return BW ? rec_words<R, KC>() + acc_words<R, KC>() : (rec_words<R, KC>() > 4 ? rec_words<R, KC>() : 4);
}

template <typename R, int KC, bool BW>
__host__ __device__ constexpr size_t warp_smem_bytes() {
  // queue [32][queue_stride] of 16-bit entries, stage [32][stage_words] R,
  // half-shell starts and ends [2][14] and queue offsets [33] int (padded
  // to 256 bytes)
  return size_t(32) * queue_stride<BW>() * 2 + size_t(32) * stage_words<R, KC, BW>() * sizeof(R) + 256;
}
static_assert(size_t(32) * queue_stride<false>() * 2 % 16 == 0 && size_t(32) * queue_stride<true>() * 2 % 16 == 0,
              "aligned stage");

int channel_class(int K) { return K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : kRsMaxK; }

template <typename R>
__device__ inline void store_vec(R* p, const R (&v)[kPerVec<R>]) {
  if constexpr (std::is_same<R, float>::value)
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}

template <typename R, int W>
__device__ inline void load_words(const R* __restrict__ p, R (&v)[W]) {
#pragma unroll
  for (int k = 0; k < W; k += kPerVec<R>) {
    const Vec<R> x = *reinterpret_cast<const Vec<R>*>(p + k);
    if constexpr (std::is_same<R, float>::value) {
      v[k] = x.x;
      v[k + 1] = x.y;
      v[k + 2] = x.z;
      v[k + 3] = x.w;
    } else {
      v[k] = x.x;
      v[k + 1] = x.y;
    }
  }
}

// row += (p_0 .. p_{KC-1}, fx, fy, fz): FP32 as 16-byte vector atomics,
// FP64 one atomic per word (channels past K skipped)
template <typename R, int KC>
__device__ inline void add_row(R* row, const R (&p)[KC], R fx, R fy, R fz, int K) {
  constexpr int AW = acc_words<R, KC>();
  if constexpr (std::is_same<R, float>::value) {
    float v[AW];
#pragma unroll
    for (int w = 0; w < AW; ++w) v[w] = 0.f;
#pragma unroll
    for (int c = 0; c < KC; ++c) v[c] = p[c];
    v[KC] = fx;
    v[KC + 1] = fy;
    v[KC + 2] = fz;
#pragma unroll
    for (int w = 0; w < AW; w += 4)
      atomicAdd(reinterpret_cast<float4*>(row + w), make_float4(v[w], v[w + 1], v[w + 2], v[w + 3]));
  } else {
#pragma unroll
    for (int c = 0; c < KC; ++c)
      if (c < K) atomicAdd(row + c, p[c]);
    atomicAdd(row + KC, fx);
    atomicAdd(row + KC + 1, fy);
    atomicAdd(row + KC + 2, fz);
  }
}

// cell of a wrapped position (count and rank within the cell).  With ufix
// (FP32 plans) also the fixed-point cell-local coordinates and the cell,
// ufix[i] = (u_x, u_y, u_z, cell), so that the scatter needs no FP64
// arithmetic: the position along each lattice vector, in units of the
// list cell's edge / 2^kFixBits, is rounded once to a 64-bit integer W
// (for a box one FP64 product r_d (n_c[d] 2^kFixBits / L_d)), whose high
// bits give the cell (wrapped mod n_c) and whose low kFixBits bits the
// coordinate; FP64 runs at a small fraction of the FP32 rate here.  FP64
// plans: fractional coordinates s = r H^-1 wrapped by floor, the cell from
// s n_c (boxes take the diagonal of H^-1 alone: the off-diagonal terms are
// exact zeros).
template <typename PosT>
__global__ void k_rs_bin(int64_t n, const PosT* __restrict__ pos, RealSpaceGeom g, int* __restrict__ cell_of,
                         int* __restrict__ rank, int* __restrict__ count, int4* __restrict__ ufix,
                         int* __restrict__ err) {
  double scale[3], abox[3];   // n_c 2^kFixBits, and for boxes times the diagonal of H^-1
  for (int d = 0; d < 3; ++d) {
    scale[d] = double(g.nc[d]) * double(1 << kFixBits);
    abox[d] = g.hinv[4 * d] * scale[d];
  }
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    double r[3];
    for (int d = 0; d < 3; ++d) {
      r[d] = double(pos[3 * i + d]);
      if (((__double_as_longlong(r[d]) >> 52) & 0x7FF) == 0x7FF) {
        atomicCAS(err, 0, PSWF_ENONFINITE);
        r[d] = 0.0;
      }
    }
    int ci[3], u[3];
    if (ufix) {
      for (int d = 0; d < 3; ++d) {
        const double v = g.tric ? (r[0] * g.hinv[d] + r[1] * g.hinv[3 + d] + r[2] * g.hinv[6 + d]) * scale[d]
                                : r[d] * abox[d];
        const long long w = __double2ll_rn(v);
        const long long ct = w >> kFixBits;   // floor(w / 2^kFixBits)
        u[d] = int(w & ((1LL << kFixBits) - 1));
        int c = int(ct);
        if (ct < 0 || ct >= g.nc[d]) {
          c = int(ct % g.nc[d]);
          c += c < 0 ? g.nc[d] : 0;
        }
        ci[d] = c;
      }
    } else {
      for (int d = 0; d < 3; ++d) {
        const double sv = g.tric ? r[0] * g.hinv[d] + r[1] * g.hinv[3 + d] + r[2] * g.hinv[6 + d]
                                 : r[d] * g.hinv[4 * d];   // in box fractions
        const double fs = sv - floor(sv);                  // [0, 1]
        const int c = int(fs * g.nc[d]);
        ci[d] = c < 0 ? 0 : (c >= g.nc[d] ? g.nc[d] - 1 : c);
      }
    }
    const int cell = (ci[2] * g.nc[1] + ci[1]) * g.nc[0] + ci[0];
    cell_of[i] = cell;
    rank[i] = atomicAdd(count + cell, 1);
    if (ufix) ufix[i] = make_int4(u[0], u[1], u[2], cell);
  }
}

// FP32 scatter from k_rs_bin's ufix: test coordinates t = u . (edges /
// 2^kFixBits) in FP32, records as whole 16-byte vectors, zeroed accumulator
// rows.  ew[9] = the list cell's edge vectors per fixed-point step.
struct EdgeStep {
  float ew[9];
};
__global__ void k_rs_scatter_fix(int64_t n, int K, int rw, const float* __restrict__ q, EdgeStep es,
                                 const int4* __restrict__ ufix, const int* __restrict__ rank,
                                 const int* __restrict__ cell_start, float4* __restrict__ lchk,
                                 float* __restrict__ rec, int* __restrict__ perm, float4* __restrict__ acc, int aw) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int4 u = ufix[i];
    const int64_t dst = int64_t(cell_start[u.w]) + rank[i];
    if (!in_bounds(dst, n, kBoundsRsScatter)) continue;
    const float fu[3] = {float(u.x), float(u.y), float(u.z)};
    float t[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = fmaf(fu[0], es.ew[k], fmaf(fu[1], es.ew[3 + k], fu[2] * es.ew[6 + k]));
    lchk[dst] = make_float4(t[0], t[1], t[2], 0.0f);
    float4* r4 = reinterpret_cast<float4*>(rec + dst * rw);
    for (int w = 0; w < rw; w += 4) {
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int x = w + e;
        v[e] = x < 3 ? __int_as_float(x == 0 ? u.x : (x == 1 ? u.y : u.z))
                     : (x - 3 < K ? q[int64_t(x - 3) * n + i] : 0.0f);
      }
      r4[w / 4] = make_float4(v[0], v[1], v[2], v[3]);
    }
    perm[dst] = int(i);
    for (int w = 0; w < aw; w += 4) acc[(dst * aw + w) / 4] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
}

// FP32 scatter in two passes (random 16-byte and 4-byte stores to the
// sorted arrays fill partial sectors, which cost DRAM read-modify-writes
// once the arrays exceed L2).  k_rs_scatter_rec moves each atom's
// fixed-point coordinates, original index and charges as one aligned record
// [4 + 4 ceil(K / 4)] words to its slot in the backward's record area (row
// stride aw words); k_rs_unpack then writes the test coordinates, records,
// order and zeroed accumulator rows in slot order, coalesced.
__global__ void k_rs_scatter_rec(int64_t n, int K, int aw, const float* __restrict__ q,
                                 const int4* __restrict__ ufix, const int* __restrict__ rank,
                                 const int* __restrict__ cell_start, float4* __restrict__ brec) {
  const int nq4 = (K + 3) / 4;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int4 u = ufix[i];
    const int64_t dst = int64_t(cell_start[u.w]) + rank[i];
    if (!in_bounds(dst, n, kBoundsRsScatter)) continue;
    float4* r = brec + dst * (aw / 4);
    r[0] = make_float4(__int_as_float(u.x), __int_as_float(u.y), __int_as_float(u.z), __int_as_float(int(i)));
    for (int c4 = 0; c4 < nq4; ++c4) {
      const int c = 4 * c4;
      r[1 + c4] = make_float4(q[int64_t(c) * n + i], c + 1 < K ? q[int64_t(c + 1) * n + i] : 0.0f,
                              c + 2 < K ? q[int64_t(c + 2) * n + i] : 0.0f, c + 3 < K ? q[int64_t(c + 3) * n + i] : 0.0f);
    }
  }
}

__global__ void k_rs_unpack(int64_t n, int K, int rw, int aw, EdgeStep es, const float* __restrict__ brec,
                            float4* __restrict__ lchk, float* __restrict__ rec, int* __restrict__ perm,
                            float4* __restrict__ acc) {
  for (int64_t m = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; m < n; m += int64_t(gridDim.x) * blockDim.x) {
    const float* rf = brec + m * aw;
    const float4 h = reinterpret_cast<const float4*>(rf)[0];
    const float fu[3] = {float(__float_as_int(h.x)), float(__float_as_int(h.y)), float(__float_as_int(h.z))};
    float t[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = fmaf(fu[0], es.ew[k], fmaf(fu[1], es.ew[3 + k], fu[2] * es.ew[6 + k]));
    lchk[m] = make_float4(t[0], t[1], t[2], 0.0f);
    float4* r4 = reinterpret_cast<float4*>(rec + m * rw);
    for (int w = 0; w < rw; w += 4) {
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int x = w + e;
        v[e] = x < 3 ? (x == 0 ? h.x : (x == 1 ? h.y : h.z)) : (x - 3 < K ? rf[x + 1] : 0.0f);
      }
      r4[w / 4] = make_float4(v[0], v[1], v[2], v[3]);
    }
    perm[m] = __float_as_int(h.w);
    for (int w = 0; w < aw; w += 4) acc[(m * aw + w) / 4] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
}

// FP64 plans: cell-local test coordinates [nmax][4] and records [nmax][rw]
// (exact coordinates, charges), the original index, and zeroed accumulator
// rows [nmax][aw]
template <typename PosT, typename R>
__global__ void k_rs_scatter(int64_t n, int K, int rw, const PosT* __restrict__ pos, const R* __restrict__ q,
                             RealSpaceGeom g, const int* __restrict__ cell_of, const int* __restrict__ rank,
                             const int* __restrict__ cell_start, R* __restrict__ lchk, R* __restrict__ rec,
                             int* __restrict__ perm, R* __restrict__ acc, int aw) {
  static_assert(std::is_same<R, double>::value, "FP32 plans scatter with k_rs_scatter_fix");
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int cell = cell_of[i];
    const int64_t dst = int64_t(cell_start[cell]) + rank[i];
    if (!in_bounds(dst, n, kBoundsRsScatter)) continue;
    int ci[3] = {cell % g.nc[0], (cell / g.nc[0]) % g.nc[1], cell / (g.nc[0] * g.nc[1])};
    R* r = rec + dst * rw;
    double x[3];
    for (int d = 0; d < 3; ++d) {
      x[d] = double(pos[3 * i + d]);
      if (((__double_as_longlong(x[d]) >> 52) & 0x7FF) == 0x7FF) x[d] = 0.0;
    }
    double u[3];   // position in the list cell, in units of its edges (0 .. 1)
    for (int d = 0; d < 3; ++d) {
      const double s = x[0] * g.hinv[d] + x[1] * g.hinv[3 + d] + x[2] * g.hinv[6 + d];
      u[d] = (s - floor(s)) * g.nc[d] - ci[d];
      r[d] = u[d];
    }
    R t4[4] = {R(0), R(0), R(0), R(0)};   // Cartesian, from the list cell's corner
    for (int k = 0; k < 3; ++k) t4[k] = R(u[0] * g.cw[k] + u[1] * g.cw[3 + k] + u[2] * g.cw[6 + k]);
    const R a2[2] = {t4[0], t4[1]}, b2[2] = {t4[2], R(0)};
    store_vec<R>(lchk + 4 * dst, a2);
    store_vec<R>(lchk + 4 * dst + 2, b2);
    for (int w = 3; w < rw; ++w) r[w] = w - 3 < K ? q[int64_t(w - 3) * n + i] : R(0);
    perm[dst] = int(i);
    if (acc) {
      const R z[kPerVec<R>] = {};
      for (int w = 0; w < aw; w += kPerVec<R>) store_vec<R>(acc + dst * aw + w, z);
    }
  }
}

template <typename R>
struct PairArgs {
  RealSpaceGeom g;
  int64_t n;
  int K, deg;
  const int* cell_start;
  const R* lchk;     // [nmax][4]
  const R* rec;      // [nmax][rec_words]
  const int* pch;
  const R* coef;     // [6][kMultSeg][deg + 1]
  R* acc;            // [nmax][acc_words], zeroed
  const R* brec;     // backward: [nmax][acc_words] gphi, gF per atom (cell order)
  const double* g_energy;   // backward: [K] or null
  int* err;
};

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

template <typename R>
__device__ inline void coords(const R* v, typename LocalT<R>::type& x, typename LocalT<R>::type& y,
                              typename LocalT<R>::type& z) {
  if constexpr (std::is_same<R, float>::value) {
    x = __float_as_int(v[0]);
    y = __float_as_int(v[1]);
    z = __float_as_int(v[2]);
  } else {
    x = v[0];
    y = v[1];
    z = v[2];
  }
}

// KC channels per pair evaluation, fully unrolled (channels past K carry
// zero charges); NC coefficients per mollifier piece (zero-padded, NC =
// deg + 1 for the common degrees, so the Horner chains have no idle step).
// The coefficient table in shared memory is [exponent][coefficient][piece]
// of scalars: the 32 pieces lie in 32 banks, so a warp's loads are free of
// bank conflicts whichever pieces its lanes need.  BW: the same sweep and
// drain evaluate the backward (a.brec holds each atom's upstream gphi and gF
// in cell order; the rows receive dL/dq and dL/dr).
template <typename R, int NC, int KC, bool TRIC, bool BW>
__global__ void __launch_bounds__(kRsThreads, 2) k_rs_pairs(PairArgs<R> a) {
  using L = typename LocalT<R>::type;
  constexpr int RW = rec_words<R, KC>();
  constexpr int AW = acc_words<R, KC>();
  constexpr int SW = stage_words<R, KC, BW>();
  constexpr int QS = queue_stride<BW>();
  extern __shared__ __align__(16) unsigned char rs_smem[];
  R* coefs = reinterpret_cast<R*>(rs_smem);   // [6][NC][kMultSeg]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  R* shv = reinterpret_cast<R*>(rs_smem + size_t(6) * kMultSeg * NC * sizeof(R));   // [kHalf][4] neighbour shifts
  unsigned char* wbase = rs_smem + size_t(6) * kMultSeg * NC * sizeof(R) + kHalf * 4 * sizeof(R) +
                         size_t(warp) * warp_smem_bytes<R, KC, BW>();
  uint16_t* queues = reinterpret_cast<uint16_t*>(wbase);                        // [32][QS]
  uint16_t* queue = queues + lane * QS;                                         // this lane's column
  R* stage = reinterpret_cast<R*>(wbase + 32 * QS * 2);   // [32][4] candidates or [32][SW] records
  int* nbs = reinterpret_cast<int*>(stage + 32 * SW);                           // [kHalf] neighbour starts
  int* nbe = nbs + kHalf;                                                       // [kHalf] ends
  int* pref = nbe + kHalf;                                                      // [33] queue offsets
  {
    for (int t = threadIdx.x; t < 6 * kMultSeg * NC; t += blockDim.x) {
      const int seg = t % kMultSeg, k = (t / kMultSeg) % NC, row = t / (kMultSeg * NC);
      coefs[t] = k <= a.deg ? a.coef[(size_t(row) * kMultSeg + seg) * (a.deg + 1) + k] : R(0);
    }
    // the neighbour o's corner relative to a cell's corner: o . (a_d / n_c)
    // (list cells are congruent, so also across the periodic boundary)
    if (threadIdx.x < kHalf) {
      const int o = kSelf + threadIdx.x;
      const double od[3] = {double(o % 3 - 1), double((o / 3) % 3 - 1), double(o / 9 - 1)};
      for (int k = 0; k < 3; ++k)
        shv[4 * threadIdx.x + k] = R(od[0] * a.g.cw[k] + od[1] * a.g.cw[3 + k] + od[2] * a.g.cw[6 + k]);
      shv[4 * threadIdx.x + 3] = R(0);
    }
  }
  __syncthreads();

  const RealSpaceGeom& g = a.g;
  const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
  const R rc2 = R(g.r_c * g.r_c), inv_rc = R(1.0 / g.r_c);
  // list-cell edge vectors per unit of the exact coordinates (FP32: one
  // fixed-point step; FP64: one edge); a box uses the diagonal only
  R ew[9];
  const double us = std::is_same<R, float>::value ? 1.0 / double(1 << kFixBits) : 1.0;
  for (int k = 0; k < 9; ++k) ew[k] = R(g.cw[k] * us);
  int prow[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) prow[c] = c < a.K ? a.pch[c] - 1 : 0;
  R* const accp = a.acc;
  R gEc[KC];   // backward: upstream gradient of the channel energies
#pragma unroll
  for (int c = 0; c < KC; ++c) gEc[c] = (BW && c < a.K && a.g_energy) ? R(a.g_energy[c]) : R(0);

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
      {
        const Vec<R> v = reinterpret_cast<const Vec<R>*>(a.lchk + 4 * int64_t(i))[0];
        xi = v.x;
        yi = v.y;
        if constexpr (std::is_same<R, float>::value)
          zi = v.z;
        else
          zi = a.lchk[4 * int64_t(i) + 2];
      }
      int len = 0;

      // the half shell's atom ranges, one lane each; the cell itself from
      // this chunk on (earlier atoms pair with it from their own chunk)
      if (lane < kHalf) {
        const int o = kSelf + lane;
        const int od[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
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
          atomicCAS(a.err, 0, PSWF_ECELL);
          b1 = b0;
        }
        if (lane == 0 && b1 > b0) b0 = base;
        nbs[lane] = b0;
        nbe[lane] = b1;
      }
      __syncwarp();

      // Balanced drain: the 32 lanes' queues, concatenated in lane order,
      // are cut into 32 ranges of equal length, one per lane.  A lane walks
      // its range in order, crossing from one queue (one atom i) to the
      // next; the i side of the pairs stays in registers until it crosses,
      // and is then added to i's accumulator row.  The j side goes to j's
      // row with vector atomics at once.
      auto drain = [&]() {
        int incl = len;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, off);
          if (lane >= off) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        pref[lane + 1] = incl;
        if (lane == 0) pref[0] = 0;
        // the chunk's own records, one per slot, for the lanes that cross
        // into another atom's queue (the stage is free between sweeps)
        if (lane < m) {
          R rs[RW];
          load_words<R, RW>(a.rec + int64_t(base + lane) * RW, rs);
#pragma unroll
          for (int w = 0; w < RW; w += kPerVec<R>) {
            R v[kPerVec<R>];
#pragma unroll
            for (int e = 0; e < kPerVec<R>; ++e) v[e] = rs[w + e];
            store_vec<R>(stage + lane * SW + w, v);
          }
          if constexpr (BW) {
            R bs[AW];
            load_words<R, AW>(a.brec + int64_t(base + lane) * AW, bs);
#pragma unroll
            for (int w = 0; w < AW; w += kPerVec<R>) {
              R v[kPerVec<R>];
#pragma unroll
              for (int e = 0; e < kPerVec<R>; ++e) v[e] = bs[w + e];
              store_vec<R>(stage + lane * SW + RW + w, v);
            }
          }
        }
        __syncwarp();
        const int e0 = (lane * total) >> 5, e1 = ((lane + 1) * total) >> 5;
        if (e0 < e1) {
          int mo = 0;   // the queue holding entry e0: the last one starting at or before it
#pragma unroll
          for (int step = 16; step > 0; step >>= 1)
            if (pref[mo + step] <= e0) mo += step;
          int t = e0 - pref[mo], tend = pref[mo + 1] - pref[mo];
          int io = base + mo / G;
          io = in_bounds(io, a.n, kBoundsRsPair) ? io : 0;   // checked build: a bad index reads row 0
          R ro[RW], bo[BW ? AW : 1];
          load_words<R, RW>(stage + (mo / G) * SW, ro);
          if constexpr (BW) load_words<R, AW>(stage + (mo / G) * SW + RW, bo);
          L ix, iy, iz;
          coords<R>(ro, ix, iy, iz);
          // the i side: phi_i (forward) or dL/dq_i (backward) partial sums,
          // and F_i or dL/dr_i
          R ph[KC];
#pragma unroll
          for (int c = 0; c < KC; ++c) ph[c] = R(0);
          R fx = 0, fy = 0, fz = 0;
          // software-pipelined: the next entry's record is fetched while the
          // current pair is evaluated (the records come from L2)
          uint32_t en = queues[mo * QS + t];
          int jn = nbs[en >> kCellBits] + int(en & (kMaxCellAtoms - 1));
          jn = in_bounds(jn, a.n, kBoundsRsPair) ? jn : 0;
          R rn[RW], bn[BW ? AW : 1];
          load_words<R, RW>(a.rec + int64_t(jn) * RW, rn);
          if constexpr (BW) load_words<R, AW>(a.brec + int64_t(jn) * AW, bn);
          for (int e = e0; e < e1; ++e) {
            R rj[RW], bj[BW ? AW : 1];
#pragma unroll
            for (int w = 0; w < RW; ++w) rj[w] = rn[w];
            if constexpr (BW) {
#pragma unroll
              for (int w = 0; w < AW; ++w) bj[w] = bn[w];
            }
            const int j = jn;
            const int o = kSelf + int(en >> kCellBits);
            const bool more = e + 1 < e1;
            int mn = mo, tn = t + 1;
            if (more) {
              if (tn == tend) {   // on to the next non-empty queue
                do {
                  ++mn;
                } while (pref[mn + 1] == pref[mn]);
                tn = 0;
              }
              en = queues[mn * QS + tn];
              jn = nbs[en >> kCellBits] + int(en & (kMaxCellAtoms - 1));
              jn = in_bounds(jn, a.n, kBoundsRsPair) ? jn : 0;
              load_words<R, RW>(a.rec + int64_t(jn) * RW, rn);
              if constexpr (BW) load_words<R, AW>(a.brec + int64_t(jn) * AW, bn);
            }
            const int o3 = o / 3;
            const int ox = o - 3 * o3 - 1, oy = o3 - 3 * (o3 / 3) - 1, oz = o3 / 3 - 1;
            L jx, jy, jz;
            coords<R>(rj, jx, jy, jz);
            R du0, du1, du2;   // displacement r_j - r_i in list-cell units
            if constexpr (std::is_same<R, float>::value) {
              du0 = __int2float_rn(jx + ox * (1 << kFixBits) - ix);
              du1 = __int2float_rn(jy + oy * (1 << kFixBits) - iy);
              du2 = __int2float_rn(jz + oz * (1 << kFixBits) - iz);
            } else {
              du0 = jx + ox - ix;
              du1 = jy + oy - iy;
              du2 = jz + oz - iz;
            }
            R dx, dy, dz;
            if constexpr (TRIC) {
              dx = du0 * ew[0] + du1 * ew[3] + du2 * ew[6];
              dy = du0 * ew[1] + du1 * ew[4] + du2 * ew[7];
              dz = du0 * ew[2] + du1 * ew[5] + du2 * ew[8];
            } else {
              dx = du0 * ew[0];
              dy = du1 * ew[4];
              dz = du2 * ew[8];
            }
            const R r2 = dx * dx + dy * dy + dz * dz;
            // atoms within one fixed-point step of each other (their FP32 test
            // coordinates may still differ) count as coincident: excluded
            if (r2 > R(0)) {
              const R inv_r = inv_sqrt(r2);
              const R r = r2 * inv_r;
              const R ir2 = inv_r * inv_r, ir4 = ir2 * ir2;
              R x = r * inv_rc;
              if (x >= R(1)) x = R(1) - R(1e-7);
              int seg = int(x * R(kMultSeg));
              if (seg > kMultSeg - 1) seg = kMultSeg - 1;
              const R sv = R(2) * (x * R(kMultSeg) - R(seg)) - R(1);
              // forward: pj = q_i^c f_p (phi_j), g = the force on i (F_j -= g);
              // backward: pj = dL/dq_j^c, g = dL/dr_i (dL/dr_j -= g)
              R pj[KC];
              R gx, gy, gz;
              if constexpr (!BW) {
                R fsum = 0;   // sum_c q_i^c q_j^c f_p'(r)
#pragma unroll
                for (int c = 0; c < KC; ++c) {
                  R cf[NC];
                  const R* cp = coefs + prow[c] * NC * kMultSeg + seg;
#pragma unroll
                  for (int k = 0; k < NC; ++k) cf[k] = cp[k * kMultSeg];
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
                  const R fc = one_m * rp;
                  const R qj = rj[3 + c];
                  ph[c] += qj * fc;
                  pj[c] = ro[3 + c] * fc;
                  fsum -= ro[3 + c] * qj * (dG * inv_rc + R(p) * one_m * inv_r) * rp;
                }
                const R sc = fsum * inv_r;
                gx = sc * dx;
                gy = sc * dy;
                gz = sc * dz;
              } else {
                // the vector-Jacobian product of (E_c, phi, F) for upstream
                // (g_E, g_phi, g_F), per pair: with d = r_i - r_j, f = f_p,
                // h = -f'/r, h' = dh/dr and u = (gF_i - gF_j) . d,
                //   dL/dq_i^c += (g_E q_j + gphi_j) f + q_j h u  (j: i <-> j)
                //   dL/dr_i  += [-sum_c (g_E q_i q_j + gphi_i q_j + gphi_j q_i) h
                //               + sum_c q_i q_j h' u / r] d + sum_c q_i q_j h (gF_i - gF_j)
                // and dL/dr_j the opposite (the force term's Jacobian is
                // w I + (w'/r) d d^T); G_p with two derivatives
                const R dg0 = bo[KC] - bj[KC], dg1 = bo[KC + 1] - bj[KC + 1], dg2 = bo[KC + 2] - bj[KC + 2];
                const R u = -(dx * dg0 + dy * dg1 + dz * dg2);   // (dx, dy, dz) = r_j - r_i
                const R dsx = R(2 * kMultSeg) * inv_rc;          // d sv / d r
                R scal = 0, w = 0;
#pragma unroll
                for (int c = 0; c < KC; ++c) {
                  const R* cp = coefs + prow[c] * NC * kMultSeg + seg;
                  R g0 = cp[(NC - 1) * kMultSeg], g1 = R(0), g2 = R(0);   // G, G' and G'' / 2 in sv
#pragma unroll
                  for (int k = NC - 2; k >= 0; --k) {
                    g2 = g2 * sv + g1;
                    g1 = g1 * sv + g0;
                    g0 = g0 * sv + cp[k * kMultSeg];
                  }
                  const R Gr = g1 * dsx, Grr = R(2) * g2 * dsx * dsx;   // dG/dr, d2G/dr2
                  const int p = prow[c] + 1;
                  const R rp = ((p & 1) ? inv_r : R(1)) * ((p & 2) ? ir2 : R(1)) * ((p & 4) ? ir4 : R(1));
                  const R f = (R(1) - g0) * rp;
                  const R f1 = -Gr * rp - R(p) * f * inv_r;
                  const R f2 = -Grr * rp + R(2 * p) * Gr * rp * inv_r + R(p * (p + 1)) * f * ir2;
                  const R h = -f1 * inv_r, h1 = -f2 * inv_r + f1 * ir2;
                  const R qi = ro[3 + c], qj = rj[3 + c], gpi = bo[c], gpj = bj[c];
                  ph[c] += (gEc[c] * qj + gpj) * f + qj * h * u;
                  pj[c] = (gEc[c] * qi + gpi) * f + qi * h * u;
                  scal += -(gEc[c] * qi * qj + gpi * qj + gpj * qi) * h + qi * qj * h1 * u * inv_r;
                  w += qi * qj * h;
                }
                gx = w * dg0 - scal * dx;
                gy = w * dg1 - scal * dy;
                gz = w * dg2 - scal * dz;
              }
              fx += gx;
              fy += gy;
              fz += gz;
              add_row<R, KC>(accp + int64_t(j) * AW, pj, -gx, -gy, -gz, a.K);
            }
            if (!more || mn != mo) {   // atom io is done in this range
              add_row<R, KC>(accp + int64_t(io) * AW, ph, fx, fy, fz, a.K);
              if (more) {
                mo = mn;
                tend = pref[mo + 1] - pref[mo];
                io = base + mo / G;
                io = in_bounds(io, a.n, kBoundsRsPair) ? io : 0;
                load_words<R, RW>(stage + (mo / G) * SW, ro);
                if constexpr (BW) load_words<R, AW>(stage + (mo / G) * SW + RW, bo);
                coords<R>(ro, ix, iy, iz);
#pragma unroll
                for (int c = 0; c < KC; ++c) ph[c] = R(0);
                fx = fy = fz = R(0);
              }
            }
            t = tn;
          }
        }
        __syncwarp();   // the queues and offsets are rewritten next
        len = 0;
      };

      for (int s = 0; s < kHalf; ++s) {
        const R ax = xi - shv[4 * s], ay = yi - shv[4 * s + 1], az = zi - shv[4 * s + 2];
        const int b0 = nbs[s], b1 = nbe[s];
        const uint32_t tag = uint32_t(s) << kCellBits;
        const int jlo = s == 0 ? i + 1 : 0;   // within the cell: j > i only
        for (int jb = b0; jb < b1; jb += 32) {
          if (__reduce_max_sync(0xffffffffu, len) > queue_cap<BW>() - 32) drain();
          const int cnt = min(32, b1 - jb);
          // one coalesced load of up to 32 candidates into the warp's stage
          if (lane < cnt)
            reinterpret_cast<Vec<R>*>(stage)[(4 / kPerVec<R>) * lane] =
                reinterpret_cast<const Vec<R>*>(a.lchk)[(4 / kPerVec<R>) * (int64_t(jb) + lane)];
          if constexpr (!std::is_same<R, float>::value)
            if (lane < cnt) stage[4 * lane + 2] = a.lchk[4 * (int64_t(jb) + lane) + 2];
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
              // r2 = 0 only for a coincident atom, which the sum excludes
              if (r2 < rc2 && r2 > R(0) && jb + jj >= jlo) queue[len++] = uint16_t(tag | uint32_t(jb - b0 + jj));
            }
          }
          __syncwarp();
        }
      }
      drain();
      __syncwarp();   // nbs / nbe are rewritten for the next chunk
    }
  }
}

// Sum of products q phi per thread.  FP32: double-float (a float sum and
// its running rounding error by TwoSum, each product split exactly by an
// FMA), merged across the warp in that form and converted to FP64 once per
// warp, since FP64 runs at a small fraction of the FP32 rate here.  FP64:
// plain FP64.
template <typename R>
struct EnergyAcc {
  double s = 0.0;
  __device__ void add_prod(R a, R b) { s += double(a) * double(b); }
  __device__ void warp_reduce() {
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __device__ double value() const { return s; }
};
template <>
struct EnergyAcc<float> {
  float s = 0.0f, e = 0.0f;
  __device__ void add(float x) {
    const float t = s + x;
    const float bp = t - s;
    e += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ void add_prod(float a, float b) {
    const float p = a * b;
    e += fmaf(a, b, -p);
    add(p);
  }
  __device__ void warp_reduce() {
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_down_sync(0xffffffffu, s, o), oe = __shfl_down_sync(0xffffffffu, e, o);
      add(os);
      e += oe;
    }
  }
  __device__ double value() const { return double(s) + double(e); }
};

// accumulator rows (cell order) to the caller's layouts, phi real [K][n]
// and forces real [n][3] (either may be null), and the channel energies
// E_c = 1/2 sum_i q_i^c phi_i^c (EnergyAcc per thread, FP64 block sums, one
// atomic per block and channel).  Threads walk the atoms in their original order: atom i's row
// is the scatter's slot cell_start[cell_of[i]] + rank[i], so the writes are
// coalesced and each row is one or two whole sectors read.
template <typename R, int KC>
__global__ void __launch_bounds__(kRsThreads) k_rs_finish(int64_t n, int K, const R* __restrict__ acc,
                                                          const R* __restrict__ q, const int* __restrict__ cell_of,
                                                          const int* __restrict__ rank,
                                                          const int* __restrict__ cell_start, R* __restrict__ phi,
                                                          R* __restrict__ forces, double* __restrict__ energy) {
  constexpr int AW = acc_words<R, KC>();
  __shared__ double part[kRsWarps][KC];
  EnergyAcc<R> e[KC];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t m = int64_t(cell_start[cell_of[i]]) + rank[i];
    if (!in_bounds(m, n, kBoundsRsFinish)) continue;
    R row[AW];
    load_words<R, AW>(acc + m * AW, row);
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      if (c >= K) break;
      e[c].add_prod(q[int64_t(c) * n + i], row[c]);
      if (phi) phi[int64_t(c) * n + i] = row[c];
    }
    if (forces) {
      forces[3 * i] = row[KC];
      forces[3 * i + 1] = row[KC + 1];
      forces[3 * i + 2] = row[KC + 2];
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    e[c].warp_reduce();
    if (lane == 0) part[warp][c] = e[c].value();
  }
  __syncthreads();
  if (threadIdx.x < KC && threadIdx.x < K) {
    double t = 0.0;
    for (int w = 0; w < kRsWarps; ++w) t += part[w][threadIdx.x];
    if (t != 0.0) atomicAdd(energy + threadIdx.x, 0.5 * t);
  }
}

// Direct mode: one thread per atom i, every atom j in shared-memory tiles,
// every image n H of the image table.  Both atoms are wrapped into the
// primary cell; a FP32 test on the wrapped Cartesian positions selects the
// pairs closer than r_c, whose displacement is then formed in FP64 and
// rounded once.
constexpr int kDirectThreads = 128;

template <typename PosT>
__device__ inline void wrapped(const PosT* __restrict__ pos, int64_t i, const RealSpaceGeom& g, double (&x)[3],
                               int* err) {
  double r[3];
  for (int d = 0; d < 3; ++d) {
    r[d] = double(pos[3 * i + d]);
    if (((__double_as_longlong(r[d]) >> 52) & 0x7FF) == 0x7FF) {
      if (err) atomicCAS(err, 0, PSWF_ENONFINITE);
      r[d] = 0.0;
    }
  }
  double s[3];
  for (int d = 0; d < 3; ++d) {
    s[d] = r[0] * g.hinv[d] + r[1] * g.hinv[3 + d] + r[2] * g.hinv[6 + d];
    s[d] -= floor(s[d]);
  }
  for (int k = 0; k < 3; ++k) x[k] = s[0] * g.h[k] + s[1] * g.h[3 + k] + s[2] * g.h[6 + k];
}

template <typename R, typename PosT, int NC, int KC>
__global__ void __launch_bounds__(kDirectThreads) k_rs_direct(int64_t n, int K, const PosT* __restrict__ pos,
                                                              const R* __restrict__ q, RealSpaceGeom g,
                                                              const int* __restrict__ pch,
                                                              const R* __restrict__ coef_src, int deg,
                                                              double* __restrict__ energy, R* __restrict__ phi,
                                                              R* __restrict__ forces, int* __restrict__ err) {
  constexpr int NV = NC / kPerVec<R>;
  extern __shared__ __align__(16) unsigned char rs_smem[];
  Vec<R>* coefv = reinterpret_cast<Vec<R>*>(rs_smem);                          // [6][NV][kMultSeg]
  double* img = reinterpret_cast<double*>(rs_smem + size_t(6) * kMultSeg * NC * sizeof(R));   // [nimg][3]
  const int nimages = (2 * g.nimg[0] + 1) * (2 * g.nimg[1] + 1) * (2 * g.nimg[2] + 1);
  double* tpos = img + 3 * nimages;                                            // [kDirectThreads][3]
  R* tq = reinterpret_cast<R*>(tpos + 3 * kDirectThreads);                     // [KC][kDirectThreads]
  {
    R* cs = reinterpret_cast<R*>(rs_smem);
    for (int t = threadIdx.x; t < 6 * kMultSeg * NC; t += blockDim.x) {
      const int e = t % kPerVec<R>, seg = (t / kPerVec<R>) % kMultSeg, v = (t / (kPerVec<R> * kMultSeg)) % NV,
                row = t / (kPerVec<R> * kMultSeg * NV);
      const int k = v * kPerVec<R> + e;
      cs[t] = k <= deg ? coef_src[(size_t(row) * kMultSeg + seg) * (deg + 1) + k] : R(0);
    }
    for (int t = threadIdx.x; t < nimages; t += blockDim.x) {
      const int n0 = t % (2 * g.nimg[0] + 1) - g.nimg[0];
      const int n1 = (t / (2 * g.nimg[0] + 1)) % (2 * g.nimg[1] + 1) - g.nimg[1];
      const int n2 = t / ((2 * g.nimg[0] + 1) * (2 * g.nimg[1] + 1)) - g.nimg[2];
      for (int k = 0; k < 3; ++k) img[3 * t + k] = n0 * g.h[k] + n1 * g.h[3 + k] + n2 * g.h[6 + k];
    }
  }
  const R rc2 = R(g.r_c * g.r_c), inv_rc = R(1.0 / g.r_c);
  int prow[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) prow[c] = c < K ? pch[c] - 1 : 0;
  const int64_t i = blockIdx.x * int64_t(kDirectThreads) + threadIdx.x;
  const bool own = i < n;
  double xi[3] = {0.0, 0.0, 0.0};
  if (own) wrapped(pos, i, g, xi, err);
  R qi[KC], ph[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    qi[c] = own && c < K ? q[int64_t(c) * n + i] : R(0);
    ph[c] = R(0);
  }
  R fx = 0, fy = 0, fz = 0;
  for (int64_t j0 = 0; j0 < n; j0 += kDirectThreads) {
    __syncthreads();   // the previous tile is consumed (and the tables are written)
    const int64_t jl = j0 + threadIdx.x;
    if (jl < n) {
      double xj[3];
      wrapped(pos, jl, g, xj, nullptr);
      for (int k = 0; k < 3; ++k) tpos[3 * threadIdx.x + k] = xj[k];
#pragma unroll
      for (int c = 0; c < KC; ++c) tq[c * kDirectThreads + threadIdx.x] = c < K ? q[int64_t(c) * n + jl] : R(0);
    }
    __syncthreads();
    const int cnt = int(n - j0 < kDirectThreads ? n - j0 : int64_t(kDirectThreads));
    if (!own) continue;
    for (int jj = 0; jj < cnt; ++jj) {
      const double b0 = tpos[3 * jj] - xi[0], b1 = tpos[3 * jj + 1] - xi[1], b2 = tpos[3 * jj + 2] - xi[2];
      for (int t = 0; t < nimages; ++t) {
        const float tx = float(b0 + img[3 * t]), ty = float(b1 + img[3 * t + 1]), tz = float(b2 + img[3 * t + 2]);
        const float t2 = tx * tx + ty * ty + tz * tz;
        if (!(t2 < float(rc2) * 1.0001f)) continue;   // FP32 test with margin; the exact test follows
        const R dx = R(b0 + img[3 * t]), dy = R(b1 + img[3 * t + 1]), dz = R(b2 + img[3 * t + 2]);
        const R r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < rc2) || !(r2 > R(0))) continue;   // outside r_c, or the atom itself
        const R inv_r = inv_sqrt(r2);
        const R r = r2 * inv_r;
        const R ir2 = inv_r * inv_r, ir4 = ir2 * ir2;
        R x = r * inv_rc;
        if (x >= R(1)) x = R(1) - R(1e-7);
        int seg = int(x * R(kMultSeg));
        if (seg > kMultSeg - 1) seg = kMultSeg - 1;
        const R sv = R(2) * (x * R(kMultSeg) - R(seg)) - R(1);
        R fsum = 0;
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          R cf[NC];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const Vec<R> cv = coefv[(prow[c] * NV + v) * kMultSeg + seg];
            if constexpr (std::is_same<R, float>::value) {
              cf[4 * v] = cv.x;
              cf[4 * v + 1] = cv.y;
              cf[4 * v + 2] = cv.z;
              cf[4 * v + 3] = cv.w;
            } else {
              cf[2 * v] = cv.x;
              cf[2 * v + 1] = cv.y;
            }
          }
          R Gv = cf[NC - 1], dG = R(0);
#pragma unroll
          for (int k = NC - 2; k >= 0; --k) {
            dG = dG * sv + Gv;
            Gv = Gv * sv + cf[k];
          }
          dG *= R(2 * kMultSeg);
          const int p = prow[c] + 1;
          const R rp = ((p & 1) ? inv_r : R(1)) * ((p & 2) ? ir2 : R(1)) * ((p & 4) ? ir4 : R(1));
          const R one_m = R(1) - Gv;
          const R qj = tq[c * kDirectThreads + jj];
          ph[c] += qj * one_m * rp;
          fsum -= qi[c] * qj * (dG * inv_rc + R(p) * one_m * inv_r) * rp;
        }
        const R sc = fsum * inv_r;
        fx += sc * dx;
        fy += sc * dy;
        fz += sc * dz;
      }
    }
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    if (c >= K) break;
    double e = own ? 0.5 * double(qi[c]) * double(ph[c]) : 0.0;
    for (int off = 16; off > 0; off >>= 1) e += __shfl_down_sync(0xffffffffu, e, off);
    if (lane == 0 && e != 0.0) atomicAdd(energy + c, e);
    if (own && phi) phi[int64_t(c) * n + i] = ph[c];
  }
  if (own && forces) {
    forces[3 * i] = fx;
    forces[3 * i + 1] = fy;
    forces[3 * i + 2] = fz;
  }
}

template <typename R, typename PosT, int NC, int KC>
cudaError_t launch_direct_k(const RealSpaceArgs& a, cudaStream_t s) {
  const RealSpaceGeom& g = a.geo;
  const int nimages = (2 * g.nimg[0] + 1) * (2 * g.nimg[1] + 1) * (2 * g.nimg[2] + 1);
  const size_t smem = size_t(6) * kMultSeg * NC * sizeof(R) + size_t(nimages) * 3 * sizeof(double) +
                      size_t(kDirectThreads) * 3 * sizeof(double) + size_t(KC) * kDirectThreads * sizeof(R);
  const cudaError_t ea = cudaFuncSetAttribute(k_rs_direct<R, PosT, NC, KC>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (ea != cudaSuccess) return ea;
  const int blocks = int((a.n + kDirectThreads - 1) / kDirectThreads);
  k_rs_direct<R, PosT, NC, KC><<<blocks, kDirectThreads, smem, s>>>(
      a.n, a.K, static_cast<const PosT*>(a.pos), static_cast<const R*>(a.q), g, a.pch,
      static_cast<const R*>(a.coef_g), a.deg_g, a.energy, static_cast<R*>(a.phi), static_cast<R*>(a.forces), a.err);
  return cudaGetLastError();
}

template <typename R, typename PosT, int NC>
cudaError_t launch_direct(const RealSpaceArgs& a, cudaStream_t s) {
  switch (channel_class(a.K)) {
    case 1: return launch_direct_k<R, PosT, NC, 1>(a, s);
    case 2: return launch_direct_k<R, PosT, NC, 2>(a, s);
    case 4: return launch_direct_k<R, PosT, NC, 4>(a, s);
    case 8: return launch_direct_k<R, PosT, NC, 8>(a, s);
    default: return launch_direct_k<R, PosT, NC, kRsMaxK>(a, s);
  }
}

// ---- backward of the real-space complement ------------------------------------
// Vector-Jacobian product of (E_c, phi_i^c, F_i) for upstream (gE_c, gphi_i^c,
// gF_i), summed per atom over its neighbours (each pair seen from both of its
// atoms, so no atomics).  With d = r_i - r_j, r = |d|, f = f_p(r), h = -f'/r
// and h' = dh/dr per channel:
//   dL/dq_i^c = gE_c phi_i^c + sum_j gphi_j^c f + sum_j q_j^c h (gF_i - gF_j) . d
//   dL/dr_i   = sum_j [ -sum_c (gE_c q_i^c q_j^c + gphi_i^c q_j^c + gphi_j^c q_i^c) h
//                       + (w' / r) d . (gF_i - gF_j) ] d + w (gF_i - gF_j),
//   w = sum_c q_i^c q_j^c h,  w' = sum_c q_i^c q_j^c h'
// (the force term's Jacobian is w I + (w'/r) d d^T), so G_p is evaluated with
// its first two derivatives.  Direct mode (cells too small for a list): one
// thread per atom over every atom and image.  With a cell list the pair
// kernel's backward mode evaluates the same terms once per pair.
constexpr int kRsBwThreads = 128;

template <typename R>
struct RsBwAcc {
  R phi, psi, tq;
};

template <typename R, int NC, int KC>
__device__ inline void rs_bw_pair(const R (&d)[3], R r2, const R* __restrict__ cs, const int (&prow)[KC], R inv_rc,
                                  const R (&qi)[KC], const R (&gpi)[KC], const R (&gEc)[KC], const R (&gFi)[3],
                                  const R* qj, const R* gpj, const R (&gFj)[3], RsBwAcc<R> (&acc)[KC], R (&gr)[3]) {
  const R inv_r = inv_sqrt(r2);
  const R r = r2 * inv_r;
  R x = r * inv_rc;
  if (x >= R(1)) x = R(1) - R(1e-7);
  int seg = int(x * R(kMultSeg));
  if (seg > kMultSeg - 1) seg = kMultSeg - 1;
  const R sv = R(2) * (x * R(kMultSeg) - R(seg)) - R(1);
  const R dsx = R(2 * kMultSeg) * inv_rc;   // d sv / d r
  const R dg[3] = {gFi[0] - gFj[0], gFi[1] - gFj[1], gFi[2] - gFj[2]};
  const R ddg = d[0] * dg[0] + d[1] * dg[1] + d[2] * dg[2];
  R scal = 0, w = 0;
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    const R* cf = cs + (prow[c] * kMultSeg + seg) * NC;
    R g0 = cf[NC - 1], g1 = 0, g2 = 0;   // G, G' and G'' / 2 in sv
#pragma unroll
    for (int k = NC - 2; k >= 0; --k) {
      g2 = g2 * sv + g1;
      g1 = g1 * sv + g0;
      g0 = g0 * sv + cf[k];
    }
    const R Gr = g1 * dsx, Grr = R(2) * g2 * dsx * dsx;   // dG/dr, d2G/dr2
    const int p = prow[c] + 1;
    const R ir2 = inv_r * inv_r;
    const R rp = ((p & 1) ? inv_r : R(1)) * ((p & 2) ? ir2 : R(1)) * ((p & 4) ? ir2 * ir2 : R(1));
    const R om = R(1) - g0;
    const R f = om * rp;
    const R f1 = -Gr * rp - R(p) * om * rp * inv_r;
    const R f2 = -Grr * rp + R(2 * p) * Gr * rp * inv_r + R(p * (p + 1)) * om * rp * ir2;
    const R h = -f1 * inv_r, h1 = -f2 * inv_r + f1 * ir2;
    const R qq = qi[c] * qj[c];
    acc[c].phi += qj[c] * f;
    acc[c].psi += gpj[c] * f;
    acc[c].tq += qj[c] * h * ddg;
    scal += -(gEc[c] * qq + gpi[c] * qj[c] + gpj[c] * qi[c]) * h + qq * h1 * ddg * inv_r;
    w += qq * h;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) gr[k] += scal * d[k] + w * dg[k];
}

template <typename R, typename PosT, int NC, int KC>
__global__ void __launch_bounds__(kRsBwThreads) k_rs_bw(RealSpaceBwArgs a) {
  extern __shared__ __align__(16) unsigned char bw_smem[];
  R* cs = reinterpret_cast<R*>(bw_smem);   // [6][kMultSeg][NC]
  double* img = reinterpret_cast<double*>(bw_smem + (size_t(6) * kMultSeg * NC * sizeof(R) + 15) / 16 * 16);
  const RealSpaceGeom& g = a.geo;
  const R* coef = static_cast<const R*>(a.coef_g);
  for (int t = threadIdx.x; t < 6 * kMultSeg * NC; t += blockDim.x) {
    const int k = t % NC, rs = t / NC;   // rs = row * kMultSeg + seg
    cs[t] = k <= a.deg_g ? coef[size_t(rs) * (a.deg_g + 1) + k] : R(0);
  }
  const int nimages = (2 * g.nimg[0] + 1) * (2 * g.nimg[1] + 1) * (2 * g.nimg[2] + 1);
  for (int t = threadIdx.x; t < nimages; t += blockDim.x) {
    const int n0 = t % (2 * g.nimg[0] + 1) - g.nimg[0];
    const int n1 = (t / (2 * g.nimg[0] + 1)) % (2 * g.nimg[1] + 1) - g.nimg[1];
    const int n2 = t / ((2 * g.nimg[0] + 1) * (2 * g.nimg[1] + 1)) - g.nimg[2];
    for (int k = 0; k < 3; ++k) img[3 * t + k] = n0 * g.h[k] + n1 * g.h[3 + k] + n2 * g.h[6 + k];
  }
  __syncthreads();
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= a.n) return;
  const int64_t n = a.n;
  const PosT* pos = static_cast<const PosT*>(a.pos);
  const R* q = static_cast<const R*>(a.q);
  const R* gphi = static_cast<const R*>(a.g_phi);
  const R* gF = static_cast<const R*>(a.g_forces);
  int prow[KC];
  R qi[KC], gpi[KC], gEc[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    prow[c] = c < a.K ? a.pch[c] - 1 : 0;
    qi[c] = c < a.K ? q[int64_t(c) * n + i] : R(0);
    gpi[c] = (c < a.K && gphi) ? gphi[int64_t(c) * n + i] : R(0);
    gEc[c] = (c < a.K && a.g_energy) ? R(a.g_energy[c]) : R(0);
  }
  const R gFi[3] = {gF ? gF[3 * i] : R(0), gF ? gF[3 * i + 1] : R(0), gF ? gF[3 * i + 2] : R(0)};
  double xi[3];
  wrapped(pos, i, g, xi, a.err);
  const double rc2 = g.r_c * g.r_c;
  const R inv_rc = R(1.0 / g.r_c);
  RsBwAcc<R> acc[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) acc[c] = {R(0), R(0), R(0)};
  R gr[3] = {0, 0, 0};
  auto visit = [&](int64_t j, const double* shift) {
    double xj[3];
    wrapped(pos, j, g, xj, nullptr);
    const double dd[3] = {xi[0] - xj[0] - shift[0], xi[1] - xj[1] - shift[1], xi[2] - xj[2] - shift[2]};
    const double r2d = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
    if (!(r2d < rc2) || !(r2d > 0.0)) return;   // outside r_c, or the atom itself
    const R d[3] = {R(dd[0]), R(dd[1]), R(dd[2])};
    R qj[KC], gpj[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      qj[c] = c < a.K ? q[int64_t(c) * n + j] : R(0);
      gpj[c] = (c < a.K && gphi) ? gphi[int64_t(c) * n + j] : R(0);
    }
    const R gFj[3] = {gF ? gF[3 * j] : R(0), gF ? gF[3 * j + 1] : R(0), gF ? gF[3 * j + 2] : R(0)};
    rs_bw_pair<R, NC, KC>(d, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], cs, prow, inv_rc, qi, gpi, gEc, gFi, qj, gpj,
                          gFj, acc, gr);
  };
  for (int64_t j = 0; j < n; ++j)
    for (int t = 0; t < nimages; ++t) visit(j, img + 3 * t);
  R* gq = static_cast<R*>(a.grad_q);
  R* gp = static_cast<R*>(a.grad_pos);
#pragma unroll
  for (int c = 0; c < KC; ++c)
    if (c < a.K && gq) gq[int64_t(c) * n + i] = gEc[c] * acc[c].phi + acc[c].psi + acc[c].tq;
  if (gp) {
    gp[3 * i] = gr[0];
    gp[3 * i + 1] = gr[1];
    gp[3 * i + 2] = gr[2];
  }
}

template <typename R, typename PosT, int NC, int KC>
cudaError_t launch_bw_k(const RealSpaceBwArgs& a, cudaStream_t s) {
  const RealSpaceGeom& g = a.geo;
  const int nimages = (2 * g.nimg[0] + 1) * (2 * g.nimg[1] + 1) * (2 * g.nimg[2] + 1);
  const size_t smem = (size_t(6) * kMultSeg * NC * sizeof(R) + 15) / 16 * 16 + size_t(nimages) * 3 * sizeof(double);
  const cudaError_t ea =
      cudaFuncSetAttribute(k_rs_bw<R, PosT, NC, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (ea != cudaSuccess) return ea;
  const int blocks = int((a.n + kRsBwThreads - 1) / kRsBwThreads);
  k_rs_bw<R, PosT, NC, KC><<<blocks, kRsBwThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename R, typename PosT, int NC>
cudaError_t launch_bw(const RealSpaceBwArgs& a, cudaStream_t s) {
  switch (channel_class(a.K)) {
    case 1: return launch_bw_k<R, PosT, NC, 1>(a, s);
    case 2: return launch_bw_k<R, PosT, NC, 2>(a, s);
    case 4: return launch_bw_k<R, PosT, NC, 4>(a, s);
    case 8: return launch_bw_k<R, PosT, NC, 8>(a, s);
    default: return launch_bw_k<R, PosT, NC, kRsMaxK>(a, s);
  }
}

// backward of the cell-list path: each atom's upstream gphi (KC) and gF (3)
// to a record in cell order (the accumulator rows are cleared by a memset:
// zero rows written at random slots would cost a second random sector per
// atom)
template <typename R, int KC>
__global__ void __launch_bounds__(kRsThreads) k_rs_bw_scatter(int64_t n, int K, const R* __restrict__ g_phi,
                                                              const R* __restrict__ g_forces,
                                                              const int* __restrict__ cell_of,
                                                              const int* __restrict__ rank,
                                                              const int* __restrict__ cell_start,
                                                              R* __restrict__ brec) {
  constexpr int AW = acc_words<R, KC>();
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t m = int64_t(cell_start[cell_of[i]]) + rank[i];
    if (!in_bounds(m, n, kBoundsRsScatter)) continue;
    R v[AW];
#pragma unroll
    for (int w = 0; w < AW; ++w) v[w] = R(0);
#pragma unroll
    for (int c = 0; c < KC; ++c)
      if (c < K && g_phi) v[c] = g_phi[int64_t(c) * n + i];
    if (g_forces) {
      v[KC] = g_forces[3 * i];
      v[KC + 1] = g_forces[3 * i + 1];
      v[KC + 2] = g_forces[3 * i + 2];
    }
#pragma unroll
    for (int w = 0; w < AW; w += kPerVec<R>) {
      R x[kPerVec<R>];
#pragma unroll
      for (int e = 0; e < kPerVec<R>; ++e) x[e] = v[w + e];
      store_vec<R>(brec + m * AW + w, x);
    }
  }
}

// rows (dL/dq, dL/dr in cell order) to grad_q real [K][n] and grad_pos real
// [n][3] (either may be null), atoms in their original order
template <typename R, int KC>
__global__ void __launch_bounds__(kRsThreads) k_rs_bw_finish(int64_t n, int K, const R* __restrict__ acc,
                                                             const int* __restrict__ cell_of,
                                                             const int* __restrict__ rank,
                                                             const int* __restrict__ cell_start,
                                                             R* __restrict__ grad_q, R* __restrict__ grad_pos) {
  constexpr int AW = acc_words<R, KC>();
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t m = int64_t(cell_start[cell_of[i]]) + rank[i];
    if (!in_bounds(m, n, kBoundsRsFinish)) continue;
    R row[AW];
    load_words<R, AW>(acc + m * AW, row);
    if (grad_q) {
#pragma unroll
      for (int c = 0; c < KC; ++c)
        if (c < K) grad_q[int64_t(c) * n + i] = row[c];
    }
    if (grad_pos) {
      grad_pos[3 * i] = row[KC];
      grad_pos[3 * i + 1] = row[KC + 1];
      grad_pos[3 * i + 2] = row[KC + 2];
    }
  }
}

template <typename R>
cudaError_t launch_bw_rows(const RealSpaceBwArgs& a, R* brec, R* acc, bool finish, int blocks, cudaStream_t s) {
  const R* gp = static_cast<const R*>(a.g_phi);
  const R* gf = static_cast<const R*>(a.g_forces);
  R* gq = static_cast<R*>(a.grad_q);
  R* gr = static_cast<R*>(a.grad_pos);
#define PSWF_RS_BW_ROWS(KC)                                                                                        \
  if (finish)                                                                                                      \
    k_rs_bw_finish<R, KC><<<blocks, kRsThreads, 0, s>>>(a.n, a.K, acc, a.cell_of, a.rank, a.cell_start, gq, gr);    \
  else                                                                                                             \
    k_rs_bw_scatter<R, KC><<<blocks, kRsThreads, 0, s>>>(a.n, a.K, gp, gf, a.cell_of, a.rank, a.cell_start, brec)
  if (!finish) {
    const int aw = channel_class(a.K) == 1 ? acc_words<R, 1>()
                   : channel_class(a.K) == 2 ? acc_words<R, 2>()
                   : channel_class(a.K) == 4 ? acc_words<R, 4>()
                   : channel_class(a.K) == 8 ? acc_words<R, 8>()
                                             : acc_words<R, kRsMaxK>();
    const cudaError_t e = cudaMemsetAsync(acc, 0, size_t(a.n) * aw * sizeof(R), s);
    if (e != cudaSuccess) return e;
  }
  switch (channel_class(a.K)) {
    case 1: PSWF_RS_BW_ROWS(1); break;
    case 2: PSWF_RS_BW_ROWS(2); break;
    case 4: PSWF_RS_BW_ROWS(4); break;
    case 8: PSWF_RS_BW_ROWS(8); break;
    default: PSWF_RS_BW_ROWS(kRsMaxK); break;
  }
#undef PSWF_RS_BW_ROWS
  return cudaGetLastError();
}

__global__ void k_rs_total(int K, double* __restrict__ energy) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int c = 0; c < K; ++c) t += energy[c];
    energy[K] = t;
  }
}

template <typename R, int NC, int KC, bool TRIC, bool BW>
cudaError_t launch_pairs_t(const PairArgs<R>& pa, int ncell, cudaStream_t s) {
  const size_t smem = size_t(6) * kMultSeg * NC * sizeof(R) + kHalf * 4 * sizeof(R) +
                      size_t(kRsWarps) * warp_smem_bytes<R, KC, BW>();
  // set on every launch: the opt-in is per device and cheap
  const cudaError_t ea = cudaFuncSetAttribute(k_rs_pairs<R, NC, KC, TRIC, BW>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (ea != cudaSuccess) return ea;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rs_pairs<R, NC, KC, TRIC, BW>, kRsThreads, smem);
  const int64_t want = (int64_t(ncell) + kRsWarps - 1) / kRsWarps;
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(std::max(nsm, 1)) * std::max(per_sm, 1))));
  k_rs_pairs<R, NC, KC, TRIC, BW><<<blocks, kRsThreads, smem, s>>>(pa);
  return cudaGetLastError();
}

// general cells transform displacements with the full 3 x 3 edge matrix
template <typename R, int NC, int KC, bool BW>
cudaError_t launch_pairs_k(const PairArgs<R>& pa, int ncell, cudaStream_t s) {
  return pa.g.tric ? launch_pairs_t<R, NC, KC, true, BW>(pa, ncell, s)
                   : launch_pairs_t<R, NC, KC, false, BW>(pa, ncell, s);
}

template <typename R, int NC, bool BW>
cudaError_t launch_pairs_nc(const PairArgs<R>& pa, int ncell, cudaStream_t s) {
  switch (channel_class(pa.K)) {
    case 1: return launch_pairs_k<R, NC, 1, BW>(pa, ncell, s);
    case 2: return launch_pairs_k<R, NC, 2, BW>(pa, ncell, s);
    case 4: return launch_pairs_k<R, NC, 4, BW>(pa, ncell, s);
    case 8: return launch_pairs_k<R, NC, 8, BW>(pa, ncell, s);
    default: return launch_pairs_k<R, NC, kRsMaxK, BW>(pa, ncell, s);
  }
}

// coefficients per piece: the FP32 fit's usual degree 6 exactly, else padded
// (the planner's degree is at most kMaxMultDeg = 16)
template <typename R, bool BW>
cudaError_t launch_pairs(const PairArgs<R>& pa, int ncell, cudaStream_t s) {
  static_assert(kMaxMultDeg + 1 <= 17, "coefficient rows");
  if constexpr (std::is_same<R, float>::value) {
    if (pa.deg + 1 <= 7) return launch_pairs_nc<R, 7, BW>(pa, ncell, s);
    if constexpr (!BW)
      if (pa.deg + 1 <= 8) return launch_pairs_nc<R, 8, BW>(pa, ncell, s);
  }
  return launch_pairs_nc<R, 17, BW>(pa, ncell, s);
}

template <typename R>
int record_words(int K) {
  switch (channel_class(K)) {
    case 1: return rec_words<R, 1>();
    case 2: return rec_words<R, 2>();
    case 4: return rec_words<R, 4>();
    case 8: return rec_words<R, 8>();
    default: return rec_words<R, kRsMaxK>();
  }
}

template <typename R>
int accumulator_words(int K) {
  switch (channel_class(K)) {
    case 1: return acc_words<R, 1>();
    case 2: return acc_words<R, 2>();
    case 4: return acc_words<R, 4>();
    case 8: return acc_words<R, 8>();
    default: return acc_words<R, kRsMaxK>();
  }
}

template <typename R>
cudaError_t launch_finish(const RealSpaceArgs& a, const R* acc, int blocks, cudaStream_t s) {
  const R* q = static_cast<const R*>(a.q);
  R* phi = static_cast<R*>(a.phi);
  R* forces = static_cast<R*>(a.forces);
#define PSWF_RS_FINISH(KC)                                                                                     \
  k_rs_finish<R, KC><<<blocks, kRsThreads, 0, s>>>(a.n, a.K, acc, q, a.cell_of, a.rank, a.cell_start, phi, forces, \
                                                   a.energy)
  switch (channel_class(a.K)) {
    case 1: PSWF_RS_FINISH(1); break;
    case 2: PSWF_RS_FINISH(2); break;
    case 4: PSWF_RS_FINISH(4); break;
    case 8: PSWF_RS_FINISH(8); break;
    default: PSWF_RS_FINISH(kRsMaxK); break;
  }
#undef PSWF_RS_FINISH
  return cudaGetLastError();
}

}  // namespace

size_t real_space_bytes_per_atom(int K, int real_size) {
  // test coordinates, records, accumulator rows, the backward's upstream records
  return real_size == 4 ? (4 + size_t(record_words<float>(K)) + size_t(2 * accumulator_words<float>(K))) * 4
                        : (4 + size_t(record_words<double>(K)) + size_t(2 * accumulator_words<double>(K))) * 8;
}

bool real_space_geometry_cell(const double H[9], double r_c, RealSpaceGeom& g) {
  const double det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                     H[2] * (H[3] * H[7] - H[4] * H[6]);
  if (!(std::fabs(det) > 0.0) || !(r_c > 0.0)) return false;
  // H^-1 = adj(H) / det
  const double inv[9] = {(H[4] * H[8] - H[5] * H[7]) / det, (H[2] * H[7] - H[1] * H[8]) / det,
                         (H[1] * H[5] - H[2] * H[4]) / det, (H[5] * H[6] - H[3] * H[8]) / det,
                         (H[0] * H[8] - H[2] * H[6]) / det, (H[2] * H[3] - H[0] * H[5]) / det,
                         (H[3] * H[7] - H[4] * H[6]) / det, (H[1] * H[6] - H[0] * H[7]) / det,
                         (H[0] * H[4] - H[1] * H[3]) / det};
  bool diag = true;
  double height[3];
  g.direct = 0;
  for (int d = 0; d < 3; ++d) {
    // height across the faces spanned by the other two vectors: V / |a_e x a_f|
    const double* ae = H + 3 * ((d + 1) % 3);
    const double* af = H + 3 * ((d + 2) % 3);
    const double cx = ae[1] * af[2] - ae[2] * af[1], cy = ae[2] * af[0] - ae[0] * af[2],
                 cz = ae[0] * af[1] - ae[1] * af[0];
    height[d] = std::fabs(det) / std::sqrt(cx * cx + cy * cy + cz * cz);
    const double ncd = std::floor(height[d] / r_c);
    if (ncd > 1e6) return false;
    if (!(ncd >= 3.0)) g.direct = 1;
    g.nc[d] = ncd >= 3.0 ? int(ncd) : 1;
    for (int k = 0; k < 3; ++k)
      if (k != d && H[3 * d + k] != 0.0) diag = false;
  }
  long long nimages = 1;
  for (int d = 0; d < 3; ++d) {
    if (g.direct) g.nc[d] = 1;
    for (int k = 0; k < 3; ++k) {
      g.cw[3 * d + k] = H[3 * d + k] / g.nc[d];
      g.h[3 * d + k] = H[3 * d + k];
    }
    // with both atoms in the primary cell a displacement closer than r_c
    // needs |n_d| <= ceil(r_c / height_d) + 1
    g.nimg[d] = int(std::ceil(r_c / height[d])) + 1;
    nimages *= 2 * g.nimg[d] + 1;
  }
  if (g.direct && nimages > kRsDirectMaxImages) return false;
  for (int k = 0; k < 9; ++k) g.hinv[k] = inv[k];
  g.tric = diag ? 0 : 1;
  g.r_c = r_c;
  return true;
}

bool real_space_geometry(const double box[3], double r_c, RealSpaceGeom& g) {
  const double H[9] = {box[0], 0.0, 0.0, 0.0, box[1], 0.0, 0.0, 0.0, box[2]};
  return real_space_geometry_cell(H, r_c, g);
}

template <typename R>
cudaError_t real_space_run(const RealSpaceArgs& a, cudaStream_t s, int* nlaunch) {
  const RealSpaceGeom& g = a.geo;
  const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
  if (a.deg_g > kMaxMultDeg) return cudaErrorInvalidValue;
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.energy, 0, size_t(a.K + 1) * sizeof(double), s)) != cudaSuccess) return e;
  if (g.direct) {
    if (a.n > 0) {
      if constexpr (std::is_same<R, float>::value) {
        const bool wide = a.deg_g + 1 > 8;
        if (a.pos_dtype == 1)
          e = wide ? launch_direct<R, double, 20>(a, s) : launch_direct<R, double, 8>(a, s);
        else
          e = wide ? launch_direct<R, float, 20>(a, s) : launch_direct<R, float, 8>(a, s);
      } else {
        e = a.pos_dtype == 1 ? launch_direct<R, double, 18>(a, s) : launch_direct<R, float, 18>(a, s);
      }
      if (e != cudaSuccess) return e;
      ++*nlaunch;
    }
    k_rs_total<<<1, 32, 0, s>>>(a.K, a.energy);
    ++*nlaunch;
    return cudaGetLastError();
  }
  if ((e = cudaMemsetAsync(a.count, 0, size_t(ncell) * sizeof(int), s)) != cudaSuccess) return e;
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((a.n + kRsThreads - 1) / kRsThreads, 148 * 16)));
  const int rw = record_words<R>(a.K);
  const int aw = accumulator_words<R>(a.K);
  R* lchk = static_cast<R*>(a.lpos);
  R* rec = lchk + 4 * a.nmax;              // records follow the test coordinates
  R* acc = rec + int64_t(rw) * a.nmax;     // accumulator rows follow the records
  // FP32: the fixed-point coordinates wait between the bin and the scatter
  // in the accumulator rows (by original index; the records then go to the
  // backward's record area, idle during the forward, which unpack clears
  // the rows after) or, where a record does not fit an accumulator row
  // (one channel), in the backward's record area
  const bool recs = std::is_same<R, float>::value && 4 + 4 * ((a.K + 3) / 4) <= aw;
  R* brec = acc + int64_t(aw) * a.nmax;
  int4* ufix = !std::is_same<R, float>::value ? nullptr : reinterpret_cast<int4*>(recs ? acc : brec);
  if (a.n > 0) {
    if (a.pos_dtype == 1)
      k_rs_bin<double><<<blocks, kRsThreads, 0, s>>>(a.n, static_cast<const double*>(a.pos), g, a.cell_of, a.rank,
                                                     a.count, ufix, a.err);
    else
      k_rs_bin<float><<<blocks, kRsThreads, 0, s>>>(a.n, static_cast<const float*>(a.pos), g, a.cell_of, a.rank,
                                                    a.count, ufix, a.err);
    ++*nlaunch;
  }
  const int nsb = (ncell + a.scan_per_block - 1) / a.scan_per_block;
  k_scan_block_sums<<<nsb, kScanBlock, 0, s>>>(ncell, a.count, a.scan_sums, a.scan_per_block);
  k_scan_sums<<<1, 32, 0, s>>>(nsb, a.scan_sums);
  k_scan_apply<<<nsb, kScanBlock, 0, s>>>(ncell, a.count, a.scan_sums, a.scan_per_block, a.cell_start);
  *nlaunch += 3;
  if (a.n > 0) {
    if constexpr (std::is_same<R, float>::value) {
      EdgeStep es;
      for (int k = 0; k < 9; ++k) es.ew[k] = float(g.cw[k] / double(1 << kFixBits));
      if (recs) {
        k_rs_scatter_rec<<<blocks, kRsThreads, 0, s>>>(a.n, a.K, aw, static_cast<const float*>(a.q), ufix, a.rank,
                                                       a.cell_start, reinterpret_cast<float4*>(brec));
        k_rs_unpack<<<blocks, kRsThreads, 0, s>>>(a.n, a.K, rw, aw, es, brec, reinterpret_cast<float4*>(lchk), rec,
                                                  a.perm, reinterpret_cast<float4*>(acc));
        ++*nlaunch;
      } else {
        k_rs_scatter_fix<<<blocks, kRsThreads, 0, s>>>(a.n, a.K, rw, static_cast<const float*>(a.q), es, ufix,
                                                       a.rank, a.cell_start, reinterpret_cast<float4*>(lchk), rec,
                                                       a.perm, reinterpret_cast<float4*>(acc), aw);
      }
    } else if (a.pos_dtype == 1)
      k_rs_scatter<double, R><<<blocks, kRsThreads, 0, s>>>(a.n, a.K, rw, static_cast<const double*>(a.pos),
                                                            static_cast<const R*>(a.q), g, a.cell_of, a.rank,
                                                            a.cell_start, lchk, rec, a.perm, acc, aw);
    else
      k_rs_scatter<float, R><<<blocks, kRsThreads, 0, s>>>(a.n, a.K, rw, static_cast<const float*>(a.pos),
                                                           static_cast<const R*>(a.q), g, a.cell_of, a.rank,
                                                           a.cell_start, lchk, rec, a.perm, acc, aw);
    PairArgs<R> pa;
    pa.g = g;
    pa.n = a.n;
    pa.K = a.K;
    pa.deg = a.deg_g;
    pa.cell_start = a.cell_start;
    pa.lchk = lchk;
    pa.rec = rec;
    pa.pch = a.pch;
    pa.coef = static_cast<const R*>(a.coef_g);
    pa.acc = acc;
    pa.brec = nullptr;
    pa.g_energy = nullptr;
    pa.err = a.err;
    if ((e = launch_pairs<R, false>(pa, ncell, s)) != cudaSuccess) return e;
    *nlaunch += 2;
    if ((e = launch_finish<R>(a, acc, blocks, s)) != cudaSuccess) return e;
    ++*nlaunch;
  }
  k_rs_total<<<1, 32, 0, s>>>(a.K, a.energy);
  ++*nlaunch;
  return cudaGetLastError();
}

int bounds_word_real_space() { return take_bounds_word(); }

template cudaError_t real_space_run<float>(const RealSpaceArgs&, cudaStream_t, int*);
template cudaError_t real_space_run<double>(const RealSpaceArgs&, cudaStream_t, int*);

// Backward: direct mode one thread per atom over every pair and image
// (k_rs_bw); cell lists reuse the forward's list, records and test
// coordinates: the upstream gradients to records in cell order, the pair
// kernel in its backward mode, the rows to the caller's layouts.
template <typename R>
cudaError_t real_space_backward_run(const RealSpaceBwArgs& a, cudaStream_t s, int* nlaunch) {
  if (a.n == 0) return cudaSuccess;
  if (a.deg_g + 1 > 18) return cudaErrorInvalidValue;
  cudaError_t e;
  if (a.geo.direct) {
    e = a.pos_dtype == 1 ? launch_bw<R, double, 18>(a, s) : launch_bw<R, float, 18>(a, s);
    if (e == cudaSuccess) ++*nlaunch;
    return e;
  }
  const int rw = record_words<R>(a.K), aw = accumulator_words<R>(a.K);
  R* lchk = static_cast<R*>(a.lpos);
  R* rec = lchk + 4 * a.nmax;
  R* acc = rec + int64_t(rw) * a.nmax;
  R* brec = acc + int64_t(aw) * a.nmax;
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((a.n + kRsThreads - 1) / kRsThreads, 148 * 16)));
  if ((e = launch_bw_rows<R>(a, brec, acc, false, blocks, s)) != cudaSuccess) return e;
  PairArgs<R> pa;
  pa.g = a.geo;
  pa.n = a.n;
  pa.K = a.K;
  pa.deg = a.deg_g;
  pa.cell_start = a.cell_start;
  pa.lchk = lchk;
  pa.rec = rec;
  pa.pch = a.pch;
  pa.coef = static_cast<const R*>(a.coef_g);
  pa.acc = acc;
  pa.brec = brec;
  pa.g_energy = a.g_energy;
  pa.err = a.err;
  const int ncell = a.geo.nc[0] * a.geo.nc[1] * a.geo.nc[2];
  if ((e = launch_pairs<R, true>(pa, ncell, s)) != cudaSuccess) return e;
  if ((e = launch_bw_rows<R>(a, brec, acc, true, blocks, s)) != cudaSuccess) return e;
  *nlaunch += 3;
  return cudaSuccess;
}

template cudaError_t real_space_backward_run<float>(const RealSpaceBwArgs&, cudaStream_t, int*);
template cudaError_t real_space_backward_run<double>(const RealSpaceBwArgs&, cudaStream_t, int*);

}  // namespace pswf
