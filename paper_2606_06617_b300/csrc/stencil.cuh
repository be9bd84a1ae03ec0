// Tiled stencil kernels: spreading (step (i)) and the gather of potentials
// and forces.  A CTA works on one tile of kTile^3 stencil-start cells at a
// time; the tile's atoms are contiguous in the sorted arrays.  The padded
// region of a tile, S^3 grid points with S = kTile + P - 1, is the union of
// its atoms' stencils and is held in shared memory (layout: TilePad).
#pragma once

#include <type_traits>

#include "kernels.cuh"

namespace pswf {

__device__ inline int wrap_index(int v, int M) {
  while (v >= M) v -= M;
  return v;
}

// Accumulator type of the spreading region: 32-bit fixed point for the FP32
// path (see k_spread), double for the FP64 path.
template <typename R>
struct SpreadAcc {
  using T = int;
};
template <>
struct SpreadAcc<double> {
  using T = double;
};

// ---- shared-memory layout of a tile ------------------------------------------
//
// Element (x, y, z) of channel c of a padded region is at c N + z R2 + y R1 + x.
// Lane mapping: a warp is cut into slots of G lanes (G = the power of two
// >= P); the lanes of a slot are the P y-rows j of one atom's stencil in one
// channel, each lane sweeping its row's P z-planes and P x-points.  With all
// K channels of a tile staged, the slots of a warp are the channels of ONE
// atom, so the window weights are shared by the whole warp and no two lanes
// hit the same shared-memory bank (layout below).  With fewer channels than
// slots, a warp takes several atoms.
template <int P>
struct TilePad {
  static constexpr int G = P <= 4 ? 4 : P <= 8 ? 8 : 16;
  static constexpr int NS = 32 / G;     // slots per warp
  static constexpr int S = kTile + P - 1;
  static constexpr int R1 = S | 1;      // odd: the G rows of a slot fall in G banks
  static constexpr int R2 = S * R1;
  // Channel stride: N = R1 G (mod 32) puts slot s at banks R1 (G s + j), so the
  // NS slots of a warp occupy disjoint bank sets.
  static constexpr int find_n() {
    int n = S * R2;
    while (((n - R1 * G) % 32 + 32) % 32 != 0) ++n;
    return n;
  }
  static constexpr int N = find_n();
};

// Threads of the spread and gather CTAs resident on one SM: 1024 in FP32 (64
// registers a thread), 512 in FP64; split over CTAS CTAs per SM (each with
// its own padded region).
template <typename R>
constexpr int kGatherThreadsFor = sizeof(R) == 4 ? 1024 : 512;

// Per-batch window tables in shared memory: for each atom of a batch, rows
// of PW >= P entries (16-byte aligned, read as vectors): W_x, W_y, W_z and,
// for the gather, (2/h_d) dW/ds in x, y, z.  One thread per (atom, direction)
// evaluates the P pieces (coefficient reads uniform across the warp).
template <int P>
constexpr int kRowW = P <= 4 ? 4 : P <= 8 ? 8 : 16;

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename R, int P>
constexpr size_t stencil_smem_bytes(int kc, int kb, int rows, size_t acc_size) {
  return align16(size_t(kc) * TilePad<P>::N * acc_size) + size_t(kb) * (rows * kRowW<P> * sizeof(R) + 2 * sizeof(int));
}
// The gather's batch also holds each atom's charges of the staged channels
// (8 entries: the most slots a warp has).
template <typename R, int P>
constexpr size_t gather_smem_bytes(int kc, int kb) {
  return stencil_smem_bytes<R, P>(kc, kb, 6, sizeof(R)) + size_t(kb) * 8 * sizeof(R);
}

// P consecutive reals from 16-byte-aligned shared memory, as vector loads.
template <typename R, int P>
__device__ inline void lds_row(const R* p, R (&v)[P]) {
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int i = 0; i < P; i += 4) {
      const float4 t = *reinterpret_cast<const float4*>(p + i);
      v[i] = t.x;
      if (i + 1 < P) v[i + 1] = t.y;
      if (i + 2 < P) v[i + 2] = t.z;
      if (i + 3 < P) v[i + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < P; i += 2) {
      const double2 t = *reinterpret_cast<const double2*>(p + i);
      v[i] = t.x;
      if (i + 1 < P) v[i + 1] = t.y;
    }
  }
}

template <typename R>
__device__ inline void cp_async_elem(R* dst, const R* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(int(sizeof(R))) : "memory");
}
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Slot bookkeeping shared by the spread and the gather.  kc channels are
// staged; the slots of one atom are a power-of-two group of kcp >= kc slots
// (slots beyond kc idle), so xor shuffles over the slot bits reduce exactly
// over one atom's channels.
struct Slots {
  int lane, warp, nwarp, j, sbase, kcp, apw, asub, cc;
  bool used;
  template <int G, int NS>
  __device__ static Slots make(int kc) {
    Slots s;
    s.lane = threadIdx.x & 31;
    s.warp = threadIdx.x >> 5;
    s.nwarp = blockDim.x >> 5;
    const int slot = s.lane / G;
    s.j = s.lane % G;
    s.sbase = s.lane - s.j;
    s.kcp = 1;
    while (s.kcp < kc) s.kcp <<= 1;
    s.apw = NS / s.kcp;
    s.asub = slot / s.kcp;
    s.cc = slot - s.asub * s.kcp;
    s.used = s.asub < s.apw && s.cc < kc;
    return s;
  }
};

// Origin (in grid points) of tile `tile` (index within its structure).
__device__ inline void tile_origin(const Geometry& g, int tile, int& ox, int& oy, int& oz) {
  const int tx = tile % g.ntile[0], ty = (tile / g.ntile[0]) % g.ntile[1], tz = tile / (g.ntile[0] * g.ntile[1]);
  ox = tx * kTile;
  oy = ty * kTile;
  oz = tz * kTile;
}

// Fills the batch's window rows (values, and derivatives times two_h[d] =
// 2 / h_d when rows == 6), the packed local start cell and (gather) the
// original index.
template <typename R, int P, int ROWS>
__device__ inline void batch_tables(const Geometry& g, const R* two_h, int64_t nmax, int b0, int nb,
                                    int ox, int oy, int oz,
                                    const R* __restrict__ st, const uint64_t* __restrict__ scell,
                                    const int* __restrict__ sperm, const WinCoef<R>& wc, R* wts, int* loc,
                                    int* perm) {
  constexpr int PW = kRowW<P>;
  for (int t = threadIdx.x; t < nb * 3; t += blockDim.x) {
    const int a = t / 3, d = t - 3 * a;
    R* row = wts + (a * ROWS + d) * PW;
    if constexpr (ROWS == 6) {
      R w[P], dw[P];
      window_weights<R, P>(st[d * nmax + b0 + a], wc, w, dw);
      const R th = two_h[d];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        row[i] = w[i];
        row[3 * PW + i] = dw[i] * th;
      }
    } else {
      R w[P];
      window_values<R, P>(st[d * nmax + b0 + a], wc, w);
#pragma unroll
      for (int i = 0; i < P; ++i) row[i] = w[i];
    }
  }
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    int cx, cy, cz;
    unpack_cell(scell[b0 + t], cx, cy, cz);
    loc[t] = (cx - ox) | ((cy - oy) << 8) | ((cz - oz) << 16);
    if (perm) perm[t] = sperm[b0 + t];
  }
}

// Spreading (step (i)).  Work items are (tile, chunk of kc channels); the
// kc padded regions live in shared memory with the layout above.  The tile's
// atoms go in batches of kb: their window rows are tabulated, then each warp
// takes an atom (several when K is small) and lane j of slot cc adds
// q_c W_x(i) W_y(j) W_z(k) for all (i, k) of row j with shared-memory atomics
// (the warp's lanes hit 32 distinct banks).  The region is then added into
// the grid with global atomics, one warp per (channel, z) plane, lanes along
// x (neighbouring tiles overlap by P - 1 planes); the grid is zeroed before
// the launch.
//
// FP32 path: contributions are rounded to integers of a per-(tile, channel)
// fixed point 1/s and summed exactly in 32 bits.  The rounding is one FFMA
// with the constant 1.5 * 2^23 (the sum's low mantissa bits are then the
// rounded integer, exact for |value| < 2^22), so s = min(0.99 * 2^22 /
// max|q|, 0.999 * 2^31 / (1.0001 sum|q|)) keeps every contribution below 2^22
// and every grid sum below 2^31 (the window is at most 1).  FP64 path:
// double atomics.
template <typename R, int P>
constexpr size_t spread_smem_bytes(int kc, int kb) {
  return stencil_smem_bytes<R, P>(kc, kb, 3, sizeof(typename SpreadAcc<R>::T));
}

template <typename R, int P, int CTAS>
__global__ void __launch_bounds__(kGatherThreadsFor<R> / CTAS, CTAS) k_spread(Geometry g, const double* __restrict__ smol,
                                                                   int64_t nmax, const int* __restrict__ tile_start,
                                                                   const R* __restrict__ st,
                                                                   const uint64_t* __restrict__ scell,
                                                                   const R* __restrict__ sq, WinCoef<R> wc, int kc,
                                                                   int kb, R* __restrict__ grid) {
  using A = typename SpreadAcc<R>::T;
  constexpr bool kFixed = std::is_same<A, int>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  using L = TilePad<P>;
  constexpr int G = L::G, NS = L::NS, S = L::S, R1 = L::R1, R2 = L::R2, N = L::N, PW = kRowW<P>;
  A* region = reinterpret_cast<A*>(smraw);   // [kc][N]
  R* wts = reinterpret_cast<R*>(smraw + align16(size_t(kc) * N * sizeof(A)));   // [kb][3][PW]
  int* loc = reinterpret_cast<int*>(wts + kb * 3 * PW);
  __shared__ float red_sum[32][NS], red_max[32][NS];
  __shared__ float sscale[NS];
  const Slots sl = Slots::template make<G, NS>(kc);
  const int lane = sl.lane, warp = sl.warp, nwarp = sl.nwarp, j = sl.j, cc = sl.cc;
  const int nchunk = (g.K + kc - 1) / kc;
  const int ntiles = g.B * g.nts;
  const int64_t plane = int64_t(g.M[1]) * g.Mxp, chan = int64_t(g.M[2]) * plane;
  for (int item = blockIdx.x; item < ntiles * nchunk; item += gridDim.x) {
    const int tile = item / nchunk, chunk = item - tile * nchunk;
    const int a0 = tile_start[tile], a1 = tile_start[tile + 1];
    if (a0 == a1) continue;
    const int sidx = tile / g.nts;
    const int c0 = chunk * kc, nk = min(kc, g.K - c0);
    const int gc0 = sidx * g.K + c0;   // first grid channel of the item
    int ox, oy, oz;
    tile_origin(g, tile - sidx * g.nts, ox, oy, oz);
    __syncthreads();   // the previous item's flush is done with the region
    {
      const int nbytes = nk * N * int(sizeof(A));
      int4* r4 = reinterpret_cast<int4*>(region);
      for (int t = threadIdx.x; t < nbytes / 16; t += blockDim.x) r4[t] = make_int4(0, 0, 0, 0);
      int* r1 = reinterpret_cast<int*>(region);
      for (int t = (nbytes / 16) * 4 + threadIdx.x; t < nbytes / 4; t += blockDim.x) r1[t] = 0;
    }
    if constexpr (kFixed) {
      float s1[NS], mx[NS];
#pragma unroll
      for (int c = 0; c < NS; ++c) s1[c] = mx[c] = 0.0f;
      for (int a = a0 + threadIdx.x; a < a1; a += blockDim.x)
#pragma unroll
        for (int c = 0; c < NS; ++c)
          if (c < nk) {
            const float v = fabsf(float(sq[int64_t(c0 + c) * nmax + a]));
            s1[c] += v;
            mx[c] = fmaxf(mx[c], v);
          }
#pragma unroll
      for (int c = 0; c < NS; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
          s1[c] += __shfl_xor_sync(0xffffffffu, s1[c], o);
          mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
        if (lane == 0) {
          red_sum[warp][c] = s1[c];
          red_max[warp][c] = mx[c];
        }
      }
      __syncthreads();
      if (threadIdx.x < nk) {
        float tot = 0.0f, m = 0.0f;
        for (int w = 0; w < nwarp; ++w) {
          tot += red_sum[w][threadIdx.x];
          m = fmaxf(m, red_max[w][threadIdx.x]);
        }
        sscale[threadIdx.x] =
            tot > 0.0f ? fminf(0.99f * 4194304.0f / m, 0.999f * 2147483647.0f / (tot * 1.0001f)) : 1.0f;
      }
    }
    const bool use_slot = sl.used && cc < nk;
    for (int b0 = a0; b0 < a1; b0 += kb) {
      const int nb = min(kb, a1 - b0);
      __syncthreads();   // previous batch done with the tables (and sscale written)
      batch_tables<R, P, 3>(g, nullptr, nmax, b0, nb, ox, oy, oz, st, scell, nullptr, wc, wts, loc, nullptr);
      __syncthreads();
      const R qscale = kFixed && use_slot ? R(sscale[cc]) : R(1);
      for (int ab = warp * sl.apw; ab < nb; ab += nwarp * sl.apw) {
        const int al = ab + sl.asub;
        if (!(use_slot && al < nb && j < P)) continue;
        const R* wa = wts + al * 3 * PW;
        R wx[P], wz[P];
        lds_row<R, P>(wa, wx);
        lds_row<R, P>(wa + 2 * PW, wz);
        const int l = loc[al];
        A* row = region + cc * N + ((l >> 16) & 0xff) * R2 + (((l >> 8) & 0xff) + j) * R1 + (l & 0xff);
        const R qy = sq[int64_t(c0 + cc) * nmax + b0 + al] * qscale * wa[PW + j];
#pragma unroll
        for (int k = 0; k < P; ++k) {
          const R coef = qy * wz[k];
#pragma unroll
          for (int i = 0; i < P; ++i) {
            if constexpr (kFixed) {
              const float f = fmaf(float(coef), float(wx[i]), 12582912.0f);
              atomicAdd(reinterpret_cast<int*>(row) + k * R2 + i, __float_as_int(f) - 0x4B400000);
            } else {
              atomicAdd(reinterpret_cast<double*>(row) + k * R2 + i, double(coef * wx[i]));
            }
          }
        }
      }
    }
    __syncthreads();
    {
      // two rows per warp iteration (half-warps), each lane adds an x pair;
      // FP32 pairs that do not straddle the periodic wrap go as one 8-byte
      // atomic (grid rows start at even offsets, tile origins are even)
      const int half = lane >> 4, x0 = 2 * (lane & 15);
      const bool has0 = x0 < S, has1 = x0 + 1 < S;
      const int gx0 = has0 ? wrap_index(ox + x0, g.M[0]) : 0;
      const int gx1 = has1 ? wrap_index(ox + x0 + 1, g.M[0]) : 0;
      const bool pair = has1 && gx1 == gx0 + 1 && (gx0 & 1) == 0;
      for (int pl = warp; pl < nk * S; pl += nwarp) {
        const int c = pl / S, lz = pl - c * S;
        const R inv = kFixed ? R(1) / R(sscale[c]) : R(1);
        R* base = grid + (gc0 + c) * chan + wrap_index(oz + lz, g.M[2]) * plane;
        const A* src = region + c * N + lz * R2;
        if (!has0) continue;
        for (int ly = half; ly < S; ly += 2) {
          R* row = base + int64_t(wrap_index(oy + ly, g.M[1])) * g.Mxp;
          const A v0 = src[ly * R1 + x0];
          const A v1 = has1 ? src[ly * R1 + x0 + 1] : A(0);
          if constexpr (kFixed) {
            if (pair) {
              atomicAdd(reinterpret_cast<float2*>(row + gx0), make_float2(float(v0) * inv, float(v1) * inv));
              continue;
            }
          }
          atomicAdd(row + gx0, R(v0) * inv);
          if (has1) atomicAdd(row + gx1, R(v1) * inv);
        }
      }
    }
  }
}

// Spreading without shared-memory staging, for plans whose padded region does
// not fit in shared memory (FP64 with large P): one thread per sorted atom,
// global atomics.
template <typename R, int P>
__global__ void k_spread_direct(int64_t nmax, Geometry g, const int* __restrict__ soff,
                                const int* __restrict__ tile_start, const R* __restrict__ st,
                                const uint64_t* __restrict__ scell, const R* __restrict__ sq, WinCoef<R> wc,
                                R* __restrict__ grid) {
  const int64_t n = soff[g.B];
  const int64_t chan = int64_t(g.M[2]) * g.M[1] * g.Mxp;
  for (int64_t a = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; a < n; a += int64_t(gridDim.x) * blockDim.x) {
    const int sidx = find_struct(tile_start, g.nts, g.B, a);
    R wx[P], wy[P], wz[P];
    window_values<R, P>(st[a], wc, wx);
    window_values<R, P>(st[nmax + a], wc, wy);
    window_values<R, P>(st[2 * nmax + a], wc, wz);
    int cx, cy, cz;
    unpack_cell(scell[a], cx, cy, cz);
    for (int c = 0; c < g.K; ++c) {
      const R qc = sq[int64_t(c) * nmax + a];
      R* gc = grid + (int64_t(sidx) * g.K + c) * chan;
      for (int k = 0; k < P; ++k) {
        const int z = wrap_index(cz + k, g.M[2]);
        for (int j = 0; j < P; ++j) {
          const int y = wrap_index(cy + j, g.M[1]);
          const R coef = qc * wy[j] * wz[k];
          R* row = gc + (int64_t(z) * g.M[1] + y) * g.Mxp;
#pragma unroll
          for (int i = 0; i < P; ++i) atomicAdd(row + wrap_index(cx + i, g.M[0]), coef * wx[i]);
        }
      }
    }
  }
}

// Gather of phi_c = sum Psi_c W + 2 a_c Q_c and F = sum_c q_c sum Psi_c grad W
// (grad_d W = (2 / h_d) dW/ds).  Work items are (tile, chunk of kc channels);
// per item the kc padded regions of Psi are staged with asynchronous copies
// (one warp per (channel, z) plane, lanes along x) while the first batch's
// window rows are tabulated.  Lane j of slot cc sweeps row j of the atom's
// stencil in channel cc.  The four sums (phi, and the three components of
// q_c f_c) are reduced over the slot's lanes by a transposing butterfly
// (after it, lane group v of the slot holds sum v), the force components
// then over the atom's slots.  With more than one chunk the force is
// accumulated with global atomics (zeroed before the launch).
template <typename R, int P, int CTAS>
__global__ void __launch_bounds__(kGatherThreadsFor<R> / CTAS, CTAS) k_interp(int64_t nmax, Geometry g,
                                                                   const double* __restrict__ smol,
                                                                   const int* __restrict__ soff,
                                                                   const int* __restrict__ tile_start,
                                                                   const R* __restrict__ st,
                                                                   const uint64_t* __restrict__ scell,
                                                                   const R* __restrict__ sq,
                                                                   const int* __restrict__ sperm, WinCoef<R> wc,
                                                                   int kc, int kb, const R* __restrict__ grid,
                                                                   const double* __restrict__ zero_coef,
                                                                   const double* __restrict__ charges,
                                                                   R* __restrict__ phi, R* __restrict__ forces) {
  extern __shared__ __align__(16) unsigned char smraw[];
  using L = TilePad<P>;
  constexpr int G = L::G, NS = L::NS, S = L::S, R1 = L::R1, R2 = L::R2, N = L::N, PW = kRowW<P>;
  constexpr int GQ = G / 4;   // lanes per reduced sum after the butterfly
  R* region = reinterpret_cast<R*>(smraw);   // [kc][N]
  R* wts = reinterpret_cast<R*>(smraw + align16(size_t(kc) * N * sizeof(R)));   // [kb][6][PW]
  R* qs = wts + kb * 6 * PW;                                                     // [kb][8]
  int* loc = reinterpret_cast<int*>(qs + kb * 8);
  int* perm = loc + kb;
  __shared__ R two_h[3];   // 2 / h_d = 2 M_d / L_d of the item's structure
  const Slots sl = Slots::template make<G, NS>(kc);
  const int lane = sl.lane, warp = sl.warp, nwarp = sl.nwarp, j = sl.j, cc = sl.cc;
  const int nchunk = (g.K + kc - 1) / kc;
  const int jr = j < P ? j : P - 1;        // row read by lanes beyond the stencil
  const int vi = j / GQ;                   // which sum this lane ends up holding
  const int64_t n = soff[g.B];
  const int ntiles = g.B * g.nts;
  const int64_t plane = int64_t(g.M[1]) * g.Mxp, chan = int64_t(g.M[2]) * plane;
  for (int item = blockIdx.x; item < ntiles * nchunk; item += gridDim.x) {
    const int tile = item / nchunk, chunk = item - tile * nchunk;
    const int a0 = tile_start[tile], a1 = tile_start[tile + 1];
    if (a0 == a1) continue;
    const int sidx = tile / g.nts;
    const int c0 = chunk * kc, nk = min(kc, g.K - c0);
    const int gc0 = sidx * g.K + c0;   // first grid channel of the item
    int ox, oy, oz;
    tile_origin(g, tile - sidx * g.nts, ox, oy, oz);
    // (every thread is past the previous item's last table fill)
    if (threadIdx.x < 3) two_h[threadIdx.x] = R(2.0 * smol[3 * sidx + threadIdx.x]);
    __syncthreads();   // the previous item's reads of the region and tables are done
    {
      const int gx = lane < S ? wrap_index(ox + lane, g.M[0]) : 0;
      for (int pl = warp; pl < nk * S; pl += nwarp) {
        const int c = pl / S, lz = pl - c * S;
        const R* src = grid + (gc0 + c) * chan + wrap_index(oz + lz, g.M[2]) * plane + gx;
        R* dst = region + c * N + lz * R2 + lane;
        if (lane < S) {
          int gy = oy;
#pragma unroll 2
          for (int ly = 0; ly < S; ++ly, ++gy) {
            if (gy == g.M[1]) gy = 0;
            cp_async_elem(dst + ly * R1, src + int64_t(gy) * g.Mxp);
          }
        }
      }
    }
    const bool use_slot = sl.used && cc < nk;
    // zero-frequency shift 2 a_c Q_c of the lane's channel
    const R zshift = use_slot ? R(2.0 * zero_coef[gc0 + cc] * charges[2 * (gc0 + cc)]) : R(0);
    for (int b0 = a0; b0 < a1; b0 += kb) {
      const int nb = min(kb, a1 - b0);
      if (b0 != a0) __syncthreads();   // previous batch done with the tables
      batch_tables<R, P, 6>(g, two_h, nmax, b0, nb, ox, oy, oz, st, scell, sperm, wc, wts, loc, perm);
      for (int t = threadIdx.x; t < nb * nk; t += blockDim.x) {
        const int a = t / nk, c = t - a * nk;
        qs[a * 8 + c] = sq[int64_t(c0 + c) * nmax + b0 + a];
      }
      if (b0 == a0) cp_async_wait_all();
      __syncthreads();
      for (int ab = warp * sl.apw; ab < nb; ab += nwarp * sl.apw) {
        const int al_raw = ab + sl.asub;
        const bool valid = use_slot && al_raw < nb;
        const int al = min(al_raw, nb - 1);
        const R* wa = wts + al * 6 * PW;
        R wx[P], dx[P], wz[P], dz[P];
        lds_row<R, P>(wa, wx);
        lds_row<R, P>(wa + 3 * PW, dx);
        lds_row<R, P>(wa + 2 * PW, wz);
        lds_row<R, P>(wa + 5 * PW, dz);
        const R wy = j < P ? wa[PW + j] : R(0), dy = j < P ? wa[4 * PW + j] : R(0);
        const int l = loc[al];
        const R* row = region + (use_slot ? cc : 0) * N + ((l >> 16) & 0xff) * R2 + (((l >> 8) & 0xff) + jr) * R1 +
                       (l & 0xff);
        R A = 0, Az = 0, B = 0;
#pragma unroll
        for (int k = 0; k < P; ++k) {
          R sx = 0, dsx = 0;
#pragma unroll
          for (int i = 0; i < P; ++i) {
            const R v = row[k * R2 + i];
            sx += v * wx[i];
            dsx += v * dx[i];
          }
          A += sx * wz[k];
          Az += sx * dz[k];
          B += dsx * wz[k];
        }
        const R q = valid ? qs[al * 8 + cc] : R(0);
        // butterfly over the slot: (phi, q f_x, q f_y, q f_z) -> one sum per lane group
        R v;
        {
          const R v0 = A * wy, v1 = q * B * wy, v2 = q * A * dy, v3 = q * Az * wy;
          const bool hi = (j & (G / 2)) != 0;
          R k0 = hi ? v2 : v0, k1 = hi ? v3 : v1;
          const R s0 = hi ? v0 : v2, s1 = hi ? v1 : v3;
          k0 += __shfl_xor_sync(0xffffffffu, s0, G / 2);
          k1 += __shfl_xor_sync(0xffffffffu, s1, G / 2);
          const bool hi2 = (j & GQ) != 0;
          v = hi2 ? k1 : k0;
          v += __shfl_xor_sync(0xffffffffu, hi2 ? k0 : k1, GQ);
#pragma unroll
          for (int o = GQ / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        }
        // force components over the atom's slots (idle slots carry q = 0)
        R fsum = v;
        for (int o = G; o < G * sl.kcp; o <<= 1) fsum += __shfl_xor_sync(0xffffffffu, fsum, o);
        if (valid && j % GQ == 0) {
          const int o = perm[al];
          if (vi == 0) {
            if (phi) phi[int64_t(c0 + cc) * n + o] = v + zshift;
          } else if (forces && cc == 0) {
            R* fo = forces + 3 * int64_t(o) + (vi - 1);
            if (nchunk == 1)
              *fo = fsum;
            else
              atomicAdd(fo, fsum);
          }
        }
      }
    }
  }
}

}  // namespace pswf
