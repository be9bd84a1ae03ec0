// FP32 stencil kernels for stencils of up to 8 points per dimension:
// spreading of the latent charges (step (i) of "Accelerating atom-grid
// spreading with PSWFs") and the gather of potentials and forces, with up to
// four channels per work item.
//
// Both work on one tile of kTile^3 stencil-start cells at a time; the tile's
// atoms are contiguous in the sorted arrays and its padded region, S^3 grid
// points with S = kTile + P - 1, is the union of their stencils.  Per atom
// the window pieces are evaluated by the lanes that use them (piece j by
// lane j of an 8-lane group, one Horner chain per lane, coefficients held in
// registers) and passed around the group by shuffles, so no per-batch window
// tables, batch barriers or table shared memory are needed.
//
// Gather: the region holds Psi of four channels interleaved (one float4 per
// grid point, row stride R1 odd).  An 8-lane group handles one atom (four
// atoms per warp); lane j sweeps row j of the stencil (its P planes and P
// points), so one 16-byte shared load feeds the eight products (value and
// x-derivative window) of the four channels.  The eight lanes of a group hit
// eight distinct 16-byte bank groups (j R1 mod 8), so each quarter-warp load
// is one wavefront.  Seven sums per lane (four potentials and the three
// force components) are reduced over the group by a transposing butterfly.
//
// Spread: the region holds one 32-bit fixed-point accumulator per grid point
// and channel (channel planes, layout SPad); a warp takes one atom, its
// lanes being four channels x eight stencil rows, so every shared atomic of
// the warp hits 32 distinct banks.  The region is then added into the grid
// with global atomics; points that received nothing are skipped (sparse
// tiles), and the flush zeroes what it read, so the region is cleared once
// per launch rather than per work item.
#pragma once

#include "bounds.cuh"
#include "stencil.cuh"

namespace pswf {

// Tile of the t-th visit: the tiles' own order (structure-major, x fastest).
// Neighbouring tiles, whose padded regions overlap, then run close together
// in time, so their shared halo lines meet in L2.  A blocked order (z-columns
// in x-strips of four tiles) measured slower for the spread (384^3 melt: 2.01
// against 1.94 ms).
__device__ inline int tile_for_visit(const Geometry&, int t) { return t; }

// Window piece j of the lane (zero for j >= P): monomial coefficients in
// s = 2t - 1, read once per thread.
template <int P>
struct LanePiece {
  static constexpr int D = WinCoef<float>::kDeg;
  float c[D + 1];
  __device__ void load(const WinCoef<float>& wc, int j) {
#pragma unroll
    for (int n = 0; n <= D; ++n) c[n] = j < P ? wc.c[j * (D + 1) + n] : 0.0f;
  }
  __device__ float value(float t) const {
    const float s = 2.0f * t - 1.0f;
    float v = c[D];
#pragma unroll
    for (int n = D - 1; n >= 0; --n) v = fmaf(v, s, c[n]);
    return v;
  }
  // value and dW/ds
  __device__ void value_deriv(float t, float& v, float& dv) const {
    const float s = 2.0f * t - 1.0f;
    v = c[D];
    dv = 0.0f;
#pragma unroll
    for (int n = D - 1; n >= 0; --n) {
      dv = fmaf(dv, s, v);
      v = fmaf(v, s, c[n]);
    }
  }
};

// 16-byte asynchronous global-to-shared copy (both addresses 16-byte aligned).
__device__ inline void cp_async16(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

template <int P>
struct Pad4 {
  static constexpr int S = kTile + P - 1;
  static constexpr int R1 = S | 1;        // odd row stride (in float4)
  static constexpr int R2 = S * R1;       // plane stride
  static constexpr int ELEMS = S * R2;    // float4 elements of the region
};

template <int P>
constexpr size_t gather4_smem_bytes() {
  return size_t(Pad4<P>::ELEMS) * 16;
}

// ---- gather -------------------------------------------------------------------
// phi_c = sum Psi_c W + 2 a_c Q_c, F = sum_c q_c sum Psi_c grad W (grad_d W =
// (2 / h_d) dW/ds).  Work items are (tile, chunk of four channels); with
// more than one chunk the forces are accumulated with global atomics (the
// caller zeroes them).
//
// Staging: when Psi is stored as channel quadruples (psi_il, written so by
// the own inverse x pass), one 16-byte asynchronous copy per grid point.
// Otherwise a job is an x-pair of one region row; its four channels' pairs
// are read as 8-byte loads (grid rows start at even offsets and tile origins
// are even, so a pair that does not straddle the periodic wrap is aligned)
// and written as two float4 (x, then x + 1), several jobs' loads in flight
// per thread.  Atom inputs of the next group of four atoms are loaded while
// the current group is evaluated.  Window coefficients sit in shared memory
// as [n][j], so the eight lanes of a group read eight banks and the four
// groups of a warp share them.
template <int P, int NT>
__global__ void __launch_bounds__(NT, 1) k_gather4(int64_t nmax, Geometry g, const double* __restrict__ smol,
                                                   const int* __restrict__ soff, const int* __restrict__ tile_start,
                                                   const float* __restrict__ st, const uint64_t* __restrict__ scell,
                                                   const float* __restrict__ sq, const int* __restrict__ sperm,
                                                   const __grid_constant__ WinCoef<float> wc,
                                                   const float* __restrict__ grid,
                                                   const double* __restrict__ zero_coef,
                                                   const double* __restrict__ charges, float* __restrict__ phi,
                                                   float* __restrict__ forces, bool psi_il,
                                                   float* __restrict__ out_rec) {
  static_assert(P <= 8, "one 8-lane group per atom");
  using L = Pad4<P>;
  constexpr int S = L::S, R1 = L::R1, R2 = L::R2;
  constexpr int NW = NT / 32;
  constexpr int D = WinCoef<float>::kDeg;
  constexpr int NPAIR = (S + 1) / 2;     // x-pairs per region row
  constexpr int NJOB = S * S * NPAIR;    // staging jobs per item
  constexpr int U = 2;                   // staging jobs in flight per thread
  extern __shared__ __align__(16) float4 reg4[];   // [S][S][R1] x 4 channels
  __shared__ float cf_s[D + 1][8];                 // window coefficients [monomial][piece]
  __shared__ float item_s[8];                      // 2 / h_d (3), zero-frequency shifts (4)
  __shared__ int gx_s[L::S];                       // wrapped x of the region (channel-quadruple staging)
  __shared__ int64_t yoff_s[L::S], zoff_s[L::S];   // wrapped row and plane offsets
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = lane & 7, grp = lane >> 3, gbase = lane & ~7;
  const int jr = j < P ? j : P - 1;
  for (int t = threadIdx.x; t < (D + 1) * 8; t += NT) {
    const int n = t >> 3, pj = t & 7;
    cf_s[n][pj] = pj < P ? wc.c[pj * (D + 1) + n] : 0.0f;
  }
  const int nchunk = (g.K + 3) / 4;
  const int64_t n = soff[g.B];
  const int nitems = g.B * g.nts * nchunk;
  const int64_t plane = int64_t(g.M[1]) * g.Mxp, chan = int64_t(g.M[2]) * plane;
  const bool xeven = (g.M[0] & 1) == 0;
  const int64_t grid_elems = int64_t(g.B) * g.K * chan;   // reals of the grid (checked build)
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int visit = item / nchunk, chunk = item - visit * nchunk;
    const int tile = tile_for_visit(g, visit);
    const int a0 = tile_start[tile], a1 = tile_start[tile + 1];
    if (a0 == a1 || !in_bounds(a1 - 1, n, kBoundsTile) || !in_bounds(a0, n, kBoundsTile)) continue;
    const int sidx = tile / g.nts;
    const int c0 = chunk * 4, nk = min(4, g.K - c0);
    const int gc0 = sidx * g.K + c0;
    int ox, oy, oz;
    tile_origin(g, tile - sidx * g.nts, ox, oy, oz);
    __syncthreads();   // the previous item's reads of the region and item_s are done
    if (threadIdx.x < 3) {
      item_s[threadIdx.x] = float(2.0 * smol[3 * sidx + threadIdx.x]);
    } else if (threadIdx.x < 7) {
      const int c = threadIdx.x - 3;
      item_s[threadIdx.x] = c < nk ? float(2.0 * zero_coef[gc0 + c] * charges[2 * (gc0 + c)]) : 0.0f;
    }
    if (psi_il) {
      // Psi as channel quadruples: one 16-byte asynchronous copy per grid
      // point, wrapped offsets from the item's tables
      if (threadIdx.x < S) {
        gx_s[threadIdx.x] = wrap_index(ox + threadIdx.x, g.M[0]);
      } else if (threadIdx.x < 2 * S) {
        yoff_s[threadIdx.x - S] = int64_t(wrap_index(oy + threadIdx.x - S, g.M[1])) * g.Mxp;
      } else if (threadIdx.x < 3 * S) {
        zoff_s[threadIdx.x - 2 * S] = wrap_index(oz + threadIdx.x - 2 * S, g.M[2]) * plane;
      }
      __syncthreads();
      const float4* g4 = reinterpret_cast<const float4*>(grid) + int64_t(gc0 / 4) * chan;
      for (int e = threadIdx.x; e < S * S * S; e += NT) {
        const int row = e / S, x = e - row * S;
        const int lz = row / S, ly = row - lz * S;
        const int64_t srcq = zoff_s[lz] + yoff_s[ly] + gx_s[x];
        if (in_bounds(row * R1 + x, L::ELEMS, kBoundsGatherStage) &&
            in_bounds(int64_t(gc0 / 4) * chan + srcq, grid_elems / 4, kBoundsGatherGrid))
          cp_async16(reg4 + row * R1 + x, g4 + srcq);
      }
      cp_async_wait_all();
    } else {
      const float* gch = grid + int64_t(gc0) * chan;
      for (int e0 = threadIdx.x; e0 < NJOB; e0 += U * NT) {
        float2 pr[U][4];
        int dsti[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = e0 + u * NT;
          dsti[u] = -1;
#pragma unroll
          for (int c = 0; c < 4; ++c) pr[u][c] = make_float2(0.0f, 0.0f);
          if (e < NJOB) {
            const int row = e / NPAIR, x = 2 * (e - row * NPAIR);
            const int lz = row / S, ly = row - lz * S;
            dsti[u] = row * R1 + x;
            const int gx = wrap_index(ox + x, g.M[0]);
            const int64_t off = wrap_index(oz + lz, g.M[2]) * plane + int64_t(wrap_index(oy + ly, g.M[1])) * g.Mxp;
            if (!in_bounds(int64_t(gc0 + nk - 1) * chan + off + gx + 1, grid_elems, kBoundsGatherGrid)) {
              dsti[u] = -1;
            } else if (xeven && gx + 1 < g.M[0]) {
#pragma unroll
              for (int c = 0; c < 4; ++c)
                if (c < nk) pr[u][c] = __ldg(reinterpret_cast<const float2*>(gch + c * chan + off + gx));
            } else {
              const int gx1 = wrap_index(gx + 1, g.M[0]);
#pragma unroll
              for (int c = 0; c < 4; ++c)
                if (c < nk) pr[u][c] = make_float2(__ldg(gch + c * chan + off + gx), __ldg(gch + c * chan + off + gx1));
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (dsti[u] < 0) continue;
          if (!in_bounds(dsti[u] + 1, L::ELEMS + 1, kBoundsGatherStage)) continue;
          reg4[dsti[u]] = make_float4(pr[u][0].x, pr[u][1].x, pr[u][2].x, pr[u][3].x);
          if ((dsti[u] % R1) + 1 < S) reg4[dsti[u] + 1] = make_float4(pr[u][0].y, pr[u][1].y, pr[u][2].y, pr[u][3].y);
        }
      }
    }
    __syncthreads();
    const float th0 = item_s[0], th1 = item_s[1], th2 = item_s[2];
    const float zshift = j < 4 ? item_s[3 + j] : 0.0f;
    // group loop: four atoms per warp, the next group's inputs loaded ahead
    int ab = a0 + 4 * warp;
    float tnx = 0.0f, tny = 0.0f, tnz = 0.0f;
    uint64_t celln = 0;
    if (ab < a1) {
      const int a = min(ab + grp, a1 - 1);
      tnx = st[a];
      tny = st[nmax + a];
      tnz = st[2 * nmax + a];
      celln = scell[a];
    }
    for (; ab < a1; ab += 4 * NW) {
      const int a_raw = ab + grp;
      const bool valid = a_raw < a1;
      const int a = valid ? a_raw : a1 - 1;
      const float tx = tnx, ty = tny, tz = tnz;
      const uint64_t cell = celln;
      if (ab + 4 * NW < a1) {
        const int an = min(ab + 4 * NW + grp, a1 - 1);
        tnx = st[an];
        tny = st[nmax + an];
        tnz = st[2 * nmax + an];
        celln = scell[an];
      }
      float q[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) q[c] = (valid && c < nk) ? sq[int64_t(c0 + c) * nmax + a] : 0.0f;
      const int o = sperm[a];
      // window piece j in x, y, z: values and dW/ds (Horner, coefficients from shared memory)
      float wxj, dxj, wyj, dyj, wzj, dzj;
      {
        const float sx_ = 2.0f * tx - 1.0f, sy_ = 2.0f * ty - 1.0f, sz_ = 2.0f * tz - 1.0f;
        const float cD = cf_s[D][j];
        wxj = wyj = wzj = cD;
        dxj = dyj = dzj = 0.0f;
#pragma unroll
        for (int m = D - 1; m >= 0; --m) {
          const float cm = cf_s[m][j];
          dxj = fmaf(dxj, sx_, wxj);
          wxj = fmaf(wxj, sx_, cm);
          dyj = fmaf(dyj, sy_, wyj);
          wyj = fmaf(wyj, sy_, cm);
          dzj = fmaf(dzj, sz_, wzj);
          wzj = fmaf(wzj, sz_, cm);
        }
      }
      dxj *= th0;
      dyj *= th1;
      dzj *= th2;
      float wx[P], dx[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        wx[i] = __shfl_sync(0xffffffffu, wxj, gbase + i);
        dx[i] = __shfl_sync(0xffffffffu, dxj, gbase + i);
      }
      int cx, cy, cz;
      unpack_cell(cell, cx, cy, cz);
      int rbase = ((cz - oz) * S + (cy - oy) + jr) * R1 + (cx - ox);
      if (!in_bounds(rbase, L::ELEMS, kBoundsGatherRegion) ||
          !in_bounds(rbase + (P - 1) * R2 + (P - 1), L::ELEMS, kBoundsGatherRegion))
        rbase = 0;   // checked build: read a valid place instead (the result is wrong, the status says so)
      const float4* row = reg4 + rbase;
      float A[4] = {0, 0, 0, 0}, Az[4] = {0, 0, 0, 0}, B[4] = {0, 0, 0, 0};
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const float wz = __shfl_sync(0xffffffffu, wzj, gbase + k);
        const float dz = __shfl_sync(0xffffffffu, dzj, gbase + k);
        float sx[4] = {0, 0, 0, 0}, dsx[4] = {0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < P; ++i) {
          const float4 v = row[k * R2 + i];
          sx[0] = fmaf(v.x, wx[i], sx[0]);
          sx[1] = fmaf(v.y, wx[i], sx[1]);
          sx[2] = fmaf(v.z, wx[i], sx[2]);
          sx[3] = fmaf(v.w, wx[i], sx[3]);
          dsx[0] = fmaf(v.x, dx[i], dsx[0]);
          dsx[1] = fmaf(v.y, dx[i], dsx[1]);
          dsx[2] = fmaf(v.z, dx[i], dsx[2]);
          dsx[3] = fmaf(v.w, dx[i], dsx[3]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          A[c] = fmaf(sx[c], wz, A[c]);
          Az[c] = fmaf(sx[c], dz, Az[c]);
          B[c] = fmaf(dsx[c], wz, B[c]);
        }
      }
      // lane j of the stencil's y rows (j >= P: weights zero)
      const float wy = j < P ? wyj : 0.0f, dy = j < P ? dyj : 0.0f;
      float v[8];
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] = A[c] * wy;
      v[4] = wy * (q[0] * B[0] + q[1] * B[1] + q[2] * B[2] + q[3] * B[3]);
      v[5] = dy * (q[0] * A[0] + q[1] * A[1] + q[2] * A[2] + q[3] * A[3]);
      v[6] = wy * (q[0] * Az[0] + q[1] * Az[1] + q[2] * Az[2] + q[3] * Az[3]);
      v[7] = 0.0f;
      // transposing butterfly over the group: afterwards lane j holds sum j
      {
        const bool h4 = (j & 4) != 0;
        float r4[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const float keep = h4 ? v[4 + m] : v[m], give = h4 ? v[m] : v[4 + m];
          r4[m] = keep + __shfl_xor_sync(0xffffffffu, give, 4);
        }
        const bool h2 = (j & 2) != 0;
        float r2[2];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          const float keep = h2 ? r4[2 + m] : r4[m], give = h2 ? r4[m] : r4[2 + m];
          r2[m] = keep + __shfl_xor_sync(0xffffffffu, give, 2);
        }
        const bool h1 = (j & 1) != 0;
        const float keep = h1 ? r2[1] : r2[0], give = h1 ? r2[0] : r2[1];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, give, 1);
      }
      if (valid && out_rec) {
        // one channel chunk: the atom's record in its sorted slot (the 8
        // lanes of the group fill one 32-byte sector); k_unpack_gather
        // writes the caller's layouts
        if (j < 7 && in_bounds(8 * int64_t(a) + j, 8 * nmax, kBoundsGatherOut))
          out_rec[8 * int64_t(a) + j] = j < 4 ? v[0] + zshift : v[0];
      } else if (valid) {
        if (j < 4) {
          if (phi && j < nk && in_bounds(int64_t(c0 + j) * n + o, int64_t(g.K) * n, kBoundsGatherOut))
            phi[int64_t(c0 + j) * n + o] = v[0] + zshift;
        } else if (j < 7 && forces && in_bounds(3 * int64_t(o) + (j - 4), 3 * n, kBoundsGatherOut)) {
          float* fo = forces + 3 * int64_t(o) + (j - 4);
          if (nchunk == 1)
            *fo = v[0];
          else
            atomicAdd(fo, v[0]);
        }
      }
    }
  }
}

// Records of k_gather4 (sorted slot m: four potentials, three force
// components) to phi [K][n] and forces [n][3] in the caller's order: atom
// i's slot is tile_start[tile_of[i]] + rank[i], so the writes are coalesced
// and each record is one 32-byte sector read.
static __global__ void k_unpack_gather(Geometry g, int64_t nmax, const int* __restrict__ soff, const int* __restrict__ tile_of,
                                const int* __restrict__ rank, const int* __restrict__ tile_start,
                                const float4* __restrict__ rec, float* __restrict__ phi, float* __restrict__ forces) {
  const int64_t n = soff[g.B];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t m = int64_t(tile_start[tile_of[i]]) + rank[i];
    if (!in_bounds(m, nmax, kBoundsGatherOut)) continue;
    const float4 a = rec[2 * m], b = rec[2 * m + 1];
    if (phi) {
      const float v[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < g.K) phi[int64_t(c) * n + i] = v[c];
    }
    if (forces) {
      forces[3 * i] = b.x;
      forces[3 * i + 1] = b.y;
      forces[3 * i + 2] = b.z;
    }
  }
}

// ---- spread -------------------------------------------------------------------
// Work items (tile, chunk of four channels).  FP32 fixed point as in k_spread:
// contributions are rounded to integers of a per-(tile, channel) unit 1/s by
// one FFMA with 1.5 * 2^23 and summed exactly in 32 bits; s (from
// k_tile_scale, computed when the points are set) keeps every contribution
// below 2^22 and every sum below 2^31.  The grid is zeroed before the launch.
// Spreading region: channel c, point (x, y, z) at c N + z R2 + y R1 + x; R1
// odd and N = 8 R1 (mod 32), so lane (c, j) of a warp (row j) is in bank
// R1 (8 c + j) + const (mod 32): 32 distinct banks.
template <int P>
struct SPad {
  static constexpr int S = kTile + P - 1;
  static constexpr int R1 = S | 1;
  static constexpr int R2 = S * R1;
  static constexpr int find_n() {
    int n = S * R2;
    while (((n - R1 * 8) % 32 + 32) % 32 != 0) ++n;
    return n;
  }
  static constexpr int N = (find_n() + 3) / 4 * 4;   // whole int4 per channel
};

template <int P>
constexpr size_t spread4_smem_bytes() {
  return size_t(4) * SPad<P>::N * sizeof(int);
}

template <int P, int NT>
__global__ void __launch_bounds__(NT, 1) k_spread4(Geometry g, int64_t nmax, const int* __restrict__ tile_start,
                                                   const float* __restrict__ st, const uint64_t* __restrict__ scell,
                                                   const float* __restrict__ sq,
                                                   const float* __restrict__ tscale,
                                                   const __grid_constant__ WinCoef<float> wc,
                                                   float* __restrict__ grid) {
  static_assert(P <= 8, "eight lanes per channel");
  using L = SPad<P>;
  constexpr int S = L::S, R1 = L::R1, R2 = L::R2, N = L::N;
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) int regi[];   // [4][N], layout SPad
  __shared__ float sscale[4], inv_s[4];
  __shared__ int64_t zoff_s[SPad<P>::S], yoff_s[SPad<P>::S];   // wrapped plane and row offsets of the item
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = lane & 7, cl = lane >> 3;   // stencil row and channel of the lane
  const int jr = j < P ? j : P - 1;
  LanePiece<P> pc;
  pc.load(wc, j);
  // the window piece a lane evaluates: piece j of direction cl (cl = 3 idle)
  const int nchunk = (g.K + 3) / 4;
  const int nitems = g.B * g.nts * nchunk;
  const int64_t plane = int64_t(g.M[1]) * g.Mxp, chan = int64_t(g.M[2]) * plane;
  const float* st_l = st + int64_t(min(cl, 2)) * nmax;
  {
    // the region starts zeroed; each item's flush zeroes what it read
    int4* r4 = reinterpret_cast<int4*>(regi);   // 4 N ints = N int4
    for (int t = threadIdx.x; t < N; t += NT) r4[t] = make_int4(0, 0, 0, 0);
  }
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int visit = item / nchunk, chunk = item - visit * nchunk;
    const int tile = tile_for_visit(g, visit);
    const int a0 = tile_start[tile], a1 = tile_start[tile + 1];
    if (a0 == a1 || !in_bounds(a1 - 1, nmax, kBoundsTile) || !in_bounds(a0, nmax, kBoundsTile)) continue;
    const int sidx = tile / g.nts;
    const int c0 = chunk * 4, nk = min(4, g.K - c0);
    const int gc0 = sidx * g.K + c0;
    int ox, oy, oz;
    tile_origin(g, tile - sidx * g.nts, ox, oy, oz);
    __syncthreads();   // the previous item's flush is done with the region (and zeroed it)
    {
      if (threadIdx.x < S)
        zoff_s[threadIdx.x] = wrap_index(oz + threadIdx.x, g.M[2]) * plane;
      else if (threadIdx.x < 2 * S)
        yoff_s[threadIdx.x - S] = int64_t(wrap_index(oy + threadIdx.x - S, g.M[1])) * g.Mxp;
    }
    if (threadIdx.x < 4) {
      const float sc = int(threadIdx.x) < nk ? tscale[int64_t(tile) * g.K + c0 + threadIdx.x] : 1.0f;
      sscale[threadIdx.x] = sc;
      inv_s[threadIdx.x] = 1.0f / sc;
    }
    __syncthreads();
    const bool active = j < P && cl < nk;
    const float qscale = active ? sscale[cl] : 0.0f;
    // one atom per warp; the next atom's inputs are loaded ahead
    int a = a0 + warp;
    float t_n = 0.0f, q_n = 0.0f;
    uint64_t cell_n = 0;
    if (a < a1) {
      t_n = st_l[a];
      cell_n = scell[a];
      q_n = cl < nk ? sq[int64_t(c0 + cl) * nmax + a] : 0.0f;
    }
    for (; a < a1; a += NW) {
      const float t = t_n, qv = q_n;
      const uint64_t cell = cell_n;
      if (a + NW < a1) {
        t_n = st_l[a + NW];
        cell_n = scell[a + NW];
        q_n = cl < nk ? sq[int64_t(c0 + cl) * nmax + a + NW] : 0.0f;
      }
      const float w = pc.value(t);   // piece j of direction cl
      float wx[P], wz[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        wx[i] = __shfl_sync(0xffffffffu, w, i);
        wz[i] = __shfl_sync(0xffffffffu, w, 16 + i);
      }
      const float wy = __shfl_sync(0xffffffffu, w, 8 + jr);
      int cx, cy, cz;
      unpack_cell(cell, cx, cy, cz);
      const int rb = cl * N + (cz - oz) * R2 + ((cy - oy) + j) * R1 + (cx - ox);
      if (active && in_bounds(rb, 4 * N, kBoundsSpreadRegion) &&
          in_bounds(rb + (P - 1) * R2 + (P - 1), 4 * N, kBoundsSpreadRegion)) {
        int* row = regi + rb;
        const float qy = qv * qscale * wy;
#pragma unroll
        for (int k = 0; k < P; ++k) {
          const float coef = qy * wz[k];
#pragma unroll
          for (int i = 0; i < P; ++i) {
            const float f = fmaf(coef, wx[i], 12582912.0f);
            atomicAdd(row + k * R2 + i, __float_as_int(f) - 0x4B400000);
          }
        }
      }
    }
    __syncthreads();
    {
      // two rows per warp iteration (half-warps), each lane adds an x pair;
      // pairs that do not straddle the periodic wrap go as one 8-byte atomic
      // (grid rows start at even offsets, tile origins are even)
      const int half = lane >> 4, x0 = 2 * (lane & 15);
      const bool has0 = x0 < S, has1 = x0 + 1 < S;
      const int gx0 = has0 ? wrap_index(ox + x0, g.M[0]) : 0;
      const int gx1 = has1 ? wrap_index(ox + x0 + 1, g.M[0]) : 0;
      const bool pair = has1 && gx1 == gx0 + 1 && (gx0 & 1) == 0;
      for (int pl = warp; pl < nk * S; pl += NW) {
        const int c = pl / S, lz = pl - c * S;
        const float inv = inv_s[c];
        float* base = grid + (gc0 + c) * chan + zoff_s[lz];
        int* src = regi + c * N + lz * R2;
        if (!has0) continue;
        for (int ly = half; ly < S; ly += 2) {
          float* rowg = base + yoff_s[ly];
          if (!in_bounds(int64_t(c * N + lz * R2 + ly * R1 + x0 + (has1 ? 1 : 0)), 4 * N, kBoundsSpreadFlush) ||
              !in_bounds((rowg - grid) + max(gx0, gx1), int64_t(g.B) * g.K * chan, kBoundsSpreadFlush))
            continue;
          const int v0 = src[ly * R1 + x0];
          const int v1 = has1 ? src[ly * R1 + x0 + 1] : 0;
          if ((v0 | v1) == 0) continue;   // nothing reached these points
          src[ly * R1 + x0] = 0;          // zeroed for the next item
          if (has1) src[ly * R1 + x0 + 1] = 0;
          if (pair) {
            atomicAdd(reinterpret_cast<float2*>(rowg + gx0), make_float2(float(v0) * inv, float(v1) * inv));
          } else {
            atomicAdd(rowg + gx0, float(v0) * inv);
            if (has1) atomicAdd(rowg + gx1, float(v1) * inv);
          }
        }
      }
    }
  }
}

// ---- backward spread ----------------------------------------------------------
// The backward's source for channel c, rhobar_c(r) = sum_i gphi_i^c W(r - r_i)
// + q_i^c gF_i . grad W(r - r_i), spread like k_spread4: one atom per warp,
// lanes = 4 channels x 8 stencil rows, 32-bit fixed point per (tile,
// channel) with the unit 1/s of k_tile_scale_bw.  Per point the contribution
// is wx(i) A(k) + dwx(i) B(k) with A(k) = (gphi wy + v_y dwy) wz(k) +
// v_z wy dwz(k), B(k) = v_x wy wz(k), v = q gF (grid-coordinate components
// in general cells), dw the window derivatives along each axis.
template <int P, int NT>
__global__ void __launch_bounds__(NT, 1) k_spread4_bw(Geometry g, int64_t nmax, const double* __restrict__ smol,
                                                      const int* __restrict__ soff,
                                                      const int* __restrict__ tile_start,
                                                      const float* __restrict__ st, const uint64_t* __restrict__ scell,
                                                      const float* __restrict__ sq, const int* __restrict__ sperm,
                                                      const float* __restrict__ tscale,
                                                      const __grid_constant__ WinCoef<float> wc,
                                                      const float* __restrict__ gphi, const float* __restrict__ gF,
                                                      float* __restrict__ grid2) {
  static_assert(P <= 8, "eight lanes per channel");
  using L = SPad<P>;
  constexpr int S = L::S, R1 = L::R1, R2 = L::R2, N = L::N;
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) int regi[];   // [4][N], layout SPad
  __shared__ float sscale[4], inv_s[4], two_h[3];
  __shared__ int64_t zoff_s[SPad<P>::S], yoff_s[SPad<P>::S];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = lane & 7, cl = lane >> 3;   // stencil row and channel of the lane
  const int jr = j < P ? j : P - 1;
  LanePiece<P> pc;
  pc.load(wc, j);
  const int64_t n = soff[g.B];
  const int nchunk = (g.K + 3) / 4;
  const int nitems = g.B * g.nts * nchunk;
  const int64_t plane = int64_t(g.M[1]) * g.Mxp, chan = int64_t(g.M[2]) * plane;
  const float* st_l = st + int64_t(min(cl, 2)) * nmax;
  {
    // the region starts zeroed; each item's flush zeroes what it read
    int4* r4 = reinterpret_cast<int4*>(regi);   // 4 N ints = N int4
    for (int t = threadIdx.x; t < N; t += NT) r4[t] = make_int4(0, 0, 0, 0);
  }
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int visit = item / nchunk, chunk = item - visit * nchunk;
    const int tile = tile_for_visit(g, visit);
    const int a0 = tile_start[tile], a1 = tile_start[tile + 1];
    if (a0 == a1 || !in_bounds(a1 - 1, nmax, kBoundsTile) || !in_bounds(a0, nmax, kBoundsTile)) continue;
    const int sidx = tile / g.nts;
    const int c0 = chunk * 4, nk = min(4, g.K - c0);
    const int gc0 = sidx * g.K + c0;
    int ox, oy, oz;
    tile_origin(g, tile - sidx * g.nts, ox, oy, oz);
    __syncthreads();   // the previous item's flush is done with the region (and zeroed it)
    {
      if (threadIdx.x < S)
        zoff_s[threadIdx.x] = wrap_index(oz + threadIdx.x, g.M[2]) * plane;
      else if (threadIdx.x < 2 * S)
        yoff_s[threadIdx.x - S] = int64_t(wrap_index(oy + threadIdx.x - S, g.M[1])) * g.Mxp;
    }
    if (threadIdx.x < 4) {
      const float sc = int(threadIdx.x) < nk ? tscale[int64_t(tile) * g.K + c0 + threadIdx.x] : 1.0f;
      sscale[threadIdx.x] = sc;
      inv_s[threadIdx.x] = 1.0f / sc;
    } else if (threadIdx.x < 7) {
      two_h[threadIdx.x - 4] = float(2.0 * smol[3 * sidx + threadIdx.x - 4]);
    }
    __syncthreads();
    const bool active = j < P && cl < nk;
    const float qscale = active ? sscale[cl] : 0.0f;
    const float th_l = two_h[min(cl, 2)];   // d s / d(grid coordinate) of the lane's direction, times the window's 2
    // one atom per warp; the next atom's inputs are loaded ahead
    int a = a0 + warp;
    float t_n = 0.0f, q_n = 0.0f;
    uint64_t cell_n = 0;
    int o_n = 0;
    if (a < a1) {
      t_n = st_l[a];
      cell_n = scell[a];
      q_n = cl < nk ? sq[int64_t(c0 + cl) * nmax + a] : 0.0f;
      o_n = sperm[a];
    }
    for (; a < a1; a += NW) {
      const float t = t_n, qv = q_n;
      const uint64_t cell = cell_n;
      const int o = o_n;
      if (a + NW < a1) {
        t_n = st_l[a + NW];
        cell_n = scell[a + NW];
        q_n = cl < nk ? sq[int64_t(c0 + cl) * nmax + a + NW] : 0.0f;
        o_n = sperm[a + NW];
      }
      const float gp = (gphi && cl < nk && in_bounds(int64_t(c0 + cl) * n + o, int64_t(g.K) * n, kBoundsSpreadRegion))
                           ? gphi[int64_t(c0 + cl) * n + o] : 0.0f;
      float gf0 = 0.0f, gf1 = 0.0f, gf2 = 0.0f;
      if (gF && in_bounds(3 * int64_t(o) + 2, 3 * n, kBoundsSpreadRegion)) {
        gf0 = gF[3 * int64_t(o)];
        gf1 = gF[3 * int64_t(o) + 1];
        gf2 = gF[3 * int64_t(o) + 2];
      }
      float w, dw;
      pc.value_deriv(t, w, dw);   // piece j of direction cl
      dw *= th_l;
      float wx[P], dx[P], wz[P], dz[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        wx[i] = __shfl_sync(0xffffffffu, w, i);
        dx[i] = __shfl_sync(0xffffffffu, dw, i);
        wz[i] = __shfl_sync(0xffffffffu, w, 16 + i);
        dz[i] = __shfl_sync(0xffffffffu, dw, 16 + i);
      }
      const float wy = __shfl_sync(0xffffffffu, w, 8 + jr);
      const float dy = __shfl_sync(0xffffffffu, dw, 8 + jr);
      int cx, cy, cz;
      unpack_cell(cell, cx, cy, cz);
      const int rb = cl * N + (cz - oz) * R2 + ((cy - oy) + j) * R1 + (cx - ox);
      if (active && in_bounds(rb, 4 * N, kBoundsSpreadRegion) &&
          in_bounds(rb + (P - 1) * R2 + (P - 1), 4 * N, kBoundsSpreadRegion)) {
        int* row = regi + rb;
        const float vq = qv * qscale;
        const float al = gp * qscale * wy + vq * gf1 * dy;   // A(k) = al wz(k) + be dz(k)
        const float be = vq * gf2 * wy;
        const float ga = vq * gf0 * wy;                      // B(k) = ga wz(k)
#pragma unroll
        for (int k = 0; k < P; ++k) {
          const float A = fmaf(al, wz[k], be * dz[k]);
          const float B = ga * wz[k];
#pragma unroll
          for (int i = 0; i < P; ++i) {
            const float f = fmaf(dx[i], B, fmaf(wx[i], A, 12582912.0f));
            atomicAdd(row + k * R2 + i, __float_as_int(f) - 0x4B400000);
          }
        }
      }
    }
    __syncthreads();
    {
      const int half = lane >> 4, x0 = 2 * (lane & 15);
      const bool has0 = x0 < S, has1 = x0 + 1 < S;
      const int gx0 = has0 ? wrap_index(ox + x0, g.M[0]) : 0;
      const int gx1 = has1 ? wrap_index(ox + x0 + 1, g.M[0]) : 0;
      const bool pair = has1 && gx1 == gx0 + 1 && (gx0 & 1) == 0;
      for (int pl = warp; pl < nk * S; pl += NW) {
        const int c = pl / S, lz = pl - c * S;
        const float inv = inv_s[c];
        float* base = grid2 + (gc0 + c) * chan + zoff_s[lz];
        int* src = regi + c * N + lz * R2;
        if (!has0) continue;
        for (int ly = half; ly < S; ly += 2) {
          float* rowg = base + yoff_s[ly];
          if (!in_bounds(int64_t(c * N + lz * R2 + ly * R1 + x0 + (has1 ? 1 : 0)), 4 * N, kBoundsSpreadFlush) ||
              !in_bounds((rowg - grid2) + max(gx0, gx1), int64_t(g.B) * g.K * chan, kBoundsSpreadFlush))
            continue;
          const int v0 = src[ly * R1 + x0];
          const int v1 = has1 ? src[ly * R1 + x0 + 1] : 0;
          if ((v0 | v1) == 0) continue;   // nothing reached these points
          src[ly * R1 + x0] = 0;          // zeroed for the next item
          if (has1) src[ly * R1 + x0 + 1] = 0;
          if (pair) {
            atomicAdd(reinterpret_cast<float2*>(rowg + gx0), make_float2(float(v0) * inv, float(v1) * inv));
          } else {
            atomicAdd(rowg + gx0, float(v0) * inv);
            if (has1) atomicAdd(rowg + gx1, float(v1) * inv);
          }
        }
      }
    }
  }
}

// Fixed-point units of k_spread4_bw per (tile, channel).  An atom's
// contribution at any point is at most M_i = |gphi_i^c| mw_x mw_y mw_z +
// |q_i^c| (|gF_x| md_x mw_y mw_z + |gF_y| mw_x md_y mw_z + |gF_z| mw_x mw_y md_z)
// with mw_d, md_d the largest |W| and |dW/dx_d| over the atom's P window
// pieces at its own offsets (evaluated as the spread evaluates them); s keeps
// every contribution below 2^22 and every sum below 2^31 (as k_tile_scale).
// One warp per tile.
template <int P>
__global__ void k_tile_scale_bw(int ntl, int nts, int K, int64_t nmax, const int* __restrict__ soff,
                                const int* __restrict__ tile_start, const float* __restrict__ st,
                                const float* __restrict__ sq, const int* __restrict__ sperm,
                                const double* __restrict__ smol, const __grid_constant__ WinCoef<float> wc,
                                const float* __restrict__ gphi, const float* __restrict__ gF,
                                float* __restrict__ tscale) {
  constexpr int D = WinCoef<float>::kDeg;
  const int lane = threadIdx.x & 31;
  const int nw = int((int64_t(gridDim.x) * blockDim.x) >> 5);
  const int64_t n = soff[ntl / nts];   // atoms of all structures (rows of gphi)
  for (int t = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); t < ntl; t += nw) {
    const int a0 = tile_start[t], a1 = tile_start[t + 1];
    const int sidx = t / nts;
    for (int c = 0; c < K; ++c) {
      float s1 = 0.0f, mq = 0.0f;
      for (int a = a0 + lane; a < a1; a += 32) {
        float mw[3], md[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float sv = 2.0f * st[int64_t(d) * nmax + a] - 1.0f;
          float vmax = 0.0f, dmax = 0.0f;
#pragma unroll
          for (int j = 0; j < P; ++j) {
            float v = wc.c[j * (D + 1) + D], dv = 0.0f;
#pragma unroll
            for (int m = D - 1; m >= 0; --m) {
              dv = fmaf(dv, sv, v);
              v = fmaf(v, sv, wc.c[j * (D + 1) + m]);
            }
            vmax = fmaxf(vmax, fabsf(v));
            dmax = fmaxf(dmax, fabsf(dv));
          }
          mw[d] = vmax;
          md[d] = dmax * float(2.0 * smol[3 * sidx + d]);
        }
        const int o = sperm[a];
        float m = 0.0f;
        if (gF)
          m = fabsf(sq[int64_t(c) * nmax + a]) *
              (fabsf(gF[3 * int64_t(o)]) * md[0] * mw[1] * mw[2] + fabsf(gF[3 * int64_t(o) + 1]) * mw[0] * md[1] * mw[2] +
               fabsf(gF[3 * int64_t(o) + 2]) * mw[0] * mw[1] * md[2]);
        if (gphi) m += fabsf(gphi[int64_t(c) * n + o]) * mw[0] * mw[1] * mw[2];
        m *= 1.0001f;   // the spread's two roundings per contribution and FP32 products here
        s1 += m;
        mq = fmaxf(mq, m);
      }
      for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        mq = fmaxf(mq, __shfl_xor_sync(0xffffffffu, mq, o));
      }
      if (lane == 0)
        tscale[int64_t(t) * K + c] =
            s1 > 0.0f ? fminf(0.99f * 4194304.0f / mq, 0.999f * 2147483647.0f / (s1 * 1.0001f)) : 1.0f;
    }
  }
}

}  // namespace pswf
