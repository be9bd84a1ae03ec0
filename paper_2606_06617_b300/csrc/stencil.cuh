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

// Threads of a spread or gather CTA: 1024 in FP32 (64 registers a thread), 512 in FP64.
template <typename R>
constexpr int kGatherThreadsFor = sizeof(R) == 4 ? 1024 : 512;

template <typename R, int P>
constexpr size_t gather_smem_bytes(int kc) {
  return size_t(kc) * TilePad<P>::N * sizeof(R);
}

template <typename R>
__device__ inline void cp_async_elem(R* dst, const R* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(int(sizeof(R))) : "memory");
}
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Spreading (step (i)).  Work items are (tile, chunk of kc channels); the
// kc padded regions live in shared memory with the layout above.  Lane j of
// a slot adds the contributions q W_x(i) W_y(j) W_z(k) of its row j for all
// (i, k) with shared-memory atomics; the slots of a warp are the channels of
// one atom (or several atoms when K is small), so no two lanes of a warp
// touch the same bank.  The region is then added into the grid with global
// atomics, one warp per (channel, z) plane, lanes along x (neighbouring
// tiles overlap by P - 1 planes); the grid is zeroed before the launch.
//
// FP32 path: contributions are rounded to integers of a per-(tile, channel)
// fixed point 1/s and summed exactly in 32 bits.  The rounding is one FFMA
// with the constant 1.5 * 2^23 (the sum's low mantissa bits are then the
// rounded integer, exact for |value| < 2^22), so s = min(0.99 * 2^22 /
// max|q|, 0.999 * 2^31 / (1.0001 sum|q|)) keeps every contribution below 2^22
// and every grid sum below 2^31 (the window is at most 1).  FP64 path:
// double atomics.
template <typename R, int P>
constexpr size_t spread_smem_bytes(int kc) {
  return size_t(kc) * TilePad<P>::N * sizeof(typename SpreadAcc<R>::T);
}

template <typename R, int P>
__global__ void __launch_bounds__(kGatherThreadsFor<R>, 1) k_spread(Geometry g, int64_t nmax,
                                                                   const int* __restrict__ tile_start,
                                                                   const R* __restrict__ st,
                                                                   const uint64_t* __restrict__ scell,
                                                                   const R* __restrict__ sq, WinCoef<R> wc, int kc,
                                                                   R* __restrict__ grid) {
  using A = typename SpreadAcc<R>::T;
  constexpr bool kFixed = std::is_same<A, int>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  using L = TilePad<P>;
  constexpr int G = L::G, NS = L::NS, S = L::S, R1 = L::R1, R2 = L::R2, N = L::N;
  A* region = reinterpret_cast<A*>(smraw);   // [kc][N]
  __shared__ float red_sum[32][NS], red_max[32][NS];
  __shared__ float sscale[NS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int slot = lane / G, j = lane % G, sbase = lane - j;
  const int nchunk = (g.K + kc - 1) / kc;
  const int apw = NS / kc;
  const int asub = slot / kc, cc = slot - asub * kc;
  const bool slot_used = asub < apw;
  const int jr = j < P ? j : P - 1;
  const int ntiles = g.ntile[0] * g.ntile[1] * g.ntile[2];
  const int64_t plane = int64_t(g.M[1]) * g.Mxp, chan = int64_t(g.M[2]) * plane;
  for (int item = blockIdx.x; item < ntiles * nchunk; item += gridDim.x) {
    const int tile = item / nchunk, chunk = item - tile * nchunk;
    const int a0 = tile_start[tile], a1 = tile_start[tile + 1];
    if (a0 == a1) continue;
    const int c0 = chunk * kc, nk = min(kc, g.K - c0);
    const int tx = tile % g.ntile[0], ty = (tile / g.ntile[0]) % g.ntile[1], tz = tile / (g.ntile[0] * g.ntile[1]);
    const int ox = tx * kTile, oy = ty * kTile, oz = tz * kTile;
    __syncthreads();   // the previous item's flush is done with the region
    {
      const int nbytes = nk * N * int(sizeof(A));
      int4* r4 = reinterpret_cast<int4*>(region);
      for (int t = threadIdx.x; t < nbytes / 16; t += blockDim.x) r4[t] = make_int4(0, 0, 0, 0);
      int* r1 = reinterpret_cast<int*>(region);
      for (int t = (nbytes / 16) * 4 + threadIdx.x; t < nbytes / 4; t += blockDim.x) r1[t] = 0;
    }
    if (kFixed) {
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
        sscale[threadIdx.x] = tot > 0.0f ? fminf(0.99f * 4194304.0f / m, 0.999f * 2147483647.0f / (tot * 1.0001f)) : 1.0f;
      }
    }
    __syncthreads();
    const bool use_slot = slot_used && cc < nk;
    const R qscale = kFixed && use_slot ? R(sscale[cc]) : R(1);
    for (int base = a0 + warp * apw; base < a1; base += nwarp * apw) {
      const int a_raw = base + asub;
      const bool valid = use_slot && a_raw < a1;
      const int a = min(a_raw, a1 - 1);
      R wj[3];
      {
        const R s0 = R(2) * st[a] - R(1), s1 = R(2) * st[nmax + a] - R(1), s2 = R(2) * st[2 * nmax + a] - R(1);
        const int deg = wc.deg;
        const R* c = wc.c + jr * (deg + 1);
        R v0 = c[deg], v1 = v0, v2 = v0;
        for (int m = deg - 1; m >= 0; --m) {
          const R cm = c[m];
          v0 = v0 * s0 + cm;
          v1 = v1 * s1 + cm;
          v2 = v2 * s2 + cm;
        }
        wj[0] = v0;
        wj[1] = v1;
        wj[2] = v2;
      }
      R wx[P], wz[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        wx[i] = __shfl_sync(0xffffffffu, wj[0], sbase + i);
        wz[i] = __shfl_sync(0xffffffffu, wj[2], sbase + i);
      }
      if (valid && j < P) {
        int cx, cy, cz;
        unpack_cell(scell[a], cx, cy, cz);
        A* row = region + cc * N + (cz - oz) * R2 + (cy - oy + j) * R1 + (cx - ox);
        const R qy = sq[int64_t(c0 + cc) * nmax + a] * qscale * wj[1];
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
      const int gx = lane < S ? wrap_index(ox + lane, g.M[0]) : 0;
      for (int pl = warp; pl < nk * S; pl += nwarp) {
        const int c = pl / S, lz = pl - c * S;
        const R inv = kFixed ? R(1) / R(sscale[c]) : R(1);
        R* dst = grid + (c0 + c) * chan + wrap_index(oz + lz, g.M[2]) * plane + gx;
        const A* src = region + c * N + lz * R2 + lane;
        if (lane < S) {
          int gy = oy;
          for (int ly = 0; ly < S; ++ly, ++gy) {
            if (gy == g.M[1]) gy = 0;
            const A v = src[ly * R1];
            if (v != A(0)) atomicAdd(dst + int64_t(gy) * g.Mxp, R(v) * inv);
          }
        }
      }
    }
  }
}

// Spreading without shared-memory staging, for plans whose padded region does
// not fit in shared memory (FP64 with large P): one thread per sorted atom,
// global atomics.
template <typename R, int P>
__global__ void k_spread_direct(int64_t n, int64_t nmax, Geometry g, const R* __restrict__ st,
                                const uint64_t* __restrict__ scell, const R* __restrict__ sq, WinCoef<R> wc,
                                R* __restrict__ grid) {
  for (int64_t a = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; a < n; a += int64_t(gridDim.x) * blockDim.x) {
    R wx[P], wy[P], wz[P];
    window_values<R, P>(st[a], wc, wx);
    window_values<R, P>(st[nmax + a], wc, wy);
    window_values<R, P>(st[2 * nmax + a], wc, wz);
    int cx, cy, cz;
    unpack_cell(scell[a], cx, cy, cz);
    for (int c = 0; c < g.K; ++c) {
      const R qc = sq[int64_t(c) * nmax + a];
      R* gc = grid + int64_t(c) * g.M[2] * g.M[1] * g.Mxp;
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
// (one warp per (channel, z) plane, lanes along x), then every warp walks the
// tile's atoms.  Lane j of a slot evaluates window piece j in x, y and z and
// the slot exchanges them by shuffles; the potential of a channel is reduced
// over its slot, the force over the atom's slots.  With more than one chunk
// the force is accumulated with global atomics (zeroed before the launch).
template <typename R, int P>
__global__ void __launch_bounds__(kGatherThreadsFor<R>, 1) k_interp(int64_t n, int64_t nmax, Geometry g,
                                                   const int* __restrict__ tile_start, const R* __restrict__ st,
                                                   const uint64_t* __restrict__ scell, const R* __restrict__ sq,
                                                   const int* __restrict__ sperm, WinCoef<R> wc, int kc,
                                                   const R* __restrict__ grid, const double* __restrict__ zero_coef,
                                                   const double* __restrict__ charges, R* __restrict__ phi,
                                                   R* __restrict__ forces) {
  extern __shared__ __align__(16) unsigned char smraw[];
  using L = TilePad<P>;
  constexpr int G = L::G, NS = L::NS, S = L::S, R1 = L::R1, R2 = L::R2, N = L::N;
  R* region = reinterpret_cast<R*>(smraw);   // [kc][N]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int slot = lane / G, j = lane % G, sbase = lane - j;
  const int nchunk = (g.K + kc - 1) / kc;
  const int apw = NS / kc;                 // atoms per warp
  const int asub = slot / kc, cc = slot - asub * kc;
  const bool slot_used = asub < apw;
  const int jr = j < P ? j : P - 1;        // row read by lanes beyond the stencil
  const R two_h[3] = {R(2.0 * g.M[0] / g.L[0]), R(2.0 * g.M[1] / g.L[1]), R(2.0 * g.M[2] / g.L[2])};
  const int ntiles = g.ntile[0] * g.ntile[1] * g.ntile[2];
  const int64_t plane = int64_t(g.M[1]) * g.Mxp, chan = int64_t(g.M[2]) * plane;
  for (int item = blockIdx.x; item < ntiles * nchunk; item += gridDim.x) {
    const int tile = item / nchunk, chunk = item - tile * nchunk;
    const int a0 = tile_start[tile], a1 = tile_start[tile + 1];
    if (a0 == a1) continue;
    const int c0 = chunk * kc, nk = min(kc, g.K - c0);
    const int tx = tile % g.ntile[0], ty = (tile / g.ntile[0]) % g.ntile[1], tz = tile / (g.ntile[0] * g.ntile[1]);
    const int ox = tx * kTile, oy = ty * kTile, oz = tz * kTile;
    __syncthreads();   // the previous item's reads of the region are done
    {
      const int gx = lane < S ? wrap_index(ox + lane, g.M[0]) : 0;
      for (int pl = warp; pl < nk * S; pl += nwarp) {
        const int c = pl / S, lz = pl - c * S;
        const R* src = grid + (c0 + c) * chan + wrap_index(oz + lz, g.M[2]) * plane + gx;
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
      cp_async_wait_all();
    }
    __syncthreads();
    const bool use_slot = slot_used && cc < nk;
    for (int base = a0 + warp * apw; base < a1; base += nwarp * apw) {
      const int a_raw = base + asub;
      const bool valid = use_slot && a_raw < a1;
      const int a = min(a_raw, a1 - 1);
      // window pieces: lane j of the slot evaluates piece j in each direction
      R wj[3], dj[3];
      {
        const R s0 = R(2) * st[a] - R(1), s1 = R(2) * st[nmax + a] - R(1), s2 = R(2) * st[2 * nmax + a] - R(1);
        const int deg = wc.deg;
        const R* c = wc.c + jr * (deg + 1);
        R v0 = c[deg], v1 = v0, v2 = v0, e0 = 0, e1 = 0, e2 = 0;
        for (int m = deg - 1; m >= 0; --m) {
          const R cm = c[m];
          e0 = e0 * s0 + v0;
          e1 = e1 * s1 + v1;
          e2 = e2 * s2 + v2;
          v0 = v0 * s0 + cm;
          v1 = v1 * s1 + cm;
          v2 = v2 * s2 + cm;
        }
        wj[0] = v0; wj[1] = v1; wj[2] = v2;
        dj[0] = e0 * two_h[0]; dj[1] = e1 * two_h[1]; dj[2] = e2 * two_h[2];
      }
      R wx[P], dx[P], wz[P], dz[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        wx[i] = __shfl_sync(0xffffffffu, wj[0], sbase + i);
        dx[i] = __shfl_sync(0xffffffffu, dj[0], sbase + i);
        wz[i] = __shfl_sync(0xffffffffu, wj[2], sbase + i);
        dz[i] = __shfl_sync(0xffffffffu, dj[2], sbase + i);
      }
      const R wy = j < P ? wj[1] : R(0), dy = j < P ? dj[1] : R(0);
      int cx, cy, cz;
      unpack_cell(scell[a], cx, cy, cz);
      const int lx = cx - ox, ly = cy - oy, lz = cz - oz;
      const R* row = region + (use_slot ? cc : 0) * N + lz * R2 + (ly + jr) * R1 + lx;
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
      const R q = valid ? sq[int64_t(c0 + cc) * nmax + a] : R(0);
      R ph = A * wy, f0 = q * B * wy, f1 = q * A * dy, f2 = q * Az * wy;
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        ph += __shfl_xor_sync(0xffffffffu, ph, o);
        f0 += __shfl_xor_sync(0xffffffffu, f0, o);
        f1 += __shfl_xor_sync(0xffffffffu, f1, o);
        f2 += __shfl_xor_sync(0xffffffffu, f2, o);
      }
      // channels of the same atom sit in neighbouring slots: cc = 0 collects
      const R e0 = f0, e1 = f1, e2 = f2;
      for (int s2 = 1; s2 < kc; ++s2) {
        const int src = min(lane + s2 * G, 31);
        const R g0 = __shfl_sync(0xffffffffu, e0, src), g1 = __shfl_sync(0xffffffffu, e1, src),
                g2 = __shfl_sync(0xffffffffu, e2, src);
        if (cc + s2 < nk) {
          f0 += g0;
          f1 += g1;
          f2 += g2;
        }
      }
      if (valid && j == 0) {
        const int o = sperm[a];
        if (phi) phi[int64_t(c0 + cc) * n + o] = ph + R(2.0 * zero_coef[c0 + cc] * charges[2 * (c0 + cc)]);
        if (forces && cc == 0) {
          R* fo = forces + 3 * int64_t(o);
          if (nchunk == 1) {
            fo[0] = f0;
            fo[1] = f1;
            fo[2] = f2;
          } else {
            atomicAdd(fo, f0);
            atomicAdd(fo + 1, f1);
            atomicAdd(fo + 2, f2);
          }
        }
      }
    }
  }
}

}  // namespace pswf
