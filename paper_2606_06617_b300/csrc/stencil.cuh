// Tiled stencil kernels: spreading (step (i)) and the gather of potentials
// and forces.  One CTA per tile of kTile^3 stencil-start cells at a time;
// the tile's atoms are contiguous in the sorted arrays.  The padded region of
// a tile, S^3 grid points with S = kTile + P - 1, is the union of its atoms'
// stencils.
//
// Shared-memory layout of a padded region: element (x, y, z) at
// z * R2 + y * R1 + x, with R1 = S | 1 and R2 >= S * R1 chosen so that the
// P^2 stencil rows (j, k) of one atom, taken 32 at a time in the order
// r = k P + j, fall in 32 different banks (for any start cell).  Lanes of a
// warp that work on the rows of one atom therefore never conflict.
#pragma once

#include <type_traits>

#include "kernels.cuh"

namespace pswf {

template <int P>
struct Padded {
  static constexpr int S = kTile + P - 1;
  static constexpr int R1 = S | 1;
  static constexpr bool conflict_free(int r2) {
    for (int base = 0; base < P * P; base += 32) {
      unsigned mask = 0;
      for (int r = base; r < base + 32 && r < P * P; ++r) {
        const int b = (R1 * (r % P) + r2 * (r / P)) % 32;
        if (mask & (1u << b)) return false;
        mask |= 1u << b;
      }
    }
    return true;
  }
  static constexpr int find_r2() {
    for (int r2 = S * R1; r2 < S * R1 + 64; ++r2)
      if (conflict_free(r2)) return r2;
    return S * R1;
  }
  static constexpr int R2 = find_r2();
  static constexpr int N = S * R2;   // elements of one padded region
};


template <typename R, int P>
constexpr size_t spread_smem_bytes(int batch) {
  return size_t(Padded<P>::N) * sizeof(R) + size_t(batch) * (3 * P * sizeof(R) + sizeof(R) + sizeof(int));
}

__device__ inline int wrap_index(int v, int M) {
  while (v >= M) v -= M;
  return v;
}

// Integer accumulator type of the spreading region: FP32 contributions are
// accumulated exactly in 32-bit fixed point (scale chosen per tile and
// channel so that the sum of all |contributions| stays below 2^31), FP64
// contributions in double.
template <typename R>
struct SpreadAcc {
  using T = int;
};
template <>
struct SpreadAcc<double> {
  using T = double;
};

// Spreading.  Channel by channel: zero the padded region; every warp takes
// atoms of the tile in turn, its lanes take the P^2 (y, z) rows of that
// atom's stencil and add q W_x(i) W_y(j) W_z(k) into the region with
// shared-memory atomics (FP32 path: rounded to a 32-bit fixed-point grid of
// step 1/s, s = 0.999 (2^31 - 1) / (1.0001 sum_tile |q|), so the exact integer
// sums never overflow); then the region is added into the grid with coalesced
// global atomics (neighbouring tiles overlap by P - 1 planes).  The grid is
// zeroed before the launch.
template <typename R, int P>
__global__ void __launch_bounds__(512) k_spread(Geometry g, int64_t nmax, const int* __restrict__ tile_start,
                                                const R* __restrict__ st, const uint64_t* __restrict__ scell,
                                                const R* __restrict__ sq, WinCoef<R> wc, int batch,
                                                R* __restrict__ grid) {
  using A = typename SpreadAcc<R>::T;
  constexpr bool kFixed = std::is_same<A, int>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int S = Padded<P>::S, R1 = Padded<P>::R1, R2 = Padded<P>::R2, N = Padded<P>::N;
  A* region = reinterpret_cast<A*>(smraw);
  R* wts = reinterpret_cast<R*>(region + N);
  R* qs = wts + batch * 3 * P;
  int* loc = reinterpret_cast<int*>(qs + batch);
  __shared__ float red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int ntiles = g.ntile[0] * g.ntile[1] * g.ntile[2];
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int a0 = tile_start[tile], a1 = tile_start[tile + 1];
    if (a0 == a1) continue;
    const int tx = tile % g.ntile[0], ty = (tile / g.ntile[0]) % g.ntile[1], tz = tile / (g.ntile[0] * g.ntile[1]);
    const int ox = tx * kTile, oy = ty * kTile, oz = tz * kTile;
    const int nbat = (a1 - a0 + batch - 1) / batch;
    for (int c = 0; c < g.K; ++c) {
      const R* qc = sq + int64_t(c) * nmax;
      float scale = 1.0f;
      if (kFixed) {
        float s = 0.0f;
        for (int a = a0 + threadIdx.x; a < a1; a += blockDim.x) s += fabsf(float(qc[a]));
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        __syncthreads();
        if (lane == 0) red[warp] = s;
        __syncthreads();
        float tot = 0.0f;
        for (int w = 0; w < nwarp; ++w) tot += red[w];
        scale = tot > 0.0f ? 0.999f * 2147483647.0f / (tot * 1.0001f) : 1.0f;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < N; i += blockDim.x) region[i] = A(0);
      for (int bi = 0; bi < nbat; ++bi) {
        const int b0 = a0 + bi * batch;
        const int nb = min(batch, a1 - b0);
        __syncthreads();
        if (c == 0 || nbat > 1) {
          for (int t = threadIdx.x; t < nb * 3; t += blockDim.x) {
            const int a = t / 3, d = t - 3 * a;
            R w[P];
            window_values<R, P>(st[d * nmax + b0 + a], wc, w);
#pragma unroll
            for (int j = 0; j < P; ++j) wts[(a * 3 + d) * P + j] = w[j];
          }
          for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            int cx, cy, cz;
            unpack_cell(scell[b0 + t], cx, cy, cz);
            loc[t] = (cx - ox) | ((cy - oy) << 8) | ((cz - oz) << 16);
          }
        }
        for (int t = threadIdx.x; t < nb; t += blockDim.x) qs[t] = qc[b0 + t] * R(scale);
        __syncthreads();
        for (int a = warp; a < nb; a += nwarp) {
          const R* wa = wts + a * 3 * P;
          const int l = loc[a];
          const int lx = l & 0xff, ly = (l >> 8) & 0xff, lz = (l >> 16) & 0xff;
          R wx[P];
#pragma unroll
          for (int i = 0; i < P; ++i) wx[i] = wa[i];
          const R qa = qs[a];
          for (int r = lane; r < P * P; r += 32) {
            const int j = r % P, k = r / P;
            const R coef = wa[P + j] * wa[2 * P + k] * qa;
            A* row = region + (lz + k) * R2 + (ly + j) * R1 + lx;
#pragma unroll
            for (int i = 0; i < P; ++i) {
              if (kFixed)
                atomicAdd(reinterpret_cast<int*>(row) + i, __float2int_rn(float(coef * wx[i])));
              else
                atomicAdd(reinterpret_cast<double*>(row) + i, double(coef * wx[i]));
            }
          }
        }
      }
      __syncthreads();
      const R inv = R(1) / R(scale);
      R* gc = grid + int64_t(c) * g.M[2] * g.M[1] * g.Mxp;
      for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
        const int lz = idx / R2, rem = idx - lz * R2, ly = rem / R1, lx = rem - ly * R1;
        if (ly >= S || lx >= S) continue;
        const A v = region[idx];
        if (v != A(0)) {
          const int gx = wrap_index(ox + lx, g.M[0]), gy = wrap_index(oy + ly, g.M[1]),
                    gz = wrap_index(oz + lz, g.M[2]);
          atomicAdd(gc + (int64_t(gz) * g.M[1] + gy) * g.Mxp + gx, R(v) * inv);
        }
      }
    }
    __syncthreads();
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

// ---- gather ------------------------------------------------------------------
//
// Lane mapping: a warp is cut into slots of G lanes (G = the power of two
// >= P); the lanes of a slot are the P y-rows j of one atom's stencil in one
// channel, each lane sweeping its row's P z-planes and P x-points.  With all
// K channels of a tile staged, the slots of a warp are the channels of ONE
// atom, so the window weights are shared by the whole warp and no two lanes
// hit the same shared-memory bank (layout below).  With fewer channels than
// slots, a warp takes several atoms.
template <int P>
struct GatherPad {
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

// Threads of a gather CTA: 1024 in FP32 (64 registers a thread), 512 in FP64.
template <typename R>
constexpr int kGatherThreadsFor = sizeof(R) == 4 ? 1024 : 512;

template <typename R, int P>
constexpr size_t gather_smem_bytes(int kc) {
  return size_t(kc) * GatherPad<P>::N * sizeof(R);
}

template <typename R>
__device__ inline void cp_async_elem(R* dst, const R* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(int(sizeof(R))) : "memory");
}
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

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
  using L = GatherPad<P>;
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
      for (int s2 = 1; s2 < kc; ++s2) {
        const int src = min(lane + s2 * G, 31);
        const R g0 = __shfl_sync(0xffffffffu, f0, src), g1 = __shfl_sync(0xffffffffu, f1, src),
                g2 = __shfl_sync(0xffffffffu, f2, src);
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
