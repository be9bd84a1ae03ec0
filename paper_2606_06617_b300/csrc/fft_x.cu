// Pruned real transforms along x (FP32), see fft_x.hpp.
//
// One warp transforms one complex row of length N = 32 N1 holding two real
// grid rows (real and imaginary parts), as the four-step split N = N1 x 32:
// an N1-point DFT in registers (radix 2, odd remainders directly, twiddles
// compile-time constants), a twiddle, and a 32-point DFT across the lanes
// (decimation in frequency, five butterfly stages of xor shuffles; each lane
// applies v' = (v + s p) w with its own sign s and pre-signed twiddle w, so
// that the lanes' outputs come in bit-reversed order r = brev5(lane)).
//
// Forward (coalesced loads): lane l holds x[l + 32 m]; registers first, then
// the twiddle e^{-2 pi i l k1 / N}, then the lanes: register k1 of lane l
// ends as X[k1 + N1 r].  The two real rows' spectra are split from X[k] and
// X[N - k] (one more shuffle) and staged per row.  Inverse (coalesced
// stores): lane l takes X[n1 + N1 l] from the staged rows; lanes first, then
// the twiddle e^{+2 pi i n1 r / N}, then registers: register k1 of lane l
// ends as x[32 k1 + r].
//
// A CTA of 8 warps covers 16 rows of one (c, z) line; the staged spectra
// are [y][pos(kx)] with pos(k) = k + k / N1 for even N1 (so that the lanes'
// strided accesses fall in distinct banks) and an odd row stride, and each
// kx plane gets one 128-byte store (forward) or load (inverse).  Planes
// kx >= nkx are neither written nor read.
#include "fft_x.hpp"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <utility>

namespace pswf {
namespace {

constexpr int kRows = 16;                // rows of a (c, z) line per CTA
constexpr int kXThreads = 16 * kRows;    // a warp per pair of rows
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// cos and sin of 2 pi j / n by their Taylor series after reducing the angle
// to [-pi, pi]; only ever evaluated by the compiler (template constants).
__host__ __device__ constexpr double series_sin(double x) {
  double term = x, s = x;
  for (int j = 1; j < 24; ++j) {
    term *= -x * x / double((2 * j) * (2 * j + 1));
    s += term;
  }
  return s;
}
__host__ __device__ constexpr double series_cos(double x) {
  double term = 1.0, s = 1.0;
  for (int j = 1; j < 24; ++j) {
    term *= -x * x / double((2 * j - 1) * (2 * j));
    s += term;
  }
  return s;
}
__host__ __device__ constexpr double turn_angle(int j, int n) {
  int r = j % n;
  if (2 * r > n) r -= n;
  return 2.0 * 3.14159265358979323846 * double(r) / double(n);
}

// W_n^j = e^{-2 pi i j / n} (forward) or its conjugate (inverse).
template <int J, int N, bool INV>
struct Tw {
  static constexpr float re = float(series_cos(turn_angle(J, N)));
  static constexpr float im = float(INV ? series_sin(turn_angle(J, N)) : -series_sin(turn_angle(J, N)));
};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
  return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}

// v W_N^J with the quarter turns exact.
template <int J, int N, bool INV>
__device__ __forceinline__ float2 mul_tw(float2 v) {
  constexpr int r = J % N;
  if constexpr (r == 0) {
    return v;
  } else if constexpr (2 * r == N) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (4 * r == N) {   // -i forward, +i inverse
    return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
  } else if constexpr (4 * r == 3 * N) {   // +i forward, -i inverse
    return INV ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
  } else {
    return cmul(v, make_float2(Tw<r, N, INV>::re, Tw<r, N, INV>::im));
  }
}

template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// In-register DFT of length N, natural order in and out.
template <int N, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&x)[N]) {
  if constexpr (N == 1) {
    return;
  } else if constexpr (N % 2 == 0) {
    constexpr int H = N / 2;
    float2 e[H], o[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      e[j] = x[2 * j];
      o[j] = x[2 * j + 1];
    }
    dft_reg<H, INV>(e);
    dft_reg<H, INV>(o);
    static_for<H>([&](auto kk) {
      constexpr int k = decltype(kk)::value;
      const float2 t = mul_tw<k, N, INV>(o[k]);
      x[k] = cadd(e[k], t);
      x[k + H] = csub(e[k], t);
    });
  } else {
    float2 y[N];
    static_for<N>([&](auto kk) {
      constexpr int k = decltype(kk)::value;
      float2 s = x[0];
      static_for<N - 1>([&](auto mm) {
        constexpr int m = decltype(mm)::value + 1;
        s = cadd(s, mul_tw<(m * k) % N, N, INV>(x[m]));
      });
      y[k] = s;
    });
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = y[j];
  }
}

// The 32-point DFT across the lanes (bit-reversed output order); stw are the
// five stages' pre-signed twiddles.
template <int N1, bool INV>
__device__ __forceinline__ void lane_dft(float2 (&v)[N1], const float2* __restrict__ stw, int lane) {
#pragma unroll
  for (int st = 0; st < 4; ++st) {
    const int d = 16 >> st;
    // lower lane: a + b; upper lane: (a - b) W_{2d}^{lane mod d}, as
    // (v + s p) w with s = -1 and w = -W on the upper lane
    float2 w = __ldg(stw + st * 32 + lane);
    if (INV) w.y = -w.y;
    const float sg = (lane & d) ? -1.0f : 1.0f;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const float px = __shfl_xor_sync(kFull, v[k1].x, d);
      const float py = __shfl_xor_sync(kFull, v[k1].y, d);
      v[k1] = cmul(make_float2(fmaf(sg, px, v[k1].x), fmaf(sg, py, v[k1].y)), w);
    }
  }
  {
    // the last stage's twiddles are 1 (lower lane) and -1 (upper): v' = s v + p
    const float sg = (lane & 1) ? -1.0f : 1.0f;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const float px = __shfl_xor_sync(kFull, v[k1].x, 1);
      const float py = __shfl_xor_sync(kFull, v[k1].y, 1);
      v[k1] = make_float2(fmaf(sg, v[k1].x, px), fmaf(sg, v[k1].y, py));
    }
  }
}

// Register j of the lane times tw[j * 32 + lane] (conjugated for INV), j >= 1.
template <int N1, bool INV>
__device__ __forceinline__ void lane_twiddle(float2 (&v)[N1], const float2* __restrict__ tw, int lane) {
#pragma unroll
  for (int j = 1; j < N1; ++j) {
    float2 w = __ldg(tw + j * 32 + lane);
    if (INV) w.y = -w.y;
    v[j] = cmul(v[j], w);
  }
}

// The inverse 32-point DFT across the lanes for bit-reversed input order
// (decimation in time): the upper lane multiplies by its twiddle first, then
// lower = t + p, upper = p - t; stw are the stages' twiddles (1 on lower
// lanes).  Output in natural lane order.
template <int N1, bool INV>
__device__ __forceinline__ void lane_dit(float2 (&v)[N1], const float2* __restrict__ stw, int lane) {
  {
    // the first stage's twiddles are 1: lower = v + p, upper = p - v
    const float sg = (lane & 1) ? -1.0f : 1.0f;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const float px = __shfl_xor_sync(kFull, v[k1].x, 1);
      const float py = __shfl_xor_sync(kFull, v[k1].y, 1);
      v[k1] = make_float2(fmaf(sg, v[k1].x, px), fmaf(sg, v[k1].y, py));
    }
  }
#pragma unroll
  for (int st = 1; st < 5; ++st) {
    const int d = 1 << st;
    float2 w = __ldg(stw + st * 32 + lane);
    if (INV) w.y = -w.y;
    const float sg = (lane & d) ? -1.0f : 1.0f;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const float2 t = cmul(v[k1], w);
      const float px = __shfl_xor_sync(kFull, t.x, d);
      const float py = __shfl_xor_sync(kFull, t.y, d);
      v[k1] = make_float2(fmaf(sg, t.x, px), fmaf(sg, t.y, py));
    }
  }
}

// Complex line of N = 32 N1 points in registers, lane l holding x[l + 32 m]:
// forward -> register k1 of lane l = X[k1 + N1 brev5(l)]; the inverse takes
// that order back to natural order (unnormalised).  tw is the length's table.
template <int N1>
__device__ __forceinline__ void line_forward(float2 (&v)[N1], const float2* __restrict__ tw, int lane) {
  dft_reg<N1, false>(v);
  lane_twiddle<N1, false>(v, tw, lane);
  lane_dft<N1, false>(v, tw + 32 * N1, lane);
}
template <int N1>
__device__ __forceinline__ void line_inverse(float2 (&v)[N1], const float2* __restrict__ tw, int lane) {
  lane_dit<N1, true>(v, tw + 2 * 32 * N1 + 160, lane);
  lane_twiddle<N1, true>(v, tw, lane);
  dft_reg<N1, true>(v);
}

// Position of frequency k in a staged row.
template <int N1>
__device__ __forceinline__ int stage_pos(int k) {
  if constexpr (N1 % 2 == 0) {
    return k + k / N1;
  } else {
    return k;
  }
}

template <int N1>
__global__ void __launch_bounds__(kXThreads) k_rfft_x(const float* __restrict__ grid, int My, int Mz, int nkx,
                                                      int rs, const float2* __restrict__ tw,
                                                      float2* __restrict__ spec) {
  constexpr int N = 32 * N1, Mxp = N + 2;
  extern __shared__ float2 stage[];   // [kRows][rs]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ychunks = (My + kRows - 1) / kRows;
  const int yc = blockIdx.x % ychunks, cz = blockIdx.x / ychunks;   // cz = c Mz + z
  const int z = cz % Mz, c = cz / Mz;
  const int y0 = yc * kRows, ya = y0 + 2 * warp;
  const int64_t plane = int64_t(Mz) * My;
  if (ya < My) {
    const bool hasb = ya + 1 < My;
    const float* ra = grid + (int64_t(cz) * My + ya) * Mxp;
    float2 v[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      v[m].x = ra[lane + 32 * m];
      v[m].y = hasb ? ra[Mxp + lane + 32 * m] : 0.0f;
    }
    dft_reg<N1, false>(v);
    lane_twiddle<N1, false>(v, tw, lane);
    lane_dft<N1, false>(v, tw + N, lane);
    // Z[k], k = k1 + N1 r with r = brev5(lane); Z[N - k] is register N1 - k1
    // of lane 31 - lane (k1 > 0) or register 0 of lane brev5((32 - r) mod 32)
    // (k1 = 0).  Row a's spectrum is (Z[k] + conj Z[N-k]) / 2, row b's
    // (Z[k] - conj Z[N-k]) / 2i.
    const int r = int(__brev(unsigned(lane)) >> 27);
    float2* sa = stage + (2 * warp) * rs;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      float2 zm;
      if (k1 == 0) {
        const int src = int(__brev(unsigned((32 - r) & 31)) >> 27);
        zm.x = __shfl_sync(kFull, v[0].x, src);
        zm.y = __shfl_sync(kFull, v[0].y, src);
      } else {
        zm.x = __shfl_xor_sync(kFull, v[N1 - k1].x, 31);
        zm.y = __shfl_xor_sync(kFull, v[N1 - k1].y, 31);
      }
      const int k = k1 + N1 * r;
      if (k < nkx) {
        const float2 zk = v[k1];
        const int pk = stage_pos<N1>(k);
        sa[pk] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        sa[rs + pk] = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
      }
    }
  }
  __syncthreads();
  const int ny = min(kRows, My - y0);
  float2* out = spec + int64_t(c) * (N / 2 + 1) * plane + int64_t(z) * My + y0;
  for (int e = threadIdx.x; e < nkx * kRows; e += kXThreads) {
    const int k = e / kRows, yl = e % kRows;
    if (yl < ny) out[int64_t(k) * plane + yl] = stage[yl * rs + stage_pos<N1>(k)];
  }
}

// Inverse real transform of two staged rows (sa and sa + rs, spectra at the
// staged positions of k < nkx) packed as one complex row: the Hermitian
// spectra at k are given for k < nkx, conjugate mirrors for N - k < nkx,
// zero between (the DC imaginary parts dropped); afterwards register k1 of
// lane l holds x[32 k1 + brev5(l)] of the first row (.x) and second (.y).
template <int N1>
__device__ __forceinline__ void irfft_rows(const float2* sa, int rs, int nkx, const float2* __restrict__ tw,
                                           int lane, float2 (&v)[N1]) {
  constexpr int N = 32 * N1;
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) {
    const int k = n1 + N1 * lane;
    float2 a = make_float2(0.0f, 0.0f), b = a;
    if (k < nkx) {
      const int pk = stage_pos<N1>(k);
      a = sa[pk];
      b = sa[rs + pk];
      if (k == 0) a.y = b.y = 0.0f;
    } else if (N - k < nkx) {
      const int pk = stage_pos<N1>(N - k);
      a = sa[pk];
      b = sa[rs + pk];
      a.y = -a.y;
      b.y = -b.y;
    }
    v[n1] = make_float2(a.x - b.y, a.y + b.x);   // A + i B
  }
  lane_dft<N1, true>(v, tw + N, lane);
  lane_twiddle<N1, true>(v, tw + N + 160, lane);
  dft_reg<N1, true>(v);
}

template <int N1>
__global__ void __launch_bounds__(kXThreads) k_irfft_x(const float2* __restrict__ spec, int My, int Mz, int nkx,
                                                       int rs, const float2* __restrict__ tw,
                                                       float* __restrict__ grid) {
  constexpr int N = 32 * N1, Mxp = N + 2;
  extern __shared__ float2 stage[];   // [kRows][rs]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ychunks = (My + kRows - 1) / kRows;
  const int yc = blockIdx.x % ychunks, cz = blockIdx.x / ychunks;
  const int z = cz % Mz, c = cz / Mz;
  const int y0 = yc * kRows, ya = y0 + 2 * warp;
  const int64_t plane = int64_t(Mz) * My;
  const int ny = min(kRows, My - y0);
  const float2* in = spec + int64_t(c) * (N / 2 + 1) * plane + int64_t(z) * My + y0;
#pragma unroll 4
  for (int e = threadIdx.x; e < nkx * kRows; e += kXThreads) {
    const int k = e / kRows, yl = e % kRows;
    stage[yl * rs + stage_pos<N1>(k)] = yl < ny ? in[int64_t(k) * plane + yl] : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  if (ya >= My) return;
  const bool hasb = ya + 1 < My;
  float2 v[N1];
  irfft_rows<N1>(stage + (2 * warp) * rs, rs, nkx, tw, lane, v);
  // register k1 of lane l is x[32 k1 + brev5(l)]: 128 contiguous bytes per store
  float* ra = grid + (int64_t(cz) * My + ya) * Mxp + int(__brev(unsigned(lane)) >> 27);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    ra[32 * k1] = v[k1].x;
    if (hasb) ra[Mxp + 32 * k1] = v[k1].y;
  }
}

// The same inverse writing the grid as channel quadruples: a CTA takes one
// y row per warp of one z plane for the four channels of a quadruple; warp
// w transforms its row's channels (0, 1) and (2, 3) as two complex rows,
// so each lane holds the four channels of its points (register k1 of lane
// l is x = 32 k1 + brev5(l)) and stores them as 16-byte words, the warp's
// 32 lanes covering 32 consecutive points.  Four CTAs per SM (at most 64
// registers): 0.787 -> 0.772 ms per 384^3 inverse transform against the
// row stage in shared memory, and 0.934 ms at the 104 registers the
// compiler takes unbounded.
constexpr int kRowsQ = kXThreads / 32;   // y rows per quadruple CTA
template <int N1>
__global__ void __launch_bounds__(kXThreads, 4) k_irfft_x4(const float2* __restrict__ spec, int My, int Mz, int nkx,
                                                        int rs, const float2* __restrict__ tw,
                                                        float4* __restrict__ grid4) {
  constexpr int N = 32 * N1, Mxp = N + 2;
  extern __shared__ float2 stage[];   // [kRowsQ y rows][4 channels][rs]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ychunks = (My + kRowsQ - 1) / kRowsQ;
  const int yc = blockIdx.x % ychunks, qz = blockIdx.x / ychunks;
  const int z = qz % Mz, q = qz / Mz;
  const int y0 = yc * kRowsQ;
  const int64_t plane = int64_t(Mz) * My;
  const int ny = min(kRowsQ, My - y0);
  {
    // a thread's line (channel c, row yl) is the same at every step; the
    // rows of one channel are adjacent in the spectrum
    static_assert(kXThreads % (4 * kRowsQ) == 0, "whole line groups per step");
    const int r = threadIdx.x % (4 * kRowsQ), c = r / kRowsQ, yl = r % kRowsQ;
    const bool ok = yl < ny;
    const float2* src = spec + int64_t(4 * q + c) * (N / 2 + 1) * plane + int64_t(z) * My + y0 + (ok ? yl : 0);
    float2* dst = stage + (yl * 4 + c) * rs;
#pragma unroll 4
    for (int k = threadIdx.x / (4 * kRowsQ); k < nkx; k += kXThreads / (4 * kRowsQ))
      dst[stage_pos<N1>(k)] = ok ? src[int64_t(k) * plane] : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  if (warp < ny) {
    float2 v[N1], w[N1];
    irfft_rows<N1>(stage + (warp * 4) * rs, rs, nkx, tw, lane, v);       // channels 0 and 1
    irfft_rows<N1>(stage + (warp * 4 + 2) * rs, rs, nkx, tw, lane, w);   // channels 2 and 3
    float4* out = grid4 + ((int64_t(q) * Mz + z) * My + y0 + warp) * Mxp + int(__brev(unsigned(lane)) >> 27);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) out[32 * k1] = make_float4(v[k1].x, v[k1].y, w[k1].x, w[k1].y);
  }
}

// ---- (z, y) passes of the fully own transform ---------------------------------
constexpr int kColTile = 16;   // y columns per z-pass CTA
constexpr int kColStride = kColTile + 1;

// z pass over the nkx planes: a CTA stages 16 y columns of one (c, kx) plane
// ([z][y], odd stride, cp.async), a warp transforms one column at a time in
// place.  Forward: natural z in, column position l + 32 k1 holds
// kz = k1 + N1 brev5(l), and only positions whose (kx, kz) line can hold
// band modes (lmask[kx][pos]) are stored; inverse: that order in (other
// positions read as zero), natural z out.
template <int N1, bool INV>
__global__ void __launch_bounds__(256) k_fft_z(float2* __restrict__ spec, int My, int nkx, int64_t chan,
                                               const float2* __restrict__ tw, const unsigned char* __restrict__ lmask) {
  constexpr int Mz = 32 * N1;
  extern __shared__ float2 tile[];   // [Mz][kColStride]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ych = (My + kColTile - 1) / kColTile;
  const int yc = blockIdx.x % ych, ck = blockIdx.x / ych;   // ck = c nkx + kx
  const int kx = ck % nkx, c = ck / nkx;
  const int y0 = yc * kColTile, ny = min(kColTile, My - y0);
  float2* base = spec + int64_t(c) * chan + int64_t(kx) * Mz * My + y0;
  const unsigned char* mk = lmask + int64_t(kx) * Mz;
  for (int e = threadIdx.x; e < Mz * kColTile; e += 256) {
    const int z = e / kColTile, yl = e % kColTile;
    float2* dst = tile + z * kColStride + yl;
    if (yl < ny && (!INV || mk[z]))
      cp_async8(dst, base + int64_t(z) * My + yl);
    else
      *dst = make_float2(0.0f, 0.0f);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  for (int col = warp; col < ny; col += 8) {
    float2 v[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) v[m] = tile[(lane + 32 * m) * kColStride + col];
    if (INV)
      line_inverse<N1>(v, tw, lane);
    else
      line_forward<N1>(v, tw, lane);
#pragma unroll
    for (int m = 0; m < N1; ++m) tile[(lane + 32 * m) * kColStride + col] = v[m];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < Mz * kColTile; e += 256) {
    const int z = e / kColTile, yl = e % kColTile;
    if (yl < ny && (INV || mk[z])) base[int64_t(z) * My + yl] = tile[z * kColStride + yl];
  }
}

// Steps (iii)-(iv) fused with the y transforms.  A warp takes y lines from
// the list of lines that can hold band modes (lines[j] = kx << 16 | pz, pz a
// column position of the z pass, kz = (pz >> 5) + N1z brev5(pz & 31)),
// double-buffered in shared memory by cp.async; transforms the line forward
// in registers, writes it back in its output order (position l + 32 k1 =
// ky = k1 + N1 brev5(l)) and multiplies each mode by
//   G = scale_c sing_p(k) (S_p(u) + log part) iw2x iw2y iw2z
// (zero outside |k| < k_c and at k = 0), adding w_m G |rho-hat|^2 / 2 to the
// energy (kx = 0 counted once) and, with vpart, the virial's log-derivative
// sums; then transforms it back and stores it.  Energy partials per block in
// FP64 (part[c][blocks]).  Three CTAs per SM (at most 80 registers): 0.315
// against 0.346 ms per 384^3 step at the 64 registers, with spills, that
// the compiler took for four.
template <int N1>
__global__ void __launch_bounds__(256, 3) k_mult_y(float2* __restrict__ spec, MultParams mp, int64_t chan,
                                                const int* __restrict__ lines, int nlines,
                                                const int* __restrict__ pch, const double* __restrict__ scale,
                                                const double* __restrict__ bmat, const float* __restrict__ coef,
                                                const float* __restrict__ iw2, int iw2_stride,
                                                const float2* __restrict__ tw, double* __restrict__ part,
                                                int want_energy, double* __restrict__ vpart) {
  constexpr int My = 32 * N1;
  extern __shared__ float2 lbuf[];   // [8 warps][2][My]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* wbuf = lbuf + warp * 2 * My;
  const int c = blockIdx.y;
  const int p = pch[c];
  const int Mz = mp.M[2], N1z = Mz >> 5;
  const float sc = float(scale[c]);
  const float* cf = coef + size_t(p - 1) * kMultSeg * (mp.deg + 1);
  const float* iw2x = iw2;
  const float* iw2y = iw2x + iw2_stride;
  const float* iw2z = iw2y + iw2_stride;
  const float kc2 = float(1.0 / (mp.inv_kc * mp.inv_kc));
  const float inv_kc = float(mp.inv_kc);
  float bm[9];   // k = B m, B = 2 pi H^-1 (diagonal for a box)
#pragma unroll
  for (int i = 0; i < 9; ++i) bm[i] = float(bmat[i]);
  float2* sp = spec + int64_t(c) * chan;
  auto line_at = [&](int j) { return sp + (int64_t(lines[j] >> 16) * Mz + (lines[j] & 0xFFFF)) * My; };
  auto fetch = [&](int j, float2* dst) {
    const float2* src = line_at(j);
#pragma unroll
    for (int m = 0; m < N1; ++m) cp_async8(dst + lane + 32 * m, src + lane + 32 * m);
  };
  EnergyAcc<float> e;
  double vt[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const int jstep = gridDim.x * 8;
  int j = blockIdx.x * 8 + warp, cur = 0;
  if (j < nlines) fetch(j, wbuf);
  cp_async_commit();
  for (; j < nlines; j += jstep, cur ^= 1) {
    __syncwarp();   // the other buffer's previous line is consumed
    if (j + jstep < nlines) fetch(j + jstep, wbuf + (cur ^ 1) * My);
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();
    float2* b = wbuf + cur * My;
    const int kx = lines[j] >> 16, pz = lines[j] & 0xFFFF;
    const int kz = (pz >> 5) + N1z * int(__brev(unsigned(pz & 31)) >> 27);
    const int mz = kz <= Mz / 2 ? kz : kz - Mz;
    // the line's part of k (kx and kz modes); + my b_y per mode
    const float lx = bm[0] * float(kx) + bm[2] * float(mz), ly = bm[3] * float(kx) + bm[5] * float(mz),
                lz = bm[6] * float(kx) + bm[8] * float(mz);
    float2 v[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) v[m] = b[lane + 32 * m];
    line_forward<N1>(v, tw, lane);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) b[lane + 32 * k1] = v[k1];
    __syncwarp();
    const float wxz = sc * iw2x[kx] * iw2z[mz < 0 ? -mz : mz];
    const float wedge = kx == 0 ? 0.5f : 1.0f;
    for (int q = lane; q < My; q += 32) {
      const int ky = (q >> 5) + N1 * int(__brev(unsigned(q & 31)) >> 27);
      const int my = ky <= My / 2 ? ky : ky - My;
      const float fkx = lx + bm[1] * float(my), fky = ly + bm[4] * float(my), fkz = lz + bm[7] * float(my);
      const float k2 = fkx * fkx + fky * fky + fkz * fkz;
      float2 x = b[q];
      if (!(k2 < kc2) || k2 == 0.0f) {
        x = make_float2(0.0f, 0.0f);
      } else {
        const float k = sqrtf(k2);
        float u = k * inv_kc;
        if (u >= 1.0f) u = 1.0f - 1e-7f;
        int seg = int(u * float(kMultSeg));
        if (seg > kMultSeg - 1) seg = kMultSeg - 1;
        const float sv = 2.0f * (u * float(kMultSeg) - float(seg)) - 1.0f;
        const float* cs = cf + seg * (mp.deg + 1);
        const float S = mult_horner(cs, mp.deg, sv);
        const float phi = mult_value(p, S, k, k2, u);
        const float G = phi * wxz * iw2y[my < 0 ? -my : my];
        if (want_energy) {
          const float em = wedge * G * (x.x * x.x + x.y * x.y);
          e.add(em);
          if (vpart) {
            const float dS = mult_horner_d(cs, mp.deg, sv);
            const double dl = double(mult_dlog(p, S, dS * float(2 * kMultSeg), u, phi)) / double(k2);
            virial_add(vt, double(em) * dl, double(fkx), double(fky), double(fkz));
          }
        }
        x.x *= G;
        x.y *= G;
      }
      b[q] = x;
    }
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = b[lane + 32 * k1];
    line_inverse<N1>(v, tw, lane);
    float2* ln = line_at(j);
#pragma unroll
    for (int m = 0; m < N1; ++m) ln[lane + 32 * m] = v[m];
  }
  cp_async_wait<0>();
  if (!want_energy) return;
  block_partials(e.value(), vt, part, vpart, size_t(c) * gridDim.x + blockIdx.x);
}

template <int N1>
cudaError_t launch_n1(bool forward, const void* in, int My, int Mz, int K, int nkx, const void* tw, void* out,
                      cudaStream_t s, bool il) {
  // staged row stride: past the last position, odd
  int rs = (nkx - 1) + ((N1 % 2 == 0) ? (nkx - 1) / N1 : 0) + 1;
  rs += (rs % 2 == 0) ? 1 : 0;
  const size_t smem = size_t(kRows) * rs * sizeof(float2);
  const int64_t blocks = int64_t(K) * Mz * ((My + kRows - 1) / kRows);
  if (blocks == 0 || nkx <= 0) return cudaSuccess;
  if (forward) {
    if (smem > 32 * 1024) {   // opt in early: static shared memory counts too
      const cudaError_t e = cudaFuncSetAttribute(k_rfft_x<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    k_rfft_x<N1><<<unsigned(blocks), kXThreads, smem, s>>>(static_cast<const float*>(in), My, Mz, nkx, rs,
                                                             static_cast<const float2*>(tw), static_cast<float2*>(out));
  } else {
    if (il) {
      const size_t smem4 = size_t(4 * kRowsQ) * rs * sizeof(float2);
      const int64_t blocks4 = int64_t(K / 4) * Mz * ((My + kRowsQ - 1) / kRowsQ);
      if (smem4 > 32 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_irfft_x4<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem4));
        if (e != cudaSuccess) return e;
      }
      k_irfft_x4<N1><<<unsigned(blocks4), kXThreads, smem4, s>>>(static_cast<const float2*>(in), My, Mz, nkx, rs,
                                                                  static_cast<const float2*>(tw),
                                                                  static_cast<float4*>(out));
      return cudaGetLastError();
    }
    if (smem > 32 * 1024) {   // opt in early: static shared memory counts too
      const cudaError_t e = cudaFuncSetAttribute(k_irfft_x<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    k_irfft_x<N1><<<unsigned(blocks), kXThreads, smem, s>>>(static_cast<const float2*>(in), My, Mz, nkx, rs,
                                                              static_cast<const float2*>(tw), static_cast<float*>(out));
  }
  return cudaGetLastError();
}

cudaError_t dispatch(bool forward, int Mx, const void* in, int My, int Mz, int K, int nkx, const void* tw, void* out,
                     cudaStream_t s, bool il = false) {
  if (!xfft_supported(Mx) || nkx > Mx / 2 || (il && K % 4 != 0)) return cudaErrorInvalidValue;
  switch (Mx / 32) {
    case 2: return launch_n1<2>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 3: return launch_n1<3>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 4: return launch_n1<4>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 5: return launch_n1<5>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 6: return launch_n1<6>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 7: return launch_n1<7>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 8: return launch_n1<8>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 9: return launch_n1<9>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 10: return launch_n1<10>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 11: return launch_n1<11>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 12: return launch_n1<12>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 13: return launch_n1<13>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 14: return launch_n1<14>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 15: return launch_n1<15>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    case 16: return launch_n1<16>(forward, in, My, Mz, K, nkx, tw, out, s, il);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool xfft_supported(int Mx) { return Mx % 32 == 0 && Mx >= 64 && Mx <= 512; }

int xfft_table_size(int Mx) { return 2 * Mx + 10 * 32; }

void xfft_twiddles(int Mx, std::vector<float>& out) {
  const int N1 = Mx / 32;
  out.assign(2 * size_t(xfft_table_size(Mx)), 0.0f);
  const double two_pi = 2.0 * 3.14159265358979323846;
  auto put = [&](int idx, long j, long n) {
    const double a = two_pi * double(j % n) / double(n);
    out[2 * size_t(idx)] = float(std::cos(a));
    out[2 * size_t(idx) + 1] = float(-std::sin(a));
  };
  for (int k1 = 0; k1 < N1; ++k1)
    for (int l = 0; l < 32; ++l) put(k1 * 32 + l, long(l) * k1, Mx);
  // stage st (distance d = 16 >> st): 1 on lower lanes, -W_{2d}^{l mod d}
  // on upper lanes
  for (int st = 0; st < 5; ++st) {
    const int d = 16 >> st;
    for (int l = 0; l < 32; ++l) {
      const int idx = Mx + st * 32 + l;
      if (l & d) {
        put(idx, l % d, 2L * d);
        out[2 * size_t(idx)] = -out[2 * size_t(idx)];
        out[2 * size_t(idx) + 1] = -out[2 * size_t(idx) + 1];
      } else {
        out[2 * size_t(idx)] = 1.0f;
        out[2 * size_t(idx) + 1] = 0.0f;
      }
    }
  }
  // inverse twiddles between the lanes and the registers
  for (int n1 = 0; n1 < N1; ++n1)
    for (int l = 0; l < 32; ++l) {
      int r = 0;
      for (int b = 0; b < 5; ++b) r |= ((l >> b) & 1) << (4 - b);
      put(Mx + 160 + n1 * 32 + l, long(n1) * r, Mx);
    }
  // decimation-in-time stages st < 5 (distance d = 1 << st): e^{-2 pi i
  // (l mod d) / 2d} on lanes with l & d set, 1 on the others
  for (int st = 0; st < 5; ++st) {
    const int d = 1 << st;
    for (int l = 0; l < 32; ++l) {
      const int idx = 2 * Mx + 160 + st * 32 + l;
      if (l & d) {
        put(idx, l % d, 2L * d);
      } else {
        out[2 * size_t(idx)] = 1.0f;
        out[2 * size_t(idx) + 1] = 0.0f;
      }
    }
  }
}

cudaError_t launch_rfft_x(const float* grid, int Mx, int My, int Mz, int K, int nkx, const void* tw, void* spec,
                          cudaStream_t s) {
  return dispatch(true, Mx, grid, My, Mz, K, nkx, tw, spec, s);
}

cudaError_t launch_irfft_x(const void* spec, int Mx, int My, int Mz, int K, int nkx, const void* tw, float* grid,
                           cudaStream_t s, bool interleave4) {
  return dispatch(false, Mx, spec, My, Mz, K, nkx, tw, grid, s, interleave4);
}

namespace {
template <int N1, bool INV>
cudaError_t launch_z_n1(void* spec, int My, int K, int nkx, int64_t chan, const void* tw, const unsigned char* lmask,
                        cudaStream_t s) {
  const size_t smem = size_t(32 * N1) * kColStride * sizeof(float2);
  if (smem > 32 * 1024) {   // opt in early: static shared memory counts too
    const cudaError_t e = cudaFuncSetAttribute(k_fft_z<N1, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = int64_t(K) * nkx * ((My + kColTile - 1) / kColTile);
  k_fft_z<N1, INV><<<unsigned(blocks), 256, smem, s>>>(static_cast<float2*>(spec), My, nkx, chan,
                                                      static_cast<const float2*>(tw), lmask);
  return cudaGetLastError();
}
template <bool INV>
cudaError_t launch_z(int Mz, void* spec, int My, int K, int nkx, int64_t chan, const void* tw,
                     const unsigned char* lmask, cudaStream_t s) {
  switch (Mz / 32) {
    case 2: return launch_z_n1<2, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 3: return launch_z_n1<3, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 4: return launch_z_n1<4, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 5: return launch_z_n1<5, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 6: return launch_z_n1<6, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 7: return launch_z_n1<7, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 8: return launch_z_n1<8, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 9: return launch_z_n1<9, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 10: return launch_z_n1<10, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 11: return launch_z_n1<11, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 12: return launch_z_n1<12, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 13: return launch_z_n1<13, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 14: return launch_z_n1<14, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 15: return launch_z_n1<15, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    case 16: return launch_z_n1<16, INV>(spec, My, K, nkx, chan, tw, lmask, s);
    default: return cudaErrorInvalidValue;
  }
}
template <int N1>
cudaError_t launch_mult_n1(const MultArgs& a, cudaStream_t s) {
  const size_t smem = size_t(8) * 2 * 32 * N1 * sizeof(float2);
  if (smem > 32 * 1024) {   // opt in early: static shared memory counts too
    const cudaError_t e = cudaFuncSetAttribute(k_mult_y<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  k_mult_y<N1><<<dim3(a.blocks, a.K), 256, smem, s>>>(
      static_cast<float2*>(a.spec), a.mp, a.chan, a.lines, a.nlines, a.pch, a.scale, a.bmat,
      static_cast<const float*>(a.coef), static_cast<const float*>(a.iw2), a.iw2_stride,
      static_cast<const float2*>(a.tw), a.part, a.want_energy, a.vpart);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_fft_z(bool inverse, void* spec, int Mz, int My, int K, int nkx, int64_t chan, const void* tw,
                         const unsigned char* lmask, cudaStream_t s) {
  if (!xfft_supported(Mz)) return cudaErrorInvalidValue;
  if (K == 0 || nkx <= 0 || My <= 0) return cudaSuccess;
  return inverse ? launch_z<true>(Mz, spec, My, K, nkx, chan, tw, lmask, s)
                 : launch_z<false>(Mz, spec, My, K, nkx, chan, tw, lmask, s);
}

void xfft_band_lines(int nkx, int My, int Mz, const double bmat[9], double k_c, std::vector<unsigned char>& mask,
                     std::vector<int>& lines) {
  const int n1z = Mz / 32;
  const double by[3] = {bmat[1], bmat[4], bmat[7]};
  const double bb = by[0] * by[0] + by[1] * by[1] + by[2] * by[2];
  const int mlo = -((My - 1) / 2), mhi = My / 2;   // signed y modes of the kernels
  mask.assign(size_t(nkx) * Mz, 0);
  lines.clear();
  for (int kx = 0; kx < nkx; ++kx)
    for (int pz = 0; pz < Mz; ++pz) {
      int r = 0;
      for (int b = 0; b < 5; ++b) r |= (((pz & 31) >> b) & 1) << (4 - b);
      const int kz = (pz >> 5) + n1z * r;
      const int mz = kz <= Mz / 2 ? kz : kz - Mz;
      const double l[3] = {bmat[0] * kx + bmat[2] * mz, bmat[3] * kx + bmat[5] * mz, bmat[6] * kx + bmat[8] * mz};
      // |l + my b_y|^2 is convex in my: its integer minimum over the line's
      // modes is at the clamped floor or ceiling of the real minimiser
      const double mstar = -(l[0] * by[0] + l[1] * by[1] + l[2] * by[2]) / bb;
      double best = 1e300;
      for (double mc : {std::floor(mstar), std::floor(mstar) + 1.0}) {
        const double my = std::min(double(mhi), std::max(double(mlo), mc));
        double k2 = 0.0;
        for (int e = 0; e < 3; ++e) k2 += (l[e] + my * by[e]) * (l[e] + my * by[e]);
        best = std::min(best, k2);
      }
      if (best < k_c * k_c) {
        mask[size_t(kx) * Mz + pz] = 1;
        lines.push_back((kx << 16) | pz);
      }
    }
}

cudaError_t launch_mult_y(const MultArgs& a, cudaStream_t s) {
  if (!xfft_supported(a.mp.M[1]) || !xfft_supported(a.mp.M[2])) return cudaErrorInvalidValue;
  if (a.K == 0 || a.blocks <= 0 || a.nlines <= 0) return cudaSuccess;
  switch (a.mp.M[1] / 32) {
    case 2: return launch_mult_n1<2>(a, s);
    case 3: return launch_mult_n1<3>(a, s);
    case 4: return launch_mult_n1<4>(a, s);
    case 5: return launch_mult_n1<5>(a, s);
    case 6: return launch_mult_n1<6>(a, s);
    case 7: return launch_mult_n1<7>(a, s);
    case 8: return launch_mult_n1<8>(a, s);
    case 9: return launch_mult_n1<9>(a, s);
    case 10: return launch_mult_n1<10>(a, s);
    case 11: return launch_mult_n1<11>(a, s);
    case 12: return launch_mult_n1<12>(a, s);
    case 13: return launch_mult_n1<13>(a, s);
    case 14: return launch_mult_n1<14>(a, s);
    case 15: return launch_mult_n1<15>(a, s);
    case 16: return launch_mult_n1<16>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pswf
