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

#include <cmath>
#include <cstdint>
#include <utility>

namespace pswf {
namespace {

constexpr int kRows = 16;                // rows of a (c, z) line per CTA
constexpr int kXThreads = 16 * kRows;    // a warp per pair of rows
constexpr unsigned kFull = 0xffffffffu;

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
  for (int st = 0; st < 5; ++st) {
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
  const float2* sa = stage + (2 * warp) * rs;
  float2 v[N1];
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) {
    // both rows' Hermitian spectra at k: given for k < nkx, conjugate
    // mirrors for N - k < nkx, zero between; the DC imaginary parts dropped
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
  // register k1 of lane l is x[32 k1 + brev5(l)]: 128 contiguous bytes per store
  float* ra = grid + (int64_t(cz) * My + ya) * Mxp + int(__brev(unsigned(lane)) >> 27);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    ra[32 * k1] = v[k1].x;
    if (hasb) ra[Mxp + 32 * k1] = v[k1].y;
  }
}

template <int N1>
cudaError_t launch_n1(bool forward, const void* in, int My, int Mz, int K, int nkx, const void* tw, void* out,
                      cudaStream_t s) {
  // staged row stride: past the last position, odd
  int rs = (nkx - 1) + ((N1 % 2 == 0) ? (nkx - 1) / N1 : 0) + 1;
  rs += (rs % 2 == 0) ? 1 : 0;
  const size_t smem = size_t(kRows) * rs * sizeof(float2);
  const int64_t blocks = int64_t(K) * Mz * ((My + kRows - 1) / kRows);
  if (blocks == 0 || nkx <= 0) return cudaSuccess;
  if (forward) {
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(k_rfft_x<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    k_rfft_x<N1><<<unsigned(blocks), kXThreads, smem, s>>>(static_cast<const float*>(in), My, Mz, nkx, rs,
                                                             static_cast<const float2*>(tw), static_cast<float2*>(out));
  } else {
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(k_irfft_x<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    k_irfft_x<N1><<<unsigned(blocks), kXThreads, smem, s>>>(static_cast<const float2*>(in), My, Mz, nkx, rs,
                                                              static_cast<const float2*>(tw), static_cast<float*>(out));
  }
  return cudaGetLastError();
}

cudaError_t dispatch(bool forward, int Mx, const void* in, int My, int Mz, int K, int nkx, const void* tw, void* out,
                     cudaStream_t s) {
  if (!xfft_supported(Mx) || nkx > Mx / 2) return cudaErrorInvalidValue;
  switch (Mx / 32) {
    case 2: return launch_n1<2>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 3: return launch_n1<3>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 4: return launch_n1<4>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 5: return launch_n1<5>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 6: return launch_n1<6>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 7: return launch_n1<7>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 8: return launch_n1<8>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 9: return launch_n1<9>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 10: return launch_n1<10>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 11: return launch_n1<11>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 12: return launch_n1<12>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 13: return launch_n1<13>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 14: return launch_n1<14>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 15: return launch_n1<15>(forward, in, My, Mz, K, nkx, tw, out, s);
    case 16: return launch_n1<16>(forward, in, My, Mz, K, nkx, tw, out, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool xfft_supported(int Mx) { return Mx % 32 == 0 && Mx >= 64 && Mx <= 512; }

int xfft_table_size(int Mx) { return 2 * Mx + 5 * 32; }

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
}

cudaError_t launch_rfft_x(const float* grid, int Mx, int My, int Mz, int K, int nkx, const void* tw, void* spec,
                          cudaStream_t s) {
  return dispatch(true, Mx, grid, My, Mz, K, nkx, tw, spec, s);
}

cudaError_t launch_irfft_x(const void* spec, int Mx, int My, int Mz, int K, int nkx, const void* tw, float* grid,
                           cudaStream_t s) {
  return dispatch(false, Mx, spec, My, Mz, K, nkx, tw, grid, s);
}

}  // namespace pswf
