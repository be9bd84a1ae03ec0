// Pruned real transforms along x (FP32), see fft_x.hpp.
//
// One warp transforms one complex row of length N = 32 N1 holding two real
// grid rows (real and imaginary parts).  Lane l starts with the N1 samples
// x[brev5(l) + 32 m], m < N1, and the transform is the four-step split
// N = N1 x 32:
//   1. an N1-point DFT over m in registers (radix 2, odd remainders directly,
//      twiddles compile-time constants),
//   2. the twiddle e^{-+2 pi i brev5(l) k1 / N},
//   3. a 32-point transform across the lanes (decimation in time: the lanes
//      hold bit-reversed inputs, five butterfly stages of xor shuffles),
// after which lane l, register k1 holds X[k1 + N1 l].  The two real rows'
// spectra are split from X[k] and X[N - k] (one more shuffle), and a CTA of
// 16 warps (32 rows of one (c, z) line) stages the kx < nkx part as
// [kx][y] in shared memory so that each kx is one 256-byte store.  The
// inverse runs the same steps backwards: staged loads, the Hermitian
// completion of both rows' spectra packed as A + i B, the inverse transform,
// and the two real rows as the real and imaginary parts.
#include "fft_x.hpp"

#include <cmath>
#include <cstdint>
#include <utility>

namespace pswf {
namespace {

constexpr int kXThreads = 512;     // 16 warps, two rows each: 32 rows of a (c, z) line
constexpr int kStage = 33;         // float2 per kx in the staging tile (32 rows + 1)
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

// Length-32 N1 transform of a warp's row (layout in the file comment).
template <int N1, bool INV>
__device__ __forceinline__ void warp_fft(float2 (&v)[N1], const float2* __restrict__ tw, int lane) {
  constexpr int N = 32 * N1;
  dft_reg<N1, INV>(v);
#pragma unroll
  for (int k1 = 1; k1 < N1; ++k1) {
    float2 w = __ldg(tw + k1 * 32 + lane);
    if (INV) w.y = -w.y;
    v[k1] = cmul(v[k1], w);
  }
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int d = 1 << s;
    float2 w = __ldg(tw + N + s * 32 + lane);   // W_{2d}^{lane mod d}
    if (INV) w.y = -w.y;
    const bool upper = (lane & d) != 0;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      float2 p;
      p.x = __shfl_xor_sync(kFull, v[k1].x, d);
      p.y = __shfl_xor_sync(kFull, v[k1].y, d);
      // lower lane: a + W b (b = partner); upper lane: a - W b (a = partner)
      const float2 a = upper ? p : v[k1];
      const float2 t = cmul(upper ? v[k1] : p, w);
      v[k1] = upper ? csub(a, t) : cadd(a, t);
    }
  }
}

template <int N1>
__global__ void __launch_bounds__(kXThreads) k_rfft_x(const float* __restrict__ grid, int My, int Mz, int nkx,
                                                      const float2* __restrict__ tw, float2* __restrict__ spec) {
  constexpr int N = 32 * N1, Mxp = N + 2;
  extern __shared__ float2 stage[];   // [nkx][kStage]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ychunks = (My + 31) >> 5;
  const int yc = blockIdx.x % ychunks, cz = blockIdx.x / ychunks;   // cz = c Mz + z
  const int z = cz % Mz, c = cz / Mz;
  const int y0 = yc * 32, ya = y0 + 2 * warp;
  const int64_t plane = int64_t(Mz) * My;
  if (ya < My) {
    const bool hasb = ya + 1 < My;
    const float* ra = grid + (int64_t(cz) * My + ya) * Mxp;
    const int n2 = int(__brev(unsigned(lane)) >> 27);
    float2 v[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      v[m].x = ra[n2 + 32 * m];
      v[m].y = hasb ? ra[Mxp + n2 + 32 * m] : 0.0f;
    }
    warp_fft<N1, false>(v, tw, lane);
    // Z[k], k = k1 + N1 lane; Z[N - k] is register N1 - k1 of lane 31 - lane
    // (k1 > 0) or register 0 of lane (32 - lane) mod 32 (k1 = 0).  Row a's
    // spectrum is (Z[k] + conj Z[N-k]) / 2, row b's (Z[k] - conj Z[N-k]) / 2i.
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      float2 zm;
      if (k1 == 0) {
        const int src = (32 - lane) & 31;
        zm.x = __shfl_sync(kFull, v[0].x, src);
        zm.y = __shfl_sync(kFull, v[0].y, src);
      } else {
        zm.x = __shfl_xor_sync(kFull, v[N1 - k1].x, 31);
        zm.y = __shfl_xor_sync(kFull, v[N1 - k1].y, 31);
      }
      const int k = k1 + N1 * lane;
      if (k < nkx) {
        const float2 zk = v[k1];
        stage[k * kStage + 2 * warp] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        stage[k * kStage + 2 * warp + 1] = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
      }
    }
  }
  __syncthreads();
  const int ny = min(32, My - y0);
  float2* out = spec + int64_t(c) * (N / 2 + 1) * plane + int64_t(z) * My + y0;
  for (int e = threadIdx.x; e < nkx * 32; e += kXThreads) {
    const int k = e >> 5, yl = e & 31;
    if (yl < ny) out[int64_t(k) * plane + yl] = stage[k * kStage + yl];
  }
}

template <int N1>
__global__ void __launch_bounds__(kXThreads) k_irfft_x(const float2* __restrict__ spec, int My, int Mz, int nkx,
                                                       const float2* __restrict__ tw, float* __restrict__ grid) {
  constexpr int N = 32 * N1, Mxp = N + 2;
  extern __shared__ float2 stage[];   // [nkx][kStage]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ychunks = (My + 31) >> 5;
  const int yc = blockIdx.x % ychunks, cz = blockIdx.x / ychunks;
  const int z = cz % Mz, c = cz / Mz;
  const int y0 = yc * 32, ya = y0 + 2 * warp;
  const int64_t plane = int64_t(Mz) * My;
  const int ny = min(32, My - y0);
  const float2* in = spec + int64_t(c) * (N / 2 + 1) * plane + int64_t(z) * My + y0;
  for (int e = threadIdx.x; e < nkx * 32; e += kXThreads) {
    const int k = e >> 5, yl = e & 31;
    stage[k * kStage + yl] = yl < ny ? in[int64_t(k) * plane + yl] : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  if (ya >= My) return;
  const bool hasb = ya + 1 < My;
  const int n2 = int(__brev(unsigned(lane)) >> 27);
  float2 v[N1];
#pragma unroll
  for (int m = 0; m < N1; ++m) {
    // both rows' Hermitian spectra at k: given for k < nkx, conjugate
    // mirrors for N - k < nkx, zero between; the DC imaginary parts dropped
    const int k = n2 + 32 * m;
    float2 a = make_float2(0.0f, 0.0f), b = a;
    if (k < nkx) {
      a = stage[k * kStage + 2 * warp];
      b = stage[k * kStage + 2 * warp + 1];
      if (k == 0) a.y = b.y = 0.0f;
    } else if (N - k < nkx) {
      a = stage[(N - k) * kStage + 2 * warp];
      b = stage[(N - k) * kStage + 2 * warp + 1];
      a.y = -a.y;
      b.y = -b.y;
    }
    v[m] = make_float2(a.x - b.y, a.y + b.x);   // A + i B
  }
  warp_fft<N1, true>(v, tw, lane);
  float* ra = grid + (int64_t(cz) * My + ya) * Mxp + N1 * lane;
  if constexpr (N1 % 2 == 0) {
#pragma unroll
    for (int k1 = 0; k1 < N1; k1 += 2) {
      *reinterpret_cast<float2*>(ra + k1) = make_float2(v[k1].x, v[k1 + 1].x);
      if (hasb) *reinterpret_cast<float2*>(ra + Mxp + k1) = make_float2(v[k1].y, v[k1 + 1].y);
    }
  } else {
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      ra[k1] = v[k1].x;
      if (hasb) ra[Mxp + k1] = v[k1].y;
    }
  }
}

template <int N1>
cudaError_t launch_n1(bool forward, const void* in, int My, int Mz, int K, int nkx, const void* tw, void* out,
                      cudaStream_t s) {
  const size_t smem = size_t(nkx) * kStage * sizeof(float2);
  const int64_t blocks = int64_t(K) * Mz * ((My + 31) / 32);
  if (blocks == 0 || nkx <= 0) return cudaSuccess;
  if (forward) {
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(k_rfft_x<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    k_rfft_x<N1><<<unsigned(blocks), kXThreads, smem, s>>>(static_cast<const float*>(in), My, Mz, nkx,
                                                             static_cast<const float2*>(tw), static_cast<float2*>(out));
  } else {
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(k_irfft_x<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
    }
    k_irfft_x<N1><<<unsigned(blocks), kXThreads, smem, s>>>(static_cast<const float2*>(in), My, Mz, nkx,
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

int xfft_table_size(int Mx) { return Mx + 5 * 32; }

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
    for (int l = 0; l < 32; ++l) {
      int r = 0;
      for (int b = 0; b < 5; ++b) r |= ((l >> b) & 1) << (4 - b);
      put(k1 * 32 + l, long(r) * k1, Mx);
    }
  for (int s = 0; s < 5; ++s)
    for (int l = 0; l < 32; ++l) put(Mx + s * 32 + l, l % (1 << s), 2L << s);
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
