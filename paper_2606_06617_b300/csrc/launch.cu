// Per-precision instantiation of the stencil kernels (spread / interp) for
// every stencil width P in 2..16.  Compiled with -DPSWF_REAL=float|double.
#include <algorithm>
#include <cstring>

#include "launch.cuh"

#ifndef PSWF_REAL
#error "define PSWF_REAL as float or double"
#endif
#define PSWF_CAT2(a, b) a##_##b
#define PSWF_CAT(a, b) PSWF_CAT2(a, b)

namespace pswf {
namespace {

using R = PSWF_REAL;
constexpr int kThreads = 256;

WinCoef<R> win_coef(const LaunchCtx& c) {
  WinCoef<R> w;
  std::memset(&w, 0, sizeof(w));
  w.deg = c.deg_w;
  const int n = c.geo.P * (c.deg_w + 1);
  for (int i = 0; i < n; ++i) w.c[i] = R(c.coef_w[i]);
  return w;
}

template <int P>
cudaError_t spread_P(const LaunchCtx& c, int* nlaunch) {
  constexpr int S = kTile + P - 1;
  const int64_t S3 = int64_t(S) * S * S;
  const int max_smem = 96 * 1024;
  int kc = int(std::max<int64_t>(1, max_smem / (S3 * int64_t(sizeof(R)))));
  kc = std::min(kc, c.geo.K);
  const size_t smem = size_t(kc) * S3 * sizeof(R);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_spread<R, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  const WinCoef<R> wc = win_coef(c);
  const int blocks = std::min(c.ntiles, 148 * 16);
  for (int c0 = 0; c0 < c.geo.K; c0 += kc) {
    const int nk = std::min(kc, c.geo.K - c0);
    k_spread<R, P><<<blocks, kThreads, smem, c.stream>>>(c.geo, c.nmax, c.tile_start, static_cast<const R*>(c.st),
                                                         c.scell, static_cast<const R*>(c.sq), c0, nk, wc,
                                                         static_cast<R*>(c.grid));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ++*nlaunch;
  }
  return cudaSuccess;
}

template <int P>
cudaError_t interp_P(const LaunchCtx& c, void* phi, void* forces, int* nlaunch) {
  if (c.n == 0) return cudaSuccess;
  ++*nlaunch;
  const WinCoef<R> wc = win_coef(c);
  const int blocks = int(std::min<int64_t>((c.n + kThreads - 1) / kThreads, 148 * 32));
  k_interp<R, P><<<blocks, kThreads, 0, c.stream>>>(c.n, c.nmax, c.geo, static_cast<const R*>(c.st), c.scell,
                                                    static_cast<const R*>(c.sq), c.sperm, wc,
                                                    static_cast<const R*>(c.grid), c.zero_coef, c.charges,
                                                    static_cast<R*>(phi), static_cast<R*>(forces));
  return cudaGetLastError();
}

}  // namespace

#define PSWF_P_CASES(F, ...)                                                                              \
  switch (c.geo.P) {                                                                                      \
    case 2: return F<2>(__VA_ARGS__);   case 3: return F<3>(__VA_ARGS__);   case 4: return F<4>(__VA_ARGS__); \
    case 5: return F<5>(__VA_ARGS__);   case 6: return F<6>(__VA_ARGS__);   case 7: return F<7>(__VA_ARGS__); \
    case 8: return F<8>(__VA_ARGS__);   case 9: return F<9>(__VA_ARGS__);   case 10: return F<10>(__VA_ARGS__); \
    case 11: return F<11>(__VA_ARGS__); case 12: return F<12>(__VA_ARGS__); case 13: return F<13>(__VA_ARGS__); \
    case 14: return F<14>(__VA_ARGS__); case 15: return F<15>(__VA_ARGS__); case 16: return F<16>(__VA_ARGS__); \
  }                                                                                                       \
  return cudaErrorInvalidValue;

cudaError_t PSWF_CAT(launch_spread, PSWF_REAL)(const LaunchCtx& c, int* nlaunch) {
  PSWF_P_CASES(spread_P, c, nlaunch)
}

cudaError_t PSWF_CAT(launch_interp, PSWF_REAL)(const LaunchCtx& c, void* phi, void* forces, int* nlaunch) {
  PSWF_P_CASES(interp_P, c, phi, forces, nlaunch)
}

}  // namespace pswf
