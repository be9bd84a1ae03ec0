// Per-precision instantiation of the stencil kernels (spread / interp) for
// every stencil width P in 2..16.  Compiled with -DPSWF_REAL=float|double.
#include <algorithm>
#include <cstring>

#include "launch.cuh"
#include "stencil.cuh"
#include "stencil4.cuh"
#include "backward.cuh"

#ifndef PSWF_REAL
#error "define PSWF_REAL as float or double"
#endif
#define PSWF_CAT2(a, b) a##_##b
#define PSWF_CAT(a, b) PSWF_CAT2(a, b)

namespace pswf {
namespace {

using R = PSWF_REAL;
constexpr int kSmemPerSm = 228 * 1024;   // shared memory per SM on sm_103a (1 KB of it reserved per CTA)
// CTAs of the stencil kernels per SM, each with its own padded region.  Two
// (two channels each, so one CTA's staging, flush and barriers could overlap
// the other's atom loop) measured slower on the 384^3 melt: spread 2.79 /
// gather 3.42 ms against 2.37 / 2.64 ms with one CTA holding all four
// channels (window tables filled twice per atom, half the slots per item).
constexpr int kStencilCtas = 1;
constexpr int kGatherThreads = kGatherThreadsFor<R>;
constexpr int kDirectThreads = 256;

template <typename T = R>
static WinCoef<T> win_coef(const LaunchCtx& c) {
  constexpr int D = WinCoef<T>::kDeg;
  WinCoef<T> w;
  std::memset(&w, 0, sizeof(w));
  w.deg = c.deg_w;
  for (int j = 0; j < c.geo.P; ++j)
    for (int n = 0; n <= c.deg_w && n <= D; ++n) w.c[j * (D + 1) + n] = T(c.coef_w[j * (c.deg_w + 1) + n]);
  return w;
}

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
  }
  return n;
}

// Channels staged per work item (as many as a warp has slots, all of them
// when K is small) and atoms per table batch, within the shared memory left
// beside the kernel's static arrays; false if not even one channel fits.
template <int P, typename Kern, typename F>
bool pick_kc_kb(Kern kern, int K, F bytes, int* kc_out, int* kb_out) {
  cudaFuncAttributes attr;
  if (cudaFuncGetAttributes(&attr, kern) != cudaSuccess) return false;
  const size_t budget = size_t(kSmemPerSm) / kStencilCtas - 1024 - attr.sharedSizeBytes;
  for (int kc = std::min(K, TilePad<P>::NS); kc >= 1; --kc)
    for (int kb = 256; kb >= 64; kb -= 32)
      if (bytes(kc, kb) <= budget) {
        *kc_out = kc;
        *kb_out = kb;
        return true;
      }
  return false;
}

template <int P, typename Kern>
cudaError_t persistent_blocks(Kern kern, size_t smem, int64_t items, int* blocks,
                              int threads = kGatherThreads / kStencilCtas) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  *blocks = int(std::min<int64_t>(items, int64_t(sm_count()) * std::max(per_sm, 1)));
  return cudaSuccess;
}

// Threads of the FP32 four-channel stencil kernels (one CTA per SM).
[[maybe_unused]] constexpr int kSpread4Threads = 1024;
[[maybe_unused]] constexpr int kGather4Threads = 512;
[[maybe_unused]] constexpr int kSpread4BwThreads = 1024;

// FP32 kernels for P <= 8: four channels per work item, windows evaluated in
// the lanes (stencil4.cuh).
template <int P>
cudaError_t spread4_P(const LaunchCtx& c, int* nlaunch) {
  const WinCoef<float> wc = win_coef<float>(c);
  const size_t smem = spread4_smem_bytes<P>();
  const int nchunk = (c.geo.K + 3) / 4;
  int blocks = 0;
  cudaError_t e = persistent_blocks<P>(k_spread4<P, kSpread4Threads>, smem, int64_t(c.ntiles) * nchunk, &blocks,
                                       kSpread4Threads);
  if (e != cudaSuccess) return e;
  k_spread4<P, kSpread4Threads><<<blocks, kSpread4Threads, smem, c.stream>>>(
      c.geo, c.nmax, c.tile_start, static_cast<const float*>(c.st), c.scell, static_cast<const float*>(c.sq),
      c.tscale, wc, static_cast<float*>(c.grid));
  ++*nlaunch;
  return cudaGetLastError();
}

template <int P>
cudaError_t interp4_P(const LaunchCtx& c, void* phi, void* forces, int* nlaunch) {
  const WinCoef<float> wc = win_coef<float>(c);
  const int nchunk = (c.geo.K + 3) / 4;
  cudaError_t e;
  if (nchunk > 1 && forces) {
    e = cudaMemsetAsync(forces, 0, size_t(c.n) * 3 * sizeof(float), c.stream);
    if (e != cudaSuccess) return e;
  }
  const size_t smem = gather4_smem_bytes<P>();
  int blocks = 0;
  e = persistent_blocks<P>(k_gather4<P, kGather4Threads>, smem, int64_t(c.ntiles) * nchunk, &blocks, kGather4Threads);
  if (e != cudaSuccess) return e;
  // one channel chunk and an idle buffer of 32 bytes per atom: outputs as
  // records in sorted order, then one coalesced pass to the caller's order
  float* rec = (nchunk == 1 && c.out_scratch && c.out_scratch_bytes >= c.nmax * 32 && c.tile_of && c.rank)
                   ? static_cast<float*>(c.out_scratch)
                   : nullptr;
  k_gather4<P, kGather4Threads><<<blocks, kGather4Threads, smem, c.stream>>>(
      c.nmax, c.geo, c.smol, c.soff, c.tile_start, static_cast<const float*>(c.st), c.scell,
      static_cast<const float*>(c.sq), c.sperm, wc, static_cast<const float*>(c.grid), c.zero_coef, c.charges,
      static_cast<float*>(phi), static_cast<float*>(forces), c.psi_il, rec);
  ++*nlaunch;
  if (rec) {
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int ub = int(std::min<int64_t>((c.nmax + 255) / 256, 148 * 16));
    k_unpack_gather<<<std::max(ub, 1), 256, 0, c.stream>>>(c.geo, c.nmax, c.soff, c.tile_of, c.rank, c.tile_start,
                                                           reinterpret_cast<const float4*>(rec),
                                                           static_cast<float*>(phi), static_cast<float*>(forces));
    ++*nlaunch;
  }
  return cudaGetLastError();
}

template <int P>
cudaError_t spread_P(const LaunchCtx& c, int* nlaunch) {
  if constexpr (sizeof(R) == 4 && P <= 8) return spread4_P<P>(c, nlaunch);
  const WinCoef<R> wc = win_coef(c);
  int kc = 0, kb = 0;
  if (!pick_kc_kb<P>(k_spread<R, P, kStencilCtas>, c.geo.K, [](int k, int b) { return spread_smem_bytes<R, P>(k, b); }, &kc, &kb)) {
    const int blocks = int(std::min<int64_t>((c.nmax + kDirectThreads - 1) / kDirectThreads, 148 * 32));
    k_spread_direct<R, P><<<std::max(blocks, 1), kDirectThreads, 0, c.stream>>>(
        c.nmax, c.geo, c.soff, c.tile_start, static_cast<const R*>(c.st), c.scell, static_cast<const R*>(c.sq), wc,
        static_cast<R*>(c.grid));
    ++*nlaunch;
    return cudaGetLastError();
  }
  const size_t smem = spread_smem_bytes<R, P>(kc, kb);
  const int nchunk = (c.geo.K + kc - 1) / kc;
  int blocks = 0;
  cudaError_t e = persistent_blocks<P>(k_spread<R, P, kStencilCtas>, smem, int64_t(c.ntiles) * nchunk, &blocks);
  if (e != cudaSuccess) return e;
  k_spread<R, P, kStencilCtas><<<blocks, kGatherThreads / kStencilCtas, smem, c.stream>>>(c.geo, c.smol, c.nmax, c.tile_start, static_cast<const R*>(c.st),
                                                             c.scell, static_cast<const R*>(c.sq), wc, kc, kb,
                                                             static_cast<R*>(c.grid));
  ++*nlaunch;
  return cudaGetLastError();
}

template <int P>
cudaError_t interp_P(const LaunchCtx& c, void* phi, void* forces, int* nlaunch) {
  if (c.n == 0) return cudaSuccess;
  if constexpr (sizeof(R) == 4 && P <= 8) return interp4_P<P>(c, phi, forces, nlaunch);
  const WinCoef<R> wc = win_coef(c);
  int kc = 0, kb = 0;
  if (!pick_kc_kb<P>(k_interp<R, P, kStencilCtas>, c.geo.K,
                     [](int k, int b) { return gather_smem_bytes<R, P>(k, b); }, &kc, &kb)) {
    const int blocks = int(std::min<int64_t>((c.nmax + kDirectThreads - 1) / kDirectThreads, 148 * 32));
    k_interp_direct<R, P><<<std::max(blocks, 1), kDirectThreads, 0, c.stream>>>(
        c.nmax, c.geo, c.smol, c.soff, c.tile_start, static_cast<const R*>(c.st), c.scell,
        static_cast<const R*>(c.sq), c.sperm, wc, static_cast<const R*>(c.grid), c.zero_coef, c.charges,
        static_cast<R*>(phi), static_cast<R*>(forces));
    ++*nlaunch;
    return cudaGetLastError();
  }
  const int nchunk = (c.geo.K + kc - 1) / kc;
  cudaError_t e;
  if (nchunk > 1 && forces) {
    e = cudaMemsetAsync(forces, 0, size_t(c.n) * 3 * sizeof(R), c.stream);
    if (e != cudaSuccess) return e;
  }
  const size_t smem = gather_smem_bytes<R, P>(kc, kb);
  int blocks = 0;
  e = persistent_blocks<P>(k_interp<R, P, kStencilCtas>, smem, int64_t(c.ntiles) * nchunk, &blocks);
  if (e != cudaSuccess) return e;
  const int threads = kGatherThreads / kStencilCtas;
  k_interp<R, P, kStencilCtas><<<blocks, threads, smem, c.stream>>>(
      c.nmax, c.geo, c.smol, c.soff, c.tile_start, static_cast<const R*>(c.st), c.scell,
      static_cast<const R*>(c.sq), c.sperm, wc, kc, kb, static_cast<const R*>(c.grid), c.zero_coef, c.charges,
      static_cast<R*>(phi), static_cast<R*>(forces));
  ++*nlaunch;
  return cudaGetLastError();
}

// FP32, P <= 8: the backward spread as k_spread4_bw (four channels per item,
// fixed point in shared memory) after its per-(tile, channel) units.
template <int P>
cudaError_t spread4_bw_P(const LaunchCtx& c, const BackwardArgs& b, int* nlaunch) {
  const WinCoef<float> wc = win_coef<float>(c);
  const int ntl = c.ntiles;
  const int tb = int(std::min<int64_t>((int64_t(ntl) * 32 + 255) / 256, 148 * 8));
  k_tile_scale_bw<P><<<std::max(tb, 1), 256, 0, c.stream>>>(
      ntl, c.geo.nts, c.geo.K, c.nmax, c.soff, c.tile_start, static_cast<const float*>(c.st),
      static_cast<const float*>(c.sq), c.sperm, c.smol, wc, static_cast<const float*>(b.g_phi),
      static_cast<const float*>(b.g_forces), c.tscale_bw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = spread4_smem_bytes<P>();
  const int nchunk = (c.geo.K + 3) / 4;
  int blocks = 0;
  e = persistent_blocks<P>(k_spread4_bw<P, kSpread4BwThreads>, smem, int64_t(ntl) * nchunk, &blocks,
                           kSpread4BwThreads);
  if (e != cudaSuccess) return e;
  k_spread4_bw<P, kSpread4BwThreads><<<blocks, kSpread4BwThreads, smem, c.stream>>>(
      c.geo, c.nmax, c.smol, c.soff, c.tile_start, static_cast<const float*>(c.st), c.scell,
      static_cast<const float*>(c.sq), c.sperm, c.tscale_bw, wc, static_cast<const float*>(b.g_phi),
      static_cast<const float*>(b.g_forces), static_cast<float*>(c.grid2));
  *nlaunch += 2;
  return cudaGetLastError();
}

template <int P>
cudaError_t backward_P(const LaunchCtx& c, const BackwardArgs& b, int stage, int* nlaunch) {
  if (c.n == 0) return cudaSuccess;
  if constexpr (sizeof(R) == 4 && P <= 8)
    if (stage == 0 && c.tscale_bw) return spread4_bw_P<P>(c, b, nlaunch);
  const WinCoef<R> wc = win_coef(c);
  const int64_t work = std::max<int64_t>(1, c.nmax * c.geo.K);
  const int blocks = int(std::min<int64_t>((work + kDirectThreads - 1) / kDirectThreads, 148 * 64));
  ++*nlaunch;
  if (stage == 0) {
    k_spread_bw<R, P><<<blocks, kDirectThreads, 0, c.stream>>>(
        c.nmax, c.geo, c.smol, c.soff, c.tile_start, static_cast<const R*>(c.st), c.scell,
        static_cast<const R*>(c.sq), c.sperm, wc, static_cast<const R*>(b.g_phi), static_cast<const R*>(b.g_forces),
        static_cast<R*>(c.grid2));
  } else {
    if (b.grad_pos) {
      const cudaError_t e = cudaMemsetAsync(b.grad_pos, 0, size_t(c.n_set) * 3 * sizeof(R), c.stream);
      if (e != cudaSuccess) return e;
    }
    k_interp_bw<R, P><<<blocks, kDirectThreads, 0, c.stream>>>(
        c.nmax, c.geo, c.smol, c.soff, c.tile_start, static_cast<const R*>(c.st), c.scell,
        static_cast<const R*>(c.sq), c.sperm, wc,
        static_cast<const R*>(c.grid), static_cast<const R*>(c.grid2), c.zero_coef, c.charges, c.gsum, b.g_energy,
        static_cast<const R*>(b.g_phi), static_cast<const R*>(b.g_forces), static_cast<R*>(b.grad_q),
        static_cast<R*>(b.grad_pos));
  }
  return cudaGetLastError();
}

}  // namespace

#define PSWF_P_CASES(F, ...)                                                                           \
  switch (c.geo.P) {                                                                                      \
    case 2: return F<2>(__VA_ARGS__);   case 3: return F<3>(__VA_ARGS__);   case 4: return F<4>(__VA_ARGS__); \
    case 5: return F<5>(__VA_ARGS__);   case 6: return F<6>(__VA_ARGS__);   case 7: return F<7>(__VA_ARGS__); \
    case 8: return F<8>(__VA_ARGS__);   case 9: return F<9>(__VA_ARGS__);   case 10: return F<10>(__VA_ARGS__); \
    case 11: return F<11>(__VA_ARGS__); case 12: return F<12>(__VA_ARGS__); case 13: return F<13>(__VA_ARGS__); \
    case 14: return F<14>(__VA_ARGS__); case 15: return F<15>(__VA_ARGS__); case 16: return F<16>(__VA_ARGS__); \
  }                                                                                                       \
  return cudaErrorInvalidValue;

int PSWF_CAT(bounds_word, PSWF_REAL)() { return take_bounds_word(); }

cudaError_t PSWF_CAT(launch_spread, PSWF_REAL)(const LaunchCtx& c, int* nlaunch) {
  PSWF_P_CASES(spread_P, c, nlaunch)
}

cudaError_t PSWF_CAT(launch_interp, PSWF_REAL)(const LaunchCtx& c, void* phi, void* forces, int* nlaunch) {
  PSWF_P_CASES(interp_P, c, phi, forces, nlaunch)
}

cudaError_t PSWF_CAT(launch_backward, PSWF_REAL)(const LaunchCtx& c, const BackwardArgs& b, int stage,
                                                 int* nlaunch) {
  PSWF_P_CASES(backward_P, c, b, stage, nlaunch)
}

}  // namespace pswf
