// C-ABI of the PSWF-LR hot path: plan, workspace, launches, cuFFT.
// The public contract is in include/pswf_lr.h.
#include <cuda_runtime.h>

#include <chrono>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <functional>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "fft_x.hpp"
#include "realspace.hpp"
#include "internal.hpp"
#include "kernels.cuh"
#include "launch.cuh"
#include "planner.hpp"
#include "pswf_lr.h"

namespace pswf {

// ---- small non-templated kernels ---------------------------------------------------
__global__ void k_charge_final(int nblk, int K, const double* __restrict__ part, double* __restrict__ charges) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= K) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nblk; ++i) {
    a += part[(size_t(i) * K + c) * 2 + 0];
    b += part[(size_t(i) * K + c) * 2 + 1];
  }
  charges[c * 2 + 0] = a;
  charges[c * 2 + 1] = b;
}

__global__ void k_scan_block_sums(int n, const int* __restrict__ in, int* __restrict__ sums, int per_block) {
  __shared__ int sh[32];
  const int64_t base = int64_t(blockIdx.x) * per_block;
  int s = 0;
  for (int i = threadIdx.x; i < per_block; i += blockDim.x) {
    const int64_t j = base + i;
    if (j < n) s += in[j];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += sh[w];
    sums[blockIdx.x] = t;
  }
}

// Single thread: exclusive scan of the (few) block sums in place.
__global__ void k_scan_sums(int nb, int* __restrict__ sums) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int acc = 0;
    for (int i = 0; i < nb; ++i) {
      const int v = sums[i];
      sums[i] = acc;
      acc += v;
    }
  }
}

// Each block scans its chunk: per-thread strips, block-wide inclusive scan of
// strip sums, then writes the exclusive prefix; out[n] = total.
__global__ void k_scan_apply(int n, const int* __restrict__ in, const int* __restrict__ sums, int per_block,
                             int* __restrict__ out) {
  __shared__ int sh[kScanBlock];
  const int64_t base = int64_t(blockIdx.x) * per_block;
  const int per_thread = (per_block + blockDim.x - 1) / blockDim.x;
  const int64_t my0 = base + int64_t(threadIdx.x) * per_thread;
  int local = 0;
  for (int i = 0; i < per_thread; ++i) {
    const int64_t j = my0 + i;
    if (j < n && j < base + per_block) local += in[j];
  }
  sh[threadIdx.x] = local;
  __syncthreads();
  for (int o = 1; o < int(blockDim.x); o <<= 1) {
    const int v = (int(threadIdx.x) >= o) ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  int acc = sums[blockIdx.x] + sh[threadIdx.x] - local;
  for (int i = 0; i < per_thread; ++i) {
    const int64_t j = my0 + i;
    if (j < n && j < base + per_block) {
      out[j] = acc;
      acc += in[j];
    }
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = acc;
}

// One block per structure s: energy[s][c] = sum of the partials of channel
// g = s K + c + zero_coef[g] Q_net^2; energy[s][K] = total.
__global__ void k_energy_final(int K, int nblk, const double* __restrict__ part, const double* __restrict__ zero_coef,
                               const double* __restrict__ charges, double* __restrict__ energy,
                               const double* __restrict__ vpart, double* __restrict__ virial) {
  // one block per structure, one warp per channel (channels strided over the warps)
  __shared__ double tw[32];
  const int s = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = int(blockDim.x >> 5);
  double tot = 0.0;   // this warp's channels (lane 0)
  for (int c = warp; c < K; c += nw) {
    const int g = s * K + c;
    double t = 0.0, v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = lane; i < nblk; i += 32) {
      t += part[size_t(g) * nblk + i];
      if (vpart)
        for (int d = 0; d < 6; ++d) v[d] += vpart[(size_t(g) * nblk + i) * 6 + d];
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (vpart)
      for (int d = 0; d < 6; ++d)
        for (int o = 16; o > 0; o >>= 1) v[d] += __shfl_down_sync(0xffffffffu, v[d], o);
    if (lane == 0) {
      const double Q = charges[2 * g];
      const double ec = t + zero_coef[g] * Q * Q;
      energy[size_t(s) * (K + 1) + c] = ec;
      tot += ec;
      // W_ab = -dE/d epsilon_ab: E delta_ab (the 1/V prefactor and E^0 ~ 1/V)
      // plus the log-derivative sums of the multiplier
      if (vpart && virial)
        for (int d = 0; d < 6; ++d) virial[size_t(g) * 6 + d] = (d < 3 ? ec : 0.0) + v[d];
    }
  }
  if (lane == 0) tw[warp] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += tw[w];
    energy[size_t(s) * (K + 1) + K] = t;
  }
}

// FP32 scatter in two passes.  Written in place, k_scatter's nine 4- and
// 8-byte stores per atom land on nine partly filled 32-byte sectors at
// random places, and the L2 write traffic is about eleven times the useful
// bytes.  Here each atom's sorted slot instead receives two aligned records
// (rec [n_max][2] float4: t, original index; packed start cell; and per
// chunk of four channels qrec [nchunk][n_max] float4), placed in a scratch
// area (the spectrum buffer, else the grid: both idle during set_points;
// record_buffer), and k_unpack_rec then writes the
// sorted arrays in slot order with coalesced stores.
__global__ void k_scatter_rec(int64_t nmax, const float* __restrict__ q, Geometry g, const int* __restrict__ soff,
                              const int* __restrict__ tile_of, const int* __restrict__ rank,
                              const int* __restrict__ tile_start, const float* __restrict__ tmp_t,
                              const uint64_t* __restrict__ tmp_cell, float4* __restrict__ rec,
                              float4* __restrict__ qrec) {
  const int64_t n = soff[g.B];
  const int nchunk = (g.K + 3) / 4;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t dst = int64_t(tile_start[tile_of[i]]) + rank[i];
    if (!in_bounds(dst, nmax, kBoundsScatter)) continue;
    const uint64_t cell = tmp_cell[i];
    rec[2 * dst] = make_float4(tmp_t[i], tmp_t[nmax + i], tmp_t[2 * nmax + i], __int_as_float(int(i)));
    rec[2 * dst + 1] = make_float4(__int_as_float(int(uint32_t(cell))), __int_as_float(int(uint32_t(cell >> 32))),
                                   0.0f, 0.0f);
    for (int c4 = 0; c4 < nchunk; ++c4) {
      const int c = 4 * c4;
      qrec[int64_t(c4) * nmax + dst] =
          make_float4(q[int64_t(c) * n + i], c + 1 < g.K ? q[int64_t(c + 1) * n + i] : 0.0f,
                      c + 2 < g.K ? q[int64_t(c + 2) * n + i] : 0.0f, c + 3 < g.K ? q[int64_t(c + 3) * n + i] : 0.0f);
    }
  }
}

__global__ void k_unpack_rec(int64_t nmax, int K, int B, const int* __restrict__ soff, const float4* __restrict__ rec,
                             const float4* __restrict__ qrec, float* __restrict__ st, uint64_t* __restrict__ scell,
                             float* __restrict__ sq, int* __restrict__ sperm) {
  const int64_t n = soff[B];
  const int nchunk = (K + 3) / 4;
  for (int64_t m = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; m < n; m += int64_t(gridDim.x) * blockDim.x) {
    const float4 a = rec[2 * m], b = rec[2 * m + 1];
    st[m] = a.x;
    st[nmax + m] = a.y;
    st[2 * nmax + m] = a.z;
    sperm[m] = __float_as_int(a.w);
    scell[m] = uint64_t(uint32_t(__float_as_int(b.x))) | (uint64_t(uint32_t(__float_as_int(b.y))) << 32);
    for (int c4 = 0; c4 < nchunk; ++c4) {
      const float4 v = qrec[int64_t(c4) * nmax + m];
      const int c = 4 * c4;
      sq[int64_t(c) * nmax + m] = v.x;
      if (c + 1 < K) sq[int64_t(c + 1) * nmax + m] = v.y;
      if (c + 2 < K) sq[int64_t(c + 2) * nmax + m] = v.z;
      if (c + 3 < K) sq[int64_t(c + 3) * nmax + m] = v.w;
    }
  }
}

__global__ void k_set_count(int* __restrict__ soff, int n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    soff[0] = 0;
    soff[1] = n;
  }
}

__global__ void k_tile_scale(int ntl, int K, int64_t nmax, const int* __restrict__ tile_start,
                             const float* __restrict__ sq, float* __restrict__ tscale) {
  const int lane = threadIdx.x & 31;
  const int nw = int((int64_t(gridDim.x) * blockDim.x) >> 5);
  for (int t = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); t < ntl; t += nw) {
    const int a0 = tile_start[t], a1 = tile_start[t + 1];
    for (int c = 0; c < K; ++c) {
      float s1 = 0.0f, mq = 0.0f;
      for (int a = a0 + lane; a < a1; a += 32) {
        const float v = fabsf(sq[int64_t(c) * nmax + a]);
        s1 += v;
        mq = fmaxf(mq, v);
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

__global__ void k_charge_final_seg(int nblk, int K, int B, const double* __restrict__ part,
                                   double* __restrict__ charges) {
  // one block per (structure, channel): threads stride over the block
  // partials (several loads in flight each), then warp and block sums
  const int g = blockIdx.x;
  if (g >= B * K) return;
  const int s = g / K, c = g - s * K;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    const size_t o = ((size_t(s) * nblk + i) * K + c) * 2;
    a += part[o];
    b += part[o + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  __shared__ double sh[2][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = a;
    sh[1][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      x += sh[0][w];
      y += sh[1][w];
    }
    charges[2 * g] = x;
    charges[2 * g + 1] = y;
  }
}

}  // namespace pswf

using namespace pswf;

namespace {

constexpr int kThreads = 256;
constexpr int kEnergyBlocks = 592;   // 4 x 148 SMs
constexpr int kQBlocks = 148;        // charge-sum blocks of pswf_self_energy_noalloc
constexpr int kQBlocksPlan = 1184;   // charge-sum blocks of a single-structure plan (8 per SM)
constexpr int kQBlocksBatch = 8;     // per structure in a batch plan

int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

// Host worker threads for the copies and conversions of the end-to-end path:
// created once, woken per parallel_for (up to 15 workers plus the caller).
class HostPool {
 public:
  static HostPool& get() {
    static HostPool pool;
    return pool;
  }
  int size() const { return int(workers_.size()) + 1; }
  // Runs f(t) for t in [0, nt) on nt threads (the caller runs t = 0).
  void run(int nt, const std::function<void(int)>& f) {
    std::lock_guard<std::mutex> one_job(run_mu_);   // callers from several threads take turns
    nt = std::min(nt, size());
    if (nt <= 1) {
      f(0);
      return;
    }
    {
      std::unique_lock<std::mutex> lk(mu_);
      job_ = &f;
      njobs_ = nt;
      next_ = 1;
      pending_ = nt - 1;
      ++gen_;
    }
    cv_.notify_all();
    f(0);
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [&] { return pending_ == 0; });
    job_ = nullptr;
  }

 private:
  HostPool() {
    const int hw = int(std::max<unsigned>(1, std::thread::hardware_concurrency()));
    const int nw = std::min(15, hw - 1);
    for (int i = 0; i < nw; ++i) workers_.emplace_back([this] { loop(); });
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : workers_) t.join();
  }
  void loop() {
    int64_t seen = 0;
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
      cv_.wait(lk, [&] { return stop_ || (gen_ != seen && next_ < njobs_); });
      if (stop_) return;
      const int t = next_++;
      if (next_ >= njobs_) seen = gen_;
      const std::function<void(int)>* f = job_;
      lk.unlock();
      (*f)(t);
      lk.lock();
      if (--pending_ == 0) done_.notify_all();
    }
  }
  std::vector<std::thread> workers_;
  std::mutex run_mu_, mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int)>* job_ = nullptr;
  int njobs_ = 0, next_ = 0, pending_ = 0;
  int64_t gen_ = 0;
  bool stop_ = false;
};

// Splits [0, n) into contiguous shares over the host pool; small ranges run
// inline.
template <typename F>
void parallel_for(int64_t n, F f) {
  HostPool& pool = HostPool::get();
  const int nt = int(std::min<int64_t>(pool.size(), std::max<int64_t>(1, n / 16384)));
  if (nt <= 1) {
    f(0, n);
    return;
  }
  const int64_t per = (n + nt - 1) / nt;
  pool.run(nt, [&](int t) {
    const int64_t lo = t * per, hi = std::min(n, lo + per);
    if (lo < hi) f(lo, hi);
  });
}

}  // namespace

struct pswf_plan_s {
  Plan host;
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t n_max = 0;
  int64_t n = -1;            // atoms of the last set_points (-1: none)
  bool psi_valid = false;    // grid holds Psi of the last execute (backward plans)
  int64_t rs_n = -1;         // atoms of the last pswf_real_space (its cell list is kept)
  int flags = 0;
  bool batch = false;        // created by pswf_batch_plan_create
  int B = 1;                 // structures (slots)
  int nrun = 1;              // slots processed per launch (a planned size >= the set count)
  int nts = 0;               // tiles per structure
  int nqb = kQBlocks;        // charge-sum blocks per structure
  int eblk = kEnergyBlocks;  // multiplier blocks per (structure, channel)
  int Mh = 0;                // max_d (M_d / 2 + 1): row stride of the iw2 tables
  size_t real_size = 4;
  Geometry geo{};
  int ntiles = 0;
  int scan_blocks = 0;
  int scan_per_block = 0;
  int64_t grid_elems = 0;    // K * Mz * My * Mxp
  // workspace
  void* ws = nullptr;
  int64_t ws_bytes = 0;
  bool ws_owned = false;
  // device pointers inside the workspace
  void* grid = nullptr;      // real [K][Mz][My][Mxp]
  void* grid2 = nullptr;     // second grid (backward)
  void* tmp_t = nullptr;     // real [3][n_max] window offsets, caller order
  uint64_t* tmp_cell = nullptr;  // [n_max] packed start cells, caller order
  void* st = nullptr;        // real [3][n_max]
  uint64_t* scell = nullptr; // [n_max]
  void* sq = nullptr;        // real [K][n_max]
  int* sperm = nullptr;      // [n_max]
  int* tile_of = nullptr;    // [n_max]
  int* rank = nullptr;       // [n_max]
  int* tile_count = nullptr; // [ntiles]
  int* tile_start = nullptr; // [ntiles + 1]
  float* tscale = nullptr;   // [ntiles][K] fixed-point unit of the FP32 four-channel spread (P <= 8)
  float* tscale_bw = nullptr;   // the same for the backward's spread (PSWF_FLAG_BACKWARD)
  int* scan_sums = nullptr;  // [scan_blocks]
  double* qpart = nullptr;   // [B][nqb][K][2]
  double* charges = nullptr; // [B K][2]: Q_net, Q_self
  double* bsum = nullptr;    // [B K][2]: sum and sum of squares of the upstream gphi (backward)
  double* epart = nullptr;   // [B K][eblk]
  double* vpart = nullptr;   // [B K][eblk][3] (PSWF_FLAG_VIRIAL)
  double* virial = nullptr;  // [B][K][3] (PSWF_FLAG_VIRIAL)
  bool virial_valid = false;
  double* energy_tmp = nullptr; // [B][K + 1]
  int* err = nullptr;        // device status flag
  void* coef_m = nullptr;    // real [6][kMultSeg][deg_m + 1], row p - 1
  // per-structure tables, one contiguous region (uploaded in one copy):
  void* stab = nullptr;
  int64_t stab_bytes = 0;
  int64_t stab_off[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double* sbox = nullptr;    // [B][3] box edges
  double* scale = nullptr;   // [B K] multiplier scale (includes dV^2 / V)
  double* zero_coef = nullptr;  // [B K]
  int* soff = nullptr;       // [B + 1] atom offsets per structure
  int* pch = nullptr;        // [B K] exponents
  void* iw2 = nullptr;       // real [B][3][Mh]
  double* smol = nullptr;    // [B][3] M_d / L_d (stencil location and 2/h without a division; 1 for a general cell)
  double* bmat = nullptr;    // [B][9] B = 2 pi H^-1 (k_m = B m; diag(2 pi / L) for a box)
  double* tmat = nullptr;    // [B][9] T = diag(M) H^-T (grid coordinates u = T r; general cells)
  bool tric = false;         // single structure in a general (non-orthorhombic) cell
  void* h_stab = nullptr;    // pinned host mirror of stab (batch plans)
  cudaEvent_t stab_ev = nullptr;  // last upload from h_stab
  std::vector<int> h_pch;    // host copy of pch
  void* fft_work = nullptr;
  // cuFFT: one plan pair per planned launch size (single plans: 1; batch
  // plans: 1, 2, 4, ... and b_max), all on one work area
  std::vector<int> fft_sizes;
  std::vector<cufftHandle> fwd, inv;
  bool fft_made = false;
  // Pruned transform of single-structure plans: only the nkx lowest x
  // frequencies can be inside the band |k| < k_c, so the 3-D transform is a
  // 1-D real transform along x over all rows plus 2-D (z, y) transforms of
  // those nkx columns only (per channel).
  bool pruned = false;
  int nkx = 0;
  cufftHandle pr_r2c = 0, pr_c2r = 0, pr_2d = 0;
  void* spec = nullptr;      // complex [K][Mxh][Mz][My] (pruned plans)
  // FP32 pruned plans with Mx = 32 N1: the x passes are the kernels of
  // fft_x.cu (only the kx < nkx planes written and read) instead of cuFFT
  bool xfft = false;
  // ... and when My and Mz are of that form too, the (z, y) passes as well:
  // z pass, then the multiplier fused with the y transforms (no cuFFT)
  bool yzfft = false;
  // Psi written by the own inverse x pass as channel quadruples (K a multiple
  // of 4, FP32 four-channel gather, no backward: the backward kernels read
  // Psi channel-planar)
  bool psi_il = false;
  void* xtw = nullptr;       // twiddle tables (float2) of Mx, then My and Mz (yzfft)
  int64_t tw_off[3] = {0, 0, 0};
  // real-space complement (PSWF_FLAG_REAL_SPACE): its cell list and scratch
  RealSpaceGeom rs_geo;
  int rs_ncell = 0, rs_nsb = 0;
  int *rs_count = nullptr, *rs_start = nullptr, *rs_cellof = nullptr, *rs_rank = nullptr, *rs_perm = nullptr,
      *rs_scan = nullptr;
  void *rs_lpos = nullptr, *coef_g = nullptr;
  unsigned char* lmask = nullptr;   // yzfft: [nkx][Mz] lines that can hold band modes
  int* lines = nullptr;             // yzfft: those lines, kx << 16 | pz
  int nlines = 0;
  size_t fft_work_bytes = 0;
  // host staging for pswf_compute_host
  double* h_pin = nullptr;
  // pswf_compute_host: the charges' copy on a second stream after the
  // positions' (ev_pos), so that the bin and the scan run meanwhile; while
  // set via q_ready, set_points waits for it before reading the charges
  cudaStream_t q_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_pos = nullptr, ev_q = nullptr, q_ready = nullptr;
  // the grid is being cleared for the next spread on the side stream (by
  // pswf_compute_host, under the positions' copy), done at ev_clear.
  // Clearing it there during set_points instead gained nothing: the sort's
  // kernels slowed by what the spread saved (HBM shared by both)
  bool grid_zeroed = false;
  cudaEvent_t ev_clear = nullptr;
  int64_t h_pin_elems = 0;
  void* d_stage = nullptr;
  int64_t d_stage_bytes = 0;
  std::string last_error;
  // measurement: stage event pairs (when enabled) and own-kernel launch counts
  struct StageRec {
    int stage;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<StageRec> recs;
  std::vector<cudaEvent_t> pool;
  int64_t launches[PSWF_NSTAGE] = {};
  int cur_stage = PSWF_STAGE_OTHER;   // innermost open StageScope
};

namespace {

int set_err(pswf_plan p, int code, const std::string& msg) {
  if (p) p->last_error = msg;
  return code;
}

int cuda_check(pswf_plan p, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PSWF_OK;
  return set_err(p, e == cudaErrorMemoryAllocation ? PSWF_ENOMEM : PSWF_ECUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

int launch_check(pswf_plan p, const char* what) { return cuda_check(p, cudaGetLastError(), what); }

cudaEvent_t take_event(pswf_plan p) {
  cudaEvent_t e = nullptr;
  if (!p->pool.empty()) {
    e = p->pool.back();
    p->pool.pop_back();
  } else {
    cudaEventCreate(&e);
  }
  return e;
}

// Records an event pair around one stage on the plan's stream when
// measurement is enabled.
struct StageScope {
  pswf_plan p;
  int stage, outer;
  cudaEvent_t a = nullptr;
  StageScope(pswf_plan p_, int stage_) : p(p_), stage(stage_), outer(p_->cur_stage) {
    p->cur_stage = stage;
    if (p->prof_on) {
      a = take_event(p);
      cudaEventRecord(a, p->stream);
    }
  }
  // the stage's time starts here instead (work before it overlaps another phase)
  void restart() {
    if (a) {
      p->pool.push_back(a);
      a = take_event(p);
      cudaEventRecord(a, p->stream);
    }
  }
  ~StageScope() {
    p->cur_stage = outer;
    if (a) {
      cudaEvent_t b = take_event(p);
      cudaEventRecord(b, p->stream);
      p->recs.push_back({stage, a, b});
    }
  }
};

// Grid elements of the slots processed per launch.
int64_t run_grid_elems(pswf_plan p) { return p->grid_elems / p->B * p->nrun; }

// Bytes of the spectrum buffer (pruned and own-transform plans; 0 without one).
int64_t spec_bytes(pswf_plan p) {
  return p->spec ? int64_t(p->host.K) * (p->host.M[0] / 2 + 1) * p->host.M[1] * p->host.M[2] * 2 *
                       int64_t(p->real_size)
                 : 0;
}

// The side stream and its events (created on first use).
int ensure_side_stream(pswf_plan p) {
  if (p->q_stream) return PSWF_OK;
  int rc;
  if ((rc = cuda_check(p, cudaStreamCreateWithFlags(&p->q_stream, cudaStreamNonBlocking), "side stream")) ||
      (rc = cuda_check(p, cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming), "side event")) ||
      (rc = cuda_check(p, cudaEventCreateWithFlags(&p->ev_pos, cudaEventDisableTiming), "side event")) ||
      (rc = cuda_check(p, cudaEventCreateWithFlags(&p->ev_q, cudaEventDisableTiming), "side event")) ||
      (rc = cuda_check(p, cudaEventCreateWithFlags(&p->ev_clear, cudaEventDisableTiming), "side event")))
    return rc;
  return PSWF_OK;
}

// Clears the grid for the next spread on the side stream, after all work
// enqueued so far on the plan's stream; execute waits for ev_clear.
int clear_grid_aside(pswf_plan p) {
  int rc;
  if ((rc = ensure_side_stream(p)) || (rc = cuda_check(p, cudaEventRecord(p->ev_in, p->stream), "side event")) ||
      (rc = cuda_check(p, cudaStreamWaitEvent(p->q_stream, p->ev_in, 0), "order the grid clearing")) ||
      (rc = cuda_check(p, cudaMemsetAsync(p->grid, 0, size_t(run_grid_elems(p)) * size_t(p->real_size), p->q_stream),
                       "clear grid")) ||
      (rc = cuda_check(p, cudaEventRecord(p->ev_clear, p->q_stream), "side event")))
    return rc;
  p->grid_zeroed = true;
  return PSWF_OK;
}

// Where the FP32 set_points parks its per-atom records before unpacking
// them: the spectrum buffer when it holds them, else the grid (both idle
// until execute), else nowhere (the direct scatter).
void* record_buffer(pswf_plan p) {
  if (p->real_size != 4) return nullptr;
  const int64_t bytes = p->n_max * (32 + 16 * int64_t((p->host.K + 3) / 4));
  if (p->spec && bytes <= spec_bytes(p)) return p->spec;
  if (bytes <= p->grid_elems * int64_t(p->real_size)) return p->grid;
  return nullptr;
}

// Smallest planned launch size holding b structures.
int run_size(pswf_plan p, int b) {
  for (int sz : p->fft_sizes)
    if (sz >= b) return sz;
  return p->B;
}

// Layout of the per-structure table region (also the pinned host mirror):
// sbox double [B][3] | scale double [B K] | zero_coef double [B K] |
// soff int [B + 1] | pch int [B K] | iw2 real [B][3][Mh] | M/L double [B][3] |
// B = 2 pi H^-1 double [B][9] | T = diag(M) H^-T double [B][9]; returns bytes.
int64_t stab_layout(pswf_plan p) {
  const int64_t B = p->B, K = p->host.K, rs = int64_t(p->real_size);
  auto a16 = [](int64_t b) { return (b + 15) & ~int64_t(15); };
  int64_t off = 0;
  p->stab_off[0] = off; off = a16(off + B * 3 * 8);
  p->stab_off[1] = off; off = a16(off + B * K * 8);
  p->stab_off[2] = off; off = a16(off + B * K * 8);
  p->stab_off[3] = off; off = a16(off + (B + 1) * 4);
  p->stab_off[4] = off; off = a16(off + B * K * 4);
  p->stab_off[5] = off; off = a16(off + B * 3 * int64_t(p->Mh) * rs);
  p->stab_off[6] = off; off = a16(off + B * 3 * 8);
  p->stab_off[7] = off; off = a16(off + B * 9 * 8);
  p->stab_off[8] = off; off = a16(off + B * 9 * 8);
  return off;
}

// Workspace layout (each region 256-byte aligned).  Returns total bytes and,
// when base != nullptr, assigns the pointers.
int64_t layout(pswf_plan p, char* base) {
  const Plan& h = p->host;
  const int64_t K = h.K, B = p->B, BK = B * K;
  const int64_t rs = int64_t(p->real_size);
  int64_t off = 0;
  auto take = [&](int64_t bytes) -> char* {
    char* ptr = base ? base + off : nullptr;
    off += align256(std::max<int64_t>(bytes, 1));
    return ptr;
  };
  p->grid = take(p->grid_elems * rs);
  p->grid2 = (p->flags & PSWF_FLAG_BACKWARD) ? take(p->grid_elems * rs) : nullptr;
  p->spec = p->pruned ? take(int64_t(h.K) * (h.M[0] / 2 + 1) * h.M[1] * h.M[2] * 2 * rs) : nullptr;
  const int64_t nm = std::max<int64_t>(p->n_max, 1);
  p->tmp_t = take(3 * nm * rs);
  p->tmp_cell = reinterpret_cast<uint64_t*>(take(nm * 8));
  p->st = take(3 * nm * rs);
  p->scell = reinterpret_cast<uint64_t*>(take(nm * 8));
  p->sq = take(K * nm * rs);
  p->sperm = reinterpret_cast<int*>(take(nm * 4));
  p->tile_of = reinterpret_cast<int*>(take(nm * 4));
  p->rank = reinterpret_cast<int*>(take(nm * 4));
  p->tile_count = reinterpret_cast<int*>(take(int64_t(p->ntiles) * 4));
  p->tile_start = reinterpret_cast<int*>(take(int64_t(p->ntiles + 1) * 4));
  p->tscale = (p->real_size == 4 && h.P <= 8) ? reinterpret_cast<float*>(take(int64_t(p->ntiles) * K * 4)) : nullptr;
  p->tscale_bw = (p->tscale && (p->flags & PSWF_FLAG_BACKWARD)) ? reinterpret_cast<float*>(take(int64_t(p->ntiles) * K * 4))
                                                              : nullptr;
  p->scan_sums = reinterpret_cast<int*>(take(int64_t(p->scan_blocks) * 4));
  p->qpart = reinterpret_cast<double*>(take(B * p->nqb * K * 2 * 8));
  p->charges = reinterpret_cast<double*>(take(BK * 2 * 8));
  p->bsum = reinterpret_cast<double*>(take(BK * 2 * 8));
  p->epart = reinterpret_cast<double*>(take(BK * p->eblk * 8));
  p->energy_tmp = reinterpret_cast<double*>(take(B * (K + 1) * 8));
  const bool vir = (p->flags & PSWF_FLAG_VIRIAL) != 0;
  p->vpart = vir ? reinterpret_cast<double*>(take(BK * p->eblk * 6 * 8)) : nullptr;
  p->virial = vir ? reinterpret_cast<double*>(take(BK * 6 * 8)) : nullptr;
  p->err = reinterpret_cast<int*>(take(4));
  p->coef_m = take(int64_t(6) * kMultSeg * (h.deg_m + 1) * rs);
  p->coef_g = take(int64_t(6) * kMultSeg * (h.deg_g + 1) * rs);
  if (p->flags & PSWF_FLAG_REAL_SPACE) {
    p->rs_count = reinterpret_cast<int*>(take(int64_t(p->rs_ncell) * 4));
    p->rs_start = reinterpret_cast<int*>(take(int64_t(p->rs_ncell + 1) * 4));
    p->rs_cellof = reinterpret_cast<int*>(take(nm * 4));
    p->rs_rank = reinterpret_cast<int*>(take(nm * 4));
    p->rs_perm = reinterpret_cast<int*>(take(nm * 4));
    p->rs_scan = reinterpret_cast<int*>(take(int64_t(p->rs_nsb) * 4));
    p->rs_lpos = take(int64_t(real_space_bytes_per_atom(K, int(rs))) * nm);   // coordinates, records, rows
  }
  {
    int64_t tw_pairs = 0;
    for (int d = 0; d < (p->yzfft ? 3 : p->xfft ? 1 : 0); ++d) {
      p->tw_off[d] = tw_pairs;
      tw_pairs += xfft_table_size(h.M[d]);
    }
    p->xtw = tw_pairs ? take(tw_pairs * 8) : nullptr;
    const int64_t nl = p->yzfft ? int64_t(p->nkx) * h.M[2] : 0;
    p->lmask = p->yzfft ? reinterpret_cast<unsigned char*>(take(nl)) : nullptr;
    p->lines = p->yzfft ? reinterpret_cast<int*>(take(nl * 4)) : nullptr;
  }
  p->stab_bytes = stab_layout(p);
  char* st = take(p->stab_bytes);
  p->stab = st;
  if (st) {
    p->sbox = reinterpret_cast<double*>(st + p->stab_off[0]);
    p->scale = reinterpret_cast<double*>(st + p->stab_off[1]);
    p->zero_coef = reinterpret_cast<double*>(st + p->stab_off[2]);
    p->soff = reinterpret_cast<int*>(st + p->stab_off[3]);
    p->pch = reinterpret_cast<int*>(st + p->stab_off[4]);
    p->iw2 = st + p->stab_off[5];
    p->smol = reinterpret_cast<double*>(st + p->stab_off[6]);
    p->bmat = reinterpret_cast<double*>(st + p->stab_off[7]);
    p->tmat = reinterpret_cast<double*>(st + p->stab_off[8]);
  }
  p->fft_work = take(int64_t(p->fft_work_bytes));
  return off;
}

template <typename R>
std::vector<R> to_real(const std::vector<double>& v) {
  return std::vector<R>(v.begin(), v.end());
}

template <typename T>
int upload(pswf_plan p, void* dst, const std::vector<T>& v, const char* what) {
  return cuda_check(p, cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), what);
}

// Fills a host image of the table region for structures 0..b-1 (boxes
// [b][3], exponents [b][K], atom offsets [b + 1]); slots b..B-1 are empty
// (no atoms, zero scale).  Exponents must be ones the plan was built for.
int fill_stab(pswf_plan p, int b, const double* boxes, const int* ps, const int64_t* offsets, char* dst) {
  const Plan& h = p->host;
  const int K = h.K, B = p->B;
  double* sbox = reinterpret_cast<double*>(dst + p->stab_off[0]);
  double* scale = reinterpret_cast<double*>(dst + p->stab_off[1]);
  double* zero = reinterpret_cast<double*>(dst + p->stab_off[2]);
  int* soff = reinterpret_cast<int*>(dst + p->stab_off[3]);
  int* pch = reinterpret_cast<int*>(dst + p->stab_off[4]);
  char* iw2 = dst + p->stab_off[5];
  double* smol = reinterpret_cast<double*>(dst + p->stab_off[6]);
  double* bmat = reinterpret_cast<double*>(dst + p->stab_off[7]);
  double* tmat = reinterpret_cast<double*>(dst + p->stab_off[8]);
  int pdef = 0;
  for (int q = 1; q <= 6 && !pdef; ++q)
    if (h.mult_scale_p[q] != 0.0) pdef = q;
  p->h_pch.assign(size_t(B) * K, pdef);
  StructTables t;
  std::string err;
  for (int sidx = 0; sidx < B; ++sidx) {
    const bool used = sidx < b;
    if (used && !p->batch) {
      t = h.st;   // the single structure's cell, tabulated by the planner
    } else if (used) {
      int rc = struct_tables(h, boxes + 3 * sidx, t, err);
      if (rc) return set_err(p, rc, "structure " + std::to_string(sidx) + ": " + err);
    } else {
      // empty slot: valid box, zero multiplier (no W-hat tables needed)
      for (int d = 0; d < 3; ++d) {
        t.box[d] = h.box_max[d];
        t.iw2[d].clear();
      }
      t.V = t.dV = 1.0;
      t.tric = false;
      for (int i = 0; i < 9; ++i) t.tmat[i] = t.bmat[i] = 0.0;
      for (int d = 0; d < 3; ++d) {
        t.tmat[4 * d] = double(h.M[d]) / t.box[d];
        t.bmat[4 * d] = 2.0 * 3.14159265358979323846 / t.box[d];
      }
    }
    for (int d = 0; d < 3; ++d) {
      sbox[3 * sidx + d] = t.box[d];
      // general cells: the gathers work in grid coordinates (unit M / L) and
      // the forces go through T^T afterwards
      smol[3 * sidx + d] = t.tric ? 1.0 : double(h.M[d]) / t.box[d];
    }
    for (int i = 0; i < 9; ++i) {
      bmat[9 * sidx + i] = t.bmat[i];
      tmat[9 * sidx + i] = t.tmat[i];
    }
    const double dv2v = t.dV * t.dV / t.V;
    for (int c = 0; c < K; ++c) {
      const int g = sidx * K + c;
      const int pp = used ? ps[size_t(sidx) * K + c] : pdef;
      if (pp < 1 || pp > 6 || h.mult_scale_p[pp] == 0.0)
        return set_err(p, PSWF_EINVAL, "exponent p of structure " + std::to_string(sidx) + " was not planned for");
      pch[g] = pp;
      p->h_pch[g] = pp;
      scale[g] = used ? h.mult_scale_p[pp] * dv2v : 0.0;
      zero[g] = used ? h.zero_num_p[pp] / t.V : 0.0;
    }
    for (int d = 0; d < 3; ++d)
      for (int m = 0; m < p->Mh; ++m) {
        const double v = m < int(t.iw2[d].size()) ? t.iw2[d][m] : 0.0;
        const size_t o = (size_t(sidx) * 3 + d) * p->Mh + m;
        if (p->real_size == 4)
          reinterpret_cast<float*>(iw2)[o] = float(v);
        else
          reinterpret_cast<double*>(iw2)[o] = v;
      }
  }
  for (int sidx = 0; sidx <= B; ++sidx) soff[sidx] = int(offsets ? offsets[std::min(sidx, b)] : 0);
  return PSWF_OK;
}

int upload_tables(pswf_plan p) {
  const Plan& h = p->host;
  int rc;
  if (p->real_size == 4) {
    if ((rc = upload(p, p->coef_m, to_real<float>(h.coef_m), "upload coef"))) return rc;
    if ((rc = upload(p, p->coef_g, to_real<float>(h.coef_g), "upload real-space coef"))) return rc;
    if (p->xfft) {
      std::vector<float> all, tw;
      for (int d = 0; d < (p->yzfft ? 3 : 1); ++d) {
        xfft_twiddles(h.M[d], tw);
        all.insert(all.end(), tw.begin(), tw.end());
      }
      if ((rc = upload(p, p->xtw, all, "upload transform twiddles"))) return rc;
    }
    if (p->yzfft) {
      std::vector<unsigned char> mask;
      std::vector<int> lines;
      const double two_pi = 2.0 * 3.14159265358979323846;
      (void)two_pi;
      xfft_band_lines(p->nkx, h.M[1], h.M[2], h.st.bmat, h.k_c, mask, lines);
      p->nlines = int(lines.size());
      if ((rc = upload(p, p->lmask, mask, "upload band mask"))) return rc;
      if (!lines.empty() && (rc = upload(p, p->lines, lines, "upload band lines"))) return rc;
    }
  } else {
    if ((rc = upload(p, p->coef_m, h.coef_m, "upload coef"))) return rc;
    if ((rc = upload(p, p->coef_g, h.coef_g, "upload real-space coef"))) return rc;
  }
  std::vector<char> img(size_t(p->stab_bytes), 0);
  if (!p->batch) {
    const int64_t offs[2] = {0, 0};
    if ((rc = fill_stab(p, 1, h.box, h.p.data(), offs, img.data()))) return rc;
  } else {
    if ((rc = fill_stab(p, 0, nullptr, nullptr, nullptr, img.data()))) return rc;
  }
  if ((rc = upload(p, p->stab, img, "upload structure tables"))) return rc;
  return cuda_check(p, cudaMemset(p->err, 0, 4), "clear err");
}

int attach_fft_work(pswf_plan p) {
  if (!p->fft_made) return PSWF_OK;
  for (cufftHandle hd : {p->pr_r2c, p->pr_c2r, p->pr_2d})
    if (hd && cufftSetWorkArea(hd, p->fft_work) != CUFFT_SUCCESS) return set_err(p, PSWF_ECUFFT, "cufftSetWorkArea failed");
  for (size_t i = 0; i < p->fwd.size(); ++i)
    if (cufftSetWorkArea(p->fwd[i], p->fft_work) != CUFFT_SUCCESS ||
        cufftSetWorkArea(p->inv[i], p->fft_work) != CUFFT_SUCCESS)
      return set_err(p, PSWF_ECUFFT, "cufftSetWorkArea failed");
  return PSWF_OK;
}

int ensure_workspace(pswf_plan p) {
  if (p->ws) return PSWF_OK;
  void* mem = nullptr;
  int rc = cuda_check(p, cudaMalloc(&mem, size_t(p->ws_bytes)), "workspace cudaMalloc");
  if (rc) return rc;
  p->ws = mem;
  p->ws_owned = true;
  layout(p, static_cast<char*>(mem));
  if ((rc = attach_fft_work(p))) return rc;
  return upload_tables(p);
}

LaunchCtx make_ctx(pswf_plan p) {
  LaunchCtx c;
  c.geo = p->geo;
  c.geo.B = p->nrun;
  c.nmax = p->n_max;
  // batch plans: outputs hold n_max rows and every launch is made whatever
  // the count (so that a captured sequence serves any batch)
  c.n = p->batch ? p->n_max : p->n;
  c.n_set = p->n;
  c.ntiles = p->nrun * p->nts;
  c.smol = p->smol;
  c.soff = p->soff;
  c.tile_start = p->tile_start;
  c.tscale = p->tscale;
  c.tscale_bw = p->tscale_bw;
  c.psi_il = p->psi_il;
  c.st = p->st;
  c.scell = p->scell;
  c.sq = p->sq;
  c.sperm = p->sperm;
  c.tile_of = p->tile_of;
  c.rank = p->rank;
  c.out_scratch = p->spec;
  c.out_scratch_bytes = spec_bytes(p);
  c.grid = p->grid;
  c.zero_coef = p->zero_coef;
  c.charges = p->charges;
  c.coef_w = p->host.coef_w.data();
  c.deg_w = p->host.deg_w;
  c.stream = p->stream;
  c.grid2 = p->grid2;
  c.gsum = p->bsum;
  return c;
}

template <typename R>
int multiply(pswf_plan p, int want_energy, void* data) {
  const Plan& h = p->host;
  MultParams mp;
  for (int d = 0; d < 3; ++d) mp.M[d] = h.M[d];
  mp.inv_kc = 1.0 / h.k_c;
  mp.Mxh = h.M[0] / 2 + 1;
  mp.deg = h.deg_m;
  mp.K = h.K;
  dim3 grid(p->eblk, p->nrun * h.K);
  if (p->yzfft) {
    MultArgs a;
    a.spec = p->spec;
    a.mp = mp;
    a.lines = p->lines;
    a.nlines = p->nlines;
    a.nkx = p->nkx;
    a.K = h.K;
    a.blocks = p->eblk;
    a.chan = int64_t(mp.Mxh) * h.M[1] * h.M[2];
    a.pch = p->pch;
    a.scale = p->scale;
    a.bmat = p->bmat;
    a.coef = p->coef_m;
    a.iw2 = p->iw2;
    a.iw2_stride = p->Mh;
    a.tw = static_cast<const float2*>(p->xtw) + p->tw_off[1];
    a.part = p->epart;
    a.want_energy = want_energy;
    a.vpart = want_energy ? p->vpart : nullptr;
    return cuda_check(p, launch_mult_y(a, p->stream), "k_mult_y");
  }
  if (p->pruned) {
    (void)data;   // the pruned spectrum lives in p->spec
    k_multiply_planes<R><<<grid, kThreads, 0, p->stream>>>(static_cast<Cplx<R>*>(p->spec), mp, p->nkx, p->pch, p->scale,
                                                           p->bmat, static_cast<const R*>(p->coef_m),
                                                           static_cast<const R*>(p->iw2), p->Mh, p->epart,
                                                           want_energy, want_energy ? p->vpart : nullptr);
    return launch_check(p, "k_multiply_planes");
  }
  if (!(want_energy && p->vpart)) {
    // channels in chunks of kMultGroup per work item, the multiplier once per distinct exponent
    static_assert(kThreads == 256, "k_multiply_group's block sums assume 8 warps");
    const dim3 ggrid(p->eblk, p->nrun * ((h.K + kMultGroup - 1) / kMultGroup));
    k_multiply_group<R><<<ggrid, kThreads, 0, p->stream>>>(static_cast<Cplx<R>*>(data), mp, p->pch, p->scale, p->bmat,
                                                           static_cast<const R*>(p->coef_m),
                                                           static_cast<const R*>(p->iw2), p->Mh, p->epart,
                                                           want_energy);
    return launch_check(p, "k_multiply_group");
  }
  k_multiply<R><<<grid, kThreads, 0, p->stream>>>(static_cast<Cplx<R>*>(data), mp, p->pch, p->scale, p->bmat,
                                                  static_cast<const R*>(p->coef_m), static_cast<const R*>(p->iw2),
                                                  p->Mh, p->epart, want_energy, p->vpart);
  return launch_check(p, "k_multiply");
}

// Pruned 3-D transform of a single structure (per channel): forward = 1-D
// R2C along x writing the spectrum in [kx][z][y] order, zero the planes
// kx >= nkx, 2-D (z, y) transforms of the nkx planes that can hold band
// modes; inverse = the 2-D transforms, then 1-D C2R along x back to the grid.
int fft_exec_pruned(pswf_plan p, void* data, bool forward) {
  const Plan& h = p->host;
  const int Mxh = h.M[0] / 2 + 1;
  const int64_t plane = int64_t(h.M[2]) * h.M[1];
  const int64_t spec_ch = int64_t(Mxh) * plane;                 // complex per channel
  const int64_t grid_ch = plane * 2 * Mxh;                       // real per channel
  for (cufftHandle hd : {p->pr_r2c, p->pr_c2r, p->pr_2d})
    if (hd && cufftSetStream(hd, p->stream) != CUFFT_SUCCESS)
      return set_err(p, PSWF_ECUFFT, "cufftSetStream failed");
  cufftResult r = CUFFT_SUCCESS;
  const bool f32 = p->real_size == 4;
  auto cplx = [&](int c) -> void* {
    return static_cast<char*>(p->spec) + size_t(c) * spec_ch * 2 * p->real_size;
  };
  auto real = [&](int c) -> void* { return static_cast<char*>(data) + size_t(c) * grid_ch * p->real_size; };
  auto planes = [&](int c) {
    const int dir = forward ? CUFFT_FORWARD : CUFFT_INVERSE;
    if (f32) return cufftExecC2C(p->pr_2d, static_cast<cufftComplex*>(cplx(c)), static_cast<cufftComplex*>(cplx(c)), dir);
    return cufftExecZ2Z(p->pr_2d, static_cast<cufftDoubleComplex*>(cplx(c)), static_cast<cufftDoubleComplex*>(cplx(c)),
                        dir);
  };
  if (p->xfft) {
    // x passes by the pruned kernels: planes kx >= nkx are never touched;
    // with yzfft the (z, y) passes are own kernels too (the y transforms run
    // inside the multiplier)
    const float2* tw = static_cast<const float2*>(p->xtw);
    auto zpass = [&](bool inverse) {
      const int rc = cuda_check(p, launch_fft_z(inverse, p->spec, h.M[2], h.M[1], h.K, p->nkx, spec_ch,
                                                tw + p->tw_off[2], p->lmask, p->stream), "k_fft_z");
      if (!rc) ++p->launches[p->cur_stage];
      return rc;
    };
    if (forward) {
      int rc = cuda_check(p, launch_rfft_x(static_cast<const float*>(data), h.M[0], h.M[1], h.M[2], h.K, p->nkx,
                                           p->xtw, p->spec, p->stream), "k_rfft_x");
      if (rc) return rc;
      ++p->launches[p->cur_stage];
      if (p->yzfft) return zpass(false);
      for (int c = 0; c < h.K && r == CUFFT_SUCCESS; ++c) r = planes(c);
    } else {
      if (p->yzfft) {
        if (int rc = zpass(true)) return rc;
      }
      for (int c = 0; c < h.K && r == CUFFT_SUCCESS && !p->yzfft; ++c) r = planes(c);
      if (r == CUFFT_SUCCESS) {
        int rc = cuda_check(p, launch_irfft_x(p->spec, h.M[0], h.M[1], h.M[2], h.K, p->nkx, p->xtw,
                                              static_cast<float*>(data), p->stream, p->psi_il), "k_irfft_x");
        if (rc) return rc;
        ++p->launches[p->cur_stage];
      }
    }
    if (r != CUFFT_SUCCESS) return set_err(p, PSWF_ECUFFT, "cufftExec failed (" + std::to_string(int(r)) + ")");
    return PSWF_OK;
  }
  if (forward) {
    for (int c = 0; c < h.K && r == CUFFT_SUCCESS; ++c)
      r = f32 ? cufftExecR2C(p->pr_r2c, static_cast<cufftReal*>(real(c)), static_cast<cufftComplex*>(cplx(c)))
              : cufftExecD2Z(p->pr_r2c, static_cast<cufftDoubleReal*>(real(c)), static_cast<cufftDoubleComplex*>(cplx(c)));
    if (r == CUFFT_SUCCESS && p->nkx < Mxh) {
      const size_t cs = 2 * p->real_size;
      int rc = cuda_check(p, cudaMemset2DAsync(static_cast<char*>(p->spec) + size_t(p->nkx) * plane * cs,
                                               size_t(spec_ch) * cs, 0, size_t(Mxh - p->nkx) * plane * cs, size_t(h.K),
                                               p->stream), "clear pruned planes");
      if (rc) return rc;
    }
    for (int c = 0; c < h.K && r == CUFFT_SUCCESS; ++c) r = planes(c);
  } else {
    for (int c = 0; c < h.K && r == CUFFT_SUCCESS; ++c) r = planes(c);
    for (int c = 0; c < h.K && r == CUFFT_SUCCESS; ++c)
      r = f32 ? cufftExecC2R(p->pr_c2r, static_cast<cufftComplex*>(cplx(c)), static_cast<cufftReal*>(real(c)))
              : cufftExecZ2D(p->pr_c2r, static_cast<cufftDoubleComplex*>(cplx(c)), static_cast<cufftDoubleReal*>(real(c)));
  }
  if (r != CUFFT_SUCCESS) return set_err(p, PSWF_ECUFFT, "cufftExec failed (" + std::to_string(int(r)) + ")");
  return PSWF_OK;
}

int fft_exec(pswf_plan p, void* data, bool forward) {
  if (p->pruned) return fft_exec_pruned(p, data, forward);
  cufftResult r;
  size_t fi = 0;
  while (fi + 1 < p->fft_sizes.size() && p->fft_sizes[fi] != p->nrun) ++fi;
  cufftHandle hdl = forward ? p->fwd[fi] : p->inv[fi];
  if (cufftSetStream(hdl, p->stream) != CUFFT_SUCCESS) return set_err(p, PSWF_ECUFFT, "cufftSetStream failed");
  if (p->real_size == 4) {
    r = forward ? cufftExecR2C(hdl, static_cast<cufftReal*>(data), static_cast<cufftComplex*>(data))
                : cufftExecC2R(hdl, static_cast<cufftComplex*>(data), static_cast<cufftReal*>(data));
  } else {
    r = forward ? cufftExecD2Z(hdl, static_cast<cufftDoubleReal*>(data), static_cast<cufftDoubleComplex*>(data))
                : cufftExecZ2D(hdl, static_cast<cufftDoubleComplex*>(data), static_cast<cufftDoubleReal*>(data));
  }
  if (r != CUFFT_SUCCESS) return set_err(p, PSWF_ECUFFT, "cufftExec failed (" + std::to_string(int(r)) + ")");
  return PSWF_OK;
}

// Q_net and Q_self per (structure, channel) of values [K][n] in caller order:
// batch plans one warp per (structure, channel) (1 launch), single plans
// block partials and a final pass (2 launches).
template <typename R>
int charge_sums(pswf_plan p, const void* vals, double* out) {
  const int K = p->host.K;
  if (p->batch) {
    k_charge_sums_warp<R><<<(p->nrun * K + 7) / 8, 256, 0, p->stream>>>(static_cast<const R*>(vals), K, p->nrun,
                                                                         p->soff, out);
    return launch_check(p, "k_charge_sums_warp");
  }
  k_charge_partials_seg<R><<<dim3(p->nqb, p->nrun), kThreads, 0, p->stream>>>(static_cast<const R*>(vals), K, p->nrun,
                                                                          p->soff, p->qpart);
  int rc = launch_check(p, "k_charge_partials_seg");
  if (rc) return rc;
  k_charge_final_seg<<<p->nrun * K, 256, 0, p->stream>>>(p->nqb, K, p->nrun, p->qpart, out);
  return launch_check(p, "k_charge_final_seg");
}

// Counts (batch plans: the atom offsets arrive with the structure tables;
// single plans: written here), bins, scans, scatters, and sums the charges.
// Launch shapes depend only on the plan's capacity; kernels read the atom
// count from soff.
template <typename R>
int do_set_points(pswf_plan p, int64_t n, const void* pos, int pos_dtype, const void* q) {
  cudaStream_t s = p->stream;
  int rc;
  p->n = n;
  p->psi_valid = false;
  p->virial_valid = false;
  StageScope scope(p, PSWF_STAGE_SET_POINTS);
  p->launches[PSWF_STAGE_SET_POINTS] += p->batch ? 6 : 8;
  if (!p->batch) {
    k_set_count<<<1, 32, 0, s>>>(p->soff, int(n));
    if ((rc = launch_check(p, "k_set_count"))) return rc;
  }
  const int ntl = p->nrun * p->nts;
  const int nsb = (ntl + p->scan_per_block - 1) / p->scan_per_block;
  Geometry geo = p->geo;
  geo.B = p->nrun;
  if ((rc = cuda_check(p, cudaMemsetAsync(p->tile_count, 0, size_t(ntl) * 4, s), "clear counts"))) return rc;
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((p->n_max + kThreads - 1) / kThreads, 148 * 32)));
  if (pos_dtype == 0)
    k_bin<float, R><<<blocks, kThreads, 0, s>>>(static_cast<const float*>(pos), geo, p->smol, p->tmat, p->soff, p->tile_of,
                                                p->rank, p->tile_count, static_cast<R*>(p->tmp_t), p->tmp_cell,
                                                p->n_max, p->err);
  else
    k_bin<double, R><<<blocks, kThreads, 0, s>>>(static_cast<const double*>(pos), geo, p->smol, p->tmat, p->soff,
                                                 p->tile_of, p->rank, p->tile_count, static_cast<R*>(p->tmp_t),
                                                 p->tmp_cell, p->n_max, p->err);
  if ((rc = launch_check(p, "k_bin"))) return rc;
  k_scan_block_sums<<<nsb, kScanBlock, 0, s>>>(ntl, p->tile_count, p->scan_sums, p->scan_per_block);
  if ((rc = launch_check(p, "k_scan_block_sums"))) return rc;
  k_scan_sums<<<1, 32, 0, s>>>(nsb, p->scan_sums);
  if ((rc = launch_check(p, "k_scan_sums"))) return rc;
  k_scan_apply<<<nsb, kScanBlock, 0, s>>>(ntl, p->tile_count, p->scan_sums, p->scan_per_block,
                                                      p->tile_start);
  if ((rc = launch_check(p, "k_scan_apply"))) return rc;
  // the charges are read from here on; when their copy runs on another
  // stream, the binning and the scan above overlap it and the stage's time
  // starts once they have arrived
  if (p->q_ready) {
    if ((rc = cuda_check(p, cudaStreamWaitEvent(s, p->q_ready, 0), "wait for the charges"))) return rc;
    scope.restart();
  }
  void* recbuf = record_buffer(p);
  if (recbuf == p->grid) p->grid_zeroed = false;
  if (recbuf) {
    // records in slot order first (in a buffer unused until execute), then unpacked
    float4* rec = static_cast<float4*>(recbuf);
    float4* qrec = rec + 2 * p->n_max;
    k_scatter_rec<<<blocks, kThreads, 0, s>>>(p->n_max, static_cast<const float*>(q), geo, p->soff, p->tile_of,
                                              p->rank, p->tile_start, static_cast<const float*>(p->tmp_t),
                                              p->tmp_cell, rec, qrec);
    if ((rc = launch_check(p, "k_scatter_rec"))) return rc;
    k_unpack_rec<<<blocks, kThreads, 0, s>>>(p->n_max, p->host.K, p->nrun, p->soff, rec, qrec,
                                             static_cast<float*>(p->st), p->scell, static_cast<float*>(p->sq),
                                             p->sperm);
    if ((rc = launch_check(p, "k_unpack_rec"))) return rc;
    ++p->launches[PSWF_STAGE_SET_POINTS];
  } else {
    k_scatter<R><<<blocks, kThreads, 0, s>>>(p->n_max, static_cast<const R*>(q), geo, p->soff, p->tile_of, p->rank,
                                             p->tile_start, static_cast<const R*>(p->tmp_t), p->tmp_cell,
                                             static_cast<R*>(p->st), p->scell, static_cast<R*>(p->sq), p->sperm);
    if ((rc = launch_check(p, "k_scatter"))) return rc;
  }
  if (p->tscale && ntl > 0) {
    const int tb = int(std::min<int64_t>((int64_t(ntl) * 32 + kThreads - 1) / kThreads, 148 * 64));
    k_tile_scale<<<tb, kThreads, 0, s>>>(ntl, p->host.K, p->n_max, p->tile_start,
                                          static_cast<const float*>(p->sq), p->tscale);
    if ((rc = launch_check(p, "k_tile_scale"))) return rc;
    ++p->launches[PSWF_STAGE_SET_POINTS];
  }
  return charge_sums<R>(p, q, p->charges);
}

template <typename R>
int do_execute(pswf_plan p, double* energy, void* phi, void* forces) {
  cudaStream_t s = p->stream;
  int rc;
  const LaunchCtx ctx = make_ctx(p);
  {
    StageScope scope(p, PSWF_STAGE_SPREAD);
    if (p->grid_zeroed) {   // cleared on the side stream meanwhile
      p->grid_zeroed = false;
      if ((rc = cuda_check(p, cudaStreamWaitEvent(s, p->ev_clear, 0), "wait for the grid clearing"))) return rc;
    } else if ((rc = cuda_check(p, cudaMemsetAsync(p->grid, 0, size_t(run_grid_elems(p)) * sizeof(R), s),
                              "clear grid")))
      return rc;
    if (p->n > 0 || p->batch) {
      int nl = 0;
      cudaError_t e = sizeof(R) == 4 ? launch_spread_float(ctx, &nl) : launch_spread_double(ctx, &nl);
      p->launches[PSWF_STAGE_SPREAD] += nl;
      if ((rc = cuda_check(p, e, "spread"))) return rc;
    }
  }
  {
    StageScope scope(p, PSWF_STAGE_FFT_FWD);
    if ((rc = fft_exec(p, p->grid, true))) return rc;
  }
  {
    StageScope scope(p, PSWF_STAGE_MULTIPLY);
    if ((rc = multiply<R>(p, 1, p->grid))) return rc;
    k_energy_final<<<p->nrun, 256, 0, s>>>(p->host.K, p->eblk, p->epart, p->zero_coef, p->charges,
                                           energy ? energy : p->energy_tmp, p->vpart, p->virial);
    p->virial_valid = p->virial != nullptr;
    if (energy && p->nrun < p->B &&
        (rc = cuda_check(p, cudaMemsetAsync(energy + size_t(p->nrun) * (p->host.K + 1), 0,
                                            size_t(p->B - p->nrun) * (p->host.K + 1) * 8, s), "clear energies")))
      return rc;
    if ((rc = launch_check(p, "k_energy_final"))) return rc;
    p->launches[PSWF_STAGE_MULTIPLY] += 2;
  }
  const bool keep_psi = (p->flags & PSWF_FLAG_BACKWARD) != 0;
  if (p->n == 0 && !p->batch) {
    p->psi_valid = keep_psi;   // nothing to gather; a backward has nothing to do
    return PSWF_OK;
  }
  if (phi || forces || keep_psi) {
    {
      StageScope scope(p, PSWF_STAGE_FFT_INV);
      if ((rc = fft_exec(p, p->grid, false))) return rc;
    }
    p->psi_valid = keep_psi;
    if (!(phi || forces)) return PSWF_OK;
    StageScope scope(p, PSWF_STAGE_INTERP);
    int nl = 0;
    cudaError_t e = sizeof(R) == 4 ? launch_interp_float(ctx, phi, forces, &nl)
                                   : launch_interp_double(ctx, phi, forces, &nl);
    if ((rc = cuda_check(p, e, "interp"))) return rc;
    if (p->tric && forces && p->n > 0) {
      // grid-coordinate gradients -> Cartesian forces, F = T^T f_u
      const int blocks = int(std::min<int64_t>((p->n + kThreads - 1) / kThreads, 148 * 8));
      k_force_cell<R><<<blocks, kThreads, 0, s>>>(p->n, p->tmat, static_cast<R*>(forces));
      if ((rc = launch_check(p, "k_force_cell"))) return rc;
      ++nl;
    }
    p->launches[PSWF_STAGE_INTERP] += nl;
  }
  return PSWF_OK;
}

// Vector-Jacobian product (the formulas are on the kernels in backward.cuh):
// sum of the upstream gphi per channel, rhobar spread into the second grid,
// FFT / the same multiplier / inverse FFT (A is symmetric), then one gather
// that reads Psi (kept by execute) and A rhobar.
template <typename R>
int do_backward(pswf_plan p, const double* g_energy, const void* g_phi, const void* g_forces, void* grad_q,
                void* grad_pos) {
  cudaStream_t s = p->stream;
  int rc;
  if (!grad_q && !grad_pos) return PSWF_OK;
  StageScope scope(p, PSWF_STAGE_BACKWARD);
  const LaunchCtx ctx = make_ctx(p);
  const int K = p->host.K;
  int nl = 0;
  cudaError_t e;
  const int cblocks = int(std::min<int64_t>((std::max<int64_t>(p->n, 1) + kThreads - 1) / kThreads, 148 * 8));
  if (p->tric && g_forces && p->n > 0) {
    // general cell: g_F into grid coordinates, g_u = T g_F, in the binning
    // scratch (free once set_points has sorted the atoms; n x 3 fits its
    // 3 x n_max reals); the kernels below then run as for a box
    k_grad_to_cell<R><<<cblocks, kThreads, 0, s>>>(p->n, p->tmat, static_cast<const R*>(g_forces),
                                                    static_cast<R*>(p->tmp_t));
    if ((rc = launch_check(p, "k_grad_to_cell"))) return rc;
    ++nl;
    g_forces = p->tmp_t;
  }
  const BackwardArgs b{g_energy, g_phi, g_forces, grad_q, grad_pos};
  if (g_phi) {
    if ((rc = charge_sums<R>(p, g_phi, p->bsum))) return rc;
    nl += p->batch ? 1 : 2;
  } else if ((rc = cuda_check(p, cudaMemsetAsync(p->bsum, 0, size_t(p->nrun) * K * 2 * sizeof(double), s),
                              "clear bsum"))) {
    return rc;
  }
  if ((rc = cuda_check(p, cudaMemsetAsync(p->grid2, 0, size_t(run_grid_elems(p)) * sizeof(R), s), "clear grid2")))
    return rc;
  if (g_phi || g_forces) {
    e = sizeof(R) == 4 ? launch_backward_float(ctx, b, 0, &nl) : launch_backward_double(ctx, b, 0, &nl);
    if ((rc = cuda_check(p, e, "backward spread"))) return rc;
    if ((rc = fft_exec(p, p->grid2, true))) return rc;
    if ((rc = multiply<R>(p, 0, p->grid2))) return rc;
    ++nl;
    if ((rc = fft_exec(p, p->grid2, false))) return rc;
  }
  e = sizeof(R) == 4 ? launch_backward_float(ctx, b, 1, &nl) : launch_backward_double(ctx, b, 1, &nl);
  if ((rc = cuda_check(p, e, "backward gather"))) return rc;
  if (p->tric && grad_pos && p->n > 0) {
    // dL/dr = T^T dL/du
    k_force_cell<R><<<cblocks, kThreads, 0, s>>>(p->n, p->tmat, static_cast<R*>(grad_pos));
    if ((rc = launch_check(p, "k_force_cell"))) return rc;
    ++nl;
  }
  p->launches[PSWF_STAGE_BACKWARD] += nl;
  return PSWF_OK;
}

// Per-batch structure tables: filled on the host into the plan's pinned
// mirror (after the previous upload from it has completed) and copied to the
// device on the plan's stream.
int batch_tables_async(pswf_plan p, int b, const double* boxes, const int* ps, const int64_t* offsets) {
  int rc;
  if (!p->h_stab) {
    if ((rc = cuda_check(p, cudaMallocHost(&p->h_stab, size_t(p->stab_bytes)), "pinned table mirror"))) return rc;
    if ((rc = cuda_check(p, cudaEventCreateWithFlags(&p->stab_ev, cudaEventDisableTiming), "table event"))) return rc;
  } else if ((rc = cuda_check(p, cudaEventSynchronize(p->stab_ev), "wait for the previous table upload"))) {
    return rc;
  }
  if ((rc = fill_stab(p, b, boxes, ps, offsets, static_cast<char*>(p->h_stab)))) return rc;
  if ((rc = cuda_check(p, cudaMemcpyAsync(p->stab, p->h_stab, size_t(p->stab_bytes), cudaMemcpyHostToDevice,
                                          p->stream), "upload structure tables")))
    return rc;
  return cuda_check(p, cudaEventRecord(p->stab_ev, p->stream), "record table upload");
}

}  // namespace

namespace pswf {

int plan_fill_tables(pswf_plan p, int b, const double* boxes, const int* ps, const int64_t* offsets) {
  int rc = ensure_workspace(p);
  if (rc) return rc;
  if (!p->h_stab) {
    if ((rc = cuda_check(p, cudaMallocHost(&p->h_stab, size_t(p->stab_bytes)), "pinned table mirror"))) return rc;
    if ((rc = cuda_check(p, cudaEventCreateWithFlags(&p->stab_ev, cudaEventDisableTiming), "table event"))) return rc;
  }
  if ((rc = fill_stab(p, b, boxes, ps, offsets, static_cast<char*>(p->h_stab)))) return rc;
  p->nrun = run_size(p, b);
  return PSWF_OK;
}

int plan_run_size(pswf_plan p) { return p->nrun; }

const int* plan_run_sizes(pswf_plan p, int* count) {
  *count = int(p->fft_sizes.size());
  return p->fft_sizes.data();
}

int plan_upload_tables(pswf_plan p) {
  return cuda_check(p, cudaMemcpyAsync(p->stab, p->h_stab, size_t(p->stab_bytes), cudaMemcpyHostToDevice, p->stream),
                    "upload structure tables");
}

int plan_run_set_points(pswf_plan p, int64_t n, const void* pos, int pos_dtype, const void* q) {
  return p->real_size == 4 ? do_set_points<float>(p, n, pos, pos_dtype, q) : do_set_points<double>(p, n, pos, pos_dtype, q);
}

int plan_run_execute(pswf_plan p, double* energy, void* phi, void* forces) {
  return p->real_size == 4 ? do_execute<float>(p, energy, phi, forces) : do_execute<double>(p, energy, phi, forces);
}

cudaStream_t plan_stream(pswf_plan p) { return p->stream; }
int plan_precision(pswf_plan p) { return p->real_size == 8 ? 1 : 0; }
const char* plan_error(pswf_plan p) { return p->last_error.c_str(); }

}  // namespace pswf

namespace {

int make_fft(pswf_plan p) {
  const Plan& h = p->host;
  int n[3] = {h.M[2], h.M[1], h.M[0]};
  const int Mxh = h.M[0] / 2 + 1;
  int embed_r[3] = {h.M[2], h.M[1], 2 * Mxh};
  int embed_c[3] = {h.M[2], h.M[1], Mxh};
  const int dist_r = h.M[2] * h.M[1] * 2 * Mxh;
  const int dist_c = h.M[2] * h.M[1] * Mxh;
  const cufftType tf = p->real_size == 4 ? CUFFT_R2C : CUFFT_D2Z;
  const cufftType ti = p->real_size == 4 ? CUFFT_C2R : CUFFT_Z2D;
  p->fft_made = true;
  p->fft_work_bytes = 0;
  if (p->B == 1) {
    const double kmax_idx = h.k_c * h.box[0] / (2.0 * 3.14159265358979323846);
    p->nkx = int(std::min<double>(Mxh, std::floor(kmax_idx) + 2));
    p->pruned = p->nkx * 4 <= Mxh * 3 && h.M[0] >= 64;
    p->xfft = p->pruned && p->real_size == 4 && xfft_supported(h.M[0]);
    p->yzfft = p->xfft && xfft_supported(h.M[1]) && xfft_supported(h.M[2]);
    p->psi_il = p->xfft && h.K % 4 == 0 && h.P <= 8 && !(p->flags & PSWF_FLAG_BACKWARD);
  }
  if (p->yzfft) {   // no cuFFT plan
    p->fft_sizes.assign(1, 1);
    return PSWF_OK;
  }
  if (p->pruned) {
    const cufftType c2c = p->real_size == 4 ? CUFFT_C2C : CUFFT_Z2Z;
    const int plane = h.M[2] * h.M[1];
    int n1[1] = {h.M[0]};
    int er[1] = {2 * Mxh}, ec[1] = {Mxh};
    int n2[2] = {h.M[2], h.M[1]};
    size_t w1 = 0, w2 = 0, w3 = 0;
    for (cufftHandle* hd : {&p->pr_r2c, &p->pr_c2r, &p->pr_2d}) {
      if (p->xfft && hd != &p->pr_2d) continue;
      if (cufftCreate(hd) != CUFFT_SUCCESS) return set_err(p, PSWF_ECUFFT, "cufftCreate failed");
      cufftSetAutoAllocation(*hd, 0);
    }
    // rows (z, y) of the grid -> spectrum element (kx, z, y) at kx * plane + (z My + y)
    const cufftResult r1 =
        p->xfft ? CUFFT_SUCCESS : cufftMakePlanMany(p->pr_r2c, 1, n1, er, 1, 2 * Mxh, ec, plane, 1, tf, plane, &w1);
    const cufftResult r2 =
        p->xfft ? CUFFT_SUCCESS : cufftMakePlanMany(p->pr_c2r, 1, n1, ec, plane, 1, er, 1, 2 * Mxh, ti, plane, &w2);
    const cufftResult r3 = cufftMakePlanMany(p->pr_2d, 2, n2, n2, 1, plane, n2, 1, plane, c2c, p->nkx, &w3);
    if (r1 != CUFFT_SUCCESS || r2 != CUFFT_SUCCESS || r3 != CUFFT_SUCCESS)
      return set_err(p, PSWF_ECUFFT, "cufftMakePlanMany (pruned) failed");
    p->fft_work_bytes = std::max(w1, std::max(w2, w3));
    p->fft_sizes.assign(1, 1);
    return PSWF_OK;
  }
  p->fft_sizes.clear();
  for (int sz = 1; sz < p->B; sz *= 2) p->fft_sizes.push_back(sz);
  p->fft_sizes.push_back(p->B);
  for (int sz : p->fft_sizes) {
    cufftHandle f = 0, g = 0;
    if (cufftCreate(&f) != CUFFT_SUCCESS) return set_err(p, PSWF_ECUFFT, "cufftCreate failed");
    p->fwd.push_back(f);
    if (cufftCreate(&g) != CUFFT_SUCCESS) return set_err(p, PSWF_ECUFFT, "cufftCreate failed");
    p->inv.push_back(g);
    cufftSetAutoAllocation(f, 0);
    cufftSetAutoAllocation(g, 0);
    size_t w1 = 0, w2 = 0;
    const int nb = sz * h.K;
    const cufftResult r1 = cufftMakePlanMany(f, 3, n, embed_r, 1, dist_r, embed_c, 1, dist_c, tf, nb, &w1);
    const cufftResult r2 = cufftMakePlanMany(g, 3, n, embed_c, 1, dist_c, embed_r, 1, dist_r, ti, nb, &w2);
    if (r1 != CUFFT_SUCCESS || r2 != CUFFT_SUCCESS)
      return set_err(p, PSWF_ECUFFT,
                     "cufftMakePlanMany failed (" + std::to_string(int(r1)) + "," + std::to_string(int(r2)) + ")");
    p->fft_work_bytes = std::max(p->fft_work_bytes, std::max(w1, w2));
  }
  return PSWF_OK;
}

Options to_options(const pswf_opts* opts) {
  Options o;
  o.tol = opts->tol > 0 ? opts->tol : 1e-5;
  o.r_c = opts->r_c;
  o.c = opts->c;
  o.c_w = opts->c_w;
  o.eta = opts->eta;
  o.P = opts->P;
  for (int d = 0; d < 3; ++d) o.grid[d] = opts->grid[d];
  o.precision = opts->precision;
  return o;
}

void fill_info(const Plan& h, int flags, pswf_info* out) {
  std::memset(out, 0, sizeof(*out));
  out->c = h.c;
  out->c_w = h.c_w;
  out->r_c = h.r_c;
  out->k_c = h.k_c;
  out->eta = h.eta;
  out->tol = h.tol;
  out->est_err_spread = h.est_spread;
  out->est_err_band = h.est_band;
  out->lambda0 = h.moll.lambda0;
  out->C0 = h.moll.C0;
  for (int d = 0; d < 3; ++d) {
    out->box[d] = h.box[d];
    out->h[d] = h.h[d];
    out->grid[d] = h.M[d];
  }
  out->P = h.P;
  out->K = h.K;
  out->precision = h.opt.precision;
  out->deg_window = h.deg_w;
  out->deg_mult = h.deg_m;
  out->deg_real = h.deg_g;
  out->flags = flags;
  out->B = 1;
  out->batch = 0;
}

}  // namespace

// ---- allocation-free self energy ------------------------------------------------
// Scratch of pswf_self_energy_noalloc: the per-block FP64 partial sums of q and
// q^2 ([kQBlocks][kMaxK][2]) followed by the per-channel totals ([kMaxK][2]),
// 152,576 bytes in all, resident on every GPU that loads this library.
static __device__ __align__(256) double pswf_noalloc_scratch[kQBlocks * kMaxK * 2 + kMaxK * 2];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {};

struct SelfCoef {
  double s[kMaxK];
};

// out[c] = s_c * Q_self^(c) from the charge totals in charges[c][2].
__global__ void k_self_energy_out(int K, SelfCoef sc, const double* __restrict__ charges, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < K) out[c] = sc.s[c] * charges[2 * c + 1];
}

// Device address of the scratch on the current device, looked up once per
// device with that device current (cudaGetSymbolAddress, no allocation).
int noalloc_scratch(pswf_plan p, double** out) {
  int dev = 0;
  int rc = cuda_check(p, cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev != p->device)
    return set_err(p, PSWF_EINVAL,
                   "pswf_self_energy_noalloc: the current device is not the plan's device (make it current)");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return set_err(p, PSWF_EINVAL, "pswf_self_energy_noalloc: device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    if ((rc = cuda_check(p, cudaGetSymbolAddress(&ptr, pswf_noalloc_scratch), "cudaGetSymbolAddress"))) return rc;
    g_noalloc_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return PSWF_OK;
}
}  // namespace

extern "C" {

int pswf_self_energy_noalloc(pswf_plan pl, int64_t n, const void* q, double* out, void* stream) {
  if (!pl || !out || (n > 0 && !q)) return PSWF_EINVAL;
  if (pl->batch) return set_err(pl, PSWF_EINVAL, "pswf_self_energy_noalloc takes a single-structure plan");
  const int K = pl->host.K;
  if (n < 0 || n > pl->n_max) return set_err(pl, PSWF_EINVAL, "pswf_self_energy_noalloc: n outside 0..n_max");
  if (K > kMaxK) return set_err(pl, PSWF_EINVAL, "pswf_self_energy_noalloc: more than 64 channels do not fit the scratch");
  double* scratch = nullptr;
  int rc = noalloc_scratch(pl, &scratch);
  if (rc) return rc;
  double* part = scratch;                           // [kQBlocks][K][2], every entry written below
  double* charges = scratch + kQBlocks * kMaxK * 2; // [K][2]
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (pl->real_size == 4)
    k_charge_partials<float><<<kQBlocks, kThreads, 0, s>>>(n, static_cast<const float*>(q), K, part);
  else
    k_charge_partials<double><<<kQBlocks, kThreads, 0, s>>>(n, static_cast<const double*>(q), K, part);
  if ((rc = launch_check(pl, "k_charge_partials (noalloc)"))) return rc;
  k_charge_final<<<1, 64, 0, s>>>(kQBlocks, K, part, charges);
  if ((rc = launch_check(pl, "k_charge_final (noalloc)"))) return rc;
  SelfCoef sc;
  for (int k = 0; k < kMaxK; ++k) sc.s[k] = k < K ? pl->host.self_coef[k] : 0.0;
  k_self_energy_out<<<1, 64, 0, s>>>(K, sc, charges, out);
  return launch_check(pl, "k_self_energy_out (noalloc)");
}

void pswf_opts_default(pswf_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-5;
}

int pswf_plan_params(const double box[3], int K, const int* p, const pswf_opts* opts, pswf_info* out) {
  if (!box || !p || !opts || !out) return PSWF_EINVAL;
  Plan h;
  const int rc = make_plan(box, K, p, to_options(opts), h);
  if (rc) return rc;
  fill_info(h, opts->flags, out);
  return PSWF_OK;
}

}  // extern "C"

namespace {
// Device-side shape of a plan whose host tables are made: geometry, tiles,
// scan, grid size, cuFFT plans and the workspace size.
int finish_create(pswf_plan pl, int64_t n_max, int b, const pswf_opts* opts, void* stream) {
  cudaGetDevice(&pl->device);
  pl->stream = static_cast<cudaStream_t>(stream);
  pl->n_max = n_max;
  pl->flags = opts->flags;
  pl->real_size = opts->precision == 1 ? 8 : 4;
  pl->B = b;
  const Plan& h = pl->host;
  pl->Mh = 0;
  for (int d = 0; d < 3; ++d) {
    pl->geo.M[d] = h.M[d];
    pl->geo.ntile[d] = (h.M[d] + kTile - 1) / kTile;
    pl->Mh = std::max(pl->Mh, h.M[d] / 2 + 1);
  }
  pl->geo.Mxp = 2 * (h.M[0] / 2 + 1);
  pl->geo.P = h.P;
  pl->geo.K = h.K;
  pl->tric = b == 1 && h.st.tric;
  pl->geo.tric = pl->tric ? 1 : 0;
  if (opts->flags & PSWF_FLAG_REAL_SPACE) {
    if (b != 1) return set_err(pl, PSWF_EINVAL, "real space: single structures only");
    if (h.K > kRsMaxK) return set_err(pl, PSWF_EINVAL, "real space: at most 16 channels");
    const bool ok = pl->tric ? real_space_geometry_cell(h.st.cell, h.r_c, pl->rs_geo)
                             : real_space_geometry(h.box, h.r_c, pl->rs_geo);
    if (!ok) return set_err(pl, PSWF_EINVAL, "real space: r_c needs more than 4096 images of the cell");
    if (pl->rs_geo.direct && n_max > kRsDirectMaxAtoms)
      return set_err(pl, PSWF_EINVAL,
                     "real space: a cell height below 3 r_c takes the direct pair sum, at most 16384 atoms");
    pl->rs_ncell = pl->rs_geo.nc[0] * pl->rs_geo.nc[1] * pl->rs_geo.nc[2];
    pl->rs_nsb = (pl->rs_ncell + 16383) / 16384;
  }
  pl->geo.nts = pl->geo.ntile[0] * pl->geo.ntile[1] * pl->geo.ntile[2];
  pl->geo.B = b;
  pl->nts = pl->geo.nts;
  pl->ntiles = b * pl->nts;
  pl->nqb = b > 1 ? kQBlocksBatch : kQBlocksPlan;
  // multiplier blocks per channel: about 8 half-spectrum elements a thread
  pl->eblk = int(std::max<int64_t>(
      1, std::min<int64_t>(kEnergyBlocks, int64_t(h.M[1]) * h.M[2] * (h.M[0] / 2 + 1) / (8 * kThreads))));
  pl->scan_per_block = 2048;   // two tiles per thread: short strips, several blocks in flight
  pl->scan_blocks = (pl->ntiles + pl->scan_per_block - 1) / pl->scan_per_block;
  pl->grid_elems = int64_t(b) * h.K * h.M[2] * h.M[1] * pl->geo.Mxp;
  int rc = make_fft(pl);
  if (rc) return rc;
  pl->ws_bytes = layout(pl, nullptr);
  return PSWF_OK;
}
}  // namespace

extern "C" {

int pswf_plan_create(const double box[3], int64_t n_max, int K, const int* p, const pswf_opts* opts, void* stream,
                     pswf_plan* out) {
  if (!out) return PSWF_EINVAL;
  *out = nullptr;
  if (!box || !p || !opts || n_max < 0 || n_max > (int64_t(1) << 31) - 1) return PSWF_EINVAL;
  pswf_plan pl = new (std::nothrow) pswf_plan_s();
  if (!pl) return PSWF_ENOMEM;
  int rc = make_plan(box, K, p, to_options(opts), pl->host);
  if (rc) {
    delete pl;
    return rc;
  }
  if ((rc = finish_create(pl, n_max, 1, opts, stream))) {
    pswf_plan_destroy(pl);
    return rc;
  }
  *out = pl;
  return PSWF_OK;
}

int pswf_plan_create_cell(const double cell[9], int64_t n_max, int K, const int* p, const pswf_opts* opts,
                          void* stream, pswf_plan* out) {
  if (!out) return PSWF_EINVAL;
  *out = nullptr;
  if (!cell || !p || !opts || n_max < 0 || n_max > (int64_t(1) << 31) - 1) return PSWF_EINVAL;
  pswf_plan pl = new (std::nothrow) pswf_plan_s();
  if (!pl) return PSWF_ENOMEM;
  int rc = make_plan_cell(cell, K, p, to_options(opts), pl->host);
  if (rc) {
    delete pl;
    return rc;
  }
  if ((rc = finish_create(pl, n_max, 1, opts, stream))) {
    pswf_plan_destroy(pl);
    return rc;
  }
  *out = pl;
  return PSWF_OK;
}

int pswf_batch_plan_create(const double box_max[3], int b_max, int64_t n_max, int K, const int* pset, int npset,
                           const pswf_opts* opts, void* stream, pswf_plan* out) {
  if (!out) return PSWF_EINVAL;
  *out = nullptr;
  if (!box_max || !pset || !opts || b_max < 1 || b_max > (1 << 16) || n_max < 0 ||
      n_max > (int64_t(1) << 31) - 1)
    return PSWF_EINVAL;
  pswf_plan pl = new (std::nothrow) pswf_plan_s();
  if (!pl) return PSWF_ENOMEM;
  int rc = make_batch_plan(box_max, K, pset, npset, to_options(opts), pl->host);
  if (rc) {
    delete pl;
    return rc;
  }
  pl->batch = true;
  if ((rc = finish_create(pl, n_max, b_max, opts, stream))) {
    pswf_plan_destroy(pl);
    return rc;
  }
  *out = pl;
  return PSWF_OK;
}

int pswf_batch_set_points(pswf_plan pl, int b, const double* boxes, const int* ps, const int64_t* offsets,
                          const void* pos, int pos_dtype, const void* q) {
  if (!pl) return PSWF_EINVAL;
  if (!pl->batch) return set_err(pl, PSWF_EINVAL, "pswf_batch_set_points needs a batch plan");
  if (b < 0 || b > pl->B) return set_err(pl, PSWF_EINVAL, "number of structures outside 0..b_max");
  if (b > 0 && (!boxes || !ps || !offsets)) return set_err(pl, PSWF_EINVAL, "boxes, ps and offsets are required");
  if (pos_dtype != 0 && pos_dtype != 1) return set_err(pl, PSWF_EINVAL, "pos_dtype must be 0 (float) or 1 (double)");
  int64_t n = 0;
  if (b > 0) {
    if (offsets[0] != 0) return set_err(pl, PSWF_EINVAL, "offsets[0] must be 0");
    for (int i = 0; i < b; ++i)
      if (offsets[i + 1] < offsets[i]) return set_err(pl, PSWF_EINVAL, "offsets must be non-decreasing");
    n = offsets[b];
  }
  if (n > pl->n_max) return set_err(pl, PSWF_EINVAL, "total atoms exceed n_max");
  if (n > 0 && (!pos || !q)) return set_err(pl, PSWF_EINVAL, "pos and q are required");
  int rc = ensure_workspace(pl);
  if (rc) return rc;
  if ((rc = batch_tables_async(pl, b, boxes, ps, offsets))) return rc;
  pl->nrun = run_size(pl, b);
  return pl->real_size == 4 ? do_set_points<float>(pl, n, pos, pos_dtype, q)
                            : do_set_points<double>(pl, n, pos, pos_dtype, q);
}

int pswf_plan_info(pswf_plan pl, pswf_info* out) {
  if (!pl || !out) return PSWF_EINVAL;
  fill_info(pl->host, pl->flags, out);
  out->n_max = pl->n_max;
  out->workspace_bytes = pl->ws_bytes;
  out->B = pl->B;
  out->batch = pl->batch ? 1 : 0;
  for (int i = 0; i < 9; ++i) out->cell[i] = pl->batch ? (i % 4 == 0 ? pl->host.box_max[i / 4] : 0.0) : pl->host.st.cell[i];
  out->transform = pl->yzfft  ? PSWF_TRANSFORM_OWN
                   : pl->xfft ? PSWF_TRANSFORM_PRUNED_X
                   : pl->pruned ? PSWF_TRANSFORM_PRUNED
                                : PSWF_TRANSFORM_FULL;
  out->nkx = pl->pruned ? pl->nkx : 0;
  return PSWF_OK;
}

int pswf_plan_set_workspace(pswf_plan pl, void* ws, int64_t bytes) {
  if (!pl || !ws) return PSWF_EINVAL;
  if (bytes < pl->ws_bytes) return set_err(pl, PSWF_ENOMEM, "workspace smaller than info.workspace_bytes");
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return set_err(pl, PSWF_EINVAL, "workspace must be 256-byte aligned");
  if (pl->ws_owned) {
    cudaFree(pl->ws);
    pl->ws_owned = false;
  }
  pl->ws = ws;
  layout(pl, static_cast<char*>(ws));
  pl->n = -1;
  int rc = attach_fft_work(pl);
  if (rc) return rc;
  return upload_tables(pl);
}

int pswf_plan_set_stream(pswf_plan pl, void* stream) {
  if (!pl) return PSWF_EINVAL;
  pl->stream = static_cast<cudaStream_t>(stream);
  return PSWF_OK;
}

int pswf_set_points(pswf_plan pl, int64_t n, const void* pos, int pos_dtype, const void* q) {
  if (!pl) return PSWF_EINVAL;
  if (pl->batch) return set_err(pl, PSWF_EINVAL, "batch plans take pswf_batch_set_points");
  if (n < 0 || n > pl->n_max) return set_err(pl, PSWF_EINVAL, "n outside 0..n_max");
  if (n > 0 && (!pos || !q)) return set_err(pl, PSWF_EINVAL, "pos and q are required");
  if (pos_dtype != 0 && pos_dtype != 1) return set_err(pl, PSWF_EINVAL, "pos_dtype must be 0 (float) or 1 (double)");
  const int rc = ensure_workspace(pl);
  if (rc) return rc;
  return pl->real_size == 4 ? do_set_points<float>(pl, n, pos, pos_dtype, q)
                            : do_set_points<double>(pl, n, pos, pos_dtype, q);
}

int pswf_execute(pswf_plan pl, double* energy, void* phi, void* forces) {
  if (!pl) return PSWF_EINVAL;
  if (pl->n < 0) return set_err(pl, PSWF_ESTATE, "pswf_execute before pswf_set_points");
  return pl->real_size == 4 ? do_execute<float>(pl, energy, phi, forces) : do_execute<double>(pl, energy, phi, forces);
}

int pswf_backward(pswf_plan pl, const double* g_energy, const void* g_phi, const void* g_forces, void* grad_q,
                  void* grad_pos) {
  if (!pl) return PSWF_EINVAL;
  if (!(pl->flags & PSWF_FLAG_BACKWARD)) return set_err(pl, PSWF_ESTATE, "plan was created without PSWF_FLAG_BACKWARD");
  if (pl->n < 0 || !pl->psi_valid) return set_err(pl, PSWF_ESTATE, "pswf_backward needs a preceding pswf_execute");
  if (pl->n == 0) return PSWF_OK;
  return pl->real_size == 4 ? do_backward<float>(pl, g_energy, g_phi, g_forces, grad_q, grad_pos)
                            : do_backward<double>(pl, g_energy, g_phi, g_forces, grad_q, grad_pos);
}

int pswf_self_energy(pswf_plan pl, double* out) {
  if (!pl || !out) return PSWF_EINVAL;
  if (pl->n < 0) return set_err(pl, PSWF_ESTATE, "pswf_self_energy before pswf_set_points");
  const int BK = pl->B * pl->host.K;
  std::vector<double> ch(2 * size_t(BK));
  int rc = cuda_check(pl, cudaMemcpyAsync(ch.data(), pl->charges, 2 * BK * sizeof(double), cudaMemcpyDeviceToHost,
                                          pl->stream), "read charges");
  if (rc) return rc;
  if ((rc = cuda_check(pl, cudaStreamSynchronize(pl->stream), "sync"))) return rc;
  const int nk = pl->nrun * pl->host.K;   // slots beyond the last launch hold no atoms
  for (int g = 0; g < BK; ++g) out[g] = g < nk ? pl->host.self_coef_p[pl->h_pch[g]] * ch[2 * g + 1] : 0.0;
  return PSWF_OK;
}

int pswf_virial(pswf_plan pl, double* virial) {
  if (!pl || !virial) return PSWF_EINVAL;
  if (!(pl->flags & PSWF_FLAG_VIRIAL)) return set_err(pl, PSWF_ESTATE, "plan was created without PSWF_FLAG_VIRIAL");
  if (!pl->virial_valid) return set_err(pl, PSWF_ESTATE, "pswf_virial needs a preceding pswf_execute");
  const size_t bytes = size_t(pl->B) * pl->host.K * 3 * 8;
  if (pl->nrun < pl->B) {
    int rc = cuda_check(pl, cudaMemsetAsync(virial, 0, bytes, pl->stream), "clear virial");
    if (rc) return rc;
  }
  // the diagonal (xx, yy, zz) of each channel's six components
  return cuda_check(pl, cudaMemcpy2DAsync(virial, 3 * 8, pl->virial, 6 * 8, 3 * 8, size_t(pl->nrun) * pl->host.K,
                                          cudaMemcpyDeviceToDevice, pl->stream), "copy virial");
}

int pswf_stress(pswf_plan pl, double* virial) {
  if (!pl || !virial) return PSWF_EINVAL;
  if (!(pl->flags & PSWF_FLAG_VIRIAL)) return set_err(pl, PSWF_ESTATE, "plan was created without PSWF_FLAG_VIRIAL");
  if (!pl->virial_valid) return set_err(pl, PSWF_ESTATE, "pswf_stress needs a preceding pswf_execute");
  const size_t bytes = size_t(pl->B) * pl->host.K * 6 * 8;
  if (pl->nrun < pl->B) {
    int rc = cuda_check(pl, cudaMemsetAsync(virial, 0, bytes, pl->stream), "clear virial");
    if (rc) return rc;
  }
  return cuda_check(pl, cudaMemcpyAsync(virial, pl->virial, size_t(pl->nrun) * pl->host.K * 6 * 8,
                                        cudaMemcpyDeviceToDevice, pl->stream), "copy virial tensor");
}

int pswf_real_space(pswf_plan pl, int64_t n, const void* pos, int pos_dtype, const void* q, double* energy,
                    void* phi, void* forces) {
  if (!pl || !energy) return PSWF_EINVAL;
  if (!(pl->flags & PSWF_FLAG_REAL_SPACE))
    return set_err(pl, PSWF_ESTATE, "plan was created without PSWF_FLAG_REAL_SPACE");
  if (n < 0 || n > pl->n_max) return set_err(pl, PSWF_EINVAL, "n outside 0..n_max");
  if (n > 0 && (!pos || !q)) return set_err(pl, PSWF_EINVAL, "pos and q are required");
  if (pos_dtype != 0 && pos_dtype != 1) return set_err(pl, PSWF_EINVAL, "pos_dtype must be 0 (float) or 1 (double)");
  int rc = ensure_workspace(pl);
  if (rc) return rc;
  StageScope scope(pl, PSWF_STAGE_REAL_SPACE);
  RealSpaceArgs a;
  a.geo = pl->rs_geo;
  a.n = n;
  a.nmax = std::max<int64_t>(pl->n_max, 1);
  a.K = pl->host.K;
  a.pos = pos;
  a.pos_dtype = pos_dtype;
  a.q = q;
  a.pch = pl->pch;
  a.coef_g = pl->coef_g;
  a.deg_g = pl->host.deg_g;
  a.count = pl->rs_count;
  a.cell_start = pl->rs_start;
  a.cell_of = pl->rs_cellof;
  a.rank = pl->rs_rank;
  a.lpos = pl->rs_lpos;
  a.perm = pl->rs_perm;
  a.scan_sums = pl->rs_scan;
  a.scan_per_block = 16384;
  a.err = pl->err;
  a.energy = energy;
  a.phi = phi;
  a.forces = forces;
  int nl = 0;
  const cudaError_t e = pl->real_size == 4 ? real_space_run<float>(a, pl->stream, &nl)
                                           : real_space_run<double>(a, pl->stream, &nl);
  pl->launches[PSWF_STAGE_REAL_SPACE] += nl;
  rc = cuda_check(pl, e, "real space");
  pl->rs_n = rc ? -1 : n;
  return rc;
}

int pswf_real_space_backward(pswf_plan pl, int64_t n, const void* pos, int pos_dtype, const void* q,
                             const double* g_energy, const void* g_phi, const void* g_forces, void* grad_q,
                             void* grad_pos) {
  if (!pl) return PSWF_EINVAL;
  if (!(pl->flags & PSWF_FLAG_REAL_SPACE))
    return set_err(pl, PSWF_ESTATE, "plan was created without PSWF_FLAG_REAL_SPACE");
  if (pl->rs_n < 0 || n != pl->rs_n)
    return set_err(pl, PSWF_ESTATE, "pswf_real_space_backward needs a preceding pswf_real_space on the same atoms");
  if (n > 0 && (!pos || !q)) return set_err(pl, PSWF_EINVAL, "pos and q are required");
  if (pos_dtype != 0 && pos_dtype != 1) return set_err(pl, PSWF_EINVAL, "pos_dtype must be 0 (float) or 1 (double)");
  if (!grad_q && !grad_pos) return PSWF_OK;
  StageScope scope(pl, PSWF_STAGE_REAL_SPACE);
  RealSpaceBwArgs a;
  a.geo = pl->rs_geo;
  a.n = n;
  a.K = pl->host.K;
  a.pos = pos;
  a.pos_dtype = pos_dtype;
  a.q = q;
  a.pch = pl->pch;
  a.coef_g = pl->coef_g;
  a.deg_g = pl->host.deg_g;
  a.cell_of = pl->rs_cellof;
  a.rank = pl->rs_rank;
  a.cell_start = pl->rs_start;
  a.perm = pl->rs_perm;
  a.lpos = pl->rs_lpos;
  a.nmax = std::max<int64_t>(pl->n_max, 1);
  a.g_energy = g_energy;
  a.g_phi = g_phi;
  a.g_forces = g_forces;
  a.grad_q = grad_q;
  a.grad_pos = grad_pos;
  a.err = pl->err;
  int nl = 0;
  const cudaError_t e = pl->real_size == 4 ? real_space_backward_run<float>(a, pl->stream, &nl)
                                           : real_space_backward_run<double>(a, pl->stream, &nl);
  pl->launches[PSWF_STAGE_REAL_SPACE] += nl;
  return cuda_check(pl, e, "real space backward");
}

int pswf_sync(pswf_plan pl) { return pswf_sync_for(pl, -1.0); }

int pswf_sync_for(pswf_plan pl, double timeout_ms) {
  if (!pl) return PSWF_EINVAL;
  int rc;
  if (timeout_ms < 0) {
    if ((rc = cuda_check(pl, cudaStreamSynchronize(pl->stream), "stream synchronize"))) return rc;
  } else {
    // poll the stream until it is idle or the deadline passes
    using SC = std::chrono::steady_clock;
    const auto limit =
        SC::now() + std::chrono::duration_cast<SC::duration>(std::chrono::duration<double, std::milli>(timeout_ms));
    for (;;) {
      const cudaError_t q = cudaStreamQuery(pl->stream);
      if (q == cudaSuccess) break;
      if (q != cudaErrorNotReady) return cuda_check(pl, q, "stream query");
      if (SC::now() >= limit) return set_err(pl, PSWF_ETIMEOUT, "pswf_sync_for: work still running at the deadline");
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
  {
    // bounds-checked build: the first failed index check of any kernel
    int bw = take_bounds_word();
    if (!bw) bw = bounds_word_float();
    if (!bw) bw = bounds_word_double();
    if (!bw) bw = bounds_word_real_space();
    if (bw)
      return set_err(pl, PSWF_EBOUNDS, "kernel index out of its buffer (bounds check " + std::to_string(bw) + ")");
  }
  if (!pl->err) return PSWF_OK;
  int flag = 0;
  if ((rc = cuda_check(pl, cudaMemcpy(&flag, pl->err, 4, cudaMemcpyDeviceToHost), "read status"))) return rc;
  if (flag) {
    cudaMemset(pl->err, 0, 4);
    return set_err(pl, flag, flag == PSWF_ENONFINITE ? "non-finite positions" : "device status");
  }
  return PSWF_OK;
}

}  // extern "C"

namespace {
// True for memory the GPU can copy from directly: page-locked host memory
// (cudaHostAlloc / cudaMallocHost or registered with cudaHostRegister).
// NULL counts as pinned (nothing to copy).
bool host_pinned(const void* ptr) {
  if (!ptr) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// out[i] = double(in[i]) for i < n (FP32 results widened for the caller).
__global__ void k_widen(int64_t n, const float* __restrict__ in, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = double(in[i]);
}

// out[i] = float(in[i]) for i < n (the caller's charges rounded to the FP32 path).
__global__ void k_narrow(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = float(in[i]);
}
}  // namespace

extern "C" {

namespace {

// pswf_compute_host (real_io false: charges and results double) and
// pswf_compute_host_real (real_io true: in the plan's precision)
int compute_host(pswf_plan pl, int64_t n, const double* pos, const void* qv, double* energy, void* phiv,
                 void* forcesv, bool real_io) {
  const double* q = static_cast<const double*>(qv);
  double* phi = static_cast<double*>(phiv);
  double* forces = static_cast<double*>(forcesv);
  if (!pl || !energy || (n > 0 && (!pos || !q))) return PSWF_EINVAL;
  if (pl->batch) return set_err(pl, PSWF_EINVAL, "pswf_compute_host takes a single-structure plan");
  if (n < 0 || n > pl->n_max) return set_err(pl, PSWF_EINVAL, "n outside 0..n_max");
  const int K = pl->host.K;
  const int64_t rs = int64_t(pl->real_size);
  int rc = ensure_workspace(pl);
  if (rc) return rc;
  // Pinned caller arrays are copied directly (positions in; potentials and
  // forces out, widened to double on the device first); pageable ones go
  // through the plan's pinned staging buffers.
  const bool pos_direct = host_pinned(pos);
  const bool q_direct = host_pinned(q);
  const bool narrow = q_direct && rs == 4 && !real_io;
  const bool out_direct = host_pinned(phi) && host_pinned(forces);
  const bool widen = out_direct && rs == 4 && !real_io;
  const int64_t qs = real_io ? rs : 8;   // bytes per charge in the caller's array
  // device staging: pos double [n][3] | q real [K][n] | energy [K+1] | phi real [K][n] | forces real [n][3]
  //                 (| phi double [K][n] | forces double [n][3] when widening on the device)
  const int64_t need = align256(n * 3 * 8) + align256(K * n * rs) + align256((K + 1) * 8) + align256(K * n * rs) +
                       align256(n * 3 * rs) + (widen ? align256(K * n * 8) + align256(n * 3 * 8) : 0) +
                       (narrow ? align256(K * n * 8) : 0);
  if (need > pl->d_stage_bytes) {
    if (pl->d_stage) cudaFree(pl->d_stage);
    pl->d_stage = nullptr;
    pl->d_stage_bytes = 0;
    if ((rc = cuda_check(pl, cudaMalloc(&pl->d_stage, size_t(need)), "staging cudaMalloc"))) return rc;
    pl->d_stage_bytes = need;
  }
  // pinned host staging (bytes): pos double [n][3] | q real [K][n] | energy | phi real [K][n] | forces real [n][3]
  const int64_t hneed_b = std::max<int64_t>(n * 24 + K * n * rs + (K + 1) * 8 + K * n * rs + n * 3 * rs, 8);
  const int64_t hneed = (hneed_b + 7) / 8;
  if (hneed > pl->h_pin_elems) {
    if (pl->h_pin) cudaFreeHost(pl->h_pin);
    pl->h_pin = nullptr;
    pl->h_pin_elems = 0;
    if ((rc = cuda_check(pl, cudaMallocHost(&pl->h_pin, size_t(hneed) * 8), "pinned cudaMallocHost"))) return rc;
    pl->h_pin_elems = hneed;
  }
  char* d = static_cast<char*>(pl->d_stage);
  double* d_pos = reinterpret_cast<double*>(d);
  d += align256(n * 3 * 8);
  char* d_q = d;
  d += align256(K * n * rs);
  double* d_e = reinterpret_cast<double*>(d);
  d += align256((K + 1) * 8);
  char* d_phi = d;
  d += align256(K * n * rs);
  char* d_f = d;
  d += align256(n * 3 * rs);
  double* d_phi64 = widen ? reinterpret_cast<double*>(d) : nullptr;
  double* d_f64 = widen ? reinterpret_cast<double*>(d + align256(K * n * 8)) : nullptr;
  if (widen) d += align256(K * n * 8) + align256(n * 3 * 8);
  double* d_q64 = narrow ? reinterpret_cast<double*>(d) : nullptr;
  // measurement (profiling on): stream events around the input and output copy phases
  cudaEvent_t ev_in0 = nullptr;
  if (pl->prof_on) {
    ev_in0 = take_event(pl);
    cudaEventRecord(ev_in0, pl->stream);
  }
  char* hb = reinterpret_cast<char*>(pl->h_pin);
  double* h_pos = reinterpret_cast<double*>(hb);
  char* h_q = hb + n * 24;
  double* h_e = reinterpret_cast<double*>(h_q + K * n * rs);
  char* h_phi = reinterpret_cast<char*>(h_e + K + 1);
  char* h_f = h_phi + K * n * rs;
  cudaStream_t s = pl->stream;
  const bool split = pos_direct && q_direct && n > 0;   // the charges' copy on its own stream
  if (split && (rc = ensure_side_stream(pl))) return rc;
  // the grid is cleared for the spread while the positions are copied,
  // unless set_points parks its records there
  if (split && record_buffer(pl) != pl->grid && (rc = clear_grid_aside(pl))) return rc;
  if (pos_direct && n > 0 &&
      (rc = cuda_check(pl, cudaMemcpyAsync(d_pos, pos, size_t(n) * 24, cudaMemcpyHostToDevice, s), "h2d pos")))
    return rc;
  // the charges' stream: with both arrays page-locked, their copy (and the
  // rounding of float64 charges) runs on it after the positions' copy, and
  // set_points waits for it only before its first kernel that reads them
  cudaStream_t sq = s;
  if (split) {
    if ((rc = cuda_check(pl, cudaEventRecord(pl->ev_pos, s), "record positions copied")) ||
        (rc = cuda_check(pl, cudaStreamWaitEvent(pl->q_stream, pl->ev_pos, 0), "order the charges' copy")))
      return rc;
    sq = pl->q_stream;
  }
  if (q_direct && n > 0) {
    // pinned charges: copied as double, rounded to FP32 on the device
    if ((rc = cuda_check(pl, cudaMemcpyAsync(narrow ? static_cast<void*>(d_q64) : static_cast<void*>(d_q), q,
                                             size_t(K * n * qs), cudaMemcpyHostToDevice, sq), "h2d q")))
      return rc;
    if (narrow) {
      const int nb = int(std::min<int64_t>((K * n + kThreads - 1) / kThreads, 148 * 16));
      k_narrow<<<nb, kThreads, 0, sq>>>(K * n, d_q64, reinterpret_cast<float*>(d_q));
      if ((rc = launch_check(pl, "k_narrow"))) return rc;
      ++pl->launches[PSWF_STAGE_OTHER];
    }
  }
  cudaEvent_t q_done = nullptr;
  if (sq != s) {
    if ((rc = cuda_check(pl, cudaEventRecord(pl->ev_q, sq), "record charges copied"))) return rc;
    q_done = pl->ev_q;
  }
  // Inputs in chunks of atoms: the host threads fill chunk i of the pinned
  // staging (q rounded to the plan's precision; positions only when the
  // caller's are pageable) while the copies already enqueued run.
  const int64_t nchunk = std::max<int64_t>(1, std::min<int64_t>(16, n / 65536));
  const int64_t csz = (n + nchunk - 1) / nchunk;
  for (int64_t ci = 0; ci < nchunk && n > 0 && !(pos_direct && q_direct); ++ci) {
    const int64_t a0 = ci * csz, a1 = std::min(n, a0 + csz);
    if (a0 >= a1) break;
    parallel_for(a1 - a0, [&](int64_t lo, int64_t hi) {
      if (!pos_direct) std::memcpy(h_pos + 3 * (a0 + lo), pos + 3 * (a0 + lo), size_t(hi - lo) * 24);
      for (int k = 0; k < K && !q_direct; ++k) {
        const double* src = q + size_t(k) * n + a0;
        if (real_io) {
          std::memcpy(h_q + (size_t(k) * n + a0 + lo) * rs, static_cast<const char*>(qv) + (size_t(k) * n + a0 + lo) * rs,
                      size_t(hi - lo) * rs);
        } else if (rs == 4) {
          float* dst = reinterpret_cast<float*>(h_q) + size_t(k) * n + a0;
          for (int64_t i = lo; i < hi; ++i) dst[i] = float(src[i]);
        } else {
          std::memcpy(reinterpret_cast<double*>(h_q) + size_t(k) * n + a0 + lo, src + lo, size_t(hi - lo) * 8);
        }
      }
    });
    if (!pos_direct && (rc = cuda_check(pl, cudaMemcpyAsync(d_pos + 3 * a0, h_pos + 3 * a0, size_t(a1 - a0) * 24,
                                                            cudaMemcpyHostToDevice, s), "h2d pos")))
      return rc;
    if (!q_direct && (rc = cuda_check(pl, cudaMemcpy2DAsync(d_q + a0 * rs, size_t(n * rs), h_q + a0 * rs,
                                                             size_t(n * rs), size_t((a1 - a0) * rs), size_t(K),
                                                             cudaMemcpyHostToDevice, s), "h2d q")))
      return rc;
  }
  if (ev_in0) {
    cudaEvent_t b = take_event(pl);
    cudaEventRecord(b, sq);   // the end of the last copy (the charges' stream when it has its own)
    pl->recs.push_back({PSWF_STAGE_H2D, ev_in0, b});
  }
  pl->q_ready = q_done;
  rc = pswf_set_points(pl, n, d_pos, 1, d_q);
  pl->q_ready = nullptr;
  if (rc) return rc;
  if ((rc = pswf_execute(pl, d_e, phi ? d_phi : nullptr, forces ? d_f : nullptr))) return rc;
  cudaEvent_t ev_out0 = nullptr;
  if (pl->prof_on) {
    ev_out0 = take_event(pl);
    cudaEventRecord(ev_out0, s);
  }
  if ((rc = cuda_check(pl, cudaMemcpyAsync(h_e, d_e, size_t(K + 1) * 8, cudaMemcpyDeviceToHost, s), "d2h energy")))
    return rc;
  std::vector<cudaEvent_t> evs;
  const int64_t nchunk_out = out_direct ? 0 : nchunk;
  if (out_direct && n > 0) {
    // straight into the caller's pinned arrays (FP32 results widened first)
    const int wb = int(std::min<int64_t>((K * n + kThreads - 1) / kThreads, 148 * 16));
    if (phi) {
      const void* src = d_phi;
      if (widen) {
        k_widen<<<wb, kThreads, 0, s>>>(K * n, reinterpret_cast<const float*>(d_phi), d_phi64);
        if ((rc = launch_check(pl, "k_widen"))) return rc;
        ++pl->launches[PSWF_STAGE_OTHER];
        src = d_phi64;
      }
      if ((rc = cuda_check(pl, cudaMemcpyAsync(phi, src, size_t(K * n) * (widen ? 8 : rs), cudaMemcpyDeviceToHost, s),
                           "d2h phi")))
        return rc;
    }
    if (forces) {
      const void* src = d_f;
      if (widen) {
        k_widen<<<wb, kThreads, 0, s>>>(3 * n, reinterpret_cast<const float*>(d_f), d_f64);
        if ((rc = launch_check(pl, "k_widen"))) return rc;
        ++pl->launches[PSWF_STAGE_OTHER];
        src = d_f64;
      }
      if ((rc = cuda_check(pl, cudaMemcpyAsync(forces, src, size_t(3 * n) * (widen ? 8 : rs), cudaMemcpyDeviceToHost,
                                               s), "d2h forces")))
        return rc;
    }
  }
  // Pageable outputs in chunks: copy chunk i down, then the host threads
  // widen it into the caller's arrays while chunk i + 1 is in flight.
  for (int64_t ci = 0; ci < nchunk_out && n > 0; ++ci) {
    const int64_t a0 = ci * csz, a1 = std::min(n, a0 + csz);
    if (a0 >= a1) break;
    if (phi && (rc = cuda_check(pl, cudaMemcpy2DAsync(h_phi + a0 * rs, size_t(n * rs), d_phi + a0 * rs, size_t(n * rs),
                                                      size_t((a1 - a0) * rs), size_t(K), cudaMemcpyDeviceToHost, s),
                                "d2h phi")))
      return rc;
    if (forces && (rc = cuda_check(pl, cudaMemcpyAsync(h_f + 3 * a0 * rs, d_f + 3 * a0 * rs, size_t(a1 - a0) * 3 * rs,
                                                       cudaMemcpyDeviceToHost, s), "d2h forces")))
      return rc;
    cudaEvent_t ev = take_event(pl);
    if ((rc = cuda_check(pl, cudaEventRecord(ev, s), "record chunk"))) return rc;
    evs.push_back(ev);
  }
  if (ev_out0) {
    cudaEvent_t b = take_event(pl);
    cudaEventRecord(b, s);
    pl->recs.push_back({PSWF_STAGE_D2H, ev_out0, b});
  }
  for (int64_t ci = 0; ci < int64_t(evs.size()); ++ci) {
    const int64_t a0 = ci * csz, a1 = std::min(n, a0 + csz);
    if ((rc = cuda_check(pl, cudaEventSynchronize(evs[ci]), "wait for chunk"))) break;
    parallel_for(a1 - a0, [&](int64_t lo, int64_t hi) {
      if (real_io) {   // same precision: plain copies
        if (phi)
          for (int k = 0; k < K; ++k)
            std::memcpy(static_cast<char*>(phiv) + (size_t(k) * n + a0 + lo) * rs, h_phi + (size_t(k) * n + a0 + lo) * rs,
                        size_t(hi - lo) * rs);
        if (forces)
          std::memcpy(static_cast<char*>(forcesv) + size_t(3 * (a0 + lo)) * rs, h_f + size_t(3 * (a0 + lo)) * rs,
                      size_t(3 * (hi - lo)) * rs);
        return;
      }
      if (phi)
        for (int k = 0; k < K; ++k)
          for (int64_t i = a0 + lo; i < a0 + hi; ++i)
            phi[size_t(k) * n + i] = rs == 4 ? double(reinterpret_cast<const float*>(h_phi)[size_t(k) * n + i])
                                             : reinterpret_cast<const double*>(h_phi)[size_t(k) * n + i];
      if (forces)
        for (int64_t i = 3 * (a0 + lo); i < 3 * (a0 + hi); ++i)
          forces[i] = rs == 4 ? double(reinterpret_cast<const float*>(h_f)[i]) : reinterpret_cast<const double*>(h_f)[i];
    });
  }
  for (auto e : evs) pl->pool.push_back(e);
  if (rc) return rc;
  if ((rc = pswf_sync(pl))) return rc;
  std::memcpy(energy, h_e, size_t(K + 1) * 8);
  return PSWF_OK;
}

}  // namespace

int pswf_compute_host(pswf_plan pl, int64_t n, const double* pos, const double* q, double* energy, double* phi,
                      double* forces) {
  return compute_host(pl, n, pos, q, energy, phi, forces, false);
}

int pswf_compute_host_real(pswf_plan pl, int64_t n, const double* pos, const void* q, double* energy, void* phi,
                           void* forces) {
  return compute_host(pl, n, pos, q, energy, phi, forces, true);
}

void pswf_plan_destroy(pswf_plan pl) {
  if (!pl) return;
  for (auto hdl : pl->fwd) cufftDestroy(hdl);
  for (auto hdl : pl->inv) cufftDestroy(hdl);
  for (cufftHandle hdl : {pl->pr_r2c, pl->pr_c2r, pl->pr_2d})
    if (hdl) cufftDestroy(hdl);
  if (pl->ws_owned && pl->ws) cudaFree(pl->ws);
  if (pl->d_stage) cudaFree(pl->d_stage);
  if (pl->h_pin) cudaFreeHost(pl->h_pin);
  if (pl->h_stab) cudaFreeHost(pl->h_stab);
  if (pl->stab_ev) cudaEventDestroy(pl->stab_ev);
  if (pl->ev_in) cudaEventDestroy(pl->ev_in);
  if (pl->ev_clear) cudaEventDestroy(pl->ev_clear);
  if (pl->ev_pos) cudaEventDestroy(pl->ev_pos);
  if (pl->ev_q) cudaEventDestroy(pl->ev_q);
  if (pl->q_stream) cudaStreamDestroy(pl->q_stream);
  for (auto& r : pl->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : pl->pool) cudaEventDestroy(e);
  delete pl;
}

int pswf_profile_enable(pswf_plan pl, int enable) {
  if (!pl) return PSWF_EINVAL;
  pl->prof_on = enable != 0;
  return PSWF_OK;
}

int pswf_profile_read(pswf_plan pl, double* stage_ms, int64_t* launches) {
  if (!pl) return PSWF_EINVAL;
  int rc = cuda_check(pl, cudaStreamSynchronize(pl->stream), "stream synchronize");
  if (rc) return rc;
  double ms[PSWF_NSTAGE] = {};
  for (auto& r : pl->recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.stage] += t;
    pl->pool.push_back(r.a);
    pl->pool.push_back(r.b);
  }
  pl->recs.clear();
  for (int i = 0; i < PSWF_NSTAGE; ++i) {
    if (stage_ms) stage_ms[i] = ms[i];
    if (launches) launches[i] = pl->launches[i];
    pl->launches[i] = 0;
  }
  return PSWF_OK;
}

const char* pswf_strerror(int status) {
  switch (status) {
    case PSWF_OK: return "ok";
    case PSWF_EINVAL: return "invalid argument";
    case PSWF_ENOMEM: return "out of device memory";
    case PSWF_ECUFFT: return "cuFFT error";
    case PSWF_ECUDA: return "CUDA error";
    case PSWF_ETIMEOUT: return "wait timed out";
    case PSWF_ENONFINITE: return "non-finite positions";
    case PSWF_ETOLUNREACHABLE: return "tolerance unreachable on this grid";
    case PSWF_ESTATE: return "call out of order";
    case PSWF_ECELL: return "a real-space cell holds more than 2048 atoms";
    case PSWF_EBOUNDS: return "kernel index out of bounds (checked build)";
  }
  return "unknown status";
}

int pswf_plan_last_error(pswf_plan pl, char* buf, int len) {
  if (!pl || !buf || len <= 0) return PSWF_EINVAL;
  std::snprintf(buf, size_t(len), "%s", pl->last_error.c_str());
  return PSWF_OK;
}

}  // extern "C"
