// Launch interface between the host API (api.cu) and the stencil kernels,
// which are instantiated per precision in launch.cu (compiled once with
// PSWF_REAL=float and once with PSWF_REAL=double).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace pswf {

struct LaunchCtx {
  Geometry geo;
  int64_t nmax = 0;        // capacity of the sorted atom arrays
  int64_t n = 0;           // output rows: atoms of the last set_points (batch plans: n_max)
  int64_t n_set = 0;       // atoms of the last set_points
  int ntiles = 0;          // B * nts
  const double* smol = nullptr;     // [B][3] M_d / L_d
  const int* soff = nullptr;        // [B + 1] atom offsets per structure (device)
  const int* tile_start = nullptr;
  const float* tscale = nullptr;    // [B nts][K] fixed-point units of the FP32 four-channel spread
  float* tscale_bw = nullptr;       // [B nts][K] the same for the backward's spread (backward plans)
  bool psi_il = false;              // Psi stored as channel quadruples [K / 4][Mz][My][Mxp][4]
  const void* st = nullptr;         // real [3][nmax]
  const uint64_t* scell = nullptr;  // [nmax]
  const void* sq = nullptr;         // real [K][nmax]
  const int* sperm = nullptr;       // [nmax]
  const int* tile_of = nullptr;     // [nmax] tile of each atom (caller order)
  const int* rank = nullptr;        // [nmax] its slot within the tile
  void* out_scratch = nullptr;      // idle during the gather (single structures' spectrum), or null
  int64_t out_scratch_bytes = 0;
  void* grid = nullptr;             // real [B][K][Mz][My][Mxp]
  const double* zero_coef = nullptr;   // [B K]
  const double* charges = nullptr;     // [B K][2]
  const double* coef_w = nullptr;   // host [P][deg_w + 1]
  int deg_w = 0;
  cudaStream_t stream = nullptr;
  // backward
  void* grid2 = nullptr;            // real [B][K][Mz][My][Mxp]
  const double* gsum = nullptr;     // [B K][2]: sum_j gphi_j^c (first entry)
};

struct BackwardArgs {
  const double* g_energy;   // device [B K] or null
  const void* g_phi;        // device real [K][n] or null
  const void* g_forces;     // device real [n][3] or null
  void* grad_q;             // device real [K][n] or null
  void* grad_pos;           // device real [n][3] or null
};

// Each returns cudaSuccess or the launch error.
cudaError_t launch_spread_float(const LaunchCtx& c, int* nlaunch);
cudaError_t launch_spread_double(const LaunchCtx& c, int* nlaunch);
cudaError_t launch_interp_float(const LaunchCtx& c, void* phi, void* forces, int* nlaunch);
cudaError_t launch_interp_double(const LaunchCtx& c, void* phi, void* forces, int* nlaunch);
// backward: spread of rhobar into grid2 (stage 0) or the final gather (stage 1)
cudaError_t launch_backward_float(const LaunchCtx& c, const BackwardArgs& b, int stage, int* nlaunch);
cudaError_t launch_backward_double(const LaunchCtx& c, const BackwardArgs& b, int stage, int* nlaunch);
// Bounds-check status word of the stencil kernels of either precision
// (checked build; read and cleared; 0 otherwise).
int bounds_word_float();
int bounds_word_double();

}  // namespace pswf
