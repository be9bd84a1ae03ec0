// Real-space complement: cell list and pair kernel, see
// realspace.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pswf {

constexpr int kRsMaxK = 16;   // channels of one real-space call

// Cells of an orthorhombic box: n_c per axis (>= 3), width w = L / n_c >= r_c.
struct RealSpaceGeom {
  int nc[3];
  double len[3], inv_len[3], w[3];
  double r_c;
};

// Device bytes per atom of the cell-local coordinates and records.
size_t real_space_bytes_per_atom(int K, int real_size);

// False when a box edge holds fewer than 3 cells of width >= r_c.
bool real_space_geometry(const double box[3], double r_c, RealSpaceGeom& g);

struct RealSpaceArgs {
  RealSpaceGeom geo;
  int64_t n, nmax;
  int K;
  const void* pos;      // [n][3], float or double (pos_dtype 0 / 1), any real value
  int pos_dtype;
  const void* q;        // real [K][n]
  const int* pch;       // device [K] exponents
  const void* coef_g;   // device real [6][kMultSeg][deg_g + 1]
  int deg_g;
  // scratch (device): counts and starts per cell, per-atom cell and rank,
  // cell-local test coordinates real [nmax][4] followed by the records
  // (exact coordinates and charges; real_space_bytes_per_atom in all), order
  int* count;
  int* cell_start;      // [ncell + 1]
  int* cell_of;
  int* rank;
  void* lpos;
  int* perm;
  int* scan_sums;
  int scan_per_block;
  int* err;
  // outputs: energy device double [K + 1] (per channel, total), phi real
  // [K][n] and forces real [n][3] (either may be null)
  double* energy;
  void* phi;
  void* forces;
};

template <typename R>
cudaError_t real_space_run(const RealSpaceArgs& a, cudaStream_t s, int* nlaunch);

}  // namespace pswf
