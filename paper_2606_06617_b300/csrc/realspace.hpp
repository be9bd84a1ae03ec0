// Real-space complement: cell list and pair kernel, see
// realspace.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pswf {

constexpr int kRsMaxK = 16;   // channels of one real-space call

// Cell list of a periodic cell H (lattice vectors a_d as rows): n_c per axis
// along each a_d (>= 3), each list cell the parallelepiped spanned by
// a_d / n_c[d], whose height across every pair of faces is >= r_c.  For an
// orthorhombic box H = diag(L) and the list cells are boxes of width L / n_c.
struct RealSpaceGeom {
  int nc[3];
  int tric;            // 0: orthorhombic box (the pair kernel's 3-multiply path)
  double hinv[9];      // H^-1, row-major: fractional s_d = sum_k r_k hinv[3 k + d]
  double cw[9];        // rows a_d / n_c[d]: the list cell's edge vectors
  double r_c;
  // direct mode (a height below 3 r_c: no cell list): every pair of atoms
  // over the images n H, |n_d| <= nimg[d]
  int direct;
  int nimg[3];
  double h[9];         // H, rows a_d
};

constexpr int kRsDirectMaxAtoms = 16384;   // direct mode: O(n^2 images) work
constexpr int kRsDirectMaxImages = 4096;

// Device bytes per atom of the cell-local coordinates, records, accumulator
// rows and the backward's upstream records.
size_t real_space_bytes_per_atom(int K, int real_size);

// Cell list when every height of the cell holds 3 list cells of height
// >= r_c; otherwise direct mode with the image ranges that hold every pair
// closer than r_c.  False for a singular cell or more than
// kRsDirectMaxImages images.
bool real_space_geometry(const double box[3], double r_c, RealSpaceGeom& g);
bool real_space_geometry_cell(const double cell[9], double r_c, RealSpaceGeom& g);

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

// Backward of the real-space complement (see realspace.cu): needs the cell
// list of a preceding real_space_run on the same points (cell-list mode).
struct RealSpaceBwArgs {
  RealSpaceGeom geo;
  int64_t n;
  int K;
  const void* pos;      // [n][3], float or double (pos_dtype 0 / 1)
  int pos_dtype;
  const void* q;        // real [K][n]
  const int* pch;       // device [K] exponents
  const void* coef_g;   // device real [6][kMultSeg][deg_g + 1]
  int deg_g;
  const int* cell_of;     // [n] list cell of each atom (cell-list mode)
  const int* rank;        // [n] its slot within the cell
  const int* cell_start;  // [ncell + 1]
  const int* perm;        // [n] original index of each sorted slot
  void* lpos;             // the forward's test coordinates, records and rows
  int64_t nmax;
  const double* g_energy; // device [K] or null
  const void* g_phi;      // real [K][n] or null
  const void* g_forces;   // real [n][3] or null
  void* grad_q;           // real [K][n] or null (written, not accumulated)
  void* grad_pos;         // real [n][3] or null (written, not accumulated)
  int* err;
};

template <typename R>
cudaError_t real_space_backward_run(const RealSpaceBwArgs& a, cudaStream_t s, int* nlaunch);

// Checked build: reads and clears the status word of this file's kernels
// (0 in the normal build).
int bounds_word_real_space();

}  // namespace pswf
