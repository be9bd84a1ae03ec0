// Pruned transforms along x for the FP32 path of single-structure plans
// (step (ii) and its inverse, first and last 1-D pass of the 3-D transform).
//
// Forward: each real grid row (z, y) of length Mx = 32 N1 (2 <= N1 <= 16) is
// transformed (unnormalised, e^{-2 pi i k x / Mx}) and only the nkx lowest
// frequencies are written, into the spectrum layout [c][kx][z][y] (plane
// stride Mz My, channel stride Mxh Mz My).  Inverse: the Hermitian spectrum
// whose kx < nkx entries are given and whose other non-negative kx are zero is
// transformed back (unnormalised, e^{+2 pi i k x / Mx}) to the real rows.
// Planes kx >= nkx are neither written nor read.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "kernels.cuh"

namespace pswf {

// True when the row length has a kernel here (Mx = 32 N1, 2 <= N1 <= 16).
bool xfft_supported(int Mx);

// Twiddle table of a row length (host, float pairs): entries [k1 * 32 + l] =
// e^{-2 pi i l k1 / Mx} for k1 < N1 (forward); for the lane stages s < 5
// (distance d = 16 >> s) [Mx + s * 32 + l] = 1 on lanes with l & d = 0 and
// -e^{-2 pi i (l mod d) / 2d} on the others; then [Mx + 160 + n1 * 32 + l] =
// e^{-2 pi i n1 brev5(l) / Mx} for n1 < N1 (inverse x pass, conjugated in
// use); then the decimation-in-time stages st < 5 (d = 1 << st)
// [2 Mx + 160 + st * 32 + l] = e^{-2 pi i (l mod d) / 2d} on lanes with
// l & d set and 1 on the others; xfft_table_size() pairs.
int xfft_table_size(int Mx);
void xfft_twiddles(int Mx, std::vector<float>& out);

// grid: K channels of real rows (row stride Mxp = 2 (Mx / 2 + 1) floats,
// channel stride Mz My Mxp); spec: complex (float2) [K][Mx / 2 + 1][Mz][My];
// tw: the device copy of the twiddle table.  One launch each.
cudaError_t launch_rfft_x(const float* grid, int Mx, int My, int Mz, int K, int nkx, const void* tw, void* spec,
                          cudaStream_t s);
// interleave4 (K a multiple of 4): the inverse writes the grid as channel
// quadruples, float [K / 4][Mz][My][Mxp][4] (element (c, z, y, x) at
// (((c / 4) Mz + z) My + y) Mxp + x) * 4 + c % 4), so one 16-byte word holds
// four channels of a grid point (a CTA transforms the four channels of its
// rows and writes whole quadruples).
cudaError_t launch_irfft_x(const void* spec, int Mx, int My, int Mz, int K, int nkx, const void* tw, float* grid,
                           cudaStream_t s, bool interleave4 = false);

// Lines of the nkx planes that can hold band modes after the z pass: for kx
// < nkx and column position pz (kz = (pz >> 5) + (Mz / 32) brev5(pz & 31),
// signed mz), some signed y mode my gives |B (kx, my, mz)| < k_c, B = 2 pi
// H^-1 (row-major bmat; for a box: (2 pi kx / L_x)^2 + (2 pi mz / L_z)^2 <
// k_c^2).  mask[kx * Mz + pz] = 1 for those, lines lists them as kx << 16 | pz.
void xfft_band_lines(int nkx, int My, int Mz, const double bmat[9], double k_c, std::vector<unsigned char>& mask,
                     std::vector<int>& lines);

// z pass of the fully own transform over the nkx planes of spec ([K][.][Mz][My],
// channel stride chan complex): forward leaves column position l + 32 k1 =
// kz = k1 + (Mz / 32) brev5(l) and stores only the masked lines; the inverse
// takes that order back, reading unmasked lines as zero.  tw: the Mz table.
cudaError_t launch_fft_z(bool inverse, void* spec, int Mz, int My, int K, int nkx, int64_t chan, const void* tw,
                         const unsigned char* lmask, cudaStream_t s);

// Forward y transform, multiplier (and energy / virial partials), inverse y
// transform of the listed lines (xfft_band_lines); grid (blocks, K); part and
// vpart as k_multiply_planes ([c][blocks], [c][blocks][3]).  tw: the My table.
struct MultArgs {
  void* spec;
  MultParams mp;
  const int* lines;
  int nlines;
  int nkx, K, blocks;
  int64_t chan;
  const int* pch;
  const double* scale;
  const double* bmat;
  const void* coef;
  const void* iw2;
  int iw2_stride;
  const void* tw;
  double* part;
  int want_energy;
  double* vpart;
};
cudaError_t launch_mult_y(const MultArgs& a, cudaStream_t s);

}  // namespace pswf
