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

namespace pswf {

// True when the row length has a kernel here (Mx = 32 N1, 2 <= N1 <= 16).
bool xfft_supported(int Mx);

// Twiddle table of a row length (host, float pairs): entries [k1 * 32 + l] =
// e^{-2 pi i l k1 / Mx} for k1 < N1 (forward); for the lane stages s < 5
// (distance d = 16 >> s) [Mx + s * 32 + l] = 1 on lanes with l & d = 0 and
// -e^{-2 pi i (l mod d) / 2d} on the others; then [Mx + 160 + n1 * 32 + l] =
// e^{-2 pi i n1 brev5(l) / Mx} for n1 < N1 (inverse, conjugated in use);
// xfft_table_size() pairs.
int xfft_table_size(int Mx);
void xfft_twiddles(int Mx, std::vector<float>& out);

// grid: K channels of real rows (row stride Mxp = 2 (Mx / 2 + 1) floats,
// channel stride Mz My Mxp); spec: complex (float2) [K][Mx / 2 + 1][Mz][My];
// tw: the device copy of the twiddle table.  One launch each.
cudaError_t launch_rfft_x(const float* grid, int Mx, int My, int Mz, int K, int nkx, const void* tw, void* spec,
                          cudaStream_t s);
cudaError_t launch_irfft_x(const void* spec, int Mx, int My, int Mz, int K, int nkx, const void* tw, float* grid,
                           cudaStream_t s);

}  // namespace pswf
