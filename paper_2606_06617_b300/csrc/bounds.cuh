// Non-trapping bounds checks.  Compiled with -DPSWF_BOUNDS_CHECK (the checked
// build of the library), an index outside its buffer records a code in this
// translation unit's device status word and the access is skipped, so a
// kernel with a bad index finishes and the status reaches the host
// (pswf_sync: PSWF_EBOUNDS) instead of faulting the GPU.  In the normal build
// every check is the constant true and compiles away.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pswf {

#ifdef PSWF_BOUNDS_CHECK
static __device__ int g_bounds_word;   // first failed check's code (0: none)

__device__ __forceinline__ bool in_bounds(int64_t i, int64_t n, int code) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_bounds_word, 0, code);
  return false;
}

// Reads and clears this translation unit's status word (host).
static inline int take_bounds_word() {
  int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_word, sizeof(int)) != cudaSuccess) return 0;
  if (v) cudaMemcpyToSymbol(g_bounds_word, &zero, sizeof(int));
  return v;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(int64_t, int64_t, int) { return true; }
static inline int take_bounds_word() { return 0; }
#endif

// Codes of the checks (which access failed).
enum BoundsCode : int {
  kBoundsGatherStage = 1,     // gather: staging write into the tile region
  kBoundsGatherGrid = 2,      // gather: grid read
  kBoundsGatherRegion = 3,    // gather: an atom's stencil in the tile region
  kBoundsGatherOut = 4,       // gather: potential or force write
  kBoundsSpreadRegion = 5,    // spread: an atom's stencil in the tile region
  kBoundsSpreadFlush = 6,     // spread: region read or grid write of the flush
  kBoundsScatter = 7,         // set_points: sorted position out of range
  kBoundsTile = 8,            // a tile's atom range outside the sorted arrays
  kBoundsRsScatter = 9,       // real space: sorted position out of range
  kBoundsRsPair = 10,         // real space: a queued neighbour or pair atom outside the sorted arrays
  kBoundsRsFinish = 11,       // real space: original index out of range
};

}  // namespace pswf
