// Library-internal entry points on a batch plan, used by the request server
// (server.cu).  Not part of the public C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pswf_lr.h"

namespace pswf {

// Host side only: fills the plan's pinned table mirror for structures
// 0..b-1 (allocating it on first use).  The caller guarantees that no upload
// from the mirror is in flight.
int plan_fill_tables(pswf_plan p, int b, const double* boxes, const int* ps, const int64_t* offsets);
// Slots the next launch processes (a planned size >= b, set by
// plan_fill_tables); captured sequences are per size.
int plan_run_size(pswf_plan p);
// Every size plan_run_size can return, ascending.
const int* plan_run_sizes(pswf_plan p, int* count);
// Copies the mirror to the device on the plan's stream (plain async copy).
int plan_upload_tables(pswf_plan p);
// The kernels of set_points / execute on the plan's stream; for a batch plan
// their launch shapes depend only on the plan's capacity, so the sequence can
// be captured into a CUDA graph once and replayed for any batch.
int plan_run_set_points(pswf_plan p, int64_t n, const void* pos, int pos_dtype, const void* q);
int plan_run_execute(pswf_plan p, double* energy, void* phi, void* forces);
cudaStream_t plan_stream(pswf_plan p);
int plan_precision(pswf_plan p);
const char* plan_error(pswf_plan p);

}  // namespace pswf
