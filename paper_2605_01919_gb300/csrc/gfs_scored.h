// Launchers of the scored value (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gfs_kernels.h"

namespace gfs {

// Rewrite a plain query's outputs in place with the scored value (a.fl_out
// and a.arg_out read and rewritten; a.s_out / a.s64_out rewritten where
// non-null); csr_ids: the survivor ids sorted ascending, csr_off: n + 1
// offsets of each sphere's ids in that list; status: bits of the phases in
// which a point ran out of its work budget (ORed in).
cudaError_t launch_query_scored(const QueryArgs& a, int box_cull, const uint32_t* csr_ids, const int64_t* csr_off,
                                unsigned* status, cudaStream_t st);
// csr_off[i] for i <= n from the sorted ids (nid of them)
cudaError_t launch_csr_offsets(const uint32_t* ids, int64_t nid, int64_t n, int KS, int64_t* off, cudaStream_t st);

// kernels this file has launched in this process
unsigned long long scored_launch_count();

}  // namespace gfs
