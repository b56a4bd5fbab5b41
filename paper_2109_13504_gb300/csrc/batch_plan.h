// batch_plan.h -- the plan builder behind mego_batch_plan, with a choice of
// host staging for the plan's copy to the device.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/megopolis.h"

namespace mego {

// Validates the filters, writes the plan's host part and queues its copy to
// d_plan on `stream`, then fills *out like mego_batch_plan.  The host part is
// built either in *pageable (resized here; cudaMemcpyAsync has read a
// pageable source by the time it returns) or, when pageable is null, in
// `staging`: page-locked memory of at least the plan's host size that the
// caller keeps unchanged until the copy has run on the stream (the copy is
// then truly asynchronous and does not wait for earlier work on the stream).
// smem_max_n: filters of at most this many weights take the shared-memory
// phase (0: none).  replan: *out already describes a plan in d_plan built
// from the same filters; only the shared-memory split changes, and the
// per-filter B, status and q already in d_plan are kept, as is out's shape.
mego_status batch_plan_staged(const mego_filter* h_filters, int32_t count, int variant,
                              int layout, uint64_t seed, int32_t smem_max_n, void* d_plan,
                              size_t plan_bytes, std::vector<unsigned char>* pageable,
                              void* staging, size_t staging_bytes, mego_batch* out,
                              void* stream, bool replan);

// Largest shared-memory threshold (weights per filter) the device allows.
int32_t smem_limit_n();

}  // namespace mego
