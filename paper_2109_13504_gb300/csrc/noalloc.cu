// noalloc.cu -- mego_compute_B_noalloc: the iteration bound without a
// caller workspace, for callers that cannot allocate device memory.
//
// The per-CTA partial results of the reduction live in a fixed array in
// this file (every GPU that loads the library holds it until the process
// exits).  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// while that device is current, and later calls reuse it (for the life of
// the process: a device reset while the library is loaded is unsupported).
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/megopolis.h"
#include "bound.cuh"

namespace {

// Capacity of the fixed scratch: one per-CTA partial (16 bytes) for every
// CTA the reduction grid can have, 16 KiB in all.  The grid is then the one
// mego_compute_B uses, so both add the same partials in the same order.
constexpr int kNoAllocParts = mego::kMaxParts;
static_assert(kNoAllocParts * sizeof(mego::Partial) == 16384, "16 KiB of partials");

static __device__ __align__(256) mego::Partial g_noalloc_parts[kNoAllocParts];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
mego::Partial* g_parts_addr[kMaxDevices] = {};

// Device address of the scratch for the current device, looked up once.
mego_status scratch_for_current_device(mego::Partial** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MEGO_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return MEGO_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_parts_addr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_parts);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return MEGO_ECUDA;
    }
    g_parts_addr[dev] = static_cast<mego::Partial*>(p);
  }
  *out = g_parts_addr[dev];
  return MEGO_OK;
}

}  // namespace

extern "C" mego_status mego_compute_B_noalloc(const float* d_w, int32_t n, double eps,
                                              int32_t b_max, int32_t* d_B, int32_t* d_status,
                                              double* d_q, void* stream) {
  if (!d_w || !d_B || !d_status) return MEGO_EINVAL;
  if (n < 1 || n > MEGO_N_MAX) return MEGO_EINVAL;
  if (!(eps > 0.0 && eps <= 1.0)) return MEGO_EINVAL;
  if (b_max < 1 || b_max > MEGO_B_MAX) return MEGO_EINVAL;
  const uint32_t un = static_cast<uint32_t>(n);
  const int grid = mego::reduce_grid(un);  // at most mego::kMaxParts CTAs
  if (grid > kNoAllocParts) return MEGO_EINVAL;
  mego::Partial* parts = nullptr;
  const mego_status s = scratch_for_current_device(&parts);
  if (s != MEGO_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Every partial the finalize step reads is written by the reduction first,
  // so nothing in the scratch needs clearing between calls.
  if (mego::launch_partials(d_w, un, false, 0.0f, nullptr, parts, grid, st) != cudaSuccess)
    return MEGO_ECUDA;
  if (mego::launch_finalize(parts, grid, un, eps, b_max, d_B, d_status, d_q, st) !=
      cudaSuccess)
    return MEGO_ECUDA;
  mego::count_launches(2);
  return MEGO_OK;
}
