// resample_dispatch.cuh -- instantiates resample_kernel for one variant over
// (particles per thread, weight path, gather layout) and launches it.
// Included once per variant translation unit, with MEGO_VARIANT defined.
#pragma once

#include <mutex>

#include "resample_kernels.cuh"

namespace mego {
namespace {

// Fault word of this variant's kernels (set when the shared-memory staging
// gives up waiting for its bulk copy); read and cleared by mego_device_fault.
__device__ int32_t g_fault_word;

int32_t* fault_word_address() {
  static std::mutex mu;
  static int32_t* addr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_fault_word) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    addr[dev] = static_cast<int32_t*>(p);
  }
  return addr[dev];
}

template <int V, int P, bool S, int G>
cudaError_t launch_one(const LaunchShape& s, const ResampleArgs& a, cudaStream_t st) {
  auto* k = &resample_kernel<V, P, S, G>;
  if (S) {
    const cudaError_t e = enable_large_smem(reinterpret_cast<const void*>(k));
    if (e != cudaSuccess) return e;
  }
  return launch_after(k, dim3(static_cast<unsigned>(s.grid)), dim3(static_cast<unsigned>(s.threads)),
                      s.smem_bytes, st, a);
}

template <int V, int P, bool S, int G>
const void* ptr_one() {
  return reinterpret_cast<const void*>(&resample_kernel<V, P, S, G>);
}

template <int V, bool S, int G>
cudaError_t by_ppt(const LaunchShape& s, const ResampleArgs& a, cudaStream_t st) {
  switch (s.ppt) {
    case 1: return launch_one<V, 1, S, G>(s, a, st);
    case 2: return launch_one<V, 2, S, G>(s, a, st);
    case 4: return launch_one<V, 4, S, G>(s, a, st);
    case 6:
      if constexpr (V == kMegopolis) return launch_one<V, 6, S, G>(s, a, st);
      return cudaErrorInvalidValue;
    case 8: return launch_one<V, 8, S, G>(s, a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int V, bool S, int G>
const void* ptr_by_ppt(int ppt) {
  switch (ppt) {
    case 1: return ptr_one<V, 1, S, G>();
    case 2: return ptr_one<V, 2, S, G>();
    case 4: return ptr_one<V, 4, S, G>();
    case 6:
      if constexpr (V == kMegopolis) return ptr_one<V, 6, S, G>();
      return nullptr;
    case 8: return ptr_one<V, 8, S, G>();
    default: return nullptr;
  }
}

template <int V, bool S>
cudaError_t by_gather(const LaunchShape& s, int gather, const ResampleArgs& a, cudaStream_t st) {
  switch (gather) {
    case kGatherNone: return by_ppt<V, S, kGatherNone>(s, a, st);
    case kGatherSoa: return by_ppt<V, S, kGatherSoa>(s, a, st);
    case kGatherAos4: return by_ppt<V, S, kGatherAos4>(s, a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int V, bool S>
const void* ptr_by_gather(int ppt, int gather) {
  switch (gather) {
    case kGatherNone: return ptr_by_ppt<V, S, kGatherNone>(ppt);
    case kGatherSoa: return ptr_by_ppt<V, S, kGatherSoa>(ppt);
    case kGatherAos4: return ptr_by_ppt<V, S, kGatherAos4>(ppt);
    default: return nullptr;
  }
}

}  // namespace

template <>
cudaError_t launch_resample<MEGO_VARIANT>(const LaunchShape& s, int gather,
                                          const ResampleArgs& a, cudaStream_t st) {
#ifdef MEGO_BOUNDS_CHECK
  const bool report = true;  // index checks report on every path
#else
  const bool report = s.smem;
#endif
  if (!report) return by_gather<MEGO_VARIANT, false>(s, gather, a, st);
  ResampleArgs b = a;
  b.p.fault = fault_word_address();
  return s.smem ? by_gather<MEGO_VARIANT, true>(s, gather, b, st)
                : by_gather<MEGO_VARIANT, false>(s, gather, b, st);
}

template <>
int32_t* resample_fault_word<MEGO_VARIANT>() {
  return fault_word_address();
}

template <>
const void* resample_kernel_ptr<MEGO_VARIANT>(int ppt, bool smem, int gather) {
  return smem ? ptr_by_gather<MEGO_VARIANT, true>(ppt, gather)
              : ptr_by_gather<MEGO_VARIANT, false>(ppt, gather);
}

}  // namespace mego
