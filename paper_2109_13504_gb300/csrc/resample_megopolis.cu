// resample_megopolis.cu -- kernel instances for one resampling variant, and
// the Megopolis-only TMA window path.
#include "resample_kernels.cuh"
#define MEGO_VARIANT ::mego::kMegopolis
#include "resample_dispatch.cuh"

namespace mego {
namespace {

template <int P, int G>
cudaError_t launch_tma_one(const LaunchShape& s, const ResampleArgs& a, cudaStream_t st) {
  return launch_after(&resample_tma_kernel<P, G>, dim3(static_cast<unsigned>(s.grid)),
                      dim3(static_cast<unsigned>(s.threads)), 0, st, a);
}

template <int P>
cudaError_t launch_tma_p(const LaunchShape& s, int gather, const ResampleArgs& a,
                         cudaStream_t st) {
  switch (gather) {
    case kGatherNone: return launch_tma_one<P, kGatherNone>(s, a, st);
    case kGatherSoa: return launch_tma_one<P, kGatherSoa>(s, a, st);
    case kGatherAos4: return launch_tma_one<P, kGatherAos4>(s, a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int P>
const void* tma_ptr_p(int gather) {
  switch (gather) {
    case kGatherNone: return reinterpret_cast<const void*>(&resample_tma_kernel<P, kGatherNone>);
    case kGatherSoa: return reinterpret_cast<const void*>(&resample_tma_kernel<P, kGatherSoa>);
    case kGatherAos4: return reinterpret_cast<const void*>(&resample_tma_kernel<P, kGatherAos4>);
    default: return nullptr;
  }
}

}  // namespace

cudaError_t launch_resample_tma(const LaunchShape& s, int gather, const ResampleArgs& a,
                                cudaStream_t st) {
  ResampleArgs b = a;
  b.p.fault = resample_fault_word<kMegopolis>();
  switch (s.ppt) {
    case 4: return launch_tma_p<4>(s, gather, b, st);
    case 6: return launch_tma_p<6>(s, gather, b, st);
    default: return cudaErrorInvalidValue;
  }
}

const void* resample_tma_kernel_ptr(int ppt, int gather) {
  switch (ppt) {
    case 4: return tma_ptr_p<4>(gather);
    case 6: return tma_ptr_p<6>(gather);
    default: return nullptr;
  }
}

}  // namespace mego
