// bound.cuh -- host-side launchers for the reduction / bound kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mego {

constexpr int kReduceThreads = 256;
constexpr int kMaxParts = 1024;
constexpr int32_t kStatusWeights = 5;  // MEGO_EWEIGHTS

struct Partial {
  float mx;
  int32_t bad;
  double sum;
};
static_assert(sizeof(Partial) == 16, "partial layout");

int reduce_grid(uint32_t n);
void count_launches(uint64_t k);
cudaError_t launch_partials(const float* src, uint32_t n, bool likelihood, float y,
                            float* w_out, Partial* parts, int grid, cudaStream_t st);
cudaError_t launch_finalize(const Partial* parts, int nparts, uint32_t n, double eps,
                            int32_t b_max, int32_t* d_B, int32_t* d_status, double* d_q,
                            cudaStream_t st);
cudaError_t launch_probe_read(const void* buf, size_t bytes, int reps, float* sink,
                              int grid, cudaStream_t st);

}  // namespace mego
