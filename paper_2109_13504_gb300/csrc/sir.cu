// sir.cu -- the stages around the resampler in the modified SIR filter
// (Algorithm 6, model of Eqs. 22-23): predict + update in one pass, and the
// estimate (mean of the resampled particles) as a deterministic reduction.
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/megopolis.h"

namespace mego {
void count_launches(uint64_t k);
}

namespace {

constexpr int kThreads = 256;
constexpr int kMaxMeanParts = 1024;

// Per particle: x' = x/2 + 25 x / (1 + x^2) + drift + v  (Eq. 22, drift =
// 8 cos(1.2 t) precomputed by the caller, v the process noise), then the
// likelihood of the measurement z = x'^2 / 20 + n with n ~ N(0, 1) (Eq. 23):
// w = exp(-(z - x'^2/20)^2 / 2).  Every operation is one binary32 operation
// rounded to nearest in this order (no contraction), so x' is reproducible.
__global__ void __launch_bounds__(kThreads)
predict_update_kernel(const float* __restrict__ x, const float* __restrict__ v, uint32_t n,
                      float drift, float z, float* __restrict__ x_pred, float* __restrict__ w) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float xi = __ldg(x + i);
    const float den = __fadd_rn(1.0f, __fmul_rn(xi, xi));
    const float frac = __fdiv_rn(__fmul_rn(25.0f, xi), den);
    float xp = __fadd_rn(__fmul_rn(0.5f, xi), frac);
    xp = __fadd_rn(xp, drift);
    xp = __fadd_rn(xp, __ldg(v + i));
    const float d = __fsub_rn(z, __fdiv_rn(__fmul_rn(xp, xp), 20.0f));
    const float a = __fmul_rn(0.5f, __fmul_rn(d, d));
    x_pred[i] = xp;
    w[i] = expf(-a);
  }
}

// Per-CTA partial sums in double, then one warp folds them in index order.
__global__ void __launch_bounds__(kThreads)
mean_partials_kernel(const float* __restrict__ x, uint32_t n, double* __restrict__ parts) {
  double s = 0.0;
  const uint32_t stride = gridDim.x * blockDim.x;
  // Compensated float accumulation per thread, in index order; one
  // conversion to double.  Sixteen loads are issued before they are summed,
  // so a pass costs one memory latency per sixteen values.
  constexpr int kPer = 16;
  float hi = 0.0f, lo = 0.0f;
  for (uint32_t base = blockIdx.x * blockDim.x + threadIdx.x; base < n; base += kPer * stride) {
    float v[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t i = base + static_cast<uint32_t>(k) * stride;
      v[k] = i < n ? __ldg(x + i) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      if (base + static_cast<uint32_t>(k) * stride >= n) break;
      const float t = __fadd_rn(hi, v[k]);
      lo = __fadd_rn(lo, fabsf(hi) >= fabsf(v[k]) ? __fadd_rn(__fsub_rn(hi, t), v[k])
                                                  : __fadd_rn(__fsub_rn(v[k], t), hi));
      hi = t;
    }
  }
  s = static_cast<double>(hi) + static_cast<double>(lo);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, off);
  __shared__ double sw[kThreads / 32];
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sw[k];
    parts[blockIdx.x] = t;
  }
}

__global__ void mean_finalize_kernel(const double* __restrict__ parts, int nparts, uint32_t n,
                                     double* __restrict__ out) {
  // Each lane folds its strided partials in index order, eight loads ahead.
  double s = 0.0;
  for (int k0 = threadIdx.x; k0 < nparts; k0 += 8 * 32) {
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = k0 + 32 * j < nparts ? parts[k0 + 32 * j] : 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (k0 + 32 * j < nparts) s += v[j];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, off);
  if (threadIdx.x == 0) *out = s / static_cast<double>(n);
}

int grid_for(uint32_t n, int cap) {
  uint32_t g = (n + kThreads * 16u - 1u) / (kThreads * 16u);
  if (g < 1u) g = 1u;
  if (g > static_cast<uint32_t>(cap)) g = static_cast<uint32_t>(cap);
  return static_cast<int>(g);
}

}  // namespace

extern "C" {

mego_status mego_sir_predict_update(const float* d_x, const float* d_v, int32_t n, float drift,
                                    float z, float* d_x_pred, float* d_w, void* stream) {
  if (!d_x || !d_v || !d_x_pred || !d_w || n < 1 || n > MEGO_N_MAX) return MEGO_EINVAL;
  // One particle per thread: every load of the launch is in flight at once
  // (a grid-stride loop would wait one memory latency per element).
  const int grid = static_cast<int>((static_cast<uint32_t>(n) + kThreads - 1u) / kThreads);
  predict_update_kernel<<<grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      d_x, d_v, static_cast<uint32_t>(n), drift, z, d_x_pred, d_w);
  if (cudaGetLastError() != cudaSuccess) return MEGO_ECUDA;
  mego::count_launches(1);
  return MEGO_OK;
}

size_t mego_mean_workspace_bytes(void) { return sizeof(double) * kMaxMeanParts + 256u; }

mego_status mego_mean(const float* d_x, int32_t n, double* d_out, void* d_ws, size_t ws_bytes,
                      void* stream) {
  if (!d_x || !d_out || !d_ws || n < 1 || n > MEGO_N_MAX) return MEGO_EINVAL;
  if (ws_bytes < mego_mean_workspace_bytes()) return MEGO_ENOMEM;
  if (reinterpret_cast<uintptr_t>(d_ws) & 7u) return MEGO_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = grid_for(static_cast<uint32_t>(n), kMaxMeanParts);
  double* parts = static_cast<double*>(d_ws);
  mean_partials_kernel<<<grid, kThreads, 0, st>>>(d_x, static_cast<uint32_t>(n), parts);
  if (cudaGetLastError() != cudaSuccess) return MEGO_ECUDA;
  mean_finalize_kernel<<<1, 32, 0, st>>>(parts, grid, static_cast<uint32_t>(n), d_out);
  if (cudaGetLastError() != cudaSuccess) return MEGO_ECUDA;
  mego::count_launches(2);
  return MEGO_OK;
}

}  // extern "C"
