// bound.cu -- weight reduction and the iteration bound (Eq. 3), optionally
// fused with the likelihood weight (Eq. 12), plus a read-bandwidth probe.
//
// Deterministic: a fixed grid writes one partial (max, sum, bad flag) per CTA
// (float-float inside the CTA, stored as a double); a single warp then folds
// the partials in a fixed order.  The result depends only on n and the
// weight bits.
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "bound.cuh"
#include "device_common.cuh"

namespace mego {

namespace {

struct Acc {
  float mx;
  int bad;
  FloatFloat sum;
};

// Per-thread accumulator: max, validity and a compensated (Neumaier) float
// sum s + c.  No FP64 operation is used per element or in the tree (FP64 is
// slow on this part): threads combine float-float values and each CTA
// converts its partial to double once.  The compensated sum of a thread's
// weights is exact to about 2 ulp of float squared.
struct ThreadAcc {
  float mx = 0.0f;
  int bad = 0;
  float s = 0.0f;
  float c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    bad |= (!(v >= 0.0f) || isinf(v)) ? 1 : 0;
    mx = fmaxf(mx, v);
    const float t = __fadd_rn(s, v);
    c = __fadd_rn(c, fabsf(s) >= fabsf(v) ? __fadd_rn(__fsub_rn(s, t), v)
                                            : __fadd_rn(__fsub_rn(v, t), s));
    s = t;
  }
  __device__ __forceinline__ Acc to_acc() const { return Acc{mx, bad, ff_from_pair(s, c)}; }
};

__device__ __forceinline__ void acc_merge(Acc& a, const Acc& b) {
  a.bad |= b.bad;
  a.mx = fmaxf(a.mx, b.mx);
  a.sum = ff_add(a.sum, b.sum);
}

__device__ __forceinline__ Acc acc_shfl_down(const Acc& a, int off) {
  Acc o;
  o.mx = __shfl_down_sync(0xFFFFFFFFu, a.mx, off);
  o.bad = __shfl_down_sync(0xFFFFFFFFu, a.bad, off);
  o.sum.hi = __shfl_down_sync(0xFFFFFFFFu, a.sum.hi, off);
  o.sum.lo = __shfl_down_sync(0xFFFFFFFFu, a.sum.lo, off);
  return o;
}

// Warp then CTA reduction in a fixed tree order; result valid in thread 0.
__device__ __forceinline__ Acc block_reduce(Acc a) {
  __shared__ Acc s[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc_merge(a, acc_shfl_down(a, off));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s[warp] = a;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    a = lane < nw ? s[lane] : Acc{0.0f, 0, FloatFloat{0.0f, 0.0f}};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc_merge(a, acc_shfl_down(a, off));
  }
  return a;
}

// One partial per CTA.  LIKELIHOOD: src is state row 0 and the weight
// w = exp(-(x - y)^2 / 2) is written to w_out before it is reduced.
template <bool LIKELIHOOD>
__device__ __forceinline__ float4 weight4(float4 v, float y, float4* w_out, uint32_t t) {
  if constexpr (LIKELIHOOD) {
    float d;
    d = v.x - y; v.x = expf(-0.5f * d * d);
    d = v.y - y; v.y = expf(-0.5f * d * d);
    d = v.z - y; v.z = expf(-0.5f * d * d);
    d = v.w - y; v.w = expf(-0.5f * d * d);
    w_out[t] = v;
  }
  return v;
}

template <bool LIKELIHOOD>
__global__ void __launch_bounds__(kReduceThreads)
partials_kernel(const float* __restrict__ src, uint32_t n, float y,
                float* __restrict__ w_out, Partial* __restrict__ parts) {
  grid_launch_dependents();  // the finalize may be scheduled now; it waits for us
  ThreadAcc a;
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0u) &&
                   (!LIKELIHOOD || ((reinterpret_cast<uintptr_t>(w_out) & 15u) == 0u));
  uint32_t tail = 0u;
  if (vec) {
    const uint32_t n4 = n / 4u;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* w4 = reinterpret_cast<float4*>(w_out);
    // Four independent 16-byte loads in flight per thread before any
    // accumulation (one DRAM latency per four vectors); the values are still
    // added in index order t0, t0 + stride, t0 + 2 stride, ...
    uint32_t t = t0;
    for (; t + 3u * stride < n4; t += 4u * stride) {
      float4 v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = __ldg(s4 + t + k * stride);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 x = weight4<LIKELIHOOD>(v[k], y, w4, t + k * stride);
        a.add(x.x);
        a.add(x.y);
        a.add(x.z);
        a.add(x.w);
      }
    }
    for (; t < n4; t += stride) {
      const float4 x = weight4<LIKELIHOOD>(__ldg(s4 + t), y, w4, t);
      a.add(x.x);
      a.add(x.y);
      a.add(x.z);
      a.add(x.w);
    }
    tail = n4 * 4u;
  }
  for (uint32_t i = tail + t0; i < n; i += stride) {
    float v = __ldg(src + i);
    if constexpr (LIKELIHOOD) {
      const float d = v - y;
      v = expf(-0.5f * d * d);
      w_out[i] = v;
    }
    a.add(v);
  }
  const Acc r = block_reduce(a.to_acc());
  if (threadIdx.x == 0) parts[blockIdx.x] = Partial{r.mx, r.bad, ff_to_double(r.sum)};
}

__global__ void __launch_bounds__(32)
finalize_kernel(const Partial* __restrict__ parts, int nparts, uint32_t n, double log_eps,
                int32_t b_max, int32_t* __restrict__ d_B, int32_t* __restrict__ d_status,
                double* __restrict__ d_q) {
  // One warp: each lane folds its strided partials in index order, then a
  // fixed shuffle tree combines the lanes.
  // Loads go out eight at a time, ahead of the (order-dependent) merges.
  grid_launch_dependents();  // a resample launched after us may be scheduled
  grid_dependency_wait();    // the partials are complete and visible
  // The partials are few: the fold stays in double.
  float mx = 0.0f;
  int bad = 0;
  double sum = 0.0;
  for (int t0 = threadIdx.x; t0 < nparts; t0 += 8 * 32) {
    Partial p[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (t0 + 32 * k < nparts) p[k] = parts[t0 + 32 * k];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (t0 + 32 * k < nparts) {
        mx = fmaxf(mx, p[k].mx);
        bad |= p[k].bad;
        sum += p[k].sum;
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mx = fmaxf(mx, __shfl_down_sync(0xFFFFFFFFu, mx, off));
    bad |= __shfl_down_sync(0xFFFFFFFFu, bad, off);
    sum += __shfl_down_sync(0xFFFFFFFFu, sum, off);
  }
  const Acc a{mx, bad, FloatFloat{0.0f, 0.0f}};
  if (threadIdx.x != 0) return;
  int32_t B = -1, status = kStatusWeights;
  double q = __longlong_as_double(0x7FF8000000000000LL);  // NaN
  // A sum that overflowed binary32 inside a chunk (finite weights of order
  // FLT_MAX / 4096 or more) cannot give B: reported like invalid weights.
  if (!a.bad && a.mx > 0.0f && isfinite(sum)) {
    // r = E(w) / max(w) with one division; log(eps) comes from the host.
    const double r = sum / (static_cast<double>(n) * static_cast<double>(a.mx));
    q = (r >= 1.0) ? 0.0 : log_eps / log1p(-r);
    double c = ceil(q);
    if (c < 0.0) c = 0.0;
    if (c <= static_cast<double>(b_max)) {
      B = static_cast<int32_t>(c);
      status = 0;
    }
  }
  *d_B = B;
  *d_status = status;
  if (d_q) *d_q = q;
}

// Read `n16` 16-byte words `reps` times; CTAs stride through the buffer
// so each pass is one coalesced sweep.
__global__ void __launch_bounds__(512)
probe_read_kernel(const float4* __restrict__ buf, size_t n16, int reps,
                  float* __restrict__ sink) {
  float acc = 0.0f;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (int r = 0; r < reps; ++r) {
    for (size_t t = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < n16;
         t += stride) {
      const float4 v = __ldcg(buf + t);
      acc += (v.x + v.y) + (v.z + v.w);
    }
  }
  // Practically never true; keeps the loads alive.
  if (acc == 1.2345678e-30f) sink[blockIdx.x] = acc;
}

}  // namespace

int reduce_grid(uint32_t n) {
  const uint32_t per_cta = kReduceThreads * 16u;
  uint32_t g = (n + per_cta - 1u) / per_cta;
  if (g < 1u) g = 1u;
  if (g > static_cast<uint32_t>(kMaxParts)) g = kMaxParts;
  return static_cast<int>(g);
}

cudaError_t launch_partials(const float* src, uint32_t n, bool likelihood, float y,
                            float* w_out, Partial* parts, int grid, cudaStream_t st) {
  if (likelihood) {
    partials_kernel<true><<<grid, kReduceThreads, 0, st>>>(src, n, y, w_out, parts);
  } else {
    partials_kernel<false><<<grid, kReduceThreads, 0, st>>>(src, n, y, w_out, parts);
  }
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Partial* parts, int nparts, uint32_t n, double eps,
                            int32_t b_max, int32_t* d_B, int32_t* d_status, double* d_q,
                            cudaStream_t st) {
  return launch_after(finalize_kernel, dim3(1), dim3(32), 0, st,
                      static_cast<const Partial*>(parts), nparts, n, std::log(eps), b_max, d_B,
                      d_status, d_q);
}

cudaError_t launch_probe_read(const void* buf, size_t bytes, int reps, float* sink,
                              int grid, cudaStream_t st) {
  probe_read_kernel<<<grid, 512, 0, st>>>(reinterpret_cast<const float4*>(buf), bytes / 16u,
                                          reps, sink);
  return cudaGetLastError();
}

}  // namespace mego
