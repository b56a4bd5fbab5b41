// resample_kernels.cuh -- Megopolis, Metropolis and Metropolis-C1/C2 chains
// with the fused ancestor gather, for sm_103a.
//
// Work decomposition.  Particles are grouped in 32-particle segments (the
// paper's warp partition, Section 4).  The grid's warps split the ceil(n/32)
// segments into equal contiguous ranges; a warp walks its range P segments
// at a time, one particle of each segment per lane, so a thread carries P
// independent chains (instruction-level parallelism).  B is read once per
// kernel, from the host argument or from device memory.
//
// Weight source.  SMEM: the whole weight vector is staged once per CTA in
// shared memory by a bulk async copy (cp.async.bulk + mbarrier); GLOBAL:
// weights are read through L1/L2 with 32-bit loads, one aligned 128-byte
// partition per warp and iteration for Megopolis.
#pragma once

#include "device_common.cuh"

namespace mego {

enum Variant : int { kMegopolis = 0, kMetropolis = 1, kC1 = 2, kC2 = 3 };
enum Gather : int { kGatherNone = 0, kGatherSoa = 1, kGatherAos4 = 2 };

struct ResampleArgs {
  const float* w;
  const int32_t* B_dev;  // non-null: read B here (device-side bound)
  int32_t* anc;          // [n] ancestors, may be null
  const float* x_in;     // gather source, may be null
  float* x_out;
  int32_t* fault;        // device fault word, may be null
  int64_t ld;
  uint32_t n;
  uint32_t nseg;         // ceil(n / 32)
  int32_t B;
  uint32_t k0, k1, sid;
  int32_t dim;
  uint32_t nw;           // C1/C2: weights per partition
  uint32_t npart;        // C1/C2: number of partitions
};

extern __shared__ float4 g_dyn_smem[];

constexpr uint32_t kStageChunk = 32768u;
constexpr uint32_t kMaxPolls = 1u << 21;

template <bool SMEM>
__device__ __forceinline__ float ldw(const float* __restrict__ w, uint32_t j) {
  if constexpr (SMEM) {
    return reinterpret_cast<const float*>(g_dyn_smem)[j];
  } else {
    return __ldg(w + j);
  }
}

// Stage w[0, n) into dynamic shared memory.  Returns false (uniformly for the
// CTA) if the bulk copy did not complete within the poll budget.
__device__ __forceinline__ bool stage_weights(const ResampleArgs& a) {
  __shared__ __align__(8) uint64_t bar;
  float* s_w = reinterpret_cast<float*>(g_dyn_smem);
  const uint32_t bytes = a.n * 4u;
  const bool bulk = ((reinterpret_cast<uintptr_t>(a.w) & 15u) == 0u) &&
                    ((bytes & 15u) == 0u);
  if (!bulk) {
    for (uint32_t t = threadIdx.x; t < a.n; t += blockDim.x) s_w[t] = __ldg(a.w + t);
    __syncthreads();
    return true;
  }
  if (threadIdx.x == 0) mbar_init(&bar, 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, bytes);
    for (uint32_t off = 0; off < bytes; off += kStageChunk) {
      const uint32_t len = (bytes - off) < kStageChunk ? (bytes - off) : kStageChunk;
      bulk_g2s(reinterpret_cast<char*>(s_w) + off,
               reinterpret_cast<const char*>(a.w) + off, len, &bar);
    }
  }
  const bool done = mbar_wait_bounded(&bar, 0u, kMaxPolls);
  if (__syncthreads_and(done ? 1 : 0)) return true;
  if (threadIdx.x == 0) {
    if (a.fault) atomicExch(a.fault, kFaultStageTimeout);
    mbar_wait_bounded(&bar, 0u, kMaxPolls);  // let copies in flight land
  }
  __syncthreads();
  return false;
}

// Ancestor output and gather for the P particles of one batch.
template <int P, int GATHER>
__device__ __forceinline__ void finish_batch(const ResampleArgs& a, uint32_t ibase,
                                             const uint32_t (&k)[P],
                                             const bool (&live)[P]) {
#pragma unroll
  for (int p = 0; p < P; ++p)
    if (live[p] && a.anc) a.anc[ibase + 32u * p] = static_cast<int32_t>(k[p]);
  if constexpr (GATHER == kGatherSoa) {
    for (int d = 0; d < a.dim; ++d) {
      const float* src = a.x_in + static_cast<int64_t>(d) * a.ld;
      float* dst = a.x_out + static_cast<int64_t>(d) * a.ld;
      float v[P];
#pragma unroll
      for (int p = 0; p < P; ++p) v[p] = live[p] ? __ldg(src + k[p]) : 0.0f;
#pragma unroll
      for (int p = 0; p < P; ++p)
        if (live[p]) dst[ibase + 32u * p] = v[p];
    }
  } else if constexpr (GATHER == kGatherAos4) {
    const float4* src = reinterpret_cast<const float4*>(a.x_in);
    float4* dst = reinterpret_cast<float4*>(a.x_out);
    float4 v[P];
#pragma unroll
    for (int p = 0; p < P; ++p)
      v[p] = live[p] ? __ldg(src + k[p]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int p = 0; p < P; ++p)
      if (live[p]) dst[ibase + 32u * p] = v[p];
  }
}

// ---------------------------------------------------------------------------
// Megopolis (Algorithm 5).  Iteration b, particle i = 32 s + lane:
//   j = (32 s + o_al + (lane + o) mod 32) mod n,  o_al = o - o mod 32.
// The warp reads one aligned 32-weight partition per segment and iteration.
// Chains keep k - 32 p ("relative" ancestor) so that in the common case, where
// the P partitions do not wrap past n, every particle's candidate is the one
// shared window index x0.
template <int P, bool SMEM, int GATHER>
__device__ __forceinline__ void megopolis_batch(const ResampleArgs& a, int B,
                                                uint32_t s0, uint32_t seg_hi,
                                                uint32_t lane) {
  const uint32_t n = a.n;
  const uint32_t ibase = s0 * 32u + lane;
  float wk[P];
  uint32_t kr[P];
  bool live[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint32_t i = ibase + 32u * p;
    live[p] = (s0 + p < seg_hi) && (i < n);
    wk[p] = ldw<SMEM>(a.w, i < n ? i : n - 1u);
    kr[p] = ibase;
  }
  uint32_t o_reg = 0u;
  for (int b0 = 0; b0 < B; b0 += 4) {
    if ((b0 & 31) == 0)
      o_reg = mego_offset(a.k0, a.k1, a.sid, static_cast<uint32_t>(b0) + lane, n);
    const int nb = (B - b0) < 4 ? (B - b0) : 4;
    float wj[4][P];
    uint32_t cj[4][P];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q < nb) {
        const uint32_t o = __shfl_sync(0xFFFFFFFFu, o_reg, (b0 + q) & 31);
        uint32_t base = s0 * 32u + (o & ~31u);
        base = base >= n ? base - n : base;
        const uint32_t x0 = base + ((lane + o) & 31u);
        if (base + 32u * P <= n) {
#pragma unroll
          for (int p = 0; p < P; ++p) {
            wj[q][p] = ldw<SMEM>(a.w, x0 + 32u * p);
            cj[q][p] = x0;
          }
        } else {
#pragma unroll
          for (int p = 0; p < P; ++p) {
            uint32_t j = x0 + 32u * p;
            if (j >= n) j -= n;
            if (j >= n) j %= n;
            wj[q][p] = ldw<SMEM>(a.w, j);
            cj[q][p] = j - 32u * p;
          }
        }
      }
    }
    uint4 r[P];
#pragma unroll
    for (int p = 0; p < P; ++p)
      r[p] = philox4x32_10(ibase + 32u * p, static_cast<uint32_t>(b0) >> 2, a.sid,
                           kTagMegoU, a.k0, a.k1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q < nb) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const bool acc = accept(u_of(word_of(r[p], q)), wk[p], wj[q][p]);
          wk[p] = acc ? wj[q][p] : wk[p];
          kr[p] = acc ? cj[q][p] : kr[p];
        }
      }
    }
  }
  uint32_t k[P];
#pragma unroll
  for (int p = 0; p < P; ++p) k[p] = kr[p] + 32u * p;
  finish_batch<P, GATHER>(a, ibase, k, live);
}

// ---------------------------------------------------------------------------
// Metropolis (Algorithm 2): independent j ~ U{0, n-1} per particle and
// iteration; two iterations per Philox call.
template <int P, bool SMEM, int GATHER>
__device__ __forceinline__ void metropolis_batch(const ResampleArgs& a, int B,
                                                 uint32_t s0, uint32_t seg_hi,
                                                 uint32_t lane) {
  const uint32_t n = a.n;
  const uint32_t ibase = s0 * 32u + lane;
  float wk[P];
  uint32_t k[P];
  bool live[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint32_t i = ibase + 32u * p;
    live[p] = (s0 + p < seg_hi) && (i < n);
    k[p] = i < n ? i : n - 1u;
    wk[p] = ldw<SMEM>(a.w, k[p]);
  }
  for (int b0 = 0; b0 < B; b0 += 2) {
    const int nb = (B - b0) < 2 ? (B - b0) : 2;
    uint4 r[P];
#pragma unroll
    for (int p = 0; p < P; ++p)
      r[p] = philox4x32_10(ibase + 32u * p, static_cast<uint32_t>(b0) >> 1, a.sid,
                           kTagMetro, a.k0, a.k1);
    float wj[2][P];
    uint32_t jj[2][P];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q < nb) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          jj[q][p] = index32(q == 0 ? r[p].x : r[p].z, n);
          wj[q][p] = ldw<SMEM>(a.w, jj[q][p]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q < nb) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const bool acc = accept(u_of(q == 0 ? r[p].y : r[p].w), wk[p], wj[q][p]);
          wk[p] = acc ? wj[q][p] : wk[p];
          k[p] = acc ? jj[q][p] : k[p];
        }
      }
    }
  }
  finish_batch<P, GATHER>(a, ibase, k, live);
}

// ---------------------------------------------------------------------------
// Metropolis-C1 / C2 (Algorithms 3, 4): j uniform inside partition p of nw
// weights; p drawn per 32-particle segment once (C1) or per iteration (C2).
template <int VARIANT, int P, bool SMEM, int GATHER>
__device__ __forceinline__ void partition_batch(const ResampleArgs& a, int B,
                                                uint32_t s0, uint32_t seg_hi,
                                                uint32_t lane) {
  const uint32_t n = a.n;
  const uint32_t ibase = s0 * 32u + lane;
  float wk[P];
  uint32_t k[P];
  bool live[P];
  uint32_t part[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint32_t i = ibase + 32u * p;
    live[p] = (s0 + p < seg_hi) && (i < n);
    k[p] = i < n ? i : n - 1u;
    wk[p] = ldw<SMEM>(a.w, k[p]);
    part[p] = 0u;
    if constexpr (VARIANT == kC1) {
      const uint4 x = philox4x32_10(s0 + p, 0u, a.sid, kTagCPart, a.k0, a.k1);
      part[p] = index64(x.x, x.y, a.npart);
    }
  }
  // C2: lane l holds the partition of segment s0 + (l % P) for iteration
  // b0 + l / P, refilled every 32 / P iterations.
  constexpr int kStepsPerFill = 32 / P;
  uint32_t part_reg = 0u;
  for (int b0 = 0; b0 < B; b0 += 2) {
    const int nb = (B - b0) < 2 ? (B - b0) : 2;
    if constexpr (VARIANT == kC2) {
      if ((b0 % kStepsPerFill) == 0) {
        const uint32_t bb = static_cast<uint32_t>(b0) + lane / P;
        const uint4 x = philox4x32_10(s0 + lane % P, bb + 1u, a.sid, kTagCPart, a.k0, a.k1);
        part_reg = index64(x.x, x.y, a.npart);
      }
    }
    uint4 r[P];
#pragma unroll
    for (int p = 0; p < P; ++p)
      r[p] = philox4x32_10(ibase + 32u * p, static_cast<uint32_t>(b0) >> 1, a.sid,
                           kTagCDraw, a.k0, a.k1);
    float wj[2][P];
    uint32_t jj[2][P];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q < nb) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          uint32_t pp = part[p];
          if constexpr (VARIANT == kC2) {
            const int src = ((b0 + q) % kStepsPerFill) * P + p;
            pp = __shfl_sync(0xFFFFFFFFu, part_reg, src);
          }
          jj[q][p] = pp * a.nw + index32(q == 0 ? r[p].x : r[p].z, a.nw);
          wj[q][p] = ldw<SMEM>(a.w, jj[q][p]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q < nb) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const bool acc = accept(u_of(q == 0 ? r[p].y : r[p].w), wk[p], wj[q][p]);
          wk[p] = acc ? wj[q][p] : wk[p];
          k[p] = acc ? jj[q][p] : k[p];
        }
      }
    }
  }
  finish_batch<P, GATHER>(a, ibase, k, live);
}

// ---------------------------------------------------------------------------
template <int VARIANT, int P, bool SMEM, int GATHER>
__global__ void __launch_bounds__(256) resample_kernel(const ResampleArgs a) {
  const int B = a.B_dev ? *a.B_dev : a.B;
  if (B < 0) return;  // device-side bound failed: write nothing
  if constexpr (SMEM) {
    if (!stage_weights(a)) return;
  }
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t wpb = blockDim.x >> 5;
  const uint64_t gw = static_cast<uint64_t>(blockIdx.x) * wpb + (threadIdx.x >> 5);
  const uint64_t tw = static_cast<uint64_t>(gridDim.x) * wpb;
  const uint32_t seg_lo = static_cast<uint32_t>(a.nseg * gw / tw);
  const uint32_t seg_hi = static_cast<uint32_t>(a.nseg * (gw + 1u) / tw);
  for (uint32_t s0 = seg_lo; s0 < seg_hi; s0 += P) {
    if constexpr (VARIANT == kMegopolis) {
      megopolis_batch<P, SMEM, GATHER>(a, B, s0, seg_hi, lane);
    } else if constexpr (VARIANT == kMetropolis) {
      metropolis_batch<P, SMEM, GATHER>(a, B, s0, seg_hi, lane);
    } else {
      partition_batch<VARIANT, P, SMEM, GATHER>(a, B, s0, seg_hi, lane);
    }
  }
}

// Host-side launcher for one variant (defined in resample_<variant>.cu).
struct LaunchShape {
  int threads;
  int ppt;
  bool smem;
  int grid;
  size_t smem_bytes;
};

// Opt a kernel in to the largest dynamic shared-memory size it can use
// (the per-block opt-in limit minus its static shared memory), once per
// device and kernel.  Defined in capi.cu.
cudaError_t enable_large_smem(const void* kernel);

template <int VARIANT>
cudaError_t launch_resample(const LaunchShape& s, int gather, const ResampleArgs& a,
                            cudaStream_t stream);

template <int VARIANT>
const void* resample_kernel_ptr(int ppt, bool smem, int gather);

}  // namespace mego
