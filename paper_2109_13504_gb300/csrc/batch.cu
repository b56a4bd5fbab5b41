// batch.cu -- many independent resampling problems ("filters") in one
// persistent launch.
//
// Plan (a caller-provided device buffer, written by mego_batch_plan):
//   header (queue counters, counts) | filter descriptors | item prefix sums |
//   chunk prefix sums | per-filter B, status, q | bound partials.
// Resample work items are (filter, 6 or 4 consecutive 32-particle segments,
// chosen per plan);
// warps of a persistent grid take items from a queue (one atomic per item),
// so filters of very different cost (size times B) balance themselves.  The
// last warp to leave resets the queue, so the plan can be launched again.
// The bound runs one CTA per (filter, 4096-weight chunk) and one warp per
// filter for the fold, in fixed order (deterministic).
// One seed per batch; every filter has its own stream id, so a filter's
// ancestors are the same alone (mego_resample_gather with that seed and
// stream id) and in any batch.
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/megopolis.h"
#include "batch_plan.h"
#include "bound.cuh"
#include "resample_kernels.cuh"

namespace mego {
namespace {

// Segments (32 particles each) per work item, fixed in the plan: one batch
// of the default particles per thread.  Megopolis takes six chains per thread
// (items of 6) when filters of at least 2^17 particles hold most of the
// segments -- long items over long chains, where the extra ILP pays -- and
// four otherwise (many small filters: shorter items balance better and the
// per-item start-up is amortised over fewer chains); Metropolis takes 4.
constexpr uint32_t kItemSegsWide = 6;
constexpr uint32_t kItemSegs = 4;
constexpr uint64_t kWideMinSegs = (1u << 17) / 32u;
uint32_t item_segs_for(int variant, const mego_filter* h, int32_t count) {
  if (variant != MEGO_MEGOPOLIS) return kItemSegs;
  uint64_t big = 0, all = 0;
  for (int32_t f = 0; f < count; ++f) {
    const uint64_t nseg = (static_cast<uint64_t>(h[f].n) + 31u) / 32u;
    all += nseg;
    if (nseg >= kWideMinSegs) big += nseg;
  }
  return 2u * big >= all ? kItemSegsWide : kItemSegs;
}
constexpr uint32_t kChunk = 4096;        // weights per bound work item
constexpr int kBoundThreads = 256;       // 16 weights per thread per chunk

struct FilterDev {
  const float* w;
  int32_t* anc;
  const float* x_in;
  float* x_out;
  int64_t ld;
  uint32_t n;
  int32_t B;        // >= 0: fixed; < 0: the batch bound's value
  uint32_t sid;
  int32_t dim;
  const float* w_host;  // non-null: the bound reads here and writes w
};

struct PlanHeader {
  uint32_t next;         // resample queue head
  uint32_t done;         // warps that left the resample kernel
  uint32_t count;
  uint32_t total_items;
  uint32_t total_chunks;
  uint32_t item_segs;    // segments per work item
  // The batch's most expensive filter, whose items the queue hands out first
  // (its chains set the length of the launch): (bits of float((B + 1) x
  // items) << 32) | ~f, the largest wins (ties: the lowest f); 0 = none.
  unsigned long long heavy;
  // Shared-memory phase: filters of at most smem_max_n weights are resampled
  // whole by one CTA each (their weights staged in shared memory), claimed
  // through smem_next before the warp-level queue; they own no work items.
  uint32_t smem_next;
  uint32_t smem_count;
  uint32_t smem_max_n;
  uint32_t reserved;
};
static_assert(sizeof(PlanHeader) == 48, "plan header layout");

struct PlanLayout {
  size_t filters, item_prefix, chunk_prefix, B, status, q, smem_list, parts, total;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

PlanLayout layout_for(uint32_t count, uint64_t total_chunks) {
  PlanLayout L;
  size_t off = sizeof(PlanHeader);
  off = align_up(off, 16);
  L.filters = off;
  off += sizeof(FilterDev) * count;
  off = align_up(off, 16);
  L.item_prefix = off;
  off += sizeof(uint32_t) * (count + 1);
  off = align_up(off, 16);
  L.chunk_prefix = off;
  off += sizeof(uint32_t) * (count + 1);
  off = align_up(off, 16);
  L.B = off;
  off += sizeof(int32_t) * count;
  off = align_up(off, 16);
  L.status = off;
  off += sizeof(int32_t) * count;
  off = align_up(off, 16);
  L.q = off;
  off += sizeof(double) * count;
  off = align_up(off, 16);
  L.smem_list = off;  // filter indices of the shared-memory phase, largest first
  off += sizeof(uint32_t) * count;
  off = align_up(off, 16);
  L.parts = off;
  off += sizeof(Partial) * total_chunks;
  L.total = align_up(off, 256);
  return L;
}

struct BatchArgs {
  unsigned char* plan;
  size_t off_filters, off_item_prefix, off_chunk_prefix, off_B, off_status, off_q, off_smem_list,
      off_parts;
  RoundKeys K;
};

// Largest f with prefix[f] <= x (prefix non-decreasing, prefix[0] = 0).
__device__ __forceinline__ uint32_t find_owner(const uint32_t* prefix, uint32_t count,
                                               uint32_t x) {
  uint32_t lo = 0, hi = count;  // answer in [lo, hi)
  while (hi - lo > 1u) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__host__ __device__ inline unsigned long long heavy_key(float cost, uint32_t f) {
  uint32_t bits;
  memcpy(&bits, &cost, sizeof bits);
  return (static_cast<unsigned long long>(bits) << 32) | static_cast<uint32_t>(~f);
}

// Queue position -> (filter, item within it): the heavy filter's items come
// first, then every other filter's in plan order.
__device__ __forceinline__ uint32_t item_owner(const uint32_t* ip, uint32_t count,
                                               unsigned long long heavy, uint32_t item,
                                               uint32_t* local) {
  if ((heavy >> 32) != 0u) {
    const uint32_t h = ~static_cast<uint32_t>(heavy);
    const uint32_t nh = __ldg(ip + h + 1) - __ldg(ip + h);
    if (item < nh) {
      *local = item;
      return h;
    }
    item -= nh;
    if (item >= __ldg(ip + h)) item += nh;
  }
  const uint32_t f = find_owner(ip, count, item);
  *local = item - __ldg(ip + f);
  return f;
}

// ---------------------------------------------------------------------------
// Bound: partial per (filter, chunk), then one warp per filter.

struct BAcc {
  float mx = 0.0f;
  int bad = 0;
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    bad |= (!(v >= 0.0f) || isinf(v)) ? 1 : 0;
    mx = fmaxf(mx, v);
    const float t = __fadd_rn(s, v);
    c = __fadd_rn(c, fabsf(s) >= fabsf(v) ? __fadd_rn(__fsub_rn(s, t), v)
                                            : __fadd_rn(__fsub_rn(v, t), s));
    s = t;
  }
};

__global__ void __launch_bounds__(kBoundThreads) batch_partials_kernel(const __grid_constant__ BatchArgs a) {
  const PlanHeader* h = reinterpret_cast<const PlanHeader*>(a.plan);
  const FilterDev* F = reinterpret_cast<const FilterDev*>(a.plan + a.off_filters);
  const uint32_t* cp = reinterpret_cast<const uint32_t*>(a.plan + a.off_chunk_prefix);
  Partial* parts = reinterpret_cast<Partial*>(a.plan + a.off_parts);
  const uint32_t count = h->count;
  const uint32_t chunk = blockIdx.x;
  grid_launch_dependents();  // the finalize may be scheduled now; it waits for us
  // The finalize that follows picks the heavy filter anew from this bound.
  if (chunk == 0u && threadIdx.x == 0u) const_cast<PlanHeader*>(h)->heavy = 0ull;
  const uint32_t f = find_owner(cp, count, chunk);
  const uint32_t n = F[f].n;
  const float* w_host = F[f].w_host;
  const float* w = F[f].w;
  const uint32_t lo = (chunk - cp[f]) * kChunk;
  const uint32_t hi = min(n, lo + kChunk);
  // All of a thread's weights are loaded before the (sequential) compensated
  // sum starts, so the chunk costs one memory latency; the sum still runs in
  // index order.
  constexpr int kPer = static_cast<int>(kChunk) / kBoundThreads;
  float v[kPer];
  // A whole, 16-byte aligned device chunk is read with 16-byte loads: thread t
  // takes floats 4 t + 1024 k .. +3 (k < 4), four loads instead of sixteen.
  const bool vec = !w_host && hi - lo == kChunk &&
                   (reinterpret_cast<uintptr_t>(w + lo) & 15u) == 0u;
  if (vec) {
    const float4* w4 = reinterpret_cast<const float4*>(w + lo);
#pragma unroll
    for (int k = 0; k < kPer / 4; ++k) {
      const float4 q = __ldg(w4 + threadIdx.x + k * kBoundThreads);
      v[4 * k] = q.x;
      v[4 * k + 1] = q.y;
      v[4 * k + 2] = q.z;
      v[4 * k + 3] = q.w;
    }
  } else if (w_host) {
    // Page-locked host memory, read once over the CPU-GPU link (plain loads).
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t i = lo + threadIdx.x + static_cast<uint32_t>(k) * kBoundThreads;
      v[k] = i < hi ? w_host[i] : 0.0f;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t i = lo + threadIdx.x + static_cast<uint32_t>(k) * kBoundThreads;
      v[k] = i < hi ? __ldg(w + i) : 0.0f;
    }
  }
  if (w_host) {
    // Upload: the device copy that the resample reads.
    float* w_dev = const_cast<float*>(F[f].w);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t i = lo + threadIdx.x + static_cast<uint32_t>(k) * kBoundThreads;
      if (i < hi) w_dev[i] = v[k];
    }
  }
  BAcc acc;
  if (vec) {
#pragma unroll
    for (int k = 0; k < kPer; ++k) acc.add(v[k]);
  } else {
#pragma unroll
    for (int k = 0; k < kPer; ++k)
      if (lo + threadIdx.x + static_cast<uint32_t>(k) * kBoundThreads < hi) acc.add(v[k]);
  }
  // Fixed-order tree in float-float (no FP64 work per thread: this part's
  // FP64 pipe is narrow): warp shuffles, then thread 0 over the warp results;
  // the chunk's partial is converted to double once.
  FloatFloat sum = ff_from_pair(acc.s, acc.c);
  float mx = acc.mx;
  int bad = acc.bad;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    FloatFloat o;
    o.hi = __shfl_down_sync(0xFFFFFFFFu, sum.hi, off);
    o.lo = __shfl_down_sync(0xFFFFFFFFu, sum.lo, off);
    sum = ff_add(sum, o);
    mx = fmaxf(mx, __shfl_down_sync(0xFFFFFFFFu, mx, off));
    bad |= __shfl_down_sync(0xFFFFFFFFu, bad, off);
  }
  __shared__ FloatFloat s_sum[kBoundThreads / 32];
  __shared__ float s_mx[kBoundThreads / 32];
  __shared__ int s_bad[kBoundThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_sum[warp] = sum;
    s_mx[warp] = mx;
    s_bad[warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    FloatFloat t{0.0f, 0.0f};
    float m = 0.0f;
    int b = 0;
    for (int k = 0; k < kBoundThreads / 32; ++k) {
      t = ff_add(t, s_sum[k]);
      m = fmaxf(m, s_mx[k]);
      b |= s_bad[k];
    }
    parts[chunk] = Partial{m, b, ff_to_double(t)};
  }
}

__global__ void __launch_bounds__(256) batch_finalize_kernel(const __grid_constant__ BatchArgs a,
                                                             double log_eps, int32_t b_max) {
  const PlanHeader* h = reinterpret_cast<const PlanHeader*>(a.plan);
  const FilterDev* F = reinterpret_cast<const FilterDev*>(a.plan + a.off_filters);
  const uint32_t* cp = reinterpret_cast<const uint32_t*>(a.plan + a.off_chunk_prefix);
  const Partial* parts = reinterpret_cast<const Partial*>(a.plan + a.off_parts);
  int32_t* Bout = reinterpret_cast<int32_t*>(a.plan + a.off_B);
  int32_t* Sout = reinterpret_cast<int32_t*>(a.plan + a.off_status);
  double* Qout = reinterpret_cast<double*>(a.plan + a.off_q);
  const uint32_t f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint32_t lane = threadIdx.x & 31u;
  grid_launch_dependents();  // the resample may be scheduled now; it waits for us
  grid_dependency_wait();    // the partials are complete and visible
  if (f >= h->count) return;
  double sum = 0.0;
  float mx = 0.0f;
  int bad = 0;
  // Loads go out eight at a time, ahead of the (order-dependent) sums.
  const uint32_t c_end = cp[f + 1];
  for (uint32_t c0 = cp[f] + lane; c0 < c_end; c0 += 8u * 32u) {
    Partial p[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (c0 + 32u * k < c_end) p[k] = parts[c0 + 32u * k];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (c0 + 32u * k < c_end) {
        sum += p[k].sum;
        mx = fmaxf(mx, p[k].mx);
        bad |= p[k].bad;
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sum += __shfl_down_sync(0xFFFFFFFFu, sum, off);
    mx = fmaxf(mx, __shfl_down_sync(0xFFFFFFFFu, mx, off));
    bad |= __shfl_down_sync(0xFFFFFFFFu, bad, off);
  }
  if (lane != 0) return;
  int32_t B = -1, status = kStatusWeights;
  double q = __longlong_as_double(0x7FF8000000000000LL);
  if (!bad && mx > 0.0f && isfinite(sum)) {  // an overflowed chunk sum cannot give B
    const double r = sum / (static_cast<double>(F[f].n) * static_cast<double>(mx));
    q = (r >= 1.0) ? 0.0 : log_eps / log1p(-r);
    double c = ceil(q);
    if (c < 0.0) c = 0.0;
    if (c <= static_cast<double>(b_max)) {
      B = static_cast<int32_t>(c);
      status = 0;
    }
  }
  Bout[f] = B;
  Sout[f] = status;
  Qout[f] = q;
  // Candidate for the heavy filter: cost = (B + 1) x its work items, with the
  // B the resample will use (a fixed B where the filter has one).
  const int32_t Beff = F[f].B >= 0 ? F[f].B : B;
  if (Beff >= 0) {
    const uint32_t* ip = reinterpret_cast<const uint32_t*>(a.plan + a.off_item_prefix);
    const float cost = static_cast<float>(Beff + 1) * static_cast<float>(ip[f + 1] - ip[f]);
    atomicMax(&const_cast<PlanHeader*>(h)->heavy, heavy_key(cost, f));
  }
}

// ---------------------------------------------------------------------------
// Persistent resample over the work queue.

// Stage w[0, n) of one filter into dynamic shared memory for a CTA that
// stages filter after filter: the 16-byte aligned whole part by bulk async
// copies on the CTA's barrier `bar` (phase parity `phase`, flipped by each
// bulk staging), the rest by plain loads.  Returns 0 when staged; 1 when the
// bounded wait expired but a second bounded wait saw the copy land (the
// filter is skipped); 2 when the copy did not land either (the CTA must stop
// using its shared memory).  Uniform across the CTA.
__device__ __forceinline__ int stage_filter(const float* w, uint32_t n, uint64_t* bar,
                                            uint32_t& phase) {
  float* s_w = reinterpret_cast<float*>(g_dyn_smem);
  const uint32_t n4 = n & ~3u;
  const bool bulk = ((reinterpret_cast<uintptr_t>(w) & 15u) == 0u) && n4 > 0u;
  if (bulk && threadIdx.x == 0) {
    const uint32_t bytes = n4 * 4u;
    mbar_expect_tx(bar, bytes);
    for (uint32_t off = 0; off < bytes; off += kStageChunk) {
      const uint32_t len = (bytes - off) < kStageChunk ? (bytes - off) : kStageChunk;
      bulk_g2s(reinterpret_cast<char*>(s_w) + off, reinterpret_cast<const char*>(w) + off, len,
               bar);
    }
  }
  for (uint32_t t = (bulk ? n4 : 0u) + threadIdx.x; t < n; t += blockDim.x) s_w[t] = __ldg(w + t);
  int status = 0;
  if (bulk) {
    const bool done = mbar_wait_bounded(bar, phase, kMaxPolls);
    if (!__syncthreads_and(done ? 1 : 0)) {
      int lost = 0;
      if (threadIdx.x == 0) lost = mbar_wait_bounded(bar, phase, kMaxPolls) ? 0 : 1;
      status = __syncthreads_or(lost) ? 2 : 1;
    }
    phase ^= 1u;
  }
  __syncthreads();
  return status;
}

// WITH_SMEM: first the shared-memory phase -- each CTA claims whole small
// filters (the plan's smem list), stages a filter's weights once and splits
// its 32-particle segments among its warps (run on the shared-memory path) --
// then the warp-level queue over the other filters' work items.  Without it
// the kernel is the warp-level queue alone.
template <int VARIANT, int P, int GATHER, bool WITH_SMEM>
__global__ void __launch_bounds__(max_threads_for(P))
batch_resample_kernel(const __grid_constant__ BatchArgs a) {
  __shared__ int2 s_win[kMaxWarps][32];
  PlanHeader* h = reinterpret_cast<PlanHeader*>(a.plan);
  const FilterDev* F = reinterpret_cast<const FilterDev*>(a.plan + a.off_filters);
  const uint32_t* ip = reinterpret_cast<const uint32_t*>(a.plan + a.off_item_prefix);
  const int32_t* Bb = reinterpret_cast<const int32_t*>(a.plan + a.off_B);
  const uint32_t lane = threadIdx.x & 31u;
  grid_dependency_wait();  // the bound's B and heavy filter are complete and visible
  const uint32_t count = h->count;
  const uint32_t total = h->total_items;
  const unsigned long long heavy = h->heavy;
  const uint32_t item_segs = h->item_segs;
  int2* win = s_win[threadIdx.x >> 5];
  bool healthy = true;
  if constexpr (WITH_SMEM) {
    const uint32_t* sl = reinterpret_cast<const uint32_t*>(a.plan + a.off_smem_list);
    int32_t* St = reinterpret_cast<int32_t*>(a.plan + a.off_status);
    const uint32_t nsm = h->smem_count;
    __shared__ uint32_t s_claim;
    __shared__ __align__(8) uint64_t s_bar;
    if (threadIdx.x == 0) mbar_init(&s_bar, 1u);
    __syncthreads();
    uint32_t phase = 0u;
    const uint32_t wpb = blockDim.x >> 5, wi = threadIdx.x >> 5;
    for (;;) {
      if (threadIdx.x == 0) s_claim = atomicAdd(&h->smem_next, 1u);
      __syncthreads();
      const uint32_t e = s_claim;
      __syncthreads();  // every thread has read the claim before the next one
      if (e >= nsm) break;
      const uint32_t f = __ldg(sl + e);
      const FilterDev d = F[f];
      const int B = d.B >= 0 ? d.B : Bb[f];
      if (B < 0) continue;  // the bound failed for this filter: write nothing
      const int st = stage_filter(d.w, d.n, &s_bar, phase);
      if (st != 0) {
        if (threadIdx.x == 0) St[f] = MEGO_ETIMEOUT;
        if (st == 2) {
          healthy = false;
          break;
        }
        continue;
      }
      Problem p;
      p.w = d.w;
      p.anc = d.anc;
      p.x_in = d.x_in;
      p.x_out = d.x_out;
      p.fault = nullptr;
      p.ld = d.ld;
      p.n = d.n;
      p.nseg = (d.n + 31u) / 32u;
      p.dim = d.dim;
      p.nw = 1u;
      p.npart = d.n;
      p.stage_polls = kMaxPolls;
      p.S = stream_key(a.K, d.sid);
      // The warps of the CTA split the filter's batches of P segments.
      const uint64_t nbat = (p.nseg + P - 1u) / P;
      const uint32_t seg_lo = static_cast<uint32_t>(nbat * wi / wpb) * P;
      const uint32_t seg_hi =
          min(p.nseg, static_cast<uint32_t>(nbat * (wi + 1u) / wpb) * static_cast<uint32_t>(P));
      OffsetWindow ow{0u, false};
      run_segments<VARIANT, P, true, GATHER, false>(p, a.K, B, seg_lo, seg_hi, lane, win, ow);
      __syncthreads();  // all warps are done with the weights before the next staging
    }
  }
  for (;;) {
    if (!healthy) break;
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(&h->next, 1u);
    item = __shfl_sync(0xFFFFFFFFu, item, 0);
    if (item >= total) break;
    uint32_t local = 0;
    const uint32_t f = item_owner(ip, count, heavy, item, &local);
    const FilterDev d = F[f];
    const int B = d.B >= 0 ? d.B : Bb[f];
    if (B < 0) continue;  // the bound failed for this filter: write nothing
    Problem p;
    p.w = d.w;
    p.anc = d.anc;
    p.x_in = d.x_in;
    p.x_out = d.x_out;
    p.fault = nullptr;
    p.ld = d.ld;
    p.n = d.n;
    p.nseg = (d.n + 31u) / 32u;
    p.dim = d.dim;
    p.nw = 1u;
    p.npart = d.n;
    p.stage_polls = kMaxPolls;
    p.S = stream_key(a.K, d.sid);
    const uint32_t seg_lo = local * item_segs;
    const uint32_t seg_hi = min(p.nseg, seg_lo + item_segs);
    // Items are single batches, so the short-chain path (which saves the
    // offset draws of a warp's later batches) has nothing to save here; the
    // general path keeps the kernel's register allocation free of it.
    OffsetWindow ow{0u, false};
    run_segments<VARIANT, P, false, GATHER, false>(p, a.K, B, seg_lo, seg_hi, lane, win, ow);
  }
  // The last warp out resets the queues for the next launch of this plan.
  if (lane == 0) {
    __threadfence();
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    if (atomicAdd(&h->done, 1u) == warps - 1u) {
      h->next = 0u;
      h->smem_next = 0u;
      h->done = 0u;
      __threadfence();
    }
  }
}

template <int V, int P, int G, bool S>
cudaError_t launch_batch_one(int grid, int threads, size_t smem, const BatchArgs& a,
                             cudaStream_t st) {
  auto* k = &batch_resample_kernel<V, P, G, S>;
  if (S) {
    const cudaError_t e = enable_large_smem(reinterpret_cast<const void*>(k));
    if (e != cudaSuccess) return e;
  }
  return launch_after(k, dim3(grid), dim3(threads), smem, st, a);
}

template <int V, int P, int G, bool S>
const void* batch_ptr_one() {
  return reinterpret_cast<const void*>(&batch_resample_kernel<V, P, G, S>);
}

template <int V, int G, bool S>
cudaError_t launch_batch_p(int ppt, int grid, int threads, size_t smem, const BatchArgs& a,
                           cudaStream_t st) {
  switch (ppt) {
    case 1: return launch_batch_one<V, 1, G, S>(grid, threads, smem, a, st);
    case 2: return launch_batch_one<V, 2, G, S>(grid, threads, smem, a, st);
    case 4: return launch_batch_one<V, 4, G, S>(grid, threads, smem, a, st);
    case 6:
      if constexpr (V == kMegopolis) return launch_batch_one<V, 6, G, S>(grid, threads, smem, a, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template <int V, int G, bool S>
const void* batch_ptr_p(int ppt) {
  switch (ppt) {
    case 1: return batch_ptr_one<V, 1, G, S>();
    case 2: return batch_ptr_one<V, 2, G, S>();
    case 4: return batch_ptr_one<V, 4, G, S>();
    case 6:
      if constexpr (V == kMegopolis) return batch_ptr_one<V, 6, G, S>();
      return nullptr;
    default: return nullptr;
  }
}

template <int V, bool S>
cudaError_t launch_batch_v(int gather, int ppt, int grid, int threads, size_t smem,
                           const BatchArgs& a, cudaStream_t st) {
  switch (gather) {
    case kGatherNone: return launch_batch_p<V, kGatherNone, S>(ppt, grid, threads, smem, a, st);
    case kGatherSoa: return launch_batch_p<V, kGatherSoa, S>(ppt, grid, threads, smem, a, st);
    case kGatherAos4: return launch_batch_p<V, kGatherAos4, S>(ppt, grid, threads, smem, a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int V, bool S>
const void* batch_ptr_v(int gather, int ppt) {
  switch (gather) {
    case kGatherNone: return batch_ptr_p<V, kGatherNone, S>(ppt);
    case kGatherSoa: return batch_ptr_p<V, kGatherSoa, S>(ppt);
    case kGatherAos4: return batch_ptr_p<V, kGatherAos4, S>(ppt);
    default: return nullptr;
  }
}

const void* batch_kernel_ptr(int variant, int gather, int ppt, bool smem) {
  if (smem)
    return variant == MEGO_MEGOPOLIS ? batch_ptr_v<kMegopolis, true>(gather, ppt)
                                     : batch_ptr_v<kMetropolis, true>(gather, ppt);
  return variant == MEGO_MEGOPOLIS ? batch_ptr_v<kMegopolis, false>(gather, ppt)
                                   : batch_ptr_v<kMetropolis, false>(gather, ppt);
}

cudaError_t launch_batch(int variant, int gather, int ppt, int grid, int threads, size_t smem,
                         const BatchArgs& a, cudaStream_t st) {
  if (smem > 0)
    return variant == MEGO_MEGOPOLIS
               ? launch_batch_v<kMegopolis, true>(gather, ppt, grid, threads, smem, a, st)
               : launch_batch_v<kMetropolis, true>(gather, ppt, grid, threads, smem, a, st);
  return variant == MEGO_MEGOPOLIS
             ? launch_batch_v<kMegopolis, false>(gather, ppt, grid, threads, 0, a, st)
             : launch_batch_v<kMetropolis, false>(gather, ppt, grid, threads, 0, a, st);
}

int gather_of(int layout, bool has_state) {
  if (!has_state) return kGatherNone;
  return layout == MEGO_LAYOUT_AOS4 ? kGatherAos4 : kGatherSoa;
}

BatchArgs args_of(const mego_batch* b) {
  BatchArgs a;
  std::memset(&a, 0, sizeof a);
  const PlanLayout L = layout_for(static_cast<uint32_t>(b->count), b->total_chunks);
  a.plan = static_cast<unsigned char*>(b->d_plan);
  a.off_filters = L.filters;
  a.off_item_prefix = L.item_prefix;
  a.off_chunk_prefix = L.chunk_prefix;
  a.off_B = L.B;
  a.off_status = L.status;
  a.off_q = L.q;
  a.off_smem_list = L.smem_list;
  a.off_parts = L.parts;
  a.K = make_round_keys(b->seed);
  return a;
}

// Grid of the persistent kernel: every SM full of resident CTAs (with
// `smem` bytes of dynamic shared memory each when the plan has a
// shared-memory phase).
// The grid per (device, kernel, CTA size, shared memory) is computed once and
// cached: the serving loop plans a batch for every launch.
mego_status shape_for(int variant, int gather, int threads, int ppt, size_t smem, int* grid) {
  const void* k = batch_kernel_ptr(variant, gather, ppt, smem > 0);
  if (!k) return MEGO_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MEGO_ECUDA;
  using Key = std::tuple<int, const void*, int, size_t>;
  static std::mutex mu;
  static std::map<Key, int> cache;
  const Key key(dev, k, threads, smem);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *grid = it->second;
      return MEGO_OK;
    }
  }
  int sms = 0, occ = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MEGO_ECUDA;
  if (smem > 0 && enable_large_smem(k) != cudaSuccess) return MEGO_EINVAL;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return MEGO_ECUDA;
  }
  if (occ < 1) return MEGO_EINVAL;
  *grid = sms * occ;
  std::lock_guard<std::mutex> lock(mu);
  cache.emplace(key, *grid);
  return MEGO_OK;
}

bool sizes(const mego_filter* h, int32_t count, uint64_t* items, uint64_t* chunks) {
  uint64_t it = 0, ch = 0;
  for (int32_t f = 0; f < count; ++f) {
    if (h[f].n < 1 || h[f].n > MEGO_N_MAX) return false;
    const uint64_t nseg = (static_cast<uint64_t>(h[f].n) + 31u) / 32u;
    it += (nseg + kItemSegs - 1) / kItemSegs;
    ch += (static_cast<uint64_t>(h[f].n) + kChunk - 1) / kChunk;
  }
  if (it >= (1ull << 31) || ch >= (1ull << 31)) return false;
  *items = it;
  *chunks = ch;
  return true;
}

}  // namespace
}  // namespace mego

extern "C" {

size_t mego_batch_plan_bytes(const mego_filter* h_filters, int32_t count) {
  uint64_t items = 0, chunks = 0;
  if (!h_filters || count < 1 || !mego::sizes(h_filters, count, &items, &chunks)) return 0;
  return mego::layout_for(static_cast<uint32_t>(count), chunks).total;
}

mego_status mego_batch_plan(const mego_filter* h_filters, int32_t count, int variant,
                            int layout, uint64_t seed, void* d_plan, size_t plan_bytes,
                            mego_batch* out, void* stream) {
  // Pageable staging: the copy has read it by the time cudaMemcpyAsync returns.
  std::vector<unsigned char> host;
  if (!out) return MEGO_EINVAL;
  return mego::batch_plan_staged(h_filters, count, variant, layout, seed, 0, d_plan, plan_bytes,
                                 &host, nullptr, 0, out, stream, false);
}

}  // extern "C"

namespace mego {

// Largest smem_max_n the device allows: the filter's weights (rounded up to
// 16 bytes) next to the kernel's static shared memory (the per-warp offset
// tables, the claim and the barrier: under 4 KiB).
int32_t smem_limit_n() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
      cudaSuccess)
    return 0;
  return optin > 4096 ? ((optin - 4096) / 16) * 4 : 0;
}

// The limit only matters for a shared-memory phase (the serving loop plans
// every batch without one and skips the device query).
bool smem_threshold_ok(int32_t smem_max_n) {
  return smem_max_n == 0 || (smem_max_n > 0 && smem_max_n <= smem_limit_n());
}

mego_status batch_plan_staged(const mego_filter* h_filters, int32_t count, int variant,
                              int layout, uint64_t seed, int32_t smem_max_n, void* d_plan,
                              size_t plan_bytes, std::vector<unsigned char>* pageable,
                              void* staging, size_t staging_bytes, mego_batch* out,
                              void* stream, bool replan) {
  if (!h_filters || count < 1 || !d_plan || !out) return MEGO_EINVAL;
  if (!smem_threshold_ok(smem_max_n)) return MEGO_EINVAL;
  if (variant != MEGO_MEGOPOLIS && variant != MEGO_METROPOLIS) return MEGO_EINVAL;
  if (layout != MEGO_LAYOUT_SOA && layout != MEGO_LAYOUT_AOS4) return MEGO_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_plan) & 255u) return MEGO_EINVAL;
  uint64_t items = 0, chunks = 0;
  if (!sizes(h_filters, count, &items, &chunks)) return MEGO_EINVAL;
  const PlanLayout L = layout_for(static_cast<uint32_t>(count), chunks);
  if (plan_bytes < L.total) return MEGO_ENOMEM;
  bool has_state = false, no_state = false;
  for (int32_t f = 0; f < count; ++f) {
    const mego_filter& d = h_filters[f];
    if (!d.w || d.B > MEGO_B_MAX) return MEGO_EINVAL;
    const bool st = d.x_in || d.x_out;
    if (st) {
      if (!d.x_in || !d.x_out) return MEGO_EINVAL;
      if (layout == MEGO_LAYOUT_SOA && (d.dim < 1 || d.ld < d.n)) return MEGO_EINVAL;
      if (layout == MEGO_LAYOUT_AOS4 &&
          (d.dim != 4 ||
           ((reinterpret_cast<uintptr_t>(d.x_in) | reinterpret_cast<uintptr_t>(d.x_out)) & 15u)))
        return MEGO_EINVAL;
      has_state = true;
    } else {
      if (!d.anc) return MEGO_EINVAL;
      no_state = true;
    }
  }
  if (has_state && no_state) return MEGO_EINVAL;  // one gather layout per batch
  unsigned char* host = nullptr;
  if (pageable) {
    pageable->assign(L.parts, 0);
    host = pageable->data();
  } else {
    if (!staging || staging_bytes < L.parts) return MEGO_ENOMEM;
    host = static_cast<unsigned char*>(staging);
    std::memset(host, 0, L.parts);
  }
  const uint32_t item_segs = item_segs_for(variant, h_filters, count);
  PlanHeader hdr{};
  hdr.item_segs = item_segs;
  hdr.count = static_cast<uint32_t>(count);
  hdr.total_items = static_cast<uint32_t>(items);
  hdr.total_chunks = static_cast<uint32_t>(chunks);
  std::memcpy(host, &hdr, sizeof hdr);
  FilterDev* F = reinterpret_cast<FilterDev*>(host + L.filters);
  uint32_t* ip = reinterpret_cast<uint32_t*>(host + L.item_prefix);
  uint32_t* cp = reinterpret_cast<uint32_t*>(host + L.chunk_prefix);
  int32_t* Bv = reinterpret_cast<int32_t*>(host + L.B);
  uint32_t* sl = reinterpret_cast<uint32_t*>(host + L.smem_list);
  uint64_t it = 0, ch = 0;
  uint32_t nsm = 0, smem_n = 0;
  for (int32_t f = 0; f < count; ++f) {
    const mego_filter& d = h_filters[f];
    F[f] = FilterDev{d.w, d.anc, d.x_in, d.x_out, d.ld, static_cast<uint32_t>(d.n), d.B,
                     d.stream_id, d.dim, d.w_host};
    ip[f] = static_cast<uint32_t>(it);
    cp[f] = static_cast<uint32_t>(ch);
    Bv[f] = d.B;
    ch += (static_cast<uint64_t>(d.n) + kChunk - 1) / kChunk;
    if (d.n <= smem_max_n) {  // shared-memory phase: a whole filter per CTA, no items
      sl[nsm++] = static_cast<uint32_t>(f);
      if (static_cast<uint32_t>(d.n) > smem_n) smem_n = static_cast<uint32_t>(d.n);
      continue;
    }
    const uint64_t nseg = (static_cast<uint64_t>(d.n) + 31u) / 32u;
    it += (nseg + item_segs - 1) / item_segs;
  }
  // Largest filters first, so the long stagings start early.
  std::stable_sort(sl, sl + nsm, [&](uint32_t x, uint32_t y) {
    return h_filters[x].n > h_filters[y].n;
  });
  reinterpret_cast<PlanHeader*>(host)->smem_count = nsm;
  reinterpret_cast<PlanHeader*>(host)->smem_max_n = static_cast<uint32_t>(smem_max_n);
  reinterpret_cast<PlanHeader*>(host)->total_items = static_cast<uint32_t>(it);
  items = it;
  ip[count] = static_cast<uint32_t>(it);
  cp[count] = static_cast<uint32_t>(ch);
  // Heavy filter among those with a fixed B; a bound recomputes it over all.
  unsigned long long heavy = 0ull;
  for (int32_t f = 0; f < count; ++f) {
    if (h_filters[f].B < 0) continue;
    const float cost = static_cast<float>(h_filters[f].B + 1) *
                       static_cast<float>(ip[f + 1] - ip[f]);
    const unsigned long long k = heavy_key(cost, static_cast<uint32_t>(f));
    if (k > heavy) heavy = k;
  }
  reinterpret_cast<PlanHeader*>(host)->heavy = heavy;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!replan) {
    if (cudaMemcpyAsync(d_plan, host, L.parts, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return MEGO_ECUDA;
  } else {
    // A new shared-memory threshold for a plan in use: keep the heavy filter
    // the last bound found (a stale one only reorders the queue) and the
    // per-filter B, status and q, which a bound may already have written.
    const size_t heavy_off = offsetof(PlanHeader, heavy);
    const size_t after = heavy_off + sizeof(unsigned long long);
    if (cudaMemcpyAsync(d_plan, host, heavy_off, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(static_cast<unsigned char*>(d_plan) + after, host + after, L.B - after,
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(static_cast<unsigned char*>(d_plan) + L.smem_list, host + L.smem_list,
                        L.parts - L.smem_list, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return MEGO_ECUDA;
  }
  const mego_launch_cfg keep = out->cfg;
  std::memset(out, 0, sizeof *out);
  out->h_filters = h_filters;
  out->smem_max_n = smem_max_n;
  out->smem_filters = static_cast<int32_t>(nsm);
  out->smem_bytes = nsm ? (static_cast<size_t>(smem_n) * 4u + 15u) & ~static_cast<size_t>(15u)
                        : 0u;
  out->d_plan = d_plan;
  out->plan_bytes = L.total;
  out->count = count;
  out->variant = variant;
  out->layout = layout;
  out->gather = gather_of(layout, has_state);
  out->seed = seed;
  out->total_items = items;
  out->total_chunks = chunks;
  out->d_B = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(d_plan) + L.B);
  out->d_status = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(d_plan) + L.status);
  out->d_q = reinterpret_cast<double*>(static_cast<unsigned char*>(d_plan) + L.q);
  // Default shape: Megopolis takes one whole work item per warp (six chains
  // per thread in 128-thread CTAs, or four in 256-thread CTAs, following the
  // item size); Metropolis is bound by scattered loads and takes two.
  // A re-plan keeps the caller's shape.
  int ppt = variant == MEGO_MEGOPOLIS ? static_cast<int>(item_segs) : 2;
  int threads = ppt == 6 ? 128 : 256;
  if (replan && keep.threads > 0) {
    ppt = keep.ppt;
    threads = keep.threads;
  }
  out->cfg.threads = threads;
  out->cfg.ppt = ppt;
  out->cfg.path = nsm ? MEGO_PATH_SMEM : MEGO_PATH_GLOBAL;
  out->cfg.ctas_per_sm = 0;
  int grid = 0;
  const mego_status s = shape_for(variant, out->gather, threads, ppt, out->smem_bytes, &grid);
  if (s != MEGO_OK) return s;
  out->grid = grid;
  return MEGO_OK;
}

}  // namespace mego

extern "C" {

mego_status mego_batch_bound(const mego_batch* b, double eps, int32_t b_max, void* stream) {
  using namespace mego;
  if (!b || !b->d_plan || !(eps > 0.0 && eps <= 1.0) || b_max < 1 || b_max > MEGO_B_MAX)
    return MEGO_EINVAL;
  const BatchArgs a = args_of(b);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  batch_partials_kernel<<<static_cast<unsigned>(b->total_chunks), kBoundThreads, 0, st>>>(a);
  if (cudaGetLastError() != cudaSuccess) return MEGO_ECUDA;
  const unsigned fgrid = static_cast<unsigned>((b->count + 7) / 8);
  if (launch_after(batch_finalize_kernel, dim3(fgrid), dim3(256), 0, st, a, std::log(eps),
                   b_max) != cudaSuccess)
    return MEGO_ECUDA;
  count_launches(2);
  return MEGO_OK;
}

mego_status mego_batch_resample(const mego_batch* b, void* stream) {
  using namespace mego;
  if (!b || !b->d_plan || b->grid < 1) return MEGO_EINVAL;
  const BatchArgs a = args_of(b);
  if (launch_batch(b->variant, b->gather, b->cfg.ppt, b->grid, b->cfg.threads, b->smem_bytes, a,
                   static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return MEGO_ECUDA;
  count_launches(1);
  return MEGO_OK;
}

mego_status mego_batch_set_shape(mego_batch* b, int32_t threads, int32_t ppt) {
  using namespace mego;
  if (!b || threads < 64 || threads > (ppt == 6 ? 128 : 256) || threads % 32 ||
      (ppt != 1 && ppt != 2 && ppt != 4 && ppt != 6))
    return MEGO_EINVAL;
  int grid = 0;
  const mego_status s = shape_for(b->variant, b->gather, threads, ppt, b->smem_bytes, &grid);
  if (s != MEGO_OK) return s;
  b->cfg.threads = threads;
  b->cfg.ppt = ppt;
  b->grid = grid;
  return MEGO_OK;
}

mego_status mego_batch_set_smem(mego_batch* b, int32_t smem_max_n, void* stream) {
  if (!b || !b->d_plan || !b->h_filters || b->count < 1) return MEGO_EINVAL;
  if (b->graph_exec) return MEGO_EINVAL;  // a captured graph holds the old launch
  std::vector<unsigned char> host;
  mego_batch nb = *b;
  const mego_status s = mego::batch_plan_staged(
      b->h_filters, b->count, b->variant, b->layout, b->seed, smem_max_n, b->d_plan,
      b->plan_bytes, &host, nullptr, 0, &nb, stream, true);
  if (s != MEGO_OK) return s;
  *b = nb;
  return MEGO_OK;
}

mego_status mego_batch_autotune(mego_batch* b, int32_t reps, float* best_ms, void* stream) {
  if (!b || reps < 1 || reps > 100) return MEGO_EINVAL;
  if (b->graph_exec) return MEGO_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return MEGO_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MEGO_ECUDA;
  }
  const int threads_c[] = {64, 128, 256};
  const int ppt_c[] = {1, 2, 4, 6};
  // Shared-memory thresholds: none, then filters of up to 16, 64 and 192 KiB
  // of weights (only with the caller's filters at hand, to re-plan).
  const int32_t smem_c[] = {0, 4096, 16384, 49152};
  const int32_t smem_cap = mego::smem_limit_n();
  int best_t = b->cfg.threads, best_p = b->cfg.ppt;
  int32_t best_sm = b->smem_max_n;
  float best = 1e30f;
  mego_status status = MEGO_OK;
  for (int32_t sm : smem_c) {
    if (sm > 0 && (!b->h_filters || sm > smem_cap)) continue;
    if (b->h_filters) {
      status = mego_batch_set_smem(b, sm, stream);
      if (status != MEGO_OK) break;
    } else if (sm != b->smem_max_n) {
      continue;
    }
    for (int t : threads_c) {
      for (int p : ppt_c) {
        mego_status s = mego_batch_set_shape(b, t, p);
        if (s == MEGO_EINVAL) continue;
        if (s == MEGO_OK) s = mego_batch_resample(b, stream);  // warm-up
        float total = 0.0f;
        for (int r = 0; r < reps && s == MEGO_OK; ++r) {
          float ms = 0.0f;
          if (cudaEventRecord(e0, st) != cudaSuccess) s = MEGO_ECUDA;
          if (s == MEGO_OK) s = mego_batch_resample(b, stream);
          if (s == MEGO_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                               cudaEventSynchronize(e1) != cudaSuccess ||
                               cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            s = MEGO_ECUDA;
          total += ms;
        }
        if (s != MEGO_OK) {
          status = s;
          break;
        }
        if (total / reps < best) {
          best = total / reps;
          best_t = t;
          best_p = p;
          best_sm = sm;
        }
      }
      if (status != MEGO_OK) break;
    }
    if (status != MEGO_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != MEGO_OK) return status;
  mego_status s = MEGO_OK;
  if (b->h_filters && best_sm != b->smem_max_n) s = mego_batch_set_smem(b, best_sm, stream);
  if (s == MEGO_OK) s = mego_batch_set_shape(b, best_t, best_p);
  if (s == MEGO_OK && best_ms) *best_ms = best;
  return s;
}

mego_status mego_batch_graph(mego_batch* b, double eps, int32_t b_max, void* stream) {
  if (!b || !stream) return MEGO_EINVAL;  // capture needs a non-default stream
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (b->graph_exec) {
    cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(b->graph_exec));
    b->graph_exec = nullptr;
  }
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return MEGO_ECUDA;
  mego_status s = MEGO_OK;
  if (eps > 0.0) s = mego_batch_bound(b, eps, b_max, stream);
  if (s == MEGO_OK) s = mego_batch_resample(b, stream);
  // Captured, not run: take the capture's launches back out of the count.
  const int32_t kernels = (eps > 0.0 ? 2 : 0) + 1;
  mego::count_launches(static_cast<uint64_t>(-static_cast<int64_t>(kernels)));
  b->graph_kernels = kernels;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (s != MEGO_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess || !g) return MEGO_ECUDA;
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return MEGO_ECUDA;
  b->graph_exec = exec;
  return MEGO_OK;
}

mego_status mego_batch_launch_graph(const mego_batch* b, void* stream) {
  if (!b || !b->graph_exec) return MEGO_EINVAL;
  if (cudaGraphLaunch(static_cast<cudaGraphExec_t>(b->graph_exec),
                      static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return MEGO_ECUDA;
  mego::count_launches(static_cast<uint64_t>(b->graph_kernels));
  return MEGO_OK;
}

mego_status mego_batch_destroy(mego_batch* b) {
  if (!b) return MEGO_EINVAL;
  if (b->graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(b->graph_exec));
  b->graph_exec = nullptr;
  return MEGO_OK;
}

}  // extern "C"
