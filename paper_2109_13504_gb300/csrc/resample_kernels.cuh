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

#include <cuda.h>  // CUtensorMap (the TMA window path's tensor map)

#include "device_common.cuh"

namespace mego {

enum Variant : int { kMegopolis = 0, kMetropolis = 1, kC1 = 2, kC2 = 3 };
enum Gather : int { kGatherNone = 0, kGatherSoa = 1, kGatherAos4 = 2 };

// One resampling problem (one weight vector and its outputs).
struct Problem {
  const float* w;
  int32_t* anc;          // [n] ancestors, may be null
  const float* x_in;     // gather source, may be null
  float* x_out;
  int32_t* fault;        // device fault word, may be null
  int64_t ld;
  uint32_t n;
  uint32_t nseg;         // ceil(n / 32)
  int32_t dim;
  uint32_t nw;           // C1/C2: weights per partition
  uint32_t npart;        // C1/C2: number of partitions
  uint32_t stage_polls;  // SMEM path: polls of the first staging wait
  StreamKey S;           // stream constants for (seed, stream id)
};

// Kernel parameters of a single resample.
struct ResampleArgs {
  Problem p;
  const int32_t* B_dev;  // non-null: read B here (device-side bound)
  int32_t B;
  RoundKeys K;           // round keys of the seed
  CUtensorMap tmap;      // TMA window path: w as a 1-D tensor, box of 32 P weights
};

// TMA window path state of one warp: a shared-memory ring of the five
// windows of a group of iterations, the warp's barrier and its phase.
struct TmaRing {
  float* ring;             // [kMegoPerCall][32 P] floats
  uint64_t* bar;
  const CUtensorMap* map;  // in the kernel's parameter space
  uint32_t parity;
  bool ok;                 // false once a window copy missed its bounded wait
};

// One window: 32 P consecutive weights from w[x] (x a multiple of 32, so
// the copy starts on a 128-byte boundary) into shared memory, completing
// on `bar` (1-D tensor copy through the TMA unit).
__device__ __forceinline__ void tma_window(float* dst, const CUtensorMap* map, uint32_t x,
                                           uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2}], [%3];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(smem_addr(bar))
      : "memory");
}

// Bounds-checked builds (-DMEGO_BOUNDS_CHECK): every weight or state index a
// chain forms is checked against n before it is used (for a window of
// consecutive loads, its last index); a bad one is recorded in the fault
// word (kFaultIndex) and replaced by 0, so nothing is read out of range.
// The normal build compiles these checks away.
__device__ __forceinline__ uint32_t checked(const Problem& a, uint32_t j, uint32_t span = 0u) {
#ifdef MEGO_BOUNDS_CHECK
  if (j + span >= a.n || j + span < j) {
    if (a.fault) atomicOr(a.fault, kFaultIndex);
    return 0u;
  }
#else
  (void)a;
  (void)span;
#endif
  return j;
}

// Per-warp table of the 32 iterations of the current offset window:
// (wrapped partition base of the warp's first segment, offset o^(b)).
constexpr int kMaxWarps = 8;

// Largest CTA a kernel with P particles per thread is compiled for.  Six
// chains per thread (Megopolis) need ~160 registers; a 128-thread bound lets
// the compiler use them and still fit three CTAs per SM.
constexpr int max_threads_for(int P) { return P == 6 ? 128 : 256; }

// Resident CTAs per SM the single-resample kernel's register allocation must
// allow (the second __launch_bounds__ argument): three for six chains per
// thread (up to 168 registers), pinned so that the short-chain path added to
// the kernel cannot move the allocation of the long-chain loop; measured
// faster than four CTAs of 128 registers on 2^20 weights at B = 356.
constexpr int min_ctas_single(int P) { return P == 6 ? 3 : 1; }

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

// w[x0 + off] with the constant off added to the pointer, not to the 32-bit
// index: the address of (w + x0) is formed once per x0 and each constant off
// becomes the load's immediate offset.  (An index sum x0 + off in 32 bits may
// wrap, so the compiler would form a separate 64-bit address for each off.)
template <bool SMEM>
__device__ __forceinline__ float ldw_at(const float* __restrict__ w, uint32_t x0, uint32_t off) {
  if constexpr (SMEM) {
    return (reinterpret_cast<const float*>(g_dyn_smem) + x0)[off];
  } else {
    return __ldg((w + x0) + off);
  }
}

// Stage w[0, n) into dynamic shared memory.  Returns false (uniformly for the
// CTA) if the bulk copy did not complete within the poll budget
// a.stage_polls (kMaxPolls by default, about two seconds of polling with
// back-off); the CTA then records the fault and waits again, with the full
// budget, for the copies it issued to land before it leaves, so no copy
// writes into shared memory that the SM has handed to another CTA.  (Should
// that second wait also expire, the memory system itself has stopped; the
// CTA leaves with the fault recorded.)
__device__ __forceinline__ bool stage_weights(const Problem& a) {
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
  const bool done = mbar_wait_bounded(&bar, 0u, a.stage_polls);
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
__device__ __forceinline__ void finish_batch(const Problem& a, uint32_t ibase,
                                             const uint32_t (&k_in)[P],
                                             const bool (&live)[P]) {
  uint32_t k[P];
#pragma unroll
  for (int p = 0; p < P; ++p) k[p] = live[p] ? checked(a, k_in[p]) : k_in[p];
#pragma unroll
  for (int p = 0; p < P; ++p)
    if (live[p] && a.anc) (a.anc + ibase)[32u * p] = static_cast<int32_t>(k[p]);
  if constexpr (GATHER == kGatherSoa) {
    // Rows in rounds of three: all of a round's random loads are in flight
    // before its stores (x_out never overlaps x_in, so the order is free),
    // one memory latency per three rows instead of one per row.
    constexpr int kRows = 3;
    for (int d0 = 0; d0 < a.dim; d0 += kRows) {
      float v[kRows][P];
#pragma unroll
      for (int dd = 0; dd < kRows; ++dd) {
        if (d0 + dd < a.dim) {
          const float* src = a.x_in + static_cast<int64_t>(d0 + dd) * a.ld;
#pragma unroll
          for (int p = 0; p < P; ++p) v[dd][p] = live[p] ? __ldg(src + k[p]) : 0.0f;
        }
      }
#pragma unroll
      for (int dd = 0; dd < kRows; ++dd) {
        if (d0 + dd < a.dim) {
          float* dst = a.x_out + static_cast<int64_t>(d0 + dd) * a.ld;
#pragma unroll
          for (int p = 0; p < P; ++p)
            if (live[p]) (dst + ibase)[32u * p] = v[dd][p];
        }
      }
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
      if (live[p]) (dst + ibase)[32u * p] = v[p];
  }
}

// Column of one Megopolis iteration for a lane: x0 = base + (lane + o) mod 32,
// where (base, o) is the iteration's table entry.  Segment p of the batch
// reads index x0 + 32 p, reduced modulo n (wrap_index) where it may run past
// n.
__device__ __forceinline__ uint32_t mego_column(int2 e, uint32_t lane) {
  return static_cast<uint32_t>(e.x) + ((lane + static_cast<uint32_t>(e.y)) & 31u);
}

__device__ __forceinline__ uint32_t wrap_index(uint32_t j, uint32_t n) {
  if (j >= n) j -= n;
  if (j >= n) j %= n;
  return j;
}

// The same reduction for the short-chain path, where the choice is made once
// per launch: a batch forms indices j < n + 32 P (a column is below n + 32
// and a batch adds at most 32 (P - 1)), so for n >= 32 P one conditional
// subtraction suffices (SMALL = false) and only n < 32 P needs the division.
template <bool SMALL>
__device__ __forceinline__ uint32_t wrap_small(uint32_t j, uint32_t n) {
  if constexpr (SMALL) {
    return j % n;
  } else {
    return j >= n ? j - n : j;
  }
}

// Loads of one Megopolis iteration for the P segments of a batch when the
// partitions may run past n: each index is reduced modulo n.
template <int P, bool SMEM>
__device__ __forceinline__ void mego_wrapped_loads(const Problem& a, uint32_t x0,
                                                   float (&wj)[P]) {
#pragma unroll
  for (int p = 0; p < P; ++p) wj[p] = ldw<SMEM>(a.w, checked(a, wrap_index(x0 + 32u * p, a.n)));
}

// ---------------------------------------------------------------------------
// Megopolis (Algorithm 5).  Iteration b, particle i = 32 s + lane:
//   j = (32 s + o_al + (lane + o) mod 32) mod n,  o_al = o - o mod 32.
// The warp reads one aligned 32-weight partition per segment and iteration.
// Iterations run in groups of five (one Philox call per particle and group).
// The warp's table holds 32 consecutive offsets: each lane draws the offset of
// one iteration and stores (wrapped base of the warp's first segment, offset);
// the table is refilled every six groups (30 iterations), so a group never
// straddles two tables.  A ballot marks the iterations whose P partitions do
// not run past n, so the common case loads at x0 + 32 p with immediate
// offsets.  A chain keeps the column x0 of its last accepted proposal (its
// index less 32 p, before the reduction modulo n); the ancestor is that
// column plus 32 p, reduced once after the last iteration.
//
// TMA (the window path): for a group whose five windows do not run past n,
// lane 0 fetches the five 32 P-weight windows into the warp's ring by TMA
// before the generator runs, and the lanes read their rotated columns from
// shared memory after it; other groups load directly.
template <int P, bool SMEM, int GATHER, bool TMA = false>
__device__ __forceinline__ void megopolis_batch(const Problem& a, const RoundKeys& K, int B,
                                                uint32_t s0, uint32_t seg_hi,
                                                uint32_t lane, int2* win,
                                                TmaRing* tr = nullptr) {
  const uint32_t n = a.n;
  const uint32_t ibase = s0 * 32u + lane;
  float wk[P];
  uint32_t kx[P];  // column of the current state: ancestor = (kx + 32 p) mod n
  bool live[P];
  PhiloxLane ph[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint32_t i = ibase + 32u * p;
    live[p] = (s0 + p < seg_hi) && (i < n);
    wk[p] = ldw<SMEM>(a.w, i < n ? i : n - 1u);
    kx[p] = ibase;
    ph[p].init(i, kTagMegoU, K, a.S);
  }
  constexpr int U = kMegoPerCall;
  constexpr uint32_t kFull = (1u << U) - 1u;
  uint32_t fast_mask = 0u;
  int t0 = 32;  // position of iteration b0 in the table; 32 forces a refill
  uint32_t g = 0u;
  for (int b0 = 0; b0 < B; b0 += U, ++g, t0 += U) {
    if (t0 + U > 32) {
      const uint32_t o = mego_offset(K, a.S, static_cast<uint32_t>(b0) + lane, n);
      uint32_t base = s0 * 32u + (o & ~31u);
      base = base >= n ? base - n : base;
      // TMA: a tensor copy must also start on a 16-byte boundary (base a
      // multiple of 4 weights); a base wrapped modulo a ragged n may not be.
      fast_mask = __ballot_sync(0xFFFFFFFFu,
                                base + 32u * P <= n && (!TMA || (base & 3u) == 0u));
      __syncwarp();
      win[lane] = make_int2(static_cast<int>(base), static_cast<int>(o));
      __syncwarp();
      t0 = 0;
    }
    uint32_t mh, ml;
    PhiloxLane::group(g, a.S, mh, ml);
    float wj[U][P];
    uint32_t x0[U];
    if (B - b0 >= U) {
      // A full group of five iterations.
#pragma unroll
      for (int q = 0; q < U; ++q) x0[q] = mego_column(win[t0 + q], lane);
      bool fast = ((fast_mask >> t0) & kFull) == kFull;
      if constexpr (TMA) {
        // Every window copy in bounds and 16-byte aligned, checked again from
        // the table itself (the same entries for every lane: uniform).
#pragma unroll
        for (int q = 0; q < U; ++q) {
          const uint32_t x = static_cast<uint32_t>(win[t0 + q].x);
          fast = fast && (x & 3u) == 0u && x + 32u * P <= n;
        }
      }
      if (fast) {
        if constexpr (TMA) {
          if (lane == 0) {
            // The ring's previous reads (generic proxy) before these writes.
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(tr->bar, static_cast<uint32_t>(U) * 32u * P * 4u);
#pragma unroll
            for (int q = 0; q < U; ++q)
              tma_window(tr->ring + q * 32 * P, tr->map, static_cast<uint32_t>(win[t0 + q].x),
                         tr->bar);
          }
        } else {
#pragma unroll
          for (int q = 0; q < U; ++q) {
            const uint32_t xq = checked(a, x0[q], 32u * (P - 1));
#pragma unroll
            for (int p = 0; p < P; ++p) wj[q][p] = ldw_at<SMEM>(a.w, xq, 32u * p);
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < U; ++q) mego_wrapped_loads<P, SMEM>(a, x0[q], wj[q]);
      }
      uint4 r[P];
#pragma unroll
      for (int p = 0; p < P; ++p) r[p] = ph[p].gen(mh, ml, K);
      if constexpr (TMA) {
        if (fast) {
          if (!mbar_wait_bounded(tr->bar, tr->parity, kMaxPolls)) {
            // Record the miss, let the copies land before the ring is
            // abandoned, and write nothing for this batch.
            tr->ok = false;
            if (lane == 0) mbar_wait_bounded(tr->bar, tr->parity, kMaxPolls);
            __syncwarp();
            return;
          }
          tr->parity ^= 1u;
#pragma unroll
          for (int q = 0; q < U; ++q) {
            const uint32_t off = x0[q] - static_cast<uint32_t>(win[t0 + q].x);
#pragma unroll
            for (int p = 0; p < P; ++p) wj[q][p] = tr->ring[q * 32 * P + off + 32u * p];
          }
          __syncwarp();  // every lane has read the ring before it is refilled
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const bool acc = accept(u_of(mego_word(r[p], q)), wk[p], wj[q][p]);
          wk[p] = acc ? wj[q][p] : wk[p];
          kx[p] = acc ? x0[q] : kx[p];
        }
      }
    } else {
      // Tail: 1..4 iterations (words 0..3 of the call).
      const int nb = B - b0;
#pragma unroll
      for (int q = 0; q < U - 1; ++q) {
        if (q < nb) {
          x0[q] = mego_column(win[t0 + q], lane);
          mego_wrapped_loads<P, SMEM>(a, x0[q], wj[q]);
        }
      }
      uint4 r[P];
#pragma unroll
      for (int p = 0; p < P; ++p) r[p] = ph[p].gen(mh, ml, K);
#pragma unroll
      for (int q = 0; q < U - 1; ++q) {
        if (q < nb) {
#pragma unroll
          for (int p = 0; p < P; ++p) {
            const bool acc = accept(u_of(word_of(r[p], q)), wk[p], wj[q][p]);
            wk[p] = acc ? wj[q][p] : wk[p];
            kx[p] = acc ? x0[q] : kx[p];
          }
        }
      }
    }
  }
  uint32_t k[P];
#pragma unroll
  for (int p = 0; p < P; ++p) k[p] = wrap_index(kx[p] + 32u * p, n);
  finish_batch<P, GATHER>(a, ibase, k, live);
}

// ---------------------------------------------------------------------------
// Megopolis for short chains, B <= kShortB (the first 30 iterations fit one
// offset table, so it is filled once per batch and never refilled).  The
// offsets depend only on (seed, stream, b, n), not on the batch: each lane
// keeps o^(lane) in a register (OffsetWindow) for all the batches a warp runs
// on one problem, so only the first batch runs the generator for them; a
// later batch recomputes just the bases.  Loads take the immediate-offset
// path whenever none of the iterations' partitions runs past n, the tail
// group included, and the index reduction modulo n is chosen per launch
// (wrap_small).  Same results as megopolis_batch, bit for bit.
constexpr int kShortB = 30;

struct OffsetWindow {
  uint32_t o;   // o^(lane) of the first window (iterations 0..31)
  bool valid;
};

template <int P, bool SMEM, int GATHER, bool SMALL>
__device__ __forceinline__ void megopolis_short(const Problem& a, const RoundKeys& K, int B,
                                                uint32_t s0, uint32_t seg_hi,
                                                uint32_t lane, int2* win, OffsetWindow& ow) {
  const uint32_t n = a.n;
  const uint32_t ibase = s0 * 32u + lane;
  float wk[P];
  uint32_t kx[P];
  bool live[P];
  PhiloxLane ph[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint32_t i = ibase + 32u * p;
    live[p] = (s0 + p < seg_hi) && (i < n);
    wk[p] = ldw<SMEM>(a.w, i < n ? i : n - 1u);
    kx[p] = ibase;
    ph[p].init(i, kTagMegoU, K, a.S);
  }
  if (!ow.valid) {  // warp-uniform
    ow.o = mego_offset(K, a.S, lane, n);
    ow.valid = true;
  }
  const uint32_t o = ow.o;
  uint32_t base = s0 * 32u + (o & ~31u);
  base = base >= n ? base - n : base;
  const uint32_t fast_mask = __ballot_sync(0xFFFFFFFFu, base + 32u * P <= n);
  __syncwarp();
  win[lane] = make_int2(static_cast<int>(base), static_cast<int>(o));
  __syncwarp();
  constexpr int U = kMegoPerCall;
  uint32_t g = 0u;
  for (int b0 = 0; b0 < B; b0 += U, ++g) {
    uint32_t mh, ml;
    PhiloxLane::group(g, a.S, mh, ml);
    const int nb = B - b0 < U ? B - b0 : U;
    const uint32_t need = (1u << nb) - 1u;
    const bool fast = ((fast_mask >> b0) & need) == need;
    float wj[U][P];
    uint32_t x0[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (q < nb) {
        x0[q] = mego_column(win[b0 + q], lane);
        if (fast) {
          const uint32_t xq = checked(a, x0[q], 32u * (P - 1));
#pragma unroll
          for (int p = 0; p < P; ++p) wj[q][p] = ldw_at<SMEM>(a.w, xq, 32u * p);
        } else {
#pragma unroll
          for (int p = 0; p < P; ++p)
            wj[q][p] = ldw<SMEM>(a.w, checked(a, wrap_small<SMALL>(x0[q] + 32u * p, n)));
        }
      }
    }
    uint4 r[P];
#pragma unroll
    for (int p = 0; p < P; ++p) r[p] = ph[p].gen(mh, ml, K);
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (q < nb) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const bool acc = accept(u_of(mego_word(r[p], q)), wk[p], wj[q][p]);
          wk[p] = acc ? wj[q][p] : wk[p];
          kx[p] = acc ? x0[q] : kx[p];
        }
      }
    }
  }
  uint32_t k[P];
#pragma unroll
  for (int p = 0; p < P; ++p) k[p] = wrap_small<SMALL>(kx[p] + 32u * p, n);
  finish_batch<P, GATHER>(a, ibase, k, live);
}

// ---------------------------------------------------------------------------
// Metropolis (Algorithm 2): independent j ~ U{0, n-1} per particle and
// iteration; two iterations per Philox call.
template <int P, bool SMEM, int GATHER>
__device__ __forceinline__ void metropolis_batch(const Problem& a, const RoundKeys& K, int B,
                                                 uint32_t s0, uint32_t seg_hi,
                                                 uint32_t lane) {
  const uint32_t n = a.n;
  const uint32_t ibase = s0 * 32u + lane;
  float wk[P];
  uint32_t k[P];
  bool live[P];
  PhiloxLane ph[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint32_t i = ibase + 32u * p;
    live[p] = (s0 + p < seg_hi) && (i < n);
    k[p] = i < n ? i : n - 1u;
    wk[p] = ldw<SMEM>(a.w, k[p]);
    ph[p].init(i, kTagMetro, K, a.S);
  }
  for (int b0 = 0; b0 < B; b0 += 2) {
    const int nb = (B - b0) < 2 ? (B - b0) : 2;
    uint32_t mh, ml;
    PhiloxLane::group(static_cast<uint32_t>(b0) >> 1, a.S, mh, ml);
    uint4 r[P];
#pragma unroll
    for (int p = 0; p < P; ++p) r[p] = ph[p].gen(mh, ml, K);
    float wj[2][P];
    uint32_t jj[2][P];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (q < nb) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          jj[q][p] = checked(a, index32(q == 0 ? r[p].x : r[p].z, n));
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
__device__ __forceinline__ void partition_batch(const Problem& a, const RoundKeys& K, int B,
                                                uint32_t s0, uint32_t seg_hi,
                                                uint32_t lane) {
  const uint32_t n = a.n;
  const uint32_t ibase = s0 * 32u + lane;
  float wk[P];
  uint32_t k[P];
  bool live[P];
  uint32_t part[P];
  PhiloxLane ph[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint32_t i = ibase + 32u * p;
    live[p] = (s0 + p < seg_hi) && (i < n);
    k[p] = i < n ? i : n - 1u;
    wk[p] = ldw<SMEM>(a.w, k[p]);
    ph[p].init(i, kTagCDraw, K, a.S);
    part[p] = 0u;
    if constexpr (VARIANT == kC1) {
      const uint4 x = philox4x32_10(s0 + p, 0u, a.S.sid, kTagCPart, K);
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
        const uint4 x = philox4x32_10(s0 + lane % P, bb + 1u, a.S.sid, kTagCPart, K);
        part_reg = index64(x.x, x.y, a.npart);
      }
    }
    uint32_t mh, ml;
    PhiloxLane::group(static_cast<uint32_t>(b0) >> 1, a.S, mh, ml);
    uint4 r[P];
#pragma unroll
    for (int p = 0; p < P; ++p) r[p] = ph[p].gen(mh, ml, K);
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
          jj[q][p] = checked(a, pp * a.nw + index32(q == 0 ? r[p].x : r[p].z, a.nw));
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
// The chains of whole batches [seg_lo, seg_hi) of one problem for one warp.
template <int VARIANT, int P, bool SMEM, int GATHER, bool SHORT = true>
__device__ __forceinline__ void run_segments(const Problem& a, const RoundKeys& K, int B,
                                             uint32_t seg_lo, uint32_t seg_hi, uint32_t lane,
                                             int2* win, OffsetWindow& ow) {
  if constexpr (VARIANT == kMegopolis) {
    if (SHORT && B <= kShortB) {  // uniform for the problem
      // n < 32 P: a batch's indices may pass 2n and need the division.
      if (a.n < 32u * P) {
        for (uint32_t s0 = seg_lo; s0 < seg_hi; s0 += P)
          megopolis_short<P, SMEM, GATHER, true>(a, K, B, s0, seg_hi, lane, win, ow);
      } else {
        for (uint32_t s0 = seg_lo; s0 < seg_hi; s0 += P)
          megopolis_short<P, SMEM, GATHER, false>(a, K, B, s0, seg_hi, lane, win, ow);
      }
    } else {
      for (uint32_t s0 = seg_lo; s0 < seg_hi; s0 += P)
        megopolis_batch<P, SMEM, GATHER>(a, K, B, s0, seg_hi, lane, win);
    }
    return;
  }
  for (uint32_t s0 = seg_lo; s0 < seg_hi; s0 += P) {
    if constexpr (VARIANT == kMetropolis) {
      metropolis_batch<P, SMEM, GATHER>(a, K, B, s0, seg_hi, lane);
    } else {
      partition_batch<VARIANT, P, SMEM, GATHER>(a, K, B, s0, seg_hi, lane);
    }
  }
}

template <int VARIANT, int P, bool SMEM, int GATHER>
__global__ void __launch_bounds__(max_threads_for(P), min_ctas_single(P))
resample_kernel(const __grid_constant__ ResampleArgs a) {
  __shared__ int2 s_win[kMaxWarps][32];
  grid_dependency_wait();  // inputs (weights, a device-side B) written by the predecessor
  const int B = a.B_dev ? *a.B_dev : a.B;
  if (B < 0) return;  // device-side bound failed: write nothing
  if constexpr (SMEM) {
    if (!stage_weights(a.p)) return;
  }
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t wpb = blockDim.x >> 5;
  const uint64_t gw = static_cast<uint64_t>(blockIdx.x) * wpb + (threadIdx.x >> 5);
  const uint64_t tw = static_cast<uint64_t>(gridDim.x) * wpb;
  // Whole batches of P segments per warp, in equal contiguous ranges.
  const uint64_t nbat = (a.p.nseg + P - 1u) / P;
  const uint32_t seg_lo = static_cast<uint32_t>(nbat * gw / tw) * P;
  uint32_t seg_hi = static_cast<uint32_t>(nbat * (gw + 1u) / tw) * P;
  if (seg_hi > a.p.nseg) seg_hi = a.p.nseg;
  OffsetWindow ow{0u, false};
  run_segments<VARIANT, P, SMEM, GATHER>(a.p, a.K, B, seg_lo, seg_hi, lane,
                                         s_win[threadIdx.x >> 5], ow);
}

// Megopolis on the TMA window path (global weights): as resample_kernel, with
// each warp's windows fetched by TMA into a shared-memory ring.  A window
// copy that misses its bounded wait marks the fault word and the warp stops.
template <int P, int GATHER>
__global__ void __launch_bounds__(max_threads_for(P), min_ctas_single(P))
resample_tma_kernel(const __grid_constant__ ResampleArgs a) {
  constexpr int W = max_threads_for(P) / 32;
  __shared__ int2 s_win[kMaxWarps][32];
  __shared__ __align__(128) float s_ring[W][kMegoPerCall * 32 * P];
  __shared__ __align__(8) uint64_t s_bar[W];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t wi = threadIdx.x >> 5;
  if (lane == 0) mbar_init(&s_bar[wi], 1u);
  __syncwarp();
  grid_dependency_wait();  // inputs (weights, a device-side B) written by the predecessor
  const int B = a.B_dev ? *a.B_dev : a.B;
  if (B < 0) return;
  const uint32_t wpb = blockDim.x >> 5;
  const uint64_t gw = static_cast<uint64_t>(blockIdx.x) * wpb + wi;
  const uint64_t tw = static_cast<uint64_t>(gridDim.x) * wpb;
  const uint64_t nbat = (a.p.nseg + P - 1u) / P;
  const uint32_t seg_lo = static_cast<uint32_t>(nbat * gw / tw) * P;
  uint32_t seg_hi = static_cast<uint32_t>(nbat * (gw + 1u) / tw) * P;
  if (seg_hi > a.p.nseg) seg_hi = a.p.nseg;
  TmaRing tr{s_ring[wi], &s_bar[wi], &a.tmap, 0u, true};
  for (uint32_t s0 = seg_lo; s0 < seg_hi; s0 += P) {
    megopolis_batch<P, false, GATHER, true>(a.p, a.K, B, s0, seg_hi, lane, s_win[wi], &tr);
    if (!tr.ok) {
      if (lane == 0 && a.p.fault) atomicExch(a.p.fault, kFaultStageTimeout);
      break;
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
  bool tma;  // Megopolis TMA window path (ppt 4 or 6)
};

// Host-side count of kernel launches (capi.cu), reported by mego_launch_count.
void count_launches(uint64_t k);

// Host helpers (capi.cu): round keys of a seed, constants of a stream.
RoundKeys make_round_keys(uint64_t seed);
StreamKey make_stream_key(const RoundKeys& K, uint32_t sid);

// Opt a kernel in to the largest dynamic shared-memory size it can use
// (the per-block opt-in limit minus its static shared memory), once per
// device and kernel.  Defined in capi.cu.
cudaError_t enable_large_smem(const void* kernel);

template <int VARIANT>
cudaError_t launch_resample(const LaunchShape& s, int gather, const ResampleArgs& a,
                            cudaStream_t stream);

template <int VARIANT>
const void* resample_kernel_ptr(int ppt, bool smem, int gather);

// The TMA window path (Megopolis only; defined in resample_megopolis.cu).
cudaError_t launch_resample_tma(const LaunchShape& s, int gather, const ResampleArgs& a,
                                cudaStream_t stream);
const void* resample_tma_kernel_ptr(int ppt, int gather);
// Tensor map of w[0, n) as a 1-D float tensor with a box of 32 ppt weights
// (capi.cu); false if the driver cannot encode it.
bool encode_window_map(CUtensorMap* map, const float* w, uint32_t n, int ppt);

// Device address of the variant's fault word (for the current device).
template <int VARIANT>
int32_t* resample_fault_word();

}  // namespace mego
