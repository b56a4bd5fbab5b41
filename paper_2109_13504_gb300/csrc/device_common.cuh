// device_common.cuh -- generator, mappings and async-copy helpers for the
// sm_103a resampling kernels.
#pragma once

#include <cstdint>
#include <utility>

#include <cuda_runtime.h>

namespace mego {

// Counter tags (fourth Philox counter word): one random stream per purpose.
constexpr uint32_t kTagOffset = 1u;  // Megopolis offsets o^(b)
constexpr uint32_t kTagMegoU = 2u;   // Megopolis acceptance uniforms
constexpr uint32_t kTagMetro = 3u;   // Metropolis (j, u) pairs
constexpr uint32_t kTagCPart = 4u;   // C1/C2 per-warp partition
constexpr uint32_t kTagCDraw = 5u;   // C1/C2 (j in partition, u) pairs

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

// Round keys of one launch (one seed), computed on the host: rk0[r] = k0 +
// r W0, rk1[r] = k1 + r W1, the key of round r.  Passed in the kernel
// parameters, so every round reads its key from the constant bank.
struct RoundKeys {
  uint32_t rk0[10];
  uint32_t rk1[10];
};

// Constants of one random stream (counter word c2 = sid) under a seed:
// H = hi(M1 sid) ^ rk0[0], L = lo(M1 sid), the parts of round 0 that do not
// depend on the particle or the iteration.
struct StreamKey {
  uint32_t H, L;
  uint32_t sid;
};

__device__ __forceinline__ uint64_t mulwide(uint32_t a, uint32_t b) {
  return static_cast<uint64_t>(a) * static_cast<uint64_t>(b);
}
__device__ __forceinline__ uint32_t hi32(uint64_t x) { return static_cast<uint32_t>(x >> 32); }
__device__ __forceinline__ uint32_t lo32(uint64_t x) { return static_cast<uint32_t>(x); }

// One Philox4x32 round with key (k0, k1):
//   (c0,c1,c2,c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                             uint32_t& c3, uint32_t k0, uint32_t k1) {
  const uint64_t p0 = mulwide(kPhiloxM0, c0);
  const uint64_t p1 = mulwide(kPhiloxM1, c2);
  c0 = hi32(p1) ^ c1 ^ k0;
  c1 = lo32(p1);
  c2 = hi32(p0) ^ c3 ^ k1;
  c3 = lo32(p0);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, round r
// keyed by (k0 + r W0, k1 + r W1).
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                               uint32_t c3, const RoundKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) philox_round(c0, c1, c2, c3, K.rk0[r], K.rk1[r]);
  return make_uint4(c0, c1, c2, c3);
}

// Philox4x32-10 for the counter family (i, g, sid, tag) with the particle i
// and the tag fixed and g varying.  Everything that depends only on (i, tag)
// -- round 0, the c0/c1 half of round 1 and the c0 product of round 2 -- is
// computed once by init(); the part that depends only on g (the c0 product of
// round 1) is shared by all particles of a thread (group()).  gen() finishes
// the ten rounds.  The output equals philox4x32_10(i, g, sid, tag).
struct PhiloxLane {
  uint32_t x1;    // c3 after round 0, xored with the round-1 key word rk1[1]
  uint32_t c1_2;  // c1 after round 1
  uint32_t h3;    // hi(M0 * c0) in round 2
  uint32_t l3;    // lo(M0 * c0) in round 2 (= c3 after round 2)

  __device__ __forceinline__ void init(uint32_t i, uint32_t tag, const RoundKeys& K,
                                       const StreamKey& S) {
    const uint64_t p0 = mulwide(kPhiloxM0, i);
    const uint32_t c2_1 = hi32(p0) ^ tag ^ K.rk1[0];
    x1 = lo32(p0) ^ K.rk1[1];
    const uint64_t p1 = mulwide(kPhiloxM1, c2_1);
    const uint32_t c0_2 = hi32(p1) ^ S.L ^ K.rk0[1];
    c1_2 = lo32(p1);
    const uint64_t p2 = mulwide(kPhiloxM0, c0_2);
    h3 = hi32(p2);
    l3 = lo32(p2);
  }

  // Shared per g: round-1 c0 product of c0_1 = H ^ g.
  static __device__ __forceinline__ void group(uint32_t g, const StreamKey& S,
                                               uint32_t& mh, uint32_t& ml) {
    const uint64_t m = mulwide(kPhiloxM0, S.H ^ g);
    mh = hi32(m);
    ml = lo32(m);
  }

  __device__ __forceinline__ uint4 gen(uint32_t mh, uint32_t ml, const RoundKeys& K) const {
    // after round 1: (c0_2, c1_2, mh ^ x1, ml); round 2 needs c2_2 = mh ^ x1.
    const uint64_t p = mulwide(kPhiloxM1, mh ^ x1);
    uint32_t c0 = hi32(p) ^ c1_2 ^ K.rk0[2];
    uint32_t c1 = lo32(p);
    uint32_t c2 = h3 ^ ml ^ K.rk1[2];
    uint32_t c3 = l3;
#pragma unroll
    for (int r = 3; r < 10; ++r) philox_round(c0, c1, c2, c3, K.rk0[r], K.rk1[r]);
    return make_uint4(c0, c1, c2, c3);
  }
};

// u in (0,1] from the top 23 bits of a word (bits 9..31): 2 - 1.m, exact.
// The shift-and-or form costs one ALU operation per uniform where a
// mask-and-or of the low bits cost two (ncu pipe counters on the batched
// kernel: 9.70 -> 8.70 ALU instructions per warp-proposal).
__device__ __forceinline__ float u_of(uint32_t word) {
  return __fsub_rn(2.0f, __uint_as_float(0x3F800000u | (word >> 9)));
}

// Acceptance u <= w_j / w_k as fl(u * w_k) <= w_j (no contraction).
__device__ __forceinline__ bool accept(float u, float wk, float wj) {
  return __fmul_rn(u, wk) <= wj;
}

// floor(x * n / 2^64) for x = hi:lo.
__device__ __forceinline__ uint32_t index64(uint32_t lo, uint32_t hi, uint32_t n) {
  const uint64_t t = __umulhi(lo, n);
  return static_cast<uint32_t>((static_cast<uint64_t>(hi) * n + t) >> 32);
}

// floor(x * n / 2^32).
__device__ __forceinline__ uint32_t index32(uint32_t x, uint32_t n) {
  return __umulhi(x, n);
}

// Megopolis offset o^(b) ~ U{0, n-1}: Philox counter (b, 0, sid, 1).
__device__ __forceinline__ uint32_t mego_offset(const RoundKeys& K, const StreamKey& S,
                                                uint32_t b, uint32_t n) {
  const uint4 x = philox4x32_10(b, 0u, S.sid, kTagOffset, K);
  return index64(x.x, x.y, n);
}

// Stream constants for stream id sid (device side).
__device__ __forceinline__ StreamKey stream_key(const RoundKeys& K, uint32_t sid) {
  const uint64_t m = mulwide(kPhiloxM1, sid);
  return StreamKey{hi32(m) ^ K.rk0[0], lo32(m), sid};
}

__device__ __forceinline__ uint32_t word_of(const uint4& x, int q) {
  return q == 0 ? x.x : (q == 1 ? x.y : (q == 2 ? x.z : x.w));
}

// Megopolis draws five uniforms from one Philox call: iteration 5 g + q of
// particle i uses call (i, g, sid, kTagMegoU); q < 4 takes word q (its top 23
// bits, through u_of); q = 4 takes the word whose bytes 1, 2, 3 are the low
// bytes (bits 0-7) of words 0, 1, 2 -- bits no other iteration reads.
constexpr int kMegoPerCall = 5;

__device__ __forceinline__ uint32_t mego_word(const uint4& x, int q) {
  if (q < 4) return word_of(x, q);
  // byte_perm selectors: (x.b0, x.b0, y.b0, x.b0), then (that.b0, that.b1,
  // that.b2, z.b0); u_of reads bytes 1-3 only (bits 1-7 of byte 1).
  return __byte_perm(__byte_perm(x.x, x.y, 0x0400u), x.z, 0x4210u);
}

// ---------------------------------------------------------------------------
// Float-float sums: hi + lo with |lo| <= ulp(hi) / 2, about 48 significant bits
// from binary32 arithmetic alone (this part's FP64 pipe is narrow, its FP32
// pipes are not).  ff_add is Dekker's addition: Knuth's TwoSum of the high
// parts, the low parts and the rounding error added, then Fast2Sum to
// renormalise.  The bound adds only non-negative values, so no cancellation
// degrades it.
struct FloatFloat {
  float hi, lo;
};

// From a compensated pair (s, c) with |c| <= |s|: Fast2Sum.
__device__ __forceinline__ FloatFloat ff_from_pair(float s, float c) {
  const float hi = __fadd_rn(s, c);
  return FloatFloat{hi, __fsub_rn(c, __fsub_rn(hi, s))};
}

__device__ __forceinline__ FloatFloat ff_add(FloatFloat a, FloatFloat b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bv = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
  const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
  return ff_from_pair(s, lo);
}

__device__ __forceinline__ double ff_to_double(FloatFloat a) {
  return static_cast<double>(a.hi) + static_cast<double>(a.lo);
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched with the programmatic
// stream serialization attribute may be scheduled while its predecessor on
// the stream is still running; grid_dependency_wait() returns once the
// predecessor has completed and its writes are visible (immediately when
// there is no such predecessor), so everything that reads the predecessor's
// results comes after it.  grid_launch_dependents() lets the next such kernel
// be scheduled before this one finishes.
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Host: launch `kernel` with programmatic stream serialization (it may be
// scheduled while its predecessor drains; it must call grid_dependency_wait()
// before reading anything the predecessor writes).
template <typename... Params, typename... Args>
cudaError_t launch_after(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem,
                         cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------
// Bulk async copy global -> shared with mbarrier completion (sm_90+ PTX).

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem,
                                         uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0u;
}

// Wait for phase `parity` of the barrier, giving up after max_polls polls
// (with a growing back-off).  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint32_t max_polls) {
  uint32_t ns = 32;
  for (uint32_t it = 0; it < max_polls; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
  }
  return false;
}

// Fault word: set when a bounded wait times out.  Read by mego_sync_status
// callers through the library's own diagnostics.
// kFaultIndex: a bounds-checked build (-DMEGO_BOUNDS_CHECK) met an index
// out of range.
enum : int32_t { kFaultNone = 0, kFaultStageTimeout = 1, kFaultIndex = 2 };

}  // namespace mego
