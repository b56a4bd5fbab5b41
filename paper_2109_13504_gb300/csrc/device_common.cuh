// device_common.cuh -- generator, mappings and async-copy helpers for the
// sm_103a resampling kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mego {

// Counter tags (fourth Philox counter word): one random stream per purpose.
constexpr uint32_t kTagOffset = 1u;  // Megopolis offsets o^(b)
constexpr uint32_t kTagMegoU = 2u;   // Megopolis acceptance uniforms
constexpr uint32_t kTagMetro = 3u;   // Metropolis (j, u) pairs
constexpr uint32_t kTagCPart = 4u;   // C1/C2 per-warp partition
constexpr uint32_t kTagCDraw = 5u;   // C1/C2 (j in partition, u) pairs

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (c0,c1,c2,c3) <- (hi(M1 c2) ^ c1 ^ k0, M1 c2, hi(M0 c0) ^ c3 ^ k1, M0 c0)
// with the key advanced by the Weyl increments between rounds.  Loop
// invariant parts (a fixed c0 or c2) are hoisted by the compiler.
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1,
                                               uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t h0 = __umulhi(M0, c0), l0 = M0 * c0;
    const uint32_t h1 = __umulhi(M1, c2), l1 = M1 * c2;
    c0 = h1 ^ c1 ^ k0;
    c1 = l1;
    c2 = h0 ^ c3 ^ k1;
    c3 = l0;
    k0 += W0;
    k1 += W1;
  }
  return make_uint4(c0, c1, c2, c3);
}

// u in (0,1] from the low 23 bits of a word: 2 - 1.m, exact.
__device__ __forceinline__ float u_of(uint32_t word) {
  return __fsub_rn(2.0f, __uint_as_float(0x3F800000u | (word & 0x007FFFFFu)));
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

// Megopolis offset o^(b) ~ U{0, n-1}.
__device__ __forceinline__ uint32_t mego_offset(uint32_t k0, uint32_t k1,
                                                uint32_t sid, uint32_t b,
                                                uint32_t n) {
  const uint4 x = philox4x32_10(b, 0u, sid, kTagOffset, k0, k1);
  return index64(x.x, x.y, n);
}

__device__ __forceinline__ uint32_t word_of(const uint4& x, int q) {
  return q == 0 ? x.x : (q == 1 ? x.y : (q == 2 ? x.z : x.w));
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
enum : int32_t { kFaultNone = 0, kFaultStageTimeout = 1 };

}  // namespace mego
