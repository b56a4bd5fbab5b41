/*
 * megopolis_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * A plain, slow, single-threaded CPU restatement of what the resampling hot
 * path computes, written from the paper ("The Megopolis Resampler: Memory
 * Coalesced Resampling on GPUs", arXiv 2109.13504).  It exists only so that
 * the tests, the smoke check and the benchmark's CPU-baseline leg can check
 * and time the CUDA path against it.  It shares no code, header, table or
 * constant generator with the CUDA path; the product never loads it.
 *
 * Build flags: -O2 -ffp-contract=off, no fast-math.  Every float operation
 * below is a single IEEE-754 binary32 operation rounded to nearest-even with
 * no contraction, so the acceptance test is bit-reproducible.
 *
 * Contents, each following one passage of the paper:
 *   - Philox4x32-10 (Salmon et al., SC'11), the counter-based generator that
 *     stands in for the paper's cuRAND XORWOW (Section 5, implementation
 *     details).  Written from the published round definition.
 *   - The u and integer mappings, which the paper leaves unstated
 *     (Section 2.1 notation; Algorithms 2 and 5 draw u ~ U[0,1]).
 *   - Metropolis resampling, Algorithm 2 (Section 3).
 *   - Megopolis resampling, Algorithm 5 (Section 4): offsets first, then the
 *     per-particle chain with the aligned/unaligned index.
 *   - Metropolis-C1 and -C2, Algorithms 3 and 4 (Section 3.1).
 *   - The iteration bound B, Eq. 3 (Section 3) and Proposition 1 (Eq. 4).
 *   - The ancestor gather (last step of Algorithms 2 and 5).
 *   - The Gaussian likelihood weight of Eq. 12 without its constant factor.
 *   - The predict/update and estimate stages of the modified SIR filter
 *     (Algorithm 6, model of Eqs. 22-23).
 *
 * Parity status: every function here is pinned by a CPU test against
 * something other than itself (a library routine, a closed form, an exact
 * Markov-chain computation or the paper's printed tables), except
 * oracle_likelihood and the SIR stages, whose pins are their closed forms
 * evaluated by the tests in double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* Status codes (same numeric meaning as the C-ABI's, defined here on their
 * own so that the oracle includes no product header).                      */
enum {
  ORC_OK = 0,
  ORC_EINVAL = 1,
  ORC_ENOMEM = 2,
  ORC_EWEIGHTS = 5
};

/* Variant numbering used by the tests (mirrors the C-ABI's enum values). */
enum { ORC_MEGOPOLIS = 0, ORC_METROPOLIS = 1, ORC_C1 = 2, ORC_C2 = 3 };

/* Counter tags: the fourth counter word separates the random streams. */
enum {
  TAG_OFFSET = 1,   /* Megopolis offsets o^(b)                       */
  TAG_MEGO_U = 2,   /* Megopolis acceptance uniforms                 */
  TAG_METRO = 3,    /* Metropolis (j, u) pairs                        */
  TAG_C_PART = 4,   /* C1/C2 per-warp partition choice               */
  TAG_C_DRAW = 5    /* C1/C2 per-particle (j-in-partition, u) pairs  */
};

/* ---------------------------------------------------------------------- */
/* Philox4x32-10.  State (c0,c1,c2,c3), key (k0,k1).  One round maps
 *   (c0,c1,c2,c3) -> (hi(B*c2)^c1^k0, lo(B*c2), hi(A*c0)^c3^k1, lo(A*c0))
 * with multipliers A = 0xD2511F53, B = 0xCD9E8D57, and the key is bumped by
 * the Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds.            */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  int round;
  for (round = 0; round < 10; ++round) {
    uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)pb;
    uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)pa;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

static void draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t sid,
                 uint32_t tag, uint32_t out[4]) {
  uint32_t ctr[4];
  uint32_t key[2];
  ctr[0] = c0;
  ctr[1] = c1;
  ctr[2] = sid;
  ctr[3] = tag;
  key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
  key[1] = (uint32_t)(seed >> 32);
  oracle_philox4x32_10(ctr, key, out);
}

/* u in (0,1]: one 32-bit word -> 2 - f, f = 1.m in [1,2) whose 23-bit
 * fraction m is the word's top 23 bits (bits 9..31; bits 0..8 are not
 * read).  2 - f is exact (Sterbenz), so u takes the 2^23 values k*2^-23,
 * k = 1..2^23, uniformly.  (0,1] rather than [0,1): u = 0 would accept a
 * zero-weight proposal from a positive-weight state, and u > 1 would reject
 * an equal-weight proposal.                                               */
float oracle_u_from_word(uint32_t word) {
  uint32_t bits = 0x3F800000u | (word >> 9);
  float f;
  memcpy(&f, &bits, sizeof f);
  return 2.0f - f;
}

/* U{0, n-1} from 64 random bits: floor(x * n / 2^64).  Exact for n a power
 * of two; otherwise each value has probability within n/2^64 of 1/n.      */
static uint32_t uniform_index64(uint32_t lo, uint32_t hi, uint32_t n) {
  /* (hi*2^32 + lo) * n / 2^64 = (hi*n + floor(lo*n / 2^32)) / 2^32 */
  uint64_t t = ((uint64_t)lo * (uint64_t)n) >> 32;
  uint64_t s = (uint64_t)hi * (uint64_t)n + t;
  return (uint32_t)(s >> 32);
}

/* U{0, n-1} from 32 random bits: floor(x * n / 2^32).  Exact for n a power
 * of two; otherwise within n/2^32 relative of 1/n.                         */
static uint32_t uniform_index32(uint32_t x, uint32_t n) {
  return (uint32_t)(((uint64_t)x * (uint64_t)n) >> 32);
}

/* o^(b) ~ U{0, N-1}, the b-th Megopolis offset (Algorithm 5, first loop). */
uint32_t oracle_offset(uint64_t seed, uint32_t sid, uint32_t b, uint32_t n) {
  uint32_t x[4];
  draw(seed, b, 0u, sid, TAG_OFFSET, x);
  return uniform_index64(x[0], x[1], n);
}

/* The uniform u that particle i uses at Megopolis iteration b.  Five
 * consecutive iterations share one Philox call, the one for counter
 * (i, floor(b/5), sid, TAG_MEGO_U).  With q = b mod 5: q < 4 uses word q;
 * q = 4 uses the word whose bytes 1, 2 and 3 are the least significant
 * bytes of words 0, 1 and 2 (byte 0 is not read).  The u mapping reads
 * only the top 23 bits of a word (bits 9..31), so the five uniforms of a
 * call are built from disjoint bits.                                       */
float oracle_megopolis_u(uint64_t seed, uint32_t sid, uint32_t i, uint32_t b) {
  uint32_t x[4];
  uint32_t q = b % 5u;
  draw(seed, i, b / 5u, sid, TAG_MEGO_U, x);
  if (q < 4u) return oracle_u_from_word(x[q]);
  return oracle_u_from_word(((x[0] & 0xFFu) << 8) | ((x[1] & 0xFFu) << 16) |
                            ((x[2] & 0xFFu) << 24));
}

/* Proposal and uniform for Metropolis particle i at iteration b: two
 * iterations share one Philox call for counter (i, floor(b/2), sid,
 * TAG_METRO); even b uses words (0,1), odd b words (2,3): j from the first
 * word of the pair, u from the second.                                    */
void oracle_metropolis_draw(uint64_t seed, uint32_t sid, uint32_t i,
                            uint32_t b, uint32_t n, uint32_t* j, float* u) {
  uint32_t x[4];
  uint32_t h = (b & 1u) * 2u;
  draw(seed, i, b >> 1, sid, TAG_METRO, x);
  *j = uniform_index32(x[h], n);
  *u = oracle_u_from_word(x[h + 1u]);
}

/* The Megopolis proposal index of Algorithm 5:
 *   i_aligned   = i - (i mod 32)
 *   o_aligned   = o - (o mod 32)
 *   o_unaligned = (i + o) mod 32
 *   j = (i_aligned + o_aligned + o_unaligned) mod N                        */
uint32_t oracle_megopolis_index(uint32_t i, uint32_t o, uint32_t n) {
  uint64_t i_aligned = (uint64_t)i - (uint64_t)(i % 32u);
  uint64_t o_aligned = (uint64_t)o - (uint64_t)(o % 32u);
  uint64_t o_unaligned = ((uint64_t)i + (uint64_t)o) % 32u;
  return (uint32_t)((i_aligned + o_aligned + o_unaligned) % (uint64_t)n);
}

/* Acceptance test of Algorithms 2-5, u <= w_j / w_k, restated without the
 * division as fl(u * w_k) <= w_j (binary32 product, rounded to nearest). */
static int accept(float u, float wk, float wj) {
  float t = u * wk;
  return t <= wj;
}

static int check_common(const float* w, uint32_t n, int32_t B,
                        uint32_t i0, uint32_t i1, const int32_t* anc) {
  if (w == NULL || anc == NULL) return ORC_EINVAL;
  if (n < 1u || n > 0x40000000u) return ORC_EINVAL;
  if (B < 0) return ORC_EINVAL;
  if (i0 > i1 || i1 > n) return ORC_EINVAL;
  return ORC_OK;
}

/* Megopolis resampling, Algorithm 5, for particles i in [i0, i1).
 * anc[i - i0] receives the ancestor index k of particle i.               */
int oracle_megopolis(const float* w, uint32_t n, int32_t B, uint64_t seed,
                     uint32_t sid, uint32_t i0, uint32_t i1, int32_t* anc) {
  uint32_t* o;
  uint32_t i;
  int32_t b;
  int st = check_common(w, n, B, i0, i1, anc);
  if (st != ORC_OK) return st;
  /* Algorithm 5, first loop: draw all B offsets before resampling. */
  o = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(B > 0 ? B : 1));
  if (o == NULL) return ORC_ENOMEM;
  for (b = 0; b < B; ++b) o[b] = oracle_offset(seed, sid, (uint32_t)b, n);
  /* Algorithm 5, second loop: one chain per particle. */
  for (i = i0; i < i1; ++i) {
    uint32_t k = i;
    for (b = 0; b < B; ++b) {
      uint32_t j = oracle_megopolis_index(i, o[b], n);
      float u = oracle_megopolis_u(seed, sid, i, (uint32_t)b);
      if (accept(u, w[k], w[j])) k = j;
    }
    anc[i - i0] = (int32_t)k;
  }
  free(o);
  return ORC_OK;
}

/* Metropolis resampling, Algorithm 2, for particles i in [i0, i1). */
int oracle_metropolis(const float* w, uint32_t n, int32_t B, uint64_t seed,
                      uint32_t sid, uint32_t i0, uint32_t i1, int32_t* anc) {
  uint32_t i;
  int32_t b;
  int st = check_common(w, n, B, i0, i1, anc);
  if (st != ORC_OK) return st;
  for (i = i0; i < i1; ++i) {
    uint32_t k = i;
    for (b = 0; b < B; ++b) {
      uint32_t j;
      float u;
      oracle_metropolis_draw(seed, sid, i, (uint32_t)b, n, &j, &u);
      if (accept(u, w[k], w[j])) k = j;
    }
    anc[i - i0] = (int32_t)k;
  }
  return ORC_OK;
}

/* Metropolis-C1 / -C2, Algorithms 3 and 4, for particles i in [i0, i1).
 * psize_bytes is P_size; N_w = P_size/4 weights per partition and
 * N_part = 4N / P_size partitions, which requires N_w | N.  The warp of
 * particle i is floor(i / 32).  The partition p is drawn once per warp
 * (C1: counter (warp, 0, sid, TAG_C_PART), 64-bit index) or once per warp
 * and iteration (C2: counter (warp, b + 1, sid, TAG_C_PART)).  The index
 * inside the partition and u come from counter (i, floor(b/2), sid,
 * TAG_C_DRAW), split like the Metropolis pair.                            */
int oracle_metropolis_c(const float* w, uint32_t n, int32_t B, uint64_t seed,
                        uint32_t sid, uint32_t psize_bytes, int variant,
                        uint32_t i0, uint32_t i1, int32_t* anc) {
  uint32_t i, nw, npart;
  int32_t b;
  int st = check_common(w, n, B, i0, i1, anc);
  if (st != ORC_OK) return st;
  if (variant != ORC_C1 && variant != ORC_C2) return ORC_EINVAL;
  if (psize_bytes < 4u || psize_bytes % 4u != 0u) return ORC_EINVAL;
  nw = psize_bytes / 4u;
  if (n % nw != 0u) return ORC_EINVAL;
  npart = n / nw;
  for (i = i0; i < i1; ++i) {
    uint32_t k = i;
    uint32_t warp = i / 32u;
    uint32_t x[4];
    uint32_t p = 0;
    if (variant == ORC_C1) {
      draw(seed, warp, 0u, sid, TAG_C_PART, x);
      p = uniform_index64(x[0], x[1], npart);
    }
    for (b = 0; b < B; ++b) {
      uint32_t y[4];
      uint32_t h = ((uint32_t)b & 1u) * 2u;
      uint32_t j;
      float u;
      if (variant == ORC_C2) {
        draw(seed, warp, (uint32_t)b + 1u, sid, TAG_C_PART, x);
        p = uniform_index64(x[0], x[1], npart);
      }
      draw(seed, i, (uint32_t)b >> 1, sid, TAG_C_DRAW, y);
      j = p * nw + uniform_index32(y[h], nw);
      u = oracle_u_from_word(y[h + 1u]);
      if (accept(u, w[k], w[j])) k = j;
    }
    anc[i - i0] = (int32_t)k;
  }
  return ORC_OK;
}

/* Dispatch on variant (psize only used by C1/C2). */
int oracle_resample(const float* w, uint32_t n, int32_t B, uint64_t seed,
                    uint32_t sid, int variant, uint32_t psize_bytes,
                    uint32_t i0, uint32_t i1, int32_t* anc) {
  switch (variant) {
    case ORC_MEGOPOLIS:
      return oracle_megopolis(w, n, B, seed, sid, i0, i1, anc);
    case ORC_METROPOLIS:
      return oracle_metropolis(w, n, B, seed, sid, i0, i1, anc);
    case ORC_C1:
    case ORC_C2:
      return oracle_metropolis_c(w, n, B, seed, sid, psize_bytes, variant, i0,
                                 i1, anc);
    default:
      return ORC_EINVAL;
  }
}

/* Run the resampler for seeds seed0 .. seed0+nseeds-1 on all n particles and
 * accumulate counts[i*n + k] += 1 whenever particle i ends at ancestor k.
 * Used for the exact small-N distribution checks.                          */
int oracle_ancestor_counts(const float* w, uint32_t n, int32_t B,
                           uint64_t seed0, uint64_t nseeds, uint32_t sid,
                           int variant, uint32_t psize_bytes,
                           uint64_t* counts) {
  uint64_t s;
  int32_t* anc;
  if (counts == NULL || n < 1u) return ORC_EINVAL;
  anc = (int32_t*)malloc(sizeof(int32_t) * n);
  if (anc == NULL) return ORC_ENOMEM;
  for (s = 0; s < nseeds; ++s) {
    uint32_t i;
    int st = oracle_resample(w, n, B, seed0 + s, sid, variant, psize_bytes, 0u,
                             n, anc);
    if (st != ORC_OK) {
      free(anc);
      return st;
    }
    for (i = 0; i < n; ++i) counts[(uint64_t)i * n + (uint32_t)anc[i]] += 1u;
  }
  free(anc);
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Weight statistics and the iteration bound.
 * Eq. 3 (and Proposition 1, Eq. 4): B = ceil(log(eps) / log(1 - E(w)/w_p))
 * with E(w) the mean weight and w_p = max(w).  Here E(w) and w_p are the
 * sample mean and the sample maximum of the given w, the sum taken in
 * double in index order.  Weights must be finite and >= 0 with at least one
 * positive weight; otherwise ORC_EWEIGHTS.  r = E(w)/w_p = 1 (all equal)
 * gives B = 0: every chain is already at the target.                       */
int oracle_reduce(const float* w, uint32_t n, float* wmax, double* wsum) {
  uint32_t i;
  float m = 0.0f;
  double s = 0.0;
  int bad = 0;
  if (w == NULL || n < 1u) return ORC_EINVAL;
  for (i = 0; i < n; ++i) {
    float v = w[i];
    if (!(v >= 0.0f) || isinf(v)) bad = 1; /* NaN, negative or infinite */
    if (v > m) m = v;
    s += (double)v;
  }
  if (wmax) *wmax = m;
  if (wsum) *wsum = s;
  if (bad || !(m > 0.0f)) return ORC_EWEIGHTS;
  return ORC_OK;
}

int oracle_compute_B(const float* w, uint32_t n, double eps, int32_t b_max,
                     int32_t* B_out, double* q_out) {
  float m;
  double s, r, q;
  int st;
  if (B_out == NULL) return ORC_EINVAL;
  if (!(eps > 0.0 && eps <= 1.0)) return ORC_EINVAL;
  st = oracle_reduce(w, n, &m, &s);
  if (st != ORC_OK) return st;
  r = (s / (double)n) / (double)m;
  if (r >= 1.0) {
    q = 0.0;
  } else {
    q = log(eps) / log1p(-r);
  }
  if (q_out) *q_out = q;
  q = ceil(q);
  if (q < 0.0) q = 0.0;
  if (q > (double)b_max) return ORC_EWEIGHTS;
  *B_out = (int32_t)q;
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Ancestor gather, x_bar^(i) = x^(k) (last line of Algorithms 2-5).
 * SoA: x[d*ld + i] for d < dim.  AoS4: four floats per particle.          */
int oracle_gather_soa(const float* x_in, float* x_out, const int32_t* anc,
                      uint32_t n, uint32_t dim, uint64_t ld) {
  uint32_t d, i;
  if (!x_in || !x_out || !anc || ld < n) return ORC_EINVAL;
  for (d = 0; d < dim; ++d)
    for (i = 0; i < n; ++i)
      x_out[(uint64_t)d * ld + i] = x_in[(uint64_t)d * ld + (uint32_t)anc[i]];
  return ORC_OK;
}

int oracle_gather_aos4(const float* x_in, float* x_out, const int32_t* anc,
                       uint32_t n) {
  uint32_t i, c;
  if (!x_in || !x_out || !anc) return ORC_EINVAL;
  for (i = 0; i < n; ++i)
    for (c = 0; c < 4u; ++c)
      x_out[(uint64_t)i * 4u + c] = x_in[(uint64_t)(uint32_t)anc[i] * 4u + c];
  return ORC_OK;
}

/* Gaussian likelihood weight against observation y, Eq. 12 without the
 * constant 1/sqrt(2 pi) (resampling ignores a common scale):
 *   w_i = exp(-(x_i - y)^2 / 2), evaluated in double, rounded once.       */
void oracle_likelihood(const float* x, uint32_t n, float y, float* w) {
  uint32_t i;
  for (i = 0; i < n; ++i) {
    double d = (double)x[i] - (double)y;
    w[i] = (float)exp(-0.5 * d * d);
  }
}

/* ---------------------------------------------------------------------- */
/* Modified SIR filter stages (Algorithm 6; model of Eqs. 22-23).
 * Predict: x' = x/2 + 25 x/(1 + x^2) + drift + v, drift = 8 cos(1.2 t) and v
 * the process noise (inputs); the paper computes in single precision, and
 * this restatement uses binary32 operations in a fixed order (no
 * contraction).  Update: w = exp(-(z - x'^2/20)^2 / 2), the exponential in
 * double and rounded once.                                                */
void oracle_sir_predict_update(const float* x, const float* v, uint32_t n, float drift,
                               float z, float* x_pred, float* w) {
  uint32_t i;
  for (i = 0; i < n; ++i) {
    float xi = x[i];
    float den = 1.0f + xi * xi;
    float frac = (25.0f * xi) / den;
    float xp = 0.5f * xi + frac;
    float d, a;
    xp = xp + drift;
    xp = xp + v[i];
    d = z - (xp * xp) / 20.0f;
    a = 0.5f * (d * d);
    x_pred[i] = xp;
    w[i] = (float)exp(-(double)a);
  }
}

/* Estimate of Algorithm 6: the mean of the resampled particles (double). */
double oracle_mean(const float* x, uint32_t n) {
  uint32_t i;
  double s = 0.0;
  for (i = 0; i < n; ++i) s += (double)x[i];
  return s / (double)n;
}
