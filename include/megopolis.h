/*
 * megopolis.h -- C ABI of libmegopolis.so, GB300 (sm_103a) resampling.
 *
 * Metropolis-style resampling of a float32 weight vector into int32
 * ancestor indices, after "The Megopolis Resampler: Memory Coalesced
 * Resampling on GPUs" (arXiv 2109.13504):
 *   - Megopolis (Algorithm 5, Section 4): iteration b proposes, for particle
 *     i, j = (i_aligned + o_aligned + (i + o^(b)) mod 32) mod N with one
 *     offset o^(b) shared by every particle;
 *   - Metropolis (Algorithm 2, Section 3): an independent uniform j per
 *     particle and iteration (the baseline);
 *   - Metropolis-C1 / -C2 (Algorithms 3, 4, Section 3.1): j uniform inside a
 *     partition of P_size bytes chosen per warp once (C1) or per iteration
 *     (C2).
 * Every variant accepts j when fl(u * w_k) <= w_j (u in (0,1], binary32,
 * round to nearest), the division-free form of u <= w_j / w_k.
 *
 * Random numbers: Philox4x32-10 keyed by `seed`, counters carry the
 * particle, the iteration, `stream_id` and a per-purpose tag.  Ancestors are
 * a pure function of (weight bits, n, B, seed, stream_id, variant, P_size):
 * they do not depend on the launch shape, the memory path or the stream.
 *
 * Conventions for every entry point:
 *   - Pointers prefixed d_ are device pointers, h_ host pointers.  The caller
 *     owns every buffer; nothing here allocates device memory, and nothing
 *     keeps a pointer after the call returns (work is queued on `stream`).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Argument errors are detected on the host and returned synchronously;
 *     nothing is launched then.  Errors found on the device (bad weights,
 *     a bound beyond its cap) are written to a caller-provided int32 status
 *     word, read with mego_sync_status.  Nothing calls abort() or exit().
 *   - Weights need not be normalised (Section 7; Section 8).
 *   - n >= 1 and n <= MEGO_N_MAX; 0 <= B <= MEGO_B_MAX.
 */
#ifndef MEGOPOLIS_H
#define MEGOPOLIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MEGO_ABI_VERSION 4
#define MEGO_N_MAX (1 << 30)
#define MEGO_B_MAX (1 << 24)

typedef enum mego_status {
  MEGO_OK = 0,
  MEGO_EINVAL = 1,    /* bad argument; nothing was launched              */
  MEGO_ENOMEM = 2,    /* caller workspace too small                       */
  MEGO_ECUDA = 3,     /* a CUDA runtime call failed                       */
  MEGO_ETIMEOUT = 4,  /* mego_sync_status: deadline passed                */
  MEGO_EWEIGHTS = 5   /* device: NaN/Inf/negative or all-zero weights,
                         weights so large that a partial sum leaves the
                         float range (about 1e32 and above), or B above
                         the cap                                          */
} mego_status;

typedef enum mego_variant {
  MEGO_MEGOPOLIS = 0,
  MEGO_METROPOLIS = 1,
  MEGO_METROPOLIS_C1 = 2,
  MEGO_METROPOLIS_C2 = 3
} mego_variant;

typedef enum mego_layout {
  MEGO_LAYOUT_SOA = 0,  /* x[d * ld + i], d < dim                         */
  MEGO_LAYOUT_AOS4 = 1  /* four floats per particle, x[4 * i + c]; 16-byte
                           aligned; one 128-bit load and store per particle */
} mego_layout;

typedef enum mego_path {
  MEGO_PATH_AUTO = 0,
  MEGO_PATH_GLOBAL = 1, /* weights read from L2/HBM with coalesced loads  */
  MEGO_PATH_SMEM = 2,   /* weights staged whole in shared memory by a bulk
                           async copy; needs 4n bytes <= the CTA's limit  */
  MEGO_PATH_TMA = 3     /* Megopolis only, ppt 4 or 6, n >= 64 ppt, d_w
                           16-byte aligned: each warp fetches the five
                           32 ppt-weight windows of a group of iterations
                           by 1-D TMA tensor copies into shared memory
                           (measured slower than MEGO_PATH_GLOBAL on GB300:
                           the chains are bound by arithmetic, not reads) */
} mego_path;

/* Launch shape.  Any field 0 selects the library's choice.  The result
 * never depends on these. */
typedef struct mego_launch_cfg {
  int32_t threads;      /* CTA size, a multiple of 32 in [64, 256]
                           ([64, 128] with ppt 6)                            */
  int32_t ppt;          /* particles per thread, 1, 2, 4, 6 (Megopolis
                           only) or 8 (each a 32-particle segment of one
                           warp)                                             */
  int32_t path;         /* mego_path                                         */
  int32_t ctas_per_sm;  /* resident CTAs per SM to aim for                   */
} mego_launch_cfg;

/* ABI version (MEGO_ABI_VERSION) and a static text for a status code. */
int mego_abi_version(void);
const char* mego_status_string(int status);

/* ----------------------------------------------------------------------
 * Resample (Algorithm 5 or Algorithm 2), B given by the host.  variant is
 * MEGO_MEGOPOLIS or MEGO_METROPOLIS; C1/C2 need a partition size and go
 * through mego_resample_gather.
 *   d_w      [n] float32, finite and >= 0 (not checked here; use
 *            mego_compute_B to validate).  Read-only.
 *   B        number of iterations, 0 <= B <= MEGO_B_MAX; B = 0 gives
 *            ancestors equal to the particle index.
 *   d_anc    [n] int32 output, must not overlap d_w.
 * Returns MEGO_EINVAL for a null pointer, n out of range, B out of range,
 * an unknown variant or overlapping buffers; MEGO_ECUDA if the launch fails.
 */
mego_status mego_resample(const float* d_w, int32_t n, int32_t B, uint64_t seed,
                          uint32_t stream_id, int variant, int32_t* d_anc,
                          void* stream);

/* ----------------------------------------------------------------------
 * Resample and gather particle state by ancestor: x_out^(i) = x_in^(k)
 * (last line of Algorithms 2 and 5).
 *   B / d_B      if d_B is non-NULL the iteration count is read on the
 *                device from *d_B (as written by mego_compute_B); a value
 *                < 0 there means "bound failed" and the kernel writes
 *                nothing.  Otherwise the host value B is used.
 *   psize_bytes  P_size for C1/C2 (a multiple of 4 with P_size/4 dividing
 *                n); ignored by the other variants.
 *   d_x_in/out   state, layout mego_layout; SoA: dim rows of stride ld >= n
 *                floats; AoS4: dim must be 4, ld ignored, both 16-byte
 *                aligned.  May both be NULL (no gather).  Must not overlap.
 *   d_anc        [n] int32 output; may be NULL when gathering.
 *   cfg          launch shape, or NULL.
 */
mego_status mego_resample_gather(const float* d_w, int32_t n, int32_t B,
                                 const int32_t* d_B, uint64_t seed,
                                 uint32_t stream_id, int variant,
                                 uint32_t psize_bytes, const float* d_x_in,
                                 float* d_x_out, int32_t dim, int64_t ld,
                                 int layout, int32_t* d_anc,
                                 const mego_launch_cfg* cfg, void* stream);

/* ----------------------------------------------------------------------
 * Iteration bound, Eq. 3 (Section 3) and Proposition 1 (Eq. 4):
 *   B = ceil(log(eps) / log(1 - E(w)/max(w)))
 * with E(w) the sample mean (compensated float-float sums inside each CTA,
 * double across CTAs, in a fixed order) and max(w) the sample maximum.
 * eps in (0, 1].  E(w) = max(w) or eps = 1 gives B = 0.
 *   d_B       [1] int32 output: B, or -1 on a device-side error.
 *   d_status  [1] int32 output: MEGO_OK, or MEGO_EWEIGHTS when a weight is
 *             NaN, infinite or negative, all weights are 0, a CTA's partial
 *             sum leaves the float range (weights of about 1e32 or more), or
 *             B > b_max.
 *   d_q       [1] double output, the value before the ceiling; may be NULL.
 *   b_max     cap on B, 0 < b_max <= MEGO_B_MAX.
 *   d_ws      caller workspace of at least mego_workspace_bytes(n) bytes,
 *             256-byte aligned; its contents need no initialisation.
 * Two kernels, no host synchronisation: graph-capturable.
 */
size_t mego_workspace_bytes(int32_t n);
mego_status mego_compute_B(const float* d_w, int32_t n, double eps,
                           int32_t b_max, int32_t* d_B, int32_t* d_status,
                           double* d_q, void* d_ws, size_t ws_bytes,
                           void* stream);

/* ----------------------------------------------------------------------
 * The iteration bound with no workspace argument and no allocation, for
 * callers that cannot allocate device memory: for example a host
 * application that hands out every byte of device memory from its own pool,
 * or a real-time loop that must not call the allocator once it is running
 * (cudaMalloc may synchronise the device and takes unbounded time).  The
 * paper has no counterpart; this is a library convenience.
 * Same inputs, outputs and device-side status as mego_compute_B, and the
 * same values bit for bit: the reduction runs the same grid and adds the
 * same partials in the same order.  Its partial results go to a fixed
 * 16 KiB array inside the library (1024 partials, the most the reduction
 * grid ever uses; every GPU that loads the library keeps it until exit).
 * The first call on a device looks up that array's device address, so make
 * that first call before any stream capture; resetting the device
 * (cudaDeviceReset) while the library is loaded is not supported, since the
 * address is kept for the life of the process.  All calls share the array:
 * calls whose work overlaps on the GPU (other streams, other threads) race
 * and may return a wrong B; order them on one stream.  Nothing in the array
 * needs to start at zero.  n above MEGO_N_MAX is rejected with MEGO_EINVAL;
 * any n up to it fits.
 */
mego_status mego_compute_B_noalloc(const float* d_w, int32_t n, double eps,
                                   int32_t b_max, int32_t* d_B,
                                   int32_t* d_status, double* d_q,
                                   void* stream);

/* ----------------------------------------------------------------------
 * Likelihood weights fused with the bound: w_i = exp(-(x_i - y)^2 / 2)
 * from row 0 of an SoA state (Eq. 12 without its constant factor, the
 * update of Algorithm 1), then B as in mego_compute_B.
 *   d_x   state row 0, [n] float32 (row 0 of an SoA array).
 *   d_w   [n] float32 output weights.
 * Other arguments as in mego_compute_B.  expf is CUDA's single-precision
 * exponential; it can differ from a double-precision evaluation by a few
 * units in the last place.
 */
mego_status mego_likelihood_B(const float* d_x, int32_t n, float y, double eps,
                              int32_t b_max, float* d_w, int32_t* d_B,
                              int32_t* d_status, double* d_q, void* d_ws,
                              size_t ws_bytes, void* stream);

/* ----------------------------------------------------------------------
 * End-to-end call on host buffers (for callers without device memory
 * management of their own): copies h_w to d_w, computes B (if B < 0, from
 * eps) and the ancestors, copies them to h_anc and B to *h_B, and waits for
 * the stream.  d_w [n] float32, d_anc [n] int32, d_ws (see above) and a
 * 16-byte device scalar area d_scalars (>= 32 bytes) are caller-provided
 * device buffers.  Host buffers should be page-locked for full copy speed.
 * Returns MEGO_EWEIGHTS if the bound failed on the device.
 */
mego_status mego_resample_host(const float* h_w, int32_t n, int32_t B,
                               double eps, uint64_t seed, uint32_t stream_id,
                               int variant, int32_t* h_anc, int32_t* h_B,
                               float* d_w, int32_t* d_anc, void* d_scalars,
                               void* d_ws, size_t ws_bytes, void* stream);

/* ----------------------------------------------------------------------
 * Batched resampling: many independent problems ("filters") of uneven size
 * in one persistent launch.  (The paper resamples one filter at a time; the
 * batch runs Algorithm 5 or Algorithm 2 on each filter unchanged.)
 *
 * One seed per batch; each filter has its own stream id, so a filter's
 * ancestors equal those of mego_resample_gather with the same seed, stream
 * id and B, whatever else is in the batch.
 *
 * Plan: mego_batch_plan copies per-filter descriptors and work-item tables
 * into a caller-provided device buffer of mego_batch_plan_bytes() bytes
 * (256-byte aligned) and fills the host handle *out.  Filters' buffers are
 * the caller's and must stay valid while the plan is used.  A plan must not
 * be launched twice concurrently (its work queue is shared).
 * Bound: mego_batch_bound computes each filter's B (Eq. 3) into the plan
 * (out->d_B, out->d_status, out->d_q: int32, int32, double per filter);
 * filters whose descriptor has B < 0 use it.  Resample: one persistent
 * kernel, warps taking (filter, 128-particle) work items from a queue.
 * Graph: mego_batch_graph captures [bound (if eps > 0)] + resample into a
 * CUDA graph held by the handle (needs a non-default stream); replay with
 * mego_batch_launch_graph; mego_batch_destroy releases it.
 * Only MEGO_MEGOPOLIS and MEGO_METROPOLIS; the global-memory path; all
 * filters of a batch gather with the same layout, or none does.
 */
typedef struct mego_filter {
  const float* w;      /* [n] weights (device)                                */
  int32_t* anc;        /* [n] ancestors (device), may be NULL when gathering  */
  const float* x_in;   /* state in the batch layout (device) or NULL          */
  float* x_out;        /* gathered state (device) or NULL                     */
  int64_t ld;          /* SoA row stride in floats (>= n)                     */
  int32_t n;           /* 1..MEGO_N_MAX                                       */
  int32_t B;           /* iterations, or < 0 for the batch bound's value      */
  uint32_t stream_id;  /* random stream of this filter                        */
  int32_t dim;         /* SoA rows to gather; 4 for AoS4                      */
  const float* w_host; /* optional: the weights in page-locked host memory.
                          The batched bound then reads them from here (over
                          the CPU-GPU link, once) and writes the device copy
                          w that the resample reads, so no separate upload
                          is needed; mego_batch_bound must then run before
                          every mego_batch_resample.  NULL: w is read.         */
} mego_filter;

typedef struct mego_batch {
  void* d_plan;
  size_t plan_bytes;
  int32_t count, variant, layout, gather;
  uint64_t seed;
  uint64_t total_items, total_chunks;
  int32_t* d_B;        /* [count] per-filter bound (device, inside the plan)  */
  int32_t* d_status;   /* [count] per-filter status                           */
  double* d_q;         /* [count] per-filter value before the ceiling         */
  mego_launch_cfg cfg; /* threads and particles per thread of the launch      */
  int32_t grid;
  void* graph_exec;    /* captured graph, or NULL                             */
  int32_t graph_kernels; /* kernels in the captured graph                     */
  /* Shared-memory phase (ABI 4): filters of at most smem_max_n weights are
   * resampled whole by one CTA each, their weights staged once in shared
   * memory, before the warp-level queue takes the other filters' items
   * (0: no such phase).  Set by mego_batch_set_smem or mego_batch_autotune. */
  int32_t smem_max_n;
  int32_t smem_filters; /* filters in the shared-memory phase                 */
  size_t smem_bytes;    /* dynamic shared memory per CTA of the launch        */
  /* The caller's filter array given to mego_batch_plan; mego_batch_set_smem
   * and mego_batch_autotune re-plan from it, so it must stay valid (and
   * unchanged) while they may be called. */
  const mego_filter* h_filters;
} mego_batch;

size_t mego_batch_plan_bytes(const mego_filter* h_filters, int32_t count);
mego_status mego_batch_plan(const mego_filter* h_filters, int32_t count,
                            int variant, int layout, uint64_t seed,
                            void* d_plan, size_t plan_bytes, mego_batch* out,
                            void* stream);
mego_status mego_batch_bound(const mego_batch* b, double eps, int32_t b_max,
                             void* stream);
mego_status mego_batch_resample(const mego_batch* b, void* stream);
/* Shape of the persistent launch (threads 64..256, particles per thread
 * 1, 2, 4 or 6 -- 6 for Megopolis only, with threads <= 128); the grid is
 * always SMs x resident CTAs.  A work item is 6 segments for a Megopolis
 * batch whose filters of >= 2^17 particles hold most of the work, else 4; it
 * is fixed in the plan, and the plan's default shape takes one item per warp
 * batch.  Any shape gives the same results. */
mego_status mego_batch_set_shape(mego_batch* b, int32_t threads, int32_t ppt);
/* Shared-memory phase threshold: re-plan (in the same plan buffer, on
 * `stream`) so that filters of at most smem_max_n weights are resampled by
 * one CTA each from shared memory.  0 turns the phase off; the maximum is
 * what fits the device's shared memory per CTA (about 56K weights on this
 * part), larger values give MEGO_EINVAL.  Keeps the launch shape and the
 * per-filter B, status and q of a previous bound.  A filter whose staging
 * copy does not land within the bounded wait is skipped and gets status
 * MEGO_ETIMEOUT.  Any threshold gives the same results. */
mego_status mego_batch_set_smem(mego_batch* b, int32_t smem_max_n, void* stream);
/* Time every launch shape (threads x particles per thread) and every
 * shared-memory threshold in {0, 4096, 16384, 49152} (those the device
 * allows) on the batch as planned (outputs are overwritten), and keep the
 * fastest pair.  The loop over iterations is not a knob: one generator call
 * serves five iterations (the Megopolis uniforms), so the chain always
 * advances five iterations per step. */
mego_status mego_batch_autotune(mego_batch* b, int32_t reps, float* best_ms,
                                void* stream);
mego_status mego_batch_graph(mego_batch* b, double eps, int32_t b_max,
                             void* stream);
mego_status mego_batch_launch_graph(const mego_batch* b, void* stream);
mego_status mego_batch_destroy(mego_batch* b);

/* ----------------------------------------------------------------------
 * Serving: a continuous-batching request loop (a library service; the paper
 * has no serving system).  One worker thread admits queued requests in FIFO
 * order while their device buffers (40 n bytes each: weights, ancestors, and
 * AoS4 state in and out) fit in the caller's arena -- the device-memory
 * budget -- and sends every admitted request through one batched launch
 * (bound + Megopolis/Metropolis + gather) on a free stream of its own, with
 * the uploads and the copies of the results to the request's host buffers
 * on the same stream.  Requests arriving while batches run join the next
 * batch, so work from different arrivals overlaps on the GPU.  A request is
 * resampled with the server's seed and stream id = (uint32) id, so its
 * result equals mego_resample_gather with that seed and stream id (B from
 * the bound) whatever it was batched with.  Host buffers of a request must
 * stay valid until its completion is polled; page-locked buffers copy fastest.
 */
typedef struct mego_request {
  uint64_t id;          /* request id; its low 32 bits are the stream id      */
  const float* h_w;     /* [n] weights (host)                                 */
  const float* h_x;     /* [n][4] state (host), or NULL if the server has none */
  int32_t* h_anc;       /* [n] ancestors out (host), or NULL                  */
  float* h_x_out;       /* [n][4] gathered state out (host), or NULL          */
  int32_t n;
} mego_request;

typedef struct mego_completion {
  uint64_t id;
  int32_t status;       /* MEGO_OK; MEGO_EWEIGHTS when the bound rejected this
                           request's weights (B = -1: no resample ran for it
                           and its output buffers hold no result); or the
                           error that failed the batch                        */
  int32_t n;
  int64_t latency_ns;   /* from submission to the results being on the host   */
  int32_t B;            /* iterations the bound gave this request (Eq. 3), or
                           -1 where it failed; a client can order its next
                           submissions by it (longest first)                  */
  int32_t reserved;
} mego_completion;

typedef struct mego_server_cfg {
  void* d_arena;        /* device memory budget (256-byte aligned, caller's)  */
  size_t arena_bytes;
  uint64_t seed;
  double eps;           /* bound of Eq. 3 per request                          */
  int32_t variant;      /* MEGO_MEGOPOLIS or MEGO_METROPOLIS                   */
  int32_t max_batch;    /* requests per batch (0: 256)                        */
  int32_t streams;      /* batches in flight (0: 2)                           */
  int32_t threads, ppt; /* batch launch shape (0: default)                    */
  int32_t poll_us;      /* worker poll interval while busy (0: 5 us)          */
  int32_t with_state;   /* 1: every request carries AoS4 state; 0: none does  */
  int32_t host_copies;  /* 0: inputs are uploaded by the copy engine;
                           results go straight into page-locked host buffers
                           (the resample writes ancestors and gathered state
                           over the CPU-GPU link), others are copied back.
                           1: copies both ways.  2: as 0, and the bound also
                           reads page-locked weights in place.               */
} mego_server_cfg;

typedef struct mego_server_stats_t {
  uint64_t batches, max_batch, peak_arena_bytes, queued, inflight;
} mego_server_stats_t;

typedef struct mego_server mego_server;

mego_status mego_server_create(const mego_server_cfg* cfg, mego_server** out);
/* Queue a request (non-blocking).  MEGO_ENOMEM if it can never fit the
 * arena; MEGO_EINVAL if its state does not match with_state. */
mego_status mego_server_submit(mego_server* s, const mego_request* r);
/* Move up to max_out completions to out; returns how many. */
int32_t mego_server_poll(mego_server* s, mego_completion* out, int32_t max_out);
/* Wait until nothing is queued or running (MEGO_ETIMEOUT after timeout_s). */
mego_status mego_server_drain(mego_server* s, double timeout_s);
mego_status mego_server_stats(mego_server* s, mego_server_stats_t* out);
mego_status mego_server_destroy(mego_server* s);
/* Submit reqs[k] at t_arrival[k] seconds after the call (open-loop arrival
 * schedule, busy-waiting between arrivals), then drain. */
mego_status mego_server_replay(mego_server* s, const mego_request* reqs,
                               const double* t_arrival, int32_t count,
                               double timeout_s);

/* ----------------------------------------------------------------------
 * Stages of the modified SIR filter around the resampler (Algorithm 6,
 * model of Eqs. 22-23).
 * mego_sir_predict_update: for each particle i,
 *   x_pred[i] = x[i]/2 + 25 x[i]/(1 + x[i]^2) + drift + v[i]
 *   w[i]      = exp(-(z - x_pred[i]^2 / 20)^2 / 2)
 * with drift = 8 cos(1.2 t) and v the process noise (both from the caller),
 * z the measurement.  Binary32 operations in that order, no contraction;
 * expf within 2 ulp.  d_x, d_v, d_x_pred, d_w: [n] float32 (device).
 * mego_mean: the estimate, mean of d_x[0, n), into *d_out (double), with a
 * deterministic reduction in a caller workspace of
 * mego_mean_workspace_bytes() bytes (8-byte aligned).
 */
mego_status mego_sir_predict_update(const float* d_x, const float* d_v, int32_t n,
                                    float drift, float z, float* d_x_pred,
                                    float* d_w, void* stream);
size_t mego_mean_workspace_bytes(void);
mego_status mego_mean(const float* d_x, int32_t n, double* d_out, void* d_ws,
                      size_t ws_bytes, void* stream);

/* ----------------------------------------------------------------------
 * Wait for `stream` up to timeout_s seconds by polling an event, then copy
 * the device status word to *h_status.  Returns MEGO_ETIMEOUT (and leaves
 * *h_status untouched) if the stream has not drained by the deadline. */
mego_status mego_sync_status(const int32_t* d_status, void* stream,
                             double timeout_s, int32_t* h_status);

/* ----------------------------------------------------------------------
 * Autotuner: time every launch shape (threads 64/128/256 x particles per
 * thread 1/2/4/8 x global/shared-memory path) on the given buffers, `reps`
 * timed runs each after one warm-up, and remember the fastest for this
 * device, variant, gather layout, floor(log2 n) and floor(log2 B); later
 * calls with cfg == NULL (host or device B) use it.  Arguments as in
 * mego_resample_gather (B from the host).  Synchronises `stream`; overwrites
 * d_anc / d_x_out.  *best and *best_ms (may be NULL) receive the winner.
 * Shapes the library rejects (weights too large for shared memory) are
 * skipped.  Results depend only on the inputs, never on the shape chosen.
 */
mego_status mego_autotune(const float* d_w, int32_t n, int32_t B, int variant,
                          uint32_t psize_bytes, const float* d_x_in,
                          float* d_x_out, int32_t dim, int64_t ld, int layout,
                          int32_t* d_anc, int32_t reps, mego_launch_cfg* best,
                          float* best_ms, void* stream);

/* ----------------------------------------------------------------------
 * Device faults of the resample kernels: the shared-memory path waits for
 * its bulk copy of the weights with a bounded number of polls; if the copy
 * has not landed by then, the CTA records a fault (1) and writes nothing.
 * The TMA window path records 1 the same way.  A library built with
 * -DMEGO_BOUNDS_CHECK also checks every index the chains form against n and
 * records an out-of-range one as 2 (using index 0 instead).
 * *h_fault receives the OR of the recorded faults since the last call
 * (0: none), and the record is cleared.  Synchronises the device.
 */
mego_status mego_device_fault(int32_t* h_fault);

/* Diagnostics (not part of the method): the number of polls the
 * shared-memory path's first staging wait makes before it gives up, for
 * resample calls queued after this one (host-wide setting).  polls < 0
 * restores the default, 2^21 polls with back-off (about two seconds); a
 * budget of 0 makes every staging wait expire at once, so a test can check
 * the fault report without a fault: the CTA records fault 1, still waits
 * with the full budget for its own copy to land, and writes nothing.
 * polls above the default: MEGO_EINVAL.
 */
mego_status mego_set_stage_poll_budget(int64_t polls);

/* ----------------------------------------------------------------------
 * Measurement helper (not part of the method): read `bytes` of d_buf
 * `reps` times with coalesced 128-bit loads, writing one float per CTA to
 * d_sink (at least four floats per SM) so the reads are not elided.  Used to
 * measure the L2 bandwidth that bounds the global-memory path when d_buf is
 * smaller than L2.  bytes must be a multiple of 16 and d_buf 16-byte
 * aligned.
 */
mego_status mego_probe_read(const void* d_buf, size_t bytes, int32_t reps,
                            float* d_sink, void* stream);

/* Kernel launches the library queued since the process started (host-side
 * count; lets a caller confirm that the CUDA path ran). */
uint64_t mego_launch_count(void);

/* Size in bytes of the public structs, for bindings that mirror them:
 * which = 0 mego_launch_cfg, 1 mego_filter, 2 mego_batch, 3 mego_request,
 * 4 mego_completion, 5 mego_server_cfg, 6 mego_server_stats_t; 0 otherwise.
 * Host only. */
size_t mego_struct_size(int32_t which);

#ifdef __cplusplus
}
#endif

#endif /* MEGOPOLIS_H */
