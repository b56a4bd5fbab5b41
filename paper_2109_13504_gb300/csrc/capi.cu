// capi.cu -- the extern "C" entry points of libmegopolis.so.
//
// Host side only: argument validation, launch-shape selection (memory path,
// particles per thread, grid sized to the SM count times resident CTAs) and
// kernel launches on the caller's stream.  No device allocation.
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <utility>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "../../include/megopolis.h"
#include "bound.cuh"
#include "resample_kernels.cuh"

namespace {

std::atomic<uint64_t> g_launches{0};
// Poll budget of the shared-memory path's first staging wait (diagnostics:
// mego_set_stage_poll_budget).
std::atomic<uint32_t> g_stage_polls{mego::kMaxPolls};

struct DevInfo {
  int sms = 0;
  int smem_optin = 0;
};

bool dev_info(DevInfo* out) {
  static std::mutex mu;
  static std::map<int, DevInfo> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it == cache.end()) {
    DevInfo d;
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return false;
    if (cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
      return false;
    it = cache.emplace(dev, d).first;
  }
  *out = it->second;
  return true;
}

int occupancy(const void* kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, kernel, threads, smem);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int occ = 0;
  if (smem > 0 && mego::enable_large_smem(kernel) != cudaSuccess) {
    cache.emplace(key, 0);
    return 0;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    occ = 0;
  }
  cache.emplace(key, occ);
  return occ;
}

bool overlaps(const void* a, size_t la, const void* b, size_t lb) {
  if (!a || !b || la == 0 || lb == 0) return false;
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + lb && y < x + la;
}

const void* kernel_ptr(int variant, int ppt, bool smem, int gather) {
  switch (variant) {
    case MEGO_MEGOPOLIS: return mego::resample_kernel_ptr<mego::kMegopolis>(ppt, smem, gather);
    case MEGO_METROPOLIS: return mego::resample_kernel_ptr<mego::kMetropolis>(ppt, smem, gather);
    case MEGO_METROPOLIS_C1: return mego::resample_kernel_ptr<mego::kC1>(ppt, smem, gather);
    case MEGO_METROPOLIS_C2: return mego::resample_kernel_ptr<mego::kC2>(ppt, smem, gather);
    default: return nullptr;
  }
}

cudaError_t launch_variant(int variant, const mego::LaunchShape& s, int gather,
                           const mego::ResampleArgs& a, cudaStream_t st) {
  switch (variant) {
    case MEGO_MEGOPOLIS: return mego::launch_resample<mego::kMegopolis>(s, gather, a, st);
    case MEGO_METROPOLIS: return mego::launch_resample<mego::kMetropolis>(s, gather, a, st);
    case MEGO_METROPOLIS_C1: return mego::launch_resample<mego::kC1>(s, gather, a, st);
    case MEGO_METROPOLIS_C2: return mego::launch_resample<mego::kC2>(s, gather, a, st);
    default: return cudaErrorInvalidValue;
  }
}

// Default shape: shared-memory path for small n (the whole vector fits
// comfortably next to other CTAs), more particles per thread as n grows.
mego_status choose_shape(int variant, uint32_t n, int gather, const mego_launch_cfg* cfg,
                         mego::LaunchShape* out) {
  DevInfo di;
  if (!dev_info(&di)) return MEGO_ECUDA;
  const uint32_t nseg = (n + 31u) / 32u;
  int ppt = (cfg && cfg->ppt) ? cfg->ppt : 0;
  if (ppt == 0) {
    // Enough segments per SM for several batches per warp: the widest ILP
    // (Megopolis: six chains per thread in 128-thread CTAs).
    const uint64_t seg_per_sm = nseg / static_cast<uint64_t>(di.sms);
    if (variant == MEGO_MEGOPOLIS && seg_per_sm >= 192)
      ppt = 6;
    else
      ppt = seg_per_sm >= 128 ? 4 : (seg_per_sm >= 32 ? 2 : 1);
  }
  if (ppt != 1 && ppt != 2 && ppt != 4 && ppt != 6 && ppt != 8) return MEGO_EINVAL;
  if (ppt == 6 && variant != MEGO_MEGOPOLIS) return MEGO_EINVAL;
  const int max_threads = ppt == 6 ? 128 : 256;
  int threads = (cfg && cfg->threads) ? cfg->threads : max_threads;
  if (threads < 64 || threads > max_threads || threads % 32) return MEGO_EINVAL;
  const size_t w_bytes = (static_cast<size_t>(n) * 4u + 15u) & ~static_cast<size_t>(15u);
  int path = (cfg && cfg->path) ? cfg->path : MEGO_PATH_AUTO;
  if (path == MEGO_PATH_AUTO)
    path = (w_bytes <= 96u * 1024u) ? MEGO_PATH_SMEM : MEGO_PATH_GLOBAL;
  if (path != MEGO_PATH_SMEM && path != MEGO_PATH_GLOBAL && path != MEGO_PATH_TMA)
    return MEGO_EINVAL;
  const bool tma = path == MEGO_PATH_TMA;
  if (tma && (variant != MEGO_MEGOPOLIS || (ppt != 4 && ppt != 6) ||
              n < 64u * static_cast<uint32_t>(ppt)))
    return MEGO_EINVAL;
  const bool smem = path == MEGO_PATH_SMEM;
  if (smem && w_bytes + 4096u > static_cast<size_t>(di.smem_optin)) return MEGO_EINVAL;
  const size_t smem_bytes = smem ? w_bytes : 0u;
  const void* kp = tma ? mego::resample_tma_kernel_ptr(ppt, gather)
                       : kernel_ptr(variant, ppt, smem, gather);
  if (!kp) return MEGO_EINVAL;
  int occ = occupancy(kp, threads, smem_bytes);
  if (occ < 1) return MEGO_EINVAL;
  if (cfg && cfg->ctas_per_sm > 0 && cfg->ctas_per_sm < occ) occ = cfg->ctas_per_sm;
  const uint64_t warps_needed = (nseg + ppt - 1u) / static_cast<uint64_t>(ppt);
  const uint64_t wpc = static_cast<uint64_t>(threads / 32);
  uint64_t grid = static_cast<uint64_t>(di.sms) * occ;
  const uint64_t ctas_needed = (warps_needed + wpc - 1u) / wpc;
  if (grid > ctas_needed) grid = ctas_needed;
  if (grid < 1u) grid = 1u;
  out->threads = threads;
  out->ppt = ppt;
  out->smem = smem;
  out->grid = static_cast<int>(grid);
  out->smem_bytes = smem_bytes;
  out->tma = tma;
  return MEGO_OK;
}

}  // namespace

namespace mego {

// Round keys of Philox4x32-10 for a seed.
RoundKeys make_round_keys(uint64_t seed) {
  RoundKeys K;
  uint32_t k0 = static_cast<uint32_t>(seed & 0xFFFFFFFFull);
  uint32_t k1 = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    K.rk0[r] = k0;
    K.rk1[r] = k1;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return K;
}

// The driver's tensor-map encoder, looked up once through the runtime (so
// the library does not link the driver library itself).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

bool encode_window_map(CUtensorMap* map, const float* w, uint32_t n, int ppt) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode || (reinterpret_cast<uintptr_t>(w) & 15u)) return false;
  const cuuint64_t gdim[1] = {static_cast<cuuint64_t>(n)};
  const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(n) * 4u};  // unused for rank 1
  const cuuint32_t box[1] = {32u * static_cast<cuuint32_t>(ppt)};
  const cuuint32_t estride[1] = {1u};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 1, const_cast<float*>(w), gdim, gstride,
                box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Constants of the stream word (c2 = stream id) used by the hoisted generator.
StreamKey make_stream_key(const RoundKeys& K, uint32_t sid) {
  const uint64_t m = static_cast<uint64_t>(kPhiloxM1) * sid;
  return StreamKey{static_cast<uint32_t>(m >> 32) ^ K.rk0[0], static_cast<uint32_t>(m), sid};
}

}  // namespace mego

namespace {

// ---------------------------------------------------------------------------
// Autotuning cache: best launch shape per (device, variant, gather layout,
// floor(log2 n), bucket of B).  Filled by mego_autotune, read when the caller
// passes no shape.

using TuneKey = std::tuple<int, int, int, int, int>;

int b_bucket(int32_t B) {
  int b = 0;
  while (b < 30 && (1 << (b + 1)) <= B) ++b;
  return B <= 0 ? -1 : b;
}

int n_bucket(uint32_t n) {
  int b = 0;
  while (b < 31 && (1u << (b + 1)) <= n) ++b;
  return b;
}

std::mutex g_tune_mu;
std::map<TuneKey, mego_launch_cfg> g_tune;

bool tune_lookup(int variant, int gather, uint32_t n, int32_t B, mego_launch_cfg* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(TuneKey(dev, variant, gather, n_bucket(n), b_bucket(B)));
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}

void tune_store(int variant, int gather, uint32_t n, int32_t B, const mego_launch_cfg& c) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[TuneKey(dev, variant, gather, n_bucket(n), b_bucket(B))] = c;
}

mego_status check_partition(int variant, uint32_t n, uint32_t psize, uint32_t* nw,
                            uint32_t* npart) {
  *nw = 1u;
  *npart = n;
  if (variant != MEGO_METROPOLIS_C1 && variant != MEGO_METROPOLIS_C2) return MEGO_OK;
  if (psize < 4u || psize % 4u) return MEGO_EINVAL;
  *nw = psize / 4u;
  if (n % *nw) return MEGO_EINVAL;
  *npart = n / *nw;
  return MEGO_OK;
}

}  // namespace

namespace mego {

void count_launches(uint64_t k) { g_launches.fetch_add(k); }

cudaError_t enable_large_smem(const void* kernel) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, cudaError_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(dev, kernel);
  auto it = done.find(key);
  if (it != done.end()) return it->second;
  int optin = 0;
  cudaFuncAttributes attr;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&attr, kernel);
  if (e == cudaSuccess) {
    const int dyn = optin - static_cast<int>(attr.sharedSizeBytes);
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  }
  if (e != cudaSuccess) cudaGetLastError();  // do not leave the error pending
  done.emplace(key, e);
  return e;
}

}  // namespace mego

extern "C" {

int mego_abi_version(void) { return MEGO_ABI_VERSION; }

const char* mego_status_string(int status) {
  switch (status) {
    case MEGO_OK: return "ok";
    case MEGO_EINVAL: return "invalid argument";
    case MEGO_ENOMEM: return "workspace too small";
    case MEGO_ECUDA: return "CUDA runtime error";
    case MEGO_ETIMEOUT: return "timed out waiting for the stream";
    case MEGO_EWEIGHTS: return "invalid weights or bound above its cap";
    default: return "unknown status";
  }
}

uint64_t mego_launch_count(void) { return g_launches.load(); }

size_t mego_struct_size(int32_t which) {
  switch (which) {
    case 0: return sizeof(mego_launch_cfg);
    case 1: return sizeof(mego_filter);
    case 2: return sizeof(mego_batch);
    case 3: return sizeof(mego_request);
    case 4: return sizeof(mego_completion);
    case 5: return sizeof(mego_server_cfg);
    case 6: return sizeof(mego_server_stats_t);
    default: return 0;
  }
}

size_t mego_workspace_bytes(int32_t n) {
  (void)n;
  return static_cast<size_t>(mego::kMaxParts) * sizeof(mego::Partial) + 256u;
}

mego_status mego_resample_gather(const float* d_w, int32_t n, int32_t B, const int32_t* d_B,
                                 uint64_t seed, uint32_t stream_id, int variant,
                                 uint32_t psize_bytes, const float* d_x_in, float* d_x_out,
                                 int32_t dim, int64_t ld, int layout, int32_t* d_anc,
                                 const mego_launch_cfg* cfg, void* stream) {
  if (!d_w || n < 1 || n > MEGO_N_MAX) return MEGO_EINVAL;
  if (!d_B && (B < 0 || B > MEGO_B_MAX)) return MEGO_EINVAL;
  if (variant < MEGO_MEGOPOLIS || variant > MEGO_METROPOLIS_C2) return MEGO_EINVAL;
  const uint32_t un = static_cast<uint32_t>(n);
  uint32_t nw = 1u, npart = un;
  if (check_partition(variant, un, psize_bytes, &nw, &npart) != MEGO_OK) return MEGO_EINVAL;
  int gather = mego::kGatherNone;
  size_t x_bytes = 0;
  if (d_x_in || d_x_out) {
    if (!d_x_in || !d_x_out) return MEGO_EINVAL;
    if (layout == MEGO_LAYOUT_SOA) {
      if (dim < 1 || ld < n) return MEGO_EINVAL;
      gather = mego::kGatherSoa;
      x_bytes = (static_cast<size_t>(dim - 1) * static_cast<size_t>(ld) + un) * 4u;
    } else if (layout == MEGO_LAYOUT_AOS4) {
      if (dim != 4) return MEGO_EINVAL;
      if ((reinterpret_cast<uintptr_t>(d_x_in) | reinterpret_cast<uintptr_t>(d_x_out)) & 15u)
        return MEGO_EINVAL;
      gather = mego::kGatherAos4;
      x_bytes = static_cast<size_t>(un) * 16u;
    } else {
      return MEGO_EINVAL;
    }
    if (overlaps(d_x_in, x_bytes, d_x_out, x_bytes)) return MEGO_EINVAL;
  } else if (!d_anc) {
    return MEGO_EINVAL;  // nothing to write
  }
  const size_t w_bytes = static_cast<size_t>(un) * 4u;
  if (d_anc && overlaps(d_anc, w_bytes, d_w, w_bytes)) return MEGO_EINVAL;
  if (d_anc && d_x_out && overlaps(d_anc, w_bytes, d_x_out, x_bytes)) return MEGO_EINVAL;
  if (d_x_out && overlaps(d_x_out, x_bytes, d_w, w_bytes)) return MEGO_EINVAL;

  mego_launch_cfg tuned;
  if (!cfg && tune_lookup(variant, gather, un, d_B ? -1 : B, &tuned)) cfg = &tuned;
  mego::LaunchShape shape;
  mego_status st = choose_shape(variant, un, gather, cfg, &shape);
  if (st != MEGO_OK) return st;

  mego::ResampleArgs a;
  std::memset(&a, 0, sizeof a);
  a.p.w = d_w;
  a.p.anc = d_anc;
  a.p.x_in = d_x_in;
  a.p.x_out = d_x_out;
  a.p.fault = nullptr;
  a.p.ld = ld;
  a.p.n = un;
  a.p.nseg = (un + 31u) / 32u;
  a.p.dim = dim;
  a.p.nw = nw;
  a.p.npart = npart;
  a.p.stage_polls = g_stage_polls.load();
  a.K = mego::make_round_keys(seed);
  a.p.S = mego::make_stream_key(a.K, stream_id);
  a.B_dev = d_B;
  a.B = d_B ? 0 : B;
  if (shape.tma && (reinterpret_cast<uintptr_t>(d_w) & 15u)) return MEGO_EINVAL;
  if (shape.tma && !mego::encode_window_map(&a.tmap, d_w, un, shape.ppt)) return MEGO_ECUDA;
  const cudaError_t e =
      shape.tma ? mego::launch_resample_tma(shape, gather, a, static_cast<cudaStream_t>(stream))
                : launch_variant(variant, shape, gather, a, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return MEGO_ECUDA;
  g_launches.fetch_add(1);
  return MEGO_OK;
}

mego_status mego_resample(const float* d_w, int32_t n, int32_t B, uint64_t seed,
                          uint32_t stream_id, int variant, int32_t* d_anc, void* stream) {
  if (!d_anc) return MEGO_EINVAL;
  if (variant != MEGO_MEGOPOLIS && variant != MEGO_METROPOLIS) return MEGO_EINVAL;
  return mego_resample_gather(d_w, n, B, nullptr, seed, stream_id, variant, 0u, nullptr,
                              nullptr, 0, 0, MEGO_LAYOUT_SOA, d_anc, nullptr, stream);
}

static mego_status bound_common(const float* src, int32_t n, bool likelihood, float y,
                                double eps, int32_t b_max, float* d_w, int32_t* d_B,
                                int32_t* d_status, double* d_q, void* d_ws, size_t ws_bytes,
                                void* stream) {
  if (!src || !d_B || !d_status || !d_ws) return MEGO_EINVAL;
  if (likelihood && !d_w) return MEGO_EINVAL;
  if (n < 1 || n > MEGO_N_MAX) return MEGO_EINVAL;
  if (!(eps > 0.0 && eps <= 1.0)) return MEGO_EINVAL;
  if (b_max < 1 || b_max > MEGO_B_MAX) return MEGO_EINVAL;
  if (ws_bytes < mego_workspace_bytes(n)) return MEGO_ENOMEM;
  if (reinterpret_cast<uintptr_t>(d_ws) & 255u) return MEGO_EINVAL;
  const uint32_t un = static_cast<uint32_t>(n);
  const size_t v_bytes = static_cast<size_t>(un) * 4u;  // up to 4 GiB: size_t, not 32 bits
  if (likelihood && overlaps(src, v_bytes, d_w, v_bytes)) return MEGO_EINVAL;
  auto* parts = static_cast<mego::Partial*>(d_ws);
  const int grid = mego::reduce_grid(un);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (mego::launch_partials(src, un, likelihood, y, d_w, parts, grid, st) != cudaSuccess)
    return MEGO_ECUDA;
  g_launches.fetch_add(1);
  if (mego::launch_finalize(parts, grid, un, eps, b_max, d_B, d_status, d_q, st) !=
      cudaSuccess)
    return MEGO_ECUDA;
  g_launches.fetch_add(1);
  return MEGO_OK;
}

mego_status mego_compute_B(const float* d_w, int32_t n, double eps, int32_t b_max,
                           int32_t* d_B, int32_t* d_status, double* d_q, void* d_ws,
                           size_t ws_bytes, void* stream) {
  return bound_common(d_w, n, false, 0.0f, eps, b_max, nullptr, d_B, d_status, d_q, d_ws,
                      ws_bytes, stream);
}

mego_status mego_likelihood_B(const float* d_x, int32_t n, float y, double eps, int32_t b_max,
                              float* d_w, int32_t* d_B, int32_t* d_status, double* d_q,
                              void* d_ws, size_t ws_bytes, void* stream) {
  return bound_common(d_x, n, true, y, eps, b_max, d_w, d_B, d_status, d_q, d_ws, ws_bytes,
                      stream);
}

mego_status mego_sync_status(const int32_t* d_status, void* stream, double timeout_s,
                             int32_t* h_status) {
  if (!d_status || !h_status || !(timeout_s >= 0.0)) return MEGO_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return MEGO_ECUDA;
  if (cudaEventRecord(ev, st) != cudaSuccess) {
    cudaEventDestroy(ev);
    return MEGO_ECUDA;
  }
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(timeout_s));
  for (;;) {
    const cudaError_t q = cudaEventQuery(ev);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) {
      cudaEventDestroy(ev);
      return MEGO_ECUDA;
    }
    if (std::chrono::steady_clock::now() >= deadline) {
      cudaEventDestroy(ev);
      return MEGO_ETIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  cudaEventDestroy(ev);
  int32_t v = 0;
  if (cudaMemcpy(&v, d_status, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess)
    return MEGO_ECUDA;
  *h_status = v;
  return MEGO_OK;
}

mego_status mego_resample_host(const float* h_w, int32_t n, int32_t B, double eps,
                               uint64_t seed, uint32_t stream_id, int variant, int32_t* h_anc,
                               int32_t* h_B, float* d_w, int32_t* d_anc, void* d_scalars,
                               void* d_ws, size_t ws_bytes, void* stream) {
  if (!h_w || !h_anc || !d_w || !d_anc || !d_scalars) return MEGO_EINVAL;
  if (n < 1 || n > MEGO_N_MAX || B > MEGO_B_MAX) return MEGO_EINVAL;
  if (variant != MEGO_MEGOPOLIS && variant != MEGO_METROPOLIS) return MEGO_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = static_cast<size_t>(n) * 4u;
  int32_t* d_Bp = static_cast<int32_t*>(d_scalars);
  int32_t* d_status = d_Bp + 1;
  double* d_q = reinterpret_cast<double*>(static_cast<char*>(d_scalars) + 8);
  if (cudaMemcpyAsync(d_w, h_w, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return MEGO_ECUDA;
  mego_status s;
  if (B < 0) {
    s = mego_compute_B(d_w, n, eps, MEGO_B_MAX, d_Bp, d_status, d_q, d_ws, ws_bytes, stream);
    if (s != MEGO_OK) return s;
    s = mego_resample_gather(d_w, n, 0, d_Bp, seed, stream_id, variant, 0u, nullptr, nullptr,
                             0, 0, MEGO_LAYOUT_SOA, d_anc, nullptr, stream);
  } else {
    s = mego_resample_gather(d_w, n, B, nullptr, seed, stream_id, variant, 0u, nullptr,
                             nullptr, 0, 0, MEGO_LAYOUT_SOA, d_anc, nullptr, stream);
  }
  if (s != MEGO_OK) return s;
  if (cudaMemcpyAsync(h_anc, d_anc, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MEGO_ECUDA;
  int32_t hb[2] = {B, 0};
  if (B < 0 &&
      cudaMemcpyAsync(hb, d_Bp, sizeof hb, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MEGO_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MEGO_ECUDA;
  if (h_B) *h_B = hb[0];
  return hb[1] == 0 ? MEGO_OK : MEGO_EWEIGHTS;
}

mego_status mego_autotune(const float* d_w, int32_t n, int32_t B, int variant,
                          uint32_t psize_bytes, const float* d_x_in, float* d_x_out,
                          int32_t dim, int64_t ld, int layout, int32_t* d_anc, int32_t reps,
                          mego_launch_cfg* best, float* best_ms, void* stream) {
  if (B < 0 || B > MEGO_B_MAX || reps < 1 || reps > 100) return MEGO_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return MEGO_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MEGO_ECUDA;
  }
  const int threads_c[] = {64, 128, 256};
  const int ppt_c[] = {1, 2, 4, 6, 8};
  const int path_c[] = {MEGO_PATH_GLOBAL, MEGO_PATH_SMEM, MEGO_PATH_TMA};
  mego_launch_cfg win{0, 0, 0, 0};
  float win_ms = 1e30f;
  mego_status status = MEGO_OK;
  for (int path : path_c) {
    for (int threads : threads_c) {
      for (int ppt : ppt_c) {
        mego_launch_cfg c{threads, ppt, path, 0};
        // Warm-up launch; shapes the library rejects (e.g. weights that do
        // not fit shared memory) are skipped.
        mego_status s = mego_resample_gather(d_w, n, B, nullptr, 1u, 0u, variant, psize_bytes,
                                             d_x_in, d_x_out, dim, ld, layout, d_anc, &c,
                                             stream);
        if (s == MEGO_EINVAL) continue;
        if (s != MEGO_OK) {
          status = s;
          break;
        }
        float total = 0.0f;
        bool ok = true;
        for (int r = 0; r < reps && ok; ++r) {
          ok = cudaEventRecord(e0, st) == cudaSuccess;
          ok = ok && mego_resample_gather(d_w, n, B, nullptr, 1u, 0u, variant, psize_bytes,
                                          d_x_in, d_x_out, dim, ld, layout, d_anc, &c,
                                          stream) == MEGO_OK;
          ok = ok && cudaEventRecord(e1, st) == cudaSuccess;
          ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
          float ms = 0.0f;
          ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
          total += ms;
        }
        if (!ok) {
          status = MEGO_ECUDA;
          break;
        }
        if (total / reps < win_ms) {
          win_ms = total / reps;
          win = c;
        }
      }
      if (status != MEGO_OK) break;
    }
    if (status != MEGO_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != MEGO_OK) return status;
  if (win.threads == 0) return MEGO_EINVAL;
  int gather = mego::kGatherNone;
  if (d_x_in) gather = layout == MEGO_LAYOUT_AOS4 ? mego::kGatherAos4 : mego::kGatherSoa;
  tune_store(variant, gather, static_cast<uint32_t>(n), B, win);
  tune_store(variant, gather, static_cast<uint32_t>(n), -1, win);  // device-side B
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  return MEGO_OK;
}

mego_status mego_device_fault(int32_t* h_fault) {
  if (!h_fault) return MEGO_EINVAL;
  int32_t* words[4] = {mego::resample_fault_word<mego::kMegopolis>(),
                       mego::resample_fault_word<mego::kMetropolis>(),
                       mego::resample_fault_word<mego::kC1>(),
                       mego::resample_fault_word<mego::kC2>()};
  int32_t any = 0;
  for (int32_t* w : words) {
    if (!w) return MEGO_ECUDA;
    int32_t v = 0;
    if (cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return MEGO_ECUDA;
    any |= v;
    if (v && cudaMemset(w, 0, sizeof v) != cudaSuccess) return MEGO_ECUDA;
  }
  *h_fault = any;
  return MEGO_OK;
}

mego_status mego_set_stage_poll_budget(int64_t polls) {
  if (polls > static_cast<int64_t>(mego::kMaxPolls)) return MEGO_EINVAL;
  g_stage_polls.store(polls < 0 ? mego::kMaxPolls : static_cast<uint32_t>(polls));
  return MEGO_OK;
}

mego_status mego_probe_read(const void* d_buf, size_t bytes, int32_t reps, float* d_sink,
                            void* stream) {
  if (!d_buf || !d_sink || bytes < 16u || bytes % 16u || reps < 1) return MEGO_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_buf) & 15u) return MEGO_EINVAL;
  DevInfo di;
  if (!dev_info(&di)) return MEGO_ECUDA;
  if (mego::launch_probe_read(d_buf, bytes, reps, d_sink, di.sms * 4,
                              static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return MEGO_ECUDA;
  g_launches.fetch_add(1);
  return MEGO_OK;
}

}  // extern "C"
