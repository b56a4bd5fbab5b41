// serve.cu -- continuous-batching request loop for resampling.
//
// A server owns one worker thread, a few CUDA streams and a first-fit
// allocator over a caller-provided device arena (the memory budget).
// Requests (weights, AoS4 state, host result buffers) are queued FIFO.  The
// worker admits queued requests while their device buffers fit in the arena,
// groups every admitted request into one batch when a stream is free, and
// on that stream uploads the inputs, runs the batched bound and the
// persistent resample with the AoS4 gather, copies the results back and
// records an event.  Requests that arrive while batches run are admitted into
// the next batch as memory frees up, so their work overlaps with the batches
// in flight.  Each request resamples with the server's seed and its id as
// stream id: its result is the same alone and in any mix.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#if defined(__linux__)
#include <sys/prctl.h>
#endif

#include "../../include/megopolis.h"
#include "batch_plan.h"

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch())
      .count();
}

// First-fit allocator over [0, size) with coalescing free blocks.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255u) & ~static_cast<size_t>(255u);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255u) & ~static_cast<size_t>(255u);
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    size_t start = off, len = bytes;
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        start = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    if (next != free_.end() && start + len == next->first) {
      len += next->second;
      free_.erase(next);
    }
    free_[start] = len;
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

struct Req {
  mego_request r;
  int64_t t_submit = 0;
  size_t off = 0, bytes = 0;   // arena slot: w | anc | x_in | x_out
  // Device addresses of the host buffers when they are page-locked (kernels
  // then read or write them in place), resolved at submission so that the
  // worker's launch path makes no pointer queries; null: copy instead.
  const float* w_dev = nullptr;
  int32_t* anc_dev = nullptr;
  float* x_out_dev = nullptr;
};

struct InFlight {
  std::vector<Req> reqs;
  size_t plan_off = 0, plan_bytes = 0;
  mego_batch batch{};
  cudaEvent_t done = nullptr;
  int stream = -1;
};

// Upper bound of one filter's share of a batch plan (descriptor, prefix
// entries, bound outputs, one 16-byte partial per 4096 weights) and the
// fixed part of a plan.
size_t plan_share(int32_t n) {
  return 128u + 16u * ((static_cast<size_t>(n) + 4095u) / 4096u);
}
constexpr size_t kPlanFixed = 1024u;

size_t slot_bytes(int32_t n) {
  const size_t un = static_cast<size_t>(n);
  // w (4n) | anc (4n) | x_in (16n) | x_out (16n), each part 256-byte aligned
  auto a = [](size_t x) { return (x + 255u) & ~static_cast<size_t>(255u); };
  return a(4 * un) + a(4 * un) + a(16 * un) + a(16 * un);
}

// Device address of page-locked host memory (kernels read and write it over
// the CPU-GPU link), or null for memory that has to be copied.
template <typename T>
T* host_device_ptr(T* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
  return static_cast<T*>(at.devicePointer);
}

}  // namespace

struct mego_server {
  mego_server_cfg cfg{};
  Arena arena;
  std::vector<cudaStream_t> streams;
  std::vector<bool> stream_busy;
  std::vector<void*> staging;     // page-locked plan staging, one per stream
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req> queue;          // submitted, not admitted
  std::vector<Req> admitted;      // in device memory, not yet launched
  std::vector<InFlight> inflight;
  std::vector<mego_completion> done;
  std::atomic<bool> stop{false};
  int launching = 0;              // batches taken from `admitted`, not yet in flight
  std::thread worker;
  size_t plan_slice = 0;          // bytes of plan space per stream (arena front)
  size_t admitted_plan = 0;       // plan bytes the admitted set will need
  int device = 0;
  mego_status error = MEGO_OK;
  uint64_t batches = 0, max_batch = 0;
  size_t peak_used = 0;

  void run();
  bool launch_batch(const std::vector<Req>& reqs, int si, InFlight* f);
  bool busy() const {
    return !(queue.empty() && admitted.empty() && inflight.empty() && launching == 0);
  }
  void finish(InFlight& f);
};

// Queues one batch on stream si: uploads, plan, bound, resample, downloads and
// the completion event.  Touches no shared server state, so the worker runs
// it without the lock (stream si and its staging buffer are reserved).
bool mego_server::launch_batch(const std::vector<Req>& reqs, int si, InFlight* f) {
  cudaStream_t st = streams[si];
  char* base = static_cast<char*>(cfg.d_arena);
  std::vector<mego_filter> filters(reqs.size());
  std::vector<char> anc_direct(reqs.size(), 0), xo_direct(reqs.size(), 0);
  const bool direct = cfg.host_copies != 1;
  for (size_t k = 0; k < reqs.size(); ++k) {
    const Req& q = reqs[k];
    const size_t un = static_cast<size_t>(q.r.n);
    auto a = [](size_t x) { return (x + 255u) & ~static_cast<size_t>(255u); };
    char* p = base + q.off;
    float* w = reinterpret_cast<float*>(p);
    int32_t* anc = reinterpret_cast<int32_t*>(p + a(4 * un));
    float* xi = reinterpret_cast<float*>(p + 2 * a(4 * un));
    float* xo = reinterpret_cast<float*>(p + 2 * a(4 * un) + a(16 * un));
    // Results go straight into page-locked host buffers (the resample writes
    // ancestors and state).  Inputs are uploaded by the copy engine, which
    // runs while other batches hold every SM; with host_copies = 2 the bound
    // reads page-locked weights itself (and writes w).  The state the
    // resample gathers from is read at random, so it is always uploaded.
    const float* w_host = cfg.host_copies == 2 ? q.w_dev : nullptr;
    if (!w_host &&
        cudaMemcpyAsync(w, q.r.h_w, 4 * un, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return false;
    const bool state = q.r.h_x != nullptr;
    if (state &&
        cudaMemcpyAsync(xi, q.r.h_x, 16 * un, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return false;
    if (direct) {
      if (q.anc_dev) {
        anc = q.anc_dev;
        anc_direct[k] = 1;
      }
      if (state && q.x_out_dev) {
        xo = q.x_out_dev;
        xo_direct[k] = 1;
      }
    }
    filters[k] = mego_filter{w, anc, state ? xi : nullptr, state ? xo : nullptr, 4,
                             q.r.n, -1, static_cast<uint32_t>(q.r.id), state ? 4 : 0, w_host};
  }
  // One gather layout per batch: all with state or all without.
  f->plan_bytes = mego_batch_plan_bytes(filters.data(), static_cast<int32_t>(filters.size()));
  if (f->plan_bytes == 0 || f->plan_bytes > plan_slice) return false;
  f->plan_off = static_cast<size_t>(si) * plan_slice;  // this stream's plan slice
  bool ok = mego::batch_plan_staged(filters.data(), static_cast<int32_t>(filters.size()),
                                    cfg.variant, MEGO_LAYOUT_AOS4, cfg.seed, 0,
                                    base + f->plan_off, f->plan_bytes, nullptr, staging[si],
                                    plan_slice, &f->batch, st, false) == MEGO_OK;
  if (ok && cfg.threads > 0)
    ok = mego_batch_set_shape(&f->batch, cfg.threads,
                              cfg.ppt > 0 ? cfg.ppt : f->batch.cfg.ppt) == MEGO_OK;
  ok = ok && mego_batch_bound(&f->batch, cfg.eps, MEGO_B_MAX, st) == MEGO_OK;
  ok = ok && mego_batch_resample(&f->batch, st) == MEGO_OK;
  for (size_t k = 0; ok && k < reqs.size(); ++k) {
    const Req& q = reqs[k];
    if (q.r.h_anc && !anc_direct[k])
      ok = cudaMemcpyAsync(q.r.h_anc, filters[k].anc, 4 * static_cast<size_t>(q.r.n),
                           cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (ok && q.r.h_x_out && filters[k].x_out && !xo_direct[k])
      ok = cudaMemcpyAsync(q.r.h_x_out, filters[k].x_out, 16 * static_cast<size_t>(q.r.n),
                           cudaMemcpyDeviceToHost, st) == cudaSuccess;
  }
  // Each request's B comes back into the stream's staging buffer (its plan
  // copy ran earlier on the same stream); finish() reads it.
  ok = ok && cudaMemcpyAsync(staging[si], f->batch.d_B, sizeof(int32_t) * reqs.size(),
                             cudaMemcpyDeviceToHost, st) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&f->done, cudaEventDisableTiming) == cudaSuccess;
  if (ok && cudaEventRecord(f->done, st) != cudaSuccess) {
    cudaEventDestroy(f->done);
    ok = false;
  }
  if (!ok) {
    // Wait for what was queued on the stream before the memory is reused.
    cudaStreamSynchronize(st);
    return false;
  }
  f->stream = si;
  return true;
}

void mego_server::finish(InFlight& f) {
  const int64_t t = now_ns();
  const int32_t* Bs = static_cast<const int32_t*>(staging[f.stream]);
  for (size_t k = 0; k < f.reqs.size(); ++k) {
    const Req& q = f.reqs[k];
    mego_completion c{};
    c.id = q.r.id;
    // B < 0: the bound rejected this request's weights (NaN, Inf, negative,
    // all zero, or B above its cap) and the resample wrote nothing for it.
    c.status = Bs[k] >= 0 ? MEGO_OK : MEGO_EWEIGHTS;
    c.latency_ns = t - q.t_submit;
    c.n = q.r.n;
    c.B = Bs[k];
    done.push_back(c);
    arena.release(q.off, q.bytes);
  }
  cudaEventDestroy(f.done);
  stream_busy[f.stream] = false;
}

void mego_server::run() {
  cudaSetDevice(device);
#if defined(__linux__)
  // The worker polls its in-flight batches every poll_us microseconds while
  // busy; Linux would otherwise let such a short sleep overrun by its default
  // 50 us of timer slack, delaying every completion and launch by as much.
  // (This thread's own setting; it ends with the thread.)
  prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
  std::unique_lock<std::mutex> lock(mu);
  while (!stop.load()) {
    // 1. Completions.
    for (size_t k = 0; k < inflight.size();) {
      const cudaError_t e = cudaEventQuery(inflight[k].done);
      if (e == cudaSuccess) {
        finish(inflight[k]);
        inflight.erase(inflight.begin() + static_cast<long>(k));
        cv.notify_all();
      } else {
        if (e != cudaErrorNotReady) error = MEGO_ECUDA;
        ++k;
      }
    }
    // 2. Admission: FIFO while the slot fits the budget (plans take a little
    // more; they are allocated at launch).
    while (!queue.empty() && static_cast<int>(admitted.size()) < cfg.max_batch) {
      Req& q = queue.front();
      const size_t share = plan_share(q.r.n);
      if (kPlanFixed + admitted_plan + share > plan_slice && !admitted.empty()) break;
      q.bytes = slot_bytes(q.r.n);
      if (!arena.alloc(q.bytes, &q.off)) break;
      admitted_plan += share;
      admitted.push_back(q);
      queue.pop_front();
    }
    if (arena.used() > peak_used) peak_used = arena.used();
    // 3. Launch the admitted requests on a free stream.
    if (!admitted.empty()) {
      int si = -1;
      for (size_t s = 0; s < streams.size(); ++s)
        if (!stream_busy[s]) {
          si = static_cast<int>(s);
          break;
        }
      if (si >= 0) {
        std::vector<Req> reqs;
        reqs.swap(admitted);
        admitted_plan = 0;
        // Launch without the lock, so submissions and polls are not held up
        // by the host side of the launch.
        stream_busy[si] = true;
        launching += 1;
        InFlight f;
        lock.unlock();
        const bool ok = launch_batch(reqs, si, &f);
        lock.lock();
        launching -= 1;
        if (ok) {
          f.reqs.swap(reqs);
          batches += 1;
          if (f.reqs.size() > max_batch) max_batch = f.reqs.size();
          inflight.push_back(std::move(f));
        } else {
          stream_busy[si] = false;
          error = MEGO_ECUDA;
          for (const Req& q : reqs) {
            mego_completion c{};
            c.id = q.r.id;
            c.status = MEGO_ECUDA;
            c.n = q.r.n;
            c.B = -1;
            done.push_back(c);
            arena.release(q.off, q.bytes);
          }
          cv.notify_all();
        }
      }
    }
    const bool idle = !busy();
    if (idle) {
      cv.wait_for(lock, std::chrono::milliseconds(1));
    } else {
      lock.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(cfg.poll_us > 0 ? cfg.poll_us : 5));
      lock.lock();
    }
  }
}

extern "C" {

mego_status mego_server_create(const mego_server_cfg* cfg, mego_server** out) {
  if (!cfg || !out || !cfg->d_arena || cfg->arena_bytes < 4096) return MEGO_EINVAL;
  if (cfg->variant != MEGO_MEGOPOLIS && cfg->variant != MEGO_METROPOLIS) return MEGO_EINVAL;
  if (!(cfg->eps > 0.0 && cfg->eps <= 1.0)) return MEGO_EINVAL;
  if (reinterpret_cast<uintptr_t>(cfg->d_arena) & 255u) return MEGO_EINVAL;
  mego_server* s = new mego_server();
  s->cfg = *cfg;
  if (s->cfg.max_batch <= 0) s->cfg.max_batch = 256;
  if (s->cfg.streams <= 0) s->cfg.streams = 2;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return MEGO_ECUDA;
  }
  // Plan slices at the front of the arena, one per stream; requests use the rest.
  size_t slice = cfg->arena_bytes / (16u * static_cast<size_t>(s->cfg.streams));
  if (slice > (16u << 20)) slice = 16u << 20;
  slice &= ~static_cast<size_t>(255u);
  s->plan_slice = slice;
  const size_t front = slice * static_cast<size_t>(s->cfg.streams);
  if (slice < 4096u || front >= cfg->arena_bytes) {
    delete s;
    return MEGO_EINVAL;
  }
  s->arena.reset(cfg->arena_bytes);
  size_t dummy = 0;
  s->arena.alloc(front, &dummy);  // offset 0: the plan slices
  for (int k = 0; k < s->cfg.streams; ++k) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
      delete s;
      return MEGO_ECUDA;
    }
    s->streams.push_back(st);
    s->stream_busy.push_back(false);
    void* h = nullptr;
    if (cudaHostAlloc(&h, slice, cudaHostAllocDefault) != cudaSuccess) {
      for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
      for (void* p : s->staging) cudaFreeHost(p);
      delete s;
      return MEGO_ECUDA;
    }
    s->staging.push_back(h);
  }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return MEGO_OK;
}

mego_status mego_server_submit(mego_server* s, const mego_request* r) {
  if (!s || !r || !r->h_w || r->n < 1 || r->n > MEGO_N_MAX) return MEGO_EINVAL;
  if ((r->h_x != nullptr) != (s->cfg.with_state != 0)) return MEGO_EINVAL;
  if (slot_bytes(r->n) + s->plan_slice * static_cast<size_t>(s->cfg.streams) >
          s->cfg.arena_bytes ||
      kPlanFixed + plan_share(r->n) > s->plan_slice)
    return MEGO_ENOMEM;  // could never fit
  Req q;
  q.r = *r;
  q.t_submit = now_ns();
  // Page-locked host buffers, resolved here (on the caller's thread) rather
  // than on the worker's launch path.
  if (s->cfg.host_copies == 2) q.w_dev = host_device_ptr(r->h_w);
  if (s->cfg.host_copies != 1) {
    q.anc_dev = host_device_ptr(r->h_anc);
    q.x_out_dev = host_device_ptr(r->h_x_out);
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->queue.push_back(q);
  }
  s->cv.notify_all();
  return MEGO_OK;
}

int32_t mego_server_poll(mego_server* s, mego_completion* out, int32_t max_out) {
  if (!s || !out || max_out < 1) return 0;
  std::lock_guard<std::mutex> lock(s->mu);
  const int32_t k = static_cast<int32_t>(
      std::min(s->done.size(), static_cast<size_t>(max_out)));
  for (int32_t i = 0; i < k; ++i) out[i] = s->done[static_cast<size_t>(i)];
  s->done.erase(s->done.begin(), s->done.begin() + k);
  return k;
}

mego_status mego_server_drain(mego_server* s, double timeout_s) {
  if (!s) return MEGO_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s));
  while (s->busy()) {
    if (s->cv.wait_until(lock, deadline) == std::cv_status::timeout &&
        Clock::now() >= deadline)
      return MEGO_ETIMEOUT;
  }
  return s->error;
}

mego_status mego_server_stats(mego_server* s, mego_server_stats_t* out) {
  if (!s || !out) return MEGO_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  out->batches = s->batches;
  out->max_batch = s->max_batch;
  out->peak_arena_bytes = s->peak_used;
  out->queued = s->queue.size();
  out->inflight = s->inflight.size();
  return MEGO_OK;
}

mego_status mego_server_destroy(mego_server* s) {
  if (!s) return MEGO_EINVAL;
  s->stop.store(true);
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (InFlight& f : s->inflight) {
    cudaEventSynchronize(f.done);
    cudaEventDestroy(f.done);
  }
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (void* p : s->staging) cudaFreeHost(p);
  delete s;
  return MEGO_OK;
}

mego_status mego_server_replay(mego_server* s, const mego_request* reqs, const double* t_arrival,
                               int32_t count, double timeout_s) {
  if (!s || !reqs || !t_arrival || count < 1) return MEGO_EINVAL;
  const auto t0 = Clock::now();
  for (int32_t k = 0; k < count; ++k) {
    const auto due = t0 + std::chrono::duration_cast<Clock::duration>(
                              std::chrono::duration<double>(t_arrival[k]));
    while (Clock::now() < due) {
    }
    const mego_status st = mego_server_submit(s, &reqs[k]);
    if (st != MEGO_OK) return st;
  }
  return mego_server_drain(s, timeout_s);
}

}  // extern "C"
