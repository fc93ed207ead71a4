// gf_server.cu -- a gauge-fixing job server: jobs of different lattices and
// gauges share one GPU.  Device memory is one arena reserved at start-up and
// sub-allocated first-fit, so link fields stay resident and admission never
// calls cudaMalloc.  A job is admitted as soon as a worker slot is free and its
// footprint (gf_footprint) fits in the arena; each admitted job runs on its
// own context and CUDA stream, so the kernels of concurrent jobs overlap on
// the device, and a finished job's slot and memory go to the next queued job
// at once (continuous batching of independent problems).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include "gf.h"
#include "gf_launch.h"

namespace {

constexpr size_t ARENA_ALIGN = 256;

// First-fit allocator over [0, size) with coalescing of free neighbours.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + ARENA_ALIGN - 1) / ARENA_ALIGN * ARENA_ALIGN;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        blocks_[*off] = bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off) {
    auto b = blocks_.find(off);
    if (b == blocks_.end()) return;
    size_t start = off, len = b->second;
    used_ -= len;
    blocks_.erase(b);
    auto next = free_.lower_bound(start);
    if (next != free_.end() && next->first == start + len) {
      len += next->second;
      free_.erase(next);
    }
    auto prev = free_.lower_bound(start);
    if (prev != free_.begin()) {
      --prev;
      if (prev->first + prev->second == start) {
        start = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    free_[start] = len;
  }
  size_t used() const { return used_; }
  size_t size() const { return size_; }

 private:
  size_t size_, used_ = 0;
  std::map<size_t, size_t> free_;    // offset -> length
  std::map<size_t, size_t> blocks_;  // offset -> length of live allocations
};

struct Pending {
  gf_job job;
  size_t bytes;
  double t_submit;
  int skipped;  // times a later job was admitted before this one
};

}  // namespace

struct gf_server {
  int device = 0;
  bool mock = false;
  double mock_seconds_per_gb = 0;
  char* base = nullptr;
  Arena* arena = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue;
  std::vector<gf_job_result> done;
  std::vector<std::thread> workers;
  int running = 0;
  uint64_t n_done_total = 0;
  bool stopping = false;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {


int sfail(int code, const char* msg) {
  gfk::set_last_error(msg);
  return code;
}

// Run one admitted job on its own context carved from the arena block.
void run_job(const gf_job& J, char* mem, size_t bytes, gf_job_result& R) {
  nvtxRangePushA("server job");
  gf_ctx* c = nullptr;
  int r = gf_create_ext(J.dims, 1, J.gauge, J.prec, nullptr, mem, bytes, &c);
  if (!r) r = gf_load_links(c, 0, J.host_links);
  if (!r && J.orbit_seed) r = gf_random_gauge_transform(c, J.orbit_seed);
  gf_fix_result fr;
  memset(&fr, 0, sizeof fr);
  if (!r) r = J.anneal ? gf_protocol(c, &J.protocol, &fr) : gf_fix(c, &J.fix, &fr);
  const int fix_status = r;
  if (c && (r == GF_OK || r == GF_ENOTCONV)) {
    int r2 = gf_functional_theta(c, &R.F, &R.theta);
    if (!r2 && J.host_out) r2 = gf_store_links(c, 0, J.host_out);
    if (r2) r = r2;
    else r = fix_status;
  }
  R.status = r;
  R.sweeps = fr.sweeps;
  R.sweeps_fp32 = fr.sweeps_fp32;
  R.sweeps_fp64 = fr.sweeps_fp64;
  R.site_updates = fr.site_updates;
  gf_destroy(c);
  nvtxRangePop();
}

void worker_main(gf_server* S) {
  if (!S->mock) cudaSetDevice(S->device);
  for (;;) {
    Pending P;
    size_t off = 0;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      for (;;) {
        if (S->stopping && S->queue.empty()) return;
        // the first queued job that fits: a large job waiting for memory does
        // not hold back smaller ones behind it, unless it has been passed over
        // 4 x slots times, after which it alone may be admitted (no starvation)
        auto it = S->queue.begin();
        const bool head_blocks = !S->queue.empty() && S->queue.front().skipped >= 4 * (int)S->workers.size();
        for (; it != S->queue.end(); ++it) {
          if (S->arena->alloc(it->bytes, &off)) break;
          if (head_blocks) {
            it = S->queue.end();
            break;
          }
        }
        if (it != S->queue.end() && it != S->queue.begin()) S->queue.front().skipped++;
        if (it != S->queue.end()) {
          P = *it;
          S->queue.erase(it);
          S->running++;
          break;
        }
        if (S->stopping) return;
        S->cv_work.wait(lock);
      }
    }
    gf_job_result R;
    memset(&R, 0, sizeof R);
    R.tag = P.job.tag;
    R.t_submit = P.t_submit;
    R.t_admit = S->now();
    R.footprint = P.bytes;
    if (S->mock) {
      // test double: no device work, a duration proportional to the footprint
      std::this_thread::sleep_for(std::chrono::duration<double>(S->mock_seconds_per_gb * P.bytes / 1e9));
      R.status = GF_OK;
    } else {
      run_job(P.job, S->base + off, P.bytes, R);
    }
    R.t_done = S->now();
    {
      std::lock_guard<std::mutex> lock(S->mu);
      S->arena->release(off);
      S->running--;
      S->n_done_total++;
      S->done.push_back(R);
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
}

int create_impl(size_t bytes, int slots, bool mock, double sec_per_gb, gf_server** out) {
  if (!out) return sfail(GF_EINVAL, "out is NULL");
  *out = nullptr;
  if (slots < 1 || slots > 64) return sfail(GF_EINVAL, "slots must be in [1, 64]");
  if (bytes < ARENA_ALIGN) return sfail(GF_EINVAL, "arena too small");
  gf_server* S = new (std::nothrow) gf_server;
  if (!S) return sfail(GF_ENOMEM, "host allocation failed");
  S->mock = mock;
  S->mock_seconds_per_gb = sec_per_gb;
  if (!mock) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      cudaGetLastError();
      delete S;
      return sfail(GF_ENOSYS, "no CUDA device available");
    }
    cudaGetDevice(&S->device);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      delete S;
      return sfail(GF_ENOMEM, "cudaMalloc of the server arena failed");
    }
    S->base = static_cast<char*>(p);
  }
  S->arena = new Arena(bytes);
  for (int k = 0; k < slots; ++k) S->workers.emplace_back(worker_main, S);
  *out = S;
  return GF_OK;
}

}  // namespace

extern "C" {

int gf_server_create(size_t hbm_bytes, int slots, gf_server** out) {
  return create_impl(hbm_bytes, slots, false, 0.0, out);
}

int gf_server_create_mock(size_t hbm_bytes, int slots, double seconds_per_gb, gf_server** out) {
  if (!(seconds_per_gb >= 0)) return sfail(GF_EINVAL, "seconds_per_gb must be >= 0");
  return create_impl(hbm_bytes, slots, true, seconds_per_gb, out);
}

int gf_server_submit(gf_server* S, const gf_job* job) {
  if (!S || !job) return sfail(GF_EINVAL, "NULL argument");
  if (!S->mock && !job->host_links) return sfail(GF_EINVAL, "host_links is NULL");
  size_t bytes = 0;
  int r = gf_footprint(job->dims, 1, job->gauge, job->prec, &bytes);
  if (r) return r;
  bytes = (bytes + ARENA_ALIGN - 1) / ARENA_ALIGN * ARENA_ALIGN;
  if (bytes > S->arena->size()) return sfail(GF_ENOMEM, "job footprint exceeds the server arena");
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stopping) return sfail(GF_EINVAL, "server is shutting down");
    S->queue.push_back(Pending{*job, bytes, S->now(), 0});
  }
  S->cv_work.notify_one();
  return GF_OK;
}

int gf_server_poll(gf_server* S, gf_job_result* out, int max_results, int wait_ms, int* n_out) {
  if (!S || !n_out || (max_results > 0 && !out)) return sfail(GF_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lock(S->mu);
  if (S->done.empty() && wait_ms > 0)
    S->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
  const int n = std::min<int>(max_results, (int)S->done.size());
  for (int k = 0; k < n; ++k) out[k] = S->done[k];
  S->done.erase(S->done.begin(), S->done.begin() + n);
  *n_out = n;
  return GF_OK;
}

int gf_server_status(gf_server* S, int* queued, int* running, uint64_t* completed, size_t* bytes_in_use) {
  if (!S) return sfail(GF_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lock(S->mu);
  if (queued) *queued = (int)S->queue.size();
  if (running) *running = S->running;
  if (completed) *completed = S->n_done_total;
  if (bytes_in_use) *bytes_in_use = S->arena->used();
  return GF_OK;
}

int gf_server_cancel(gf_server* S, uint64_t tag, int* n_canceled) {
  if (!S) return sfail(GF_EINVAL, "NULL server");
  int n = 0;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    for (auto it = S->queue.begin(); it != S->queue.end();) {
      if (it->job.tag != tag) {
        ++it;
        continue;
      }
      gf_job_result R;
      memset(&R, 0, sizeof R);
      R.tag = tag;
      R.status = GF_ECANCELED;
      R.footprint = it->bytes;
      R.t_submit = it->t_submit;
      R.t_admit = R.t_done = S->now();
      S->done.push_back(R);
      S->n_done_total++;
      it = S->queue.erase(it);
      ++n;
    }
  }
  if (n) {
    S->cv_done.notify_all();
    S->cv_work.notify_all();  // a large job at the head may have been blocking others
  }
  if (n_canceled) *n_canceled = n;
  return GF_OK;
}

void gf_server_destroy(gf_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  if (S->base) cudaFree(S->base);
  delete S->arena;
  delete S;
}

}  // extern "C"
