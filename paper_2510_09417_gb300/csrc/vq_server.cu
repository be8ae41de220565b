// vq_server.cu -- serving handle: hull requests admitted against a device
// memory budget and run together.
//
// A host thread owns a device pool.  Whenever requests are queued it admits
// as many as fit (FIFO, up to max_inflight and the memory budget), copies
// their points into the pool and runs them as one batched level-synchronous
// hull (all segments of all admitted requests share each level step).  The
// results are copied back per request; vq_server_poll / vq_server_wait hand
// them out.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/vqhull.h"

namespace {

using Clock = std::chrono::steady_clock;

// device bytes per point of a request: input (16), ping-pong buffers (40),
// keys and slots (~5), output (4), tables (~2)
constexpr double kBytesPerPoint = 68.0;
constexpr size_t kBytesFixed = 1 << 20;

struct Request {
  uint64_t ticket = 0;
  std::vector<double> x, y;
  int64_t n = 0;
  Clock::time_point t_submit;
  // result
  bool done = false;
  vq_status status = VQ_OK;
  std::vector<int32_t> hull;
  Clock::time_point t_done;
};

size_t request_bytes(int64_t n) { return (size_t)(kBytesPerPoint * (double)n) + 4096; }

}  // namespace

struct vq_server {
  vq_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread thr;
  // device pool
  double* d_x = nullptr;
  double* d_y = nullptr;
  int32_t* d_out = nullptr;
  int64_t* d_off = nullptr;
  int64_t* d_hoff = nullptr;
  int64_t pool_points = 0;
  int pool_sets = 0;
  cudaStream_t stream = nullptr;
  // stats
  std::vector<double> lat_ms;
  Clock::time_point t_first{};
  Clock::time_point t_last{};
  long long completed = 0;
  vq_status fatal = VQ_OK;
};

static vq_status ensure_pool(vq_server* s, int64_t points, int sets) {
  if (points <= s->pool_points && sets <= s->pool_sets) return VQ_OK;
  cudaFree(s->d_x); cudaFree(s->d_y); cudaFree(s->d_out); cudaFree(s->d_off); cudaFree(s->d_hoff);
  s->d_x = s->d_y = nullptr; s->d_out = nullptr; s->d_off = s->d_hoff = nullptr;
  s->pool_points = 0; s->pool_sets = 0;
  const int64_t P = std::max<int64_t>(points, 1);
  if (cudaMalloc(&s->d_x, sizeof(double) * P) != cudaSuccess ||
      cudaMalloc(&s->d_y, sizeof(double) * P) != cudaSuccess ||
      cudaMalloc(&s->d_out, sizeof(int32_t) * P) != cudaSuccess ||
      cudaMalloc(&s->d_off, sizeof(int64_t) * (sets + 1)) != cudaSuccess ||
      cudaMalloc(&s->d_hoff, sizeof(int64_t) * (sets + 1)) != cudaSuccess) {
    cudaGetLastError();
    return VQ_ERR_NOMEM;
  }
  s->pool_points = P;
  s->pool_sets = sets;
  return VQ_OK;
}

static void serve(vq_server* s) {
  cudaSetDevice(s->cfg.device);
  cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  for (;;) {
    std::vector<Request*> batch;
    {
      std::unique_lock<std::mutex> g(s->mu);
      s->cv_work.wait(g, [&] { return s->stop || !s->queue.empty(); });
      if (s->stop) break;
      size_t used = kBytesFixed;
      while (!s->queue.empty() && (int)batch.size() < s->cfg.max_inflight) {
        Request* r = s->queue.front();
        const size_t b = request_bytes(r->n);
        if (!batch.empty() && used + b > s->cfg.mem_budget_bytes) break;
        used += b;
        batch.push_back(r);
        s->queue.pop_front();
      }
    }
    // copy in, run all admitted requests together, copy out
    int64_t total = 0;
    std::vector<int64_t> offs(batch.size() + 1, 0);
    for (size_t i = 0; i < batch.size(); i++) { offs[i] = total; total += batch[i]->n; }
    offs[batch.size()] = total;
    vq_status st = ensure_pool(s, total, (int)batch.size());
    std::vector<int64_t> hoff(batch.size() + 1, 0);
    std::vector<int32_t> out;
    if (st == VQ_OK) {
      for (size_t i = 0; i < batch.size(); i++) {
        if (batch[i]->n == 0) continue;
        cudaMemcpyAsync(s->d_x + offs[i], batch[i]->x.data(), sizeof(double) * batch[i]->n,
                        cudaMemcpyHostToDevice, s->stream);
        cudaMemcpyAsync(s->d_y + offs[i], batch[i]->y.data(), sizeof(double) * batch[i]->n,
                        cudaMemcpyHostToDevice, s->stream);
      }
      cudaMemcpyAsync(s->d_off, offs.data(), sizeof(int64_t) * offs.size(), cudaMemcpyHostToDevice, s->stream);
      st = vq_hull2d_batched(s->d_x, s->d_y, s->d_off, (int32_t)batch.size(), s->d_out, s->d_hoff, s->stream);
      if (st == VQ_OK || st == VQ_ERR_NONFINITE) {
        cudaMemcpyAsync(hoff.data(), s->d_hoff, sizeof(int64_t) * hoff.size(), cudaMemcpyDeviceToHost, s->stream);
        cudaStreamSynchronize(s->stream);
        out.resize((size_t)std::max<int64_t>(hoff.back(), 1));
        if (hoff.back() > 0)
          cudaMemcpyAsync(out.data(), s->d_out, sizeof(int32_t) * hoff.back(), cudaMemcpyDeviceToHost, s->stream);
        if (cudaStreamSynchronize(s->stream) != cudaSuccess) st = VQ_ERR_CUDA;
      }
    }
    const auto now = Clock::now();
    {
      std::lock_guard<std::mutex> g(s->mu);
      for (size_t i = 0; i < batch.size(); i++) {
        Request* r = batch[i];
        if (st == VQ_OK || st == VQ_ERR_NONFINITE) {
          const int64_t a = hoff[i], b = hoff[i + 1];
          r->hull.assign(out.begin() + a, out.begin() + b);
          // a request with a non-finite point gets an empty hull; report it as such
          r->status = (st == VQ_ERR_NONFINITE && b == a && r->n > 0) ? VQ_ERR_NONFINITE : VQ_OK;
        } else {
          r->status = st;
        }
        r->x.clear(); r->x.shrink_to_fit();
        r->y.clear(); r->y.shrink_to_fit();
        r->done = true;
        r->t_done = now;
        s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
        s->completed++;
        s->t_last = now;
      }
    }
    s->cv_done.notify_all();
  }
  cudaStreamDestroy(s->stream);
}

extern "C" {

vq_status vq_server_create(const vq_server_config* cfg, vq_server** out) {
  if (!cfg || !out || cfg->max_inflight < 1 || cfg->mem_budget_bytes < kBytesFixed) return VQ_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return VQ_ERR_CUDA;
  if (cfg->device < 0 || cfg->device >= ndev) return VQ_ERR_INVALID_ARG;
  vq_server* s = new vq_server();
  s->cfg = *cfg;
  s->thr = std::thread(serve, s);
  *out = s;
  return VQ_OK;
}

vq_status vq_server_submit(vq_server* s, const double* x_host, const double* y_host, int64_t n, uint64_t* ticket) {
  if (!s || !ticket || n < 0 || (n > 0 && (!x_host || !y_host))) return VQ_ERR_INVALID_ARG;
  if (n > (int64_t)INT32_MAX - 2) return VQ_ERR_TOO_LARGE;
  if (request_bytes(n) + kBytesFixed > s->cfg.mem_budget_bytes) return VQ_ERR_BUDGET;
  Request* r = new Request();
  r->n = n;
  r->x.assign(x_host, x_host + n);
  r->y.assign(y_host, y_host + n);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> g(s->mu);
    r->ticket = s->next_ticket++;
    if (s->completed == 0 && s->all.empty()) s->t_first = r->t_submit;
    s->all[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv_work.notify_one();
  return VQ_OK;
}

static vq_status take_result(vq_server* s, uint64_t ticket, int32_t* hull_idx_host, int64_t cap, int64_t* h,
                             bool wait, int32_t timeout_ms) {
  if (!s || !h) return VQ_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> g(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return VQ_ERR_NOT_FOUND;
  Request* r = it->second;
  if (!r->done && wait) {
    auto pred = [&] { return r->done; };
    if (timeout_ms < 0) s->cv_done.wait(g, pred);
    else s->cv_done.wait_for(g, std::chrono::milliseconds(timeout_ms), pred);
  }
  if (!r->done) return VQ_PENDING;
  if (r->status != VQ_OK) {
    const vq_status st = r->status;
    s->all.erase(it);
    delete r;
    return st;
  }
  *h = (int64_t)r->hull.size();
  if (cap < *h || (*h > 0 && !hull_idx_host)) return VQ_ERR_CAPACITY;
  if (*h > 0) memcpy(hull_idx_host, r->hull.data(), sizeof(int32_t) * r->hull.size());
  s->all.erase(it);
  delete r;
  return VQ_OK;
}

vq_status vq_server_poll(vq_server* s, uint64_t ticket, int32_t* hull_idx_host, int64_t cap, int64_t* h) {
  return take_result(s, ticket, hull_idx_host, cap, h, false, 0);
}

vq_status vq_server_wait(vq_server* s, uint64_t ticket, int32_t* hull_idx_host, int64_t cap, int64_t* h,
                         int32_t timeout_ms) {
  return take_result(s, ticket, hull_idx_host, cap, h, true, timeout_ms);
}

vq_status vq_server_stats(vq_server* s, double* p50_ms, double* p99_ms, double* hulls_per_s) {
  if (!s) return VQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  std::vector<double> v = s->lat_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double q) -> double {
    if (v.empty()) return 0.0;
    size_t i = (size_t)(q * (double)(v.size() - 1) + 0.5);
    return v[std::min(i, v.size() - 1)];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (hulls_per_s) {
    const double sec = std::chrono::duration<double>(s->t_last - s->t_first).count();
    *hulls_per_s = (sec > 0.0) ? (double)s->completed / sec : 0.0;
  }
  return VQ_OK;
}

void vq_server_destroy(vq_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->thr.joinable()) s->thr.join();
  for (auto& kv : s->all) delete kv.second;
  cudaSetDevice(s->cfg.device);
  cudaFree(s->d_x); cudaFree(s->d_y); cudaFree(s->d_out); cudaFree(s->d_off); cudaFree(s->d_hoff);
  delete s;
}

}  // extern "C"
