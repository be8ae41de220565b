// vq_server.cu -- serving handle: continuous batching of hull requests.
//
// Requests are queued by vq_server_submit.  Each lane is a host thread with
// its own CUDA stream and hull context.  An idle lane takes the queued
// requests (FIFO) that fit the free request slots and the free device
// memory, copies their points into memory drawn from the server's pool,
// and runs them as one batched level-synchronous hull: all segments of all
// its requests share each level step (Sec. 3's extraction, run for many
// hulls at once).  Lanes run side by side, so requests that arrive while
// other batches are on the GPU are admitted as soon as a lane, slots and
// memory are free, and their kernels overlap with the running batches.
// Results are copied back per request; vq_server_poll / vq_server_wait hand
// them out, in any order.
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
#include "vq_admit.h"
#include "vq_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kDefaultLanes = 3;
constexpr int kMaxLanes = 16;
constexpr size_t kBytesFixed = 1 << 20;  // the budget must at least cover this
// A batch is the queue's head and the requests after it while the batch
// holds at most max(kBatchPoints, head's points) points: small requests share
// level steps, and a big request does not hold small ones back behind it.
constexpr long long kBatchPoints = 1ll << 20;
constexpr size_t kDefaultPinned = 8ull << 30;  // pinned staging area (at most the budget)

struct Request {
  uint64_t ticket = 0;
  std::vector<double> x, y;   // pageable copy (when the pinned staging area is full)
  double* px = nullptr;       // pinned copy: x then y, n doubles each
  size_t pin_off = 0, pin_len = 0;
  int64_t n = 0;
  Clock::time_point t_submit;
  // result
  bool done = false;
  vq_status status = VQ_OK;
  std::vector<int32_t> hull;
  Clock::time_point t_done;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// One batch's device memory, carved from one pool allocation: x and y,
// the output indices, offsets, hull offsets, then the hull workspace.
struct BatchLayout {
  size_t x, y, out, off, hoff, ws, ws_bytes, total;
};

BatchLayout batch_layout(long long N, int nsets) {
  BatchLayout L;
  const size_t n = (size_t)std::max<long long>(N, 1);
  size_t o = 0;
  L.x = o;
  o += align256(sizeof(double) * n);
  L.y = o;
  o += align256(sizeof(double) * n);
  L.out = o;
  o += align256(sizeof(int32_t) * n);
  L.off = o;
  o += align256(sizeof(int64_t) * (size_t)(nsets + 1));
  L.hoff = o;
  o += align256(sizeof(int64_t) * (size_t)(nsets + 1));
  L.ws = o;
  L.ws_bytes = align256(vq::batched_workspace_bytes(N, nsets));
  o += L.ws_bytes;
  L.total = o + 256;  // room to align the pool allocation's start
  return L;
}

}  // namespace

struct vq_server;

struct Lane {
  vq_server* s = nullptr;
  std::thread thr;
  cudaStream_t st = nullptr;
  vq::Ctx* ctx = nullptr;
};

struct vq_server {
  vq_server_config cfg{};
  int nlanes = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> all;
  std::deque<uint64_t> finished;  // tickets in completion order (for vq_server_wait_any)
  uint64_t next_ticket = 1;
  bool stop = false;
  std::vector<Lane*> lanes;
  cudaMemPool_t pool = nullptr;
  // pinned staging of submitted points (under mu): free extents offset -> bytes
  char* pinned = nullptr;
  size_t pinned_cap = 0;
  vq::Extents pin_free;
  // admission state (under mu)
  long long resident = 0;  // requests admitted and not finished
  size_t used = 0;         // device bytes of the admitted batches
  int busy = 0;            // lanes running a batch
  // statistics (under mu)
  std::vector<double> lat_ms;
  Clock::time_point t_first{};
  Clock::time_point t_last{};
  bool any_submitted = false;
  vq_server_info info{};
};

static size_t batch_bytes(long long points, int sets) { return batch_layout(points, sets).total; }

// How many queued requests a lane admits now, FIFO from the head, within
// the request slots and the memory budget (caller holds mu); limit > 0
// looks at no more than that many requests.
static int admit_count(const vq_server* s, int limit, long long* points, size_t* bytes) {
  int nq = (int)std::min<size_t>(s->queue.size(), (size_t)std::max<long long>(s->cfg.max_inflight - s->resident, 0));
  if (limit > 0) nq = std::min(nq, limit);
  std::vector<int64_t> sizes((size_t)nq);
  for (int i = 0; i < nq; i++) sizes[(size_t)i] = s->queue[(size_t)i]->n;
  int k = vq::admit_prefix(sizes.data(), nq, s->resident, s->used, kBytesFixed, s->cfg.max_inflight,
                           s->cfg.mem_budget_bytes, batch_bytes, points, bytes);
  if (k > 1) {
    long long pts = 0;
    const int j = vq::batch_prefix(sizes.data(), k, kBatchPoints, &pts);
    if (j < k) {
      k = j;
      *points = pts;
      *bytes = batch_bytes(pts, k);
    }
  }
  return k;
}

// The queue's head can be admitted now (caller holds mu).
static bool admissible(const vq_server* s) {
  long long pts = 0;
  size_t bytes = 0;
  return admit_count(s, 1, &pts, &bytes) > 0;
}

// Copies in, runs and copies out one batch on the lane's stream.
static vq_status run_batch(vq_server* s, Lane* L, const std::vector<Request*>& batch, long long N,
                           const BatchLayout& B, std::vector<int64_t>& hoff, std::vector<int32_t>& out) {
  const int ns = (int)batch.size();
  char* base = nullptr;
  if (cudaMallocFromPoolAsync(reinterpret_cast<void**>(&base), B.total, s->pool, L->st) != cudaSuccess) {
    cudaGetLastError();
    return VQ_ERR_NOMEM;
  }
  // every piece of the layout starts on a 256-byte boundary
  char* mem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(base) + 255) & ~uintptr_t(255));
  double* dx = reinterpret_cast<double*>(mem + B.x);
  double* dy = reinterpret_cast<double*>(mem + B.y);
  int32_t* dout = reinterpret_cast<int32_t*>(mem + B.out);
  int64_t* doff = reinterpret_cast<int64_t*>(mem + B.off);
  int64_t* dhoff = reinterpret_cast<int64_t*>(mem + B.hoff);
  std::vector<int64_t> offs(ns + 1, 0);
  for (int i = 0; i < ns; i++) offs[i + 1] = offs[i] + batch[i]->n;
  vq_status st = VQ_OK;
  long long total = 0;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < ns && e == cudaSuccess; i++) {
    const Request* r = batch[i];
    if (r->n == 0) continue;
    const double* hx = r->px ? r->px : r->x.data();
    const double* hy = r->px ? r->px + r->n : r->y.data();
    e = cudaMemcpyAsync(dx + offs[i], hx, sizeof(double) * r->n, cudaMemcpyHostToDevice, L->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy + offs[i], hy, sizeof(double) * r->n, cudaMemcpyHostToDevice, L->st);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(doff, offs.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice, L->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    st = VQ_ERR_CUDA;
  } else {
    st = vq::batched_run(L->ctx, mem + B.ws, B.ws_bytes, dx, dy, reinterpret_cast<const long long*>(doff), ns, N,
                         dout, reinterpret_cast<long long*>(dhoff), L->st, &total);
  }
  if (st == VQ_OK || st == VQ_ERR_NONFINITE) {
    // the run ended with a synchronisation and returned the total, so the
    // offsets and the vertices come back in one round trip
    hoff.assign(ns + 1, 0);
    out.resize((size_t)std::max<long long>(total, 1));
    e = cudaMemcpyAsync(hoff.data(), dhoff, sizeof(int64_t) * (ns + 1), cudaMemcpyDeviceToHost, L->st);
    if (e == cudaSuccess && total > 0)
      e = cudaMemcpyAsync(out.data(), dout, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, L->st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      st = VQ_ERR_CUDA;
    }
  }
  cudaFreeAsync(base, L->st);
  if (cudaStreamSynchronize(L->st) != cudaSuccess) {
    cudaGetLastError();
    if (st == VQ_OK) st = VQ_ERR_CUDA;
  }
  return st;
}

static void lane_main(vq_server* s, Lane* L) {
  cudaSetDevice(s->cfg.device);
  for (;;) {
    std::vector<Request*> batch;
    long long N = 0;
    BatchLayout B{};
    {
      std::unique_lock<std::mutex> g(s->mu);
      s->cv_work.wait(g, [&] { return s->stop || admissible(s); });
      if (s->stop) break;
      // FIFO from the head while request slots and memory allow
      size_t bytes = 0;
      const int k = admit_count(s, 0, &N, &bytes);
      for (int i = 0; i < k; i++) {
        batch.push_back(s->queue.front());
        s->queue.pop_front();
      }
      B = batch_layout(N, k);
      if (s->busy > 0) s->info.admitted_while_busy += (long long)batch.size();
      s->busy++;
      s->resident += (long long)batch.size();
      s->used += B.total;
      s->info.batches++;
      s->info.max_busy_lanes = std::max<int64_t>(s->info.max_busy_lanes, s->busy);
      s->info.peak_bytes = std::max<int64_t>(s->info.peak_bytes, (int64_t)s->used);
    }
    // other idle lanes may admit what is left
    s->cv_work.notify_all();
    std::vector<int64_t> hoff;
    std::vector<int32_t> out;
    const vq_status st = run_batch(s, L, batch, N, B, hoff, out);
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
        r->x.clear();
        r->x.shrink_to_fit();
        r->y.clear();
        r->y.shrink_to_fit();
        if (r->px) {  // the batch's copies are done (run_batch synchronised its stream)
          s->pin_free.give(r->pin_off, r->pin_len);
          r->px = nullptr;
        }
        r->done = true;
        r->t_done = now;
        s->finished.push_back(r->ticket);
        s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
        s->info.completed++;
        s->t_last = now;
      }
      s->busy--;
      s->resident -= (long long)batch.size();
      s->used -= B.total;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

static void server_free(vq_server* s) {
  for (Lane* L : s->lanes) {
    if (L->ctx) vq::ctx_destroy(L->ctx);
    if (L->st) cudaStreamDestroy(L->st);
    delete L;
  }
  s->lanes.clear();
  if (s->pool) cudaMemPoolDestroy(s->pool);
  s->pool = nullptr;
  if (s->pinned) cudaFreeHost(s->pinned);
  s->pinned = nullptr;
  for (auto& kv : s->all) delete kv.second;
  s->all.clear();
  delete s;
}

extern "C" {

vq_status vq_server_create(const vq_server_config* cfg, vq_server** out) {
  if (!cfg || !out || cfg->max_inflight < 1 || cfg->mem_budget_bytes < kBytesFixed || cfg->lanes < 0 ||
      cfg->lanes > kMaxLanes)
    return VQ_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return VQ_ERR_CUDA;
  if (cfg->device < 0 || cfg->device >= ndev) return VQ_ERR_INVALID_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(cfg->device) != cudaSuccess) return VQ_ERR_CUDA;
  vq_server* s = new vq_server();
  s->cfg = *cfg;
  s->nlanes = cfg->lanes > 0 ? cfg->lanes : kDefaultLanes;
  s->info.budget_bytes = (int64_t)cfg->mem_budget_bytes;
  vq_status st = VQ_OK;
  cudaMemPoolProps props;
  memset(&props, 0, sizeof props);
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = cfg->device;
  if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
    s->pool = nullptr;
    st = VQ_ERR_CUDA;
  } else {
    // freed batches stay cached in the pool up to the budget
    unsigned long long keep = (unsigned long long)cfg->mem_budget_bytes;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  // pinned staging area for submitted points (device copies from it run at
  // the link's speed and asynchronously); without it, pageable copies
  if (st == VQ_OK) {
    size_t cap = cfg->pinned_bytes ? cfg->pinned_bytes : std::min<size_t>(cfg->mem_budget_bytes, kDefaultPinned);
    cap &= ~size_t(255);
    if (cap >= 256 && cudaMallocHost(&s->pinned, cap) == cudaSuccess) {
      s->pinned_cap = cap;
      s->pin_free.give(0, cap);
    } else {
      cudaGetLastError();
      s->pinned = nullptr;
    }
  }
  for (int i = 0; i < s->nlanes && st == VQ_OK; i++) {
    Lane* L = new Lane();
    L->s = s;
    s->lanes.push_back(L);
    if (cudaStreamCreateWithFlags(&L->st, cudaStreamNonBlocking) != cudaSuccess) {
      L->st = nullptr;
      st = VQ_ERR_CUDA;
    } else if (!(L->ctx = vq::ctx_create())) {
      st = VQ_ERR_NOMEM;
    }
  }
  if (st != VQ_OK) {
    cudaGetLastError();
    server_free(s);
    cudaSetDevice(prev);
    return st;
  }
  for (Lane* L : s->lanes) L->thr = std::thread(lane_main, s, L);
  cudaSetDevice(prev);
  *out = s;
  return VQ_OK;
}

vq_status vq_server_submit(vq_server* s, const double* x_host, const double* y_host, int64_t n, uint64_t* ticket) {
  const auto t0 = Clock::now();
  if (!s || !ticket || n < 0 || (n > 0 && (!x_host || !y_host))) return VQ_ERR_INVALID_ARG;
  if (n > (int64_t)INT32_MAX - 2) return VQ_ERR_TOO_LARGE;
  if (batch_layout(n, 1).total + kBytesFixed > s->cfg.mem_budget_bytes) return VQ_ERR_BUDGET;
  Request* r = new Request();
  r->n = n;
  r->t_submit = t0;
  // the points go to the pinned staging area when it has room, else to
  // pageable memory
  size_t off = 0;
  const size_t bytes = (sizeof(double) * 2 * (size_t)n + 255) & ~size_t(255);
  bool pinned = false;
  if (n > 0 && s->pinned) {
    std::lock_guard<std::mutex> g(s->mu);
    pinned = s->pin_free.take(bytes, &off);
  }
  if (pinned) {
    r->px = reinterpret_cast<double*>(s->pinned + off);
    r->pin_off = off;
    r->pin_len = bytes;
    memcpy(r->px, x_host, sizeof(double) * (size_t)n);
    memcpy(r->px + n, y_host, sizeof(double) * (size_t)n);
  } else {
    r->x.assign(x_host, x_host + n);
    r->y.assign(y_host, y_host + n);
  }
  {
    std::lock_guard<std::mutex> g(s->mu);
    r->ticket = s->next_ticket++;
    if (!s->any_submitted) {
      s->t_first = t0;
      s->any_submitted = true;
    }
    s->all[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv_work.notify_all();
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

vq_status vq_server_wait_any(vq_server* s, uint64_t* ticket, int32_t* hull_idx_host, int64_t cap, int64_t* h,
                             int32_t timeout_ms, double* latency_ms) {
  if (!s || !ticket || !h) return VQ_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> g(s->mu);
  // the oldest finished request that poll / wait have not taken yet
  auto next = [&]() -> Request* {
    while (!s->finished.empty()) {
      auto it = s->all.find(s->finished.front());
      if (it != s->all.end()) return it->second;
      s->finished.pop_front();
    }
    return nullptr;
  };
  Request* r = next();
  if (!r) {
    auto pred = [&] { return (r = next()) != nullptr; };
    if (timeout_ms < 0) s->cv_done.wait(g, pred);
    else s->cv_done.wait_for(g, std::chrono::milliseconds(timeout_ms), pred);
  }
  if (!r) return VQ_PENDING;
  *ticket = r->ticket;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  *h = (int64_t)r->hull.size();
  if (r->status == VQ_OK && (cap < *h || (*h > 0 && !hull_idx_host))) {
    s->finished.pop_front();  // stays available to vq_server_wait / vq_server_poll
    return VQ_ERR_CAPACITY;
  }
  s->finished.pop_front();
  const vq_status st = r->status;
  if (st == VQ_OK && *h > 0) memcpy(hull_idx_host, r->hull.data(), sizeof(int32_t) * r->hull.size());
  s->all.erase(r->ticket);
  delete r;
  return st;
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
    *hulls_per_s = (sec > 0.0) ? (double)s->info.completed / sec : 0.0;
  }
  return VQ_OK;
}

vq_status vq_server_info_read(vq_server* s, vq_server_info* out) {
  if (!s || !out) return VQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  *out = s->info;
  return VQ_OK;
}

void vq_server_destroy(vq_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (Lane* L : s->lanes)
    if (L->thr.joinable()) L->thr.join();
  int prev = 0;
  const bool have_prev = cudaGetDevice(&prev) == cudaSuccess;
  cudaSetDevice(s->cfg.device);
  server_free(s);
  if (have_prev) cudaSetDevice(prev);
}

}  // extern "C"
