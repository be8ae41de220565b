// vq_api.cu -- host driver and C ABI of libvqhull (single and batched hulls).
//
// One call runs Alg. 1 (Sec. 2.1) for all point sets at once, one recursion
// level per step: extreme points (k_k0*), then per level the fused
// partition (k_k1), the per-segment finalize (k_k2) and the small-segment
// finisher (k_k3), until no segment is left; then the vertices are put in
// clockwise order (k_k4_*).
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/vqhull.h"
#include "vq_internal.h"

namespace vq {

struct Config {
  int ppt = 16;
  int small_max = 1024;
  int k1_bps = 0;
  int profile = 0;
  int ordered = 0;
  long long timeout_ns = 2000000000ll;
  int drop_tile = -1;
  int host_loop = 0;
  int prefilter = 1;
  int k1_shape = 0;
  long long wl_points = 1ll << 22;  // level-loop handover to the persistent worklist (0: never)
};

static std::mutex g_cfg_mu;
static Config g_cfg;

static Config get_cfg() {
  std::lock_guard<std::mutex> g(g_cfg_mu);
  return g_cfg;
}

long long config_timeout_ns() { return get_cfg().timeout_ns; }

static vq_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return VQ_OK;
  if (e == cudaErrorMemoryAllocation) return VQ_ERR_NOMEM;
  return VQ_ERR_CUDA;
}

// VQ_DEBUG=1 in the environment prints the failing runtime call
static bool debug_on() {
  static const int on = [] {
    const char* v = getenv("VQ_DEBUG");
    return v && v[0] == '1' ? 1 : 0;
  }();
  return on != 0;
}

#define VQ_CHECK(call)                                                                                  \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) {                                                                            \
      if (debug_on()) fprintf(stderr, "vqhull: %s:%d %s: %s\n", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return cuda_status(e_);                                                                           \
    }                                                                                                   \
  } while (0)

// A captured device-driven level loop: one CUDA graph whose WHILE node
// repeats levels >= 1 until no segment is left.  Kernel arguments are fixed
// at capture, so a graph is reused only for the same workspace layout,
// inputs and tuning (the key).
struct LevelGraph {
  std::vector<unsigned char> key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long used = 0;
  int fixed_kernels = 0;  // kernel nodes outside the loop body (level 0, the first test, the worklist)
};
constexpr int kGraphCache = 16;           // graphs kept per device (least recently used goes)
constexpr int kGraphKernelsPerIter = 13;  // two levels of 6 kernels (two partition tiers), and the condition

struct Ctx {
  std::mutex mu;
  bool init = false;
  int device = 0;
  int sms = 0;
  char* mem = nullptr;
  size_t bytes = 0;
  bool external = false;   // mem belongs to the caller (server lanes): never freed or grown here
  Ctrl* h_ctrl = nullptr;  // pinned
  Work* d_work = nullptr;  // the call's Work in device memory (the level loop's kernels read it)
  Work* h_work = nullptr;  // pinned source of its copy
  long long* h_total = nullptr;
  // staging for vq_hull2d_host
  double* stage = nullptr;
  int* stage_out = nullptr;
  long long stage_n = 0;
  // pipelined host path: copy stream, per-chunk events, merge buffers
  cudaStream_t cstream = nullptr;
  std::vector<cudaEvent_t> cev;
  double* mxy = nullptr;  // 2 * mcap doubles: merge x then merge y
  int* mid = nullptr;     // mcap original indices
  int* mout = nullptr;    // mcap merge-hull indices
  long long mcap = 0;
  // last call
  long long* d_stats = nullptr;
  int last_levels = 0;
  int bps_cache[17] = {};
  // profile: accumulated counters and an event pool for kernel timing
  vq_profile prof{};
  std::vector<cudaEvent_t> events;
  std::vector<int> ev_kind;  // one entry per (start, stop) pair
  // device-driven level loop: capture stream and the graph cache
  cudaStream_t gstream = nullptr;
  bool graph_off = false;  // a graph could not be built here: host loop from then on
  std::vector<LevelGraph> graphs;
  unsigned long long graph_clock = 0;
  // persistent worklist: where its tag array was last time (a new place is
  // cleared first) and the last epoch published there
  const unsigned* wl_tag = nullptr;
  int wl_tag_cap = 0;
  unsigned wl_epoch = 0;
};

enum { kKindOther = 0, kKindK0, kKindK1, kKindK2, kKindK3, kKindK4, kKindSample, kKindK5 };

// Brackets kernel launches with CUDA events on the call's stream when
// profiling is on; the times are summed per kernel kind after the call.
struct Timer {
  Ctx& c;
  cudaStream_t st;
  bool on;
  int open = -1;
  Timer(Ctx& c_, cudaStream_t st_, bool on_) : c(c_), st(st_), on(on_) { c.ev_kind.clear(); }
  cudaError_t begin(int kind) {
    if (!on) return cudaSuccess;
    const size_t pair = c.ev_kind.size();
    while (c.events.size() < 2 * (pair + 1)) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      c.events.push_back(e);
    }
    c.ev_kind.push_back(kind);
    open = (int)pair;
    return cudaEventRecord(c.events[2 * pair], st);
  }
  cudaError_t end() {
    if (!on || open < 0) return cudaSuccess;
    const int pair = open;
    open = -1;
    return cudaEventRecord(c.events[2 * pair + 1], st);
  }
  // call after the stream has been synchronised
  void collect() {
    if (!on) return;
    for (size_t p = 0; p < c.ev_kind.size(); p++) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c.events[2 * p], c.events[2 * p + 1]) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      switch (c.ev_kind[p]) {
        case kKindK0: c.prof.k0_ms += ms; break;
        case kKindK1: c.prof.k1_ms += ms; break;
        case kKindK2: c.prof.k2_ms += ms; break;
        case kKindK3: c.prof.k3_ms += ms; break;
        case kKindK4: c.prof.k4_ms += ms; break;
        case kKindSample: c.prof.sample_ms += ms; break;
        case kKindK5: c.prof.k5_ms += ms; break;
        default: c.prof.other_ms += ms; break;
      }
    }
  }
};

#define VQ_TIMED(timer, kind, call)          \
  do {                                       \
    VQ_CHECK((timer).begin(kind));           \
    VQ_CHECK(call);                          \
    VQ_CHECK((timer).end());                 \
  } while (0)

static Ctx g_ctx[64];


static size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

// Carves the workspace for N points, nsets sets and nkeys order keys.
// With base == nullptr only the size is computed.
static size_t layout(Work& w, char* base, long long N, int nsets, long long nkeys, const Config& cfg) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes > 0 ? bytes : 1);
    return p;
  };
  const long long n = N > 0 ? N : 1;
  for (int b = 0; b < 2; b++) {
    // 16 bytes of padding: the partition kernel's bulk copies may read up
    // to 15 bytes past a tile's last point
    w.bx[b] = reinterpret_cast<double*>(take(sizeof(double) * n + 16));
    w.by[b] = reinterpret_cast<double*>(take(sizeof(double) * n + 16));
    w.bi[b] = reinterpret_cast<int*>(take(sizeof(int) * n + 16));
  }
  w.nkeys = nkeys;
  w.slot = reinterpret_cast<int*>(take(sizeof(int) * (nkeys + 1)));
  w.bitmap = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * ((nkeys + 31) / 32 + 1)));
  w.sets = reinterpret_cast<SetRec*>(take(sizeof(SetRec) * nsets));
  w.sieve = cfg.prefilter ? 1 : 0;
  w.poly = reinterpret_cast<PolyF*>(take(w.sieve ? sizeof(PolyF) * nsets : 0));
  w.dirbest = reinterpret_cast<unsigned long long*>(take(w.sieve ? sizeof(unsigned long long) * kPolyDirs * nsets : 0));
  w.nsurv = reinterpret_cast<int*>(take(w.sieve ? sizeof(int) * nsets : 0));
  w.k0_tile_start = reinterpret_cast<int*>(take(sizeof(int) * (nsets + 1)));
  w.capT0 = (int)(n / kK0Tile + nsets + 1);
  // partials: one per extreme-pass tile, or (sieve) one per block and set
  w.k0part = reinterpret_cast<K0Part*>(take(sizeof(K0Part) * (w.sieve ? (size_t)kSvMaxBlocks + nsets : (size_t)w.capT0)));
  w.small_max = cfg.small_max;
  // partition tile: one warp's (32 x ppt points), or one look-back block's
  w.tile = (cfg.ordered ? kK1Threads : kWarp) * cfg.ppt;
  w.capS = (int)(n / (cfg.small_max + 1) + 2);
  w.capT = (int)(n / w.tile + w.capS + 1);
  w.capQ = 2 * w.capS + nsets + 16;
  w.capJ = w.capT / kFillTiles + w.capS + 1;
  for (int b = 0; b < 2; b++) {
    w.segs[b] = reinterpret_cast<SegRec*>(take(sizeof(SegRec) * w.capS));
    w.geom[b] = reinterpret_cast<SegGeom*>(take(sizeof(SegGeom) * w.capS));
    w.tile_seg[b] = reinterpret_cast<int*>(take(sizeof(int) * w.capT));
    w.tdesc[b] = reinterpret_cast<TileDesc*>(take(sizeof(TileDesc) * w.capT));
    w.fjobs[b] = reinterpret_cast<int4*>(take(sizeof(int4) * w.capJ));
    w.status[b] = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * w.capT));
    w.cand[b] = reinterpret_cast<TileRec*>(take(sizeof(TileRec) * w.capT));
    w.sstate[b] = reinterpret_cast<SegState*>(take(sizeof(SegState) * w.capS));
  }
  w.k3q = reinterpret_cast<SegRec*>(take(sizeof(SegRec) * w.capQ));
  // persistent worklist (not with look-back offsets, whose layout it would
  // not keep).  At the handover a level holds at most m points; the table
  // holds the big segments of the rest of the recursion and the queue their
  // partition tasks and the small segments.  Both bounds are generous, not
  // certain: an overflow makes the call run again with the level loop alone.
  w.wl_points = (cfg.wl_points > 0 && !cfg.ordered) ? cfg.wl_points : 0;
  if (w.wl_points > 0) {
    const long long m = n < w.wl_points ? n : w.wl_points;
    const long long ws = 8 * (m / (cfg.small_max + 1)) + 2LL * nsets + 256;
    const long long wq = 8 * (m / kWlTaskPts) + 3 * ws + nsets + 1024;
    w.capWS = (int)(ws < (1LL << 30) ? ws : (1LL << 30));
    w.capWQ = (int)(wq < (1LL << 30) ? wq : (1LL << 30));
    // test knob: VQ_WL_QUEUE_CAP=k caps the queue at k entries (the
    // overflow path: the call runs again with the level loop alone)
    if (const char* e = getenv("VQ_WL_QUEUE_CAP")) {
      const long long k = atoll(e);
      if (k > 0 && k < w.capWQ) w.capWQ = (int)k;
    }
  } else {
    w.capWS = 0;
    w.capWQ = 0;
  }
  w.wlq = reinterpret_cast<WlTask*>(take(sizeof(WlTask) * (size_t)w.capWQ));
  w.wltag = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * (size_t)w.capWQ));
  w.wlrec = reinterpret_cast<BestRec*>(take(2 * sizeof(BestRec) * (size_t)w.capWQ));
  w.wlseg = reinterpret_cast<WlSeg*>(take(sizeof(WlSeg) * (size_t)w.capWS));
  w.ctrl = reinterpret_cast<Ctrl*>(take(sizeof(Ctrl)));
  w.stats = reinterpret_cast<long long*>(take(sizeof(long long) * 3 * kMaxLevels));
  return off;
}

// scratch for the scans (int64), placed after the layout
static size_t scan_bytes(long long nkeys, int nsets) {
  const long long nwords = (nkeys + 31) / 32;
  const long long nb = (nwords + kK4Words - 1) / kK4Words;
  long long a = nb + 1 + scan_tmp_elems(nb + 1);
  if (a < order_fused_tmp_elems(nkeys)) a = order_fused_tmp_elems(nkeys);
  const long long b = scan_tmp_elems((long long)nsets + 1);
  return align_up(sizeof(long long) * (a > b ? a : b));
}

static vq_status ctx_init(Ctx& c) {
  if (c.init) return VQ_OK;
  VQ_CHECK(cudaGetDevice(&c.device));
  VQ_CHECK(cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, c.device));
  VQ_CHECK(cudaMallocHost(&c.h_ctrl, sizeof(Ctrl) + 64));
  c.h_total = reinterpret_cast<long long*>(reinterpret_cast<char*>(c.h_ctrl) + sizeof(Ctrl) + 32);
  VQ_CHECK(cudaMallocHost(&c.h_work, sizeof(Work)));
  VQ_CHECK(cudaMalloc(&c.d_work, sizeof(Work)));
  c.init = true;
  return VQ_OK;
}

static vq_status ctx_reserve(Ctx& c, size_t bytes) {
  if (bytes <= c.bytes) return VQ_OK;
  if (c.external) return VQ_ERR_CAPACITY;
  if (c.mem) {
    cudaFree(c.mem);
    c.mem = nullptr;
    c.bytes = 0;
  }
  size_t want = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&c.mem, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&c.mem, bytes);
    want = bytes;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    c.mem = nullptr;
    return VQ_ERR_NOMEM;
  }
  c.bytes = want;
  return VQ_OK;
}

static void graph_free(LevelGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  g.exec = nullptr;
  g.graph = nullptr;
}

// Returns the instantiated level-loop graph for `w` (captured on first use).
// It holds everything after the level-0 segments are made: the level-0
// tile map and level 0 (prologue, partition, finalize, next tile map,
// finisher), then a WHILE node whose body is two levels, parity 1 then
// parity 0, followed by the condition kernel, then (when the worklist is
// on) the worklist's set-up and persistent kernels.  A level whose segment
// count is zero does nothing in any of its kernels, so the second level of
// the last iteration may run empty, and after a handover every level
// kernel finds nothing to do.  All kernels read the call's Work from
// device memory, so the graph depends only on what shapes its launches
// (the key).  The partition kernel gets its persistent grid: it reads the
// level's tile count from the control block.
// With cached_only set, returns VQ_OK and *out = nullptr when no graph for
// `w` is cached yet.
static vq_status level_graph(Ctx& c, const Work& w, const Config& cfg, bool cached_only, cudaGraphExec_t* out) {
  *out = nullptr;
  const int kv[5] = {cfg.ppt, cfg.k1_shape, c.sms, w.sieve, w.capWQ > 0 ? 1 : 0};
  std::vector<unsigned char> key(sizeof kv);
  memcpy(key.data(), kv, sizeof kv);
  for (LevelGraph& g : c.graphs)
    if (g.key == key) {
      g.used = ++c.graph_clock;
      *out = g.exec;
      return VQ_OK;
    }
  if (cached_only) return VQ_OK;
  if (!c.gstream) VQ_CHECK(cudaStreamCreateWithFlags(&c.gstream, cudaStreamNonBlocking));
  LevelGraph g;
  g.key = key;
  VQ_CHECK(cudaGraphCreate(&g.graph, 0));
  const long long before = kernels_launched();
  cudaStream_t gs = c.gstream;
  cudaError_t e = cudaSuccess;
  // level 0, captured into the graph; its last node is the WHILE node's
  // first dependency
  cudaGraphNode_t level0_last = nullptr;
  {
    e = cudaStreamBeginCaptureToGraph(gs, g.graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      e = launch_tilemap(w, 0, c.sms * 4, gs);
      if (e == cudaSuccess) e = launch_prologue(w, 0, gs);
      if (e == cudaSuccess) e = launch_k1(w, 0, cfg.ppt, INT_MAX / 4, gs);
      if (e == cudaSuccess) e = launch_k2(w, 0, c.sms * 8, gs);
      if (e == cudaSuccess) e = launch_tilemap(w, 1, c.sms * 4, gs);
      if (e == cudaSuccess) e = launch_k3(w, c.sms * 2, gs);
      if (e == cudaSuccess) {
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(gs, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
        if (e == cudaSuccess && ndeps == 1) level0_last = deps[0];
        else if (e == cudaSuccess) e = cudaErrorInvalidValue;
      }
      cudaGraph_t captured = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(gs, &captured);
      if (e == cudaSuccess) e = e2;
    }
  }
  // the loop's condition starts at 0 on every launch; a kernel node ahead
  // of the WHILE node sets it from level 0's result, and the body's last
  // kernel sets it for the next iteration
  cudaGraphConditionalHandle h;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g.graph, 0, cudaGraphCondAssignDefault);
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};  // the rest zero
  cudaGraphNode_t init_node, node;
  if (e == cudaSuccess) e = add_loop_init_node(g.graph, &init_node, w, h);
  if (e == cudaSuccess) e = cudaGraphAddDependencies(g.graph, &level0_last, &init_node, nullptr, 1);
  if (e == cudaSuccess) {
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    e = cudaGraphAddNode(&node, g.graph, &init_node, nullptr, 1, &p);
  }
  if (e == cudaSuccess) {
    cudaGraph_t body = p.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(gs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      for (int level = 1; level <= 2 && e == cudaSuccess; level++) {
        if (e == cudaSuccess) e = launch_prologue(w, level, gs);
        if (e == cudaSuccess) e = launch_k1(w, level, cfg.ppt, INT_MAX / 4, gs);
        if (e == cudaSuccess) e = launch_k2(w, level, c.sms * 8, gs);
        if (e == cudaSuccess) e = launch_tilemap(w, (level + 1) & 1, c.sms * 4, gs);
        if (e == cudaSuccess) e = launch_k3(w, c.sms * 2, gs);
      }
      if (e == cudaSuccess) e = launch_level_cond(w, h, gs);
      cudaGraph_t captured = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(gs, &captured);
      if (e == cudaSuccess) e = e2;
    }
  }
  // the rest of the recursion when a level handed it over
  if (e == cudaSuccess && w.capWQ > 0) {
    e = cudaStreamBeginCaptureToGraph(gs, g.graph, &node, nullptr, 1, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      e = launch_worklist(w, gs);
      cudaGraph_t captured = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(gs, &captured);
      if (e == cudaSuccess) e = e2;
    }
  }
  g.fixed_kernels = (int)(kernels_launched() - before) - kGraphKernelsPerIter + 1;  // and the first test
  count_launches(before - kernels_launched());  // capturing launches nothing
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, g.graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    graph_free(g);
    return cuda_status(e);
  }
  if ((int)c.graphs.size() >= kGraphCache) {
    size_t lru = 0;
    for (size_t i = 1; i < c.graphs.size(); i++)
      if (c.graphs[i].used < c.graphs[lru].used) lru = i;
    graph_free(c.graphs[lru]);
    c.graphs.erase(c.graphs.begin() + (long)lru);
  }
  g.used = ++c.graph_clock;
  c.graphs.push_back(g);
  *out = g.exec;
  return VQ_OK;
}

// The level loop shared by the single and batched entry points.
// small_max_override > 0 replaces the small-segment threshold for this run
// (hull-dense inputs finish faster level-synchronously than in the
// shared-memory recursion, which walks one hull vertex per step).
static vq_status run(Ctx& c, const double* x, const double* y, const long long* offsets, long long n_single,
                     int nsets, long long N, int* out, long long* hull_offsets, long long* h_out,
                     cudaStream_t st, int small_max_override = 0, int aos = 0, int wl_off = 0) {
  Config cfg = get_cfg();
  if (small_max_override > 0) cfg.small_max = small_max_override;
  if (wl_off) cfg.wl_points = 0;
  if (aos) {  // interleaved points are read by the sieve only (the pre-filter path)
    cfg.prefilter = 1;
    cfg.ordered = 0;
  }
  const long long nkeys = N + nsets;
  Work w;
  memset(&w, 0, sizeof w);
  const size_t main_bytes = layout(w, nullptr, N, nsets, nkeys, cfg);
  const size_t total = main_bytes + scan_bytes(nkeys, nsets);
  vq_status s = ctx_reserve(c, total);
  if (s != VQ_OK) return s;
  layout(w, c.mem, N, nsets, nkeys, cfg);
  long long* scan_tmp = reinterpret_cast<long long*>(c.mem + main_bytes);
  w.x = x;
  w.y = y;
  w.aos = aos;
  w.offsets = offsets;
  w.key_base = nullptr;
  w.n_single = n_single;
  w.nsets = nsets;
  w.N = (int)N;
  w.timeout_ns = cfg.timeout_ns;
  w.drop_tile = cfg.drop_tile;
  w.ordered = cfg.ordered;
  w.k1_shape = cfg.k1_shape;
  c.d_stats = w.stats;

  // the worklist's queue entries are published with the call's epoch; a
  // tag array in a new place (or an epoch about to wrap) is cleared first
  if (w.capWQ > 0) {
    if (c.wl_tag != w.wltag || c.wl_tag_cap != w.capWQ || c.wl_epoch >= 0xfffffff0u) {
      VQ_CHECK(cudaMemsetAsync(w.wltag, 0, sizeof(unsigned) * (size_t)w.capWQ, st));
      c.wl_tag = w.wltag;
      c.wl_tag_cap = w.capWQ;
      c.wl_epoch = 0;
    }
    w.wl_epoch = ++c.wl_epoch;
  }

  // the level loop's kernels read Work from device memory (one copy per
  // call; h_work is not rewritten before the call's final synchronisation)
  w.dev = c.d_work;
  w.tier_dev = 0;
  w.key_local_clear = nsets == 1 ? 1 : 0;  // one set: the finalize clears just the words its keys reach
  *c.h_work = w;
  VQ_CHECK(cudaMemcpyAsync(c.d_work, c.h_work, sizeof(Work), cudaMemcpyHostToDevice, st));

  const long long launches0 = kernels_launched();
  Timer tm(c, st, cfg.profile != 0);
  VQ_CHECK(tm.begin(kKindOther));
  if (nsets == 1) {  // one kernel clears the counters and seeds the set
    VQ_CHECK(launch_seed_single(w, st));
  } else {
    VQ_CHECK(cudaMemsetAsync(w.ctrl, 0, sizeof(Ctrl), st));
    VQ_CHECK(cudaMemsetAsync(w.stats, 0, sizeof(long long) * 3 * kMaxLevels, st));
    if (!w.key_local_clear)
      VQ_CHECK(cudaMemsetAsync(w.bitmap, 0, sizeof(unsigned) * ((nkeys + 31) / 32 + 1), st));
    VQ_CHECK(launch_seed(w, st));
    VQ_CHECK(scan_exclusive_i32(w.k0_tile_start, (long long)nsets + 1, reinterpret_cast<int*>(scan_tmp), st));
    if (w.sieve) {
      VQ_CHECK(cudaMemsetAsync(w.dirbest, 0, sizeof(unsigned long long) * kPolyDirs * nsets, st));
      VQ_CHECK(cudaMemsetAsync(w.nsurv, 0, sizeof(int) * nsets, st));
    }
  }
  VQ_CHECK(tm.end());
  if (w.sieve) {  // pre-filter path: sample, chains, sieve (the extreme pass over the kept points)
    VQ_CHECK(tm.begin(kKindSample));
    VQ_CHECK(launch_sample(w, st));
    VQ_CHECK(launch_poly(w, st));
    VQ_CHECK(tm.end());
  }
  VQ_CHECK(tm.begin(kKindK0));
  if (w.sieve) {
    VQ_CHECK(launch_sieve(w, st));
  } else {
    VQ_CHECK(launch_k0(w, c.sms * 2, st));  // resident blocks only (2 per SM); tiles of kK0Tile points
  }
  VQ_CHECK(tm.end());
  VQ_TIMED(tm, kKindOther, launch_k0_finalize(w, st));

  int level = 0;
  int levels_run = 0;
  // levels >= 1 on the device (a graph WHILE node) unless the host loop is
  // asked for, per-kernel events are recorded or offsets come from the
  // look-back (whose grid is one block per tile)
  const bool device_loop = !cfg.host_loop && !cfg.profile && !cfg.ordered;
  bool graph_ran = false;
  int graph_fixed = 0;
  cudaGraphExec_t ex = nullptr;
  if (device_loop && !c.graph_off) {
    // the partition kernel's tier is picked on the device, so the call has
    // no host round trip before its end
    w.tier_dev = 1;
    if (level_graph(c, w, cfg, false, &ex) != VQ_OK) {
      c.graph_off = true;  // nothing was launched: the host loop runs instead
      ex = nullptr;
      fprintf(stderr, "vqhull: the device-driven level loop could not be built; using the host loop\n");
    }
    if (!ex) w.tier_dev = 0;
  }
  if (ex) {
    // level 0, every later level and the worklist in one graph launch
    for (const LevelGraph& g : c.graphs)
      if (g.exec == ex) graph_fixed = g.fixed_kernels;
    VQ_CHECK(cudaGraphLaunch(ex, st));
    c.prof.k1_launches++;
    graph_ran = true;
    levels_run = 1;
  } else {
    VQ_TIMED(tm, kKindOther, launch_tilemap(w, 0, c.sms * 4, st));
    // which partition kernel: FP32-only unless some set needs the FP64 tier
    VQ_CHECK(cudaMemcpyAsync(c.h_ctrl, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    VQ_CHECK(cudaStreamSynchronize(st));
    w.all_fast = c.h_ctrl->any_slow ? 0 : 1;
    // one partition block per tile: level 0 uses the bound (one segment per
    // point set), later levels the count the previous level produced
    long long k1_grid = N / w.tile + nsets + 1;
    for (;; level++) {
      VQ_TIMED(tm, kKindOther, launch_prologue(w, level, st));
      if (k1_grid > 0) VQ_TIMED(tm, kKindK1, launch_k1(w, level, cfg.ppt, (int)k1_grid, st));
      c.prof.k1_launches++;
      VQ_TIMED(tm, kKindK2, launch_k2(w, level, c.sms * 8, st));
      VQ_TIMED(tm, kKindOther, launch_tilemap(w, (level + 1) & 1, c.sms * 4, st));
      VQ_TIMED(tm, kKindK3, launch_k3(w, c.sms * 2, st));
      VQ_CHECK(cudaMemcpyAsync(c.h_ctrl, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
      VQ_CHECK(cudaStreamSynchronize(st));
      levels_run = level + 1;
      if (c.h_ctrl->err & kErrFatal) break;
      if (c.h_ctrl->k1_segs[(level + 1) & 1] == 0) break;
      k1_grid = c.h_ctrl->k1_tiles[(level + 1) & 1];
      if (level > N + 1) {  // every level removes at least one point per segment
        c.h_ctrl->err |= kErrInternal;
        break;
      }
    }
  }
  // the rest of the recursion, when a level handed it over (inside the graph
  // when the graph ran)
  if (w.capWQ > 0 && !graph_ran) VQ_TIMED(tm, kKindK5, launch_worklist(w, st));
  VQ_TIMED(tm, kKindK4, launch_order_fused(w, out, hull_offsets, &w.ctrl->total, scan_tmp, st));
  VQ_CHECK(cudaMemcpyAsync(c.h_ctrl, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  VQ_CHECK(cudaStreamSynchronize(st));
  tm.collect();
  if (graph_ran) {
    const long long iters = c.h_ctrl->graph_iters;
    levels_run = 1 + c.h_ctrl->live_levels;
    count_launches(graph_fixed + iters * kGraphKernelsPerIter);  // level 0, first test, worklist; the body
    c.prof.k1_launches += 2 * iters;
    c.prof.graph_launches++;
  }
  if (c.h_ctrl->wl_on && c.h_ctrl->wl_maxlevel > levels_run) levels_run = c.h_ctrl->wl_maxlevel;
  c.last_levels = levels_run;
  c.prof.calls++;
  c.prof.levels += levels_run;
  c.prof.launches += kernels_launched() - launches0;
  c.prof.k1_points_read += c.h_ctrl->k1_read;
  c.prof.k1_points_kept += c.h_ctrl->k1_kept;
  const unsigned err = c.h_ctrl->err;
#ifdef VQ_K1_PROFILE
  {
    const unsigned long long* q = c.h_ctrl->k1prof;
    fprintf(stderr,
            "vqhull k1prof tiles=%llu wait=%llu classify=%llu farthest=%llu atomic=%llu store=%llu issue=%llu "
            "total=%llu far_bounds=%llu far_searches=%llu multi_lane=%llu cands=%llu\n",
            q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], q[8], q[9], q[10], q[11]);
    const unsigned long long* r = c.h_ctrl->k2prof;
    fprintf(stderr, "vqhull k2prof segments=%llu overflow=%llu candidates=%llu scanned=%llu\n", r[0], r[1], r[2],
            r[3]);
    const unsigned long long* k = c.h_ctrl->k3prof;
    fprintf(stderr,
            "vqhull k3prof frames=%llu argmax=%llu geom=%llu classify=%llu points=%llu exact=%llu frame_total=%llu\n",
            k[0], k[1], k[2], k[3], k[4], k[5], k[6]);
  }
#endif
#ifdef VQ_WL_PROFILE
  if (c.h_ctrl->wl_on) {
    const unsigned long long* q = c.h_ctrl->k1prof;
    const unsigned long long t_init = ~q[10], t_start = ~q[6], t_end = q[7];
    fprintf(stderr,
            "vqhull wlprof tiles=%llu small=%llu small_pts=%llu wait_ns=%llu tile_ns=%llu small_ns=%llu "
            "finish_ns=%llu max_small_ns=%llu max_tile_ns=%llu init_to_start_ns=%lld span_ns=%lld "
            "segs=%d tail=%d\n",
            q[0], q[1], q[11], q[2], q[3], q[4], q[5], q[8], q[9], (long long)(t_start - t_init),
            (long long)(t_end - t_start), c.h_ctrl->wl_nseg, (int)(c.h_ctrl->wl_tp >> 32));
    if (const char* tp = getenv("VQ_WL_TRACE")) wl_trace_dump(tp);
    unsigned long long tc[8];
    wl_tier_calls(tc);
    fprintf(stderr,
            "vqhull wlprof fp64_filter_calls=%llu exact_calls=%llu classify_exact=%llu beats_exact=%llu "
            "classify_rel=%llu orient_rel=%llu (kernels of vq_kernels.cu)\n",
            tc[0], tc[1], tc[2], tc[3], tc[4], tc[5]);
    const unsigned long long* g = c.h_ctrl->k2prof;
    fprintf(stderr, "vqhull wlprof record ns: merge0=%llu merge1=%llu cursor=%llu multi_lane_merges=%llu\n", g[0],
            g[1], g[2], g[3]);
    const unsigned long long* f = c.h_ctrl->k3prof;
    fprintf(stderr,
            "vqhull wlprof tile phases ns: seg=%llu classify=%llu (loads=%llu tiers=%llu) sync=%llu record=%llu "
            "store=%llu ticket=%llu\n",
            f[0], f[1], f[6], f[7], f[2], f[3], f[4], f[5]);
  }
#endif
  if (c.h_ctrl->dbg_site)
    fprintf(stderr, "vqhull: bounds check %d failed (value %lld), level loop ran %d levels\n", c.h_ctrl->dbg_site,
            c.h_ctrl->dbg_val, levels_run);
  if ((err & kErrWorklistFull) && !wl_off) {  // the worklist overflowed: the level loop alone
    c.prof.worklist_reruns++;
    return run(c, x, y, offsets, n_single, nsets, N, out, hull_offsets, h_out, st, small_max_override, aos, 1);
  }
  if (h_out) *h_out = c.h_ctrl->total;
  if (err & kErrBadOffsets) return VQ_ERR_INVALID_ARG;
  if (err & kErrTimeout) return VQ_ERR_TIMEOUT;
  if (err & (kErrCapacity | kErrInternal)) return VQ_ERR_CAPACITY;
  if (err & kErrNonfinite) return VQ_ERR_NONFINITE;
  return VQ_OK;
}

static Ctx* current_ctx(vq_status& s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    s = VQ_ERR_CUDA;
    return nullptr;
  }
  s = VQ_OK;
  return &g_ctx[dev];
}

// ---------------------------------------------------------------------------
// Contexts with caller-provided workspaces (the server's lanes)
// ---------------------------------------------------------------------------

Ctx* ctx_create() {
  Ctx* c = new Ctx();
  if (ctx_init(*c) != VQ_OK) {
    ctx_destroy(c);
    return nullptr;
  }
  return c;
}

void ctx_destroy(Ctx* c) {
  if (!c) return;
  for (LevelGraph& g : c->graphs) graph_free(g);
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  for (cudaEvent_t e : c->cev) cudaEventDestroy(e);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  if (c->cstream) cudaStreamDestroy(c->cstream);
  if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
  if (c->h_work) cudaFreeHost(c->h_work);
  if (c->d_work) cudaFree(c->d_work);
  if (c->mem && !c->external) cudaFree(c->mem);
  if (c->stage) cudaFree(c->stage);
  if (c->stage_out) cudaFree(c->stage_out);
  if (c->mxy) cudaFree(c->mxy);
  if (c->mid) cudaFree(c->mid);
  if (c->mout) cudaFree(c->mout);
  delete c;
}

size_t batched_workspace_bytes(long long N, int nsets) {
  const Config cfg = get_cfg();
  Work w;
  memset(&w, 0, sizeof w);
  const long long nkeys = N + nsets;
  return layout(w, nullptr, N, nsets, nkeys, cfg) + scan_bytes(nkeys, nsets);
}

vq_status batched_run(Ctx* c, void* workspace, size_t bytes, const double* x, const double* y,
                      const long long* offsets, int nsets, long long N, int* hull_idx, long long* hull_offsets,
                      cudaStream_t st, long long* h_total) {
  if (!c || !workspace || !offsets || !hull_offsets || nsets < 1 || N < 0) return VQ_ERR_INVALID_ARG;
  if (N + nsets > (long long)INT_MAX - 2) return VQ_ERR_TOO_LARGE;
  if (N > 0 && (!x || !y || !hull_idx)) return VQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  c->mem = static_cast<char*>(workspace);
  c->bytes = bytes;
  c->external = true;
  const vq_status s = run(*c, x, y, offsets, 0, nsets, N, hull_idx, hull_offsets, h_total, st);
  c->mem = nullptr;
  c->bytes = 0;
  c->external = false;
  return s;
}

}  // namespace vq

using namespace vq;


extern "C" {

const char* vq_status_string(int status) {
  switch (status) {
    case VQ_OK: return "ok";
    case VQ_PENDING: return "pending";
    case VQ_ERR_INVALID_ARG: return "invalid argument";
    case VQ_ERR_NONFINITE: return "non-finite coordinate";
    case VQ_ERR_TOO_LARGE: return "too many points for int32 indices";
    case VQ_ERR_NOMEM: return "out of memory";
    case VQ_ERR_CUDA: return "CUDA error";
    case VQ_ERR_TIMEOUT: return "device wait timed out";
    case VQ_ERR_BUDGET: return "request exceeds the memory budget";
    case VQ_ERR_CAPACITY: return "capacity exceeded";
    case VQ_ERR_NOT_FOUND: return "unknown ticket";
    default: return "unknown status";
  }
}

int vq_version(void) { return 100; }

vq_status vq_hull2d(const double* x, const double* y, int64_t n, int32_t* hull_idx, int64_t* h, void* stream) {
  if (!h || n < 0) return VQ_ERR_INVALID_ARG;
  *h = 0;
  if (n == 0) return VQ_OK;
  if (!x || !y || !hull_idx) return VQ_ERR_INVALID_ARG;
  if (n > (int64_t)INT_MAX - 2) return VQ_ERR_TOO_LARGE;
  vq_status s;
  Ctx* c = current_ctx(s);
  if (!c) return s;
  std::lock_guard<std::mutex> g(c->mu);
  if ((s = ctx_init(*c)) != VQ_OK) return s;
  long long hh = 0;
  s = run(*c, x, y, nullptr, n, 1, n, hull_idx, nullptr, &hh, static_cast<cudaStream_t>(stream));
  *h = hh;
  return s;
}

vq_status vq_hull2d_aos(const double* xy, int64_t n, int32_t* hull_idx, int64_t* h, void* stream) {
  if (!h || n < 0) return VQ_ERR_INVALID_ARG;
  *h = 0;
  if (n == 0) return VQ_OK;
  if (!xy || !hull_idx || (reinterpret_cast<uintptr_t>(xy) & 7u) != 0) return VQ_ERR_INVALID_ARG;
  if (n > (int64_t)INT_MAX - 2) return VQ_ERR_TOO_LARGE;
  vq_status s;
  Ctx* c = current_ctx(s);
  if (!c) return s;
  std::lock_guard<std::mutex> g(c->mu);
  if ((s = ctx_init(*c)) != VQ_OK) return s;
  long long hh = 0;
  s = run(*c, xy, xy + 1, nullptr, n, 1, n, hull_idx, nullptr, &hh, static_cast<cudaStream_t>(stream), 0, 1);
  *h = hh;
  return s;
}

vq_status vq_hull2d_batched(const double* x, const double* y, const int64_t* offsets, int32_t nsets,
                            int32_t* hull_idx, int64_t* hull_offsets, void* stream) {
  if (!offsets || !hull_offsets || nsets < 1) return VQ_ERR_INVALID_ARG;
  vq_status s;
  Ctx* c = current_ctx(s);
  if (!c) return s;
  std::lock_guard<std::mutex> g(c->mu);
  if ((s = ctx_init(*c)) != VQ_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  long long N = 0;
  VQ_CHECK(cudaMemcpyAsync(c->h_total, offsets + nsets, sizeof(long long), cudaMemcpyDeviceToHost, st));
  VQ_CHECK(cudaStreamSynchronize(st));
  N = *c->h_total;
  if (N < 0) return VQ_ERR_INVALID_ARG;
  if (N + nsets > (long long)INT_MAX - 2) return VQ_ERR_TOO_LARGE;
  if (N > 0 && (!x || !y || !hull_idx)) return VQ_ERR_INVALID_ARG;
  return run(*c, x, y, reinterpret_cast<const long long*>(offsets), 0, nsets, N, hull_idx,
             reinterpret_cast<long long*>(hull_offsets), nullptr, st);
}

// ---------------------------------------------------------------------------
// Host entry point, pipelined.  The host-to-device link (about 211 GB/s on
// GB300 machines here) moves the points slower than the hull is computed, so
// for large pinned inputs the copy runs in chunks on a second stream while
// each arrived chunk's hull is computed; the answer is then the hull of the
// union of the chunk hulls' vertices (the strict hull of a union is the
// strict hull of the parts' hulls).  The merge buffer lists the chunk hulls
// in chunk order, so among coincident points the lowest merge index is the
// lowest original index and the output is the same as the direct hull's.
// When the chunk hulls grow large (most points on the hull), the call falls
// back to one hull over the staged points.
// ---------------------------------------------------------------------------

constexpr long long kPipeMin = 1ll << 24;       // pipelined from this size
constexpr long long kPipeMinChunk = 1ll << 23;  // chunks of at least this many points,
constexpr int kPipeChunks = 4;                  // and at most this many chunks (each chunk hull has a fixed cost)
// Chunk sizes as fractions of n: the last chunk is the smallest, so little
// hull work is left when the last copy lands; every other chunk's hull
// still finishes before the next chunk has arrived.
constexpr double kPipeFrac[kPipeChunks] = {0.30, 0.30, 0.25, 0.15};
constexpr int kMergeSmallMax = 32;              // small-segment threshold of the merge hull

static bool host_pinned(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// Returns VQ_OK with *done = false when the caller should run the plain
// path on the (fully staged) points.
static vq_status host_pipelined(Ctx& c, const double* xh, const double* yh, long long n, int32_t* out_h,
                                long long* h, cudaStream_t st, bool* done) {
  *done = false;
  // chunk k is [bnd[k], bnd[k+1]); starts stay 2 KB aligned
  long long bnd[kPipeChunks + 1];
  long long nchunks = 0;
  bnd[0] = 0;
  double acc = 0.0;
  for (int k = 0; k < kPipeChunks; k++) {
    acc += kPipeFrac[k];
    long long e = k == kPipeChunks - 1 ? n : (((long long)(acc * (double)n)) + 255) & ~255ll;
    if (e > n) e = n;
    if (e - bnd[nchunks] < kPipeMinChunk && e < n) continue;  // too small: joins the next chunk
    bnd[++nchunks] = e;
    if (e == n) break;
  }
  if (nchunks > 1 && bnd[nchunks] - bnd[nchunks - 1] < kPipeMinChunk) {  // a short tail joins its predecessor
    bnd[nchunks - 1] = n;
    nchunks--;
  }
  if (nchunks < 2) {  // nothing to overlap: stage the points for the plain path
    VQ_CHECK(cudaMemcpyAsync(c.stage, xh, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    VQ_CHECK(cudaMemcpyAsync(c.stage + n, yh, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    return VQ_OK;
  }
  const long long mmax = n / 8;  // merge budget: beyond it the plain path is cheaper
  if (!c.cstream) VQ_CHECK(cudaStreamCreateWithFlags(&c.cstream, cudaStreamNonBlocking));
  while ((long long)c.cev.size() < nchunks + 1) {
    cudaEvent_t e;
    VQ_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c.cev.push_back(e);
  }
  if (c.mcap < mmax) {
    if (c.mxy) cudaFree(c.mxy);
    if (c.mid) cudaFree(c.mid);
    if (c.mout) cudaFree(c.mout);
    c.mxy = nullptr;
    c.mid = nullptr;
    c.mout = nullptr;
    c.mcap = 0;
    if (cudaMalloc(&c.mxy, sizeof(double) * 2 * mmax) != cudaSuccess ||
        cudaMalloc(&c.mid, sizeof(int) * mmax) != cudaSuccess || cudaMalloc(&c.mout, sizeof(int) * mmax) != cudaSuccess) {
      cudaGetLastError();
      return VQ_ERR_NOMEM;
    }
    c.mcap = mmax;
  }
  // the workspace for a full-size run, reserved before any chunk runs (the
  // fallback may need it; no allocation happens between chunks)
  {
    const Config cfg = get_cfg();
    Work w;
    memset(&w, 0, sizeof w);
    const size_t total = layout(w, nullptr, n, 1, n + 1, cfg) + scan_bytes(n + 1, 1);
    vq_status s = ctx_reserve(c, total);
    if (s != VQ_OK) return s;
  }
  double* sx = c.stage;
  double* sy = c.stage + n;
  // copies: after any earlier work on `st`, all chunks back to back
  VQ_CHECK(cudaEventRecord(c.cev[nchunks], st));
  VQ_CHECK(cudaStreamWaitEvent(c.cstream, c.cev[nchunks], 0));
  for (long long k = 0; k < nchunks; k++) {
    const long long off = bnd[k], len = bnd[k + 1] - bnd[k];
    VQ_CHECK(cudaMemcpyAsync(sx + off, xh + off, sizeof(double) * len, cudaMemcpyHostToDevice, c.cstream));
    VQ_CHECK(cudaMemcpyAsync(sy + off, yh + off, sizeof(double) * len, cudaMemcpyHostToDevice, c.cstream));
    VQ_CHECK(cudaEventRecord(c.cev[k], c.cstream));
  }
  vq_status result = VQ_OK;
  long long m = 0;
  bool merge = true;
  for (long long k = 0; k < nchunks; k++) {
    const long long off = bnd[k], len = bnd[k + 1] - bnd[k];
    if (cudaStreamWaitEvent(st, c.cev[k], 0) != cudaSuccess) {
      cudaGetLastError();
      result = VQ_ERR_CUDA;
      break;
    }
    long long hk = 0;
    vq_status s = run(c, sx + off, sy + off, nullptr, len, 1, len, c.stage_out + off, nullptr, &hk, st);
    if (s != VQ_OK) {
      result = s;
      merge = false;
      break;
    }
    if (m + hk > mmax) {
      merge = false;
      break;
    }
    if (launch_gather(sx + off, sy + off, c.stage_out + off, hk, off, c.mxy + m, c.mxy + mmax + m, c.mid + m, st) !=
        cudaSuccess) {
      cudaGetLastError();
      result = VQ_ERR_CUDA;
      break;
    }
    m += hk;
  }
  // the copies read the caller's buffers: they end before this call returns
  VQ_CHECK(cudaStreamSynchronize(c.cstream));
  if (result != VQ_OK) return result;
  if (!merge) {
    VQ_CHECK(cudaStreamWaitEvent(st, c.cev[nchunks - 1], 0));
    return VQ_OK;  // *done stays false: plain path over the staged points
  }
  // the merge input is the chunk hulls' vertices: nearly every point is a
  // hull vertex, so it runs level-synchronously to the end
  long long hm = 0;
  vq_status s = run(c, c.mxy, c.mxy + mmax, nullptr, m, 1, m, c.mout, nullptr, &hm, st, kMergeSmallMax);
  if (s != VQ_OK) return s;
  VQ_CHECK(launch_map_indices(c.mout, c.mid, hm, c.stage_out, st));
  if (hm > 0) VQ_CHECK(cudaMemcpyAsync(out_h, c.stage_out, sizeof(int) * hm, cudaMemcpyDeviceToHost, st));
  VQ_CHECK(cudaStreamSynchronize(st));
  *h = hm;
  *done = true;
  return VQ_OK;
}

vq_status vq_hull2d_host(const double* x_host, const double* y_host, int64_t n, int32_t* hull_idx_host,
                         int64_t* h, void* stream) {
  if (!h || n < 0) return VQ_ERR_INVALID_ARG;
  *h = 0;
  if (n == 0) return VQ_OK;
  if (!x_host || !y_host || !hull_idx_host) return VQ_ERR_INVALID_ARG;
  if (n > (int64_t)INT_MAX - 2) return VQ_ERR_TOO_LARGE;
  vq_status s;
  Ctx* c = current_ctx(s);
  if (!c) return s;
  std::lock_guard<std::mutex> g(c->mu);
  if ((s = ctx_init(*c)) != VQ_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (c->stage_n < n) {
    if (c->stage) cudaFree(c->stage);
    if (c->stage_out) cudaFree(c->stage_out);
    c->stage = nullptr;
    c->stage_out = nullptr;
    c->stage_n = 0;
    if (cudaMalloc(&c->stage, sizeof(double) * 2 * n) != cudaSuccess ||
        cudaMalloc(&c->stage_out, sizeof(int) * n) != cudaSuccess) {
      cudaGetLastError();
      if (c->stage) cudaFree(c->stage);
      c->stage = nullptr;
      c->stage_out = nullptr;
      return VQ_ERR_NOMEM;
    }
    c->stage_n = n;
  }
  if (n >= kPipeMin && host_pinned(x_host) && host_pinned(y_host)) {
    bool done = false;
    long long hp = 0;
    s = host_pipelined(*c, x_host, y_host, n, hull_idx_host, &hp, st, &done);
    if (s != VQ_OK) return s;
    if (done) {
      *h = hp;
      return VQ_OK;
    }
  } else {
    VQ_CHECK(cudaMemcpyAsync(c->stage, x_host, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    VQ_CHECK(cudaMemcpyAsync(c->stage + n, y_host, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  }
  long long hh = 0;
  s = run(*c, c->stage, c->stage + n, nullptr, n, 1, n, c->stage_out, nullptr, &hh, st);
  if (s != VQ_OK && s != VQ_ERR_NONFINITE) return s;
  *h = hh;
  if (hh > 0) {
    VQ_CHECK(cudaMemcpyAsync(hull_idx_host, c->stage_out, sizeof(int) * hh, cudaMemcpyDeviceToHost, st));
    VQ_CHECK(cudaStreamSynchronize(st));
  }
  return s;
}

vq_status vq_autotune(const double* x, const double* y, int64_t n, int32_t reps, vq_config* best, double* best_ms,
                      void* stream) {
  if (n <= 0 || !x || !y || reps < 1 || reps > 16) return VQ_ERR_INVALID_ARG;
  if (n > (int64_t)INT_MAX - 2) return VQ_ERR_TOO_LARGE;
  vq_status s;
  Ctx* c = current_ctx(s);
  if (!c) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* out = nullptr;
  if (cudaMalloc(&out, sizeof(int) * (size_t)n) != cudaSuccess) {
    cudaGetLastError();
    return VQ_ERR_NOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    cudaFree(out);
    return VQ_ERR_CUDA;
  }
  const Config base = get_cfg();
  Config win = base;
  double win_ms = -1.0;
  long long h0 = -1;
  vq_status result = VQ_OK;
  const int ppts[2] = {8, 16}, smalls[2] = {256, 1024}, pres[2] = {0, 1};
  for (int a = 0; a < 2 && result == VQ_OK; a++)
    for (int b = 0; b < 2 && result == VQ_OK; b++)
      for (int d = 0; d < 2 && result == VQ_OK; d++)
        for (int k = 0; k < 3 && result == VQ_OK; k++) {
        Config cand = base;
        cand.ppt = ppts[a];
        cand.small_max = smalls[b];
        cand.prefilter = pres[d];
        cand.k1_shape = k;
        cand.profile = 0;
        cand.ordered = 0;
        {
          std::lock_guard<std::mutex> g(g_cfg_mu);
          g_cfg = cand;
        }
        std::vector<double> ms;
        for (int r = 0; r <= reps && result == VQ_OK; r++) {
          long long h = 0;
          std::lock_guard<std::mutex> g(c->mu);
          if ((result = ctx_init(*c)) != VQ_OK) break;
          if (r > 0 && cudaEventRecord(e0, st) != cudaSuccess) result = VQ_ERR_CUDA;
          if (result == VQ_OK) result = run(*c, x, y, nullptr, n, 1, n, out, nullptr, &h, st);
          if (result != VQ_OK) break;
          if (h0 < 0) h0 = h;
          if (h != h0) {
            result = VQ_ERR_CAPACITY;
            break;
          }
          if (r > 0) {  // run() synchronised the stream: e1 completes at once
            float t = 0.f;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
              cudaGetLastError();
              result = VQ_ERR_CUDA;
              break;
            }
            ms.push_back(t);
          }
        }
        if (result != VQ_OK) break;
        std::sort(ms.begin(), ms.end());
        const double med = ms[ms.size() / 2];
        if (win_ms < 0.0 || med < win_ms) {
          win_ms = med;
          win = cand;
        }
      }
  win.profile = base.profile;  // timed without per-kernel events and look-back; restored
  win.ordered = base.ordered;
  {
    std::lock_guard<std::mutex> g(g_cfg_mu);
    g_cfg = result == VQ_OK ? win : base;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (result != VQ_OK) return result;
  if (best) vq_get_config(best);
  if (best_ms) *best_ms = win_ms;
  return VQ_OK;
}

vq_status vq_get_config(vq_config* cfg) {
  if (!cfg) return VQ_ERR_INVALID_ARG;
  const Config c = get_cfg();
  memset(cfg, 0, sizeof *cfg);
  cfg->points_per_thread = c.ppt;
  cfg->small_max = c.small_max;
  cfg->k1_blocks_per_sm = c.k1_bps;
  cfg->profile = c.profile;
  cfg->timeout_ns = c.timeout_ns;
  cfg->debug_drop_tile = c.drop_tile;
  cfg->ordered = c.ordered;
  cfg->host_loop = c.host_loop;
  cfg->prefilter = c.prefilter;
  cfg->k1_shape = c.k1_shape;
  cfg->worklist_points = c.wl_points;
  return VQ_OK;
}

vq_status vq_set_config(const vq_config* cfg) {
  if (!cfg) return VQ_ERR_INVALID_ARG;
  if (cfg->points_per_thread != 4 && cfg->points_per_thread != 8 && cfg->points_per_thread != 16)
    return VQ_ERR_INVALID_ARG;
  if (cfg->small_max < 2 || cfg->small_max > kK3Cap) return VQ_ERR_INVALID_ARG;
  if (cfg->k1_blocks_per_sm < 0 || cfg->k1_blocks_per_sm > 32) return VQ_ERR_INVALID_ARG;
  if (cfg->timeout_ns <= 0) return VQ_ERR_INVALID_ARG;
  if (cfg->k1_shape < 0 || cfg->k1_shape > 2) return VQ_ERR_INVALID_ARG;
  if (cfg->worklist_points < 0) return VQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_cfg_mu);
  g_cfg.ppt = cfg->points_per_thread;
  g_cfg.small_max = cfg->small_max;
  g_cfg.k1_bps = cfg->k1_blocks_per_sm;
  g_cfg.profile = cfg->profile ? 1 : 0;
  g_cfg.timeout_ns = cfg->timeout_ns;
  g_cfg.drop_tile = cfg->debug_drop_tile;
  g_cfg.ordered = cfg->ordered ? 1 : 0;
  g_cfg.host_loop = cfg->host_loop ? 1 : 0;
  g_cfg.prefilter = cfg->prefilter ? 1 : 0;
  g_cfg.k1_shape = cfg->k1_shape;
  g_cfg.wl_points = cfg->worklist_points;
  return VQ_OK;
}

vq_status vq_debug_round_f32(const double* v, int64_t m, float* out, void* stream) {
  if (m < 0 || (m > 0 && (!v || !out))) return VQ_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  VQ_CHECK(launch_debug_round_f32(v, m, out, st));
  VQ_CHECK(cudaStreamSynchronize(st));
  return VQ_OK;
}

vq_status vq_debug_orient_f32(const double* tri, int64_t m, int32_t tier, float* d, float* e, void* stream) {
  if (m < 0 || (m > 0 && (!tri || !d || !e)) || tier < 0 || tier > 1) return VQ_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  VQ_CHECK(launch_debug_orient_f32(tri, m, tier, d, e, st));
  VQ_CHECK(cudaStreamSynchronize(st));
  return VQ_OK;
}

vq_status vq_last_stats(int64_t* levels, int64_t* read, int64_t* kept, int64_t* segs, int32_t cap) {
  if (!levels || cap < 0) return VQ_ERR_INVALID_ARG;
  vq_status s;
  Ctx* c = current_ctx(s);
  if (!c) return s;
  std::lock_guard<std::mutex> g(c->mu);
  *levels = 0;
  if (!c->init || !c->d_stats) return VQ_OK;
  std::vector<long long> buf(3 * kMaxLevels);
  VQ_CHECK(cudaMemcpy(buf.data(), c->d_stats, sizeof(long long) * 3 * kMaxLevels, cudaMemcpyDeviceToHost));
  int L = 0;
  for (int l = 0; l < kMaxLevels; l++)
    if (buf[2 * kMaxLevels + l] > 0) L = l + 1;
  *levels = L;
  for (int l = 0; l < L && l < cap; l++) {
    if (read) read[l] = buf[l];
    if (kept) kept[l] = buf[kMaxLevels + l];
    if (segs) segs[l] = buf[2 * kMaxLevels + l];
  }
  return VQ_OK;
}

vq_status vq_profile_read(vq_profile* out, int32_t reset) {
  vq_status s;
  Ctx* c = current_ctx(s);
  if (!c) return s;
  std::lock_guard<std::mutex> g(c->mu);
  if (out) *out = c->prof;
  if (reset) memset(&c->prof, 0, sizeof c->prof);
  return VQ_OK;
}

}  // extern "C"
