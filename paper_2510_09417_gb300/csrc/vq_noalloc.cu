// vq_noalloc.cu -- vq_hull2d_noalloc: the single-hull path for callers that
// must not allocate.
//
// Some callers cannot let a library call cudaMalloc (or cudaMallocHost, or
// any allocating routine): real-time or embedded hosts that forbid
// allocation after start-up, because an allocation can stall or fail at
// an unpredictable moment, and processes whose device memory is owned by a
// pool allocator that must account for every byte.  vq_hull2d allocates its
// workspace lazily, so this entry point runs the same kernels out of one
// fixed block of device memory instead: the file-scope array below.  It is
// part of the module, so every GPU that loads this library reserves it
// (64 MiB) until the process exits.  The call waits for its stream before
// it returns.
//
// The workspace for n points needs about 46 bytes per point plus tables;
// kNoAllocMaxPoints (2^20) is the largest n that fits, and larger n is
// rejected with VQ_ERR_TOO_LARGE before any device work.
#include <climits>
#include <cstring>
#include <mutex>

#include "../../include/vqhull.h"
#include "vq_internal.h"

namespace vq {
namespace {

constexpr long long kNoAllocMaxPoints = 1ll << 20;
constexpr size_t kNoAllocBytes = 64ull << 20;
constexpr int kNoAllocPPT = 16;          // partition tile: 32 lanes x 16 points
constexpr int kNoAllocSmallMax = 1024;   // small-segment threshold

// The scratch.  Host code must not use this name as an address: it has to
// ask the runtime for the device address of the symbol (see setup()).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct DeviceState {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  int sms = 0;
};

std::mutex g_mu;
DeviceState g_dev[64];
Ctrl g_ctrl_host;  // plain host memory: control words read back each level
Work g_work_host;  // plain host memory: the source of the Work copy in the scratch

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

// Same carving as the allocating path, into the fixed scratch, with the
// fixed tiling above.  Returns the bytes needed (base == nullptr: size only).
size_t carve(Work& w, unsigned char* base, long long n, long long** scan_tmp) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> unsigned char* {
    unsigned char* p = base ? base + off : nullptr;
    off += up256(bytes > 0 ? bytes : 1);
    return p;
  };
  const int nsets = 1;
  const long long nkeys = n + nsets;
  for (int b = 0; b < 2; b++) {
    w.bx[b] = reinterpret_cast<double*>(take(sizeof(double) * n + 16));  // 16-byte tail pad for bulk copies
    w.by[b] = reinterpret_cast<double*>(take(sizeof(double) * n + 16));
    w.bi[b] = reinterpret_cast<int*>(take(sizeof(int) * n + 16));
  }
  w.nkeys = nkeys;
  w.slot = reinterpret_cast<int*>(take(sizeof(int) * (nkeys + 1)));
  w.bitmap = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * ((nkeys + 31) / 32 + 1)));
  w.sets = reinterpret_cast<SetRec*>(take(sizeof(SetRec) * nsets));
  w.k0_tile_start = reinterpret_cast<int*>(take(sizeof(int) * (nsets + 1)));
  w.capT0 = (int)(n / kK0Tile + nsets + 1);
  w.k0part = reinterpret_cast<K0Part*>(take(sizeof(K0Part) * w.capT0));
  w.small_max = kNoAllocSmallMax;
  w.tile = kWarp * kNoAllocPPT;  // partition tile: one warp's points
  w.capS = (int)(n / (kNoAllocSmallMax + 1) + 2);
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
  w.ctrl = reinterpret_cast<Ctrl*>(take(sizeof(Ctrl)));
  w.dev = reinterpret_cast<const Work*>(take(sizeof(Work)));  // the level loop's kernels read Work there
  w.stats = reinterpret_cast<long long*>(take(sizeof(long long) * 3 * kMaxLevels));
  const long long nwords = (nkeys + 31) / 32;
  const long long nb = (nwords + kK4Words - 1) / kK4Words;
  const long long a = nb + 1 + scan_tmp_elems(nb + 1);
  const long long b = scan_tmp_elems(nsets + 1);
  unsigned char* t = take(sizeof(long long) * (a > b ? a : b));
  if (scan_tmp) *scan_tmp = reinterpret_cast<long long*>(t);
  return off;
}

// Once per device, with that device current: the device address of the
// scratch symbol, the SM count and the partition kernel's occupancy.
vq_status setup(int dev, DeviceState& d) {
  if (d.ready) return VQ_OK;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return VQ_ERR_CUDA;
  }
  if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return VQ_ERR_CUDA;
  d.scratch = static_cast<unsigned char*>(p);
  d.ready = true;
  return VQ_OK;
}

}  // namespace
}  // namespace vq

using namespace vq;

extern "C" vq_status vq_hull2d_noalloc(const double* x, const double* y, int64_t n, int32_t* hull_idx, int64_t* h,
                                       void* stream) {
  if (!h || n < 0) return VQ_ERR_INVALID_ARG;
  *h = 0;
  if (n == 0) return VQ_OK;
  if (!x || !y || !hull_idx) return VQ_ERR_INVALID_ARG;
  if (n > kNoAllocMaxPoints) return VQ_ERR_TOO_LARGE;
  Work w;
  memset(&w, 0, sizeof w);
  if (carve(w, nullptr, n, nullptr) > kNoAllocBytes) return VQ_ERR_TOO_LARGE;

  std::lock_guard<std::mutex> g(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VQ_ERR_CUDA;
  DeviceState& d = g_dev[dev];
  vq_status s = setup(dev, d);
  if (s != VQ_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  long long* scan_tmp = nullptr;
  carve(w, d.scratch, n, &scan_tmp);
  w.x = x;
  w.y = y;
  w.offsets = nullptr;
  w.key_base = nullptr;
  w.n_single = n;
  w.nsets = 1;
  w.N = (int)n;
  w.timeout_ns = config_timeout_ns();  // the bound of vq_config, as on the allocating path
  w.drop_tile = -1;
  w.ordered = 0;

  // on a failure, work already queued may still use the shared array: the
  // stream is drained before the lock is released
#define NA_CHECK(call)                                     \
  do {                                                     \
    if ((call) != cudaSuccess) {                           \
      cudaGetLastError();                                  \
      cudaStreamSynchronize(st);                           \
      cudaGetLastError();                                  \
      return VQ_ERR_CUDA;                                  \
    }                                                      \
  } while (0)

  // the scratch keeps the previous call's contents: clear what the kernels
  // expect to start at zero (control words, counters, the vertex bitmap)
  g_work_host = w;
  NA_CHECK(cudaMemcpyAsync(const_cast<Work*>(w.dev), &g_work_host, sizeof(Work), cudaMemcpyHostToDevice, st));
  NA_CHECK(cudaMemsetAsync(w.ctrl, 0, sizeof(Ctrl), st));
  NA_CHECK(cudaMemsetAsync(w.stats, 0, sizeof(long long) * 3 * kMaxLevels, st));
  NA_CHECK(cudaMemsetAsync(w.bitmap, 0, sizeof(unsigned) * ((w.nkeys + 31) / 32 + 1), st));
  NA_CHECK(launch_seed(w, st));
  NA_CHECK(scan_exclusive_i32(w.k0_tile_start, 2, reinterpret_cast<int*>(scan_tmp), st));
  NA_CHECK(launch_k0(w, d.sms * 2, st));
  NA_CHECK(launch_k0_finalize(w, st));
  NA_CHECK(launch_tilemap(w, 0, d.sms * 4, st));
  NA_CHECK(cudaMemcpyAsync(&g_ctrl_host, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  NA_CHECK(cudaStreamSynchronize(st));
  w.all_fast = g_ctrl_host.any_slow ? 0 : 1;
  long long k1_grid = n / w.tile + 2;  // level 0: at most this many tiles
  for (int level = 0;; level++) {
    NA_CHECK(launch_prologue(w, level, st));
    if (k1_grid > 0) NA_CHECK(launch_k1(w, level, kNoAllocPPT, (int)k1_grid, st));
    NA_CHECK(launch_k2(w, level, d.sms * 8, st));
    NA_CHECK(launch_tilemap(w, (level + 1) & 1, d.sms * 4, st));
    NA_CHECK(launch_k3(w, d.sms * 2, st));
    NA_CHECK(cudaMemcpyAsync(&g_ctrl_host, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    NA_CHECK(cudaStreamSynchronize(st));
    if (g_ctrl_host.err & kErrFatal) break;
    if (g_ctrl_host.k1_segs[(level + 1) & 1] == 0) break;
    k1_grid = g_ctrl_host.k1_tiles[(level + 1) & 1];
    if (level > n + 1) {
      g_ctrl_host.err |= kErrInternal;
      break;
    }
  }
  NA_CHECK(launch_order(w, hull_idx, nullptr, &w.ctrl->total, scan_tmp, st));
  NA_CHECK(cudaMemcpyAsync(&g_ctrl_host, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  NA_CHECK(cudaStreamSynchronize(st));
#undef NA_CHECK
  *h = g_ctrl_host.total;
  const unsigned err = g_ctrl_host.err;
  if (err & kErrTimeout) return VQ_ERR_TIMEOUT;
  if (err & (kErrCapacity | kErrInternal | kErrBadOffsets)) return VQ_ERR_CAPACITY;
  if (err & kErrNonfinite) return VQ_ERR_NONFINITE;
  return VQ_OK;
}
