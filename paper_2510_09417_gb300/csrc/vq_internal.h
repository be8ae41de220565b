// vq_internal.h -- declarations shared by the kernels and the host driver.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "vq_device.cuh"
#include "../../include/vqhull.h"

namespace vq {

constexpr int kK1Threads = 128;  // partition block: 4 warps, one tile per block
constexpr int kK0Threads = 256;
constexpr int kK0Tile = 32768;      // points per extreme-pass tile
constexpr int kK0Pairs = 2;         // extreme pass: point pairs per array, thread and stage
constexpr int kK0Stages = 4;        // extreme pass: shared-memory ring stages (64 KB per block)
constexpr int kSampleChunk = 4096;  // pre-filter sample: the first kSampleChunk points of every
constexpr int kSampleEvery = 16;    // kSampleEvery-th extreme-pass tile of a set (1/128 of the points)
constexpr int kSvWarps = 8;         // sieve: warps per block
constexpr int kSvMaxBlocks = 4096;  // sieve: most blocks (its partials: one per block and set)
constexpr int kK3Cap = 1024;        // points per segment in the small-segment kernel (one block each)
constexpr int kWlPPT = 4;           // worklist partition task: points per thread (256 threads)
constexpr int kWlTaskPts = 256 * kWlPPT;  // points per worklist partition task
constexpr int kK3StatLevels = 64;  // levels whose counters the small-segment kernel sums per block
constexpr int kK4Words = 1024;      // bitmap words per ordering block (256 threads x 4)
constexpr int kFillTiles = 1024;    // tiles per tile-map fill job

// Everything a kernel needs, passed by value.
struct Work {
  const double* x;           // caller's points (global index = position): x[i], y[i], or with
  const double* y;           // aos set, x = xy, y = xy + 1 and point i at xy[2 i], xy[2 i + 1]
  int aos;                   // 1: the caller's points are interleaved (x0, y0, x1, y1, ...)
  const long long* offsets;  // nsets + 1 device offsets, or null (single set of n_single)
  const long long* key_base; // optional per-set key of p (server); null: off + set
  long long n_single;
  int nsets;
  int N;
  double* bx[2];
  double* by[2];
  int* bi[2];
  int* slot;
  unsigned* bitmap;
  long long nkeys;
  SetRec* sets;
  int* k0_tile_start;        // nsets + 1
  K0Part* k0part;
  SegRec* segs[2];
  SegGeom* geom[2];
  int* tile_seg[2];
  TileDesc* tdesc[2];        // per tile: where its points are
  int4* fjobs[2];            // tile-map fill jobs: {segment, first tile, tiles, 0}
  unsigned long long* status[2];
  TileRec* cand[2];
  SegState* sstate[2];       // per big segment: cursors and farthest-point candidates
  SegRec* k3q;
  Ctrl* ctrl;
  long long* stats;          // [3][kMaxLevels]: points read, points kept, segments
  int capS, capT, capQ, capT0, capJ;
  int small_max;             // segments with len <= small_max go to the small kernel
  int tile;                  // K1 tile size (points)
  long long timeout_ns;
  int drop_tile;             // test knob: this K1 tile never publishes (-1: none)
  int ordered;               // 1: offsets by decoupled look-back (stable layout); 0: atomic cursors
  int all_fast;              // host's copy of !Ctrl::any_slow: selects the FP32-only partition kernel
  int k1_shape;              // streaming partition kernel: block shape 0..2 (warps per block, ring stages)
  int tier_dev;              // host side: 1: both partition kernels are launched and the device's
                             // Ctrl::any_slow picks the one that runs (no host round trip)
  const Work* dev;           // this struct's copy in device memory: the kernels of the level loop
                             // (prologue, partition, finalize, tile map, finisher, loop tests)
                             // read it there, so a captured level loop serves every call
  PolyF* poly;               // per set: pre-filter chains and inner box
  unsigned long long* dirbest;  // per set and sampled direction: packed (score, index) of the extreme
  int* nsurv;                // per set: points the sieve kept (written to buffer 1 from the set's offset)
  int sieve;                 // 1: the pre-filter path (sample, chains, sieve); level 0 reads buffer 1
  int key_local_clear;       // 1 (one set): the finalize clears the bitmap words the set's keys reach
                             // (the call then skips clearing the whole bitmap)
  // persistent worklist: the level loop hands over at the first level whose
  // tiles hold at most wl_points points (0: never)
  long long wl_points;
  WlTask* wlq;               // queue entries
  unsigned* wltag;           // per entry: the epoch of the call that published it
  BestRec* wlrec;            // per entry and child: the partition task's farthest point
  WlSeg* wlseg;              // segment table
  int capWQ, capWS;          // queue entries, segment slots
  unsigned wl_epoch;         // this call's tag value (never 0)
  int pad_wl;
};

// launchers (vq_kernels.cu); all enqueue on `st`
cudaError_t launch_seed(const Work& w, cudaStream_t st);
// one point set: counters cleared and the set seeded in one kernel
cudaError_t launch_seed_single(const Work& w, cudaStream_t st);
cudaError_t launch_k0(const Work& w, int grid, cudaStream_t st);
cudaError_t launch_k0_finalize(const Work& w, cudaStream_t st);
// pre-filter path: sampled direction extremes, chains per set, the sieve
cudaError_t launch_sample(const Work& w, cudaStream_t st);
cudaError_t launch_poly(const Work& w, cudaStream_t st);
cudaError_t launch_sieve(const Work& w, cudaStream_t st);
cudaError_t launch_prologue(const Work& w, int level, cudaStream_t st);
// condition kernel of the device-driven level loop (a graph WHILE node)
cudaError_t launch_level_cond(const Work& w, cudaGraphConditionalHandle h, cudaStream_t st);
// a kernel node of graph g (no dependencies) that sets h to whether the
// level after level 0 has segments (the WHILE node's first test)
cudaError_t add_loop_init_node(cudaGraph_t g, cudaGraphNode_t* node, const Work& w, cudaGraphConditionalHandle h);
cudaError_t launch_k1(const Work& w, int level, int ppt, int grid, cudaStream_t st);
// the streaming partition kernel (vq_partition.cu), block shape w.k1_shape
cudaError_t launch_k1w(const Work& w, int level, int ppt, int tiles, cudaStream_t st);
cudaError_t launch_k2(const Work& w, int level, int grid, cudaStream_t st);
cudaError_t launch_tilemap(const Work& w, int par, int grid, cudaStream_t st);
cudaError_t launch_k3(const Work& w, int grid, cudaStream_t st);
// the persistent worklist: the handed-over segments into its queue, then the
// persistent kernel (both return at once when the level loop kept going)
cudaError_t launch_worklist(const Work& w, cudaStream_t st);
#ifdef VQ_WL_PROFILE
void wl_tier_calls(unsigned long long* out);
void wl_trace_dump(const char* path);
#endif
cudaError_t launch_order(const Work& w, int* out, long long* hull_offsets, long long* total,
                         long long* tmp, cudaStream_t st);
// the same in one pass (decoupled look-back over bitmap chunks); tmp holds
// order_fused_tmp_elems(nkeys) entries
cudaError_t launch_order_fused(const Work& w, int* out, long long* hull_offsets, long long* total,
                               long long* tmp, cudaStream_t st);
long long order_fused_tmp_elems(long long nkeys);
// pipelined host path: chunk-hull points into the merge buffers, and merge
// indices back to original indices
cudaError_t launch_gather(const double* x, const double* y, const int* idx, long long m, long long base, double* mx,
                          double* my, int* mid, cudaStream_t st);
cudaError_t launch_debug_round_f32(const double* v, long long m, float* out, cudaStream_t st);
cudaError_t launch_debug_orient_f32(const double* tri, long long m, int tier, float* d, float* e, cudaStream_t st);
cudaError_t launch_map_indices(const int* mout, const int* mid, long long h, int* out, cudaStream_t st);
cudaError_t scan_exclusive_i32(int* data, long long n, int* tmp, cudaStream_t st);
cudaError_t scan_exclusive_i64(long long* data, long long n, long long* tmp, cudaStream_t st);
long long scan_tmp_elems(long long n);
int k1_blocks_per_sm(int ppt);
long long kernels_launched();  // kernels launched by this library so far (all devices)
void count_launches(long long k);  // adds k (may be negative) to that count
int k3_smem_bytes();

// vq_config.timeout_ns as currently set (vq_api.cu)
long long config_timeout_ns();

// Hull contexts with caller-provided workspaces (vq_api.cu), used by the
// server: each lane owns a context and runs its batches on its own stream.
struct Ctx;
Ctx* ctx_create();  // for the current device; null on failure
void ctx_destroy(Ctx* c);
// device bytes a batched run of N points in nsets sets needs (current config)
size_t batched_workspace_bytes(long long N, int nsets);
// vq_hull2d_batched with N known on the host and the workspace given
// (at least batched_workspace_bytes(N, nsets) bytes, 256-byte aligned)
vq_status batched_run(Ctx* c, void* workspace, size_t bytes, const double* x, const double* y,
                      const long long* offsets, int nsets, long long N, int* hull_idx, long long* hull_offsets,
                      cudaStream_t st, long long* h_total = nullptr);

}  // namespace vq
