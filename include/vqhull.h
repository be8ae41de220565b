/*
 * vqhull.h -- C ABI of libvqhull, a GB300 (sm_103a) planar convex hull
 * built on the level-synchronous subset extraction of the VQhull paper
 * (Quickhull, arxiv 2510.09417).
 *
 * The result of every hull call is the one defined by Alg. 1 (Sec. 2.1):
 * the vertices H of the convex hull of the input points, in clockwise
 * order (y axis up), starting at the leftmost point.  Readings of what the
 * paper leaves open, applied throughout:
 *   - leftmost / rightmost are the lexicographic (x, then y) minimum and
 *     maximum;
 *   - "to the left of" is strict (Sec. 2.1, first display), so points on a
 *     hull edge are not vertices: only strict (extreme) vertices are listed,
 *     each coordinate pair once, represented by its lowest input index;
 *   - the farthest point of Alg. 1 is taken with exact arithmetic; among
 *     tied points the one nearest the segment's first endpoint, then the
 *     lowest index;
 *   - 0 points give an empty hull, coincident points a single vertex, and
 *     collinear points their two extreme ends.
 * Predicates are exact for finite coordinates whose nonzero magnitudes lie
 * in [2^-400, 2^400]; coordinates outside that range are accepted but the
 * result may then differ from the exact hull.
 *
 * Points are FP64 in structure-of-arrays layout (separate x[] and y[]), the
 * layout of Sec. 4 / Sec. 5.4.  Indices are 0-based int32.
 *
 * Memory: device arrays passed in stay owned by the caller and are only
 * read (the input is never permuted).  The library keeps one workspace per
 * device (about 45 bytes per input point), grown on demand and reused
 * across calls; calls on one device are serialised.
 *
 * Errors are returned as vq_status values, never raised or trapped.  After
 * an error the output arrays hold unspecified values.
 */
#ifndef VQHULL_H
#define VQHULL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VQ_OK = 0,
  VQ_PENDING = 1,             /* server: result not ready yet               */
  VQ_ERR_INVALID_ARG = -1,    /* null pointer, negative size, bad offsets   */
  VQ_ERR_NONFINITE = -2,      /* a NaN or infinite coordinate               */
  VQ_ERR_TOO_LARGE = -3,      /* sizes beyond the int32 index range          */
  VQ_ERR_NOMEM = -4,          /* device or host allocation failed            */
  VQ_ERR_CUDA = -5,           /* a CUDA runtime call failed                  */
  VQ_ERR_TIMEOUT = -6,        /* a bounded device wait expired               */
  VQ_ERR_BUDGET = -7,         /* server: request larger than the budget      */
  VQ_ERR_CAPACITY = -8,       /* output capacity or internal table too small */
  VQ_ERR_NOT_FOUND = -9       /* server: unknown ticket                      */
} vq_status;

/* Static description of a status code (never NULL). */
const char* vq_status_string(int status);

/* Library version: major * 10000 + minor * 100 + patch. */
int vq_version(void);

/*
 * Hull of one point set (Alg. 1).
 *   x, y      device FP64 arrays of n points (caller-owned, read-only)
 *   n         0 <= n <= 2^31 - 2
 *   hull_idx  device int32 array with room for n indices (worst case h = n);
 *             receives the h vertex indices, clockwise from the lexicographic
 *             minimum
 *   h         host pointer; receives the vertex count
 *   stream    cudaStream_t to enqueue on (NULL = legacy default stream); the
 *             call synchronises it before returning
 * Returns VQ_OK, VQ_ERR_INVALID_ARG, VQ_ERR_NONFINITE, VQ_ERR_TOO_LARGE,
 * VQ_ERR_NOMEM, VQ_ERR_CUDA or VQ_ERR_TIMEOUT.
 */
vq_status vq_hull2d(const double* x, const double* y, int64_t n, int32_t* hull_idx, int64_t* h,
                    void* stream);

/*
 * vq_hull2d on interleaved points: xy holds x0, y0, x1, y1, ... (device FP64,
 * 2n values, 8-byte aligned; 16-byte alignment gives the fastest loads), the
 * array-of-structures layout of PBBS's point files that the paper's
 * comparison with PBBS describes (Sec. 5.4).  The hull and its indices are
 * those of vq_hull2d on the same points.  The interleaved array is read once
 * by the level-0 pre-filter pass (which this call always uses); the points
 * it keeps continue in the library's own SoA buffers.  Arguments, errors and
 * stream behaviour as for vq_hull2d.
 */
vq_status vq_hull2d_aos(const double* xy, int64_t n, int32_t* hull_idx, int64_t* h, void* stream);

/*
 * Hulls of nsets independent point sets in one level-synchronous run: the
 * result per set is that of Alg. 1 (Sec. 2.1), and every level of the
 * subset extraction (Sec. 3: classify, compact, farthest point) runs over
 * the live segments of all sets at once.
 *   x, y          device FP64 arrays holding the sets back to back
 *   offsets       device int64[nsets + 1]: set s is points
 *                 offsets[s] .. offsets[s+1]-1; offsets[0] = 0, non-decreasing;
 *                 empty sets are allowed
 *   nsets         >= 1; offsets[nsets] + nsets must stay below 2^31
 *   hull_idx      device int32 with room for offsets[nsets] indices; receives
 *                 the hulls back to back, each clockwise from its set's
 *                 lexicographic minimum, with indices LOCAL to the set
 *   hull_offsets  device int64[nsets + 1]; receives the hulls' boundaries
 *                 (hull s is hull_idx[hull_offsets[s] .. hull_offsets[s+1]-1])
 * Synchronises `stream`.  A set with a non-finite coordinate gets an empty
 * hull and the call returns VQ_ERR_NONFINITE (the other sets are valid).
 */
vq_status vq_hull2d_batched(const double* x, const double* y, const int64_t* offsets, int32_t nsets,
                            int32_t* hull_idx, int64_t* hull_offsets, void* stream);

/*
 * vq_hull2d on host memory: copies x, y (n doubles each, host; pinned memory
 * gives the fastest copies) to a library-owned device buffer, runs the hull
 * and copies the h indices back.  hull_idx_host needs room for n indices.
 */
vq_status vq_hull2d_host(const double* x_host, const double* y_host, int64_t n, int32_t* hull_idx_host,
                         int64_t* h, void* stream);

/*
 * vq_hull2d for callers that cannot allocate.  The paper has no counterpart:
 * this entry point exists for code that must not trigger a device or host
 * allocation from inside a library call -- hosts that forbid allocation
 * after start-up (an allocation can stall or fail at an unpredictable
 * moment) and processes whose device memory is handed out by their own pool
 * allocator, which must account for every byte.  It runs the same kernels
 * as vq_hull2d (with the host-driven level loop and without the level-0
 * pre-filter, which changes no hull), but its whole workspace is one fixed
 * 64 MiB array of device memory that is part of this library; every GPU
 * that loads the library reserves it until the process exits.  The call
 * makes no cudaMalloc, cudaMallocHost, cudaFree or other allocating call.
 *   x, y, hull_idx, h, stream   as for vq_hull2d (hull_idx: room for n)
 *   n                           0 <= n <= 1,048,576; larger n returns
 *                               VQ_ERR_TOO_LARGE without touching the device
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture begins.  All calls on a device share the array,
 * which keeps the previous call's contents (each call clears what it needs
 * zeroed); calls that overlap on the GPU would race on it.  This function
 * therefore takes a process-wide lock and waits for `stream` before it
 * returns (also when it fails), so calls made through it never overlap.
 * Device waits are bounded by vq_config.timeout_ns, as for vq_hull2d.
 */
vq_status vq_hull2d_noalloc(const double* x, const double* y, int64_t n, int32_t* hull_idx, int64_t* h,
                            void* stream);

/*
 * Test access to the FP32 tiers of the exact left-of test of Sec. 2.1: for
 * m triples tri[6k .. 6k+5] = (ax, ay, bx, by, ux, uy) (device FP64), d[k]
 * and e[k] (device FP32) receive the value and error bound with which every
 * kernel of this library evaluates orient(a, b, u) =
 * (bx-ax)(uy-ay) - (by-ay)(ux-ax) in that tier:
 *   tier 0  a and b as an FP32 line (truncated origin, rounded direction),
 *           u truncated to 24 bits (absolute coordinates);
 *   tier 1  the same direction, u - a computed in FP64 and rounded to FP32
 *           (coordinates relative to a), for near-collinear points.
 * The tiers are used only when every |coordinate| < 2^40, and they claim a
 * sign only when |d| > e; |d - orient| <= e must hold for such inputs.
 * Synchronises `stream`.  Returns VQ_ERR_INVALID_ARG for m < 0, null arrays
 * or another tier.
 */
vq_status vq_debug_orient_f32(const double* tri, int64_t m, int32_t tier, float* d, float* e, void* stream);

/*
 * Test access to the FP64 -> FP32 rounding that the FP32 tiers use for the
 * line direction D~ = fl32(fl64(e - o)) and the relative coordinates
 * T~ = fl32(fl64(u - o)) (IEEE 754 round to nearest, ties to even, done
 * with integer operations): out[k] = fl32(v[k]) for m device FP64 values.
 * Synchronises `stream`.  Returns VQ_ERR_INVALID_ARG for m < 0 or null
 * arrays.
 */
vq_status vq_debug_round_f32(const double* v, int64_t m, float* out, void* stream);

/* Tuning knobs (process-wide; take effect on the next call). */
typedef struct {
  int32_t points_per_thread; /* partition kernel: 4, 8 or 16 points per lane
                                (default 16: a warp tile of 512 points)      */
  int32_t small_max;         /* segments of <= small_max points (2..1024) are
                                finished by the shared-memory kernel          */
  int32_t k1_blocks_per_sm;  /* reserved                                     */
  int32_t profile;           /* 1: time every kernel with CUDA events (see
                                vq_profile_read); 0: off                     */
  int64_t timeout_ns;        /* bound of every device-side wait              */
  int32_t debug_drop_tile;   /* testing: this partition tile never publishes
                                its look-back status (-1 = off)              */
  int32_t ordered;           /* 1: partition offsets by decoupled look-back
                                (stable, run-to-run identical buffer layout);
                                0 (default): one atomic per tile (faster; the
                                hull is identical either way)               */
  int32_t host_loop;         /* 0 (default): levels >= 1 run as one CUDA graph
                                launch whose WHILE node repeats the level on
                                the device until no segment is left (one host
                                round trip per call instead of one per
                                level); 1: the host launches every level and
                                reads its segment count back.  Profiling and
                                ordered mode always use the host loop.      */
  int32_t prefilter;         /* 1 (default): level 0 drops the points that lie
                                certainly inside a polygon of input points
                                found by the extreme pass (the Akl-Toussaint
                                octagon the paper proposes as its next step,
                                Sec. 6); the hull is the same, the per-level
                                counters are not.  0: plain Alg. 1 counts.
                                Applies to the default partition kernel.    */
  int32_t k1_shape;          /* streaming partition kernel's block shape:
                                0 (default) 4 warps per block; 1: 8 warps,
                                a shallower ring; 2: 2 warps, a deeper ring
                                (per points_per_thread; 0..2)                */
  int64_t worklist_points;   /* the level loop hands the rest of the
                                recursion (Alg. 1 on every live segment) to
                                the persistent worklist at the first level
                                whose segments hold at most this many points
                                (default 4,194,304); there a child segment
                                starts as soon as its parent's last
                                partition task is done, with no per-level
                                launches.  0: the level loop to the end.
                                The hull is the same either way.            */
} vq_config;

vq_status vq_get_config(vq_config* cfg);
vq_status vq_set_config(const vq_config* cfg);

/*
 * Per-level counters of the last call on the current device: for each
 * partition level l < *levels (at most cap are copied), read[l] points were
 * classified, kept[l] of them went to a child, in segs[l] segments (the
 * per-call statistics of Sec. 5.2's byte model).
 */
vq_status vq_last_stats(int64_t* levels, int64_t* read, int64_t* kept, int64_t* segs, int32_t cap);

/*
 * Counters accumulated over the hull calls on the current device since the
 * last reset.  Kernel times are filled only while vq_config.profile is set;
 * they are CUDA-event times on the call's stream.
 */
typedef struct {
  int64_t calls;             /* hull calls                                    */
  int64_t launches;          /* kernels launched by the library               */
  int64_t k1_launches;       /* partition kernel launches                     */
  int64_t levels;            /* partition levels run by the level loop        */
  int64_t k1_points_read;    /* points classified by the partition kernel     */
  int64_t k1_points_kept;    /* of those, points written to a child           */
  double k0_ms;              /* extreme-point pass (with the pre-filter: the
                                sieve); the per-set finalize is in other_ms  */
  double k1_ms;              /* partition kernel                              */
  double k2_ms;              /* per-segment finalize                          */
  double k3_ms;              /* small-segment finisher                        */
  double k4_ms;              /* ordering                                      */
  double other_ms;           /* scans, tile maps, counter resets              */
  int64_t graph_launches;    /* level loops run as a device-driven graph      */
  double sample_ms;          /* pre-filter set-up: sampled extremes and chains */
  double k5_ms;              /* persistent worklist (the recursion below the
                                level where the level loop hands over)      */
  int64_t worklist_reruns;   /* calls run again with the level loop alone
                                after the worklist's queue overflowed       */
} vq_profile;

vq_status vq_profile_read(vq_profile* out, int32_t reset);

/*
 * Autotuner of the knobs above for inputs like (x, y, n) (device FP64 SoA,
 * as for vq_hull2d).  It times the hull of these points on `stream` under
 * each candidate configuration: points per lane 8 or 16, small-segment
 * threshold 256 or 1024, level-0 pre-filter on or off, and the partition
 * kernel's three block shapes (warps per block and ring depth), 24
 * candidates.  Every candidate runs
 * once untimed (workspace, graph capture), then `reps` times (1..16) between
 * CUDA events.  The fastest by its median time becomes the process-wide
 * configuration; the other fields keep their current values.
 *   best     receives that configuration (may be NULL)
 *   best_ms  receives its median time per hull in ms (may be NULL)
 * The candidates must agree on the hull's vertex count, else
 * VQ_ERR_CAPACITY.  The call allocates a temporary device buffer of n
 * indices and synchronises `stream`.
 */
vq_status vq_autotune(const double* x, const double* y, int64_t n, int32_t reps, vq_config* best,
                      double* best_ms, void* stream);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of hull requests                        */
/* ------------------------------------------------------------------ */

typedef struct vq_server vq_server;

typedef struct {
  size_t mem_budget_bytes; /* device memory the server may use in total      */
  int32_t max_inflight;    /* requests resident on the device at once (>= 1) */
  int32_t device;          /* CUDA device ordinal                            */
  int32_t lanes;           /* batches on the device at once, each on its own
                              stream (1..16; 0 = default 3)                   */
  size_t pinned_bytes;     /* pinned host memory that stages submitted points
                              (0: the smaller of the budget and 8 GiB); a
                              request that does not fit is kept in pageable
                              memory instead                                  */
} vq_server_config;

/*
 * Creates a server: continuous batching of hull requests (the level-
 * synchronous extraction of Sec. 3 applied to many requests at once).  The
 * paper has no counterpart for serving; each request's result is the hull
 * of Alg. 1 (Sec. 2.1), the same as vq_hull2d's on the same points.
 * Each of `lanes` host threads owns a CUDA stream and a hull context.  An
 * idle lane takes the queued requests (FIFO) that fit the free request
 * slots (max_inflight) and the free device memory (mem_budget_bytes),
 * copies their points in and runs them as one batched level-synchronous
 * hull, so that all segments of its requests share every level step.
 * Requests that arrive while other batches are on the GPU are admitted by
 * another lane as soon as slots and memory allow, and their kernels overlap
 * with the running batches on the device.  Device memory comes from a pool
 * owned by the server; the admitted requests' bytes (points, outputs and
 * the exact workspace of their batch) never exceed the budget.
 */
vq_status vq_server_create(const vq_server_config* cfg, vq_server** out);

/* Queues a hull of n host points (copied before return, into the server's
 * pinned staging area when it has room; the caller may free them).  VQ_ERR_BUDGET if the request alone (its batch's device bytes plus
 * the server's fixed 1 MiB reserve) exceeds the memory budget.  Serving
 * only; no counterpart in the paper. */
vq_status vq_server_submit(vq_server* s, const double* x_host, const double* y_host, int64_t n,
                           uint64_t* ticket);

/* VQ_OK with the result copied to hull_idx_host (room for cap indices; h set),
 * VQ_PENDING, VQ_ERR_CAPACITY if cap < h, VQ_ERR_NOT_FOUND, or the request's
 * own error.  A result is released once returned with VQ_OK.  The result is
 * the hull of Alg. 1 (Sec. 2.1), clockwise from the lexicographic minimum,
 * indices into the request's points. */
vq_status vq_server_poll(vq_server* s, uint64_t ticket, int32_t* hull_idx_host, int64_t cap, int64_t* h);

/* As vq_server_poll, waiting up to timeout_ms (< 0: no limit). */
vq_status vq_server_wait(vq_server* s, uint64_t ticket, int32_t* hull_idx_host, int64_t cap, int64_t* h,
                         int32_t timeout_ms);

/* Waits up to timeout_ms (< 0: no limit) for any request to finish and takes
 * the one that finished first among those not yet taken: *ticket, *h and
 * its result as for vq_server_poll, and *latency_ms (may be NULL) the time
 * from its submission to its completion on the server's clock.  Returns
 * VQ_PENDING if none finished in time.  VQ_ERR_CAPACITY (cap < h) sets
 * *ticket and *h and leaves the result to vq_server_wait / vq_server_poll. */
vq_status vq_server_wait_any(vq_server* s, uint64_t* ticket, int32_t* hull_idx_host, int64_t cap, int64_t* h,
                             int32_t timeout_ms, double* latency_ms);

/* Latency percentiles (submit to completion) and throughput so far
 * (serving only; no counterpart in the paper). */
vq_status vq_server_stats(vq_server* s, double* p50_ms, double* p99_ms, double* hulls_per_s);

/* Counters of the server since its creation. */
typedef struct {
  int64_t completed;            /* requests finished (with any status)           */
  int64_t batches;              /* batches run                                   */
  int64_t max_busy_lanes;       /* most lanes running a batch at the same time   */
  int64_t admitted_while_busy;  /* requests admitted while another lane's batch
                                   was on the device                            */
  int64_t peak_bytes;           /* most device bytes held by admitted batches    */
  int64_t budget_bytes;         /* the configured budget                         */
} vq_server_info;

vq_status vq_server_info_read(vq_server* s, vq_server_info* out);

/* Stops the server thread and frees its memory; pending requests are dropped. */
void vq_server_destroy(vq_server* s);

#ifdef __cplusplus
}
#endif

#endif /* VQHULL_H */
