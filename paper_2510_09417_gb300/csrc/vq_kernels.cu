// vq_kernels.cu -- the kernels of the level-synchronous planar Quickhull.
//
// One level of Alg. 1 (Sec. 2.1) is run for every live segment (a, b, r) at
// once: each point u of the segment is classified as left of a->r (child
// a->r), left of r->b (child r->b) or discarded (the subset extraction of
// Sec. 3), the two children are compacted into the other ping-pong buffer
// (left child forward from the segment start, right child backward from its
// end, as in the two-ended layout of Alg. 2), and each child's farthest point
// is found in the same pass (Sec. 4, "Bandwidth considerations").
//
// Kernels, in call order:
//   k_seed / k_k0 / k_k0_finalize  leftmost p and rightmost q per point set
//                                  (Alg. 1, first two steps), level-0 segments
//   k_prologue                     per-level counter reset
//   k_k1                           fused classify + compact + per-tile argmax,
//                                  offsets by decoupled look-back
//   k_k2                           per segment: exact cross-tile argmax, emit r,
//                                  child segments, next level's tile map
//   k_k3                           segments of <= small_max points, finished
//                                  whole in shared memory (one warp each)
//   k_k4_*                         clockwise order of the emitted vertices
//
// Hull order.  A vertex r emitted for segment [off, off+len) gets the order
// key off + nL + 1 + shift: the buffer position between its left child
// [off, off+nL) and right child [off+len-nR, off+len).  All descendants of
// the left child get keys inside the left range and those of the right child
// inside the right range, so sorting by key is the in-order traversal of
// Alg. 1's recursion, i.e. the clockwise hull.  p gets key off + shift.
#include <climits>
#include <cstdio>
#include <cstdlib>

#include "vq_internal.h"
#include "vq_common.cuh"

namespace vq {

static unsigned long long g_launches = 0;
static inline void count_launch(int k = 1) { __atomic_fetch_add(&g_launches, (unsigned long long)k, __ATOMIC_RELAXED); }
long long kernels_launched() { return (long long)__atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

// ---------------------------------------------------------------------------
// shared helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ void emit(const Work& w, long long key, int local) {
  if (!VQ_OK_IDX(w, 1, key, 0, w.nkeys) || !VQ_OK_IDX(w, 2, local, 0, w.N)) return;
  atomicOr(&w.bitmap[key >> 5], 1u << (unsigned)(key & 31));
  w.slot[key] = local;
}

__device__ __forceinline__ void add_stats(const Work& w, int level, long long rd, long long kept,
                                          long long segs = 1) {
  const int l = level < kMaxLevels ? level : kMaxLevels - 1;
  atomicAdd(reinterpret_cast<unsigned long long*>(&w.stats[l]), (unsigned long long)rd);
  atomicAdd(reinterpret_cast<unsigned long long*>(&w.stats[kMaxLevels + l]), (unsigned long long)kept);
  atomicAdd(reinterpret_cast<unsigned long long*>(&w.stats[2 * kMaxLevels + l]), (unsigned long long)segs);
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
  return v;
}

// Append a segment for the partition kernel (whole warp): reserve its tiles,
// write its geometry and the tile -> segment map, clear the tiles' status.
// Register a big segment for the next partition level: a slot, a range of
// tiles, its geometry and its zeroed cursor; the per-tile map is written by
// k_tilemap from fill jobs of at most kFillTiles tiles each.
__device__ int push_k1_warp(const Work& w, int par, SegRec R, int lane) {
  const int ntiles = (R.len + w.tile - 1) / w.tile;
  const int njobs = (ntiles + kFillTiles - 1) / kFillTiles;
  int slot = 0, base = 0, job = 0;
  if (lane == 0) {
    slot = atomicAdd(&w.ctrl->k1_segs[par], 1);
    base = atomicAdd(&w.ctrl->k1_tiles[par], ntiles);
    job = atomicAdd(&w.ctrl->fill_jobs[par], njobs);
  }
  slot = __shfl_sync(kFull, slot, 0);
  base = __shfl_sync(kFull, base, 0);
  job = __shfl_sync(kFull, job, 0);
  if (slot >= w.capS || base > w.capT - ntiles || job > w.capJ - njobs) {
    if (lane == 0) atomicOr(&w.ctrl->err, kErrCapacity);
    return -1;
  }
  R.tile_base = base;
  R.ntiles = ntiles;
  if (!VQ_OK_IDX(w, 3, R.a, 0, w.N) || !VQ_OK_IDX(w, 4, R.b, 0, w.N) || !VQ_OK_IDX(w, 5, R.r, 0, w.N) ||
      !VQ_OK_IDX(w, 6, (long long)R.off + R.len, 1, (long long)w.N + 1))
    return -1;
  if (lane == 0) {
    w.segs[par][slot] = R;
    SegGeom g;
    fill_geom(g, px(w, R.a), py(w, R.a), px(w, R.b), py(w, R.b), px(w, R.r), py(w, R.r));
    w.geom[par][slot] = g;
  }
  for (int i = lane; i < njobs; i += kWarp)
    w.fjobs[par][job + i] = make_int4(slot, base + i * kFillTiles, min(kFillTiles, ntiles - i * kFillTiles), 0);
  int* st = reinterpret_cast<int*>(&w.sstate[par][slot]);
  for (int i = lane; i < (int)(sizeof(SegState) / sizeof(int)); i += kWarp) st[i] = 0;
  return slot;
}

// The per-tile map of level parity `par`: segment, look-back status word
// and the partition kernel's tile descriptor, one fill job per block.
__global__ void __launch_bounds__(256) k_tilemap(const Work* __restrict__ wp, int par) {
  const Work& w = *wp;
  if (fatal(w)) return;
  const int njobs = min(*reinterpret_cast<volatile int*>(&w.ctrl->fill_jobs[par]), w.capJ);
  for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
    const int4 J = w.fjobs[par][j];
    const SegRec S = w.segs[par][J.x];
    for (int i = threadIdx.x; i < J.z; i += blockDim.x) {
      const int t = J.y + i;
      const int k = t - S.tile_base;
      if (!VQ_OK_IDX(w, 45, t, 0, w.capT)) break;
      w.tile_seg[par][t] = J.x;
      if (w.ordered) w.status[par][t] = 0ull;
      TileDesc d;
      d.sid = J.x;
      d.begin = S.off + k * w.tile;
      d.count = min(w.tile, S.len - k * w.tile);
      d.flags = S.flags;
      d.off = S.off;
      d.len = S.len;
      d.pad0 = 0;
      d.pad1 = 0;
      w.tdesc[par][t] = d;
    }
  }
}

__device__ __forceinline__ void push_k3(const Work& w, const SegRec& R) {
  const int i = atomicAdd(&w.ctrl->k3_count, 1);
  if (i < w.capQ) w.k3q[i] = R;
  else atomicOr(&w.ctrl->err, kErrCapacity);
}

// ---------------------------------------------------------------------------
// Point sets and the extreme pass
// ---------------------------------------------------------------------------

__global__ void k_seed(Work w) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) {
    w.k0_tile_start[w.nsets] = 0;
    w.ctrl->nonfinite_set = LLONG_MAX;
  }
  if (s >= w.nsets) return;
  long long off, end;
  if (w.offsets) {
    off = w.offsets[s];
    end = w.offsets[s + 1];
  } else {
    off = 0;
    end = w.n_single;
  }
  if (off < 0 || end < off || end > w.N || (s == 0 && off != 0) ||
      (s == w.nsets - 1 && end != w.N)) {
    atomicOr(&w.ctrl->err, kErrBadOffsets);
    off = 0;
    end = 0;
  }
  SetRec r;
  r.off = (int)off;
  r.len = (int)(end - off);
  r.shift = w.key_base ? w.key_base[s] - off : (long long)s;
  r.flags = 0;
  r.p = r.q = -1;
  r.pad = 0;
  w.sets[s] = r;
  w.k0_tile_start[s] = (r.len + kK0Tile - 1) / kK0Tile;
}

// One point set: the control block, the level counters and (pre-filter
// path) the set's sampled extremes and survivor count cleared, then the
// set's record and its extreme-pass tiles [0, tiles) (what k_seed and the
// scan of k0_tile_start give for one set), in one block.
__global__ void __launch_bounds__(256) k_seed_single(Work w) {
  static_assert(sizeof(Ctrl) % sizeof(int4) == 0, "Ctrl is cleared as int4");
  int4* c4 = reinterpret_cast<int4*>(w.ctrl);
  for (int i = threadIdx.x; i < (int)(sizeof(Ctrl) / sizeof(int4)); i += blockDim.x) c4[i] = make_int4(0, 0, 0, 0);
  for (int i = threadIdx.x; i < 3 * kMaxLevels; i += blockDim.x) w.stats[i] = 0;
  if (w.sieve) {
    for (int i = threadIdx.x; i < kPolyDirs; i += blockDim.x) w.dirbest[i] = 0ull;
    if (threadIdx.x == 0) w.nsurv[0] = 0;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  w.ctrl->nonfinite_set = LLONG_MAX;
  const long long off = w.offsets ? w.offsets[0] : 0;
  const long long end = w.offsets ? w.offsets[1] : w.n_single;
  SetRec r;
  if (off != 0 || end != w.N) {
    atomicOr(&w.ctrl->err, kErrBadOffsets);
    r.off = 0;
    r.len = 0;
  } else {
    r.off = 0;
    r.len = (int)end;
  }
  r.shift = w.key_base ? w.key_base[0] : 0;
  r.flags = 0;
  r.p = r.q = -1;
  r.pad = 0;
  w.sets[0] = r;
  w.k0_tile_start[0] = 0;
  w.k0_tile_start[1] = (r.len + kK0Tile - 1) / kK0Tile;
}

struct LexPt {
  long long kx, ky;
  int i;
};

__device__ __forceinline__ bool lex_min_better(const LexPt& a, const LexPt& b) {
  return a.kx < b.kx || (a.kx == b.kx && (a.ky < b.ky || (a.ky == b.ky && a.i < b.i)));
}
__device__ __forceinline__ bool lex_max_better(const LexPt& a, const LexPt& b) {
  return a.kx > b.kx || (a.kx == b.kx && (a.ky > b.ky || (a.ky == b.ky && a.i < b.i)));
}
__device__ __forceinline__ LexPt shfl_lex(const LexPt& p, int m) {
  LexPt o;
  o.kx = __shfl_xor_sync(kFull, p.kx, m);
  o.ky = __shfl_xor_sync(kFull, p.ky, m);
  o.i = __shfl_xor_sync(kFull, p.i, m);
  return o;
}

// One point's contribution to the extreme pass: lexicographic min and max
// (x, then y, then lowest index) as integer comparisons of the ordered bit
// patterns (branch-free selects: the batched loads stay in flight); am
// keeps the largest magnitude bit pattern seen, from which the flags are
// derived once (k0_flags).
__device__ __forceinline__ void k0_take(double vx, double vy, int i, LexPt& mn, LexPt& mx, unsigned& am) {
  const long long kx = order_key(vx);
  // the full lexicographic compare only when x reaches the current
  // extreme (rare after the first points)
  if (kx <= mn.kx) {
    const LexPt p{kx, order_key(vy), i};
    if (lex_min_better(p, mn)) mn = p;
  }
  if (kx >= mx.kx) {
    const LexPt p{kx, order_key(vy), i};
    if (lex_max_better(p, mx)) mx = p;
  }
  const unsigned ax = static_cast<unsigned>(__double2hiint(vx)) & 0x7fffffffu;
  const unsigned ay = static_cast<unsigned>(__double2hiint(vy)) & 0x7fffffffu;
  am = max(am, max(ax, ay));
}
// From the largest high word of |coordinate| seen: bit 0: a coordinate is
// non-finite (exponent all ones); bit 1: some |coordinate| >= 2^40 (outside
// the FP32 tier's range).  Both thresholds have a zero low word, so the
// high words decide them exactly.
__device__ __forceinline__ int k0_flags(unsigned am) {
  return (am >= 0x7ff00000u ? 1 : 0) | (am >= 0x42700000u ? 2 : 0);
}

// Asynchronous 16-byte global -> shared copies (cp.async, completion
// tracked per thread by commit groups).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One tile's points through the shared-memory ring (see k_k0).
__device__ __forceinline__ void k0_stream(const Work& w, int begin, int count, LexPt& mn, LexPt& mx, unsigned& am) {
  extern __shared__ __align__(16) double2 k0_ring[];  // [stage][x|y][pair k][thread]
  constexpr int SP = kK0Pairs * kK0Threads;           // pairs per stage
  // pair q covers points 2q, 2q+1; stage i holds pairs i*SP .. i*SP+SP-1
  const double2* px = reinterpret_cast<const double2*>(w.x + begin);
  const double2* py = reinterpret_cast<const double2*>(w.y + begin);
  const int npairs = count >> 1;
  const int nst = (npairs + SP - 1) / SP;
  auto slot = [&](int st, int a, int k) -> double2* {
    return k0_ring + ((st * 2 + a) * kK0Pairs + k) * kK0Threads + threadIdx.x;
  };
  auto issue = [&](int i) {
    const int st = i % kK0Stages;
#pragma unroll
    for (int k = 0; k < kK0Pairs; k++) {
      const int q = i * SP + k * kK0Threads + (int)threadIdx.x;
      if (q < npairs) {
        cp_async16(slot(st, 0, k), px + q);
        cp_async16(slot(st, 1, k), py + q);
      }
    }
  };
#pragma unroll
  for (int i = 0; i < kK0Stages - 1; i++) {
    if (i < nst) issue(i);
    cp_async_commit();
  }
  for (int i = 0; i < nst; i++) {
    // the slot refilled here was read by this thread in the previous step
    if (i + kK0Stages - 1 < nst) issue(i + kK0Stages - 1);
    cp_async_commit();
    cp_async_wait<kK0Stages - 1>();  // this thread's copies of stage i have landed
    const int st = i % kK0Stages;
#pragma unroll
    for (int k = 0; k < kK0Pairs; k++) {
      const int q = i * SP + k * kK0Threads + (int)threadIdx.x;
      if (q < npairs) {
        const double2 vx = *slot(st, 0, k), vy = *slot(st, 1, k);
        k0_take(vx.x, vy.x, begin + 2 * q, mn, mx, am);
        k0_take(vx.y, vy.y, begin + 2 * q + 1, mn, mx, am);
      }
    }
  }
  cp_async_wait<0>();
  if ((count & 1) && threadIdx.x == 0) {
    const int l = begin + count - 1;
    k0_take(w.x[l], w.y[l], l, mn, mx, am);
  }
}

// Lexicographic min and max (x, then y, then lowest index) of each tile and
// its flags.  Tiles whose first point is 16-byte aligned in both arrays
// (the usual case) stream through a ring of kK0Stages shared-memory stages:
// per stage every thread copies kK0Pairs pairs of x and of y (16 bytes
// each, consecutive threads on consecutive pairs) with cp.async, and reads
// back only its own slots, so no barrier is needed between stages; the
// copies of the next kK0Stages - 1 stages stay in flight while a stage is
// reduced.  Other tiles are read point by point.
__global__ void __launch_bounds__(kK0Threads) k_k0(Work w) {
  __shared__ LexPt s_mn[kK0Threads / kWarp], s_mx[kK0Threads / kWarp];
  __shared__ int s_fl[kK0Threads / kWarp];
  const int total = w.k0_tile_start[w.nsets];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = w.nsets - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (w.k0_tile_start[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const SetRec S = w.sets[lo];
    const int j = t - w.k0_tile_start[lo];
    const int begin = S.off + j * kK0Tile;
    const int count = min(kK0Tile, S.len - j * kK0Tile);
    LexPt mn{LLONG_MAX, LLONG_MAX, INT_MAX}, mx{LLONG_MIN, LLONG_MIN, INT_MAX};
    unsigned am = 0;
    const bool vec = ((reinterpret_cast<uintptr_t>(w.x + begin) | reinterpret_cast<uintptr_t>(w.y + begin)) & 15u) == 0;
    if (vec) {
      k0_stream(w, begin, count, mn, mx, am);
    } else {
#pragma unroll 8
      for (int l = threadIdx.x; l < count; l += kK0Threads) k0_take(w.x[begin + l], w.y[begin + l], begin + l, mn, mx, am);
    }
    int fl = k0_flags(am);
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      const LexPt a = shfl_lex(mn, m), b = shfl_lex(mx, m);
      if (lex_min_better(a, mn)) mn = a;
      if (lex_max_better(b, mx)) mx = b;
      fl |= __shfl_xor_sync(kFull, fl, m);
    }
    if (lane == 0) { s_mn[warp] = mn; s_mx[warp] = mx; s_fl[warp] = fl; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < kK0Threads / kWarp; q++) {
        if (lex_min_better(s_mn[q], mn)) mn = s_mn[q];
        if (lex_max_better(s_mx[q], mx)) mx = s_mx[q];
        fl |= s_fl[q];
      }
      K0Part P;
      P.minx = mn.kx; P.miny = mn.ky; P.mini = mn.i;
      P.maxx = mx.kx; P.maxy = mx.ky; P.maxi = mx.i;
      P.flags = fl;
      P.pad = 0;
      w.k0part[t] = P;
    }
    __syncthreads();
  }
}

// One warp per point set: p, q, the set's flags; emit p; make the level-0
// segment (a = p, b = p, r = q), whose children are p->q (upper, points left
// of p->q) and q->p (lower), the two calls of Alg. 1's first line.
__device__ void k0_finish_set(const Work& w, int s, SetRec S, const LexPt& mn, const LexPt& mx, int fl, int lane);

// One block per point set: the set's partials are reduced by the whole
// block, then warp 0 finishes the set.
__global__ void __launch_bounds__(kK0Threads) k_k0_finalize(Work w) {
  __shared__ LexPt s_mn[kK0Threads / kWarp], s_mx[kK0Threads / kWarp];
  __shared__ int s_fl[kK0Threads / kWarp];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (w.nsets == 1 && blockIdx.x == 0 && w.key_local_clear) {
    // one set: its keys lie in [off + shift, off + shift + len + 1] with
    // len the points it partitions; the order pass reads just those words,
    // cleared here (before any emission) instead of the whole bitmap
    const SetRec S = w.sets[0];
    const long long len = w.sieve ? min((long long)__ldcg(&w.nsurv[0]), (long long)S.len) : (long long)S.len;
    long long kw = ((long long)S.off + S.shift + len + 2 + 31) / 32 + 1;
    const long long all = (w.nkeys + 31) / 32 + 1;
    if (kw > all) kw = all;
    for (long long i = threadIdx.x; i < kw; i += blockDim.x) w.bitmap[i] = 0u;
    if (threadIdx.x == 0) w.ctrl->key_words = kw;
    __syncthreads();
  }
  for (int s = blockIdx.x; s < w.nsets; s += gridDim.x) {
    SetRec S = w.sets[s];
    if (S.len == 0) continue;  // uniform across the block
    LexPt mn{LLONG_MAX, LLONG_MAX, INT_MAX}, mx{LLONG_MIN, LLONG_MIN, INT_MAX};
    int fl = 0;
    // partials: one per extreme-pass tile, or (sieve) one per sieve block
    // that worked on the set, block g of G at slot g + s, where block g
    // holds tiles [T g / G, T (g + 1) / G): the blocks of the set's first
    // and last tiles u are ceil((u + 1) G / T) - 1, and the empty ones
    // between them wrote nothing
    long long lo = w.k0_tile_start[s], hi = w.k0_tile_start[s + 1];
    const long long T = w.k0_tile_start[w.nsets], G = w.sieve ? __ldcg(&w.ctrl->sv_grid) : 0;
    if (w.sieve) {
      if (hi <= lo || G <= 0) {
        lo = hi = 0;
      } else {
        const long long g0 = ((lo + 1) * G + T - 1) / T - 1, g1 = (hi * G + T - 1) / T - 1;
        lo = g0;
        hi = g1 + 1;
      }
    }
#pragma unroll 4
    for (long long t = lo + threadIdx.x; t < hi; t += kK0Threads) {
      if (w.sieve && T * (t + 1) / G <= T * t / G) continue;  // block t had no tile
      const K0Part P = w.k0part[w.sieve ? t + s : t];
      const LexPt a{P.minx, P.miny, P.mini}, b{P.maxx, P.maxy, P.maxi};
      if (lex_min_better(a, mn)) mn = a;
      if (lex_max_better(b, mx)) mx = b;
      fl |= P.flags;
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      const LexPt a = shfl_lex(mn, m), b = shfl_lex(mx, m);
      if (lex_min_better(a, mn)) mn = a;
      if (lex_max_better(b, mx)) mx = b;
      fl |= __shfl_xor_sync(kFull, fl, m);
    }
    if (lane == 0) { s_mn[warp] = mn; s_mx[warp] = mx; s_fl[warp] = fl; }
    __syncthreads();
    if (warp == 0) {
      mn = lane < kK0Threads / kWarp ? s_mn[lane] : LexPt{LLONG_MAX, LLONG_MAX, INT_MAX};
      mx = lane < kK0Threads / kWarp ? s_mx[lane] : LexPt{LLONG_MIN, LLONG_MIN, INT_MAX};
      fl = lane < kK0Threads / kWarp ? s_fl[lane] : 0;
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) {
        const LexPt a = shfl_lex(mn, m), b = shfl_lex(mx, m);
        if (lex_min_better(a, mn)) mn = a;
        if (lex_max_better(b, mx)) mx = b;
        fl |= __shfl_xor_sync(kFull, fl, m);
      }
      k0_finish_set(w, s, S, mn, mx, fl, lane);
    }
    __syncthreads();  // the shared partials are reused by the next set
  }
}

// Warp 0 of the finalize block: p, q and the flags of set s; emit p; make
// the level-0 segment.  On the pre-filter path the segment holds the
// sieve's survivors of the set, in buffer 1 from the set's offset; p and q
// are among them (strict vertices are never dropped), so the extremes of
// the survivors are those of the set.
__device__ void k0_finish_set(const Work& w, int s, SetRec S, const LexPt& mn, const LexPt& mx, int fl, int lane) {
  if (fl & 1) {
    if (lane == 0) {
      atomicOr(&w.ctrl->err, kErrNonfinite);
      atomicMin(reinterpret_cast<unsigned long long*>(&w.ctrl->nonfinite_set), (unsigned long long)s);
    }
    return;
  }
  const int p = mn.i, q = mx.i;
  if (p < S.off || p >= S.off + S.len || q < S.off || q >= S.off + S.len) {  // partials not written: an earlier error
    if (lane == 0) atomicOr(&w.ctrl->err, kErrInternal);
    return;
  }
  S.p = p;
  S.q = q;
  S.flags = (fl & 2) ? 0 : kSegFast;
  if ((fl & 2) && lane == 0) atomicOr(&w.ctrl->any_slow, 1);
  if (lane == 0) {
    w.sets[s] = S;
    emit(w, (long long)S.off + S.shift, p - S.off);
  }
  if (p == q) return;  // all points coincide with p
  SegRec R;
  R.shift = S.shift;
  R.off = S.off;
  R.len = w.sieve ? min(__ldcg(&w.nsurv[s]), S.len) : S.len;
  R.a = p;
  R.b = p;
  R.r = q;
  R.set_off = S.off;
  R.level = 0;
  R.tile_base = 0;
  R.ntiles = 0;
  R.flags = S.flags | (w.sieve ? kSegSrcBuf1 : kSegSrcInput);
  if (w.sieve && 2LL * R.len > (long long)S.len) R.flags |= kSegDense;
  if (R.len <= seg_small_max(w, R.flags)) {
    if (lane == 0) push_k3(w, R);
  } else {
    push_k1_warp(w, 0, R, lane);
  }
}

// Per-level counter reset.  It is also where the level loop hands over to
// the persistent worklist: when the level's tiles hold at most wl_points
// points, its big segments (and, at level 0, the small ones queued with
// them) are recorded for the worklist and the level's counts are set to
// zero, so that every later kernel of the loop finds nothing to do and the
// loop stops.
__global__ void k_prologue(const Work* __restrict__ wp, int level) {
  const Work& w = *wp;
  const int par = level & 1;
  Ctrl* c = w.ctrl;
  c->k1_ticket = 0;
  c->k1_segs[par ^ 1] = 0;
  c->k1_tiles[par ^ 1] = 0;
  c->fill_jobs[par ^ 1] = 0;
  if (level > 0) c->k3_count = 0;
  if (w.wl_points > 0 && !c->wl_on && !(c->err & kErrFatal) &&
      (long long)c->k1_tiles[par] * w.tile <= w.wl_points) {
    c->wl_on = 1;
    c->wl_par = par;
    c->wl_nbig = c->k1_segs[par];
    c->wl_nsmall = c->k3_count;
    c->wl_maxlevel = level;
    c->k1_segs[par] = 0;
    c->k1_tiles[par] = 0;
    c->k3_count = 0;
  }
  if (level > 0 && c->k1_segs[par] > 0) c->live_levels++;
  c->level = level;
}

// Condition of the device-driven level loop: a CUDA graph WHILE node whose
// body runs two partition levels (parity 1, then parity 0).  The loop goes
// on while the next level (parity 1) has segments and no fatal error was
// raised.  Every level removes at least one point from each of its
// segments, so N / 2 + 4 iterations bound the loop; reaching the bound is
// an internal error.
// A second bound is time: a loop still running kLevelLoopNs after its first
// condition stops with a timeout (far beyond any real run: a 1e8-point
// hull-dense input takes under a second).
constexpr unsigned long long kLevelLoopNs = 60ull * 1000000000ull;

// First test of the device-driven level loop: run it only if level 0 left
// segments for level 1 and raised no fatal error.
__global__ void k_loop_init(const Work* __restrict__ wp, cudaGraphConditionalHandle h) {
  const Work& w = *wp;
  const Ctrl* c = w.ctrl;
  cudaGraphSetConditional(h, (c->k1_segs[1] > 0 && !(c->err & kErrFatal)) ? 1u : 0u);
}

__global__ void k_level_cond(const Work* __restrict__ wp, cudaGraphConditionalHandle h) {
  const Work& w = *wp;
  const long long max_iters = (long long)w.N / 2 + 4;
  Ctrl* c = w.ctrl;
  const long long it = ++c->graph_iters;
  const unsigned long long now = global_ns();
  if (it == 1) c->loop_t0 = now;
  bool more = c->k1_segs[1] > 0 && !(c->err & kErrFatal);
  if (more && it >= max_iters) {
    c->err |= kErrInternal;
    more = false;
  }
  if (more && now - c->loop_t0 > kLevelLoopNs) {
    c->err |= kErrTimeout;
    more = false;
  }
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// K1: fused classify + compact + per-tile argmax
// ---------------------------------------------------------------------------

// Decoupled look-back (Merrill and Garland, "Single-pass Parallel Prefix
// Scan with Decoupled Look-back", 2016), restarted at every segment, carrying
// two sums (left and right child counts) and two running maxima (the
// children's farthest points under the exact order).  Tile t publishes its
// own counts and farthest points (aggregate), then combines predecessors of
// the same segment until one with an inclusive prefix, then publishes its
// inclusive prefix.  Records are written before the status word that makes
// them visible (release); readers load the status with acquire.  Waits are
// bounded by w.timeout_ns; on expiry the error flag is set and false returned.
__device__ __forceinline__ bool lookback_warp(const Work& w, int par, int t, int first, const SegGeom* G,
                                              unsigned long long aggL, unsigned long long aggR,
                                              const CandT<double>& own0, const CandT<double>& own1,
                                              long long& exclL, long long& exclR, CandT<double>& incl0,
                                              CandT<double>& incl1, int lane) {
  unsigned long long* st = w.status[par];
  TileRec* rec = w.cand[par];
  exclL = 0;
  exclR = 0;
  const bool publish = (t != w.drop_tile);
  incl0 = own0;
  incl1 = own1;
  if (t == first) {
    if (lane == 0) {
      rec[t].incl[0] = to_rec(own0);
      rec[t].incl[1] = to_rec(own1);
      if (publish) st_release_u64(&st[t], kStInc | st_pack(aggL, aggR));
    }
    return true;
  }
  if (lane == 0) {
    rec[t].own[0] = to_rec(own0);
    rec[t].own[1] = to_rec(own1);
    if (publish) st_release_u64(&st[t], kStAgg | st_pack(aggL, aggR));
  }
  const unsigned long long t0 = global_ns();
  CandT<double> acc0 = own0, acc1 = own1;
  int look = t - 1;
  bool ok = true;
  for (;;) {
    const int pos = look - lane;
    unsigned long long v = 0;
    if (pos >= first) {
      v = ld_acquire_u64(&st[pos]);
      while ((v & kStFlagMask) == 0) {
        if (global_ns() - t0 > (unsigned long long)w.timeout_ns) { ok = false; break; }
        __nanosleep(32);
        v = ld_acquire_u64(&st[pos]);
      }
    }
    ok = __all_sync(kFull, ok);
    if (!ok) break;
    const unsigned inc = __ballot_sync(kFull, pos >= first && (v & kStFlagMask) == kStInc);
    const int stop = inc ? __ffs(inc) - 1 : 31;
    long long l = 0, r = 0;
    CandT<double> c0 = cand_none<double>(), c1 = cand_none<double>();
    if (lane <= stop && pos >= first) {
      l = (long long)((v >> 31) & kCnt31);
      r = (long long)(v & kCnt31);
      const bool isinc = (v & kStFlagMask) == kStInc;
      c0 = from_rec(load_rec(isinc ? &rec[pos].incl[0] : &rec[pos].own[0]));
      c1 = from_rec(load_rec(isinc ? &rec[pos].incl[1] : &rec[pos].own[1]));
    }
    exclL += warp_sum_ll(l);
    exclR += warp_sum_ll(r);
    if (__any_sync(kFull, c0.idx >= 0)) {
      c0 = warp_best(&G->ax, c0);
      if (cand_beats(&G->ax, c0, acc0)) acc0 = c0;
    }
    if (__any_sync(kFull, c1.idx >= 0)) {
      c1 = warp_best(&G->rx, c1);
      if (cand_beats(&G->rx, c1, acc1)) acc1 = c1;
    }
    if (inc) break;
    look -= kWarp;
    if (look < first) { ok = false; break; }  // cannot happen: the first tile is inclusive
  }
  if (!ok) {
    if (lane == 0) atomicOr(&w.ctrl->err, kErrTimeout);
    return false;
  }
  if (lane == 0) {
    rec[t].incl[0] = to_rec(acc0);
    rec[t].incl[1] = to_rec(acc1);
    if (publish)
      st_release_u64(&st[t], kStInc | st_pack((unsigned long long)exclL + aggL, (unsigned long long)exclR + aggR));
  }
  incl0 = acc0;
  incl1 = acc1;
  return true;
}

// Unordered offsets and farthest-point candidates for one tile (lane 0 of
// warp 0): one 64-bit atomic on the segment's cursor returns both children's
// output offsets; the tile's best per child is published as a candidate when
// its upper bound reaches the largest lower bound seen so far.  The true
// farthest point's tile always qualifies (its upper bound is at least every
// tile's lower bound), so it is always listed.
__device__ __forceinline__ void tile_atomic(const Work& w, int par, int sid, int t, unsigned long long cnt0,
                                            unsigned long long cnt1, const CandT<double>& c0,
                                            const CandT<double>& c1, long long& eL, long long& eR) {
  SegState* st = &w.sstate[par][sid];
  const unsigned long long old = atomicAdd(&st->cursor, (cnt0 << 32) | cnt1);
  eL = (long long)(old >> 32);
  eR = (long long)(old & 0xffffffffull);
  TileRec* rec = &w.cand[par][t];
  rec->own[0] = to_rec(c0);
  rec->own[1] = to_rec(c1);
#pragma unroll
  for (int ch = 0; ch < 2; ch++) {
    const CandT<double>& c = ch ? c1 : c0;
    if (c.idx < 0) continue;
    const unsigned long long klo = dkey(c.lo);
    const unsigned long long prev = atomicMax(&st->lomax[ch], klo);
    const unsigned long long thr = prev > klo ? prev : klo;
    if (dkey(c.hi) >= thr) {
      const int i = atomicAdd(&st->ncand[ch], 1);
      if (i < kMaxCand) st->cand[ch][i] = t;
    }
  }
}

// ---- asynchronous global -> shared copies (cp.async, per thread) ----
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// Shared-memory layout of the partition kernel: an input stage (the tile's
// points, copied asynchronously) and an output stage (the compacted
// survivors), each split into one region per warp.
template <int PPT>
struct K1Layout {
  static constexpr int WPB = kK1Threads / kWarp;
  static constexpr int TW = kWarp * PPT;     // points per warp
  static constexpr int TB = WPB * TW;        // points per block tile
  static constexpr size_t bytes = 2ull * TB * (2 * sizeof(double) + sizeof(int));
};

struct K1Shared {
  int tot[2][kK1Threads / kWarp];
  int pre[2][kK1Threads / kWarp];
  CandT<double> best[2][kK1Threads / kWarp];
  int excl[2];
  int tick;
};

// Warp part of a block tile: classify this warp's points (read from its
// input region), find its exact farthest point per child, compact the
// survivors into its output region (left child from the start, right child
// from the end).  Points are re-read from shared memory in each pass, so no
// per-point registers are held across the rare exact paths.
template <int PPT, bool SRC_INPUT, bool FAST>
__device__ __forceinline__ void k1_warp_part(const Work& w, const SegRec& S, const SegGeom* __restrict__ G, int j,
                                             const double* ix, const double* iy, const int* ii, double* ox_,
                                             double* oy_, int* oi_, int warp, int lane, int& tot0, int& tot1,
                                             CandT<double>& best0, CandT<double>& best1) {
  typedef typename KeyOf<FAST>::T K;
  typedef K1Layout<PPT> Ly;
  const int begin = S.off + j * Ly::TB + warp * Ly::TW;
  const int count = S.len - j * Ly::TB - warp * Ly::TW;
  // pass 1: filter only; undecided points are flagged
  unsigned cls = 0, und = 0;
  K lo0 = key_neg_inf<K>(), lo1 = key_neg_inf<K>();
  const LineF l1 = line1_of(*G), l2 = line2_of(*G);
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const int l = k * kWarp + lane;
    if (l < count) {
      K key, err;
      const int c = classify_filter(*G, l1, l2, ix[l], iy[l], key, err);
      if (c == 3) {
        und |= 1u << k;
      } else {
        cls |= (unsigned)c << (2 * k);
        if (c == 1) lo0 = key_max(lo0, key_lo(key, err));
        if (c == 2) lo1 = key_max(lo1, key_lo(key, err));
      }
    }
  }
  // pass 2 (rare): exact classification of the undecided points
  if (__any_sync(kFull, und != 0)) {
#pragma unroll 1
    for (int k = 0; k < PPT; k++) {
      if (!((und >> k) & 1u)) continue;
      const int l = k * kWarp + lane;
      const double ux = ix[l], uy = iy[l];
      const int c = classify_exact(G, ux, uy);
      cls |= (unsigned)c << (2 * k);
      if (c != 0) {
        K key, err;
        if (c == 1) line_key_k(l1, &G->ax, ux, uy, key, err);
        else line_key_k(l2, &G->rx, ux, uy, key, err);
        if (c == 1) lo0 = key_max(lo0, key_lo(key, err));
        else lo1 = key_max(lo1, key_lo(key, err));
      }
    }
  }
  // pass 3: exact farthest point per child; candidates are the points whose
  // upper bound reaches the warp's best lower bound
  const K L0 = warp_max_k(lo0), L1 = warp_max_k(lo1);
  CandT<K> b0 = cand_none<K>(), b1 = cand_none<K>();
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const unsigned c = (cls >> (2 * k)) & 3u;
    if (c == 0u) continue;
    const int l = k * kWarp + lane;
    const double ux = ix[l], uy = iy[l];
    K key, err;
    if (c == 1u) line_key_k(l1, &G->ax, ux, uy, key, err);
    else line_key_k(l2, &G->rx, ux, uy, key, err);
    if (key_hi(key, err) < (c == 1u ? L0 : L1)) continue;
    const int id = SRC_INPUT ? begin + l : ii[l];
    if (c == 1u) take_best(b0, &G->ax, ux, uy, id, key, err);
    else take_best(b1, &G->rx, ux, uy, id, key, err);
  }
  if (__any_sync(kFull, b0.idx >= 0)) b0 = warp_best(&G->ax, b0);
  if (__any_sync(kFull, b1.idx >= 0)) b1 = warp_best(&G->rx, b1);
  best0 = to_double(b0);
  best1 = to_double(b1);
  // compaction into the output region, in point order per child
  tot0 = 0;
  tot1 = 0;
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const unsigned c = (cls >> (2 * k)) & 3u;
    const unsigned mL = __ballot_sync(kFull, c == 1u), mR = __ballot_sync(kFull, c == 2u);
    int q = -1;
    if (c == 1u) q = tot0 + __popc(mL & lt);
    else if (c == 2u) q = Ly::TW - 1 - (tot1 + __popc(mR & lt));
    if (q >= 0) {
      const int l = k * kWarp + lane;
      ox_[q] = ix[l];
      oy_[q] = iy[l];
      oi_[q] = SRC_INPUT ? begin + l : ii[l];
    }
    tot0 += __popc(mL);
    tot1 += __popc(mR);
  }
  __syncwarp();
}

// Partition kernel: one block per tile.  A block takes the next tile number
// when it starts (so tiles are processed in claim order and a look-back only
// waits for tiles already in progress), copies the tile's points into shared
// memory (cp.async), lets its warps classify and compact their parts
// independently, combines their counts and farthest points, runs the
// segment's decoupled look-back (warp 0) and writes the survivors out with
// contiguous, coalesced stores.
template <int PPT, bool SRC_INPUT>
__global__ void __launch_bounds__(kK1Threads) k_k1(Work w, int level) {
  typedef K1Layout<PPT> Ly;
  constexpr int WPB = Ly::WPB, TW = Ly::TW, TB = Ly::TB;
  extern __shared__ __align__(16) unsigned char k1_smem[];
  __shared__ K1Shared sh;
  if (fatal(w)) return;
  const int par = level & 1;
  const int srcb = (level + 1) & 1, dstb = level & 1;
  const int ntiles = min(*reinterpret_cast<volatile int*>(&w.ctrl->k1_tiles[par]), w.capT);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int t = blockIdx.x;
  if (w.ordered) {  // the look-back needs tiles in start order
    if (tid == 0) sh.tick = atomicAdd(&w.ctrl->k1_ticket, 1);
    __syncthreads();
    t = sh.tick;
  }
  if (t >= ntiles) return;
  const int sid = __ldg(&w.tile_seg[par][t]);
#ifdef VQ_CHECKED
  if (!VQ_OK_IDX(w, 20, sid, 0, w.capS)) return;
#endif
  const SegRec S = w.segs[par][sid];
  const SegGeom* G = &w.geom[par][sid];
  const int j = t - S.tile_base;
  double* const base = reinterpret_cast<double*>(k1_smem);
  double* ix = base + warp * TW;
  double* iy = base + TB + warp * TW;
  double* ox_ = base + 2 * TB + warp * TW;
  double* oy_ = base + 3 * TB + warp * TW;
  int* ii = reinterpret_cast<int*>(base + 4 * TB) + warp * TW;
  int* oi_ = reinterpret_cast<int*>(base + 4 * TB) + TB + warp * TW;
  {
    const int begin = S.off + j * TB + warp * TW;
    const int count = S.len - j * TB - warp * TW;
    const double* sx = SRC_INPUT ? w.x : w.bx[srcb];
    const double* sy = SRC_INPUT ? w.y : w.by[srcb];
    const int* si = w.bi[srcb];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      const int l = k * kWarp + lane;
      if (l < count && VQ_OK_IDX(w, 7, (long long)begin + l, 0, w.N)) {
        cp_async8(ix + l, sx + begin + l);
        cp_async8(iy + l, sy + begin + l);
        if (!SRC_INPUT) cp_async4(ii + l, si + begin + l);
      }
    }
    cp_async_commit();
    cp_async_wait<0>();  // each lane reads back only what it copied
  }
  int tot0, tot1;
  CandT<double> best0, best1;
  if (S.flags & kSegFast)
    k1_warp_part<PPT, SRC_INPUT, true>(w, S, G, j, ix, iy, ii, ox_, oy_, oi_, warp, lane, tot0, tot1, best0, best1);
  else
    k1_warp_part<PPT, SRC_INPUT, false>(w, S, G, j, ix, iy, ii, ox_, oy_, oi_, warp, lane, tot0, tot1, best0, best1);
  if (lane == 0) {
    sh.tot[0][warp] = tot0;
    sh.tot[1][warp] = tot1;
    sh.best[0][warp] = best0;
    sh.best[1][warp] = best1;
  }
  __syncthreads();
  if (warp == 0) {
    // warp prefixes, block totals, block farthest points, then the
    // segment's look-back for this tile
    const int t0 = lane < WPB ? sh.tot[0][lane] : 0, t1 = lane < WPB ? sh.tot[1][lane] : 0;
    int i0 = t0, i1 = t1;
#pragma unroll
    for (int o = 1; o < WPB; o <<= 1) {
      const int n0 = __shfl_up_sync(kFull, i0, o), n1 = __shfl_up_sync(kFull, i1, o);
      if (lane >= o) { i0 += n0; i1 += n1; }
    }
    if (lane < WPB) { sh.pre[0][lane] = i0 - t0; sh.pre[1][lane] = i1 - t1; }
    const int bt0 = __shfl_sync(kFull, i0, WPB - 1), bt1 = __shfl_sync(kFull, i1, WPB - 1);
    CandT<double> c0 = cand_none<double>(), c1 = cand_none<double>();
    if (lane < WPB) { c0 = sh.best[0][lane]; c1 = sh.best[1][lane]; }
    if (__any_sync(kFull, c0.idx >= 0)) c0 = warp_best(&G->ax, c0);
    if (__any_sync(kFull, c1.idx >= 0)) c1 = warp_best(&G->rx, c1);
    long long eL = 0, eR = 0;
    bool ok = true;
    if (w.ordered) {
      CandT<double> i0c, i1c;
      ok = lookback_warp(w, par, t, S.tile_base, G, (unsigned long long)bt0, (unsigned long long)bt1, c0, c1, eL, eR,
                         i0c, i1c, lane);
      if (ok && lane == 0 && t == S.tile_base + S.ntiles - 1) {
        // last tile: publish the segment's totals and farthest points in the
        // form the finalize kernel reads
        SegState* st = &w.sstate[par][sid];
        st->cursor = ((unsigned long long)(eL + bt0) << 32) | (unsigned long long)(eR + bt1);
        w.cand[par][t].own[0] = to_rec(i0c);
        w.cand[par][t].own[1] = to_rec(i1c);
        for (int ch = 0; ch < 2; ch++) {
          const CandT<double>& c = ch ? i1c : i0c;
          st->lomax[ch] = c.idx >= 0 ? dkey(c.lo) : 0ull;
          st->ncand[ch] = c.idx >= 0 ? 1 : 0;
          st->cand[ch][0] = t;
        }
      }
    } else if (lane == 0) {
      tile_atomic(w, par, sid, t, (unsigned long long)bt0, (unsigned long long)bt1, c0, c1, eL, eR);
    }
    if (lane == 0) {
      const bool fits = ok && eL + bt0 <= S.len && eR + bt1 <= S.len;
      sh.excl[0] = fits ? (int)eL : -1;
      sh.excl[1] = fits ? (int)eR : -1;
    }
  }
  __syncthreads();
  const int eL = sh.excl[0], eR = sh.excl[1];
  if (eL < 0) return;
#ifdef VQ_CHECKED
  if (!VQ_OK_IDX(w, 9, (long long)S.off + S.len, 1, (long long)w.N + 1) || !VQ_OK_IDX(w, 10, S.off, 0, w.N)) return;
#endif
  // contiguous copy-out of this warp's survivors
  double* __restrict__ dx = w.bx[dstb];
  double* __restrict__ dy = w.by[dstb];
  int* __restrict__ di = w.bi[dstb];
  const int l0 = S.off + eL + sh.pre[0][warp];
  for (int i = lane; i < tot0; i += kWarp) {
    __stcs(dx + l0 + i, ox_[i]);
    __stcs(dy + l0 + i, oy_[i]);
    __stcs(di + l0 + i, oi_[i]);
  }
  const int r0 = S.off + S.len - eR - sh.pre[1][warp] - tot1;
  for (int i = lane; i < tot1; i += kWarp) {
    const int q = TW - tot1 + i;
    __stcs(dx + r0 + i, ox_[q]);
    __stcs(dy + r0 + i, oy_[q]);
    __stcs(di + r0 + i, oi_[q]);
  }
}

#include "vq_sieve.cuh"

// ---------------------------------------------------------------------------
// K2: per segment, cross-tile argmax, emission, children
// ---------------------------------------------------------------------------

// Child ch's farthest point from the segment's candidate list (exact), or
// from every tile's record when the list overflowed.
__device__ BestRec seg_best(const Work& w, int par, int s, const SegRec& S, int ch, const double* L, int lane) {
  const SegState* st = &w.sstate[par][s];
  const int nc = __ldcg(&st->ncand[ch]);
  const double thr = dkey_inv(__ldcg(&st->lomax[ch]));
  CandT<double> best = cand_none<double>();
#ifdef VQ_K1_PROFILE
  if (lane == 0) {
    atomicAdd(&w.ctrl->k2prof[0], 1ull);
    if (nc > kMaxCand) atomicAdd(&w.ctrl->k2prof[1], 1ull);
    atomicAdd(&w.ctrl->k2prof[2], (unsigned long long)(nc < kMaxCand ? nc : kMaxCand));
    if (nc > kMaxCand) atomicAdd(&w.ctrl->k2prof[3], (unsigned long long)S.ntiles);
  }
#endif
  if (nc <= kMaxCand) {
    for (int i = lane; i < nc; i += kWarp) {
      const int t = __ldcg(&st->cand[ch][i]);
      const BestRec r = load_rec(&w.cand[par][t].own[ch]);
      if (r.idx < 0 || r.hi < thr) continue;
      const CandT<double> c = from_rec(r);
      if (cand_beats(L, c, best)) best = c;
    }
  } else if (!w.ordered) {
    // The streaming partition kernel gave warp g of nw the tile range
    // [T g / nw, T (g+1) / nw) and wrote records only at the last tile of
    // each run of one segment: visit exactly those tiles of this segment.
    const long long T = min(__ldcg(&w.ctrl->k1_tiles[par]), w.capT), nw = __ldcg(&w.ctrl->k1_nw[par]);
    const long long tb = S.tile_base, te = tb + S.ntiles;
    if (nw > 0 && T > 0 && te <= T) {
      // the warp holding tile u is the last g with T g / nw <= u, i.e.
      // g = ceil((u + 1) nw / T) - 1
      long long g0 = ((tb + 1) * nw + T - 1) / T - 1, g1 = (te * nw + T - 1) / T - 1;
      if (g0 > nw - 1) g0 = nw - 1;
      if (g1 > nw - 1) g1 = nw - 1;
      for (long long g = g0 + lane; g <= g1; g += kWarp) {
        const long long b = T * g / nw, e = T * (g + 1) / nw;
        const long long last = (e < te ? e : te) - 1;
        if (last < (b > tb ? b : tb)) continue;  // no tile of this segment in the range
        const BestRec r = load_rec(&w.cand[par][last].own[ch]);
        if (r.idx < 0 || r.hi < thr) continue;
        const CandT<double> c = from_rec(r);
        if (cand_beats(L, c, best)) best = c;
      }
    }
  } else {
    for (int t = S.tile_base + lane; t < S.tile_base + S.ntiles; t += kWarp) {
      const BestRec r = load_rec(&w.cand[par][t].own[ch]);
      if (r.idx < 0 || r.hi < thr) continue;
      const CandT<double> c = from_rec(r);
      if (cand_beats(L, c, best)) best = c;
    }
  }
  best = warp_best(L, best);
  return to_rec(best);
}

__device__ void make_child(const Work& w, const SegRec& P, int a, int b, int r, int off, int len, int level,
                           int buf, int lane) {
  if (r < 0) {
    if (lane == 0) atomicOr(&w.ctrl->err, kErrInternal);
    return;
  }
  if (len == 1) {  // a single point is its own farthest point: Alg. 1, |P| <= 1
    if (lane == 0) emit(w, (long long)off + 1 + P.shift, r - P.set_off);
    return;
  }
  SegRec C;
  C.shift = P.shift;
  C.off = off;
  C.len = len;
  C.a = a;
  C.b = b;
  C.r = r;
  C.set_off = P.set_off;
  C.level = level;
  C.tile_base = 0;
  C.ntiles = 0;
  C.flags = (P.flags & (kSegFast | kSegDense)) | (buf ? kSegSrcBuf1 : 0);
  if (len <= seg_small_max(w, C.flags)) {
    if (lane == 0) push_k3(w, C);
  } else {
    push_k1_warp(w, (level & 1), C, lane);
  }
}

__global__ void k_k2(const Work* __restrict__ wp, int level) {
  const Work& w = *wp;
  if (fatal(w)) return;
  const int par = level & 1, dstb = level & 1;
  const int nseg = min(*reinterpret_cast<volatile int*>(&w.ctrl->k1_segs[par]), w.capS);
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int s = gw; s < nseg; s += nw) {
    const SegRec S = w.segs[par][s];
    const SegGeom& G = w.geom[par][s];
    const double ax = G.ax, ay = G.ay, rx = G.rx, ry = G.ry, bx = G.bx, by = G.by;
    (void)ax; (void)ay; (void)rx; (void)ry; (void)bx; (void)by;
    const unsigned long long cur = __ldcg(&w.sstate[par][s].cursor);
    const int nL = (int)(cur >> 32), nR = (int)(cur & 0xffffffffull);
    if (nL + nR > S.len) {
      if (lane == 0) atomicOr(&w.ctrl->err, kErrInternal);
      continue;
    }
    BestRec bl, br;
    bl.idx = -1;
    br.idx = -1;
    if (nL > 0) bl = seg_best(w, par, s, S, 0, &w.geom[par][s].ax, lane);
    if (nR > 0) br = seg_best(w, par, s, S, 1, &w.geom[par][s].rx, lane);
#ifdef VQ_CHECKED
    if ((nL > 0 && !VQ_OK_IDX(w, 11, bl.idx, 0, w.N)) || (nR > 0 && !VQ_OK_IDX(w, 11, br.idx, 0, w.N))) continue;
#endif
    if (lane == 0) {
      emit(w, (long long)S.off + nL + 1 + S.shift, S.r - S.set_off);
      add_stats(w, S.level, S.len, nL + nR);
      atomicAdd(reinterpret_cast<unsigned long long*>(&w.ctrl->k1_read), (unsigned long long)S.len);
      atomicAdd(reinterpret_cast<unsigned long long*>(&w.ctrl->k1_kept), (unsigned long long)(nL + nR));
    }
    if (nL > 0) make_child(w, S, S.a, S.r, bl.idx, S.off, nL, S.level + 1, dstb, lane);
    if (nR > 0) make_child(w, S, S.r, S.b, br.idx, S.off + S.len - nR, nR, S.level + 1, dstb, lane);
  }
}

// ---------------------------------------------------------------------------
// K3: small segments, one block each, finished in shared memory
// ---------------------------------------------------------------------------

#include "vq_small.cuh"

// ---------------------------------------------------------------------------
// K5: the persistent segment worklist (the recursion below a small level)
// ---------------------------------------------------------------------------

#include "vq_worklist.cuh"

// ---------------------------------------------------------------------------
// K4: order the emitted vertices by key (bitmap compaction)
// ---------------------------------------------------------------------------

__device__ __forceinline__ int block_excl_scan_256(int v, int* sh, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < kWarp; o <<= 1) {
    const int n = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int s = lane < 8 ? sh[lane] : 0;
    int si = s;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const int n = __shfl_up_sync(kFull, si, o);
      if (lane >= o) si += n;
    }
    if (lane < 8) sh[8 + lane] = si - s;
    if (lane == 7) sh[16] = si;
  }
  __syncthreads();
  const int r = sh[8 + warp] + incl - v;
  total = sh[16];
  __syncthreads();
  return r;
}

// The bitmap words in use: all, or those a single set's finalize cleared.
__device__ __forceinline__ long long k4_words(long long nwords, const Ctrl* ctrl) {
  const long long k = *reinterpret_cast<const volatile long long*>(&ctrl->key_words);
  return k > 0 && k < nwords ? k : nwords;
}

__global__ void __launch_bounds__(256) k_k4_count(const unsigned* bm, long long nwords, long long* sums,
                                                  long long nb, const Ctrl* ctrl) {
  __shared__ int sh[24];
  if (blockIdx.x == 0 && threadIdx.x == 0) sums[nb] = 0;  // becomes the total after the scan
  nwords = k4_words(nwords, ctrl);
  if ((long long)blockIdx.x * kK4Words >= nwords) {  // beyond the words in use (uniform)
    if (threadIdx.x == 0) sums[blockIdx.x] = 0;
    return;
  }
  const long long w0 = (long long)blockIdx.x * kK4Words + threadIdx.x * 4;
  int c = 0;
#pragma unroll
  for (int q = 0; q < 4; q++)
    if (w0 + q < nwords) c += __popc(bm[w0 + q]);
  int total;
  block_excl_scan_256(c, sh, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(256) k_k4_write(const unsigned* bm, long long nwords, const long long* sums,
                                                  const int* slot, int* out, long long cap, Ctrl* ctrl) {
  __shared__ int sh[24];
  nwords = k4_words(nwords, ctrl);
  if ((long long)blockIdx.x * kK4Words >= nwords) return;  // uniform
  const long long w0 = (long long)blockIdx.x * kK4Words + threadIdx.x * 4;
  unsigned v[4];
  int c = 0;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    v[q] = (w0 + q < nwords) ? bm[w0 + q] : 0u;
    c += __popc(v[q]);
  }
  int total;
  const int pre = block_excl_scan_256(c, sh, total);
  long long pos = sums[blockIdx.x] + pre;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    unsigned m = v[q];
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
#ifdef VQ_CHECKED
      if (pos >= cap) {
        if (atomicCAS(&ctrl->dbg_site, 0, 19) == 0) ctrl->dbg_val = pos;
        atomicOr(&ctrl->err, kErrInternal);
        return;
      }
#endif
      out[pos++] = slot[(w0 + q) * 32 + b];
    }
  }
}

// One-pass ordering: chunks of kK4Words bitmap words, taken in order by a
// ticket; each chunk counts its set bits, publishes the count, finds its
// exclusive prefix by decoupled look-back over the chunks before it (their
// status words: 0 not yet, count << 2 | 1 aggregate, prefix << 2 | 2
// inclusive), publishes its inclusive prefix and writes its vertices.
// Only the chunks that hold the words in use are taken.  sums[c] gets
// chunk c's exclusive prefix and sums[nb] the total (for the per-set
// offsets); every wait is bounded by timeout_ns.
__global__ void __launch_bounds__(256) k_k4_fused(const unsigned* bm, long long nwords, unsigned long long* status,
                                                  unsigned* ticket, long long* sums, long long nb, const int* slot,
                                                  int* out, long long cap, Ctrl* ctrl, long long* total,
                                                  long long timeout_ns) {
  __shared__ int sh[24];
  __shared__ int s_t;
  __shared__ long long s_pre;
  const long long nw = k4_words(nwords, ctrl);
  const long long nch = (nw + kK4Words - 1) / kK4Words;
  if (nch == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      *total = 0;
      sums[nb] = 0;
    }
    return;
  }
  for (;;) {
    if (threadIdx.x == 0) s_t = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const long long t = s_t;
    if (t >= nch) return;  // uniform
    const long long w0 = t * kK4Words + threadIdx.x * 4;
    unsigned v[4];
    int c = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      v[q] = (w0 + q < nw) ? bm[w0 + q] : 0u;
      c += __popc(v[q]);
    }
    int cnt;
    const int pre = block_excl_scan_256(c, sh, cnt);
    if (threadIdx.x == 0) {
      long long acc = 0;
      if (t == 0) {
        st_release_u64(&status[0], ((unsigned long long)cnt << 2) | 2ull);
      } else {
        st_release_u64(&status[t], ((unsigned long long)cnt << 2) | 1ull);
        const unsigned long long t0 = global_ns();
        for (long long j = t - 1; j >= 0;) {
          const unsigned long long sv = ld_acquire_u64(&status[j]);
          if ((sv & 3ull) == 0ull) {
            if (global_ns() - t0 > (unsigned long long)timeout_ns) {
              atomicOr(&ctrl->err, kErrTimeout);
              break;
            }
            continue;
          }
          acc += (long long)(sv >> 2);
          if ((sv & 3ull) == 2ull) break;
          j--;
        }
        st_release_u64(&status[t], ((unsigned long long)(acc + cnt) << 2) | 2ull);
      }
      sums[t] = acc;
      if (t == nch - 1) {
        *total = acc + cnt;
        sums[nb] = acc + cnt;
      }
      s_pre = acc;
    }
    __syncthreads();
    long long pos = s_pre + pre;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      unsigned m = v[q];
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        if (pos < cap) out[pos] = slot[(w0 + q) * 32 + b];
        pos++;
      }
    }
    __syncthreads();  // s_t and s_pre are rewritten by the next chunk
  }
}

// Rank of a key among the emitted ones (set bits below it), one warp per
// key: the block prefix plus the bits of the words before it in its block.
__device__ __forceinline__ long long key_rank_warp(const unsigned* bm, long long nwords, const long long* sums,
                                                   long long key, int lane) {
  const long long word = key >> 5;
  const long long blk = word / kK4Words;
  long long r = 0;
  for (long long q = blk * kK4Words + lane; q < word && q < nwords; q += kWarp) r += __popc(bm[q]);
  r = warp_sum_ll(r);
  r += sums[blk];
  if (word < nwords) r += __popc(bm[word] & ((1u << (unsigned)(key & 31)) - 1u));
  return r;
}

// hull_offsets[s] = rank of set s's first key (one warp per set); the
// total is the scan's last entry.
__global__ void k_k4_offsets(Work w, const long long* sums, long long nb, long long* hull_offsets, long long* total) {
  const long long nwords = (w.nkeys + 31) >> 5;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  if (gw == 0 && lane == 0) {
    if (total) *total = sums[nb];
    if (hull_offsets) hull_offsets[w.nsets] = sums[nb];
  }
  if (!hull_offsets) return;
  for (int s = gw; s < w.nsets; s += nw) {
    const long long key = (long long)w.sets[s].off + w.sets[s].shift;
    const long long r = key_rank_warp(w.bitmap, nwords, sums, key, lane);
    if (lane == 0) hull_offsets[s] = r;
  }
}

// ---------------------------------------------------------------------------
// generic exclusive scan (in place), 2048 items per block, recursive
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(256) k_scan_block(T* data, long long n, T* sums) {
  __shared__ T sh[24];
  const long long b0 = (long long)blockIdx.x * 2048 + threadIdx.x * 8;
  T v[8];
  T s = 0;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    v[q] = (b0 + q < n) ? data[b0 + q] : (T)0;
    s += v[q];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = s;
#pragma unroll
  for (int o = 1; o < kWarp; o <<= 1) {
    const T m = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += m;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    T run = 0;
    for (int q = 0; q < 8; q++) { const T t = sh[q]; sh[8 + q] = run; run += t; }
    sh[16] = run;
  }
  __syncthreads();
  T run = sh[8 + warp] + incl - s;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    if (b0 + q < n) data[b0 + q] = run;
    run += v[q];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = sh[16];
}

template <typename T>
__global__ void k_scan_add(T* data, long long n, const T* sums) {
  const long long b0 = (long long)blockIdx.x * 2048;
  const T add = sums[blockIdx.x];
  for (int q = threadIdx.x; q < 2048; q += blockDim.x)
    if (b0 + q < n) data[b0 + q] += add;
}

template <typename T>
static cudaError_t scan_rec(T* data, long long n, T* tmp, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long nb = (n + 2047) / 2048;
  count_launch();
  k_scan_block<T><<<(unsigned)nb, 256, 0, st>>>(data, n, tmp);
  if (nb > 1) {
    cudaError_t e = scan_rec<T>(tmp, nb, tmp + nb, st);
    if (e != cudaSuccess) return e;
    count_launch();
    k_scan_add<T><<<(unsigned)nb, 256, 0, st>>>(data, n, tmp);
  }
  return cudaGetLastError();
}

long long scan_tmp_elems(long long n) {
  long long t = 0;
  while (n > 1) {
    n = (n + 2047) / 2048;
    t += n;
  }
  return t + 8;
}

cudaError_t scan_exclusive_i32(int* data, long long n, int* tmp, cudaStream_t st) {
  return scan_rec<int>(data, n, tmp, st);
}
cudaError_t scan_exclusive_i64(long long* data, long long n, long long* tmp, cudaStream_t st) {
  return scan_rec<long long>(data, n, tmp, st);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------


cudaError_t launch_seed_single(const Work& w, cudaStream_t st) {
  count_launch();
  k_seed_single<<<1, 256, 0, st>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_seed(const Work& w, cudaStream_t st) {
  const int blocks = (w.nsets + 255) / 256;
  count_launch();
  k_seed<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(w);
  return cudaGetLastError();
}

static int device_sms() {
  static int sms[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (sms[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
    sms[dev] = n;
  }
  return sms[dev];
}

// upper bound of the extreme-pass tiles (exact for one set)
static long long k0_tiles_bound(const Work& w) {
  return w.offsets ? (long long)w.N / kK0Tile + w.nsets : (w.n_single + kK0Tile - 1) / kK0Tile;
}


static constexpr int k0_ring_bytes() { return (int)(sizeof(double2) * kK0Stages * 2 * kK0Pairs * kK0Threads); }

// Extreme pass: a resident grid, sized so that every block gets the same
// number of tiles (the tile count is exact for one set, an upper bound for
// several).
cudaError_t launch_k0(const Work& w, int grid, cudaStream_t st) {
  (void)grid;
  static int occ[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (occ[dev] == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_k0, cudaFuncAttributeMaxDynamicSharedMemorySize, k0_ring_bytes());
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_k0, kK0Threads, k0_ring_bytes());
    if (e != cudaSuccess) return e;
    occ[dev] = n > 0 ? n : 1;
  }
  const long long tiles = k0_tiles_bound(w);
  long long g = (long long)occ[dev] * device_sms();
  if (tiles < g) g = tiles;
  if (g < 1) g = 1;
  const long long rounds = (tiles + g - 1) / g;
  if (rounds > 0) g = (tiles + rounds - 1) / rounds;
  if (g < 1) g = 1;
  count_launch();
  k_k0<<<(unsigned)g, kK0Threads, k0_ring_bytes(), st>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_k0_finalize(const Work& w, cudaStream_t st) {
  long long blocks = w.nsets;
  if (blocks > 4096) blocks = 4096;
  count_launch();
  k_k0_finalize<<<(unsigned)(blocks > 0 ? blocks : 1), kK0Threads, 0, st>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_sample(const Work& w, cudaStream_t st) {
  long long g = (long long)device_sms() * 8;
  const long long units = (k0_tiles_bound(w) / kSampleEvery + 1 + w.nsets) * kSampleParts;
  if (g > units) g = units;
  if (g < 1) g = 1;
  count_launch();
  k_sample<<<(unsigned)g, 256, 0, st>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_poly(const Work& w, cudaStream_t st) {
  long long g = ((long long)w.nsets + 3) / 4;
  if (g > 2048) g = 2048;
  if (g < 1) g = 1;
  count_launch();
  k_poly<<<(unsigned)g, 128, 0, st>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_sieve(const Work& w, cudaStream_t st) {
  static int occ[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  constexpr int threads = 32 * kSvWarps;
  if (occ[dev] == 0) {
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sieve, threads, 0);
    if (e != cudaSuccess) return e;
    occ[dev] = n > 0 ? n : 1;
  }
  long long g = (long long)occ[dev] * device_sms();
  const long long tiles = k0_tiles_bound(w);
  if (g > tiles) g = tiles;
  if (g > kSvMaxBlocks) g = kSvMaxBlocks;
  if (g < 1) g = 1;
  count_launch();
  k_sieve<<<(unsigned)g, threads, 0, st>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_level_cond(const Work& w, cudaGraphConditionalHandle h, cudaStream_t st) {
  count_launch();
  k_level_cond<<<1, 1, 0, st>>>(w.dev, h);
  return cudaGetLastError();
}

void count_launches(long long k) { count_launch((int)k); }

cudaError_t add_loop_init_node(cudaGraph_t g, cudaGraphNode_t* node, const Work& w, cudaGraphConditionalHandle h) {
  const Work* wd = w.dev;
  void* args[2] = {&wd, &h};
  cudaKernelNodeParams p = {};
  p.func = reinterpret_cast<void*>(k_loop_init);
  p.gridDim = dim3(1);
  p.blockDim = dim3(1);
  p.sharedMemBytes = 0;
  p.kernelParams = args;
  p.extra = nullptr;
  return cudaGraphAddKernelNode(node, g, nullptr, 0, &p);
}

cudaError_t launch_prologue(const Work& w, int level, cudaStream_t st) {
  count_launch();
  k_prologue<<<1, 1, 0, st>>>(w.dev, level);
  return cudaGetLastError();
}

template <int PPT>
static size_t k1_smem() {
  return K1Layout<PPT>::bytes;
}

template <int PPT>
static cudaError_t k1_attrs() {
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (done[dev]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_k1<PPT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k1_smem<PPT>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_k1<PPT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k1_smem<PPT>());
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

template <int PPT>
static cudaError_t launch_k1_ppt(const Work& w, int level, int grid, cudaStream_t st) {
  if (w.tile != kK1Threads * PPT) return cudaErrorInvalidValue;
  cudaError_t e = k1_attrs<PPT>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kK1Threads);
  cfg.dynamicSmemBytes = k1_smem<PPT>();
  cfg.stream = st;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  count_launch();
  if (level == 0 && !w.sieve) return cudaLaunchKernelEx(&cfg, k_k1<PPT, true>, w, level);
  return cudaLaunchKernelEx(&cfg, k_k1<PPT, false>, w, level);
}

cudaError_t launch_k1(const Work& w, int level, int ppt, int grid, cudaStream_t st) {
  if (!w.ordered) return launch_k1w(w, level, ppt, grid, st);  // vq_partition.cu
  switch (ppt) {
    case 4: return launch_k1_ppt<4>(w, level, grid, st);
    case 8: return launch_k1_ppt<8>(w, level, grid, st);
    case 16: return launch_k1_ppt<16>(w, level, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int PPT>
static int k1_occ() {
  int n = 0, n0 = 0;
  if (k1_attrs<PPT>() != cudaSuccess) return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_k1<PPT, false>, kK1Threads, k1_smem<PPT>()) != cudaSuccess) return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n0, k_k1<PPT, true>, kK1Threads, k1_smem<PPT>()) != cudaSuccess) return 1;
  n = n0 < n ? n0 : n;
  return n > 0 ? n : 1;
}

int k1_blocks_per_sm(int ppt) {
  switch (ppt) {
    case 4: return k1_occ<4>();
    case 8: return k1_occ<8>();
    case 16: return k1_occ<16>();
    default: return 1;
  }
}

cudaError_t launch_k2(const Work& w, int level, int grid, cudaStream_t st) {
  count_launch();
  k_k2<<<grid, 256, 0, st>>>(w.dev, level);
  return cudaGetLastError();
}

// Test access to the FP32 tier: for triples (ax, ay, bx, by, ux, uy) the
// evaluation of orient(a, b, u) that the partition, finalize and pre-filter
// kernels use: make_line on the exact endpoints, trunc_f32 of the point,
// orient_f32 with its bound.
__global__ void k_debug_orient_f32(const double* tri, long long m, int tier, float* d, float* e) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m; k += (long long)gridDim.x * blockDim.x) {
    const double* t = tri + 6 * k;
    const LineF L = make_line(t[0], t[1], t[2], t[3]);
    float key, err;
    if (tier == 0) line_key_k(L, nullptr, t[4], t[5], key, err);
    else orient_rel(L, t[0], t[1], t[4], t[5], key, err);
    d[k] = key;
    e[k] = err;
  }
}

__global__ void k_debug_round_f32(const double* v, long long m, float* out) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m; k += (long long)gridDim.x * blockDim.x)
    out[k] = f32_rn(v[k]);
}

cudaError_t launch_debug_round_f32(const double* v, long long m, float* out, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  long long blocks = (m + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  count_launch();
  k_debug_round_f32<<<(unsigned)blocks, 256, 0, st>>>(v, m, out);
  return cudaGetLastError();
}

cudaError_t launch_debug_orient_f32(const double* tri, long long m, int tier, float* d, float* e, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  long long blocks = (m + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  count_launch();
  k_debug_orient_f32<<<(unsigned)blocks, 256, 0, st>>>(tri, m, tier, d, e);
  return cudaGetLastError();
}

// Chunk hull -> merge buffer: point idx[i] (chunk-local) of the chunk's
// arrays, with its original index base + idx[i].
__global__ void k_gather(const double* x, const double* y, const int* idx, long long m, long long base, double* mx,
                         double* my, int* mid) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const int u = idx[i];
    mx[i] = x[u];
    my[i] = y[u];
    mid[i] = (int)(base + u);
  }
}

__global__ void k_map_indices(const int* mout, const int* mid, long long h, int* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < h; i += (long long)gridDim.x * blockDim.x)
    out[i] = mid[mout[i]];
}

cudaError_t launch_gather(const double* x, const double* y, const int* idx, long long m, long long base, double* mx,
                          double* my, int* mid, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  long long blocks = (m + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  count_launch();
  k_gather<<<(unsigned)blocks, 256, 0, st>>>(x, y, idx, m, base, mx, my, mid);
  return cudaGetLastError();
}

cudaError_t launch_map_indices(const int* mout, const int* mid, long long h, int* out, cudaStream_t st) {
  if (h <= 0) return cudaSuccess;
  long long blocks = (h + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  count_launch();
  k_map_indices<<<(unsigned)blocks, 256, 0, st>>>(mout, mid, h, out);
  return cudaGetLastError();
}

cudaError_t launch_tilemap(const Work& w, int par, int grid, cudaStream_t st) {
  count_launch();
  k_tilemap<<<grid, 256, 0, st>>>(w.dev, par);
  return cudaGetLastError();
}

int k3_smem_bytes() { return (int)sizeof(K3Smem); }

cudaError_t launch_k3(const Work& w, int grid, cudaStream_t st) {
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_k3, cudaFuncAttributeMaxDynamicSharedMemorySize, k3_smem_bytes());
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  count_launch();
  k_k3<<<grid, kK3Threads, k3_smem_bytes(), st>>>(w.dev);
  return cudaGetLastError();
}

int wl_smem_bytes() { return (int)sizeof(WlSmem); }

#ifdef VQ_WL_PROFILE
// Profiling builds: the FP64-filter and exact-expansion call counts of this
// translation unit's kernels since the last read (then cleared).
// Profiling builds: the per-task trace of the next worklist launch goes to
// a device buffer; wl_trace_dump writes it to `path` as text.
static unsigned long long* g_trace_dev = nullptr;
void wl_trace_arm(cudaStream_t st) {
  if (!g_trace_dev) {
    if (cudaMalloc(&g_trace_dev, sizeof(unsigned long long) * 8 * kWlTraceCap) != cudaSuccess) {
      g_trace_dev = nullptr;
      return;
    }
    cudaMemcpyToSymbol(g_wl_trace, &g_trace_dev, sizeof g_trace_dev);
  }
  const int z = 0;
  cudaMemcpyToSymbolAsync(g_wl_trace_n, &z, sizeof z, 0, cudaMemcpyHostToDevice, st);
}
void wl_trace_dump(const char* path) {
  int n = 0;
  cudaMemcpyFromSymbol(&n, g_wl_trace_n, sizeof n);
  if (n > kWlTraceCap) n = kWlTraceCap;
  if (!g_trace_dev || n <= 0) return;
  unsigned long long* h = (unsigned long long*)malloc(sizeof(unsigned long long) * 8 * (size_t)n);
  if (!h) return;
  cudaMemcpy(h, g_trace_dev, sizeof(unsigned long long) * 8 * (size_t)n, cudaMemcpyDeviceToHost);
  FILE* f = fopen(path, "a");
  if (f) {
    fprintf(f, "# call\n");
    for (int i = 0; i < n; i++) {
      const unsigned long long* e = h + 8 * (size_t)i;
      fprintf(f, "%llu %llu %llu %llu %llu %lld %llu %llu %llu %llu\n", e[0], e[1], e[2], e[3] >> 32,
              e[3] & 0xffffffffull, (long long)e[4], e[5] >> 32, e[5] & 0xffffffffull, e[6], e[7]);
    }
    fclose(f);
  }
  free(h);
}

void wl_tier_calls(unsigned long long* out) {
  for (int i = 0; i < 8; i++) out[i] = 0ull;
  cudaMemcpyFromSymbol(out, g_vq_tier_calls, sizeof(unsigned long long) * 8);
  const unsigned long long z[8] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
  cudaMemcpyToSymbol(g_vq_tier_calls, z, sizeof z);
}
#endif

cudaError_t launch_worklist(const Work& w, cudaStream_t st) {
  if (w.capWQ == 0 || w.wl_points <= 0) return cudaSuccess;
  static int blocks[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!blocks[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_wl, cudaFuncAttributeMaxDynamicSharedMemorySize, wl_smem_bytes());
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wl, kWlThreads, wl_smem_bytes());
    if (e != cudaSuccess) return e;
    blocks[dev] = (per_sm > 0 ? per_sm : 1) * device_sms();
  }
#ifdef VQ_WL_PROFILE
  if (const char* e = getenv("VQ_WL_BLOCKS")) {  // profiling builds: another grid
    const int b = atoi(e);
    if (b > 0 && b < blocks[dev]) {
      count_launch(2);
      k_wl_init<<<1, 256, 0, st>>>(w.dev);
      k_wl<<<b, kWlThreads, wl_smem_bytes(), st>>>(w.dev);
      return cudaGetLastError();
    }
  }
#endif
#ifdef VQ_WL_PROFILE
  wl_trace_arm(st);
#endif
  count_launch(2);
  k_wl_init<<<1, 256, 0, st>>>(w.dev);
  k_wl<<<blocks[dev], kWlThreads, wl_smem_bytes(), st>>>(w.dev);
  return cudaGetLastError();
}

// tmp: status words (nb), the ticket, the chunk prefixes and the total
// (nb + 1); 2 nb + 3 entries.
long long order_fused_tmp_elems(long long nkeys) {
  const long long nb = ((nkeys + 31) / 32 + kK4Words - 1) / kK4Words;
  return 2 * nb + 3;
}

cudaError_t launch_order_fused(const Work& w, int* out, long long* hull_offsets, long long* total, long long* tmp,
                               cudaStream_t st) {
  const long long nwords = (w.nkeys + 31) >> 5;
  const long long nb = (nwords + kK4Words - 1) / kK4Words;
  unsigned long long* status = reinterpret_cast<unsigned long long*>(tmp);
  unsigned* ticket = reinterpret_cast<unsigned*>(tmp + nb);
  long long* sums = tmp + nb + 1;
  cudaError_t e = cudaMemsetAsync(tmp, 0, sizeof(long long) * (size_t)(nb + 1), st);
  if (e != cudaSuccess) return e;
  long long grid = 2LL * device_sms();
  if (grid > nb) grid = nb;
  if (grid < 1) grid = 1;
  count_launch();
  k_k4_fused<<<(unsigned)grid, 256, 0, st>>>(w.bitmap, nwords, status, ticket, sums, nb, w.slot, out, (long long)w.N,
                                             w.ctrl, total, w.timeout_ns);
  if (hull_offsets) {
    long long blocks = ((long long)w.nsets + 7) / 8;
    if (blocks > 1024) blocks = 1024;
    count_launch();
    k_k4_offsets<<<(unsigned)blocks, 256, 0, st>>>(w, sums, nb, hull_offsets, nullptr);
  }
  return cudaGetLastError();
}

cudaError_t launch_order(const Work& w, int* out, long long* hull_offsets, long long* total, long long* tmp,
                         cudaStream_t st) {
  const long long nwords = (w.nkeys + 31) >> 5;
  const long long nb = (nwords + kK4Words - 1) / kK4Words;
  long long* sums = tmp;  // nb + 1 entries: block prefixes, then the total
  count_launch();
  k_k4_count<<<(unsigned)nb, 256, 0, st>>>(w.bitmap, nwords, sums, nb, w.ctrl);
  cudaError_t e = scan_exclusive_i64(sums, nb + 1, tmp + nb + 1, st);
  if (e != cudaSuccess) return e;
  count_launch();
  k_k4_write<<<(unsigned)nb, 256, 0, st>>>(w.bitmap, nwords, sums, w.slot, out, (long long)w.N, w.ctrl);
  long long blocks = ((long long)w.nsets + 7) / 8;
  if (blocks > 1024) blocks = 1024;
  count_launch();
  k_k4_offsets<<<(unsigned)blocks, 256, 0, st>>>(w, sums, nb, hull_offsets, total);
  return cudaGetLastError();
}

}  // namespace vq
