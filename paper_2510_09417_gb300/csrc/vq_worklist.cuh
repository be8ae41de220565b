// vq_worklist.cuh -- the persistent segment worklist (K5): Alg. 1's
// recursion below the level where the level loop hands over.  Included by
// vq_kernels.cu inside namespace vq after the small-segment finisher; not a
// standalone header.
//
// Once a level holds few points, the level-synchronous loop spends its time
// on launches and on the dependent loads that open each of its per-level
// kernels, not on points.  The worklist runs the rest of the recursion in
// one launch with no level barrier: a child segment is ready as soon as its
// parent's last partition task has finished (the task that takes the
// parent's last ticket reduces the farthest-point records and pushes the
// children), so the branches of the recursion proceed independently.
//
// Blocks are persistent: each claims the next queue index (one atomic),
// waits until that entry is published, runs it and claims again.  Tasks:
//   partition: up to kWlTaskPts points of a big segment (kWlPPT per thread):
//     Sec. 3's classification against a->r and r->b, compaction into the
//     segment's range of the other buffer (left child from the start, right
//     child from the end, one cursor atomic per task) and the task's
//     farthest point per child (Sec. 4, found in the same pass);
//   small: a segment of at most small_max points, finished whole in shared
//     memory by the finisher's rounds (k3_solve).
// Termination: wl_pending counts the tasks queued or running.  A producer
// adds before it publishes and a task subtracts itself after its own
// pushes, so the count reaches 0 exactly when the recursion is done, and no
// entry is published after that.  A block whose claimed entry is not
// published leaves when it reads 0.  Every wait is bounded by timeout_ns
// (kErrTimeout).  Overflow of the queue or of the segment table raises
// kErrWorklistFull: the blocks leave and the host runs the call again with
// the level loop alone.
// Memory ordering: a task's stores (the children's points, its record) are
// followed by a fence in every thread and a block barrier before the task
// takes its ticket; the block that takes the last ticket fences before it
// reads the records; a producer fences after writing a segment slot and its
// entries and publishes each entry's tag with a release store, which the
// consumer reads with an acquire load.  What this kernel writes it reads
// with L1-bypassing loads.
#pragma once

// Profiling builds (VQ_WL_PROFILE): thread 0 of every block sums its task
// counts and times (globaltimer ns) into Ctrl::k1prof: [0] partition tasks,
// [1] small tasks, [2] waiting for an entry, [3] in partition tasks (with
// their segment finishes), [4] in small tasks, [5] in segment finishes,
// [6] ~(first block start), [7] last block end, [8] longest small task,
// [9] longest partition task, [10] ~(init start), [11] points of the small
// tasks; and the phases of the partition tasks into Ctrl::k3prof: [0] the
// segment's record, [1] points, classification, the warps' farthest points,
// [2] the barrier after them, [3] the task's record and cursor atomic,
// [4] stores and fences, [5] the ticket.
#ifdef VQ_WL_PROFILE
// and a per-task trace (g_wl_trace, up to kWlTraceCap entries of 8 words:
// claim time, start, end, queue index << 32 | block, segment slot or -1,
// level << 32 | points, finished-the-segment flag, 0)
constexpr int kWlTraceCap = 1 << 16;
__device__ unsigned long long* g_wl_trace;
__device__ int g_wl_trace_n;
#define WL_NOW(v) const unsigned long long v = global_ns()
#define WL_ADD(i, d) atomicAdd(&w.ctrl->k1prof[i], (unsigned long long)(d))
#define WL_MAX(i, d) atomicMax(&w.ctrl->k1prof[i], (unsigned long long)(d))
#define WL_PH(i, d) atomicAdd(&w.ctrl->k3prof[i], (unsigned long long)(d))
#else
#define WL_PH(i, d)
#define WL_NOW(v)
#define WL_ADD(i, d)
#define WL_MAX(i, d)
#endif

constexpr int kWlThreads = kK3Threads;  // a block runs the finisher's rounds as well
constexpr int kWlWarps = kWlThreads / kWarp;
static_assert(kWlTaskPts == kWlThreads * kWlPPT, "a partition task: kWlPPT points per thread");

struct WlTileSmem {
  WlSeg seg;                      // the task's segment (copy; its cursor and ticket are not used)
  CandT<double> wc[2][kWlWarps];  // per child and warp: farthest point of the warp's points
  int cnt[2][kWlWarps];           // per child and warp: survivors
  int pre[2][kWlWarps];           // exclusive prefix sums of cnt
  int tot[2];
  unsigned long long old;         // the segment's cursor before this task
  int last;                       // this task completed the segment
};

struct WlSmem {
  union {
    K3Smem k3;
    WlTileSmem t;
  } u;
  WlTask task;
  int h;
};

// The protocol's fences: release before a ticket or a tag, acquire after
// one (message passing only, so no sequentially consistent fence is needed).
__device__ __forceinline__ void wl_fence() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Thread 0: claim the next queue index and wait until its entry is
// published.  Returns the index, or -1 when the block should leave (queue
// exhausted, recursion done, fatal error, timeout).
__device__ int wl_pop(const Work& w, WlTask* out) {
  Ctrl* c = w.ctrl;
  const int h = atomicAdd(&c->wl_head, 1);
  if (h >= w.capWQ) return -1;
  // the entry's own tag is polled (entries spread over the cache); the
  // shared counters only every eighth time
  const unsigned long long t0 = global_ns();
  unsigned ns = 32;
  for (int it = 1;; it++) {
    if (ld_relaxed_u32(&w.wltag[h]) == w.wl_epoch) {
      wl_fence();  // with the relaxed read: acquires the producer's release
      break;
    }
    if ((it & 7) == 0) {
      if ((unsigned)*reinterpret_cast<volatile unsigned long long*>(&c->wl_tp) == 0u) return -1;
      if (fatal(w)) return -1;
      if (global_ns() - t0 > (unsigned long long)w.timeout_ns) {
        atomicOr(&c->err, kErrTimeout);
        return -1;
      }
    }
    __nanosleep(ns);
    if (ns < 512) ns *= 2;
  }
  const int4* src = reinterpret_cast<const int4*>(&w.wlq[h]);
  int4* dst = reinterpret_cast<int4*>(out);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(WlTask) / sizeof(int4)); i++) dst[i] = __ldcg(src + i);
  return h;
}

// One thread: queue a small segment.
__device__ void wl_push_small(const Work& w, const SegRec& C) {
  Ctrl* c = w.ctrl;
  const int t = (int)(atomicAdd(&c->wl_tp, (1ull << 32) | 1ull) >> 32);
  if (t >= w.capWQ) {
    atomicOr(&c->err, kErrWorklistFull);
    atomicAdd(&c->wl_tp, ~0ull);  // not pending after all
    return;
  }
  WlTask T;
  T.R = C;
  T.seg = -1;
  T.begin = 0;
  T.count = C.len;
  T.pad = 0;
  w.wlq[t] = T;
  wl_fence();
  st_release_u32(&w.wltag[t], w.wl_epoch);
}

// Warp: a big segment into a slot of the segment table (geometry of its
// child lines for the FP32 tier) and its partition tasks into the queue.
__device__ void wl_push_big(const Work& w, const SegRec& C, int lane) {
  Ctrl* c = w.ctrl;
  const int nt = (C.len + kWlTaskPts - 1) / kWlTaskPts;
  int slot = -1, t0 = 0;
  if (lane == 0) {
    slot = atomicAdd(&c->wl_nseg, 1);
    if (slot < w.capWS) {
      t0 = (int)(atomicAdd(&c->wl_tp, ((unsigned long long)nt << 32) | (unsigned long long)nt) >> 32);
      if (t0 > w.capWQ - nt) {
        atomicAdd(&c->wl_tp, 0ull - (unsigned long long)nt);  // not pending after all
        slot = -1;
      }
    } else {
      slot = -1;
    }
    if (slot < 0) atomicOr(&c->err, kErrWorklistFull);
  }
  slot = __shfl_sync(kFull, slot, 0);
  t0 = __shfl_sync(kFull, t0, 0);
  if (slot < 0) return;
  if (lane == 0) {
    WlSeg S;
    S.R = C;
    fill_geom(S.G, px(w, C.a), py(w, C.a), px(w, C.b), py(w, C.b), px(w, C.r), py(w, C.r));
    S.cursor = 0ull;
    S.ndone = 0;
    S.ntasks = nt;
    S.t0 = t0;
    S.pad[0] = S.pad[1] = S.pad[2] = 0;
    w.wlseg[slot] = S;
    wl_fence();
  }
  __syncwarp();
  for (int i = lane; i < nt; i += kWarp) {
    WlTask T;
    T.R = C;
    T.seg = slot;
    T.begin = i * kWlTaskPts;
    T.count = min(kWlTaskPts, C.len - T.begin);
    T.pad = 0;
    w.wlq[t0 + i] = T;
  }
  wl_fence();
  for (int i = lane; i < nt; i += kWarp) st_release_u32(&w.wltag[t0 + i], w.wl_epoch);
}

// Warp: child (a, b) of P with farthest point r, its points at positions
// off .. off+len-1 of buffer buf (Alg. 1's recursion on S1 or S2).
__device__ void wl_child(const Work& w, const SegRec& P, int a, int b, int r, int off, int len, int buf,
                         int lane) {
  if (len <= 0) return;
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
  C.level = P.level + 1;
  C.tile_base = 0;
  C.ntiles = 0;
  C.flags = (P.flags & (kSegFast | kSegDense)) | (buf ? kSegSrcBuf1 : 0);
  if (len <= seg_small_max(w, C.flags)) {
    if (lane == 0) wl_push_small(w, C);
  } else {
    wl_push_big(w, C, lane);
  }
}

// Source and destination buffers of a segment's points (-1: the caller's arrays).
__device__ __forceinline__ int wl_src(int flags) {
  return (flags & kSegSrcInput) ? -1 : ((flags & kSegSrcBuf1) ? 1 : 0);
}
__device__ __forceinline__ int wl_dst(int flags) { return wl_src(flags) == 0 ? 1 : 0; }

// Block: the segment's last task is done.  Its children's farthest points
// are the exact best of the tasks' records; emit r (key: the position
// between the children), push the children.
__device__ void wl_finish(const Work& w, WlSmem& S, int sid) {
  const WlTileSmem& M = S.u.t;
  const SegRec& R = M.seg.R;
  const SegGeom& G = M.seg.G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long cur = __ldcg(&w.wlseg[sid].cursor);
  const int nL = (int)(cur >> 32), nR = (int)(cur & 0xffffffffull);
  if (nL + nR > R.len) {
    if (threadIdx.x == 0) atomicOr(&w.ctrl->err, kErrInternal);
    return;
  }
  const int t0 = M.seg.t0, nt = M.seg.ntasks;
  if (warp < 2) {
    const int ch = warp;
    const int n = ch ? nR : nL;
    if (n > 0) {
      const double* E = ch ? &G.rx : &G.ax;
      const bool fast = (R.flags & kSegFast) != 0;
      const LineF Lf = fast ? (ch ? line2_of(G) : line1_of(G)) : LineF{};
      CandT<double> b = cand_none<double>();
      for (int i = lane; i < nt; i += kWarp) {
        const BestRec r = load_rec(&w.wlrec[2 * (long long)(t0 + i) + ch]);
        if (r.idx < 0) continue;
        const CandT<double> c = from_rec(r);
        if (fast ? cand_beats(Lf, E, c, b) : cand_beats(E, c, b)) b = c;
      }
      b = fast ? warp_best(Lf, E, b) : warp_best(E, b);
      const int dst = wl_dst(R.flags);
      if (ch == 0) wl_child(w, R, R.a, R.r, b.idx, R.off, nL, dst, lane);
      else wl_child(w, R, R.r, R.b, b.idx, R.off + R.len - nR, nR, dst, lane);
    }
  } else if (warp == 2 && lane == 0) {
    emit(w, (long long)R.off + nL + 1 + R.shift, R.r - R.set_off);
    add_stats(w, R.level, R.len, nL + nR);
    atomicAdd(reinterpret_cast<unsigned long long*>(&w.ctrl->k1_read), (unsigned long long)R.len);
    atomicAdd(reinterpret_cast<unsigned long long*>(&w.ctrl->k1_kept), (unsigned long long)(nL + nR));
    atomicMax(&w.ctrl->wl_maxlevel, R.level + 1);
  }
}

// Block: one partition task (points begin .. begin+count-1 of the segment
// in S.u.t.seg).
template <bool FAST>
__device__ void wl_tile(const Work& w, WlSmem& S, const WlTask& T, int h) {
  typedef typename KeyOf<FAST>::T K;
  WlTileSmem& M = S.u.t;
  const SegRec& R = M.seg.R;
  const SegGeom& G = M.seg.G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int src = wl_src(R.flags), dst = wl_dst(R.flags);
  const int base = R.off + T.begin;
  const int count = min(T.count, kWlTaskPts);
  WL_NOW(ph0);
  LineF l1 = {}, l2 = {};
  if (FAST) {
    l1 = line1_of(G);
    l2 = line2_of(G);
  }
  // the warp's points: kWlPPT columns of 32, coalesced
  double X[kWlPPT], Y[kWlPPT];
  int I[kWlPPT];
#pragma unroll
  for (int k = 0; k < kWlPPT; k++) {
    const int l = warp * (kWarp * kWlPPT) + k * kWarp + lane;
    X[k] = 0.0;
    Y[k] = 0.0;
    I[k] = -1;
    if (l < count) {
      const int p = base + l;
      if (src < 0) {
        X[k] = px(w, p);
        Y[k] = py(w, p);
        I[k] = p;
      } else {
        X[k] = __ldcg(w.bx[src] + p);
        Y[k] = __ldcg(w.by[src] + p);
        I[k] = __ldcg(w.bi[src] + p);
      }
    }
  }
#ifdef VQ_WL_PROFILE
  {  // profiling only: wait for the loads before reading the clock
    unsigned long long z = 0;
#pragma unroll
    for (int k = 0; k < kWlPPT; k++)
      z ^= (unsigned long long)__double_as_longlong(X[k]) ^ (unsigned long long)__double_as_longlong(Y[k]) ^ (unsigned)I[k];
    if (z == 0x5a5a5a5a5a5a5a5aull) M.last = 3;
  }
  WL_NOW(phA);
#endif
  // classification: FP32 tiers, then the exact tiers for what they leave
  K key[kWlPPT], err[kWlPPT];
  unsigned m1 = 0, m2 = 0;
  K lo0 = key_neg_inf<K>(), lo1 = key_neg_inf<K>();
#pragma unroll
  for (int k = 0; k < kWlPPT; k++) {
    key[k] = K(0);
    err[k] = K(0);
    if (I[k] < 0) continue;
    K kk = K(0), ee = K(0);
    int c = classify_filter(G, l1, l2, X[k], Y[k], kk, ee);
    if (c == 3) c = classify_rel(G, l1, l2, X[k], Y[k], kk, ee);
    if (c == 3) {
      c = classify_exact(&G, X[k], Y[k]);
      if (c == 1) line_key_tight(l1, &G.ax, X[k], Y[k], kk, ee);
      if (c == 2) line_key_tight(l2, &G.rx, X[k], Y[k], kk, ee);
    }
    key[k] = kk;
    err[k] = ee;
    if (c == 1) {
      m1 |= 1u << k;
      lo0 = key_max(lo0, key_lo(kk, ee));
    } else if (c == 2) {
      m2 |= 1u << k;
      lo1 = key_max(lo1, key_lo(kk, ee));
    }
  }
#ifdef VQ_WL_PROFILE
  if ((m1 | m2) == 0xfffffffu) M.last = 3;  // profiling only: after the classification
  WL_NOW(phB);
#endif
  // farthest point per child among the warp's survivors: only points whose
  // upper bound reaches the warp's best lower bound can be it
#pragma unroll
  for (int ch = 0; ch < 2; ch++) {
    const unsigned mc = ch ? m2 : m1;
    const K Lc = warp_max_k(ch ? lo1 : lo0);
    const double* E = ch ? &G.rx : &G.ax;
    const LineF lc = ch ? l2 : l1;
    CandT<K> b = cand_none<K>();
#pragma unroll
    for (int k = 0; k < kWlPPT; k++) {
      if (!((mc >> k) & 1u) || key_hi(key[k], err[k]) < Lc) continue;
      K kk, ee;
      line_key_tight(lc, E, X[k], Y[k], kk, ee);
      if constexpr (FAST) take_best(b, lc, E, X[k], Y[k], I[k], kk, ee);
      else take_best(b, E, X[k], Y[k], I[k], kk, ee);
    }
    const unsigned lanes = __ballot_sync(kFull, b.idx >= 0);
    if (__popc(lanes) > 1) {  // usually one lane holds the only candidate
      if constexpr (FAST) b = warp_best(lc, E, b);
      else b = warp_best(E, b);
    }
    else if (lanes) b = shfl_xor_cand(b, lane ^ (__ffs(lanes) - 1));
    const int n = __reduce_add_sync(kFull, __popc(mc));
    if (lane == 0) {
      M.wc[ch][warp] = to_double(b);
      M.cnt[ch][warp] = n;
    }
  }
  WL_NOW(ph1);
  __syncthreads();
  WL_NOW(ph2);
  if (warp < 2) {  // the task's record of child `warp`
    const int ch = warp;
    const double* E = ch ? &G.rx : &G.ax;
    CandT<double> b = lane < kWlWarps ? M.wc[ch][lane] : cand_none<double>();
    // a warp's point whose upper bound is below another's lower bound
    // cannot win (ordered integer images: no FP64 compares)
    unsigned long long lo = b.idx >= 0 ? dkey(b.lo) : 0ull;
#pragma unroll
    for (int m = kWlWarps / 2; m >= 1; m >>= 1) {
      const unsigned long long o = __shfl_xor_sync(kFull, lo, m);
      lo = o > lo ? o : lo;
    }
    if (b.idx >= 0 && dkey(b.hi) < lo) b.idx = -1;
    const unsigned lanes = __ballot_sync(kFull, b.idx >= 0);
    if (__popc(lanes) > 1) {
      if constexpr (FAST) b = warp_best(ch ? l2 : l1, E, b);
      else b = warp_best(E, b);
    }
    else if (lanes) b = shfl_xor_cand(b, lane ^ (__ffs(lanes) - 1));
    if (lane == 0) w.wlrec[2 * (long long)h + ch] = to_rec(b);
#ifdef VQ_WL_PROFILE
    WL_NOW(pr1);
    if (lane == 0) atomicAdd(&w.ctrl->k2prof[ch], pr1 - ph2);
    if (lane == 0 && __popc(lanes) > 1) atomicAdd(&w.ctrl->k2prof[3], 1ull);
#endif
  } else if (warp == 2 && lane == 0) {  // output offsets: one atomic per task
    int tl = 0, tr = 0;
    for (int q = 0; q < kWlWarps; q++) {
      M.pre[0][q] = tl;
      M.pre[1][q] = tr;
      tl += M.cnt[0][q];
      tr += M.cnt[1][q];
    }
    M.tot[0] = tl;
    M.tot[1] = tr;
    M.old = (tl + tr) > 0
                ? atomicAdd(&w.wlseg[T.seg].cursor, ((unsigned long long)tl << 32) | (unsigned long long)tr)
                : 0ull;
#ifdef VQ_WL_PROFILE
    if (M.old == 0x5a5a5a5a5a5a5a5aull) M.last = 3;  // profiling only: after the atomic's result
    WL_NOW(pr2);
    atomicAdd(&w.ctrl->k2prof[2], pr2 - ph2);
#endif
  }
  __syncthreads();
  WL_NOW(ph3);
  // survivors: left child forward from the segment's start, right child
  // backward from its end
  {
    const unsigned long long old = M.old;
    const long long eL = (long long)(old >> 32), eR = (long long)(old & 0xffffffffull);
    if (eL + M.tot[0] <= R.len && eR + M.tot[1] <= R.len) {
      double* __restrict__ dx = w.bx[dst];
      double* __restrict__ dy = w.by[dst];
      int* __restrict__ di = w.bi[dst];
      const int baseL = R.off + (int)eL + M.pre[0][warp];
      const int endR = R.off + R.len - (int)eR - M.pre[1][warp];
      const unsigned lt = lanemask_lt();
      int nl = 0, nr = 0;
#pragma unroll
      for (int k = 0; k < kWlPPT; k++) {
        const bool isL = (m1 >> k) & 1u, isR = (m2 >> k) & 1u;
        const unsigned bL = __ballot_sync(kFull, isL), bR = __ballot_sync(kFull, isR);
        if (isL || isR) {
          const int pos = isL ? baseL + nl + __popc(bL & lt) : endR - 1 - (nr + __popc(bR & lt));
          if (VQ_OK_IDX(w, 60, pos, R.off, (long long)R.off + R.len)) {
            dx[pos] = X[k];
            dy[pos] = Y[k];
            di[pos] = I[k];
          }
        }
        nl += __popc(bL);
        nr += __popc(bR);
      }
    } else if (tid == 0) {
      atomicOr(&w.ctrl->err, kErrInternal);
    }
  }
  // the task's ticket; the last one finishes the segment
  wl_fence();
  __syncthreads();
  WL_NOW(ph4);
  if (tid == 0) M.last = atomicAdd(&w.wlseg[T.seg].ndone, 1) == M.seg.ntasks - 1 ? 1 : 0;
  __syncthreads();
#ifdef VQ_WL_PROFILE
  WL_NOW(ph5);
  if (tid == 0) {
    WL_PH(1, ph1 - ph0);
    WL_PH(2, ph2 - ph1);
    WL_PH(3, ph3 - ph2);
    WL_PH(4, ph4 - ph3);
    WL_PH(5, ph5 - ph4);
    WL_PH(6, phA - ph0);
    WL_PH(7, phB - phA);
  }
#endif
  if (M.last) {
    wl_fence();
    WL_NOW(tf0);
    wl_finish(w, S, T.seg);
#ifdef VQ_WL_PROFILE
    __syncthreads();
    WL_NOW(tf1);
    if (tid == 0) WL_ADD(5, tf1 - tf0);
#endif
  }
}

// Block: one small segment, finished in shared memory (Alg. 1 on at most
// small_max points, round by round as in the small-segment kernel).
__device__ void wl_small(const Work& w, WlSmem& S, const SegRec& R) {
  K3Smem& M = S.u.k3;
  const int tid = threadIdx.x;
  if (R.len < 2 || R.len > kK3Cap || R.off < 0 || (long long)R.off + R.len > (long long)w.N || R.a < 0 ||
      R.a >= w.N || R.b < 0 || R.b >= w.N || R.r < 0 || R.r >= w.N) {
    if (tid == 0) atomicOr(&w.ctrl->err, kErrInternal);
    return;
  }
  const int src = wl_src(R.flags);
  for (int i = tid; i < 3 * kK3StatLevels; i += kWlThreads) (&M.kst[0][0])[i] = 0ull;
  if (tid == 0) {
    M.X[kK3Cap] = px(w, R.a); M.Y[kK3Cap] = py(w, R.a); M.I[kK3Cap] = R.a;
    M.X[kK3Cap + 1] = px(w, R.b); M.Y[kK3Cap + 1] = py(w, R.b); M.I[kK3Cap + 1] = R.b;
    M.ncand = INT_MAX;
  }
  __syncthreads();
  for (int l = tid; l < R.len; l += kWlThreads) {
    const int p = R.off + l;
    if (src < 0) {
      M.X[l] = px(w, p);
      M.Y[l] = py(w, p);
      M.I[l] = p;
    } else {
      M.X[l] = __ldcg(w.bx[src] + p);
      M.Y[l] = __ldcg(w.by[src] + p);
      M.I[l] = __ldcg(w.bi[src] + p);
    }
    if (M.I[l] == R.r) atomicMin(&M.ncand, l);
  }
  __syncthreads();
  const int r0 = M.ncand;
  if (r0 == INT_MAX) {  // the segment's farthest point is not among its points
    if (tid == 0) atomicOr(&w.ctrl->err, kErrInternal);
    return;
  }
  if (R.flags & kSegFast) k3_solve<true>(w, R, M, R.len, r0);
  else k3_solve<false>(w, R, M, R.len, r0);
  __syncthreads();
  for (int l = tid; l < kK3StatLevels; l += kWlThreads) {
    if (M.kst[2][l] == 0ull) continue;
    atomicAdd(reinterpret_cast<unsigned long long*>(&w.stats[l]), M.kst[0][l]);
    atomicAdd(reinterpret_cast<unsigned long long*>(&w.stats[kMaxLevels + l]), M.kst[1][l]);
    atomicAdd(reinterpret_cast<unsigned long long*>(&w.stats[2 * kMaxLevels + l]), M.kst[2][l]);
    atomicMax(&w.ctrl->wl_maxlevel, l + 1);
  }
}

// The persistent kernel: claim, run, repeat until the recursion is done.
__global__ void __launch_bounds__(kWlThreads, 2) k_wl(const Work* __restrict__ wp) {
  extern __shared__ __align__(16) unsigned char wl_raw[];
  WlSmem& S = *reinterpret_cast<WlSmem*>(wl_raw);
  // the call's Work in shared memory: read on every step, and the fences
  // of the protocol would send each read of it back to L2
  __shared__ __align__(16) Work sw;
  static_assert(sizeof(Work) % sizeof(int4) == 0, "Work is copied as int4");
  for (int i = threadIdx.x; i < (int)(sizeof(Work) / sizeof(int4)); i += kWlThreads)
    reinterpret_cast<int4*>(&sw)[i] = __ldg(reinterpret_cast<const int4*>(wp) + i);
  __syncthreads();
  const Work& w = sw;
  if (w.capWQ == 0 || !*reinterpret_cast<const volatile int*>(&w.ctrl->wl_on)) return;
#ifdef VQ_WL_PROFILE
  if (threadIdx.x == 0) WL_MAX(6, ~global_ns());
#endif
  for (;;) {
    WL_NOW(tp0);
#ifdef VQ_WL_PROFILE
    const unsigned long long cc0 = clock64();
#endif
    if (threadIdx.x == 0) S.h = wl_pop(w, &S.task);
    __syncthreads();
    const int h = S.h;
#ifdef VQ_WL_PROFILE
    WL_NOW(tp1);
    if (threadIdx.x == 0) {
      WL_ADD(2, tp1 - tp0);
      if (h < 0) WL_MAX(7, tp1);
    }
#endif
    if (h < 0) return;
    const WlTask T = S.task;
    if (T.seg < 0) {
      wl_small(w, S, T.R);
    } else if (T.seg >= w.capWS || T.count <= 0 || T.count > kWlTaskPts) {
      if (threadIdx.x == 0) atomicOr(&w.ctrl->err, kErrInternal);
    } else {
      constexpr int kSegVec = (int)(sizeof(WlSeg) / sizeof(int4));
      if (threadIdx.x < kSegVec)
        reinterpret_cast<int4*>(&S.u.t.seg)[threadIdx.x] =
            __ldcg(reinterpret_cast<const int4*>(&w.wlseg[T.seg]) + threadIdx.x);
      __syncthreads();
#ifdef VQ_WL_PROFILE
      WL_NOW(tps);
      if (threadIdx.x == 0) WL_PH(0, tps - tp1);
#endif
      const SegRec& R = S.u.t.seg.R;
      if (R.off < 0 || (long long)R.off + R.len > (long long)w.N || T.begin < 0 || T.begin + T.count > R.len) {
        if (threadIdx.x == 0) atomicOr(&w.ctrl->err, kErrInternal);
      } else if (R.flags & kSegFast) {
        wl_tile<true>(w, S, T, h);
      } else {
        wl_tile<false>(w, S, T, h);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&w.ctrl->wl_tp, ~0ull);  // this task is done
#ifdef VQ_WL_PROFILE
    WL_NOW(tp2);
    if (threadIdx.x == 0) {
      const bool small = T.seg < 0;
      WL_ADD(small ? 1 : 0, 1);
      WL_ADD(small ? 4 : 3, tp2 - tp1);
      WL_MAX(small ? 8 : 9, tp2 - tp1);
      if (small) WL_ADD(11, T.R.len);
      const int i = atomicAdd(&g_wl_trace_n, 1);
      if (g_wl_trace && i < kWlTraceCap) {
        unsigned long long* e = g_wl_trace + 8 * (long long)i;
        e[0] = tp0;
        e[1] = tp1;
        e[2] = tp2;
        e[3] = ((unsigned long long)h << 32) | blockIdx.x;
        e[4] = (unsigned long long)(long long)T.seg;
        e[5] = ((unsigned long long)(small ? T.R.level : S.u.t.seg.R.level) << 32) | (unsigned)(small ? T.R.len : T.count);
        e[6] = small ? 0ull : (unsigned long long)S.u.t.last;
        e[7] = clock64() - cc0;  // SM cycles from the claim to the end
      }
    }
#endif
  }
}

// One block: the handed-over segments into the queue (big segment s of the
// level into slot s of the segment table), then the pending count.  Runs
// before the persistent kernel, so its entries need no release order.
__global__ void __launch_bounds__(256) k_wl_init(const Work* __restrict__ wp) {
  const Work& w = *wp;
  Ctrl* c = w.ctrl;
  if (w.capWQ == 0 || !c->wl_on || fatal(w)) return;
#ifdef VQ_WL_PROFILE
  if (threadIdx.x == 0) WL_MAX(10, ~global_ns());
#endif
  const int par = c->wl_par & 1;
  const int nb = c->wl_nbig, ns = min(c->wl_nsmall, w.capQ);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (nb < 0 || nb > w.capWS || nb > w.capS) {
    if (threadIdx.x == 0) atomicOr(&c->err, kErrWorklistFull);
    return;
  }
  for (int s = warp; s < nb; s += blockDim.x / kWarp) {
    const SegRec R = w.segs[par][s];
    const int nt = (R.len + kWlTaskPts - 1) / kWlTaskPts;
    int t0 = 0;
    if (lane == 0) t0 = (int)(atomicAdd(&c->wl_tp, (unsigned long long)nt << 32) >> 32);
    t0 = __shfl_sync(kFull, t0, 0);
    if (t0 > w.capWQ - nt) {
      if (lane == 0) atomicOr(&c->err, kErrWorklistFull);
      continue;
    }
    if (lane == 0) {
      WlSeg S;
      S.R = R;
      S.G = w.geom[par][s];
      S.cursor = 0ull;
      S.ndone = 0;
      S.ntasks = nt;
      S.t0 = t0;
      S.pad[0] = S.pad[1] = S.pad[2] = 0;
      w.wlseg[s] = S;
    }
    for (int i = lane; i < nt; i += kWarp) {
      WlTask T;
      T.R = R;
      T.seg = s;
      T.begin = i * kWlTaskPts;
      T.count = min(kWlTaskPts, R.len - T.begin);
      T.pad = 0;
      w.wlq[t0 + i] = T;
      w.wltag[t0 + i] = w.wl_epoch;
    }
  }
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    const int t = (int)(atomicAdd(&c->wl_tp, 1ull << 32) >> 32);
    if (t >= w.capWQ) {
      atomicOr(&c->err, kErrWorklistFull);
      continue;
    }
    WlTask T;
    T.R = w.k3q[i];
    T.seg = -1;
    T.begin = 0;
    T.count = T.R.len;
    T.pad = 0;
    w.wlq[t] = T;
    w.wltag[t] = w.wl_epoch;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned tail = (unsigned)(atomicAdd(&c->wl_tp, 0ull) >> 32);
    const unsigned pend = tail < (unsigned)w.capWQ ? tail : (unsigned)w.capWQ;
    c->wl_tp = ((unsigned long long)tail << 32) | pend;
    c->wl_nseg = nb;
  }
}
