// vq_small.cuh -- the small-segment finisher (K3): segments of at most
// kK3Cap points, one block each, finished inside shared memory.  Alg. 1's
// recursion on the segment's points runs level by level: a round takes
// every open frame of the segment at once (its farthest point, the emission
// of that vertex, the classification of the frame's points against the two
// child lines and their compaction into the children's ranges), so a
// segment needs as many rounds as its recursion is deep, not one step per
// hull vertex.  Included by vq_kernels.cu inside namespace vq after the
// shared helpers; not a standalone header.
#pragma once

constexpr int kK3Threads = 256;
constexpr int kK3PPT = kK3Cap / kK3Threads;  // point positions per thread
constexpr int kK3Frames = kK3Cap / 2;        // open frames hold two points or more
constexpr unsigned short kNoFrame = 0xffff;
constexpr int kK3FewCand = 8;  // a frame with at most this many farthest-point candidates: one thread

// Shared memory of one block.  Point slots 0 .. len-1 hold the segment's
// points, slots kK3Cap and kK3Cap + 1 its endpoints a and b.  Positions are
// the frame order: frame f holds positions [lo, hi) of P[cur].
struct K3Smem {
  double X[kK3Cap + 2], Y[kK3Cap + 2];
  int I[kK3Cap + 2];                 // original indices
  unsigned short P[2][kK3Cap];       // slot at each position (ping-pong)
  unsigned short FR[2][kK3Cap];      // frame of each position, kNoFrame outside every frame
  // open frames (ping-pong): range, endpoints (slots), FP32 line a->b
  unsigned short lo[2][kK3Frames], hi[2][kK3Frames], fa[2][kK3Frames], fb[2][kK3Frames];
  LineF lab[2][kK3Frames];
  // per round
  short fr[kK3Frames];               // farthest point's slot
  int nl[kK3Frames], nr[kK3Frames];  // children's sizes (and insertion cursors)
  unsigned long long kmax[kK3Frames];  // largest lower bound of the key (ordered image)
  int base[kK3Frames];               // first next-round frame id of frame f
  LineF l1[kK3Frames], l2[kK3Frames];  // a->r and r->b
  unsigned short cand[kK3Cap];       // positions of farthest-point candidates, in position order
  short cs[kK3Frames], ce[kK3Frames];  // each frame's range in cand
  int wsum[kK3Threads / kWarp];
  int ncand, nframes;
  unsigned long long kst[3][kK3StatLevels];
};

// Block-wide exclusive prefix sum of one value per thread; total in *tot.
__device__ __forceinline__ int k3_scan(int v, int* wsum, int* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < kWarp; o <<= 1) {
    const int n = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == kWarp - 1) wsum[warp] = incl;
  __syncthreads();
  int before = 0, all = 0;
#pragma unroll
  for (int q = 0; q < kK3Threads / kWarp; q++) {
    const int s = wsum[q];
    if (q < warp) before += s;
    all += s;
  }
  __syncthreads();
  *tot = all;
  return before + incl - v;
}

// The key of a point for the line of frame f (FP32 tier, or FP64 filter),
// as a lower and an upper bound widened to FP64.
template <bool FAST>
__device__ __forceinline__ void k3_key(const K3Smem& M, int cur, int f, double ux, double uy, double& lo,
                                       double& hi) {
  typedef typename KeyOf<FAST>::T K;
  K key, err;
  double E[4] = {M.X[M.fa[cur][f]], M.Y[M.fa[cur][f]], M.X[M.fb[cur][f]], M.Y[M.fb[cur][f]]};
  line_key_tight(M.lab[cur][f], E, ux, uy, key, err);
  lo = widen(key_lo(key, err));
  hi = widen(key_hi(key, err));
}

// One segment (len >= 2 points already in M.X/Y/I, frame 0 = the whole
// segment with its known farthest point r0 (a slot)).
template <bool FAST>
__device__ void k3_solve(const Work& w, const SegRec& S, K3Smem& M, int len, int r0) {
  const int tid = threadIdx.x;
  int cur = 0;
  int depth = 0;
  int F = 1;
  if (tid == 0) {
    M.lo[0][0] = 0; M.hi[0][0] = (unsigned short)len;
    M.fa[0][0] = kK3Cap; M.fb[0][0] = kK3Cap + 1;
    M.lab[0][0] = FAST ? make_line(M.X[kK3Cap], M.Y[kK3Cap], M.X[kK3Cap + 1], M.Y[kK3Cap + 1]) : LineF{};
    M.fr[0] = (short)r0;
  }
  for (int k = 0; k < kK3PPT; k++) {
    const int q = tid * kK3PPT + k;
    M.P[0][q] = (unsigned short)q;
    M.FR[0][q] = q < len ? 0 : kNoFrame;
  }
  __syncthreads();
  while (F > 0) {
    const int nxt = cur ^ 1;
    // A. farthest point of every frame not given one (all but the first)
    if (depth > 0) {
      for (int f = tid; f < F; f += kK3Threads) M.kmax[f] = 0ull;
      __syncthreads();
      double klo[kK3PPT], khi[kK3PPT];
#pragma unroll
      for (int k = 0; k < kK3PPT; k++) {
        const int q = tid * kK3PPT + k;
        klo[k] = -INFINITY;
        khi[k] = -INFINITY;
        const int f = M.FR[cur][q];
        if (f != kNoFrame) {
          const int u = M.P[cur][q];
          k3_key<FAST>(M, cur, f, M.X[u], M.Y[u], klo[k], khi[k]);
          atomicMax(&M.kmax[f], dkey(klo[k]));
        }
      }
      __syncthreads();
      // candidates: points whose upper bound reaches their frame's largest
      // lower bound (the farthest point always does), compacted in position
      // order so that a frame's candidates are adjacent
      unsigned cm = 0;
      int c = 0;
#pragma unroll
      for (int k = 0; k < kK3PPT; k++) {
        const int q = tid * kK3PPT + k;
        const int f = M.FR[cur][q];
        if (f != kNoFrame && khi[k] >= dkey_inv(M.kmax[f])) { cm |= 1u << k; c++; }
      }
      // a thread holds consecutive positions: one scan gives position order
      int total = 0;
      int pos = k3_scan(c, M.wsum, &total);
#pragma unroll
      for (int k = 0; k < kK3PPT; k++)
        if ((cm >> k) & 1u) M.cand[pos++] = (unsigned short)(tid * kK3PPT + k);
      if (tid == 0) M.ncand = total;
      __syncthreads();
      // each frame's candidates are adjacent in the list: its range
      const int nc = M.ncand;
      for (int i = tid; i < nc; i += kK3Threads) {
        const int f = M.FR[cur][M.cand[i]];
        if (i == 0 || M.FR[cur][M.cand[i - 1]] != f) M.cs[f] = i;
        if (i == nc - 1 || M.FR[cur][M.cand[i + 1]] != f) M.ce[f] = i + 1;
      }
      __syncthreads();
      // a frame with few candidates (the usual case once the keys are
      // tight): one thread walks them; with many, one warp: each lane keeps
      // the exact best of its share, then the warp's butterfly.  The order is
      // larger orient, then nearer a, then lower index; O(candidates) exact
      // comparisons either way
      for (int f = tid; f < F; f += kK3Threads) {
        const int c0 = M.cs[f], c1 = M.ce[f];
        if (c1 - c0 > kK3FewCand) continue;
        const double L[4] = {M.X[M.fa[cur][f]], M.Y[M.fa[cur][f]], M.X[M.fb[cur][f]], M.Y[M.fb[cur][f]]};
        CandT<double> best = cand_none<double>();
        int bslot = -1;
        for (int i = c0; i < c1; i++) {
          const int u = M.P[cur][M.cand[i]];
          CandT<double> c;
          c.x = M.X[u]; c.y = M.Y[u]; c.idx = M.I[u];
          k3_key<FAST>(M, cur, f, c.x, c.y, c.lo, c.hi);
          if (FAST ? cand_beats(M.lab[cur][f], L, c, best) : cand_beats(L, c, best)) { best = c; bslot = u; }
        }
        M.fr[f] = (short)bslot;
      }
      const int lane = tid & 31, warp = tid >> 5;
      for (int f = warp; f < F; f += kK3Threads / kWarp) {
        if (M.ce[f] - M.cs[f] <= kK3FewCand) continue;  // uniform across the warp
        const double L[4] = {M.X[M.fa[cur][f]], M.Y[M.fa[cur][f]], M.X[M.fb[cur][f]], M.Y[M.fb[cur][f]]};
        CandT<double> best = cand_none<double>();
        for (int i = M.cs[f] + lane; i < M.ce[f]; i += kWarp) {
          const int u = M.P[cur][M.cand[i]];
          CandT<double> c;
          c.x = M.X[u]; c.y = M.Y[u]; c.idx = M.I[u];
          k3_key<FAST>(M, cur, f, c.x, c.y, c.lo, c.hi);
          if (FAST ? cand_beats(M.lab[cur][f], L, c, best) : cand_beats(L, c, best)) best = c;
        }
        const unsigned lanes = __ballot_sync(kFull, best.idx >= 0);
        if (__popc(lanes) > 1) best = FAST ? warp_best(M.lab[cur][f], L, best) : warp_best(L, best);
        else if (lanes) best = shfl_xor_cand(best, lane ^ (__ffs(lanes) - 1));
        if (lane == 0) {
          // the winner's slot: the candidate with that index
          for (int i = M.cs[f]; i < M.ce[f]; i++) {
            const int u = M.P[cur][M.cand[i]];
            if (M.I[u] == best.idx) { M.fr[f] = (short)u; break; }
          }
        }
      }
      __syncthreads();
    }
    // B. the child lines of every frame; counters
    for (int f = tid; f < F; f += kK3Threads) {
      const int a = M.fa[cur][f], b = M.fb[cur][f], r = M.fr[f];
      if (FAST) {
        M.l1[f] = make_line(M.X[a], M.Y[a], M.X[r], M.Y[r]);
        M.l2[f] = make_line(M.X[r], M.Y[r], M.X[b], M.Y[b]);
      }
      M.nl[f] = 0;
      M.nr[f] = 0;
    }
    for (int k = 0; k < kK3PPT; k++) M.FR[nxt][tid * kK3PPT + k] = kNoFrame;
    __syncthreads();
    // C. classify every point of every frame; move it to its child's range
    int npos[kK3PPT], ncls[kK3PPT], nfr[kK3PPT], nu[kK3PPT];
#pragma unroll
    for (int k = 0; k < kK3PPT; k++) {
      const int q = tid * kK3PPT + k;
      ncls[k] = 0;
      npos[k] = 0;
      nfr[k] = 0;
      nu[k] = 0;
      const int f = M.FR[cur][q];
      if (f == kNoFrame) continue;
      const int u = M.P[cur][q];
      nu[k] = u;
      const int a = M.fa[cur][f], b = M.fb[cur][f], r = M.fr[f];
      SegGeom G;
      G.ax = M.X[a]; G.ay = M.Y[a]; G.rx = M.X[r]; G.ry = M.Y[r]; G.bx = M.X[b]; G.by = M.Y[b];
      typename KeyOf<FAST>::T key, err;
      int c = classify_filter(G, M.l1[f], M.l2[f], M.X[u], M.Y[u], key, err);
      if (c == 3) c = classify_rel(G, M.l1[f], M.l2[f], M.X[u], M.Y[u], key, err);
      if (c == 3) c = classify_exact(&G, M.X[u], M.Y[u]);
      ncls[k] = c;
      nfr[k] = f;
    }
    // positions in the children's ranges: the lanes of a warp that move a
    // point into the same child share one shared-memory atomic (early
    // rounds have a few large frames, whose cursors every point hits)
    {
      const int lane = tid & 31;
      const unsigned lt = lanemask_lt();
#pragma unroll
      for (int k = 0; k < kK3PPT; k++) {
        const int c = ncls[k], f = nfr[k];
        const unsigned key = (c == 1 || c == 2) ? (((unsigned)f << 1) | (unsigned)(c - 1)) : 0xffffffffu;
        const unsigned mm = __match_any_sync(kFull, key);
        if (key != 0xffffffffu) {
          const int leader = __ffs(mm) - 1;
          int base = 0;
          if (lane == leader) base = atomicAdd(c == 1 ? &M.nl[f] : &M.nr[f], __popc(mm));
          base = __shfl_sync(mm, base, leader) + __popc(mm & lt);
          npos[k] = c == 1 ? M.lo[cur][f] + base : M.hi[cur][f] - 1 - base;
          M.P[nxt][npos[k]] = (unsigned short)nu[k];
        }
      }
    }
    __syncthreads();
    // D. per frame (two per thread, in frame order): emit r and the
    // single-point children, count the children that stay open, scan
    constexpr int FPT = (kK3Frames + kK3Threads - 1) / kK3Threads;
    int nchild[FPT];
    int mine = 0;
    unsigned long long st_read = 0, st_kept = 0, st_segs = 0;  // this round's counters (one level)
#pragma unroll
    for (int k = 0; k < FPT; k++) {
      const int f = tid * FPT + k;
      nchild[k] = 0;
      if (f >= F) continue;
      const int lo = M.lo[cur][f], hi = M.hi[cur][f], nl = M.nl[f], nr = M.nr[f], r = M.fr[f];
      emit(w, (long long)S.off + lo + nl + 1 + S.shift, M.I[r] - S.set_off);
      st_read += (unsigned long long)(hi - lo);
      st_kept += (unsigned long long)(nl + nr);
      st_segs += 1ull;
      // a single point is its own farthest point: Alg. 1, |P| <= 1
      if (nl == 1) emit(w, (long long)S.off + lo + 1 + S.shift, M.I[M.P[nxt][lo]] - S.set_off);
      if (nr == 1) emit(w, (long long)S.off + hi + S.shift, M.I[M.P[nxt][hi - 1]] - S.set_off);
      nchild[k] = (nl >= 2 ? 1 : 0) + (nr >= 2 ? 1 : 0);
      mine += nchild[k];
    }
    {  // every frame of a round is at level S.level + depth: one add per warp
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) {
        st_read += __shfl_xor_sync(kFull, st_read, m);
        st_kept += __shfl_xor_sync(kFull, st_kept, m);
        st_segs += __shfl_xor_sync(kFull, st_segs, m);
      }
      const int lvl = S.level + depth;
      if ((tid & 31) == 0 && st_segs > 0) {
        if (lvl < kK3StatLevels) {
          atomicAdd(&M.kst[0][lvl], st_read);
          atomicAdd(&M.kst[1][lvl], st_kept);
          atomicAdd(&M.kst[2][lvl], st_segs);
        } else {
          add_stats(w, lvl, (long long)st_read, (long long)st_kept, (long long)st_segs);
        }
      }
    }
    int F2 = 0;
    int b0 = k3_scan(mine, M.wsum, &F2);
#pragma unroll
    for (int k = 0; k < FPT; k++) {
      const int f = tid * FPT + k;
      if (f >= F) continue;
      M.base[f] = b0;
      // the next round's frames of f: left (a, r) first, then right (r, b)
      const int lo = M.lo[cur][f], hi = M.hi[cur][f], nl = M.nl[f], nr = M.nr[f], r = M.fr[f];
      int id = b0;
      if (nl >= 2) {
        M.lo[nxt][id] = (unsigned short)lo; M.hi[nxt][id] = (unsigned short)(lo + nl);
        M.fa[nxt][id] = M.fa[cur][f]; M.fb[nxt][id] = (unsigned short)r;
        if (FAST) M.lab[nxt][id] = M.l1[f];
        id++;
      }
      if (nr >= 2) {
        M.lo[nxt][id] = (unsigned short)(hi - nr); M.hi[nxt][id] = (unsigned short)hi;
        M.fa[nxt][id] = (unsigned short)r; M.fb[nxt][id] = M.fb[cur][f];
        if (FAST) M.lab[nxt][id] = M.l2[f];
      }
      b0 += nchild[k];
    }
    __syncthreads();
    // E. the frame of every moved point in the next round
#pragma unroll
    for (int k = 0; k < kK3PPT; k++) {
      if (ncls[k] == 0) continue;
      const int f = nfr[k];
      const int nl = M.nl[f], nr = M.nr[f];
      if (ncls[k] == 1 && nl >= 2) M.FR[nxt][npos[k]] = (unsigned short)M.base[f];
      if (ncls[k] == 2 && nr >= 2) M.FR[nxt][npos[k]] = (unsigned short)(M.base[f] + (nl >= 2 ? 1 : 0));
    }
    depth++;
    cur = nxt;
    F = F2;
    __syncthreads();
  }
}

// One block per queued segment of at most kK3Cap points: its points and its
// endpoints a, b into shared memory, the slot of its known farthest point,
// then the rounds.  Per-level counters are summed in shared memory and added
// to the call's once per block.
__global__ void __launch_bounds__(kK3Threads, 2) k_k3(const Work* __restrict__ wp) {
  const Work& w = *wp;
  extern __shared__ __align__(16) unsigned char k3_raw[];
  K3Smem& M = *reinterpret_cast<K3Smem*>(k3_raw);
  if (fatal(w)) return;
  for (int i = threadIdx.x; i < 3 * kK3StatLevels; i += kK3Threads) (&M.kst[0][0])[i] = 0ull;
  const int nq = min(*reinterpret_cast<volatile int*>(&w.ctrl->k3_count), w.capQ);
  for (int e = blockIdx.x; e < nq; e += gridDim.x) {
    const SegRec S = w.k3q[e];
    if (!VQ_OK_IDX(w, 17, (long long)S.off + S.len, 1, (long long)w.N + 1) || !VQ_OK_IDX(w, 18, S.r, 0, w.N)) continue;
    if (S.len > kK3Cap || S.len < 2 || S.a < 0 || S.a >= w.N || S.b < 0 || S.b >= w.N) {
      if (threadIdx.x == 0) atomicOr(&w.ctrl->err, kErrInternal);
      continue;
    }
    const double* sx;
    const double* sy;
    const int* si = nullptr;
    if (S.flags & kSegSrcInput) {
      sx = w.x; sy = w.y;
    } else {
      const int b = (S.flags & kSegSrcBuf1) ? 1 : 0;
      sx = w.bx[b]; sy = w.by[b]; si = w.bi[b];
    }
    __syncthreads();  // the previous segment is done with M
    if (threadIdx.x == 0) {
      M.X[kK3Cap] = px(w, S.a); M.Y[kK3Cap] = py(w, S.a); M.I[kK3Cap] = S.a;
      M.X[kK3Cap + 1] = px(w, S.b); M.Y[kK3Cap + 1] = py(w, S.b); M.I[kK3Cap + 1] = S.b;
      M.ncand = INT_MAX;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < S.len; l += kK3Threads) {
      M.X[l] = sx[S.off + l];
      M.Y[l] = sy[S.off + l];
      M.I[l] = si ? si[S.off + l] : S.off + l;
      if (M.I[l] == S.r) atomicMin(&M.ncand, l);
    }
    __syncthreads();
    const int r0 = M.ncand;
    if (r0 == INT_MAX) {  // the segment's farthest point is not among its points
      if (threadIdx.x == 0) atomicOr(&w.ctrl->err, kErrInternal);
      continue;
    }
    if (S.flags & kSegFast) k3_solve<true>(w, S, M, S.len, r0);
    else k3_solve<false>(w, S, M, S.len, r0);
  }
  __syncthreads();
  for (int l = threadIdx.x; l < kK3StatLevels; l += kK3Threads) {
    if (M.kst[2][l] == 0ull) continue;
    atomicAdd(reinterpret_cast<unsigned long long*>(&w.stats[l]), M.kst[0][l]);
    atomicAdd(reinterpret_cast<unsigned long long*>(&w.stats[kMaxLevels + l]), M.kst[1][l]);
    atomicAdd(reinterpret_cast<unsigned long long*>(&w.stats[2 * kMaxLevels + l]), M.kst[2][l]);
  }
}
