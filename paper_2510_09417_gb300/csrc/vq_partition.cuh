// vq_partition.cuh -- streaming partition kernel (level k >= 0 of Alg. 1's
// subset extraction, all live big segments at once).  Included by
// vq_kernels.cu inside namespace vq after the shared helpers; not a
// standalone header.
//
// For every point u of every live segment (a, b, r) the kernel decides
// left of a->r (left child, S1), left of r->b (right child, S2) or neither
// (Alg. 1, the two partition steps after r is found), writes the survivors
// into the segment's range of the other ping-pong buffer (left child from
// the start, right child from the end) and finds, per tile and child, the
// point farthest from the child's line (the next level's r).
//
// Structure: every warp works on its own.  It owns a ring of NS
// shared-memory stages and walks the level's warp tiles (32 * PPT points of
// one segment) with a stride of the grid's warp count.  Lane 0 streams each
// tile into a stage with 1-D bulk copies (cp.async.bulk, completion on the
// stage's mbarrier) NS tiles ahead, from a per-tile descriptor written when
// the tile map was built.  Per tile the warp classifies its points from
// shared memory (FP32 filter tier, exact tiers for undecided points), takes
// the tile's output offsets with one 64-bit atomic on the segment cursor
// (issued before the farthest-point search, used after it), resolves the
// tile's farthest point per child among the few points whose upper bound
// reaches the tile's best lower bound, and stores the survivors directly:
// per step, one contiguous run per child.  There is no block-wide barrier
// after start-up.  Every wait is bounded by w.timeout_ns; a warp that gives
// up raises kErrTimeout, lets its own copies land and leaves.
#pragma once

// ---- mbarrier / bulk-copy primitives (PTX ISA: mbarrier, cp.async.bulk) ----

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of parity `parity` to complete; false after timeout_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, long long timeout_ns) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(b, parity)) return true;
    if (global_ns() - t0 > (unsigned long long)timeout_ns) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Order-preserving int image of a float (for redux.sync max).
__device__ __forceinline__ int f_ord(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float f_unord(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }
__device__ __forceinline__ float warp_max_redux(float v) { return f_unord(__reduce_max_sync(kFull, f_ord(v))); }
__device__ __forceinline__ double warp_max_redux(double v) { return warp_max_d(v); }

// ---- stage layout ----

struct alignas(16) K1Meta {
  int t, sid, begin, count;  // tile, segment, first buffer position, points
  int sx, sy, si, flags;     // slot of the tile's first point per array; segment flags
  int off, len, pad0, pad1;  // segment range
};

// One stage: the segment's geometry (bulk-copied), the tile's metadata and
// its points.  Point l of the tile is x[l + sx], y[l + sy], i[l + si]; each
// array is copied from the 16-byte boundary at or below its first point.
template <int TW>
struct alignas(16) K1Stage {
  SegGeom g;
  K1Meta m;
  double x[TW + 2];
  double y[TW + 2];
  int i[TW + 8];
};
static_assert(sizeof(SegGeom) == 96, "SegGeom is bulk-copied as 96 bytes");

// A warp's private region: its stages and their mbarriers.
template <int PPT, int NS>
struct alignas(16) K1Ring {
  static constexpr int TW = 32 * PPT;
  K1Stage<TW> st[NS];
  unsigned long long full[NS];
};

// Pass-A classification.  FP32 tier: both lines are evaluated without
// branches; 1 / 2 = left / right child, 0 = discard, 3 = undecided (the
// exact tiers decide).  key/err: the point's orient w.r.t. its child's line
// and its bound.  FP64 tier (point sets outside the FP32 range): the
// filter of classify_filter.
__device__ __forceinline__ int classify_a(const SegGeom&, const LineF& l1, const LineF& l2, double ux, double uy,
                                          float& key, float& err) {
  const float fx = trunc_f32(ux), fy = trunc_f32(uy);
  const float m = __fadd_ru(fabsf(fx), fabsf(fy));
  float d1, e1, d2, e2;
  orient_f32(l1, fx, fy, m, d1, e1);
  orient_f32(l2, fx, fy, m, d2, e2);
  const bool p1 = d1 > e1, n1 = d1 < -e1, p2 = d2 > e2, n2 = d2 < -e2;
  key = p1 ? d1 : d2;
  err = p1 ? e1 : e2;
  return p1 ? 1 : (!n1 ? 3 : (p2 ? 2 : (n2 ? 0 : 3)));
}
__device__ __forceinline__ int classify_a(const SegGeom& g, const LineF& l1, const LineF& l2, double ux, double uy,
                                          double& key, double& err) {
  key = 0.0;
  err = 0.0;
  return classify_filter(g, l1, l2, ux, uy, key, err);
}

// Stage one array.  Elements [0, count) of src (element size ES, src
// ES-aligned) go to slots sh .. sh+count-1 of dst, sh = (src mod 16) / ES.
// The bulk part is the 16-byte-aligned cover of the range, clipped to the
// aligned interior of [arr_lo, arr_hi) when the array is the caller's
// (arr_lo != null); a padded workspace array (arr_lo == null) may be read
// up to 15 bytes beyond the range on either side.  Elements outside the
// bulk part are copied here with plain loads (array ends only).
template <typename T>
struct K1Copy {
  const char* lo;
  unsigned bytes;
  int dst_off;  // byte offset of lo in the stage array
  int sh;
};
template <typename T>
__device__ __forceinline__ K1Copy<T> k1_stage_array(T* dst, const T* src, int count, const T* arr_lo,
                                                    const T* arr_hi) {
  constexpr int ES = (int)sizeof(T);
  const uintptr_t a = reinterpret_cast<uintptr_t>(src);
  const uintptr_t e = reinterpret_cast<uintptr_t>(src + count);
  const uintptr_t base = a & ~uintptr_t(15);
  uintptr_t lo = base, hi = (e + 15) & ~uintptr_t(15);
  if (arr_lo) {
    const uintptr_t al = (reinterpret_cast<uintptr_t>(arr_lo) + 15) & ~uintptr_t(15);
    const uintptr_t ah = reinterpret_cast<uintptr_t>(arr_hi) & ~uintptr_t(15);
    if (lo < al) lo = al;
    if (hi > ah) hi = ah;
    if (hi < lo) hi = lo;
  }
  K1Copy<T> c;
  c.sh = (int)((a - base) / ES);
  c.lo = reinterpret_cast<const char*>(lo);
  c.bytes = (unsigned)(hi - lo);
  c.dst_off = (int)(lo - base);
  if (lo > a || hi < e) {  // plain loads for the elements outside [lo, hi)
    for (int k = 0; k < count; k++) {
      const uintptr_t p = a + (uintptr_t)k * ES;
      if (p < lo || p >= hi) dst[c.sh + k] = src[k];
    }
  }
  return c;
}

__device__ __forceinline__ TileDesc load_desc(const TileDesc* p) {
  const int4 a = __ldg(reinterpret_cast<const int4*>(p));
  const int4 b = __ldg(reinterpret_cast<const int4*>(p) + 1);
  TileDesc d;
  d.sid = a.x; d.begin = a.y; d.count = a.z; d.flags = a.w;
  d.off = b.x; d.len = b.y; d.pad0 = 0; d.pad1 = 0;
  return d;
}

// Lane 0: stage tile t (descriptor d) into stage s of the ring.
template <int PPT, int NS, bool SRC_INPUT>
__device__ __forceinline__ void k1_issue(const Work& w, int par, K1Ring<PPT, NS>* R, int s, int t,
                                         const TileDesc& d) {
  constexpr int TW = 32 * PPT;
  const int srcb = par ^ 1;
  K1Stage<TW>* sg = &R->st[s];
  int count = d.count;
  const bool good = VQ_OK_IDX(w, 40, d.sid, 0, w.capS) && VQ_OK_IDX(w, 41, count, 1, TW + 1) &&
                    VQ_OK_IDX(w, 42, d.begin, 0, w.N) &&
                    VQ_OK_IDX(w, 43, (long long)d.begin + count, 1, (long long)w.N + 1);
  if (!good) count = 0;
  const double* px = (SRC_INPUT ? w.x : w.bx[srcb]) + d.begin;
  const double* py = (SRC_INPUT ? w.y : w.by[srcb]) + d.begin;
  const int* pi = w.bi[srcb] + d.begin;
  const K1Copy<double> cx = k1_stage_array<double>(sg->x, px, count, SRC_INPUT ? w.x : nullptr,
                                                   SRC_INPUT ? w.x + w.N : nullptr);
  const K1Copy<double> cy = k1_stage_array<double>(sg->y, py, count, SRC_INPUT ? w.y : nullptr,
                                                   SRC_INPUT ? w.y + w.N : nullptr);
  K1Copy<int> ci;
  ci.lo = nullptr; ci.bytes = 0; ci.dst_off = 0; ci.sh = 0;
  if (!SRC_INPUT) ci = k1_stage_array<int>(sg->i, pi, count, nullptr, nullptr);
  K1Meta m;
  m.t = t; m.sid = good ? d.sid : 0; m.begin = d.begin; m.count = count;
  m.sx = cx.sh; m.sy = cy.sh; m.si = ci.sh; m.flags = d.flags;
  m.off = d.off; m.len = d.len; m.pad0 = 0; m.pad1 = 0;
  sg->m = m;
  const unsigned gb = good ? (unsigned)sizeof(SegGeom) : 0u;
  unsigned long long* bar = &R->full[s];
  mbar_arrive_expect_tx(bar, gb + cx.bytes + cy.bytes + ci.bytes);
  if (gb) bulk_g2s(&sg->g, &w.geom[par][d.sid], gb, bar);
  if (cx.bytes) bulk_g2s(reinterpret_cast<char*>(sg->x) + cx.dst_off, cx.lo, cx.bytes, bar);
  if (cy.bytes) bulk_g2s(reinterpret_cast<char*>(sg->y) + cy.dst_off, cy.lo, cy.bytes, bar);
  if (ci.bytes) bulk_g2s(reinterpret_cast<char*>(sg->i) + ci.dst_off, ci.lo, ci.bytes, bar);
}

// Profiling builds (VQ_K1_PROFILE): lane 0 of every warp accumulates SM
// cycles per phase; the sums land in Ctrl::k1prof at the end of the kernel:
// [0] tiles, [1] stage wait, [2] classification, [3] farthest point,
// [4] wait for the cursor atomic, [5] stores, [6] copy issue, [7] warp total,
// [8] of [3]: bound reductions, [9] tiles that needed a candidate search,
// [10] candidate searches spanning lanes, [11] candidates.
#ifdef VQ_K1_PROFILE
#define K1_MARK(v) const unsigned long long v = clock64()
#define K1_ADD(P, i, d) ((P)[i] += (d))
#else
#define K1_MARK(v)
#define K1_ADD(P, i, d)
#endif

// A warp's running farthest point per child over its consecutive tiles of
// one segment (warp-uniform registers).  rb: the point with its bounds
// widened to FP64 (for the record); lf / hf: the same bounds in FP32 when
// the segment uses the FP32 tier (exactly representable there).
struct K1Run {
  int sid;     // segment of the running points (-1: none)
  int t_last;  // this warp's last tile of that segment: holds the record
  CandT<double> rb[2];
  float lf[2], hf[2];
};

__device__ __forceinline__ void run_bounds(const K1Run& r, int ch, float& lo, float& hi) {
  lo = r.lf[ch];
  hi = r.hf[ch];
}
__device__ __forceinline__ void run_bounds(const K1Run& r, int ch, double& lo, double& hi) {
  lo = r.rb[ch].lo;
  hi = r.rb[ch].hi;
}
__device__ __forceinline__ void run_set(K1Run& r, int ch, const CandT<float>& b) {
  r.rb[ch] = to_double(b);
  r.lf[ch] = b.lo;
  r.hf[ch] = b.hi;
}
__device__ __forceinline__ void run_set(K1Run& r, int ch, const CandT<double>& b) { r.rb[ch] = b; }

template <typename K>
__device__ __forceinline__ CandT<K> shfl_cand(const CandT<K>& c, int src) {
  CandT<K> o;
  o.x = __shfl_sync(kFull, c.x, src);
  o.y = __shfl_sync(kFull, c.y, src);
  o.lo = __shfl_sync(kFull, c.lo, src);
  o.hi = __shfl_sync(kFull, c.hi, src);
  o.idx = __shfl_sync(kFull, c.idx, src);
  return o;
}

// Close the warp's run of tiles of segment r.sid: the running farthest
// points go to the record of the run's last tile, which is listed as a
// child's candidate when its upper bound reaches the segment's largest
// lower bound (fresh copy; the bound itself was raised as the run improved).
__device__ __forceinline__ void k1w_flush(const Work& w, int par, K1Run& r, int lane) {
  if (r.sid >= 0 && lane == 0) {
    SegState* ss = &w.sstate[par][r.sid];
    TileRec* rec = &w.cand[par][r.t_last];
#pragma unroll
    for (int ch = 0; ch < 2; ch++) {
      const CandT<double>& b = r.rb[ch];
      rec->own[ch] = to_rec(b);
      if (b.idx >= 0) {
        const unsigned long long klo = dkey(b.lo), khi = dkey(b.hi);
        unsigned long long thr = __ldcg(&ss->lomax[ch]);
        if (klo > thr) thr = klo;
        if (khi >= thr) {
          const int i = atomicAdd(&ss->ncand[ch], 1);
          if (i < kMaxCand) ss->cand[ch][i] = r.t_last;
        }
      }
    }
  }
  r.sid = -1;
}

// ---- one warp tile ----

template <int PPT, bool SRC_INPUT, bool FAST>
__device__ __forceinline__ void k1w_tile(const Work& w, int par, K1Stage<32 * PPT>* __restrict__ sg, int lane,
                                         K1Run& run, unsigned long long* prof) {
  (void)prof;
  K1_MARK(c0);
  typedef typename KeyOf<FAST>::T K;
  constexpr int TW = 32 * PPT;
  const int t = sg->m.t, sid = sg->m.sid, begin = sg->m.begin;
  const int count = min(max(sg->m.count, 0), TW);
  const int soff = sg->m.off, slen = sg->m.len;
  const double* X = sg->x + (sg->m.sx & 1);
  const double* Y = sg->y + (sg->m.sy & 1);
  const int* I = sg->i + (sg->m.si & 3);
  const SegGeom* G = &sg->g;
  SegState* ss = &w.sstate[par][sid];
  if (sid != run.sid) {
    k1w_flush(w, par, run, lane);
    run.sid = sid;
    run.rb[0] = cand_none<double>();
    run.rb[1] = cand_none<double>();
    run.lf[0] = run.lf[1] = run.hf[0] = run.hf[1] = 0.0f;
  }
  run.t_last = t;
  if (lane == 0) {  // no record in this tile unless the run ends here
    w.cand[par][t].own[0].idx = -1;
    w.cand[par][t].own[1].idx = -1;
  }

  // pass A: filter tier for every point; class masks, undecided points
  // flagged, per-lane maxima of the keys' bounds per child
  unsigned m1 = 0, m2 = 0, und = 0;
  K lo0 = key_neg_inf<K>(), lo1 = key_neg_inf<K>(), hi0 = key_neg_inf<K>(), hi1 = key_neg_inf<K>();
  LineF l1 = {}, l2 = {};
  if (FAST) {
    l1 = line1_of(*G);
    l2 = line2_of(*G);
  }
  auto account = [&](int k, int c, K key, K err) {
    const K lo = key_lo(key, err), hi = key_hi(key, err);
    if (c == 3) und |= 1u << k;
    if (c == 1) { m1 |= 1u << k; lo0 = key_max(lo0, lo); hi0 = key_max(hi0, hi); }
    if (c == 2) { m2 |= 1u << k; lo1 = key_max(lo1, lo); hi1 = key_max(hi1, hi); }
  };
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const int l = k * kWarp + lane;
    if (l < count) {
      K key, err;
      const int c = classify_a(*G, l1, l2, X[l], Y[l], key, err);
      account(k, c, key, err);
    }
  }
  // the undecided points (rare, but most of them on hull-dense inputs): the
  // relative FP32 tier, then the exact tiers
  if (__any_sync(kFull, und != 0)) {
    for (unsigned u = und; u != 0; u &= u - 1) {
      const int k = __ffs(u) - 1;
      const int l = k * kWarp + lane;
      const double ux = X[l], uy = Y[l];
      K key, err;
      int c = classify_rel(*G, l1, l2, ux, uy, key, err);
      if (c == 3) {
        c = classify_exact(G, ux, uy);
        if (c == 1) line_key_tight(l1, &G->ax, ux, uy, key, err);
        if (c == 2) line_key_tight(l2, &G->rx, ux, uy, key, err);
      }
      if (c != 0) {
        const K lo = key_lo(key, err), hi = key_hi(key, err);
        if (c == 1) { m1 |= 1u << k; lo0 = key_max(lo0, lo); hi0 = key_max(hi0, hi); }
        else { m2 |= 1u << k; lo1 = key_max(lo1, lo); hi1 = key_max(hi1, hi); }
      }
    }
  }
  const int tot0 = __reduce_add_sync(kFull, __popc(m1)), tot1 = __reduce_add_sync(kFull, __popc(m2));
  // output offsets: one atomic per tile, its result first used after the
  // farthest-point search
  unsigned long long old = 0;
  if (lane == 0 && tot0 + tot1 > 0)
    old = atomicAdd(&ss->cursor, ((unsigned long long)tot0 << 32) | (unsigned long long)tot1);
  K1_MARK(c1);

  // farthest point per child.  The tile can only hold a point that beats
  // (or ties) the run's if its best upper bound reaches the run's lower
  // bound; most tiles stop at that test.  Otherwise the candidates are the
  // survivors whose upper bound reaches both the tile's best lower bound
  // and the run's (the tile's true farthest point is always among them),
  // compared exactly; the winner replaces the run's point if it beats it.
  const K L0 = warp_max_redux(lo0), L1 = warp_max_redux(lo1);
  const K H0 = warp_max_redux(hi0), H1 = warp_max_redux(hi1);
  K1_MARK(c1a);
  K1_ADD(prof, 8, c1a - c1);
#pragma unroll
  for (int ch = 0; ch < 2; ch++) {
    if ((ch ? tot1 : tot0) == 0) continue;
    K rlo, rhi;
    run_bounds(run, ch, rlo, rhi);
    const bool have = run.rb[ch].idx >= 0;
    if (have && (ch ? H1 : H0) < rlo) continue;
    K1_ADD(prof, 9, 1);
    const K Lc = ch ? L1 : L0;
    const K thr = have && rlo > Lc ? rlo : Lc;
    const unsigned mc = ch ? m2 : m1;
    const double* E = ch ? &G->rx : &G->ax;
    // the survivors' keys again, as tight as the FP32 tiers give them (any
    // valid bounds will do: the true farthest point's upper bound reaches
    // every lower bound): candidates reach the threshold
    unsigned cm = 0;
    for (unsigned u = mc; u != 0; u &= u - 1) {
      const int l = (__ffs(u) - 1) * kWarp + lane;
      K key, err;
      line_key_tight(ch ? l2 : l1, E, X[l], Y[l], key, err);
      if (key_hi(key, err) >= thr) cm |= 1u << (__ffs(u) - 1);
    }
    const unsigned lanes = __ballot_sync(kFull, cm != 0);
    if (lanes == 0) continue;
    K1_ADD(prof, 11, (unsigned long long)__reduce_add_sync(kFull, __popc(cm)));
    CandT<K> b = cand_none<K>();
    for (unsigned u = cm; u != 0; u &= u - 1) {
      const int l = (__ffs(u) - 1) * kWarp + lane;
      const double ux = X[l], uy = Y[l];
      K key, err;
      line_key_tight(ch ? l2 : l1, E, ux, uy, key, err);
      take_best(b, E, ux, uy, SRC_INPUT ? begin + l : I[l], key, err);
    }
    if (__popc(lanes) > 1) {
      b = warp_best(E, b);
      K1_ADD(prof, 10, 1);
    } else {
      b = shfl_cand(b, __ffs(lanes) - 1);
    }
    bool better = !have;
    if (have) {
      if (b.lo > rhi) better = true;
      else if (rlo > b.hi) better = false;
      else better = beats_exact(E[0], E[1], E[2], E[3], b.x, b.y, b.idx, run.rb[ch].x, run.rb[ch].y, run.rb[ch].idx);
    }
    if (better) {
      run_set(run, ch, b);
      if (lane == 0) atomicMax(&ss->lomax[ch], dkey(run.rb[ch].lo));  // result unused: a reduction
    }
  }

  // survivors: per step, one contiguous run per child
  K1_MARK(c2);
  K1_ADD(prof, 3, c2 - c1);
  old = __shfl_sync(kFull, old, 0);
  K1_MARK(c3);
  const long long eL = (long long)(old >> 32), eR = (long long)(old & 0xffffffffull);
  if (tot0 + tot1 > 0 && eL + tot0 <= slen && eR + tot1 <= slen) {
    const int dstb = par;
    double* __restrict__ dx = w.bx[dstb];
    double* __restrict__ dy = w.by[dstb];
    int* __restrict__ di = w.bi[dstb];
    const int baseL = soff + (int)eL;
    const int endR = soff + slen - (int)eR;
    const unsigned lt = lanemask_lt();
    int nl = 0, nr = 0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      const bool isL = (m1 >> k) & 1u, isR = (m2 >> k) & 1u;
      const unsigned bL = __ballot_sync(kFull, isL), bR = __ballot_sync(kFull, isR);
      if (isL || isR) {
        const int pos = isL ? baseL + nl + __popc(bL & lt) : endR - 1 - (nr + __popc(bR & lt));
        const int l = k * kWarp + lane;
        if (VQ_OK_IDX(w, 44, pos, soff, (long long)soff + slen)) {
          dx[pos] = X[l];
          dy[pos] = Y[l];
          di[pos] = SRC_INPUT ? begin + l : I[l];
        }
      }
      nl += __popc(bL);
      nr += __popc(bR);
    }
  }
  K1_MARK(c4);
  K1_ADD(prof, 2, c1 - c0);
  K1_ADD(prof, 4, c3 - c2);
  K1_ADD(prof, 5, c4 - c3);
}

template <int PPT, int WPB, int NS>
struct K1W {
  typedef K1Ring<PPT, NS> Ring;
  static constexpr int TW = 32 * PPT;
  static constexpr size_t smem = (size_t)WPB * sizeof(Ring);
  // blocks per SM that shared memory allows (227 KB usable, 1 KB reserved
  // per block), but never so many that a thread gets fewer than 112
  // registers: the register budget is sized for MINB blocks
  static constexpr int SMEMB = (int)((227u * 1024u) / (smem + 1024u));
  static constexpr int REGB = 65536 / (32 * WPB * 112);
  static constexpr int MINB = SMEMB < REGB ? (SMEMB > 0 ? SMEMB : 1) : REGB;
};

// Every warp takes a contiguous range of the level's tiles (consecutive
// tiles mostly share a segment, so the running farthest points rarely
// restart) and streams them through its ring.
// ALLFAST: every point set of the call is in the FP32 tier's range, so only
// that path is compiled in (a smaller kernel).
template <int PPT, int WPB, int NS, bool SRC_INPUT, bool ALLFAST>
__global__ void __launch_bounds__(32 * WPB, (K1W<PPT, WPB, NS>::MINB))
    k_k1w(const Work* __restrict__ wp, int level, int tier_dev) {
  const Work& w = *wp;
  typedef K1Ring<PPT, NS> Ring;
  extern __shared__ __align__(128) unsigned char k1w_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int par = level & 1;
  // warps are independent from here on: each may leave on its own
  if (fatal(w)) return;
  // launched beside its other instantiation: the device's tier flag picks one
  if (tier_dev && ALLFAST == (*reinterpret_cast<volatile int*>(&w.ctrl->any_slow) != 0)) return;
  Ring* R = reinterpret_cast<Ring*>(k1w_smem) + warp;
  const int ntiles = min(*reinterpret_cast<volatile int*>(&w.ctrl->k1_tiles[par]), w.capT);
  const long long gw = (long long)blockIdx.x * WPB + warp, nw = (long long)gridDim.x * WPB;
  const int t_begin = (int)((long long)ntiles * gw / nw), t_end = (int)((long long)ntiles * (gw + 1) / nw);
  const TileDesc* desc = w.tdesc[par];
  if (gw == 0 && lane == 0) w.ctrl->k1_nw[par] = nw;  // the finalize kernel retraces the tile split
  if (lane == 0) {
    for (int s = 0; s < NS; s++) mbar_init(&R->full[s], 1);
    mbar_fence_init();
  }
  __syncwarp();
  // prologue: the first NS tiles, and the descriptor of the one after
  int t_issue = t_begin;
  TileDesc nd;
  nd.sid = nd.begin = nd.count = nd.flags = nd.off = nd.len = nd.pad0 = nd.pad1 = 0;
  if (lane == 0) {
    for (int s = 0; s < NS && t_issue < t_end; s++, t_issue++)
      k1_issue<PPT, NS, SRC_INPUT>(w, par, R, s, t_issue, load_desc(desc + t_issue));
    if (t_issue < t_end) nd = load_desc(desc + t_issue);
  }
  t_issue = __shfl_sync(kFull, t_issue, 0);
  unsigned long long prof[12] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
  K1Run run;
  run.sid = -1;
  run.t_last = 0;
  run.rb[0] = cand_none<double>();
  run.rb[1] = cand_none<double>();
  run.lf[0] = run.lf[1] = run.hf[0] = run.hf[1] = 0.0f;
  K1_MARK(k_start);
  int it = 0;
  for (int t = t_begin; t < t_end; t++, it++) {
    const int s = it % NS;
    K1_MARK(w0);
    const bool arrived = mbar_wait(&R->full[s], (unsigned)((it / NS) & 1), w.timeout_ns);
    K1_MARK(w1);
    K1_ADD(prof, 0, 1);
    K1_ADD(prof, 1, w1 - w0);
    if (!arrived) {
      if (lane == 0) {
        atomicOr(&w.ctrl->err, kErrTimeout);
        // let this warp's other copies in flight land before leaving
        for (int q = it + 1; q < it + NS && t_begin + q < t_end; q++)
          mbar_wait(&R->full[q % NS], (unsigned)((q / NS) & 1), 10000000ll);
      }
      __syncwarp();
      return;
    }
    K1Stage<32 * PPT>* sg = &R->st[s];
    if (ALLFAST || (sg->m.flags & kSegFast))
      k1w_tile<PPT, SRC_INPUT, true>(w, par, sg, lane, run, prof);
    else
      k1w_tile<PPT, SRC_INPUT, ALLFAST>(w, par, sg, lane, run, prof);
    __syncwarp();
    K1_MARK(i0);
    if (lane == 0 && t_issue < t_end) {
      fence_proxy_async_smem();  // this warp's reads of the stage before the copy that reuses it
      k1_issue<PPT, NS, SRC_INPUT>(w, par, R, s, t_issue, nd);
      if (t_issue + 1 < t_end) nd = load_desc(desc + t_issue + 1);
    }
    K1_MARK(i1);
    K1_ADD(prof, 6, i1 - i0);
    t_issue++;
  }
  k1w_flush(w, par, run, lane);
#ifdef VQ_K1_PROFILE
  K1_MARK(k_end);
  prof[7] = k_end - k_start;
  if (lane == 0)
    for (int i = 0; i < 12; i++) atomicAdd(&w.ctrl->k1prof[i], prof[i]);
#endif
}
