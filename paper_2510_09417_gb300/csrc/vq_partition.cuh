// vq_partition.cuh -- streaming partition kernel (level k >= 0 of Alg. 1's
// subset extraction, all live big segments at once).  Included by
// vq_kernels.cu after the shared helpers; not a standalone header.
//
// For every point u of every live segment (a, b, r) the kernel decides
// left of a->r (left child, S1), left of r->b (right child, S2) or neither
// (Alg. 1, the two partition steps after r is found), writes the survivors
// into the segment's range of the other ping-pong buffer (left child from
// the start, right child from the end) and finds, per tile and child, the
// point farthest from the child's line (the next level's r).
//
// Structure (one CTA per SM slot, persistent over the level's tiles):
//   * a producer warp streams tiles into a ring of NS shared-memory stages
//     with 1-D bulk copies (cp.async.bulk, completion on an mbarrier): the
//     16-byte-aligned middle of each array in one copy, the ragged ends
//     with plain loads, so no byte outside the tile's range is read;
//   * NC consumer warps classify their 32*PPT points per tile from shared
//     memory (FP32 filter tier, exact tiers for undecided points), combine
//     counts at one named barrier, take the tile's output offsets with one
//     64-bit atomic on the segment cursor, resolve the tile's farthest
//     point per child among the few points whose upper bound reaches the
//     tile's best lower bound, and store the survivors directly (per warp
//     and step, one contiguous run per child);
//   * every wait (stage full, stage empty) is bounded by w.timeout_ns; a
//     consumer that gives up raises kErrTimeout and the CTA leaves together
//     after the next barrier.
#pragma once

// (included inside namespace vq)

// ---- mbarrier / bulk-copy primitives (PTX ISA: mbarrier, cp.async.bulk) ----

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
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
// Wait for the phase of parity `parity` to complete; false after timeout_ns
// or (abort != null) once *abort is set.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, long long timeout_ns,
                                          const volatile int* abort = nullptr) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(b, parity)) return true;
    if (abort && *abort) return false;
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
__device__ __forceinline__ void bar_consumers(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
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
  int sx, sy, si, flags;     // shared-memory slot shift per array; segment flags
  int off, len, pad0, pad1;  // segment range
};

// One stage: the segment's geometry (bulk-copied), the tile's metadata and
// its points.  Point l of the tile is x[l + sx], y[l + sy], i[l + si]; the
// shifts put each array's bulk part on a 16-byte boundary.
template <int TB>
struct alignas(16) K1Stage {
  SegGeom g;
  K1Meta m;
  double x[TB + 2];
  double y[TB + 2];
  int i[TB + 4];
};
static_assert(sizeof(SegGeom) == 96, "SegGeom is bulk-copied as 96 bytes");

template <int NC>
struct K1Sync {
  unsigned long long full[4];
  unsigned long long empty[4];
  int cnt[2][NC];
  float lof[2][NC];
  double lod[2][NC];
  CandT<double> slot[2][NC];
  int excl[2];
  int err;    // a consumer's stage wait timed out
  int abort;  // consumers stopped: the producer stops issuing
  int ntiles;
  int fatal;
};

template <int NC>
__device__ __forceinline__ void put_lo(K1Sync<NC>& sh, int ch, int q, float v) { sh.lof[ch][q] = v; }
template <int NC>
__device__ __forceinline__ void put_lo(K1Sync<NC>& sh, int ch, int q, double v) { sh.lod[ch][q] = v; }
template <int NC>
__device__ __forceinline__ void get_lo(const K1Sync<NC>& sh, int ch, int q, float& v) { v = sh.lof[ch][q]; }
template <int NC>
__device__ __forceinline__ void get_lo(const K1Sync<NC>& sh, int ch, int q, double& v) { v = sh.lod[ch][q]; }

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

// Element range of one array for the producer: `sh` = slot shift, `h`
// head elements (plain), `nb` bulk elements from h (16-byte aligned at
// both ends), the rest tail (plain).
struct K1Range {
  int sh, h, nb;
};
template <int ES>
__device__ __forceinline__ K1Range k1_range(const void* p, int count) {
  const unsigned mis = (unsigned)(reinterpret_cast<uintptr_t>(p) & 15u);
  K1Range r;
  r.sh = (int)(mis / ES);
  const int h = mis ? (int)((16u - mis) / ES) : 0;
  r.h = h < count ? h : count;
  r.nb = (((count - r.h) * ES) / 16) * 16 / ES;
  return r;
}
template <typename T>
__device__ __forceinline__ void k1_plain_ends(T* dst, const T* src, int count, const K1Range& r) {
  for (int e = 0; e < r.h; e++) dst[r.sh + e] = src[e];
  for (int e = r.h + r.nb; e < count; e++) dst[r.sh + e] = src[e];
}

// ---- producer ----

template <int PPT, int NC, int NS, bool SRC_INPUT>
__device__ __forceinline__ void k1s_produce(const Work& w, int level, K1Sync<NC>& sh, unsigned char* stages,
                                            int ntiles) {
  constexpr int TB = 32 * NC * PPT;
  typedef K1Stage<TB> Stage;
  const int par = level & 1, srcb = (level + 1) & 1;
  const volatile int* abort = &sh.abort;
  int it = 0;
  bool ok = true;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
    const int s = it % NS;
    if (it >= NS && !mbar_wait(&sh.empty[s], (unsigned)((it / NS - 1) & 1), w.timeout_ns, abort)) {
      ok = false;
      break;
    }
    Stage* sg = reinterpret_cast<Stage*>(stages + (size_t)s * sizeof(Stage));
    const int sid = __ldg(&w.tile_seg[par][t]);
    int begin = 0, count = 0, off = 0, len = 0, flags = 0;
    bool good = VQ_OK_IDX(w, 40, sid, 0, w.capS);
    if (good) {
      const SegRec S = w.segs[par][sid];
      const int j = t - S.tile_base;
      begin = S.off + j * TB;
      count = min(TB, S.len - j * TB);
      off = S.off;
      len = S.len;
      flags = S.flags;
      good = VQ_OK_IDX(w, 41, count, 1, TB + 1) && VQ_OK_IDX(w, 42, begin, 0, w.N) &&
             VQ_OK_IDX(w, 43, (long long)begin + count, 1, (long long)w.N + 1);
    }
    if (!good) count = 0;
    const double* px = (SRC_INPUT ? w.x : w.bx[srcb]) + begin;
    const double* py = (SRC_INPUT ? w.y : w.by[srcb]) + begin;
    const int* pi = w.bi[srcb] + begin;
    const K1Range rx = k1_range<8>(px, count), ry = k1_range<8>(py, count);
    K1Range ri;
    ri.sh = 0; ri.h = 0; ri.nb = 0;
    if (!SRC_INPUT) ri = k1_range<4>(pi, count);
    k1_plain_ends(sg->x, px, count, rx);
    k1_plain_ends(sg->y, py, count, ry);
    if (!SRC_INPUT) k1_plain_ends(sg->i, pi, count, ri);
    K1Meta m;
    m.t = t; m.sid = good ? sid : 0; m.begin = begin; m.count = count;
    m.sx = rx.sh; m.sy = ry.sh; m.si = ri.sh; m.flags = flags;
    m.off = off; m.len = len; m.pad0 = 0; m.pad1 = 0;
    sg->m = m;
    const unsigned gb = good ? (unsigned)sizeof(SegGeom) : 0u;
    const unsigned tx = gb + (unsigned)(rx.nb + ry.nb) * 8u + (unsigned)ri.nb * 4u;
    mbar_arrive_expect_tx(&sh.full[s], tx);
    if (gb) bulk_g2s(&sg->g, &w.geom[par][sid], gb, &sh.full[s]);
    if (rx.nb) bulk_g2s(sg->x + rx.sh + rx.h, px + rx.h, (unsigned)rx.nb * 8u, &sh.full[s]);
    if (ry.nb) bulk_g2s(sg->y + ry.sh + ry.h, py + ry.h, (unsigned)ry.nb * 8u, &sh.full[s]);
    if (!SRC_INPUT && ri.nb) bulk_g2s(sg->i + ri.sh + ri.h, pi + ri.h, (unsigned)ri.nb * 4u, &sh.full[s]);
  }
  if (!ok) {
    atomicOr(&w.ctrl->err, kErrTimeout);
    // let the copies already issued land before the CTA can exit
    const int first = it > NS ? it - NS : 0;
    for (int q = first; q < it; q++) mbar_wait(&sh.full[q % NS], (unsigned)((q / NS) & 1), 10000000ll);
  }
}

// ---- consumers: one tile ----

template <int PPT, int NC, bool SRC_INPUT, bool FAST>
__device__ __forceinline__ bool k1s_tile(const Work& w, int par, K1Stage<32 * NC * PPT>* __restrict__ sg,
                                         K1Sync<NC>& sh, unsigned char* hi_raw, int cw, int lane, int tid,
                                         unsigned long long* empty_bar) {
  typedef typename KeyOf<FAST>::T K;
  constexpr int TW = 32 * PPT, NT = 32 * NC, TB = NC * TW;
  const int t = sg->m.t, sid = sg->m.sid, begin = sg->m.begin;
  const int count = min(max(sg->m.count, 0), TB);
  const int soff = sg->m.off, slen = sg->m.len;
  const double* X = sg->x + (sg->m.sx & 1);
  const double* Y = sg->y + (sg->m.sy & 1);
  const int* I = sg->i + (sg->m.si & 3);
  const SegGeom* G = &sg->g;
  K* hs = reinterpret_cast<K*>(hi_raw);
  const int wb = cw * TW;
  const int wcount = min(max(count - wb, 0), TW);

  // pass A: filter tier for every point; upper bounds of survivors' keys
  // go to shared memory (hs[k][tid]), undecided points are flagged
  unsigned m1 = 0, m2 = 0, und = 0;
  K lo0 = key_neg_inf<K>(), lo1 = key_neg_inf<K>();
  LineF l1 = {}, l2 = {};
  if (FAST) {
    l1 = line1_of(*G);
    l2 = line2_of(*G);
  }
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const int l = k * kWarp + lane;
    K h = key_neg_inf<K>();
    if (l < wcount) {
      K key, err;
      const int c = classify_a(*G, l1, l2, X[wb + l], Y[wb + l], key, err);
      const K lo = key_lo(key, err), hi = key_hi(key, err);
      if (c == 3) und |= 1u << k;
      if (c == 1) { m1 |= 1u << k; lo0 = key_max(lo0, lo); h = hi; }
      if (c == 2) { m2 |= 1u << k; lo1 = key_max(lo1, lo); h = hi; }
    }
    hs[k * NT + tid] = h;
  }
  // exact tiers for the undecided points (rare)
  if (__any_sync(kFull, und != 0)) {
    for (unsigned u = und; u != 0; u &= u - 1) {
      const int k = __ffs(u) - 1;
      const int l = wb + k * kWarp + lane;
      const double ux = X[l], uy = Y[l];
      const int c = classify_exact(G, ux, uy);
      if (c != 0) {
        K key, err;
        if (c == 1) line_key_k(l1, &G->ax, ux, uy, key, err);
        else line_key_k(l2, &G->rx, ux, uy, key, err);
        const K lo = key_lo(key, err);
        if (c == 1) { m1 |= 1u << k; lo0 = key_max(lo0, lo); }
        else { m2 |= 1u << k; lo1 = key_max(lo1, lo); }
        hs[k * NT + tid] = key_hi(key, err);
      }
    }
  }
  {
    const int c0 = __reduce_add_sync(kFull, __popc(m1)), c1 = __reduce_add_sync(kFull, __popc(m2));
    const K wl0 = warp_max_redux(lo0), wl1 = warp_max_redux(lo1);
    if (lane == 0) {
      sh.cnt[0][cw] = c0;
      sh.cnt[1][cw] = c1;
      put_lo(sh, 0, cw, wl0);
      put_lo(sh, 1, cw, wl1);
    }
  }
  bar_consumers(NT);
  if (*reinterpret_cast<volatile int*>(&sh.err)) return false;

  // block totals, this warp's prefix, the tile's best lower bounds
  int pre0 = 0, pre1 = 0, tot0 = 0, tot1 = 0;
  K L0 = key_neg_inf<K>(), L1 = key_neg_inf<K>();
#pragma unroll
  for (int q = 0; q < NC; q++) {
    const int a = sh.cnt[0][q], b = sh.cnt[1][q];
    if (q < cw) { pre0 += a; pre1 += b; }
    tot0 += a;
    tot1 += b;
    K v0, v1;
    get_lo(sh, 0, q, v0);
    get_lo(sh, 1, q, v1);
    L0 = key_max(L0, v0);
    L1 = key_max(L1, v1);
  }
  SegState* ss = &w.sstate[par][sid];
  unsigned long long old = 0, thr0 = 0, thr1 = 0;
  if (tid == 0) {
    // output offsets (the result is first needed after the candidate pass)
    if (tot0 + tot1 > 0) old = atomicAdd(&ss->cursor, ((unsigned long long)tot0 << 32) | (unsigned long long)tot1);
    thr0 = __ldcg(&ss->lomax[0]);
    thr1 = __ldcg(&ss->lomax[1]);
  }

  // candidates: survivors whose upper bound reaches the tile's best lower
  // bound; the true farthest point of the tile is always one of them
  unsigned cm1 = 0, cm2 = 0;
#pragma unroll
  for (int k = 0; k < PPT; k++) {
    const K h = hs[k * NT + tid];
    if (((m1 >> k) & 1u) && h >= L0) cm1 |= 1u << k;
    if (((m2 >> k) & 1u) && h >= L1) cm2 |= 1u << k;
  }
#pragma unroll
  for (int ch = 0; ch < 2; ch++) {
    const unsigned cm = ch ? cm2 : cm1;
    const double* E = ch ? &G->rx : &G->ax;
    const unsigned lanes = __ballot_sync(kFull, cm != 0);
    if (lanes == 0) {
      if (lane == 0) sh.slot[ch][cw].idx = -1;
      continue;
    }
    CandT<K> b = cand_none<K>();
    for (unsigned u = cm; u != 0; u &= u - 1) {
      const int l = wb + (__ffs(u) - 1) * kWarp + lane;
      const double ux = X[l], uy = Y[l];
      K key, err;
      line_key_k(ch ? l2 : l1, E, ux, uy, key, err);
      take_best(b, E, ux, uy, SRC_INPUT ? begin + l : I[l], key, err);
    }
    if (__popc(lanes) == 1) {
      if (cm != 0) sh.slot[ch][cw] = to_double(b);
    } else {
      b = warp_best(E, b);
      if (lane == 0) sh.slot[ch][cw] = to_double(b);
    }
  }
  if (tid == 0) {
    const long long eL = (long long)(old >> 32), eR = (long long)(old & 0xffffffffull);
    const bool fits = eL + tot0 <= slen && eR + tot1 <= slen;
    sh.excl[0] = fits ? (int)eL : -1;
    sh.excl[1] = fits ? (int)eR : -1;
  }
  bar_consumers(NT);
  const int eL = sh.excl[0], eR = sh.excl[1];

  // thread 0: the tile's farthest point per child; its record, the
  // segment's largest lower bound (atomic max, issued now, result used
  // after the stores)
  unsigned long long pv[2] = {0ull, 0ull}, klo[2] = {0ull, 0ull}, khi[2] = {0ull, 0ull};
  bool has[2] = {false, false};
  if (tid == 0) {
    TileRec* rec = &w.cand[par][t];
#pragma unroll
    for (int ch = 0; ch < 2; ch++) {
      const double* E = ch ? &G->rx : &G->ax;
      CandT<double> best = cand_none<double>();
#pragma unroll
      for (int q = 0; q < NC; q++) {
        const CandT<double> c = sh.slot[ch][q];
        if (cand_beats(E, c, best)) best = c;
      }
      rec->own[ch] = to_rec(best);
      if (best.idx >= 0) {
        has[ch] = true;
        klo[ch] = dkey(best.lo);
        khi[ch] = dkey(best.hi);
        const unsigned long long th = ch ? thr1 : thr0;
        pv[ch] = klo[ch] > th ? atomicMax(&ss->lomax[ch], klo[ch]) : th;
      }
    }
  }

  // survivors: per step, one contiguous run per child and warp
  if (eL >= 0) {
    const int dstb = par;
    double* __restrict__ dx = w.bx[dstb];
    double* __restrict__ dy = w.by[dstb];
    int* __restrict__ di = w.bi[dstb];
    const int baseL = soff + eL + pre0;
    const int endR = soff + slen - eR - pre1;
    const unsigned lt = lanemask_lt();
    int nl = 0, nr = 0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
      const bool isL = (m1 >> k) & 1u, isR = (m2 >> k) & 1u;
      const unsigned bL = __ballot_sync(kFull, isL), bR = __ballot_sync(kFull, isR);
      if (isL || isR) {
        const int pos = isL ? baseL + nl + __popc(bL & lt) : endR - 1 - (nr + __popc(bR & lt));
        const int l = wb + k * kWarp + lane;
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
  __syncwarp();
  if (lane == 0) mbar_arrive(empty_bar);

  // thread 0: list the tile as a farthest-point candidate of a child when
  // its upper bound reaches the largest lower bound seen so far
  if (tid == 0) {
#pragma unroll
    for (int ch = 0; ch < 2; ch++) {
      if (!has[ch]) continue;
      const unsigned long long thr = pv[ch] > klo[ch] ? pv[ch] : klo[ch];
      if (khi[ch] >= thr) {
        const int i = atomicAdd(&ss->ncand[ch], 1);
        if (i < kMaxCand) ss->cand[ch][i] = t;
      }
    }
  }
  return true;
}

template <int PPT, int NC, int NS>
struct K1S {
  static constexpr int TB = 32 * NC * PPT;
  static constexpr int NT = 32 * NC;
  static constexpr size_t stage_bytes = sizeof(K1Stage<TB>);
  static constexpr size_t smem = NS * stage_bytes + (size_t)PPT * NT * sizeof(double);
};

template <int PPT, int NC, int NS, bool SRC_INPUT>
__global__ void __launch_bounds__(32 * NC + 32, NS) k_k1s(Work w, int level) {
  typedef K1S<PPT, NC, NS> C;
  static_assert(NS <= 4, "at most 4 stages");
  extern __shared__ __align__(128) unsigned char k1s_smem[];
  __shared__ K1Sync<NC> sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int par = level & 1;
  if (tid == 0) {
    sh.fatal = fatal(w) ? 1 : 0;
    sh.ntiles = min(*reinterpret_cast<volatile int*>(&w.ctrl->k1_tiles[par]), w.capT);
    sh.err = 0;
    sh.abort = 0;
    for (int s = 0; s < NS; s++) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], NC);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (sh.fatal) return;
  const int ntiles = sh.ntiles;
  unsigned char* stages = k1s_smem;
  unsigned char* hi_raw = k1s_smem + NS * C::stage_bytes;
  if (warp == NC) {
    if (lane == 0) k1s_produce<PPT, NC, NS, SRC_INPUT>(w, level, sh, stages, ntiles);
    return;
  }
  typedef K1Stage<C::TB> Stage;
  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
    const int s = it % NS;
    if (!mbar_wait(&sh.full[s], (unsigned)((it / NS) & 1), w.timeout_ns)) {
      *reinterpret_cast<volatile int*>(&sh.err) = 1;
      atomicOr(&w.ctrl->err, kErrTimeout);
    }
    Stage* sg = reinterpret_cast<Stage*>(stages + (size_t)s * C::stage_bytes);
    bool ok;
    if (sg->m.flags & kSegFast)
      ok = k1s_tile<PPT, NC, SRC_INPUT, true>(w, par, sg, sh, hi_raw, warp, lane, tid, &sh.empty[s]);
    else
      ok = k1s_tile<PPT, NC, SRC_INPUT, false>(w, par, sg, sh, hi_raw, warp, lane, tid, &sh.empty[s]);
    if (!ok) {
      *reinterpret_cast<volatile int*>(&sh.abort) = 1;
      return;
    }
  }
}
