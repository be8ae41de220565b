// vq_sieve.cuh -- the level-0 pre-filter path (the Akl-Toussaint heuristic
// the paper proposes as its next step, Sec. 6) fused with the extreme-point
// pass of Alg. 1:
//   k_sample  extremes of the points in kPolyDirs directions, over a sample
//             of each set (approximate scores: any choice is safe);
//   k_poly    per set, two x-monotone chains of those input points and an
//             inner box whose corners are certainly inside (see PolyF);
//   k_sieve   streams every point once into registers, drops the points
//             certainly inside an inner box or the chains' region, writes the rest
//             with their indices to buffer 1 (from the set's offset, where
//             level 0 reads them), and takes the lexicographic extremes and
//             the range flags of the points it keeps.
// p and q are strict vertices, so they are never dropped: the extremes of
// the kept points are the set's.  A dropped point is finite and in the FP32
// tier's range (the tests reject everything else), so the flags of the kept
// points are the set's as well.
// Included by vq_kernels.cu inside namespace vq after the extreme-pass
// helpers (LexPt, k0_take); not a standalone header.
#pragma once

// ---- sampled directions ----------------------------------------------------
// Direction k is the integer pair (kDirA[k], kDirB[k]): the first quadrant's
// (1,0), (4,1), (2,1), (4,3), (1,1), (3,4), (1,2), (1,4), turned by k / 8
// quarter turns, so the angle grows with k.  Directions 1..15 point up (the
// upper chain's candidates), 17..31 down (the lower chain's); 4, 12, 20 and
// 28 are the diagonals that bound the inner box.
__device__ constexpr int kDirA[kPolyDirs] = {1, 4, 2, 4, 1, 3, 1, 1, 0, -1, -1, -3, -1, -4, -2, -4,
                                             -1, -4, -2, -4, -1, -3, -1, -1, 0, 1, 1, 3, 1, 4, 2, 4};
__device__ constexpr int kDirB[kPolyDirs] = {0, 1, 1, 3, 1, 4, 2, 4, 1, 4, 2, 4, 1, 3, 1, 1,
                                             0, -1, -1, -3, -1, -4, -2, -4, -1, -4, -2, -4, -1, -3, -1, -1};

// (score, index) packed so that the unsigned maximum is the largest score,
// then the lowest index; 0 means no point.
__device__ __forceinline__ unsigned long long pack_score(float s, int idx) {
  unsigned u = __float_as_uint(s);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)u << 32) | (unsigned long long)(0xffffffffu - (unsigned)idx);
}
__device__ __forceinline__ int unpack_index(unsigned long long k) {
  return k == 0ull ? -1 : (int)(0xffffffffu - (unsigned)(k & 0xffffffffull));
}

// Sampled extremes: the first kSampleChunk points of every extreme-pass
// tile whose global number is a multiple of kSampleEvery, and of every
// set's first tile, are scored in every direction on their FP32-truncated
// coordinates; per set and direction the best (score, lowest index) is kept
// by a 64-bit atomic maximum.  A block takes kSampleBlockPts of a sampled
// chunk (a unit), eight points per thread, loaded before any is scored;
// per direction each thread keeps its best and the warps reduce them.
// Scores of non-finite or huge coordinates are meaningless; k_poly rejects
// such candidates.
constexpr int kSampleBlockPts = 2048;
constexpr int kSamplePPT = kSampleBlockPts / 256;
constexpr int kSampleParts = kSampleChunk / kSampleBlockPts;
__global__ void __launch_bounds__(256) k_sample(Work w) {
  __shared__ unsigned long long s_best[256 / kWarp][kPolyDirs];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int T = w.k0_tile_start[w.nsets];
  const long long u1 = (long long)((T + kSampleEvery - 1) / kSampleEvery) * kSampleParts;
  const long long units = u1 + (long long)w.nsets * kSampleParts;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    int t, lo, part;
    if (u < u1) {  // tile kSampleEvery * (u / parts): find its set
      t = (int)(u / kSampleParts) * kSampleEvery;
      part = (int)(u % kSampleParts);
      lo = 0;
      int hi = w.nsets - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (w.k0_tile_start[mid] <= t) lo = mid; else hi = mid - 1;
      }
    } else {  // the first tile of set lo, unless already sampled
      lo = (int)((u - u1) / kSampleParts);
      part = (int)((u - u1) % kSampleParts);
      t = w.k0_tile_start[lo];
      if (t % kSampleEvery == 0 || t >= w.k0_tile_start[lo + 1]) continue;
    }
    const int j = t - w.k0_tile_start[lo];
    const SetRec S = w.sets[lo];
    const int first = j * kK0Tile + part * kSampleBlockPts;
    const int count = min(kSampleBlockPts, S.len - first);
    if (count <= 0) continue;
    const int begin = S.off + first;
    double vx[kSamplePPT], vy[kSamplePPT];
#pragma unroll
    for (int q = 0; q < kSamplePPT; q++) {
      const int l = q * 256 + (int)threadIdx.x;
      vx[q] = l < count ? px(w, begin + l) : 0.0;
      vy[q] = l < count ? py(w, begin + l) : 0.0;
    }
    float fx[kSamplePPT], fy[kSamplePPT];
#pragma unroll
    for (int q = 0; q < kSamplePPT; q++) {
      fx[q] = trunc_f32(vx[q]);
      fy[q] = trunc_f32(vy[q]);
    }
    // directions k and k + 16 are opposite: one score, its maximum and minimum
#pragma unroll
    for (int k = 0; k < kPolyDirs / 2; k++) {
      // this thread's points come in increasing index order: a strict
      // compare keeps the lowest index among its ties
      float bmax = -INFINITY, bmin = INFINITY;
      int imax = -1, imin = -1;
#pragma unroll
      for (int q = 0; q < kSamplePPT; q++) {
        const int l = q * 256 + (int)threadIdx.x;
        const float sc = __fmaf_rn((float)kDirA[k], fx[q], __fmul_rn((float)kDirB[k], fy[q]));
        if (l < count && sc > bmax) {
          bmax = sc;
          imax = begin + l;
        }
        if (l < count && sc < bmin) {
          bmin = sc;
          imin = begin + l;
        }
      }
      // opposite direction: the score negated exactly
      unsigned long long v = imax >= 0 ? pack_score(bmax, imax) : 0ull;
      unsigned long long u = imin >= 0 ? pack_score(-bmin, imin) : 0ull;
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, v, m), p = __shfl_xor_sync(kFull, u, m);
        v = o > v ? o : v;
        u = p > u ? p : u;
      }
      if (lane == 0) {
        s_best[warp][k] = v;
        s_best[warp][k + kPolyDirs / 2] = u;
      }
    }
    __syncthreads();
    if (threadIdx.x < kPolyDirs) {
      unsigned long long v = 0ull;
      for (int q = 0; q < 256 / kWarp; q++) v = s_best[q][threadIdx.x] > v ? s_best[q][threadIdx.x] : v;
      if (v) atomicMax(&w.dirbest[(long long)lo * kPolyDirs + threadIdx.x], v);
    }
    __syncthreads();  // s_best is rewritten by the next unit
  }
}

// ---- chains per set ------------------------------------------------------

// Per-warp scratch of k_poly.
struct PolyScratch {
  double x[kPolyDirs], y[kPolyDirs];
  float fx[kPolyDirs], fy[kPolyDirs];  // trunc_f32 of the candidates (approximate turn tests)
  int idx[kPolyDirs];                  // candidate point (global index) or -1
  int cu[kChainEdges + 1], cl[kChainEdges + 1];  // chain vertices as candidate slots, L first, R last
  int nu, nl;
  float bb[kPolyBoxes];  // inner-box search: largest passing scale per box
  PolyF P;
};

// Inner boxes: box b has half sizes s (kBoxFx[b] hx, kBoxFy[b] hy) around
// the centre, i.e. corners at angle t_b from the axes on an ellipse of
// half axes sqrt(2) (hx, hy): t_b = 45, 22.5, 67.5, 33.75, 56.25 degrees,
// (sqrt(2) cos t_b, sqrt(2) sin t_b).  On a disk the union of the five
// covers about 90 % of the area (the first three 85 %, the first one 64 %).
__device__ __forceinline__ float box_fx(int b) {
  return b == 0 ? 1.0f : (b == 1 ? 1.3066f : (b == 2 ? 0.5412f : (b == 3 ? 1.1759f : 0.7857f)));
}
__device__ __forceinline__ float box_fy(int b) {
  return b == 0 ? 1.0f : (b == 1 ? 0.5412f : (b == 2 ? 1.3066f : (b == 3 ? 0.7857f : 1.1759f)));
}

// Approximate orientation of three candidates (FP32 on truncated
// coordinates): only used to choose chain vertices, which needs no
// exactness (see PolyF).
__device__ __forceinline__ float turn_f32(const PolyScratch& S, int a, int b, int c) {
  const float ux = S.fx[b] - S.fx[a], uy = S.fy[b] - S.fy[a];
  const float vx = S.fx[c] - S.fx[a], vy = S.fy[c] - S.fy[a];
  return ux * vy - uy * vx;
}

// Both chains at once.  The upper chain's candidates are the slots of
// directions 1..15, the lower chain's those of 17..31, each taken if it
// lies strictly between L and R in x.  Every lane of a group ranks its
// candidate by (x, then y downward for the upper chain and upward for the
// lower one, then index) against the others of its group; of candidates
// with equal x only the first is kept.  Lanes 0 and 16 then walk their
// chain from L to R like one half of Andrew's monotone chain, popping a
// vertex that would not turn the right way (approximately: FP32 on the
// truncated coordinates, which needs no exactness, see PolyF).  Leaves
// S.cu / S.nu and S.cl / S.nl (vertex slots, L first, R last).
__device__ void build_chains(PolyScratch& S, int L, int R, int lane) {
  const long long xl = order_key(S.x[L]), xr = order_key(S.x[R]);
  const int idx = S.idx[lane];
  const long long kx = order_key(S.x[lane]), ky = order_key(S.y[lane]);
  const int grp = lane >= 1 && lane < kPolyDirs / 2 ? 0 : (lane > kPolyDirs / 2 ? 1 : -1);
  const bool mem = grp >= 0 && idx >= 0 && kx > xl && kx < xr;
  const int g = mem ? grp : -1;
  // lane j before me in my group's order: a strict total order over the
  // lanes (a point that is the candidate of several directions is ordered
  // by lane), so the ranks below are distinct
  auto before = [&](long long jx, long long jy, int ji, int j) {
    if (jx != kx) return jx < kx;
    if (jy != ky) return grp == 0 ? jy > ky : jy < ky;
    if (ji != idx) return ji < idx;
    return j < lane;
  };
  bool drop = false;
  for (int j = 0; j < kWarp; j++) {
    const long long jx = __shfl_sync(kFull, kx, j), jy = __shfl_sync(kFull, ky, j);
    const int ji = __shfl_sync(kFull, idx, j), jg = __shfl_sync(kFull, g, j);
    if (mem && j != lane && jg == g && jx == kx && before(jx, jy, ji, j)) drop = true;
  }
  const bool keep = mem && !drop;
  int rank = 0;
  for (int j = 0; j < kWarp; j++) {
    const long long jx = __shfl_sync(kFull, kx, j), jy = __shfl_sync(kFull, ky, j);
    const int ji = __shfl_sync(kFull, idx, j), jg = __shfl_sync(kFull, keep ? g : -1, j);
    if (keep && j != lane && jg == g && before(jx, jy, ji, j)) rank++;
  }
  const unsigned ku = __ballot_sync(kFull, keep && g == 0), kl = __ballot_sync(kFull, keep && g == 1);
  const int nu = __popc(ku), nl = __popc(kl);
  int* tmpu = S.cu;  // sorted candidates at 1 .. n, L at 0 and R at n + 1
  int* tmpl = S.cl;
  if (keep) (g == 0 ? tmpu : tmpl)[1 + rank] = lane;
  if (lane == 0) { tmpu[0] = L; tmpu[nu + 1] = R; }
  if (lane == 16) { tmpl[0] = L; tmpl[nl + 1] = R; }
  __syncwarp();
  if (lane == 0 || lane == 16) {
    // in place: vertex m is written only after position m has been read
    int* C = lane == 0 ? tmpu : tmpl;
    const int n = (lane == 0 ? nu : nl) + 2;
    int m = 1;
    for (int i = 1; i < n; i++) {
      const int c = C[i];
      while (m >= 2) {
        const float t = turn_f32(S, C[m - 2], C[m - 1], c);
        if (lane == 0 ? t < 0.0f : t > 0.0f) break;
        m--;
      }
      C[m++] = c;
    }
    if (lane == 0) S.nu = m; else S.nl = m;
  }
  __syncwarp();
}

// One warp per set: candidates from k_sample, the two chains, their FP32
// tier edges (make_line on the exact endpoints) and thresholds, and the
// inner box.  A set whose candidates are out of the FP32 tier's range (or
// non-finite), or too few, gets no chains (the sieve then keeps all its
// points).
__global__ void __launch_bounds__(128) k_poly(Work w) {
  __shared__ PolyScratch sh[4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  PolyScratch& S = sh[warp];
  for (int s = blockIdx.x * 4 + warp; s < w.nsets; s += gridDim.x * 4) {
    const SetRec R = w.sets[s];
    int idx = unpack_index(w.dirbest[(long long)s * kPolyDirs + lane]);
    if (idx < R.off || idx >= R.off + R.len) idx = -1;
    double x = 0.0, y = 0.0;
    bool ok = true;
    if (idx >= 0) {
      x = px(w, idx);
      y = py(w, idx);
      const unsigned ax = static_cast<unsigned>(__double2hiint(x)) & 0x7fffffffu;
      const unsigned ay = static_cast<unsigned>(__double2hiint(y)) & 0x7fffffffu;
      ok = max(ax, ay) < 0x42700000u;  // |coordinate| < 2^40, finite
    }
    S.idx[lane] = idx;
    S.x[lane] = x;
    S.y[lane] = y;
    S.fx[lane] = trunc_f32(x);
    S.fy[lane] = trunc_f32(y);
    // L and R: the lexicographic extremes of the candidates (exact keys)
    LexPt mn{LLONG_MAX, LLONG_MAX, INT_MAX}, mx{LLONG_MIN, LLONG_MIN, INT_MAX};
    if (idx >= 0) {
      mn = LexPt{order_key(x), order_key(y), idx};
      mx = mn;
    }
    int lmin = idx >= 0 ? lane : -1, lmax = lmin;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      const LexPt a = shfl_lex(mn, m), b = shfl_lex(mx, m);
      const int la = __shfl_xor_sync(kFull, lmin, m), lb = __shfl_xor_sync(kFull, lmax, m);
      if (lex_min_better(a, mn)) { mn = a; lmin = la; }
      if (lex_max_better(b, mx)) { mx = b; lmax = lb; }
    }
    const int nvalid = __popc(__ballot_sync(kFull, idx >= 0));
    ok = __all_sync(kFull, ok) && nvalid >= 3 && lmin >= 0 && lmax >= 0 && mn.kx < mx.kx;
    __syncwarp();
    PolyF& P = S.P;
    if (ok) build_chains(S, lmin, lmax, lane);
    if (ok) {
      // thresholds (lanes 0..15 upper, 16..31 lower) and edges
      const int j = lane & (kChainEdges - 1);
      const bool up = lane < kChainEdges;
      const int* C = up ? S.cu : S.cl;
      const int nv = up ? S.nu : S.nl;
      float* T = up ? P.tu : P.tl;
      T[j] = j < nv - 2 ? trunc_f32(S.x[C[j + 1]]) : INFINITY;
      float4* E = up ? &P.eu[j][0] : &P.el[j][0];
      if (j < nv - 1) {
        const LineF L = make_line(S.x[C[j]], S.y[C[j]], S.x[C[j + 1]], S.y[C[j + 1]]);
        E[0] = make_float4(L.ox, L.oy, L.dx, L.dy);
        E[1] = make_float4(L.k, L.c, 0.0f, 0.0f);
      } else {
        E[0] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        E[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
      if (lane == 0) {
        P.xl = trunc_f32(S.x[lmin]);
        P.xr = trunc_f32(S.x[lmax]);
        P.on = 1;
        P.pad = 0;
      }
    } else if (lane == 0) {
      P.on = 0;
      P.pad = 0;
      P.xl = INFINITY;
      P.xr = -INFINITY;
    }
    if (lane < kPolyBoxes) {
      P.box[lane][0] = INFINITY; P.box[lane][1] = -INFINITY;
      P.box[lane][2] = INFINITY; P.box[lane][3] = -INFINITY;
    }
    __syncwarp();
    // inner boxes around a centre c: half sizes s (hx, hy) for box 0,
    // s (1.307 hx, 0.541 hy) (wide) and s (0.541 hx, 1.307 hy) (tall), the
    // corners of boxes 1 and 2 lying at 22.5 degrees from the axes where
    // those of box 0 lie at 45.  c and (hx, hy) come from the box of the
    // diagonal candidates (else from the chains' extent).  Per box, s is the
    // largest tried value whose four corners pass the certain inside test.
    if (ok) {
      // FP32 throughout (GB300's FP64 pipe is slow and the box is only a
      // heuristic): each tested corner is an FP32 value, widened exactly, so
      // the stored box is the one whose corners passed the test
      float cx, cy, hx, hy;
      const int i1 = S.idx[4], i2 = S.idx[12], i3 = S.idx[20], i4 = S.idx[28];
      const float x0 = fmaxf(S.fx[12], S.fx[20]), x1 = fminf(S.fx[4], S.fx[28]);
      const float y0 = fmaxf(S.fy[20], S.fy[28]), y1 = fminf(S.fy[4], S.fy[12]);
      if (i1 >= 0 && i2 >= 0 && i3 >= 0 && i4 >= 0 && x0 < x1 && y0 < y1) {
        cx = 0.5f * (x0 + x1); cy = 0.5f * (y0 + y1);
        hx = 0.5f * (x1 - x0); hy = 0.5f * (y1 - y0);
      } else {
        float sx = 0.0f, sy = 0.0f, ylo = S.fy[lmin], yhi = S.fy[lmin];
        const int nv = S.nu + S.nl;
        for (int i = 0; i < S.nu; i++) { sx += S.fx[S.cu[i]]; sy += S.fy[S.cu[i]]; ylo = fminf(ylo, S.fy[S.cu[i]]); yhi = fmaxf(yhi, S.fy[S.cu[i]]); }
        for (int i = 0; i < S.nl; i++) { sx += S.fx[S.cl[i]]; sy += S.fy[S.cl[i]]; ylo = fminf(ylo, S.fy[S.cl[i]]); yhi = fmaxf(yhi, S.fy[S.cl[i]]); }
        cx = sx / (float)nv; cy = sy / (float)nv;
        hx = 0.25f * (S.fx[lmax] - S.fx[lmin]); hy = 0.25f * (yhi - ylo);
      }
      // lane 6 b + j (j < 6, b < kPolyBoxes) tests scale j of box b (its
      // four corners in turn): a coarse round over (0, 1], then two rounds
      // that split the gap above the largest passing scale into 7 parts;
      // per box the largest passing scale is kept with an atomic maximum on
      // its bits (non-negative floats order as their bit patterns)
      constexpr int kScales = 6;
      static_assert(kScales * kPolyBoxes <= kWarp, "one try per lane");
      const float coarse[kScales] = {1.0f, 0.95f, 0.85f, 0.7f, 0.5f, 0.25f};
      if (lane < kPolyBoxes) S.bb[lane] = 0.0f;
      __syncwarp();
      const int b = lane / kScales, j = lane - b * kScales;
      const bool box = b < kPolyBoxes;
      const float fx = box ? box_fx(b) : 0.0f, fy = box ? box_fy(b) : 0.0f;
      float gap = 0.0f;  // width of the interval the next round splits
      for (int round = 0; round < 3; round++) {
        const float best = box ? S.bb[b] : 0.0f;
        float sc = coarse[j];
        if (round == 1) {  // the gap up to the next coarse scale
          gap = best >= 1.0f ? 0.0f : (best >= 0.95f ? 0.05f : (best >= 0.85f ? 0.1f : (best >= 0.7f ? 0.15f : (best >= 0.5f ? 0.2f : (best >= 0.25f ? 0.25f : 0.25f)))));
        } else if (round == 2) {
          gap = gap * (1.0f / 7.0f);
        }
        if (round > 0) sc = best + gap * (float)(kScales - j) * (1.0f / 7.0f);
        // explicit roundings (never contracted): the store below recomputes
        // the same corners
        const float ex = __fmul_rn(__fmul_rn(sc, fx), hx), ey = __fmul_rn(__fmul_rn(sc, fy), hy);
        bool in = box && sc > best && ex > 0.0f && ey > 0.0f && isfinite(__fadd_rn(cx, ex)) && isfinite(__fadd_rn(cy, ey));
#pragma unroll 1
        for (int k = 0; k < 4 && in; k++)
          in = poly_inside(P, f2d_exact((k & 1) ? __fadd_rn(cx, ex) : __fsub_rn(cx, ex)),
                           f2d_exact((k & 2) ? __fadd_rn(cy, ey) : __fsub_rn(cy, ey)));
        __syncwarp();
        if (in) atomicMax(reinterpret_cast<int*>(&S.bb[b]), __float_as_int(sc));
        __syncwarp();
      }
      if (lane < kPolyBoxes && S.bb[lane] > 0.0f) {
        const int b = lane;
        const float best = S.bb[b];
        const float ex = __fmul_rn(__fmul_rn(best, box_fx(b)), hx), ey = __fmul_rn(__fmul_rn(best, box_fy(b)), hy);
        P.box[b][0] = hword(f2d_exact(__fsub_rn(cx, ex))); P.box[b][1] = hword(f2d_exact(__fadd_rn(cx, ex)));
        P.box[b][2] = hword(f2d_exact(__fsub_rn(cy, ey))); P.box[b][3] = hword(f2d_exact(__fadd_rn(cy, ey)));
      }
    }
    __syncwarp();
    const int* src = reinterpret_cast<const int*>(&P);
    int* dst = reinterpret_cast<int*>(w.poly + s);
    for (int i = lane; i < (int)(sizeof(PolyF) / sizeof(int)); i += kWarp) dst[i] = src[i];
    __syncwarp();
  }
}

// ---- the sieve -------------------------------------------------------------

// A warp's step: 256 consecutive points of one tile, 8 per lane (lane l
// holds points 64 k + 2 l + e, k < 4, e < 2: four 16-byte loads per array).
constexpr int kSvStep = 2 * kWarp * 4;

// Per warp: the points of a step that are outside every inner box.
struct SvRest {
  double x[kSvStep];
  double y[kSvStep];
  int i[kSvStep];
};

__device__ __forceinline__ int sv_set_of(const Work& w, int t) {
  int lo = 0, hi = w.nsets - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (w.k0_tile_start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Block b takes the extreme-pass tiles [T b / G, T (b + 1) / G) (G blocks);
// the warps of a block take the steps of a tile in turn.  A step's points
// go straight into registers (16-byte streaming loads; every warp keeps
// four loads per array in flight, and a resident grid of 24 warps per SM
// keeps the memory system busy).  The box test (high words as FP32, no
// arithmetic) decides almost every point; the rest are compacted into the
// warp's shared-memory list and take the chain test on full warps; the
// points that pass neither are written to the set's range of buffer 1 after
// one atomic per warp and round reserves their slots, and feed the warp's
// running extremes and flags.  When the block leaves a set (or its range
// ends) its warps' extremes are combined and written to the partial of
// (block b, set s), slot b + s: unique, because a later block never works
// on an earlier set.
__global__ void __launch_bounds__(32 * kSvWarps, 3) k_sieve(Work w) {
  __shared__ SvRest s_rest[kSvWarps];
  __shared__ LexPt s_mn[kSvWarps], s_mx[kSvWarps];
  __shared__ int s_fl[kSvWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  SvRest& R = s_rest[warp];
  const unsigned lt = lanemask_lt();
  const long long T = w.k0_tile_start[w.nsets], G = gridDim.x;
  const int t0 = (int)(T * blockIdx.x / G), t1 = (int)(T * (blockIdx.x + 1) / G);
  if (blockIdx.x == 0 && threadIdx.x == 0) w.ctrl->sv_grid = (int)G;
  if (t0 >= t1) return;
  int set = sv_set_of(w, t0);
  int set_end = w.k0_tile_start[set + 1];
  SetRec S = w.sets[set];
  const PolyF* P = w.poly + set;
  // the first three inner boxes in registers (the test of every point);
  // the others are read on the compacted rest
  constexpr int kRegBoxes = 3;
  float bx[kRegBoxes][4];
#pragma unroll
  for (int b = 0; b < kRegBoxes; b++)
#pragma unroll
    for (int c = 0; c < 4; c++) bx[b][c] = P->box[b][c];
  int on = P->on;
  LexPt mn{LLONG_MAX, LLONG_MAX, INT_MAX}, mx{LLONG_MIN, LLONG_MIN, INT_MAX};
  unsigned am = 0;
  for (int t = t0; t < t1; t++) {
    const int j = t - w.k0_tile_start[set];
    const int tb = S.off + j * kK0Tile, tc = min(kK0Tile, S.len - j * kK0Tile);
    const bool vec = w.aos ? (reinterpret_cast<uintptr_t>(w.x + 2ll * tb) & 15u) == 0
                           : ((reinterpret_cast<uintptr_t>(w.x + tb) | reinterpret_cast<uintptr_t>(w.y + tb)) & 15u) == 0;
    for (int s0 = warp * kSvStep; s0 < tc; s0 += kSvWarps * kSvStep) {
      const int base = tb + s0, cnt = min(kSvStep, tc - s0);
      double vx[8], vy[8];
      if (vec && cnt == kSvStep && !w.aos) {
        const double2* X2 = reinterpret_cast<const double2*>(w.x + base);
        const double2* Y2 = reinterpret_cast<const double2*>(w.y + base);
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const double2 a = __ldcs(X2 + k * kWarp + lane), b = __ldcs(Y2 + k * kWarp + lane);
          vx[2 * k] = a.x; vx[2 * k + 1] = a.y;
          vy[2 * k] = b.x; vy[2 * k + 1] = b.y;
        }
      } else if (vec && cnt == kSvStep) {  // interleaved: one 16-byte load per point
        const double2* P2 = reinterpret_cast<const double2*>(w.x + 2ll * base);
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const double2 a = __ldcs(P2 + 64 * (q >> 1) + 2 * lane + (q & 1));
          vx[q] = a.x;
          vy[q] = a.y;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const int l = 64 * (q >> 1) + 2 * lane + (q & 1);
          vx[q] = l < cnt ? px(w, base + l) : 0.0;
          vy[q] = l < cnt ? py(w, base + l) : 0.0;
        }
      }
      unsigned rest = 0;
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int l = 64 * (q >> 1) + 2 * lane + (q & 1);
        if (l < cnt && !in_boxes(bx, hword(vx[q]), hword(vy[q]))) rest |= 1u << q;
      }
      if (!__any_sync(kFull, rest != 0)) continue;
      // the points outside the boxes, compacted into the warp's list
      int n = 0;
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const bool o = (rest >> q) & 1u;
        const unsigned b = __ballot_sync(kFull, o);
        if (o) {
          const int d = n + __popc(b & lt);
          R.x[d] = vx[q];
          R.y[d] = vy[q];
          R.i[d] = base + 64 * (q >> 1) + 2 * lane + (q & 1);
        }
        n += __popc(b);
      }
      __syncwarp();
      // the other boxes on full warps; what they leave is compacted again
      // in place (a lane writes at or below the position every lane read)
      if (kPolyBoxes > kRegBoxes && n > kWarp) {  // they can save a chain-test pass
        float xb[kPolyBoxes - kRegBoxes][4];
#pragma unroll
        for (int b = 0; b < kPolyBoxes - kRegBoxes; b++)
#pragma unroll
          for (int c = 0; c < 4; c++) xb[b][c] = P->box[kRegBoxes + b][c];
        int n2 = 0;
        for (int i0 = 0; i0 < n; i0 += kWarp) {
          const int i = i0 + lane;
          bool o = false;
          double ux = 0.0, uy = 0.0;
          int ui = 0;
          if (i < n) {
            ux = R.x[i];
            uy = R.y[i];
            ui = R.i[i];
            o = !in_boxes(xb, hword(ux), hword(uy));
          }
          const unsigned b = __ballot_sync(kFull, o);
          if (o) {
            const int d = n2 + __popc(b & lt);
            R.x[d] = ux;
            R.y[d] = uy;
            R.i[d] = ui;
          }
          n2 += __popc(b);
        }
        __syncwarp();
        n = n2;
      }
      // chain test on full warps; the points it cannot place inside are kept
      for (int i0 = 0; i0 < n; i0 += kWarp) {
        const int i = i0 + lane;
        bool keep = false;
        double ux = 0.0, uy = 0.0;
        int ui = 0;
        if (i < n) {
          ux = R.x[i];
          uy = R.y[i];
          ui = R.i[i];
          keep = !(on && poly_inside(*P, ux, uy));
        }
        const unsigned b = __ballot_sync(kFull, keep);
        if (b == 0u) continue;
        int pos = 0;
        if (lane == 0) pos = atomicAdd(&w.nsurv[set], __popc(b));
        pos = __shfl_sync(kFull, pos, 0) + __popc(b & lt);
        if (keep) {
          if (VQ_OK_IDX(w, 46, (long long)S.off + pos, 0, w.N)) {
            w.bx[1][S.off + pos] = ux;
            w.by[1][S.off + pos] = uy;
            w.bi[1][S.off + pos] = ui;
          }
          k0_take(ux, uy, ui, mn, mx, am);
        }
      }
      __syncwarp();  // the list is refilled by the next step
    }
    if (t + 1 < t1 && t + 1 < set_end) continue;  // same set next
    // the block leaves this set: its partial at slot blockIdx.x + set
    int fl = k0_flags(am);
#pragma unroll
    for (int q = 16; q >= 1; q >>= 1) {
      const LexPt a = shfl_lex(mn, q), b = shfl_lex(mx, q);
      if (lex_min_better(a, mn)) mn = a;
      if (lex_max_better(b, mx)) mx = b;
      fl |= __shfl_xor_sync(kFull, fl, q);
    }
    if (lane == 0) { s_mn[warp] = mn; s_mx[warp] = mx; s_fl[warp] = fl; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < kSvWarps; q++) {
        if (lex_min_better(s_mn[q], mn)) mn = s_mn[q];
        if (lex_max_better(s_mx[q], mx)) mx = s_mx[q];
        fl |= s_fl[q];
      }
      K0Part Q;
      Q.minx = mn.kx; Q.miny = mn.ky; Q.mini = mn.i;
      Q.maxx = mx.kx; Q.maxy = mx.ky; Q.maxi = mx.i;
      Q.flags = fl;
      Q.pad = 0;
      w.k0part[(long long)blockIdx.x + set] = Q;
    }
    __syncthreads();  // s_mn / s_mx are reused at the next set
    mn = LexPt{LLONG_MAX, LLONG_MAX, INT_MAX};
    mx = LexPt{LLONG_MIN, LLONG_MIN, INT_MAX};
    am = 0;
    if (t + 1 < t1) {  // the next tile's set (sets without tiles are skipped)
      while (w.k0_tile_start[set + 1] <= t + 1) set++;
      set_end = w.k0_tile_start[set + 1];
      S = w.sets[set];
      P = w.poly + set;
#pragma unroll
      for (int b = 0; b < kRegBoxes; b++)
#pragma unroll
        for (int c = 0; c < 4; c++) bx[b][c] = P->box[b][c];
      on = P->on;
    }
  }
}
