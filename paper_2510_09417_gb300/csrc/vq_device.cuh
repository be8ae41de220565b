// vq_device.cuh -- device-side records and exact predicates for the
// level-synchronous planar Quickhull (VQhull, arxiv 2510.09417).
//
// The predicates are the two tests of Sec. 2.1:
//   left-of      : (px-ux)(qy-uy) > (py-uy)(qx-ux), i.e. orient(p,q,u) > 0
//   farther-than : (qy-py)(ux-u'x) < (qx-px)(uy-u'y), i.e. (q-p) x (u-u') > 0
// evaluated exactly in three tiers:
//   1. FP32 on coordinates truncated to 24 significant bits by integer ops
//      (no FP64 instruction), with a per-point error bound derived below;
//   2. FP64 with Shewchuk's bound (3 + 16 eps) eps (|t1| + |t2|), eps = 2^-53
//      ("Adaptive Precision Floating-Point Arithmetic and Fast Robust
//      Geometric Predicates", 1997, Sec. 4);
//   3. exact expansion arithmetic: TwoProduct by FMA and Grow-Expansion
//      (Shewchuk 1997, Thm. 10) over the products of raw coordinates.
// Exactness holds for finite inputs whose nonzero magnitudes lie in
// [2^-400, 2^400]; the FP32 tier is only used on point sets with all
// |coordinates| < 2^40 (flag computed by the extreme-point pass).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vq {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxLevels = 512;

// error bits in Ctrl::err
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned kErrNonfinite = 2u;
constexpr unsigned kErrCapacity = 4u;
constexpr unsigned kErrInternal = 8u;
constexpr unsigned kErrBadOffsets = 16u;
constexpr unsigned kErrWorklistFull = 32u;  // the worklist's queue or segment table overflowed: the call
                                            // is run again with the level loop alone
constexpr unsigned kErrFatal = kErrTimeout | kErrCapacity | kErrInternal | kErrBadOffsets | kErrWorklistFull;

// segment flags
constexpr int kSegFast = 1;       // FP32 tier allowed (all |coords| < 2^40)
constexpr int kSegSrcInput = 2;   // points still in the caller's arrays (level 0)
constexpr int kSegSrcBuf1 = 4;    // points in ping-pong buffer 1 (else buffer 0)
constexpr int kSegDense = 8;      // hull-dense set (most points kept by the pre-filter): segments of up to
                                  // the finisher's capacity go to it (see seg_small_max)

// look-back status words: 2 flag bits, 31-bit left count, 31-bit right count
constexpr unsigned long long kStAgg = 1ull << 62;
constexpr unsigned long long kStInc = 2ull << 62;
constexpr unsigned long long kStFlagMask = 3ull << 62;
constexpr unsigned long long kCnt31 = 0x7fffffffull;

__host__ __device__ inline unsigned long long st_pack(unsigned long long l, unsigned long long r) {
  return (l << 31) | r;
}

// Control block: counters shared by the kernels of one call.
struct Ctrl {
  unsigned int err;
  int k1_ticket;
  int k1_segs[2];     // K1 segments per level parity
  int k1_tiles[2];    // K1 tiles per level parity
  int k3_count;       // small-segment queue length
  int k0_tiles;       // tiles of the extreme pass
  int k0_ticket;
  int level;
  unsigned long long emitted;
  long long nonfinite_set;  // first set with a non-finite coordinate
  long long total;          // vertices over all sets (written by the ordering)
  long long k1_read;        // points classified by the partition kernel
  long long k1_kept;        // of those, points written to a child
  int dbg_site;             // checked builds: first failed bounds check
  int fill_jobs[2];         // tile-map fill jobs per level parity
  int any_slow;             // some point set needs the FP64 tier (|coordinate| >= 2^40)
  int sv_grid;              // blocks of the last sieve launch (its partials are per block and set)
  long long k1_nw[2];       // warps of the last partition launch per level parity
  long long dbg_val;        // checked builds: the offending value
  unsigned long long k1prof[12];  // profiling builds: partition-kernel cycle and event counters
  unsigned long long k2prof[4];   // profiling builds: finalize counters
  unsigned long long k3prof[8];   // profiling builds: small-segment kernel counters
  long long graph_iters;    // device-driven level loop: iterations of its body (two levels each)
  int live_levels;          // levels >= 1 that started with at least one big segment
  int pad1;
  long long key_words;      // bitmap words the order pass reads (0: all); a single set's finalize
                            // sets it to the words its keys can reach and clears them
  unsigned long long loop_t0;  // device-driven level loop: time of its first condition (ns)
  // persistent worklist (taken over from the level loop once a level is
  // small).  The counters its blocks update per task or read while they
  // wait sit in cache lines of their own.
  // queue entries reserved by producers (high 32 bits) and tasks queued or
  // running (low 32 bits; 0: the recursion is done), in one word so that a
  // push is one atomic
  alignas(128) unsigned long long wl_tp;
  int wl_pad0[30];
  int wl_head;              // next queue entry a block claims
  int wl_pad1[31];
  int wl_nseg;              // worklist segment slots in use
  int wl_pad3[31];
  int wl_on;                // 1: the level loop handed its segments over
  int wl_par;               // parity of the handed-over level (its segments are segs[wl_par])
  int wl_nbig;              // handed-over big segments
  int wl_nsmall;            // handed-over small segments (the small-segment queue)
  int wl_maxlevel;          // deepest level the worklist reached, plus one
  int wl_pad4[27];
};

// A live segment: points off .. off+len-1 of its source buffer, hull edge
// a->b, farthest point r (global indices).  Children are a->r and r->b.
struct SegRec {
  long long shift;  // order key of buffer position pos is pos + 1 + shift
  int off;
  int len;
  int a, b, r;
  int set_off;      // first global index of the point set (for set-local output)
  int level;        // partition level of this segment
  int tile_base;
  int ntiles;
  int flags;
};

// Per-segment constants of the FP32 tier and the exact endpoints.
// Line 1 is a->r (left child), line 2 is r->b (right child).
struct SegGeom {
  double ax, ay, rx, ry, bx, by;  // line 1 = {ax, ay, rx, ry}, line 2 = {rx, ry, bx, by}
  float o1x, o1y, o2x, o2y;  // origins: truncated a and r (same conversion as points)
  float d1x, d1y, d2x, d2y;  // rounded r-a and b-r
  float k1, c1, k2, c2;      // error bound: E = k*(|ux~|+|uy~|) + c + 2^-22 |d~|
};

// Persistent worklist.  A big segment (more than small_max points) lives in
// a slot of the segment table while its partition tasks run: each task
// classifies and compacts up to kWlTaskPts of its points and leaves the
// farthest point per child among them in a record; the task that
// completes the segment (ticket ndone) reduces the records, emits r and
// pushes the children.
struct alignas(16) WlSeg {
  SegRec R;
  SegGeom G;
  unsigned long long cursor;  // children's counts (left << 32 | right), as SegState::cursor
  int ndone;                  // finished tasks
  int ntasks;                 // tasks of the segment
  int t0;                     // queue index of its first task (its tasks are t0 .. t0+ntasks-1)
  int pad[3];
};
// A queue entry: a partition task (seg >= 0: points begin .. begin+count-1
// of segment slot seg) or a small segment (seg < 0: R, finished whole).
// Entry i is ready when its tag equals the call's epoch.
struct alignas(16) WlTask {
  SegRec R;
  int seg;
  int begin;
  int count;
  int pad;
};

struct SetRec {
  long long shift;  // key(pos) = pos + 1 + shift; key of p = off + shift
  int off;
  int len;
  int flags;
  int p, q;
  int pad;
};

// A farthest-point candidate published through the look-back: the point,
// bounds lo <= orient(child line, point) <= hi, and its index (-1: none).
struct BestRec {
  double x, y;
  double lo, hi;
  int idx;
  int pad;
};

// Per partition tile and child (0 = left, 1 = right): the tile's own
// farthest point (written before its aggregate status) and the running
// farthest point over the segment's tiles up to this one (written before
// its inclusive status).  The last tile's inclusive records are the
// children's farthest points.
struct TileRec {
  BestRec own[2];
  BestRec incl[2];
};

// Where a partition tile's points are: written per tile when the tile map is
// built, read (one 32-byte load) by the partition kernel's copy issuer.
struct alignas(16) TileDesc {
  int sid;    // segment
  int begin;  // first buffer position of the tile
  int count;  // points in the tile
  int flags;  // segment flags
  int off, len;  // segment range
  int pad0, pad1;
};

// Per big segment and level: output cursors and farthest-point candidates.
// cursor packs the children's counts (left << 32 | right); tiles add their
// counts atomically and get their output offsets back.  lomax[c] is the
// largest lower bound of child c's key seen so far (order-preserving u64 of
// an FP64 value); a tile whose best upper bound reaches it adds its index to
// cand[c].  The child's farthest point is the exact best among the listed
// tiles' own records with hi >= the final lomax; more than kMaxCand entries
// (ncand) fall back to scanning every tile's record.
constexpr int kMaxCand = 32;
struct SegState {
  unsigned long long cursor;
  unsigned long long lomax[2];
  int ncand[2];
  int cand[2][kMaxCand];
};

__host__ __device__ inline unsigned long long dkey(double v) {
#ifdef __CUDA_ARCH__
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long b;
  __builtin_memcpy(&b, &v, 8);
#endif
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ inline double dkey_inv(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

struct K0Part {
  long long minx, miny, maxx, maxy;  // ordered-integer keys
  int mini, maxi;
  int flags;  // bit0 nonfinite, bit1 out of FP32 range
  int pad;
};

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__device__ __forceinline__ void st_volatile_u64(unsigned long long* p, unsigned long long v) {
  *reinterpret_cast<volatile unsigned long long*>(p) = v;
}

// release store / acquire load at GPU scope (look-back status words)
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Doubles as signed integers with the same order; -0 and +0 map to 0.
__device__ __forceinline__ long long order_key(double v) {
  long long b = __double_as_longlong(v);
  return b >= 0 ? b : -(b & 0x7fffffffffffffffll);
}

// FP64 -> FP32 by integer ops: keep the top 23 fraction bits (truncation)
// and rebias the exponent; magnitudes below 2^-126 become exactly -2^-126
// (negative v) or +2^-126 (positive v and both zeros).  For
// 2^-126 <= |v| < 2^128 the result is v truncated to 24 significant bits:
// |v~ - v| < 2^-23 |v|; below 2^-126, |v~ - v| < 2^-125.  The map is
// monotone (u <= v implies u~ <= v~), so u~ > v~ implies u > v.
__device__ __forceinline__ float trunc_f32(double v) {
  const unsigned lo = static_cast<unsigned>(__double2loint(v));
  const unsigned hi = static_cast<unsigned>(__double2hiint(v));
  const unsigned a = hi & 0x7fffffffu;
  const unsigned f = a < 0x38100000u ? 0x00800000u : __funnelshift_l(lo, a, 3) - 0xC0000000u;  // (1023 - 127) << 23
  const unsigned neg = (a | lo) != 0u ? (hi & 0x80000000u) : 0u;  // -0 maps like +0
  return __uint_as_float(f | neg);
}

// Exact FP32 -> FP64 widening by integer operations (GB300's FP64 pipe is
// narrow; per-tile bookkeeping stays off it).  Normal numbers rebias the
// exponent by 1023 - 127; subnormals m * 2^-149 are renormalised at their
// leading bit; zeros, infinities and NaNs keep their class.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long s = (unsigned long long)(u >> 31) << 63;
  const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned long long b;
  if (e == 0xffu) b = 0x7ff0000000000000ull | ((unsigned long long)m << 29);
  else if (e != 0u) b = ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  else if (m == 0u) b = 0ull;
  else {
    const int p = 31 - __clz(m);
    b = ((unsigned long long)(p + 874) << 52) | ((unsigned long long)(m - (1u << p)) << (52 - p));
  }
  return __longlong_as_double((long long)(s | b));
}
__device__ __forceinline__ double widen(float v) { return f2d_exact(v); }
__device__ __forceinline__ double widen(double v) { return v; }

// FP64 -> FP32 rounded to nearest (ties to even) by integer operations,
// from the IEEE 754 definition: normal results keep the top 23 fraction
// bits and round on the 29 dropped ones (a carry moves into the exponent,
// up to infinity); results below 2^-126 are FP32 subnormals m 2^-149 with m
// rounded from the full significand; infinities and NaNs keep their class.
// GB300's FP64 pipe (conversions included) has about 64 cycles of latency;
// this runs on the integer pipe.
__device__ __forceinline__ float f32_rn(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffull);
  const unsigned long long f = b & 0xfffffffffffffull;
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (f ? 0x00400000u : 0u));
  const int ef = e - 896;  // FP32 biased exponent (1023 - 127)
  unsigned r;
  if (ef > 0) {
    if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);
    r = ((unsigned)ef << 23) | (unsigned)(f >> 29);
    const unsigned rem = (unsigned)(f & 0x1fffffffull);
    if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) r++;  // may carry into the exponent
  } else {
    const int sh = 30 - ef;  // value = M 2^(e - 1075), unit 2^-149: M >> (926 - e)
    if (e == 0 || sh >= 64) return __uint_as_float(sign);  // below half the smallest subnormal
    const unsigned long long M = f | (1ull << 52);
    r = (unsigned)(M >> sh);
    const unsigned long long rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (r & 1u))) r++;
  }
  return __uint_as_float(sign | r);
}

// Profiling builds (VQ_WL_PROFILE): calls of the FP64 filter and of the
// exact expansions, per translation unit.
#ifdef VQ_WL_PROFILE
__device__ unsigned long long g_vq_tier_calls[8];
#define VQ_COUNT_TIER(i) atomicAdd(&g_vq_tier_calls[i], 1ull)
#else
#define VQ_COUNT_TIER(i)
#endif

// ---------------------------------------------------------------------------
// Tier 1: FP32 orient with a rigorous error bound.
//
// With u~, o~ the truncated point and origin (|w~ - w| <= 2^-23|w| + 2^-125),
// D~ = fl32(D) for the exact direction D (|D~ - D| <= 2^-23 |D| + 2^-149),
// t~ = fl(ux~ - ox~), s~ = fl(uy~ - oy~), p = fl(Dy~ t~),
// d~ = fl(Dx~ s~ - p) (one FMA), one finds with rho >= (1 + 2^-22) max|D~|
//   |d~ - d| <= 3.01 * 2^-23 rho (|ux|+|uy|+|ox|+|oy|) + 2^-23.99 |d~| + rho 2^-122 + 2^-104,
// and |ux| + |uy| <= (1 + 2^-22)(|ux~| + |uy~|) + 2^-124.
// The bound used, E = k (|ux~|+|uy~|) + c + 2^-22 |d~| with
// k = 4 * 2^-23 rho and c = 4 * 2^-23 rho (|ox|+|oy|) + rho 2^-100 + 2^-100,
// is evaluated with upward rounding and covers it with margin, as long as
// all |coordinates| < 2^40 (so nothing overflows FP32).
// ---------------------------------------------------------------------------

struct LineF {
  float ox, oy, dx, dy, k, c;
};

__device__ __forceinline__ void orient_f32(const LineF& L, float ux, float uy, float m, float& d,
                                           float& e) {
  const float t = __fsub_rn(ux, L.ox);
  const float s = __fsub_rn(uy, L.oy);
  const float p = __fmul_rn(L.dy, t);
  d = __fmaf_rn(L.dx, s, -p);
  e = __fmaf_ru(fabsf(d), 0x1p-22f, __fmaf_ru(L.k, m, L.c));
}

// ---------------------------------------------------------------------------
// Tier 1b: FP32 in coordinates relative to the line's first endpoint o, for
// points that the absolute tier leaves undecided because they are nearly
// collinear far from the origin (hull-dense inputs such as points on a
// circle).  With T = u - o and D = e - o (exact), T~ = fl32(fl64(u - o)),
// D~ the line's rounded direction (as above), p = fl(D~y T~x) and
// d~ = fl(D~x T~y - p) (one FMA), writing |T~ - T| <= a |T~| + b and
// |D~ - D| <= a |D~| + b with a = 2^-24 (1 + 2^-20), b = 2^-148:
//   |d~ - d| <= 2^-24 |d~| + (2a (1 + a) + 2^-24) (|D~x||T~y| + |D~y||T~x|)
//               + b (1 + a) (|D~x| + |D~y| + |T~x| + |T~y|) + 2^-149,
// and with rho = max |D~| (|D~x||T~y| + |D~y||T~x| <= rho m, m = |T~x| + |T~y|)
// this is covered by E = 2^-22 |d~| + (k + 2^-146) m + (k 2^-110 + 2^-140),
// k = 4 * 2^-23 rho (1 + 2^-21) the absolute tier's constant, evaluated with
// upward rounding: no term depends on the magnitude of o or u.  Valid for
// all |coordinates| < 2^40 (nothing overflows FP32); the two FP64
// subtractions are the tier's only FP64 work.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void orient_rel(const LineF& L, double ox, double oy, double ux, double uy, float& d,
                                           float& e) {
  VQ_COUNT_TIER(5);
  const float tx = f32_rn(__dsub_rn(ux, ox));
  const float ty = f32_rn(__dsub_rn(uy, oy));
  const float m = __fadd_ru(fabsf(tx), fabsf(ty));
  const float p = __fmul_rn(L.dy, tx);
  d = __fmaf_rn(L.dx, ty, -p);
  const float k = __fadd_ru(L.k, 0x1p-146f);
  const float c = __fmaf_ru(L.k, 0x1p-110f, 0x1p-140f);
  e = __fmaf_ru(fabsf(d), 0x1p-22f, __fmaf_ru(k, m, c));
}

// ---------------------------------------------------------------------------
// Tier 2: FP64 with separately rounded operations (never contracted).
// ---------------------------------------------------------------------------

constexpr double kEps = 1.1102230246251565404e-16;  // 2^-53
constexpr double kCcwErr = (3.0 + 16.0 * kEps) * kEps;

// sign of (p1-p0) x (q1-q0) if the filter settles it (*sure = true).
// Also returns the rounded value and its error bound.
__device__ __forceinline__ int cross_f64(double p0x, double p0y, double p1x, double p1y, double q0x,
                                         double q0y, double q1x, double q1y, double& det,
                                         double& bound, bool& sure) {
  VQ_COUNT_TIER(0);
  const double t1 = __dmul_rn(__dsub_rn(p1x, p0x), __dsub_rn(q1y, q0y));
  const double t2 = __dmul_rn(__dsub_rn(p1y, p0y), __dsub_rn(q1x, q0x));
  det = __dsub_rn(t1, t2);
  bound = __dmul_ru(kCcwErr, __dadd_ru(fabs(t1), fabs(t2)));
  if (det > bound) { sure = true; return 1; }
  if (-det > bound) { sure = true; return -1; }
  if (bound == 0.0 && det == 0.0) { sure = true; return 0; }
  sure = false;
  return 0;
}

__device__ __forceinline__ int dot_f64(double p0x, double p0y, double p1x, double p1y, double q0x,
                                       double q0y, double q1x, double q1y, bool& sure) {
  const double t1 = __dmul_rn(__dsub_rn(p1x, p0x), __dsub_rn(q1x, q0x));
  const double t2 = __dmul_rn(__dsub_rn(p1y, p0y), __dsub_rn(q1y, q0y));
  const double det = __dadd_rn(t1, t2);
  const double bound = __dmul_ru(kCcwErr, __dadd_ru(fabs(t1), fabs(t2)));
  if (det > bound) { sure = true; return 1; }
  if (-det > bound) { sure = true; return -1; }
  if (bound == 0.0 && det == 0.0) { sure = true; return 0; }
  sure = false;
  return 0;
}

// ---------------------------------------------------------------------------
// Tier 3: exact expansion arithmetic (rare path, kept out of line).
// ---------------------------------------------------------------------------

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& err) {
  s = __dadd_rn(a, b);
  const double bv = __dsub_rn(s, a);
  const double av = __dsub_rn(s, bv);
  err = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

// sign( sum_k sg_k a_k b_k ), n <= 8.  Rare path: loops are kept rolled and
// the expansion lives in local memory.  Like every helper here it is
// inlined: the kernels make no device-function calls (calls measured
// slower, through their stack traffic, than the larger inlined code).
static __device__ __forceinline__ int exact_sum_sign(int n, const double* a, const double* b, const int* sg) {
  VQ_COUNT_TIER(1);
  double e[16];
  int m = 0;
#pragma unroll 1
  for (int k = 0; k < 2 * n; k++) {
    const int t = k >> 1;
    const double hi = __dmul_rn(a[t], b[t]);
    double q = (k & 1) ? hi : __fma_rn(a[t], b[t], -hi);  // exact product error, then the product
    if (sg[t] < 0) q = -q;
#pragma unroll 1
    for (int i = 0; i < m; i++) {  // Grow-Expansion
      double sum, h;
      two_sum(q, e[i], sum, h);
      e[i] = h;
      q = sum;
    }
    e[m++] = q;
  }
#pragma unroll 1
  for (int i = m - 1; i >= 0; i--)
    if (e[i] != 0.0) return e[i] > 0.0 ? 1 : -1;
  return 0;
}

// orient(a,b,c) = (b-a) x (c-a) = bx cy - bx ay - ax cy - by cx + by ax + ay cx
static __device__ __forceinline__ int exact_orient_sign(double ax, double ay, double bx, double by, double cx,
                                              double cy) {
  const double A[6] = {bx, bx, ax, by, by, ay};
  const double B[6] = {cy, ay, cy, cx, ax, cx};
  const int S[6] = {1, -1, -1, -1, 1, 1};
  return exact_sum_sign(6, A, B, S);
}

static __device__ __forceinline__ int exact_cross_sign(double p0x, double p0y, double p1x, double p1y,
                                             double q0x, double q0y, double q1x, double q1y) {
  const double A[8] = {p1x, p1x, p0x, p0x, p1y, p1y, p0y, p0y};
  const double B[8] = {q1y, q0y, q1y, q0y, q1x, q0x, q1x, q0x};
  const int S[8] = {1, -1, -1, 1, -1, 1, 1, -1};
  return exact_sum_sign(8, A, B, S);
}

static __device__ __forceinline__ int exact_dot_sign(double p0x, double p0y, double p1x, double p1y,
                                           double q0x, double q0y, double q1x, double q1y) {
  const double A[8] = {p1x, p1x, p0x, p0x, p1y, p1y, p0y, p0y};
  const double B[8] = {q1x, q0x, q1x, q0x, q1y, q0y, q1y, q0y};
  const int S[8] = {1, -1, -1, 1, 1, -1, -1, 1};
  return exact_sum_sign(8, A, B, S);
}

// Exact orient sign via tiers 2 and 3 (used only when tier 1 is unsure).
static __device__ __forceinline__ int orient_sign_slow(double ax, double ay, double bx, double by, double cx,
                                                double cy) {
  double det, bound;
  bool sure;
  const int s = cross_f64(ax, ay, bx, by, ax, ay, cx, cy, det, bound, sure);
  if (sure) return s;
  return exact_orient_sign(ax, ay, bx, by, cx, cy);
}

// ---------------------------------------------------------------------------
// Farthest-point comparison: does u beat v as the farthest point to the left
// of o->e?  Each candidate carries bounds lo <= orient(o, e, .) <= hi.
// Order: larger orient; then the smaller projection on e - o (the tied
// point nearest o); then the lower index.  Bounds decide most pairs; the
// rest go to the exact tiers.
// ---------------------------------------------------------------------------

template <typename K>
struct CandT {
  double x, y;
  K lo, hi;
  int idx;
};

static __device__ __forceinline__ bool beats_exact(double ox, double oy, double ex, double ey, double ux, double uy, int ui,
                                         double vx, double vy, int vi) {
  if (ux == vx && uy == vy) return ui < vi;  // coincident: cross and dot are exactly 0
  VQ_COUNT_TIER(3);
  double det, bound;
  bool sure;
  int c = cross_f64(ox, oy, ex, ey, vx, vy, ux, uy, det, bound, sure);
  if (!sure) c = exact_cross_sign(ox, oy, ex, ey, vx, vy, ux, uy);
  if (c != 0) return c > 0;
  int d = dot_f64(ox, oy, ex, ey, vx, vy, ux, uy, sure);
  if (!sure) d = exact_dot_sign(ox, oy, ex, ey, vx, vy, ux, uy);
  if (d != 0) return d < 0;
  return ui < vi;
}

// L points at the line's endpoints {ox, oy, ex, ey} (read only when the
// bounds overlap, so the hot paths keep no FP64 endpoints in registers).
// Bounds compared without FP64 instructions: FP32 as is, FP64 through
// their order-preserving integer images (-0 and +0 alike).
__device__ __forceinline__ bool bound_gt(float a, float b) { return a > b; }
__device__ __forceinline__ bool bound_gt(double a, double b) { return order_key(a) > order_key(b); }

template <typename K>
__device__ __forceinline__ bool cand_beats(const double* L, const CandT<K>& u, const CandT<K>& v) {
  if (u.idx < 0) return false;
  if (v.idx < 0) return true;
  if (bound_gt(u.lo, v.hi)) return true;
  if (bound_gt(v.lo, u.hi)) return false;
  return beats_exact(L[0], L[1], L[2], L[3], u.x, u.y, u.idx, v.x, v.y, v.idx);
}

// Which of u, v is farther to the left of the line L (o -> e), decided in
// FP32 on their difference: orient(o, e, u) - orient(o, e, v) equals
// D x T with T = u - v, so the relative tier's evaluation and bound apply
// with T~ = fl32(fl64(u - v)) in place of fl32(fl64(u - o)).  Returns 1
// (u farther), -1 (v farther) or 0 (within the bound: a near tie, for the
// exact tiers).  Candidates near the farthest point are close to each
// other, so |T| and the bound are small where the keys' own bounds overlap.
__device__ __forceinline__ int beats_rel(const LineF& L, double ux, double uy, double vx, double vy) {
  float d, e;
  orient_rel(L, vx, vy, ux, uy, d, e);
  return d > e ? 1 : (d < -e ? -1 : 0);
}

// cand_beats with the line's FP32 constants: bounds, then the difference
// tier, then the exact tiers.
template <typename K>
__device__ __forceinline__ bool cand_beats(const LineF& Lf, const double* L, const CandT<K>& u, const CandT<K>& v) {
  if (u.idx < 0) return false;
  if (v.idx < 0) return true;
  if (bound_gt(u.lo, v.hi)) return true;
  if (bound_gt(v.lo, u.hi)) return false;
  if (__double_as_longlong(u.x) == __double_as_longlong(v.x) && __double_as_longlong(u.y) == __double_as_longlong(v.y))
    return u.idx < v.idx;  // the same point (other equal pairs reach the exact tiers)
  const int r = beats_rel(Lf, u.x, u.y, v.x, v.y);
  if (r != 0) return r > 0;
  return beats_exact(L[0], L[1], L[2], L[3], u.x, u.y, u.idx, v.x, v.y, v.idx);
}

template <typename K>
__device__ __forceinline__ CandT<K> cand_none() {
  CandT<K> c;
  c.x = 0.0; c.y = 0.0; c.lo = (K)0; c.hi = (K)0; c.idx = -1;
  return c;
}

template <typename K>
__device__ __forceinline__ CandT<K> shfl_xor_cand(const CandT<K>& c, int m) {
  CandT<K> o;
  o.x = __shfl_xor_sync(kFull, c.x, m);
  o.y = __shfl_xor_sync(kFull, c.y, m);
  o.lo = __shfl_xor_sync(kFull, c.lo, m);
  o.hi = __shfl_xor_sync(kFull, c.hi, m);
  o.idx = __shfl_xor_sync(kFull, c.idx, m);
  return o;
}

// Warp-wide exact argmax (all lanes get the winner).  The comparison is a
// strict total order on distinct indices, so the butterfly is consistent.
template <typename K>
__device__ __forceinline__ CandT<K> warp_best(const double* L, CandT<K> c) {
#pragma unroll 1
  for (int m = 16; m >= 1; m >>= 1) {
    const CandT<K> o = shfl_xor_cand(c, m);
    if (cand_beats(L, o, c)) c = o;
  }
  return c;
}
template <typename K>
__device__ __forceinline__ CandT<K> warp_best(const LineF& Lf, const double* L, CandT<K> c) {
#pragma unroll 1
  for (int m = 16; m >= 1; m >>= 1) {
    const CandT<K> o = shfl_xor_cand(c, m);
    if (cand_beats(Lf, L, o, c)) c = o;
  }
  return c;
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, m));
  return v;
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, m));
  return v;
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
  return v;
}

// ---------------------------------------------------------------------------
// Segment geometry for the FP32 tier, from the exact endpoints.
// ---------------------------------------------------------------------------

__device__ inline LineF make_line(double ox, double oy, double ex, double ey) {
  LineF L;
  L.ox = trunc_f32(ox);
  L.oy = trunc_f32(oy);
  // D~ = fl32(fl64(e - o)), rounded to nearest (the tiers' derivations)
  L.dx = f32_rn(__dsub_rn(ex, ox));
  L.dy = f32_rn(__dsub_rn(ey, oy));
  // rho >= (1 + 2^-22) max |D~|; the rounding of dx, dy in FP64 (2^-53) is
  // covered by the factor as well.  Everything below rounds upward in FP32,
  // so k and c are at least the derivation's values.
  const float rho = __fmul_ru(fmaxf(fabsf(L.dx), fabsf(L.dy)), 1.0f + 0x1p-21f);
  L.k = __fmul_ru(rho, 0x1p-21f);  // 4 * 2^-23 rho
  // mag >= |ox| + |oy|: |w| <= (|w~| + 2^-125)(1 + 2^-22) for the truncation w~
  const float mag =
      __fmul_ru(__fadd_ru(__fadd_ru(fabsf(L.ox), fabsf(L.oy)), 0x1p-124f), 1.0f + 0x1p-22f);
  L.c = __fadd_ru(__fadd_ru(__fmul_ru(__fmul_ru(L.k, mag), 1.0f + 0x1p-20f), __fmul_ru(rho, 0x1p-100f)), 0x1p-100f);
  return L;
}

__device__ inline void fill_geom(SegGeom& g, double ax, double ay, double bx, double by, double rx,
                                 double ry) {
  g.ax = ax; g.ay = ay; g.bx = bx; g.by = by; g.rx = rx; g.ry = ry;
  const LineF l1 = make_line(ax, ay, rx, ry);
  const LineF l2 = make_line(rx, ry, bx, by);
  g.o1x = l1.ox; g.o1y = l1.oy; g.d1x = l1.dx; g.d1y = l1.dy; g.k1 = l1.k; g.c1 = l1.c;
  g.o2x = l2.ox; g.o2y = l2.oy; g.d2x = l2.dx; g.d2y = l2.dy; g.k2 = l2.k; g.c2 = l2.c;
}

__device__ __forceinline__ LineF line1_of(const SegGeom& g) {
  LineF L; L.ox = g.o1x; L.oy = g.o1y; L.dx = g.d1x; L.dy = g.d1y; L.k = g.k1; L.c = g.c1; return L;
}
__device__ __forceinline__ LineF line2_of(const SegGeom& g) {
  LineF L; L.ox = g.o2x; L.oy = g.o2y; L.dx = g.d2x; L.dy = g.d2y; L.k = g.k2; L.c = g.c2; return L;
}

// ---------------------------------------------------------------------------
// Level-0 pre-filter: the Akl-Toussaint heuristic that the paper proposes as
// its next step (Sec. 6, the octagon p1..p8 from the extremes of x, y, x - y
// and x + y), here with kPolyDirs sampled directions instead of eight.
// Per point set, two x-monotone chains of input points run from the
// leftmost candidate L to the rightmost R: the upper chain (thresholds tu,
// edges eu) and the lower chain (tl, el), vertices in strictly increasing x.
// Let Q be the open region strictly below the upper chain and strictly
// above the lower chain over L.x < x < R.x.  Every point of Q lies on an
// open vertical segment between two points of the chains, so Q lies in the
// convex hull of the chains' vertices, and Q is open, so it lies in the
// interior of that hull: a point of Q is strictly inside the hull of its
// set.  Such a point is neither a strict vertex nor the farthest point of
// any segment (farthest points maximise a linear function over the set, so
// they lie on a supporting line of the hull), and dropping it leaves every
// result of Alg. 1 unchanged.  None of this needs the chains to be convex,
// so they are built with approximate arithmetic; only the per-point test
// must be certain: FP32 tier with its bound, and equal thresholds or
// inconclusive signs keep the point.
// An axis-parallel box whose four corners passed that same certain test
// lies in the convex hull of the corners, hence in the set's hull, and a
// point strictly inside the box is strictly inside the hull.  The box test
// compares the coordinates' high words read as FP32 numbers (hword): no
// arithmetic at all.
// ---------------------------------------------------------------------------

constexpr int kPolyDirs = 32;    // sampled directions (integer pairs, see k_sample)
constexpr int kChainEdges = 16;  // at most 16 edges (15 inner vertices) per chain

constexpr int kPolyBoxes = 5;    // inner boxes per set (corners at 45, 22.5, 67.5, 33.75, 56.25 degrees)

struct alignas(16) PolyF {
  float box[kPolyBoxes][4];  // inner boxes: hword of x0, x1, y0, y1; empty: x0 = +inf
  float xl, xr;              // trunc_f32 of L.x and R.x
  int on;                    // 1: the chains apply
  int pad;
  float tu[kChainEdges];     // trunc_f32(x) of the upper chain's inner vertices, increasing; +inf padded
  float tl[kChainEdges];     // the same for the lower chain
  float4 eu[kChainEdges][2];  // upper edge j (vertex j -> j + 1): {ox, oy, dx, dy}, {k, c, 0, 0}
  float4 el[kChainEdges][2];  // lower edges, likewise (left to right)
};

// The high word of a double read as an FP32 number.  For doubles u, v:
// hword(u) > hword(v) implies u > v.  Both positive: the high word is a
// prefix of the bit pattern, whose order is the value order.  Both
// negative: likewise with the order reversed, as for FP32.  Mixed signs and
// zeros: -0 and +0 compare equal in FP32, and a nonzero high word has a
// nonzero value.  A double of magnitude 2^1017 or more reads as an
// infinity (the implication still holds) or a NaN (every compare fails).
__device__ __forceinline__ float hword(double v) { return __int_as_float(__double2hiint(v)); }

// The point is certainly strictly inside one of the inner boxes b[0 .. NB).
template <int NB>
__device__ __forceinline__ bool in_boxes(const float (&b)[NB][4], float hx, float hy) {
  bool in = false;
#pragma unroll
  for (int k = 0; k < NB; k++) in = in || (hx > b[k][0] && hx < b[k][1] && hy > b[k][2] && hy < b[k][3]);
  return in;
}

// Edge of a chain over the truncated abscissa v: the number of inner
// thresholds below v (binary search over 16 entries, the last one +inf),
// or -1 when v equals a threshold (x undecided against that vertex).  For
// a result j, trunc_f32's monotonicity gives x(vertex j) < x < x(vertex
// j + 1) for the inner vertices involved.
__device__ __forceinline__ int chain_edge(const float* t, float v) {
  int j = 0;
#pragma unroll
  for (int s = kChainEdges / 2; s >= 1; s >>= 1) j += t[j + s - 1] < v ? s : 0;
  return t[j] == v ? -1 : j;
}

__device__ __forceinline__ LineF poly_edge(const float4 (*e)[2], int j) {
  const float4 a = e[j][0], b = e[j][1];
  LineF L;
  L.ox = a.x; L.oy = a.y; L.dx = a.z; L.dy = a.w; L.k = b.x; L.c = b.y;
  return L;
}

// The point is certainly in the region Q of the chains (see above).
__device__ __forceinline__ bool poly_inside(const PolyF& P, double ux, double uy) {
  const unsigned ax = static_cast<unsigned>(__double2hiint(ux)) & 0x7fffffffu;
  const unsigned ay = static_cast<unsigned>(__double2hiint(uy)) & 0x7fffffffu;
  if (max(ax, ay) >= 0x42700000u) return false;  // |coordinate| >= 2^40 or non-finite: outside the FP32 tier
  const float fx = trunc_f32(ux), fy = trunc_f32(uy);
  if (!(fx > P.xl && fx < P.xr)) return false;
  const int ju = chain_edge(P.tu, fx), jl = chain_edge(P.tl, fx);
  if ((ju | jl) < 0) return false;
  const float m = __fadd_ru(fabsf(fx), fabsf(fy));
  float du, eu, dl, el;
  orient_f32(poly_edge(P.eu, ju), fx, fy, m, du, eu);
  orient_f32(poly_edge(P.el, jl), fx, fy, m, dl, el);
  return du < -eu && dl > el;  // certainly below the upper edge and above the lower edge
}

// ---------------------------------------------------------------------------
// Classification of one point against a segment (a, r, b):
// 1 = left of a->r (left child), 2 = left of r->b (right child), 0 = discard.
// key/err: orient of the point w.r.t. its child's line, with a bound
// (|key - exact| <= err).  The FAST variant keeps keys in FP32 so the hot
// loop issues no FP64 instruction unless the filter is inconclusive.
// ---------------------------------------------------------------------------

template <bool FAST>
struct KeyOf { typedef double T; };
template <>
struct KeyOf<true> { typedef float T; };

__device__ __forceinline__ float key_lo(float k, float e) { return __fsub_rd(k, e); }
__device__ __forceinline__ double key_lo(double k, double e) { return __dsub_rd(k, e); }
__device__ __forceinline__ float key_hi(float k, float e) { return __fadd_ru(k, e); }
__device__ __forceinline__ double key_hi(double k, double e) { return __dadd_ru(k, e); }
__device__ __forceinline__ float key_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double key_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float warp_max_k(float v) { return warp_max_f(v); }
__device__ __forceinline__ double warp_max_k(double v) { return warp_max_d(v); }
template <typename T> __device__ __forceinline__ T key_neg_inf();
template <> __device__ __forceinline__ float key_neg_inf<float>() { return -INFINITY; }
template <> __device__ __forceinline__ double key_neg_inf<double>() { return -INFINITY; }

__device__ __forceinline__ int classify_fast(const SegGeom& g, const LineF& l1, const LineF& l2,
                                             double ux, double uy, float& key, float& err) {
  const float fx = trunc_f32(ux), fy = trunc_f32(uy);
  const float m = __fadd_ru(fabsf(fx), fabsf(fy));
  float d1, e1, d2, e2;
  orient_f32(l1, fx, fy, m, d1, e1);
  orient_f32(l2, fx, fy, m, d2, e2);
  int s1 = d1 > e1 ? 1 : (d1 < -e1 ? -1 : 2);
  if (s1 == 2) s1 = orient_sign_slow(g.ax, g.ay, g.rx, g.ry, ux, uy);
  if (s1 > 0) { key = d1; err = e1; return 1; }
  int s2 = d2 > e2 ? 1 : (d2 < -e2 ? -1 : 2);
  if (s2 == 2) s2 = orient_sign_slow(g.rx, g.ry, g.bx, g.by, ux, uy);
  if (s2 > 0) { key = d2; err = e2; return 2; }
  return 0;
}

__device__ __forceinline__ int classify_slow(const SegGeom& g, double ux, double uy, double& key,
                                             double& err) {
  double d1, b1, d2, b2;
  bool sure;
  int s1 = cross_f64(g.ax, g.ay, g.rx, g.ry, g.ax, g.ay, ux, uy, d1, b1, sure);
  if (!sure) s1 = exact_orient_sign(g.ax, g.ay, g.rx, g.ry, ux, uy);
  if (s1 > 0) { key = d1; err = b1; return 1; }
  int s2 = cross_f64(g.rx, g.ry, g.bx, g.by, g.rx, g.ry, ux, uy, d2, b2, sure);
  if (!sure) s2 = exact_orient_sign(g.rx, g.ry, g.bx, g.by, ux, uy);
  if (s2 > 0) { key = d2; err = b2; return 2; }
  return 0;
}

// Filter-only classification (no calls): returns 0, 1, 2 when the filter
// settles both signs it needs, 3 when the exact tiers must decide.
// key/err are set for results 1 and 2.
__device__ __forceinline__ int classify_filter(const SegGeom&, const LineF& l1, const LineF& l2, double ux,
                                               double uy, float& key, float& err) {
  const float fx = trunc_f32(ux), fy = trunc_f32(uy);
  const float m = __fadd_ru(fabsf(fx), fabsf(fy));
  float d1, e1;
  orient_f32(l1, fx, fy, m, d1, e1);
  if (d1 > e1) { key = d1; err = e1; return 1; }
  if (!(d1 < -e1)) return 3;
  float d2, e2;
  orient_f32(l2, fx, fy, m, d2, e2);
  if (d2 > e2) { key = d2; err = e2; return 2; }
  if (!(d2 < -e2)) return 3;
  return 0;
}
__device__ __forceinline__ int classify_filter(const SegGeom& g, const LineF&, const LineF&, double ux, double uy,
                                               double& key, double& err) {
  bool sure;
  const int s1 = cross_f64(g.ax, g.ay, g.rx, g.ry, g.ax, g.ay, ux, uy, key, err, sure);
  if (!sure) return 3;
  if (s1 > 0) return 1;
  const int s2 = cross_f64(g.rx, g.ry, g.bx, g.by, g.rx, g.ry, ux, uy, key, err, sure);
  if (!sure) return 3;
  return s2 > 0 ? 2 : 0;
}

// Exact classification (tiers 2 and 3).  A point coincident with r, a or b
// has orient exactly 0 against the child line through that point, and the
// sign against the other line is fixed by the segment (r strictly left of
// a->b, so orient(r, b, a) = -orient(a, b, r) < 0 and orient(a, r, b) < 0;
// the level-0 segment p->p through q has both orients 0): such a point is
// discarded without the expansions, which the FP64 filter cannot avoid for
// an exact zero (about 33K cycles per call on GB300).
__device__ __forceinline__ int classify_exact(const SegGeom* g, double ux, double uy) {
  if ((ux == g->rx && uy == g->ry) || (ux == g->ax && uy == g->ay) || (ux == g->bx && uy == g->by)) return 0;
  VQ_COUNT_TIER(2);
  if (orient_sign_slow(g->ax, g->ay, g->rx, g->ry, ux, uy) > 0) return 1;
  if (orient_sign_slow(g->rx, g->ry, g->bx, g->by, ux, uy) > 0) return 2;
  return 0;
}

__device__ __forceinline__ int classify_k(const SegGeom& g, const LineF& l1, const LineF& l2,
                                          double ux, double uy, float& key, float& err) {
  return classify_fast(g, l1, l2, ux, uy, key, err);
}
__device__ __forceinline__ int classify_k(const SegGeom& g, const LineF&, const LineF&, double ux,
                                          double uy, double& key, double& err) {
  return classify_slow(g, ux, uy, key, err);
}

// Key and bound of a point for one line only (farthest-point search);
// E = {ox, oy, ex, ey} is read by the FP64 variant only.
__device__ __forceinline__ void line_key_k(const LineF& L, const double*, double ux, double uy, float& key,
                                           float& err) {
  const float fx = trunc_f32(ux), fy = trunc_f32(uy);
  const float m = __fadd_ru(fabsf(fx), fabsf(fy));
  orient_f32(L, fx, fy, m, key, err);
}
__device__ __forceinline__ void line_key_k(const LineF&, const double* E, double ux, double uy, double& key,
                                           double& err) {
  bool sure;
  cross_f64(E[0], E[1], E[2], E[3], E[0], E[1], ux, uy, key, err, sure);
}

// The tighter of the FP32 evaluations: the absolute tier, and when its
// bound is wide next to the value (near-collinear points), the relative
// tier (both bound the same exact value).  The FP64 variant is line_key_k.
__device__ __forceinline__ void line_key_tight(const LineF& L, const double* E, double ux, double uy, float& key,
                                               float& err) {
  line_key_k(L, E, ux, uy, key, err);
  if (err > 0x1p-8f * fabsf(key)) {
    float k2, e2;
    orient_rel(L, E[0], E[1], ux, uy, k2, e2);
    if (e2 < err) {
      key = k2;
      err = e2;
    }
  }
}
__device__ __forceinline__ void line_key_tight(const LineF& L, const double* E, double ux, double uy, double& key,
                                               double& err) {
  line_key_k(L, E, ux, uy, key, err);
}

// Classification by the relative tier (for points the absolute tier left
// undecided): 0, 1, 2 as classify_filter, 3 when it is unsure as well.
__device__ __forceinline__ int classify_rel(const SegGeom& g, const LineF& l1, const LineF& l2, double ux,
                                            double uy, float& key, float& err) {
  VQ_COUNT_TIER(4);
  float d1, e1;
  orient_rel(l1, g.ax, g.ay, ux, uy, d1, e1);
  if (d1 > e1) { key = d1; err = e1; return 1; }
  if (!(d1 < -e1)) return 3;
  float d2, e2;
  orient_rel(l2, g.rx, g.ry, ux, uy, d2, e2);
  if (d2 > e2) { key = d2; err = e2; return 2; }
  if (!(d2 < -e2)) return 3;
  return 0;
}
__device__ __forceinline__ int classify_rel(const SegGeom&, const LineF&, const LineF&, double, double, double&,
                                            double&) {
  return 3;
}

}  // namespace vq
