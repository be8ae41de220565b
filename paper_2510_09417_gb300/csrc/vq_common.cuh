// vq_common.cuh -- device helpers shared by the kernel translation units
// (vq_kernels.cu, vq_partition.cu): checked-build index validation, the
// fatal-error test, farthest-point candidate records and shared-memory
// addresses.  Inside namespace vq; include after vq_internal.h.
#pragma once

#include "vq_internal.h"

namespace vq {

// Checked builds (VQ_CHECKED=1) validate computed indices before use: a
// failure records its site and value, raises kErrInternal and skips the access.
#ifdef VQ_CHECKED
#define VQ_OK_IDX(w, site, v, lo, hi) vq_check_idx((w), (site), (long long)(v), (long long)(lo), (long long)(hi))
__device__ __forceinline__ bool vq_check_idx(const Work& w, int site, long long v, long long lo, long long hi) {
  if (v >= lo && v < hi) return true;
  if (atomicCAS(&w.ctrl->dbg_site, 0, site) == 0) w.ctrl->dbg_val = v;
  atomicOr(&w.ctrl->err, kErrInternal);
  return false;
}
#else
#define VQ_OK_IDX(w, site, v, lo, hi) true
#endif

// Coordinates of the caller's point i (structure of arrays, or interleaved).
__device__ __forceinline__ double px(const Work& w, long long i) { return w.x[w.aos ? 2 * i : i]; }
__device__ __forceinline__ double py(const Work& w, long long i) { return w.y[w.aos ? 2 * i : i]; }

// Segments of at most this many points are finished in shared memory.  A
// hull-dense set (flag kSegDense: the pre-filter kept more than half of its
// points, so nearly every point is a hull vertex) uses the finisher's full
// capacity: its recursion is as deep as the segment is long, which the
// finisher's rounds take far faster than partition levels.  Only the
// routing changes; the result and the per-level counters do not.
__device__ __forceinline__ int seg_small_max(const Work& w, int flags) {
  return (flags & kSegDense) ? (kK3Cap > w.small_max ? kK3Cap : w.small_max) : w.small_max;
}

__device__ __forceinline__ bool fatal(const Work& w) {
  return (*reinterpret_cast<volatile unsigned*>(&w.ctrl->err) & kErrFatal) != 0;
}

// Running exact argmax of one thread: replace the best when the new point
// beats it (bounds first, exact tiers only when the bounds overlap).
template <typename K>
__device__ __forceinline__ void take_best(CandT<K>& b, const double* L, double x, double y, int idx, K key, K err) {
  const K lo = key_lo(key, err), hi = key_hi(key, err);
  if (b.idx >= 0 && hi < b.lo) return;  // clearly nearer the line
  if (b.idx < 0 || lo > b.hi || beats_exact(L[0], L[1], L[2], L[3], x, y, idx, b.x, b.y, b.idx)) {
    b.x = x; b.y = y; b.lo = lo; b.hi = hi; b.idx = idx;
  }
}
// The same with the line's FP32 constants (the difference tier first).
__device__ __forceinline__ void take_best(CandT<float>& b, const LineF& Lf, const double* L, double x, double y,
                                          int idx, float key, float err) {
  CandT<float> c;
  c.x = x; c.y = y; c.lo = key_lo(key, err); c.hi = key_hi(key, err); c.idx = idx;
  if (cand_beats(Lf, L, c, b)) b = c;
}

template <typename K>
__device__ __forceinline__ CandT<double> to_double(const CandT<K>& c) {
  CandT<double> d;
  d.x = c.x; d.y = c.y; d.lo = widen(c.lo); d.hi = widen(c.hi); d.idx = c.idx;
  return d;
}

__device__ __forceinline__ BestRec to_rec(const CandT<double>& c) {
  BestRec r;
  r.x = c.x; r.y = c.y; r.lo = c.lo; r.hi = c.hi; r.idx = c.idx; r.pad = 0;
  return r;
}
__device__ __forceinline__ CandT<double> from_rec(const BestRec& r) {
  CandT<double> c;
  c.x = r.x; c.y = r.y; c.lo = r.lo; c.hi = r.hi; c.idx = r.idx;
  return c;
}
__device__ __forceinline__ BestRec load_rec(const BestRec* p) {
  BestRec r;
  r.x = __ldcg(&p->x);
  r.y = __ldcg(&p->y);
  r.lo = __ldcg(&p->lo);
  r.hi = __ldcg(&p->hi);
  r.idx = __ldcg(&p->idx);
  r.pad = 0;
  return r;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
}  // namespace vq
