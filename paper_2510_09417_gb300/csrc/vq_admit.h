// vq_admit.h -- host-side policies of the serving handle (no CUDA): which
// queued requests an idle lane takes as its next batch, and the first-fit
// extents of the pinned area that stages submitted points.
#pragma once

#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace vq {

// The longest prefix of the FIFO queue (sizes[0], in points, is the head)
// that keeps the resident requests plus the batch within max_inflight and
// the server's fixed reserve plus the device bytes in use plus the batch's
// bytes, bytes(points, sets), within the budget.  Returns its length, 0
// when the head alone does not fit; *batch_points and *batch_bytes describe
// the prefix.
template <class BytesFn>
inline int admit_prefix(const int64_t* sizes, int nqueued, long long resident, size_t used, size_t reserve,
                        long long max_inflight, size_t budget, BytesFn bytes, long long* batch_points,
                        size_t* batch_bytes) {
  int k = 0;
  long long pts = 0;
  size_t b = 0;
  while (k < nqueued && resident + k < max_inflight) {
    const size_t b2 = bytes(pts + sizes[k], k + 1);
    if (reserve + used + b2 > budget) break;
    pts += sizes[k];
    b = b2;
    k++;
  }
  *batch_points = pts;
  *batch_bytes = b;
  return k;
}

// The batch a lane runs: of an admissible prefix of k requests, the head
// and the requests after it while the batch holds at most max(cap_points,
// the head's points) points, so that small requests share level steps and
// a big request does not hold small ones back behind it.  Returns the
// batch's length (1 <= result <= k when k >= 1) and its points.
inline int batch_prefix(const int64_t* sizes, int k, long long cap_points, long long* batch_points) {
  if (k <= 0) {
    *batch_points = 0;
    return 0;
  }
  const long long cap = cap_points > sizes[0] ? cap_points : (long long)sizes[0];
  long long pts = sizes[0];
  int j = 1;
  while (j < k && pts + sizes[j] <= cap) pts += sizes[j++];
  *batch_points = pts;
  return j;
}

// Free extents of a staging area (offset -> bytes): first-fit takes, and
// returns merged with their free neighbours.
class Extents {
 public:
  // an extent of `bytes` at *off; false when no free extent is that large
  bool take(size_t bytes, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes, at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      return true;
    }
    return false;
  }
  void give(size_t off, size_t bytes) {
    if (!bytes) return;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  size_t extents() const { return free_.size(); }
  size_t largest() const {
    size_t m = 0;
    for (const auto& kv : free_) m = kv.second > m ? kv.second : m;
    return m;
  }

 private:
  std::map<size_t, size_t> free_;
};

}  // namespace vq
