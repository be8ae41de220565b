// vq_admit.h -- admission policy of the serving handle (host code only, no
// CUDA): which queued requests an idle lane takes as its next batch.
#pragma once

#include <cstddef>
#include <cstdint>

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

}  // namespace vq
