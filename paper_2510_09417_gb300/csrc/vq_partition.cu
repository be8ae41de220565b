// vq_partition.cu -- the streaming partition kernel's instantiations and
// launcher (the kernel itself is in vq_partition.cuh): points per lane
// (PPT), and per PPT three block shapes (warps per block, ring stages), a
// runtime choice (vq_config.k1_shape) that the autotuner explores.  A
// translation unit of its own so that it compiles beside vq_kernels.cu.
#include <climits>

#include "vq_internal.h"
#include "vq_common.cuh"

namespace vq {

#include "vq_partition.cuh"

namespace {

int sm_count() {
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

// Block shapes per points-per-lane: shape 0 is the default.
template <int PPT, int S>
struct Shape;
template <> struct Shape<4, 0> { static constexpr int WPB = 4, NS = 4; };
template <> struct Shape<4, 1> { static constexpr int WPB = 8, NS = 3; };
template <> struct Shape<4, 2> { static constexpr int WPB = 2, NS = 6; };
template <> struct Shape<8, 0> { static constexpr int WPB = 4, NS = 3; };
template <> struct Shape<8, 1> { static constexpr int WPB = 8, NS = 2; };
template <> struct Shape<8, 2> { static constexpr int WPB = 2, NS = 4; };
template <> struct Shape<16, 0> { static constexpr int WPB = 4, NS = 2; };
template <> struct Shape<16, 1> { static constexpr int WPB = 8, NS = 2; };
template <> struct Shape<16, 2> { static constexpr int WPB = 2, NS = 3; };

// Resident blocks per SM of both source variants (shared memory and the
// register floor of K1W::MINB), once per device.
template <int PPT, int S, bool ALLFAST>
int blocks_per_sm() {
  constexpr int WPB = Shape<PPT, S>::WPB, NS = Shape<PPT, S>::NS;
  typedef K1W<PPT, WPB, NS> C;
  static int occ[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  if (occ[dev] > 0) return occ[dev];
  if (cudaFuncSetAttribute(k_k1w<PPT, WPB, NS, true, ALLFAST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)C::smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_k1w<PPT, WPB, NS, false, ALLFAST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)C::smem) != cudaSuccess)
    return -1;
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_k1w<PPT, WPB, NS, true, ALLFAST>, 32 * WPB, C::smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_k1w<PPT, WPB, NS, false, ALLFAST>, 32 * WPB, C::smem) !=
          cudaSuccess)
    return -1;
  const int n = a < b ? a : b;
  occ[dev] = n > 0 ? n : 1;
  return occ[dev];
}

// A persistent grid: as many blocks as are resident, fewer when the level
// has fewer tiles than warps.
template <int PPT, int S, bool ALLFAST>
cudaError_t launch_one(const Work& w, int level, int tiles, cudaStream_t st) {
  constexpr int WPB = Shape<PPT, S>::WPB, NS = Shape<PPT, S>::NS;
  typedef K1W<PPT, WPB, NS> C;
  if (w.tile != C::TW) return cudaErrorInvalidValue;
  const int occ = blocks_per_sm<PPT, S, ALLFAST>();
  if (occ < 0) return cudaErrorInvalidConfiguration;
  long long grid = (long long)occ * sm_count();
  const long long need = ((long long)tiles + WPB - 1) / WPB;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  count_launches(1);
  if (level == 0 && !w.sieve)
    k_k1w<PPT, WPB, NS, true, ALLFAST><<<(unsigned)grid, 32 * WPB, C::smem, st>>>(w.dev, level, w.tier_dev);
  else
    k_k1w<PPT, WPB, NS, false, ALLFAST><<<(unsigned)grid, 32 * WPB, C::smem, st>>>(w.dev, level, w.tier_dev);
  return cudaGetLastError();
}

// The tier: FP32-only kernel or both tiers, chosen by the host's copy of the
// flag, or both launched when the device picks (Work::tier_dev).
template <int PPT, int S>
cudaError_t launch_tier(const Work& w, int level, int tiles, cudaStream_t st) {
  if (w.tier_dev) {
    const cudaError_t e = launch_one<PPT, S, true>(w, level, tiles, st);
    return e != cudaSuccess ? e : launch_one<PPT, S, false>(w, level, tiles, st);
  }
  return w.all_fast ? launch_one<PPT, S, true>(w, level, tiles, st) : launch_one<PPT, S, false>(w, level, tiles, st);
}

template <int PPT>
cudaError_t launch_shape(const Work& w, int level, int tiles, cudaStream_t st) {
  switch (w.k1_shape) {
    case 0: return launch_tier<PPT, 0>(w, level, tiles, st);
    case 1: return launch_tier<PPT, 1>(w, level, tiles, st);
    case 2: return launch_tier<PPT, 2>(w, level, tiles, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_k1w(const Work& w, int level, int ppt, int tiles, cudaStream_t st) {
  switch (ppt) {
    case 4: return launch_shape<4>(w, level, tiles, st);
    case 8: return launch_shape<8>(w, level, tiles, st);
    case 16: return launch_shape<16>(w, level, tiles, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace vq
