// Host-only check of the serving handle's admission policy (vq_admit.h):
// prints one line per case, "name k points bytes"; the test compares them
// with the expected values.
#include <cstdio>

#include "vq_admit.h"

static size_t model_bytes(long long points, int sets) { return (size_t)(68 * points + 1000 * sets); }

static void run(const char* name, const int64_t* sizes, int nq, long long resident, size_t used, long long slots,
                size_t budget, size_t reserve = 0) {
  long long pts = -1;
  size_t bytes = 0;
  const int k = vq::admit_prefix(sizes, nq, resident, used, reserve, slots, budget, model_bytes, &pts, &bytes);
  std::printf("%s %d %lld %zu\n", name, k, pts, bytes);
}

int main() {
  const int64_t q[4] = {100, 200, 300, 400};
  run("all", q, 4, 0, 0, 64, 1u << 30);               // everything fits
  run("slots", q, 4, 1, 0, 3, 1u << 30);              // two slots left
  run("no_slot", q, 4, 3, 0, 3, 1u << 30);            // none left
  run("budget", q, 4, 0, 0, 64, 68 * 300 + 2000);     // the first two fit exactly
  run("head_too_big", q, 4, 0, 100000, 64, 100500);   // memory in use leaves too little
  run("empty", q, 0, 0, 0, 64, 1u << 30);
  // the fixed reserve counts against the budget: the first two fit exactly
  // with it, one byte less leaves room for the first only
  run("reserve_fits", q, 4, 0, 5000, 64, 5000 + 68 * 300 + 2000 + 4096, 4096);
  run("reserve_short", q, 4, 0, 5000, 64, 5000 + 68 * 300 + 2000 + 4095, 4096);
  // a lane's batch: the head and what follows while the batch holds at most
  // max(cap, head) points
  {
    const int64_t b[5] = {100, 200, 300, 5000, 50};
    long long bp = -1;
    int j = vq::batch_prefix(b, 5, 600, &bp);
    std::printf("batch_cap %d %lld\n", j, bp);  // 100 + 200 + 300 = 600 fits, 5000 does not
    j = vq::batch_prefix(b + 3, 2, 600, &bp);
    std::printf("batch_big_head %d %lld\n", j, bp);  // 5000 alone (5050 > max(600, 5000))
    j = vq::batch_prefix(b, 5, 1 << 20, &bp);
    std::printf("batch_all %d %lld\n", j, bp);
    j = vq::batch_prefix(b, 0, 600, &bp);
    std::printf("batch_none %d %lld\n", j, bp);
  }
  // pinned staging extents: first fit, merging on return
  vq::Extents e;
  e.give(0, 1000);
  size_t a = 0, b = 0, c = 0, d = 0;
  const bool ta = e.take(300, &a), tb = e.take(300, &b), tc = e.take(300, &c), td = e.take(300, &d);
  std::printf("ext_take %d %d %d %d %zu %zu %zu %zu\n", ta, tb, tc, td, a, b, c, e.largest());
  e.give(b, 300);  // a hole in the middle
  size_t f = 0;
  const bool tf = e.take(301, &f);
  std::printf("ext_hole %d %zu %zu\n", tf, e.extents(), e.largest());
  e.give(a, 300);
  e.give(c, 300);  // all free again: one extent
  std::printf("ext_merge %zu %zu\n", e.extents(), e.largest());
  return 0;
}
