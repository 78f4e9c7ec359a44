// Host test of the serving engine's ring arena (paper_1403_7295_gb300/csrc/aes_ring.h):
// random alloc/free sequences never hand out overlapping or out-of-range
// bytes, account every byte, free out of order, and refuse what does not fit.
// Exit status 0 = every check held.
#include <cstdio>
#include <random>
#include <vector>

#include "aes_ring.h"

#define CHECK(x) do { if (!(x)) { std::fprintf(stderr, "check failed: %s (line %d)\n", #x, __LINE__); return 1; } } while (0)

int main() {
  std::mt19937_64 rng(0);
  for (uint64_t size : {uint64_t(256), uint64_t(4096), uint64_t(1) << 20}) {
    aesgpu::RingArena ar(size);
    std::vector<aesgpu::RingArena::Range> live;
    for (int step = 0; step < 20000; ++step) {
      if (!live.empty() && (rng() % 100 < 45 || live.size() > 50)) {
        const size_t k = rng() % (live.size() < 4 ? live.size() : 4);  // mostly oldest first
        ar.free(live[k]);
        live.erase(live.begin() + k);
      } else {
        const uint64_t n = 1 + rng() % (size / 4 + 1);
        aesgpu::RingArena::Range r;
        if (!ar.alloc(n, &r)) continue;
        CHECK(r.start + r.bytes <= size && r.bytes >= n && r.start % 16 == 0);
        for (const auto& o : live) CHECK(r.start + r.bytes <= o.start || o.start + o.bytes <= r.start);
        live.push_back(r);
      }
      uint64_t sum = 0;
      for (const auto& o : live) sum += o.bytes;
      CHECK(ar.used() == sum);
    }
    for (const auto& o : live) ar.free(o);
    CHECK(ar.used() == 0 && ar.empty());
  }
  aesgpu::RingArena ar(1024);
  aesgpu::RingArena::Range a, b, c, d;
  CHECK(!ar.alloc(2048, &d));
  CHECK(ar.alloc(512, &a) && ar.alloc(400, &b));
  CHECK(!ar.alloc(200, &d));  // 112 bytes left at the end, the front is live
  ar.free(a);
  CHECK(ar.alloc(200, &c) && c.start == 0);  // wraps to the front
  ar.free(b);
  ar.free(c);
  CHECK(ar.used() == 0);
  std::printf("ring ok\n");
  return 0;
}
