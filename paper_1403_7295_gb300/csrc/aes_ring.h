// aes_ring.h — byte ranges of one buffer handed out in FIFO order (the
// serving engine's output arena).  Host code only, header-only, no CUDA.
//
// alloc(n) returns the start of a free range of n bytes rounded up to 16, or
// -1 when those bytes are not free.  free() may come out of order (batches
// complete on different streams); the tail advances over every freed range at
// the front.  Ranges never overlap and never leave [0, size).
#pragma once
#include <cstdint>
#include <deque>

namespace aesgpu {

class RingArena {
 public:
  explicit RingArena(uint64_t size) : size_(size) {}

  // A handle: the range's start, size and position in allocation order.
  struct Range {
    uint64_t start = 0, bytes = 0, seq = 0;
  };

  bool alloc(uint64_t nbytes, Range* out) {
    uint64_t n = (nbytes + 15) & ~uint64_t(15);
    if (n < 16) n = 16;
    if (n > size_) return false;
    uint64_t start;
    if (live_.empty()) {
      head_ = 0;
      start = 0;
    } else {
      const uint64_t tail = live_.front().start;
      if (head_ >= tail) {
        if (head_ + n <= size_) start = head_;
        else if (n < tail) start = 0;  // wrap; strict so head != tail while ranges are live
        else return false;
      } else {
        if (head_ + n < tail) start = head_;
        else return false;
      }
    }
    live_.push_back(Entry{start, n, false});
    head_ = start + n;
    used_ += n;
    *out = Range{start, n, first_seq_ + live_.size() - 1};
    return true;
  }

  void free(const Range& r) {
    Entry& e = live_[r.seq - first_seq_];
    e.freed = true;
    used_ -= e.bytes;
    while (!live_.empty() && live_.front().freed) {
      live_.pop_front();
      ++first_seq_;
    }
  }

  uint64_t used() const { return used_; }
  uint64_t size() const { return size_; }
  bool empty() const { return live_.empty(); }

 private:
  struct Entry {
    uint64_t start, bytes;
    bool freed;
  };
  uint64_t size_, head_ = 0, used_ = 0, first_seq_ = 0;
  std::deque<Entry> live_;
};

}  // namespace aesgpu
