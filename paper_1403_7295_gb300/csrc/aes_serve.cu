// aes_serve.cu — continuous-batching AES-CTR server: requests (tenant, input
// slice, length) arrive over time and run as batches of aes_batch_submit.
// Host code only; every AES step runs in the batch kernels.
//
// One call of aes_server_progress:
//   1. frees the output ranges and budget of the requests it reported last
//      time (their outputs stay readable until then);
//   2. admits waiting requests in arrival order while the budget allows
//      (each is charged its input and output bytes rounded to 16; its output
//      range comes from a ring arena of the budget's size) and gives each the
//      tenant's next counter range (IV = tenant nonce || counter, the counter
//      advanced by the request's blocks, so no keystream block repeats
//      within a tenant until 2^32 blocks);
//   3. launches every admitted request into the next batch as soon as a slot
//      is free (continuous batching: requests that arrive while batches are
//      on the GPU join the next launch): the slot's descriptors go through
//      its pinned staging buffer with one async copy, then the batch call
//      and an event, on the next stream;
//   4. reports batches whose event fired; a batch not complete after
//      batch_timeout_s is declared lost: its requests are reported with
//      AES_ERR_TIMEOUT, its slot and output ranges are quarantined (the GPU
//      might still write them) and admission stops.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <deque>
#include <vector>

#include "aes_ring.h"
#include "aesgpu.h"

namespace aesgpu {
aes_status record_cuda_failure(cudaError_t e);

namespace {

inline uint64_t up16(uint64_t x) { return (x + 15) & ~uint64_t(15); }

struct Req {
  uint64_t id;
  uint32_t tenant;
  uint64_t in_off, length;
  double t_arrival, t_admitted;
  RingArena::Range out;
  uint32_t counter;
};

// A reported completion and the output range it holds until it has been
// handed out and one more step has run.
struct Done {
  aes_server_completion c;
  RingArena::Range out;
  bool owns_range;  // false for a lost batch's request: its range stays quarantined
};

// Descriptor arrays of one batch, in the same layout in pinned host memory
// and on the device.
struct Slot {
  enum { kInOff, kInLen, kOutOff, kOutLen, kSched, kStatus, kIv, kFields };
  uint32_t max = 0;
  size_t off[kFields] = {};
  size_t bytes = 0;
  uint8_t* host = nullptr;
  uint8_t* dev = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaEvent_t ev = nullptr;
  std::vector<Req> reqs;
  int stream = 0;
  double t_launch = 0;
  uint64_t seq = 0;  // 1-based launch number
};

}  // namespace
}  // namespace aesgpu

struct aes_server {
  aes_server_config cfg{};
  const uint8_t* pool = nullptr;
  uint64_t pool_bytes = 0;
  aes_key_schedule* schedules = nullptr;  // device table
  uint32_t n_tenants = 0;
  std::vector<uint8_t> nonces;             // 12 per tenant
  std::vector<uint64_t> counters;          // running block counter per tenant
  uint8_t* out = nullptr;                  // output arena (budget bytes)
  aesgpu::RingArena arena{0};
  uint64_t charged = 0, max_charged = 0;
  std::vector<cudaStream_t> streams;
  int next_stream = 0;
  std::vector<aesgpu::Slot*> all_slots;
  std::deque<aesgpu::Slot*> free_slots, inflight;
  std::vector<aesgpu::Slot*> quarantined;
  std::deque<aesgpu::Req> waiting, admitted;
  std::deque<aesgpu::Done> pending;           // completions not yet handed out
  std::vector<aesgpu::Done> to_free;          // handed out; freed at the start of the next step
  uint64_t launches = 0, submitted = 0, completed = 0, timed_out = 0, overlapped = 0, bytes = 0;
  uint64_t batched_msgs = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
  bool healthy() const { return quarantined.empty(); }
};

namespace aesgpu {
namespace {

void free_reported(aes_server* s) {
  for (const Done& d : s->to_free) {
    if (!d.owns_range) continue;
    s->arena.free(d.out);
    s->charged -= 2 * up16(d.c.length);
  }
  s->to_free.clear();
}

// Hand out one completion: its range is freed at the start of the next step.
aes_server_completion hand_out(aes_server* s) {
  Done d = s->pending.front();
  s->pending.pop_front();
  s->to_free.push_back(d);
  return d.c;
}

void admit(aes_server* s, double now) {
  while (!s->waiting.empty()) {
    Req& r = s->waiting.front();
    const uint64_t cost = 2 * up16(r.length);
    if (s->charged + cost > s->cfg.budget_bytes) break;
    if (!s->arena.alloc(r.length, &r.out)) break;
    s->charged += cost;
    if (s->charged > s->max_charged) s->max_charged = s->charged;
    r.t_admitted = now;
    r.counter = static_cast<uint32_t>(s->counters[r.tenant]);
    s->counters[r.tenant] += (r.length + 15) / 16;
    s->admitted.push_back(r);
    s->waiting.pop_front();
  }
}

// Launch one batch of admitted requests into a free slot; false when either is missing.
aes_status launch(aes_server* s, double now, bool* launched) {
  *launched = false;
  if (s->admitted.empty() || s->free_slots.empty()) return AES_OK;
  Slot* sl = s->free_slots.front();
  s->free_slots.pop_front();
  sl->reqs.clear();
  while (!s->admitted.empty() && sl->reqs.size() < sl->max) {
    sl->reqs.push_back(s->admitted.front());
    s->admitted.pop_front();
  }
  const uint32_t n = static_cast<uint32_t>(sl->reqs.size());
  uint64_t* in_off = reinterpret_cast<uint64_t*>(sl->host + sl->off[Slot::kInOff]);
  uint64_t* in_len = reinterpret_cast<uint64_t*>(sl->host + sl->off[Slot::kInLen]);
  uint64_t* out_off = reinterpret_cast<uint64_t*>(sl->host + sl->off[Slot::kOutOff]);
  uint32_t* sched = reinterpret_cast<uint32_t*>(sl->host + sl->off[Slot::kSched]);
  uint8_t* iv = sl->host + sl->off[Slot::kIv];
  bool in_padded = true;
  for (uint32_t i = 0; i < n; ++i) {
    const Req& r = sl->reqs[i];
    in_off[i] = r.in_off;
    in_len[i] = r.length;
    out_off[i] = r.out.start;
    sched[i] = r.tenant;
    std::memcpy(iv + 16 * i, s->nonces.data() + 12 * r.tenant, 12);
    iv[16 * i + 12] = static_cast<uint8_t>(r.counter >> 24);
    iv[16 * i + 13] = static_cast<uint8_t>(r.counter >> 16);
    iv[16 * i + 14] = static_cast<uint8_t>(r.counter >> 8);
    iv[16 * i + 15] = static_cast<uint8_t>(r.counter);
    if (up16(r.in_off + r.length) > s->pool_bytes) in_padded = false;
  }
  const int si = s->next_stream;
  s->next_stream = (s->next_stream + 1) % static_cast<int>(s->streams.size());
  cudaStream_t st = s->streams[si];
  // one copy of the used part of the staging buffer (the IV field is last)
  cudaError_t e = cudaMemcpyAsync(sl->dev, sl->host, sl->off[Slot::kIv] + 16ull * n, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return record_cuda_failure(e);
  aes_batch b{};
  b.n_msgs = n;
  b.op = AES_BATCH_CTR;
  b.in = s->pool;
  b.out = s->out;
  b.in_off = reinterpret_cast<const uint64_t*>(sl->dev + sl->off[Slot::kInOff]);
  b.in_len = reinterpret_cast<const uint64_t*>(sl->dev + sl->off[Slot::kInLen]);
  b.out_off = reinterpret_cast<const uint64_t*>(sl->dev + sl->off[Slot::kOutOff]);
  b.schedules = s->schedules;
  b.sched_idx = reinterpret_cast<const uint32_t*>(sl->dev + sl->off[Slot::kSched]);
  b.n_schedules = s->n_tenants;
  // outputs sit in 16-byte-rounded ring ranges; inputs may be read to their
  // next 16-byte boundary when the pool holds it
  b.flags = AES_BATCH_OUT_PADDED | (in_padded ? AES_BATCH_IN_PADDED : 0u);
  b.iv = sl->dev + sl->off[Slot::kIv];
  b.out_len = reinterpret_cast<uint64_t*>(sl->dev + sl->off[Slot::kOutLen]);
  b.status = reinterpret_cast<int32_t*>(sl->dev + sl->off[Slot::kStatus]);
  aes_batch_config bc{0, 0, s->cfg.grid_ctas, 0};
  const aes_status as = aes_batch_submit_ex(&b, sl->ws, sl->ws_bytes, st, &bc);
  if (as != AES_OK) return as;
  e = cudaEventRecord(sl->ev, st);
  if (e != cudaSuccess) return record_cuda_failure(e);
  if (!s->inflight.empty()) ++s->overlapped;  // launched while earlier batches are on the GPU
  sl->stream = si;
  sl->t_launch = now;
  sl->seq = ++s->launches;
  s->batched_msgs += n;
  s->inflight.push_back(sl);
  *launched = true;
  return AES_OK;
}

aes_server_completion completion_of(const Req& r, int32_t status, double t_done) {
  aes_server_completion c{};
  c.id = r.id;
  c.status = status;
  c.tenant = r.tenant;
  c.out_off = r.out.start;
  c.length = r.length;
  c.counter = r.counter;
  c.t_arrival = r.t_arrival;
  c.t_admitted = r.t_admitted;
  c.t_done = t_done;
  return c;
}

// Report batches whose event fired; declare lost the ones past the timeout.
aes_status poll(aes_server* s) {
  for (auto it = s->inflight.begin(); it != s->inflight.end();) {
    Slot* sl = *it;
    const bool injected_lost = s->cfg.inject_lost_batch != 0 && sl->seq == s->cfg.inject_lost_batch;
    cudaError_t e = injected_lost ? cudaErrorNotReady : cudaEventQuery(sl->ev);
    const double t = s->now();
    if (e == cudaErrorNotReady) {
      if (t - sl->t_launch > s->cfg.batch_timeout_s) {  // lost: quarantine, report, stop admitting
        for (const Req& r : sl->reqs) {
          s->pending.push_back(Done{completion_of(r, AES_ERR_TIMEOUT, -2.0), r.out, false});
          ++s->timed_out;
        }
        s->quarantined.push_back(sl);
        it = s->inflight.erase(it);
      } else {
        ++it;
      }
      continue;
    }
    if (e != cudaSuccess) return record_cuda_failure(e);
    for (const Req& r : sl->reqs) {
      s->pending.push_back(Done{completion_of(r, AES_OK, t), r.out, true});
      ++s->completed;
      s->bytes += r.length;
    }
    sl->reqs.clear();
    s->free_slots.push_back(sl);
    it = s->inflight.erase(it);
  }
  return AES_OK;
}

// One pass of the loop; completions go to s->pending.
aes_status step(aes_server* s) {
  free_reported(s);
  const double now = s->now();
  if (s->healthy()) {
    admit(s, now);
    for (;;) {
      bool launched = false;
      const aes_status st = launch(s, now, &launched);
      if (st != AES_OK) return st;
      if (!launched) break;
    }
  }
  return poll(s);
}

void release(aes_server* s) {
  for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
  for (Slot* sl : s->all_slots) {
    if (sl->ev) cudaEventDestroy(sl->ev);
    if (sl->host) cudaFreeHost(sl->host);
    if (sl->dev) cudaFree(sl->dev);
    if (sl->ws) cudaFree(sl->ws);
    delete sl;
  }
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  if (s->out) cudaFree(s->out);
  if (s->schedules) cudaFree(s->schedules);
  delete s;
}

}  // namespace
}  // namespace aesgpu

extern "C" {

aes_status aes_server_create(const aes_server_config* cfg, const void* d_pool, uint64_t pool_bytes,
                             const aes_key_schedule* schedules, const uint8_t* nonces, uint32_t n_tenants,
                             aes_server** out) {
  using namespace aesgpu;
  if (out == nullptr || d_pool == nullptr || schedules == nullptr || nonces == nullptr || n_tenants == 0)
    return AES_ERR_ARG;
  *out = nullptr;
  aes_server* s = new aes_server;
  if (cfg) s->cfg = *cfg;
  if (s->cfg.budget_bytes == 0) s->cfg.budget_bytes = 8ull << 30;
  if (s->cfg.n_streams == 0) s->cfg.n_streams = 2;
  if (s->cfg.slots_per_stream == 0) s->cfg.slots_per_stream = 2;
  if (s->cfg.max_batch_msgs == 0) s->cfg.max_batch_msgs = 8192;
  if (s->cfg.batch_timeout_s <= 0) s->cfg.batch_timeout_s = 10.0;
  if (s->cfg.n_streams > 64 || s->cfg.slots_per_stream > 64 || s->cfg.max_batch_msgs > (1u << 24)) {
    delete s;
    return AES_ERR_ARG;
  }
  s->pool = static_cast<const uint8_t*>(d_pool);
  s->pool_bytes = pool_bytes;
  s->n_tenants = n_tenants;
  s->nonces.assign(nonces, nonces + 12ull * n_tenants);
  s->counters.assign(n_tenants, 0);
  s->arena = RingArena(s->cfg.budget_bytes);
  cudaError_t e = cudaMalloc(&s->schedules, sizeof(aes_key_schedule) * n_tenants);
  if (e == cudaSuccess)
    e = cudaMemcpy(s->schedules, schedules, sizeof(aes_key_schedule) * n_tenants, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&s->out, s->cfg.budget_bytes);
  for (uint32_t i = 0; i < s->cfg.n_streams && e == cudaSuccess; ++i) {
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) s->streams.push_back(st);
  }
  const uint32_t nslots = s->cfg.n_streams * s->cfg.slots_per_stream;
  for (uint32_t i = 0; i < nslots && e == cudaSuccess; ++i) {
    Slot* sl = new Slot;
    s->all_slots.push_back(sl);
    sl->max = s->cfg.max_batch_msgs;
    const size_t widths[Slot::kFields] = {8, 8, 8, 8, 4, 4, 16};
    size_t off = 0;
    for (int f = 0; f < Slot::kFields; ++f) {
      sl->off[f] = off;
      off = up16(off + widths[f] * sl->max);
    }
    sl->bytes = off;
    sl->ws_bytes = aes_batch_workspace_size(sl->max);
    e = cudaHostAlloc(reinterpret_cast<void**>(&sl->host), sl->bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&sl->dev, sl->bytes);
    if (e == cudaSuccess) e = cudaMalloc(&sl->ws, sl->ws_bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) s->free_slots.push_back(sl);
  }
  if (e != cudaSuccess) {
    release(s);
    return record_cuda_failure(e);
  }
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return AES_OK;
}

void aes_server_destroy(aes_server* s) {
  if (s) aesgpu::release(s);
}

aes_status aes_server_submit(aes_server* s, uint64_t id, uint32_t tenant, uint64_t in_off, uint64_t length) {
  if (s == nullptr || tenant >= s->n_tenants || (in_off & 15u) != 0 || in_off + length > s->pool_bytes)
    return AES_ERR_ARG;
  if (2 * aesgpu::up16(length) > s->cfg.budget_bytes) return AES_ERR_NOMEM;  // could never be admitted
  s->waiting.push_back(aesgpu::Req{id, tenant, in_off, length, s->now(), -1.0, {}, 0});
  ++s->submitted;
  return AES_OK;
}

uint32_t aes_server_progress(aes_server* s, aes_server_completion* done, uint32_t max_done, aes_status* status) {
  if (status) *status = AES_OK;
  if (s == nullptr) {
    if (status) *status = AES_ERR_ARG;
    return 0;
  }
  const aes_status st = aesgpu::step(s);
  if (status) *status = st;
  uint32_t k = 0;
  while (k < max_done && done != nullptr && !s->pending.empty()) done[k++] = aesgpu::hand_out(s);
  return k;
}

int aes_server_healthy(const aes_server* s) { return s && s->healthy() ? 1 : 0; }

int aes_server_idle(const aes_server* s) {  // nothing waiting, queued, on the GPU or unreported
  return s && s->waiting.empty() && s->admitted.empty() && s->inflight.empty() && s->pending.empty() ? 1 : 0;
}

void* aes_server_output(aes_server* s) { return s ? s->out : nullptr; }

double aes_server_now(const aes_server* s) { return s ? s->now() : 0.0; }

void aes_server_get_stats(const aes_server* s, aes_server_stats* st) {
  if (s == nullptr || st == nullptr) return;
  *st = aes_server_stats{};
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->timed_out = s->timed_out;
  st->batches = s->launches;
  st->batches_overlapped = s->overlapped;
  st->bytes = s->bytes;
  st->max_charged = s->max_charged;
  st->mean_batch_msgs = s->launches ? static_cast<double>(s->batched_msgs) / s->launches : 0.0;
}

aes_status aes_server_replay(aes_server* s, uint64_t n, const double* arrival_s, const uint32_t* tenants,
                             const uint64_t* in_offs, const uint64_t* lengths, double time_limit_s,
                             double* latency_s, double* wait_s, uint32_t* counters, void* capture,
                             const uint64_t* capture_off) {
  using namespace aesgpu;
  if (s == nullptr || (n && (arrival_s == nullptr || tenants == nullptr || in_offs == nullptr || lengths == nullptr)))
    return AES_ERR_ARG;
  for (uint64_t i = 0; i < n; ++i) {
    if (tenants[i] >= s->n_tenants || (in_offs[i] & 15u) || in_offs[i] + lengths[i] > s->pool_bytes ||
        2 * up16(lengths[i]) > s->cfg.budget_bytes)
      return AES_ERR_ARG;
    if (latency_s) latency_s[i] = -1.0;
    if (wait_s) wait_s[i] = -1.0;
  }
  const double start = s->now();
  uint64_t next = 0;
  aes_status result = AES_OK;
  std::vector<aes_server_completion> done;
  cudaStream_t copy_stream = s->streams.empty() ? nullptr : s->streams[0];
  for (;;) {
    const double now = s->now() - start;
    while (next < n && arrival_s[next] <= now) {
      s->waiting.push_back(Req{next, tenants[next], in_offs[next], lengths[next], start + arrival_s[next], -1.0,
                               {}, 0});
      ++s->submitted;
      ++next;
    }
    result = step(s);
    if (result != AES_OK) break;
    while (!s->pending.empty()) {
      const aes_server_completion c = hand_out(s);
      const uint64_t i = c.id;
      if (i < n) {
        if (c.status == AES_OK) {
          if (latency_s) latency_s[i] = c.t_done - c.t_arrival;
          if (capture && capture_off && capture_off[i] != UINT64_MAX) {  // a copy before the range is reused
            cudaError_t e = cudaMemcpyAsync(static_cast<uint8_t*>(capture) + capture_off[i], s->out + c.out_off,
                                            c.length, cudaMemcpyDeviceToDevice, copy_stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(copy_stream);
            if (e != cudaSuccess) {
              result = record_cuda_failure(e);
              break;
            }
          }
        } else if (latency_s) {
          latency_s[i] = -2.0;  // timed out
        }
        if (wait_s && c.t_admitted >= 0) wait_s[i] = c.t_admitted - c.t_arrival;
        if (counters) counters[i] = c.counter;
      }
    }
    if (result != AES_OK) break;
    const bool busy = !s->waiting.empty() || !s->admitted.empty() || !s->inflight.empty();
    if (next >= n && !busy) break;
    if (!s->healthy() && s->inflight.empty()) break;  // a batch was lost: report instead of waiting forever
    if (s->now() - start > time_limit_s) break;
  }
  for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
  free_reported(s);
  return result;
}

}  // extern "C"
