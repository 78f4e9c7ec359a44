// aes_file.cu — aes_file_crypt: a file in, the encrypted file out (the
// paper's workload, §IV), as a pipeline of worker threads over chunks.  Host
// code only; the cipher runs through the library's own single-buffer path.
//
// Direct path (opt-in, AES_FILE_DIRECT; the device reads and writes pageable
// host memory through the host's page tables): both files are mapped, each worker faults in its
// chunk's pages and launches the cipher on the mappings themselves, so no
// byte is copied on the host.  On the GB300 host the kernel moves mapped
// file pages over NVLink-C2C as fast as pinned buffers (about 170 GB/s each
// way).
//
// Staged path (the default): input chunks are read with pread at their offsets
// into pinned buffers (parallel reads of one file scale with the threads),
// the kernel runs on the pinned buffer in place, and output chunks are
// copied into a shared mapping of dst: writes to one file through
// write/pwrite are serialised by the kernel's per-file lock (about 12 GB/s
// on the GB300 host whatever the thread count), while stores into a shared
// mapping fault pages in parallel (88 GB/s with 16 threads).  When dst
// cannot be mapped the workers fall back to pwrite.
#include <cuda_runtime.h>
#include <fcntl.h>
#include <sys/mman.h>
#include <sys/stat.h>
#include <unistd.h>

#include <atomic>
#include <cerrno>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "aesgpu.h"

#ifndef MADV_POPULATE_READ
#define MADV_POPULATE_READ 22
#endif
#ifndef MADV_POPULATE_WRITE
#define MADV_POPULATE_WRITE 23
#endif

namespace aesgpu {
aes_status record_cuda_failure(cudaError_t e);
bool host_pageable_access();
aes_status crypt_mapped(int mode, const aes_key_schedule* ks, const uint8_t* iv, const void* in, void* out,
                        size_t nbytes, cudaStream_t stream);

namespace {

constexpr uint64_t kDefaultChunk = 4ull << 20;         // staged path: one pinned buffer per worker
constexpr uint64_t kDefaultDirectChunk = 64ull << 20;  // direct path: fewer launches, same page faults
constexpr int kMaxThreads = 64;
constexpr size_t kPoolMax = 64;  // pinned buffers kept between calls

// Pinned chunk buffers kept between calls: pinning host memory costs about
// 1 ms per MiB-buffer on the GB300 host, a sixth of a 4 GiB file's time.
// Keyed by device and size (sizes are rounded up to whole MiB); the oldest
// entries are freed beyond kPoolMax; aes_file_trim() frees them all.
struct PinnedBuf {
  int device;
  uint64_t bytes;
  uint8_t* p;
};
struct PinnedPool {
  std::mutex mu;
  std::deque<PinnedBuf> free;
};
PinnedPool& pinned_pool() {
  static PinnedPool* pool = new PinnedPool;  // never destroyed: no teardown-order issue at exit
  return *pool;
}

cudaError_t pinned_take(int device, uint64_t bytes, uint8_t** out) {
  {
    PinnedPool& pool = pinned_pool();
    std::lock_guard<std::mutex> lock(pool.mu);
    for (auto it = pool.free.begin(); it != pool.free.end(); ++it) {
      if (it->device == device && it->bytes == bytes) {
        *out = it->p;
        pool.free.erase(it);
        return cudaSuccess;
      }
    }
  }
  return cudaHostAlloc(reinterpret_cast<void**>(out), bytes, cudaHostAllocMapped);
}

void pinned_give(int device, uint64_t bytes, uint8_t* p) {
  std::vector<uint8_t*> evict;
  {
    PinnedPool& pool = pinned_pool();
    std::lock_guard<std::mutex> lock(pool.mu);
    pool.free.push_back(PinnedBuf{device, bytes, p});
    while (pool.free.size() > kPoolMax) {
      evict.push_back(pool.free.front().p);
      pool.free.pop_front();
    }
  }
  for (uint8_t* q : evict) cudaFreeHost(q);
}

// Everything the workers share.  The first failure wins; the others stop at
// their next chunk.
struct FileJob {
  int fd_in = -1, fd_out = -1;
  uint64_t size = 0, chunk = 0, nchunks = 0;
  aes_file_mode mode = AES_FILE_CTR;
  const aes_key_schedule* ks = nullptr;
  uint8_t iv[16] = {};
  int device = 0;
  uint8_t* map = nullptr;        // shared mapping of dst, or null: pwrite
  const uint8_t* src_map = nullptr;  // direct path: mapping of src (== map in place)
  uint64_t page = 4096;
  std::atomic<uint64_t> next{0};
  std::atomic<int> status{AES_OK};
  std::atomic<int> os_errno{0};
  std::atomic<int> cuda_error{0};

  void fail(aes_status s, int err = 0, cudaError_t ce = cudaSuccess) {
    int expected = AES_OK;
    if (status.compare_exchange_strong(expected, s)) {
      os_errno.store(err);
      cuda_error.store(static_cast<int>(ce));
    }
  }
};

// The IV of the chunk starting `blocks` blocks into the file: the library's
// aes_ctr_iv_advance (counter in bytes 12..15 advanced modulo 2^32).
void iv_at(const uint8_t iv[16], uint64_t blocks, uint8_t out[16]) { aes_ctr_iv_advance(iv, blocks, out); }

bool read_full(int fd, uint8_t* p, uint64_t n, uint64_t off, int* err) {
  while (n > 0) {
    const ssize_t r = pread(fd, p, n, static_cast<off_t>(off));
    if (r < 0 && errno == EINTR) continue;
    if (r <= 0) {
      *err = r < 0 ? errno : EIO;  // a file that shrank under us reads short
      return false;
    }
    p += r;
    off += static_cast<uint64_t>(r);
    n -= static_cast<uint64_t>(r);
  }
  return true;
}

bool write_full(int fd, const uint8_t* p, uint64_t n, uint64_t off, int* err) {
  while (n > 0) {
    const ssize_t w = pwrite(fd, p, n, static_cast<off_t>(off));
    if (w < 0 && errno == EINTR) continue;
    if (w <= 0) {
      *err = w < 0 ? errno : EIO;
      return false;
    }
    p += w;
    off += static_cast<uint64_t>(w);
    n -= static_cast<uint64_t>(w);
  }
  return true;
}

// One worker: its pinned buffer and stream, then chunks until none are left
// or another worker failed.
void worker(FileJob* job, uint8_t* buf, cudaStream_t stream) {
  cudaError_t ce = cudaSetDevice(job->device);
  if (ce != cudaSuccess) {
    job->fail(AES_ERR_CUDA, 0, ce);
    return;
  }
  for (;;) {
    if (job->status.load() != AES_OK) return;
    const uint64_t c = job->next.fetch_add(1);
    if (c >= job->nchunks) return;
    const uint64_t off = c * job->chunk;
    const uint64_t n = job->size - off < job->chunk ? job->size - off : job->chunk;
    int err = 0;
    if (!read_full(job->fd_in, buf, n, off, &err)) {
      job->fail(AES_ERR_IO, err);
      return;
    }
    aes_status s;
    if (job->mode == AES_FILE_CTR) {
      uint8_t ivc[16];
      iv_at(job->iv, off / 16, ivc);
      s = aes_ctr_xcrypt(job->ks, ivc, buf, buf, n, stream);
    } else if (job->mode == AES_FILE_ECB_ENCRYPT) {
      s = aes_ecb_encrypt(job->ks, buf, buf, n, stream);
    } else {
      s = aes_ecb_decrypt(job->ks, buf, buf, n, stream);
    }
    if (s != AES_OK) {
      job->fail(s, 0, s == AES_ERR_CUDA ? static_cast<cudaError_t>(aes_last_cuda_error()) : cudaSuccess);
      return;
    }
    ce = cudaStreamSynchronize(stream);
    if (ce != cudaSuccess) {
      job->fail(AES_ERR_CUDA, 0, ce);
      return;
    }
    if (job->map) {
      std::memcpy(job->map + off, buf, n);
    } else if (!write_full(job->fd_out, buf, n, off, &err)) {
      job->fail(AES_ERR_IO, err);
      return;
    }
  }
}

// How a worker faults in its chunk's pages before the device touches them.
enum class Fault {
  kRead,        // src pages: MADV_POPULATE_READ
  kWrite,       // dst pages holding data (in place): MADV_POPULATE_WRITE, which keeps every byte
  kWriteOwned,  // dst pages the device is about to overwrite: store 0 into the first byte of
                // each page inside the range (one write fault per page: about 110 GB/s for new
                // tmpfs pages on the GB300 host, against 30-45 for MADV_POPULATE_WRITE)
};

// Fault in the pages holding [off, off + n) of a mapping of map_len bytes,
// so the device never meets a missing page.  Only bytes inside the range are
// ever stored to: those outside may belong to a chunk in flight.  Kernels
// without MADV_POPULATE_* get one access per page instead (a read, or a
// store of the byte's own value).
bool populate(const uint8_t* base, uint64_t off, uint64_t n, uint64_t map_len, uint64_t page, Fault how,
              int* err) {
  volatile uint8_t* b = const_cast<volatile uint8_t*>(base);
  if (how == Fault::kWriteOwned) {
    for (uint64_t a = off; a < off + n; a = (a / page + 1) * page) b[a] = 0;
    return true;
  }
  const uint64_t lo = off / page * page;
  const uint64_t end = (map_len + page - 1) / page * page;
  uint64_t hi = (off + n + page - 1) / page * page;
  if (hi > end) hi = end;
  const int advice = how == Fault::kRead ? MADV_POPULATE_READ : MADV_POPULATE_WRITE;
  if (madvise(const_cast<uint8_t*>(base) + lo, hi - lo, advice) == 0) return true;
  if (errno != EINVAL) {  // EFAULT / ENOMEM / EHWPOISON: the pages cannot be had
    *err = errno;
    return false;
  }
  for (uint64_t a = off; a < off + n; a = (a / page + 1) * page) {
    if (how == Fault::kWrite) b[a] = b[a];
    else (void)b[a];
  }
  return true;
}

// One direct-path worker: chunks until none are left or another worker
// failed, each launched on the mappings once its pages are in; then its
// stream is drained.
void worker_direct(FileJob* job, cudaStream_t stream) {
  cudaError_t ce = cudaSetDevice(job->device);
  if (ce != cudaSuccess) {
    job->fail(AES_ERR_CUDA, 0, ce);
    return;
  }
  const bool in_place = job->src_map == job->map;
  for (;;) {
    if (job->status.load() != AES_OK) break;
    const uint64_t c = job->next.fetch_add(1);
    if (c >= job->nchunks) break;
    const uint64_t off = c * job->chunk;
    const uint64_t n = job->size - off < job->chunk ? job->size - off : job->chunk;
    int err = 0;
    const bool ok = in_place ? populate(job->map, off, n, job->size, job->page, Fault::kWrite, &err)
                             : populate(job->src_map, off, n, job->size, job->page, Fault::kRead, &err) &&
                                   populate(job->map, off, n, job->size, job->page, Fault::kWriteOwned, &err);
    if (!ok) {
      job->fail(AES_ERR_IO, err);
      break;
    }
    uint8_t ivc[16];
    if (job->mode == AES_FILE_CTR) iv_at(job->iv, off / 16, ivc);
    const aes_status s = crypt_mapped(job->mode, job->ks, job->mode == AES_FILE_CTR ? ivc : nullptr,
                                      job->src_map + off, job->map + off, n, stream);
    if (s != AES_OK) {
      job->fail(s, 0, s == AES_ERR_CUDA ? static_cast<cudaError_t>(aes_last_cuda_error()) : cudaSuccess);
      break;
    }
  }
  ce = cudaStreamSynchronize(stream);  // every launch above reads and writes the mappings
  if (ce != cudaSuccess) job->fail(AES_ERR_CUDA, 0, ce);
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace aesgpu

extern "C" aes_status aes_file_crypt(const char* src_path, const char* dst_path, aes_file_mode mode,
                                     const aes_key_schedule* ks, const uint8_t iv[16],
                                     const aes_file_config* cfg, aes_file_stats* stats) {
  using namespace aesgpu;
  const auto t0 = std::chrono::steady_clock::now();
  if (stats) *stats = aes_file_stats{};
  if (src_path == nullptr || dst_path == nullptr || ks == nullptr) return AES_ERR_ARG;
  if (mode != AES_FILE_CTR && mode != AES_FILE_ECB_ENCRYPT && mode != AES_FILE_ECB_DECRYPT) return AES_ERR_ARG;
  if (mode == AES_FILE_CTR && iv == nullptr) return AES_ERR_ARG;
  uint64_t chunk = cfg ? cfg->chunk_bytes : 0;  // 0: the path's default, set below
  int threads = cfg && cfg->threads ? cfg->threads : 0;
  const uint32_t flags = cfg ? cfg->flags : 0u;
  if ((flags & ~(AES_FILE_STAGED | AES_FILE_DIRECT)) || flags == (AES_FILE_STAGED | AES_FILE_DIRECT))
    return AES_ERR_ARG;
  if (chunk % 16 != 0 || threads < 0 || threads > kMaxThreads) return AES_ERR_ARG;
  if (threads == 0) {
    const unsigned hw = std::thread::hardware_concurrency();
    threads = hw == 0 ? 4 : static_cast<int>(hw < 16 ? hw : 16);
  }

  FileJob job;
  job.mode = mode;
  job.ks = ks;
  if (iv) std::memcpy(job.iv, iv, 16);
  auto io_fail = [&](int err) {
    if (stats) stats->os_errno = err;
    return AES_ERR_IO;
  };
  job.fd_in = open(src_path, O_RDONLY | O_CLOEXEC);
  if (job.fd_in < 0) return io_fail(errno);
  struct stat st_in {};
  if (fstat(job.fd_in, &st_in) != 0) {
    const int err = errno;
    close(job.fd_in);
    return io_fail(err);
  }
  job.size = static_cast<uint64_t>(st_in.st_size);
  if (mode != AES_FILE_CTR && job.size % 16 != 0) {
    close(job.fd_in);
    return AES_ERR_LENGTH;
  }
  // dst: the same file (in place) or a new/truncated one of the source length
  struct stat st_out {};
  const bool same = stat(dst_path, &st_out) == 0 && st_out.st_dev == st_in.st_dev && st_out.st_ino == st_in.st_ino;
  job.fd_out = open(dst_path, O_RDWR | O_CLOEXEC | (same ? 0 : O_CREAT | O_TRUNC), 0644);
  if (job.fd_out < 0 || (!same && ftruncate(job.fd_out, static_cast<off_t>(job.size)) != 0)) {
    const int err = errno;
    if (job.fd_out >= 0) close(job.fd_out);
    close(job.fd_in);
    return io_fail(err);
  }
  if (job.size > 0) {
    void* m = mmap(nullptr, job.size, PROT_READ | PROT_WRITE, MAP_SHARED, job.fd_out, 0);
    job.map = m == MAP_FAILED ? nullptr : static_cast<uint8_t*>(m);
  }
  aes_status result = AES_OK;
  // an empty file needs no GPU: dst is created empty and nothing else runs
  cudaError_t ce = job.size > 0 ? cudaGetDevice(&job.device) : cudaSuccess;
  // the direct path, only when asked for: dst mapped, src mapped (or the
  // same mapping in place), and a device that reaches pageable memory through
  // the host's page tables.  It is opt-in because a file truncated by another
  // process while a chunk is in flight would fault the device, not the host.
  bool direct = false;
  uint8_t* src_map = nullptr;  // a mapping of its own (not in place)
  if (ce == cudaSuccess && job.size > 0 && job.map && (flags & AES_FILE_DIRECT) && host_pageable_access()) {
    if (same) {
      job.src_map = job.map;
      direct = true;
    } else {
      void* m = mmap(nullptr, job.size, PROT_READ, MAP_SHARED, job.fd_in, 0);
      if (m != MAP_FAILED) {
        src_map = static_cast<uint8_t*>(m);
        job.src_map = src_map;
        direct = true;
      }
    }
    const long pg = sysconf(_SC_PAGESIZE);
    job.page = pg > 0 ? static_cast<uint64_t>(pg) : 4096;
  }
  if (chunk == 0) chunk = direct ? kDefaultDirectChunk : kDefaultChunk;
  if (chunk > job.size) chunk = (job.size + 15) / 16 * 16;
  if (chunk == 0) chunk = 16;
  job.chunk = chunk;
  job.nchunks = (job.size + chunk - 1) / chunk;
  if (static_cast<uint64_t>(threads) > job.nchunks) threads = static_cast<int>(job.nchunks > 0 ? job.nchunks : 1);
  std::vector<uint8_t*> bufs(threads, nullptr);
  std::vector<cudaStream_t> streams(threads, nullptr);
  const uint64_t buf_bytes = (chunk + (1ull << 20) - 1) >> 20 << 20;
  for (int t = 0; t < threads && ce == cudaSuccess && job.nchunks > 0; ++t) {
    if (!direct) {
      ce = pinned_take(job.device, buf_bytes, &bufs[t]);
      if (ce != cudaSuccess) bufs[t] = nullptr;
    }
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&streams[t], cudaStreamNonBlocking);
  }
  const double setup = seconds_since(t0);
  if (ce != cudaSuccess) {
    result = record_cuda_failure(ce);
  } else if (job.nchunks > 0) {
    std::vector<std::thread> pool;
    pool.reserve(threads);
    for (int t = 0; t < threads; ++t) {
      if (direct) pool.emplace_back(worker_direct, &job, streams[t]);
      else pool.emplace_back(worker, &job, bufs[t], streams[t]);
    }
    for (auto& th : pool) th.join();
    result = static_cast<aes_status>(job.status.load());
    if (result == AES_ERR_CUDA) record_cuda_failure(static_cast<cudaError_t>(job.cuda_error.load()));
  }
  for (int t = 0; t < threads; ++t) {
    if (streams[t]) cudaStreamDestroy(streams[t]);
    if (bufs[t]) pinned_give(job.device, buf_bytes, bufs[t]);
  }
  int close_err = 0;
  if (src_map && munmap(src_map, job.size) != 0) close_err = errno;
  if (job.map && munmap(job.map, job.size) != 0) close_err = errno;
  if (close(job.fd_out) != 0 && close_err == 0) close_err = errno;  // a deferred write error surfaces here
  close(job.fd_in);
  if (result == AES_OK && close_err != 0) {
    result = AES_ERR_IO;
    job.os_errno.store(close_err);
  }
  if (stats) {
    stats->bytes = job.size;
    stats->chunks = job.next.load() < job.nchunks ? job.next.load() : job.nchunks;
    stats->seconds = seconds_since(t0);
    stats->setup_seconds = setup;
    stats->threads = threads;
    stats->os_errno = result == AES_ERR_IO ? job.os_errno.load() : 0;
    stats->direct = direct ? 1 : 0;
  }
  return result;
}

extern "C" void aes_file_trim(void) {
  using namespace aesgpu;
  std::vector<uint8_t*> all;
  {
    PinnedPool& pool = pinned_pool();
    std::lock_guard<std::mutex> lock(pool.mu);
    for (const PinnedBuf& b : pool.free) all.push_back(b.p);
    pool.free.clear();
  }
  for (uint8_t* p : all) cudaFreeHost(p);
}
