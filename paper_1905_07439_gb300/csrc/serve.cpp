// Serving runtime: a queue of independent products served with continuous admission.
//
// Requests (any formula, size, depth, seed and leaf mode) are submitted from any host thread
// and get consecutive tickets.  A worker thread admits them in arrival order as soon as the
// device workspace pool (a fixed-capacity region carved once at queue creation, sub-
// allocated first-fit) and a stream are free, so requests that arrive while others run
// start immediately and their kernels overlap on the device.  Completion is detected with
// events (non-blocking polls), the workspace returns to the pool, and each request's device
// status word (bounded-wait expiries) is copied back asynchronously and reported by poll.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "rbc_internal.h"

using namespace rbc;

namespace {

// First-fit allocator over one device region (256-byte granules).
class Pool {
 public:
  void init(char* base, size_t bytes) {
    base_ = base;
    free_.clear();
    free_[0] = bytes & ~(size_t)255;
  }
  // Returns the offset, or SIZE_MAX when no free block is large enough.
  size_t alloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        used_ += bytes;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  char* base() const { return base_; }
  size_t used() const { return used_; }

 private:
  char* base_ = nullptr;
  size_t used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Job {
  uint64_t ticket;
  rbc_request req;
  size_t ws_bytes;
};

struct Running {
  Job job;
  size_t off;
  int stream;
  cudaEvent_t done;
  int* status_host;  // pinned status word of this request
};

}  // namespace

struct rbc_queue_s {
  int device = 0;
  size_t cap = 0;
  char* region = nullptr;
  Pool pool;
  std::vector<cudaStream_t> streams;
  std::vector<char> stream_busy;
  std::vector<cudaEvent_t> events;
  int* status_pinned = nullptr;  // one word per stream slot
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job> pending;
  std::vector<Running> running;
  std::map<uint64_t, int> state;  // live tickets: -1 in progress, else final status (erased when collected)
  uint64_t next_ticket = 1;
  std::atomic<bool> stop{false};
  std::thread worker;
  // statistics
  uint64_t admitted = 0, completed = 0;
  size_t peak_used = 0;
  int peak_running = 0;
};

namespace {

void worker_loop(rbc_queue_s* q) {
  cudaSetDevice(q->device);
  std::unique_lock<std::mutex> lock(q->mu);
  while (true) {
    // retire finished requests
    for (size_t i = 0; i < q->running.size();) {
      Running& r = q->running[i];
      const cudaError_t e = cudaEventQuery(r.done);
      if (e == cudaErrorNotReady) {
        ++i;
        continue;
      }
      int st = e == cudaSuccess ? *r.status_host : (int)RBC_ECUDA;
      q->state[r.job.ticket] = st;
      q->pool.release(r.off, r.job.ws_bytes);
      q->stream_busy[r.stream] = 0;
      ++q->completed;
      q->running[i] = q->running.back();
      q->running.pop_back();
    }
    // admit in arrival order while memory and a stream are free
    while (!q->pending.empty()) {
      Job& j = q->pending.front();
      int s = -1;
      for (size_t k = 0; k < q->streams.size(); ++k)
        if (!q->stream_busy[k]) {
          s = (int)k;
          break;
        }
      if (s < 0) break;
      const size_t off = q->pool.alloc(j.ws_bytes);
      if (off == SIZE_MAX) break;
      char* ws = q->pool.base() + off;
      const rbc_request& rq = j.req;
      rbc_status st = rbc_matmul(rq.plan, rq.A, rq.B, rq.C, rq.N, rq.lda, rq.ldb, rq.ldc, rq.io_dtype,
                                 rq.leaf_dtype, ws, j.ws_bytes, q->streams[s]);
      int* sh = q->status_pinned + s;
      *sh = 0;
      if (st == RBC_OK &&
          cudaMemcpyAsync(sh, ws, sizeof(int), cudaMemcpyDeviceToHost, q->streams[s]) != cudaSuccess)
        st = RBC_ECUDA;
      if (st == RBC_OK && cudaEventRecord(q->events[s], q->streams[s]) != cudaSuccess) st = RBC_ECUDA;
      if (st != RBC_OK) {
        q->pool.release(off, j.ws_bytes);
        q->state[j.ticket] = (int)st;
        ++q->completed;
        q->pending.pop_front();
        continue;
      }
      q->stream_busy[s] = 1;
      q->running.push_back(Running{j, off, s, q->events[s], sh});
      ++q->admitted;
      if (q->pool.used() > q->peak_used) q->peak_used = q->pool.used();
      if ((int)q->running.size() > q->peak_running) q->peak_running = (int)q->running.size();
      q->pending.pop_front();
    }
    if (q->stop && q->pending.empty() && q->running.empty()) break;
    if (q->running.empty() && q->pending.empty()) {
      q->cv.wait(lock, [q] { return q->stop || !q->pending.empty(); });
    } else {
      // poll completions without holding the lock
      lock.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lock.lock();
    }
  }
}

}  // namespace

extern "C" {

rbc_status rbc_queue_create(int device, size_t workspace_cap_bytes, int streams, rbc_queue_t* out) {
  if (!out || streams < 1 || streams > 256 || workspace_cap_bytes < 4096)
    return fail(RBC_EINVAL, "bad queue arguments");
  *out = nullptr;
  rbc_queue_s* q = new (std::nothrow) rbc_queue_s();
  if (!q) return fail(RBC_ENOMEM, "out of host memory");
  q->device = device;
  q->cap = workspace_cap_bytes & ~(size_t)255;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc(&q->region, q->cap);
  if (e == cudaSuccess) e = cudaMallocHost(&q->status_pinned, sizeof(int) * streams);
  for (int i = 0; e == cudaSuccess && i < streams; ++i) {
    cudaStream_t s;
    cudaEvent_t ev;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
      q->streams.push_back(s);
      q->events.push_back(ev);
      q->stream_busy.push_back(0);
    }
  }
  if (e != cudaSuccess) {
    rbc_queue_destroy(q);
    return fail(e == cudaErrorMemoryAllocation ? RBC_ENOMEM : RBC_ECUDA, cudaGetErrorString(e));
  }
  q->pool.init(q->region, q->cap);
  q->worker = std::thread(worker_loop, q);
  *out = q;
  return RBC_OK;
}

rbc_status rbc_batch_submit(rbc_queue_t q, const rbc_request* reqs, int count, uint64_t* ticket) {
  if (!q || (count > 0 && !reqs) || !ticket || count < 0) return fail(RBC_EINVAL, "null argument");
  std::vector<Job> jobs;
  jobs.reserve(count);
  for (int i = 0; i < count; ++i) {
    const rbc_request& r = reqs[i];
    Job j{0, r, 0};
    j.ws_bytes = (r.plan && r.A && r.B && r.C) ? rbc_workspace_size(r.plan, r.N, r.io_dtype, r.leaf_dtype) : 0;
    if (j.ws_bytes > q->cap) return fail(RBC_ENOMEM, "request " + std::to_string(i) + " needs more workspace than the cap");
    jobs.push_back(j);
  }
  {
    std::lock_guard<std::mutex> lock(q->mu);
    if (q->stop) return fail(RBC_EBUSY, "queue is shutting down");
    *ticket = q->next_ticket;
    for (Job& j : jobs) {
      j.ticket = q->next_ticket++;
      if (j.ws_bytes == 0) {
        q->state[j.ticket] = (int)RBC_EINVAL;  // invalid request: completes at once with an error
        continue;
      }
      q->state[j.ticket] = -1;
      q->pending.push_back(j);
    }
  }
  q->cv.notify_one();
  return RBC_OK;
}

rbc_status rbc_batch_poll(rbc_queue_t q, uint64_t ticket, int* done) {
  if (!q || !done) return fail(RBC_EINVAL, "null argument");
  std::lock_guard<std::mutex> lock(q->mu);
  auto f = q->state.find(ticket);
  if (f == q->state.end()) return fail(RBC_EINVAL, "unknown ticket, or already collected");
  if (f->second < 0) {
    *done = 0;
    return RBC_OK;
  }
  *done = 1;
  const int st = f->second;
  q->state.erase(f);
  return st == RBC_OK ? RBC_OK : fail((rbc_status)st, "request failed");
}

rbc_status rbc_queue_stats(rbc_queue_t q, rbc_queue_info* info) {
  if (!q || !info) return fail(RBC_EINVAL, "null argument");
  std::lock_guard<std::mutex> lock(q->mu);
  info->pending = (int64_t)q->pending.size();
  info->running = (int64_t)q->running.size();
  info->admitted = q->admitted;
  info->completed = q->completed;
  info->workspace_used = q->pool.used();
  info->workspace_peak = q->peak_used;
  info->workspace_cap = q->cap;
  info->peak_running = q->peak_running;
  return RBC_OK;
}

void rbc_queue_destroy(rbc_queue_t q) {
  if (!q) return;
  {
    std::lock_guard<std::mutex> lock(q->mu);
    q->stop = true;
  }
  q->cv.notify_one();
  if (q->worker.joinable()) q->worker.join();
  for (cudaStream_t s : q->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : q->events) cudaEventDestroy(e);
  if (q->status_pinned) cudaFreeHost(q->status_pinned);
  if (q->region) cudaFree(q->region);
  delete q;
}

}  // extern "C"
