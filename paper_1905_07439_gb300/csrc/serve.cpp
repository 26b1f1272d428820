// Serving runtime: a queue of independent products served with continuous batching.
//
// Requests (any formula, size, depth, seed and leaf mode) are submitted from any host thread
// and get consecutive tickets.  A worker thread forms units of work every tick:
//   * admission walks the pending requests in arrival order and admits every one for which
//     the device workspace pool (one region carved at queue creation, sub-allocated first
//     fit) has room.  A request that does not fit is passed over by later, smaller ones, but
//     at most kMaxBypass times: after that admission stops at it until it fits (aging), so a
//     large request is never starved;
//   * small requests with the same tensor-core leaf mode admitted in one tick form one unit:
//     their encodes and decodes run in turn on the unit's stream and ALL their leaf products
//     run in one grouped persistent tcgen05 launch (the instance descriptors and tensor maps
//     go up by an asynchronous copy from pinned memory); every other request is a unit of its
//     own, computed exactly as rbc_matmul computes it;
//   * each unit runs on its own stream, so units admitted while others run overlap on the
//     device.
// The queue lock is held for admission and bookkeeping only, never while work is enqueued.
// Completion is detected with events (non-blocking polls), the workspace returns to the
// pool, and each unit's device status word (bounded-wait expiries) is copied back
// asynchronously and reported by poll for every request of the unit.
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "matmul_internal.h"
#include "rbc_internal.h"
#include "tc_gemm.cuh"

using namespace rbc;
using namespace rbc::detail;

namespace {

constexpr int kMaxBatch = 32;          // requests per grouped unit
constexpr int64_t kBatchMaxN = 2048;   // larger products fill the GPU alone: units of their own
constexpr int kMaxBypass = 32;         // later admissions that may pass a request that does not fit
constexpr size_t kDescBytes = 256 + (size_t)kMaxBatch * (sizeof(TcInst) + 2 * sizeof(CUtensorMap));

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
  uint64_t ticket = 0;
  rbc_request req{};
  size_t ws_bytes = 0;  // workspace as a unit of its own (rbc_matmul's layout)
  size_t ws_group = 0;  // workspace inside a grouped unit (staged decode); 0: not batchable
  int bypassed = 0;
};

// A unit: one request alone, or several small requests sharing one grouped leaf launch.
struct Unit {
  std::vector<Job> jobs;
  std::vector<size_t> offs;
  int stream = -1;
  bool grouped = false;
  int leaf = 0;
  cudaEvent_t done = nullptr;
  int* status_host = nullptr;
};

bool batchable(const rbc_request& r) {
  return is_tc_leaf(r.leaf_dtype) && r.io_dtype == RBC_IO_F32 && r.N <= kBatchMaxN;
}

}  // namespace

struct rbc_queue_s {
  int device = 0;
  size_t cap = 0;
  char* region = nullptr;
  Pool pool;
  std::vector<cudaStream_t> streams;
  std::vector<char> stream_busy;
  std::vector<cudaEvent_t> events;
  int* status_pinned = nullptr;   // one word per stream slot
  char* desc_pinned = nullptr;    // per stream slot: staging of a grouped unit's descriptors
  char* desc_dev = nullptr;       // per stream slot: the same on the device
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job> pending;
  std::vector<Unit> running;
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

// A grouped unit on stream `st`: encodes in turn, one grouped leaf launch, decodes in turn.
rbc_status enqueue_grouped(rbc_queue_s* q, Unit& u, cudaStream_t st) {
  static thread_local std::unique_ptr<Tables<float>> tab(new Tables<float>());
  const size_t n = u.jobs.size();
  std::vector<Layout> lo(n);
  for (size_t i = 0; i < n; ++i) {
    const rbc_request& r = u.jobs[i].req;
    rbc_status s = make_layout(r.plan, r.N, RBC_IO_F32, r.leaf_dtype, 2, &lo[i]);
    if (s != RBC_OK) return s;
  }
  char* ws0 = q->pool.base() + u.offs[0];
  cudaError_t e = cudaMemsetAsync(ws0, 0, sizeof(int), st);  // the unit's status word
  if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
  // instance descriptors: tile widths and CTAs per SM as a single product of this mode takes them
  bool all256 = u.leaf != RBC_LEAF_BF16X6 && u.leaf != RBC_LEAF_F16X3, small = leaf_panels(u.leaf) == 1;
  for (size_t i = 0; i < n; ++i) {
    all256 = all256 && lo[i].mp % 256 == 0;
    small = small && lo[i].mp <= 256;
  }
  const int bn = small ? 128 : (all256 ? 256 : 128), ctas = small ? 2 : 1;
  char* hst = q->desc_pinned + (size_t)u.stream * kDescBytes;
  char* dev = q->desc_dev + (size_t)u.stream * kDescBytes;
  TcInst* insts = reinterpret_cast<TcInst*>(hst);
  const size_t maps_off = (n * sizeof(TcInst) + 127) & ~(size_t)127;
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(hst + maps_off);
  int64_t tiles = 0;
  for (size_t i = 0; i < n; ++i) {
    const rbc_request& r = u.jobs[i].req;
    char* w = q->pool.base() + u.offs[i];
    TcGemmArgs a{};
    a.S = w + lo[i].leafS;
    a.T = w + lo[i].leafT;
    a.K = lo[i].K;
    a.m = lo[i].m;
    a.mp = lo[i].mp;
    a.leaves = ipow(r.plan->R, r.plan->L);
    a.C = r.C;
    a.ldc = r.ldc;
    a.direct = r.plan->L == 0;
    a.store_m = r.plan->L > 0;
    a.M = w + lo[i].M;
    a.strideM = lo[i].mstride;
    a.leaf = u.leaf;
    a.status = reinterpret_cast<int*>(ws0);
    a.rinv = leaf_inverse(lo[i], w, 0);
    a.cinv = leaf_inverse(lo[i], w, 1);
    if (!tc_prepare_instance(a, bn, tc_default_group(u.leaf, a.mp, a.K), tiles, &insts[i], &maps[2 * i]))
      return fail(RBC_EINVAL, "grouped unit: tensor map or tile shape rejected");
    tiles += tc_instance_tiles(insts[i]);
  }
  for (size_t i = 0; i < n; ++i) {
    const rbc_request& r = u.jobs[i].req;
    char* w = q->pool.base() + u.offs[i];
    rbc_status s = leaf_scales(r.plan, lo[i], r.A, r.lda, r.B, r.ldb, r.N, w, st);
    if (s == RBC_OK) s = encode_operand<float>(r.plan, lo[i], RBC_IO_F32, 0, r.A, r.lda, w, *tab, st);
    if (s == RBC_OK) s = encode_operand<float>(r.plan, lo[i], RBC_IO_F32, 1, r.B, r.ldb, w, *tab, st);
    if (s != RBC_OK) return s;
  }
  e = cudaMemcpyAsync(dev, hst, maps_off + 2 * n * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
  TcGroupArgs ga{};
  ga.insts = reinterpret_cast<const TcInst*>(dev);
  ga.maps = dev + maps_off;
  ga.ninst = (int)n;
  ga.total_tiles = tiles;
  ga.leaf = u.leaf;
  ga.bn = bn;
  ga.ctas = ctas;
  ga.status = reinterpret_cast<int*>(ws0);
  e = launch_tc_gemm_grouped(ga, st);
  if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
  for (size_t i = 0; i < n; ++i) {
    const rbc_request& r = u.jobs[i].req;
    if (r.plan->L == 0) continue;  // the leaf launch wrote C directly
    rbc_status s = decode_passes<float>(r.plan, lo[i], r.C, r.ldc, q->pool.base() + u.offs[i], *tab, st);
    if (s != RBC_OK) return s;
  }
  return RBC_OK;
}

// Enqueue a unit's work, the copy of its status word and its completion event (no lock held).
rbc_status enqueue_unit(rbc_queue_s* q, Unit& u) {
  cudaStream_t st = q->streams[u.stream];
  rbc_status s;
  if (u.grouped) {
    s = enqueue_grouped(q, u, st);
  } else {
    const rbc_request& r = u.jobs[0].req;
    s = rbc_matmul(r.plan, r.A, r.B, r.C, r.N, r.lda, r.ldb, r.ldc, r.io_dtype, r.leaf_dtype,
                   q->pool.base() + u.offs[0], u.jobs[0].ws_bytes, st);
  }
  u.status_host = q->status_pinned + u.stream;
  *u.status_host = 0;
  if (s == RBC_OK && cudaMemcpyAsync(u.status_host, q->pool.base() + u.offs[0], sizeof(int),
                                     cudaMemcpyDeviceToHost, st) != cudaSuccess)
    s = RBC_ECUDA;
  u.done = q->events[u.stream];
  if (s == RBC_OK && cudaEventRecord(u.done, st) != cudaSuccess) s = RBC_ECUDA;
  return s;
}

void release_unit(rbc_queue_s* q, const Unit& u, int status) {
  for (size_t i = 0; i < u.jobs.size(); ++i) {
    q->pool.release(u.offs[i], u.grouped ? u.jobs[i].ws_group : u.jobs[i].ws_bytes);
    q->state[u.jobs[i].ticket] = status;
    ++q->completed;
  }
  q->stream_busy[u.stream] = 0;
}

int free_stream(const rbc_queue_s* q) {
  for (size_t k = 0; k < q->streams.size(); ++k)
    if (!q->stream_busy[k]) return (int)k;
  return -1;
}

// Admission (lock held): form this tick's units from the pending requests.
std::vector<Unit> admit(rbc_queue_s* q) {
  std::vector<Unit> units;
  for (auto it = q->pending.begin(); it != q->pending.end();) {
    Job& j = *it;
    // join a grouped unit of this tick with the same leaf mode, else start a unit
    Unit* into = nullptr;
    if (j.ws_group) {
      for (Unit& u : units)
        if (u.grouped && u.leaf == j.req.leaf_dtype && (int)u.jobs.size() < kMaxBatch) {
          into = &u;
          break;
        }
    }
    const int s = into ? -1 : free_stream(q);
    if (!into && s < 0) break;  // no stream for a new unit
    const size_t bytes = j.ws_group ? j.ws_group : j.ws_bytes;
    const size_t off = q->pool.alloc(bytes);
    if (off == SIZE_MAX) {
      if (j.bypassed >= kMaxBypass) break;  // aged: nothing later passes it any more
      ++it;
      continue;
    }
    // every request passed over so far in this tick is passed once more
    for (auto p = q->pending.begin(); p != it; ++p) ++p->bypassed;
    if (!into) {
      Unit u;
      u.stream = s;
      u.grouped = j.ws_group != 0;
      u.leaf = j.req.leaf_dtype;
      q->stream_busy[s] = 1;
      units.push_back(u);
      into = &units.back();
    }
    into->jobs.push_back(j);
    into->offs.push_back(off);
    it = q->pending.erase(it);
  }
  // a grouped unit of one request runs as an ordinary product in its rbc_matmul layout
  for (Unit& u : units)
    if (u.grouped && u.jobs.size() == 1) {
      Job& j = u.jobs[0];
      q->pool.release(u.offs[0], j.ws_group);
      const size_t off = q->pool.alloc(j.ws_bytes);  // fits: ws_bytes <= ws_group, space just freed
      u.offs[0] = off;
      u.grouped = false;
    }
  return units;
}

void worker_loop(rbc_queue_s* q) {
  cudaSetDevice(q->device);
  std::unique_lock<std::mutex> lock(q->mu);
  while (true) {
    // retire finished units
    for (size_t i = 0; i < q->running.size();) {
      Unit& u = q->running[i];
      const cudaError_t e = cudaEventQuery(u.done);
      if (e == cudaErrorNotReady) {
        ++i;
        continue;
      }
      release_unit(q, u, e == cudaSuccess ? *u.status_host : (int)RBC_ECUDA);
      q->running[i] = q->running.back();
      q->running.pop_back();
    }
    std::vector<Unit> units = admit(q);
    if (!units.empty()) {
      lock.unlock();  // submit and poll proceed while the work is enqueued
      std::vector<rbc_status> sts(units.size());
      for (size_t k = 0; k < units.size(); ++k) sts[k] = enqueue_unit(q, units[k]);
      lock.lock();
      for (size_t k = 0; k < units.size(); ++k) {
        if (sts[k] != RBC_OK) {
          if (units[k].done) cudaEventSynchronize(units[k].done);  // nothing in flight on its memory
          cudaStreamSynchronize(q->streams[units[k].stream]);
          release_unit(q, units[k], (int)sts[k]);
          continue;
        }
        q->admitted += units[k].jobs.size();
        q->running.push_back(units[k]);
      }
      if (q->pool.used() > q->peak_used) q->peak_used = q->pool.used();
      int in_flight = 0;
      for (const Unit& u : q->running) in_flight += (int)u.jobs.size();
      if (in_flight > q->peak_running) q->peak_running = in_flight;
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
  if (e == cudaSuccess) e = cudaMallocHost(&q->desc_pinned, kDescBytes * streams);
  if (e == cudaSuccess) e = cudaMalloc(&q->desc_dev, kDescBytes * streams);
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
    Job j;
    j.req = r;
    const bool ok = r.plan && r.A && r.B && r.C && r.lda >= r.N && r.ldb >= r.N && r.ldc >= r.N;
    j.ws_bytes = ok ? rbc_workspace_size(r.plan, r.N, r.io_dtype, r.leaf_dtype) : 0;
    if (j.ws_bytes > q->cap)
      return fail(RBC_ENOMEM, "request " + std::to_string(i) + " needs more workspace than the cap");
    if (j.ws_bytes && batchable(r)) {
      rbc_matmul_opts staged{};
      staged.decode = 2;
      j.ws_group = rbc_workspace_size_ex(r.plan, r.N, r.io_dtype, r.leaf_dtype, &staged);
      if (j.ws_group < j.ws_bytes || j.ws_group > q->cap) j.ws_group = 0;
    }
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
  int64_t running = 0;
  for (const Unit& u : q->running) running += (int64_t)u.jobs.size();
  info->running = running;
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
  if (q->desc_pinned) cudaFreeHost(q->desc_pinned);
  if (q->desc_dev) cudaFree(q->desc_dev);
  if (q->region) cudaFree(q->region);
  delete q;
}

}  // extern "C"
