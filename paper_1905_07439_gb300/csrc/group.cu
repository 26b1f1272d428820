// Grouped batch of independent products C_i = F^(L_i)(A_i, B_i) (Section 2.1.1) with fp32
// I/O and tensor-core leaves.  Each instance is encoded and decoded by its own passes; the
// leaf products of all instances run in ONE persistent tcgen05 launch whose tile scheduler
// walks a global tile list (instance-major, then leaf, then tile), reading each instance's
// descriptor and TMA tensor maps from device memory.  The whole sequence can be captured
// once into a CUDA graph and replayed; a small autotuner times the candidate tile widths, tile
// orders and CTAs per SM of the grouped launch and keeps the fastest for the batch's
// signature.  Every configuration computes each tile with the same instruction sequence, so
// the configuration changes the speed, not the results.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "matmul_internal.h"
#include "rbc_internal.h"
#include "tc_gemm.cuh"

using namespace rbc;
using namespace rbc::detail;

namespace {

struct Config {
  int bn = 128;
  int group = 0;  // 0: per instance default, 1: row-major, 8: groups of 8 tile rows
  int ctas = 1;   // CTAs per SM of the grouped launch (2: plain 128-wide tiles, two stages each)
};

std::mutex g_cache_mutex;
std::map<std::string, Config> g_tuned;  // autotuner results by batch signature

struct TablesHolder {
  std::unique_ptr<Tables<float>> t{new Tables<float>()};
};

}  // namespace

struct rbc_group_s {
  int leaf = 0;
  std::vector<rbc_group_item> items;
  std::vector<Layout> layouts;
  std::vector<size_t> ws_off;   // per-instance sub-workspace offsets
  size_t inst_off = 0, maps_off = 0, total = 0;
  bool bn256_ok = false;
  Config cfg;
  std::string signature;
  // binding of the device-side descriptors to a workspace
  void* bound_ws = nullptr;
  Config bound_cfg;
  int64_t total_tiles = 0;
  // captured graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* graph_ws = nullptr;
  cudaStream_t graph_stream = nullptr;
  // side streams and events for running instances' passes concurrently (fork / join)
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;
  ~rbc_group_s() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaStream_t s : side) cudaStreamDestroy(s);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

namespace {

TcGemmArgs inst_args(const rbc_group_s* g, size_t i, char* ws) {
  const Layout& lo = g->layouts[i];
  char* w = ws + g->ws_off[i];
  TcGemmArgs a{};
  a.S = w + lo.leafS;
  a.T = w + lo.leafT;
  a.K = lo.K;
  a.m = lo.m;
  a.mp = lo.mp;
  a.leaves = ipow(g->items[i].plan->R, g->items[i].plan->L);
  a.C = g->items[i].C;
  a.ldc = g->items[i].ldc;
  a.direct = g->items[i].plan->L == 0;
  a.store_m = g->items[i].plan->L > 0;
  a.M = w + lo.M;
  a.strideM = lo.mstride;
  a.leaf = g->leaf;
  a.status = reinterpret_cast<int*>(ws);
  a.rinv = leaf_inverse(lo, w, 0);
  a.cinv = leaf_inverse(lo, w, 1);
  return a;
}

// Write the instance descriptors and tensor maps for `cfg` into the workspace.
rbc_status bind(rbc_group_s* g, char* ws, const Config& cfg) {
  const size_t n = g->items.size();
  std::vector<TcInst> insts(n);
  std::vector<CUtensorMap> maps(2 * n);
  int64_t tiles = 0;
  for (size_t i = 0; i < n; ++i) {
    TcGemmArgs a = inst_args(g, i, ws);
    const int grp = cfg.group ? cfg.group : tc_default_group(g->leaf, a.mp, a.K);
    if (!tc_prepare_instance(a, cfg.bn, grp, tiles, &insts[i], &maps[2 * i]))
      return fail(RBC_EINVAL, "instance " + std::to_string(i) + ": tensor map or tile shape rejected");
    tiles += tc_instance_tiles(insts[i]);
  }
  cudaError_t e = cudaMemcpy(ws + g->inst_off, insts.data(), n * sizeof(TcInst), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(ws + g->maps_off, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
  g->bound_ws = ws;
  g->bound_cfg = cfg;
  g->total_tiles = tiles;
  return RBC_OK;
}

rbc_status grouped_gemm(rbc_group_s* g, char* ws, cudaStream_t st) {
  TcGroupArgs ga{};
  ga.insts = reinterpret_cast<const TcInst*>(ws + g->inst_off);
  ga.maps = ws + g->maps_off;
  ga.ninst = (int)g->items.size();
  ga.total_tiles = g->total_tiles;
  ga.leaf = g->leaf;
  ga.bn = g->bound_cfg.bn;
  ga.ctas = g->bound_cfg.ctas;
  ga.status = reinterpret_cast<int*>(ws);
  cudaError_t e = launch_tc_gemm_grouped(ga, st);
  ++g_launches;
  return e == cudaSuccess ? RBC_OK : fail(RBC_ECUDA, cudaGetErrorString(e));
}

constexpr int kSideStreams = 8;

rbc_status ensure_side(rbc_group_s* g) {
  if (!g->side.empty()) return RBC_OK;
  for (int i = 0; i < kSideStreams; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
      return fail(RBC_ECUDA, "stream creation failed");
    g->side.push_back(s);
  }
  for (int i = 0; i < 2 * kSideStreams + 2; ++i) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return fail(RBC_ECUDA, "event creation failed");
    g->ev.push_back(e);
  }
  return RBC_OK;
}

// Fork: every side stream waits for `st`; join: `st` waits for every side stream.
rbc_status fork(rbc_group_s* g, cudaStream_t st, cudaEvent_t e) {
  if (cudaEventRecord(e, st) != cudaSuccess) return fail(RBC_ECUDA, "event record failed");
  for (cudaStream_t s : g->side)
    if (cudaStreamWaitEvent(s, e, 0) != cudaSuccess) return fail(RBC_ECUDA, "stream wait failed");
  return RBC_OK;
}
rbc_status join(rbc_group_s* g, cudaStream_t st, const cudaEvent_t* evs) {
  for (size_t i = 0; i < g->side.size(); ++i) {
    if (cudaEventRecord(evs[i], g->side[i]) != cudaSuccess) return fail(RBC_ECUDA, "event record failed");
    if (cudaStreamWaitEvent(st, evs[i], 0) != cudaSuccess) return fail(RBC_ECUDA, "stream wait failed");
  }
  return RBC_OK;
}

// The whole batch: the instances' encodes spread over the side streams, one grouped leaf
// launch on `st`, then the decodes spread again; ordered on `st` before and after.
rbc_status enqueue(rbc_group_s* g, char* ws, cudaStream_t st) {
  static thread_local TablesHolder holder;
  Tables<float>& tab = *holder.t;
  rbc_status s = ensure_side(g);
  if (s != RBC_OK) return s;
  cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(int), st);
  if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
  const int ns = (int)g->side.size();
  if ((s = fork(g, st, g->ev[0])) != RBC_OK) return s;
  for (size_t i = 0; i < g->items.size(); ++i) {
    const rbc_group_item& it = g->items[i];
    char* w = ws + g->ws_off[i];
    cudaStream_t si = g->side[i % ns];
    s = leaf_scales(it.plan, g->layouts[i], it.A, it.lda, it.B, it.ldb, it.N, w, si);
    if (s == RBC_OK) s = encode_operand<float>(it.plan, g->layouts[i], RBC_IO_F32, 0, it.A, it.lda, w, tab, si);
    if (s == RBC_OK) s = encode_operand<float>(it.plan, g->layouts[i], RBC_IO_F32, 1, it.B, it.ldb, w, tab, si);
    if (s != RBC_OK) return s;
  }
  if ((s = join(g, st, &g->ev[2])) != RBC_OK) return s;
  if ((s = grouped_gemm(g, ws, st)) != RBC_OK) return s;
  if ((s = fork(g, st, g->ev[1])) != RBC_OK) return s;
  for (size_t i = 0; i < g->items.size(); ++i) {
    const rbc_group_item& it = g->items[i];
    if (it.plan->L == 0) continue;  // the leaf launch wrote C directly
    s = decode_passes<float>(it.plan, g->layouts[i], it.C, it.ldc, ws + g->ws_off[i], tab, g->side[i % ns]);
    if (s != RBC_OK) return s;
  }
  return join(g, st, &g->ev[2 + ns]);
}

rbc_status check_ws(const rbc_group_s* g, void* ws, size_t bytes) {
  if (!ws || ((uintptr_t)ws & 255)) return fail(RBC_EINVAL, "workspace must be a 256-byte aligned device pointer");
  if (bytes < g->total) return fail(RBC_ENOMEM, "workspace too small");
  return RBC_OK;
}

}  // namespace

extern "C" {

rbc_status rbc_group_create(const rbc_group_item* items, int count, int leaf_dtype, rbc_group_t* out) {
  if (!items || !out || count <= 0) return fail(RBC_EINVAL, "null argument or empty batch");
  *out = nullptr;
  if (!is_tc_leaf(leaf_dtype)) return fail(RBC_EUNSUPPORTED, "grouped batches use tensor-core leaf modes");
  std::unique_ptr<rbc_group_s> g(new (std::nothrow) rbc_group_s());
  if (!g) return fail(RBC_ENOMEM, "out of host memory");
  g->leaf = leaf_dtype;
  g->items.assign(items, items + count);
  size_t off = kStatusBytes;
  bool all256 = true;  // 256-wide tiles: every instance's padded leaf size divisible by 256
  std::ostringstream sig;
  sig << leaf_dtype;
  for (int i = 0; i < count; ++i) {
    const rbc_group_item& it = items[i];
    if (!it.plan || !it.A || !it.B || !it.C) return fail(RBC_EINVAL, "null pointer in item " + std::to_string(i));
    if (it.lda < it.N || it.ldb < it.N || it.ldc < it.N) return fail(RBC_EINVAL, "leading dimension below N");
    Layout lo;
    rbc_status s = make_layout(it.plan, it.N, RBC_IO_F32, leaf_dtype, 2, &lo);
    if (s != RBC_OK) return s;
    g->layouts.push_back(lo);
    g->ws_off.push_back(off);
    off = align256(off + lo.total);
    all256 = all256 && lo.mp % 256 == 0;
    sig << ';' << lo.mp << 'x' << ipow(it.plan->R, it.plan->L);
  }
  g->inst_off = off;
  off = align256(off + (size_t)count * sizeof(TcInst));
  g->maps_off = off;
  off = align256(off + (size_t)count * 2 * sizeof(CUtensorMap));
  g->total = off;
  g->bn256_ok = all256;
  g->signature = sig.str();
  g->cfg.bn = 128;
  {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    auto f = g_tuned.find(g->signature);
    if (f != g_tuned.end()) g->cfg = f->second;
  }
  *out = g.release();
  return RBC_OK;
}

size_t rbc_group_workspace_size(rbc_group_t g) { return g ? g->total : 0; }

rbc_status rbc_group_run(rbc_group_t g, void* workspace, size_t bytes, void* stream, int flags) {
  if (!g) return fail(RBC_EINVAL, "null group");
  rbc_status s = check_ws(g, workspace, bytes);
  if (s != RBC_OK) return s;
  char* ws = static_cast<char*>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (g->bound_ws != ws || g->bound_cfg.bn != g->cfg.bn || g->bound_cfg.group != g->cfg.group ||
      g->bound_cfg.ctas != g->cfg.ctas) {
    s = bind(g, ws, g->cfg);
    if (s != RBC_OK) return s;
    if (g->exec) {
      cudaGraphExecDestroy(g->exec);
      g->exec = nullptr;
    }
    if (g->graph) {
      cudaGraphDestroy(g->graph);
      g->graph = nullptr;
    }
  }
  g_launches = 0;
  if (!(flags & RBC_GROUP_GRAPH)) return enqueue(g, ws, st);
  if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread)
    return fail(RBC_EINVAL, "graph capture needs a created (non-default) stream");
  if (!g->exec || g->graph_ws != ws || g->graph_stream != st) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    g->exec = nullptr;
    g->graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
    s = enqueue(g, ws, st);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (s != RBC_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return fail(RBC_ECUDA, cudaGetErrorString(e));
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return fail(RBC_ECUDA, cudaGetErrorString(e));
    }
    g->graph = graph;
    g->graph_ws = ws;
    g->graph_stream = st;
  }
  cudaError_t e = cudaGraphLaunch(g->exec, st);
  return e == cudaSuccess ? RBC_OK : fail(RBC_ECUDA, cudaGetErrorString(e));
}

rbc_status rbc_group_tune(rbc_group_t g, void* workspace, size_t bytes, void* stream, rbc_group_tuning* out) {
  if (!g) return fail(RBC_EINVAL, "null group");
  rbc_status s = check_ws(g, workspace, bytes);
  if (s != RBC_OK) return s;
  char* ws = static_cast<char*>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // leaf operands must exist once: run the batch eagerly with the current configuration
  s = bind(g, ws, g->cfg);
  if (s == RBC_OK) s = enqueue(g, ws, st);
  if (s != RBC_OK) return s;
  std::vector<Config> cands;
  const bool split = leaf_panels(g->leaf) > 1;
  for (int bn : {128, 256}) {
    if (bn == 256 && (!g->bn256_ok || g->leaf == RBC_LEAF_BF16X6 || g->leaf == RBC_LEAF_F16X3)) continue;
    for (int ctas : {1, 2}) {
      if (ctas == 2 && (split || bn != 128)) continue;
      for (int grp : {0, 1, 8}) cands.push_back(Config{bn, grp, ctas});
    }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(RBC_ECUDA, "event creation failed");
  float best_ms = 1e30f;
  Config best = g->cfg;
  int ntried = 0;
  for (const Config& c : cands) {
    s = bind(g, ws, c);
    if (s != RBC_OK) break;
    s = grouped_gemm(g, ws, st);  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && s == RBC_OK; ++r) s = grouped_gemm(g, ws, st);
    cudaEventRecord(e1, st);
    if (s != RBC_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      s = fail(RBC_ECUDA, "tuning run failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 3.f;
    ++ntried;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != RBC_OK) return s;
  g->cfg = best;
  s = bind(g, ws, best);
  if (g->exec) {
    cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
  if (g->graph) {
    cudaGraphDestroy(g->graph);
    g->graph = nullptr;
  }
  {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    g_tuned[g->signature] = best;
  }
  if (out) {
    out->bn = best.bn;
    out->group = best.group;
    out->ctas_per_sm = best.ctas;
    out->candidates = ntried;
    out->best_ms = best_ms;
  }
  return s;
}

rbc_status rbc_group_configure(rbc_group_t g, const rbc_group_tuning* cfg) {
  if (!g || !cfg) return fail(RBC_EINVAL, "null argument");
  const bool split = leaf_panels(g->leaf) > 1;
  if (cfg->bn != 128 && cfg->bn != 256) return fail(RBC_EINVAL, "bn must be 128 or 256");
  if (cfg->bn == 256 && !g->bn256_ok) return fail(RBC_EINVAL, "bn 256 needs padded leaf sizes divisible by 256");
  if (cfg->bn == 256 && (g->leaf == RBC_LEAF_BF16X6 || g->leaf == RBC_LEAF_F16X3))
    return fail(RBC_EINVAL, "bf16x6 and f16x3 leaves take bn 128");
  const int grp = cfg->group;
  if (grp != 0 && grp != 1 && grp != 2 && grp != 4 && grp != 8 && grp != 16)
    return fail(RBC_EINVAL, "group must be 0, 1, 2, 4, 8 or 16");
  if (cfg->ctas_per_sm != 1 && cfg->ctas_per_sm != 2) return fail(RBC_EINVAL, "ctas_per_sm must be 1 or 2");
  if (cfg->ctas_per_sm == 2 && (split || cfg->bn != 128))
    return fail(RBC_EINVAL, "two CTAs per SM need bn 128 and a plain leaf mode");
  g->cfg = Config{cfg->bn, grp, cfg->ctas_per_sm};
  return RBC_OK;
}

void rbc_group_destroy(rbc_group_t g) { delete g; }

}  // extern "C"
