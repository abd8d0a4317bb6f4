// irs_batch.cu -- many maps as one CUDA graph (irs_make_maps_batched).
//
// Maps with uneven lens counts, kappa and gamma are prepared on NSIDE forked
// capture streams (each map's mass sum, cell lists and far-field series, or
// the brute-force tile setup and ray pass), joined, and their interpolated ray
// passes run as ONE persistent launch per kernel variant whose CTAs pull
// (map, cell) items from a global counter.  The whole sequence is captured once
// per distinct (plans, buffers) set and replayed from the instantiated graph.
#include <string.h>

#include <mutex>
#include <vector>

#include "irs_common.cuh"
#include "irs_interp.cuh"

namespace {

constexpr int NSIDE = 8;       // capture streams the per-map stages are spread over
constexpr int CACHE_SIZE = 4;  // graphs kept (least recently used dropped)
constexpr size_t KEY_PER_MAP = 7;  // key words per map, after the device

struct BatchEntry {
  std::vector<uintptr_t> key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* dbuf = nullptr;  // descriptors of every variant group + one queue counter each
  cudaStream_t cs = nullptr;
  cudaStream_t side[NSIDE] = {};
  cudaEvent_t ev[NSIDE + 1] = {};
  int device = -1;
  uint64_t last_use = 0;
};

std::mutex g_mu;
std::vector<BatchEntry*> g_cache;
uint64_t g_clock = 0;

void release(BatchEntry* e) {
  if (!e) return;
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  if (e->dbuf) cudaFree(e->dbuf);
  for (int k = 0; k < NSIDE; ++k)
    if (e->side[k]) cudaStreamDestroy(e->side[k]);
  for (int k = 0; k <= NSIDE; ++k)
    if (e->ev[k]) cudaEventDestroy(e->ev[k]);
  if (e->cs) cudaStreamDestroy(e->cs);
  delete e;
}

irs_status st_of(cudaError_t e) {
  if (e == cudaSuccess) return IRS_OK;
  return e == cudaErrorMemoryAllocation ? IRS_ERR_OOM : IRS_ERR_CUDA;
}

// Enqueue the whole batch on the capture stream (and its side streams).
irs_status enqueue(BatchEntry* e, irs_plan_t* const* plans, int32_t nmaps, const double* const* xy,
                   const double* const* mass, const int64_t* n, uint32_t* const* counts,
                   float* const* mag, const std::vector<std::vector<int>>& groups,
                   const std::vector<size_t>& group_off, size_t queue_off) {
  cudaStream_t cs = e->cs;
  if (cudaEventRecord(e->ev[NSIDE], cs) != cudaSuccess) return IRS_ERR_CUDA;
  for (int k = 0; k < NSIDE; ++k)
    if (cudaStreamWaitEvent(e->side[k], e->ev[NSIDE], 0) != cudaSuccess) return IRS_ERR_CUDA;
  for (int32_t m = 0; m < nmaps; ++m) {
    irs_plan_t* P = plans[m];
    cudaStream_t s = e->side[m % NSIDE];
    const size_t npix = (size_t)P->g.npix_x * P->g.npix_y;
    if (cudaMemsetAsync(counts[m], 0, npix * sizeof(uint32_t), s) != cudaSuccess) return IRS_ERR_CUDA;
    if (irs::launch_mass_sum(P, mass[m], n[m], s, xy[m]) != cudaSuccess) return IRS_ERR_CUDA;
    if (P->p.method == IRS_BRUTE) {
      if (irs::launch_brute_setup(P, s) != cudaSuccess) return IRS_ERR_CUDA;
      if (irs::launch_brute_map(P, xy[m], mass[m], n[m], 0, P->g.nry, counts[m], s) != cudaSuccess)
        return IRS_ERR_CUDA;
    } else {
      const int timing = P->timing;
      P->timing = 0;  // no stage events inside the graph
      irs_status st = irs::interp_prepare(P, xy[m], mass[m], n[m], s);
      P->timing = timing;
      if (st != IRS_OK) return st;
    }
  }
  for (int k = 0; k < NSIDE; ++k) {
    if (cudaEventRecord(e->ev[k], e->side[k]) != cudaSuccess) return IRS_ERR_CUDA;
    if (cudaStreamWaitEvent(cs, e->ev[k], 0) != cudaSuccess) return IRS_ERR_CUDA;
  }
  char* base = static_cast<char*>(e->dbuf);
  unsigned long long* queues = reinterpret_cast<unsigned long long*>(base + queue_off);
  for (size_t v = 0; v < groups.size(); ++v) {
    const std::vector<int>& gm = groups[v];
    if (gm.empty()) continue;
    // item count of the group, recomputed from the plans (cheap, host side)
    std::vector<irs_plan_t*> gp;
    std::vector<uint32_t*> gc;
    int nrow = 0;
    for (int m : gm) {
      gp.push_back(plans[m]);
      gc.push_back(counts[m]);
      const int r = irs::interp_row_entries(plans[m]);
      nrow = r > nrow ? r : nrow;
    }
    std::vector<char> tmp(irs::interp_desc_bytes((int)gm.size()));
    const int64_t items = irs::interp_fill_descs(gp.data(), gc.data(), (int)gm.size(), tmp.data());
    irs_status st = irs::interp_batch_launch((int)v, base + group_off[v], (int)gm.size(), items,
                                             queues + v, plans[gm[0]]->num_sms, nrow, cs);
    if (st != IRS_OK) return st;
  }
  if (mag) {
    for (int32_t m = 0; m < nmaps; ++m)
      if (mag[m] && irs::launch_magnify(plans[m], counts[m], mag[m], cs) != cudaSuccess)
        return IRS_ERR_CUDA;
  }
  return IRS_OK;
}

irs_status build_entry(BatchEntry* e, irs_plan_t* const* plans, int32_t nmaps,
                       const double* const* xy, const double* const* mass, const int64_t* n,
                       uint32_t* const* counts, float* const* mag) {
  // the lens buffers were grown by the caller, before the key was taken;
  // streams, events and descriptors are made here, before the capture
  if (cudaGetDevice(&e->device) != cudaSuccess) return IRS_ERR_CUDA;
  if (cudaStreamCreateWithFlags(&e->cs, cudaStreamNonBlocking) != cudaSuccess) return IRS_ERR_CUDA;
  for (int k = 0; k < NSIDE; ++k)
    if (cudaStreamCreateWithFlags(&e->side[k], cudaStreamNonBlocking) != cudaSuccess) return IRS_ERR_CUDA;
  for (int k = 0; k <= NSIDE; ++k)
    if (cudaEventCreateWithFlags(&e->ev[k], cudaEventDisableTiming) != cudaSuccess) return IRS_ERR_CUDA;

  // interpolated maps grouped by ray-pass variant; descriptors + queues in one buffer
  std::vector<std::vector<int>> groups(irs::interp_num_variants());
  for (int32_t m = 0; m < nmaps; ++m)
    if (plans[m]->p.method != IRS_BRUTE) groups[irs::interp_variant(plans[m])].push_back(m);
  std::vector<size_t> group_off(groups.size(), 0);
  size_t off = 0;
  for (size_t v = 0; v < groups.size(); ++v) {
    group_off[v] = off;
    off += (irs::interp_desc_bytes((int)groups[v].size()) + 255) & ~(size_t)255;
  }
  const size_t queue_off = off;
  off += sizeof(unsigned long long) * groups.size();
  if (cudaMalloc(&e->dbuf, off) != cudaSuccess) {
    cudaGetLastError();
    return IRS_ERR_OOM;
  }
  for (size_t v = 0; v < groups.size(); ++v) {
    if (groups[v].empty()) continue;
    std::vector<irs_plan_t*> gp;
    std::vector<uint32_t*> gc;
    for (int m : groups[v]) {
      gp.push_back(plans[m]);
      gc.push_back(counts[m]);
    }
    std::vector<char> host(irs::interp_desc_bytes((int)groups[v].size()));
    irs::interp_fill_descs(gp.data(), gc.data(), (int)groups[v].size(), host.data());
    if (cudaMemcpy(static_cast<char*>(e->dbuf) + group_off[v], host.data(), host.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return IRS_ERR_CUDA;
  }

  if (cudaStreamBeginCapture(e->cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return IRS_ERR_CUDA;
  irs_status st = enqueue(e, plans, nmaps, xy, mass, n, counts, mag, groups, group_off, queue_off);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(e->cs, &graph);
  if (st != IRS_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return st;
  }
  if (ce != cudaSuccess || !graph) return IRS_ERR_CUDA;
  e->graph = graph;
  if (cudaGraphInstantiate(&e->exec, graph, 0) != cudaSuccess) return IRS_ERR_CUDA;
  return IRS_OK;
}

}  // namespace

extern "C" irs_status irs_make_maps_batched(irs_plan_t* const* plans, int32_t nmaps,
                                            const double* const* lens_xy, const double* const* mass,
                                            const int64_t* n, uint32_t* const* counts,
                                            float* const* mag, void* stream) {
  if (nmaps < 0 || (nmaps > 0 && (!plans || !lens_xy || !mass || !n || !counts))) return IRS_ERR_ARG;
  if (nmaps == 0) return IRS_OK;
  for (int32_t m = 0; m < nmaps; ++m) {
    if (!plans[m] || !counts[m] || n[m] < 0) return IRS_ERR_ARG;
    if (n[m] > 0 && (!lens_xy[m] || !mass[m] || ((uintptr_t)lens_xy[m] & 15u))) return IRS_ERR_ARG;
    if (plans[m]->p.method == IRS_MLP) return IRS_ERR_UNSUPPORTED;
    for (int32_t q = 0; q < m; ++q)  // stages of one map run concurrently with the others':
      if (plans[q] == plans[m]) return IRS_ERR_ARG;  // a plan's workspace serves one map
  }
  std::lock_guard<std::mutex> lock(g_mu);
  // lens buffers grow (and move) before the key is taken: a graph is keyed by
  // every address its kernels use, the plans' workspace generations included,
  // so a graph captured before a plan's buffers moved is never replayed
  for (int32_t m = 0; m < nmaps; ++m)
    if (plans[m]->p.method != IRS_BRUTE) {
      irs_status st = irs::interp_ensure_capacity(plans[m], n[m]);
      if (st != IRS_OK) return st;
    }
  std::vector<uintptr_t> key;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IRS_ERR_CUDA;
  key.push_back((uintptr_t)dev);
  for (int32_t m = 0; m < nmaps; ++m) {
    key.push_back((uintptr_t)plans[m]);
    key.push_back((uintptr_t)lens_xy[m]);
    key.push_back((uintptr_t)mass[m]);
    key.push_back((uintptr_t)n[m]);
    key.push_back((uintptr_t)counts[m]);
    key.push_back((uintptr_t)(mag ? mag[m] : nullptr));
    key.push_back((uintptr_t)plans[m]->ws_gen);
  }
  BatchEntry* e = nullptr;
  for (BatchEntry* c : g_cache)
    if (c->key == key) e = c;
  if (!e) {
    e = new BatchEntry();
    e->key = key;
    irs_status st = build_entry(e, plans, nmaps, lens_xy, mass, n, counts, mag);
    if (st != IRS_OK) {
      release(e);
      return st;
    }
    if ((int)g_cache.size() >= CACHE_SIZE) {
      size_t oldest = 0;
      for (size_t k = 1; k < g_cache.size(); ++k)
        if (g_cache[k]->last_use < g_cache[oldest]->last_use) oldest = k;
      cudaDeviceSynchronize();
      release(g_cache[oldest]);
      g_cache.erase(g_cache.begin() + (long)oldest);
    }
    g_cache.push_back(e);
  }
  e->last_use = ++g_clock;
  return st_of(cudaGraphLaunch(e->exec, static_cast<cudaStream_t>(stream)));
}

// Drop every cached graph that refers to `plan` (called when the plan is destroyed).
void irs_batch_forget_plan(const irs_plan_t* plan) {
  std::lock_guard<std::mutex> lock(g_mu);
  for (size_t k = 0; k < g_cache.size();) {
    bool hit = false;
    for (size_t i = 1; i < g_cache[k]->key.size(); i += KEY_PER_MAP)
      if (g_cache[k]->key[i] == (uintptr_t)plan) hit = true;
    if (hit) {
      release(g_cache[k]);
      g_cache.erase(g_cache.begin() + (long)k);
    } else {
      ++k;
    }
  }
}
