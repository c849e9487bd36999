// Batched scan: many independent U_T builds captured into one CUDA graph (one launch per scan).
// lanes = 0: split-precision dense plans of one precision and step count run as one persistent
// launch over (instance, step, term, tile) work units (scan.cu); otherwise, or with lanes >= 1, the
// graph holds every plan's own build on `lanes` concurrent branches.
#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "internal.h"

struct fq_batch {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {
size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
double cost(const fq_plan* p) { return (double)p->n * p->n * p->n * p->steps * p->L; }
}  // namespace

// the plans' own workspaces, back to back
static size_t plans_bytes(fq_plan* const* plans, int count) {
  size_t tot = 0;
  for (int i = 0; i < count; ++i) tot += up256(floquet_workspace_size(plans[i], plans[i]->n));
  return tot;
}

extern "C" size_t floquet_batch_workspace_size(fq_plan* const* plans, int32_t count) {
  if (!plans || count < 1) return 0;
  for (int i = 0; i < count; ++i)
    if (!plans[i]) return 0;
  return plans_bytes(plans, count) + fq_scan_extra_bytes(plans, count);
}

static fq_status floquet_batch_create_body(fq_batch** out, fq_plan* const* plans, int32_t count, void* const* d_U,
                                           void* d_ws, size_t ws_bytes, int32_t lanes) {
  if (!out || !plans || !d_U || count < 1 || lanes < 0 || lanes > 32) {
    fq_set_error("floquet_batch_create: bad arguments");
    return FQ_EINVAL;
  }
  *out = nullptr;
  for (int i = 0; i < count; ++i)
    if (!plans[i] || !d_U[i]) {
      fq_set_error("floquet_batch_create: plan or output %d is NULL", i);
      return FQ_EINVAL;
    }
  const size_t need = floquet_batch_workspace_size(plans, count);
  if (!d_ws || ws_bytes < need || ((uintptr_t)d_ws & 255)) {
    fq_set_error("floquet_batch_create: workspace must be >= %zu bytes, 256-byte aligned", need);
    return FQ_EINVAL;
  }
  std::vector<size_t> off(count);
  size_t o = 0;
  for (int i = 0; i < count; ++i) {
    off[i] = o;
    o += up256(floquet_workspace_size(plans[i], plans[i]->n));
  }
  fq_batch* b = new (std::nothrow) fq_batch();
  if (!b) { fq_set_error("host allocation failed"); return FQ_ENOMEM; }
  if (lanes == 0 && fq_scan_eligible(plans, count)) {  // one persistent launch over work units
    fq_status st = fq_scan_graph(plans, count, d_U, d_ws, off.data(), plans_bytes(plans, count), &b->graph);
    if (st == FQ_OK) {
      cudaError_t e = cudaGraphInstantiate(&b->exec, b->graph, 0);
      if (e != cudaSuccess) st = fq_cuda_fail(e, "batch graph instantiate");
    }
    if (st != FQ_OK) {
      floquet_batch_destroy(b);
      return st;
    }
    *out = b;
    return FQ_OK;
  }
  if (lanes == 0) lanes = 8;  // plans the persistent scan does not take: the lane graph
  // longest-processing-time assignment of instances to lanes
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return cost(plans[a]) > cost(plans[b]); });
  std::vector<double> load(lanes, 0.0);
  std::vector<int> lane_of(count);
  for (int i : order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lane_of[i] = l;
    load[l] += cost(plans[i]);
  }
  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> ls(lanes, nullptr);
  std::vector<cudaEvent_t> joins(lanes, nullptr);
  cudaEvent_t fork = nullptr;
  fq_status st = FQ_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
  for (int l = 0; l < lanes && e == cudaSuccess; ++l) e = cudaStreamCreateWithFlags(&ls[l], cudaStreamNonBlocking);
  for (int l = 0; l < lanes && e == cudaSuccess; ++l) e = cudaEventCreateWithFlags(&joins[l], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
  bool capturing = e == cudaSuccess;
  if (e == cudaSuccess) e = cudaEventRecord(fork, origin);
  for (int l = 0; l < lanes && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(ls[l], fork, 0);
  if (e != cudaSuccess) st = fq_cuda_fail(e, "batch capture setup");
  // each persistent split product takes at most half the SMs, so products of different lanes run
  // side by side instead of one after another (5.86 -> 5.57 s for the 48-instance scan)
  const int cap = std::max(1, fq_sm_count() / 2);
  for (int k = 0; k < count && st == FQ_OK; ++k) {
    const int i = order[k];
    plans[i]->grid_cap = cap;
    st = floquet_build_UT(plans[i], d_U[i], (char*)d_ws + off[i], ws_bytes - off[i], ls[lane_of[i]]);
    plans[i]->grid_cap = 0;
  }
  for (int l = 0; l < lanes && capturing; ++l) {
    cudaEventRecord(joins[l], ls[l]);
    cudaStreamWaitEvent(origin, joins[l], 0);
  }
  if (capturing) {
    e = cudaStreamEndCapture(origin, &b->graph);
    if (st == FQ_OK && e != cudaSuccess) st = fq_cuda_fail(e, "batch capture");
  }
  if (st == FQ_OK) {
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) st = fq_cuda_fail(e, "batch graph instantiate");
  }
  for (int l = 0; l < lanes; ++l) {
    if (ls[l]) cudaStreamDestroy(ls[l]);
    if (joins[l]) cudaEventDestroy(joins[l]);
  }
  if (fork) cudaEventDestroy(fork);
  if (origin) cudaStreamDestroy(origin);
  if (st != FQ_OK) {
    floquet_batch_destroy(b);
    return st;
  }
  *out = b;
  return FQ_OK;
}

extern "C" fq_status floquet_batch_create(fq_batch** out, fq_plan* const* plans, int32_t count, void* const* d_U,
                                          void* d_ws, size_t ws_bytes, int32_t lanes) {
  return fq_guard("floquet_batch_create", [&] {
    return floquet_batch_create_body(out, plans, count, d_U, d_ws, ws_bytes, lanes);
  });
}

extern "C" fq_status floquet_batch_launch(fq_batch* b, void* stream) {
  if (!b || !b->exec) {
    fq_set_error("floquet_batch_launch: NULL batch");
    return FQ_EINVAL;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? FQ_OK : fq_cuda_fail(e, "batch graph launch");
}

extern "C" void floquet_batch_destroy(fq_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
}
