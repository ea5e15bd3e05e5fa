// batch.cu - the batched form: several blocks of uneven receiver shapes in
// one graph-captured pass (mraid_batch_*).
//
// Each unit owns a plan (its buffers are allocated at mraid_batch_plan, so
// nothing allocates during capture) bound to a side stream forked from the
// batch stream. The whole pass - every unit's Gram, eigen and masking
// kernels, and the info copies - is captured once into a CUDA graph. Two
// packings exist: the units as independent branches (the GPU runs them
// concurrently, so small units fill the SMs large ones leave idle) or
// chained one after another (no contention when every unit fills the GPU
// on its own); the first call times both and keeps the faster. A call with
// different buffers re-captures and rebinds them into the existing
// executable graph with cudaGraphExecUpdate.
#include <cuda_runtime.h>
#include <string.h>

#include <new>
#include <vector>

#include "internal.h"

struct mraid_batch_s {
  int device = 0;
  cudaStream_t user = nullptr;    // the caller's stream (may be the legacy default stream)
  cudaStream_t stream = nullptr;  // the batch's own stream: capture and graph launches
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<mraid_plan_s*> plans;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<mraid_unit_io> bound;
  std::vector<mraid_flag_info*> infos;
  int instantiations = 0, updates = 0;
  int packing = -1;                     // 0 concurrent branches, 1 chained; -1 not yet tuned
  float packing_ms[2] = {-1.f, -1.f};   // measured pass time of each packing
};

using namespace mraid;

namespace {

bool same_io(const std::vector<mraid_unit_io>& a, const mraid_unit_io* b) {
  for (size_t i = 0; i < a.size(); ++i)
    if (memcmp(&a[i], &b[i], sizeof(mraid_unit_io)) != 0) return false;
  return true;
}

mraid_status capture(mraid_batch_s* bt, const mraid_unit_io* io, int packing, cudaGraph_t* graph) {
  cudaError_t e = cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "batch capture begin");
  mraid_status st = MRAID_OK;
  e = cudaEventRecord(bt->fork, bt->stream);
  for (size_t i = 0; i < bt->plans.size() && e == cudaSuccess && st == MRAID_OK; ++i) {
    // concurrent: every unit starts at the fork; chained: after the previous unit
    e = cudaStreamWaitEvent(bt->side[i], (packing == 1 && i > 0) ? bt->join[i - 1] : bt->fork, 0);
    if (e != cudaSuccess) break;
    st = mraid_run(bt->plans[i], io[i].d_data, io[i].d_evals, io[i].d_q1, io[i].d_stat,
                   io[i].d_flags, nullptr);
    if (st == MRAID_OK) e = cudaEventRecord(bt->join[i], bt->side[i]);
    if (e == cudaSuccess && st == MRAID_OK) e = cudaStreamWaitEvent(bt->stream, bt->join[i], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(bt->stream, &g);
  if (st != MRAID_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e, "batch capture");
  }
  *graph = g;
  return MRAID_OK;
}

// Time both packings on the caller's buffers (one warm-up and two timed
// launches each, after the caller's stream) and keep the faster; its
// executable graph becomes the batch's.
mraid_status tune_packing(mraid_batch_s* bt, const mraid_unit_io* io) {
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) e = cudaEventRecord(bt->ev_in, bt->user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(bt->stream, bt->ev_in, 0);
  cudaGraphExec_t ex[2] = {nullptr, nullptr};
  mraid_status st = MRAID_OK;
  for (int p = 0; p < 2 && e == cudaSuccess && st == MRAID_OK; ++p) {
    cudaGraph_t g = nullptr;
    st = capture(bt, io, p, &g);
    if (st != MRAID_OK) break;
    e = cudaGraphInstantiate(&ex[p], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) break;
    ++bt->instantiations;
    e = cudaGraphLaunch(ex[p], bt->stream);
    if (e == cudaSuccess) e = cudaEventRecord(t0, bt->stream);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = cudaGraphLaunch(ex[p], bt->stream);
    if (e == cudaSuccess) e = cudaEventRecord(t1, bt->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    bt->packing_ms[p] = ms / 2.f;
  }
  if (e == cudaSuccess && st == MRAID_OK) {
    const int best = bt->packing_ms[1] < bt->packing_ms[0] ? 1 : 0;
    bt->packing = best;
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    bt->exec = ex[best];
    ex[best] = nullptr;
    bt->bound.assign(io, io + bt->plans.size());
  }
  for (auto x : ex)
    if (x) cudaGraphExecDestroy(x);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (st != MRAID_OK) return st;
  return e == cudaSuccess ? MRAID_OK : cuda_fail(e, "batch packing");
}

}  // namespace

extern "C" {

mraid_status mraid_batch_plan(const mraid_params* params, int32_t n_units, void* stream,
                              mraid_batch_t* out) {
  if (!out || !params || n_units < 1 || n_units > 4096) {
    set_error("mraid_batch_plan: params, out and 1..4096 units are required");
    return MRAID_ERR_INVALID_ARG;
  }
  *out = nullptr;
  for (int32_t i = 0; i < n_units; ++i) {
    mraid_status st = mraid_validate(&params[i]);
    if (st != MRAID_OK) return st;
  }
  mraid_batch_s* bt = new (std::nothrow) mraid_batch_s();
  if (!bt) {
    set_error("host allocation failed");
    return MRAID_ERR_OOM;
  }
  bt->user = static_cast<cudaStream_t>(stream);
  mraid_status st = MRAID_OK;
  cudaError_t e = cudaGetDevice(&bt->device);
  // the legacy default stream cannot be captured: the batch captures and
  // launches on a stream of its own, ordered after / before the caller's
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming);
  for (int32_t i = 0; i < n_units && e == cudaSuccess && st == MRAID_OK; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t j = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    bt->side.push_back(s);
    e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    bt->join.push_back(j);
    mraid_plan_t pl = nullptr;
    st = mraid_plan(&params[i], s, &pl);
    if (st != MRAID_OK) break;
    bt->plans.push_back(pl);
    st = plan_prepare(pl);
  }
  if (e == cudaSuccess && st == MRAID_OK) e = cudaDeviceSynchronize();
  if (e != cudaSuccess || st != MRAID_OK) {
    if (st == MRAID_OK) st = cuda_fail(e, "mraid_batch_plan");
    mraid_batch_destroy(bt);
    return st;
  }
  bt->infos.assign((size_t)n_units, nullptr);
  *out = bt;
  return MRAID_OK;
}

mraid_status mraid_batch_run(mraid_batch_t bt, const mraid_unit_io* io, mraid_flag_info* infos) {
  if (!bt || !io) {
    set_error("mraid_batch_run: batch and io are required");
    return MRAID_ERR_INVALID_ARG;
  }
  for (size_t i = 0; i < bt->plans.size(); ++i) {
    if (!io[i].d_data || !io[i].d_stat || !io[i].d_flags) {
      set_error("mraid_batch_run: unit %zu lacks d_data, d_stat or d_flags", i);
      return MRAID_ERR_INVALID_ARG;
    }
  }
  cudaError_t e = cudaSetDevice(bt->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  if (bt->packing < 0) {
    mraid_status st = tune_packing(bt, io);
    if (st != MRAID_OK) return st;
  }
  if (!bt->exec || !same_io(bt->bound, io)) {
    cudaGraph_t g = nullptr;
    mraid_status st = capture(bt, io, bt->packing, &g);
    if (st != MRAID_OK) return st;
    bool updated = false;
    if (bt->exec) {
      cudaGraphExecUpdateResultInfo res;
      if (cudaGraphExecUpdate(bt->exec, g, &res) == cudaSuccess) {
        updated = true;
        ++bt->updates;
      } else {
        cudaGetLastError();
        cudaGraphExecDestroy(bt->exec);
        bt->exec = nullptr;
      }
    }
    if (!updated) {
      e = cudaGraphInstantiate(&bt->exec, g, 0);
      if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        bt->exec = nullptr;
        return cuda_fail(e, "batch graph instantiate");
      }
      ++bt->instantiations;
    }
    cudaGraphDestroy(g);
    bt->bound.assign(io, io + bt->plans.size());
  }
  e = cudaEventRecord(bt->ev_in, bt->user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(bt->stream, bt->ev_in, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(bt->exec, bt->stream);
  if (e == cudaSuccess) e = cudaEventRecord(bt->ev_out, bt->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(bt->user, bt->ev_out, 0);
  if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
  for (size_t i = 0; i < bt->plans.size(); ++i) {
    bt->infos[i] = infos ? &infos[i] : nullptr;
    bt->plans[i]->pending_info = bt->infos[i];
  }
  return MRAID_OK;
}

mraid_status mraid_batch_sync(mraid_batch_t bt) {
  if (!bt) {
    set_error("batch is NULL");
    return MRAID_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaStreamSynchronize(bt->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mraid_batch_sync");
  mraid_status worst = MRAID_OK;
  for (auto* pl : bt->plans) {
    mraid_status st = mraid_sync(pl);  // delivers the unit's info, reports its errors
    if (st != MRAID_OK && worst == MRAID_OK) worst = st;
  }
  return worst;
}

mraid_status mraid_batch_graph_stats(mraid_batch_t bt, int32_t* instantiations, int32_t* updates) {
  if (!bt || !instantiations || !updates) {
    set_error("mraid_batch_graph_stats: bad arguments");
    return MRAID_ERR_INVALID_ARG;
  }
  *instantiations = bt->instantiations;
  *updates = bt->updates;
  return MRAID_OK;
}

mraid_status mraid_batch_packing(mraid_batch_t bt, int32_t* packing, float* ms_concurrent,
                                 float* ms_chained) {
  if (!bt || !packing) {
    set_error("mraid_batch_packing: bad arguments");
    return MRAID_ERR_INVALID_ARG;
  }
  *packing = bt->packing;
  if (ms_concurrent) *ms_concurrent = bt->packing_ms[0];
  if (ms_chained) *ms_chained = bt->packing_ms[1];
  return MRAID_OK;
}

void mraid_batch_destroy(mraid_batch_t bt) {
  if (!bt) return;
  if (bt->stream) cudaStreamSynchronize(bt->stream);
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  for (auto* pl : bt->plans) mraid_destroy(pl);
  for (auto s : bt->side) cudaStreamDestroy(s);
  for (auto j : bt->join) cudaEventDestroy(j);
  if (bt->fork) cudaEventDestroy(bt->fork);
  if (bt->ev_in) cudaEventDestroy(bt->ev_in);
  if (bt->ev_out) cudaEventDestroy(bt->ev_out);
  if (bt->stream) cudaStreamDestroy(bt->stream);
  delete bt;
}

}  // extern "C"
