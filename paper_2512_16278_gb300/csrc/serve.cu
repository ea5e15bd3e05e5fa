// serve.cu - the served form (mraid_serve_*): continuous batching of blocks
// from several concurrent observations.
//
// A server thread owns the GPU work. Submitted blocks wait in a FIFO queue;
// a block is admitted when its observation has a free staging buffer, the
// number of blocks on the GPU is below max_inflight and, for the first block
// of an observation, its buffers fit the HBM budget. An admitted block is
// enqueued on its observation's CUDA stream: the samples carried over from
// the previous block are copied to the head of the block's staging buffer,
// the new samples are copied in after them, the whole sub-integrations go
// through mraid_run, the flags are copied to the caller's buffer and an
// event marks completion. Observations have their own streams, so their
// blocks overlap on the device. The server polls events, stamps latencies
// and moves finished blocks to the result queue.
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Pending {
  int stream;
  const void* h_block;
  uint8_t* h_flags;
  int64_t seq;
  Clock::time_point t_submit;
};

struct Running {
  Pending p;
  int buf;
  int n_sub;
  cudaEvent_t start, done;
  mraid_flag_info* h_info;  // pinned, per staging buffer
};

struct Obs {
  mraid_stream_desc d;
  cudaStream_t cs = nullptr;
  bool allocated = false;
  uint8_t* d_buf[2] = {nullptr, nullptr};  // [beam][cap][chan]
  float* d_stat[2] = {nullptr, nullptr};
  uint8_t* d_flags[2] = {nullptr, nullptr};
  mraid_flag_info* h_info[2] = {nullptr, nullptr};
  bool busy[2] = {false, false};
  cudaEvent_t ev_start[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
  int64_t cap = 0;       // samples per staging buffer (block + carry room)
  int carry = 0;         // samples carried into the next block
  int carry_buf = 0;     // buffer holding the carry (tail of the last block)
  int carry_from = 0;    // first carried sample in that buffer
  int last_buf = 1;      // buffer of the last admitted block
  int n_lo = 0;          // fewest whole sub-integrations a block can hold
  mraid_plan_t plan[2] = {nullptr, nullptr};  // n_lo and n_lo + 1
  size_t bytes = 0;
  int64_t blocks = 0, flagged = 0;
};

}  // namespace

struct mraid_server_s {
  int device = 0;
  std::vector<Obs> obs;
  int64_t budget = 0, used = 0;
  int max_inflight = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Pending> queue;
  std::vector<Running> running;
  std::deque<mraid_block_result> done;
  int64_t submitted = 0, finished = 0;
  bool stop = false;
  std::thread th;
};

using namespace mraid;

namespace {

// Bytes the observation's buffers take on the device (staging, outputs and
// the plans' work buffers).
size_t obs_bytes(const Obs& o) {
  const mraid_params& p = o.d.params;
  const size_t cells = (size_t)(o.n_lo + 1) * p.n_chan;
  const size_t np = (size_t)p.n_beam * (p.n_beam + 1) / 2, psum = (size_t)(p.n_beam + 1) * (p.n_beam + 2) / 2;
  const size_t per_plan = cells * (np * 4 + psum * 8 + (size_t)p.n_beam * 4);
  return 2 * ((size_t)p.n_beam * o.cap * p.n_chan + cells * 5) + 2 * per_plan;
}

mraid_status obs_allocate(Obs& o) {
  mraid_params p = o.d.params;
  cudaError_t e = cudaStreamCreateWithFlags(&o.cs, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    const size_t cells = (size_t)(o.n_lo + 1) * p.n_chan;
    e = cudaMalloc(&o.d_buf[i], (size_t)p.n_beam * o.cap * p.n_chan);
    if (e == cudaSuccess) e = cudaMalloc(&o.d_stat[i], cells * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&o.d_flags[i], cells);
    if (e == cudaSuccess) e = cudaMallocHost(&o.h_info[i], sizeof(mraid_flag_info));
    if (e == cudaSuccess) e = cudaEventCreate(&o.ev_start[i]);
    if (e == cudaSuccess) e = cudaEventCreate(&o.ev_done[i]);
  }
  if (e != cudaSuccess) return cuda_fail(e, "serve: stream buffers");
  for (int k = 0; k < 2; ++k) {
    if (o.n_lo + k < 1) continue;  // a block with no whole sub-integration
    p.n_sub = o.n_lo + k;
    p.beam_stride = o.cap * p.n_chan;
    mraid_status st = mraid_plan(&p, o.cs, &o.plan[k]);
    if (st != MRAID_OK) return st;
    st = plan_prepare(o.plan[k]);
    if (st != MRAID_OK) return st;
  }
  o.allocated = true;
  return MRAID_OK;
}

void obs_free(Obs& o) {
  if (o.cs) cudaStreamSynchronize(o.cs);
  for (int k = 0; k < 2; ++k) {
    mraid_destroy(o.plan[k]);
    cudaFree(o.d_buf[k]);
    cudaFree(o.d_stat[k]);
    cudaFree(o.d_flags[k]);
    if (o.h_info[k]) cudaFreeHost(o.h_info[k]);
    if (o.ev_start[k]) cudaEventDestroy(o.ev_start[k]);
    if (o.ev_done[k]) cudaEventDestroy(o.ev_done[k]);
  }
  if (o.cs) cudaStreamDestroy(o.cs);
}

// Enqueue one admitted block on its observation's stream.
mraid_status launch_block(mraid_server_s* sv, const Pending& pd, Running* r) {
  Obs& o = sv->obs[pd.stream];
  const mraid_params& p = o.d.params;
  const int b = o.last_buf ^ 1;  // the other buffer; the stream order makes it free
  const int64_t total = (int64_t)o.carry + o.d.block_samples;
  const int n_sub = (int)(total / p.n_samp_sub);
  const int rest = (int)(total - (int64_t)n_sub * p.n_samp_sub);
  cudaError_t e = cudaEventRecord(o.ev_start[b], o.cs);
  const size_t row = (size_t)p.n_chan;  // bytes per sample across channels
  // carry: the last `carry` samples of the previous block, to the head
  if (e == cudaSuccess && o.carry > 0)
    e = cudaMemcpy2DAsync(o.d_buf[b], (size_t)o.cap * row,
                          o.d_buf[o.carry_buf] + (size_t)o.carry_from * row, (size_t)o.cap * row,
                          (size_t)o.carry * row, (size_t)p.n_beam, cudaMemcpyDeviceToDevice, o.cs);
  // the new block after the carry, one 2-D copy over beams
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(o.d_buf[b] + (size_t)o.carry * row, (size_t)o.cap * row, pd.h_block,
                          (size_t)o.d.block_samples * row, (size_t)o.d.block_samples * row,
                          (size_t)p.n_beam, cudaMemcpyHostToDevice, o.cs);
  if (e != cudaSuccess) return cuda_fail(e, "serve: copy in");
  mraid_status st = MRAID_OK;
  if (n_sub > 0) {
    mraid_plan_t pl = o.plan[n_sub - o.n_lo];
    st = mraid_run(pl, o.d_buf[b], nullptr, nullptr, o.d_stat[b], o.d_flags[b], nullptr);
    if (st != MRAID_OK) return st;
    e = cudaMemcpyAsync(o.h_info[b], pl->d_info, sizeof(mraid_flag_info), cudaMemcpyDeviceToHost,
                        o.cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(pd.h_flags, o.d_flags[b], (size_t)n_sub * p.n_chan,
                          cudaMemcpyDeviceToHost, o.cs);
  }
  if (e == cudaSuccess) e = cudaEventRecord(o.ev_done[b], o.cs);
  if (e != cudaSuccess) return cuda_fail(e, "serve: launch");
  // the next block's carry is this block's tail
  o.carry_buf = b;
  o.carry_from = (int)((int64_t)n_sub * p.n_samp_sub);
  o.carry = rest;
  o.last_buf = b;
  o.busy[b] = true;
  r->p = pd;
  r->buf = b;
  r->n_sub = n_sub;
  r->start = o.ev_start[b];
  r->done = o.ev_done[b];
  r->h_info = o.h_info[b];
  return MRAID_OK;
}

void server_loop(mraid_server_s* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    // admission, FIFO: a block of an observation whose both buffers are busy
    // holds back later blocks of the same observation only
    bool progressed = false;
    for (auto it = sv->queue.begin(); it != sv->queue.end();) {
      if ((int)sv->running.size() >= sv->max_inflight) break;
      Obs& o = sv->obs[it->stream];
      bool blocked_earlier = false;
      for (auto jt = sv->queue.begin(); jt != it; ++jt)
        if (jt->stream == it->stream) blocked_earlier = true;
      if (blocked_earlier || o.busy[o.last_buf ^ 1]) {
        ++it;
        continue;
      }
      if (!o.allocated) {
        const size_t need = obs_bytes(o);
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        if (sv->used + (int64_t)need > sv->budget || need > fr) {
          ++it;
          continue;  // wait for memory: nothing is freed before close, so only
                     // observations already holding buffers progress
        }
        if (obs_allocate(o) != MRAID_OK) {
          obs_free(o);
          Obs fresh;
          fresh.d = o.d;
          fresh.cap = o.cap;
          fresh.n_lo = o.n_lo;
          o = fresh;
          ++it;
          continue;
        }
        sv->used += (int64_t)need;
        o.bytes = need;
      }
      Running r;
      mraid_status st = launch_block(sv, *it, &r);
      if (st != MRAID_OK) {
        mraid_block_result res = {};
        res.stream = it->stream;
        res.seq = it->seq;
        res.status = st;
        sv->done.push_back(res);
        ++sv->finished;
      } else {
        sv->running.push_back(r);
      }
      it = sv->queue.erase(it);
      progressed = true;
    }
    // completion
    for (size_t i = 0; i < sv->running.size();) {
      Running& r = sv->running[i];
      cudaError_t q = cudaEventQuery(r.done);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      Obs& o = sv->obs[r.p.stream];
      mraid_block_result res = {};
      res.stream = r.p.stream;
      res.seq = r.p.seq;
      res.n_sub = r.n_sub;
      res.n_cells = (int64_t)r.n_sub * o.d.params.n_chan;
      res.latency_ms = ms_since(r.p.t_submit, Clock::now());
      float dms = 0.f;
      cudaEventElapsedTime(&dms, r.start, r.done);
      res.device_ms = dms;
      res.status = (q == cudaSuccess) ? MRAID_OK : MRAID_ERR_CUDA;
      if (r.n_sub > 0 && q == cudaSuccess) {
        res.n_flagged = r.h_info->n_flagged;
        res.mu = r.h_info->mu;
        res.sigma = r.h_info->sigma;
        res.thresh = r.h_info->thresh;
        o.flagged += res.n_flagged;
      }
      o.blocks += 1;
      o.busy[r.buf] = false;
      sv->done.push_back(res);
      ++sv->finished;
      sv->running.erase(sv->running.begin() + (long)i);
      progressed = true;
    }
    if (sv->stop && sv->queue.empty() && sv->running.empty()) break;
    if (progressed) {
      sv->cv.notify_all();
      continue;
    }
    // idle: short waits while blocks are on the GPU, else until a submit
    if (!sv->running.empty())
      sv->cv.wait_for(lk, std::chrono::microseconds(50));
    else
      sv->cv.wait_for(lk, std::chrono::milliseconds(5));
  }
  sv->cv.notify_all();
}

}  // namespace

extern "C" {

mraid_status mraid_serve_open(const mraid_stream_desc* streams, int32_t n_streams,
                              int64_t hbm_budget, int32_t max_inflight, mraid_server_t* out) {
  if (!out || !streams || n_streams < 1 || n_streams > 1024 || max_inflight < 1 ||
      hbm_budget < 0) {
    set_error("mraid_serve_open: bad arguments");
    return MRAID_ERR_INVALID_ARG;
  }
  *out = nullptr;
  for (int32_t i = 0; i < n_streams; ++i) {
    mraid_params p = streams[i].params;
    if (streams[i].block_samples < 1 || streams[i].reserved != 0) {
      set_error("mraid_serve_open: stream %d: block_samples must be >= 1", i);
      return MRAID_ERR_INVALID_ARG;
    }
    p.n_sub = 1;
    p.beam_stride = 0;
    mraid_status st = mraid_validate(&p);
    if (st != MRAID_OK) return st;
  }
  mraid_server_s* sv = new (std::nothrow) mraid_server_s();
  if (!sv) {
    set_error("host allocation failed");
    return MRAID_ERR_OOM;
  }
  cudaError_t e = cudaGetDevice(&sv->device);
  size_t fr = 0, tot = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
  if (e != cudaSuccess) {
    delete sv;
    return cuda_fail(e, "mraid_serve_open");
  }
  sv->budget = hbm_budget > 0 ? hbm_budget : (int64_t)(0.8 * (double)fr);
  sv->max_inflight = max_inflight;
  sv->obs.resize((size_t)n_streams);
  for (int32_t i = 0; i < n_streams; ++i) {
    Obs& o = sv->obs[(size_t)i];
    o.d = streams[i];
    o.d.params.keep = nullptr;
    const int ns = o.d.params.n_samp_sub;
    o.cap = (int64_t)o.d.block_samples + ns;  // room for a carry of < N_s samples
    o.n_lo = o.d.block_samples / ns;          // whole sub-integrations without carry
  }
  sv->th = std::thread(server_loop, sv);
  *out = sv;
  return MRAID_OK;
}

mraid_status mraid_serve_submit(mraid_server_t sv, int32_t stream, const void* h_block,
                                uint8_t* h_flags, int64_t seq) {
  if (!sv || !h_block || !h_flags || stream < 0 || stream >= (int32_t)sv->obs.size()) {
    set_error("mraid_serve_submit: bad arguments");
    return MRAID_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) {
    set_error("mraid_serve_submit: server is closing");
    return MRAID_ERR_INVALID_ARG;
  }
  sv->queue.push_back(Pending{stream, h_block, h_flags, seq, Clock::now()});
  ++sv->submitted;
  sv->cv.notify_all();
  return MRAID_OK;
}

mraid_status mraid_serve_poll(mraid_server_t sv, mraid_block_result* out, int32_t max,
                              int32_t* n) {
  if (!sv || !n || max < 0 || (max > 0 && !out)) {
    set_error("mraid_serve_poll: bad arguments");
    return MRAID_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  int32_t k = 0;
  while (k < max && !sv->done.empty()) {
    out[k++] = sv->done.front();
    sv->done.pop_front();
  }
  *n = k;
  return MRAID_OK;
}

mraid_status mraid_serve_drain(mraid_server_t sv, int32_t timeout_ms) {
  if (!sv) {
    set_error("server is NULL");
    return MRAID_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(sv->mu);
  const bool ok = sv->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                  [&] { return sv->finished == sv->submitted; });
  if (!ok) {
    set_error("mraid_serve_drain: %lld of %lld blocks finished", (long long)sv->finished,
              (long long)sv->submitted);
    return MRAID_ERR_TIMEOUT;
  }
  return MRAID_OK;
}

void mraid_serve_close(mraid_server_t sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->queue.clear();  // not yet admitted: dropped
    sv->cv.notify_all();
  }
  if (sv->th.joinable()) sv->th.join();
  int dev = -1;
  cudaGetDevice(&dev);
  cudaSetDevice(sv->device);
  for (auto& o : sv->obs) obs_free(o);
  if (dev >= 0) cudaSetDevice(dev);
  delete sv;
}

}  // extern "C"
