// Serving loop: continuous batching of TNEP evaluation requests.
//
// Requests (one structure each, any size, open or periodic) are copied in by
// tnep_submit and admitted while the device-memory budget and the request
// slots allow.  Up to `n_pipelines` batches are in flight, each on its own
// stream with its own resident workspace: whenever a pipeline is free, every
// pending request (up to max_batch_atoms) is launched on it as one batch
// through the whole path (cell lists, neighbour lists, radial moments, fused
// kernels, FP64 reduction), so requests that arrive while others run are
// batched together and overlap them on the device.  A request that finds a
// pipeline free and nothing queued is launched by the submitting thread
// itself (no hand-off to the worker); the worker launches everything else
// and, while batches are in flight, polls their completion events without
// sleeping.  Each structure's result is bitwise the same alone or in any
// batch (fixed per-structure reduction order).  All waits are bounded.

#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "engine.h"

using namespace tnep;
using Clock = std::chrono::steady_clock;

namespace {

struct ServeRequest {
  uint64_t ticket = 0;
  int n_atoms = 0;
  std::vector<float> pos;
  std::vector<int> types;
  float box[3] = {0.f, 0.f, 0.f};
  size_t bytes = 0;
  Clock::time_point t_submit;
  std::vector<double> out;
  bool done = false;
  tnep_status status = TNEP_OK;
  double latency_s = 0.0;
};
using ReqPtr = std::shared_ptr<ServeRequest>;

struct Pipeline {
  Workspace ws;
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  PinBuf<float> h_pos, h_box;
  PinBuf<int> h_types;
  PinBuf<double> h_out;
  DevBuf<float> d_pos, d_box;
  DevBuf<int> d_types;
  std::vector<ReqPtr> batch;
  std::vector<int> offsets;
  bool busy = false;
};

// Device bytes one atom of a request occupies while it is in flight
// (positions, lists, moments, per-atom outputs).
size_t bytes_per_atom(const tnep_ctx* c) {
  return 16 + 12 + 4 + (size_t)(2 * c->cap_R + c->cap_A) * 4 + (size_t)c->n_types * kMomBasis * 10 * 4 +
         (size_t)9 * 4 * c->models.size() + (c->pair_cache ? (size_t)c->cap_A * 4 * sizeof(float4) : 0) + 64;
}

}  // namespace

struct tnep_server {
  tnep_ctx* ctx = nullptr;
  size_t budget = 0, in_use = 0;
  int max_slots = 0, max_batch_atoms = 0;
  int n_inflight = 0;  // admitted, not yet completed
  std::vector<std::unique_ptr<Pipeline>> pipes;
  std::deque<ReqPtr> pending;
  std::unordered_map<uint64_t, ReqPtr> table;
  std::mutex mu;           // requests: pending queue, ticket table, counters
  std::mutex dispatch_mu;  // pipelines: busy flags, batches, launches (taken before mu)
  std::condition_variable cv_done, cv_work;
  std::thread worker;
  std::atomic<bool> stop{false};
  std::atomic<int> callers{0};  // calls on the server in progress; stop waits for them
  uint64_t next_ticket = 1;
  uint64_t n_completed = 0, n_batches = 0, n_atoms_done = 0;
};

namespace {

// Counts a call in progress for the lifetime of the guard.
struct CallGuard {
  tnep_server* s;
  explicit CallGuard(tnep_server* srv) : s(srv) { if (s) s->callers.fetch_add(1); }
  ~CallGuard() { if (s) s->callers.fetch_sub(1); }
};

void finish_request(tnep_server* s, const ReqPtr& r, tnep_status st) {
  r->status = st;
  r->done = true;
  r->latency_s = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
  s->in_use -= r->bytes;
  s->n_inflight -= 1;
  s->n_completed += 1;
}

// Stages the batch's inputs and enqueues the whole path on the pipeline stream.
tnep_status launch_batch(tnep_server* s, Pipeline& p) {
  tnep_ctx* c = s->ctx;
  const int S = (int)p.batch.size();
  p.offsets.assign(S + 1, 0);
  for (int k = 0; k < S; ++k) p.offsets[k + 1] = p.offsets[k] + p.batch[k]->n_atoms;
  const int N = p.offsets[S];
  TNEP_CUDA(p.h_pos.ensure((size_t)std::max(N, 1) * 3));
  TNEP_CUDA(p.h_types.ensure((size_t)std::max(N, 1)));
  TNEP_CUDA(p.h_box.ensure((size_t)S * 3));
  TNEP_CUDA(p.h_out.ensure((size_t)S * total_C(c) + 1));
  for (int k = 0; k < S; ++k) {
    const ServeRequest& r = *p.batch[k];
    std::memcpy(p.h_pos.p + (size_t)p.offsets[k] * 3, r.pos.data(), sizeof(float) * 3 * r.n_atoms);
    std::memcpy(p.h_types.p + p.offsets[k], r.types.data(), sizeof(int) * r.n_atoms);
    std::memcpy(p.h_box.p + 3 * k, r.box, sizeof(float) * 3);
  }
  TNEP_CUDA(p.d_pos.ensure((size_t)std::max(N, 1) * 3));
  TNEP_CUDA(p.d_types.ensure((size_t)std::max(N, 1)));
  TNEP_CUDA(p.d_box.ensure((size_t)S * 3));
  cudaStream_t st = p.stream;
  if (N > 0) {
    TNEP_CUDA(cudaMemcpyAsync(p.d_pos.p, p.h_pos.p, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, st));
    TNEP_CUDA(cudaMemcpyAsync(p.d_types.p, p.h_types.p, sizeof(int) * N, cudaMemcpyHostToDevice, st));
  }
  TNEP_CUDA(cudaMemcpyAsync(p.d_box.p, p.h_box.p, sizeof(float) * 3 * S, cudaMemcpyHostToDevice, st));
  TNEP_TRY(reset_status(p.ws, st));
  TNEP_TRY(build_lists(c, p.ws, st, S, p.offsets.data(), p.d_pos.p, p.d_box.p, p.d_types.p, std::max(N, 1)));
  TNEP_TRY(run_models(c, p.ws, st, S, N, nullptr));
  TNEP_CUDA(cudaMemcpyAsync(p.h_out.p, p.ws.out.p, sizeof(double) * S * total_C(c), cudaMemcpyDeviceToHost, st));
  TNEP_CUDA(cudaMemcpyAsync(p.ws.h_status.p, p.ws.d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  TNEP_CUDA(cudaEventRecord(p.done_ev, st));
  return TNEP_OK;
}

// Called with the pipeline's event complete.  Returns true when the batch was
// relaunched (neighbour lists regrown) instead of completed.
bool complete_batch(tnep_server* s, Pipeline& p) {
  tnep_ctx* c = s->ctx;
  bool regrow = false;
  tnep_status st = check_status(c, *p.ws.h_status.p, &regrow);
  if (st == TNEP_OK && regrow) {
    st = launch_batch(s, p);
    if (st == TNEP_OK) return true;
  }
  const int S = (int)p.batch.size();
  const int Ctot = total_C(c);
  std::lock_guard<std::mutex> lock(s->mu);
  for (int k = 0; k < S; ++k) {
    ServeRequest& r = *p.batch[k];
    if (st == TNEP_OK) {
      r.out.resize(Ctot);
      size_t off = 0, o = 0;
      for (const auto& m : c->models) {
        for (int q = 0; q < m.C; ++q) r.out[o + q] = p.h_out.p[off + (size_t)k * m.C + q];
        off += (size_t)S * m.C;
        o += m.C;
      }
      s->n_atoms_done += r.n_atoms;
    }
    finish_request(s, p.batch[k], st);
  }
  s->n_batches += 1;
  p.batch.clear();
  p.busy = false;
  s->cv_done.notify_all();
  return false;
}

// Launches pending requests on every free pipeline.  Caller holds
// dispatch_mu.  Returns true if anything was launched.
bool dispatch_pending(tnep_server* s) {
  bool launched = false;
  for (auto& pp : s->pipes) {
    Pipeline& p = *pp;
    if (p.busy) continue;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if (s->pending.empty()) break;
      long long atoms = 0;
      while (!s->pending.empty()) {
        const ReqPtr& r = s->pending.front();
        if (!p.batch.empty() && atoms + r->n_atoms > s->max_batch_atoms) break;
        atoms += r->n_atoms;
        p.batch.push_back(r);
        s->pending.pop_front();
      }
    }
    p.busy = true;
    launched = true;
    const tnep_status st = launch_batch(s, p);
    if (st != TNEP_OK) {
      std::lock_guard<std::mutex> lock(s->mu);
      for (auto& r : p.batch) finish_request(s, r, st);
      p.batch.clear();
      p.busy = false;
      s->cv_done.notify_all();
    }
  }
  return launched;
}

// Completes every finished batch.  Caller holds dispatch_mu.  Returns
// (progressed, pipelines still busy).
std::pair<bool, int> poll_completions(tnep_server* s) {
  bool progressed = false;
  int busy = 0;
  for (auto& pp : s->pipes) {
    Pipeline& p = *pp;
    if (!p.busy) continue;
    const cudaError_t q = cudaEventQuery(p.done_ev);
    if (q == cudaSuccess) {
      complete_batch(s, p);
      progressed = true;
    } else if (q != cudaErrorNotReady) {
      cudaGetLastError();
      std::lock_guard<std::mutex> lock(s->mu);
      for (auto& r : p.batch) finish_request(s, r, TNEP_ERR_CUDA);
      p.batch.clear();
      p.busy = false;
      s->cv_done.notify_all();
      progressed = true;
    }
    busy += p.busy;
  }
  return {progressed, busy};
}

void worker_loop(tnep_server* s) {
  cudaSetDevice(s->ctx->device);
  for (;;) {
    bool progressed;
    int busy;
    {
      std::lock_guard<std::mutex> dl(s->dispatch_mu);
      auto pr = poll_completions(s);
      progressed = pr.first;
      busy = pr.second;
      if (dispatch_pending(s)) {
        progressed = true;
        busy = 0;
        for (auto& pp : s->pipes) busy += pp->busy;
      }
    }
    if (s->stop.load() && busy == 0) {
      std::lock_guard<std::mutex> lock(s->mu);
      if (s->pending.empty()) break;
    }
    if (progressed) continue;
    if (busy) {
      // batches in flight: poll their events again at once (the result is on
      // the host as soon as the event completes)
      std::this_thread::yield();
      continue;
    }
    std::unique_lock<std::mutex> lock(s->mu);
    // idle: a submit or stop wakes us; bounded so that nothing is missed
    if (s->pending.empty() && !s->stop.load()) s->cv_work.wait_for(lock, std::chrono::milliseconds(2));
  }
}

}  // namespace

extern "C" {

tnep_status tnep_server_start(tnep_ctx* ctx, size_t mem_budget_bytes, int max_slots, int n_pipelines,
                              int max_batch_atoms, tnep_server** out) {
  if (!out) return fail(TNEP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!ctx) return fail(TNEP_ERR_INVALID, "ctx is NULL");
  if (max_slots < 1 || n_pipelines < 1 || n_pipelines > 16 || max_batch_atoms < 1 ||
      max_batch_atoms >= kMaxBatchAtoms || mem_budget_bytes == 0)
    return fail(TNEP_ERR_INVALID, "bad server limits");
  TNEP_CUDA(cudaSetDevice(ctx->device));
  auto* s = new (std::nothrow) tnep_server();
  if (!s) return fail(TNEP_ERR_OOM, "host allocation failed");
  s->ctx = ctx;
  s->budget = mem_budget_bytes;
  s->max_slots = max_slots;
  s->max_batch_atoms = max_batch_atoms;
  for (int k = 0; k < n_pipelines; ++k) {
    auto p = std::make_unique<Pipeline>();
    cudaError_t e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void**>(&p->ws.d_status), sizeof(DevStatus));
    if (e == cudaSuccess) e = p->ws.h_status.ensure(1);
    s->pipes.push_back(std::move(p));
    if (e != cudaSuccess) {
      tnep_server_stop(s);
      return cuda_fail(e, "server pipeline setup");
    }
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return TNEP_OK;
}

tnep_status tnep_submit(tnep_server* s, const tnep_request* req, uint64_t* ticket) {
  CallGuard guard(s);
  if (!s || !req || !ticket) return fail(TNEP_ERR_INVALID, "NULL argument");
  if (s->stop.load()) return fail(TNEP_ERR_INVALID, "server is stopping");
  const int n = req->n_atoms;
  if (n < 0 || n >= s->max_batch_atoms + 1 || (n > 0 && (!req->pos || !req->types)))
    return fail(TNEP_ERR_INVALID, "bad request size or NULL buffer");
  for (int a = 0; a < n; ++a)
    if (req->types[a] < 0 || req->types[a] >= s->ctx->n_types) return fail(TNEP_ERR_INVALID, "type out of range");
  if (req->box)
    for (int d = 0; d < 3; ++d)
      if (req->box[d] > 0.f && req->box[d] < 2.f * s->ctx->rc_R)
        return fail(TNEP_ERR_BOX_TOO_SMALL, "periodic edge < 2 rc_R");
  auto r = std::make_shared<ServeRequest>();
  r->n_atoms = n;
  r->pos.assign(req->pos, req->pos + 3 * (size_t)n);
  r->types.assign(req->types, req->types + n);
  if (req->box) std::memcpy(r->box, req->box, sizeof(float) * 3);
  r->bytes = (size_t)std::max(n, 1) * bytes_per_atom(s->ctx);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    // checked again under the lock the worker takes before it exits: a
    // submit that races tnep_server_stop is either served or refused here
    if (s->stop.load()) return fail(TNEP_ERR_INVALID, "server is stopping");
    if (s->n_inflight >= s->max_slots) return fail(TNEP_ERR_BUSY, "no free request slot");
    if (s->in_use + r->bytes > s->budget && s->n_inflight > 0)
      return fail(TNEP_ERR_BUSY, "device-memory budget exhausted");
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    s->in_use += r->bytes;
    s->n_inflight += 1;
    s->table[r->ticket] = r;
    s->pending.push_back(r);
  }
  *ticket = r->ticket;
  // A free pipeline: launch from this thread at once.  If the worker holds
  // the pipelines, it launches the request on its next pass.
  {
    std::unique_lock<std::mutex> dl(s->dispatch_mu, std::try_to_lock);
    if (dl.owns_lock()) {
      int prev = -1;
      const bool switch_dev = cudaGetDevice(&prev) == cudaSuccess && prev != s->ctx->device;
      if (!switch_dev || cudaSetDevice(s->ctx->device) == cudaSuccess) {
        dispatch_pending(s);
        if (switch_dev) cudaSetDevice(prev);
      } else {
        cudaGetLastError();  // the worker launches the request instead
      }
    }
  }
  s->cv_work.notify_one();
  return TNEP_OK;
}

static tnep_status take_result(tnep_server* s, uint64_t ticket, double* out, double* latency_s) {
  auto it = s->table.find(ticket);
  const ReqPtr r = it->second;
  s->table.erase(it);
  if (latency_s) *latency_s = r->latency_s;
  if (r->status != TNEP_OK) return fail(r->status, "request failed on the device");
  if (out) std::memcpy(out, r->out.data(), sizeof(double) * r->out.size());
  return TNEP_OK;
}

tnep_status tnep_poll(tnep_server* s, uint64_t ticket, double* out, int* done, double* latency_s) {
  CallGuard guard(s);
  if (!s || !done) return fail(TNEP_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return fail(TNEP_ERR_INVALID, "unknown ticket");
  *done = it->second->done ? 1 : 0;
  if (!*done) return TNEP_OK;
  return take_result(s, ticket, out, latency_s);
}

tnep_status tnep_wait(tnep_server* s, uint64_t ticket, double* out, double timeout_s, double* latency_s) {
  CallGuard guard(s);
  if (!s) return fail(TNEP_ERR_INVALID, "NULL argument");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return fail(TNEP_ERR_INVALID, "unknown ticket");
  const ReqPtr r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration<double>(std::max(timeout_s, 0.0));
  while (!r->done) {
    if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && !r->done)
      return fail(TNEP_ERR_TIMEOUT, "request not finished before the timeout");
  }
  return take_result(s, ticket, out, latency_s);
}

tnep_status tnep_server_stats(tnep_server* s, double stats[6]) {
  CallGuard guard(s);
  if (!s || !stats) return fail(TNEP_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  stats[0] = (double)s->n_completed;
  stats[1] = (double)s->n_batches;
  stats[2] = (double)s->n_atoms_done;
  stats[3] = (double)s->in_use;
  stats[4] = (double)s->n_inflight;
  stats[5] = (double)s->pending.size();
  return TNEP_OK;
}

void tnep_server_stop(tnep_server* s) {
  if (!s) return;
  s->stop.store(true);
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  // every admitted request has finished, so waiting callers wake; calls
  // already in progress return before the server is freed
  while (s->callers.load() != 0) {
    s->cv_done.notify_all();
    std::this_thread::yield();
  }
  {
    std::lock_guard<std::mutex> dl(s->dispatch_mu);  // a submit's own dispatch has finished
    cudaSetDevice(s->ctx->device);
    for (auto& p : s->pipes) {
      if (p->stream) cudaStreamSynchronize(p->stream);
      p->ws.release();
      p->h_pos.release(); p->h_box.release(); p->h_types.release(); p->h_out.release();
      p->d_pos.release(); p->d_box.release(); p->d_types.release();
      if (p->done_ev) cudaEventDestroy(p->done_ev);
      if (p->stream) cudaStreamDestroy(p->stream);
    }
  }
  delete s;
}

}  // extern "C"
