// Population evaluation for training-style use (Sec. II.D: the separable
// natural evolution strategy evaluates a population of parameter vectors on
// the training structures every generation).
//
// The neighbour lists and the radial moments depend only on the structures,
// so tnep_population_create builds them once.  The per-generation work --
// upload of the packed parameter vectors, one fused-kernel launch over all
// individuals x atoms, the FP64 per-structure reduction, the RMSE per
// individual and the read-back -- is captured once into a CUDA graph and
// replayed by tnep_population_eval.  The launch shape (atoms per CTA, and
// whether consecutive CTAs vary the individual or the atom block) is picked
// by timing the candidates on the actual structures.

#include <cuda_runtime.h>

#include <cstring>
#include <memory>
#include <vector>

#include "engine.h"

using namespace tnep;

struct tnep_population {
  tnep_ctx* ctx = nullptr;
  int model = 0, n_pop = 0, S = 0, N = 0, C = 0;
  Workspace ws;
  cudaStream_t stream = nullptr;
  std::vector<int> offsets;
  DevBuf<float> d_pos, d_box;
  DevBuf<int> d_types;
  DevBuf<float> d_params;
  PinBuf<float> h_params;
  DevBuf<double> d_target, d_rmse, d_pred;
  PinBuf<double> h_rmse, h_pred;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int block = 128, pop_major = 0;
  double tune_ms[4] = {0, 0, 0, 0};
  double last_ms = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

FusedArgs pop_args(tnep_population* p) {
  const Model& m = p->ctx->models[p->model];
  FusedArgs f = fused_args(p->ctx, p->ws, m, p->N);
  f.model = p->d_params.p;
  f.model_stride = m.lay.words;
  f.per_atom = p->ws.per_atom.p;
  f.per_atom_stride = (size_t)m.C * p->ws.atom_stride;
  f.pop_major = p->pop_major;
  return f;
}

// The per-generation device work on p->stream (no host synchronisation).
tnep_status enqueue_generation(tnep_population* p, bool with_copies) {
  const Model& m = p->ctx->models[p->model];
  cudaStream_t st = p->stream;
  if (with_copies)
    TNEP_CUDA(cudaMemcpyAsync(p->d_params.p, p->h_params.p, sizeof(float) * (size_t)p->n_pop * m.lay.words,
                              cudaMemcpyHostToDevice, st));
  FusedArgs f = pop_args(p);
  TNEP_CUDA(launch_fused(m.variant, m.d.rank, f, p->n_pop, p->block, m.d.mlp_precision, st));
  TNEP_CUDA(launch_reduce(p->S, p->n_pop, p->ws.offsets.p, p->ws.max_atoms, p->ws.per_atom.p, f.per_atom_stride,
                          p->ws.atom_stride, m.C, p->ws.partial.p, p->d_pred.p, (size_t)p->S * m.C, st));
  TNEP_CUDA(launch_rmse(p->n_pop, p->S, m.C, p->d_pred.p, p->d_target.p, p->d_rmse.p, st));
  if (with_copies) {
    TNEP_CUDA(cudaMemcpyAsync(p->h_rmse.p, p->d_rmse.p, sizeof(double) * p->n_pop, cudaMemcpyDeviceToHost, st));
    TNEP_CUDA(cudaMemcpyAsync(p->h_pred.p, p->d_pred.p, sizeof(double) * (size_t)p->n_pop * p->S * m.C,
                              cudaMemcpyDeviceToHost, st));
  }
  return TNEP_OK;
}

tnep_status pack_all(tnep_population* p, const float* params) {
  const Model& m = p->ctx->models[p->model];
  const size_t np = m.params.size();
  for (int k = 0; k < p->n_pop; ++k)
    pack_params(m, p->ctx->n_types, params + (size_t)k * np, m.scaler.data(), p->h_params.p + (size_t)k * m.lay.words);
  return TNEP_OK;
}

// Times the fused launch for each candidate shape and keeps the fastest.
tnep_status autotune(tnep_population* p) {
  const int blocks[2] = {128, 64};
  double best = 1e30;
  int best_b = 128, best_o = 0, idx = 0;
  TNEP_CUDA(cudaMemcpyAsync(p->d_params.p, p->h_params.p,
                            sizeof(float) * (size_t)p->n_pop * p->ctx->models[p->model].lay.words,
                            cudaMemcpyHostToDevice, p->stream));
  for (int b : blocks) {
    for (int order = 0; order < 2; ++order, ++idx) {
      p->block = b;
      p->pop_major = order;
      const int nblk = (p->N + b - 1) / b;
      const bool tc = p->ctx->models[p->model].d.mlp_precision != 0;
      if ((order == 1 && nblk > 65535) || (tc && b != 128)) { p->tune_ms[idx] = -1; continue; }
      TNEP_TRY(enqueue_generation(p, false));  // warm-up
      TNEP_CUDA(cudaEventRecord(p->ev0, p->stream));
      for (int r = 0; r < 3; ++r) TNEP_TRY(enqueue_generation(p, false));
      TNEP_CUDA(cudaEventRecord(p->ev1, p->stream));
      TNEP_CUDA(cudaEventSynchronize(p->ev1));
      float ms = 0.f;
      TNEP_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
      p->tune_ms[idx] = ms / 3.0;
      if (ms < best) { best = ms; best_b = b; best_o = order; }
    }
  }
  p->block = best_b;
  p->pop_major = best_o;
  return TNEP_OK;
}

void destroy_pop(tnep_population* p) {
  if (!p) return;
  cudaSetDevice(p->ctx->device);
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  p->ws.release();
  p->d_pos.release(); p->d_box.release(); p->d_types.release(); p->d_params.release(); p->h_params.release();
  p->d_target.release(); p->d_rmse.release(); p->d_pred.release(); p->h_rmse.release(); p->h_pred.release();
  if (p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

tnep_status create_pop(tnep_population* p, const float* params0, const float* pos, const float* box,
                       const int* types, const double* target) {
  tnep_ctx* c = p->ctx;
  const Model& m = c->models[p->model];
  const int S = p->S, N = p->N;
  TNEP_CUDA(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
  TNEP_CUDA(cudaEventCreate(&p->ev0));
  TNEP_CUDA(cudaEventCreate(&p->ev1));
  TNEP_CUDA(cudaMalloc(&p->ws.d_status, sizeof(DevStatus)));
  TNEP_CUDA(p->ws.h_status.ensure(1));
  cudaStream_t st = p->stream;
  TNEP_CUDA(p->d_pos.ensure((size_t)std::max(N, 1) * 3));
  TNEP_CUDA(p->d_types.ensure((size_t)std::max(N, 1)));
  TNEP_CUDA(p->d_box.ensure((size_t)S * 3));
  if (N > 0) {
    TNEP_CUDA(cudaMemcpyAsync(p->d_pos.p, pos, sizeof(float) * 3 * N, cudaMemcpyDefault, st));
    TNEP_CUDA(cudaMemcpyAsync(p->d_types.p, types, sizeof(int) * N, cudaMemcpyDefault, st));
  }
  if (box) {
    TNEP_CUDA(cudaMemcpyAsync(p->d_box.p, box, sizeof(float) * 3 * S, cudaMemcpyDefault, st));
  } else {
    TNEP_CUDA(cudaMemsetAsync(p->d_box.p, 0, sizeof(float) * 3 * S, st));
  }
  // lists and moments, regrown until they fit
  for (int attempt = 0;; ++attempt) {
    if (attempt == 4) return fail(TNEP_ERR_NEIGHBOR_OVERFLOW, "neighbour lists kept overflowing");
    TNEP_TRY(reset_status(p->ws, st));
    TNEP_TRY(build_lists(c, p->ws, st, S, p->offsets.data(), p->d_pos.p, p->d_box.p, p->d_types.p, std::max(N, 1)));
    bool regrow = false;
    TNEP_TRY(finish(c, p->ws, st, &regrow));
    if (!regrow) break;
  }
  TNEP_TRY(compute_moments(c, p->ws, st, N, m.d.rank == 1, m.d.rank == 2));
  const size_t pa = (size_t)m.C * p->ws.atom_stride * p->n_pop;
  TNEP_CUDA(p->ws.per_atom.ensure(pa));
  TNEP_CUDA(p->ws.partial.ensure((size_t)p->n_pop * S * reduce_chunks(p->ws.max_atoms) * m.C));
  TNEP_CUDA(p->d_params.ensure((size_t)p->n_pop * m.lay.words));
  TNEP_CUDA(p->h_params.ensure((size_t)p->n_pop * m.lay.words));
  TNEP_CUDA(p->d_target.ensure((size_t)S * m.C));
  TNEP_CUDA(cudaMemcpyAsync(p->d_target.p, target, sizeof(double) * S * m.C, cudaMemcpyDefault, st));
  TNEP_CUDA(p->d_rmse.ensure(p->n_pop));
  TNEP_CUDA(p->h_rmse.ensure(p->n_pop));
  TNEP_CUDA(p->d_pred.ensure((size_t)p->n_pop * S * m.C));
  TNEP_CUDA(p->h_pred.ensure((size_t)p->n_pop * S * m.C));
  TNEP_TRY(pack_all(p, params0));
  TNEP_TRY(autotune(p));
  TNEP_CUDA(cudaStreamSynchronize(st));
  // capture one generation
  TNEP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const tnep_status cap = enqueue_generation(p, true);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (cap != TNEP_OK) {
    if (g) cudaGraphDestroy(g);
    return cap;
  }
  TNEP_CUDA(e);
  p->graph = g;
  TNEP_CUDA(cudaGraphInstantiate(&p->exec, g, 0));
  return TNEP_OK;
}

}  // namespace

extern "C" {

tnep_status tnep_population_create(tnep_ctx* ctx, int model, int n_pop, const float* params, int n_structs,
                                   const int* atom_offsets, const float* pos, const float* box, const int* types,
                                   const double* target, tnep_population** out) {
  if (!out) return fail(TNEP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!ctx || model < 0 || model >= (int)ctx->models.size()) return fail(TNEP_ERR_INVALID, "bad context or model");
  if (n_pop < 1 || n_pop > 65535 || n_structs < 1) return fail(TNEP_ERR_INVALID, "need 1 <= n_pop <= 65535, n_structs >= 1");
  if (!params || !atom_offsets || !target) return fail(TNEP_ERR_INVALID, "NULL buffer");
  if (is_device_ptr(atom_offsets) || is_device_ptr(params))
    return fail(TNEP_ERR_INVALID, "atom_offsets and params must be host memory");
  if (atom_offsets[0] != 0) return fail(TNEP_ERR_INVALID, "atom_offsets[0] must be 0");
  for (int s = 0; s < n_structs; ++s)
    if (atom_offsets[s + 1] < atom_offsets[s]) return fail(TNEP_ERR_INVALID, "atom_offsets must not decrease");
  const int N = atom_offsets[n_structs];
  if (N >= kMaxBatchAtoms) return fail(TNEP_ERR_INVALID, "fewer than 2^29 atoms");
  if (N > 0 && (!pos || !types)) return fail(TNEP_ERR_INVALID, "NULL buffer");
  if (!is_device_ptr(types))
    for (int a = 0; a < N; ++a)
      if (types[a] < 0 || types[a] >= ctx->n_types) return fail(TNEP_ERR_INVALID, "type index out of range");
  TNEP_CUDA(cudaSetDevice(ctx->device));
  auto* p = new (std::nothrow) tnep_population();
  if (!p) return fail(TNEP_ERR_OOM, "host allocation failed");
  p->ctx = ctx;
  p->model = model;
  p->n_pop = n_pop;
  p->S = n_structs;
  p->N = N;
  p->C = ctx->models[model].C;
  p->offsets.assign(atom_offsets, atom_offsets + n_structs + 1);
  const tnep_status st = create_pop(p, params, pos, box, types, target);
  if (st != TNEP_OK) {
    destroy_pop(p);
    return st;
  }
  *out = p;
  return TNEP_OK;
}

tnep_status tnep_population_eval(tnep_population* p, const float* params, double* rmse, double* out) {
  if (!p || !params || !rmse) return fail(TNEP_ERR_INVALID, "NULL argument");
  TNEP_CUDA(cudaSetDevice(p->ctx->device));
  TNEP_TRY(pack_all(p, params));
  TNEP_CUDA(cudaEventRecord(p->ev0, p->stream));
  TNEP_CUDA(cudaGraphLaunch(p->exec, p->stream));
  TNEP_CUDA(cudaEventRecord(p->ev1, p->stream));
  TNEP_CUDA(cudaStreamSynchronize(p->stream));
  count_launches(4);  // fused, two reduction stages, RMSE
  float ms = 0.f;
  TNEP_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
  p->last_ms = ms;
  std::memcpy(rmse, p->h_rmse.p, sizeof(double) * p->n_pop);
  if (out) std::memcpy(out, p->h_pred.p, sizeof(double) * (size_t)p->n_pop * p->S * p->C);
  return TNEP_OK;
}

tnep_status tnep_population_info(const tnep_population* p, double info[8]) {
  if (!p || !info) return fail(TNEP_ERR_INVALID, "NULL argument");
  info[0] = p->block;
  info[1] = p->pop_major;
  for (int k = 0; k < 4; ++k) info[2 + k] = p->tune_ms[k];
  info[6] = p->last_ms;
  info[7] = p->N;
  return TNEP_OK;
}

void tnep_population_destroy(tnep_population* p) { destroy_pop(p); }

}  // extern "C"
