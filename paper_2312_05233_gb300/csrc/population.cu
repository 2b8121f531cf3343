// Population evaluation for training-style use (Sec. II.D: the separable
// natural evolution strategy evaluates a population of parameter vectors on
// the training structures every generation).
//
// The neighbour lists, the radial moments and the angular moments (g_n is
// linear in the coefficients that differ between individuals; angmom.cu)
// depend only on the structures, so tnep_population_create builds them once.  The per-generation work --
// upload of the packed parameter vectors, one fused-kernel launch over all
// individuals x atoms, the FP64 per-structure reduction, the RMSE per
// individual and the read-back -- is captured once into a CUDA graph and
// replayed by tnep_population_eval.  The launch shape (atoms per CTA, and
// whether consecutive CTAs vary the individual or the atom block) is picked
// by timing the candidates on the actual structures, together with the choice
// between the per-pair angular walk and the factored form through the angular
// moments.

#include <cuda_runtime.h>

#include <cmath>
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
  int block = 128, pop_major = 0, fact = 0;  // fact: 0 walk, 1 factored (CUDA cores), 2 factored (tensor cores)
  bool fact_ok = false;          // angular moments available
  DevBuf<float> amom;            // angular moments (factored form)
  bool tc_ok = false;            // tensor-core form available (pop_tc.cu)
  DevBuf<unsigned char> mom_tc, coef_tc;
  DevBuf<int> tc_tiles;
  int n_tiles = 0, n_mt = 0;
  double tc_ms = -1.0;
  double tune_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
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
  if (p->fact) {
    f.amom = p->amom.p;
    f.amom_slots = (int)angular_moment_slots(p->ctx->models[p->model].variant, p->ctx->models[p->model].d.rank,
                                             p->ctx->n_types);
  }
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
  if (p->fact == 2) {
    TNEP_CUDA(launch_coef_tc(p->n_pop, p->ctx->n_types, p->n_mt, p->d_params.p, m.lay, p->coef_tc.p, st));
    PopTcArgs t{};
    t.n_tiles = p->n_tiles;
    t.n_mt = p->n_mt;
    t.n_pop = p->n_pop;
    t.n_types = p->ctx->n_types;
    t.n_atoms = p->N;
    t.tiles = p->tc_tiles.p;
    t.mom_tc = p->mom_tc.p;
    t.mom_tc_stride = pop_tc_moment_stride(m.d.rank);
    t.coef_tc = p->coef_tc.p;
    t.params = p->d_params.p;
    t.lay = m.lay;
    t.mom = f.mom;
    t.mom_stride = f.mom_stride;
    t.v0 = f.v0;
    t.w0 = f.w0;
    t.per_atom = f.per_atom;
    t.per_atom_stride = f.per_atom_stride;
    t.atom_stride = f.atom_stride;
    t.status = f.status;
    TNEP_CUDA(launch_pop_tc(m.d.rank, t, st));
  } else {
    TNEP_CUDA(launch_fused(m.variant, m.d.rank, f, p->n_pop, p->block, m.d.mlp_precision, st));
  }
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

// Times the fused launch for each candidate shape (and, where the angular
// moments exist, the factored form) and keeps the fastest.
tnep_status autotune(tnep_population* p) {
  const int blocks[2] = {128, 64};
  double best = 1e30;
  int best_b = 128, best_o = 0, best_f = 0, idx = 0;
  TNEP_CUDA(cudaMemcpyAsync(p->d_params.p, p->h_params.p,
                            sizeof(float) * (size_t)p->n_pop * p->ctx->models[p->model].lay.words,
                            cudaMemcpyHostToDevice, p->stream));
  for (int fact = 0; fact < 2; ++fact) {
    for (int b : blocks) {
      for (int order = 0; order < 2; ++order, ++idx) {
        p->block = b;
        p->pop_major = order;
        p->fact = fact;
        const int nblk = (p->N + b - 1) / b;
        const bool tc = p->ctx->models[p->model].d.mlp_precision != 0;
        const int form = p->ctx->population_form;
        if ((order == 1 && nblk > 65535) || (tc && b != 128) || (fact && !p->fact_ok) ||
            (form == 1 && fact) || (form == 2 && p->fact_ok && !fact)) {
          p->tune_ms[idx] = -1;
          continue;
        }
        TNEP_TRY(enqueue_generation(p, false));  // warm-up
        TNEP_CUDA(cudaEventRecord(p->ev0, p->stream));
        for (int r = 0; r < 3; ++r) TNEP_TRY(enqueue_generation(p, false));
        TNEP_CUDA(cudaEventRecord(p->ev1, p->stream));
        TNEP_CUDA(cudaEventSynchronize(p->ev1));
        float ms = 0.f;
        TNEP_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        p->tune_ms[idx] = ms / 3.0;
        if (ms < best) { best = ms; best_b = b; best_o = order; best_f = fact; }
      }
    }
  }
  // the tensor-core form (one launch shape)
  p->tc_ms = -1.0;
  const int form = p->ctx->population_form;
  if (p->tc_ok && (form == 0 || form == 3)) {
    p->fact = 2;
    TNEP_TRY(enqueue_generation(p, false));  // warm-up
    TNEP_CUDA(cudaEventRecord(p->ev0, p->stream));
    for (int r = 0; r < 3; ++r) TNEP_TRY(enqueue_generation(p, false));
    TNEP_CUDA(cudaEventRecord(p->ev1, p->stream));
    TNEP_CUDA(cudaEventSynchronize(p->ev1));
    float ms = 0.f;
    TNEP_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
    p->tc_ms = ms / 3.0;
    if (ms < best || form == 3) { best = ms; best_f = 2; }
  }
  p->block = best_b;
  p->pop_major = best_o;
  p->fact = best_f;
  return TNEP_OK;
}

// Tiles of the tensor-core form: the atoms of each centre type in sorted
// order, kPopTcAtoms per tile (the zero block, index N, fills the last one),
// and the per-atom moment blocks in the layout the products read.
tnep_status setup_tc(tnep_population* p) {
  const Model& m = p->ctx->models[p->model];
  const int N = p->N, T = p->ctx->n_types;
  std::vector<float4> pos4(N);
  TNEP_CUDA(cudaMemcpyAsync(pos4.data(), p->ws.pos4.p, sizeof(float4) * N, cudaMemcpyDeviceToHost, p->stream));
  TNEP_CUDA(cudaStreamSynchronize(p->stream));
  std::vector<int> tiles;
  for (int t = 0; t < T; ++t) {
    std::vector<int> at;
    for (int i = 0; i < N; ++i) {
      int ti;
      std::memcpy(&ti, &pos4[i].w, sizeof(int));
      if (ti == t) at.push_back(i);
    }
    for (size_t k = 0; k < at.size(); k += kPopTcAtoms) {
      int rec[8] = {N, N, N, N, N, t, 0, 0};
      const int cnt = (int)std::min<size_t>(kPopTcAtoms, at.size() - k);
      for (int u = 0; u < cnt; ++u) rec[u] = at[k + u];
      rec[6] = cnt;
      tiles.insert(tiles.end(), rec, rec + 8);
    }
  }
  p->n_tiles = (int)tiles.size() / 8;
  p->n_mt = (p->n_pop + kPopTcIndividuals - 1) / kPopTcIndividuals;
  if ((long long)p->n_tiles * p->n_mt > 0x7fffffffLL) return fail(TNEP_ERR_UNSUPPORTED, "too many tiles");
  TNEP_CUDA(p->tc_tiles.ensure(std::max<size_t>(tiles.size(), 1)));
  TNEP_CUDA(cudaMemcpyAsync(p->tc_tiles.p, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice,
                            p->stream));
  TNEP_CUDA(p->mom_tc.ensure((size_t)(N + 1) * pop_tc_moment_stride(m.d.rank)));
  TNEP_CUDA(p->coef_tc.ensure((size_t)T * p->n_mt * pop_tc_coef_bytes()));
  const int slots = (int)angular_moment_slots(m.variant, m.d.rank, T);
  TNEP_CUDA(launch_moments_tc(N, T, m.d.rank, p->amom.p, slots, p->mom_tc.p, p->stream));
  TNEP_CUDA(cudaStreamSynchronize(p->stream));
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
  p->amom.release();
  p->mom_tc.release(); p->coef_tc.release(); p->tc_tiles.release();
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
  TNEP_CUDA(dev_malloc(reinterpret_cast<void**>(&p->ws.d_status), sizeof(DevStatus)));
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
  // angular moments for the factored form (FP32 network only); without the
  // memory for them the per-pair walk is used
  if (m.d.mlp_precision == 0 && N > 0) {
    const size_t slots = angular_moment_slots(m.variant, m.d.rank, c->n_types);
    if (p->amom.ensure(slots * p->ws.atom_stride) == cudaSuccess) {
      AngMomArgs am{};
      am.n_atoms = N;
      am.n_types = c->n_types;
      am.pos4 = p->ws.pos4.p;
      am.sorted_struct = p->ws.sorted_struct.p;
      am.boxes = p->ws.boxes.p;
      am.nbr_A = p->ws.nbr_A.p;
      am.cnt_A = p->ws.cnt_A.p;
      am.cap_A = p->ws.cap_A;
      am.rc_A = c->rc_A;
      am.amom = p->amom.p;
      am.amom_slots = (int)slots;
      TNEP_CUDA(launch_angular_moments(m.variant, m.d.rank, am, st));
      p->fact_ok = true;
    } else {
      cudaGetLastError();
      p->amom.release();
    }
  }
  // tensor-core form: standard descriptor, <= 3 types, FP32 network; without
  // the memory for its moment blocks the other forms are used
  if (p->fact_ok && m.variant == kVarStd && c->n_types <= 3 && m.d.mlp_precision == 0 &&
      (c->population_form == 0 || c->population_form == 3)) {
    const tnep_status ts = setup_tc(p);
    p->tc_ok = ts == TNEP_OK;
    if (!p->tc_ok) {
      cudaGetLastError();
      p->mom_tc.release(); p->coef_tc.release(); p->tc_tiles.release();
      if (ts != TNEP_ERR_OOM) return ts;
    }
  }
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

tnep_status tnep_population_info(const tnep_population* p, double info[14]) {
  if (!p || !info) return fail(TNEP_ERR_INVALID, "NULL argument");
  info[0] = p->block;
  info[1] = p->pop_major;
  info[2] = p->fact;
  for (int k = 0; k < 8; ++k) info[3 + k] = p->tune_ms[k];
  info[11] = p->last_ms;
  info[12] = p->N;
  info[13] = p->tc_ms;
  return TNEP_OK;
}

void tnep_population_destroy(tnep_population* p) { destroy_pop(p); }

}  // extern "C"

// ---- SNES training loop around the population evaluation (Sec. II.D) ----

struct tnep_snes {
  tnep_population* pop = nullptr;
  int P = 0, d = 0;
  double eta_mu = 1.0, eta_sigma = 0.0, lambda1 = 0.0, lambda2 = 0.0;
  unsigned long long seed = 0;
  DevBuf<double> mu, sigma, s, loss, hist;
  DevBuf<int> dst;
  DevBuf<long long> gen;
  PinBuf<double> h_hist;
  long long generation = 0;
  double last_ms = 0.0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

tnep_status enqueue_snes(tnep_snes* sn) {
  tnep_population* p = sn->pop;
  const Model& m = p->ctx->models[p->model];
  cudaStream_t st = p->stream;
  SnesSampleArgs sa{sn->seed, sn->gen.p, sn->P, sn->d, sn->mu.p, sn->sigma.p, sn->s.p, p->d_params.p,
                    (size_t)m.lay.words, sn->dst.p};
  TNEP_CUDA(launch_snes_sample(sa, st));
  TNEP_TRY(enqueue_generation(p, false));
  SnesFitnessArgs fa{sn->P, sn->d, sn->mu.p, sn->sigma.p, sn->s.p, p->d_rmse.p, sn->lambda1, sn->lambda2,
                     sn->loss.p};
  TNEP_CUDA(launch_snes_fitness(fa, st));
  SnesUpdateArgs ua{sn->P, sn->d, sn->loss.p, sn->s.p, p->d_rmse.p, sn->mu.p, sn->sigma.p, sn->eta_mu,
                    sn->eta_sigma, sn->hist.p, sn->gen.p};
  TNEP_CUDA(launch_snes_update(ua, st));
  return TNEP_OK;
}

void destroy_snes(tnep_snes* sn) {
  if (!sn) return;
  if (sn->pop) {
    cudaSetDevice(sn->pop->ctx->device);
    cudaStreamSynchronize(sn->pop->stream);
  }
  if (sn->exec) cudaGraphExecDestroy(sn->exec);
  if (sn->graph) cudaGraphDestroy(sn->graph);
  sn->mu.release(); sn->sigma.release(); sn->s.release(); sn->loss.release(); sn->hist.release();
  sn->dst.release(); sn->gen.release(); sn->h_hist.release();
  destroy_pop(sn->pop);
  delete sn;
}

tnep_status check_snes_sizes(int n_pop, int dim) {
  if (n_pop < 2 || n_pop > kMaxSnesPop) return fail(TNEP_ERR_INVALID, "SNES needs 2 <= n_pop <= 1024");
  if (dim < 1) return fail(TNEP_ERR_INVALID, "SNES needs dim >= 1");
  return TNEP_OK;
}

double default_eta_sigma(int d) { return (3.0 + std::log((double)d)) / (5.0 * std::sqrt((double)d)); }

}  // namespace

extern "C" {

tnep_status tnep_snes_create(tnep_ctx* ctx, int model, const tnep_snes_config* cfg, const double* mu0,
                             const double* sigma0, int n_structs, const int* atom_offsets, const float* pos,
                             const float* box, const int* types, const double* target, tnep_snes** out) {
  if (!out) return fail(TNEP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!ctx || !cfg || !mu0 || !sigma0) return fail(TNEP_ERR_INVALID, "NULL argument");
  if (model < 0 || model >= (int)ctx->models.size()) return fail(TNEP_ERR_INVALID, "bad model index");
  const int d = (int)ctx->models[model].params.size();
  TNEP_TRY(check_snes_sizes(cfg->n_pop, d));
  if (!(cfg->lambda1 >= 0.0) || !(cfg->lambda2 >= 0.0)) return fail(TNEP_ERR_INVALID, "lambda1, lambda2 must be >= 0");
  if (is_device_ptr(mu0) || is_device_ptr(sigma0)) return fail(TNEP_ERR_INVALID, "mu0 and sigma0 must be host memory");
  for (int i = 0; i < d; ++i) {
    if (!std::isfinite(mu0[i])) return fail(TNEP_ERR_INVALID, "mu0 must be finite");
    if (!(sigma0[i] > 0.0) || !std::isfinite(sigma0[i])) return fail(TNEP_ERR_INVALID, "sigma0 must be > 0 and finite");
  }
  // the population object holds the structures; its parameters start at mu0
  std::vector<float> p0((size_t)cfg->n_pop * d);
  for (int k = 0; k < cfg->n_pop; ++k)
    for (int i = 0; i < d; ++i) p0[(size_t)k * d + i] = (float)mu0[i];
  tnep_population* pop = nullptr;
  TNEP_TRY(tnep_population_create(ctx, model, cfg->n_pop, p0.data(), n_structs, atom_offsets, pos, box, types,
                                  target, &pop));
  auto* sn = new (std::nothrow) tnep_snes();
  if (!sn) {
    destroy_pop(pop);
    return fail(TNEP_ERR_OOM, "host allocation failed");
  }
  sn->pop = pop;
  sn->P = cfg->n_pop;
  sn->d = d;
  sn->eta_mu = cfg->eta_mu > 0.0 ? cfg->eta_mu : 1.0;
  sn->eta_sigma = cfg->eta_sigma > 0.0 ? cfg->eta_sigma : default_eta_sigma(d);
  sn->lambda1 = cfg->lambda1;
  sn->lambda2 = cfg->lambda2;
  sn->seed = cfg->seed;
  auto setup = [&]() -> tnep_status {
    const Model& m = ctx->models[model];
    cudaStream_t st = pop->stream;
    std::vector<int> dst(d);
    pack_index_map(m, ctx->n_types, dst.data());
    TNEP_CUDA(sn->mu.ensure(d));
    TNEP_CUDA(sn->sigma.ensure(d));
    TNEP_CUDA(sn->s.ensure((size_t)sn->P * d));
    TNEP_CUDA(sn->loss.ensure(sn->P));
    TNEP_CUDA(sn->hist.ensure(3));
    TNEP_CUDA(sn->dst.ensure(d));
    TNEP_CUDA(sn->gen.ensure(1));
    TNEP_CUDA(cudaMemcpyAsync(sn->mu.p, mu0, sizeof(double) * d, cudaMemcpyHostToDevice, st));
    TNEP_CUDA(cudaMemcpyAsync(sn->sigma.p, sigma0, sizeof(double) * d, cudaMemcpyHostToDevice, st));
    TNEP_CUDA(cudaMemcpyAsync(sn->dst.p, dst.data(), sizeof(int) * d, cudaMemcpyHostToDevice, st));
    TNEP_CUDA(cudaMemsetAsync(sn->gen.p, 0, sizeof(long long), st));
    // the packed template (scaler, padding) is already on the device: the
    // population upload of p0 wrote it for every individual
    TNEP_CUDA(cudaMemcpyAsync(pop->d_params.p, pop->h_params.p, sizeof(float) * (size_t)sn->P * m.lay.words,
                              cudaMemcpyHostToDevice, st));
    TNEP_CUDA(cudaStreamSynchronize(st));
    TNEP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const tnep_status cap = enqueue_snes(sn);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (cap != TNEP_OK) {
      if (g) cudaGraphDestroy(g);
      return cap;
    }
    TNEP_CUDA(e);
    sn->graph = g;
    TNEP_CUDA(cudaGraphInstantiate(&sn->exec, g, 0));
    return TNEP_OK;
  };
  const tnep_status st = setup();
  if (st != TNEP_OK) {
    destroy_snes(sn);
    return st;
  }
  *out = sn;
  return TNEP_OK;
}

tnep_status tnep_snes_run(tnep_snes* sn, int n_gen, double* history) {
  if (!sn || n_gen < 0) return fail(TNEP_ERR_INVALID, "bad SNES handle or n_gen");
  if (n_gen == 0) return TNEP_OK;
  tnep_population* p = sn->pop;
  TNEP_CUDA(cudaSetDevice(p->ctx->device));
  cudaStream_t st = p->stream;
  if (history) TNEP_CUDA(sn->h_hist.ensure((size_t)3 * n_gen));
  TNEP_CUDA(cudaEventRecord(p->ev0, st));
  for (int g = 0; g < n_gen; ++g) {
    TNEP_CUDA(cudaGraphLaunch(sn->exec, st));
    if (history)
      TNEP_CUDA(cudaMemcpyAsync(sn->h_hist.p + 3 * (size_t)g, sn->hist.p, 3 * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
  }
  TNEP_CUDA(cudaEventRecord(p->ev1, st));
  TNEP_CUDA(cudaStreamSynchronize(st));
  count_launches(7 * n_gen);  // sample, fused, two reduction stages, RMSE, fitness, update
  float ms = 0.f;
  TNEP_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
  sn->last_ms = ms / n_gen;
  sn->generation += n_gen;
  if (history) std::memcpy(history, sn->h_hist.p, sizeof(double) * 3 * (size_t)n_gen);
  return TNEP_OK;
}

tnep_status tnep_snes_state(const tnep_snes* sn, double* mu, double* sigma, long long* generation) {
  if (!sn) return fail(TNEP_ERR_INVALID, "NULL SNES handle");
  if ((mu && is_device_ptr(mu)) || (sigma && is_device_ptr(sigma)))
    return fail(TNEP_ERR_INVALID, "mu and sigma must be host memory");
  TNEP_CUDA(cudaSetDevice(sn->pop->ctx->device));
  TNEP_CUDA(cudaStreamSynchronize(sn->pop->stream));
  if (mu) TNEP_CUDA(cudaMemcpy(mu, sn->mu.p, sizeof(double) * sn->d, cudaMemcpyDeviceToHost));
  if (sigma) TNEP_CUDA(cudaMemcpy(sigma, sn->sigma.p, sizeof(double) * sn->d, cudaMemcpyDeviceToHost));
  if (generation) *generation = sn->generation;
  return TNEP_OK;
}

tnep_status tnep_snes_info(const tnep_snes* sn, double info[4]) {
  if (!sn || !info) return fail(TNEP_ERR_INVALID, "NULL argument");
  info[0] = (double)sn->generation;
  info[1] = sn->d;
  info[2] = sn->P;
  info[3] = sn->last_ms;
  return TNEP_OK;
}

void tnep_snes_destroy(tnep_snes* sn) { destroy_snes(sn); }

tnep_status tnep_snes_normals(unsigned long long seed, long long generation, int n_pop, int dim, double* s,
                              void* stream) {
  TNEP_TRY(check_snes_sizes(n_pop, dim));
  if (generation < 0) return fail(TNEP_ERR_INVALID, "generation must be >= 0");
  if (!s || !is_device_ptr(s)) return fail(TNEP_ERR_INVALID, "s must be device memory");
  TNEP_CUDA(launch_snes_normals(seed, generation, n_pop, dim, s, (cudaStream_t)stream));
  return TNEP_OK;
}

tnep_status tnep_snes_update(int n_pop, int dim, const double* loss, const double* s, double* mu, double* sigma,
                             double eta_mu, double eta_sigma, void* stream) {
  TNEP_TRY(check_snes_sizes(n_pop, dim));
  for (const void* q : {(const void*)loss, (const void*)s, (const void*)mu, (const void*)sigma})
    if (!q || !is_device_ptr(q)) return fail(TNEP_ERR_INVALID, "loss, s, mu and sigma must be device memory");
  if (!(eta_mu > 0.0)) return fail(TNEP_ERR_INVALID, "eta_mu must be > 0");
  SnesUpdateArgs ua{n_pop, dim, loss, s, nullptr, mu, sigma, eta_mu,
                    eta_sigma > 0.0 ? eta_sigma : default_eta_sigma(dim), nullptr, nullptr};
  TNEP_CUDA(launch_snes_update(ua, (cudaStream_t)stream));
  count_launches(1);
  return TNEP_OK;
}

}  // extern "C"
