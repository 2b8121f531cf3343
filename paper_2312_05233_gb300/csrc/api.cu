// C ABI of libtnep: argument validation and the synchronous entry points.
//
// Every entry point validates its arguments, returns a tnep_status and never
// lets an exception cross the ABI.  A context owns one CUDA stream, a copy
// stream, and device buffers that grow on demand and stay resident between
// calls (positions, cell lists, neighbour lists, per-atom partials).

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "engine.h"

using namespace tnep;

extern "C" {

const char* tnep_last_error(void) { return last_error_cstr(); }

tnep_status tnep_create(const tnep_model_desc* models, int n_models, int n_types, const char* const* type_names,
                        const float cutoffs[2], int device, tnep_ctx** out) {
  if (!out) return fail(TNEP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!models || n_models < 1) return fail(TNEP_ERR_INVALID, "need at least one model");
  if (n_types < 1 || n_types > kMaxTypes) return fail(TNEP_ERR_INVALID, "n_types must be in [1, 8]");
  if (!cutoffs || !(cutoffs[0] > 0.f) || !(cutoffs[1] > 0.f) || cutoffs[1] > cutoffs[0] ||
      !std::isfinite(cutoffs[0]))
    return fail(TNEP_ERR_INVALID, "cutoffs must satisfy 0 < rc_A <= rc_R");
  for (int k = 0; k < n_models; ++k) TNEP_TRY(validate_model(models[k], n_types));
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(TNEP_ERR_NO_DEVICE, "no CUDA device");
  }
  if (device < 0 || device >= ndev) return fail(TNEP_ERR_INVALID, "device index out of range");
  cudaDeviceProp prop{};
  TNEP_CUDA(cudaGetDeviceProperties(&prop, device));
  if (prop.major * 10 + prop.minor != 103)
    return fail(TNEP_ERR_NO_DEVICE, std::string("library built for sm_103a, device is ") + prop.name);
  TNEP_CUDA(cudaSetDevice(device));
  tnep_ctx* c = new (std::nothrow) tnep_ctx();
  if (!c) return fail(TNEP_ERR_OOM, "host allocation failed");
  c->device = device;
  c->n_types = n_types;
  c->rc_R = cutoffs[0];
  c->rc_A = cutoffs[1];
  if (type_names)
    for (int t = 0; t < n_types; ++t) c->type_names.emplace_back(type_names[t] ? type_names[t] : "");
  auto bail = [&](tnep_status s) {
    tnep_destroy(c);
    return s;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->red_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fused, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_reduced, cudaEventDisableTiming);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&c->ev_copied[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_consumed[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev_k0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev_k1);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void**>(&c->ws.d_status), sizeof(DevStatus));
  if (e == cudaSuccess) e = c->ws.h_status.ensure(1);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void**>(&c->skin_ws.d_status), sizeof(DevStatus));
  if (e == cudaSuccess) e = c->skin_ws.h_status.ensure(1);
  if (e != cudaSuccess) return bail(cuda_fail(e, "context setup"));
  for (int k = 0; k < n_models; ++k) {
    Model m;
    m.d = models[k];
    m.nR = m.d.n_max_R + 1;
    m.nA = m.d.n_max_A + 1;
    m.bR = m.d.basis_R + 1;
    m.bA = m.d.basis_A + 1;
    m.D = m.nR + m.nA * (m.d.l_max + (m.d.use_4body ? 1 : 0));
    m.nets = m.d.per_type_nn ? n_types : 1;
    m.variant = variant_of(m.nR, m.nA, m.bR, m.bA, m.d.l_max, m.d.use_4body);
    m.C = m.d.rank == 1 ? 3 : 9;
    m.params.assign(m.d.params, m.d.params + m.d.n_params);
    m.scaler.assign(m.D, 1.f);
    if (m.d.q_scaler) m.scaler.assign(m.d.q_scaler, m.d.q_scaler + m.D);
    m.d.params = nullptr;
    m.d.q_scaler = nullptr;
    pack_model(c, m);
    std::vector<float> packed(m.lay.words);
    pack_params(m, n_types, m.params.data(), m.scaler.data(), packed.data());
    e = dev_malloc(reinterpret_cast<void**>(&m.d_packed), sizeof(float) * m.lay.words);
    if (e == cudaSuccess)
      e = cudaMemcpy(m.d_packed, packed.data(), sizeof(float) * m.lay.words, cudaMemcpyHostToDevice);
    c->models.push_back(std::move(m));
    if (e != cudaSuccess) return bail(cuda_fail(e, "model upload"));
    if (fused_smem_bytes(c->models.back().variant, c->models.back().lay, kFusedBlockMax,
                         c->models.back().d.mlp_precision) > 227 * 1024)
      return bail(fail(TNEP_ERR_UNSUPPORTED, "model too large for shared memory"));
  }
  *out = c;
  return TNEP_OK;
}

void tnep_destroy(tnep_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  if (c->red_stream) cudaStreamSynchronize(c->red_stream);
  for (auto& m : c->models)
    if (m.d_packed) cudaFree(m.d_packed);
  c->ws.release();
  c->skin_ws.release();
  c->pop_params.release();
  c->pop_target.release();
  c->pop_rmse.release();
  c->h_out.release();
  c->h_stage_f.release();
  c->h_stage_i.release();
  for (int k = 0; k < 2; ++k) {
    if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
    if (c->ev_consumed[k]) cudaEventDestroy(c->ev_consumed[k]);
  }
  if (c->ev_k0) cudaEventDestroy(c->ev_k0);
  if (c->ev_k1) cudaEventDestroy(c->ev_k1);
  for (auto e : c->ev_pass) cudaEventDestroy(e);
  if (c->stream) cudaStreamDestroy(c->stream);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->red_stream) cudaStreamDestroy(c->red_stream);
  if (c->ev_fused) cudaEventDestroy(c->ev_fused);
  if (c->ev_reduced) cudaEventDestroy(c->ev_reduced);
  delete c;
}

int tnep_output_dim(const tnep_ctx* c, int model) {
  if (!c || model < 0 || model >= (int)c->models.size()) return 0;
  return c->models[model].C;
}

tnep_status tnep_set_option(tnep_ctx* c, int option, double value) {
  if (!c) return fail(TNEP_ERR_INVALID, "ctx is NULL");
  switch (option) {
    case TNEP_OPT_FRAMES_PER_BATCH:
      if (value < 0 || value > (1 << 24)) return fail(TNEP_ERR_INVALID, "frames per batch out of range");
      c->frames_per_batch = (int)value;
      return TNEP_OK;
    case TNEP_OPT_MAX_NEIGHBORS:
      if (value < 32 || value > 16384) return fail(TNEP_ERR_INVALID, "max neighbours must be in [32, 16384]");
      c->max_neighbors = (int)value;
      return TNEP_OK;
    case TNEP_OPT_BLOCK_ATOMS:
      if (value != 64 && value != 128) return fail(TNEP_ERR_INVALID, "atoms per CTA must be 64 or 128");
      c->block_atoms = (int)value;
      return TNEP_OK;
    case TNEP_OPT_CELL_DIV:
      if (value != 1 && value != 2 && value != 3) return fail(TNEP_ERR_INVALID, "cell subdivision must be 1, 2 or 3");
      c->cell_div = (int)value;
      return TNEP_OK;
    case TNEP_OPT_CELL_XDIV:
      if (value != 1 && value != 2 && value != 3 && value != 4)
        return fail(TNEP_ERR_INVALID, "x subdivision must be 1, 2, 3 or 4");
      c->x_div = (int)value;
      return TNEP_OK;
    case TNEP_OPT_SKIN:
      if (!(value >= 0.0) || value > 2.0) return fail(TNEP_ERR_INVALID, "skin must be in [0, 2] Angstrom");
      c->skin = (float)value;
      return TNEP_OK;
    case TNEP_OPT_POPULATION_FORM:
      if (value != 0.0 && value != 1.0 && value != 2.0 && value != 3.0)
        return fail(TNEP_ERR_INVALID, "population form must be 0, 1, 2 or 3");
      c->population_form = (int)value;
      return TNEP_OK;
    case TNEP_OPT_WAIT_TRIES:
      if (!(value >= 0.0) || value > 9.0e15) return fail(TNEP_ERR_INVALID, "wait limit must be in [0, 9e15]");
      c->wait_tries = (long long)value;
      return TNEP_OK;
    case TNEP_OPT_PAIR_CACHE:
      if (value != 0.0 && value != 1.0) return fail(TNEP_ERR_INVALID, "pair cache must be 0 or 1");
      c->pair_cache = (int)value;
      return TNEP_OK;
    default:
      return fail(TNEP_ERR_INVALID, "unknown or read-only option");
  }
}

tnep_status tnep_get_option(const tnep_ctx* c, int option, double* value) {
  if (!c || !value) return fail(TNEP_ERR_INVALID, "NULL argument");
  switch (option) {
    case TNEP_OPT_FRAMES_PER_BATCH: *value = c->frames_per_batch; return TNEP_OK;
    case TNEP_OPT_MAX_NEIGHBORS: *value = c->max_neighbors; return TNEP_OK;
    case TNEP_OPT_BLOCK_ATOMS: *value = c->block_atoms; return TNEP_OK;
    case TNEP_OPT_LAST_KERNEL_MS: *value = c->last_kernel_ms; return TNEP_OK;
    case TNEP_OPT_CELL_DIV: *value = c->cell_div; return TNEP_OK;
    case TNEP_OPT_LAST_KERNEL_LAUNCHES: *value = c->last_launches; return TNEP_OK;
    case TNEP_OPT_LAST_NBR_MS: *value = c->last_nbr_ms; return TNEP_OK;
    case TNEP_OPT_KERNEL_LAUNCHES_TOTAL: *value = (double)launches_total(); return TNEP_OK;
    case TNEP_OPT_SKIN: *value = c->skin; return TNEP_OK;
    case TNEP_OPT_POPULATION_FORM: *value = c->population_form; return TNEP_OK;
    case TNEP_OPT_CELL_XDIV: *value = c->x_div; return TNEP_OK;
    case TNEP_OPT_LAST_SKIN_USED: *value = c->last_skin_used; return TNEP_OK;
    case TNEP_OPT_ALLOC_COUNT: *value = (double)alloc_count(); return TNEP_OK;
    case TNEP_OPT_WAIT_TRIES: *value = (double)c->wait_tries; return TNEP_OK;
    case TNEP_OPT_PAIR_CACHE: *value = c->pair_cache; return TNEP_OK;
    default: return fail(TNEP_ERR_INVALID, "unknown option");
  }
}

tnep_status tnep_eval(tnep_ctx* c, int n_frames, int n_atoms, const float* pos, const float* box,
                      const int* types, double* out, void* stream) {
  if (!c) return fail(TNEP_ERR_INVALID, "ctx is NULL");
  if (n_frames < 0 || n_atoms < 0) return fail(TNEP_ERR_INVALID, "negative size");
  if (n_frames == 0) return TNEP_OK;
  if (!out || (n_atoms > 0 && (!pos || !types))) return fail(TNEP_ERR_INVALID, "NULL buffer");
  if ((long long)n_frames * n_atoms > (1LL << 30)) return fail(TNEP_ERR_INVALID, "too many atoms in one call");
  TNEP_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = pick_stream(c, stream);
  const int Ctot = total_C(c);
  int fb = c->frames_per_batch > 0 ? std::min(c->frames_per_batch, n_frames)
                                   : default_frames_per_batch(n_atoms, n_frames);
  if (n_atoms >= kMaxBatchAtoms) return fail(TNEP_ERR_INVALID, "a frame must hold fewer than 2^29 atoms");
  fb = std::max(1, std::min(fb, (kMaxBatchAtoms - 1) / std::max(n_atoms, 1)));
  const bool pos_dev = is_device_ptr(pos);
  const bool box_dev = box && is_device_ptr(box);
  const bool out_dev = is_device_ptr(out);
  const int* d_types = nullptr;
  TNEP_TRY(stage_in(types, (size_t)n_atoms, c->ws.types_stage, &d_types, st));
  if (n_atoms > 0 && !d_types) return fail(TNEP_ERR_INVALID, "types is NULL");
  // type range check on the host copy when available
  if (!is_device_ptr(types))
    for (int a = 0; a < n_atoms; ++a)
      if (types[a] < 0 || types[a] >= c->n_types) return fail(TNEP_ERR_INVALID, "type index out of range");
  const float* d_box_all = nullptr;
  if (box) TNEP_TRY(stage_in(box, (size_t)3 * n_frames, c->ws.box_stage, &d_box_all, st));
  if (!out_dev) TNEP_CUDA(c->h_out.ensure((size_t)n_frames * Ctot));
  std::vector<int> offs(fb + 1);
  // Verlet-skin reuse needs one box for the whole pass and n_atoms > 0; any
  // violation found on the device (displacement above skin / 2, changed box,
  // box too small for the enlarged cutoff) redoes the call with fresh lists
  // for every frame.
  bool use_skin = c->skin > 0.f && n_atoms > 0;
  for (int attempt = 0; attempt < 6; ++attempt) {
    TNEP_TRY(reset_status(c->ws, st));
    if (use_skin) TNEP_TRY(reset_status(c->skin_ws, st));
    int n_pass = 0;
    for (int f0 = 0, b = 0; f0 < n_frames; f0 += fb, ++b) {
      cudaEvent_t* ev = nullptr;
      TNEP_TRY(pass_events(c, b, &ev));
      n_pass = b + 1;
      const int nf = std::min(fb, n_frames - f0);
      for (int k = 0; k <= nf; ++k) offs[k] = k * n_atoms;
      const float* d_pos = pos + (size_t)f0 * n_atoms * 3;
      if (!pos_dev && n_atoms > 0) {
        const int slot = b & 1;
        const size_t cnt = (size_t)nf * n_atoms * 3;
        TNEP_CUDA(c->ws.pos_stage[slot].ensure((size_t)fb * n_atoms * 3));
        TNEP_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_consumed[slot], 0));
        TNEP_CUDA(cudaMemcpyAsync(c->ws.pos_stage[slot].p, pos + (size_t)f0 * n_atoms * 3, sizeof(float) * cnt,
                                  cudaMemcpyHostToDevice, c->copy_stream));
        TNEP_CUDA(cudaEventRecord(c->ev_copied[slot], c->copy_stream));
        TNEP_CUDA(cudaStreamWaitEvent(st, c->ev_copied[slot], 0));
        d_pos = c->ws.pos_stage[slot].p;
      }
      const float* d_box = d_box_all ? d_box_all + (size_t)3 * f0 : nullptr;
      TNEP_CUDA(cudaEventRecord(ev[0], st));
      if (use_skin)
        TNEP_TRY(skin_lists(c, c->ws, c->skin_ws, st, nf, n_atoms, d_pos, d_box, d_types));
      else
        TNEP_TRY(build_lists(c, c->ws, st, nf, offs.data(), d_pos, d_box, d_types, n_atoms));
      if (!pos_dev && n_atoms > 0) TNEP_CUDA(cudaEventRecord(c->ev_consumed[b & 1], st));
      TNEP_CUDA(cudaEventRecord(ev[1], st));
      // the pass's per-frame sums and their copy-out run on the side stream,
      // overlapping the next pass's cell lists and neighbour build
      TNEP_TRY(run_models(c, c->ws, st, nf, nf * n_atoms, ev[2], nullptr, c->red_stream));
      // scatter results: model m block [n_frames][C_m]
      size_t src_off = 0, dst_base = 0;
      for (const auto& m : c->models) {
        double* dst = out_dev ? out : c->h_out.p;
        TNEP_TRY(copy_out(dst + dst_base + (size_t)f0 * m.C, c->ws.out.p + src_off, (size_t)nf * m.C,
                          c->red_stream));
        src_off += (size_t)nf * m.C;
        dst_base += (size_t)n_frames * m.C;
      }
      TNEP_CUDA(cudaEventRecord(c->ev_reduced, c->red_stream));
    }
    TNEP_CUDA(cudaStreamWaitEvent(st, c->ev_reduced, 0));
    if (use_skin) {
      TNEP_CUDA(cudaMemcpyAsync(c->skin_ws.h_status.p, c->skin_ws.d_status, sizeof(DevStatus),
                                cudaMemcpyDeviceToHost, st));
      TNEP_CUDA(cudaStreamSynchronize(st));
      const DevStatus sk = *c->skin_ws.h_status.p;
      if (sk.error) {  // e.g. a box shorter than 2 (rc + skin): plain lists instead
        use_skin = false;
        continue;
      }
      if (sk.max_cnt_R > c->skin_cap) {
        c->skin_cap = round_up(sk.max_cnt_R + 16, 32);
        if (c->skin_cap > c->max_neighbors) use_skin = false;
        continue;
      }
    }
    bool regrow = false;
    TNEP_TRY(finish(c, c->ws, st, &regrow));
    TNEP_TRY(sum_pass_times(c, n_pass));
    if (use_skin && c->ws.h_status.p->skin_violation) {
      use_skin = false;
      continue;
    }
    if (!regrow) {
      c->last_skin_used = use_skin ? 1 : 0;
      if (!out_dev) std::memcpy(out, c->h_out.p, sizeof(double) * (size_t)n_frames * Ctot);
      return TNEP_OK;
    }
  }
  return fail(TNEP_ERR_NEIGHBOR_OVERFLOW, "neighbour lists kept overflowing");
}

tnep_status tnep_eval_batch(tnep_ctx* c, int n_structs, const int* atom_offsets, const float* pos,
                            const float* box, const int* types, double* out, float* per_atom, void* stream) {
  if (!c) return fail(TNEP_ERR_INVALID, "ctx is NULL");
  if (n_structs < 0) return fail(TNEP_ERR_INVALID, "negative size");
  if (n_structs == 0) return TNEP_OK;
  if (!atom_offsets || !out) return fail(TNEP_ERR_INVALID, "NULL buffer");
  if (is_device_ptr(atom_offsets)) return fail(TNEP_ERR_INVALID, "atom_offsets must be host memory");
  if (atom_offsets[0] != 0) return fail(TNEP_ERR_INVALID, "atom_offsets[0] must be 0");
  for (int s = 0; s < n_structs; ++s)
    if (atom_offsets[s + 1] < atom_offsets[s]) return fail(TNEP_ERR_INVALID, "atom_offsets must not decrease");
  const int N = atom_offsets[n_structs];
  if (N >= kMaxBatchAtoms) return fail(TNEP_ERR_INVALID, "a batch must hold fewer than 2^29 atoms");
  if (N > 0 && (!pos || !types)) return fail(TNEP_ERR_INVALID, "NULL buffer");
  TNEP_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = pick_stream(c, stream);
  if (types && !is_device_ptr(types))
    for (int a = 0; a < N; ++a)
      if (types[a] < 0 || types[a] >= c->n_types) return fail(TNEP_ERR_INVALID, "type index out of range");
  const float* d_pos = nullptr;
  const int* d_types = nullptr;
  const float* d_box = nullptr;
  TNEP_TRY(stage_in(pos, (size_t)N * 3, c->ws.pos_stage[0], &d_pos, st));
  TNEP_TRY(stage_in(types, (size_t)N, c->ws.types_stage, &d_types, st));
  if (box) TNEP_TRY(stage_in(box, (size_t)n_structs * 3, c->ws.box_stage, &d_box, st));
  const int Ctot = total_C(c);
  for (int attempt = 0; attempt < 4; ++attempt) {
    TNEP_TRY(reset_status(c->ws, st));
    cudaEvent_t* ev = nullptr;
    TNEP_TRY(pass_events(c, 0, &ev));
    TNEP_CUDA(cudaEventRecord(ev[0], st));
    TNEP_TRY(build_lists(c, c->ws, st, n_structs, atom_offsets, d_pos, d_box, d_types, std::max(N, 1)));
    TNEP_CUDA(cudaEventRecord(ev[1], st));
    TNEP_TRY(run_models(c, c->ws, st, n_structs, N, ev[2]));
    bool regrow = false;
    TNEP_TRY(finish(c, c->ws, st, &regrow));
    TNEP_TRY(sum_pass_times(c, 1));
    if (regrow) continue;
    TNEP_TRY(copy_out(out, c->ws.out.p, (size_t)n_structs * Ctot, st));
    if (per_atom && N > 0) {
      const size_t per_model = (size_t)9 * c->ws.atom_stride;
      const bool pa_dev = is_device_ptr(per_atom);
      size_t dst_off = 0;
      DevBuf<float> tmp;
      for (size_t k = 0; k < c->models.size(); ++k) {
        const Model& m = c->models[k];
        float* dst = per_atom + dst_off;
        if (!pa_dev) {
          TNEP_CUDA(tmp.ensure((size_t)N * m.C));
          dst = tmp.p;
        }
        TNEP_CUDA(launch_gather_per_atom(N, c->ws.orig_sorted.p, c->ws.per_atom.p + k * per_model,
                                         c->ws.atom_stride, m.C, dst, st));
        if (!pa_dev) {
          TNEP_CUDA(cudaMemcpyAsync(per_atom + dst_off, tmp.p, sizeof(float) * N * m.C, cudaMemcpyDeviceToHost, st));
          TNEP_CUDA(cudaStreamSynchronize(st));
        }
        dst_off += (size_t)N * m.C;
      }
      tmp.release();
    }
    TNEP_CUDA(cudaStreamSynchronize(st));
    return TNEP_OK;
  }
  return fail(TNEP_ERR_NEIGHBOR_OVERFLOW, "neighbour lists kept overflowing");
}

tnep_status tnep_neighbors(tnep_ctx* c, int n_structs, const int* atom_offsets, const float* pos,
                           const float* box, int* counts_R, int* counts_A, int* list_R, int cap_R, int* list_A,
                           int cap_A, void* stream) {
  if (!c) return fail(TNEP_ERR_INVALID, "ctx is NULL");
  if (n_structs <= 0) return n_structs == 0 ? TNEP_OK : fail(TNEP_ERR_INVALID, "negative size");
  if (!atom_offsets || !counts_R || !counts_A || !list_R || !list_A || cap_R < 0 || cap_A < 0)
    return fail(TNEP_ERR_INVALID, "NULL buffer or negative cap");
  if (is_device_ptr(atom_offsets)) return fail(TNEP_ERR_INVALID, "atom_offsets must be host memory");
  if (atom_offsets[0] != 0) return fail(TNEP_ERR_INVALID, "atom_offsets[0] must be 0");
  for (int s = 0; s < n_structs; ++s)
    if (atom_offsets[s + 1] < atom_offsets[s]) return fail(TNEP_ERR_INVALID, "atom_offsets must not decrease");
  const int N = atom_offsets[n_structs];
  if (N == 0) return TNEP_OK;
  if (N >= kMaxBatchAtoms) return fail(TNEP_ERR_INVALID, "a batch must hold fewer than 2^29 atoms");
  if (!pos) return fail(TNEP_ERR_INVALID, "pos is NULL");
  TNEP_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = pick_stream(c, stream);
  const float* d_pos = nullptr;
  const float* d_box = nullptr;
  TNEP_TRY(stage_in(pos, (size_t)N * 3, c->ws.pos_stage[0], &d_pos, st));
  if (box) TNEP_TRY(stage_in(box, (size_t)n_structs * 3, c->ws.box_stage, &d_box, st));
  DevBuf<int> zeros;
  TNEP_CUDA(zeros.ensure(1));
  TNEP_CUDA(cudaMemsetAsync(zeros.p, 0, sizeof(int), st));
  for (int attempt = 0; attempt < 4; ++attempt) {
    TNEP_TRY(reset_status(c->ws, st));
    TNEP_TRY(build_lists(c, c->ws, st, n_structs, atom_offsets, d_pos, d_box, zeros.p, 1));
    bool regrow = false;
    TNEP_TRY(finish(c, c->ws, st, &regrow));
    if (regrow) continue;
    const bool dev = is_device_ptr(list_R);
    DevBuf<int> tR, tA, tcR, tcA;
    int *oR = list_R, *oA = list_A, *ocR = counts_R, *ocA = counts_A;
    if (!dev) {
      TNEP_CUDA(tR.ensure((size_t)N * std::max(cap_R, 1)));
      TNEP_CUDA(tA.ensure((size_t)N * std::max(cap_A, 1)));
      TNEP_CUDA(tcR.ensure(N));
      TNEP_CUDA(tcA.ensure(N));
      oR = tR.p; oA = tA.p; ocR = tcR.p; ocA = tcA.p;
    }
    TNEP_CUDA(launch_export_neighbors(N, c->ws.sorted_orig.p, c->ws.orig_sorted.p, c->ws.nbr_R.p, c->ws.cnt_R.p,
                                      c->ws.cap_R, c->ws.seg_R.p, c->ws.two_ended, c->ws.nbr_A.p, c->ws.cnt_A.p, c->ws.cap_A, ocR, ocA, oR, cap_R,
                                      oA, cap_A, st));
    if (!dev) {
      TNEP_CUDA(cudaMemcpyAsync(list_R, tR.p, sizeof(int) * (size_t)N * cap_R, cudaMemcpyDeviceToHost, st));
      TNEP_CUDA(cudaMemcpyAsync(list_A, tA.p, sizeof(int) * (size_t)N * cap_A, cudaMemcpyDeviceToHost, st));
      TNEP_CUDA(cudaMemcpyAsync(counts_R, tcR.p, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
      TNEP_CUDA(cudaMemcpyAsync(counts_A, tcA.p, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
    }
    TNEP_CUDA(cudaStreamSynchronize(st));
    tR.release(); tA.release(); tcR.release(); tcA.release(); zeros.release();
    return TNEP_OK;
  }
  zeros.release();
  return fail(TNEP_ERR_NEIGHBOR_OVERFLOW, "neighbour lists kept overflowing");
}

tnep_status tnep_eval_population(tnep_ctx* c, int model, int n_pop, const float* params, int n_structs,
                                 const int* atom_offsets, const float* pos, const float* box, const int* types,
                                 const double* target, double* rmse, double* out, void* stream) {
  if (!c) return fail(TNEP_ERR_INVALID, "ctx is NULL");
  if (model < 0 || model >= (int)c->models.size()) return fail(TNEP_ERR_INVALID, "model index out of range");
  if (n_pop < 1 || n_structs < 1) return fail(TNEP_ERR_INVALID, "need n_pop >= 1 and n_structs >= 1");
  if (!params || !atom_offsets || !target || !rmse) return fail(TNEP_ERR_INVALID, "NULL buffer");
  if (is_device_ptr(atom_offsets) || is_device_ptr(params))
    return fail(TNEP_ERR_INVALID, "atom_offsets and params must be host memory");
  if (atom_offsets[0] != 0) return fail(TNEP_ERR_INVALID, "atom_offsets[0] must be 0");
  for (int s = 0; s < n_structs; ++s)
    if (atom_offsets[s + 1] < atom_offsets[s]) return fail(TNEP_ERR_INVALID, "atom_offsets must not decrease");
  const int N = atom_offsets[n_structs];
  if (N >= kMaxBatchAtoms) return fail(TNEP_ERR_INVALID, "a batch must hold fewer than 2^29 atoms");
  if (N > 0 && (!pos || !types)) return fail(TNEP_ERR_INVALID, "NULL buffer");
  TNEP_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = pick_stream(c, stream);
  if (types && !is_device_ptr(types))
    for (int a = 0; a < N; ++a)
      if (types[a] < 0 || types[a] >= c->n_types) return fail(TNEP_ERR_INVALID, "type index out of range");
  Model& m = c->models[model];
  const size_t np = m.params.size();
  std::vector<float> packed((size_t)n_pop * m.lay.words);
  for (int p = 0; p < n_pop; ++p)
    pack_params(m, c->n_types, params + (size_t)p * np, m.scaler.data(), packed.data() + (size_t)p * m.lay.words);
  TNEP_CUDA(c->pop_params.ensure(packed.size()));
  TNEP_CUDA(cudaMemcpyAsync(c->pop_params.p, packed.data(), sizeof(float) * packed.size(), cudaMemcpyHostToDevice,
                            st));
  const float* d_pos = nullptr;
  const int* d_types = nullptr;
  const float* d_box = nullptr;
  const double* d_target = nullptr;
  TNEP_TRY(stage_in(pos, (size_t)N * 3, c->ws.pos_stage[0], &d_pos, st));
  TNEP_TRY(stage_in(types, (size_t)N, c->ws.types_stage, &d_types, st));
  if (box) TNEP_TRY(stage_in(box, (size_t)n_structs * 3, c->ws.box_stage, &d_box, st));
  TNEP_TRY(stage_in(target, (size_t)n_structs * m.C, c->pop_target, &d_target, st));
  for (int attempt = 0; attempt < 4; ++attempt) {
    TNEP_TRY(reset_status(c->ws, st));
    TNEP_TRY(build_lists(c, c->ws, st, n_structs, atom_offsets, d_pos, d_box, d_types, std::max(N, 1)));
    Workspace& w = c->ws;
    const size_t pa_pop = (size_t)m.C * w.atom_stride;
    TNEP_CUDA(w.per_atom.ensure(pa_pop * n_pop));
    TNEP_CUDA(w.out.ensure((size_t)n_pop * n_structs * m.C));
    TNEP_CUDA(c->pop_rmse.ensure(n_pop));
    cudaEvent_t* ev0 = nullptr;
    TNEP_TRY(pass_events(c, 0, &ev0));
    TNEP_CUDA(cudaEventRecord(ev0[1], st));
    TNEP_TRY(compute_moments(c, c->ws, st, N, m.d.rank == 1, m.d.rank == 2));
    FusedArgs f = fused_args(c, c->ws, m, N);
    f.model = c->pop_params.p;
    f.model_stride = m.lay.words;
    f.per_atom = w.per_atom.p;
    f.per_atom_stride = pa_pop;
    cudaEvent_t* ev = nullptr;
    TNEP_TRY(pass_events(c, 0, &ev));
    TNEP_CUDA(launch_fused(m.variant, m.d.rank, f, n_pop, c->block_atoms, m.d.mlp_precision, st));
    TNEP_CUDA(cudaEventRecord(ev[2], st));
    TNEP_CUDA(w.partial.ensure((size_t)n_pop * n_structs * reduce_chunks(w.max_atoms) * m.C));
    TNEP_CUDA(launch_reduce(n_structs, n_pop, w.offsets.p, w.max_atoms, w.per_atom.p, pa_pop, w.atom_stride, m.C,
                            w.partial.p, w.out.p, (size_t)n_structs * m.C, st));
    TNEP_CUDA(launch_rmse(n_pop, n_structs, m.C, w.out.p, d_target, c->pop_rmse.p, st));
    bool regrow = false;
    TNEP_TRY(finish(c, c->ws, st, &regrow));
    if (regrow) continue;
    float ms = 0.f;
    TNEP_CUDA(cudaEventElapsedTime(&ms, ev[1], ev[2]));
    c->last_kernel_ms = ms;
    c->last_launches = 1;
    TNEP_TRY(copy_out(rmse, c->pop_rmse.p, (size_t)n_pop, st));
    if (out) TNEP_TRY(copy_out(out, w.out.p, (size_t)n_pop * n_structs * m.C, st));
    TNEP_CUDA(cudaStreamSynchronize(st));
    return TNEP_OK;
  }
  return fail(TNEP_ERR_NEIGHBOR_OVERFLOW, "neighbour lists kept overflowing");
}

tnep_status tnep_spectrum(const double* series, int T, int C, double dt_fs, int kind, int max_lag,
                          int subtract_mean, double* freq_cm1, double* spec, double* acf_out, void* stream) {
  if (!series || !freq_cm1 || !spec) return fail(TNEP_ERR_INVALID, "NULL buffer");
  if (T < 2) return fail(TNEP_ERR_INVALID, "need at least two samples");
  if (!(dt_fs > 0.0)) return fail(TNEP_ERR_INVALID, "dt must be positive");
  if (kind == TNEP_SPECTRUM_IR) {
    if (C != 3) return fail(TNEP_ERR_INVALID, "IR needs C = 3");
  } else if (kind == TNEP_SPECTRUM_RAMAN_ISO || kind == TNEP_SPECTRUM_RAMAN_ANISO) {
    if (C != 9) return fail(TNEP_ERR_INVALID, "Raman needs C = 9");
  } else {
    return fail(TNEP_ERR_INVALID, "unknown spectrum kind");
  }
  const int M = max_lag <= 0 ? T / 2 : max_lag;
  if (M < 1 || M >= T) return fail(TNEP_ERR_INVALID, "max_lag must be in [1, T)");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(TNEP_ERR_NO_DEVICE, "no CUDA device");
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t n_series = (size_t)T * C;
  const size_t n_work = (size_t)T * 9 + 3 * (size_t)(M + 1) + 2 * (size_t)M + 8;
  // the direct time-origin sums while cheap, the Fourier route for long series
  const bool use_fft = (double)spectrum_channels(kind) * (double)T * (double)(M + 1) > 1.0e9;
  int N = 2;
  while (N < T + M) N <<= 1;
  const size_t n_z = use_fft ? (size_t)18 * N + (size_t)N / 2 : 0;  // double2
  double* d = nullptr;
  const size_t total = 2 * n_z + n_series + n_work + 2 * (size_t)(M + 1) + (M + 1);
  TNEP_CUDA(dev_malloc_async((void**)&d, sizeof(double) * total, st));
  double2* d_z = reinterpret_cast<double2*>(d);  // first: the allocation's alignment holds
  double* d_series = d + 2 * n_z;
  double* d_work = d_series + n_series;
  double* d_freq = d_work + n_work;
  double* d_spec = d_freq + (M + 1);
  double* d_acf = d_spec + (M + 1);
  tnep_status rc = TNEP_OK;
  cudaError_t e = cudaMemcpyAsync(d_series, series, sizeof(double) * n_series, cudaMemcpyDefault, st);
  if (e == cudaSuccess)
    e = use_fft ? launch_spectrum_fft(d_series, T, C, dt_fs, kind, M, subtract_mean, d_work, d_z, N, d_freq, d_spec,
                                      d_acf, st)
                : launch_spectrum(d_series, T, C, dt_fs, kind, M, subtract_mean, d_work, d_freq, d_spec, d_acf, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(freq_cm1, d_freq, sizeof(double) * (M + 1), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(spec, d_spec, sizeof(double) * (M + 1), cudaMemcpyDefault, st);
  if (e == cudaSuccess && acf_out)
    e = cudaMemcpyAsync(acf_out, d_acf, sizeof(double) * (M + 1), cudaMemcpyDefault, st);
  if (e != cudaSuccess) rc = cuda_fail(e, "spectrum");
  cudaFreeAsync(d, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess && rc == TNEP_OK) rc = cuda_fail(e, "spectrum sync");
  return rc;
}

}  // extern "C"
