// Host-side engine of libtnep: device workspaces, the batch pipeline and
// error reporting.  Shared by the C entry points (api.cu) and the serving
// loop (serve.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "tnep_internal.cuh"

namespace tnep {

tnep_status fail(tnep_status s, const std::string& msg);
const char* last_error_cstr();
tnep_status cuda_fail(cudaError_t e, const char* what);

#define TNEP_CUDA(expr)                                     \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return ::tnep::cuda_fail(_e, #expr); \
  } while (0)

#define TNEP_TRY(expr)                    \
  do {                                    \
    tnep_status _s = (expr);              \
    if (_s != TNEP_OK) return _s;         \
  } while (0)

// Every allocation of the library goes through these three calls.  They
// count allocations (process-wide) and implement host-side fault injection:
// with the environment variable TNEP_FAULT=oom@N set when the library loads,
// the N-th allocation fails once with cudaErrorMemoryAllocation (nothing is
// allocated and the device is not touched), so callers can check that every
// entry point returns TNEP_ERR_OOM and that the context stays usable.
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st);
cudaError_t host_alloc(void** p, size_t bytes);
long long alloc_count();

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t m) {
    if (m <= n && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    const size_t want = std::max<size_t>(std::max<size_t>(m, 1), m + m / 4);
    cudaError_t e = dev_malloc(reinterpret_cast<void**>(&p), want * sizeof(T));
    if (e != cudaSuccess) { p = nullptr; return e; }
    n = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

template <class T>
struct PinBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t m) {
    if (m <= n && p) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
    const size_t want = std::max<size_t>(m, 1);
    cudaError_t e = host_alloc(reinterpret_cast<void**>(&p), want * sizeof(T));
    if (e != cudaSuccess) { p = nullptr; return e; }
    n = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
  }
};

struct Model {
  tnep_model_desc d{};
  int nR = 0, nA = 0, bR = 0, bA = 0, D = 0, nets = 0, variant = -1, C = 0;
  ModelLayout lay{};
  std::vector<float> params;
  std::vector<float> scaler;
  float* d_packed = nullptr;
};

// Device workspace of one in-flight batch.
struct Workspace {
  DevBuf<int> offsets, atom_struct, atom_cell, atom_slot, cell_count, cell_start, cell_atoms;
  DevBuf<int> sorted_orig, orig_sorted, sorted_struct, struct_cells, cnt_R, cnt_A, nbr_R, nbr_A;
  DevBuf<int> nbr_tmp, seg_R, struct_flags;
  DevBuf<float> mom;        // radial moments [slots][atom_stride]
  DevBuf<float4> pcache;    // per-pair cache of the angular walk (see FusedArgs)
  DevBuf<int> red_offsets;  // structure offsets of the pass whose sums run on the side stream
  int mom_v0 = -1, mom_w0 = -1;
  DevBuf<float4> pos4;
  DevBuf<StructGrid> grids;
  DevBuf<StructBox> boxes;
  DevBuf<float> per_atom;   // [model][pop][C][atom_stride]
  DevBuf<double> out;       // [model][S][C]
  DevBuf<double> partial;   // reduction partials
  int max_atoms = 0;        // largest structure of the batch
  DevBuf<float> pos_stage[2], box_stage;
  DevBuf<int> types_stage;
  DevStatus* d_status = nullptr;  // device status word of this workspace
  PinBuf<DevStatus> h_status;     // pinned host copy
  int atom_stride = 0;
  int cells_cap = 0;
  int cap_R = 0, cap_A = 0;  // caps the lists were built with
  int two_ended = 0;         // radial list layout of the last build (see NbrArgs)
  void release() {
    for (auto* b : {&offsets, &atom_struct, &atom_cell, &atom_slot, &cell_count, &cell_start, &cell_atoms,
                    &sorted_orig, &orig_sorted, &sorted_struct, &struct_cells, &cnt_R, &cnt_A, &nbr_R, &nbr_A,
                    &types_stage, &nbr_tmp, &seg_R, &struct_flags})
      b->release();
    pos4.release(); grids.release(); boxes.release(); per_atom.release(); out.release(); partial.release();
    mom.release(); pcache.release(); red_offsets.release();
    pos_stage[0].release(); pos_stage[1].release(); box_stage.release();
    if (d_status) cudaFree(d_status);
    d_status = nullptr;
    h_status.release();
  }
};

bool is_device_ptr(const void* p);
int round_up(int x, int m);

}  // namespace tnep

struct tnep_ctx {
  using Workspace = tnep::Workspace;
  using Model = tnep::Model;
  template <class T> using PinBuf = tnep::PinBuf<T>;
  template <class T> using DevBuf = tnep::DevBuf<T>;
  int device = 0;
  cudaStream_t stream = nullptr, copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_consumed[2] = {nullptr, nullptr};
  // trajectories: the per-frame sums of a pass run on red_stream while the
  // next pass's lists are built (ev_fused: the pass's fused kernels are done;
  // ev_reduced: its sums and output copy are done)
  cudaStream_t red_stream = nullptr;
  cudaEvent_t ev_fused = nullptr, ev_reduced = nullptr;
  cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;
  std::vector<cudaEvent_t> ev_pass;  // 3 timing events per pass, created on demand
  int n_types = 0;
  float rc_R = 0.f, rc_A = 0.f;
  std::vector<Model> models;
  std::vector<std::string> type_names;
  std::vector<double> masses;  // per type (amu), for the centre-of-mass dipole
  Workspace ws;
  PinBuf<double> h_out;
  PinBuf<float> h_stage_f;
  PinBuf<int> h_stage_i;
  DevBuf<float> pop_params;
  DevBuf<double> pop_target, pop_rmse;
  int cap_R = 128, cap_A = 64;
  int max_neighbors = 1024;
  int frames_per_batch = 0;
  int cell_div = 1;
  int x_div = 2;
  float skin = 0.f;        // Verlet skin for trajectories (0 = lists rebuilt every frame)
  int skin_cap = 160;      // radial capacity of the skin lists
  Workspace skin_ws;       // skin lists of the current pass's first frame
  int last_skin_used = 0;  // the last tnep_eval reused skin lists in every pass
  int block_atoms = 128;  // atoms per CTA of the fused kernel (64 or 128)
  int population_form = 0;  // 0 = timed choice, 1 = per-pair walk, 2 = factored, 3 = factored on the tensor cores
  long long wait_tries = tnep::kDefaultWaitTries;  // bounded-wait limit of the tensor-core network
  int pair_cache = 1;      // the fused kernel caches each angular pair's values between its walks
  double last_kernel_ms = 0.0;
  double last_nbr_ms = 0.0;
  int last_launches = 0;
};


namespace tnep {

tnep_status pack_model(tnep_ctx* c, Model& m);
void pack_params(const Model& m, int T, const float* flat, const float* scaler, float* out);
void pack_index_map(const Model& m, int T, int* dst);
size_t expected_params(const tnep_model_desc& d, int T);
tnep_status validate_model(const tnep_model_desc& d, int T);
// Cutoffs and capacities of one list build (default: the context's).
struct ListSpec {
  float rc_R, rc_A;
  int cap_R, cap_A;
};
tnep_status ensure_batch(tnep_ctx* c, Workspace& w, cudaStream_t st, int S, const int* h_offsets, int cap_R,
                         int cap_A);
tnep_status build_lists(tnep_ctx* c, Workspace& w, cudaStream_t st, int S, const int* h_offsets, const float* d_pos,
                        const float* d_box, const int* d_types, int types_period, const ListSpec* spec = nullptr);
tnep_status skin_lists(tnep_ctx* c, Workspace& w, Workspace& sw, cudaStream_t st, int nf, int N, const float* d_pos,
                       const float* d_box, const int* d_types);
tnep_status compute_moments(tnep_ctx* c, Workspace& w, cudaStream_t st, int N, bool need_v, bool need_w);
bool any_rank(const tnep_ctx* c, int rank);
FusedArgs fused_args(tnep_ctx* c, Workspace& w, const Model& m, int N);
int total_C(const tnep_ctx* c);
tnep_status pass_events(tnep_ctx* c, int b, cudaEvent_t** ev);
tnep_status sum_pass_times(tnep_ctx* c, int n_pass);
// ghost: NULL, or one flag per atom of the batch (input order) marking image
// atoms whose contributions are left out of the per-structure sums.
// red_st: NULL, or a stream for the per-structure sums (the caller records
// c->ev_reduced on it once it has consumed w.out); the fused kernels on st
// first wait for the previous pass's sums (c->ev_reduced) to have read the
// per-atom outputs.
tnep_status run_models(tnep_ctx* c, Workspace& w, cudaStream_t st, int S, int N, cudaEvent_t ev_done,
                       const unsigned char* ghost = nullptr, cudaStream_t red_st = nullptr);
cudaError_t launch_zero_ghosts(int N, const int* sorted_orig, const unsigned char* ghost, float* per_atom,
                               int atom_stride, int C, cudaStream_t st);
tnep_status check_status(tnep_ctx* c, const DevStatus& s, bool* regrow);
tnep_status reset_status(Workspace& w, cudaStream_t st);
tnep_status finish(tnep_ctx* c, Workspace& w, cudaStream_t st, bool* regrow);
tnep_status copy_out_bytes(void* dst, const void* src, size_t bytes, cudaStream_t st);
template <class T>
tnep_status copy_out(T* dst, const T* src, size_t count, cudaStream_t st) {
  return copy_out_bytes(dst, src, sizeof(T) * count, st);
}
template <class T>
tnep_status stage_in(const T* src, size_t n, DevBuf<T>& buf, const T** dev, cudaStream_t st) {
  if (!src || n == 0) { *dev = src; return TNEP_OK; }
  if (is_device_ptr(src)) { *dev = src; return TNEP_OK; }
  TNEP_CUDA(buf.ensure(n));
  TNEP_CUDA(cudaMemcpyAsync(buf.p, src, sizeof(T) * n, cudaMemcpyHostToDevice, st));
  *dev = buf.p;
  return TNEP_OK;
}
cudaStream_t pick_stream(tnep_ctx* c, void* stream);
int default_frames_per_batch(int n_atoms, int n_frames);

}  // namespace tnep
