// C ABI of libtnep: contexts, resident device workspaces and the batch engine.
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

#include "tnep_internal.cuh"

using namespace tnep;

namespace {

thread_local std::string g_last_error;

tnep_status fail(tnep_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

tnep_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free error
  return fail(e == cudaErrorMemoryAllocation ? TNEP_ERR_OOM : TNEP_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define TNEP_CUDA(expr)                                     \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return cuda_fail(_e, #expr);     \
  } while (0)

#define TNEP_TRY(expr)                    \
  do {                                    \
    tnep_status _s = (expr);              \
    if (_s != TNEP_OK) return _s;         \
  } while (0)

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
    cudaError_t e = cudaMalloc(&p, want * sizeof(T));
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
    cudaError_t e = cudaHostAlloc((void**)&p, want * sizeof(T), cudaHostAllocDefault);
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
  int atom_stride = 0;
  int cells_cap = 0;
  int cap_R = 0, cap_A = 0;  // caps the lists were built with
  void release() {
    for (auto* b : {&offsets, &atom_struct, &atom_cell, &atom_slot, &cell_count, &cell_start, &cell_atoms,
                    &sorted_orig, &orig_sorted, &sorted_struct, &struct_cells, &cnt_R, &cnt_A, &nbr_R, &nbr_A,
                    &types_stage, &nbr_tmp, &seg_R, &struct_flags})
      b->release();
    pos4.release(); grids.release(); boxes.release(); per_atom.release(); out.release(); partial.release();
    mom.release();
    pos_stage[0].release(); pos_stage[1].release(); box_stage.release();
  }
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) { cudaGetLastError(); return false; }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

int coeff_stride(int words) {
  int s = round_up(words, 4);
  if (s % 32 == 0 || s % 32 == 16) s += 4;  // spread (ti, tj) blocks over banks
  return s;
}

}  // namespace

void tnep::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

struct tnep_ctx {
  int device = 0;
  cudaStream_t stream = nullptr, copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_consumed[2] = {nullptr, nullptr};
  cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;
  std::vector<cudaEvent_t> ev_pass;  // 3 timing events per pass, created on demand
  int n_types = 0;
  float rc_R = 0.f, rc_A = 0.f;
  std::vector<Model> models;
  std::vector<std::string> type_names;
  Workspace ws;
  DevStatus* d_status = nullptr;
  PinBuf<DevStatus> h_status;
  PinBuf<double> h_out;
  PinBuf<float> h_stage_f;
  PinBuf<int> h_stage_i;
  DevBuf<float> pop_params;
  DevBuf<double> pop_target, pop_rmse;
  int cap_R = 128, cap_A = 64;
  int max_neighbors = 1024;
  int frames_per_batch = 0;
  int cell_div = 1;
  double last_kernel_ms = 0.0;
  double last_nbr_ms = 0.0;
  int last_launches = 0;
};

namespace {

tnep_status pack_model(tnep_ctx* c, Model& m) {
  const int T = c->n_types;
  ModelLayout& L = m.lay;
  L.n_types = T;
  L.nets = m.nets;
  L.H = m.d.n_hidden;
  L.D = m.D;
  L.Dp = round_up(m.D, 4);
  L.stride_cR = coeff_stride(m.nR * m.bR);
  L.stride_cA = coeff_stride(m.nA * m.bA);
  L.off_cR = 0;
  L.off_cA = L.off_cR + T * T * L.stride_cR;
  L.off_W0 = L.off_cA + T * T * L.stride_cA;
  L.off_b0 = L.off_W0 + m.nets * L.H * L.Dp;
  L.off_w1 = L.off_b0 + m.nets * L.H;
  L.off_b1 = L.off_w1 + m.nets * L.H;
  L.off_scaler = round_up(L.off_b1 + m.nets, 4);
  L.words = round_up(L.off_scaler + L.Dp, 4);
  return TNEP_OK;
}

// Flat parameters -> device layout (one individual).
void pack_params(const Model& m, int T, const float* flat, const float* scaler, float* out) {
  const ModelLayout& L = m.lay;
  std::fill(out, out + L.words, 0.f);
  size_t o = 0;
  for (int net = 0; net < m.nets; ++net) {
    for (int h = 0; h < L.H; ++h)
      for (int d = 0; d < m.D; ++d) out[L.off_W0 + (net * L.H + h) * L.Dp + d] = flat[o++];
    for (int h = 0; h < L.H; ++h) out[L.off_b0 + net * L.H + h] = flat[o++];
    for (int h = 0; h < L.H; ++h) out[L.off_w1 + net * L.H + h] = flat[o++];
    out[L.off_b1 + net] = flat[o++];
  }
  for (int p = 0; p < T * T; ++p)
    for (int k = 0; k < m.nR * m.bR; ++k) out[L.off_cR + p * L.stride_cR + k] = flat[o++];
  for (int p = 0; p < T * T; ++p)
    for (int k = 0; k < m.nA * m.bA; ++k) out[L.off_cA + p * L.stride_cA + k] = flat[o++];
  for (int d = 0; d < m.D; ++d) out[L.off_scaler + d] = scaler[d];
}

size_t expected_params(const tnep_model_desc& d, int T) {
  const int D = (d.n_max_R + 1) + (d.n_max_A + 1) * (d.l_max + (d.use_4body ? 1 : 0));
  const int nets = d.per_type_nn ? T : 1;
  return (size_t)nets * (d.n_hidden * D + 2 * d.n_hidden + 1) +
         (size_t)T * T * ((d.n_max_R + 1) * (d.basis_R + 1) + (d.n_max_A + 1) * (d.basis_A + 1));
}

tnep_status validate_model(const tnep_model_desc& d, int T) {
  if (d.rank != 1 && d.rank != 2) return fail(TNEP_ERR_INVALID, "model rank must be 1 or 2");
  if (d.n_hidden < 1 || d.n_hidden > 64) return fail(TNEP_ERR_INVALID, "n_hidden must be in [1, 64]");
  if (!d.params) return fail(TNEP_ERR_INVALID, "model params is NULL");
  if (d.n_max_R < 0 || d.n_max_A < 0 || d.basis_R < 0 || d.basis_A < 0 || d.l_max < 1)
    return fail(TNEP_ERR_INVALID, "negative descriptor size");
  if (variant_of(d.n_max_R + 1, d.n_max_A + 1, d.basis_R + 1, d.basis_A + 1, d.l_max, d.use_4body) < 0)
    return fail(TNEP_ERR_UNSUPPORTED, "no compiled kernel for these descriptor sizes");
  if (d.mlp_precision != 0 && d.mlp_precision != 1) return fail(TNEP_ERR_INVALID, "mlp_precision must be 0 or 1");
  if (d.mlp_precision == 1) return fail(TNEP_ERR_UNSUPPORTED, "BF16 tensor-core MLP not built in this library");
  const size_t want = expected_params(d, T);
  if (d.n_params != want)
    return fail(TNEP_ERR_INVALID, "n_params " + std::to_string(d.n_params) + " != layout " + std::to_string(want));
  return TNEP_OK;
}

// Builds cell and neighbour lists for a batch whose inputs are on the device.
tnep_status build_lists(tnep_ctx* c, cudaStream_t st, int S, const int* h_offsets, const float* d_pos,
                        const float* d_box, const int* d_types, int types_period) {
  Workspace& w = c->ws;
  const int N = h_offsets[S];
  const int stride = round_up(std::max(N, 1), 32);
  int mx = 0;
  for (int s = 0; s < S; ++s) mx = std::max(mx, h_offsets[s + 1] - h_offsets[s]);
  w.max_atoms = mx;
  w.atom_stride = stride;
  w.cells_cap = 2 * N + 8 * S;
  w.cap_R = c->cap_R;
  w.cap_A = c->cap_A;
  TNEP_CUDA(w.offsets.ensure(S + 1));
  TNEP_CUDA(w.struct_cells.ensure(S + 1));
  TNEP_CUDA(w.struct_flags.ensure(S));
  TNEP_CUDA(w.grids.ensure(S));
  TNEP_CUDA(w.boxes.ensure(S));
  TNEP_CUDA(w.atom_struct.ensure(stride));
  TNEP_CUDA(w.atom_cell.ensure(stride));
  TNEP_CUDA(w.atom_slot.ensure(stride));
  TNEP_CUDA(w.cell_atoms.ensure(stride));
  TNEP_CUDA(w.sorted_orig.ensure(stride));
  TNEP_CUDA(w.orig_sorted.ensure(stride));
  TNEP_CUDA(w.sorted_struct.ensure(stride));
  TNEP_CUDA(w.pos4.ensure(stride));
  TNEP_CUDA(w.cnt_R.ensure(stride));
  TNEP_CUDA(w.cnt_A.ensure(stride));
  TNEP_CUDA(w.cell_count.ensure(w.cells_cap + 1));
  TNEP_CUDA(w.cell_start.ensure(w.cells_cap + 1));
  TNEP_CUDA(w.nbr_R.ensure((size_t)stride * w.cap_R));
  TNEP_CUDA(w.nbr_tmp.ensure((size_t)stride * w.cap_R));
  TNEP_CUDA(w.nbr_A.ensure((size_t)stride * w.cap_A));
  TNEP_CUDA(w.seg_R.ensure((size_t)stride * c->n_types));
  TNEP_CUDA(cudaMemcpyAsync(w.offsets.p, h_offsets, sizeof(int) * (S + 1), cudaMemcpyHostToDevice, st));
  TNEP_CUDA(cudaMemsetAsync(w.cell_count.p, 0, sizeof(int) * (w.cells_cap + 1), st));
  TNEP_CUDA(cudaMemsetAsync(w.struct_flags.p, 0, sizeof(int) * S, st));
  NbrArgs a{};
  a.n_structs = S;
  a.n_atoms = N;
  a.offsets = w.offsets.p;
  a.pos = d_pos;
  a.box = d_box;
  a.types = d_types;
  a.types_period = std::max(types_period, 1);
  a.n_types = c->n_types;
  a.rc_R = c->rc_R;
  a.rc_A = c->rc_A;
  a.cell_div = c->cell_div;
  a.grids = w.grids.p;
  a.boxes = w.boxes.p;
  a.struct_cells = w.struct_cells.p;
  a.struct_flags = w.struct_flags.p;
  a.atom_struct = w.atom_struct.p;
  a.atom_cell = w.atom_cell.p;
  a.atom_slot = w.atom_slot.p;
  a.cell_count = w.cell_count.p;
  a.cell_start = w.cell_start.p;
  a.cell_atoms = w.cell_atoms.p;
  a.sorted_orig = w.sorted_orig.p;
  a.orig_sorted = w.orig_sorted.p;
  a.sorted_struct = w.sorted_struct.p;
  a.pos4 = w.pos4.p;
  a.nbr_R = w.nbr_R.p;
  a.nbr_A = w.nbr_A.p;
  a.nbr_tmp = w.nbr_tmp.p;
  a.seg_R = w.seg_R.p;
  a.seg_stride = stride;
  a.cnt_R = w.cnt_R.p;
  a.cnt_A = w.cnt_A.p;
  a.cap_R = w.cap_R;
  a.cap_A = w.cap_A;
  a.cells_cap = w.cells_cap;
  a.status = c->d_status;
  TNEP_CUDA(launch_neighbor_pipeline(a, st));
  return TNEP_OK;
}

// Radial moments of the lists in the workspace (F always; V for rank-1 and W
// for rank-2 models).
tnep_status compute_moments(tnep_ctx* c, cudaStream_t st, int N, bool need_v, bool need_w) {
  Workspace& w = c->ws;
  const int T = c->n_types;
  const int per = T * kMomBasis;
  w.mom_v0 = need_v ? per : -1;
  w.mom_w0 = need_w ? per * (need_v ? 4 : 1) : -1;
  const int slots = per * (1 + (need_v ? 3 : 0) + (need_w ? 6 : 0));
  TNEP_CUDA(w.mom.ensure((size_t)slots * w.atom_stride));
  RadialArgs r{};
  r.n_atoms = N;
  r.n_types = T;
  r.pos4 = w.pos4.p;
  r.sorted_struct = w.sorted_struct.p;
  r.boxes = w.boxes.p;
  r.nbr_R = w.nbr_R.p;
  r.cap_R = w.cap_R;
  r.seg_R = w.seg_R.p;
  r.seg_stride = w.atom_stride;
  r.rc_R = c->rc_R;
  r.mom = w.mom.p;
  r.mom_stride = w.atom_stride;
  r.v0 = w.mom_v0;
  r.w0 = w.mom_w0;
  TNEP_CUDA(launch_radial_moments(r, st));
  return TNEP_OK;
}

bool any_rank(const tnep_ctx* c, int rank) {
  for (const auto& m : c->models)
    if (m.d.rank == rank) return true;
  return false;
}

FusedArgs fused_args(tnep_ctx* c, const Model& m, int N) {
  Workspace& w = c->ws;
  FusedArgs f{};
  f.n_atoms = N;
  f.pos4 = w.pos4.p;
  f.sorted_struct = w.sorted_struct.p;
  f.boxes = w.boxes.p;
  f.mom = w.mom.p;
  f.mom_stride = w.atom_stride;
  f.v0 = w.mom_v0;
  f.w0 = w.mom_w0;
  f.nbr_A = w.nbr_A.p;
  f.cnt_A = w.cnt_A.p;
  f.cap_A = w.cap_A;
  f.model = m.d_packed;
  f.model_stride = 0;
  f.lay = m.lay;
  f.rc_R = c->rc_R;
  f.rc_A = c->rc_A;
  f.atom_stride = w.atom_stride;
  return f;
}

int total_C(const tnep_ctx* c) {
  int t = 0;
  for (const auto& m : c->models) t += m.C;
  return t;
}

// Runs every model on the lists in the workspace; out_dev [model][S][C].
// Timing events of pass `b` (0: before the neighbour pipeline, 1: before the
// fused kernels, 2: after them).
tnep_status pass_events(tnep_ctx* c, int b, cudaEvent_t** ev) {
  while ((int)c->ev_pass.size() < 3 * (b + 1)) {
    cudaEvent_t e;
    TNEP_CUDA(cudaEventCreate(&e));
    c->ev_pass.push_back(e);
  }
  *ev = &c->ev_pass[3 * b];
  return TNEP_OK;
}

tnep_status sum_pass_times(tnep_ctx* c, int n_pass) {
  double nbr = 0.0, fused = 0.0;
  for (int b = 0; b < n_pass; ++b) {
    float m1 = 0.f, m2 = 0.f;
    TNEP_CUDA(cudaEventElapsedTime(&m1, c->ev_pass[3 * b], c->ev_pass[3 * b + 1]));
    TNEP_CUDA(cudaEventElapsedTime(&m2, c->ev_pass[3 * b + 1], c->ev_pass[3 * b + 2]));
    nbr += m1;
    fused += m2;
  }
  c->last_nbr_ms = nbr;
  c->last_kernel_ms = fused;
  c->last_launches = n_pass * (int)c->models.size();
  return TNEP_OK;
}

tnep_status run_models(tnep_ctx* c, cudaStream_t st, int S, int N, cudaEvent_t ev_done) {
  Workspace& w = c->ws;
  const size_t per_model = (size_t)9 * w.atom_stride;
  TNEP_CUDA(w.per_atom.ensure(per_model * c->models.size()));
  TNEP_CUDA(w.out.ensure((size_t)std::max(S, 1) * total_C(c)));
  TNEP_TRY(compute_moments(c, st, N, any_rank(c, 1), any_rank(c, 2)));
  for (size_t k = 0; k < c->models.size(); ++k) {
    const Model& m = c->models[k];
    FusedArgs f = fused_args(c, m, N);
    f.per_atom = w.per_atom.p + k * per_model;
    f.per_atom_stride = 0;
    TNEP_CUDA(launch_fused(m.variant, m.d.rank, f, 1, st));
  }
  if (ev_done) TNEP_CUDA(cudaEventRecord(ev_done, st));
  TNEP_CUDA(w.partial.ensure((size_t)std::max(S, 1) * reduce_chunks(w.max_atoms) * 9));
  size_t off = 0;
  for (size_t k = 0; k < c->models.size(); ++k) {
    const Model& m = c->models[k];
    TNEP_CUDA(launch_reduce(S, 1, w.offsets.p, w.max_atoms, w.per_atom.p + k * per_model, 0, w.atom_stride, m.C,
                            w.partial.p, w.out.p + off, 0, st));
    off += (size_t)S * m.C;
  }
  return TNEP_OK;
}

// Reads the device status after the stream has synchronised.
tnep_status check_status(tnep_ctx* c, bool* regrow) {
  const DevStatus& s = *c->h_status.p;
  *regrow = false;
  if (s.error == TNEP_ERR_BOX_TOO_SMALL)
    return fail(TNEP_ERR_BOX_TOO_SMALL, "structure " + std::to_string(s.bad_struct) + ": periodic edge < 2 rc_R");
  if (s.error) return fail((tnep_status)s.error, "invalid input in structure " + std::to_string(s.bad_struct));
  if (s.max_cnt_R > c->cap_R || s.max_cnt_A > c->cap_A) {
    const int need_R = std::max(c->cap_R, round_up(s.max_cnt_R + 8, 32));
    const int need_A = std::max(c->cap_A, round_up(s.max_cnt_A + 8, 32));
    if (need_R > c->max_neighbors || need_A > c->max_neighbors)
      return fail(TNEP_ERR_NEIGHBOR_OVERFLOW,
                  "neighbour count " + std::to_string(std::max(s.max_cnt_R, s.max_cnt_A)) + " above the cap " +
                      std::to_string(c->max_neighbors));
    c->cap_R = need_R;
    c->cap_A = need_A;
    *regrow = true;
  }
  return TNEP_OK;
}

tnep_status reset_status(tnep_ctx* c, cudaStream_t st) {
  TNEP_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(DevStatus), st));
  return TNEP_OK;
}

tnep_status finish(tnep_ctx* c, cudaStream_t st, bool* regrow) {
  TNEP_CUDA(cudaMemcpyAsync(c->h_status.p, c->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  TNEP_CUDA(cudaStreamSynchronize(st));
  return check_status(c, regrow);
}

// Copies `count` elements of T to the caller's buffer (host or device) on `st`.
template <class T>
tnep_status copy_out(T* dst, const T* src, size_t count, cudaStream_t st) {
  if (count == 0) return TNEP_OK;
  TNEP_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyDefault, st));
  return TNEP_OK;
}

// Makes `n` elements of a caller input available on the device.
template <class T>
tnep_status stage_in(const T* src, size_t n, DevBuf<T>& buf, const T** dev, cudaStream_t st) {
  if (!src || n == 0) { *dev = src; return TNEP_OK; }
  if (is_device_ptr(src)) { *dev = src; return TNEP_OK; }
  TNEP_CUDA(buf.ensure(n));
  TNEP_CUDA(cudaMemcpyAsync(buf.p, src, sizeof(T) * n, cudaMemcpyHostToDevice, st));
  *dev = buf.p;
  return TNEP_OK;
}

cudaStream_t pick_stream(tnep_ctx* c, void* stream) {
  return stream ? reinterpret_cast<cudaStream_t>(stream) : c->stream;
}

int default_frames_per_batch(int n_atoms, int n_frames) {
  const long long target = 1 << 20;  // ~1 M atoms per pass: >= 20 waves of 304 CTAs
  long long fb = std::max<long long>(1, target / std::max(n_atoms, 1));
  return (int)std::min<long long>(fb, std::max(n_frames, 1));
}

}  // namespace

extern "C" {

const char* tnep_last_error(void) { return g_last_error.c_str(); }

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
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&c->ev_copied[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_consumed[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev_k0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev_k1);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(DevStatus));
  if (e == cudaSuccess) e = c->h_status.ensure(1);
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
    e = cudaMalloc(&m.d_packed, sizeof(float) * m.lay.words);
    if (e == cudaSuccess)
      e = cudaMemcpy(m.d_packed, packed.data(), sizeof(float) * m.lay.words, cudaMemcpyHostToDevice);
    c->models.push_back(std::move(m));
    if (e != cudaSuccess) return bail(cuda_fail(e, "model upload"));
    if (fused_smem_bytes(c->models.back().variant, c->models.back().lay) > 227 * 1024)
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
  for (auto& m : c->models)
    if (m.d_packed) cudaFree(m.d_packed);
  c->ws.release();
  c->pop_params.release();
  c->pop_target.release();
  c->pop_rmse.release();
  if (c->d_status) cudaFree(c->d_status);
  c->h_status.release();
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
      if (value != kFusedBlock) return fail(TNEP_ERR_UNSUPPORTED, "this build uses 128 atoms per CTA");
      return TNEP_OK;
    case TNEP_OPT_CELL_DIV:
      if (value != 1 && value != 2) return fail(TNEP_ERR_INVALID, "cell subdivision must be 1 or 2");
      c->cell_div = (int)value;
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
    case TNEP_OPT_BLOCK_ATOMS: *value = kFusedBlock; return TNEP_OK;
    case TNEP_OPT_LAST_KERNEL_MS: *value = c->last_kernel_ms; return TNEP_OK;
    case TNEP_OPT_CELL_DIV: *value = c->cell_div; return TNEP_OK;
    case TNEP_OPT_LAST_KERNEL_LAUNCHES: *value = c->last_launches; return TNEP_OK;
    case TNEP_OPT_LAST_NBR_MS: *value = c->last_nbr_ms; return TNEP_OK;
    case TNEP_OPT_KERNEL_LAUNCHES_TOTAL: *value = (double)launches_total(); return TNEP_OK;
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
  for (int attempt = 0; attempt < 4; ++attempt) {
    TNEP_TRY(reset_status(c, st));
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
      TNEP_TRY(build_lists(c, st, nf, offs.data(), d_pos, d_box, d_types, n_atoms));
      if (!pos_dev && n_atoms > 0) TNEP_CUDA(cudaEventRecord(c->ev_consumed[b & 1], st));
      TNEP_CUDA(cudaEventRecord(ev[1], st));
      TNEP_TRY(run_models(c, st, nf, nf * n_atoms, ev[2]));
      // scatter results: model m block [n_frames][C_m]
      size_t src_off = 0, dst_base = 0;
      for (const auto& m : c->models) {
        double* dst = out_dev ? out : c->h_out.p;
        TNEP_TRY(copy_out(dst + dst_base + (size_t)f0 * m.C, c->ws.out.p + src_off, (size_t)nf * m.C, st));
        src_off += (size_t)nf * m.C;
        dst_base += (size_t)n_frames * m.C;
      }
    }
    bool regrow = false;
    TNEP_TRY(finish(c, st, &regrow));
    TNEP_TRY(sum_pass_times(c, n_pass));
    if (!regrow) {
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
    TNEP_TRY(reset_status(c, st));
    cudaEvent_t* ev = nullptr;
    TNEP_TRY(pass_events(c, 0, &ev));
    TNEP_CUDA(cudaEventRecord(ev[0], st));
    TNEP_TRY(build_lists(c, st, n_structs, atom_offsets, d_pos, d_box, d_types, std::max(N, 1)));
    TNEP_CUDA(cudaEventRecord(ev[1], st));
    TNEP_TRY(run_models(c, st, n_structs, N, ev[2]));
    bool regrow = false;
    TNEP_TRY(finish(c, st, &regrow));
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
    TNEP_TRY(reset_status(c, st));
    TNEP_TRY(build_lists(c, st, n_structs, atom_offsets, d_pos, d_box, zeros.p, 1));
    bool regrow = false;
    TNEP_TRY(finish(c, st, &regrow));
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
                                      c->ws.cap_R, c->ws.nbr_A.p, c->ws.cnt_A.p, c->ws.cap_A, ocR, ocA, oR, cap_R,
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
    TNEP_TRY(reset_status(c, st));
    TNEP_TRY(build_lists(c, st, n_structs, atom_offsets, d_pos, d_box, d_types, std::max(N, 1)));
    Workspace& w = c->ws;
    const size_t pa_pop = (size_t)m.C * w.atom_stride;
    TNEP_CUDA(w.per_atom.ensure(pa_pop * n_pop));
    TNEP_CUDA(w.out.ensure((size_t)n_pop * n_structs * m.C));
    TNEP_CUDA(c->pop_rmse.ensure(n_pop));
    cudaEvent_t* ev0 = nullptr;
    TNEP_TRY(pass_events(c, 0, &ev0));
    TNEP_CUDA(cudaEventRecord(ev0[1], st));
    TNEP_TRY(compute_moments(c, st, N, m.d.rank == 1, m.d.rank == 2));
    FusedArgs f = fused_args(c, m, N);
    f.model = c->pop_params.p;
    f.model_stride = m.lay.words;
    f.per_atom = w.per_atom.p;
    f.per_atom_stride = pa_pop;
    cudaEvent_t* ev = nullptr;
    TNEP_TRY(pass_events(c, 0, &ev));
    TNEP_CUDA(launch_fused(m.variant, m.d.rank, f, n_pop, st));
    TNEP_CUDA(cudaEventRecord(ev[2], st));
    TNEP_CUDA(w.partial.ensure((size_t)n_pop * n_structs * reduce_chunks(w.max_atoms) * m.C));
    TNEP_CUDA(launch_reduce(n_structs, n_pop, w.offsets.p, w.max_atoms, w.per_atom.p, pa_pop, w.atom_stride, m.C,
                            w.partial.p, w.out.p, (size_t)n_structs * m.C, st));
    TNEP_CUDA(launch_rmse(n_pop, n_structs, m.C, w.out.p, d_target, c->pop_rmse.p, st));
    bool regrow = false;
    TNEP_TRY(finish(c, st, &regrow));
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
  double* d = nullptr;
  const size_t total = n_series + n_work + 2 * (size_t)(M + 1) + (M + 1);
  TNEP_CUDA(cudaMallocAsync((void**)&d, sizeof(double) * total, st));
  double* d_series = d;
  double* d_work = d + n_series;
  double* d_freq = d_work + n_work;
  double* d_spec = d_freq + (M + 1);
  double* d_acf = d_spec + (M + 1);
  tnep_status rc = TNEP_OK;
  cudaError_t e = cudaMemcpyAsync(d_series, series, sizeof(double) * n_series, cudaMemcpyDefault, st);
  if (e == cudaSuccess)
    e = launch_spectrum(d_series, T, C, dt_fs, kind, M, subtract_mean, d_work, d_freq, d_spec, d_acf, st);
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
