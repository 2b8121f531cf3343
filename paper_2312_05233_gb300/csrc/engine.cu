// Host-side engine of libtnep (see engine.h).

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "engine.h"

namespace {

thread_local std::string g_last_error;

std::atomic<long long> g_allocs{0};
long long g_fault_at = 0;  // 0 = no injected failure
std::once_flag g_fault_once;

// True if this allocation is the one TNEP_FAULT=oom@N asks to fail.
bool injected_oom() {
  std::call_once(g_fault_once, [] {
    const char* v = std::getenv("TNEP_FAULT");
    if (v && std::strncmp(v, "oom@", 4) == 0) g_fault_at = std::atoll(v + 4);
  });
  const long long k = g_allocs.fetch_add(1, std::memory_order_relaxed) + 1;
  return g_fault_at > 0 && k == g_fault_at;
}

}  // namespace

namespace tnep {

cudaError_t dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_oom()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (injected_oom()) return cudaErrorMemoryAllocation;
  return cudaMallocAsync(p, bytes, st);
}

cudaError_t host_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_oom()) return cudaErrorMemoryAllocation;
  return cudaHostAlloc(p, bytes, cudaHostAllocDefault);
}

long long alloc_count() { return g_allocs.load(std::memory_order_relaxed); }

tnep_status fail(tnep_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

tnep_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free error
  return fail(e == cudaErrorMemoryAllocation ? TNEP_ERR_OOM : TNEP_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

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

void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }
const char* last_error_cstr() { return g_last_error.c_str(); }


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
// Packed word of every flat parameter (the flat order is the one documented
// for tnep_model_desc.params); padding words and the scaler are not mapped.
void pack_index_map(const Model& m, int T, int* dst) {
  const ModelLayout& L = m.lay;
  size_t o = 0;
  for (int net = 0; net < m.nets; ++net) {
    for (int h = 0; h < L.H; ++h)
      for (int d = 0; d < m.D; ++d) dst[o++] = L.off_W0 + (net * L.H + h) * L.Dp + d;
    for (int h = 0; h < L.H; ++h) dst[o++] = L.off_b0 + net * L.H + h;
    for (int h = 0; h < L.H; ++h) dst[o++] = L.off_w1 + net * L.H + h;
    dst[o++] = L.off_b1 + net;
  }
  for (int p = 0; p < T * T; ++p)
    for (int k = 0; k < m.nR * m.bR; ++k) dst[o++] = L.off_cR + p * L.stride_cR + k;
  for (int p = 0; p < T * T; ++p)
    for (int k = 0; k < m.nA * m.bA; ++k) dst[o++] = L.off_cA + p * L.stride_cA + k;
}

void pack_params(const Model& m, int T, const float* flat, const float* scaler, float* out) {
  const ModelLayout& L = m.lay;
  std::fill(out, out + L.words, 0.f);
  std::vector<int> dst(m.params.size());
  pack_index_map(m, T, dst.data());
  for (size_t i = 0; i < dst.size(); ++i) out[dst[i]] = flat[i];
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
  if (d.mlp_precision < 0 || d.mlp_precision > 2) return fail(TNEP_ERR_INVALID, "mlp_precision must be 0, 1 or 2");
  if (d.mlp_precision != 0) {
    const int D = (d.n_max_R + 1) + (d.n_max_A + 1) * (d.l_max + (d.use_4body ? 1 : 0));
    if (D > 32 || d.n_hidden > 32)
      return fail(TNEP_ERR_UNSUPPORTED, "the tensor-core network takes at most 32 descriptor components and 32 hidden units");
  }
  const size_t want = expected_params(d, T);
  if (d.n_params != want)
    return fail(TNEP_ERR_INVALID, "n_params " + std::to_string(d.n_params) + " != layout " + std::to_string(want));
  return TNEP_OK;
}

// Builds cell and neighbour lists for a batch whose inputs are on the device.
tnep_status ensure_batch(tnep_ctx* c, Workspace& w, cudaStream_t st, int S, const int* h_offsets, int cap_R,
                         int cap_A) {
  const int N = h_offsets[S];
  const int stride = round_up(std::max(N, 1), 32);
  int mx = 0;
  for (int s = 0; s < S; ++s) mx = std::max(mx, h_offsets[s + 1] - h_offsets[s]);
  w.max_atoms = mx;
  w.atom_stride = stride;
  w.cells_cap = 2 * N + 8 * S;
  w.cap_R = cap_R;
  w.cap_A = cap_A;
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
  return TNEP_OK;
}

tnep_status build_lists(tnep_ctx* c, Workspace& w, cudaStream_t st, int S, const int* h_offsets, const float* d_pos,
                        const float* d_box, const int* d_types, int types_period, const ListSpec* spec) {
  const float rc_R = spec ? spec->rc_R : c->rc_R, rc_A = spec ? spec->rc_A : c->rc_A;
  TNEP_TRY(ensure_batch(c, w, st, S, h_offsets, spec ? spec->cap_R : c->cap_R, spec ? spec->cap_A : c->cap_A));
  const int N = h_offsets[S];
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
  a.rc_R = rc_R;
  a.rc_A = rc_A;
  a.cell_div = c->cell_div;
  a.x_div = c->x_div;
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
  a.seg_stride = w.atom_stride;
  w.two_ended = c->n_types == 2 ? 1 : 0;
  a.two_ended = w.two_ended;
  a.cnt_R = w.cnt_R.p;
  a.cnt_A = w.cnt_A.p;
  a.cap_R = w.cap_R;
  a.cap_A = w.cap_A;
  a.cells_cap = w.cells_cap;
  a.status = w.d_status;
  TNEP_CUDA(launch_neighbor_pipeline(a, st));
  return TNEP_OK;
}

// Trajectory pass with Verlet-skin reuse: skin lists (cutoffs + skin) of the
// pass's first frame in `sw`, then every frame's exact lists compacted from
// them into `w` (frames in the first frame's cell order).  Raises
// skin_violation in w's status when an atom moved more than skin / 2.
tnep_status skin_lists(tnep_ctx* c, Workspace& w, Workspace& sw, cudaStream_t st, int nf, int N, const float* d_pos,
                       const float* d_box, const int* d_types) {
  const int one[2] = {0, N};
  ListSpec spec{c->rc_R + c->skin, c->rc_A + c->skin, c->skin_cap, 4};
  TNEP_TRY(build_lists(c, sw, st, 1, one, d_pos, d_box, d_types, N, &spec));
  std::vector<int> offs(nf + 1);
  for (int k = 0; k <= nf; ++k) offs[k] = k * N;
  TNEP_TRY(ensure_batch(c, w, st, nf, offs.data(), c->cap_R, c->cap_A));
  SkinArgs a{};
  a.nf = nf;
  a.N = N;
  a.pos = d_pos;
  a.box = d_box;
  a.types = d_types;
  a.types_period = std::max(N, 1);
  a.n_types = c->n_types;
  a.sorted_orig = sw.sorted_orig.p;
  a.ref4 = sw.pos4.p;
  a.ref_box = sw.boxes.p;
  a.skin_nbr = sw.nbr_R.p;
  a.skin_seg = sw.seg_R.p;
  a.skin_cap = sw.cap_R;
  a.skin_seg_stride = sw.atom_stride;
  a.skin_two_ended = sw.two_ended;
  a.rc2R = c->rc_R * c->rc_R;
  a.rc2A = c->rc_A * c->rc_A;
  const float hs = 0.5f * c->skin * 0.999f;
  a.half_skin2 = hs * hs;
  a.pos4 = w.pos4.p;
  a.sorted_struct = w.sorted_struct.p;
  a.boxes = w.boxes.p;
  a.nbr_R = w.nbr_R.p;
  a.nbr_A = w.nbr_A.p;
  a.cnt_R = w.cnt_R.p;
  a.cnt_A = w.cnt_A.p;
  a.seg_R = w.seg_R.p;
  a.seg_stride = w.atom_stride;
  a.cap_R = w.cap_R;
  a.cap_A = w.cap_A;
  a.status = w.d_status;
  w.two_ended = 0;  // the compacted lists are front-packed per type
  TNEP_CUDA(launch_skin_compact(a, st));
  return TNEP_OK;
}

// Radial moments of the lists in the workspace (F always; V for rank-1 and W
// for rank-2 models).
tnep_status compute_moments(tnep_ctx* c, Workspace& w, cudaStream_t st, int N, bool need_v, bool need_w) {
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
  r.two_ended = w.two_ended;
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

FusedArgs fused_args(tnep_ctx* c, Workspace& w, const Model& m, int N) {
  FusedArgs f{};
  f.n_atoms = N;
  f.pos4 = w.pos4.p;
  f.sorted_struct = w.sorted_struct.p;
  f.boxes = w.boxes.p;
  f.mom = w.mom.p;
  f.mom_stride = w.atom_stride;
  f.v0 = w.mom_v0;
  f.w0 = w.mom_w0;
  f.status = w.d_status;
  f.nbr_A = w.nbr_A.p;
  f.cnt_A = w.cnt_A.p;
  f.cap_A = w.cap_A;
  f.model = m.d_packed;
  f.model_stride = 0;
  f.lay = m.lay;
  f.rc_R = c->rc_R;
  f.rc_A = c->rc_A;
  f.atom_stride = w.atom_stride;
  f.wait_tries = c->wait_tries;
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

tnep_status run_models(tnep_ctx* c, Workspace& w, cudaStream_t st, int S, int N, cudaEvent_t ev_done,
                       const unsigned char* ghost, cudaStream_t red_st) {
  const size_t per_model = (size_t)9 * w.atom_stride;
  TNEP_CUDA(w.per_atom.ensure(per_model * c->models.size()));
  TNEP_CUDA(w.out.ensure((size_t)std::max(S, 1) * total_C(c)));
  TNEP_TRY(compute_moments(c, w, st, N, any_rank(c, 1), any_rank(c, 2)));
  // per-pair cache of the angular walks, reused by every model in turn
  // (skipped when the lists' cap would make it larger than 16 GB: a pass of
  // 2^21 atoms at cap_A = 64 takes 8.6 GB)
  constexpr size_t kPairCacheMaxBytes = size_t(16) << 30;
  int quads = 0;
  for (const auto& m : c->models) quads = std::max(quads, pair_cache_quads(m.d.n_max_A + 1));
  const int pc_stride = round_up(std::max(N, 1), 128);
  const size_t pc_elems = (size_t)w.cap_A * quads * pc_stride;
  const bool use_pc = c->pair_cache && pc_elems * sizeof(float4) <= kPairCacheMaxBytes;
  if (use_pc) TNEP_CUDA(w.pcache.ensure(pc_elems));
  const int* offsets = w.offsets.p;
  if (red_st) {
    // the previous pass's sums have read the per-atom outputs and offsets
    TNEP_CUDA(cudaStreamWaitEvent(st, c->ev_reduced, 0));
    TNEP_CUDA(w.red_offsets.ensure((size_t)S + 1));
    TNEP_CUDA(cudaMemcpyAsync(w.red_offsets.p, w.offsets.p, sizeof(int) * ((size_t)S + 1), cudaMemcpyDeviceToDevice,
                              st));
    offsets = w.red_offsets.p;
  }
  for (size_t k = 0; k < c->models.size(); ++k) {
    const Model& m = c->models[k];
    FusedArgs f = fused_args(c, w, m, N);
    f.per_atom = w.per_atom.p + k * per_model;
    f.per_atom_stride = 0;
    f.pcache = use_pc ? w.pcache.p : nullptr;
    f.pc_stride = pc_stride;
    TNEP_CUDA(launch_fused(m.variant, m.d.rank, f, 1, c->block_atoms, m.d.mlp_precision, st));
  }
  if (ev_done) TNEP_CUDA(cudaEventRecord(ev_done, st));
  if (ghost)
    for (size_t k = 0; k < c->models.size(); ++k)
      TNEP_CUDA(launch_zero_ghosts(N, w.sorted_orig.p, ghost, w.per_atom.p + k * per_model, w.atom_stride,
                                   c->models[k].C, st));
  TNEP_CUDA(w.partial.ensure((size_t)std::max(S, 1) * reduce_chunks(w.max_atoms) * 9));
  cudaStream_t rs = st;
  if (red_st) {
    TNEP_CUDA(cudaEventRecord(c->ev_fused, st));
    TNEP_CUDA(cudaStreamWaitEvent(red_st, c->ev_fused, 0));
    rs = red_st;
  }
  size_t off = 0;
  for (size_t k = 0; k < c->models.size(); ++k) {
    const Model& m = c->models[k];
    TNEP_CUDA(launch_reduce(S, 1, offsets, w.max_atoms, w.per_atom.p + k * per_model, 0, w.atom_stride, m.C,
                            w.partial.p, w.out.p + off, 0, rs));
    off += (size_t)S * m.C;
  }
  return TNEP_OK;
}

// Reads the device status after the stream has synchronised.
tnep_status check_status(tnep_ctx* c, const DevStatus& s, bool* regrow) {
  *regrow = false;
  if (s.error == TNEP_ERR_BOX_TOO_SMALL)
    return fail(TNEP_ERR_BOX_TOO_SMALL, "structure " + std::to_string(s.bad_struct) + ": periodic edge < 2 rc_R");
  if (s.error == TNEP_ERR_TIMEOUT)
    return fail(TNEP_ERR_TIMEOUT, "a device-side bounded wait gave up (tensor-core product not completed in time)");
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

tnep_status reset_status(Workspace& w, cudaStream_t st) {
  TNEP_CUDA(cudaMemsetAsync(w.d_status, 0, sizeof(DevStatus), st));
  return TNEP_OK;
}

tnep_status finish(tnep_ctx* c, Workspace& w, cudaStream_t st, bool* regrow) {
  TNEP_CUDA(cudaMemcpyAsync(w.h_status.p, w.d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  TNEP_CUDA(cudaStreamSynchronize(st));
  return check_status(c, *w.h_status.p, regrow);
}

// Copies bytes to the caller's buffer (host or device) on `st`.
tnep_status copy_out_bytes(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return TNEP_OK;
  TNEP_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
  return TNEP_OK;
}


cudaStream_t pick_stream(tnep_ctx* c, void* stream) {
  return stream ? reinterpret_cast<cudaStream_t>(stream) : c->stream;
}

int default_frames_per_batch(int n_atoms, int n_frames) {
  // ~2 M atoms per pass: > 50 waves of 304 CTAs of the fused kernel, and the
  // fixed costs of a pass (small neighbour kernels, reductions, kernel tails)
  // spread over many frames (bulk water, 2,000 frames: 418.6 ms per step at
  // 25 frames per pass, 409.1 ms at 50, 407.7 ms at 64)
  const long long target = 1 << 21;
  long long fb = std::max<long long>(1, target / std::max(n_atoms, 1));
  return (int)std::min<long long>(fb, std::max(n_frames, 1));
}


}  // namespace tnep
