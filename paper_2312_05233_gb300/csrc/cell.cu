// General periodic cells: triclinic, and cells shorter than twice the cutoff
// (Sec. II.A: U_i is a function of the pair vectors r_ij to every neighbour
// within the cutoff; in a small or skewed cell a neighbour may appear
// through several images).
//
// Each periodic structure is expanded into an open one: its atoms wrapped
// into the cell, followed by every image r_j + n H (n != 0) whose fractional
// coordinates lie within delta_a = rc_R / d_a of the cell (d_a the spacing of
// the lattice planes normal to axis a).  Any image within rc_R of an atom of
// the cell lies in that region, so the open structure holds every pair of the
// periodic one.  The ordinary batch path then runs on the expanded batch;
// the contributions of the image atoms ("ghosts") are zeroed before the
// per-structure reduction, so only the cell's own atoms are summed.
//
//   k_cell_plan     per structure: H^-1, plane spacings, delta (float64)
//   k_cell_expand   one CTA per structure, atoms in chunks of 256: per atom
//                   the image ranges, a block-wide scan of the counts, then
//                   (write pass) the wrapped atom and its images in a fixed
//                   order (atom, then n0, n1, n2)
//   k_zero_ghosts   per sorted atom of the expanded batch

#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "engine.h"

namespace tnep {

namespace {

struct CellInfo {
  double H[9];
  double Hinv[9];
  double delta[3];
  int periodic;
};

constexpr int kExpandThreads = 256;

__global__ void k_cell_plan(int S, const float* __restrict__ cell, float rc, CellInfo* __restrict__ info,
                            DevStatus* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  CellInfo ci{};
  bool any = false;
  for (int k = 0; k < 9; ++k) {
    ci.H[k] = (double)cell[9 * s + k];
    any |= cell[9 * s + k] != 0.0f;
  }
  ci.periodic = any ? 1 : 0;
  if (any) {
    const double* H = ci.H;
    // rows a = H[0..2], b = H[3..5], c = H[6..8]; Hinv columns from cross products
    const double bc[3] = {H[4] * H[8] - H[5] * H[7], H[5] * H[6] - H[3] * H[8], H[3] * H[7] - H[4] * H[6]};
    const double ca[3] = {H[7] * H[2] - H[8] * H[1], H[8] * H[0] - H[6] * H[2], H[6] * H[1] - H[7] * H[0]};
    const double ab[3] = {H[1] * H[5] - H[2] * H[4], H[2] * H[3] - H[0] * H[5], H[0] * H[4] - H[1] * H[3]};
    const double det = H[0] * bc[0] + H[1] * bc[1] + H[2] * bc[2];
    if (!(fabs(det) > 1e-9)) {
      atomicCAS(&status->error, 0, (int)TNEP_ERR_INVALID);
      atomicCAS(&status->bad_struct, 0, s);
      ci.periodic = 0;
    } else {
      // s = r Hinv with Hinv[:, a] = (row cross product) / det
      for (int k = 0; k < 3; ++k) {
        ci.Hinv[3 * k + 0] = bc[k] / det;
        ci.Hinv[3 * k + 1] = ca[k] / det;
        ci.Hinv[3 * k + 2] = ab[k] / det;
      }
      const double vol = fabs(det);
      const double nrm[3] = {sqrt(bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]),
                             sqrt(ca[0] * ca[0] + ca[1] * ca[1] + ca[2] * ca[2]),
                             sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2])};
      for (int a = 0; a < 3; ++a) ci.delta[a] = (double)rc / (vol / nrm[a]) + 1e-6;
    }
  }
  info[s] = ci;
}

__device__ __forceinline__ void frac_of(const CellInfo& ci, const float* p, double* sf) {
  for (int a = 0; a < 3; ++a) {
    const double v = (double)p[0] * ci.Hinv[a] + (double)p[1] * ci.Hinv[3 + a] + (double)p[2] * ci.Hinv[6 + a];
    sf[a] = v - floor(v);
  }
}

// Image range of one fractional coordinate: n with s + n in [-delta, 1 + delta).
__device__ __forceinline__ void image_range(double s, double delta, int& lo, int& hi) {
  lo = (int)ceil(-delta - s);
  hi = (int)ceil(1.0 + delta - s) - 1;
}

// count pass (out_pos == nullptr): n_ghost[s]; write pass: expanded atoms.
__global__ void __launch_bounds__(kExpandThreads) k_cell_expand(int S, const int* __restrict__ off,
                                                                const float* __restrict__ pos,
                                                                const int* __restrict__ types,
                                                                const CellInfo* __restrict__ info,
                                                                int* __restrict__ n_ghost,
                                                                const int* __restrict__ new_off,
                                                                float* __restrict__ out_pos,
                                                                int* __restrict__ out_types,
                                                                unsigned char* __restrict__ ghost) {
  __shared__ int scan[kExpandThreads];
  __shared__ int base_sh;
  const int s = blockIdx.x;
  const int a0 = off[s], a1 = off[s + 1], n = a1 - a0;
  const CellInfo ci = info[s];
  const int o0 = new_off ? new_off[s] : 0;
  // the structure's own atoms first
  if (out_pos) {
    for (int k = threadIdx.x; k < n; k += kExpandThreads) {
      const int a = a0 + k;
      float* q = out_pos + 3 * (size_t)(o0 + k);
      if (ci.periodic) {
        double sf[3];
        frac_of(ci, pos + 3 * (size_t)a, sf);
        for (int c = 0; c < 3; ++c)
          q[c] = (float)(sf[0] * ci.H[c] + sf[1] * ci.H[3 + c] + sf[2] * ci.H[6 + c]);
      } else {
        q[0] = pos[3 * (size_t)a]; q[1] = pos[3 * (size_t)a + 1]; q[2] = pos[3 * (size_t)a + 2];
      }
      out_types[o0 + k] = types[a];
      ghost[o0 + k] = 0;
    }
  }
  if (!ci.periodic) {
    if (!out_pos && threadIdx.x == 0) n_ghost[s] = 0;
    return;
  }
  if (threadIdx.x == 0) base_sh = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += kExpandThreads) {
    const int k = c0 + threadIdx.x;
    int cnt = 0, lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
    double sf[3] = {0.0, 0.0, 0.0};
    if (k < n) {
      frac_of(ci, pos + 3 * (size_t)(a0 + k), sf);
      for (int a = 0; a < 3; ++a) image_range(sf[a], ci.delta[a], lo[a], hi[a]);
      cnt = (hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1) - 1;  // n = 0 is the atom itself
    }
    scan[threadIdx.x] = cnt;
    __syncthreads();
    // inclusive Hillis-Steele scan (fixed order)
    for (int w = 1; w < kExpandThreads; w <<= 1) {
      const int v = threadIdx.x >= w ? scan[threadIdx.x - w] : 0;
      __syncthreads();
      scan[threadIdx.x] += v;
      __syncthreads();
    }
    const int excl = scan[threadIdx.x] - cnt;
    const int base = base_sh;
    if (out_pos && cnt > 0) {
      int g = o0 + n + base + excl;
      const int t = types[a0 + k];
      for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
        for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
          for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
            if (n0 == 0 && n1 == 0 && n2 == 0) continue;
            const double f0 = sf[0] + n0, f1 = sf[1] + n1, f2 = sf[2] + n2;
            float* q = out_pos + 3 * (size_t)g;
            for (int c = 0; c < 3; ++c) q[c] = (float)(f0 * ci.H[c] + f1 * ci.H[3 + c] + f2 * ci.H[6 + c]);
            out_types[g] = t;
            ghost[g] = 1;
            ++g;
          }
    }
    __syncthreads();
    if (threadIdx.x == kExpandThreads - 1) base_sh = base + scan[kExpandThreads - 1];
    __syncthreads();
  }
  if (!out_pos && threadIdx.x == 0) n_ghost[s] = base_sh;
}

__global__ void k_zero_ghosts(int N, const int* __restrict__ sorted_orig, const unsigned char* __restrict__ ghost,
                              float* __restrict__ per_atom, int atom_stride, int C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || !ghost[sorted_orig[i]]) return;
  for (int c = 0; c < C; ++c) per_atom[(size_t)c * atom_stride + i] = 0.f;
}

}  // namespace

cudaError_t launch_zero_ghosts(int N, const int* sorted_orig, const unsigned char* ghost, float* per_atom,
                               int atom_stride, int C, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  count_launches(1);
  k_zero_ghosts<<<(N + 255) / 256, 256, 0, st>>>(N, sorted_orig, ghost, per_atom, atom_stride, C);
  return cudaGetLastError();
}

}  // namespace tnep

using namespace tnep;

extern "C" {

tnep_status tnep_eval_batch_cell(tnep_ctx* c, int n_structs, const int* atom_offsets, const float* pos,
                                 const float* cell, const int* types, double* out, void* stream) {
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
  if (!is_device_ptr(types))
    for (int a = 0; a < N; ++a)
      if (types[a] < 0 || types[a] >= c->n_types) return fail(TNEP_ERR_INVALID, "type index out of range");
  Workspace& w = c->ws;
  DevBuf<float> d_pos_in, d_cell, d_epos, d_ebox;
  DevBuf<int> d_types_in, d_off, d_newoff, d_nghost, d_etypes;
  DevBuf<unsigned char> d_ghost;
  DevBuf<CellInfo> d_info;
  auto release = [&]() {
    d_pos_in.release(); d_cell.release(); d_epos.release(); d_ebox.release(); d_types_in.release();
    d_off.release(); d_newoff.release(); d_nghost.release(); d_etypes.release(); d_ghost.release();
    d_info.release();
  };
  auto body = [&]() -> tnep_status {
    TNEP_CUDA(d_pos_in.ensure((size_t)std::max(N, 1) * 3));
    TNEP_CUDA(d_types_in.ensure(std::max(N, 1)));
    TNEP_CUDA(d_cell.ensure((size_t)n_structs * 9));
    TNEP_CUDA(d_off.ensure(n_structs + 1));
    TNEP_CUDA(d_nghost.ensure(n_structs));
    TNEP_CUDA(d_info.ensure(n_structs));
    if (N > 0) {
      TNEP_CUDA(cudaMemcpyAsync(d_pos_in.p, pos, sizeof(float) * 3 * N, cudaMemcpyDefault, st));
      TNEP_CUDA(cudaMemcpyAsync(d_types_in.p, types, sizeof(int) * N, cudaMemcpyDefault, st));
    }
    if (cell)
      TNEP_CUDA(cudaMemcpyAsync(d_cell.p, cell, sizeof(float) * 9 * n_structs, cudaMemcpyDefault, st));
    else
      TNEP_CUDA(cudaMemsetAsync(d_cell.p, 0, sizeof(float) * 9 * n_structs, st));
    TNEP_CUDA(cudaMemcpyAsync(d_off.p, atom_offsets, sizeof(int) * (n_structs + 1), cudaMemcpyHostToDevice, st));
    TNEP_TRY(reset_status(w, st));
    k_cell_plan<<<(n_structs + 127) / 128, 128, 0, st>>>(n_structs, d_cell.p, c->rc_R, d_info.p, w.d_status);
    k_cell_expand<<<n_structs, kExpandThreads, 0, st>>>(n_structs, d_off.p, d_pos_in.p, d_types_in.p, d_info.p,
                                                        d_nghost.p, nullptr, nullptr, nullptr, nullptr);
    count_launches(2);
    TNEP_CUDA(cudaGetLastError());
    std::vector<int> ng(n_structs);
    TNEP_CUDA(cudaMemcpyAsync(ng.data(), d_nghost.p, sizeof(int) * n_structs, cudaMemcpyDeviceToHost, st));
    bool regrow = false;
    TNEP_TRY(finish(c, w, st, &regrow));  // synchronises; reports a degenerate cell
    std::vector<int> eoff(n_structs + 1, 0);
    long long tot = 0;
    for (int s = 0; s < n_structs; ++s) {
      tot += (long long)(atom_offsets[s + 1] - atom_offsets[s]) + ng[s];
      if (tot >= kMaxBatchAtoms) return fail(TNEP_ERR_INVALID, "expanded batch (cell atoms + images) exceeds 2^29 atoms");
      eoff[s + 1] = (int)tot;
    }
    const int Ne = (int)tot;
    TNEP_CUDA(d_newoff.ensure(n_structs + 1));
    TNEP_CUDA(d_epos.ensure((size_t)std::max(Ne, 1) * 3));
    TNEP_CUDA(d_etypes.ensure(std::max(Ne, 1)));
    TNEP_CUDA(d_ghost.ensure(std::max(Ne, 1)));
    TNEP_CUDA(d_ebox.ensure((size_t)n_structs * 3));
    TNEP_CUDA(cudaMemsetAsync(d_ebox.p, 0, sizeof(float) * 3 * n_structs, st));
    TNEP_CUDA(cudaMemcpyAsync(d_newoff.p, eoff.data(), sizeof(int) * (n_structs + 1), cudaMemcpyHostToDevice, st));
    k_cell_expand<<<n_structs, kExpandThreads, 0, st>>>(n_structs, d_off.p, d_pos_in.p, d_types_in.p, d_info.p,
                                                        d_nghost.p, d_newoff.p, d_epos.p, d_etypes.p, d_ghost.p);
    count_launches(1);
    TNEP_CUDA(cudaGetLastError());
    const int Ctot = total_C(c);
    for (int attempt = 0; attempt < 4; ++attempt) {
      TNEP_TRY(reset_status(w, st));
      TNEP_TRY(build_lists(c, w, st, n_structs, eoff.data(), d_epos.p, d_ebox.p, d_etypes.p, std::max(Ne, 1)));
      TNEP_TRY(run_models(c, w, st, n_structs, Ne, nullptr, d_ghost.p));
      regrow = false;
      TNEP_TRY(finish(c, w, st, &regrow));
      if (regrow) continue;
      TNEP_TRY(copy_out(out, w.out.p, (size_t)n_structs * Ctot, st));
      TNEP_CUDA(cudaStreamSynchronize(st));
      return TNEP_OK;
    }
    return fail(TNEP_ERR_NEIGHBOR_OVERFLOW, "neighbour lists kept overflowing");
  };
  const tnep_status rc = body();
  cudaStreamSynchronize(st);
  release();
  return rc;
}

}  // extern "C"
