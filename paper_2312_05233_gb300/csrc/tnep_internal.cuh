// Internal declarations shared by the CUDA translation units of libtnep.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tnep.h"

namespace tnep {

constexpr int kMaxTypes = 8;
constexpr int kFusedBlockMax = 128;  // atoms per CTA of the fused kernel (one atom per thread): 64 or 128
// Radial scratch entries carry the neighbour type in bits 29-31, so a batch
// holds fewer than 2^29 atoms.
constexpr int kTypeShift = 29;
constexpr int kIndexMask = (1 << kTypeShift) - 1;
constexpr int kMaxBatchAtoms = 1 << kTypeShift;
constexpr int kMomBasis = 9;  // radial moments are computed for k = 0..8 (basis_R <= 8)

// Device-side status word, reset before each batch and read back after it.
struct DevStatus {
  int error;        // first tnep_status raised on the device (0 = none)
  int bad_struct;   // structure that raised it
  int max_cnt_R;    // largest radial neighbour count seen above the cap
  int max_cnt_A;    // largest angular neighbour count seen above the cap
  int skin_violation;  // an atom moved more than skin / 2 (or the box changed) within a pass
  int work_next;    // work counter of the persistent fused kernel (zeroed before each of its launches)
};

// Per-structure cell grid (orthorhombic, periodic or open per axis).
struct StructGrid {
  float L[3];       // periodic edge (0 = open axis)
  float invL[3];    // 1/L rounded to float32 (0 on open axes)
  float origin[3];  // grid origin (0 on periodic axes, min corner on open axes)
  float cinv[3];    // cells per Angstrom
  int nc[3];        // cells per axis
  int cell_offset;  // first global cell of this structure
};

// Per-structure box as the fused kernel needs it.
struct StructBox {
  float L[3];
  float invL[3];
};

// Neighbour lists are stored warp-tiled: entry k of atom i lives at
// ((i >> 5) * cap + k) * 32 + (i & 31), so one warp's lists are contiguous
// and every row of 32 entries is one 128-byte line.
__host__ __device__ __forceinline__ size_t nbr_index(int i, int k, int cap) {
  return ((size_t)(i >> 5) * cap + k) * 32 + (i & 31);
}

// Arguments of the neighbour-list pipeline.
struct NbrArgs {
  int n_structs;
  int n_atoms;
  const int* offsets;       // [S+1] device
  const float* pos;         // [N][3] input order, device
  const float* box;         // [S][3] device or null
  const int* types;         // input types, device
  int types_period;         // type of atom g = types[g % types_period]
  int n_types;              // types outside [0, n_types) raise TNEP_ERR_INVALID (and read as 0)
  float rc_R, rc_A;
  int cell_div;             // cells have edge >= rc_R / cell_div
  int x_div;                // with cell_div = 1: cells have edge >= rc_R / x_div along x (window scan)
  // outputs / scratch
  StructGrid* grids;        // [S]
  StructBox* boxes;         // [S]
  int* struct_cells;        // [S+1] cells per structure, then exclusive scan
  int* struct_flags;        // [S] bit 0: a coordinate lies outside [0, L) on a periodic axis
  int* atom_struct;         // [N] structure of each input atom
  int* atom_cell;           // [N]
  int* atom_slot;           // [N]
  int* cell_count;          // [cells_cap]
  int* cell_start;          // [cells_cap + 1]
  int* cell_atoms;          // [N] scatter target
  int* sorted_orig;         // [N] sorted -> input index
  int* orig_sorted;         // [N] input -> sorted index
  int* sorted_struct;       // [N]
  float4* pos4;             // [N] sorted positions, w = type bits
  int* nbr_R; int* nbr_A;   // warp-tiled lists (sorted indices); radial sorted by neighbour type
  int* nbr_tmp;             // radial scratch (type-tagged), same layout as nbr_R
  int* seg_R;               // [n_types][seg_stride] radial neighbours of each type
  int seg_stride;
  int two_ended;            // two types: type 0 from entry 0 up, type 1 from entry cap_R - 1 down
  int* cnt_R; int* cnt_A;   // [N] true counts (may exceed caps)
  int cap_R, cap_A;
  int cells_cap;
  DevStatus* status;
};

// First radial-list entry of neighbour type t: the running start of the
// front-packed layout, or cap - n for type 1 of a two-ended list.
__host__ __device__ inline int radial_segment_start(int two_ended, int t, int running, int n, int cap) {
  return (two_ended && t == 1) ? cap - n : running;
}

// Sets the thread-local message returned by tnep_last_error().
void set_last_error(const char* msg);

// Process-wide count of kernels this library has launched.
void count_launches(int n);
long long launches_total();

// Verlet-skin reuse within a trajectory pass (see skin_lists in engine.cu).
struct SkinArgs {
  int nf, N;
  const float* pos;           // [nf][N][3] input order (device)
  const float* box;           // [nf][3] or null
  const int* types; int types_period;
  int n_types;
  const int* sorted_orig;     // first frame: sorted -> input index
  const float4* ref4;         // first frame positions, sorted
  const StructBox* ref_box;   // first frame box
  const int* skin_nbr; const int* skin_seg; int skin_cap, skin_seg_stride;  // type-sorted skin lists
  int skin_two_ended;
  float rc2R, rc2A, half_skin2;
  float4* pos4; int* sorted_struct; StructBox* boxes;   // batch outputs
  int* nbr_R; int* nbr_A; int* cnt_R; int* cnt_A; int* seg_R; int seg_stride; int cap_R, cap_A;
  DevStatus* status;
};
cudaError_t launch_skin_compact(const SkinArgs& a, cudaStream_t st);

// Launches the cell-list + neighbour pipeline on `st`.
cudaError_t launch_neighbor_pipeline(const NbrArgs& a, cudaStream_t st);

// Radial moments per atom and neighbour type t (SoA, slot-major, stride mom_stride):
//   F^t_k     = sum_{j of type t} f_k(r_ij)                       slots  t*B + k
//   V^t_k,a   = sum_j r_ij f_k'(r_ij) r_ij^a                      slots  v0 + (t*B + k)*3 + a
//   W^t_k,ab  = sum_j f_k'(r_ij) / r_ij  r_ij^a r_ij^b  (ab in xx xy xz yy yz zz)  slots w0 + (t*B + k)*6 + c
// with B = kMomBasis.  They hold everything the radial descriptor and the
// radial part of Eqs. 3-4 need, for every model sharing rc_R.
struct RadialArgs {
  int n_atoms, n_types;
  const float4* pos4;
  const int* sorted_struct;
  const StructBox* boxes;
  const int* nbr_R; int cap_R;
  const int* seg_R; int seg_stride;
  int two_ended;
  float rc_R;
  float* mom; int mom_stride;
  int v0, w0;  // slot bases, -1 when not computed
};
cudaError_t launch_radial_moments(const RadialArgs& a, cudaStream_t st);

// Packed model layout in device memory (floats).
struct ModelLayout {
  int n_types, nets, H, D, Dp;
  int stride_cR, stride_cA;        // floats per (ti, tj) coefficient block
  int off_cR, off_cA, off_W0, off_b0, off_w1, off_b1, off_scaler;
  int words;                       // total floats, multiple of 4
};

// Layout of the packed model as the fused kernel keeps it in shared memory:
// without W0 (its FP32 block of nets x H x Dp floats, which the tensor-core
// network does not read there) the words after it move down by that size.
__host__ __device__ inline ModelLayout smem_layout(const ModelLayout& g, bool drop_w0) {
  ModelLayout s = g;
  if (drop_w0) {
    const int w0n = g.off_b0 - g.off_W0;
    s.off_W0 = -1;
    s.off_b0 -= w0n;
    s.off_w1 -= w0n;
    s.off_b1 -= w0n;
    s.off_scaler -= w0n;
    s.words -= w0n;
  }
  return s;
}

// Arguments of the fused descriptor -> network -> partial force -> contraction kernel.
struct FusedArgs {
  int n_atoms;
  const float4* pos4;
  const int* sorted_struct;
  const StructBox* boxes;
  const float* mom; int mom_stride; int v0, w0;   // radial moments (see RadialArgs)
  const int* nbr_A; const int* cnt_A; int cap_A;
  const float* model;        // packed model (first individual)
  size_t model_stride;       // floats between individuals (population), 0 otherwise
  ModelLayout lay;
  float rc_R, rc_A;
  float* per_atom;           // [pop][C][atom_stride] (SoA, sorted order)
  size_t per_atom_stride;    // floats between individuals
  int atom_stride;           // row stride of the SoA output
  int pop_major;             // 1: the individual varies fastest over the work items
  int n_pop;                 // individuals (set by the launcher)
  const float* amom; int amom_slots;   // angular moments (factored population path), else null
  DevStatus* status;         // error word (bounded waits of the tensor-core path)
  long long wait_tries;      // try_wait limit of the tensor-core network's product waits
  // Per-pair cache of the angular walk (single-individual launches, else
  // null): the forward walk stores, for pair k of atom i, r_ij and 1/|r_ij|,
  // g_n and g_n' in pair_cache_quads(NA) float4 at
  // pcache[(k * quads + q) * pc_stride + i]; the backward walk reads them back
  // instead of repeating the neighbour gather, the minimum image, the basis
  // and the coefficient sums.
  float4* pcache;
  int pc_stride;
};
__host__ __device__ constexpr int pair_cache_quads(int na) { return (4 + 2 * na + 3) / 4; }
// Default try_wait limit of the device-side bounded waits.
constexpr long long kDefaultWaitTries = 1LL << 22;

// Angular moments of the basis for population evaluation (angmom.cu): B, and
// Phi (rank 1) or Psi (rank 2).  Per (t, k) the B block holds NLM slots padded
// to a multiple of 4 and the Phi / Psi block NLM * C slots padded likewise;
// all B blocks come first.  Layout (warp-tiled, four slots per float4): slot
// s of atom i at ((i / 32) * n_slots + (s & ~3)) * 32 + (i % 32) * 4 + (s & 3),
// so a warp reads four consecutive slots of its 32 atoms as one 512-byte load.
struct AngMomArgs {
  int n_atoms, n_types;
  const float4* pos4;
  const int* sorted_struct;
  const StructBox* boxes;
  const int* nbr_A; const int* cnt_A; int cap_A;
  float rc_A;
  float* amom; int amom_slots;
};
__host__ __device__ constexpr int pad4(int n) { return (n + 3) & ~3; }
__host__ __device__ inline size_t amom_index(int i, int s, int n_slots) {
  return ((size_t)(i >> 5) * n_slots + (s & ~3)) * 32 + (size_t)(i & 31) * 4 + (s & 3);
}
size_t angular_moment_slots(int variant, int rank, int n_types);
cudaError_t launch_angular_moments(int variant, int rank, const AngMomArgs& a, cudaStream_t st);

// Population evaluation with the angular products on the tensor cores
// (pop_tc.cu): tiles of kPopTcAtoms atoms of one centre type x
// kPopTcIndividuals individuals per CTA.  Standard descriptor sizes only
// (5 x 9 radial and angular, l_max 4, 4-body), at most 3 types, FP32 network.
constexpr int kPopTcIndividuals = 25;
constexpr int kPopTcAtoms = 5;
struct PopTcArgs {
  int n_tiles, n_mt, n_pop, n_types, n_atoms;
  const int* tiles;               // [n_tiles][8]: atoms 0..4 (n_atoms = empty), centre type, count
  const unsigned char* mom_tc;    // per-atom moment blocks (pop_tc_moment_stride bytes each), atom n_atoms = 0
  size_t mom_tc_stride;
  const unsigned char* coef_tc;   // [n_types][n_mt] coefficient tiles
  const float* params;            // [n_pop][lay.words] packed
  ModelLayout lay;
  const float* mom; int mom_stride; int v0, w0;   // radial moments (see RadialArgs)
  float* per_atom; size_t per_atom_stride; int atom_stride;
  DevStatus* status;
};
size_t pop_tc_moment_stride(int rank);
size_t pop_tc_coef_bytes();
cudaError_t launch_moments_tc(int n_atoms, int n_types, int rank, const float* amom, int amom_slots,
                              unsigned char* dst, cudaStream_t st);
cudaError_t launch_coef_tc(int n_pop, int n_types, int n_mt, const float* params, const ModelLayout& lay,
                           unsigned char* dst, cudaStream_t st);
cudaError_t launch_pop_tc(int rank, const PopTcArgs& a, cudaStream_t st);

// Kernel variant keys (must match the compiled instantiations).
enum Variant { kVarStd = 0, kVarSmall = 1, kVarCount = 2 };

int variant_of(int nR, int nA, int bR, int bA, int lmax, int fb);
// tcm: network products on the CUDA cores in FP32 (0), on the tensor cores
// with BF16 operands and FP32 accumulation (1), or on the tensor cores with
// split high/low BF16 operands, three products (2); 1 and 2 use 128 atoms per CTA.
size_t fused_smem_bytes(int variant, const ModelLayout& lay, int block, int tcm);
cudaError_t launch_fused(int variant, int rank, const FusedArgs& a, int n_pop, int block, int tcm, cudaStream_t st);

// Per-structure FP64 reduction of per-atom contributions.  `max_atoms` is
// the largest structure; `partial` holds n_pop * n_structs * reduce_chunks(max_atoms) * C doubles.
constexpr int kReduceChunk = 2048;
inline int reduce_chunks(int max_atoms) { return max_atoms > 0 ? (max_atoms + kReduceChunk - 1) / kReduceChunk : 1; }
cudaError_t launch_reduce(int n_structs, int n_pop, const int* offsets, int max_atoms, const float* per_atom,
                          size_t per_atom_stride, int atom_stride, int C, double* partial, double* out,
                          size_t out_pop_stride, cudaStream_t st);

// Gathers per-atom contributions back to input order: out[g][c] = pa[c][orig_sorted[g]].
cudaError_t launch_gather_per_atom(int n_atoms, const int* orig_sorted, const float* per_atom,
                                   int atom_stride, int C, float* out, cudaStream_t st);

// Converts warp-tiled sorted-index lists to row-major input-order lists.
cudaError_t launch_export_neighbors(int n_atoms, const int* sorted_orig, const int* orig_sorted,
                                    const int* nbr_R, const int* cnt_R, int cap_R, const int* seg_R, int two_ended,
                                    const int* nbr_A, const int* cnt_A, int cap_A,
                                    int* out_cnt_R, int* out_cnt_A, int* out_R, int out_cap_R,
                                    int* out_A, int out_cap_A, cudaStream_t st);

// RMSE per individual: rmse[p] = sqrt(mean_{s,c} (pred[p][s][c] - target[s][c])^2).
cudaError_t launch_rmse(int n_pop, int n_structs, int C, const double* pred, const double* target,
                        double* rmse, cudaStream_t st);

// Batched float64 complex FFT (fft.cu): twiddles tw[N/2] for length N (a
// power of two); launch_fft transforms `batch` arrays of length N held in *a
// (forward: exp(-i ...), inverse: exp(+i ...), no 1/N), using *b as the other
// buffer, and swaps the pointers so that *a holds the result.
cudaError_t launch_fft_twiddles(int N, double2* tw, cudaStream_t st);
cudaError_t launch_fft(double2** a, double2** b, const double2* tw, int N, int batch, int inverse, cudaStream_t st);

// Spectrum tail.
cudaError_t launch_spectrum(const double* series, int T, int C, double dt_fs, int kind, int M,
                            int subtract_mean, double* work /* >= T*9 + 2*(M+1) + 2*M doubles */,
                            double* freq, double* spec, double* acf_out, cudaStream_t st);
// The same through the Fourier transform for long series: N >= T + M a power
// of two; work >= T*9 + 2*(M+1) + 2*M doubles as above, zwork >= (2*9*N + N/2)
// double2.
cudaError_t launch_spectrum_fft(const double* series, int T, int C, double dt_fs, int kind, int M,
                                int subtract_mean, double* work, double2* zwork, int N, double* freq, double* spec,
                                double* acf_out, cudaStream_t st);
// Channels whose correlations a spectrum kind sums (IR 3, Raman iso 1, aniso 9).
inline int spectrum_channels(int kind) { return kind == TNEP_SPECTRUM_IR ? 3 : (kind == TNEP_SPECTRUM_RAMAN_ISO ? 1 : 9); }

// SNES training loop (snes.cu).
constexpr int kMaxSnesPop = 1024;
struct SnesSampleArgs {
  uint64_t seed;
  const long long* generation;  // device counter
  int P, d;
  const double* mu;
  const double* sigma;
  double* s;          // [P][d]
  float* packed;      // [P][words] packed parameters of the fused kernel
  size_t words;
  const int* dst;     // packed word of flat parameter i
};
struct SnesFitnessArgs {
  int P, d;
  const double* mu;
  const double* sigma;
  const double* s;
  const double* rmse;
  double lambda1, lambda2;
  double* loss;
};
struct SnesUpdateArgs {
  int P, d;
  const double* loss;
  const double* s;
  const double* rmse;   // may be null
  double* mu;
  double* sigma;
  double eta_mu, eta_sigma;
  double* history;      // [3] or null
  long long* generation;  // advanced by one, or null
};
cudaError_t launch_snes_normals(uint64_t seed, long long generation, int P, int d, double* s, cudaStream_t st);
cudaError_t launch_snes_sample(const SnesSampleArgs& a, cudaStream_t st);
cudaError_t launch_snes_fitness(const SnesFitnessArgs& a, cudaStream_t st);
cudaError_t launch_snes_update(const SnesUpdateArgs& a, cudaStream_t st);

}  // namespace tnep
