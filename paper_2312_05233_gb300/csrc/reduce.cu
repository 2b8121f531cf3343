// Per-structure reductions and population scoring after the fused kernel:
// the deterministic FP64 sums of the per-atom contributions of Eqs. 3-4
// into one tensor per structure, the per-atom export in input order, and the
// RMSE of each individual's predictions against the target tensors (the
// loss of Sec. II.D before regularization).

#include "tnep_internal.cuh"

namespace tnep {

namespace {

// Per-structure FP64 sums in two deterministic stages: CTA (s, chunk) sums a
// fixed 2048-atom chunk of structure s (strided per-thread sums, a shuffle
// tree in each warp, then the eight warp sums in order), then one warp per
// structure adds its chunk partials (strided per-lane sums, shuffle tree).
// Chunks are aligned to the structure start, so a structure's result does
// not depend on what else is in the batch.
__global__ void __launch_bounds__(256) k_reduce_partial(const int* offsets, int n_chunks, const float* per_atom,
                                                        size_t pa_pop_stride, int atom_stride, int C,
                                                        double* partial) {
  const int s = blockIdx.x / n_chunks, chunk = blockIdx.x % n_chunks, p = blockIdx.y;
  const int S = gridDim.x / n_chunks;
  const int a0 = offsets[s] + chunk * kReduceChunk;
  const int a1 = min(offsets[s + 1], a0 + kReduceChunk);
  const float* pa = per_atom + (size_t)p * pa_pop_stride;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double acc[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) acc[c] = 0.0;
  for (int g = a0 + threadIdx.x; g < a1; g += blockDim.x) {
#pragma unroll
    for (int c = 0; c < 9; ++c)
      if (c < C) acc[c] += (double)pa[(size_t)c * atom_stride + g];
  }
  __shared__ double red[9][8];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    if (c < C) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o);
      if (lane == 0) red[c][w] = acc[c];
    }
  }
  __syncthreads();
  if (threadIdx.x < C) {
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) v += red[threadIdx.x][k];
    partial[(((size_t)p * S + s) * n_chunks + chunk) * C + threadIdx.x] = v;
  }
}

// One warp per (individual, structure).
__global__ void k_reduce_final(int S, int n_chunks, int C, int n_pop, const double* partial, double* out,
                               size_t out_pop_stride) {
  const int wid = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (wid >= S * n_pop) return;  // whole warps
  const int p = wid / S, s = wid % S;
  const double* src = partial + ((size_t)p * S + s) * n_chunks * C;
  double v[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) v[c] = 0.0;
  for (int k = lane; k < n_chunks; k += 32) {
#pragma unroll
    for (int c = 0; c < 9; ++c)
      if (c < C) v[c] += src[(size_t)k * C + c];
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    if (c < C) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
      if (lane == 0) out[(size_t)p * out_pop_stride + (size_t)s * C + c] = v[c];
    }
  }
}

__global__ void k_gather(int n, const int* orig_sorted, const float* pa, int atom_stride, int C, float* out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const int i = orig_sorted[g];
  for (int c = 0; c < C; ++c) out[(size_t)g * C + c] = pa[(size_t)c * atom_stride + i];
}

__global__ void k_rmse(int S, int C, const double* pred, const double* target, double* rmse) {
  const int p = blockIdx.x;
  const double* pp = pred + (size_t)p * S * C;
  double acc = 0.0;
  for (int k = threadIdx.x; k < S * C; k += blockDim.x) {
    const double d = pp[k] - target[k];
    acc += d * d;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) rmse[p] = S * C > 0 ? sqrt(red[0] / (double)(S * C)) : 0.0;
}

}  // namespace

cudaError_t launch_reduce(int n_structs, int n_pop, const int* offsets, int max_atoms, const float* per_atom,
                          size_t per_atom_stride, int atom_stride, int C, double* partial, double* out,
                          size_t out_pop_stride, cudaStream_t st) {
  if (n_structs <= 0 || n_pop <= 0) return cudaSuccess;
  count_launches(2);
  const int n_chunks = reduce_chunks(max_atoms);
  k_reduce_partial<<<dim3(n_structs * n_chunks, n_pop), 256, 0, st>>>(offsets, n_chunks, per_atom, per_atom_stride,
                                                                     atom_stride, C, partial);
  const long long nt = 32LL * n_structs * n_pop;
  k_reduce_final<<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(n_structs, n_chunks, C, n_pop, partial, out,
                                                                out_pop_stride);
  return cudaGetLastError();
}

cudaError_t launch_gather_per_atom(int n_atoms, const int* orig_sorted, const float* per_atom,
                                   int atom_stride, int C, float* out, cudaStream_t st) {
  if (n_atoms <= 0) return cudaSuccess;
  count_launches(1);
  k_gather<<<(n_atoms + 255) / 256, 256, 0, st>>>(n_atoms, orig_sorted, per_atom, atom_stride, C, out);
  return cudaGetLastError();
}

cudaError_t launch_rmse(int n_pop, int n_structs, int C, const double* pred, const double* target,
                        double* rmse, cudaStream_t st) {
  if (n_pop <= 0) return cudaSuccess;
  count_launches(1);
  k_rmse<<<n_pop, 256, 0, st>>>(n_structs, C, pred, target, rmse);
  return cudaGetLastError();
}

}  // namespace tnep
