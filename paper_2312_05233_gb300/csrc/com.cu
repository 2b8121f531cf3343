// Dipole of charged molecules about the origin (Sec. III.A): a TNEP dipole
// model trained on relative dipoles mu_r (about the centre of mass) gives
// the dipole of a molecule with net charge Q as mu = mu_r + Q r_COM.
//
// One CTA per structure: float64 sums of m_i r_i and m_i over the atoms in a
// fixed order (strided partial sums, then a tree), then mu += Q r_COM.

#include <cuda_runtime.h>

#include "engine.h"

namespace tnep {

namespace {

constexpr int kComThreads = 256;

__global__ void __launch_bounds__(kComThreads) k_com_dipole(const int* __restrict__ offsets,
                                                            const float* __restrict__ pos,
                                                            const int* __restrict__ types,
                                                            const double* __restrict__ masses,
                                                            const double* __restrict__ charge, double* mu,
                                                            int stride) {
  __shared__ double red[4][kComThreads];
  const int s = blockIdx.x;
  const double q = charge[s];
  if (q == 0.0) return;
  const int a0 = offsets[s], a1 = offsets[s + 1];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int a = a0 + threadIdx.x; a < a1; a += kComThreads) {
    const double m = masses[types[a]];
    acc[0] += m * (double)pos[3 * (size_t)a];
    acc[1] += m * (double)pos[3 * (size_t)a + 1];
    acc[2] += m * (double)pos[3 * (size_t)a + 2];
    acc[3] += m;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = kComThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3 && red[3][0] > 0.0) mu[(size_t)s * stride + threadIdx.x] += q * (red[threadIdx.x][0] / red[3][0]);
}

}  // namespace

}  // namespace tnep

using namespace tnep;

extern "C" {

tnep_status tnep_set_masses(tnep_ctx* c, const double* masses) {
  if (!c || !masses) return fail(TNEP_ERR_INVALID, "NULL argument");
  for (int t = 0; t < c->n_types; ++t)
    if (!(masses[t] > 0.0) || !std::isfinite(masses[t])) return fail(TNEP_ERR_INVALID, "masses must be > 0 and finite");
  c->masses.assign(masses, masses + c->n_types);
  return TNEP_OK;
}

tnep_status tnep_add_com_dipole(tnep_ctx* c, int n_structs, const int* atom_offsets, const float* pos,
                                const float* box, const int* types, const double* charge, double* mu, int mu_stride,
                                void* stream) {
  if (!c || !atom_offsets || !charge || !mu) return fail(TNEP_ERR_INVALID, "NULL argument");
  if (n_structs < 1 || mu_stride < 3) return fail(TNEP_ERR_INVALID, "need n_structs >= 1 and mu_stride >= 3");
  if ((int)c->masses.size() != c->n_types) return fail(TNEP_ERR_INVALID, "set the type masses first (tnep_set_masses)");
  if (is_device_ptr(atom_offsets)) return fail(TNEP_ERR_INVALID, "atom_offsets must be host memory");
  if (atom_offsets[0] != 0) return fail(TNEP_ERR_INVALID, "atom_offsets[0] must be 0");
  for (int s = 0; s < n_structs; ++s)
    if (atom_offsets[s + 1] < atom_offsets[s]) return fail(TNEP_ERR_INVALID, "atom_offsets must not decrease");
  const int N = atom_offsets[n_structs];
  if (N > 0 && (!pos || !types)) return fail(TNEP_ERR_INVALID, "NULL buffer");
  // a net charge needs an open structure (the centre of mass of a periodic one is not defined)
  const bool host_q = !is_device_ptr(charge), host_box = box && !is_device_ptr(box);
  if (host_q && box && host_box)
    for (int s = 0; s < n_structs; ++s)
      if (charge[s] != 0.0 && (box[3 * s] > 0.f || box[3 * s + 1] > 0.f || box[3 * s + 2] > 0.f))
        return fail(TNEP_ERR_INVALID, "a charged structure must be open (box 0 0 0)");
  if (!is_device_ptr(types))
    for (int a = 0; a < N; ++a)
      if (types[a] < 0 || types[a] >= c->n_types) return fail(TNEP_ERR_INVALID, "type index out of range");
  TNEP_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = stream ? reinterpret_cast<cudaStream_t>(stream) : c->stream;
  const size_t nmu = (size_t)(n_structs - 1) * mu_stride + 3;
  // one scratch block: offsets, masses, charges, mu, positions, types
  const size_t bytes = sizeof(int) * (n_structs + 1) + sizeof(double) * (c->n_types + n_structs + nmu) +
                       sizeof(float) * 3 * (size_t)N + sizeof(int) * (size_t)N + 64;
  char* d = nullptr;
  TNEP_CUDA(dev_malloc_async((void**)&d, bytes, st));
  double* d_mass = reinterpret_cast<double*>(d);
  double* d_q = d_mass + c->n_types;
  double* d_mu = d_q + n_structs;
  float* d_pos = reinterpret_cast<float*>(d_mu + nmu);
  int* d_types = reinterpret_cast<int*>(d_pos + 3 * (size_t)N);
  int* d_off = d_types + N;
  cudaError_t e = cudaMemcpyAsync(d_mass, c->masses.data(), sizeof(double) * c->n_types, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_q, charge, sizeof(double) * n_structs, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_mu, mu, sizeof(double) * nmu, cudaMemcpyDefault, st);
  if (e == cudaSuccess && N > 0) e = cudaMemcpyAsync(d_pos, pos, sizeof(float) * 3 * N, cudaMemcpyDefault, st);
  if (e == cudaSuccess && N > 0) e = cudaMemcpyAsync(d_types, types, sizeof(int) * N, cudaMemcpyDefault, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_off, atom_offsets, sizeof(int) * (n_structs + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_com_dipole<<<n_structs, kComThreads, 0, st>>>(d_off, d_pos, d_types, d_mass, d_q, d_mu, mu_stride);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(mu, d_mu, sizeof(double) * nmu, cudaMemcpyDefault, st);
  tnep_status rc = e == cudaSuccess ? TNEP_OK : cuda_fail(e, "centre-of-mass dipole");
  cudaFreeAsync(d, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess && rc == TNEP_OK) rc = cuda_fail(e, "centre-of-mass dipole sync");
  return rc;
}

}  // extern "C"
