// Device steps of the SNES training loop (Sec. II.D: the parameters are
// trained with the separable natural evolution strategy on the RMSE of the
// tensor plus L1 / L2 regularization).
//
//   k_snes_sample   standard normals s_k (Philox4x64-10 + Box-Muller),
//                   z_k = mu + sigma * s_k, z_k rounded to float32 and
//                   scattered into the packed parameter layout of the fused
//                   kernel
//   k_snes_fitness  L_k = RMSE_k + lambda1 mean|z_k| + lambda2 sqrt(mean z_k^2)
//   k_snes_update   ranks, utilities, natural-gradient update of mu and sigma
//
// Every sum has a fixed order, so a run is bitwise reproducible.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tnep_internal.cuh"

namespace tnep {

namespace {

constexpr int kSnesThreads = 256;

// Philox4x64-10 (Salmon, Moraes, Dror and Shaw 2011): multipliers and Weyl
// key increments of the published definition.
constexpr uint64_t kPhM0 = 0xD2E7470EE14C6C93ull, kPhM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhW0 = 0x9E3779B97F4A7C15ull, kPhW1 = 0xBB67AE8584CAA73Bull;

__device__ __forceinline__ void philox(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(kPhM0, c[0]), lo0 = kPhM0 * c[0];
    const uint64_t hi1 = __umul64hi(kPhM1, c[2]), lo1 = kPhM1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += kPhW0;
    k1 += kPhW1;
  }
}

// u in (0, 1) from the top 52 bits.
__device__ __forceinline__ double unit_open(uint64_t x) {
  return ((double)(x >> 12) + 0.5) * 0x1p-52;
}

// The four normals of block b of individual k at generation g.
__device__ __forceinline__ void normals4(uint64_t seed, long long g, int k, int b, double n[4]) {
  uint64_t c[4] = {(uint64_t)b, (uint64_t)k, (uint64_t)g, 0ull};
  philox(c, seed, 0ull);
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const double rad = sqrt(-2.0 * log(unit_open(c[2 * p])));
    double sn, cs;
    sincospi(2.0 * unit_open(c[2 * p + 1]), &sn, &cs);
    n[2 * p] = rad * cs;
    n[2 * p + 1] = rad * sn;
  }
}

__global__ void k_snes_normals(uint64_t seed, long long g, int P, int d, double* __restrict__ s) {
  const int nb = (d + 3) >> 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)P * nb) return;
  const int k = (int)(t / nb), b = (int)(t % nb);
  double n[4];
  normals4(seed, g, k, b, n);
  double* row = s + (size_t)k * d;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (4 * b + q < d) row[4 * b + q] = n[q];
}

__global__ void k_snes_sample(SnesSampleArgs a) {
  const int nb = (a.d + 3) >> 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)a.P * nb) return;
  const int k = (int)(t / nb), b = (int)(t % nb);
  double n[4];
  normals4(a.seed, *a.generation, k, b, n);
  double* row = a.s + (size_t)k * a.d;
  float* packed = a.packed + (size_t)k * a.words;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 4 * b + q;
    if (i < a.d) {
      row[i] = n[q];
      packed[a.dst[i]] = (float)(a.mu[i] + a.sigma[i] * n[q]);
    }
  }
}

// One CTA per individual: fixed-order tree over a strided partition.
__global__ void __launch_bounds__(kSnesThreads) k_snes_fitness(SnesFitnessArgs a) {
  const int k = blockIdx.x;
  const double* row = a.s + (size_t)k * a.d;
  double l1 = 0.0, l2 = 0.0;
  for (int i = threadIdx.x; i < a.d; i += kSnesThreads) {
    const double z = a.mu[i] + a.sigma[i] * row[i];
    l1 += fabs(z);
    l2 += z * z;
  }
  __shared__ double r1[kSnesThreads], r2[kSnesThreads];
  r1[threadIdx.x] = l1;
  r2[threadIdx.x] = l2;
  __syncthreads();
  for (int w = kSnesThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      r1[threadIdx.x] += r1[threadIdx.x + w];
      r2[threadIdx.x] += r2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    a.loss[k] = a.rmse[k] + a.lambda1 * (r1[0] / a.d) + a.lambda2 * sqrt(r2[0] / a.d);
}

// Ascending loss, NaN last, ties by index.
__device__ __forceinline__ bool before(double a, int i, double b, int j) {
  const bool na = isnan(a), nb = isnan(b);
  if (na != nb) return nb;
  if (!na && a != b) return a < b;
  return i < j;
}

// Every CTA ranks the P losses itself (P <= 1024), then updates its slice of
// the parameters; CTA 0 also writes the generation summary and advances the
// generation counter (read only by the next generation's sampling launch).
__global__ void __launch_bounds__(kSnesThreads) k_snes_update(SnesUpdateArgs a) {
  __shared__ double util[kMaxSnesPop];
  __shared__ double w[kMaxSnesPop];
  __shared__ double wsum;
  const int P = a.P;
  const double lhalf = log(P / 2.0 + 1.0);
  for (int r = threadIdx.x; r < P; r += kSnesThreads) w[r] = fmax(0.0, lhalf - log((double)(r + 1)));
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int r = 0; r < P; ++r) acc += w[r];
    wsum = acc;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < P; k += kSnesThreads) {
    const double lk = a.loss[k];
    int rank = 0;
    for (int j = 0; j < P; ++j) rank += before(a.loss[j], j, lk, k) ? 1 : 0;
    util[k] = w[rank] / wsum - 1.0 / P;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.history) {
    int best = 0;
    double mean = 0.0;
    for (int k = 0; k < P; ++k) {
      if (before(a.loss[k], k, a.loss[best], best)) best = k;
      mean += a.loss[k];
    }
    a.history[0] = a.loss[best];
    a.history[1] = a.rmse ? a.rmse[best] : 0.0;
    a.history[2] = mean / P;
  }
  const int i = blockIdx.x * kSnesThreads + threadIdx.x;
  if (i < a.d) {
    double gm = 0.0, gs = 0.0;
    for (int k = 0; k < P; ++k) {
      const double sk = a.s[(size_t)k * a.d + i];
      gm += util[k] * sk;
      gs += util[k] * (sk * sk - 1.0);
    }
    const double sg = a.sigma[i];
    a.mu[i] = a.mu[i] + a.eta_mu * sg * gm;
    a.sigma[i] = sg * exp(0.5 * a.eta_sigma * gs);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.generation) *a.generation += 1;
}

}  // namespace

cudaError_t launch_snes_normals(uint64_t seed, long long generation, int P, int d, double* s, cudaStream_t st) {
  const long long n = (long long)P * ((d + 3) / 4);
  k_snes_normals<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(seed, generation, P, d, s);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_snes_sample(const SnesSampleArgs& a, cudaStream_t st) {
  const long long n = (long long)a.P * ((a.d + 3) / 4);
  k_snes_sample<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_snes_fitness(const SnesFitnessArgs& a, cudaStream_t st) {
  k_snes_fitness<<<a.P, kSnesThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_snes_update(const SnesUpdateArgs& a, cudaStream_t st) {
  k_snes_update<<<(a.d + kSnesThreads - 1) / kSnesThreads, kSnesThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tnep
