// Polarized Raman tail in float64 (Sec. II.G, Eqs. 7-8).
//
//   mean   per component of alpha(t) (or chi(t)), one CTA per component
//   prep   x [9][T] channel-major, mean removed if asked
//   corr   C_pq(tau) = sum_t x_p(t) x_q(t + tau), all 81 ordered pairs; one
//          thread owns one pair and four consecutive lags and walks t in order
//          (direct sums, used while 81 T M is small), or for long series
//   fft    the symmetrised sums S_pq(tau) through the Fourier transform: the
//          nine channels, zero-padded to N >= T + M (a power of two, so the
//          circular correlation equals the linear one for tau <= M), are
//          transformed (radix-2 Stockham, float64), the real cross spectra
//          Re(conj(X_p) X_q) of the 45 pairs p <= q are transformed back two
//          per complex transform, and S_pq(tau) = (1/N) IDFT[...](tau)
//   cos    L_pq(nu_k) = dt [S_pq(0) + 2 sum_tau S_pq(tau) cos(pi k tau / M)],
//          S_pq = (C_pq + C_qp) / (2 (T - tau)); one CTA per frequency, one
//          warp per group of pairs
//   polar  spec_o(nu_k) = sum_pq w_p w_q L_pq(nu_k), w = vec(n_o eps_o^T) (Eq. 7)
//   porto  the same for Z(XX)Z-bar / Z(XY)Z-bar of a crystal turned by theta
// Every sum runs in a fixed order, so results do not depend on the launch.

#include <cuda_runtime.h>

#include <utility>

#include "engine.h"

namespace tnep {

namespace {

constexpr double kCmPerInvFs = 1.0 / 2.99792458e-5;
constexpr int kLagsPerThread = 4;
// 81 T (M + 1) above which the correlations go through the Fourier transform
constexpr double kFftAbove = 1.0e9;
constexpr int kCorrThreads = 128;

__global__ void __launch_bounds__(1024) k_rmean(const double* __restrict__ s, int T, int subtract_mean,
                                                double* __restrict__ mean) {
  __shared__ double red[1024];
  const int c = blockIdx.x;
  double acc = 0.0;
  if (subtract_mean)
    for (int t = threadIdx.x; t < T; t += blockDim.x) acc += s[(size_t)t * 9 + c];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) mean[c] = red[0] / (double)T;
}

__global__ void k_rprep(const double* __restrict__ s, int T, const double* __restrict__ mean,
                        double* __restrict__ x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9LL * T) return;
  const int t = (int)(i / 9), c = (int)(i % 9);
  x[(size_t)c * T + t] = s[i] - mean[c];
}

// grid (lag tiles, 81 pairs); thread: lags tau0..tau0+3 of pair (p, q).
__global__ void __launch_bounds__(kCorrThreads) k_rcorr(const double* __restrict__ x, int T, int M,
                                                        double* __restrict__ C) {
  const int pair = blockIdx.y;
  const int p = pair / 9, q = pair % 9;
  const int tau0 = (blockIdx.x * kCorrThreads + threadIdx.x) * kLagsPerThread;
  if (tau0 > M) return;
  const double* xp = x + (size_t)p * T;
  const double* xq = x + (size_t)q * T;
  double acc[kLagsPerThread] = {0.0, 0.0, 0.0, 0.0};
  double win[kLagsPerThread];
#pragma unroll
  for (int j = 0; j < kLagsPerThread; ++j) win[j] = (tau0 + j < T) ? xq[tau0 + j] : 0.0;
  // x_q(t + tau0 + j) slides along t; terms with t + tau >= T are left out
  const int n = T - tau0;
  for (int t = 0; t < n; ++t) {
    const double a = xp[t];
#pragma unroll
    for (int j = 0; j < kLagsPerThread; ++j)
      if (t + j < n) acc[j] = fma(a, win[j], acc[j]);
#pragma unroll
    for (int j = 0; j < kLagsPerThread - 1; ++j) win[j] = win[j + 1];
    const int nxt = t + tau0 + kLagsPerThread;
    win[kLagsPerThread - 1] = nxt < T ? xq[nxt] : 0.0;
  }
#pragma unroll
  for (int j = 0; j < kLagsPerThread; ++j)
    if (tau0 + j <= M) C[((size_t)(tau0 + j)) * 81 + pair] = acc[j];
}

// ---- Fourier route (float64 complex as double2) ----

// Channel c of the mean-removed series, zero-padded to N, as complex.
__global__ void k_fft_load(const double* __restrict__ x, int T, int N, double2* __restrict__ z) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 9LL * N) return;
  const int c = (int)(g / N), t = (int)(g % N);
  z[g] = make_double2(t < T ? x[(size_t)c * T + t] : 0.0, 0.0);
}

// Cross spectra of the 45 pairs p <= q, two per complex array:
// z_w[f] = Re(conj(X_p) X_q)[f] + i Re(conj(X_p') X_q')[f].
__global__ void k_fft_cross(const double2* __restrict__ X, int N, double2* __restrict__ z) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 23LL * N) return;
  const int w = (int)(g / N), f = (int)(g % N);
  double re[2] = {0.0, 0.0};
  for (int h = 0; h < 2; ++h) {
    const int u = 2 * w + h;
    if (u >= 45) break;
    int p = 0, rem = u;
    while (rem >= 9 - p) { rem -= 9 - p; ++p; }
    const int q = p + rem;
    const double2 xp = X[(size_t)p * N + f], xq = X[(size_t)q * N + f];
    re[h] = xp.x * xq.x + xp.y * xq.y;
  }
  z[g] = make_double2(re[0], re[1]);
}

// C[tau][81] (both p q and q p) = S_pq(tau): the inverse transform carries
// no 1/N, so divide by N here.
__global__ void k_fft_store(const double2* __restrict__ z, int N, int M, double* __restrict__ C) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 45LL * (M + 1)) return;
  const int u = (int)(g / (M + 1)), tau = (int)(g % (M + 1));
  int p = 0, rem = u;
  while (rem >= 9 - p) { rem -= 9 - p; ++p; }
  const int q = p + rem;
  const double2 v = z[(size_t)(u >> 1) * N + tau];
  const double sv = ((u & 1) ? v.y : v.x) / (double)N;
  C[(size_t)tau * 81 + p * 9 + q] = sv;
  C[(size_t)tau * 81 + q * 9 + p] = sv;
}

__global__ void k_rcostab(int M, double* tab) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < 2 * M) tab[m] = cospi((double)m / (double)M);
}

// One CTA (8 warps) per frequency k; warp w handles the unique pairs
// u = w, w + 8, ... of the 45 (p <= q).
__global__ void __launch_bounds__(256) k_rcos(const double* __restrict__ C, const double* __restrict__ tab, int T,
                                              int M, double dt, double* __restrict__ freq, double* __restrict__ L) {
  const int k = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int u = warp; u < 45; u += 8) {
    int p = 0, rem = u;
    while (rem >= 9 - p) { rem -= 9 - p; ++p; }
    const int q = p + rem;
    double acc = 0.0;
    for (int tau = 1 + lane; tau <= M; tau += 32) {
      const double* c = C + (size_t)tau * 81;
      const double s = 0.5 * (c[p * 9 + q] + c[q * 9 + p]) / (double)(T - tau);
      acc = fma(s, tab[(long long)k * tau % (2LL * M)], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const double s0 = 0.5 * (C[p * 9 + q] + C[q * 9 + p]) / (double)T;
      const double v = dt * (s0 + 2.0 * acc);
      L[(size_t)k * 81 + p * 9 + q] = v;
      L[(size_t)k * 81 + q * 9 + p] = v;
    }
  }
  if (threadIdx.x == 0) freq[k] = (double)k / (2.0 * M * dt) * kCmPerInvFs;
}

__device__ __forceinline__ double contract(const double* __restrict__ Lk, const double w[9]) {
  double acc = 0.0;
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    double r = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) r = fma(Lk[p * 9 + q], w[q], r);
    acc = fma(w[p], r, acc);
  }
  return acc;
}

__global__ void k_rpolar(const double* __restrict__ L, int M, int O, const double* __restrict__ n,
                         const double* __restrict__ eps, double* __restrict__ spec) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)O * (M + 1)) return;
  const int o = (int)(i / (M + 1)), k = (int)(i % (M + 1));
  double w[9];
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int d = 0; d < 3; ++d) w[g * 3 + d] = n[o * 3 + g] * eps[o * 3 + d];
  spec[i] = contract(L + (size_t)k * 81, w);
}

// Crystal turned by theta about `axis` (the laser direction): incoming
// polarization R^T X, observed R^T X (parallel) or R^T Y (crossed), with X, Y
// the two crystal axes orthogonal to `axis` in cyclic order.
__global__ void k_rporto(const double* __restrict__ L, int M, int O, const double* __restrict__ theta, int axis,
                         double* __restrict__ par, double* __restrict__ crs) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)O * (M + 1)) return;
  const int o = (int)(i / (M + 1)), k = (int)(i % (M + 1));
  const int a = (axis + 1) % 3, b = (axis + 2) % 3;
  double sn, cs;
  sincos(theta[o], &sn, &cs);
  double e[3] = {0.0, 0.0, 0.0}, y[3] = {0.0, 0.0, 0.0};
  e[a] = cs; e[b] = -sn;
  y[a] = sn; y[b] = cs;
  double wp[9], wc[9];
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      wp[g * 3 + d] = e[g] * e[d];
      wc[g * 3 + d] = y[g] * e[d];
    }
  par[i] = contract(L + (size_t)k * 81, wp);
  crs[i] = contract(L + (size_t)k * 81, wc);
}

unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

bool have_device() {
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return false;
  }
  return true;
}

}  // namespace

}  // namespace tnep

using namespace tnep;

extern "C" {

tnep_status tnep_raman_tensor(const double* series, int T, double dt_fs, int max_lag, int subtract_mean,
                              double* freq_cm1, double* L, void* stream) {
  if (!series || !freq_cm1 || !L) return fail(TNEP_ERR_INVALID, "NULL buffer");
  if (T < 2) return fail(TNEP_ERR_INVALID, "need at least two samples");
  if (!(dt_fs > 0.0)) return fail(TNEP_ERR_INVALID, "dt must be positive");
  const int M = max_lag <= 0 ? T / 2 : max_lag;
  if (M < 1 || M >= T) return fail(TNEP_ERR_INVALID, "max_lag must be in [1, T)");
  if (!have_device()) return fail(TNEP_ERR_NO_DEVICE, "no CUDA device");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t nS = (size_t)T * 9, nX = (size_t)T * 9, nC = (size_t)(M + 1) * 81, nT = 2 * (size_t)M;
  const size_t nF = (size_t)(M + 1), nL = (size_t)(M + 1) * 81;
  // direct time-origin sums while they are cheap, the Fourier route beyond
  const bool use_fft = 81.0 * (double)T * (double)(M + 1) > kFftAbove;
  int N = 2;
  while (N < T + M) N <<= 1;
  const size_t nZ = use_fft ? (size_t)2 * 23 * N + (size_t)N / 2 : 0;  // double2: two work arrays + twiddles
  double* d = nullptr;
  TNEP_CUDA(dev_malloc_async((void**)&d, sizeof(double) * (nS + nX + nC + nT + nF + nL + 16 + 2 * nZ), st));
  // the FFT work area (double2) first, where the allocation's alignment holds
  double2* zwork = reinterpret_cast<double2*>(d);
  double* d_s = d + 2 * nZ;
  double* d_x = d_s + nS;
  double* d_c = d_x + nX;
  double* d_tab = d_c + nC;
  double* d_f = d_tab + nT;
  double* d_l = d_f + nF;
  double* d_mean = d_l + nL;
  cudaError_t e = cudaMemcpyAsync(d_s, series, sizeof(double) * nS, cudaMemcpyDefault, st);
  if (e == cudaSuccess) {
    k_rmean<<<9, 1024, 0, st>>>(d_s, T, subtract_mean, d_mean);
    k_rprep<<<blocks_for(9LL * T, 256), 256, 0, st>>>(d_s, T, d_mean, d_x);
    if (!use_fft) {
      const int tiles = (M + 1 + kCorrThreads * kLagsPerThread - 1) / (kCorrThreads * kLagsPerThread);
      k_rcorr<<<dim3(tiles, 81), kCorrThreads, 0, st>>>(d_x, T, M, d_c);
      count_launches(1);
    } else {
      double2* za = zwork;
      double2* zb = za + (size_t)23 * N;
      double2* tw = zb + (size_t)23 * N;
      launch_fft_twiddles(N, tw, st);
      k_fft_load<<<blocks_for(9LL * N, 256), 256, 0, st>>>(d_x, T, N, za);
      launch_fft(&za, &zb, tw, N, 9, 0, st);
      k_fft_cross<<<blocks_for(23LL * N, 256), 256, 0, st>>>(za, N, zb);
      std::swap(za, zb);
      launch_fft(&za, &zb, tw, N, 23, 1, st);
      k_fft_store<<<blocks_for(45LL * (M + 1), 256), 256, 0, st>>>(za, N, M, d_c);
      count_launches(3);
    }
    k_rcostab<<<blocks_for(2LL * M, 256), 256, 0, st>>>(M, d_tab);
    k_rcos<<<M + 1, 256, 0, st>>>(d_c, d_tab, T, M, dt_fs, d_f, d_l);
    count_launches(4);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(freq_cm1, d_f, sizeof(double) * nF, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L, d_l, sizeof(double) * nL, cudaMemcpyDefault, st);
  tnep_status rc = e == cudaSuccess ? TNEP_OK : cuda_fail(e, "raman tensor");
  cudaFreeAsync(d, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess && rc == TNEP_OK) rc = cuda_fail(e, "raman tensor sync");
  return rc;
}

tnep_status tnep_raman_polarized(const double* L, int max_lag, int n_orient, const double* n, const double* eps,
                                 double* spec, void* stream) {
  if (!L || !n || !eps || !spec) return fail(TNEP_ERR_INVALID, "NULL buffer");
  if (max_lag < 1 || n_orient < 1) return fail(TNEP_ERR_INVALID, "need max_lag >= 1 and n_orient >= 1");
  if (!have_device()) return fail(TNEP_ERR_NO_DEVICE, "no CUDA device");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t nL = (size_t)(max_lag + 1) * 81, nV = (size_t)n_orient * 3, nO = (size_t)n_orient * (max_lag + 1);
  double* d = nullptr;
  TNEP_CUDA(dev_malloc_async((void**)&d, sizeof(double) * (nL + 2 * nV + nO), st));
  double *d_l = d, *d_n = d_l + nL, *d_e = d_n + nV, *d_o = d_e + nV;
  cudaError_t e = cudaMemcpyAsync(d_l, L, sizeof(double) * nL, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_n, n, sizeof(double) * nV, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_e, eps, sizeof(double) * nV, cudaMemcpyDefault, st);
  if (e == cudaSuccess) {
    k_rpolar<<<blocks_for((long long)nO, 256), 256, 0, st>>>(d_l, max_lag, n_orient, d_n, d_e, d_o);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(spec, d_o, sizeof(double) * nO, cudaMemcpyDefault, st);
  tnep_status rc = e == cudaSuccess ? TNEP_OK : cuda_fail(e, "raman polarized");
  cudaFreeAsync(d, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess && rc == TNEP_OK) rc = cuda_fail(e, "raman polarized sync");
  return rc;
}

tnep_status tnep_raman_porto_map(const double* L, int max_lag, int n_theta, const double* theta, int axis,
                                 double* spec_parallel, double* spec_crossed, void* stream) {
  if (!L || !theta || !spec_parallel || !spec_crossed) return fail(TNEP_ERR_INVALID, "NULL buffer");
  if (max_lag < 1 || n_theta < 1) return fail(TNEP_ERR_INVALID, "need max_lag >= 1 and n_theta >= 1");
  if (axis < 0 || axis > 2) return fail(TNEP_ERR_INVALID, "axis must be 0, 1 or 2");
  if (!have_device()) return fail(TNEP_ERR_NO_DEVICE, "no CUDA device");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t nL = (size_t)(max_lag + 1) * 81, nO = (size_t)n_theta * (max_lag + 1);
  double* d = nullptr;
  TNEP_CUDA(dev_malloc_async((void**)&d, sizeof(double) * (nL + n_theta + 2 * nO), st));
  double *d_l = d, *d_t = d_l + nL, *d_p = d_t + n_theta, *d_c = d_p + nO;
  cudaError_t e = cudaMemcpyAsync(d_l, L, sizeof(double) * nL, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_t, theta, sizeof(double) * n_theta, cudaMemcpyDefault, st);
  if (e == cudaSuccess) {
    k_rporto<<<blocks_for((long long)nO, 256), 256, 0, st>>>(d_l, max_lag, n_theta, d_t, axis, d_p, d_c);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(spec_parallel, d_p, sizeof(double) * nO, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(spec_crossed, d_c, sizeof(double) * nO, cudaMemcpyDefault, st);
  tnep_status rc = e == cudaSuccess ? TNEP_OK : cuda_fail(e, "raman porto map");
  cudaFreeAsync(d, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess && rc == TNEP_OK) rc = cuda_fail(e, "raman porto map sync");
  return rc;
}

}  // extern "C"
