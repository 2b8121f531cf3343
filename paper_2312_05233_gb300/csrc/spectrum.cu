// Spectrum tail in float64 (Sec. II.F, Eqs. 5-6; Sec. II.G, Eqs. 7-9).
//
//   prep   signal x(t): IR mu (3 comps); Raman iso gamma = Tr(alpha)/3;
//          Raman aniso beta = alpha - gamma I (9 comps); mean removed if asked
//   acf    one CTA per lag tau: C(tau) = 1/(T - tau) sum_t x(t).x'(t + tau),
//          with x' = x (IR: times 1/3) or x'_{ab} = x_{ba} (Tr[beta beta])
//   cos    one CTA per frequency k:
//          S_k = dt [C(0) + 2 sum_{tau=1}^{M} C(tau) cos(pi k tau / M)]
//          (IR times (2 pi nu_k)^2), nu_k = k / (2 M dt)
// Every sum runs in a fixed order (strided partial sums, then a tree), so the
// results do not depend on the launch.
// Long series (channels x T x M above 1e9) take the Fourier route for the
// autocorrelation: the prepared channels, zero-padded to N >= T + M (a power
// of two), are transformed (fft.cu), the real product spectrum
//   IR: sum_c |X_c|^2 / 3,  iso: |X|^2,  aniso: sum_ab Re(conj(B_ab) B_ba)
// is transformed back, and C(tau) = IDFT(...)(tau) / (N (T - tau)).

#include <utility>

#include "tnep_internal.cuh"

namespace tnep {

namespace {

constexpr double kCmPerInvFs = 1.0 / 2.99792458e-5;

__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// One CTA: x [T][cx] from the series.
__global__ void __launch_bounds__(256) k_prep(const double* series, int T, int C, int kind, int subtract_mean,
                                              double* x) {
  __shared__ double red[256];
  const int cx = kind == TNEP_SPECTRUM_IR ? 3 : (kind == TNEP_SPECTRUM_RAMAN_ISO ? 1 : 9);
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    const double* s = series + (size_t)t * C;
    double* o = x + (size_t)t * cx;
    if (kind == TNEP_SPECTRUM_IR) {
      o[0] = s[0]; o[1] = s[1]; o[2] = s[2];
    } else {
      const double g = (s[0] + s[4] + s[8]) / 3.0;
      if (kind == TNEP_SPECTRUM_RAMAN_ISO) {
        o[0] = g;
      } else {
        for (int k = 0; k < 9; ++k) o[k] = s[k] - ((k == 0 || k == 4 || k == 8) ? g : 0.0);
      }
    }
  }
  __syncthreads();
  if (!subtract_mean) return;
  for (int c = 0; c < cx; ++c) {
    double acc = 0.0;
    for (int t = threadIdx.x; t < T; t += blockDim.x) acc += x[(size_t)t * cx + c];
    const double mean = block_sum(acc, red) / (double)T;
    for (int t = threadIdx.x; t < T; t += blockDim.x) x[(size_t)t * cx + c] -= mean;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_acf(const double* x, int T, int kind, double* acf) {
  __shared__ double red[256];
  const int tau = blockIdx.x;
  const int n = T - tau;
  double acc = 0.0;
  if (kind == TNEP_SPECTRUM_IR) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const double* a = x + (size_t)t * 3;
      const double* b = x + (size_t)(t + tau) * 3;
      acc += a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    }
  } else if (kind == TNEP_SPECTRUM_RAMAN_ISO) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) acc += x[t] * x[t + tau];
  } else {
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const double* a = x + (size_t)t * 9;
      const double* b = x + (size_t)(t + tau) * 9;
      for (int u = 0; u < 3; ++u)
        for (int v = 0; v < 3; ++v) acc += a[3 * u + v] * b[3 * v + u];
    }
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) acf[tau] = s / (double)n / (kind == TNEP_SPECTRUM_IR ? 3.0 : 1.0);
}

__global__ void k_costab(int M, double* tab) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < 2 * M) tab[m] = cospi((double)m / (double)M);
}

__global__ void __launch_bounds__(256) k_costransform(const double* acf, const double* tab, int M, double dt,
                                                      int kind, double* freq, double* spec) {
  __shared__ double red[256];
  const int k = blockIdx.x;
  double acc = 0.0;
  for (int tau = 1 + threadIdx.x; tau <= M; tau += blockDim.x)
    acc += acf[tau] * tab[(long long)k * tau % (2LL * M)];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) {
    const double nu = (double)k / (2.0 * M * dt);
    double S = dt * (acf[0] + 2.0 * s);
    if (kind == TNEP_SPECTRUM_IR) {
      const double w = 2.0 * 3.14159265358979323846 * nu;
      S *= w * w;
    }
    freq[k] = nu * kCmPerInvFs;
    spec[k] = S;
  }
}

// Channel c of the prepared signal x [T][cx], zero-padded to N, as complex.
__global__ void k_spec_load(const double* __restrict__ x, int T, int cx, int N, double2* __restrict__ z) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)cx * N) return;
  const int c = (int)(g / N), t = (int)(g % N);
  z[g] = make_double2(t < T ? x[(size_t)t * cx + c] : 0.0, 0.0);
}

__global__ void k_spec_product(const double2* __restrict__ X, int N, int kind, double2* __restrict__ z) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= N) return;
  double v = 0.0;
  if (kind == TNEP_SPECTRUM_IR) {
    for (int c = 0; c < 3; ++c) {
      const double2 a = X[(size_t)c * N + f];
      v += a.x * a.x + a.y * a.y;
    }
    v /= 3.0;
  } else if (kind == TNEP_SPECTRUM_RAMAN_ISO) {
    const double2 a = X[f];
    v = a.x * a.x + a.y * a.y;
  } else {
    for (int u = 0; u < 3; ++u)
      for (int w = 0; w < 3; ++w) {
        const double2 a = X[(size_t)(3 * u + w) * N + f], b = X[(size_t)(3 * w + u) * N + f];
        v += a.x * b.x + a.y * b.y;
      }
  }
  z[f] = make_double2(v, 0.0);
}

__global__ void k_spec_acf(const double2* __restrict__ z, int N, int T, int M, double* __restrict__ acf) {
  const int tau = blockIdx.x * blockDim.x + threadIdx.x;
  if (tau > M) return;
  acf[tau] = z[tau].x / (double)N / (double)(T - tau);
}

}  // namespace

cudaError_t launch_spectrum(const double* series, int T, int C, double dt_fs, int kind, int M,
                            int subtract_mean, double* work, double* freq, double* spec, double* acf_out,
                            cudaStream_t st) {
  double* x = work;                           // [T][9]
  double* acf = work + (size_t)T * 9;         // [M+1]
  double* tab = acf + (M + 1);                // [2M]
  count_launches(4);
  k_prep<<<1, 256, 0, st>>>(series, T, C, kind, subtract_mean, x);
  k_acf<<<M + 1, 256, 0, st>>>(x, T, kind, acf);
  k_costab<<<(2 * M + 255) / 256, 256, 0, st>>>(M, tab);
  k_costransform<<<M + 1, 256, 0, st>>>(acf, tab, M, dt_fs, kind, freq, spec);
  if (acf_out) {
    cudaError_t e = cudaMemcpyAsync(acf_out, acf, sizeof(double) * (M + 1), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_spectrum_fft(const double* series, int T, int C, double dt_fs, int kind, int M,
                                int subtract_mean, double* work, double2* zwork, int N, double* freq, double* spec,
                                double* acf_out, cudaStream_t st) {
  const int cx = spectrum_channels(kind);
  double* x = work;                           // [T][9]
  double* acf = work + (size_t)T * 9;         // [M+1]
  double* tab = acf + (M + 1);                // [2M]
  double2* za = zwork;
  double2* zb = za + (size_t)9 * N;
  double2* tw = zb + (size_t)9 * N;
  k_prep<<<1, 256, 0, st>>>(series, T, C, kind, subtract_mean, x);
  cudaError_t e = launch_fft_twiddles(N, tw, st);
  if (e != cudaSuccess) return e;
  k_spec_load<<<(unsigned)(((long long)cx * N + 255) / 256), 256, 0, st>>>(x, T, cx, N, za);
  e = launch_fft(&za, &zb, tw, N, cx, 0, st);
  if (e != cudaSuccess) return e;
  k_spec_product<<<(N + 255) / 256, 256, 0, st>>>(za, N, kind, zb);
  std::swap(za, zb);
  e = launch_fft(&za, &zb, tw, N, 1, 1, st);
  if (e != cudaSuccess) return e;
  k_spec_acf<<<(M + 1 + 255) / 256, 256, 0, st>>>(za, N, T, M, acf);
  k_costab<<<(2 * M + 255) / 256, 256, 0, st>>>(M, tab);
  k_costransform<<<M + 1, 256, 0, st>>>(acf, tab, M, dt_fs, kind, freq, spec);
  count_launches(6);
  if (acf_out) {
    e = cudaMemcpyAsync(acf_out, acf, sizeof(double) * (M + 1), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace tnep
