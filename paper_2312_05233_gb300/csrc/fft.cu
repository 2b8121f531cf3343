// Batched complex FFT in float64 (radix-2 Stockham, out of place), shared by
// the long-series routes of the spectrum tail and of the polarized Raman
// tensor: correlations of series of length T up to lag M are taken from
// transforms of length N >= T + M (a power of two), where the circular
// correlation of the zero-padded series equals the linear one.
//
// Stage with half-size p (p = 1, 2, 4, ..., N/2), on each transform:
//   b[2j - k] = a[j] + w a[j + N/2],  b[2j - k + p] = a[j] - w a[j + N/2],
//   k = j mod p, w = exp(-+2 pi i k / (2p)) = tw[k N / (2p)],
// which leaves the result in natural order after log2 N stages.

#include <utility>

#include "tnep_internal.cuh"

namespace tnep {

namespace {

__global__ void k_fft_twiddles(int N, double2* __restrict__ tw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N / 2) return;
  double s, c;
  sincospi(-2.0 * (double)k / (double)N, &s, &c);  // exp(-2 pi i k / N)
  tw[k] = make_double2(c, s);
}

__global__ void k_fft_stage(const double2* __restrict__ a, double2* __restrict__ b, const double2* __restrict__ tw,
                            int N, int p, int batch, int inverse) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int half = N >> 1;
  if (g >= (long long)batch * half) return;
  const int f = (int)(g / half), j = (int)(g % half);
  const int k = j & (p - 1);
  double2 w = tw[(size_t)k * (half / p)];
  if (inverse) w.y = -w.y;
  const double2* A = a + (size_t)f * N;
  double2* B = b + (size_t)f * N;
  const double2 u = A[j], v0 = A[j + half];
  const double2 v = make_double2(v0.x * w.x - v0.y * w.y, v0.x * w.y + v0.y * w.x);
  const int o = 2 * j - k;
  B[o] = make_double2(u.x + v.x, u.y + v.y);
  B[o + p] = make_double2(u.x - v.x, u.y - v.y);
}

unsigned fft_blocks(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t launch_fft_twiddles(int N, double2* tw, cudaStream_t st) {
  k_fft_twiddles<<<fft_blocks(N / 2), 256, 0, st>>>(N, tw);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fft(double2** a, double2** b, const double2* tw, int N, int batch, int inverse, cudaStream_t st) {
  int n = 0;
  for (int p = 1; p < N; p <<= 1, ++n) {
    k_fft_stage<<<fft_blocks((long long)batch * (N / 2)), 256, 0, st>>>(*a, *b, tw, N, p, batch, inverse);
    std::swap(*a, *b);
  }
  count_launches(n);
  return cudaGetLastError();
}

}  // namespace tnep
