// Device helpers shared by the fused and the radial-moment kernels.
#pragma once

#include "tnep_internal.cuh"

namespace tnep {

constexpr float kPi = 3.14159265358979323846f;

// Chebyshev basis f_k = (T_k(x) + 1) f_c / 2, x = 2 (r/rc - 1)^2 - 1.
template <int B>
__device__ __forceinline__ void basis_fwd(float r, float rcinv, float* f) {
  float sn, cs;
  __sincosf(kPi * r * rcinv, &sn, &cs);
  const float fc = 0.5f + 0.5f * cs;
  const float t = r * rcinv - 1.f;
  const float x = 2.f * t * t - 1.f;
  const float hfc = 0.5f * fc;
  f[0] = fc;
  float T0 = 1.f, T1 = x;
  if constexpr (B > 1) f[1] = hfc * (x + 1.f);
#pragma unroll
  for (int k = 2; k < B; ++k) {
    const float T2 = 2.f * x * T1 - T0;
    f[k] = hfc * (T2 + 1.f);
    T0 = T1; T1 = T2;
  }
}

// Basis and its radial derivative.
template <int B>
__device__ __forceinline__ void basis_fwd_bwd(float r, float rcinv, float* f, float* df) {
  float sn, cs;
  __sincosf(kPi * r * rcinv, &sn, &cs);
  const float fc = 0.5f + 0.5f * cs;
  const float dfc = -0.5f * kPi * rcinv * sn;
  const float t = r * rcinv - 1.f;
  const float x = 2.f * t * t - 1.f;
  const float dx = 4.f * t * rcinv;
  const float hfc = 0.5f * fc, hdfc = 0.5f * dfc, hdxfc = 0.5f * dx * fc;
  f[0] = fc; df[0] = dfc;
  float T0 = 1.f, T1 = x, dT0 = 0.f, dT1 = 1.f;
  if constexpr (B > 1) { f[1] = hfc * (x + 1.f); df[1] = hdxfc + hdfc * (x + 1.f); }
#pragma unroll
  for (int k = 2; k < B; ++k) {
    const float T2 = 2.f * x * T1 - T0;
    const float dT2 = 2.f * T1 + 2.f * x * dT1 - dT0;
    f[k] = hfc * (T2 + 1.f);
    df[k] = hdxfc * dT2 + hdfc * (T2 + 1.f);
    T0 = T1; T1 = T2; dT0 = dT1; dT1 = dT2;
  }
}

// Minimum-image component of r_ij = r_j - r_i.  The image shift k is taken
// from the plain difference; the box edge is then subtracted from the operand
// that lies near the far face before the final difference, which is exact
// (Sterbenz) for positions wrapped into [0, L): pairs across a face keep the
// precision of short vectors instead of rounding at ulp(L).
__device__ __forceinline__ float min_image(float xj, float xi, float L, float invL) {
  if (L > 0.f) {
    const float k = rintf((xj - xi) * invL);
    const float aj = fmaf(-fmaxf(k, 0.f), L, xj);
    const float ai = fmaf(-fmaxf(-k, 0.f), L, xi);
    return aj - ai;
  }
  return xj - xi;
}

// Software-pipelined walk over one atom's neighbour list: the neighbour index
// is fetched two iterations ahead and its position one iteration ahead, so
// the dependent index -> position gather overlaps the current pair's math.
// Out-of-range slots re-use a valid index (loads stay in bounds).
constexpr int kPrefetch = 8;

struct NbrWalk {
  const int* __restrict__ list;
  const float4* __restrict__ pos;
  int i, cap, s, n;
  int j_ahead;
  float4 p_ahead;
  // entries [s, s + n) of atom i's list
  __device__ __forceinline__ NbrWalk(const int* l, const float4* p, int i_, int cap_, int s_, int n_, float4 self)
      : list(l), pos(p), i(i_), cap(cap_), s(s_), n(n_) {
    const int j0 = n > 0 ? list[nbr_index(i, s, cap)] : i;
    j_ahead = n > 1 ? list[nbr_index(i, s + 1, cap)] : j0;
    p_ahead = n > 0 ? pos[j0] : self;
  }
  __device__ __forceinline__ float4 next(int k) {
    const float4 pj = p_ahead;
    p_ahead = pos[j_ahead];
    if (k + 2 < n) j_ahead = list[nbr_index(i, s + k + 2, cap)];
    // pull the index row kPrefetch entries ahead into L1 (one 128-byte line per warp)
    if (k + kPrefetch < n) asm volatile("prefetch.global.L1 [%0];" ::"l"(list + nbr_index(i, s + k + kPrefetch, cap)));
    return pj;
  }
};

}  // namespace tnep
