// Device helpers shared by the fused and the radial-moment kernels.
#pragma once

#include "tnep_internal.cuh"

namespace tnep {

constexpr float kPi = 3.14159265358979323846f;

// Packed FP32 pairs (sm_100 family): two float32 lanes in one 64-bit
// register and fma.rn.f32x2, which rounds each lane exactly like fmaf but
// takes one issue slot for two multiply-adds.
using f32x2 = unsigned long long;
__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpk2(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

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
constexpr int kPrefetch = 4;

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

// (2 2 2; 0 0 0) = -sqrt(2/35);  C4 = -sqrt(2/35) * (5/(4 pi))^1.5 * 9/2
constexpr float kC4 = -0.26998130975990770f;

// Addition-theorem weights of the real polynomials, l = 1..4 (see real_harmonics):
// w = (4 pi / (2l+1)) * (normalisation of the orthonormal real harmonic)^2.
constexpr float wlm(int k) {
  constexpr float w[24] = {1.f, 1.f, 1.f, 3.f, 3.f, 3.f, 0.75f, 0.25f, 0.625f, 15.f, 0.375f, 0.25f,
                           0.375f, 3.75f, 0.625f, 8.75f, 4.375f, 1.25f, 0.625f, 0.015625f, 0.625f,
                           0.3125f, 4.375f, 0.546875f};
  return w[k];
}
constexpr int l_of(int k) { return k < 3 ? 1 : (k < 8 ? 2 : (k < 15 ? 3 : 4)); }

// Tr(M^3) of the traceless symmetric M built from the l=2 sums a[0..4]
// (xy, yz, xz, x^2-y^2, 3z^2-1), and its gradient with respect to a.
__device__ __forceinline__ float trace_m3(const float* a, float* grad) {
  const float mxy = a[0], myz = a[1], mxz = a[2];
  const float mzz = a[4] * (1.f / 3.f);
  const float mxx = 0.5f * (a[3] - mzz), myy = 0.5f * (-a[3] - mzz);
  const float nxx = mxx * mxx + mxy * mxy + mxz * mxz;
  const float nyy = mxy * mxy + myy * myy + myz * myz;
  const float nzz = mxz * mxz + myz * myz + mzz * mzz;
  const float nxy = mxx * mxy + mxy * myy + mxz * myz;
  const float nyz = mxy * mxz + myy * myz + myz * mzz;
  const float nxz = mxx * mxz + mxy * myz + mxz * mzz;
  // Tr(M^3) = sum_ij M_ij (M^2)_ji
  const float tr = mxx * nxx + myy * nyy + mzz * nzz + 2.f * (mxy * nxy + myz * nyz + mxz * nxz);
  // d Tr(M^3) = 3 Tr(M^2 dM)
  grad[0] = 6.f * nxy;
  grad[1] = 6.f * nyz;
  grad[2] = 6.f * nxz;
  grad[3] = 1.5f * (nxx - nyy);
  grad[4] = nzz - 0.5f * (nxx + nyy);
  return tr;
}

// Real polynomials p_lm(x, y, z) on the unit sphere:
// l=1: x, y, z
// l=2: xy, yz, xz, x^2-y^2, 3z^2-1
// l=3: y(3x^2-y^2), xyz, y(5z^2-1), z(5z^2-3), x(5z^2-1), z(x^2-y^2), x(x^2-3y^2)
// l=4: xy(x^2-y^2), yz(3x^2-y^2), xy(7z^2-1), yz(7z^2-3), 35z^4-30z^2+3,
//      xz(7z^2-3), (x^2-y^2)(7z^2-1), xz(x^2-3y^2), x^4-6x^2y^2+y^4
template <int LMAX>
__device__ __forceinline__ void real_harmonics(float x, float y, float z, float* p) {
  p[0] = x; p[1] = y; p[2] = z;
  if constexpr (LMAX >= 2) {
    const float x2 = x * x, y2 = y * y, z2 = z * z;
    p[3] = x * y; p[4] = y * z; p[5] = x * z; p[6] = x2 - y2; p[7] = 3.f * z2 - 1.f;
    if constexpr (LMAX >= 3) {
      const float t5 = 5.f * z2;
      p[8] = y * (3.f * x2 - y2);
      p[9] = x * y * z;
      p[10] = y * (t5 - 1.f);
      p[11] = z * (t5 - 3.f);
      p[12] = x * (t5 - 1.f);
      p[13] = z * (x2 - y2);
      p[14] = x * (x2 - 3.f * y2);
      if constexpr (LMAX >= 4) {
        const float t7 = 7.f * z2;
        p[15] = x * y * (x2 - y2);
        p[16] = y * z * (3.f * x2 - y2);
        p[17] = x * y * (t7 - 1.f);
        p[18] = y * z * (t7 - 3.f);
        p[19] = (35.f * z2 - 30.f) * z2 + 3.f;
        p[20] = x * z * (t7 - 3.f);
        p[21] = (x2 - y2) * (t7 - 1.f);
        p[22] = x * z * (x2 - 3.f * y2);
        p[23] = x2 * (x2 - 3.f * y2) - y2 * (3.f * x2 - y2);
      }
    }
  }
}

// Gradients of the same polynomials (as polynomials of x, y, z), one
// vector per (l, m): (gx[k], gy[k], gz[k]) = grad p_k.
template <int LMAX>
__device__ __forceinline__ void real_harmonics_grad(float x, float y, float z, float* gx, float* gy, float* gz) {
  gx[0] = 1.f; gy[0] = 0.f; gz[0] = 0.f;
  gx[1] = 0.f; gy[1] = 1.f; gz[1] = 0.f;
  gx[2] = 0.f; gy[2] = 0.f; gz[2] = 1.f;
  if constexpr (LMAX >= 2) {
    gx[3] = y;         gy[3] = x;          gz[3] = 0.f;
    gx[4] = 0.f;       gy[4] = z;          gz[4] = y;
    gx[5] = z;         gy[5] = 0.f;        gz[5] = x;
    gx[6] = 2.f * x;   gy[6] = -2.f * y;   gz[6] = 0.f;
    gx[7] = 0.f;       gy[7] = 0.f;        gz[7] = 6.f * z;
    if constexpr (LMAX >= 3) {
      const float x2 = x * x, y2 = y * y, z2 = z * z;
      const float xy = x * y, yz = y * z, xz = x * z;
      const float t5 = 5.f * z2 - 1.f, d3 = 3.f * x2 - 3.f * y2;
      gx[8] = 6.f * xy;    gy[8] = d3;           gz[8] = 0.f;
      gx[9] = yz;          gy[9] = xz;           gz[9] = xy;
      gx[10] = 0.f;        gy[10] = t5;          gz[10] = 10.f * yz;
      gx[11] = 0.f;        gy[11] = 0.f;         gz[11] = 15.f * z2 - 3.f;
      gx[12] = t5;         gy[12] = 0.f;         gz[12] = 10.f * xz;
      gx[13] = 2.f * xz;   gy[13] = -2.f * yz;   gz[13] = x2 - y2;
      gx[14] = d3;         gy[14] = -6.f * xy;   gz[14] = 0.f;
      if constexpr (LMAX >= 4) {
        const float t7 = 7.f * z2 - 1.f, t73 = 7.f * z2 - 3.f, xyz = xy * z;
        const float a15 = 3.f * x2 * y - y2 * y, b15 = x2 * x - 3.f * x * y2;
        gx[15] = a15;                 gy[15] = b15;                 gz[15] = 0.f;
        gx[16] = 6.f * xyz;           gy[16] = d3 * z;              gz[16] = a15;
        gx[17] = y * t7;              gy[17] = x * t7;              gz[17] = 14.f * xyz;
        gx[18] = 0.f;                 gy[18] = t73 * z;             gz[18] = (21.f * z2 - 3.f) * y;
        gx[19] = 0.f;                 gy[19] = 0.f;                 gz[19] = (140.f * z2 - 60.f) * z;
        gx[20] = t73 * z;             gy[20] = 0.f;                 gz[20] = (21.f * z2 - 3.f) * x;
        gx[21] = 2.f * x * t7;        gy[21] = -2.f * y * t7;       gz[21] = 14.f * z * (x2 - y2);
        gx[22] = d3 * z;              gy[22] = -6.f * xyz;          gz[22] = b15;
        gx[23] = 4.f * x2 * x - 12.f * x * y2;  gy[23] = 4.f * y2 * y - 12.f * x2 * y;  gz[23] = 0.f;
      }
    }
  }
}

}  // namespace tnep
