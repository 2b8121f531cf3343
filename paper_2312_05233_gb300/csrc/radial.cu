// Radial moments: one pass over each atom's type-sorted radial list.
//
// g_n^{t_i t_j}(r) = sum_k c^{t_i t_j}_{nk} f_k(r) is linear in c, so the
// radial descriptor and the radial part of Eqs. 3-4 need only per-type sums
// of basis values over the neighbours, computed once per frame and shared by
// every model (and every individual of a population) with the same rc_R:
//   F^t_k    = sum_{j of type t} f_k(r_ij)
//   V^t_k    = sum_j r_ij f_k'(r_ij) r_ij_vec                 (rank 1)
//   W^t_k    = sum_j f_k'(r_ij) / r_ij  r_ij_vec (x) r_ij_vec  (rank 2, symmetric)
// since -|r|^2 dU_i/dr_ij = -r g'(r) r_vec and -r_vec (x) dU_i/dr_ij =
// -g'(r)/r r_vec (x) r_vec with g' = sum_k D_k f_k'.

#include "tnep_device.cuh"
#include "tnep_internal.cuh"

namespace tnep {

namespace {

template <bool HV, bool HW>
__global__ void __launch_bounds__(128, 3) k_radial(const __grid_constant__ RadialArgs a) {
  constexpr int B = kMomBasis;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_atoms) return;
  const float4 pi = a.pos4[i];
  const StructBox bx = a.boxes[a.sorted_struct[i]];
  const float rcinv = 1.f / a.rc_R;
  float* mom = a.mom + i;
  const size_t ms = a.mom_stride;
  int start = 0;
  for (int t = 0; t < a.n_types; ++t) {
    const int n = a.seg_R[(size_t)t * a.seg_stride + i];
    // accumulators in basis pairs (k = 2q, 2q + 1), one packed multiply-add
    // per pair; the last index of an odd basis size is accumulated alone
    constexpr int BP = B / 2;
    constexpr bool ODD = (B & 1) != 0;
    f32x2 F2[BP], V2[HV ? 3 * BP : 1], W2[HW ? 6 * BP : 1];
    float Ft = 0.f, Vt[3] = {0.f, 0.f, 0.f}, Wt[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < BP; ++q) F2[q] = 0ull;
#pragma unroll
    for (int k = 0; k < (HV ? 3 * BP : 1); ++k) V2[k] = 0ull;
#pragma unroll
    for (int k = 0; k < (HW ? 6 * BP : 1); ++k) W2[k] = 0ull;
    NbrWalk w(a.nbr_R, a.pos4, i, a.cap_R, radial_segment_start(a.two_ended, t, start, n, a.cap_R), n, pi);
    // two pairs per iteration interleave their (serial) basis recursions;
    // 166 registers, three CTAs per SM
#pragma unroll 2
    for (int kk = 0; kk < n; ++kk) {
      const float4 pj = w.next(kk);
      const float dx = min_image(pj.x, pi.x, bx.L[0], bx.invL[0]);
      const float dy = min_image(pj.y, pi.y, bx.L[1], bx.invL[1]);
      const float dz = min_image(pj.z, pi.z, bx.L[2], bx.invL[2]);
      const float r2 = dx * dx + dy * dy + dz * dz;
      const float rinv = rsqrtf(r2);
      const float r = r2 * rinv;
      // basis: f_k = fc (T_k(x) + 1) / 2 enters F only through its sum, so
      // F accumulates sum fc T_k (slot k) and is finished after the walk as
      // F_k = (FT_k + FT_0) / 2 (T_0 = 1); f_k' = (fc' (T_k + 1) + fc x' T_k') / 2
      float sn, cs;
      __sincosf(kPi * r * rcinv, &sn, &cs);
      const float fc = 0.5f + 0.5f * cs;
      const float hdfc = -0.25f * kPi * rcinv * sn;
      const float tt = r * rcinv - 1.f;
      const float x = 2.f * tt * tt - 1.f, x2 = 2.f * x;
      const float hdxfc = 2.f * tt * rcinv * fc;
      float Tk[B], df[B];
      {
        float T0 = 1.f, T1 = x, d0 = 0.f, d1 = 1.f;
        Tk[0] = 1.f; df[0] = 2.f * hdfc;
        if constexpr (B > 1) { Tk[1] = x; df[1] = fmaf(hdxfc, 1.f, hdfc * (x + 1.f)); }
#pragma unroll
        for (int k = 2; k < B; ++k) {
          const float T2 = fmaf(x2, T1, -T0);
          const float d2 = fmaf(2.f, T1, fmaf(x2, d1, -d0));
          Tk[k] = T2;
          df[k] = fmaf(hdxfc, d2, hdfc * (T2 + 1.f));
          T0 = T1; T1 = T2; d0 = d1; d1 = d2;
        }
      }
      // pair factors shared by every basis index k
      float rv[3], rr[6];
      if constexpr (HV) { rv[0] = r * dx; rv[1] = r * dy; rv[2] = r * dz; }
      if constexpr (HW) {
        const float ux = dx * rinv, uy = dy * rinv;
        rr[0] = ux * dx; rr[1] = ux * dy; rr[2] = ux * dz;
        rr[3] = uy * dy; rr[4] = uy * dz; rr[5] = dz * rinv * dz;
      }
      const f32x2 fcc = pk2(fc, fc);
      f32x2 rv2[3], rr2[6];
      if constexpr (HV) {
#pragma unroll
        for (int c = 0; c < 3; ++c) rv2[c] = pk2(rv[c], rv[c]);
      }
      if constexpr (HW) {
#pragma unroll
        for (int c = 0; c < 6; ++c) rr2[c] = pk2(rr[c], rr[c]);
      }
#pragma unroll
      for (int q = 0; q < BP; ++q) {
        const f32x2 t2 = pk2(Tk[2 * q], Tk[2 * q + 1]);
        F2[q] = fma2(fcc, t2, F2[q]);
        if constexpr (HV || HW) {
          const f32x2 d2 = pk2(df[2 * q], df[2 * q + 1]);
          if constexpr (HV) {
#pragma unroll
            for (int c = 0; c < 3; ++c) V2[c * BP + q] = fma2(d2, rv2[c], V2[c * BP + q]);
          }
          if constexpr (HW) {
#pragma unroll
            for (int c = 0; c < 6; ++c) W2[c * BP + q] = fma2(d2, rr2[c], W2[c * BP + q]);
          }
        }
      }
      if constexpr (ODD) {
        Ft = fmaf(fc, Tk[B - 1], Ft);
        if constexpr (HV) {
#pragma unroll
          for (int c = 0; c < 3; ++c) Vt[c] = fmaf(df[B - 1], rv[c], Vt[c]);
        }
        if constexpr (HW) {
#pragma unroll
          for (int c = 0; c < 6; ++c) Wt[c] = fmaf(df[B - 1], rr[c], Wt[c]);
        }
      }
    }
    start += n;
    float F[B];
#pragma unroll
    for (int q = 0; q < BP; ++q) unpk2(F2[q], F[2 * q], F[2 * q + 1]);
    if constexpr (ODD) F[B - 1] = Ft;
#pragma unroll
    for (int k = 0; k < B; ++k) mom[(size_t)(t * B + k) * ms] = k == 0 ? F[0] : 0.5f * (F[k] + F[0]);
    if constexpr (HV) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int q = 0; q < BP; ++q) {
          float lo, hi;
          unpk2(V2[c * BP + q], lo, hi);
          mom[(size_t)(a.v0 + 3 * t * B + 3 * (2 * q) + c) * ms] = lo;
          mom[(size_t)(a.v0 + 3 * t * B + 3 * (2 * q + 1) + c) * ms] = hi;
        }
        if constexpr (ODD) mom[(size_t)(a.v0 + 3 * t * B + 3 * (B - 1) + c) * ms] = Vt[c];
      }
    }
    if constexpr (HW) {
#pragma unroll
      for (int c = 0; c < 6; ++c) {
#pragma unroll
        for (int q = 0; q < BP; ++q) {
          float lo, hi;
          unpk2(W2[c * BP + q], lo, hi);
          mom[(size_t)(a.w0 + 6 * t * B + 6 * (2 * q) + c) * ms] = lo;
          mom[(size_t)(a.w0 + 6 * t * B + 6 * (2 * q + 1) + c) * ms] = hi;
        }
        if constexpr (ODD) mom[(size_t)(a.w0 + 6 * t * B + 6 * (B - 1) + c) * ms] = Wt[c];
      }
    }
  }
}

}  // namespace

cudaError_t launch_radial_moments(const RadialArgs& a, cudaStream_t st) {
  if (a.n_atoms <= 0) return cudaSuccess;
  count_launches(1);
  const int grid = (a.n_atoms + 127) / 128;
  const bool hv = a.v0 >= 0, hw = a.w0 >= 0;
  if (hv && hw) k_radial<true, true><<<grid, 128, 0, st>>>(a);
  else if (hv) k_radial<true, false><<<grid, 128, 0, st>>>(a);
  else if (hw) k_radial<false, true><<<grid, 128, 0, st>>>(a);
  else k_radial<false, false><<<grid, 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tnep
