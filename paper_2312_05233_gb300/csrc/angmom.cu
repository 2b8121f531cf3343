// Angular moments for population evaluation (the linear-in-c factorisation
// of the angular descriptor and of its share of Eqs. 3-4).
//
// g^A_n(r) = sum_k c^{t_i t_j}_{nk} f_k(r) is linear in the coefficients c,
// which are what differs between the individuals of a population (Sec. II.D).
// So the angular sums and the angular partial-force contractions of every
// individual follow from per-atom moments of the basis, computed once for a
// resident structure set:
//   B^t_{k,lm}     = sum_{j of type t} f_k(r_ij) p_lm(u_ij)
//   Phi^t_{k,lm}   = sum_j |r_ij|^2 grad_j [f_k p_lm](r_ij)          (rank 1, 3 components)
//   Psi^t_{k,lm}   = sum_j r_ij (x) grad_j [f_k p_lm](r_ij)          (rank 2, 9 components)
// with grad [f_k p_lm] = f_k' p_lm u + f_k (grad p_lm - (u . grad p_lm) u) / r.
// Then A_nlm = sum_{t,k} c^{t_i t}_{nk} B^t_{k,lm}, and with
// H^t_{k,lm} = sum_n (dU/dA_nlm) c^{t_i t}_{nk} the angular part of Eq. 3 is
// -sum H . Phi and that of Eq. 4 is -sum H . Psi.
//
// Storage (see AngMomArgs; NLMP = NLM and GBP = NLM * C, each padded to 4):
//   B slot      (t * BA + k) * NLMP + lm
//   Phi / Psi   T * BA * NLMP + (t * BA + k) * GBP + lm * C + c
// One thread per atom walks its angular list once per (t, k, lm block),
// keeping that block's sums in registers.

#include "tnep_device.cuh"
#include "tnep_internal.cuh"

namespace tnep {

namespace {

template <int BA, int LMAX, int RANK, int LB>
__global__ void __launch_bounds__(128) k_angular_moments(const __grid_constant__ AngMomArgs a) {
  constexpr int NLM = LMAX * (LMAX + 2);
  constexpr int C = RANK == 1 ? 3 : 9;
  static_assert(NLM % LB == 0, "the lm blocks must tile the harmonics");
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_atoms) return;
  const float4 pi = a.pos4[i];
  const StructBox bx = a.boxes[a.sorted_struct[i]];
  const float rcinv = 1.f / a.rc_A;
  const int nA = min(a.cnt_A[i], a.cap_A);
  constexpr int NLMP = pad4(NLM), GBP = pad4(NLM * C);
  const int T = a.n_types;
  const int gbase = T * BA * NLMP;
  for (int t = 0; t < T; ++t) {
    for (int k = 0; k < BA; ++k) {
#pragma unroll
      for (int l0 = 0; l0 < NLM; l0 += LB) {
        float Bs[LB], G[LB * C];
#pragma unroll
        for (int u = 0; u < LB; ++u) Bs[u] = 0.f;
#pragma unroll
        for (int u = 0; u < LB * C; ++u) G[u] = 0.f;
        NbrWalk w(a.nbr_A, a.pos4, i, a.cap_A, 0, nA, pi);
        for (int kk = 0; kk < nA; ++kk) {
          const float4 pj = w.next(kk);
          if (__float_as_int(pj.w) != t) continue;
          const float dx = min_image(pj.x, pi.x, bx.L[0], bx.invL[0]);
          const float dy = min_image(pj.y, pi.y, bx.L[1], bx.invL[1]);
          const float dz = min_image(pj.z, pi.z, bx.L[2], bx.invL[2]);
          const float r2 = dx * dx + dy * dy + dz * dz;
          const float rinv = rsqrtf(r2);
          const float r = r2 * rinv;
          const float ux = dx * rinv, uy = dy * rinv, uz = dz * rinv;
          float f[BA], df[BA];
          basis_fwd_bwd<BA>(r, rcinv, f, df);
          float fk = f[0], dfk = df[0];
#pragma unroll
          for (int q = 1; q < BA; ++q)
            if (q == k) { fk = f[q]; dfk = df[q]; }
          float p[NLM], gx[NLM], gy[NLM], gz[NLM];
          real_harmonics<LMAX>(ux, uy, uz, p);
          real_harmonics_grad<LMAX>(ux, uy, uz, gx, gy, gz);
#pragma unroll
          for (int u = 0; u < LB; ++u) {
            const float pv = p[l0 + u], vx = gx[l0 + u], vy = gy[l0 + u], vz = gz[l0 + u];
            Bs[u] += fk * pv;
            const float ug = ux * vx + uy * vy + uz * vz;
            const float s = fk * rinv;
            const float hx = dfk * pv * ux + s * (vx - ug * ux);
            const float hy = dfk * pv * uy + s * (vy - ug * uy);
            const float hz = dfk * pv * uz + s * (vz - ug * uz);
            if constexpr (RANK == 1) {
              G[3 * u] += r2 * hx; G[3 * u + 1] += r2 * hy; G[3 * u + 2] += r2 * hz;
            } else {
              G[9 * u + 0] += dx * hx; G[9 * u + 1] += dx * hy; G[9 * u + 2] += dx * hz;
              G[9 * u + 3] += dy * hx; G[9 * u + 4] += dy * hy; G[9 * u + 5] += dy * hz;
              G[9 * u + 6] += dz * hx; G[9 * u + 7] += dz * hy; G[9 * u + 8] += dz * hz;
            }
          }
        }
        const int b0 = (t * BA + k) * NLMP + l0;
        const int g0 = gbase + (t * BA + k) * GBP + l0 * C;
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          a.amom[amom_index(i, b0 + u, a.amom_slots)] = Bs[u];
#pragma unroll
          for (int c = 0; c < C; ++c) a.amom[amom_index(i, g0 + u * C + c, a.amom_slots)] = G[u * C + c];
        }
      }
    }
  }
}

}  // namespace

size_t angular_moment_slots(int variant, int rank, int n_types) {
  const int BA = variant == kVarStd ? 9 : 6, LMAX = variant == kVarStd ? 4 : 3;
  const int NLM = LMAX * (LMAX + 2);
  return (size_t)n_types * BA * (pad4(NLM) + pad4(NLM * (rank == 1 ? 3 : 9)));
}

cudaError_t launch_angular_moments(int variant, int rank, const AngMomArgs& a, cudaStream_t st) {
  if (a.n_atoms <= 0) return cudaSuccess;
  count_launches(1);
  const int grid = (a.n_atoms + 127) / 128;
  if (variant == kVarStd) {
    if (rank == 1) k_angular_moments<9, 4, 1, 8><<<grid, 128, 0, st>>>(a);
    else k_angular_moments<9, 4, 2, 4><<<grid, 128, 0, st>>>(a);
  } else if (variant == kVarSmall) {
    if (rank == 1) k_angular_moments<6, 3, 1, 5><<<grid, 128, 0, st>>>(a);
    else k_angular_moments<6, 3, 2, 5><<<grid, 128, 0, st>>>(a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace tnep
