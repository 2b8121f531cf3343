// Fused TNEP kernel: descriptor -> network -> partial forces -> tensor contraction.
//
// One thread owns one atom i:
//   1. radial descriptor q_n = sum_{t,k} c^{t_i t}_{nk} F^t_k from the per-type
//      radial moments (radial.cu; g_n is linear in c)
//   2. angular forward  A_nlm = sum_j g^A_n(r_ij) p_lm(u_ij)   (120 register accumulators)
//      then q_nl = sum_m w_lm A_nlm^2 and the 4-body invariant
//   3. network U_i = w1 . tanh(W0 s - b0) - b1 and dU/dq (Eq. 1)
//   4. radial part of the contraction through the moments V (rank 1) or W (rank 2)
//   5. angular backward: partial force
//        dU_i/dr_ij = s1 u + (V - (u.V) u) / r,
//        s1 = sum_lm T_lm p_lm = sum_n g_n'(r) P_n,  V = sum_lm S_lm grad p_lm,
//        S_lm = sum_n G_nlm g_n(r),  T_lm = sum_n G_nlm g_n'(r),
//        P_n = sum_lm G_nlm p_lm,  G = dU/dA
// and contracts each angular partial force on the fly (Sec. II.B-C):
//   rank 1 (Eq. 3):  mu_i    -= |r_ij|^2 dU_i/dr_ij
//   rank 2 (Eq. 4):  alpha_i -= r_ij (x) dU_i/dr_ij,  plus U_i on the diagonal.
// With the pair cache (the default for single-model launches) the forward walk
// stores each angular pair's r_ij, 1/|r_ij|, g_n and g_n' and the backward
// walk reads them back; without it the backward walk recomputes them.
// Per-atom results go out in float32 (SoA) and are summed per structure in
// float64 by the reduce kernel.
//
// Angular functions: real Cartesian polynomials p_lm(u) of the unit vector u
// with weights w_lm such that P_l(a.b) = sum_m w_lm p_lm(a) p_lm(b) (the
// addition theorem in a real, unnormalised basis).  With this basis
// q_nl = sum_{j,k} g g P_l(cos theta_ijk) = sum_m w_lm A_nlm^2 exactly.
// The l = 2 four-body invariant sum_m (2 2 2; m1 m2 m3) A A A equals
// C4 * Tr(M^3), where M is the traceless symmetric tensor
// sum_j g_n(r_ij) (u u^T - I/3) built from the five l = 2 sums, and
// C4 = (2 2 2; 0 0 0) (5 / 4 pi)^(3/2) / (2/9) (evaluate both sides at
// a = b = c = z_hat; the invariant is unique up to scale).

#include <algorithm>
#include <atomic>
#include <climits>

#include "tc_sm100.cuh"
#include "tnep_device.cuh"
#include "tnep_internal.cuh"

namespace tnep {

namespace {

// V += sum_lm S_lm * grad p_lm(x, y, z)  (gradient of the polynomial as written).
// Each order l accumulates into its own partial sums so that the four
// dependency chains run side by side.
template <int LMAX>
__device__ __forceinline__ void harmonic_grad(const float* S, float x, float y, float z, float& vx, float& vy,
                                              float& vz) {
  float ax = S[0], ay = S[1], az = S[2];
  float bx = 0.f, by = 0.f, bz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, dx = 0.f, dy = 0.f, dz = 0.f;
  if constexpr (LMAX >= 2) {
    bx = y * S[3] + z * S[5] + 2.f * x * S[6];
    by = x * S[3] + z * S[4] - 2.f * y * S[6];
    bz = y * S[4] + x * S[5] + 6.f * z * S[7];
    if constexpr (LMAX >= 3) {
      const float x2 = x * x, y2 = y * y, z2 = z * z;
      const float xy = x * y, yz = y * z, xz = x * z;
      const float t5 = 5.f * z2 - 1.f;
      // p8 = 3x^2y - y^3, p9 = xyz, p10 = y(5z^2-1), p11 = 5z^3 - 3z,
      // p12 = x(5z^2-1), p13 = z(x^2-y^2), p14 = x^3 - 3xy^2
      cx = 6.f * xy * S[8] + yz * S[9] + t5 * S[12] + 2.f * xz * S[13] + (3.f * x2 - 3.f * y2) * S[14];
      cy = (3.f * x2 - 3.f * y2) * S[8] + xz * S[9] + t5 * S[10] - 2.f * yz * S[13] - 6.f * xy * S[14];
      cz = xy * S[9] + 10.f * yz * S[10] + (15.f * z2 - 3.f) * S[11] + 10.f * xz * S[12] + (x2 - y2) * S[13];
      if constexpr (LMAX >= 4) {
        const float t7 = 7.f * z2 - 1.f, t73 = 7.f * z2 - 3.f;
        const float xyz = xy * z;
        // p15 = x^3 y - x y^3, p16 = 3x^2yz - y^3 z, p17 = xy(7z^2-1),
        // p18 = 7yz^3 - 3yz, p19 = 35z^4 - 30z^2 + 3, p20 = xz(7z^2-3),
        // p21 = (x^2-y^2)(7z^2-1), p22 = x^3 z - 3 x y^2 z, p23 = x^4 - 6x^2y^2 + y^4
        dx = (3.f * x2 * y - y2 * y) * S[15] + 6.f * xyz * S[16] + y * t7 * S[17] + t73 * z * S[20] +
             2.f * x * t7 * S[21] + (3.f * x2 - 3.f * y2) * z * S[22] + (4.f * x2 * x - 12.f * x * y2) * S[23];
        dy = (x2 * x - 3.f * x * y2) * S[15] + (3.f * x2 - 3.f * y2) * z * S[16] + x * t7 * S[17] +
             t73 * z * S[18] - 2.f * y * t7 * S[21] - 6.f * xyz * S[22] + (4.f * y2 * y - 12.f * x2 * y) * S[23];
        dz = (3.f * x2 * y - y2 * y) * S[16] + 14.f * xyz * S[17] + (21.f * z2 - 3.f) * y * S[18] +
             (140.f * z2 - 60.f) * z * S[19] + (21.f * z2 - 3.f) * x * S[20] + 14.f * z * (x2 - y2) * S[21] +
             (x2 * x - 3.f * x * y2) * S[22];
      }
    }
  }
  vx += (ax + bx) + (cx + dx);
  vy += (ay + by) + (cy + dy);
  vz += (az + bz) + (cz + dz);
}

// Loads one (t_i, t_j) coefficient block c[n][k] from shared memory.
template <int NN, int B>
__device__ __forceinline__ void load_coeffs(const float* blk, float* cc) {
  constexpr int NV = (NN * B + 3) / 4;
  const float4* c4 = reinterpret_cast<const float4*>(blk);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float4 t = c4[v];
    cc[4 * v] = t.x; cc[4 * v + 1] = t.y; cc[4 * v + 2] = t.z; cc[4 * v + 3] = t.w;
  }
}

// Bytes of shared memory the tensor-core network needs after the scratch:
// mbarrier + TMEM slot (128 B), the A tile (128 rows x 64: a high and a low
// bf16 part of 32 columns each) and, per network, the two B tiles (32 rows x
// 64, high and low parts of the weights).
__host__ __device__ constexpr int tc_smem_bytes(int nets) { return 128 + 128 * 64 * 2 + nets * 2 * 32 * 64 * 2; }
__host__ __device__ constexpr uint32_t tc_tmem_cols(int nets) {
  return nets * 32 <= 32 ? 32u : nets * 32 <= 64 ? 64u : nets * 32 <= 128 ? 128u : 256u;
}
constexpr long long kMbarTries = kDefaultWaitTries;

// TCM: 0 = FP32 network on the CUDA cores; 1 = network products on the
// tensor cores with BF16 operands and FP32 accumulation; 2 = the same with
// every operand split into a high and a low BF16 part and three products
// (hi*hi + hi*lo + lo*hi), which is accurate to about 2^-17.
// FACT: the angular sums and the angular part of Eqs. 3-4 come from the
// per-atom angular moments (angmom.cu) instead of a walk over the angular
// list: A_nlm = sum_{t,k} c_nk B^t_{k,lm}, and -sum_{t,k,lm} H^t_{k,lm} Phi
// (or Psi) with H^t_{k,lm} = sum_n G_nlm c_nk.  Exact up to rounding; used
// for populations, whose individuals share the moments.
// PC: the forward walk stores each pair's r_ij, 1/|r_ij|, g_n and g_n' in
// a.pcache and the backward walk reads them back (bitwise the same values it
// would recompute).
template <int NR, int NA, int BR, int BA, int LMAX, bool FB, int RANK, int BLK, int TCM, bool FACT = false,
          bool PC = false>
__global__ void __launch_bounds__(BLK, 256 / BLK) k_fused(const __grid_constant__ FusedArgs a) {
  static_assert(!(PC && FACT), "the pair cache belongs to the walked form");
  constexpr bool TC = TCM != 0;
  static_assert(!TC || BLK == 128, "the tensor-core network uses M = 128 rows, one per atom");
  constexpr int NLM = LMAX * (LMAX + 2);
  constexpr int D = NR + NA * LMAX + (FB ? NA : 0);
  constexpr int DP = (D + 3) & ~3;
  constexpr int C = RANK == 1 ? 3 : 9;
  constexpr int NBR4 = ((NR * BR + 3) / 4) * 4;
  constexpr int NBA4 = ((NA * BA + 3) / 4) * 4;
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  const ModelLayout& Ly = a.lay;  // the packed model (global memory)
  // Its copy in shared memory: with the tensor cores the FP32 W0 block
  // (nets x H x Dp floats) is left out -- the products read the BF16 tiles
  // made from it, which are built from global memory -- and every word after
  // it moves down by w0n.  The offsets stay expressions of the kernel
  // parameters (no layout copy held in registers).
  const int w0n = TC ? Ly.off_b0 - Ly.off_W0 : 0;
  const int sm_words = Ly.words - w0n;
  const int tid = threadIdx.x;
  float* scratch = sm + sm_words + tid;  // slot s at scratch[s * BLK]

  // ---------------------------------------------------------------- tensor-core set-up (once per CTA)
  uint32_t tmem_base = 0, mbar = 0;
  __nv_bfloat16* tileA = nullptr;
  __nv_bfloat16* tileB1 = nullptr;
  __nv_bfloat16* tileB2 = nullptr;
  int* next_item = nullptr;  // the CTA's next work item (tensor-core path)
  if constexpr (TC) {
    constexpr int NSLOT = NA * LMAX * (LMAX + 2);
    unsigned char* tcb = reinterpret_cast<unsigned char*>(sm + sm_words + NSLOT * BLK);
    uint64_t* mb = reinterpret_cast<uint64_t*>(tcb);
    uint32_t* slot = reinterpret_cast<uint32_t*>(tcb + 8);
    next_item = reinterpret_cast<int*>(tcb + 16);
    tileA = reinterpret_cast<__nv_bfloat16*>(tcb + 128);
    tileB1 = tileA + 128 * 64;
    tileB2 = tileB1 + Ly.nets * 32 * 64;
    if (tid == 0) {
      tc::mbar_init(tc::smem_addr(mb), 1);
      tc::fence_mbar_init();
    }
    if (tid < 32) tc::tmem_alloc(tc::smem_addr(slot), tc_tmem_cols(Ly.nets));
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tmem_base = *slot;
    mbar = tc::smem_addr(mb);
  }

  // Work item w = (atom block, individual); with pop_major the individual
  // varies fastest so that CTAs running together share an atom block's lists.
  // Without the tensor cores each CTA takes item blockIdx.x.  With them the
  // CTAs are persistent: each starts with item blockIdx.x and takes the next
  // from the counter a.status->work_next (gridDim.x + its value, zeroed before
  // the launch), fetched by thread 0 between the two network products and
  // handed to the CTA through shared memory across the second product's
  // barrier; the model, the weight tiles made from it, the mbarrier and the
  // TMEM columns are then set up once per CTA (the model again only when the
  // individual changes).  Extra CTAs find the counter exhausted and exit, so
  // the grid need not match the number of CTAs resident at once.
  const int nblk = (a.n_atoms + BLK - 1) / BLK;
  const int n_work = nblk * a.n_pop;
  // loads individual `pop`'s model into shared memory (and, with the tensor
  // cores, the weight tiles made from it)
  auto load_model = [&](const int pop) {
    const float* model = a.model + (size_t)pop * a.model_stride;
    const float4* src = reinterpret_cast<const float4*>(model);
    // words [0, off_W0) in place, then (tensor cores) the words after W0 moved
    // down over it; off_W0 and off_b0 are multiples of 4
    const int skip4 = w0n >> 2, w4 = Ly.off_W0 >> 2;
    for (int k = tid; k < (sm_words >> 2); k += BLK) sm4[k] = src[k < w4 ? k : k + skip4];
    __syncthreads();
    if constexpr (TC) {
      // B1[net]: row = hidden unit h, column = descriptor d  (W0[h][d])
      // B2[net]: row = descriptor d, column = hidden unit h  (W0[h][d])
      // columns 0-31 hold the bf16 rounding of the weight, 32-63 the bf16
      // rounding of what is left over
      for (int idx = tid; idx < Ly.nets * 32 * 32; idx += BLK) {
        const int nt = idx >> 10, r = (idx >> 5) & 31, k = idx & 31;
        const float* W = model + Ly.off_W0 + nt * Ly.H * DP;
        const float w1v = (r < Ly.H && k < Ly.D) ? W[r * DP + k] : 0.f;
        const float w2v = (k < Ly.H && r < Ly.D) ? W[k * DP + r] : 0.f;
        const __nv_bfloat16 h1 = __float2bfloat16_rn(w1v), h2 = __float2bfloat16_rn(w2v);
        tileB1[nt * 2048 + (tc::kmajor_offset(r, k, 64) >> 1)] = h1;
        tileB1[nt * 2048 + (tc::kmajor_offset(r, 32 + k, 64) >> 1)] = __float2bfloat16_rn(w1v - __bfloat162float(h1));
        tileB2[nt * 2048 + (tc::kmajor_offset(r, k, 64) >> 1)] = h2;
        tileB2[nt * 2048 + (tc::kmajor_offset(r, 32 + k, 64) >> 1)] = __float2bfloat16_rn(w2v - __bfloat162float(h2));
      }
      // the tiles are made visible to the tensor cores by the fence and the
      // barrier that precede every product
    }
  };

  // one work item; false when the tensor-core network gave up (the CTA then
  // returns at once)
  auto item = [&](const int pop, const int ablk) -> bool {
  const int i_raw = ablk * BLK + tid;
  const bool valid = i_raw < a.n_atoms;
  // The tensor-core path has CTA-wide barriers: threads past the end work on
  // the last atom and store nothing.
  if (!TC && !valid) return true;
  const int i = valid ? i_raw : a.n_atoms - 1;

  const float4 pi = a.pos4[i];
  const int ti = __float_as_int(pi.w);
  const StructBox bx = a.boxes[a.sorted_struct[i]];
  const int T = Ly.n_types;
  const float rcAinv = 1.f / a.rc_A;

  // ---------------------------------------------------------------- radial descriptor
  // q_n = sum_t sum_k c^{t_i t}_{nk} F^t_k from the per-type radial moments
  float q[DP];
#pragma unroll
  for (int d = 0; d < DP; ++d) q[d] = 0.f;
  const float* cR_i = sm + Ly.off_cR + ti * T * Ly.stride_cR;
  const float* mom = a.mom + i;
  for (int t = 0; t < T; ++t) {
    float Fk[BR];
#pragma unroll
    for (int k = 0; k < BR; ++k) Fk[k] = mom[(size_t)(t * kMomBasis + k) * a.mom_stride];
    float cc[NBR4];
    load_coeffs<NR, BR>(cR_i + t * Ly.stride_cR, cc);
#pragma unroll
    for (int n = 0; n < NR; ++n)
#pragma unroll
      for (int k = 0; k < BR; ++k) q[n] += cc[n * BR + k] * Fk[k];
  }

  // ---------------------------------------------------------------- angular forward
  const int nA = min(a.cnt_A[i], a.cap_A);
  const float* cA_i = sm + Ly.off_cA + ti * T * Ly.stride_cA;
  {
    float A[NA * NLM];
#pragma unroll
    for (int k = 0; k < NA * NLM; ++k) A[k] = 0.f;
    // the walk accumulates A in lm pairs, one packed multiply-add per pair
    constexpr int NP = NLM / 2;
    f32x2 A2[NA * NP];
#pragma unroll
    for (int k = 0; k < NA * NP; ++k) A2[k] = 0ull;
    if constexpr (FACT) {
      constexpr int NLMP = pad4(NLM);
      // float4 group g (slots 4g..4g+3) of this atom at m4[g * 32]
      const float4* m4 = reinterpret_cast<const float4*>(a.amom) + (size_t)(i >> 5) * (a.amom_slots / 4) * 32 + (i & 31);
      for (int t = 0; t < T; ++t) {
        const float* cblk = cA_i + t * Ly.stride_cA;
#pragma unroll 1
        for (int k = 0; k < BA; ++k) {
          float ck[NA];
#pragma unroll
          for (int n = 0; n < NA; ++n) ck[n] = cblk[n * BA + k];
          const float4* b = m4 + (size_t)((t * BA + k) * (NLMP / 4)) * 32;
          // pull the next (t, k) slice towards L1 while this one is used
          if (t * BA + k + 1 < T * BA) {
#pragma unroll
            for (int q = 0; q < NLMP / 4; ++q)
              asm volatile("prefetch.global.L1 [%0];" ::"l"(b + (size_t)(NLMP / 4 + q) * 32));
          }
#pragma unroll
          for (int q = 0; q < NLMP / 4; ++q) {
            const float4 v = b[(size_t)q * 32];
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (4 * q + u < NLM) {
#pragma unroll
                for (int n = 0; n < NA; ++n) A[n * NLM + 4 * q + u] += ck[n] * vv[u];
              }
            }
          }
        }
      }
    }
    NbrWalk wA(a.nbr_A, a.pos4, i, a.cap_A, 0, FACT ? 0 : nA, pi);
    for (int kk = 0; kk < (FACT ? 0 : nA); ++kk) {
      const float4 pj = wA.next(kk);
      const float dx = min_image(pj.x, pi.x, bx.L[0], bx.invL[0]);
      const float dy = min_image(pj.y, pi.y, bx.L[1], bx.invL[1]);
      const float dz = min_image(pj.z, pi.z, bx.L[2], bx.invL[2]);
      const float r2 = dx * dx + dy * dy + dz * dz;
      const float rinv = rsqrtf(r2);
      const float r = r2 * rinv;
      float cc[NBA4];
      load_coeffs<NA, BA>(cA_i + __float_as_int(pj.w) * Ly.stride_cA, cc);
      float g[NA];
      if constexpr (PC) {
        // the backward walk's g_n and g_n', computed here once and cached
        float f[BA], df[BA], dg[NA];
        basis_fwd_bwd<BA>(r, rcAinv, f, df);
#pragma unroll
        for (int n = 0; n < NA; ++n) {
          float s0 = 0.f, s1 = 0.f;
#pragma unroll
          for (int k = 0; k < BA; ++k) { s0 += cc[n * BA + k] * f[k]; s1 += cc[n * BA + k] * df[k]; }
          g[n] = s0; dg[n] = s1;
        }
        constexpr int NQ = pair_cache_quads(NA);
        float v[4 * NQ];
        v[0] = dx; v[1] = dy; v[2] = dz; v[3] = rinv;
#pragma unroll
        for (int n = 0; n < NA; ++n) { v[4 + n] = g[n]; v[4 + NA + n] = dg[n]; }
#pragma unroll
        for (int u = 4 + 2 * NA; u < 4 * NQ; ++u) v[u] = 0.f;
        float4* dst = a.pcache + (size_t)kk * NQ * a.pc_stride + i_raw;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
          __stcg(dst + (size_t)q * a.pc_stride, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
      } else {
        float f[BA];
        basis_fwd<BA>(r, rcAinv, f);
#pragma unroll
        for (int n = 0; n < NA; ++n) {
          float s = 0.f;
#pragma unroll
          for (int k = 0; k < BA; ++k) s += cc[n * BA + k] * f[k];
          g[n] = s;
        }
      }
      float p[NLM];
      real_harmonics<LMAX>(dx * rinv, dy * rinv, dz * rinv, p);
      f32x2 p2[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) p2[q] = pk2(p[2 * q], p[2 * q + 1]);
#pragma unroll
      for (int n = 0; n < NA; ++n) {
        const f32x2 gg = pk2(g[n], g[n]);
#pragma unroll
        for (int q = 0; q < NP; ++q) A2[n * NP + q] = fma2(gg, p2[q], A2[n * NP + q]);
        if constexpr (NLM & 1) A[n * NLM + NLM - 1] += g[n] * p[NLM - 1];
      }
    }
    if constexpr (!FACT) {
#pragma unroll
      for (int n = 0; n < NA; ++n)
#pragma unroll
        for (int q = 0; q < NP; ++q) unpk2(A2[n * NP + q], A[n * NLM + 2 * q], A[n * NLM + 2 * q + 1]);
    }
    // descriptor components and stash of A for the backward pass
#pragma unroll
    for (int n = 0; n < NA; ++n) {
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm) {
        const float v = A[n * NLM + lm];
        q[NR + (l_of(lm) - 1) * NA + n] += wlm(lm) * v * v;
        scratch[(n * NLM + lm) * BLK] = v;
      }
      if constexpr (FB) {
        float gr[5];
        q[NR + LMAX * NA + n] = kC4 * trace_m3(&A[n * NLM + 3], gr);
      }
    }
  }

  // ---------------------------------------------------------------- network (Eq. 1)
  const int net = Ly.nets > 1 ? ti : 0;
  const float* W0 = TC ? nullptr : sm + Ly.off_W0 + net * Ly.H * DP;  // FP32 network only
  const float* b0 = sm + (Ly.off_b0 - w0n) + net * Ly.H;
  const float* w1 = sm + (Ly.off_w1 - w0n) + net * Ly.H;
  const float* sc = sm + (Ly.off_scaler - w0n);
  float e[DP];
  float U = -sm[Ly.off_b1 - w0n + net];
  if constexpr (TC) {
    // z = W0 s on the tensor cores: A = s (bf16, one row per atom), B1 = W0,
    // D (F32) in TMEM columns [32 net, 32 net + 32); then e = W0^T v likewise.
    static_assert(DP <= 32, "the tensor-core network takes at most 32 descriptor components");
    const int warp = tid >> 5;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 32);
    const uint32_t a_base = tc::smem_addr(tileA);
    // row `tid` of A: columns 0-31 the bf16 rounding of v, 32-63 the remainder
    auto write_row = [&](const float* v) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        __nv_bfloat162 hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float x0 = v[8 * c + 2 * u], x1 = v[8 * c + 2 * u + 1];
          hi[u] = __floats2bfloat162_rn(x0, x1);
          lo[u] = __floats2bfloat162_rn(x0 - __low2float(hi[u]), x1 - __high2float(hi[u]));
        }
        unsigned char* base = reinterpret_cast<unsigned char*>(tileA);
        *reinterpret_cast<uint4*>(base + tc::kmajor_offset(tid, 8 * c, 64)) = *reinterpret_cast<uint4*>(hi);
        if constexpr (TCM == 2)
          *reinterpret_cast<uint4*>(base + tc::kmajor_offset(tid, 32 + 8 * c, 64)) = *reinterpret_cast<uint4*>(lo);
      }
    };
    // D = sum over (A block, B block) pairs: TCM 1: (hi, hi) -- plain BF16
    // operands; TCM 2: (hi, hi) + (hi, lo) + (lo, hi) -- both operands to ~2^-17.
    auto gemm = [&](const __nv_bfloat16* B, uint32_t parity) -> bool {
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        constexpr int NPAIR = TCM == 2 ? 3 : 1;
        const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};
        for (int t = 0; t < Ly.nets; ++t) {
          const uint32_t b_base = tc::smem_addr(B + t * 2048);
          int step = 0;
          for (int q2 = 0; q2 < NPAIR; ++q2)
#pragma unroll
            for (int ks = 0; ks < 2; ++ks, ++step)
              tc::mma_bf16(tmem_base + 32 * t, tc::smem_desc(a_base + 512 * pa[q2] + 256 * ks, 128, 1024),
                           tc::smem_desc(b_base + 512 * pb[q2] + 256 * ks, 128, 1024), idesc, step > 0);
        }
        tc::commit_to(mbar);
      }
      // every thread polls the mbarrier itself; the barrier-and makes the
      // give-up decision the same for the whole CTA
      const bool ok = __syncthreads_and(tc::mbar_wait_bounded(mbar, parity, a.wait_tries)) != 0;
      tc::fence_after_sync();
      return ok;
    };
    auto read_row = [&](float* v) {
      for (int t = 0; t < Ly.nets; ++t) {
        float r[32];
        tc::tmem_ld32(tmem_base + ((uint32_t)(32 * warp) << 16) + 32 * t, r);
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = (t == net) ? r[k] : v[k];
      }
    };
    float buf[32];
#pragma unroll
    for (int d = 0; d < 32; ++d) buf[d] = d < DP ? q[d] * sc[d] : 0.f;
    write_row(buf);
    // Give-up path: when a product's completion does not arrive in time, the
    // CTA reads no TMEM, rewrites no operand tile and issues no further
    // product (an unfinished product may still read the tile and write its
    // columns).  It raises TNEP_ERR_TIMEOUT, waits once more (bounded) for
    // that completion, frees its columns only if it arrived -- a late write
    // can then never land in columns that another CTA has since been given
    // -- and returns without storing a result.  If the completion never
    // arrives, the CTA exits with its columns still allocated rather than
    // free columns a product may still write; the host gets TNEP_ERR_TIMEOUT.
    // The product waits use the context's limit (TNEP_OPT_WAIT_TRIES); the
    // drain always uses the default one, so that a small limit only makes
    // the call give up, never leaves TMEM allocated.
    uint32_t pending = 0;  // parity of the product whose completion is awaited
    bool ok = gemm(tileB1, 0);
    float z[32];
    if (ok) {
      // the next work item; its latency is hidden behind the network
      int nxt = 0;
      if (tid == 0) nxt = (int)gridDim.x + atomicAdd(&a.status->work_next, 1);
#pragma unroll
      for (int k = 0; k < 32; ++k) z[k] = 0.f;
      read_row(z);
#pragma unroll
      for (int h = 0; h < 32; ++h) {
        if (h < Ly.H) {
          const float hh = tanhf(z[h] - b0[h]);
          const float wh = w1[h];
          U += wh * hh;
          buf[h] = wh * (1.f - hh * hh);
        } else {
          buf[h] = 0.f;
        }
      }
      // the first product has completed, so the A tile may be rewritten; its
      // TMEM columns are rewritten only by the second product, which is
      // issued after the CTA-wide barrier in gemm, i.e. after every warp's
      // tcgen05.ld (each followed by tcgen05.wait::ld) above
      write_row(buf);
      // published before the second product's barrier; read after the item,
      // and rewritten only after the next item's first barrier
      if (tid == 0) *next_item = nxt;
      pending = 1;
      ok = gemm(tileB2, 1);
    }
    if (!ok) {
      if (tid == 0 && a.status) atomicCAS(&a.status->error, 0, TNEP_ERR_TIMEOUT);
      const bool drained = __syncthreads_and(tc::mbar_wait_bounded(mbar, pending, kMbarTries)) != 0;
      if (drained) {
        tc::fence_after_sync();
        tc::fence_before_sync();
        __syncthreads();
        if (tid < 32) tc::tmem_dealloc(tmem_base, tc_tmem_cols(Ly.nets));
      }
      return false;
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) z[k] = 0.f;
    read_row(z);
#pragma unroll
    for (int d = 0; d < DP; ++d) e[d] = z[d] * sc[d];
  } else if constexpr (FACT) {
    // scalar products: measured faster than the packed form below in the
    // factored population kernel
    float s[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) { s[d] = q[d] * sc[d]; e[d] = 0.f; }
    for (int h = 0; h < Ly.H; ++h) {
      const float4* row = reinterpret_cast<const float4*>(W0 + h * DP);
      float z = -b0[h];
#pragma unroll
      for (int v = 0; v < DP / 4; ++v) {
        const float4 w = row[v];
        z += w.x * s[4 * v] + w.y * s[4 * v + 1] + w.z * s[4 * v + 2] + w.w * s[4 * v + 3];
      }
      const float hh = tanhf(z);
      const float wh = w1[h];
      U += wh * hh;
      const float vh = wh * (1.f - hh * hh);
#pragma unroll
      for (int v = 0; v < DP / 4; ++v) {
        const float4 w = row[v];
        e[4 * v] += vh * w.x; e[4 * v + 1] += vh * w.y; e[4 * v + 2] += vh * w.z; e[4 * v + 3] += vh * w.w;
      }
    }
#pragma unroll
    for (int d = 0; d < DP; ++d) e[d] *= sc[d];
  } else {
    // both products in descriptor pairs with packed multiply-adds: z from
    // partial sums over alternate pairs, e accumulated pairwise
    f32x2 s2[DP / 2], e2[DP / 2];
#pragma unroll
    for (int v = 0; v < DP / 2; ++v) {
      s2[v] = pk2(q[2 * v] * sc[2 * v], q[2 * v + 1] * sc[2 * v + 1]);
      e2[v] = 0ull;
    }
    for (int h = 0; h < Ly.H; ++h) {
      const float4* row = reinterpret_cast<const float4*>(W0 + h * DP);
      // four independent partial sums keep the dependency chains short
      f32x2 z2[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
      for (int v = 0; v < DP / 4; ++v) {
        const float4 w = row[v];
        z2[v & 1] = fma2(pk2(w.x, w.y), s2[2 * v], z2[v & 1]);
        z2[2 + (v & 1)] = fma2(pk2(w.z, w.w), s2[2 * v + 1], z2[2 + (v & 1)]);
      }
      float zp[8];
#pragma unroll
      for (int u = 0; u < 4; ++u) unpk2(z2[u], zp[2 * u], zp[2 * u + 1]);
      const float zs = ((zp[0] + zp[1]) + (zp[2] + zp[3])) + ((zp[4] + zp[5]) + (zp[6] + zp[7]));
      const float hh = tanhf(zs - b0[h]);
      const float wh = w1[h];
      U += wh * hh;
      const float vh = wh * (1.f - hh * hh);
      const f32x2 vv = pk2(vh, vh);
#pragma unroll
      for (int v = 0; v < DP / 4; ++v) {
        const float4 w = row[v];
        e2[2 * v] = fma2(vv, pk2(w.x, w.y), e2[2 * v]);
        e2[2 * v + 1] = fma2(vv, pk2(w.z, w.w), e2[2 * v + 1]);
      }
    }
#pragma unroll
    for (int v = 0; v < DP / 2; ++v) {
      unpk2(e2[v], e[2 * v], e[2 * v + 1]);
      e[2 * v] *= sc[2 * v];
      e[2 * v + 1] *= sc[2 * v + 1];
    }
  }

  float acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = 0.f;

  // ---------------------------------------------------------------- radial part of Eqs. 3-4
  // dU_i/dr_ij (radial) = (sum_k D^{t_j}_k f_k'(r)) r_ij / r with
  // D^t_k = sum_n (dU/dq_n) c^{t_i t}_{nk}; contracted through the moments:
  //   rank 1: mu_i    -= sum_{t,k} D^t_k V^t_k
  //   rank 2: alpha_i -= sum_{t,k} D^t_k W^t_k
  for (int t = 0; t < T; ++t) {
    float cc[NBR4];
    load_coeffs<NR, BR>(cR_i + t * Ly.stride_cR, cc);
#pragma unroll
    for (int k = 0; k < BR; ++k) {
      float Dk = 0.f;
#pragma unroll
      for (int n = 0; n < NR; ++n) Dk += e[n] * cc[n * BR + k];
      const int tk = t * kMomBasis + k;
      if constexpr (RANK == 1) {
        const float* v = mom + (size_t)(a.v0 + 3 * tk) * a.mom_stride;
        acc[0] -= Dk * v[0];
        acc[1] -= Dk * v[(size_t)a.mom_stride];
        acc[2] -= Dk * v[2 * (size_t)a.mom_stride];
      } else {
        const float* w = mom + (size_t)(a.w0 + 6 * tk) * a.mom_stride;
        const size_t ms = a.mom_stride;
        const float wxx = w[0], wxy = w[ms], wxz = w[2 * ms], wyy = w[3 * ms], wyz = w[4 * ms], wzz = w[5 * ms];
        acc[0] -= Dk * wxx; acc[1] -= Dk * wxy; acc[2] -= Dk * wxz;
        acc[3] -= Dk * wxy; acc[4] -= Dk * wyy; acc[5] -= Dk * wyz;
        acc[6] -= Dk * wxz; acc[7] -= Dk * wyz; acc[8] -= Dk * wzz;
      }
    }
  }

  // ---------------------------------------------------------------- angular backward
  {
    float G[NA * NLM];
#pragma unroll
    for (int n = 0; n < NA; ++n) {
#pragma unroll
      for (int lm = 0; lm < NLM; ++lm)
        G[n * NLM + lm] = 2.f * wlm(lm) * e[NR + (l_of(lm) - 1) * NA + n] * scratch[(n * NLM + lm) * BLK];
      if constexpr (FB) {
        float a2[5], gr[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) a2[m] = scratch[(n * NLM + 3 + m) * BLK];
        trace_m3(a2, gr);
        const float e4 = kC4 * e[NR + LMAX * NA + n];
#pragma unroll
        for (int m = 0; m < 5; ++m) G[n * NLM + 3 + m] += e4 * gr[m];
      }
    }
    // G in lm pairs for the packed products of the pair walk
    constexpr int NP = NLM / 2;
    f32x2 G2[NA * NP];
#pragma unroll
    for (int n = 0; n < NA; ++n)
#pragma unroll
      for (int q = 0; q < NP; ++q) G2[n * NP + q] = pk2(G[n * NLM + 2 * q], G[n * NLM + 2 * q + 1]);
    if constexpr (FACT) {
      constexpr int CC = RANK == 1 ? 3 : 9;
      constexpr int NLMP = pad4(NLM), GBP = pad4(NLM * CC);
      const float4* m4 = reinterpret_cast<const float4*>(a.amom) + (size_t)(i >> 5) * (a.amom_slots / 4) * 32 + (i & 31);
      const int gbase4 = T * BA * NLMP / 4;
      for (int t = 0; t < T; ++t) {
        const float* cblk = cA_i + t * Ly.stride_cA;
#pragma unroll 1
        for (int k = 0; k < BA; ++k) {
          float ck[NA];
#pragma unroll
          for (int n = 0; n < NA; ++n) ck[n] = cblk[n * BA + k];
          const float4* g = m4 + (size_t)(gbase4 + (t * BA + k) * (GBP / 4)) * 32;
          if (t * BA + k + 1 < T * BA) {
#pragma unroll
            for (int q = 0; q < GBP / 4; ++q)
              asm volatile("prefetch.global.L1 [%0];" ::"l"(g + (size_t)(GBP / 4 + q) * 32));
          }
          // four lm at a time: their 4 * CC slots are CC float4 groups
#pragma unroll
          for (int l0 = 0; l0 < NLM; l0 += 4) {
            const int nv = (GBP - l0 * CC) / 4 < CC ? (GBP - l0 * CC) / 4 : CC;
            float vals[4 * CC];
#pragma unroll
            for (int q = 0; q < CC; ++q) {
              if (q < nv) {
                const float4 v = g[(size_t)(l0 * CC / 4 + q) * 32];
                vals[4 * q] = v.x; vals[4 * q + 1] = v.y; vals[4 * q + 2] = v.z; vals[4 * q + 3] = v.w;
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int lm = l0 + u;
              if (lm < NLM) {
                float h = 0.f;
#pragma unroll
                for (int n = 0; n < NA; ++n) h += G[n * NLM + lm] * ck[n];
#pragma unroll
                for (int c = 0; c < CC; ++c) acc[c] -= h * vals[u * CC + c];
              }
            }
          }
        }
      }
    }
    constexpr int NQ = pair_cache_quads(NA);
    NbrWalk wB(a.nbr_A, a.pos4, i, a.cap_A, 0, (FACT || PC) ? 0 : nA, pi);
    // cached pairs: the next pair's quads are loaded one iteration ahead
    const float4* pcs = PC ? a.pcache + i_raw : nullptr;  // own slots also past the end (tensor-core path)
    float4 nxt[PC ? NQ : 1];
    if constexpr (PC) {
      if (nA > 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) nxt[q] = __ldcs(pcs + (size_t)q * a.pc_stride);
      }
    }
    for (int kk = 0; kk < (FACT ? 0 : nA); ++kk) {
      float dx, dy, dz, rinv;
      float g[NA], dg[NA];
      if constexpr (PC) {
        float v[4 * NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          v[4 * q] = nxt[q].x; v[4 * q + 1] = nxt[q].y; v[4 * q + 2] = nxt[q].z; v[4 * q + 3] = nxt[q].w;
        }
        // pair kk + 2 towards L1 (the register copy is one pair ahead)
        if (kk + 2 < nA) {
          const float4* pf = pcs + (size_t)(kk + 2) * NQ * a.pc_stride;
#pragma unroll
          for (int q = 0; q < NQ; ++q) asm volatile("prefetch.global.L1 [%0];" ::"l"(pf + (size_t)q * a.pc_stride));
        }
        if (kk + 1 < nA) {
          const float4* src = pcs + (size_t)(kk + 1) * NQ * a.pc_stride;
#pragma unroll
          for (int q = 0; q < NQ; ++q) nxt[q] = __ldcs(src + (size_t)q * a.pc_stride);
        }
        dx = v[0]; dy = v[1]; dz = v[2]; rinv = v[3];
#pragma unroll
        for (int n = 0; n < NA; ++n) { g[n] = v[4 + n]; dg[n] = v[4 + NA + n]; }
      } else {
        const float4 pj = wB.next(kk);
        dx = min_image(pj.x, pi.x, bx.L[0], bx.invL[0]);
        dy = min_image(pj.y, pi.y, bx.L[1], bx.invL[1]);
        dz = min_image(pj.z, pi.z, bx.L[2], bx.invL[2]);
        const float r2w = dx * dx + dy * dy + dz * dz;
        rinv = rsqrtf(r2w);
        const float r = r2w * rinv;
        float f[BA], df[BA];
        basis_fwd_bwd<BA>(r, rcAinv, f, df);
        float cc[NBA4];
        load_coeffs<NA, BA>(cA_i + __float_as_int(pj.w) * Ly.stride_cA, cc);
#pragma unroll
        for (int n = 0; n < NA; ++n) {
          float s0 = 0.f, s1 = 0.f;
#pragma unroll
          for (int k = 0; k < BA; ++k) { s0 += cc[n * BA + k] * f[k]; s1 += cc[n * BA + k] * df[k]; }
          g[n] = s0; dg[n] = s1;
        }
      }
      const float r2 = dx * dx + dy * dy + dz * dz;
      const float ux = dx * rinv, uy = dy * rinv, uz = dz * rinv;
      float p[NLM];
      real_harmonics<LMAX>(ux, uy, uz, p);
      // S_lm = sum_n G_nlm g_n; sum_lm T_lm p_lm = sum_n g'_n P_n with
      // P_n = sum_lm G_nlm p_lm.  Both run over lm pairs with packed
      // multiply-adds; P_n is summed as its even-lm and odd-lm halves.
      float S[NLM];
      f32x2 gg[NA], P2[NA];
#pragma unroll
      for (int n = 0; n < NA; ++n) { gg[n] = pk2(g[n], g[n]); P2[n] = 0ull; }
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const f32x2 pq = pk2(p[2 * q], p[2 * q + 1]);
        f32x2 sv = 0ull;
#pragma unroll
        for (int n = 0; n < NA; ++n) {
          sv = fma2(G2[n * NP + q], gg[n], sv);
          P2[n] = fma2(G2[n * NP + q], pq, P2[n]);
        }
        unpk2(sv, S[2 * q], S[2 * q + 1]);
      }
      float P[NA];
#pragma unroll
      for (int n = 0; n < NA; ++n) {
        float lo, hi;
        unpk2(P2[n], lo, hi);
        P[n] = lo + hi;
      }
      if constexpr (NLM & 1) {
        float sv = 0.f;
#pragma unroll
        for (int n = 0; n < NA; ++n) {
          sv += G[n * NLM + NLM - 1] * g[n];
          P[n] += G[n * NLM + NLM - 1] * p[NLM - 1];
        }
        S[NLM - 1] = sv;
      }
      float srad = 0.f;
#pragma unroll
      for (int n = 0; n < NA; ++n) srad += dg[n] * P[n];
      float vx = 0.f, vy = 0.f, vz = 0.f;
      harmonic_grad<LMAX>(S, ux, uy, uz, vx, vy, vz);
      const float uv = ux * vx + uy * vy + uz * vz;
      const float fx = srad * ux + rinv * (vx - uv * ux);
      const float fy = srad * uy + rinv * (vy - uv * uy);
      const float fz = srad * uz + rinv * (vz - uv * uz);
      if constexpr (RANK == 1) {
        acc[0] -= r2 * fx; acc[1] -= r2 * fy; acc[2] -= r2 * fz;
      } else {
        acc[0] -= dx * fx; acc[1] -= dx * fy; acc[2] -= dx * fz;
        acc[3] -= dy * fx; acc[4] -= dy * fy; acc[5] -= dy * fz;
        acc[6] -= dz * fx; acc[7] -= dz * fy; acc[8] -= dz * fz;
      }
    }
  }

  // ---------------------------------------------------------------- per-atom output
  if (valid) {
    float* out = a.per_atom + (size_t)pop * a.per_atom_stride;
    if constexpr (RANK == 2) { acc[0] += U; acc[4] += U; acc[8] += U; }
#pragma unroll
    for (int c = 0; c < C; ++c) out[(size_t)c * a.atom_stride + i] = acc[c];
  }
  return true;
  };

  if constexpr (TC) {
    int loaded = -1;
    for (int wi = blockIdx.x; wi < n_work;) {
      const int pop = a.pop_major ? wi % a.n_pop : wi / nblk;
      const int ablk = a.pop_major ? wi / a.n_pop : wi % nblk;
      if (pop != loaded) {
        __syncthreads();  // every thread is done with the previous model and tiles
        load_model(pop);
        loaded = pop;
      }
      if (!item(pop, ablk)) return;
      wi = *next_item;
    }
    // every warp's last tcgen05.ld has completed (tcgen05.wait::ld in tmem_ld32)
    tc::fence_before_sync();
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(tmem_base, tc_tmem_cols(Ly.nets));
  } else {
    // grid (atom blocks, individuals), or (individuals, atom blocks) with pop_major
    const int pop = a.pop_major ? blockIdx.x : blockIdx.y;
    load_model(pop);
    item(pop, a.pop_major ? blockIdx.y : blockIdx.x);
  }
}

// One CTA per work item (atom block, individual), or, for the tensor-core
// network, persistent CTAs: two per SM (what fits; the runtime's occupancy
// figure for this kernel is one, but two are resident), extra ones exit at once.
template <int NR, int NA, int BR, int BA, int LMAX, bool FB, int BLK, int TCM, bool FACT = false, bool PC = false>
cudaError_t launch_block(int rank, const FusedArgs& a_in, int n_pop, size_t smem, cudaStream_t st) {
  FusedArgs a = a_in;
  a.n_pop = n_pop;
  const long long n_work = (long long)((a.n_atoms + BLK - 1) / BLK) * n_pop;
  if (n_work > INT_MAX) return cudaErrorInvalidConfiguration;
  auto fn = rank == 1 ? k_fused<NR, NA, BR, BA, LMAX, FB, 1, BLK, TCM, FACT, PC>
                      : k_fused<NR, NA, BR, BA, LMAX, FB, 2, BLK, TCM, FACT, PC>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid;
  if constexpr (TCM != 0) {
    if (!a.status) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    grid = dim3((unsigned)std::min<long long>(n_work, 2LL * sms));
    e = cudaMemsetAsync(&a.status->work_next, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
  } else {
    const int nblk = (a.n_atoms + BLK - 1) / BLK;
    if (a.pop_major && nblk > 65535) return cudaErrorInvalidConfiguration;
    if (!a.pop_major && n_pop > 65535) return cudaErrorInvalidConfiguration;
    grid = a.pop_major ? dim3(n_pop, nblk) : dim3(nblk, n_pop);
  }
  fn<<<grid, BLK, smem, st>>>(a);
  return cudaGetLastError();
}

template <int NR, int NA, int BR, int BA, int LMAX, bool FB>
cudaError_t launch_variant(int rank, const FusedArgs& a, int n_pop, int block, int tcm, size_t smem,
                           cudaStream_t st) {
  if (a.amom && tcm == 0) {
    if (block == 64) return launch_block<NR, NA, BR, BA, LMAX, FB, 64, 0, true>(rank, a, n_pop, smem, st);
    return launch_block<NR, NA, BR, BA, LMAX, FB, 128, 0, true>(rank, a, n_pop, smem, st);
  }
  // the pair cache holds one individual's pairs
  if (a.pcache && n_pop == 1 && !a.amom && (block == 128 || tcm != 0)) {
    if (tcm == 1) return launch_block<NR, NA, BR, BA, LMAX, FB, 128, 1, false, true>(rank, a, n_pop, smem, st);
    if (tcm == 2) return launch_block<NR, NA, BR, BA, LMAX, FB, 128, 2, false, true>(rank, a, n_pop, smem, st);
    return launch_block<NR, NA, BR, BA, LMAX, FB, 128, 0, false, true>(rank, a, n_pop, smem, st);
  }
  if (tcm == 1) return launch_block<NR, NA, BR, BA, LMAX, FB, 128, 1>(rank, a, n_pop, smem, st);
  if (tcm == 2) return launch_block<NR, NA, BR, BA, LMAX, FB, 128, 2>(rank, a, n_pop, smem, st);
  if (block == 64) return launch_block<NR, NA, BR, BA, LMAX, FB, 64, 0>(rank, a, n_pop, smem, st);
  return launch_block<NR, NA, BR, BA, LMAX, FB, 128, 0>(rank, a, n_pop, smem, st);
}

}  // namespace

static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

int variant_of(int nR, int nA, int bR, int bA, int lmax, int fb) {
  if (nR == 5 && nA == 5 && bR == 9 && bA == 9 && lmax == 4 && fb) return kVarStd;
  if (nR == 4 && nA == 3 && bR == 7 && bA == 6 && lmax == 3 && fb) return kVarSmall;
  return -1;
}

size_t fused_smem_bytes(int variant, const ModelLayout& lay, int block, int tcm) {
  const bool tc = tcm != 0;
  int slots = 0;
  if (variant == kVarStd) slots = 5 * 24;
  if (variant == kVarSmall) slots = 3 * 15;
  if (tc) block = 128;
  return (size_t)(smem_layout(lay, tc).words + slots * block) * sizeof(float) + (tc ? tc_smem_bytes(lay.nets) : 0);
}

cudaError_t launch_fused(int variant, int rank, const FusedArgs& a, int n_pop, int block, int tcm,
                         cudaStream_t st) {
  if (a.n_atoms <= 0 || n_pop <= 0) return cudaSuccess;
  if (block != 64 && block != 128) return cudaErrorInvalidValue;
  if (tcm < 0 || tcm > 2) return cudaErrorInvalidValue;
  count_launches(1);
  const size_t smem = fused_smem_bytes(variant, a.lay, block, tcm);
  switch (variant) {
    case kVarStd: return launch_variant<5, 5, 9, 9, 4, true>(rank, a, n_pop, block, tcm, smem, st);
    case kVarSmall: return launch_variant<4, 3, 7, 6, 3, true>(rank, a, n_pop, block, tcm, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tnep
