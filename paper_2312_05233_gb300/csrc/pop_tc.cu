// Population evaluation with the angular contractions on the tensor cores.
//
// Sec. II.D: the evolution strategy evaluates a population of parameter
// vectors on the training structures every generation.  g^A_n is linear in
// the angular coefficients c, so for a centre atom i of type tau and an
// individual p (angmom.cu holds the per-atom moments B and Phi / Psi):
//   A_{p,n,lm}(i)    = sum_{(t,k)} c^{tau t}_{p,n,k} B^t_{k,lm}(i)
// and the angular share of Eqs. 3-4, with G = dU/dA and
// H^t_{k,lm} = sum_n G_nlm c_nk, is
//   -sum_{t,k,lm} H^t_{k,lm} Phi^t_{k,lm,c}(i) = -sum_n sum_lm G_{p,n,lm} X_{p,n,lm,c}(i),
//   X_{p,n,lm,c}(i)  = sum_{(t,k)} c^{tau t}_{p,n,k} Phi^t_{k,lm,c}(i).
// Both A and X are dense products with the same left operand
// C[(p, n)][(t, k)] (one 128-row tile holds 25 individuals x 5 orders n;
// K = T * 9 <= 32) and the atoms' moments as the right operand: rows (i, lm)
// for A, rows (lm, c) for X.  They run as tcgen05.mma (kind::f16, BF16
// operands, FP32 accumulation in TMEM).  For FP32 accuracy every operand is
// split into three BF16 terms, x = x1 + x2 + x3 (|x - x1 - x2 - x3| <= 2^-24
// |x|), and the six products whose order is <= 2 are accumulated
// (x1 y1, x1 y2, x2 y1, x1 y3, x2 y2, x3 y1; the rest is below 2^-24).
//
// One CTA (128 threads) takes one tile of 5 atoms of one centre type and 25
// individuals.  TMEM lane r = 5 p + n holds row (p, n).
//   1. bulk copies (cp.async.bulk, mbarrier) of the coefficient tile and of
//      the 5 atoms' B blocks; one product A for all 5 atoms (N = 128
//      columns); lane (p, n) reads its A_{n,lm}(i) and forms q_nl and the
//      4-body term of its n for each atom.  As soon as the product has read
//      its operands, the 25 individuals' W0 blocks are bulk-copied over them.
//   2. thread (p, i): radial descriptor from the radial moments; the FP32
//      network (Eq. 1) on the staged weights (b0, w1 in the rows' padding
//      columns; packed multiply-adds over descriptor pairs), dU/dq written
//      over the descriptor row; the radial part of
//      Eqs. 3-4.  Meanwhile the coefficient tile and the B blocks are loaded
//      again, with the first round's Phi / Psi blocks.
//   3. rounds of AG atoms (2 for rank 1, 1 for rank 2): the product A again
//      (N = 32 or 48) and X over the round's Phi / Psi rows (N = 144 or
//      224); lane (p, n) forms G_{n,lm} and its partial contraction; thread
//      (p, i) sums the five n in a fixed order and writes the per-atom
//      tensor.  The next round's copy starts once this round's products
//      have read their buffer.
// Each structure's per-atom results depend only on its atoms, so the usual
// FP64 per-structure reduction follows.  All waits are bounded; on give-up
// the CTA raises TNEP_ERR_TIMEOUT, issues nothing further, waits (bounded)
// for what it has in flight, frees TMEM only if that arrived and stores
// nothing.

#include <cuda_bf16.h>

#include "tc_sm100.cuh"
#include "tnep_device.cuh"
#include "tnep_internal.cuh"

namespace tnep {

namespace {

// hidden units per iteration of the per-thread network loop (best of 1, 2,
// 3, 5, 6 measured)
constexpr int kNetUnroll = 6;
constexpr int kPT = kPopTcIndividuals;  // individuals per 128-row tile (125 rows used)
constexpr int kNT = kPopTcAtoms;        // atoms per CTA
constexpr int kKW = 96;                 // bf16 per operand row: three terms x K = 32
constexpr int kGroup = 8 * kKW * 2;     // bytes of 8 rows
constexpr int kBBytes = 3 * kGroup;     // one atom's B block: 24 rows (lm)
// Phase 3 works in rounds of AG atoms (2 for rank 1, 1 for rank 2): one
// product A over their 24 AG rows of B and one product X over their rows
// (lm, c) of the Phi / Psi blocks, 72 per atom for rank 1 and 216 for rank
// 2.  Each N is rounded up to a multiple of 16; the extra rows read whatever
// follows in shared memory into result columns that are never read.
template <int RANK> constexpr int x_rows() { return RANK == 1 ? 72 : 216; }
template <int RANK> constexpr int x_bytes() { return x_rows<RANK>() / 8 * (8 * 96 * 2); }
template <int RANK> constexpr int round_atoms() { return RANK == 1 ? 2 : 1; }
constexpr int kCoefBytes = 16 * kGroup;  // 128 rows
constexpr int kW0Bytes = 30 * 128;      // one individual's W0 (30 rows x 32 floats), staged in phase 2
constexpr long long kTries = 1LL << 22;

// smem layout (bytes)
constexpr int kOffC = 0;
constexpr int kOffB = kOffC + kCoefBytes;              // 16 groups: 5 atoms x 3 + one pad group
constexpr int kOffX0 = kOffB + 16 * kGroup;            // the X buffer of one round
// the n-sums of one round, float [AG][25][5][C], after the X buffer
template <int RANK> constexpr int off_nsum() { return kOffX0 + round_atoms<RANK>() * x_bytes<RANK>(); }
template <int RANK> constexpr int nsum_bytes() { return round_atoms<RANK>() * kPT * 5 * (RANK == 1 ? 3 : 9) * 4; }
// Phase 2 stages the 25 individuals' W0 over [0, kW0Area): individual p at
// p * kW0Stride (30 rows of 128 B; the stride is 16 B more than the block so
// that the threads of a warp, which take up to 8 individuals, read rows of
// different individuals from different banks).  Column 30 of row h holds
// b0_h and column 31 holds w1_h (the weights there are zero padding).
constexpr int kW0Stride = kW0Bytes + 16;
constexpr int kW0Area = ((kPT * kW0Stride + 127) / 128) * 128;
// rows of 36 floats (s, then e; slot 30: U): a stride of 144 B puts the rows
// read by eight consecutive threads in different banks
constexpr int kQS = 36;
constexpr int kOffQ = kW0Area;                           // float [25][5][kQS]
constexpr int kOffBar = kOffQ + kPT * kNT * kQS * 4;    // 6 mbarriers + TMEM slot + flag
constexpr int kSmemBytes = kOffBar + 64;
static_assert(kW0Area >= off_nsum<1>() + nsum_bytes<1>() && kW0Area >= off_nsum<2>() + nsum_bytes<2>(),
              "the W0 area covers the operand, X and n-sum buffers");
static_assert(kOffQ % 16 == 0 && kOffBar % 8 == 0, "alignment");

__device__ __forceinline__ uint32_t tile_off(int row, int part, int k) {
  return tc::kmajor_offset(row, part * 32 + k, kKW);
}

// x = x1 + x2 + x3 in BF16; each residual is exact in FP32.
__device__ __forceinline__ void split3(float x, __nv_bfloat16* t) {
  t[0] = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(t[0]);
  t[1] = __float2bfloat16_rn(r1);
  t[2] = __float2bfloat16_rn(r1 - __bfloat162float(t[1]));
}

// Writes one operand row (32 K values, three terms) in the canonical layout.
__device__ __forceinline__ void store_row(unsigned char* tile, int row, const float* v) {
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    __nv_bfloat16 h[3][8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      __nv_bfloat16 t[3];
      split3(v[8 * kc + u], t);
      h[0][u] = t[0]; h[1][u] = t[1]; h[2][u] = t[2];
    }
#pragma unroll
    for (int part = 0; part < 3; ++part)
      *reinterpret_cast<uint4*>(tile + tile_off(row, part, 8 * kc)) = *reinterpret_cast<const uint4*>(h[part]);
  }
}

// Per-atom moment blocks in the tensor-core layout: B (24 rows lm), then Phi
// (rank 1) or Psi (rank 2) (24 * C rows (lm, c)); K = (t, k), zero beyond T * 9.
// Atom n_atoms is an all-zero block (padding of partial tiles).
__global__ void __launch_bounds__(128) k_moments_tc(int n_atoms, int T, int C, const float* __restrict__ amom,
                                                    int amom_slots, unsigned char* __restrict__ dst,
                                                    size_t stride) {
  const int rows = 24 + 24 * C;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)(n_atoms + 1) * rows) return;
  const int a = (int)(g / rows), row = (int)(g % rows);
  const int GBP = pad4(24 * C);
  float v[32];
#pragma unroll
  for (int kk = 0; kk < 32; ++kk) {
    const int t = kk / 9, k = kk % 9;
    float x = 0.f;
    if (a < n_atoms && t < T) {
      const int slot = row < 24 ? (t * 9 + k) * 24 + row : T * 9 * 24 + (t * 9 + k) * GBP + (row - 24);
      x = amom[amom_index(a, slot, amom_slots)];
    }
    v[kk] = x;
  }
  unsigned char* blk = dst + (size_t)a * stride;
  if (row < 24) store_row(blk, row, v);
  else store_row(blk + kBBytes, row - 24, v);
}

// Per generation: the left operand C[(p, n)][(t, k)] of every (centre type,
// individual tile), rows p * 5 + n (zero beyond the population and K).
__global__ void __launch_bounds__(128) k_coef_tc(int n_pop, int T, int n_mt, const float* __restrict__ params,
                                                 int words, int off_cA, int stride_cA, unsigned char* __restrict__ dst) {
  const int tau = blockIdx.x / n_mt, mt = blockIdx.x % n_mt;
  const int r = threadIdx.x;
  const int pl = r / 5, n = r % 5, p = mt * kPT + pl;
  const bool valid = r < kPT * 5 && p < n_pop;
  float v[32];
#pragma unroll
  for (int kk = 0; kk < 32; ++kk) {
    const int t = kk / 9, k = kk % 9;
    v[kk] = (valid && t < T) ? params[(size_t)p * words + off_cA + (tau * T + t) * stride_cA + n * 9 + k] : 0.f;
  }
  store_row(dst + (size_t)blockIdx.x * kCoefBytes, r, v);
}

// Issues the six split products of one K = 32 operand pair into `d`.
__device__ __forceinline__ void issue_split_products(uint32_t d, uint32_t a_base, uint32_t b_base, uint32_t idesc) {
  const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
  int step = 0;
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int q = 0; q < 6; ++q, ++step)
      tc::mma_bf16(d, tc::smem_desc(a_base + 512 * pa[q] + 256 * ks, 128, kGroup),
                   tc::smem_desc(b_base + 512 * pb[q] + 256 * ks, 128, kGroup), idesc, step > 0);
}

template <int RANK>
__global__ void __launch_bounds__(128, 2) k_pop_tc(const __grid_constant__ PopTcArgs a) {
  constexpr int C = RANK == 1 ? 3 : 9;
  constexpr int AG = round_atoms<RANK>(), NROUND = (kNT + AG - 1) / AG;
  constexpr int XR = x_rows<RANK>(), XB = x_bytes<RANK>();
  constexpr int XN = (AG * XR + 15) / 16 * 16, AN = (AG * 24 + 15) / 16 * 16;
  constexpr uint32_t TCOLS = 256;
  static_assert(AN + XN <= (int)TCOLS, "one round fits the TMEM allocation");
  constexpr int NR = 5, NA = 5, BR = 9, NLM = 24, DP = 32;
  extern __shared__ __align__(16) unsigned char smem[];
  float* qbuf = reinterpret_cast<float*>(smem + kOffQ);
  float* nsum = reinterpret_cast<float*>(smem + off_nsum<RANK>());
  // mbarriers (each has at most one phase outstanding, so its k-th use
  // completes with parity k & 1): bulk loads of the coefficient tile and B
  // blocks (phase 1, again for phase 3), the first product, the X copy of
  // each round, the weight blocks of phase 2, the products of each round
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kOffBar + 48);
  const uint32_t s_base = tc::smem_addr(smem);
  const uint32_t bar_load = tc::smem_addr(&bars[0]), bar_mma = tc::smem_addr(&bars[1]);
  const uint32_t bar_x = tc::smem_addr(&bars[2]), bar_w = tc::smem_addr(&bars[3]);
  const uint32_t bar_r = tc::smem_addr(&bars[4]);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int tile = blockIdx.x / a.n_mt, mt = blockIdx.x % a.n_mt;
  const int* td = a.tiles + (size_t)tile * 8;
  const int tau = td[5], count = td[6];
  const int pl = tid / 5, x = tid % 5;            // (individual, n) in phases 1 and 3; (individual, atom) in 2
  const int p = mt * kPT + pl;
  const bool prow = tid < kPT * 5 && p < a.n_pop;  // a real (individual, .) row
  const int T = a.n_types;
  const size_t xs = a.mom_tc_stride;
  auto atom_of = [&](int i) { return td[i]; };      // a.n_atoms (zero block) for empty slots
  auto x_src = [&](int i) { return a.mom_tc + (size_t)atom_of(i) * xs + kBBytes; };
  // thread 0: bulk copies of round r's X blocks (the zero block past the tile)
  auto load_round = [&](int r) {
    tc::mbar_expect_tx(bar_x, AG * XB);
    for (int ia = 0; ia < AG; ++ia) {
      const int i = AG * r + ia;
      tc::bulk_g2s(s_base + kOffX0 + ia * XB, i < kNT ? x_src(i) : a.mom_tc + (size_t)a.n_atoms * xs + kBBytes,
                   XB, bar_x);
    }
  };

  // ---------------------------------------------------------------- set-up
  if (tid == 0) {
    for (int b = 0; b < 5; ++b) tc::mbar_init(tc::smem_addr(&bars[b]), 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), TCOLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);

  // what thread 0 has issued and seen complete, per barrier (for the give-up path)
  int n_commit = 0, x_issued = 0, x_seen = 0, r_issued = 0, r_seen = 0;
  int load_issued = 1, load_seen = 0;  // uses of bar_load: phase 1, then phase 3
  bool w_issued = false, w_seen = false;
  volatile int* s_flag = reinterpret_cast<volatile int*>(smem + kOffBar + 52);
  if (tid == 0) {
    tc::mbar_expect_tx(bar_load, kCoefBytes + kNT * kBBytes);
    tc::bulk_g2s(s_base + kOffC, a.coef_tc + (size_t)(tau * a.n_mt + mt) * kCoefBytes, kCoefBytes, bar_load);
    for (int i = 0; i < kNT; ++i)
      tc::bulk_g2s(s_base + kOffB + i * kBBytes, a.mom_tc + (size_t)atom_of(i) * xs, kBBytes, bar_load);
  }

  // ---------------------------------------------------------------- 1. A for all atoms, q_nl
  bool ok = true;
  int mma_done = 0;  // completions of bar_mma observed by every thread
  if (tid == 0) {
    ok = tc::mbar_wait_bounded(bar_load, 0, kTries);
    if (ok) load_seen = 1;
    if (ok) {
      tc::fence_after_sync();
      issue_split_products(tmem, s_base + kOffC, s_base + kOffB, tc::idesc_bf16_f32(128, 128));
      tc::commit_to(bar_mma);
      ++n_commit;
    }
  }
  ok = __syncthreads_and(ok && tc::mbar_wait_bounded(bar_mma, 0, kTries)) != 0;
  if (!ok) goto give_up;
  mma_done = 1;
  // the product has read the operand buffers: stage every individual's W0
  // block over them now (one bulk copy each, issued by thread ip), to land
  // during q and 2a.  Thread 0 arms the byte count; a copy that completes
  // first cannot end the phase, which also waits for that arrival.
  {
    const int nw = min(kPT, a.n_pop - mt * kPT);
    if (tid == 0) {
      tc::mbar_expect_tx(bar_w, nw * kW0Bytes);
      w_issued = true;
    }
    if (tid < nw) {
      const int net = a.lay.nets > 1 ? tau : 0;
      tc::bulk_g2s(s_base + tid * kW0Stride,
                   a.params + (size_t)(mt * kPT + tid) * a.lay.words + a.lay.off_W0 + net * a.lay.H * DP, kW0Bytes,
                   bar_w);
    }
  }
  tc::fence_after_sync();
#pragma unroll 1
  for (int i = 0; i < kNT; ++i) {
    float A[32];
    tc::tmem_ld32(lane_base + i * 24, A);
    if (prow) {
      float* qd = qbuf + (pl * kNT + i) * kQS;
#pragma unroll
      for (int l = 1; l <= 4; ++l) {
        float s = 0.f;
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm)
          if (l_of(lm) == l) s += wlm(lm) * A[lm] * A[lm];
        qd[NR + (l - 1) * NA + x] = s;
      }
      float gr[5];
      qd[NR + 4 * NA + x] = kC4 * trace_m3(&A[3], gr);
    }
  }
  tc::fence_before_sync();
  __syncthreads();

  // ---------------------------------------------------------------- 2. network (Eq. 1), radial part
  {
    const ModelLayout& Ly = a.lay;
    const bool mine = prow && x < count;  // thread (p, atom x)
    // 2a. thread (p, atom x): radial descriptor q_n from the radial moments,
    // then the scaled descriptor s = q * q_scaler in place
    if (mine) {
      const float* model = a.params + (size_t)p * Ly.words;
      const float* cR_i = model + Ly.off_cR + tau * T * Ly.stride_cR;
      const float* mom = a.mom + atom_of(x);
      float q[NR];
#pragma unroll
      for (int n = 0; n < NR; ++n) q[n] = 0.f;
      for (int t = 0; t < T; ++t) {
        float Fk[BR];
#pragma unroll
        for (int k = 0; k < BR; ++k) Fk[k] = mom[(size_t)(t * kMomBasis + k) * a.mom_stride];
        const float* cc = cR_i + t * Ly.stride_cR;
#pragma unroll
        for (int n = 0; n < NR; ++n)
#pragma unroll
          for (int k = 0; k < BR; ++k) q[n] += __ldg(cc + n * BR + k) * Fk[k];
      }
      float* qd = qbuf + (pl * kNT + x) * kQS;
      // all scaler loads first (generic stores below would otherwise order them)
      float scl[DP];
      const float4* sc4 = reinterpret_cast<const float4*>(model + Ly.off_scaler);
#pragma unroll
      for (int v = 0; v < DP / 4; ++v) {
        const float4 g = __ldg(sc4 + v);
        scl[4 * v] = g.x; scl[4 * v + 1] = g.y; scl[4 * v + 2] = g.z; scl[4 * v + 3] = g.w;
      }
      float4* q4 = reinterpret_cast<float4*>(qd);
#pragma unroll
      for (int v = 0; v < DP / 4; ++v) {
        float4 t4 = q4[v];
        float r4[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int d = 4 * v + u;
          r4[u] = d < NR ? q[d < NR ? d : 0] * scl[d] : (d < 30 ? r4[u] * scl[d] : 0.f);
        }
        q4[v] = make_float4(r4[0], r4[1], r4[2], r4[3]);
      }
    }
    // 2b. every individual's W0 block has been staged by bulk copies (issued
    // after the first product); b0_h and w1_h go into its padding columns 30,
    // 31 of row h.
    {
      const int net = Ly.nets > 1 ? tau : 0;
      const int H = Ly.H;
      constexpr int NPR = (kPT * 30 + 127) / 128;  // rows patched per thread
      float pb0[NPR], pw1[NPR];
#pragma unroll
      for (int u = 0; u < NPR; ++u) {
        const int r = tid + 128 * u, ip = r / 30, h = r % 30, pp = mt * kPT + ip;
        const bool v = r < kPT * 30 && pp < a.n_pop && h < H;
        const float* model = a.params + (size_t)(v ? pp : 0) * Ly.words;
        pb0[u] = v ? __ldg(model + Ly.off_b0 + net * H + h) : 0.f;
        pw1[u] = v ? __ldg(model + Ly.off_w1 + net * H + h) : 0.f;
      }
      const bool okw = __syncthreads_and(tc::mbar_wait_bounded(bar_w, 0, kTries)) != 0;
      if (!okw) goto give_up;
      if (tid == 0) w_seen = true;
#pragma unroll
      for (int u = 0; u < NPR; ++u) {
        const int r = tid + 128 * u, ip = r / 30, h = r % 30;
        if (r < kPT * 30) {
          float* row = reinterpret_cast<float*>(smem + ip * kW0Stride + h * 128);
          row[30] = pb0[u];
          row[31] = pw1[u];
        }
      }
      __syncthreads();
      // thread (p, atom x): U = sum_h w1_h tanh(z_h) - b1, z = W0 s - b0,
      // e = q_scaler * W0^T (w1 * (1 - tanh^2)), written over s in its row
      if (mine) {
        const float* model = a.params + (size_t)p * Ly.words;
        float* row_s = qbuf + (pl * kNT + x) * kQS;
        float sv[DP], e[DP];
#pragma unroll
        for (int v = 0; v < DP / 4; ++v) {
          const float4 t4 = reinterpret_cast<const float4*>(row_s)[v];
          sv[4 * v] = t4.x; sv[4 * v + 1] = t4.y; sv[4 * v + 2] = t4.z; sv[4 * v + 3] = t4.w;
        }
        sv[30] = 0.f;
        sv[31] = 0.f;
#pragma unroll
        for (int d = 0; d < DP; ++d) e[d] = 0.f;
        float U = -__ldg(model + Ly.off_b1 + net);
        const unsigned char* Wp = smem + pl * kW0Stride;
        // z and e in descriptor pairs, one packed multiply-add per pair
        f32x2 s2[15], e2[15];
#pragma unroll
        for (int v = 0; v < 15; ++v) { s2[v] = pk2(sv[2 * v], sv[2 * v + 1]); e2[v] = 0ull; }
#pragma unroll kNetUnroll
        for (int h = 0; h < H; ++h) {
          const float4* w4 = reinterpret_cast<const float4*>(Wp + h * 128);
          float w[DP];
#pragma unroll
          for (int v = 0; v < DP / 4; ++v) {
            const float4 t4 = w4[v];
            w[4 * v] = t4.x; w[4 * v + 1] = t4.y; w[4 * v + 2] = t4.z; w[4 * v + 3] = t4.w;
          }
          f32x2 z2[2] = {0ull, 0ull};
#pragma unroll
          for (int v = 0; v < 15; ++v) z2[v & 1] = fma2(pk2(w[2 * v], w[2 * v + 1]), s2[v], z2[v & 1]);
          float za, zb, zc, zd;
          unpk2(z2[0], za, zb);
          unpk2(z2[1], zc, zd);
          const float z = ((za + zb) + (zc + zd)) - w[30];
          const float hh = tanhf(z);
          const float w1h = w[31];
          U += w1h * hh;
          const float vh = w1h * (1.f - hh * hh);
          const f32x2 vv = pk2(vh, vh);
#pragma unroll
          for (int v = 0; v < 15; ++v) e2[v] = fma2(vv, pk2(w[2 * v], w[2 * v + 1]), e2[v]);
        }
#pragma unroll
        for (int v = 0; v < 15; ++v) unpk2(e2[v], e[2 * v], e[2 * v + 1]);
        float scl[DP];
        const float4* sc4 = reinterpret_cast<const float4*>(model + Ly.off_scaler);
#pragma unroll
        for (int v = 0; v < DP / 4; ++v) {
          const float4 g = __ldg(sc4 + v);
          scl[4 * v] = g.x; scl[4 * v + 1] = g.y; scl[4 * v + 2] = g.z; scl[4 * v + 3] = g.w;
        }
        e[30] = U;
        e[31] = 0.f;
        scl[30] = 1.f;
        scl[31] = 1.f;
#pragma unroll
        for (int v = 0; v < DP / 4; ++v)
          reinterpret_cast<float4*>(row_s)[v] =
              make_float4(e[4 * v] * scl[4 * v], e[4 * v + 1] * scl[4 * v + 1], e[4 * v + 2] * scl[4 * v + 2],
                          e[4 * v + 3] * scl[4 * v + 3]);
      }
    }
    // the W0 area is refilled by bulk copies (async proxy): order this
    // phase's generic accesses before them
    tc::fence_proxy_async_smem();
    __syncthreads();
    // reload the coefficient tile and the B blocks for phase 3, and round 0's X blocks
    if (tid == 0) {
      tc::mbar_expect_tx(bar_load, kCoefBytes + kNT * kBBytes);
      tc::bulk_g2s(s_base + kOffC, a.coef_tc + (size_t)(tau * a.n_mt + mt) * kCoefBytes, kCoefBytes, bar_load);
      for (int i = 0; i < kNT; ++i)
        tc::bulk_g2s(s_base + kOffB + i * kBBytes, a.mom_tc + (size_t)atom_of(i) * xs, kBBytes, bar_load);
      load_issued = 2;
      load_round(0);
      ++x_issued;
    }
    // 2c. thread (p, atom x): radial part of Eqs. 3-4 through the moments V
    // (rank 1) or W (rank 2), and U on the diagonal (rank 2)
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = 0.f;
    if (mine) {
      const float* model = a.params + (size_t)p * Ly.words;
      const float* cR_i = model + Ly.off_cR + tau * T * Ly.stride_cR;
      const float* mom = a.mom + atom_of(x);
      const float* ed = qbuf + (pl * kNT + x) * kQS;
      float e[NR];
#pragma unroll
      for (int n = 0; n < NR; ++n) e[n] = ed[n];
      for (int t = 0; t < T; ++t) {
        const float* cc = cR_i + t * Ly.stride_cR;
#pragma unroll
        for (int k = 0; k < BR; ++k) {
          float Dk = 0.f;
#pragma unroll
          for (int n = 0; n < NR; ++n) Dk += e[n] * __ldg(cc + n * BR + k);
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
      if constexpr (RANK == 2) {
        const float U = ed[30];
        acc[0] += U; acc[4] += U; acc[8] += U;
      }
    }

    // -------------------------------------------------------------- 3. per round: A again, X, contraction
    // Round r (atoms AG r ...): the product A (N = AN, TMEM columns [0, AN))
    // and X (N = XN, columns [AN, AN + XN)).  One X buffer, refilled for
    // round r + 1 as soon as round r's products have read it (during round
    // r's epilogue).
    bool okl = true;
    if (tid == 0) {
      okl = tc::mbar_wait_bounded(bar_load, 1, kTries);
      if (okl) load_seen = 2;
    }
#pragma unroll 1
    for (int r = 0; r < NROUND; ++r) {
      bool ok0 = okl;
      if (tid == 0 && ok0) {
        ok0 = tc::mbar_wait_bounded(bar_x, r & 1, kTries);
        if (ok0) {
          ++x_seen;
          tc::fence_after_sync();
          issue_split_products(tmem, s_base + kOffC, s_base + kOffB + 3 * AG * r * kGroup, tc::idesc_bf16_f32(128, AN));
          issue_split_products(tmem + AN, s_base + kOffC, s_base + kOffX0, tc::idesc_bf16_f32(128, XN));
          tc::commit_to(bar_r);
          ++r_issued;
        }
      }
      ok = __syncthreads_and(ok0 && tc::mbar_wait_bounded(bar_r, r & 1, kTries)) != 0;
      if (!ok) goto give_up;
      if (tid == 0) {
        ++r_seen;
        if (r + 1 < NROUND) {  // round r's products have read the buffer
          load_round(r + 1);
          ++x_issued;
        }
      }
      tc::fence_after_sync();
#pragma unroll
      for (int ia = 0; ia < AG; ++ia) {
        const int i = AG * r + ia;
        if (i >= kNT) break;
        float G[NLM], part[C];
        {
          float Av[32];
          tc::tmem_ld32(lane_base + 24 * ia, Av);
          const float* ed = qbuf + (pl * kNT + i) * kQS;
#pragma unroll
          for (int lm = 0; lm < NLM; ++lm)
            G[lm] = prow ? 2.f * wlm(lm) * ed[NR + (l_of(lm) - 1) * NA + x] * Av[lm] : 0.f;
          if (prow) {
            float gr[5];
            trace_m3(&Av[3], gr);
            const float e4 = kC4 * ed[NR + 4 * NA + x];
#pragma unroll
            for (int m = 0; m < 5; ++m) G[3 + m] += e4 * gr[m];
          }
#pragma unroll
          for (int c = 0; c < C; ++c) part[c] = 0.f;
        }
        // X column AN + XR ia + f, f = lm * C + c
#pragma unroll
        for (int blk = 0; blk < (XR + 31) / 32; ++blk) {
          float Xv[32];
          tc::tmem_ld32(lane_base + AN + XR * ia + 32 * blk, Xv);
#pragma unroll
          for (int v = 0; v < 32; ++v) {
            const int f = 32 * blk + v;
            if (f < XR) part[f % C] += G[f / C] * Xv[v];
          }
        }
        float* red = nsum + ia * (kPT * 5 * C);
        if (prow) {
#pragma unroll
          for (int c = 0; c < C; ++c) red[(pl * 5 + x) * C + c] = part[c];
        }
      }
      tc::fence_before_sync();
      __syncthreads();
#pragma unroll
      for (int ia = 0; ia < AG; ++ia) {
        const int i = AG * r + ia;
        if (i < kNT && mine && x == i) {
          const float* red = nsum + ia * (kPT * 5 * C);
          float* out = a.per_atom + (size_t)p * a.per_atom_stride + atom_of(i);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            float sum = 0.f;
#pragma unroll
            for (int n = 0; n < 5; ++n) sum += red[(pl * 5 + n) * C + c];
            out[(size_t)c * a.atom_stride] = acc[c] - sum;
          }
        }
      }
      __syncthreads();  // the n-sums are read before the next round rewrites them
    }
  }
  if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
  return;

give_up:
  // Nothing further is issued.  Thread 0 knows what it started: the bulk
  // loads, the last committed product, the X copy and the weight blocks.  It
  // waits (bounded) for each of them; TMEM is freed only if all arrived, so
  // no late product can write columns another CTA has been given since, and
  // no late copy can land in shared memory the CTA no longer owns.
  if (tid == 0) {
    if (a.status) atomicCAS(&a.status->error, 0, TNEP_ERR_TIMEOUT);
    bool drained = true;
    if (load_issued > load_seen) drained = tc::mbar_wait_bounded(bar_load, (load_issued - 1) & 1, kTries) && drained;
    if (n_commit > mma_done) drained = tc::mbar_wait_bounded(bar_mma, 0, kTries) && drained;
    if (x_issued > x_seen) drained = tc::mbar_wait_bounded(bar_x, (x_issued - 1) & 1, kTries) && drained;
    if (r_issued > r_seen) drained = tc::mbar_wait_bounded(bar_r, (r_issued - 1) & 1, kTries) && drained;
    if (w_issued && !w_seen) drained = tc::mbar_wait_bounded(bar_w, 0, kTries) && drained;
    *s_flag = drained ? 1 : 0;
  }
  __syncthreads();
  if (*s_flag) {
    tc::fence_after_sync();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
  }
}

}  // namespace

size_t pop_tc_moment_stride(int rank) { return (size_t)kBBytes + (size_t)(rank == 1 ? x_bytes<1>() : x_bytes<2>()); }
size_t pop_tc_coef_bytes() { return kCoefBytes; }

cudaError_t launch_moments_tc(int n_atoms, int n_types, int rank, const float* amom, int amom_slots,
                              unsigned char* dst, cudaStream_t st) {
  const int C = rank == 1 ? 3 : 9;
  const long long threads = (long long)(n_atoms + 1) * (24 + 24 * C);
  count_launches(1);
  k_moments_tc<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(n_atoms, n_types, C, amom, amom_slots, dst,
                                                                  pop_tc_moment_stride(rank));
  return cudaGetLastError();
}

cudaError_t launch_coef_tc(int n_pop, int n_types, int n_mt, const float* params, const ModelLayout& lay,
                           unsigned char* dst, cudaStream_t st) {
  count_launches(1);
  k_coef_tc<<<n_types * n_mt, 128, 0, st>>>(n_pop, n_types, n_mt, params, lay.words, lay.off_cA, lay.stride_cA, dst);
  return cudaGetLastError();
}

cudaError_t launch_pop_tc(int rank, const PopTcArgs& a, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  count_launches(1);
  auto fn = rank == 1 ? k_pop_tc<1> : k_pop_tc<2>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)a.n_tiles * a.n_mt, 128, kSmemBytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tnep
