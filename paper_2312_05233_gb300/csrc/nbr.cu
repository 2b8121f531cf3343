// Cell lists and neighbour lists for batches of structures (periodic or open).
//
// The TNEP descriptor only sees atoms inside the cutoffs rc_R and rc_A, with
// r_ij = r_j - r_i taken under the minimum image (Sec. II.A).  The pipeline
// per batch is:
//   plan    one CTA per structure: box checks, bounding box of open axes,
//           cell grid with edge >= rc_R / cell_div (>= rc_R / x_div along x
//           when cell_div = 1; at most 2n + 8 cells)
//   scan    exclusive scan of cells per structure
//   bin     cell of every atom, atomic slot inside the cell
//   scan    exclusive scan of cell counts
//   scatter atoms into their cells
//   sort    one warp per cell orders its atoms by input index (so the whole
//           pipeline is deterministic) and writes cell-ordered float4
//           positions with the type in .w
//   build   one thread per atom scans the stencil cells (with x-thin cells:
//           only the x-cells of each stencil row that its cutoff sphere
//           reaches) and writes the radial (rc_R) and angular (rc_A) lists,
//           warp-tiled.
// Pair selection follows the exact float32 recipe documented in tnep.h.

#include "tnep_internal.cuh"

namespace tnep {

namespace {

__device__ __forceinline__ void raise_error(DevStatus* st, int code, int s) {
  if (atomicCAS(&st->error, 0, code) == 0) st->bad_struct = s;
}

__global__ void k_plan(NbrArgs a) {
  const int s = blockIdx.x;
  const int a0 = a.offsets[s], a1 = a.offsets[s + 1];
  const int n = a1 - a0;
  float L[3];
  for (int d = 0; d < 3; ++d) L[d] = a.box ? a.box[3 * s + d] : 0.0f;
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  const bool any_open = !(L[0] > 0.0f && L[1] > 0.0f && L[2] > 0.0f);
  if (any_open) {  // bounding box of the open axes
    for (int g = a0 + threadIdx.x; g < a1; g += blockDim.x) {
      for (int d = 0; d < 3; ++d) {
        const float x = a.pos[3 * (size_t)g + d];
        mn[d] = fminf(mn[d], x);
        mx[d] = fmaxf(mx[d], x);
      }
    }
  }
  __shared__ float smn[3][32], smx[3][32];
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
      mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int d = 0; d < 3; ++d) { smn[d][w] = mn[d]; smx[d][w] = mx[d]; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int d = 0; d < 3; ++d) {
    mn[d] = smn[d][0]; mx[d] = smx[d][0];
    for (int k = 1; k < nw; ++k) { mn[d] = fminf(mn[d], smn[d][k]); mx[d] = fmaxf(mx[d], smx[d][k]); }
  }
  StructGrid G;
  StructBox B;
  const float edge_min = a.rc_R / (float)a.cell_div * (1.0f + 1e-5f);
  // x_div thins the cells along x (cell_div = 1 only)
  const float edge_min_x = a.cell_div == 1 ? edge_min / (float)a.x_div : edge_min;
  int nc[3];
  float ext[3];
  for (int d = 0; d < 3; ++d) {
    const float em = d == 0 ? edge_min_x : edge_min;
    if (L[d] > 0.0f) {
      if (L[d] < 2.0f * a.rc_R) raise_error(a.status, TNEP_ERR_BOX_TOO_SMALL, s);
      nc[d] = max(1, (int)floorf(L[d] / em));
      ext[d] = L[d];
    } else if (L[d] < 0.0f || isnan(L[d])) {
      raise_error(a.status, TNEP_ERR_INVALID, s);
      nc[d] = 1; ext[d] = 0.0f; L[d] = 0.0f;
    } else {
      ext[d] = n > 0 ? mx[d] - mn[d] : 0.0f;
      if (!(ext[d] < 1e30f)) { raise_error(a.status, TNEP_ERR_INVALID, s); ext[d] = 0.0f; }
      nc[d] = max(1, min(1 << 20, (int)floorf(ext[d] / em) + 1));
    }
  }
  const long long cap = 2LL * n + 8;
  while ((long long)nc[0] * nc[1] * nc[2] > cap) {
    int d = 0;
    if (nc[1] > nc[d]) d = 1;
    if (nc[2] > nc[d]) d = 2;
    nc[d] = max(1, (nc[d] + 1) / 2);
  }
  for (int d = 0; d < 3; ++d) {
    G.nc[d] = nc[d];
    if (L[d] > 0.0f) {
      G.L[d] = L[d];
      G.invL[d] = __fdiv_rn(1.0f, L[d]);
      G.origin[d] = 0.0f;
      G.cinv[d] = (float)nc[d] / L[d];
    } else {
      G.L[d] = 0.0f;
      G.invL[d] = 0.0f;
      G.origin[d] = n > 0 ? mn[d] : 0.0f;
      const float e = fmaxf(d == 0 ? edge_min_x : edge_min, ext[d] / (float)nc[d] * (1.0f + 1e-6f));
      G.cinv[d] = 1.0f / e;
    }
    B.L[d] = G.L[d];
    B.invL[d] = G.invL[d];
  }
  G.cell_offset = 0;
  a.grids[s] = G;
  a.boxes[s] = B;
  a.struct_cells[s] = nc[0] * nc[1] * nc[2];
}

// Exclusive scan of in[0..n) into out[0..n], out[n] = total, one CTA of 1024.
// Tiles of 4 consecutive elements per thread (coalesced), scanned across the
// warps and carried into the next tile.  in and out may alias: each thread
// reads its own elements before writing them.
__device__ void block_exclusive_scan(const int* in, int* out, int n) {
  constexpr int V = 4;
  __shared__ int warp_sums[32];
  __shared__ int carry;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x * V) {
    const int k0 = base + tid * V;
    int v[V];
    int local = 0;
#pragma unroll
    for (int q = 0; q < V; ++q) {
      v[q] = k0 + q < n ? in[k0 + q] : 0;
      local += v[q];
    }
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
      int x = lane < nw ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
      }
      if (lane < nw) warp_sums[lane] = x;
    }
    __syncthreads();
    int run = carry + incl - local + (w > 0 ? warp_sums[w - 1] : 0);
#pragma unroll
    for (int q = 0; q < V; ++q) {
      if (k0 + q < n) out[k0 + q] = run;
      run += v[q];
    }
    __syncthreads();  // carry and warp_sums are read before they change
    if (tid == blockDim.x - 1) carry = run;
    __syncthreads();
  }
  if (tid == 0) out[n] = carry;
}

__global__ void k_scan_structs(NbrArgs a) {
  block_exclusive_scan(a.struct_cells, a.struct_cells, a.n_structs);
  __syncthreads();
  for (int s = threadIdx.x; s < a.n_structs; s += blockDim.x) a.grids[s].cell_offset = a.struct_cells[s];
  if (threadIdx.x == 0 && a.struct_cells[a.n_structs] > a.cells_cap) raise_error(a.status, TNEP_ERR_INVALID, -1);
}

__device__ __forceinline__ int cell_coord(float x, const StructGrid& G, int d) {
  float xw;
  if (G.L[d] > 0.0f) {
    xw = x - G.L[d] * floorf(x * G.invL[d]);
  } else {
    xw = x - G.origin[d];
  }
  int c = (int)floorf(xw * G.cinv[d]);
  return min(max(c, 0), G.nc[d] - 1);
}

__global__ void k_bin(NbrArgs a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n_atoms) return;
  // structure of atom g: last s with offsets[s] <= g
  int lo = 0, hi = a.n_structs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.offsets[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const int s = lo;
  a.atom_struct[g] = s;
  const StructGrid G = a.grids[s];
  const float x0 = a.pos[3 * (size_t)g + 0], x1 = a.pos[3 * (size_t)g + 1], x2 = a.pos[3 * (size_t)g + 2];
  const int c0 = cell_coord(x0, G, 0);
  const int c1 = cell_coord(x1, G, 1);
  const int c2 = cell_coord(x2, G, 2);
  const bool outside = (G.L[0] > 0.0f && !(x0 >= 0.0f && x0 < G.L[0])) ||
                       (G.L[1] > 0.0f && !(x1 >= 0.0f && x1 < G.L[1])) ||
                       (G.L[2] > 0.0f && !(x2 >= 0.0f && x2 < G.L[2]));
  if (outside) atomicOr(&a.struct_flags[s], 1);
  const int cell = G.cell_offset + (c2 * G.nc[1] + c1) * G.nc[0] + c0;
  if (cell >= a.cells_cap) {  // unreachable: cells per structure <= 2n + 8
    raise_error(a.status, TNEP_ERR_INVALID, s);
    a.atom_cell[g] = -1;
    return;
  }
  a.atom_cell[g] = cell;
  a.atom_slot[g] = atomicAdd(&a.cell_count[cell], 1);
}

__global__ void k_scan_cells(NbrArgs a) {
  const int n_cells = min(a.struct_cells[a.n_structs], a.cells_cap);
  block_exclusive_scan(a.cell_count, a.cell_start, n_cells);
}

__global__ void k_scatter(NbrArgs a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n_atoms) return;
  const int cell = a.atom_cell[g];
  if (cell < 0 || cell >= a.cells_cap) return;
  a.cell_atoms[a.cell_start[cell] + a.atom_slot[g]] = g;
}

// One warp per cell: order by input index, write sorted arrays.
__global__ void k_cell_sort(NbrArgs a, int* sorted_cell) {
  const int n_cells = min(a.struct_cells[a.n_structs], a.cells_cap);
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n_cells; c += warps) {
  const int start = a.cell_start[c], m = a.cell_start[c + 1] - start;
  for (int e = lane; e < m; e += 32) {
    const int id = a.cell_atoms[start + e];
    int rank = 0;
    for (int f = 0; f < m; ++f) rank += (a.cell_atoms[start + f] < id);
    const int dst = start + rank;
    a.sorted_orig[dst] = id;
    a.orig_sorted[id] = dst;
    a.sorted_struct[dst] = a.atom_struct[id];
    sorted_cell[dst] = c;
    int t = a.types[id % a.types_period];
    if (t < 0 || t >= a.n_types) {
      raise_error(a.status, TNEP_ERR_INVALID, a.atom_struct[id]);
      t = 0;
    }
    a.pos4[dst] = make_float4(a.pos[3 * (size_t)id], a.pos[3 * (size_t)id + 1], a.pos[3 * (size_t)id + 2],
                              __int_as_float(t));
  }
  }
}

// Stencil cells along one axis with their image shift (in units of the box
// edge, as the float32 product L * k) and their distance in whole cells,
// max(|offset| - 1, 0), from the centre cell (0 where it is not known).
// Periodic axes with at least 2k+1 cells wrap and carry the shift that the
// minimum-image rule would pick for any pair within the cutoff; shorter
// periodic axes list every cell once and leave the shift to rint (flagged by
// the return value < 0).
// `off` receives each stencil cell's offset from the centre cell before wrapping.
__device__ __forceinline__ int axis_stencil(int c, int nc, float L, int k, int* cell, float* sh, int* unit,
                                            int* off) {
  int n = 0;
  if (L > 0.0f) {
    if (nc >= 2 * k + 1) {
      for (int o = -k; o <= k; ++o) {
        int cc = c + o;
        float s = 0.0f;
        if (cc < 0) { cc += nc; s = L; }
        else if (cc >= nc) { cc -= nc; s = -L; }
        cell[n] = cc; sh[n] = s; unit[n] = max(abs(o) - 1, 0); off[n] = o; ++n;
      }
    } else {
      for (int o = 0; o < nc; ++o) { cell[n] = o; sh[n] = 0.0f; unit[n] = 0; off[n] = o - c; ++n; }
      return -n;
    }
  } else {
    const int lo = max(0, c - k), hi = min(nc - 1, c + k);
    for (int o = lo; o <= hi; ++o) {
      cell[n] = o; sh[n] = 0.0f; unit[n] = max(abs(o - c) - 1, 0); off[n] = o - c; ++n;
    }
  }
  return n;
}

// Lower bound on the distance between points of two cells `u` whole cells
// apart along an axis of edge e, less a margin for positions binned across
// a face by rounding.
__device__ __forceinline__ float cell_gap(int u, float e) { return fmaxf((float)u * e - 1e-3f, 0.0f); }

// Margin (Angstrom) for float32 rounding of cell bounds, of binning and of
// the pair rule in the window scan below.
constexpr float kWindowMargin = 1e-3f;

// Lower bound on the distance along one axis between a point at x (relative
// to the grid origin) in cell c and the points of cell c + o, edge e.
__device__ __forceinline__ float point_cell_gap(float x, int c, int o, float e) {
  float g = 0.0f;
  if (o > 0) g = (float)(c + o) * e - x;
  else if (o < 0) g = x - (float)(c + o + 1) * e;
  return fmaxf(g - kWindowMargin, 0.0f);
}

// Minimum-image difference with every operation rounded separately.
__device__ __forceinline__ float mi_diff(float xj, float xi, float L, float invL) {
  float d = __fsub_rn(xj, xi);
  d = __fsub_rn(d, __fmul_rn(L, rintf(__fmul_rn(d, invL))));
  return d;
}

// One thread per atom.  Radial entries go to a scratch list tagged with the
// neighbour type (bits 29-31), then the same thread counting-sorts its own
// entries by type into the final radial list (stable: ascending scan order
// inside each type) and records the per-type counts; the radial moments
// kernel walks one type segment at a time.  (Staging the scratch in shared
// memory instead was measured slower: it limits the candidate scan to 12
// warps per SM.)
// Tests candidates jb..je-1 (at most 32) against atom i with the float32 pair
// rule of the header, setting bit j - jb of mR / mA for r^2 < rc2R / rc2A.
// MODE 0: no image shift; 1: a per-cell shift (s_x, s_y, s_z); 2: rint per
// pair.  (For a zero shift modes 0 and 1 agree bit for bit.)
template <int MODE>
__device__ __forceinline__ void test_candidates(const float4* __restrict__ pos4, int jb, int je, float4 pi,
                                                float sx, float sy, float sz, const StructGrid& G, float rc2R,
                                                float rc2A, unsigned& mR, unsigned& mA, unsigned& mT) {
  unsigned bit = 1u;
#pragma unroll 4
  for (int j = jb; j < je; ++j, bit <<= 1) {
    const float4 pj = __ldg(&pos4[j]);
    float dx, dy, dz;
    if constexpr (MODE == 0) {
      dx = __fsub_rn(pj.x, pi.x);
      dy = __fsub_rn(pj.y, pi.y);
      dz = __fsub_rn(pj.z, pi.z);
    } else if constexpr (MODE == 1) {
      dx = __fsub_rn(__fsub_rn(pj.x, pi.x), sx);
      dy = __fsub_rn(__fsub_rn(pj.y, pi.y), sy);
      dz = __fsub_rn(__fsub_rn(pj.z, pi.z), sz);
    } else {
      dx = mi_diff(pj.x, pi.x, G.L[0], G.invL[0]);
      dy = mi_diff(pj.y, pi.y, G.L[1], G.invL[1]);
      dz = mi_diff(pj.z, pi.z, G.L[2], G.invL[2]);
    }
    const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    mR |= (r2 < rc2R) ? bit : 0u;
    mA |= (r2 < rc2A) ? bit : 0u;
    mT |= (__float_as_int(pj.w) != 0) ? bit : 0u;
  }
}

// TWO: two atom types, radial entries written straight into their final
// places (type 0 from entry 0 up, type 1 from entry cap_R - 1 down), with no
// scratch list and no sort.
template <bool TWO>
__global__ void __launch_bounds__(128) k_build(NbrArgs a, const int* sorted_cell, float rc2R, float rc2A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_atoms) return;
  const float4 pi = a.pos4[i];
  const int s = a.sorted_struct[i];
  const StructGrid G = a.grids[s];
  const int lc = sorted_cell[i] - G.cell_offset;
  const int cx = lc % G.nc[0], cy = (lc / G.nc[0]) % G.nc[1], cz = lc / (G.nc[0] * G.nc[1]);
  const int k = a.cell_div;
  const int kx = k == 1 ? a.x_div : k;  // x_div subdivides x only, and only with cell_div = 1
  int xc[9], yc[7], zc[7], xu[9], yu[7], zu[7], xo[9], yo[7], zo[7];
  float xs[9], ys[7], zs[7];
  int nx = axis_stencil(cx, G.nc[0], G.L[0], kx, xc, xs, xu, xo);
  int ny = axis_stencil(cy, G.nc[1], G.L[1], k, yc, ys, yu, yo);
  int nz = axis_stencil(cz, G.nc[2], G.L[2], k, zc, zs, zu, zo);
  // stencil cells farther than the cutoff from the centre cell are skipped
  const float ex = 1.0f / G.cinv[0], ey = 1.0f / G.cinv[1], ez = 1.0f / G.cinv[2];
  // The shift of a stencil cell equals L * rint((p_j - p_i) / L) for every pair
  // the cutoff can accept when all coordinates lie in [0, L); otherwise (or
  // when an axis has too few cells to carry shifts) use rint per pair.  Both
  // give the float32 rule of the header bit for bit.
  const bool use_rint = nx < 0 || ny < 0 || nz < 0 || (a.struct_flags[s] & 1);
  nx = abs(nx); ny = abs(ny); nz = abs(nz);
  // scratch entry e of this thread lives at wR[e * ws]
  int* wR = a.nbr_tmp + (size_t)(i >> 5) * a.cap_R * 32 + (i & 31);
  constexpr int ws = 32;
  int* wA = a.nbr_A + (size_t)(i >> 5) * a.cap_A * 32 + (i & 31);
  int* outR = a.nbr_R + (size_t)(i >> 5) * a.cap_R * 32 + (i & 31);
  int cR = 0, cA = 0, c1 = 0;
  // Tests candidates j0..j1-1 (one contiguous range of cells sharing a shift)
  // and appends the accepted ones.
  auto scan = [&](int j0, int j1, float sx, float sy, float sz, bool rint_pairs) {
    const bool noshift = !rint_pairs && sx == 0.0f && sy == 0.0f && sz == 0.0f;
    // Test up to 32 candidates into acceptance bit masks, then append only
    // the accepted ones (about one candidate in seven is accepted).
    for (int jb = j0; jb < j1; jb += 32) {
      const int je = min(jb + 32, j1);
      unsigned mR = 0u, mA = 0u, mT = 0u;
      if (noshift)
        test_candidates<0>(a.pos4, jb, je, pi, sx, sy, sz, G, rc2R, rc2A, mR, mA, mT);
      else if (!rint_pairs)
        test_candidates<1>(a.pos4, jb, je, pi, sx, sy, sz, G, rc2R, rc2A, mR, mA, mT);
      else
        test_candidates<2>(a.pos4, jb, je, pi, sx, sy, sz, G, rc2R, rc2A, mR, mA, mT);
      if (i >= jb && i < je) {  // an atom is not its own neighbour
        mR &= ~(1u << (i - jb));
        mA &= ~(1u << (i - jb));
      }
      if constexpr (TWO) {
        // type 0 from the front, then type 1 from the back: one store stream each
        unsigned m0 = mR & ~mT, m1 = mR & mT;
        while (m0) {
          const int j = jb + __ffs(m0) - 1;
          m0 &= m0 - 1;
          if (cR - c1 < a.cap_R) outR[(size_t)(cR - c1) * 32] = j;
          ++cR;
        }
        while (m1) {
          const int j = jb + __ffs(m1) - 1;
          m1 &= m1 - 1;
          if (c1 < a.cap_R) outR[(size_t)(a.cap_R - 1 - c1) * 32] = j;
          ++c1;
          ++cR;
        }
      } else {
        while (mR) {
          const int j = jb + __ffs(mR) - 1;
          mR &= mR - 1;
          if (cR < a.cap_R) wR[(size_t)cR * 32] = j | (__float_as_int(a.pos4[j].w) << kTypeShift);
          ++cR;
        }
      }
      while (mA) {
        const int j = jb + __ffs(mA) - 1;
        mA &= mA - 1;
        if (cA < a.cap_A) wA[(size_t)cA * 32] = j;
        ++cA;
      }
    }
  };
  if (kx > 1 && k == 1 && !use_rint) {
    // Window scan: cells are thin along x.  In each (y, z) row of the stencil
    // only the x-cells meeting [x_i - h, x_i + h] can hold pairs, where
    // h^2 = rc_R^2 - (distance from atom i to the row)^2; on a periodic axis
    // the window splits at the box faces into ranges with shifts +L, 0, -L.
    // A window longer than the row falls back to the whole row with rint.
    const float xr = pi.x - G.origin[0], yr = pi.y - G.origin[1], zr = pi.z - G.origin[2];
    const float rcm = a.rc_R + kWindowMargin, rcm2 = rcm * rcm;
    const int ncx = G.nc[0];
    for (int iz = 0; iz < nz; ++iz) {
      const float gz = point_cell_gap(zr, cz, zo[iz], ez);
      if (gz * gz >= rcm2) continue;
      for (int iy = 0; iy < ny; ++iy) {
        const float gy = point_cell_gap(yr, cy, yo[iy], ey);
        const float h2 = rcm2 - gy * gy - gz * gz;
        if (h2 <= 0.0f) continue;
        const float h = sqrtf(h2) + kWindowMargin;
        int clo = (int)floorf((xr - h) * G.cinv[0]);
        int chi = (int)floorf((xr + h) * G.cinv[0]);
        const int row = G.cell_offset + (zc[iz] * G.nc[1] + yc[iy]) * ncx;
        const float sy = ys[iy], sz = zs[iz];
        if (G.L[0] > 0.0f) {
          if (chi - clo + 1 > ncx) {
            scan(a.cell_start[row], a.cell_start[row + ncx], 0.0f, sy, sz, true);
            continue;
          }
          if (clo < 0) scan(a.cell_start[row + clo + ncx], a.cell_start[row + ncx], G.L[0], sy, sz, false);
          const int b0 = max(clo, 0), b1 = min(chi, ncx - 1);
          if (b0 <= b1) scan(a.cell_start[row + b0], a.cell_start[row + b1 + 1], 0.0f, sy, sz, false);
          if (chi >= ncx) scan(a.cell_start[row], a.cell_start[row + chi - ncx + 1], -G.L[0], sy, sz, false);
        } else {
          clo = max(clo, 0);
          chi = min(chi, ncx - 1);
          if (clo <= chi) scan(a.cell_start[row + clo], a.cell_start[row + chi + 1], 0.0f, sy, sz, false);
        }
      }
    }
  } else {
    for (int iz = 0; iz < nz; ++iz) {
      const float gz = cell_gap(zu[iz], ez);
      if (gz * gz >= rc2R) continue;
      for (int iy = 0; iy < ny; ++iy) {
        const float gy = cell_gap(yu[iy], ey);
        const float gyz = gy * gy + gz * gz;
        if (gyz >= rc2R) continue;
        const int row = G.cell_offset + (zc[iz] * G.nc[1] + yc[iy]) * G.nc[0];
        const float sy = ys[iy], sz = zs[iz];
        int ix = 0;
        while (ix < nx) {
          const float gx = cell_gap(xu[ix], ex);
          if (gx * gx + gyz >= rc2R) { ++ix; continue; }
          // merge x-cells that are contiguous, within reach and share a shift into one range
          int ie = ix + 1;
          while (ie < nx && xc[ie] == xc[ie - 1] + 1 && xs[ie] == xs[ix]) {
            const float ge = cell_gap(xu[ie], ex);
            if (ge * ge + gyz >= rc2R) break;
            ++ie;
          }
          const float sx = xs[ix];
          const int j0 = a.cell_start[row + xc[ix]], j1 = a.cell_start[row + xc[ie - 1] + 1];
          ix = ie;
          scan(j0, j1, sx, sy, sz, use_rint);
        }
      }
    }
  }
  a.cnt_R[i] = cR;
  a.cnt_A[i] = cA;
  if (cR > a.cap_R) atomicMax(&a.status->max_cnt_R, cR);
  if (cA > a.cap_A) atomicMax(&a.status->max_cnt_A, cA);
  if constexpr (TWO) {
    a.seg_R[i] = cR - c1;
    a.seg_R[(size_t)a.seg_stride + i] = c1;
    return;
  }
  // counting sort of the radial entries by neighbour type; the scratch rows
  // are read eight at a time so that eight loads are in flight per warp
  const int n = min(cR, a.cap_R);
  int cnt[kMaxTypes];
#pragma unroll
  for (int u = 0; u < kMaxTypes; ++u) cnt[u] = 0;
  for (int e0 = 0; e0 < n; e0 += 8) {
    int v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (e0 + q < n) ? wR[(size_t)(e0 + q) * ws] : 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int t = (e0 + q < n) ? (int)((unsigned)v[q] >> kTypeShift) : -1;
#pragma unroll
      for (int u = 0; u < kMaxTypes; ++u) cnt[u] += (t == u);
    }
  }
  int off[kMaxTypes];
  int run = 0;
#pragma unroll
  for (int u = 0; u < kMaxTypes; ++u) { off[u] = run; run += cnt[u]; }
  for (int e0 = 0; e0 < n; e0 += 8) {
    int v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (e0 + q < n) ? wR[(size_t)(e0 + q) * ws] : 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (e0 + q < n) {
        const int t = (unsigned)v[q] >> kTypeShift;
        int dst = 0;
#pragma unroll
        for (int u = 0; u < kMaxTypes; ++u)
          if (t == u) { dst = off[u]; off[u] = dst + 1; }
        outR[(size_t)dst * 32] = v[q] & kIndexMask;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kMaxTypes; ++u)
    if (u < a.n_types) a.seg_R[(size_t)u * a.seg_stride + i] = cnt[u];
}

// Frames of a pass in the first frame's cell order, with their boxes.
__global__ void k_skin_gather(SkinArgs a) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)a.nf * a.N) return;
  const int f = (int)(g / a.N), i = (int)(g % a.N);
  const int o = a.sorted_orig[i];
  const float* p = a.pos + ((size_t)f * a.N + o) * 3;
  const int t = a.types[o % a.types_period];
  a.pos4[g] = make_float4(p[0], p[1], p[2], __int_as_float(t));
  a.sorted_struct[g] = f;
  if (i == 0) {
    StructBox B;
    for (int d = 0; d < 3; ++d) {
      const float L = a.box ? a.box[3 * f + d] : 0.0f;
      B.L[d] = L > 0.0f ? L : 0.0f;
      B.invL[d] = L > 0.0f ? __fdiv_rn(1.0f, L) : 0.0f;
    }
    a.boxes[f] = B;
  }
}

// Each frame's exact lists from the first frame's skin lists: every skin
// candidate is re-tested with the float32 pair rule of the header under this
// frame's positions.  The radial list keeps the type segments; the angular
// list is taken from the same candidates.  Flags skin_violation when an atom
// moved more than skin / 2 from the first frame or the box changed.
__global__ void __launch_bounds__(128) k_skin_compact(SkinArgs a) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)a.nf * a.N) return;
  const int f = (int)(g / a.N), i = (int)(g % a.N);
  const int base = f * a.N;
  const float4 pi = a.pos4[g];
  const StructBox B = a.boxes[f];
  const StructBox R = a.ref_box[0];
  bool bad = false;
  for (int d = 0; d < 3; ++d) bad |= (B.L[d] != R.L[d]);
  {
    const float4 p0 = a.ref4[i];
    const float dx = mi_diff(pi.x, p0.x, B.L[0], B.invL[0]);
    const float dy = mi_diff(pi.y, p0.y, B.L[1], B.invL[1]);
    const float dz = mi_diff(pi.z, p0.z, B.L[2], B.invL[2]);
    bad |= (dx * dx + dy * dy + dz * dz) > a.half_skin2;
  }
  if (bad) atomicOr(&a.status->skin_violation, 1);
  int cR = 0, cA = 0, start = 0;
  for (int t = 0; t < a.n_types; ++t) {
    const int n_seg = a.skin_seg[(size_t)t * a.skin_seg_stride + i];
    // entries of this type inside the row: all of them unless the skin lists
    // overflowed, in which case the call is redone with a larger capacity and
    // the reads only have to stay in bounds
    const int s0 = radial_segment_start(a.skin_two_ended, t, start, n_seg, a.skin_cap);
    const int e0 = max(s0, 0), n = max(min(s0 + n_seg, a.skin_cap) - e0, 0);
    int kept = 0;
    // Software-pipelined gather: the list index two entries ahead, the
    // position one ahead, list rows four ahead pulled into L1 (a warp's row is
    // one 128-byte line).  The same candidates in the same order as a plain
    // loop over entries e0 .. e0 + n - 1; past the end the last index is
    // re-used, so every load stays in bounds.
    int jn = n > 0 ? a.skin_nbr[nbr_index(i, e0, a.skin_cap)] : 0;
    int ja = n > 1 ? a.skin_nbr[nbr_index(i, e0 + 1, a.skin_cap)] : jn;
    float4 pn = n > 0 ? a.pos4[base + jn] : pi;
    for (int k = 0; k < n; ++k) {
      const int j = jn;
      const float4 pj = pn;
      jn = ja;
      pn = a.pos4[base + ja];
      if (k + 2 < n) ja = a.skin_nbr[nbr_index(i, e0 + k + 2, a.skin_cap)];
      if (k + 4 < n)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.skin_nbr + nbr_index(i, e0 + k + 4, a.skin_cap)));
      const float dx = mi_diff(pj.x, pi.x, B.L[0], B.invL[0]);
      const float dy = mi_diff(pj.y, pi.y, B.L[1], B.invL[1]);
      const float dz = mi_diff(pj.z, pi.z, B.L[2], B.invL[2]);
      const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
      if (r2 < a.rc2R) {
        if (cR < a.cap_R) a.nbr_R[nbr_index((int)g, cR, a.cap_R)] = base + j;
        ++cR;
        ++kept;
        if (r2 < a.rc2A) {
          if (cA < a.cap_A) a.nbr_A[nbr_index((int)g, cA, a.cap_A)] = base + j;
          ++cA;
        }
      }
    }
    start += n_seg;
    a.seg_R[(size_t)t * a.seg_stride + g] = kept;
  }
  a.cnt_R[g] = cR;
  a.cnt_A[g] = cA;
  if (cR > a.cap_R) atomicMax(&a.status->max_cnt_R, cR);
  if (cA > a.cap_A) atomicMax(&a.status->max_cnt_A, cA);
}

__global__ void k_export(int n, const int* sorted_orig, const int* nbr_R, const int* cnt_R, int cap_R,
                         const int* seg_R, int two_ended, const int* nbr_A, const int* cnt_A, int cap_A, int* out_cnt_R, int* out_cnt_A,
                         int* out_R, int out_cap_R, int* out_A, int out_cap_A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int o = sorted_orig[i];
  const int nR = cnt_R[i], nA = cnt_A[i];
  out_cnt_R[o] = nR;
  out_cnt_A[o] = nA;
  // two-ended lists (nR <= cap_R here): type 1 occupies [cap_R - n1, cap_R)
  const int n0 = two_ended ? seg_R[i] : nR;
  for (int k = 0; k < min(nR, min(cap_R, out_cap_R)); ++k) {
    const int e = k < n0 ? k : cap_R - nR + k;
    out_R[(size_t)o * out_cap_R + k] = sorted_orig[nbr_R[nbr_index(i, e, cap_R)]];
  }
  for (int k = 0; k < min(nA, min(cap_A, out_cap_A)); ++k)
    out_A[(size_t)o * out_cap_A + k] = sorted_orig[nbr_A[nbr_index(i, k, cap_A)]];
}

}  // namespace

cudaError_t launch_neighbor_pipeline(const NbrArgs& a, cudaStream_t st) {
  const int S = a.n_structs, N = a.n_atoms;
  if (S <= 0) return cudaSuccess;
  count_launches(N > 0 ? 7 : 3);
  k_plan<<<S, 256, 0, st>>>(a);
  k_scan_structs<<<1, 1024, 0, st>>>(a);
  // The number of cells in use is known only on the device; the cell scan
  // and the per-cell sort read it from struct_cells[S].
  if (N > 0) k_bin<<<(N + 255) / 256, 256, 0, st>>>(a);
  k_scan_cells<<<1, 1024, 0, st>>>(a);
  if (N > 0) {
    k_scatter<<<(N + 255) / 256, 256, 0, st>>>(a);
    // sorted_cell reuses atom_slot (dead after the scatter)
    k_cell_sort<<<1216, 256, 0, st>>>(a, a.atom_slot);
    const float rc2R = a.rc_R * a.rc_R, rc2A = a.rc_A * a.rc_A;
    if (a.two_ended)
      k_build<true><<<(N + 127) / 128, 128, 0, st>>>(a, a.atom_slot, rc2R, rc2A);
    else
      k_build<false><<<(N + 127) / 128, 128, 0, st>>>(a, a.atom_slot, rc2R, rc2A);
  }
  return cudaGetLastError();
}

cudaError_t launch_skin_compact(const SkinArgs& a, cudaStream_t st) {
  const long long n = (long long)a.nf * a.N;
  if (n <= 0) return cudaSuccess;
  count_launches(2);
  const int blocks = (int)((n + 127) / 128);
  k_skin_gather<<<blocks, 128, 0, st>>>(a);
  k_skin_compact<<<blocks, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_export_neighbors(int n_atoms, const int* sorted_orig, const int* orig_sorted,
                                    const int* nbr_R, const int* cnt_R, int cap_R, const int* seg_R, int two_ended,
                                    const int* nbr_A, const int* cnt_A, int cap_A,
                                    int* out_cnt_R, int* out_cnt_A, int* out_R, int out_cap_R,
                                    int* out_A, int out_cap_A, cudaStream_t st) {
  (void)orig_sorted;
  if (n_atoms <= 0) return cudaSuccess;
  count_launches(1);
  k_export<<<(n_atoms + 127) / 128, 128, 0, st>>>(n_atoms, sorted_orig, nbr_R, cnt_R, cap_R, seg_R, two_ended,
                                                   nbr_A, cnt_A,
                                                   cap_A, out_cnt_R, out_cnt_A, out_R, out_cap_R, out_A,
                                                   out_cap_A);
  return cudaGetLastError();
}

}  // namespace tnep
