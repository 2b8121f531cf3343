"""FP64 CPU oracle for the TNEP tensor path -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py`` (its cpu_baseline leg
and ``--impl reference`` arm) may import this module.  The product path never
does, and this module imports nothing from the product package; it shares no
code with the CUDA kernels.

What it computes (paper: arXiv 2312.05233, Sec. II):

* site-energy decomposition U = sum_i U_i with U_i = NN(q_i)      (Sec. II.A, Eq. 1)
* partial force dU_i/dr_ij, r_ij = r_j - r_i (minimum image)       (Sec. II.A, below Eq. 2)
* virial W = -sum_i sum_j r_ij (x) dU_i/dr_ij                      (Eq. 2)
* dipole mu = -sum_i sum_j |r_ij|^2 dU_i/dr_ij                     (Eq. 3, second line)
* polarizability alpha = sum_i U_i I - sum_i sum_j r_ij (x) dU_i/dr_ij  (Eq. 4)
* dipole / polarizability autocorrelations and their cosine transforms
  (Sec. II.F, Eqs. 5-6 for IR; Sec. II.G, Eqs. 7-9 for Raman iso/aniso)

The paper defers the descriptor q_i, the network and the partial force to the
original NEP papers (Sec. II.A).  The readings used here (the published NEP
form) are:

* cutoff f_c(r) = (1 + cos(pi r / rc)) / 2 for r < rc, else 0;
  x = 2 (r/rc - 1)^2 - 1;  f_k(r) = (T_k(x) + 1) f_c(r) / 2, k = 0..K,
  T_k Chebyshev polynomials of the first kind;
  g_n(r) = sum_k c^{t_i t_j}_{nk} f_k(r), separate c for the radial and the
  angular sets.
* radial  q_n = sum_{j: r_ij < rc_R} g^R_n(r_ij).
* angular q_nl = sum_{j,k} g^A_n(r_ij) g^A_n(r_ik) P_l(cos theta_ijk),
  l = 1..l_max, j = k included; equivalently (addition theorem)
  q_nl = 4 pi / (2l+1) sum_m |A_nlm|^2 with A_nlm = sum_j g^A_n(r_ij) Y_lm(r_ij/r_ij),
  complex orthonormal Y_lm with the Condon-Shortley phase.
* 4-body q_n = sum_{m1+m2+m3=0} (2 2 2; m1 m2 m3) A_n2m1 A_n2m2 A_n2m3.
* network U_i = sum_mu w1_mu tanh(sum_nu W0_mu,nu s_nu - b0_mu) - b1,
  s = q * q_scaler, one network per centre type (or one shared network).

Two evaluation modes:

* factorized (default): A_nlm sums, complex Y_lm from the Cartesian textbook
  formula Y_lm = (-1)^m N_lm (x + i y)^m d^m P_l(z)/dz^m (m >= 0), 3j symbols
  from the Racah formula.  O(neighbours) per atom.
* definition: Legendre double sums for q_nl and the explicit triple sum over
  neighbours for the 4-body term, using the closed form of the l=2 invariant
  sum_m (2 2 2; m) Y Y Y = C Tr(Q_a Q_b Q_c), Q_u = u u^T - I/3,
  C = (2 2 2; 0 0 0) (5/4pi)^(3/2) / (2/9).  Tiny inputs only.

Partial forces are the literal definition: the pair vectors r_ij are leaves
of the computation graph and dU_i/dr_ij is obtained with reverse-mode
automatic differentiation (torch.autograd) of U = sum_i U_i, which is exact to
rounding.

Parity pins (tests/test_oracle_*.py): addition theorem (definition ==
factorized), Y_lm against scipy, 3j against sympy and closed forms, 4-body
(definition == factorized), central finite differences of U_i, diatomic 1-D
closed form (pins the r_ij sign), rotations, translation, permutation,
inversion, symmetric alpha, the W0 = 0 closed form, the cubic perovskite, a
parameter-layout probe, the FP32 pair list against the FP64 one, and the
spectrum tail against numpy's FFT (Wiener-Khinchin) and closed forms.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch
from numpy.polynomial import legendre as _npleg
from numpy.polynomial import polynomial as _nppoly

DT = torch.float64
WAVENUMBER_PER_INV_FS = 1.0 / 2.99792458e-5  # 1 fs^-1 in cm^-1

__all__ = [
    "OracleModel", "pairs_fp64", "neighbours_fp32", "wigner3j",
    "sph_harm_complex", "evaluate", "evaluate_frames", "site_energies_from_pairs",
    "acf", "spectrum", "KIND_IR", "KIND_RAMAN_ISO", "KIND_RAMAN_ANISO", "com_dipole", "pairs_cell",
]

KIND_IR, KIND_RAMAN_ISO, KIND_RAMAN_ANISO = 0, 1, 2


# --------------------------------------------------------------------------
# model and its flat parameter layout
# --------------------------------------------------------------------------
@dataclass
class OracleModel:
    """Parsed TNEP model in float64.

    Flat layout of ``params`` (the C header documents the same layout):
    for each network (n_types networks if per_type_nn else one):
        W0 [H][D] row-major, b0 [H], w1 [H], b1 [1]
    then c_R [T][T][n_max_R+1][basis_R+1] (centre type, neighbour type, n, k)
    then c_A [T][T][n_max_A+1][basis_A+1].
    Descriptor order: radial n; then for l = 1..l_max the angular q_nl over n;
    then the 4-body term over n.
    """

    n_types: int
    rank: int
    nR: int
    nA: int
    KR: int
    KA: int
    lmax: int
    four_body: bool
    H: int
    per_type_nn: bool
    rc_R: float
    rc_A: float
    W0: torch.Tensor  # [nets,H,D]
    b0: torch.Tensor  # [nets,H]
    w1: torch.Tensor  # [nets,H]
    b1: torch.Tensor  # [nets]
    cR: torch.Tensor  # [T,T,nR,KR+1]
    cA: torch.Tensor  # [T,T,nA,KA+1]
    scaler: torch.Tensor  # [D]

    @property
    def D(self) -> int:
        return self.nR + self.nA * (self.lmax + (1 if self.four_body else 0))

    @classmethod
    def from_flat(cls, hp, params, q_scaler, rc_R: float, rc_A: float) -> "OracleModel":
        T = hp.n_types
        nR, nA = hp.n_max_R + 1, hp.n_max_A + 1
        KR, KA = hp.basis_R, hp.basis_A
        D = nR + nA * (hp.l_max + (1 if hp.use_4body else 0))
        H = hp.n_hidden
        nets = T if hp.per_type_nn else 1
        p = torch.as_tensor(np.asarray(params, dtype=np.float64))
        o = 0
        W0, b0, w1, b1 = [], [], [], []
        for _ in range(nets):
            W0.append(p[o:o + H * D].reshape(H, D)); o += H * D
            b0.append(p[o:o + H]); o += H
            w1.append(p[o:o + H]); o += H
            b1.append(p[o]); o += 1
        cR = p[o:o + T * T * nR * (KR + 1)].reshape(T, T, nR, KR + 1); o += T * T * nR * (KR + 1)
        cA = p[o:o + T * T * nA * (KA + 1)].reshape(T, T, nA, KA + 1); o += T * T * nA * (KA + 1)
        if o != p.numel():
            raise ValueError(f"parameter vector has {p.numel()} entries, layout needs {o}")
        sc = torch.ones(D, dtype=DT) if q_scaler is None else torch.as_tensor(
            np.asarray(q_scaler, dtype=np.float64))
        return cls(T, hp.rank, nR, nA, KR, KA, hp.l_max, bool(hp.use_4body), H,
                   bool(hp.per_type_nn), float(rc_R), float(rc_A),
                   torch.stack(W0), torch.stack(b0), torch.stack(w1), torch.stack(b1),
                   cR, cA, sc)


# --------------------------------------------------------------------------
# pairs (Sec. II.A: r_ij = r_j - r_i; cutoff model)
# --------------------------------------------------------------------------
def _check_box(box, rc):
    for L in box:
        if L > 0 and L < 2.0 * rc:
            raise ValueError("periodic box edge shorter than twice the cutoff")


def pairs_fp64(pos, box, rc, centers=None):
    """All (i, j != i) with |r_ij| < rc, minimum image on periodic axes.

    Brute force over every atom for every centre.  Returns (i, j, r_ij) with
    r_ij = r_j - r_i as float64, sorted by i then j.
    """
    pos = np.asarray(pos, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    _check_box(box, rc)
    n = len(pos)
    centers = np.arange(n) if centers is None else np.asarray(centers)
    per = box > 0
    I, J, R = [], [], []
    chunk = max(1, 2_000_000 // max(n, 1))
    for s in range(0, len(centers), chunk):
        c = centers[s:s + chunk]
        d = pos[None, :, :] - pos[c][:, None, :]
        if per.any():
            L = np.where(per, box, 1.0)
            d = np.where(per, d - L * np.round(d / L), d)
        r2 = np.einsum("cja,cja->cj", d, d)
        mask = r2 < rc * rc
        mask[np.arange(len(c)), c] = False
        ci, jj = np.nonzero(mask)
        I.append(c[ci]); J.append(jj); R.append(d[ci, jj])
    if not I:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros((0, 3))
    return np.concatenate(I), np.concatenate(J), np.concatenate(R)


def pairs_cell(pos, cell, rc, centers=None):
    """Pairs under a general periodic cell (rows of ``cell`` are the lattice
    vectors a, b, c; r = s H for fractional s): every (i, j, n) with
    |r_j + n H - r_i| < rc and (j, n) != (i, 0), so a neighbour appears once
    per image within the cutoff (cells of any shape, also shorter than twice
    the cutoff).  Positions are first wrapped into the cell; the images are
    enumerated by brute force over n in [-k, k]^3 with k_a = ceil(rc / d_a) + 1,
    d_a the spacing of the lattice planes normal to axis a.  Returns
    (i, j, r_ij) with r_ij = r_j + n H - r_i, sorted by i, then j, then n.
    """
    H = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    vol = abs(np.linalg.det(H))
    if vol <= 0:
        raise ValueError("degenerate cell")
    s = np.asarray(pos, dtype=np.float64) @ np.linalg.inv(H)
    r = (s - np.floor(s)) @ H
    n_at = len(r)
    centers = np.arange(n_at) if centers is None else np.asarray(centers)
    spacing = [vol / np.linalg.norm(np.cross(H[(a + 1) % 3], H[(a + 2) % 3])) for a in range(3)]
    k = [int(np.ceil(rc / d)) + 1 for d in spacing]
    I, J, N, R = [], [], [], []
    for n0 in range(-k[0], k[0] + 1):
        for n1 in range(-k[1], k[1] + 1):
            for n2 in range(-k[2], k[2] + 1):
                shift = np.array([n0, n1, n2], dtype=np.float64) @ H
                d = r[None, :, :] + shift - r[centers][:, None, :]
                r2 = np.einsum("cja,cja->cj", d, d)
                mask = r2 < rc * rc
                if n0 == 0 and n1 == 0 and n2 == 0:
                    mask[np.arange(len(centers)), centers] = False
                ci, jj = np.nonzero(mask)
                nid = ((n0 + k[0]) * (2 * k[1] + 1) + (n1 + k[1])) * (2 * k[2] + 1) + (n2 + k[2])
                I.append(centers[ci]); J.append(jj); N.append(np.full(len(ci), nid)); R.append(d[ci, jj])
    I, J, N, R = (np.concatenate(x) for x in (I, J, N, R))
    order = np.lexsort((N, J, I))
    return I[order], J[order], R[order]


def neighbours_fp32(pos, box, rc, atoms=None):
    """Pair sets under the exact FP32 recipe the C header specifies.

    d = p_j - p_i; on a periodic axis d = d - L * rint(d * (1/L)); every
    operation rounded to float32 separately (no fused multiply-add);
    r2 = (dx*dx + dy*dy) + dz*dz; pair iff r2 < rc*rc (rounded to float32).
    Returns a list of sorted int arrays, one per atom (per atom of `atoms`
    when given: each atom's set is computed on its own against all atoms).
    """
    p = np.asarray(pos, dtype=np.float32)
    b = np.asarray(box, dtype=np.float32)
    n = len(p)
    rc32 = np.float32(rc)
    rc2 = np.float32(rc32 * rc32)
    inv = np.where(b > 0, np.float32(1.0) / np.where(b > 0, b, np.float32(1.0)), np.float32(0.0)).astype(np.float32)
    out = []
    for i in (range(n) if atoms is None else atoms):
        d = (p - p[i]).astype(np.float32)
        for a in range(3):
            if b[a] > 0:
                k = np.rint((d[:, a] * inv[a]).astype(np.float32)).astype(np.float32)
                d[:, a] = (d[:, a] - (b[a] * k).astype(np.float32)).astype(np.float32)
        sq = (d * d).astype(np.float32)
        r2 = ((sq[:, 0] + sq[:, 1]).astype(np.float32) + sq[:, 2]).astype(np.float32)
        m = r2 < rc2
        m[i] = False
        out.append(np.nonzero(m)[0])
    return out


# --------------------------------------------------------------------------
# radial basis (NEP form)
# --------------------------------------------------------------------------
def cutoff_fn(r, rc):
    return torch.where(r < rc, 0.5 * (1.0 + torch.cos(math.pi * r / rc)), torch.zeros_like(r))


def chebyshev_basis(r, rc, K):
    """f_k(r) = (T_k(x) + 1) f_c(r) / 2, x = 2 (r/rc - 1)^2 - 1, k = 0..K -> [P, K+1]."""
    fc = cutoff_fn(r, rc)
    x = 2.0 * (r / rc - 1.0) ** 2 - 1.0
    T = [torch.ones_like(x), x]
    for k in range(2, K + 1):
        T.append(2.0 * x * T[-1] - T[-2])
    return torch.stack([0.5 * (T[k] + 1.0) * fc for k in range(K + 1)], dim=-1)


def radial_functions(r, ti, tj, c, rc, K):
    """g_n(r_ij) = sum_k c[t_i, t_j, n, k] f_k(r_ij) -> [P, n]."""
    f = chebyshev_basis(r, rc, K)
    return torch.einsum("pk,pnk->pn", f, c[ti, tj])


# --------------------------------------------------------------------------
# complex spherical harmonics and Wigner 3j symbols
# --------------------------------------------------------------------------
def _legendre_deriv_power_coeffs(l, m):
    """Power-series coefficients of d^m P_l(z) / dz^m."""
    leg = np.zeros(l + 1); leg[l] = 1.0
    return _nppoly.polyder(_npleg.leg2poly(leg), m) if m else _npleg.leg2poly(leg)


def sph_harm_complex(u, l):
    """Complex orthonormal Y_lm(u), m = -l..l, for unit vectors u [P,3].

    Cartesian textbook form: for m >= 0,
    Y_lm = (-1)^m sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) (x + i y)^m P_l^{(m)}(z),
    and Y_{l,-m} = (-1)^m conj(Y_lm).  Returns (re, im), each [P, 2l+1].
    """
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    re_m = [None] * (l + 1); im_m = [None] * (l + 1)
    pr, pi_ = torch.ones_like(x), torch.zeros_like(x)  # (x+iy)^m
    for m in range(l + 1):
        coef = _legendre_deriv_power_coeffs(l, m)
        poly = torch.zeros_like(z)
        for cf in coef[::-1]:
            poly = poly * z + float(cf)
        N = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
        s = (-1.0) ** m * N
        re_m[m] = s * pr * poly
        im_m[m] = s * pi_ * poly
        pr, pi_ = pr * x - pi_ * y, pr * y + pi_ * x
    re, im = [], []
    for m in range(-l, l + 1):
        if m >= 0:
            re.append(re_m[m]); im.append(im_m[m])
        else:
            sg = (-1.0) ** (-m)
            re.append(sg * re_m[-m]); im.append(-sg * im_m[-m])
    return torch.stack(re, -1), torch.stack(im, -1)


def wigner3j(j1, j2, j3, m1, m2, m3) -> float:
    """Wigner 3j symbol for integer arguments by the Racah formula."""
    if m1 + m2 + m3 != 0:
        return 0.0
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    f = math.factorial
    tri = f(j1 + j2 - j3) * f(j1 - j2 + j3) * f(-j1 + j2 + j3) / f(j1 + j2 + j3 + 1)
    pre = math.sqrt(tri * f(j1 + m1) * f(j1 - m1) * f(j2 + m2) * f(j2 - m2) * f(j3 + m3) * f(j3 - m3))
    kmin = max(0, j2 - j3 - m1, j1 - j3 + m2)
    kmax = min(j1 + j2 - j3, j1 - m1, j2 + m2)
    s = 0.0
    for k in range(kmin, kmax + 1):
        s += (-1) ** k / (f(k) * f(j3 - j2 + k + m1) * f(j3 - j1 + k - m2)
                          * f(j1 + j2 - j3 - k) * f(j1 - k - m1) * f(j2 - k + m2))
    return (-1) ** (j1 - j2 - m3) * pre * s


# --------------------------------------------------------------------------
# descriptors
# --------------------------------------------------------------------------
def _descriptor_factorized(m: OracleModel, n_atoms, i, ti, tj, rij):
    """q [n_atoms, D] from pair vectors (factorized mode)."""
    r = torch.linalg.norm(rij, dim=1)
    u = rij / r[:, None]
    q = []
    gR = radial_functions(r, ti, tj, m.cR, m.rc_R, m.KR)
    qR = torch.zeros(n_atoms, m.nR, dtype=DT).index_add(0, i, gR)
    q.append(qR)
    maskA = r < m.rc_A
    iA, rA, uA = i[maskA], r[maskA], u[maskA]
    gA = radial_functions(rA, ti[maskA], tj[maskA], m.cA, m.rc_A, m.KA)
    A = {}
    for l in range(1, m.lmax + 1):
        yr, yi = sph_harm_complex(uA, l)
        Ar = torch.zeros(n_atoms, m.nA, 2 * l + 1, dtype=DT).index_add(0, iA, gA[:, :, None] * yr[:, None, :])
        Ai = torch.zeros(n_atoms, m.nA, 2 * l + 1, dtype=DT).index_add(0, iA, gA[:, :, None] * yi[:, None, :])
        A[l] = (Ar, Ai)
        q.append(4.0 * math.pi / (2 * l + 1) * (Ar * Ar + Ai * Ai).sum(-1))
    if m.four_body:
        Ar, Ai = A[2]
        q4 = torch.zeros(n_atoms, m.nA, dtype=DT)
        for m1 in range(-2, 3):
            for m2 in range(-2, 3):
                m3 = -m1 - m2
                if abs(m3) > 2:
                    continue
                w = wigner3j(2, 2, 2, m1, m2, m3)
                ar, ai = Ar[..., m1 + 2], Ai[..., m1 + 2]
                br, bi = Ar[..., m2 + 2], Ai[..., m2 + 2]
                cr, ci = Ar[..., m3 + 2], Ai[..., m3 + 2]
                pr, pi_ = ar * br - ai * bi, ar * bi + ai * br
                q4 = q4 + w * (pr * cr - pi_ * ci)
        q.append(q4)
    return torch.cat(q, dim=1)


def _legendre(l, c):
    """P_l(c) by the Bonnet recurrence."""
    p0, p1 = torch.ones_like(c), c
    if l == 0:
        return p0
    for k in range(1, l):
        p0, p1 = p1, ((2 * k + 1) * c * p1 - k * p0) / (k + 1)
    return p1


C4B = -math.sqrt(2.0 / 35.0) * (5.0 / (4.0 * math.pi)) ** 1.5 / (2.0 / 9.0)


def _descriptor_definition(m: OracleModel, n_atoms, i, ti, tj, rij):
    """q [n_atoms, D] by explicit neighbour double / triple sums (tiny inputs)."""
    r = torch.linalg.norm(rij, dim=1)
    u = rij / r[:, None]
    gR = radial_functions(r, ti, tj, m.cR, m.rc_R, m.KR)
    rows = []
    for a in range(n_atoms):
        sel = torch.nonzero(i == a).flatten()
        qa = [gR[sel].sum(0)]
        selA = sel[r[sel] < m.rc_A]
        gA = radial_functions(r[selA], ti[selA], tj[selA], m.cA, m.rc_A, m.KA)  # [k, nA]
        ua = u[selA]
        cos = ua @ ua.T
        for l in range(1, m.lmax + 1):
            P = _legendre(l, cos)
            qa.append(torch.einsum("jn,kn,jk->n", gA, gA, P))
        if m.four_body:
            cjk = cos[:, :, None]
            ckp = cos[None, :, :]
            cpj = cos.T[:, None, :]
            tr = cjk * ckp * cpj - (cjk ** 2 + ckp ** 2 + cpj ** 2) / 3.0 + 2.0 / 9.0
            qa.append(C4B * torch.einsum("jn,kn,pn,jkp->n", gA, gA, gA, tr))
        rows.append(torch.cat(qa))
    return torch.stack(rows) if rows else torch.zeros(0, m.D, dtype=DT)


def _network(m: OracleModel, q, types):
    """U_i = sum_mu w1 tanh(W0 s - b0) - b1, s = q * scaler (Eq. 1)."""
    s = q * m.scaler
    U = torch.zeros(q.shape[0], dtype=DT)
    nets = m.n_types if m.per_type_nn else 1
    for t in range(nets):
        sel = (types == t) if m.per_type_nn else torch.ones_like(types, dtype=torch.bool)
        if not bool(sel.any()):
            continue
        h = torch.tanh(s[sel] @ m.W0[t].T - m.b0[t])
        U = U.index_put((torch.nonzero(sel).flatten(),), h @ m.w1[t] - m.b1[t])
    return U


def site_energies_from_pairs(m: OracleModel, n_atoms, types, i, j, rij, mode="factorized"):
    """U_i for every atom as a function of the pair vectors r_ij (differentiable)."""
    types_t = torch.as_tensor(types, dtype=torch.long)
    i_t = torch.as_tensor(i, dtype=torch.long)
    ti = types_t[i_t]
    tj = types_t[torch.as_tensor(j, dtype=torch.long)]
    if mode == "factorized":
        q = _descriptor_factorized(m, n_atoms, i_t, ti, tj, rij)
    elif mode == "definition":
        q = _descriptor_definition(m, n_atoms, i_t, ti, tj, rij)
    else:
        raise ValueError(mode)
    return _network(m, q, types_t), q


# --------------------------------------------------------------------------
# tensors (Eqs. 2-4)
# --------------------------------------------------------------------------
@dataclass
class OracleResult:
    U: np.ndarray          # [n] site values (centres only, else 0)
    q: np.ndarray          # [n, D]
    i: np.ndarray          # pair centre
    j: np.ndarray          # pair neighbour
    rij: np.ndarray        # [P,3]
    dUdr: np.ndarray       # [P,3] partial forces dU_i/dr_ij
    per_atom: np.ndarray   # [n, 3] (rank 1) or [n, 9] (rank 2)
    tensor: np.ndarray     # [3] or [9] row-major
    virial: np.ndarray     # [9] (Eq. 2)


def evaluate(m: OracleModel, pos, box, types, centers=None, mode="factorized", cell=None) -> OracleResult:
    """One structure.  ``centers`` restricts the sum over i to a subset.
    With ``cell`` (3x3, rows = lattice vectors) the structure is periodic in
    that cell with every image within the cutoff (see pairs_cell) and
    ``box`` is ignored."""
    pos = np.asarray(pos, dtype=np.float64)
    box = np.zeros(3) if box is None else np.asarray(box, dtype=np.float64)
    n = len(pos)
    if cell is not None:
        i, j, R = pairs_cell(pos, cell, m.rc_R, centers)
    else:
        i, j, R = pairs_fp64(pos, box, m.rc_R, centers)
    rij = torch.tensor(R, dtype=DT, requires_grad=True)
    U, q = site_energies_from_pairs(m, n, types, i, j, rij, mode)
    cmask = np.zeros(n, bool)
    cmask[np.arange(n) if centers is None else np.asarray(centers)] = True
    Ucen = U * torch.as_tensor(cmask, dtype=DT)
    (g,) = torch.autograd.grad(Ucen.sum(), rij) if rij.numel() else (torch.zeros_like(rij),)
    F = g.detach().numpy()
    Rn = R
    Un = Ucen.detach().numpy()
    if m.rank == 1:
        contrib = -(np.einsum("pa,pa->p", Rn, Rn)[:, None] * F)
        per_atom = np.zeros((n, 3))
        np.add.at(per_atom, i, contrib)
    else:
        contrib = -np.einsum("pa,pb->pab", Rn, F).reshape(-1, 9)
        per_atom = np.zeros((n, 9))
        np.add.at(per_atom, i, contrib)
        per_atom[:, [0, 4, 8]] += Un[:, None]
    per_atom[~cmask] = 0.0
    vir = -np.einsum("pa,pb->ab", Rn, F).reshape(9)
    return OracleResult(Un, q.detach().numpy(), i, j, Rn, F, per_atom, per_atom.sum(0), vir)


def evaluate_frames(m: OracleModel, frames, box, types, mode="factorized"):
    """Tensor per frame: frames [F,N,3]; box [3] or [F,3] -> [F,3|9]."""
    frames = np.asarray(frames)
    out = []
    for f in range(len(frames)):
        b = box if box is None or np.ndim(box) == 1 else box[f]
        out.append(evaluate(m, frames[f], b, types, mode=mode).tensor)
    return np.asarray(out)


# --------------------------------------------------------------------------
# charged molecules (Sec. III.A)
# --------------------------------------------------------------------------
def com_dipole(pos, types, masses, charge):
    """Q r_COM, the term that turns the relative dipole mu_r of a molecule
    with net charge Q (in e) into its dipole about the origin,
    mu = mu_r + Q r_COM, r_COM = sum_i m_i r_i / sum_i m_i (Sec. III.A)."""
    r = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    m = np.asarray(masses, dtype=np.float64)[np.asarray(types)]
    return float(charge) * (m[:, None] * r).sum(0) / m.sum()


# --------------------------------------------------------------------------
# spectra (Sec. II.F / II.G)
# --------------------------------------------------------------------------
def acf(series, max_lag=None, kind=KIND_IR, subtract_mean=True):
    """Time-origin averaged autocorrelation C(tau), tau = 0..max_lag.

    C(tau) = 1/(T - tau) sum_{t=0}^{T-1-tau} x(t) . x(t + tau)  (unbiased)
    IR: x = mu, one third of the trace (isotropic sample, Sec. II.F).
    Raman iso: x = gamma = Tr(alpha)/3.  Raman aniso: Tr[beta(t) beta(t+tau)]
    with beta = alpha - gamma I (Eq. 9).  Mean removed first if asked.
    """
    s = np.asarray(series, dtype=np.float64)
    T = s.shape[0]
    M = T // 2 if max_lag is None else int(max_lag)
    if kind == KIND_IR:
        x = s.reshape(T, 3)
        if subtract_mean:
            x = x - x.mean(0)
        return np.array([(x[:T - t] * x[t:]).sum() / (T - t) / 3.0 for t in range(M + 1)])
    a = s.reshape(T, 3, 3)
    gam = np.trace(a, axis1=1, axis2=2) / 3.0
    if kind == KIND_RAMAN_ISO:
        x = gam - gam.mean() if subtract_mean else gam
        return np.array([(x[:T - t] * x[t:]).sum() / (T - t) for t in range(M + 1)])
    beta = a - gam[:, None, None] * np.eye(3)
    if subtract_mean:
        beta = beta - beta.mean(0)
    return np.array([np.einsum("tab,tba->", beta[:T - t], beta[t:]) / (T - t) for t in range(M + 1)])


def spectrum(series, dt_fs, kind=KIND_IR, max_lag=None, subtract_mean=True, k_sel=None):
    """One-sided cosine transform of the ACF.

    S(nu_k) = dt [C(0) + 2 sum_{tau=1}^{M} C(tau) cos(2 pi nu_k tau dt)],
    nu_k = k / (2 M dt), k = 0..M.  IR is multiplied by omega^2 (Eq. 6).
    Returns (frequency in cm^-1, spectrum); with k_sel, only the rows k in
    k_sel (same formula, for lags too long to hold the full M x M table).
    """
    C = acf(series, max_lag, kind, subtract_mean)
    M = len(C) - 1
    k = np.arange(M + 1) if k_sel is None else np.asarray(k_sel, dtype=np.int64)
    tau = np.arange(1, M + 1)
    nu = k / (2.0 * M * dt_fs) if M > 0 else np.zeros(1)
    S = dt_fs * (C[0] + 2.0 * (C[1:][None, :] * np.cos(np.pi * np.outer(k, tau) / max(M, 1))).sum(1))
    if kind == KIND_IR:
        S = S * (2.0 * math.pi * nu) ** 2
    return nu * WAVENUMBER_PER_INV_FS, S
