"""Pins of the FP64 oracle against facts outside itself (no GPU).

Each test checks the oracle against mathematics or a library routine that the
oracle does not call: Wigner 3j symbols against sympy and closed forms, Y_lm
against scipy, the addition theorem (Legendre double sums vs factorized
sums), the 4-body invariant (explicit triple sum with the traceless-tensor
closed form vs 3j contraction), finite differences of U_i against the
autograd partial forces, the diatomic closed form that fixes the sign of
r_ij = r_j - r_i (Sec. II.A), equivariance of Eqs. 3-4, and closed forms.
"""

import math

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.tnep_oracle import (DT, OracleModel, _descriptor_definition, _descriptor_factorized,
                                chebyshev_basis, pairs_fp64, sph_harm_complex, wigner3j)

RC_R, RC_A = 6.0, 4.0


def make_model(rank=1, n_types=2, seed=7, **kw):
    hp = synth.HyperParams(n_types=n_types, rank=rank, **kw)
    rng = np.random.default_rng(seed)
    p = synth.model_params(hp, rng)
    return hp, p, OracleModel.from_flat(hp, p, synth.default_q_scaler(hp), RC_R, RC_A)


def small_cluster(n_mol=4, seed=3):
    rng = np.random.default_rng(seed)
    pos, types, box = synth.water_cluster(n_mol, rng)
    return pos, types, box


# ----------------------------------------------------------------- 3j / Y_lm
def test_wigner3j_closed_forms():
    assert wigner3j(2, 2, 2, 0, 0, 0) == pytest.approx(-math.sqrt(2.0 / 35.0), abs=1e-15)
    assert wigner3j(1, 1, 0, 0, 0, 0) == pytest.approx(-1.0 / math.sqrt(3.0), abs=1e-15)
    assert wigner3j(2, 2, 2, 1, 0, 1) == 0.0  # m sum != 0
    # (j j 0; m -m 0) = (-1)^(j-m) / sqrt(2j+1)
    for j in range(5):
        for m in range(-j, j + 1):
            assert wigner3j(j, j, 0, m, -m, 0) == pytest.approx((-1) ** (j - m) / math.sqrt(2 * j + 1), abs=1e-14)


def test_wigner3j_orthogonality():
    # sum_{m1,m2} (2j3+1) (j1 j2 j3; m1 m2 m3)(j1 j2 j3'; m1 m2 m3') = delta
    j1 = j2 = 2
    for j3 in range(0, 5):
        for j3p in range(0, 5):
            for m3 in range(-min(j3, j3p), min(j3, j3p) + 1):
                s = sum((2 * j3 + 1) * wigner3j(j1, j2, j3, m1, -m1 - m3, m3)
                        * wigner3j(j1, j2, j3p, m1, -m1 - m3, m3)
                        for m1 in range(-j1, j1 + 1) if abs(-m1 - m3) <= j2)
                assert s == pytest.approx(1.0 if j3 == j3p else 0.0, abs=1e-13)


def test_wigner3j_vs_sympy():
    wig = pytest.importorskip("sympy.physics.wigner")
    for j1, j2, j3 in [(2, 2, 2), (1, 2, 3), (2, 2, 4), (3, 3, 2), (4, 4, 4)]:
        for m1 in range(-j1, j1 + 1):
            for m2 in range(-j2, j2 + 1):
                m3 = -m1 - m2
                if abs(m3) > j3:
                    continue
                assert wigner3j(j1, j2, j3, m1, m2, m3) == pytest.approx(
                    float(wig.wigner_3j(j1, j2, j3, m1, m2, m3)), abs=1e-14)


def test_sph_harm_vs_scipy():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(0)
    u = rng.normal(size=(50, 3)); u /= np.linalg.norm(u, axis=1)[:, None]
    th = np.arccos(u[:, 2]); ph = np.arctan2(u[:, 1], u[:, 0])
    for l in range(0, 5):
        re, im = sph_harm_complex(torch.tensor(u, dtype=DT), l)
        for m in range(-l, l + 1):
            ref = sp.sph_harm_y(l, m, th, ph)
            np.testing.assert_allclose(re[:, m + l].numpy(), ref.real, atol=1e-13)
            np.testing.assert_allclose(im[:, m + l].numpy(), ref.imag, atol=1e-13)


# ---------------------------------------------------------- basis functions
def test_chebyshev_basis_closed_form():
    r = torch.linspace(0.1, 5.9, 37, dtype=DT)
    f = chebyshev_basis(r, 6.0, 8).numpy()
    x = 2 * (r.numpy() / 6.0 - 1) ** 2 - 1
    fc = 0.5 * (1 + np.cos(np.pi * r.numpy() / 6.0))
    for k in range(9):
        Tk = np.cos(k * np.arccos(np.clip(x, -1, 1)))  # T_k(cos t) = cos(k t)
        np.testing.assert_allclose(f[:, k], 0.5 * (Tk + 1) * fc, atol=1e-13)
    assert float(chebyshev_basis(torch.tensor([6.0, 7.0], dtype=DT), 6.0, 8).abs().max()) == 0.0


# ------------------------------------------------ descriptor: two derivations
@pytest.mark.parametrize("periodic", [False, True])
def test_addition_theorem_and_4body(periodic):
    _, _, m = make_model()
    if periodic:
        rng = np.random.default_rng(5)
        pos, types, box = synth.water_grid_box(4, 12.42, rng)
        pos = pos[:60]; types = types[:60]
    else:
        pos, types, box = small_cluster(6)
    i, j, R = pairs_fp64(pos, box, RC_R)
    n = len(pos)
    it = torch.as_tensor(i); tt = torch.as_tensor(types, dtype=torch.long)
    ti, tj = tt[it], tt[torch.as_tensor(j)]
    rij = torch.tensor(R, dtype=DT)
    qf = _descriptor_factorized(m, n, it, ti, tj, rij).numpy()
    qd = _descriptor_definition(m, n, it, ti, tj, rij).numpy()
    np.testing.assert_allclose(qf, qd, rtol=1e-11, atol=1e-13)
    assert np.abs(qf[:, -5:]).max() > 1e-6  # 4-body term is exercised


# ---------------------------------------------------- partial forces (Eq. 2)
def test_partial_force_finite_differences():
    _, _, m = make_model(rank=2)
    pos, types, box = small_cluster(3)
    n = len(pos)
    i, j, R = pairs_fp64(pos, box, RC_R)
    res = oracle.evaluate(m, pos, box, types)
    h = 1e-5
    rng = np.random.default_rng(1)
    for p in rng.choice(len(i), size=min(12, len(i)), replace=False):
        for a in range(3):
            Rp = R.copy(); Rp[p, a] += h
            Rm = R.copy(); Rm[p, a] -= h
            Up, _ = oracle.site_energies_from_pairs(m, n, types, i, j, torch.tensor(Rp, dtype=DT))
            Um, _ = oracle.site_energies_from_pairs(m, n, types, i, j, torch.tensor(Rm, dtype=DT))
            fd = (Up[i[p]] - Um[i[p]]).item() / (2 * h)
            assert fd == pytest.approx(res.dUdr[p, a], rel=1e-6, abs=1e-9)


def test_total_force_from_positions():
    """F_k = -dU/dr_k assembled from partial forces (pins pair conventions and
    the minimum image): F_k = sum_i dU_i/dr_ik - sum_j dU_k/dr_kj."""
    _, _, m = make_model()
    rng = np.random.default_rng(9)
    pos, types, box = synth.water_grid_box(4, 12.42, rng)
    pos = np.mod(pos + 0.05 * rng.standard_normal(pos.shape), box)
    res = oracle.evaluate(m, pos, box, types)
    n = len(pos)
    F = np.zeros((n, 3))
    np.add.at(F, res.j, res.dUdr)
    np.add.at(F, res.i, -res.dUdr)
    h = 1e-5
    for k in [0, 5, 100]:
        for a in range(3):
            pp = pos.copy(); pp[k, a] += h
            pm = pos.copy(); pm[k, a] -= h
            Up = oracle.evaluate(m, pp, box, types).U.sum()
            Um = oracle.evaluate(m, pm, box, types).U.sum()
            assert -(Up - Um) / (2 * h) == pytest.approx(-F[k, a], rel=1e-6, abs=1e-8)
    # Newton's third law over the structure (Sec. II.B)
    np.testing.assert_allclose(F.sum(0), 0.0, atol=1e-10)


def test_diatomic_closed_form():
    """Two atoms a, b at distance r along d: mu = -r^2 (U_a' - U_b') d_hat and
    alpha = (U_a + U_b) I - r (U_a' + U_b') d_hat d_hat^T, with r_ab = r_b - r_a."""
    for rank in (1, 2):
        _, _, m = make_model(rank=rank)
        types = np.array([0, 1])
        d = np.array([0.3, -0.5, 0.8]); d /= np.linalg.norm(d)
        r0 = 2.1

        def Us(r):
            pos = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0]]) + np.array([[0, 0, 0], r * d])
            return oracle.evaluate(m, pos, None, types).U

        h = 1e-5
        dU = (Us(r0 + h) - Us(r0 - h)) / (2 * h)
        U = Us(r0)
        pos = np.array([[1.0, 2.0, 3.0], [1.0 + r0 * d[0], 2.0 + r0 * d[1], 3.0 + r0 * d[2]]])
        t = oracle.evaluate(m, pos, None, types).tensor
        if rank == 1:
            np.testing.assert_allclose(t, -r0 ** 2 * (dU[0] - dU[1]) * d, rtol=1e-7, atol=1e-10)
        else:
            ref = (U[0] + U[1]) * np.eye(3) - r0 * (dU[0] + dU[1]) * np.outer(d, d)
            np.testing.assert_allclose(t.reshape(3, 3), ref, rtol=1e-7, atol=1e-10)


# ------------------------------------------------------------- equivariance
def test_rotation_covariance():
    pos, types, box = small_cluster(8, seed=11)
    R = synth.random_rotation(np.random.default_rng(2))
    for rank in (1, 2):
        _, _, m = make_model(rank=rank)
        t0 = oracle.evaluate(m, pos, box, types).tensor
        t1 = oracle.evaluate(m, pos @ R.T, box, types).tensor
        if rank == 1:
            np.testing.assert_allclose(t1, R @ t0, atol=1e-11)
        else:
            a0 = t0.reshape(3, 3)
            np.testing.assert_allclose(t1.reshape(3, 3), R @ a0 @ R.T, atol=1e-11)
            np.testing.assert_allclose(a0, a0.T, atol=1e-11)


def test_translation_permutation_inversion():
    rng = np.random.default_rng(4)
    pos, types, box = synth.water_grid_box(4, 12.42, rng)
    for rank in (1, 2):
        _, _, m = make_model(rank=rank)
        t0 = oracle.evaluate(m, pos, box, types).tensor
        shifted = np.mod(pos + np.array([3.3, -1.7, 5.2]), box)
        np.testing.assert_allclose(oracle.evaluate(m, shifted, box, types).tensor, t0, atol=1e-10)
        perm = rng.permutation(len(pos))
        np.testing.assert_allclose(oracle.evaluate(m, pos[perm], box, types[perm]).tensor, t0, atol=1e-10)
        inv = oracle.evaluate(m, np.mod(-pos, box), box, types).tensor
        np.testing.assert_allclose(inv, -t0 if rank == 1 else t0, atol=1e-10)


# ------------------------------------------------------------- closed forms
def test_zero_W0_closed_form():
    hp, p, m = make_model(rank=2)
    m.W0.zero_()
    pos, types, box = small_cluster(5)
    r = oracle.evaluate(m, pos, box, types)
    Ut = [float((m.w1[t] * torch.tanh(-m.b0[t])).sum() - m.b1[t]) for t in range(2)]
    np.testing.assert_allclose(r.U, [Ut[t] for t in types], atol=1e-13)
    np.testing.assert_allclose(r.tensor.reshape(3, 3), sum(Ut[t] for t in types) * np.eye(3), atol=1e-12)
    hp1, p1, m1 = make_model(rank=1)
    m1.W0.zero_()
    np.testing.assert_allclose(oracle.evaluate(m1, pos, box, types).tensor, 0.0, atol=1e-13)


def test_isolated_atom():
    _, _, m = make_model(rank=2)
    r = oracle.evaluate(m, np.array([[0.0, 0.0, 0.0]]), None, np.array([1]))
    assert np.all(r.q == 0)
    U0 = float(m.w1[1] @ torch.tanh(-m.b0[1]) - m.b1[1])
    np.testing.assert_allclose(r.tensor.reshape(3, 3), U0 * np.eye(3), atol=1e-14)


def test_cubic_perovskite_symmetry():
    pos, types, box = synth.bzo_supercell(3)
    for rank in (1, 2):
        _, _, m = make_model(rank=rank, n_types=3)
        t = oracle.evaluate(m, pos, box, types).tensor
        if rank == 1:
            np.testing.assert_allclose(t, 0.0, atol=1e-10)
        else:
            a = t.reshape(3, 3)
            np.testing.assert_allclose(a - a[0, 0] * np.eye(3), 0.0, atol=1e-10)


def test_linearity_of_output_layer():
    _, _, m = make_model(rank=2)
    pos, types, box = small_cluster(4)
    t0 = oracle.evaluate(m, pos, box, types).tensor
    m.w1.mul_(2.5); m.b1.mul_(2.5)
    np.testing.assert_allclose(oracle.evaluate(m, pos, box, types).tensor, 2.5 * t0, rtol=1e-12, atol=1e-13)


def test_parameter_layout_probe():
    """One nonzero W0[t=1][mu=2][d=7] and w1[t=1][2]: only H atoms feel it."""
    hp = synth.HyperParams(n_types=2, rank=2)
    D, H = hp.dim, hp.n_hidden
    p = np.zeros(synth.n_params(hp), np.float32)
    per_net = H * D + 2 * H + 1
    p[per_net + 2 * D + 7] = 1.0            # W0[1][2][7]
    p[per_net + H * D + H + 2] = 1.0        # w1[1][2]
    coff = 2 * per_net
    nRk = 5 * 9
    p[coff: coff + 4 * nRk] = 0.0
    cA = coff + 4 * nRk
    # c_A[ti=1][tj=0][n=2][k=0] = 1 -> g_2 = f_0 for H centres with O neighbours
    p[cA + (1 * 2 + 0) * nRk + 2 * 9 + 0] = 1.0
    m = OracleModel.from_flat(hp, p, None, RC_R, RC_A)
    pos, types, box = small_cluster(3)
    r = oracle.evaluate(m, pos, box, types)
    assert np.all(r.U[types == 0] == 0)
    i, j, R = r.i, r.j, r.rij
    d = np.linalg.norm(R, axis=1)
    for a in np.nonzero(types == 1)[0]:
        sel = (i == a) & (d < RC_A) & (types[j] == 0)
        f0 = 0.5 * (1 + np.cos(np.pi * d[sel] / RC_A))
        u = R[sel] / d[sel][:, None]
        q_21 = np.sum(f0[:, None] * f0[None, :] * (u @ u.T))   # l=1, n=2 -> d = 5 + 0*5 + 2 = 7
        assert r.U[a] == pytest.approx(math.tanh(q_21), abs=1e-12)


# ------------------------------------------------------------ neighbour sets
def test_fp32_pairs_match_fp64():
    frames, types, box = synth.water_small(1)
    pos = frames[0]
    i, j, R = pairs_fp64(pos.astype(np.float64), box.astype(np.float64), RC_R)
    lists = oracle.neighbours_fp32(pos, box, RC_R)
    d = np.linalg.norm(R, axis=1)
    for a in range(len(pos)):
        ref = set(j[(i == a)].tolist())
        got = set(lists[a].tolist())
        diff = ref ^ got
        for b in diff:  # only pairs within rounding of the cutoff may differ
            dd = pos[b].astype(np.float64) - pos[a]
            dd -= box * np.round(dd / box)
            assert abs(np.linalg.norm(dd) - RC_R) < 1e-4
    assert sum(len(x) for x in lists) == pytest.approx(len(i), abs=4)
    assert d.max() < RC_R


def test_fp32_pairs_subset_matches_full():
    """The per-atom subset form (used on large frames) gives the same rows,
    on a periodic box and on a slab open along z."""
    rng = np.random.default_rng(5)
    for box in (np.array([15.1, 19.0, 19.0], np.float32), np.array([20.0, 19.0, 0.0], np.float32)):
        ext = np.where(box > 0, box, 15.0)
        pos = (rng.random((400, 3)) * ext).astype(np.float32)
        full = oracle.neighbours_fp32(pos, box, RC_R)
        atoms = rng.choice(len(pos), size=50, replace=False)
        sub = oracle.neighbours_fp32(pos, box, RC_R, atoms=atoms)
        for a, row in zip(atoms, sub):
            assert np.array_equal(row, full[a])


# ------------------------------------------------------------------ spectra
def test_acf_matches_fft_wiener_khinchin():
    rng = np.random.default_rng(3)
    T = 257
    s = rng.normal(size=(T, 3))
    C = oracle.acf(s, max_lag=100, kind=oracle.KIND_IR, subtract_mean=True)
    x = s - s.mean(0)
    F = np.fft.rfft(x, n=2 * T, axis=0)
    raw = np.fft.irfft(np.abs(F) ** 2, axis=0)[:101].sum(1)
    ref = raw / (T - np.arange(101)) / 3.0
    np.testing.assert_allclose(C, ref, atol=1e-12)


def test_spectrum_peak_and_constant():
    dt = 1.0
    T = 4000
    nu0 = 0.05  # fs^-1
    t = np.arange(T) * dt
    mu = np.stack([np.cos(2 * np.pi * nu0 * t), np.zeros(T), np.zeros(T)], 1)
    f, S = oracle.spectrum(mu, dt, oracle.KIND_IR, max_lag=1000)
    assert f[np.argmax(S)] == pytest.approx(nu0 / 2.99792458e-5, rel=2e-3)
    f, S = oracle.spectrum(np.ones((T, 3)), dt, oracle.KIND_IR, max_lag=100)
    np.testing.assert_allclose(S, 0.0, atol=1e-20)


def test_raman_iso_aniso_split():
    rng = np.random.default_rng(8)
    T = 300
    g = rng.normal(size=T)
    iso = g[:, None, None] * np.eye(3)
    C_aniso = oracle.acf(iso.reshape(T, 9), 50, oracle.KIND_RAMAN_ANISO)
    np.testing.assert_allclose(C_aniso, 0.0, atol=1e-14)
    C_iso = oracle.acf(iso.reshape(T, 9), 50, oracle.KIND_RAMAN_ISO)
    x = g - g.mean()
    np.testing.assert_allclose(C_iso[3], (x[:-3] * x[3:]).sum() / (T - 3), rtol=1e-13)
    # traceless symmetric part alone gives zero isotropic signal
    B = rng.normal(size=(T, 3, 3)); B = B + B.transpose(0, 2, 1)
    B -= np.trace(B, axis1=1, axis2=2)[:, None, None] * np.eye(3) / 3
    np.testing.assert_allclose(oracle.acf(B.reshape(T, 9), 20, oracle.KIND_RAMAN_ISO), 0.0, atol=1e-14)
    Bc = B - B.mean(0)
    ref = np.einsum("tab,tba->", Bc[:-2], Bc[2:]) / (T - 2)
    assert oracle.acf(B.reshape(T, 9), 20, oracle.KIND_RAMAN_ANISO)[2] == pytest.approx(ref, rel=1e-12)


def test_com_dipole_closed_forms():
    rng = np.random.default_rng(12)
    pos = rng.normal(size=(7, 3))
    types = np.array([0, 1, 1, 2, 0, 1, 2])
    masses = np.array([15.999, 1.008, 12.011])
    q = -1.0
    base = oracle.com_dipole(pos, types, masses, q)
    d = np.array([0.3, -1.2, 2.5])
    # translating the molecule by d moves the origin-referenced dipole by Q d
    np.testing.assert_allclose(oracle.com_dipole(pos + d, types, masses, q) - base, q * d, atol=1e-12)
    # neutral: no correction; one atom: Q r; equal masses: Q times the centroid
    assert np.all(oracle.com_dipole(pos, types, masses, 0.0) == 0.0)
    np.testing.assert_allclose(oracle.com_dipole(pos[:1], types[:1], masses, 2.0), 2.0 * pos[0])
    np.testing.assert_allclose(oracle.com_dipole(pos, np.zeros(7, int), masses, 1.0), pos.mean(0), atol=1e-14)
    # only mass ratios matter
    np.testing.assert_allclose(oracle.com_dipole(pos, types, 3.7 * masses, q), base, atol=1e-13)


# ----------------------------------------------------------------- general periodic cells
def test_cell_pairs_equal_minimum_image_for_large_orthorhombic_cells():
    rng = np.random.default_rng(40)
    pos, types, box = synth.water_box(64, rng, L=12.42)
    i0, j0, r0 = pairs_fp64(pos, box, RC_R)
    i1, j1, r1 = oracle.pairs_cell(pos, np.diag(box), RC_R)
    o0, o1 = np.lexsort((j0, i0)), np.lexsort((j1, i1))
    assert np.array_equal(i0[o0], i1[o1]) and np.array_equal(j0[o0], j1[o1])
    np.testing.assert_allclose(r0[o0], r1[o1], atol=1e-12)


@pytest.mark.parametrize("rank,L,n_mol,reps", [(1, 9.0, 24, 2), (2, 9.0, 24, 2), (2, 5.0, 3, 3)])
def test_small_cell_equals_its_supercell(rank, L, n_mol, reps):
    # cells shorter than 2 rc (the 5 A cube even shorter than rc: an atom sees
    # its own images): every image within the cutoff counts; the supercell of
    # edge >= 2 rc uses the plain minimum image instead
    _, _, m = make_model(rank=rank)
    rng = np.random.default_rng(41)
    pos, types, box = synth.water_box(n_mol, rng, L=L)
    small = oracle.evaluate(m, pos, None, types, cell=np.diag(box))
    shifts = [np.array([a, b, c]) for a in range(reps) for b in range(reps) for c in range(reps)]
    big_pos = np.concatenate([pos + L * sh for sh in shifts])
    big = oracle.evaluate(m, big_pos, np.full(3, reps * L), np.tile(types, len(shifts)))
    np.testing.assert_allclose(big.per_atom[:len(types)], small.per_atom, atol=1e-10 * np.abs(small.per_atom).max())
    np.testing.assert_allclose(big.tensor, len(shifts) * small.tensor, atol=1e-10 * np.abs(big.per_atom).sum())


def _sheared_cell():
    return np.array([[8.0, 0.0, 0.0], [2.5, 7.5, 0.0], [-1.5, 2.0, 8.5]])


def test_triclinic_cell_basis_change_and_supercell():
    _, _, m = make_model(rank=2)
    H = _sheared_cell()
    pos, types, _ = synth.cell_water(14, H, np.random.default_rng(42))
    ref = oracle.evaluate(m, pos, None, types, cell=H)
    # the same lattice in another basis (unimodular integer change)
    M = np.array([[1, 1, 0], [0, 1, 0], [1, 0, 1]])
    alt = oracle.evaluate(m, pos, None, types, cell=M @ H)
    np.testing.assert_allclose(alt.per_atom, ref.per_atom, atol=1e-10 * np.abs(ref.per_atom).max())
    # 2x1x1 supercell along a: every atom keeps its contribution
    big_pos = np.concatenate([pos, pos + H[0]])
    big = oracle.evaluate(m, big_pos, None, np.tile(types, 2), cell=np.diag([2, 1, 1]) @ H)
    np.testing.assert_allclose(big.per_atom[:len(types)], ref.per_atom, atol=1e-10 * np.abs(ref.per_atom).max())
    np.testing.assert_allclose(big.per_atom[len(types):], ref.per_atom, atol=1e-10 * np.abs(ref.per_atom).max())


def test_triclinic_cell_rotates_with_the_structure():
    _, _, m1 = make_model(rank=1)
    _, _, m2 = make_model(rank=2)
    H = _sheared_cell()
    pos, types, _ = synth.cell_water(12, H, np.random.default_rng(43))
    R = synth.random_rotation(np.random.default_rng(44))
    for m in (m1, m2):
        a = oracle.evaluate(m, pos, None, types, cell=H).tensor
        b = oracle.evaluate(m, pos @ R.T, None, types, cell=H @ R.T).tensor
        if m.rank == 1:
            np.testing.assert_allclose(b, R @ a, atol=1e-10 * np.abs(a).max())
        else:
            np.testing.assert_allclose(b.reshape(3, 3), R @ a.reshape(3, 3) @ R.T, atol=1e-10 * np.abs(a).max())


def test_lattice_translations_of_single_atoms_change_nothing():
    # moving atoms by whole lattice vectors (far outside the cell) is no change;
    # a strongly sheared cell, whose plane spacings are well below its edges
    _, _, m = make_model(rank=2)
    H = np.array([[7.0, 0.0, 0.0], [5.5, 6.5, 0.0], [4.0, -3.0, 7.5]])
    pos, types, _ = synth.cell_water(10, H, np.random.default_rng(45))
    ref = oracle.evaluate(m, pos, None, types, cell=H)
    moved = pos.copy()
    moved[3] += 3 * H[0] - 2 * H[2]
    moved[10] -= 4 * H[1]
    moved[17] += H[0] + H[1] + H[2]
    got = oracle.evaluate(m, moved, None, types, cell=H)
    np.testing.assert_allclose(got.per_atom, ref.per_atom, atol=1e-10 * np.abs(ref.per_atom).max())


def test_spectrum_row_selection_equals_full_rows():
    """oracle.spectrum(k_sel=...) returns the selected rows of the full
    transform (used where the full M x M cosine table would not fit)."""
    rng = np.random.default_rng(3)
    s = rng.normal(size=(300, 9))
    for kind in (oracle.KIND_IR, oracle.KIND_RAMAN_ANISO):
        ser = s[:, :3] if kind == oracle.KIND_IR else s
        f, S = oracle.spectrum(ser, 0.5, kind, max_lag=120)
        ks = np.array([0, 3, 77, 120])
        fk, Sk = oracle.spectrum(ser, 0.5, kind, max_lag=120, k_sel=ks)
        assert np.array_equal(fk, f[ks])
        np.testing.assert_allclose(Sk, S[ks], rtol=1e-14, atol=1e-14 * np.abs(S).max())
