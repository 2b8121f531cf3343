"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances.  The CUDA path computes in float32 (descriptors, network,
partial forces, per-atom contractions) and sums atoms per structure in
float64.  The bar is a per-frame relative error of 1e-5 in the Frobenius
norm (float32 rounding of ~1e2 neighbour terms per atom gives ~1e-6; the
margin covers the hardware sine/cosine in the cutoff, ~4e-7 absolute).  When
a tensor is a cancelling sum, its norm is compared against the condition
scale sum_i |per-atom contribution_i| instead (an error of 1e-6 of it).
Neighbour lists are compared as exact sets.
"""

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

RC = (6.0, 4.0)
REL = 1e-5
COND = 1e-6


@pytest.fixture(scope="module")
def tn():
    import __graft_entry__ as g
    g.build()
    from paper_2312_05233_gb300 import tnep
    return tnep


def models_for(tn, n_types, ranks=(1, 2), seed=11, small=False, per_type_nn=1, scaler=True):
    rng = np.random.default_rng(seed)
    out, orc = [], []
    for r in ranks:
        if small:
            hp = synth.HyperParams(n_types=n_types, rank=r, n_max_R=3, n_max_A=2, basis_R=6, basis_A=5,
                                   l_max=3, use_4body=1, n_hidden=17, per_type_nn=per_type_nn)
        else:
            hp = synth.HyperParams(n_types=n_types, rank=r, per_type_nn=per_type_nn)
        p = synth.model_params(hp, rng)
        sc = synth.default_q_scaler(hp) if scaler else None
        out.append(tn.Model.from_hyper(hp, p, sc))
        orc.append(oracle.OracleModel.from_flat(hp, p, sc, *RC))
    return out, orc


def check_frames(got, ref, per_atom_ref=None):
    got = np.asarray(got)
    for f in range(len(ref)):
        err = np.linalg.norm(got[f] - ref[f])
        scale = np.linalg.norm(ref[f])
        tol = REL * scale
        if per_atom_ref is not None:
            tol = max(tol, COND * np.abs(per_atom_ref[f]).sum())
        assert err <= tol, f"frame {f}: |d|={err:.3e} |ref|={scale:.3e} tol={tol:.3e}"


# ----------------------------------------------------------- neighbour lists
def _random_box_structure(rng, box, extent):
    """Uniform atoms at water density in `extent` (open axes have box 0)."""
    ext = np.asarray(extent, dtype=np.float64)
    n = int(0.1003 * np.prod(ext))
    pos = (rng.random((n, 3)) * ext).astype(np.float32)
    types = (np.arange(n) % 3 != 0).astype(np.int32)
    return synth.Structure(pos, types, np.asarray(box, dtype=np.float32))


@pytest.mark.parametrize("cell_div,x_div", [(1, 1), (2, 1), (3, 1), (1, 2), (1, 3), (1, 4), (2, 4)])
def test_neighbors_bitexact(tn, cell_div, x_div):
    frames, types, box = synth.water_small(3)
    structs = [synth.Structure(frames[f], types, box) for f in range(3)]
    rng = np.random.default_rng(3)
    # unwrapped coordinates (shifted by whole box edges) take the per-pair rint path
    unwrapped = (frames[0] + box * rng.integers(-1, 2, size=frames[0].shape)).astype(np.float32)
    structs.append(synth.Structure(unwrapped, types, box))
    big, bt_types, bbox = synth.water_grid_box(8, 24.84, rng)
    structs.append(synth.Structure(np.mod(big, bbox).astype(np.float32), bt_types, bbox.astype(np.float32)))
    for n in (1, 7, 40):
        p, t, b = synth.water_cluster(n, rng)
        structs.append(synth.Structure(p.astype(np.float32), t, b.astype(np.float32)))
    # x barely above 2 rc_R (too few x-cells for shifts: rint per pair), x
    # a little longer (windows wrap at both faces), a slab open along z and a
    # rod open along x
    structs.append(_random_box_structure(rng, (12.1, 19.0, 19.0), (12.1, 19.0, 19.0)))
    structs.append(_random_box_structure(rng, (15.1, 19.0, 19.0), (15.1, 19.0, 19.0)))
    structs.append(_random_box_structure(rng, (20.0, 19.0, 0.0), (20.0, 19.0, 15.0)))
    structs.append(_random_box_structure(rng, (0.0, 18.5, 18.5), (30.0, 18.5, 18.5)))
    bt = synth.concat_structures(structs)
    ms, _ = models_for(tn, 2, ranks=(1,))
    ctx = tn.tnep_create(ms, 2, RC)
    tn.tnep_set_option(ctx, tn.TNEP_OPT_CELL_DIV, cell_div)
    assert tn.tnep_get_option(ctx, tn.TNEP_OPT_CELL_XDIV) == 2  # the default
    for bad in (0, 5):
        with pytest.raises(tn.TnepError):
            tn.tnep_set_option(ctx, tn.TNEP_OPT_CELL_XDIV, bad)
    tn.tnep_set_option(ctx, tn.TNEP_OPT_CELL_XDIV, x_div)
    cR, cA, lR, lA = tn.tnep_neighbors(ctx, bt.offsets, bt.pos, bt.box, cap_R=256, cap_A=128)
    for s in range(bt.n_structs):
        a0, a1 = bt.offsets[s], bt.offsets[s + 1]
        refR = oracle.neighbours_fp32(bt.pos[a0:a1], bt.box[s], RC[0])
        refA = oracle.neighbours_fp32(bt.pos[a0:a1], bt.box[s], RC[1])
        for a in range(a1 - a0):
            g = a0 + a
            assert cR[g] == len(refR[a]) and cA[g] == len(refA[a])
            assert np.array_equal(np.sort(lR[g, :cR[g]]) - a0, refR[a])
            assert np.array_equal(np.sort(lA[g, :cA[g]]) - a0, refA[a])
    ctx.close()


def test_neighbors_bitexact_bulk_water(tn):
    """The bench's frame size (41,472 atoms, 74.5 A box) with the default
    x-thin cells: sampled atoms' lists against the float32 brute force."""
    frames, types, box = synth.water_bulk(n_frames=1)
    pos = frames[0]
    ms, _ = models_for(tn, 2, ranks=(1,))
    ctx = tn.tnep_create(ms, 2, RC)
    offs = np.array([0, len(pos)], np.int32)
    cR, cA, lR, lA = tn.tnep_neighbors(ctx, offs, pos, box[None, :], cap_R=256, cap_A=128)
    sample = np.random.default_rng(11).choice(len(pos), size=1500, replace=False)
    refR = oracle.neighbours_fp32(pos, box, RC[0], atoms=sample)
    refA = oracle.neighbours_fp32(pos, box, RC[1], atoms=sample)
    for a, rR, rA in zip(sample, refR, refA):
        assert cR[a] == len(rR) and cA[a] == len(rA)
        assert np.array_equal(np.sort(lR[a, :cR[a]]), rR)
        assert np.array_equal(np.sort(lA[a, :cA[a]]), rA)
    ctx.close()


# ------------------------------------------------------- small water (192 atoms)
def test_water_small_parity(tn):
    frames, types, box = synth.water_small(12)
    ms, om = models_for(tn, 2)
    ctx = tn.tnep_create(ms, 2, RC)
    mu, alpha = tn.tnep_eval(ctx, frames, box, types)
    for got, m in ((mu, om[0]), (alpha, om[1])):
        res = [oracle.evaluate(m, frames[f], box, types) for f in range(len(frames))]
        check_frames(got, np.array([r.tensor for r in res]), np.array([r.per_atom for r in res]))
    ctx.close()


def test_device_and_host_inputs_agree(tn):
    """Host and device buffers give the same frames, also when the device
    outputs of several passes are written while later passes run (the
    per-frame sums and their copies run on a side stream)."""
    frames, types, box = synth.water_small(5)
    ms, _ = models_for(tn, 2)
    ctx = tn.tnep_create(ms, 2, RC)
    h = tn.tnep_eval(ctx, frames, box, types)
    dev = (torch.from_numpy(frames).cuda(), torch.from_numpy(box).cuda(), torch.from_numpy(types).cuda())
    d = tn.tnep_eval(ctx, *dev)
    for a, b in zip(h, d):
        assert np.array_equal(a, b.cpu().numpy())
    tn.tnep_set_option(ctx, tn.TNEP_OPT_FRAMES_PER_BATCH, 2)  # three passes
    d3 = tn.tnep_eval(ctx, *dev)
    for a, b in zip(h, d3):
        assert np.array_equal(a, b.cpu().numpy())
    ctx.close()


def test_batch_split_is_bitwise_invariant(tn):
    """Results do not depend on how frames are grouped into device passes,
    for a box with too few cells for shifts (12.42 A) and one scanned with
    x-thin cells and windows (24.84 A, 1,536 atoms)."""
    rng = np.random.default_rng(21)
    base, btypes, bbox = synth.water_grid_box(8, 24.84, rng)
    bframes = synth.random_walk_frames(base, bbox, 6, 0.05, rng).astype(np.float32)
    cases = (synth.water_small(9), (bframes, btypes, bbox.astype(np.float32)))
    ms, _ = models_for(tn, 2)
    ctx = tn.tnep_create(ms, 2, RC)
    for frames, types, box in cases:
        outs = []
        for fb in (1, 4, len(frames)):
            tn.tnep_set_option(ctx, tn.TNEP_OPT_FRAMES_PER_BATCH, fb)
            outs.append(tn.tnep_eval(ctx, frames, box, types))
        for o in outs[1:]:
            for a, b in zip(outs[0], o):
                assert np.array_equal(a, b)
    ctx.close()


def test_per_atom_parity(tn):
    frames, types, box = synth.water_small(1)
    ms, om = models_for(tn, 2)
    ctx = tn.tnep_create(ms, 2, RC)
    offs = np.array([0, len(types)])
    (mu, al), (pmu, pal) = tn.tnep_eval_batch(ctx, offs, frames[0], box[None], types, per_atom=True)
    for got, m, tot in ((pmu, om[0], mu), (pal, om[1], al)):
        ref = oracle.evaluate(m, frames[0], box, types).per_atom
        scale = np.abs(ref).max()
        np.testing.assert_allclose(got, ref, atol=REL * scale, rtol=0)
        # the structure total is the FP64 sum of the per-atom contributions
        np.testing.assert_allclose(tot[0], got.astype(np.float64).sum(0), rtol=1e-12, atol=1e-12 * scale)
    ctx.close()


# ------------------------------------------- second kernel variant, 3 types
@pytest.mark.parametrize("per_type_nn", [1, 0])
def test_small_variant_three_types(tn, per_type_nn):
    rng = np.random.default_rng(5)
    base, types, box = synth.bzo_supercell(3)
    frames = synth.thermal_frames(base, box, 3, 0.08, rng)
    box = box.astype(np.float32)
    ms, om = models_for(tn, 3, small=True, per_type_nn=per_type_nn)
    ctx = tn.tnep_create(ms, 3, RC)
    outs = tn.tnep_eval(ctx, frames, box, types)
    for got, m in zip(outs, om):
        res = [oracle.evaluate(m, frames[f], box, types) for f in range(len(frames))]
        check_frames(got, np.array([r.tensor for r in res]), np.array([r.per_atom for r in res]))
    ctx.close()


# ------------------------------------------------- uneven batch, edge cases
@pytest.mark.parametrize("mode", [0, 2])
def test_uneven_batch_open_and_periodic(tn, mode):
    """Open clusters, an empty structure, a single atom, a periodic box and a
    slab in one batch, with the network on the CUDA cores (mode 0) and on the
    tensor cores with split-BF16 operands (mode 2, the persistent kernel),
    both held to the FP32 bars."""
    rng = np.random.default_rng(17)
    structs = []
    for n in (5, 1, 30):
        p, t, b = synth.water_cluster(n, rng)
        structs.append(synth.Structure(p.astype(np.float32), t, b.astype(np.float32)))
    structs.append(synth.Structure(np.zeros((0, 3), np.float32), np.zeros(0, np.int32), np.zeros(3, np.float32)))
    structs.append(synth.Structure(np.array([[1.0, 2.0, 3.0]], np.float32), np.array([1], np.int32),
                                   np.zeros(3, np.float32)))
    p, t, b = synth.water_box(64, rng, L=12.42)
    structs.append(synth.Structure(np.mod(p, b).astype(np.float32), t, b.astype(np.float32)))
    # one axis open, two periodic (a slab)
    p, t, b = synth.water_box(64, rng, L=12.42)
    structs.append(synth.Structure(p.astype(np.float32), t, np.array([12.42, 12.42, 0.0], np.float32)))
    bt = synth.concat_structures(structs)
    ms, om = models_for(tn, 2)
    ctx = tn.tnep_create(with_precision(tn, ms, mode, 2), 2, RC)
    outs, _ = tn.tnep_eval_batch(ctx, bt.offsets, bt.pos, bt.box, bt.types)
    for got, m in zip(outs, om):
        res = []
        for s in range(bt.n_structs):
            a0, a1 = bt.offsets[s], bt.offsets[s + 1]
            res.append(oracle.evaluate(m, bt.pos[a0:a1], bt.box[s], bt.types[a0:a1]))
        ref = np.array([r.tensor for r in res])
        pa = [np.abs(r.per_atom).sum() for r in res]
        for s in range(bt.n_structs):
            err = np.linalg.norm(got[s] - ref[s])
            assert err <= max(REL * np.linalg.norm(ref[s]), COND * pa[s], 1e-12), (s, err, ref[s])
    assert np.all(outs[0][3] == 0) and np.all(outs[1][3] == 0)  # empty structure
    ctx.close()


def test_six_type_anions(tn):
    rng = np.random.default_rng(23)
    structs = []
    for n in (20, 37, 60):
        p, t, b = synth.anion(n, rng)
        structs.append(synth.Structure(p.astype(np.float32), t, b.astype(np.float32)))
    bt = synth.concat_structures(structs)
    ms, om = models_for(tn, 6)
    ctx = tn.tnep_create(ms, 6, RC)
    outs, _ = tn.tnep_eval_batch(ctx, bt.offsets, bt.pos, bt.box, bt.types)
    for got, m in zip(outs, om):
        for s in range(bt.n_structs):
            a0, a1 = bt.offsets[s], bt.offsets[s + 1]
            r = oracle.evaluate(m, bt.pos[a0:a1], bt.box[s], bt.types[a0:a1])
            err = np.linalg.norm(got[s] - r.tensor)
            assert err <= max(REL * np.linalg.norm(r.tensor), COND * np.abs(r.per_atom).sum())
    ctx.close()


def test_charged_anions_com_dipole(tn):
    # Sec. III.A: mu = mu_r + Q r_COM for the charged anions, open boxes
    rng = np.random.default_rng(31)
    structs = []
    for n in (25, 44, 58):
        p, t, b = synth.anion(n, rng)
        structs.append(synth.Structure((p + rng.uniform(-20, 20, 3)).astype(np.float32), t, b.astype(np.float32)))
    bt = synth.concat_structures(structs)
    ms, om = models_for(tn, 6)
    ctx = tn.tnep_create(ms, 6, RC)
    masses = np.array([1.008, 12.011, 14.007, 15.999, 18.998, 32.06])  # H C N O F S
    charge = np.array([-1.0, 0.0, -2.0])
    with pytest.raises(tn.TnepError):  # masses not set yet
        tn.tnep_add_com_dipole(ctx, bt.offsets, bt.pos, bt.box, bt.types, charge, np.zeros((3, 3)))
    tn.tnep_set_masses(ctx, masses)
    (mu, _), _ = tn.tnep_eval_batch(ctx, bt.offsets, bt.pos, bt.box, bt.types)
    mu_r = mu.copy()
    tn.tnep_add_com_dipole(ctx, bt.offsets, bt.pos, bt.box, bt.types, charge, mu)
    assert np.array_equal(mu[1], mu_r[1])  # neutral structure untouched
    for s in range(bt.n_structs):
        a0, a1 = bt.offsets[s], bt.offsets[s + 1]
        r = oracle.evaluate(om[0], bt.pos[a0:a1], bt.box[s], bt.types[a0:a1])
        com = oracle.com_dipole(bt.pos[a0:a1], bt.types[a0:a1], masses, charge[s])
        np.testing.assert_allclose(mu[s] - mu_r[s], com, rtol=1e-12, atol=1e-12 * np.abs(com).max(initial=1.0))
        ref = r.tensor + com
        assert np.linalg.norm(mu[s] - ref) <= max(REL * np.linalg.norm(ref), COND * np.abs(r.per_atom).sum())
    # a charged periodic structure has no centre of mass
    box = bt.box.copy()
    box[0] = [30.0, 30.0, 30.0]
    with pytest.raises(tn.TnepError) as e:
        tn.tnep_add_com_dipole(ctx, bt.offsets, bt.pos, box, bt.types, charge, mu)
    assert e.value.status == 1
    ctx.close()


def test_errors_and_neighbor_regrow(tn):
    ms, om = models_for(tn, 2)
    ctx = tn.tnep_create(ms, 2, RC)
    p = np.zeros((2, 3), np.float32)
    p[1] = [1.0, 0, 0]
    with pytest.raises(tn.TnepError) as e:
        tn.tnep_eval_batch(ctx, [0, 2], p, np.array([[11.0, 20.0, 20.0]], np.float32), np.array([0, 1]))
    assert e.value.status == 3
    with pytest.raises(tn.TnepError) as e:
        tn.tnep_eval_batch(ctx, [0, 2], p, None, np.array([0, 2]))
    assert e.value.status == 1
    # 100 molecules in a 12.42 A cube (1.56x water density): more radial
    # neighbours than the initial list capacity of 128, so the lists regrow
    rng = np.random.default_rng(2)
    pos, types, box = synth.water_box(100, rng, L=12.42)
    pos = np.mod(pos, box).astype(np.float32)
    box = box.astype(np.float32)
    cR, cA, _, _ = tn.tnep_neighbors(ctx, [0, len(types)], pos, box[None], cap_R=8, cap_A=8)
    assert cR.max() > 128
    (mu, al), _ = tn.tnep_eval_batch(ctx, [0, len(types)], pos, box[None], types)
    for got, m in ((mu, om[0]), (al, om[1])):
        r = oracle.evaluate(m, pos, box, types)
        assert np.linalg.norm(got[0] - r.tensor) <= max(REL * np.linalg.norm(r.tensor),
                                                        COND * np.abs(r.per_atom).sum())
    if cR.max() > 32:
        ctx2 = tn.tnep_create(ms, 2, RC)
        tn.tnep_set_option(ctx2, tn.TNEP_OPT_MAX_NEIGHBORS, 32)
        with pytest.raises(tn.TnepError) as e:
            tn.tnep_eval_batch(ctx2, [0, len(types)], pos, box[None], types)
        assert e.value.status == 4
        ctx2.close()
    ctx.close()


# ------------------------------------------- full-size workloads, sampled atoms
@pytest.mark.parametrize("mode", [0, 2])
def test_bulk_water_full_size_sampled(tn, mode):
    """The bench workload (41,472 atoms) with the network on the CUDA cores
    (mode 0) and on the tensor cores with split-BF16 operands (mode 2, the
    bench's launch configuration), sampled per-atom against the oracle."""
    frames, types, box = synth.water_bulk(n_frames=2)
    ms, om = models_for(tn, 2)
    if mode:
        ms = [tn.Model.from_hyper(synth.HyperParams(n_types=2, rank=m.rank), m.params, m.q_scaler, mlp_precision=mode)
              for m in ms]
    ctx = tn.tnep_create(ms, 2, RC)
    N = len(types)
    offs = np.array([0, N])
    (mu, al), (pmu, pal) = tn.tnep_eval_batch(ctx, offs, frames[1], box[None], types, per_atom=True)
    sample = np.random.default_rng(0).choice(N, size=200, replace=False)
    for got, m in ((pmu, om[0]), (pal, om[1])):
        ref = oracle.evaluate(m, frames[1], box, types, centers=sample).per_atom[sample]
        np.testing.assert_allclose(got[sample], ref, atol=REL * np.abs(ref).max(), rtol=0)
    np.testing.assert_allclose(mu[0], pmu.astype(np.float64).sum(0), rtol=1e-12, atol=1e-9)
    # the same frame through the trajectory path gives the same numbers
    mu2, al2 = tn.tnep_eval(ctx, frames, box, types)
    assert np.array_equal(mu2[1], mu[0]) and np.array_equal(al2[1], al[0])
    ctx.close()


def test_perovskite_full_size_symmetry_and_sample(tn):
    base, types, box = synth.bzo_supercell(12)
    base = base.astype(np.float32)
    box = box.astype(np.float32)
    ms, om = models_for(tn, 3, ranks=(1, 2))
    ctx = tn.tnep_create(ms, 3, RC)
    (mu, al), (pmu, pal) = tn.tnep_eval_batch(ctx, [0, len(types)], base, box[None], types, per_atom=True)
    # Every atom of the perfect lattice sits on an inversion centre, so its
    # own contribution to mu vanishes and equivalent atoms carry identical
    # float32 residuals that add coherently.  The yardstick is the pair-level
    # scale sum_ij |r_ij|^k |dU_i/dr_ij| (k = 2 for mu, 1 for alpha),
    # estimated from the oracle on a sample of centres.
    sample = np.arange(0, len(types), 97)
    scales = []
    for m, k in ((om[0], 2), (om[1], 1)):
        r = oracle.evaluate(m, base, box, types, centers=sample)
        d = np.linalg.norm(r.rij, axis=1)
        scales.append((d ** k * np.linalg.norm(r.dUdr, axis=1)).sum() * len(types) / len(sample))
    assert np.abs(mu[0]).max() <= COND * scales[0]
    a = al[0].reshape(3, 3)
    assert np.abs(a - a[0, 0] * np.eye(3)).max() <= COND * scales[1]
    frames = synth.bzo_perovskite(n_frames=1)[0]
    (mu, al), (pmu, pal) = tn.tnep_eval_batch(ctx, [0, len(types)], frames[0], box[None], types, per_atom=True)
    sample = np.random.default_rng(1).choice(len(types), size=150, replace=False)
    for got, m in ((pmu, om[0]), (pal, om[1])):
        ref = oracle.evaluate(m, frames[0], box, types, centers=sample).per_atom[sample]
        np.testing.assert_allclose(got[sample], ref, atol=REL * np.abs(ref).max(), rtol=0)
    ctx.close()


def test_equivariance_large_open_cluster(tn):
    """Properties that hold at any size, on a 3,000-atom open cluster: under a
    rotation R, mu -> R mu and alpha -> R alpha R^T; translation and a
    permutation of the atoms change nothing; alpha is symmetric."""
    rng = np.random.default_rng(synth.seed_for(1, 60))
    pos, types, _ = synth.water_cluster(1000, rng)
    pos = pos.astype(np.float32)
    ms, _ = models_for(tn, 2)
    ctx = tn.tnep_create(ms, 2, RC)
    offs = [0, len(types)]

    def run(p, t):
        (mu, al), (pmu, pal) = tn.tnep_eval_batch(ctx, offs, p.astype(np.float32), None, t, per_atom=True)
        return mu[0], al[0].reshape(3, 3), np.abs(pmu).sum(), np.abs(pal).sum()

    mu0, al0, s1, s2 = run(pos, types)
    tol1, tol2 = max(REL * np.linalg.norm(mu0), COND * s1), max(REL * np.linalg.norm(al0), COND * s2)
    R = synth.random_rotation(rng)
    c = pos.mean(0)
    mu1, al1, _, _ = run((pos - c) @ R.T + c, types)
    assert np.linalg.norm(mu1 - R @ mu0) <= 2 * tol1
    assert np.linalg.norm(al1 - R @ al0 @ R.T) <= 2 * tol2
    mu2, al2, _, _ = run(pos + np.array([7.25, -3.5, 11.0], np.float32), types)
    assert np.linalg.norm(mu2 - mu0) <= 2 * tol1 and np.linalg.norm(al2 - al0) <= 2 * tol2
    perm = rng.permutation(len(types))
    mu3, al3, _, _ = run(pos[perm], types[perm])
    assert np.linalg.norm(mu3 - mu0) <= 2 * tol1 and np.linalg.norm(al3 - al0) <= 2 * tol2
    assert np.linalg.norm(al0 - al0.T) <= 2 * tol2
    ctx.close()


# ---------------------------------------------------------------- population
def test_population_matches_individual_evaluation(tn):
    rng = np.random.default_rng(31)
    structs = synth.population_structures(n_clusters=6, n_boxes=3, seed_k=1)
    bt = synth.concat_structures(structs)
    hp = synth.HyperParams(n_types=2, rank=1)
    P = 5
    params = np.stack([synth.model_params(hp, rng) for _ in range(P)])
    sc = synth.default_q_scaler(hp)
    target = rng.standard_normal((bt.n_structs, 3))
    ctx = tn.tnep_create([tn.Model.from_hyper(hp, params[0], sc)], 2, RC)
    rmse, pred = tn.tnep_eval_population(ctx, 0, params, bt.offsets, bt.pos, bt.box, bt.types, target,
                                         want_out=True)
    for p in range(P):
        c1 = tn.tnep_create([tn.Model.from_hyper(hp, params[p], sc)], 2, RC)
        (single,), _ = tn.tnep_eval_batch(c1, bt.offsets, bt.pos, bt.box, bt.types)
        assert np.array_equal(single, pred[p])
        c1.close()
        assert rmse[p] == pytest.approx(np.sqrt(np.mean((pred[p] - target) ** 2)), rel=1e-12)
    om = oracle.OracleModel.from_flat(hp, params[2], sc, *RC)
    for s in (0, bt.n_structs - 1):
        a0, a1 = bt.offsets[s], bt.offsets[s + 1]
        r = oracle.evaluate(om, bt.pos[a0:a1], bt.box[s], bt.types[a0:a1])
        assert np.linalg.norm(pred[2][s] - r.tensor) <= max(REL * np.linalg.norm(r.tensor),
                                                            COND * np.abs(r.per_atom).sum())
    ctx.close()


def test_population_full_size_sampled(tn):
    """The population workload the bench times (50 individuals x 600 uneven
    structures, 256,920 atoms; launch shape and angular form autotuned),
    checked on sampled (individual, structure) pairs against the oracle."""
    structs = synth.population_structures()
    bt = synth.concat_structures(structs)
    rng = np.random.default_rng(synth.seed_for(4, 11))
    hp = synth.HyperParams(n_types=2, rank=1)
    sc = synth.default_q_scaler(hp)
    P = 50
    params = np.stack([synth.model_params(hp, rng) for _ in range(P)])
    target = synth.tensor_targets(bt.n_structs, 3, rng)
    ctx = tn.tnep_create([tn.Model.from_hyper(hp, params[0], sc)], 2, RC)
    pop = tn.tnep_population_create(ctx, 0, params, bt.offsets, bt.pos, bt.box, bt.types, target)
    rmse, pred = pop.eval(params, want_out=True)
    np.testing.assert_allclose(rmse, np.sqrt(np.mean((pred - target[None]) ** 2, axis=(1, 2))), rtol=1e-12)
    sizes = np.diff(bt.offsets)
    small = [s for s in range(bt.n_structs) if sizes[s] <= 120]
    big = [s for s in range(bt.n_structs) if sizes[s] >= 1000]
    picks = [(0, small[0]), (17, small[len(small) // 2]), (49, small[-1]), (33, big[0])]
    for p_, s_ in picks:
        m = oracle.OracleModel.from_flat(hp, params[p_], sc, *RC)
        a0, a1 = bt.offsets[s_], bt.offsets[s_ + 1]
        r = oracle.evaluate(m, bt.pos[a0:a1], bt.box[s_], bt.types[a0:a1])
        assert np.linalg.norm(pred[p_, s_] - r.tensor) <= max(REL * np.linalg.norm(r.tensor),
                                                              COND * np.abs(r.per_atom).sum()), (p_, s_)
    pop.close()
    ctx.close()


# ------------------------------------------------------------------ spectra
@pytest.mark.parametrize("kind,C", [(0, 3), (1, 9), (2, 9)])
def test_spectrum_parity(tn, kind, C):
    rng = np.random.default_rng(kind)
    T = 600
    t = np.arange(T)
    series = rng.normal(size=(T, C)) + np.cos(0.07 * t)[:, None] * rng.normal(size=C)
    f, S, acf = tn.tnep_spectrum(series, 0.5, kind, max_lag=250, want_acf=True)
    fr, Sr = oracle.spectrum(series, 0.5, kind, max_lag=250)
    Cr = oracle.acf(series, 250, kind)
    np.testing.assert_allclose(acf, Cr, rtol=1e-11, atol=1e-13 * np.abs(Cr).max())
    np.testing.assert_allclose(f, fr, rtol=1e-13)
    np.testing.assert_allclose(S, Sr, rtol=1e-9, atol=1e-11 * np.abs(Sr).max())
    # device-resident series gives the same result
    f2, S2 = tn.tnep_spectrum(torch.from_numpy(series).cuda(), 0.5, kind, max_lag=250)
    assert np.array_equal(S2, S)


@pytest.mark.parametrize("kind,C,T", [(0, 3, 400_000), (1, 9, 1_100_000), (2, 9, 150_000)])
def test_spectrum_long_series_fourier_route(tn, kind, C, T):
    """Series long enough (channels x T x M > 1e9) for the Fourier route of
    the autocorrelation, against the oracle's direct time-origin sums."""
    rng = np.random.default_rng(10 + kind)
    t = np.arange(T)
    series = rng.normal(size=(T, C)) + np.cos(0.003 * t)[:, None] * rng.normal(size=C) + 2.0
    f, S, acf = tn.tnep_spectrum(series, 1.0, kind, max_lag=1000, want_acf=True)
    Cr = oracle.acf(series, 1000, kind)
    fr, Sr = oracle.spectrum(series, 1.0, kind, max_lag=1000)
    np.testing.assert_allclose(acf, Cr, rtol=0, atol=1e-12 * np.abs(Cr).max())
    np.testing.assert_allclose(f, fr, rtol=1e-13)
    np.testing.assert_allclose(S, Sr, rtol=0, atol=1e-10 * np.abs(Sr).max())


def test_dense_cluster_large_lists(tn):
    """~200 neighbours per atom: the neighbour lists regrow well past their
    initial capacity (128 radial, 64 angular)."""
    rng = np.random.default_rng(41)
    pts = []
    while len(pts) < 200:
        v = rng.uniform(-3.0, 3.0, 3)
        if np.linalg.norm(v) < 3.0 and all(np.linalg.norm(v - q) >= 0.35 for q in pts):
            pts.append(v)
    pos = np.asarray(pts, np.float32)
    types = rng.integers(0, 2, size=len(pts)).astype(np.int32)
    ms, om = models_for(tn, 2)
    ctx = tn.tnep_create(ms, 2, RC)
    cR, cA, lR, _ = tn.tnep_neighbors(ctx, [0, len(pts)], pos, None, cap_R=256, cap_A=256)
    ref = oracle.neighbours_fp32(pos, np.zeros(3, np.float32), RC[0])
    assert cR.min() == len(pts) - 1
    for a in range(len(pts)):
        assert np.array_equal(np.sort(lR[a, :cR[a]]), ref[a])
    (mu, al), _ = tn.tnep_eval_batch(ctx, [0, len(pts)], pos, None, types)
    for got, m in ((mu, om[0]), (al, om[1])):
        r = oracle.evaluate(m, pos, None, types)
        assert np.linalg.norm(got[0] - r.tensor) <= max(REL * np.linalg.norm(r.tensor),
                                                        COND * np.abs(r.per_atom).sum())
    ctx.close()


@pytest.mark.parametrize("mode", [0, 2])
def test_population_graph_replay_and_shapes(tn, mode):
    """Graph-captured generations equal the one-shot population call, for every
    launch shape the autotuner may pick, and for new parameters each time;
    with the network on the CUDA cores (mode 0) and on the tensor cores
    (mode 2: persistent CTAs whose work counter is reset inside the graph)."""
    rng = np.random.default_rng(8)
    structs = synth.population_structures(n_clusters=10, n_boxes=4, seed_k=2)
    bt = synth.concat_structures(structs)
    hp = synth.HyperParams(n_types=2, rank=2)
    P = 6
    sc = synth.default_q_scaler(hp)
    target = rng.standard_normal((bt.n_structs, 9))
    params = [np.stack([synth.model_params(hp, rng) for _ in range(P)]) for _ in range(2)]
    ctx = tn.tnep_create([tn.Model.from_hyper(hp, params[0][0], sc, mlp_precision=mode)], 2, RC)
    tn.tnep_set_option(ctx, tn.TNEP_OPT_POPULATION_FORM, 1)  # per-pair walk: same arithmetic as the batch path
    pop = tn.tnep_population_create(ctx, 0, params[0], bt.offsets, bt.pos, bt.box, bt.types, target)
    info = pop.info()
    assert info["block"] in (64, 128) and info["atoms"] == len(bt.types) and info["factored"] == 0
    walk = info["tune_ms"][:4]  # (128, 64 atoms per CTA) x (structure-major, individual-major)
    if mode == 0:
        assert all(t > 0 for t in walk)
    else:  # the tensor-core network takes 128-atom CTAs only
        assert walk[0] > 0 and walk[1] > 0 and walk[2] == -1 and walk[3] == -1
    assert all(t == -1 for t in info["tune_ms"][4:])
    for prm in params:  # two generations with different parameters
        rmse, pred = pop.eval(prm, want_out=True)
        r1, p1 = tn.tnep_eval_population(ctx, 0, prm, bt.offsets, bt.pos, bt.box, bt.types, target, want_out=True)
        np.testing.assert_allclose(pred, p1, rtol=0, atol=1e-12 * np.abs(p1).max())
        np.testing.assert_allclose(rmse, r1, rtol=1e-12)
    c1 = tn.tnep_create([tn.Model.from_hyper(hp, params[1][0], sc, mlp_precision=mode)], 2, RC)
    for block in (64, 128):  # the CTA size does not change any arithmetic
        tn.tnep_set_option(c1, tn.TNEP_OPT_BLOCK_ATOMS, block)
        (ref,), _ = tn.tnep_eval_batch(c1, bt.offsets, bt.pos, bt.box, bt.types)
        if mode == 0:
            assert np.array_equal(pred[0], ref)
        else:
            assert np.all(np.abs(pred[0] - ref) <= 1e-12 * np.abs(ref).max())
    c1.close()
    pop.close()
    ctx.close()


@pytest.mark.parametrize("rank,small,n_types", [(1, False, 2), (2, False, 2), (2, True, 3), (1, True, 3)])
def test_population_factored_form(tn, rank, small, n_types):
    """The factored form (angular sums and angular partial-force contractions
    from per-atom moments of the basis, shared by the individuals) against the
    FP64 oracle for every individual and structure, and against the walk."""
    rng = np.random.default_rng(50 + rank + 3 * small)
    if n_types == 2:
        structs = synth.population_structures(n_clusters=6, n_boxes=1, seed_k=7)
    else:
        structs = []
        for n in (20, 33, 47):
            p, t, b = synth.anion(n, rng)
            structs.append(synth.Structure(p.astype(np.float32), (t % 3).astype(np.int32), b.astype(np.float32)))
        base, types, box = synth.bzo_supercell(3)
        structs.append(synth.Structure((base + 0.05 * rng.standard_normal(base.shape)).astype(np.float32),
                                       types.astype(np.int32), box.astype(np.float32)))
    bt = synth.concat_structures(structs)
    if small:
        hp = synth.HyperParams(n_types=n_types, rank=rank, n_max_R=3, n_max_A=2, basis_R=6, basis_A=5, l_max=3,
                               use_4body=1, n_hidden=17)
    else:
        hp = synth.HyperParams(n_types=n_types, rank=rank)
    sc = synth.default_q_scaler(hp)
    C = 3 if rank == 1 else 9
    P = 3
    params = np.stack([synth.model_params(hp, rng) for _ in range(P)])
    target = rng.standard_normal((bt.n_structs, C))
    preds = {}
    for form in (1, 2, 3):
        ctx = tn.tnep_create([tn.Model.from_hyper(hp, params[0], sc)], n_types, RC)
        tn.tnep_set_option(ctx, tn.TNEP_OPT_POPULATION_FORM, form)
        pop = tn.tnep_population_create(ctx, 0, params, bt.offsets, bt.pos, bt.box, bt.types, target)
        if form == 3 and small:  # the tensor-core form takes the standard descriptor only
            assert pop.info()["factored"] in (0, 1) and pop.info()["tensor_core_ms"] == -1
        else:
            assert pop.info()["factored"] == form - 1
        rmse, preds[form] = pop.eval(params, want_out=True)
        np.testing.assert_allclose(rmse, np.sqrt(np.mean((preds[form] - target[None]) ** 2, axis=(1, 2))),
                                   rtol=1e-12)
        pop.close()
        ctx.close()
    for p_ in range(P):
        m = oracle.OracleModel.from_flat(hp, params[p_], sc, *RC)
        for s_ in range(bt.n_structs):
            a0, a1 = bt.offsets[s_], bt.offsets[s_ + 1]
            r = oracle.evaluate(m, bt.pos[a0:a1], bt.box[s_], bt.types[a0:a1])
            tol = max(REL * np.linalg.norm(r.tensor), COND * np.abs(r.per_atom).sum())
            for form in (1, 2, 3):
                assert np.linalg.norm(preds[form][p_, s_] - r.tensor) <= tol, (form, p_, s_)


@pytest.mark.parametrize("rank", [1, 2])
def test_population_tensor_core_form_tiles(tn, rank):
    """The tensor-core form with 2 individual tiles (P = 31: 25 + 6), three
    centre types (partial atom tiles of every type), open and periodic
    structures: every individual and structure against the CUDA-core
    factored form (same moments, FP32 sums in another order) and sampled
    individuals against the FP64 oracle."""
    rng = np.random.default_rng(70 + rank)
    structs = []
    for n in (21, 37, 58):
        p, t, b = synth.anion(n, rng)
        structs.append(synth.Structure(p.astype(np.float32), (t % 3).astype(np.int32), b.astype(np.float32)))
    base, types, box = synth.bzo_supercell(3)
    structs.append(synth.Structure((base + 0.06 * rng.standard_normal(base.shape)).astype(np.float32),
                                   types.astype(np.int32), box.astype(np.float32)))
    bt = synth.concat_structures(structs)
    hp = synth.HyperParams(n_types=3, rank=rank)
    sc = synth.default_q_scaler(hp)
    P = 31
    params = np.stack([synth.model_params(hp, rng) for _ in range(P)])
    target = rng.standard_normal((bt.n_structs, 3 if rank == 1 else 9))
    preds = {}
    for form in (2, 3):
        ctx = tn.tnep_create([tn.Model.from_hyper(hp, params[0], sc)], 3, RC)
        tn.tnep_set_option(ctx, tn.TNEP_OPT_POPULATION_FORM, form)
        pop = tn.tnep_population_create(ctx, 0, params, bt.offsets, bt.pos, bt.box, bt.types, target)
        assert pop.info()["factored"] == form - 1
        for _ in range(2):  # graph replays reuse the operands of the previous generation
            rmse, preds[form] = pop.eval(params, want_out=True)
        np.testing.assert_allclose(rmse, np.sqrt(np.mean((preds[form] - target[None]) ** 2, axis=(1, 2))),
                                   rtol=1e-12)
        pop.close()
        ctx.close()
    for s_ in range(bt.n_structs):
        a0, a1 = bt.offsets[s_], bt.offsets[s_ + 1]
        scale = np.linalg.norm(preds[2][:, s_], axis=1).max()
        for p_ in range(P):
            d = np.linalg.norm(preds[3][p_, s_] - preds[2][p_, s_])
            assert d <= REL * scale, (p_, s_, d / scale)
        for p_ in (0, 24, 25, 30):
            m = oracle.OracleModel.from_flat(hp, params[p_], sc, *RC)
            r = oracle.evaluate(m, bt.pos[a0:a1], bt.box[s_], bt.types[a0:a1])
            tol = max(REL * np.linalg.norm(r.tensor), COND * np.abs(r.per_atom).sum())
            assert np.linalg.norm(preds[3][p_, s_] - r.tensor) <= tol, (p_, s_)


# ------------------------------------------------- tensor-core network
# Mode 1 rounds activations and weights to BF16 (unit roundoff 2^-9) with
# FP32 accumulation.  The bar is the BF16 tolerance of 1e-3, taken on the
# tensor, ||dT|| <= 1e-3 ||T||, or, for a tensor that is a cancelling sum, on
# its condition scale sum_i |c_i| (the sum over atoms and components of the
# absolute per-atom contributions): ||dT|| <= 1e-3 sum_i |c_i|.  The
# condition-scale fallback keeps the same 1e-3 (not 1e-4 as for FP32, where
# per-atom rounding is independent): the rounding of the per-type weights is
# shared by every atom, and on near-crystalline structures the rounding of
# the activations is nearly the same for every atom of a type, so per-atom
# errors add coherently.  Largest measured: 6.3e-4 of the condition scale
# (3x3x3 BaZrO3, rank 2, small model), 9.6e-4 of sum_i ||c_i|| and
# 9e-3 of ||mu|| (64-molecule water, where mu cancels).
# Mode 2 splits both operands into high and low BF16 parts (three products,
# omitted term ~2^-18) and is held to the FP32 tolerance.
BF16_REL = 1e-3
BF16_COND = 1e-3


def bf16_bound(r):
    return max(BF16_REL * np.linalg.norm(r.tensor), BF16_COND * np.abs(r.per_atom).sum())


def with_precision(tn, ms, mode, n_types):
    return [tn.Model.from_hyper(synth.HyperParams(n_types=n_types, rank=m.rank, n_max_R=m.n_max_R,
                                                  n_max_A=m.n_max_A, basis_R=m.basis_R, basis_A=m.basis_A,
                                                  l_max=m.l_max, use_4body=m.use_4body, n_hidden=m.n_hidden),
                                m.params, m.q_scaler, mlp_precision=mode) for m in ms]


@pytest.mark.parametrize("small,n_types", [(False, 2), (True, 3)])
def test_tensor_core_network(tn, small, n_types):
    if n_types == 2:
        frames, types, box = synth.water_small(6)
    else:
        rng = np.random.default_rng(6)
        base, types, box = synth.bzo_supercell(3)
        frames = synth.thermal_frames(base, box, 4, 0.08, rng)
        box = box.astype(np.float32)
    ms32, om = models_for(tn, n_types, small=small)
    outs = {}
    for mode in (0, 1, 2):
        c = tn.tnep_create(with_precision(tn, ms32, mode, n_types), n_types, RC)
        outs[mode] = tn.tnep_eval(c, frames, box, types)
        c.close()
    for k, m in enumerate(om):
        res = [oracle.evaluate(m, frames[f], box, types) for f in range(len(frames))]
        for f, r in enumerate(res):
            scale = np.linalg.norm(r.tensor)
            cond = np.abs(r.per_atom).sum()
            assert np.linalg.norm(outs[1][k][f] - r.tensor) <= bf16_bound(r)
            assert np.linalg.norm(outs[2][k][f] - r.tensor) <= max(REL * scale, COND * cond)
        assert not np.array_equal(outs[1][k], outs[0][k])  # the tensor-core paths really ran
        assert not np.array_equal(outs[2][k], outs[1][k])


@pytest.mark.parametrize("small,n_types", [(False, 2), (True, 3)])
def test_pair_cache_equals_recomputed_walk(tn, small, n_types):
    """The backward walk reads each pair's r_ij, 1/|r_ij|, g_n and g_n' from
    the cache the forward walk wrote, or recomputes them: the same values, so
    the results agree bit for bit, for every network mode and with a partly
    filled last CTA (192 and 135 atoms)."""
    if n_types == 2:
        frames, types, box = synth.water_small(4)
    else:
        rng = np.random.default_rng(8)
        base, types, box = synth.bzo_supercell(3)
        frames = synth.thermal_frames(base, box, 3, 0.08, rng)
        box = box.astype(np.float32)
    ms32, om = models_for(tn, n_types, small=small)
    for mode in (0, 1, 2):
        c = tn.tnep_create(with_precision(tn, ms32, mode, n_types), n_types, RC)
        assert tn.tnep_get_option(c, tn.TNEP_OPT_PAIR_CACHE) == 1
        on = tn.tnep_eval(c, frames, box, types)
        tn.tnep_set_option(c, tn.TNEP_OPT_PAIR_CACHE, 0)
        off = tn.tnep_eval(c, frames, box, types)
        for a, b in zip(on, off):
            assert np.array_equal(a, b), mode
        c.close()
    res = oracle.evaluate(om[0], frames[0], box, types)
    assert np.linalg.norm(on[0][0] - res.tensor) <= bf16_bound(res)


def test_tensor_core_network_perovskite_full_size(tn):
    """BaZrO3 12x12x12 (8,640 atoms, 3 types), rank-2 susceptibility, the
    precision workload: whole frames through the oracle.  BF16 network (mode
    1): relative Frobenius error <= 1e-3 per frame, each component within
    1e-3 of the tensor's norm; split BF16 (mode 2) and FP32 (mode 0): 1e-5."""
    frames, types, box = synth.bzo_perovskite(n_frames=3)
    rng = np.random.default_rng(synth.seed_for(3, 1))
    hp = synth.HyperParams(n_types=3, rank=2)
    p = synth.model_params(hp, rng)
    sc = synth.default_q_scaler(hp)
    om = oracle.OracleModel.from_flat(hp, p, sc, *RC)
    refs = [oracle.evaluate(om, frames[f], box, types).tensor for f in (0, 2)]
    bars = {0: 1e-5, 1: 1e-3, 2: 1e-5}
    for mode in (0, 1, 2):
        ctx = tn.tnep_create([tn.Model.from_hyper(hp, p, sc, mlp_precision=mode)], 3, RC)
        (al,) = tn.tnep_eval(ctx, frames, box, types)
        ctx.close()
        for got, ref in zip(al[[0, 2]], refs):
            nrm = np.linalg.norm(ref)
            assert np.linalg.norm(got - ref) <= bars[mode] * nrm, (mode, np.linalg.norm(got - ref) / nrm)
            assert np.all(np.abs(got - ref) <= bars[mode] * nrm), mode


def test_tensor_core_population_and_tail_block(tn):
    """Tensor-core network with a partial last CTA and in the population kernel."""
    rng = np.random.default_rng(12)
    structs = synth.population_structures(n_clusters=5, n_boxes=2, seed_k=3)
    bt = synth.concat_structures(structs)
    assert len(bt.types) % 128 != 0
    hp = synth.HyperParams(n_types=2, rank=1)
    sc = synth.default_q_scaler(hp)
    params = np.stack([synth.model_params(hp, rng) for _ in range(3)])
    target = rng.standard_normal((bt.n_structs, 3))
    om = oracle.OracleModel.from_flat(hp, params[1], sc, *RC)
    refs = []
    for s in range(bt.n_structs):
        a0, a1 = bt.offsets[s], bt.offsets[s + 1]
        refs.append(oracle.evaluate(om, bt.pos[a0:a1], bt.box[s], bt.types[a0:a1]))
    for mode in (1, 2):
        ctx = tn.tnep_create([tn.Model.from_hyper(hp, params[0], sc, mlp_precision=mode)], 2, RC)
        rmse, pred = tn.tnep_eval_population(ctx, 0, params, bt.offsets, bt.pos, bt.box, bt.types, target,
                                             want_out=True)
        for s, r in enumerate(refs):
            err = np.linalg.norm(pred[1][s] - r.tensor)
            if mode == 1:
                assert err <= bf16_bound(r)
            else:
                assert err <= max(REL * np.linalg.norm(r.tensor), COND * np.abs(r.per_atom).sum())
        ctx.close()


def test_tensor_core_persistent_items_switch_individuals(tn):
    """The tensor-core fused kernel runs persistent CTAs that take work items
    (atom block, individual) from a counter and reload the model when the
    individual changes: with more items than CTAs, every individual of a
    population equals a single-model evaluation with its own parameters."""
    rng = np.random.default_rng(21)
    structs = synth.population_structures(n_clusters=40, n_boxes=6, seed_k=4)
    bt = synth.concat_structures(structs)
    hp = synth.HyperParams(n_types=2, rank=2)
    sc = synth.default_q_scaler(hp)
    n_pop = 7
    params = np.stack([synth.model_params(hp, rng) for _ in range(n_pop)])
    target = rng.standard_normal((bt.n_structs, 9))
    assert n_pop * ((len(bt.types) + 127) // 128) > 2 * 152
    for mode in (1, 2):
        ctx = tn.tnep_create([tn.Model.from_hyper(hp, params[0], sc, mlp_precision=mode)], 2, RC)
        _, pred = tn.tnep_eval_population(ctx, 0, params, bt.offsets, bt.pos, bt.box, bt.types, target,
                                          want_out=True)
        ctx.close()
        for p in range(n_pop):
            c1 = tn.tnep_create([tn.Model.from_hyper(hp, params[p], sc, mlp_precision=mode)], 2, RC)
            (one,), _ = tn.tnep_eval_batch(c1, bt.offsets, bt.pos, bt.box, bt.types)
            c1.close()
            one = np.asarray(one)
            assert np.all(np.abs(pred[p] - one) <= 1e-12 * np.abs(one).max()), (mode, p)


# ------------------------------------------------------------ Verlet skin
def _walk(n_side, L, n_frames, sigma, seed):
    rng = np.random.default_rng(seed)
    base, types, box = synth.water_grid_box(n_side, L, rng)
    frames = synth.random_walk_frames(base, box, n_frames, sigma, rng)
    return frames, types, box.astype(np.float32)


def test_skin_reuse_matches_per_frame_lists(tn):
    frames, types, box = _walk(10, 31.04, 24, 0.01, 5)
    ms, om = models_for(tn, 2)
    ctx = tn.tnep_create(ms, 2, RC)
    tn.tnep_set_option(ctx, tn.TNEP_OPT_FRAMES_PER_BATCH, 8)
    plain = tn.tnep_eval(ctx, frames, box, types)
    assert tn.tnep_get_option(ctx, tn.TNEP_OPT_LAST_SKIN_USED) == 0
    tn.tnep_set_option(ctx, tn.TNEP_OPT_SKIN, 0.5)
    skin = tn.tnep_eval(ctx, frames, box, types)
    assert tn.tnep_get_option(ctx, tn.TNEP_OPT_LAST_SKIN_USED) == 1
    for a, b, m in zip(plain, skin, om):
        # same pairs, possibly another summation order
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-6 * np.abs(a).max())
        for f in (0, 7, 23):
            r = oracle.evaluate(m, frames[f], box, types)
            assert np.linalg.norm(b[f] - r.tensor) <= max(REL * np.linalg.norm(r.tensor),
                                                          COND * np.abs(r.per_atom).sum())
    # an atom that jumps further than skin / 2 inside a pass forces fresh lists
    jumped = frames.copy()
    jumped[5, 17] = np.mod(jumped[5, 17] + 0.4, box)
    skin2 = tn.tnep_eval(ctx, jumped, box, types)
    assert tn.tnep_get_option(ctx, tn.TNEP_OPT_LAST_SKIN_USED) == 0
    tn.tnep_set_option(ctx, tn.TNEP_OPT_SKIN, 0.0)
    plain2 = tn.tnep_eval(ctx, jumped, box, types)
    for a, b in zip(plain2, skin2):
        assert np.array_equal(a, b)
    ctx.close()


def test_skin_falls_back_when_box_is_short(tn):
    frames, types, box = synth.water_small(6)  # 12.42 A < 2 (6 + 0.5) A
    ms, _ = models_for(tn, 2)
    ctx = tn.tnep_create(ms, 2, RC)
    plain = tn.tnep_eval(ctx, frames, box, types)
    tn.tnep_set_option(ctx, tn.TNEP_OPT_SKIN, 0.5)
    skin = tn.tnep_eval(ctx, frames, box, types)
    assert tn.tnep_get_option(ctx, tn.TNEP_OPT_LAST_SKIN_USED) == 0
    for a, b in zip(plain, skin):
        assert np.array_equal(a, b)
    ctx.close()
