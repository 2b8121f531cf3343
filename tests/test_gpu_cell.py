"""General periodic cells (triclinic; shorter than twice the cutoff, where a
neighbour counts once per image) through the C ABI against the FP64 oracle,
whose image enumeration is pinned by supercell identities."""

import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def setup(tn):
    rng = np.random.default_rng(synth.seed_for(8, 0))
    ms, om = [], []
    for r in (1, 2):
        hp = synth.HyperParams(n_types=2, rank=r)
        p = synth.model_params(hp, rng)
        sc = synth.default_q_scaler(hp)
        ms.append(tn.Model.from_hyper(hp, p, sc))
        om.append(oracle.OracleModel.from_flat(hp, p, sc, *RC))
    ctx = tn.tnep_create(ms, 2, RC)
    yield ctx, om
    ctx.close()


def _check(got, m, pos, types, cell):
    ref = oracle.evaluate(m, pos, None, types, cell=cell) if cell is not None else oracle.evaluate(m, pos, None,
                                                                                                  types)
    err = np.linalg.norm(got - ref.tensor)
    assert err <= max(REL * np.linalg.norm(ref.tensor), COND * np.abs(ref.per_atom).sum()), (err, ref.tensor)


def _structures():
    rng = np.random.default_rng(synth.seed_for(8, 1))
    out = []
    pos, types, box = synth.water_box(24, rng, L=9.0)          # shorter than 2 rc
    out.append((pos, types, np.diag(box)))
    pos, types, box = synth.water_box(3, rng, L=5.0)           # shorter than rc: own images
    out.append((pos, types, np.diag(box)))
    H = np.array([[8.0, 0.0, 0.0], [2.5, 7.5, 0.0], [-1.5, 2.0, 8.5]])
    pos, types, _ = synth.cell_water(14, H, rng)               # triclinic
    out.append((pos + 3.0 * H[0] - 2.0 * H[2], types, H))      # positions far outside the cell
    pos, types, box = synth.water_box(64, rng, L=12.42)        # orthorhombic, >= 2 rc
    out.append((pos, types, np.diag(box)))
    pos, types, _ = synth.water_cluster(9, rng)                # open
    out.append((pos, types, None))
    return out


def test_cells_match_oracle_and_batches_are_invariant(tn, setup):
    ctx, om = setup
    sts = _structures()
    offs = np.cumsum([0] + [len(t) for _, t, _ in sts])
    pos = np.concatenate([p for p, _, _ in sts]).astype(np.float32)
    types = np.concatenate([t for _, t, _ in sts]).astype(np.int32)
    cells = np.stack([np.zeros((3, 3)) if c is None else c for _, _, c in sts]).astype(np.float32)
    outs = tn.tnep_eval_batch_cell(ctx, offs, pos, cells, types)
    for s, (p, t, c) in enumerate(sts):
        p32 = p.astype(np.float32).astype(np.float64)
        c32 = None if c is None else c.astype(np.float32).astype(np.float64)
        for k in range(2):
            _check(outs[k][s], om[k], p32, t, c32)
        alone = tn.tnep_eval_batch_cell(ctx, [0, len(t)], p.astype(np.float32), cells[s:s + 1], t)
        for k in range(2):
            assert np.array_equal(alone[k][0], outs[k][s])


def test_orthorhombic_cell_equals_minimum_image_path(tn, setup):
    ctx, _ = setup
    rng = np.random.default_rng(synth.seed_for(8, 2))
    pos, types, box = synth.water_box(64, rng, L=12.42)
    pos = np.mod(pos, box).astype(np.float32)
    a = tn.tnep_eval_batch_cell(ctx, [0, len(types)], pos, np.diag(box)[None].astype(np.float32), types)
    (mu, al), _ = tn.tnep_eval_batch(ctx, [0, len(types)], pos, box[None].astype(np.float32), types)
    np.testing.assert_allclose(a[0][0], mu[0], rtol=0, atol=REL * np.abs(mu).max() * 10)
    np.testing.assert_allclose(a[1][0], al[0], rtol=0, atol=REL * np.abs(al).max() * 10)


def test_sheared_perovskite_supercell(tn):
    # a 6x6x6 BaZrO3 supercell (1,080 atoms) under a monoclinic shear
    rng = np.random.default_rng(synth.seed_for(8, 3))
    frames, types, box = synth.bzo_perovskite(n_frames=1, n=6)
    H = np.diag(box).astype(np.float64)
    S = np.array([[1.0, 0.0, 0.0], [0.08, 1.0, 0.0], [0.0, 0.05, 1.0]])
    Hs = S @ H
    frac = frames[0] @ np.linalg.inv(H)
    pos = (frac @ Hs).astype(np.float32)
    hp = synth.HyperParams(n_types=3, rank=2)
    p = synth.model_params(hp, rng)
    sc = synth.default_q_scaler(hp)
    ctx = tn.tnep_create([tn.Model.from_hyper(hp, p, sc)], 3, RC)
    got = tn.tnep_eval_batch_cell(ctx, [0, len(types)], pos, Hs[None].astype(np.float32), types)[0][0]
    m = oracle.OracleModel.from_flat(hp, p, sc, *RC)
    _check(got, m, pos.astype(np.float64), types, Hs.astype(np.float32).astype(np.float64))
    ctx.close()


def test_degenerate_cell_is_rejected(tn, setup):
    ctx, _ = setup
    pos = np.zeros((3, 3), np.float32)
    pos[1, 0] = 1.0
    pos[2, 1] = 1.0
    cell = np.array([[[5.0, 0, 0], [10.0, 0, 0], [0, 0, 5.0]]], np.float32)
    with pytest.raises(tn.TnepError) as e:
        tn.tnep_eval_batch_cell(ctx, [0, 3], pos, cell, np.array([0, 1, 1], np.int32))
    assert e.value.status == 1


def test_rotated_periodic_cell_is_covariant(tn, setup):
    # a periodic box seen in a rotated frame: the cell rows and the positions
    # rotate together, so mu -> R mu and alpha -> R alpha R^T
    ctx, _ = setup
    rng = np.random.default_rng(synth.seed_for(8, 4))
    pos, types, box = synth.water_box(216, rng, L=18.62)
    R = synth.random_rotation(rng)
    H = np.diag(box)
    a = tn.tnep_eval_batch_cell(ctx, [0, len(types)], pos.astype(np.float32), H[None].astype(np.float32), types)
    b = tn.tnep_eval_batch_cell(ctx, [0, len(types)], (pos @ R.T).astype(np.float32),
                                (H @ R.T)[None].astype(np.float32), types)
    mu0, al0 = a[0][0], a[1][0].reshape(3, 3)
    np.testing.assert_allclose(b[0][0], R @ mu0, rtol=0, atol=1e-4 * np.abs(mu0).max())
    np.testing.assert_allclose(b[1][0].reshape(3, 3), R @ al0 @ R.T, rtol=0, atol=1e-4 * np.abs(al0).max())
