"""SNES training loop (Sec. II.D) through the C ABI against the FP64 oracle.

The normals and the update are compared element by element; the full loop
(sampling, evaluation of every individual, loss, ranking, update) is compared
generation by generation with the oracle evaluating each individual in FP64.
The ranking is an integer decision taken from losses the GPU computes in
float32: the test first checks that the oracle's losses are separated by far
more than the evaluation tolerance, so both sides must rank identically.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

RC = (6.0, 4.0)


@pytest.fixture(scope="module")
def tn():
    import __graft_entry__ as g
    g.build()
    from paper_2312_05233_gb300 import tnep
    return tnep


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.mark.parametrize("seed,gen,P,d", [(2312005233, 0, 7, 1001), (2 ** 63 + 5, 123456, 50, 2282),
                                          (0, 3, 2, 1), (17, 9, 1024, 5)])
def test_normals_match_oracle(tn, torch, seed, gen, P, d):
    s = torch.empty((P, d), dtype=torch.float64, device="cuda")
    tn.tnep_snes_normals(seed, gen, P, d, s)
    torch.cuda.synchronize()
    ref = oracle.snes_normals(seed, gen, P, d)
    np.testing.assert_allclose(s.cpu().numpy(), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("P,d,ties,nan", [(13, 517, True, False), (2, 3, False, False), (64, 2282, True, True),
                                          (1024, 33, True, False)])
def test_update_matches_oracle(tn, torch, P, d, ties, nan):
    rng = np.random.default_rng(synth.seed_for(6, P))
    mu, sigma, s, loss = synth.snes_update_inputs(P, d, rng, ties=ties, nan=nan)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    mu_d, sg_d = dev(mu), dev(sigma)
    eta_s = oracle.default_eta_sigma(d)
    tn.tnep_snes_update(dev(loss), dev(s), mu_d, sg_d, 1.0, 0.0)
    torch.cuda.synchronize()
    mu_o, sg_o = oracle.snes_update(mu, sigma, s, loss, 1.0, eta_s)
    np.testing.assert_allclose(mu_d.cpu().numpy(), mu_o, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(sg_d.cpu().numpy(), sg_o, rtol=1e-12)


def _training_set(n_clusters, n_boxes, seed_k):
    structs = synth.population_structures(n_clusters=n_clusters, n_boxes=n_boxes, seed_k=seed_k)
    return structs, synth.concat_structures(structs)


def _models(tn, rank, seed=21):
    hp = synth.HyperParams(n_types=2, rank=rank)
    rng = np.random.default_rng(synth.seed_for(6, seed))
    p = synth.model_params(hp, rng)
    sc = synth.default_q_scaler(hp)
    return hp, p, sc, tn.Model.from_hyper(hp, p, sc)


@pytest.mark.parametrize("rank", [1, 2])
def test_training_loop_matches_oracle(tn, rank):
    hp, p0, sc, model = _models(tn, rank)
    ctx = tn.tnep_create([model], 2, RC)
    structs, bt = _training_set(3, 0, seed_k=5)
    C = 3 if rank == 1 else 9
    target = synth.tensor_targets(len(structs), C, np.random.default_rng(synth.seed_for(6, 40 + rank)))
    P, G, seed, lam1, lam2 = 6, 3, 99, 0.01, 0.02
    sigma0 = np.full(p0.size, 0.05)
    mu0 = p0.astype(np.float64)
    with tn.tnep_snes_create(ctx, 0, P, mu0, sigma0, bt.offsets, bt.pos, bt.box, bt.types, target, seed=seed,
                             lambda1=lam1, lambda2=lam2) as sn:
        hist = sn.run(G)
        mu_g, sg_g, gen = sn.state()
    assert gen == G

    def rmse_fn(z):
        zf = z.astype(np.float32).astype(np.float64)  # the evaluation takes z rounded to float32
        om = oracle.OracleModel.from_flat(hp, zf, sc, *RC)
        pred = np.array([oracle.evaluate(om, st.pos, st.box, st.types).tensor.ravel() for st in structs])
        return float(np.sqrt(np.mean((pred - target) ** 2)))

    mu, sg = mu0.copy(), sigma0.copy()
    for g in range(G):
        mu_n, sg_n, loss, rmse = oracle.snes_generation(mu, sg, g, seed, P, rmse_fn, lam1, lam2)
        srt = np.sort(loss)
        assert np.min(np.diff(srt) / srt[1:]) > 1e-4, "oracle losses too close to rank unambiguously"
        best = int(np.argmin(loss))
        assert hist[g, 0] == pytest.approx(loss[best], rel=1e-5)
        assert hist[g, 1] == pytest.approx(rmse[best], rel=1e-5)
        assert hist[g, 2] == pytest.approx(loss.mean(), rel=1e-5)
        mu, sg = mu_n, sg_n
    np.testing.assert_allclose(mu_g, mu, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(sg_g, sg, rtol=1e-11)
    ctx.close()


def test_training_is_reproducible_resumable_and_descends(tn):
    hp, p0, sc, model = _models(tn, 1, seed=22)
    ctx = tn.tnep_create([model], 2, RC)
    structs, bt = _training_set(40, 8, seed_k=6)
    target = synth.tensor_targets(len(structs), 3, np.random.default_rng(synth.seed_for(6, 50)))
    args = (ctx, 0, 24, p0.astype(np.float64), 0.1, bt.offsets, bt.pos, bt.box, bt.types, target)
    with tn.tnep_snes_create(*args, seed=7, lambda1=1e-3, lambda2=1e-3) as a:
        h_a = np.concatenate([a.run(5), a.run(295)])
        mu_a, sg_a, _ = a.state()
        info = a.info()
    with tn.tnep_snes_create(*args, seed=7, lambda1=1e-3, lambda2=1e-3) as b:
        h_b = b.run(300)
        mu_b, sg_b, _ = b.state()
    assert np.array_equal(h_a, h_b) and np.array_equal(mu_a, mu_b) and np.array_equal(sg_a, sg_b)
    assert info["generation"] == 300 and info["n_pop"] == 24 and info["ms_per_generation"] > 0
    # the best loss of the last generations is well below that of the first
    print("best loss per 20 generations:", h_a[::20, 0])
    assert h_a[-10:, 0].mean() < 0.8 * h_a[:10, 0].mean()
    assert np.all(h_a[:, 0] <= h_a[:, 2])
    ctx.close()
