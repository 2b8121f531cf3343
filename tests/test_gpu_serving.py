"""Serving loop (continuous batching) through the C ABI.

Each result must be bitwise identical alone and in a mixed batch (the
per-structure reductions have a fixed order), equal to the plain batch entry
point, and within the parity tolerance of the FP64 oracle.  Admission is
bounded by slots and by the device-memory budget, and waits are bounded.
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


def six_type_models(tn, seed=3):
    rng = np.random.default_rng(seed)
    ms, om = [], []
    for rank in (1, 2):
        hp = synth.HyperParams(n_types=6, rank=rank)
        p = synth.model_params(hp, rng)
        sc = synth.default_q_scaler(hp)
        ms.append(tn.Model.from_hyper(hp, p, sc))
        om.append(oracle.OracleModel.from_flat(hp, p, sc, *RC))
    return ms, om


def test_alone_equals_mixed_equals_plain(tn):
    ms, om = six_type_models(tn)
    ctx = tn.tnep_create(ms, 6, RC)
    reqs = synth.serving_requests(40, np.random.default_rng(11), max_mol=600)
    probe = reqs[7]
    with tn.tnep_server_start(ctx, n_pipelines=3, max_batch_atoms=8192) as srv:
        t = srv.submit(probe.pos, probe.types, probe.box)
        alone, _ = srv.wait(t)
        tickets = [srv.submit(r.pos, r.types, r.box) for r in reqs]
        assert all(tk is not None for tk in tickets)
        mixed = [srv.wait(tk)[0] for tk in tickets]
        st = srv.stats()
    assert st["completed"] == 41 and st["batches"] >= 2
    assert np.array_equal(alone, mixed[7])
    for r, got in zip(reqs, mixed):
        (mu, al), _ = tn.tnep_eval_batch(ctx, [0, len(r.types)], r.pos, r.box[None], r.types)
        assert np.array_equal(got, np.concatenate([mu[0], al[0]]))
    for k in (0, 7, 20):
        r = reqs[k]
        for m, sl in ((om[0], slice(0, 3)), (om[1], slice(3, 12))):
            ref = oracle.evaluate(m, r.pos, r.box, r.types)
            err = np.linalg.norm(mixed[k][sl] - ref.tensor)
            assert err <= max(1e-5 * np.linalg.norm(ref.tensor), 1e-6 * np.abs(ref.per_atom).sum())
    ctx.close()


def test_admission_budget_slots_and_timeout(tn):
    ms, _ = six_type_models(tn)
    ctx = tn.tnep_create(ms[:1], 6, RC)
    big = synth.serving_requests(1, np.random.default_rng(2), max_mol=64)[0]
    frames, types, box = synth.water_bulk(n_frames=1)
    wtypes = np.where(types == 0, 3, 0).astype(np.int32)
    # a request that keeps the GPU busy for milliseconds (8 bulk-water
    # frames side by side, 331,776 atoms): it is still in flight when the
    # zero-timeout wait below is made, although a lone request is launched
    # inside submit itself
    shifts = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], np.float32) * box
    big_pos = (frames[0][None] + shifts[:, None]).reshape(-1, 3)
    big_types = np.tile(wtypes, 8)
    # one slot: the second request is refused until the first finishes
    with tn.tnep_server_start(ctx, max_slots=1, n_pipelines=1) as srv:
        t1 = srv.submit(big_pos, big_types, 2 * box)
        assert t1 is not None
        assert srv.submit(big.pos, big.types, big.box) is None
        with pytest.raises(tn.TnepError) as e:
            srv.wait(t1, timeout_s=0.0)
        assert e.value.status == tn.TNEP_ERR_TIMEOUT
        out, lat = srv.wait(t1, timeout_s=60.0)
        assert lat > 0 and np.all(np.isfinite(out))
        assert srv.submit(big.pos, big.types, big.box) is not None
    # a budget below one large request admits it only when nothing else is in flight
    with tn.tnep_server_start(ctx, mem_budget_bytes=1 << 20, n_pipelines=2) as srv:
        t1 = srv.submit(frames[0], wtypes, box)
        assert t1 is not None
        t2 = srv.submit(frames[0], wtypes, box)
        if t2 is None:
            srv.wait(t1)
        else:  # the first one already finished
            srv.wait(t2)
    ctx.close()


def test_stop_finishes_admitted_requests_and_waiting_calls(tn):
    """A wait in progress when the stop begins returns its result: the stop
    finishes every admitted request and lets calls in progress return before
    it frees the server."""
    import threading
    import time
    ms, _ = six_type_models(tn)
    ctx = tn.tnep_create(ms[:1], 6, RC)
    frames, types, box = synth.water_bulk(n_frames=1)
    wtypes = np.where(types == 0, 3, 0).astype(np.int32)
    shifts = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], np.float32) * box
    big_pos = (frames[0][None] + shifts[:, None]).reshape(-1, 3)
    big_types = np.tile(wtypes, 8)
    plain, _ = tn.tnep_eval_batch(ctx, [0, len(big_types)], big_pos, (2 * box)[None], big_types)
    srv = tn.tnep_server_start(ctx, mem_budget_bytes=96 << 30, n_pipelines=1, max_batch_atoms=len(big_types))
    # queued one batch at a time on one pipeline: tens of milliseconds of work
    tickets = [srv.submit(big_pos, big_types, 2 * box) for _ in range(24)]
    assert all(t is not None for t in tickets)
    entered, got = threading.Event(), {}

    def waiter():
        entered.set()
        got["out"], got["lat"] = srv.wait(tickets[-1], timeout_s=120.0)

    th = threading.Thread(target=waiter)
    th.start()
    entered.wait()
    time.sleep(0.02)  # the waiter is blocked inside the call
    t0 = time.perf_counter()
    srv.stop()
    th.join(timeout=120.0)
    assert not th.is_alive()
    assert np.array_equal(got["out"], plain[0][0])
    assert got["lat"] > 0 and time.perf_counter() - t0 < 120.0
    ctx.close()
