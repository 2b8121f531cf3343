"""Host-side logic of bench.py that needs no GPU: the oracle process pool
(the CPU baseline and the accuracy reference) splits the centres of a
structure across spawned processes and must return exactly the per-atom
contributions of one oracle call over all centres, in centre order."""

import numpy as np

import oracle
import synth


def test_oracle_pool_equals_one_call():
    import bench
    frames, types, box = synth.water_small(1)
    _, hps, params = bench.make_models(None, synth)
    centers = np.array([0, 3, 4, 17, 60, 61, 100, 150, 191])
    pool = bench.OraclePool(nproc=2)
    try:
        got, wall = pool.per_atom(hps, params, frames[0], box, types, centers)
    finally:
        pool.close()
    assert wall > 0
    for m, (hp, p) in enumerate(zip(hps, params)):
        om = oracle.OracleModel.from_flat(hp, p, synth.default_q_scaler(hp), *bench.RC)
        ref = oracle.evaluate(om, frames[0], box, types, centers=centers).per_atom[centers]
        np.testing.assert_array_equal(got[m], ref)


def test_rel_errors_definition():
    import bench
    e = bench.rel_errors([1.0, 2.0, 2.0], [1.0, 2.0, 2.0 + 3e-4])
    assert abs(e["rel_frobenius"] - 3e-4 / np.linalg.norm([1.0, 2.0, 2.0 + 3e-4])) < 1e-15
    assert e["rel_per_component"][0] == 0.0
