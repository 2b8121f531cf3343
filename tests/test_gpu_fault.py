"""Host-side fault injection: allocation failures (TNEP_FAULT=oom@N).

The library's N-th allocation is made to fail on the host (nothing is
allocated; no GPU fault, trap or hang is involved).  For allocation numbers
spread over a whole run -- context creation, a trajectory in three passes,
three served requests, a population -- the call that hits the failure must
return TNEP_ERR_OOM, and the same call made again must succeed, with results
equal to those of a run without the failure.  Each run is a child process
(tests/fault_child.py), because the fault is read from the environment when
the library loads.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CHILD = os.path.join(HERE, "fault_child.py")


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    return True


def run_child(fault=None):
    env = dict(os.environ)
    env.pop("TNEP_FAULT", None)
    if fault:
        env["TNEP_FAULT"] = fault
    r = subprocess.run([sys.executable, CHILD], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, f"{fault}: {r.stderr[-3000:]}"
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_allocation_failures_return_oom_and_leave_the_context_usable(built):
    ref = run_child()
    assert ref["ooms"] == []
    total = int(ref["allocs"])
    assert total >= 20
    picks = sorted(set([1, 2, 3, 5, 8] + [int(x) for x in np.linspace(9, total, 14)]))
    hit = set()
    for n in picks:
        got = run_child(f"oom@{n}")
        assert len(got["ooms"]) == 1, (n, got["ooms"])
        hit.update(got["ooms"])
        assert got["mu"] == ref["mu"] and got["alpha"] == ref["alpha"], n
        assert got["served"] == ref["served"], n
        p, pr = np.asarray(got["pop"]), np.asarray(ref["pop"])
        np.testing.assert_allclose(p, pr, rtol=0, atol=1e-6 * np.abs(pr).max())
    # every kind of call met an allocation failure in some run
    assert {"create", "eval", "submit", "population_create"} <= hit, hit


def test_tensor_core_wait_give_up_reports_timeout_and_context_recovers(built):
    """Device-side bounded waits: with TNEP_OPT_WAIT_TRIES = 0 every wait of
    the tensor-core network for its product gives up at once.  Each CTA then
    stores nothing, waits (with the default limit) for the product it issued,
    frees its tensor memory and raises TNEP_ERR_TIMEOUT, which the call
    returns.  No wait is left unbounded and nothing faults; afterwards the
    same context gives the results of a fault-free call bit for bit."""
    import synth
    from paper_2312_05233_gb300 import tnep as tn
    frames, types, box = synth.water_small(3)
    rng = np.random.default_rng(5)
    models = []
    for rank in (1, 2):
        hp = synth.HyperParams(n_types=2, rank=rank)
        models.append(tn.Model.from_hyper(hp, synth.model_params(hp, rng), synth.default_q_scaler(hp),
                                          mlp_precision=2))
    ctx = tn.tnep_create(models, 2, (6.0, 4.0))
    ref = tn.tnep_eval(ctx, frames, box, types)
    default = tn.tnep_get_option(ctx, tn.TNEP_OPT_WAIT_TRIES)
    tn.tnep_set_option(ctx, tn.TNEP_OPT_WAIT_TRIES, 0)
    with pytest.raises(tn.TnepError) as e:
        tn.tnep_eval(ctx, frames, box, types)
    assert e.value.status == tn.TNEP_ERR_TIMEOUT and "bounded wait" in str(e.value)
    tn.tnep_set_option(ctx, tn.TNEP_OPT_WAIT_TRIES, default)
    again = tn.tnep_eval(ctx, frames, box, types)
    for a, b in zip(ref, again):
        assert np.array_equal(a, b)
    ctx.close()
