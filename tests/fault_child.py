"""Child process of tests/test_gpu_fault.py (not collected by pytest).

Runs one fixed sequence of library calls -- context creation, a trajectory
through tnep_eval, three requests through the serving loop, a population --
retrying any call that fails with TNEP_ERR_OOM once, and prints one JSON line
with the results, the calls that reported an allocation failure, and the
library's allocation count.  With TNEP_FAULT=oom@N in the environment, the
library's N-th allocation fails (host-side injection; the device is never
faulted)."""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from paper_2312_05233_gb300 import tnep as tn  # noqa: E402

RC = (6.0, 4.0)


def main():
    ooms = []

    def retry(name, fn):
        try:
            return fn()
        except tn.TnepError as e:
            if e.status != 2:
                raise
            ooms.append(name)
            return fn()

    rng = np.random.default_rng(3)
    frames, types, box = synth.water_small(5)
    models = []
    for rank in (1, 2):
        hp = synth.HyperParams(n_types=2, rank=rank)
        models.append(tn.Model.from_hyper(hp, synth.model_params(hp, rng), synth.default_q_scaler(hp)))
    ctx = retry("create", lambda: tn.tnep_create(models, 2, RC))
    tn.tnep_set_option(ctx, tn.TNEP_OPT_FRAMES_PER_BATCH, 2)  # three passes
    mu, al = retry("eval", lambda: tn.tnep_eval(ctx, frames, box, types))

    reqs = [synth.anion(n, rng) for n in (20, 41)] + [(frames[0], types, box)]
    srv = retry("server_start", lambda: tn.tnep_server_start(ctx, mem_budget_bytes=1 << 30, max_slots=64))
    served = []
    for p, t, b in reqs:
        t = np.asarray(t) % 2
        b = np.asarray(b, np.float32)
        served.append(retry("submit", lambda: srv.wait(srv.submit(p, t, b))[0]).tolist())
    srv.stop()

    structs = synth.population_structures(n_clusters=4, n_boxes=1, seed_k=5)
    bt = synth.concat_structures(structs)
    hp = synth.HyperParams(n_types=2, rank=1)
    params = np.stack([synth.model_params(hp, rng) for _ in range(3)])
    target = rng.standard_normal((bt.n_structs, 3))
    pctx = retry("create", lambda: tn.tnep_create([tn.Model.from_hyper(hp, params[0], synth.default_q_scaler(hp))],
                                                 2, RC))
    tn.tnep_set_option(pctx, tn.TNEP_OPT_POPULATION_FORM, 1)
    pop = retry("population_create", lambda: tn.tnep_population_create(pctx, 0, params, bt.offsets, bt.pos,
                                                                         bt.box, bt.types, target))
    rmse, pred = retry("population_eval", lambda: pop.eval(params, want_out=True))
    pop.close()
    allocs = tn.tnep_get_option(ctx, tn.TNEP_OPT_ALLOC_COUNT)
    pctx.close()
    ctx.close()
    print(json.dumps({"mu": mu.tolist(), "alpha": al.tolist(), "served": served, "pop": pred.tolist(),
                      "rmse": rmse.tolist(), "ooms": ooms, "allocs": allocs}))


if __name__ == "__main__":
    main()
