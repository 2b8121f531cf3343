"""Benchmark of the TNEP tensor path on bulk water (one JSON line on rank 0).

Workload: 13,824 H2O (41,472 atoms) in a 74.5 A periodic cube, a 2,000-frame
random walk (0.01 A per atom per step); per frame the dipole (rank 1) and
polarizability (rank 2) of two random TNEP models (rc_R = 6 A, rc_A = 4 A,
n_max 4/4, basis 8/8, l_max 4 + 4-body, 30 hidden units, 2 types), then the
IR and Raman (iso, aniso) spectra of the 2,000-frame series (dt = 1 fs).
One step = the whole path over the whole trajectory.

value: atom-frames/s with positions resident in HBM (1.0 GB, larger than L2)
e2e:   the same through the public API with pinned host inputs and host outputs
--impl reference: the FP64 CPU oracle on the host cores, bounded samples.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

RC = (6.0, 4.0)
N_SIDE, L_BOX = 24, 74.5
DT_FS = 1.0
METRIC = "TNEP atom-frames/s served vs plain at rel err <=1e-4 vs FP64; p50/p99 latency"
# Algorithmic flop model per atom and model evaluation (forward + backward):
# radial pair 235, angular pair 1380, per atom 4500 (descriptor products and
# the 30x30 network forward and backward).
PHI_R, PHI_A, PHI_ATOM = 235.0, 1380.0, 4500.0
SMS, FP32_LANES = 152, 128


TRAFFIC_SOURCES = ("tnep_fused.cu", "tnep_device.cuh", "tc_sm100.cuh", "tnep_internal.cuh", "radial.cu")


def traffic_record(atoms_per_pass):
    """DRAM bytes of the compute kernels of one pass (k_radial and both
    k_fused launches), scaled from the ncu capture recorded under profiles/,
    or None when the kernel sources changed since that capture."""
    import hashlib
    rec_path = os.path.join(ROOT, "profiles", "k_fused_traffic.txt")
    if not os.path.exists(rec_path):
        return None, None
    rec = {}
    for ln in open(rec_path):
        if "=" in ln and not ln.startswith("#"):
            k, v = ln.strip().split("=", 1)
            rec[k] = v
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2312_05233_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != rec.get("sources_sha256_16"):
        return None, None
    per_atom = {k: float(rec[k + "_bytes_per_atom"]) for k in ("k_radial", "k_fused_rank1", "k_fused_rank2")}
    return sum(per_atom.values()) * atoms_per_pass, per_atom


NETWORK = {0: "FP32 on the CUDA cores", 1: "BF16 tensor cores (tcgen05), FP32 accumulation",
           2: "split-BF16 tensor cores (tcgen05; hi/lo operands, three products, FP32 accumulation)"}


def workload_config(n_frames, mlp_precision=2):
    return {
        "workload": f"bulk water 13,824 H2O (41,472 atoms), 74.5 A periodic cube, {n_frames}-frame random walk; "
                    "dipole (rank 1) + polarizability (rank 2) TNEP models; IR + Raman iso/aniso spectra",
        "atoms": N_SIDE ** 3 * 3,
        "frames": n_frames,
        "models": "rank1 + rank2, n_max 4/4, basis 8/8, l_max 4 + 4-body, H=30, rc 6/4 A",
        "l2": "inputs larger than L2 (positions 1.0 GB resident, no flush needed)",
        "network": NETWORK[mlp_precision],
    }


def make_models(tn, synth, mlp_precision=0):
    rng = np.random.default_rng(synth.seed_for(2, 1))
    out, hps, params = [], [], []
    for rank in (1, 2):
        hp = synth.HyperParams(n_types=2, rank=rank)
        p = synth.model_params(hp, rng)
        out.append(tn.Model.from_hyper(hp, p, synth.default_q_scaler(hp), mlp_precision) if tn else None)
        hps.append(hp)
        params.append(p)
    return out, hps, params


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        if not getattr(self, "lines", None):
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_chunk(task):
    """Worker of the oracle pool (a spawned process, one torch thread): the
    FP64 oracle's per-atom contributions of every model for a chunk of
    centres of one structure, and the time it took."""
    import torch
    import oracle
    import synth
    torch.set_num_threads(1)
    hps, params, frame, box, types, centers = task
    if centers is None:
        return None, 0.0
    t0 = time.perf_counter()
    per = []
    for hp, p in zip(hps, params):
        om = oracle.OracleModel.from_flat(hp, p, synth.default_q_scaler(hp), *RC)
        per.append(oracle.evaluate(om, frame, box, types, centers=centers).per_atom[centers])
    return per, time.perf_counter() - t0


class OraclePool:
    """The FP64 oracle run as one process per host core over chunks of atom
    centres (the oracle's sum over i is a sum of independent per-atom terms,
    Sec. II.B-C).  Started with `spawn`, so it is safe after CUDA is up."""

    def __init__(self, nproc=None):
        import multiprocessing as mp
        self.nproc = int(nproc or os.cpu_count() or 1)
        self.pool = mp.get_context("spawn").Pool(self.nproc)
        # warm-up: every worker imports torch and the oracle once
        self.pool.map(_oracle_chunk, [(None, None, None, None, None, None)] * (4 * self.nproc), chunksize=1)

    def per_atom(self, hps, params, frame, box, types, centers):
        """Per-atom contributions [model][len(centers)][C] and the wall time."""
        centers = np.asarray(centers)
        # one chunk per process: each oracle call has a fixed cost that grows
        # with the structure (about 0.75 s per model for 41,472 atoms), the
        # per-centre cost is uniform
        n_chunks = min(len(centers), self.nproc)
        chunks = [c for c in np.array_split(centers, n_chunks) if len(c)]
        tasks = [(hps, params, frame, box, types, c) for c in chunks]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_chunk, tasks, chunksize=1)
        wall = time.perf_counter() - t0
        out = [np.concatenate([r[0][m] for r in res]) for m in range(len(hps))]
        return out, wall

    def close(self):
        self.pool.close()
        self.pool.join()


def host_cpu():
    """CPU model and core count of the host (for the baseline's record)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        if model is None:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu model", "hardware")):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"model": model, "nproc": os.cpu_count(), "machine": os.uname().machine}


def rel_errors(got, ref):
    """Relative errors of per-structure tensors: Frobenius (N12) and
    per-component |d| / max |ref_c|."""
    got, ref = np.asarray(got, float), np.asarray(ref, float)
    return {"rel_frobenius": float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)),
            "rel_per_component": (np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)).tolist()}


def oracle_sample(hps, params, frame, box, types, n_centers, seed=0, threads=None):
    """Times the FP64 oracle (both models) on n_centers atoms of one frame,
    with all host threads or the number given."""
    import torch
    import oracle
    import synth
    oms = [oracle.OracleModel.from_flat(hp, p, synth.default_q_scaler(hp), *RC) for hp, p in zip(hps, params)]
    centers = np.random.default_rng(seed).choice(len(types), size=n_centers, replace=False)
    old = torch.get_num_threads()
    if threads:
        torch.set_num_threads(threads)
    try:
        used = torch.get_num_threads()
        t0 = time.perf_counter()
        for om in oms:
            oracle.evaluate(om, frame, box, types, centers=centers)
        dt = time.perf_counter() - t0
    finally:
        torch.set_num_threads(old)
    return dt, used


def serving_bench(tn, synth, device, rates, n_req):
    """Poisson arrivals of mixed requests (open anions, periodic water) served
    by the continuous-batching server vs the plain per-request path."""
    import threading
    old_switch = sys.getswitchinterval()
    sys.setswitchinterval(2e-5)  # the client and the result thread share the GIL

    def wait_until(t):
        while True:
            dt = t - time.perf_counter()
            if dt <= 0:
                return
            time.sleep(dt if dt > 2e-4 else 0)

    rng = np.random.default_rng(synth.seed_for(5))
    reqs = synth.serving_requests(n_req, rng)
    atoms = np.array([len(r.types) for r in reqs])
    hp = synth.HyperParams(n_types=6, rank=1)
    model = tn.Model.from_hyper(hp, synth.model_params(hp, rng), synth.default_q_scaler(hp))
    ctx = tn.tnep_create([model], 6, RC, device=device)
    for r in reqs[:8]:  # warm-up of both paths
        tn.tnep_eval_batch(ctx, [0, len(r.types)], r.pos, r.box[None], r.types)
    out = []
    for rate in rates:
        arr = synth.poisson_arrivals(rate, n_req, np.random.default_rng(synth.seed_for(5, int(rate))))
        # served
        srv = tn.tnep_server_start(ctx, mem_budget_bytes=16 << 30, max_slots=4096, n_pipelines=3,
                                   max_batch_atoms=1 << 19)
        for r in reqs[:8]:
            srv.wait(srv.submit(r.pos, r.types, r.box))
        tickets = [None] * n_req
        t_sub = np.zeros(n_req)    # host clock just before the (accepted) submit
        lat_srv = np.zeros(n_req)  # server: submit -> result on the host
        seen = np.zeros(n_req)     # when the client thread got the result
        t0 = time.perf_counter()

        def waiter():
            for i in range(n_req):
                while tickets[i] is None:
                    time.sleep(2e-5)
                _, lat_srv[i] = srv.wait(tickets[i], timeout_s=120.0)
                seen[i] = time.perf_counter()

        th = threading.Thread(target=waiter)
        th.start()
        for i, r in enumerate(reqs):
            wait_until(t0 + arr[i])
            t_sub[i] = time.perf_counter()
            tk = srv.submit(r.pos, r.types, r.box)
            while tk is None:
                time.sleep(5e-5)
                t_sub[i] = time.perf_counter()
                tk = srv.submit(r.pos, r.types, r.box)
            tickets[i] = tk
        th.join()
        st = srv.stats()
        srv.stop()
        # latency from arrival to the result being on the host (the server's
        # completion stamp); `client_*` adds the one waiter thread's wake-up,
        # which takes the tickets in arrival order
        done = t_sub + lat_srv
        lat_s = done - (t0 + arr)
        lat_c = seen - (t0 + arr)
        served = {"atom_frames_per_s": float(atoms.sum() / (done.max() - t0)),
                  "p50_ms": float(np.percentile(lat_s, 50) * 1e3), "p99_ms": float(np.percentile(lat_s, 99) * 1e3),
                  "client_p50_ms": float(np.percentile(lat_c, 50) * 1e3),
                  "client_p99_ms": float(np.percentile(lat_c, 99) * 1e3),
                  "batches": int(st["batches"])}
        # plain: one tnep_eval_batch per request, first come first served
        done_p = np.zeros(n_req)
        t0 = time.perf_counter()
        for i, r in enumerate(reqs):
            wait_until(t0 + arr[i])
            tn.tnep_eval_batch(ctx, [0, len(r.types)], r.pos, r.box[None], r.types)
            done_p[i] = time.perf_counter()
        lat_p = done_p - (t0 + arr)
        plain = {"atom_frames_per_s": float(atoms.sum() / (done_p.max() - t0)),
                 "p50_ms": float(np.percentile(lat_p, 50) * 1e3), "p99_ms": float(np.percentile(lat_p, 99) * 1e3)}
        out.append({"rate_per_s": rate, "served": served, "plain": plain})
    ctx.close()
    sys.setswitchinterval(old_switch)
    return {"workload": f"{n_req} requests per rate, 50/50 open anions (20-60 atoms, 6 types) and periodic "
                        f"water (192-24,000 atoms), rank-1 model, Poisson arrivals; latency from arrival",
            "mean_atoms": float(atoms.mean()), "rates": out}


def population_bench(tn, synth, device, n_pop=50, gens=5, rank=1):
    """50 parameter vectors x 600 uneven structures per generation (open water
    clusters of 3-300 atoms, periodic boxes of 192-1,536 atoms), RMSE of the
    dipole (rank 1) or polarizability (rank 2) against seeded random targets;
    structures resident, generations replayed from a CUDA graph with the
    autotuned form and launch shape (per-pair walk, factored on the CUDA
    cores, factored with tensor-core products)."""
    rng = np.random.default_rng(synth.seed_for(4, 9 + 10 * (rank - 1)))
    structs = synth.population_structures()
    bt = synth.concat_structures(structs)
    hp = synth.HyperParams(n_types=2, rank=rank)
    sc = synth.default_q_scaler(hp)
    target = rng.standard_normal((bt.n_structs, 3 if rank == 1 else 9))
    gen_params = [np.stack([synth.model_params(hp, rng) for _ in range(n_pop)]) for _ in range(gens + 1)]
    ctx = tn.tnep_create([tn.Model.from_hyper(hp, gen_params[0][0], sc)], 2, RC, device=device)
    pop = tn.tnep_population_create(ctx, 0, gen_params[0], bt.offsets, bt.pos, bt.box, bt.types, target)
    pop.eval(gen_params[0])
    t0 = time.perf_counter()
    dev_ms = 0.0
    for g_ in range(1, gens + 1):
        rmse, _ = pop.eval(gen_params[g_])
        dev_ms += pop.info()["last_ms"]
    wall = (time.perf_counter() - t0) / gens
    info = pop.info()
    t1 = time.perf_counter()
    tn.tnep_eval_population(ctx, 0, gen_params[1], bt.offsets, bt.pos, bt.box, bt.types, target)
    oneshot = time.perf_counter() - t1
    pop.close()
    ctx.close()
    atoms = len(bt.types)
    forms = {0: "per-pair walk", 1: "factored, CUDA cores", 2: "factored, tensor-core products"}
    return {"workload": f"{n_pop} parameter vectors x {bt.n_structs} structures ({atoms} atoms), rank {rank}",
            "generation_ms": wall * 1e3, "generation_device_ms": dev_ms / gens,
            "atom_evals_per_s": n_pop * atoms / wall, "oneshot_ms": oneshot * 1e3,
            "chosen": {"atoms_per_cta": info["block"], "individual_major": info["pop_major"],
                       "factored": info["factored"], "form": forms[info["factored"]]},
            "candidates_ms": info["tune_ms"], "tensor_core_form_ms": info["tensor_core_ms"],
            "rmse_first": float(rmse[0])}


def snes_bench(tn, synth, device, n_pop=50, gens=100):
    """The SNES training loop on the population workload: 50 individuals x
    600 structures per generation, dipole loss against seeded random targets
    with L1 / L2 terms (lambda 2e-3 each); every generation (sampling,
    evaluation, loss, ranking, update) is one CUDA graph replay."""
    rng = np.random.default_rng(synth.seed_for(4, 10))
    structs = synth.population_structures()
    bt = synth.concat_structures(structs)
    hp = synth.HyperParams(n_types=2, rank=1)
    sc = synth.default_q_scaler(hp)
    target = synth.tensor_targets(bt.n_structs, 3, rng)
    mu0 = synth.model_params(hp, rng).astype(np.float64)
    ctx = tn.tnep_create([tn.Model.from_hyper(hp, mu0.astype(np.float32), sc)], 2, RC, device=device)
    sn = tn.tnep_snes_create(ctx, 0, n_pop, mu0, 0.1, bt.offsets, bt.pos, bt.box, bt.types, target, seed=11,
                             lambda1=2e-3, lambda2=2e-3)
    sn.run(3)
    t0 = time.perf_counter()
    hist = sn.run(gens)
    wall = (time.perf_counter() - t0) / gens
    info = sn.info()
    sn.close()
    ctx.close()
    atoms = len(bt.types)
    return {"workload": f"SNES, {n_pop} individuals x {bt.n_structs} structures ({atoms} atoms), rank 1, "
                        f"d = {info['dim']}, {gens} generations",
            "generation_ms": wall * 1e3, "generation_device_ms": info["ms_per_generation"],
            "generations_per_s": 1.0 / wall, "atom_evals_per_s": n_pop * atoms / wall,
            "best_loss_first": float(hist[0, 0]), "best_loss_last": float(hist[-1, 0])}


def raman_bench(tn, synth, T=100_000, M=2000, n_theta=181):
    """Polarized Raman tail at the BaZrO3 production length: a synthetic
    susceptibility trajectory of 100,000 samples (500 ps at 5 fs), lineshape
    tensor up to 10 ps lag, then the Z(XX)Z-bar / Z(XY)Z-bar orientation map
    for 181 crystal angles about z.  Wall time of the synchronous calls,
    host series in, host spectra out."""
    a = synth.tensor_series(T, np.random.default_rng(synth.seed_for(7, 5)))
    tn.tnep_raman_tensor(a[:4000], 5.0, 100)  # warm-up
    t0 = time.perf_counter()
    _, L = tn.tnep_raman_tensor(a, 5.0, M)
    t1 = time.perf_counter()
    th = np.linspace(0.0, np.pi, n_theta)
    tn.tnep_raman_porto_map(L, th, 2)
    t2 = time.perf_counter()
    return {"workload": f"susceptibility series T = {T} (500 ps at 5 fs), M = {M} lags, {n_theta} angles",
            "tensor_ms": (t1 - t0) * 1e3, "porto_map_ms": (t2 - t1) * 1e3,
            "route": "fourier" if 81.0 * T * (M + 1) > 1.0e9 else "direct"}


def precision_report(tn, synth, device, pool, n_frames=500, oracle_frames=(0, 1)):
    """BaZrO3 12x12x12 (8,640 atoms), 500 frames, rank-2 susceptibility:
    the network on the CUDA cores in FP32 (mode 0), on the tensor cores in
    BF16 (mode 1) and as split BF16 with three products (mode 2).  Errors per
    tensor component: max over frames of |T_mode - T_0| / max_frames |T_0,c|,
    and against the FP64 oracle (whole frames, every atom) on the frames
    `oracle_frames`: relative Frobenius error per frame and per component."""
    import torch
    frames, types, box = synth.bzo_perovskite(n_frames=n_frames)
    rng = np.random.default_rng(synth.seed_for(3, 1))
    hp = synth.HyperParams(n_types=3, rank=2)
    p = synth.model_params(hp, rng)
    sc = synth.default_q_scaler(hp)
    F = len(frames)
    pos = torch.from_numpy(frames).to(torch.device("cuda", device))
    bx = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(box, (F, 3)))).to(pos.device)
    ty = torch.from_numpy(types).to(pos.device)
    res, outs = {}, {}
    for mode in (0, 1, 2):
        ctx = tn.tnep_create([tn.Model.from_hyper(hp, p, sc, mode)], 3, RC, device=device)
        tn.tnep_eval(ctx, pos, bx, ty)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        (al,) = tn.tnep_eval(ctx, pos, bx, ty)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        outs[mode] = al.cpu().numpy()
        res[mode] = {"atom_frames_per_s": F * len(types) / dt}
        ctx.close()
    scale = np.abs(outs[0]).max(0)
    for mode in (1, 2):
        d = np.abs(outs[mode] - outs[0]) / np.maximum(scale, 1e-30)
        res[mode]["vs_fp32_max_rel_per_component"] = d.max(0).tolist()
    refs = []
    for f in oracle_frames:
        (per,), _ = pool.per_atom([hp], [p], frames[f], box, types, np.arange(len(types)))
        refs.append(per.sum(0))
    ref = np.array(refs)
    for mode in (0, 1, 2):
        got = outs[mode][list(oracle_frames)]
        e = np.abs(got - ref)
        res[mode]["vs_fp64_rel_per_component"] = (e.max(0) / np.maximum(np.abs(ref).max(0), 1e-30)).tolist()
        res[mode]["vs_fp64_rel_frobenius"] = float(max(np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k])
                                                       for k in range(len(ref))))
    bars = {0: 1e-5, 1: 1e-3, 2: 1e-5}
    for mode in (0, 1, 2):
        res[mode]["bar_rel_frobenius"] = bars[mode]
        res[mode]["within_bar"] = bool(res[mode]["vs_fp64_rel_frobenius"] <= bars[mode])
    return {"workload": f"BaZrO3 12x12x12 (8,640 atoms), {F} frames, rank 2, 3 types; oracle on frames "
                        f"{list(oracle_frames)} (every atom)",
            "modes": {"fp32_cuda_cores": res[0], "bf16_tensor_cores": res[1], "split_bf16_tensor_cores": res[2]}}


def accuracy_report(tn, ctx, hps, params, frames, box, types, timed_out, pool, n_sample=2048):
    """Error of the timed workload's tensors against the FP64 oracle.

    Frame 0: every atom through the oracle, so the frame tensor of the timed
    run is compared as a whole (relative Frobenius error, N12; and against
    the condition scale sum_i |c_i|).  Two more frames (middle, last):
    n_sample atoms each, per-atom errors.  On all three frames the timed
    frame tensor is also checked against the FP64 sum of the per-atom
    outputs of the same library (tnep_eval_batch), which the oracle samples
    are compared with."""
    F, N = frames.shape[0], frames.shape[1]
    C = [3, 9]
    T_timed = [timed_out[:F * 3].reshape(F, 3), timed_out[F * 3:].reshape(F, 9)]
    rng = np.random.default_rng(2312)
    rows, per_atom_rel, consist = [], [[], []], 0.0
    for f in (0, F // 2, F - 1):
        _, pa = tn.tnep_eval_batch(ctx, [0, N], frames[f], box[None], types, per_atom=True)
        for m in range(2):
            s = pa[m].astype(np.float64).sum(0)
            consist = max(consist, float(np.linalg.norm(s - T_timed[m][f]) / np.linalg.norm(T_timed[m][f])))
        centers = np.arange(N) if f == 0 else np.sort(rng.choice(N, size=n_sample, replace=False))
        ref, wall = pool.per_atom(hps, params, frames[f], box, types, centers)
        for m in range(2):
            got = pa[m][centers].astype(np.float64)
            r = ref[m]
            per_atom_rel[m].append(np.linalg.norm(got - r, axis=1) / np.maximum(np.linalg.norm(r, axis=1), 1e-300))
            if f == 0:
                T_ref = r.sum(0)
                e = rel_errors(T_timed[m][f], T_ref)
                e["cond_rel"] = float(np.linalg.norm(T_timed[m][f] - T_ref) /
                                      np.linalg.norm(r, axis=1).sum())
                rows.append({"model": f"rank {m + 1}", "frame": int(f), "atoms": int(N), **e})
        if f == 0:
            full_wall = wall
    out = {"workload": "bulk water (the timed workload): frame 0 with every atom through the FP64 oracle; "
                       f"frames {F // 2} and {F - 1} with {n_sample} sampled atoms each",
           "frame_errors": rows,
           "max_rel_frobenius": max(r["rel_frobenius"] for r in rows),
           "per_atom": {f"rank {m + 1}": {"max_rel": float(np.concatenate(per_atom_rel[m]).max()),
                                          "median_rel": float(np.median(np.concatenate(per_atom_rel[m]))),
                                          "atoms": int(sum(len(x) for x in per_atom_rel[m]))} for m in range(2)},
           "timed_vs_per_atom_sum_rel": consist,
           "bar_rel": 1e-4, "fp32_bar_rel": 1e-5}
    out["within_bar"] = bool(out["max_rel_frobenius"] <= out["bar_rel"])
    return out, full_wall


# ------------------------------------------------------------------ multi-rank
def shard_seed_k(rank: int) -> int:
    """Each rank evaluates its own trajectory (weak scaling over frames):
    rank r draws the bulk-water random walk with seed offset r."""
    return int(rank)


def max_over_ranks(dist, x: float, device, world: int) -> float:
    """The slowest rank's time (the job's time)."""
    if world == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_units(frames: int, atoms: int, world: int) -> int:
    """Atom-frames processed by the whole job per step."""
    return int(frames) * int(atoms) * int(world)


def run_reference(args, rank, world):
    """FP64 CPU oracle arm: bounded samples of the same workload."""
    import synth
    if rank != 0:
        return 0
    frames, types, box = synth.water_bulk(n_frames=max(args.warmup + args.steps, 1))
    _, hps, params = make_models(None, synth)
    n_c = args.ref_centers
    pool = OraclePool()
    rng = np.random.default_rng(100)
    for w in range(args.warmup):
        pool.per_atom(hps, params, frames[w], box, types, rng.choice(len(types), max(8, n_c // 8), replace=False))
    times, cores = [], pool.nproc
    for k in range(args.steps):
        c = np.sort(rng.choice(len(types), n_c, replace=False))
        _, dt = pool.per_atom(hps, params, frames[args.warmup + k], box, types, c)
        times.append(dt)
    pool.close()
    t = float(np.mean(times))
    value = n_c / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "atom-frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.frames),
        "cpu_baseline": {"value": value, "unit": "atom-frames/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n_c} atoms of one frame per step, both models, one process per host "
                                   "core over chunks of atom centres", "host": host_cpu()},
        "e2e": {"value": value, "unit": "atom-frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--frames", type=int, default=2000)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-centers", type=int, default=8192)
    ap.add_argument("--cpu-centers", type=int, default=1500,
                    help="atoms of the single-process oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=5000)
    ap.add_argument("--serve-rates", default="100,300,1000,3000,5000,20000",
                    help="Poisson arrival rates (req/s): the five of the serving workload plus a saturating one")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-population", action="store_true")
    ap.add_argument("--no-network-variants", action="store_true",
                    help="skip timing the step with the network in the other precisions")
    ap.add_argument("--mlp-precision", type=int, default=2,
                    help="network products: 0 FP32 CUDA cores, 1 BF16 tensor cores, 2 split-BF16 tensor cores")
    ap.add_argument("--no-precision-report", action="store_true",
                    help="skip the BaZrO3 network-precision table (printed by default)")
    ap.add_argument("--skin", type=float, default=1.0, help="Verlet skin of the extra skin-reuse measurement")
    ap.add_argument("--cell-div", type=int, default=0, help="cell subdivision of the neighbour search (0 = library default)")
    ap.add_argument("--x-div", type=int, default=0, help="x-only cell subdivision with window scan (0 = library default)")
    ap.add_argument("--frames-per-batch", type=int, default=0, help="frames per device pass (0 = library default)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    import __graft_entry__ as g
    import synth

    g.build()
    from paper_2312_05233_gb300 import tnep as tn

    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # each rank evaluates its own trajectory (weak scaling over frames)
    frames, types, box = synth.water_bulk(n_frames=args.frames, seed_k=shard_seed_k(rank))
    F, N = frames.shape[0], frames.shape[1]
    models, hps, params = make_models(tn, synth, args.mlp_precision)
    ctx = tn.tnep_create(models, 2, RC, device=local)
    if args.cell_div:
        tn.tnep_set_option(ctx, tn.TNEP_OPT_CELL_DIV, args.cell_div)
    if args.x_div:
        tn.tnep_set_option(ctx, tn.TNEP_OPT_CELL_XDIV, args.x_div)
    if args.frames_per_batch:
        tn.tnep_set_option(ctx, tn.TNEP_OPT_FRAMES_PER_BATCH, args.frames_per_batch)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream

    pos_d = torch.from_numpy(frames).to(dev)
    box_all = np.ascontiguousarray(np.broadcast_to(box, (F, 3)), dtype=np.float32)
    box_d = torch.from_numpy(box_all).to(dev)
    types_d = torch.from_numpy(types).to(dev)
    out_d = torch.empty(F * 12, dtype=torch.float64, device=dev)
    pos_h = torch.from_numpy(frames).pin_memory()
    box_h = torch.from_numpy(box_all).pin_memory()
    types_h = torch.from_numpy(types).pin_memory()
    out_h = torch.empty(F * 12, dtype=torch.float64).pin_memory()
    M = F // 2

    def step_device():
        tn.tnep_eval(ctx, pos_d, box_d, types_d, out=out_d, stream=sp)
        mu = out_d[:F * 3].view(F, 3)
        al = out_d[F * 3:].view(F, 9)
        tn.tnep_spectrum(mu, DT_FS, tn.TNEP_SPECTRUM_IR, M, stream=sp)
        tn.tnep_spectrum(al, DT_FS, tn.TNEP_SPECTRUM_RAMAN_ISO, M, stream=sp)
        tn.tnep_spectrum(al, DT_FS, tn.TNEP_SPECTRUM_RAMAN_ANISO, M, stream=sp)

    def step_e2e():
        tn.tnep_eval(ctx, pos_h, box_h, types_h, out=out_h, stream=sp)
        mu = out_h[:F * 3].view(F, 3)
        al = out_h[F * 3:].view(F, 9)
        tn.tnep_spectrum(mu, DT_FS, tn.TNEP_SPECTRUM_IR, M, stream=sp)
        tn.tnep_spectrum(al, DT_FS, tn.TNEP_SPECTRUM_RAMAN_ISO, M, stream=sp)
        tn.tnep_spectrum(al, DT_FS, tn.TNEP_SPECTRUM_RAMAN_ANISO, M, stream=sp)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step_device()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fused_ms, nbr_ms, fused_launches = 0.0, 0.0, 0
    l0 = tn.tnep_get_option(ctx, tn.TNEP_OPT_KERNEL_LAUNCHES_TOTAL)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            step_device()
            fused_ms += tn.tnep_get_option(ctx, tn.TNEP_OPT_LAST_KERNEL_MS)
            nbr_ms += tn.tnep_get_option(ctx, tn.TNEP_OPT_LAST_NBR_MS)
            fused_launches += int(tn.tnep_get_option(ctx, tn.TNEP_OPT_LAST_KERNEL_LAUNCHES))
        ev1.record(stream)
        barrier()
    launches = tn.tnep_get_option(ctx, tn.TNEP_OPT_KERNEL_LAUNCHES_TOTAL) - l0
    timed_out = out_d.cpu().numpy().copy()  # frame tensors of the last timed step
    ms = max_over_ranks(dist, ev0.elapsed_time(ev1) / args.steps, dev, world)

    # end to end through the public API with pinned host buffers
    for _ in range(1):
        step_e2e()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    barrier()
    e2e_ms = max_over_ranks(dist, (time.perf_counter() - t0) * 1e3 / args.steps, dev, world)

    # the same trajectory with Verlet-skin list reuse (every frame still uses
    # exactly the pairs within the cutoffs; reported beside the headline,
    # which rebuilds the lists for every frame)
    skin_line = None
    if args.skin > 0:
        tn.tnep_set_option(ctx, tn.TNEP_OPT_SKIN, args.skin)
        step_device()
        barrier()
        es0, es1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es0.record(stream)
        for _ in range(args.steps):
            step_device()
        es1.record(stream)
        barrier()
        sk_ms = max_over_ranks(dist, es0.elapsed_time(es1) / args.steps, dev, world)
        skin_line = {"skin_A": args.skin, "value": job_units(F, N, world) / (sk_ms * 1e-3), "ms_per_step": sk_ms,
                     "lists_reused_every_pass": bool(tn.tnep_get_option(ctx, tn.TNEP_OPT_LAST_SKIN_USED)),
                     "nbr_ms_per_step": tn.tnep_get_option(ctx, tn.TNEP_OPT_LAST_NBR_MS)}
        tn.tnep_set_option(ctx, tn.TNEP_OPT_SKIN, 0.0)

    # the same step with the network in the other precisions (same weights)
    variants = {}
    if rank == 0 and not args.no_network_variants:
        for mp in (0, 1, 2):
            if mp == args.mlp_precision:
                continue
            vmodels, _, _ = make_models(tn, synth, mp)
            vctx = tn.tnep_create(vmodels, 2, RC, device=local)
            if args.cell_div:
                tn.tnep_set_option(vctx, tn.TNEP_OPT_CELL_DIV, args.cell_div)
            if args.x_div:
                tn.tnep_set_option(vctx, tn.TNEP_OPT_CELL_XDIV, args.x_div)

            def vstep():
                tn.tnep_eval(vctx, pos_d, box_d, types_d, out=out_d, stream=sp)
                tn.tnep_spectrum(out_d[:F * 3].view(F, 3), DT_FS, tn.TNEP_SPECTRUM_IR, M, stream=sp)
                tn.tnep_spectrum(out_d[F * 3:].view(F, 9), DT_FS, tn.TNEP_SPECTRUM_RAMAN_ISO, M, stream=sp)
                tn.tnep_spectrum(out_d[F * 3:].view(F, 9), DT_FS, tn.TNEP_SPECTRUM_RAMAN_ANISO, M, stream=sp)

            for _ in range(2):
                vstep()
            torch.cuda.synchronize(dev)
            ev0.record(stream)
            for _ in range(args.steps):
                vstep()
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            v_ms = ev0.elapsed_time(ev1) / args.steps
            variants[NETWORK[mp]] = {"value": F * N / (v_ms * 1e-3), "ms_per_step": v_ms}
            vctx.close()

    # neighbour statistics of the last frame for the flop model
    offs = np.array([0, N])
    cR, cA, _, _ = tn.tnep_neighbors(ctx, offs, frames[-1], box[None], cap_R=1, cap_A=1)
    nn_R, nn_A = float(cR.mean()), float(cA.mean())
    flops_atom = nn_R * PHI_R + nn_A * PHI_A + PHI_ATOM
    atom_evals = F * N * 2 * args.steps
    achieved_tflops = flops_atom * atom_evals / (fused_ms * 1e-3) / 1e12 if fused_ms > 0 else None
    clocks = clk.summary()
    peak_tflops = SMS * FP32_LANES * 2 * 2070e6 / 1e12
    passes = fused_launches / args.steps / 2 if fused_launches else 1
    atoms_per_pass = F * N / passes
    traffic, traffic_per_atom = traffic_record(atoms_per_pass)

    units = job_units(F, N, world)
    value = units / (ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "atom-frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(F, args.mlp_precision),
        "e2e": {"value": units / (e2e_ms * 1e-3), "unit": "atom-frames/s",
                "h2d_bytes_per_step": int(F * N * 12 + F * 12 + N * 4),
                "d2h_bytes_per_step": int(F * 12 * 8 + 3 * 2 * (M + 1) * 8), "ms_per_step": e2e_ms},
        "gpu_launches": int(launches / args.steps),
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": (achieved_tflops / peak_tflops) if achieved_tflops else None, "traffic": traffic,
                     "kernel": "k_radial + k_fused x2 (descriptor + network + partial force + contraction)",
                     "traffic_scope": "DRAM bytes of k_radial and both k_fused launches of one pass "
                                      f"({atoms_per_pass:.0f} atoms), scaled per atom from an ncu capture",
                     "traffic_bytes_per_atom": traffic_per_atom,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (unit counts and max clock)",
                     "flops_per_atom_eval": flops_atom, "nn_R": nn_R, "nn_A": nn_A,
                     "fused_ms_per_step": fused_ms / args.steps, "nbr_ms_per_step": nbr_ms / args.steps,
                     "fused_launches_per_step": fused_launches / args.steps},
        "clocks": clocks,
        "skin_reuse": skin_line,
        "network_variants": variants or None,
    }
    # the FP64 oracle on the host cores: one process per core (spawned)
    pool = OraclePool() if rank == 0 and world == 1 and not args.no_cpu_baseline else None
    if pool is not None:
        line["accuracy"], full_wall = accuracy_report(tn, ctx, hps, params, frames, box, types, timed_out, pool)
        if not args.no_precision_report:
            line["precision"] = precision_report(tn, synth, local, pool)
    if rank == 0 and not args.no_population:
        line["population"] = population_bench(tn, synth, local)
        line["population_rank2"] = population_bench(tn, synth, local, rank=2)
    if rank == 0 and not args.no_population:
        line["snes"] = snes_bench(tn, synth, local)
    if rank == 0 and not args.no_population:
        line["raman"] = raman_bench(tn, synth)
    if rank == 0 and not args.no_serve:
        rates = [float(x) for x in args.serve_rates.split(",") if x]
        line["served"] = serving_bench(tn, synth, local, rates, args.serve_requests)
    if pool is not None:
        n1 = args.cpu_centers
        dt1, _ = oracle_sample(hps, params, frames[0], box, types, n1, threads=1)
        line["cpu_baseline"] = {"value": N / full_wall, "unit": "atom-frames/s", "cores": pool.nproc,
                                "kind": "oracle",
                                "sample": f"frame 0 whole ({N} atoms), both models, FP64 oracle, one process "
                                          f"per host core over chunks of atom centres ({full_wall:.1f} s)",
                                "single_process": {"value": n1 / dt1, "cores": 1,
                                                   "sample": f"{n1} atoms of frame 0, one thread"},
                                "host": host_cpu()}
        pool.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
