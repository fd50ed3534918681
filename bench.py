"""Benchmark of the msDEM hot path on GB300 (one JSON line on rank 0).

Workload: the batched configuration of 128 x 128 coarse cells of 25 km with
lognormal(median 96, sigma 0.69) floes per cell clipped to [8, 1024]
(~1.98M floes), FP32 floe state with FP64 moments and coarse solve, seeded
synthetic inputs.

One bench step = one coarse interval of Algorithm 1: N0 = 100 fine steps of
every cell's DEM (contact search, contact and drag forces, forward Euler,
moment reduction, 10 gradual updates) plus the coarse Lax-Friedrichs step,
i.e. one pass over every row of the hot path.  The state (64 MB) fits in L2,
so L2 is flushed (a 512 MB write) before every timed step and each step is
timed alone with CUDA events on the library's stream.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
BYTES_PER_FLOE_STEP = 56.0     # read x,y,theta,u,v,omega,r,h (8 x 4 B), write x,y,theta,u,v,omega (6 x 4 B)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", HBM_FALLBACK_GBS)), "measured", d
    return HBM_FALLBACK_GBS, "fallback", {}


PROFILE_SOURCES = ("cell_run.cu", "common.cuh", "classes.cuh")   # the resident kernels and their launch classes


def sources_sha16():
    import hashlib
    h = hashlib.sha256()
    for f in PROFILE_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2303_07819_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic():
    """DRAM bytes per coarse interval of the resident cell kernels (the three
    class launches of one interval, live caches) from the committed ncu
    summary, if the kernel sources have not changed since (else None)."""
    path = os.path.join(ROOT, "profiles", "cell_run32_batched128x128.txt")
    if not os.path.exists(path):
        return None, None
    rec = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    if sources_sha16() != rec.get("sources_sha256_16"):
        return None, rec
    return float(rec["dram_bytes_per_interval"]), rec


# FLOP per sample of the closure network (16 -> 128 -> 128 -> 128 -> 4):
# forward 2 (16*128 + 2*128*128 + 128*4); training adds about twice that
MLP_FWD_FLOP = 2 * (16 * 128 + 2 * 128 * 128 + 128 * 4)
MLP_TRAIN_FLOP = 3 * MLP_FWD_FLOP


def closure_training_rate(msdem, batch, n=65536, epochs=4):
    """Adam epochs over n synthetic samples at `batch` on each engine (one
    epoch of warm-up, then `epochs` timed by the host around ms_mlp_train,
    which waits for the device once at its end)."""
    from paper_2303_07819_gb300 import inputs as I
    rng = np.random.default_rng(4)
    X = rng.normal(size=(n, 16)).astype(np.float32)
    Y = np.stack([np.sin(X[:, 0]), 0.1 * X[:, 1], np.tanh(X[:, 3]), 0.01 * X[:, 4] ** 2], 1).astype(np.float32)
    norm = msdem.fit_norm(X, Y)
    out = {"samples": n, "batch": batch, "epochs": epochs}
    for eng, name in ((1, "tcgen05"), (0, "mma_sync")):
        net = msdem.MLP(I.mlp_init(), norm, max_batch=batch)
        net.set_engine(eng)
        net.train(X, Y, epochs=1, batch=batch, lr=1e-3, seed=1)
        t = time.perf_counter()
        net.train(X, Y, epochs=epochs, batch=batch, lr=1e-3, seed=2)
        dt = time.perf_counter() - t
        net.close()
        out[name] = {"samples_per_s": epochs * n / dt, "tflops": epochs * n * MLP_TRAIN_FLOP / dt / 1e12,
                     "us_per_batch": dt / (epochs * (n // batch)) * 1e6}
    return out


def closure_inference_rate(net, X, n=256 * 256, reps=20):
    """The network on a 256 x 256 grid's cells (features drawn from the
    training set), device-timed over `reps` calls of the inference kernel."""
    import torch
    idx = np.random.default_rng(5).integers(0, X.shape[0], n)
    Xd = torch.as_tensor(X[idx].astype(np.float32), device="cuda")
    Yd = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(3):
        net.forward_device(Xd.data_ptr(), n, Yd.data_ptr(), st.cuda_stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        net.forward_device(Xd.data_ptr(), n, Yd.data_ptr(), st.cuda_stream)
    b.record(st)
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    return {"cells": n, "ms_per_call": ms, "cells_per_s": n / (ms * 1e-3),
            "tflops": n * MLP_FWD_FLOP / (ms * 1e-3) / 1e12, "engine": "tcgen05 (kind::f16, BF16, FP32 in TMEM)"}


def closure_eval(msdem, s, seeds=(101, 102, 103), nx_train=128, spin=15, nint=21, K=10,
                 tols=(0.01, 0.015, 0.02, 0.025, 0.03, 0.05, 0.1, 0.2), target_err=1e-2, mode=0, epochs=40):
    """The learned closure on the timed workload.  Training data come from the
    particle path of other seeds of the same workload (after spin-up;
    1.03e6 cell-intervals: 3 seeds x 21 intervals x 16,384 cells); the
    network trains on the GPU; then K coarse intervals of the particle-only
    model are compared with the
    closure-plus-fallback model at a sweep of bounds on the network's checked
    error, the mean-field closure, and, as the noise floor, the particle path
    with another reduction order (the warp-per-cell kernels), all from the
    same spun-up state.  A closure cell's coarse interval counts as N0
    cell-steps.  `crossover` names the bound with the highest speed-up among
    those faster than the particle path at a coarse-state error of at most
    target_err, or says that none is."""
    from paper_2303_07819_gb300 import inputs as I
    t0 = time.perf_counter()
    Xs, Ys = [], []
    for sd in seeds:
        ss = I.batched_128x128(seed=sd, nx=nx_train)
        m = msdem.Model(ss["params"], ss["floes"], msdem.MS_FP32)
        m.step(ss["dt"], ss["params"]["N0"] * spin)
        X, Y = m.closure_collect(nint)
        Xs.append(X.reshape(-1, 16)); Ys.append(Y.reshape(-1, 4))
        m.close()
    X, Y = np.concatenate(Xs), np.concatenate(Ys)
    # mode 2: the network learns the change of the tendencies from the
    # interval before (the lagged features 12-15), which the closure adds back
    T = Y - X[:, 12:16] if mode == 2 else Y
    norm = msdem.fit_norm(X, T)
    net = msdem.MLP(I.mlp_init(), norm, max_batch=8192)
    tt = time.perf_counter()
    losses = net.train(X, T, epochs=epochs, batch=1024, lr=2e-3, seed=3)
    t_train = time.perf_counter() - tt
    infer = closure_inference_rate(net, X)
    box = np.stack([X.min(0) - 0.05 * np.abs(X.min(0)), X.max(0) + 0.05 * np.abs(X.max(0))])
    p, dt, N0 = s["params"], s["dt"], int(s["params"]["N0"])
    cells = p["nx"] * p["ny"]

    def run(mode, tol, variant=-1):
        mm = msdem.Model(p, s["floes"], msdem.MS_FP32)
        if variant >= 0:
            mm.set_launch(variant, 128, 0)
        mm.step(dt, N0 * spin)
        if mode >= 0:
            mm.closure_attach(net if mode != 1 else None, mode, tol, box if mode != 1 else None)
        mm.step(dt, N0)                       # first interval: builds the interval graph
        c0 = mm.closure_stats()["closure_cell_intervals"]
        mm.sync()
        ta = time.perf_counter()
        mm.step(dt, N0 * K)
        el = time.perf_counter() - ta
        st = mm.closure_stats()
        q = mm.coupling()["q"]
        if mode < 0 and variant < 0:
            Xh, Yh = mm.closure_collect(5)
        else:
            Xh = Yh = None
        mm.close()
        return q, el, (st["closure_cell_intervals"] - c0) / (cells * K), Xh, Yh

    qp, tp, _, Xh, Yh = run(-1, 0.0)
    Xh, Yh = Xh.reshape(-1, 16), Yh.reshape(-1, 4)
    P = net.predict(Xh) + (Xh[:, 12:16] if mode == 2 else 0.0)
    r2 = 1 - ((P - Yh) ** 2).sum(0) / ((Yh - Yh.mean(0)) ** 2).sum(0)
    Pl = Xh[:, 12:16]
    r2_lag = 1 - ((Pl - Yh) ** 2).sum(0) / ((Yh - Yh.mean(0)) ** 2).sum(0)
    names = ["rho", "rho_u", "rho_v", "P_omega"]

    def err(q):
        return {n: float(np.linalg.norm(q[f] - qp[f]) / np.linalg.norm(qp[f])) for f, n in enumerate(names)}

    out = {"workload": f"the timed workload, spun up {spin} coarse intervals, then {K} intervals timed "
                       f"(wall clock, graph replays); error = normwise relative difference of the coarse "
                       f"state from the particle-only run after those {K} intervals",
           "train": {"samples": int(X.shape[0]), "from": f"particle path, seeds {list(seeds)}, {nx_train}^2 cells, "
                                                          f"{nint} intervals after {spin} of spin-up",
                     "epochs": epochs, "seconds": t_train,
                     "samples_per_s": epochs * int(X.shape[0]) / t_train,
                     "tflops": epochs * int(X.shape[0]) * MLP_TRAIN_FLOP / t_train / 1e12,
                     "loss_first_last": [float(losses[0]), float(losses[-1])],
                     "mode": mode,
                     "heldout_r2_drag_x_y_torque_var": [float(v) for v in r2],
                     "heldout_r2_of_last_interval": [float(v) for v in r2_lag]},
           "inference_256x256": infer,
           "particle": {"cell_steps_per_s": cells * N0 * K / tp}}
    qn, tn, _, _, _ = run(-1, 0.0, variant=4)
    out["noise_floor_other_reduction_order"] = {"coarse_state_rel_err": err(qn)}
    sweep = []
    for tol in tols:
        q, t, frac, _, _ = run(mode, tol)
        e = err(q)
        sweep.append({"tol": tol, "closure_fraction": frac, "cell_steps_per_s": cells * N0 * K / t,
                      "speedup": tp / t, "coarse_state_rel_err": e, "max_rel_err": max(e.values())})
    out["network"] = sweep
    q, t, frac, _, _ = run(1, 0.0)
    out["mean_field_all"] = {"closure_fraction": frac, "cell_steps_per_s": cells * N0 * K / t, "speedup": tp / t,
                             "coarse_state_rel_err": err(q)}
    ok = [r for r in sweep if r["speedup"] > 1.0 and r["max_rel_err"] <= target_err]
    if ok:
        best = max(ok, key=lambda r: r["speedup"])
        out["crossover"] = {"target_err": target_err, "tol": best["tol"], "speedup": best["speedup"],
                            "max_rel_err": best["max_rel_err"], "closure_fraction": best["closure_fraction"]}
    else:
        out["crossover"] = {"target_err": target_err, "tol": None,
                            "statement": "no bound in the sweep is both faster than the particle path and "
                                         "within the error target"}
    out["seconds"] = time.perf_counter() - t0
    net.close()
    return out


def ensemble_eval(msdem, warmup=2, steps=5):
    """The ensemble workload (16 seeded realizations of 256 x 256 cells,
    about 8M floes, one model): device-timed coarse intervals after warm-up,
    an L2 flush before each."""
    import torch
    s = load_scenario("ensemble_16x256x256")
    p, dt, N0 = s["params"], s["dt"], int(s["params"]["N0"])
    st = torch.cuda.Stream()
    m = msdem.Model(p, s["floes"], msdem.MS_FP32)
    m.set_stream(st.cuda_stream)
    for _ in range(warmup):
        m.step(dt, N0)
    m.sync()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ms = []
    for k in range(steps):
        with torch.cuda.stream(st):
            flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        m.step_async(dt, N0)
        e1.record(st)
        st.synchronize()
        ms.append(e0.elapsed_time(e1))
    m.sync()
    n, nc = m.n, m.ncell
    info = m.info()
    m.close()
    tot = sum(ms) / 1e3
    return {"workload": workload_config(s, "flushed before every timed interval (512 MB write)")["workload"],
            "floes": int(n), "cells": int(nc), "intervals_timed": steps, "ms_per_interval": 1e3 * tot / steps,
            "floe_steps_per_s": n * N0 * steps / tot, "cell_steps_per_s": nc * N0 * steps / tot,
            "launch_variant": info["variant"]}


def load_scenario(name: str):
    from paper_2303_07819_gb300 import inputs as I
    cache = os.path.join(tempfile.gettempdir(), f"msdem_inputs_{name}_{I.BASE_SEED}.npz")
    if os.path.exists(cache):
        z = np.load(cache, allow_pickle=True)
        s = z["s"].item()
        return s
    s = I.WORKLOADS[name]()
    try:
        np.savez(cache, s=np.array(s, dtype=object))
    except OSError:
        pass
    return s


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"msdem_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def oracle_sample_rate(s, ncells: int, steps: int, seed: int = 0, threads: int | None = None):
    """Floe-steps/s of the FP64 oracle (all host cores, or `threads`) on
    `ncells` random cells of the workload for `steps` fine steps."""
    from oracle import oracle as O
    O.build()
    cores = threads if threads else len(os.sched_getaffinity(0))
    O.set_threads(cores)
    p = dict(s["params"], nens=1)           # an ensemble: cells of its first realization
    fl = s["floes"]
    if "cell" in s["meta"]:
        cell = s["meta"]["cell"]
    else:
        cell = (np.floor(fl["y"] / (p["Ly"] / p["ny"])).astype(np.int64) * p["nx"] +
                np.floor(fl["x"] / (p["Lx"] / p["nx"])).astype(np.int64))
    rng = np.random.default_rng(seed)
    pick = rng.choice(p["nx"] * p["ny"], size=min(ncells, p["nx"] * p["ny"]), replace=False)
    sel = np.isin(cell, pick)
    sub = {k: v[sel] for k, v in fl.items()}
    m = O.Model(p, sub)
    t0 = time.perf_counter()
    m.step(s["dt"], steps)
    dt = time.perf_counter() - t0
    n = int(sel.sum())
    m.close()
    return n * steps / dt, n, dt, cores


def calibrated_oracle(s, target_s: float, ncells: int = 4096):
    """A sample of `ncells` random cells and the number of fine steps that
    takes the oracle about target_s seconds on all host cores."""
    p = s["params"]
    ncells = min(ncells, p["nx"] * p["ny"])
    rate, n, dt, cores = oracle_sample_rate(s, ncells, 1, seed=1)
    steps = int(max(1, min(1000, round(target_s * rate / max(n, 1)))))
    return ncells, steps


def job_rate(units_per_rank, ms_local, world, dist=None, device="cpu"):
    """Whole-job throughput of `world` ranks that each processed
    `units_per_rank` units (replicas of one workload, one per GPU): all ranks'
    units over the slowest rank's timed milliseconds.  Returns (rate, max ms)."""
    import torch
    tot_ms = float(ms_local)
    if dist is not None:
        t = torch.tensor([tot_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    return world * units_per_rank / (tot_ms / 1e3), tot_ms


def run_reference(args, s, rank):
    if rank != 0:
        return
    from paper_2303_07819_gb300 import inputs as I  # noqa: F401
    p = s["params"]
    ncells, steps = calibrated_oracle(s, 8.0)
    for w in range(args.warmup):
        oracle_sample_rate(s, max(64, ncells // 8), 1, seed=100 + w)
    tot_fs, tot_t, cores, nsum = 0.0, 0.0, 0, 0
    for k in range(args.steps):
        rate, n, dt, cores = oracle_sample_rate(s, ncells, steps, seed=k)
        tot_fs += n * steps
        tot_t += dt
        nsum += n
    value = tot_fs / tot_t
    sample = (f"{ncells} random cells (~{nsum // args.steps} floes) of the workload, {steps} fine steps "
              f"per bench step, FP64 oracle, OpenMP over cells")
    line = {
        "impl": "reference", "metric": "floe-steps/s", "value": value, "unit": "floe-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(s, "none (CPU)"),
        "cpu_baseline": {"value": value, "unit": "floe-steps/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "floe-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(s, l2):
    p = s["params"]
    nens = int(p.get("nens", 1))
    if nens > 1:
        w = (f"msDEM ensemble batch: {nens} realizations x {p['nx']}x{p['ny']} cells of 25 km, lognormal(6, 0.69) "
             f"floes/cell clipped [1,64], power-law radii 0.2-3 km, one 8-mode ocean and rotating 6 h wind, "
             f"dt 5 s, N0 100, n_t 10")
    else:
        w = ("msDEM batched cells: 128x128 cells of 25 km, lognormal(96, 0.69) floes/cell "
             "clipped [8,1024], power-law radii 0.2-3 km, 8-mode ocean, rotating 6 h wind, "
             "dt 5 s, N0 100, n_t 10")
    return {"workload": w,
            "floes": int(s["floes"]["x"].shape[0]), "cells": int(p["nx"] * p["ny"] * nens),
            "fine_steps_per_step": int(p["N0"]), "state": "FP32 floes, FP64 moments and coarse solve",
            "l2": l2}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_128x128",
                    choices=["square_4x4", "powerlaw_32x32", "batched_128x128", "ensemble_16x256x256"])
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, cpu baseline and autotune")
    ap.add_argument("--variant", type=int, default=-1, help="force the cell-kernel variant (profiling)")
    ap.add_argument("--profile", type=int, default=0,
                    help="no timing: build the model, run N fine steps and exit (for ncu captures)")
    ap.add_argument("--truth", type=int, default=0,
                    help="the truth DEM of --workload alone: run N steps and exit (for ncu captures), "
                         "or with --truth-time time it")
    ap.add_argument("--truth-time", action="store_true", help="print the truth DEM's time per step")
    ap.add_argument("--closure-train", type=int, default=0,
                    help="the closure network's training alone at batch B on 65,536 synthetic samples "
                         "(random-init weights), each engine: time it and exit (for ncu captures)")
    ap.add_argument("--closure-infer", type=int, default=0,
                    help="the closure network's inference kernel alone on N cells of synthetic features "
                         "(random-init weights): time it and exit (for ncu captures)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    s = load_scenario(args.workload)
    if args.impl == "reference":
        run_reference(args, s, rank)
        return

    import torch
    from paper_2303_07819_gb300 import msdem
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    msdem.load()
    if args.closure_train:
        print(json.dumps(closure_training_rate(msdem, args.closure_train)), flush=True)
        return
    if args.closure_infer:
        from paper_2303_07819_gb300 import inputs as I
        rng = np.random.default_rng(3)
        X = rng.normal(size=(4096, 16)).astype(np.float32)
        Y = rng.normal(size=(4096, 4)).astype(np.float32)
        net = msdem.MLP(I.mlp_init(), msdem.fit_norm(X, Y), max_batch=4096)
        out = closure_inference_rate(net, X, n=args.closure_infer, reps=5)
        net.close()
        print(json.dumps(out), flush=True)
        return
    if args.truth:
        tp = dict(s["params"], couple=0)
        tm = msdem.Model(tp, s["floes"], msdem.MS_FP32)
        tm.truth_step(s["dt"], args.truth)
        out = {"truth_steps": args.truth}
        if args.truth_time:
            ms = min(tm.time_kernel(1, s["dt"], 50) for _ in range(3))
            n = int(s["floes"]["x"].shape[0])
            out.update({"floes": n, "ms_per_truth_step": ms, "floe_steps_per_s": n / (ms * 1e-3)})
        tm.sync()
        print(json.dumps(out), flush=True)
        tm.close()
        return
    p = s["params"]
    dt = s["dt"]
    N0 = int(p["N0"])
    stream = torch.cuda.Stream()
    sharded = None
    if world > 1:
        # one grid split into tiles of cells, one per rank; the coarse
        # inputs are all-gathered (NCCL) once per coarse interval
        from paper_2303_07819_gb300 import shard
        sharded = shard.ShardedModel(p, s["floes"], world, rank, precision=msdem.MS_FP32)
        model = sharded.model
    else:
        model = msdem.Model(p, s["floes"], msdem.MS_FP32)
    model.set_stream(stream.cuda_stream)
    n_floes, ncell = int(s["floes"]["x"].shape[0]), model.ncell   # the whole grid's
    if args.profile:
        if args.variant >= 0:
            model.set_launch(args.variant, 128, 0)
        model.step(dt, args.profile)
        print(json.dumps({"profile_steps": args.profile, "info": model.info()}), flush=True)
        model.close()
        return
    if args.variant >= 0:
        model.set_launch(args.variant, 128, 0)
    elif not args.no_extras:
        model.autotune(dt, reps=3)
    info = model.info()

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        model.step(dt, N0)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        ev[k][0].record(stream)
        model.step_async(dt, N0)
        ev[k][1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    model.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    fine_steps = args.steps * N0
    # the ranks share one grid: all its floes over the slowest rank's time
    value, tot_ms = job_rate(n_floes * fine_steps, float(sum(step_ms)), 1, dist, "cuda")
    cell_rate = ncell * fine_steps / (tot_ms / 1e3)

    hbm, peak_kind, _ = peaks()
    traffic, prof = profile_traffic()
    if args.workload != "batched_128x128":     # the committed capture is of this workload only
        traffic, prof = None, None
    kern_ms_live = tot_ms / fine_steps          # per fine step, incl. the coarse step's share
    kern_ms_interval = model.time_kernel(2, dt, 10)   # cell kernels of one interval alone, out of place
    # per GPU: this rank's floes (all of them at N = 1) over the step time
    achieved = model.n * BYTES_PER_FLOE_STEP / (kern_ms_live / 1e3) / 1e9
    # the FP32 side of the roofline: the FMA rate this GPU reaches (probe),
    # the FMA-pipe activity ncu measured on the cell kernels, and the issue
    # rate the live step implies for ncu's instruction count (of the peak
    # 4 warp instructions per SM per cycle at the sampled clock)
    fp32_peak = msdem.probe_fp32(5)
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    issue_frac = None
    if prof is not None and traffic is not None and clk.get("sm_mhz"):
        wi = float(prof["warp_instructions_per_interval"])
        issue_frac = wi / (tot_ms / args.steps / 1e3) / (nsm * 4 * clk["sm_mhz"] * 1e6)

    line = {
        "metric": "floe-steps/s", "value": value, "unit": "floe-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "cell_steps_per_s": cell_rate,
        "config": workload_config(s, "flushed before every timed step (512 MB write); state 64 MB"),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": (traffic if traffic is not None and info["variant"] == 5 else None),
                     "traffic_per": "coarse interval (one launch of each resident class)",
                     "kernel": "msd::k_cell_run32_block<1|2|4> (resident for a coarse interval)",
                     "peak_source": peak_kind,
                     "bytes_per_floe_step": BYTES_PER_FLOE_STEP,
                     "algorithmic_bytes_per_interval": model.n * BYTES_PER_FLOE_STEP * N0,
                     "kernel_ms_live": kern_ms_live, "cell_kernels_ms_per_interval_alone": kern_ms_interval,
                     "fp32_peak_tflops_probe": fp32_peak,
                     "fp32_pipe_frac_ncu": (float(prof["fp32_pipe_frac"]) if traffic is not None else None),
                     "issue_frac": issue_frac},
        "clocks": clk,
        "gpu_launches": args.steps * (info["launches_per_interval"] + info["launches_per_coarse"]
                                      + (2 if sharded else 0)),   # + pack and scatter of the exchange
        "launch": {"variant": info["variant"], "threads": info["threads"], "persistent": info["persistent"]},
        "wall_s": t_wall,
    }

    if not args.no_extras:
        # end to end through the public API with host buffers: upload the
        # state, one coarse interval, read the moments back (every rank, as
        # the interval's exchange needs them all).  Each step's input is the
        # state the model holds (fetched before the timer starts), so the
        # run continues as the device-resident one does; an older state
        # uploaded again while the coarse solution moves on is not a state
        # of the method, and drives it unstable within a few intervals.
        # The step's input sits in page-locked host memory (as a loader
        # would leave it), which ms_set_floes sends without a host copy.
        ke = max(1, min(args.steps, 5))
        model.set_floes(model.floes())
        model.step(dt, N0)
        pinned = torch.empty((8, model.n), dtype=torch.float64).pin_memory().numpy()
        host = {k: pinned[i] for i, k in enumerate(msdem.FLOE_KEYS)}
        te = 0.0
        for _ in range(ke):
            for k, v in model.floes().items():
                host[k][:] = v
            t0 = time.perf_counter()
            model.set_floes(host)
            model.step_async(dt, N0)
            mom = model.moments()
            te += time.perf_counter() - t0
        _, te_ms = job_rate(1, te * 1e3, 1, dist, "cuda")
        line["e2e"] = {"value": n_floes * N0 * ke / (te_ms / 1e3), "unit": "floe-steps/s",
                       "h2d_bytes_per_step": int(64 * n_floes), "d2h_bytes_per_step": int(world * mom.nbytes),
                       "host_buffers": "page-locked (torch pin_memory), sent without a host copy"}
    if sharded is not None:
        line["config"]["parallelism"] = (f"{world} tiles of cells (recursive bisection balanced by floe "
                                         f"pairs), coarse inputs all-gathered once per coarse interval (NCCL)")
        line["shard_floes"] = int(model.n)
    if not args.no_extras and rank == 0:
        ncells, steps = calibrated_oracle(s, 15.0)
        rate, n, tdt, cores = oracle_sample_rate(s, ncells, steps)
        # the same oracle on one thread, a 32nd of the cells (about the same wall time)
        n1cells = max(8, ncells // 32)
        rate1, n1, tdt1, _ = oracle_sample_rate(s, n1cells, steps, seed=2, threads=1)
        line["cpu_baseline"] = {"value": rate, "unit": "floe-steps/s", "cores": cores, "kind": "oracle",
                                "cell_steps_per_s": ncells * steps / tdt,
                                "sample": f"{ncells} random cells ({n} floes) x {steps} fine steps, "
                                          f"{tdt:.1f} s wall, FP64, OpenMP over cells",
                                "one_thread": {"value": rate1, "unit": "floe-steps/s",
                                               "cell_steps_per_s": n1cells * steps / tdt1,
                                               "sample": f"{n1cells} random cells ({n1} floes) x {steps} "
                                                         f"fine steps, {tdt1:.1f} s wall"}}
        if args.workload == "batched_128x128":
            line["closure"] = closure_eval(msdem, s)
            line["ensemble"] = ensemble_eval(msdem)
    model.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
