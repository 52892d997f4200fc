"""Benchmark of the MOT hot path (one JSON line on rank 0).

A step is one pass of the whole hot path for all right-hand sides of the workload: plane-wave
tests, history sum with the right-hand-side blocks, T_0 solve, projector and post-processing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

N > 1 (torchrun): every rank marches its own copy of the workload (independent incident-wave
batches; weak scaling, no data-path collective); value = all ranks' steps / max time.
--impl reference times the FP64 CPU oracle (a deliberately slow reference program) on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "sphere7680_r64"
L2_BYTES = 126 * 2 ** 20
METRIC = "MOT steps/s"


def workload(name: str, precision: str | None = None, waves: int | None = None, form: str = "dense"):
    from synth import workloads
    w = {
        "sphere480_fp64": workloads.sphere480_fp64,
        "torus864_fp32": workloads.torus864_fp32,
        "sphere7680_r64": workloads.sphere7680_r64,
        "sphere1920_r64": workloads.sphere1920_r64,
        "ellipsoid12288": workloads.ellipsoid12288,
    }[name]()
    if precision:
        w["precision"] = precision
    if waves:
        w["pw"] = {k: v[:waves] for k, v in w["pw"].items()}
        w["name"] = f"{w['name']}_waves{waves}"
    w["form"] = form
    if form != "dense":
        w["name"] = f"{w['name']}_{form}"
    if name == "torus864_fp32":
        # alpha = 1 puts a real polynomial eigenvalue of modulus 1.89 outside the unit circle at
        # this time step on this torus; alpha = 0.5 keeps the spectrum inside (radius 0.84)
        w["alpha"] = 0.5
    return w


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def whole_job_rate(dev_ms: float, steps: int, ws: int, pg=None, device="cpu"):
    """Whole-job steps/s of N replicas: every rank marched `steps` steps of its own batch in
    dev_ms; the job takes the slowest rank's time (all-reduce MAX), and the value counts the steps
    of all ranks.  Returns (value, max_ms)."""
    import torch
    tot_ms = float(dev_ms)
    if pg is not None:
        t = torch.tensor([float(dev_ms)], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        tot_ms = float(t.item())
    return ws * steps / (tot_ms / 1e3), tot_ms


def oracle_threads() -> int:
    """Threads the oracle's BLAS may use: the thread-count variable when one is set, else every core."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k, "").isdigit():
            return int(os.environ[k])
    return os.cpu_count()


def cpu_oracle_dense_rate(w, steps: int = 3):
    """Oracle dense march (oracle.mot.march_dense, FP64 numpy) on blocks of the workload's size.

    For meshes whose FP64 oracle assembly takes hours, the timed sample is the oracle's own
    marching step applied to dense FP64 blocks of the workload's size (N edges, K blocks, R
    waves) filled with synthetic values; the arithmetic per step does not depend on the values."""
    import numpy as np

    from oracle import mot
    from oracle.topology import Topology, n_lags
    t = Topology(w["V"], w["F"])
    K = n_lags(t.D, w["dt"])
    R = int(w["pw"]["k"].shape[0])
    T = np.empty((K, t.ne, t.ne))
    rng = np.random.default_rng(0)
    row = rng.standard_normal(t.ne) / t.ne
    T[:] = row[None, None, :]
    T[0] += 4.0 * np.eye(t.ne)
    r = rng.standard_normal((K + steps, t.ne, R))
    mot.march_dense(T, r[:2])              # warm-up (LU of T_0 and BLAS threads)
    t1 = time.time()
    mot.march_dense(T, r[: K + steps])
    el = time.time() - t1
    # the march of K + steps steps: the first K - 1 steps see fewer history blocks; count the
    # block-matvec work and express the rate in full steps (K - 1 history blocks each)
    full_equiv = sum(min(n, K - 1) for n in range(K + steps)) / (K - 1)
    return full_equiv / el, K + steps, K


def cpu_oracle_rate(w, max_steps: int, budget_s: float = 20.0):
    """Oracle (FP64, numpy + plain C) march on the host cores: steps/s over a bounded sample."""
    import numpy as np
    if w["F"].shape[0] > 2000:
        rate, n, K = cpu_oracle_dense_rate(w)
        return rate, n, None
    from oracle import mot, rhs
    from oracle.assemble import Operators
    from oracle.formulation import Formulation
    t0 = time.time()
    ops = Operators(w["V"], w["F"], dt=w["dt"], alpha=w["alpha"])
    fm = Formulation(ops)
    t_asm = time.time() - t0
    # calibrate the sample so the march takes about budget_s
    n = min(max_steps, w["Nt"])
    e, h = rhs.incident_tests(ops, w["pw"], w["dt"] * np.arange(1, n + 1))
    r = fm.rhs(e, h)
    t1 = time.time()
    mot.march_factored(fm, r[: min(n, 20)])
    per = (time.time() - t1) / min(n, 20)
    n = int(max(10, min(n, budget_s / max(per, 1e-6))))
    t1 = time.time()
    mot.march_factored(fm, r[:n])
    dt = time.time() - t1
    return n / dt, n, t_asm


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    rate, n, t_asm = cpu_oracle_rate(w, args.steps * 20, budget_s=min(60.0, 5.0 * args.steps))
    cores = oracle_threads()
    sample = (f"{n} march steps after an untimed {t_asm:.1f} s assembly" if t_asm is not None else
              f"oracle dense march, {n} steps on dense FP64 blocks of the workload's size (synthetic values; "
              f"the FP64 oracle assembly of this mesh is out of reach), rate in full-history steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / rate, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "edges": int(w["F"].shape[0] * 3 // 2), "R": int(w["pw"]["k"].shape[0]),
                   "dt": w["dt"], "alpha": w["alpha"]},
        "cpu_baseline": {"value": rate, "unit": "steps/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_guess_study(args, w):
    """GMRES initial guesses on the 12288-edge ellipsoid (FP32, GMRES tol 1e-8), against the direct
    T_0^-1 solve (the plain GPU march): zero, previous step, cubic extrapolation of the last four
    steps, and two learned networks trained on 7680-edge sphere trajectories -- the increment over
    y_{n-1} and the correction to the extrapolation.  Reported per guess: steps/s, GMRES iterations,
    the guess error |x0 - y_n| / |y_n| over the march, rel-L2 against the direct march."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2312_06367_gb300 import Solver, mlp_predict, mlp_samples, mlp_train
    from synth import workloads
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    info = {}
    # 1. training trajectories (plain FP32 direct march of 8 waves) on the GPU
    tw = workloads.sphere7680_train8()
    t0 = time.time()
    st = Solver(tw["V"], tw["F"], dt=tw["dt"], nt=tw["Nt"], precision="fp32", R=8, stream=stream.cuda_stream).assemble()
    info["train_assemble_s"] = round(time.time() - t0, 1)
    y = torch.empty((tw["Nt"], 8, st.ne), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        st.set_excitation(tw["pw"])
        st.step_y(tw["Nt"], None, y)
        torch.cuda.synchronize()
    st.close()
    # 2. one network per base (Adam, GPU kernels); seeded uniform(+-1/sqrt(fan_in)) weights, zero biases
    nets = {}
    for base in ("prev", "extrap"):
        with torch.cuda.stream(stream):
            X, Y = mlp_samples(y, base=base)
        rng = np.random.default_rng(2312063672)
        parts = []
        for fan_in, n_w, n_b in ((8, 64 * 8, 64), (64, 64 * 64, 64), (64, 64, 1)):
            lim = 1.0 / np.sqrt(fan_in)
            parts += [rng.uniform(-lim, lim, n_w), np.zeros(n_b)]
        params = torch.tensor(np.concatenate(parts), dtype=torch.float32, device="cuda")
        t0 = time.time()
        with torch.cuda.stream(stream):
            hist = mlp_train(params, X, Y, epochs=args.train_epochs, batch=4096, lr=1e-3, seed=7)
        torch.cuda.synchronize()
        info[base] = dict(train_samples=int(X.shape[0]), train_epochs=args.train_epochs,
                          train_s=round(time.time() - t0, 2), loss_first=float(hist[0]), loss_last=float(hist[-1]))
        nets[base] = params
        del X, Y
    del y
    torch.cuda.empty_cache()                      # the evaluation assembly needs most of the HBM
    # 3. evaluation handle; the direct march's y gives the guess errors
    t0 = time.time()
    s = Solver(w["V"], w["F"], dt=w["dt"], nt=w["Nt"], alpha=w["alpha"], precision="fp32", R=1,
               stream=stream.cuda_stream, solver="gmres", guess="zero", gmres_tol=w["gmres_tol"]).assemble()
    t_asm = time.time() - t0
    nt = w["Nt"]
    outs, rows = {}, {}
    yd = torch.empty((nt, 1, s.ne), dtype=torch.float32, device="cuda")
    for mode in ("direct", "zero", "prev", "extrap", "mlp", "mlp_extrap"):
        if mode == "direct":
            s.set_solver("direct")
        else:
            s.set_solver("gmres", mode, w["gmres_tol"])
            if mode.startswith("mlp"):
                s.mlp_load(nets["extrap" if mode == "mlp_extrap" else "prev"].cpu().numpy())
        out = torch.empty((nt, 1, s.ne), dtype=torch.float32, device="cuda")
        with torch.cuda.stream(stream):
            s.set_excitation(w["pw"])
            s.step(args.warmup)                   # warm-up: captures the step graph
            torch.cuda.synchronize()
            with Clocks(local) as clk:
                s.set_excitation(w["pw"])
                if mode == "direct":
                    s.step_y(nt, out, yd)
                else:
                    s.step(nt, out)
                torch.cuda.synchronize()
        tm = s.timing()
        row = {"steps_s": 1e3 / tm["step_ms"], "ms_per_step": tm["step_ms"], "history_ms": tm["history_ms"],
               "launches": tm["launches"], "clocks": clk.summary()}
        if mode != "direct":
            row.update(s.gmres_stats())
            row["iterations_per_step"] = row["iterations"] / max(row["steps"], 1)
        rows[mode] = row
        outs[mode] = out[:, 0, :].double()
    ref = outs["direct"]
    for mode in rows:
        rows[mode]["rel_l2_vs_direct"] = float(torch.linalg.norm(outs[mode] - ref) / torch.linalg.norm(ref))
    # guess errors |x0 - y_n| / |y_n| over steps 9 .. nt of the direct march (analysis, on the device)
    yv = yd[:, 0, :].double()
    yn, y1, y2, y3, y4 = yv[8:], yv[7:-1], yv[6:-2], yv[5:-3], yv[4:-4]
    ext = 4 * y1 - 6 * y2 + 4 * y3 - y4
    sc = torch.sqrt(torch.mean(y1 ** 2, dim=1, keepdim=True))
    sc = torch.where(sc > 0, sc, torch.ones_like(sc))
    Xf, _ = mlp_samples(yd)
    den = torch.linalg.norm(yn)
    gerr = {"zero": 1.0, "prev": float(torch.linalg.norm(yn - y1) / den), "extrap": float(torch.linalg.norm(yn - ext) / den)}
    for mode, base in (("mlp", y1), ("mlp_extrap", ext)):
        f = mlp_predict(nets["extrap" if mode == "mlp_extrap" else "prev"], Xf).double().reshape(nt - 8, s.ne)
        gerr[mode] = float(torch.linalg.norm(yn - (base + sc.float().double() * f)) / den)
    for mode in gerr:
        rows[mode]["guess_error"] = gerr[mode]
    best = min(("zero", "prev", "extrap", "mlp", "mlp_extrap"), key=lambda m: rows[m]["ms_per_step"])
    m = rows[best]
    pk = peaks()
    hb = s.timing()["history_bytes"]
    line = {
        "metric": METRIC, "value": m["steps_s"], "unit": "steps/s", "n_gpus": 1, "steps": nt, "warmup": args.warmup,
        "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["name"], "edges": s.ne, "triangles": s.nc, "R": 1, "K": s.K, "dt": w["dt"],
                   "solver": "gmres", "guess": best, "gmres_tol": w["gmres_tol"], "assemble_s": round(t_asm, 1),
                   "cache": "inputs larger than L2"},
        "gpu_launches": int(m["launches"]),
        "roofline": {"bound": "hbm", "achieved": hb / (m["history_ms"] / 1e3) / 1e9 if m["history_ms"] else None,
                     "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                     "frac": (hb / (m["history_ms"] / 1e3) / 1e9 / pk["hbm_gbs"]) if m["history_ms"] else None,
                     "traffic": None, "kernel": "history sum (k_history + k_reduce)",
                     "algorithmic_bytes_per_launch": hb},
        "guess_study": rows, "training": info,
    }
    print(json.dumps(line), flush=True)
    s.close()
    return 0


def run_accuracy(args, w):
    """Full-size accuracy of the reduced-precision paths: the workload's mesh and waves marched in
    FP64 (the path that matches the oracle to 1e-10 on every case the oracle can assemble) as the
    reference for 8 waves, then the same FP64-formed blocks re-planned for FP32 (R = 8) and for the
    tensor-core FP16X3 path (all R waves); rel-L2 of the currents over all steps, edges and the 8 waves."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2312_06367_gb300 import Solver
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    R = int(w["pw"]["k"].shape[0])
    nt = args.steps
    pw8 = {k: v[:8] for k, v in w["pw"].items()}
    t0 = time.time()
    s = Solver(w["V"], w["F"], dt=w["dt"], nt=nt, alpha=w["alpha"], precision="fp64", R=8).assemble()
    t_asm = time.time() - t0

    def march(prec, r, pw):
        s.replan(prec, r)
        out = torch.zeros((nt, r, s.ne), dtype=s.dtype, device="cuda")
        s.march(pw, out)
        torch.cuda.synchronize()
        return out[:, :8].double().cpu().numpy(), 1e3 / s.timing()["step_ms"]

    ref, r64 = march("fp64", 8, pw8)
    res = {"fp64": {"steps_s": r64}}
    runs = [("fp32", 8, pw8)]
    if R == 64:
        runs.append(("fp16x3", 64, w["pw"]))
    for prec, r, pw in runs:
        j, rate = march(prec, r, pw)
        err = float(np.linalg.norm(j - ref) / np.linalg.norm(ref))
        win = {}
        for a, b in ((0, nt // 4), (nt // 4, nt // 2), (nt // 2, nt)):
            win[f"steps_{a}_{b}"] = float(np.linalg.norm(j[a:b] - ref[a:b]) / max(np.linalg.norm(ref[a:b]), 1e-300))
        res[prec] = {"rel_l2_vs_fp64": err, "by_window": win, "steps_s": rate, "R": r}
    line = {"metric": "rel-L2 of the surface current vs the FP64 path", "workload": w["name"],
            "edges": s.ne, "K": s.K, "dt": w["dt"], "steps": nt, "waves_compared": 8,
            "assemble_fp64_s": round(t_asm, 1), "results": res}
    print(json.dumps(line), flush=True)
    s.close()
    return 0


def run_batch(args, probs, name):
    """Uneven batch: every scatterer FP32 with one wave, all advanced by one graph launch per step
    (tdcfie_batch_step: the persistent cooperative kernel, launch shape from tdcfie_batch_tune),
    against the same handles stepped one after another (tdcfie_step each)."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2312_06367_gb300 import Batch, Solver
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    t0 = time.time()
    ss = []
    for p in sorted(probs, key=lambda p: -p["F"].shape[0]):     # largest first: the FP64 peak is lowest
        s = Solver(p["V"], p["F"], dt=p["dt"], nt=args.steps, alpha=p["alpha"], precision="fp32", R=1).assemble()
        s.release_assembly()                 # keep only the FP32 step plan on the device
        s.set_excitation(p["pw"])
        s._p = p
        ss.append(s)
    t_asm = time.time() - t0
    # one after another: each handle's own graph, warmed up, then timed
    seq_ms = 0.0
    for s in ss:
        s.step(args.warmup)
        s.step(args.steps)
        seq_ms += s.timing()["step_ms"]
    for s in ss:
        s.set_excitation(s._p["pw"])
    b = Batch(ss)
    t1 = time.time()
    cfg = b.tune(3)
    t_tune = time.time() - t1
    b.step(args.warmup)
    outs = [torch.empty((args.steps, 1, s.ne), dtype=torch.float32, device="cuda") for s in ss]
    with Clocks(local) as clk:
        b.step(args.steps, outs)
    t = b.timing()
    finite = all(bool(torch.isfinite(o).all().item()) for o in outs)
    hb = sum(s.timing()["history_bytes"] for s in ss)
    pk = peaks()
    line = {
        "metric": METRIC, "value": 1e3 / t["step_ms"], "unit": "steps/s (all scatterers advance one step)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t["step_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": name, "scatterers": len(ss), "edges": [s.ne for s in ss], "K": [s.K for s in ss],
                   "dt": probs[0]["dt"], "assemble_s": round(t_asm, 1), "tune_s": round(t_tune, 2), "launch": cfg,
                   "cache": f"history operands of all scatterers ({hb / 1e9:.2f} GB) stream each step",
                   "finite": finite},
        "gpu_launches": int(t["launches"]) * args.steps,
        "sequential": {"ms_per_step": seq_ms, "steps_s": 1e3 / seq_ms, "how": "each handle's own step graph, one after another"},
        "speedup_vs_sequential": seq_ms / t["step_ms"],
        "roofline": {"bound": "hbm", "achieved": hb / (t["step_ms"] / 1e3) / 1e9, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                     "frac": hb / (t["step_ms"] / 1e3) / 1e9 / pk["hbm_gbs"], "traffic": None,
                     "kernel": "whole batch step (k_batch_step; history rows dominate)", "algorithmic_bytes_per_launch": hb},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    b.close()
    for s in ss:
        s.close()
    return 0


def accuracy_in_run(s, w, nt, stream):
    """Measured in this run on the same FP64-formed blocks: the FP64 path (the path that matches
    the oracle to 1e-10 wherever the oracle can assemble) marches the first 8 waves for nt steps;
    the timed path (all waves) and the plain single-wave FP32 path march the same steps; rel-L2 of
    the currents over steps x edges x waves against the FP64 march."""
    import numpy as np
    import torch
    R = int(w["pw"]["k"].shape[0])
    prec = w["precision"]
    pw8 = {k: v[:8] for k, v in w["pw"].items()}
    pw1 = {k: v[:1] for k, v in w["pw"].items()}

    def march(p, r, pw):
        s.replan(p, r)
        out = torch.zeros((nt, r, s.ne), dtype=s.dtype, device="cuda")
        with torch.cuda.stream(stream):
            s.set_excitation(pw)
            s.step(nt, out)
        torch.cuda.synchronize()
        return out.double().cpu().numpy()

    ref = march("fp64", min(8, R), pw8)
    got = march(prec, R, w["pw"])[:, :ref.shape[1]]
    one = march("fp32", 1, pw1)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    res = {"steps": nt, "waves": ref.shape[1], "reference": "FP64 path on the same FP64-formed blocks",
           "rel_l2_vs_fp64_path": rel(got, ref), "plain_fp32_rel_l2_vs_fp64_path": rel(one, ref[:, :1]),
           "bar": 1e-5}
    res["meets_bar"] = res["rel_l2_vs_fp64_path"] <= 1e-5
    return res


def factored_study(s, w, steps, warmup, nt_acc, stream):
    """The two forms of the history sum on the workload's mesh with one incident wave, same FP64
    assembly: the dense T_k stream (k_history + k_reduce) against the shell-sparse factored form
    (k_shells, then one dense product with T_0^-1 [-A | alpha L2 | -L1 Sigma]); per path precision
    the step rate, the history kernels' time and algorithmic bytes, the matrix bytes per step, and
    the rel-L2 of the factored currents against the dense ones over nt_acc steps."""
    import numpy as np
    import torch
    one = {k: v[:1] for k, v in w["pw"].items()}
    pk = peaks()
    res = {}
    for prec in ("fp32", "fp64"):
        s.replan(prec, 1)                  # keeps the handle's history form: measure that one first
        first = s.history_stats()["form"]
        row = {}
        cur = {}
        for form in (first, "factored" if first == "dense" else "dense"):
            if form != first:
                s.set_history_form(form)
            st = s.history_stats()
            acc = torch.zeros((nt_acc, 1, s.ne), dtype=s.dtype, device="cuda")
            with torch.cuda.stream(stream):
                s.set_excitation(one)
                s.step(nt_acc, acc)
                s.set_excitation(one)
                s.step(warmup)
                s.step(steps)
            torch.cuda.synchronize()
            t = s.timing()
            cur[form] = acc.double().cpu().numpy()
            h_ms = t["history_ms"]
            gbs = st["history_bytes"] / (h_ms / 1e3) / 1e9 if h_ms > 0 else None
            row[form] = {"steps_s": 1e3 / t["step_ms"], "step_ms": t["step_ms"], "history_ms": h_ms,
                         "history_bytes": st["history_bytes"], "step_bytes": st["step_bytes"],
                         "history_gbs": gbs, "history_frac_hbm": gbs / pk["hbm_gbs"] if gbs else None,
                         "launches_per_step": t["launches"] // max(1, steps)}
            if form == "factored":
                row[form]["shell_nnz"] = st["nnz"]
                row[form]["shell_nnz_per_ne2"] = st["nnz"] / s.ne ** 2
        d, f = cur["dense"], cur["factored"]
        row["rel_l2_factored_vs_dense"] = float(np.linalg.norm(f - d) / np.linalg.norm(d))
        row["speedup"] = row["factored"]["steps_s"] / row["dense"]["steps_s"]
        row["step_bytes_ratio"] = row["factored"]["step_bytes"] / row["dense"]["step_bytes"]
        res[prec] = row
    res["R"] = 1
    res["accuracy_steps"] = nt_acc
    return res


def run_ours(args, w):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2312_06367_gb300 import Solver

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    R = int(w["pw"]["k"].shape[0])
    prec = w["precision"]
    tensor = prec in ("bf16x3", "fp16x3")
    t0 = time.time()
    # the blocks are formed in FP64 so that the FP64 path can check the timed path in this run
    s = Solver(w["V"], w["F"], dt=w["dt"], nt=args.steps, alpha=w["alpha"], precision="fp64",
               R=R if not tensor else 8, stream=stream.cuda_stream, device=local).assemble()
    if prec != "fp64" or tensor:
        s.replan(prec, R)
    factored = w.get("form", "dense") == "factored"
    if factored:
        s.set_history_form("factored")
    t_asm = time.time() - t0
    esz = 8 if prec == "fp64" else 4
    work_bytes = s.timing()["history_bytes"]
    flush = work_bytes < 2 * L2_BYTES
    flush_buf = torch.empty(int(2 * L2_BYTES // 4), dtype=torch.float32, device=dev) if flush else None
    out = torch.empty((args.steps, R, s.ne), dtype=s.dtype, device=dev)
    s.set_excitation(w["pw"])

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize(dev)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            s.step(1)
            if flush:
                flush_buf.fill_(1.0)
        barrier()
        step_ms, hist_ms = [], []
        with Clocks(local) as clk:
            barrier()
            wall0 = time.perf_counter()
            if flush:
                for i in range(args.steps):
                    flush_buf.fill_(float(i))       # evict the L2 between timed steps
                    s.step(1, out[i:i + 1])
                    t = s.timing()
                    step_ms.append(t["step_ms"])
                    hist_ms.append(t["history_ms"])
            else:
                s.step(args.steps, out)
                t = s.timing()
                step_ms = [t["step_ms"]] * args.steps
                hist_ms = [t["history_ms"]]
            barrier()
            wall1 = time.perf_counter()
    dev_ms = sum(step_ms)
    launches = s.timing()["launches"] if not flush else s.timing()["launches"] * args.steps
    finite = bool(torch.isfinite(out).all().item())
    value, tot_ms = whole_job_rate(dev_ms, args.steps, ws, pg, dev)
    # end-to-end through the C ABI with host buffers: excitation from host, currents to pinned host
    host_out = torch.empty((args.steps, R, s.ne), dtype=s.dtype, pin_memory=True).numpy()
    barrier()
    e0 = time.perf_counter()
    s.march(w["pw"], host_out, out_on_host=True)
    barrier()
    e1 = time.perf_counter()
    e2e = ws * args.steps / (e1 - e0)
    # roofline of the dominant kernel (history sum: streams every history and right-hand-side block)
    pk = peaks()
    h_ms = statistics.mean(hist_ms) if hist_ms and hist_ms[0] > 0 else None
    achieved = work_bytes / (h_ms / 1e3) / 1e9 if h_ms else None
    traffic = None
    prof = os.path.join(ROOT, "profiles", f"history_{w['name']}.json")
    if os.path.exists(prof):
        try:
            traffic = json.load(open(prof)).get("dram_bytes_per_launch")
        except Exception:
            traffic = None
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "bf16x3": "bf16x3", "fp16x3": "fp16x3"}[prec],
        "data": "synthetic",
        "config": {"workload": w["name"], "edges": s.ne, "triangles": s.nc, "R": R, "K": s.K, "dt": w["dt"],
                   "alpha": w["alpha"], "precision": prec, "history_form": s.history_stats()["form"],
                   "step_matrix_bytes": s.history_stats()["step_bytes"],
                   "cache": "L2 flushed between timed steps" if flush else "inputs larger than L2",
                   "assemble_s": round(t_asm, 2), "wall_s": round(wall1 - wall0, 4), "finite": finite},
        "e2e": {"value": e2e, "unit": "steps/s", "h2d_bytes_per_step": 88 * R / args.steps,
                "d2h_bytes_per_step": R * s.ne * esz},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                     "frac": (achieved / pk["hbm_gbs"]) if achieved else None, "traffic": traffic,
                     "kernel": ("factored history sum over all lags of S_k, MM'_k, Phi_k (k_shells)" if factored else
                                "history sum (k_history + k_reduce)" if prec in ("fp64", "fp32") else
                                "tcgen05 split-precision history GEMM (k_tc_gemm, fixup in-kernel)"),
                     "algorithmic_bytes_per_launch": work_bytes, "history_ms": h_ms,
                     "peak_source": "measured" if not pk.get("fallback") else "fallback"},
        "clocks": clk.summary(),
    }
    if ws == 1 and tensor and not args.no_accuracy:
        acc = accuracy_in_run(s, w, args.accuracy_steps, stream)
        line["accuracy"] = acc
        # batched vs plain: the plain single-wave FP32 march on the same blocks, timed here
        s.replan("fp32", 1)
        one = {k: v[:1] for k, v in w["pw"].items()}
        o1 = torch.empty((args.steps, 1, s.ne), dtype=torch.float32, device=dev)
        with torch.cuda.stream(stream):
            s.set_excitation(one)
            s.step(args.warmup)
            s.step(args.steps, o1)
            torch.cuda.synchronize()
        plain = 1e3 / s.timing()["step_ms"]
        line["batched_vs_plain"] = {
            "plain": "FP32 history sum, R = 1 (one incident wave per march), same blocks", "plain_steps_s": plain,
            "batched_wave_steps_s": value / ws * R, "speedup_per_wave": value / ws * R / plain,
            "rel_l2_batched_vs_fp64": acc["rel_l2_vs_fp64_path"],
            "rel_l2_plain_vs_fp64": acc["plain_fp32_rel_l2_vs_fp64_path"]}
        if not args.no_factored:
            line["factored_form"] = factored_study(s, w, 20, 3, min(args.accuracy_steps, 200), stream)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, n, t_casm = cpu_oracle_rate(w, 4 * args.steps + 50)
        sample = (f"{n} march steps of the same workload (assembly {t_casm:.1f} s untimed)" if t_casm is not None else
                  f"oracle dense march, {n} steps on dense FP64 blocks of the workload's size (synthetic values; "
                  f"the FP64 oracle assembly of this mesh is out of reach), rate in full-history steps")
        line["cpu_baseline"] = {"value": rate, "unit": "steps/s", "cores": oracle_threads(), "kind": "oracle",
                                "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    s.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, help="override the workload's path precision")
    ap.add_argument("--waves", type=int, default=None, help="march only the first N incident waves")
    ap.add_argument("--history-form", default="dense", choices=["dense", "factored"],
                    help="history sum over the dense T_k or the shell-sparse factored form (FP64/FP32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the in-run accuracy check")
    ap.add_argument("--accuracy-steps", type=int, default=300, help="steps of the in-run accuracy check")
    ap.add_argument("--no-factored", action="store_true",
                    help="skip the dense-versus-factored history comparison on the workload's mesh")
    ap.add_argument("--accuracy", action="store_true",
                    help="full-size accuracy of the reduced-precision paths against the FP64 path")
    ap.add_argument("--train-epochs", type=int, default=4, help="learned-guess training passes (ellipsoid12288)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.workload.startswith("batch_uneven") or args.workload == "batch32":
        from synth import workloads
        if args.workload == "batch32":
            probs = workloads.batch32()
        else:
            probs = workloads.batch_uneven(int(args.workload[len("batch_uneven"):] or 16))
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the uneven batch is measured against the "
                              "same GPU handles stepped one after another, not against the oracle"}))
            return 0
        return run_batch(args, probs, args.workload)
    w = workload(args.workload, args.precision, args.waves, args.history_form)
    if args.impl == "reference":
        return run_reference(args, w)
    if args.accuracy:
        return run_accuracy(args, w)
    if args.workload == "ellipsoid12288":
        return run_guess_study(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
