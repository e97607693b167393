"""Benchmark: CA-SGD samples/s on one GB300 (and N independent replicas).

Workload (default, the headline): binary logistic regression, dense A
1,048,576 x 512 FP32 with entries N(0, 1/512), planted w*, 5% label flips;
CA-SGD with s = 8, b = 64, eta = 0.5, lambda = 0, 65,536 SGD-equivalent
iterations; Gram, margin and gradient operands in BF16 with FP32
accumulation, FP32 recurrence and master weights.  One bench step = one full
training run (x reset to 0, then 65,536 iterations through the C ABI,
replayed as a CUDA graph).

Roofline (every line): the run's roofline time T_roof sums, over its outer
iterations, the slower of the gathered bytes s b (n e_A + 4) at the measured
HBM bandwidth and the strictly block-lower Gram flops b^2 s (s-1) n at the
Gram type's peak; "step_frac" = T_roof / measured run time.  The dominant
kernel's own roofline uses the same per-outer-iteration units (bytes for
the gather and the chain, Gram flops for the Gram) over its average launch.

Extra legs (skipped with --no-extras): the other s of the headline workload,
TF32 and FP32 Grams, the FP32 plain-SGD GPU path, the end-to-end number with
host buffers, the CPU oracle (one core and every core), time to target loss,
the wide 400,000 x 2048 workload (per-column-scaled BF16/FP16 storage; FP8,
BF16 and FP32 Grams; s = 16, 32, 64 with the FP64 recurrence on and off),
the large 4,194,304 x 1024 BF16 least-squares workload (s = 64, b = 256)
and the 256-problem batched workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU: one process per GPU (torchrun); each rank runs an independent
replica of the single fit (the column partition of glm_slab_* is not used
here), value = all ranks' samples / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "samples/s & time-to-target-loss: CA-SGD BF16/TF32 vs FP32 SGD, one GB300"
WORKLOAD = {"m": 1 << 20, "n": 512, "flip": 0.05, "b": 64, "eta": 0.5, "lam": 0.0,
            "iters": 65536, "seed": 0, "data_seed": 0}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--s", type=int, default=8)
    ap.add_argument("--gram", default="bf16", choices=["f32", "tf32", "bf16", "f16"])
    ap.add_argument("--cluster", type=int, default=0)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-wide", action="store_true", help="skip the 400,000 x 2048 legs")
    ap.add_argument("--no-large", action="store_true", help="skip the 4,194,304 x 1024 legs")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip SGD baseline, time-to-target, e2e and CPU legs")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(base: int, rank: int) -> int:
    """Index-stream seed of replica `rank`: replicas draw independent streams."""
    return base + 1000 * rank


def batch_seed(rank: int, p: int) -> int:
    """Seed of problem p of replica `rank` in the batched workload."""
    return 1000 * (rank + 1) + p


def job_ms(ms: float, ws: int, device) -> float:
    """Whole-job time of a timed region: the maximum over ranks, one MAX
    all-reduce of a scalar (the replicas' data paths have no collective)."""
    if ws <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(ws: int, samples_per_rank: int, ms: float) -> float:
    """Whole-job throughput: every rank's samples over the slowest rank's time."""
    return ws * samples_per_rank / (ms / 1e3)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm": d["hbm_gbs"], "bf16": d["bf16_tflops"],
                "bf16_sustained": d["bf16_tflops_sustained"], "src": "measured"}
    return {"hbm": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "src": "fallback"}


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None
        self.path = None

    def start(self):
        self.p = None
        fd, self.path = tempfile.mkstemp(prefix=f".glm_clocks_rank{self.index}_", suffix=".csv",
                                         dir=ROOT)
        self.f = os.fdopen(fd, "w")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                       f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
            self.f.close()
            os.unlink(self.path)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _src_hash(*files):
    h = hashlib.sha1()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:12]


KERNEL_FILES = {"gather": "paper_2606_18463_gb300/csrc/k_gather.cu",
                "gram": "paper_2606_18463_gb300/csrc/k_gram_tc.cu",
                "gram_simt": "paper_2606_18463_gb300/csrc/k_gram_simt.cu",
                "chain": "paper_2606_18463_gb300/csrc/k_chain.cu",
                "chain_stream": "paper_2606_18463_gb300/csrc/k_chain_stream.cu"}


def _traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu capture, if it was taken on
    the current source of that kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(f"{kernel}:{workload}")
    if not e or e.get("src") != _src_hash(KERNEL_FILES[kernel], "paper_2606_18463_gb300/csrc/glm_internal.cuh"):
        return None
    return e.get("bytes_per_launch")


def _cpu_baseline(pr, w, budget_s=15.0):
    """The FP64 oracle (plain SGD == CA-SGD iterate) on the host cores, on a
    bounded sample of the same workload: the first T_s iterations, on one
    core; then the same sample on every core at once (one independent index
    stream per core, threads: the oracle's C call releases the GIL)."""
    import concurrent.futures as cf
    import oracle
    oracle.build()
    T = 256
    t0 = time.perf_counter()
    oracle.sgd(pr.A, pr.y, pr.loss, w["b"], w["eta"], w["lam"], T, w["seed"])
    dt = time.perf_counter() - t0
    Ts = int(min(w["iters"], max(T, T * budget_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    x = oracle.sgd(pr.A, pr.y, pr.loss, w["b"], w["eta"], w["lam"], Ts, w["seed"])
    dt = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    Tm = max(1, Ts // 3)   # a third of the sample per core keeps this leg ~5 s
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda k: oracle.sgd(pr.A, pr.y, pr.loss, w["b"], w["eta"], w["lam"], Tm,
                                         w["seed"] + 1 + k), range(cores)))
        dt_all = time.perf_counter() - t0
    return {"value": Ts * w["b"] / dt, "unit": "samples/s", "cores": 1, "kind": "oracle",
            "sample": f"first {Ts} of {w['iters']} iterations (b={w['b']}), FP64 SGD, "
                      "single-threaded C", "seconds": dt, "iters": Ts,
            "all_cores": {"value": cores * Tm * w["b"] / dt_all, "unit": "samples/s",
                          "cores": cores, "seconds": dt_all,
                          "sample": f"{cores} independent index streams of {Tm} iterations "
                                    "each, one per host core (os.cpu_count)"}}, x, Ts


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import synth
    w = WORKLOAD
    pr = synth.logistic_planted(w["m"], w["n"], seed=w["data_seed"], flip=w["flip"])
    per_step_budget = max(5.0, 150.0 / max(args.steps + args.warmup, 1))
    cb, _, Ts = _cpu_baseline(pr, w, budget_s=per_step_budget)
    import oracle
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.sgd(pr.A, pr.y, pr.loss, w["b"], w["eta"], w["lam"], Ts, w["seed"])
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps * Ts * w["b"] / tot
    cb["value"] = value
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(args, w), "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _config(args, w):
    return {"workload": f"logistic {w['m']}x{w['n']} FP32, N(0,1/{w['n']}), planted w*, "
                        f"5% flips; CA-SGD s={args.s} b={w['b']} eta={w['eta']} "
                        f"lambda={w['lam']} T={w['iters']}",
            "m": w["m"], "n": w["n"], "s": args.s, "b": w["b"], "eta": w["eta"],
            "lambda": w["lam"], "iters": w["iters"], "storage": "f32",
            "gram_dtype": args.gram, "recurrence": "f32", "master_weights": "f32",
            "l2": "inputs larger than L2 (A is 2 GiB, rows gathered at random)",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


E_BYTES = {"f32": 4, "tf32": 4, "bf16": 2, "f16": 2, "e4m3": 1}


def roofline(kms, kl, ms_run, T, s, b, n, e_A, gram, peaks, clocks, gram_impl=2,
             workload=None, chain_impl=1):
    """Roofline of one run: T_roof over the run (gathered bytes at HBM, Gram
    flops at the Gram type's sustained peak, the slower per outer iteration)
    against the measured run time, and the dominant kernel's own fraction
    (same per-outer-iteration units over its average CUDA-event launch time;
    the gather and the chain are held to the bytes, the Gram to its flops)."""
    from paper_2606_18463_gb300 import accounting as acc
    sm = (clocks or {}).get("sm_mhz") or 2070.0
    simt = gram == "f32" or gram_impl in (1, 3)
    p_tc = acc.gram_peak_tflops("f32" if simt else gram, peaks["bf16_sustained"], sm)
    t_roof = acc.roof_seconds(T, s, b, n, e_A, peaks["hbm"], p_tc) * 1e3
    by, fl = acc.run_bytes_flops(T, s, b, n, e_A)
    names = ["gather", "gram", "chain"]
    dom = max(range(3), key=lambda k: kms[k])
    avg_ms = kms[dom] / max(kl[dom], 1)
    frac_units = 1.0 / max(kl[dom], 1)          # share of the run one launch covers
    if names[dom] == "gram":
        p_burst = acc.gram_peak_tflops("f32" if simt else gram, peaks["bf16"], sm)
        achieved = fl * frac_units / (avg_ms / 1e3) / 1e12
        peak, unit = p_burst, "TFLOP/s"
        bound = "alu" if simt else "tensor"
        psrc = ("FP32 FMA: 152 SMs x 128 lanes x 2 flop x median SM clock" if simt else
                f"{peaks['src']} bf16 burst x {acc.TC_RATIO[gram]} ({gram} nominal ratio)")
    else:
        achieved = by * frac_units / (avg_ms / 1e3) / 1e9
        peak, unit, bound = peaks["hbm"], "GB/s", "hbm"
        psrc = f"{peaks['src']} HBM copy"
    kern = names[dom] if not (names[dom] == "gram" and simt) else "gram_simt"
    if kern == "chain" and chain_impl == 2:
        kern = "chain_stream"
    return {"kernel": kern, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "peak_source": psrc,
            "traffic": _traffic(kern, workload) if workload else None,
            "avg_launch_ms": avg_ms, "launches_per_step": kl[dom],
            "kernel_ms_per_step": {names[k]: kms[k] for k in range(3)},
            "step_T_roof_ms": t_roof, "step_T_meas_ms": ms_run, "step_frac": t_roof / ms_run,
            "step_bound": "tensor" if fl / (p_tc * 1e12) > by / (peaks["hbm"] * 1e9) else "hbm",
            "units": "per outer iteration: B_Y = s b (n e_A + 4) bytes, "
                     "F_G = b^2 s (s-1) n flops; e_A = %d" % e_A}


def time_run(stream, torch, fn, reps=2):
    """Median CUDA-event time (ms) of reps calls of fn after one warm-up."""
    fn()
    stream.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def gram_isolated(torch, glm, peaks):
    """The tcgen05 Gram alone (glm_gram_lower, BF16 operands, FP32
    accumulation) at the paper's roofline shape -- n = 16,384, b = 32, s in
    {2, 8, 16, 32, 64}, one outer step -- and at one outer step of the wide and
    the large least-squares shapes: strictly block-lower flops b^2 s (s-1) n
    over the CUDA-event time of one launch (median of 5 after a warm-up),
    against the measured BF16 burst peak.  Random N(0,1) rows, L2-resident
    operands (one outer step's rows fit in L2), as a kernel timed alone."""
    from paper_2606_18463_gb300 import accounting as acc
    out = []
    shapes = [("paper roofline shape", 1, s, 32, 16384) for s in (2, 8, 16, 32, 64)]
    shapes += [("wide, 8 outer steps", 8, 16, 128, 2048), ("large lsq, 1 outer step", 1, 64, 256, 1024)]
    for name, nouter, s, b, n in shapes:
        torch.manual_seed(0)
        Y = torch.randn(nouter * s * b, n, device="cuda").to(torch.bfloat16)
        G = torch.empty(nouter * acc.gram_lower_floats(s, b), device="cuda")
        run = lambda: glm.glm_gram_lower(Y, glm.GLM_BF16, nouter, s, b, n, n, None, G, 2)  # noqa
        run()
        ts = []
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = sorted(ts)[2]
        tf = acc.gram_flops(s, b, n) * nouter / (ms / 1e3) / 1e12
        out.append({"shape": name, "s": s, "b": b, "n": n, "nouter": nouter, "ms": ms,
                    "tflops": tf, "frac_of_bf16_burst": tf / peaks["bf16"]})
        del Y, G
    return out


def leg(ds, stream, torch, glm, peaks, clocks, *, name, s, b, eta, lam, T, seed, e_A, gram,
        n, x, reps=2, workload=None, **opts):
    """One timed configuration on an existing dataset handle."""
    o = dict(opts, gram_dtype=gram, timing=1)

    def run():
        x.zero_()
        ds.ca_sgd(x, s, b, eta, lam, T, seed, **o)
    with torch.cuda.stream(stream):
        ms = time_run(stream, torch, run, reps)
    ds.sync()
    kms, kl = glm.glm_kernel_times(ds.h)
    plan = glm.glm_ca_plan(ds.h, s, b, eta, lam, T, glm.default_ca_opts(**o))
    r = {"workload": name, "value": T * b / (ms / 1e3), "unit": "samples/s", "ms_per_run": ms,
         "s": s, "b": b, "eta": eta, "lambda": lam, "iters": T, "gram_dtype": gram,
         "recurrence": {0: "f32", 1: "f64", 2: "compensated f32"}[plan.recurrence_f64],
         "gram_impl": plan.gram_impl, "chain": {1: "resident", 2: "streaming"}[plan.chain_impl],
         "cluster": plan.cluster, "launches_per_run": plan.launches,
         "final_loss": ds.loss_value(x, lam)}
    r["roofline"] = roofline(kms, kl, ms, T, s, b, n, e_A, gram, peaks, clocks,
                             gram_impl=plan.gram_impl, chain_impl=plan.chain_impl,
                             workload=workload)
    return r


def wide_legs(args, torch, synth, glm, peaks, clocks):
    """The wide logistic workload: 400,000 x 2048, N(0,1) features times
    log-uniform column scales in [0.1, 10], lambda = 1e-3, b = 128, eta =
    2^-10 (the largest of 2^-k giving the lowest loss in an FP32 sweep at
    T = 16,384), T = 16,384; storage BF16 / FP16 with per-column scales."""
    pr = synth.logistic_wide(400_000, 2048, seed=0, lam=1e-3)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        A = torch.from_numpy(pr.A).cuda()
        y = torch.from_numpy(pr.y).cuda()
    stream.synchronize()
    ds = {"bf16": glm.Dataset(A, y, pr.loss, "bf16", fp8_copy=True, stream=stream),
          "f16": glm.Dataset(A, y, pr.loss, "f16", stream=stream)}
    del A, y
    x = torch.zeros(pr.n, dtype=torch.float32, device="cuda")
    common = dict(b=128, eta=2.0 ** -10, lam=1e-3, T=16384, seed=0, n=2048, x=x)
    out = []
    for st, gram, s, rec in [("bf16", "bf16", 16, -1), ("bf16", "e4m3", 16, -1),
                             ("bf16", "f32", 16, -1), ("f16", "f16", 16, -1),
                             ("bf16", "bf16", 32, 1), ("bf16", "bf16", 32, 2),
                             ("bf16", "bf16", 32, 0), ("bf16", "bf16", 64, 1),
                             ("bf16", "bf16", 64, 2), ("bf16", "bf16", 64, 0)]:
        r = leg(ds[st], stream, torch, glm, peaks, clocks, name=f"wide 400000x2048 {st} storage",
                s=s, e_A=2, gram=gram, recurrence_f64=rec, reps=1, **common)
        r["storage"] = st
        out.append(r)
    for d in ds.values():
        d.close()
    return out


def large_legs(args, torch, synth, glm, peaks, clocks):
    """The large least-squares workload: 4,194,304 x 1024, A ~ N(0, 1/1024)
    rounded to BF16 (the BF16 values are the data, 8 GiB), y = A x* +
    N(0, 0.01^2), lambda = 1e-5, s = 64, b = 256, BF16 Gram, T = 65,536,
    eta = 50 (as the least-squares parity case at this shape)."""
    A, y, _ = synth.lsq_bf16_device(4_194_304, 1024, seed=5)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    ds = glm.Dataset(A.view(torch.int16), y, synth.LSQ, "bf16", input_dtype="bf16",
                     stream=stream)
    del A, y
    x = torch.zeros(1024, dtype=torch.float32, device="cuda")
    out = []
    for rec in (1, 2, 0):
        r = leg(ds, stream, torch, glm, peaks, clocks, name="large lsq 4194304x1024 bf16",
                s=64, b=256, eta=50.0, lam=1e-5, T=65536, seed=0, e_A=2, gram="bf16", n=1024,
                x=x, recurrence_f64=rec, reps=1)
        out.append(r)
    ds.close()
    return out


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import synth
    from paper_2606_18463_gb300 import accounting as acc
    from paper_2606_18463_gb300 import glm
    glm.load()

    w = dict(WORKLOAD)
    s, b, T = args.s, w["b"], w["iters"]
    pr = synth.logistic_planted(w["m"], w["n"], seed=w["data_seed"], flip=w["flip"])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        A = torch.from_numpy(pr.A).cuda()
        y = torch.from_numpy(pr.y).cuda()
    stream.synchronize()
    ds = glm.Dataset(A, y, pr.loss, "f32", stream=stream)
    del A, y
    x = torch.zeros(pr.n, dtype=torch.float32, device="cuda")
    opts = dict(gram_dtype=args.gram, cluster=args.cluster, timing=1)
    seed = replica_seed(w["seed"], rank)
    plan = glm.glm_ca_plan(ds.h, s, b, w["eta"], w["lam"], T, glm.default_ca_opts(**opts))

    def step():
        x.zero_()
        ds.ca_sgd(x, s, b, w["eta"], w["lam"], T, seed, **opts)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        stream.synchronize()
        ds.sync()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = Clocks(local)
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        stream.synchronize()
        clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ds.sync()
    kms, kl = glm.glm_kernel_times(ds.h)   # last step's per-kernel event times
    ms = job_ms(ms, ws, "cuda")
    value = job_value(ws, T * b, ms)

    # ---- roofline (run and dominant kernel) -------------------------------
    peaks = _peaks()
    roof = roofline(kms, kl, ms, T, s, b, w["n"], 4, args.gram, peaks, clocks,
                    gram_impl=plan.gram_impl, workload="c2")

    out = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": args.gram, "data": "synthetic", "config": _config(args, w),
           "roofline": roof, "gpu_launches": int(plan.launches) * args.steps,
           "clocks": clocks,
           "plan": {"chunk_outer": plan.chunk_outer, "chunks": plan.chunks,
                    "cluster": plan.cluster, "gram_impl": plan.gram_impl}}

    if not args.no_extras:
        # ---- the other s of the workload, one timed run each ------------------
        sweep = {}
        with torch.cuda.stream(stream):
            for s2 in (8, 16, 32):
                o2 = dict(opts, timing=0)

                def run2():
                    x.zero_()
                    ds.ca_sgd(x, s2, b, w["eta"], w["lam"], T, seed, **o2)
                run2()
                stream.synchronize()
                g0 = torch.cuda.Event(enable_timing=True)
                g1 = torch.cuda.Event(enable_timing=True)
                g0.record(stream)
                run2()
                g1.record(stream)
                stream.synchronize()
                ms2 = g0.elapsed_time(g1)
                sweep[f"s={s2}"] = {"samples_per_s": T * b / (ms2 / 1e3), "ms_per_run": ms2,
                                    "recurrence": "f64" if s2 >= 32 else "f32"}
        out["s_sweep"] = sweep

        # ---- TF32 and FP32 Grams of the headline workload ---------------------
        xg = torch.zeros(pr.n, dtype=torch.float32, device="cuda")
        out["gram_legs"] = [
            leg(ds, stream, torch, glm, peaks, clocks, name="c2 " + g, s=s, b=b, eta=w["eta"],
                lam=w["lam"], T=T, seed=seed, e_A=4, gram=g, n=w["n"], x=xg,
                cluster=args.cluster)
            for g in ("tf32", "f32")]

        # ---- FP32 plain-SGD GPU baseline (same data, same index stream) -------
        with torch.cuda.stream(stream):
            xs = torch.zeros(pr.n, dtype=torch.float32, device="cuda")

            def sgd_step():
                xs.zero_()
                ds.sgd(xs, b, w["eta"], w["lam"], T, seed)
            sgd_step()
            stream.synchronize()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(2):
                sgd_step()
            f1.record(stream)
            stream.synchronize()
        sgd_ms = f0.elapsed_time(f1) / 2
        out["sgd_fp32"] = {"value": T * b / (sgd_ms / 1e3), "unit": "samples/s",
                           "ms_per_run": sgd_ms, "speedup_ca_over_sgd": sgd_ms / ms}

        # ---- end to end through the public API with host buffers --------------
        x0h = torch.zeros(pr.n, dtype=torch.float32).pin_memory()
        xTh = torch.empty(pr.n, dtype=torch.float32).pin_memory()
        xd = torch.empty(pr.n, dtype=torch.float32, device="cuda")
        with torch.cuda.stream(stream):
            def e2e_step():
                xd.copy_(x0h, non_blocking=True)
                ds.ca_sgd(xd, s, b, w["eta"], w["lam"], T, seed, **opts)
                xTh.copy_(xd, non_blocking=True)
                return ds.loss_value(xd, w["lam"])   # blocks: reads the loss on the host
            e2e_step()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                loss_e2e = e2e_step()
            dt = time.perf_counter() - t0
        out["e2e"] = {"value": ws * T * b * args.steps / dt, "unit": "samples/s",
                      "h2d_bytes_per_step": 4 * pr.n, "d2h_bytes_per_step": 4 * pr.n + 8,
                      "includes": "x0 H2D, run, x_T D2H, full-data loss D2H; the "
                                  "one-time dataset upload (glm_create) is excluded",
                      "final_loss": loss_e2e}

        if rank == 0:
            # ---- CPU oracle baseline + target loss --------------------------------
            cb, x_or, Ts = _cpu_baseline(pr, w)
            out["cpu_baseline"] = cb
            # time to target: (1 + 1e-3) x the oracle's loss after the same
            # number of iterations it managed in the sample, measured on the GPU
            # in segments (loss evaluation excluded from the training time)
            import oracle
            f_or = oracle.loss(pr.A, pr.y, pr.loss, w["lam"], x_or)
            target = (1 + 1e-3) * f_or
            out["time_to_target"] = _ttt(ds, pr, w, s, b, seed, target, Ts, opts, stream,
                                         torch, glm)
            out["time_to_target"].update({"target_loss": target, "oracle_loss": f_or,
                                          "oracle_iters": Ts})
    ds.close()
    del pr
    if not args.no_extras and ws == 1:
        if not args.no_wide:
            out["wide"] = wide_legs(args, torch, synth, glm, peaks, clocks)
        if not args.no_large:
            out["large"] = large_legs(args, torch, synth, glm, peaks, clocks)
    if not args.no_extras and ws == 1:
        out["gram_isolated"] = gram_isolated(torch, glm, peaks)
    if not args.no_extras and not args.no_batch:
        out["batched"] = _batched(args, torch, synth, glm, rank, peaks)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


BATCH = {"P": 256, "b": 64, "iters": 4096, "eta": 0.25, "data_seed": 0}


def _batched(args, torch, synth, glm, rank, peaks):
    """The batched workload: 256 independent fits in one run (gather, grouped
    Gram and a persistent work-queue chain per round; all rounds one CUDA
    graph); m log-uniform in [4096, 131072], n cycling 64..1024, lambda on
    10^(-6 + 5 p / 255), even p logistic, odd p least squares; BF16 storage
    with per-column scales; s chosen by the library's autotuner."""
    cfg = dict(BATCH)
    probs = []
    for sp in synth.batch_specs(P=cfg["P"], seed=cfg["data_seed"]):
        pr = synth.batch_problem(sp, seed=cfg["data_seed"])
        probs.append(dict(A=pr.A, y=pr.y, loss=sp["loss"], lam=sp["lam"], eta=cfg["eta"],
                          iters=cfg["iters"], seed=batch_seed(rank, sp["p"]), b=cfg["b"],
                          s=0))
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    bt = glm.Batch(probs, dtype="bf16", stream=stream)
    t_create = time.perf_counter() - t0
    xs = [torch.zeros(p["A"].shape[1], dtype=torch.float32, device="cuda") for p in probs]
    samples = cfg["P"] * cfg["iters"] * cfg["b"]
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 1)):
            for x in xs:
                x.zero_()
            bt.run(xs)
        times = []
        for _ in range(max(args.steps, 1)):
            for x in xs:
                x.zero_()
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            status = bt.run(xs)
            e1.record(stream)
            stream.synchronize()
            times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    choice = {}
    for p, pr in enumerate(probs):
        n = int(pr["A"].shape[1])
        choice.setdefault(str(n), {})
        sp = str(bt.choice(p)[0])
        choice[str(n)][sp] = choice[str(n)].get(sp, 0) + 1
    losses = bt.loss(xs)
    # roofline of the whole batch: every problem's gathered bytes (BF16
    # storage) and strictly block-lower Gram flops at its chosen s; the
    # problems share the GPU, so the bound is the slower of the two totals
    from paper_2606_18463_gb300 import accounting as acc
    tby = tfl = 0
    for p, pr in enumerate(probs):
        sp = bt.choice(p)[0]
        by, fl = acc.run_bytes_flops(cfg["iters"], sp, cfg["b"], int(pr["A"].shape[1]), 2)
        tby += by
        tfl += fl
    t_roof = max(tby / (peaks["hbm"] * 1e9), tfl / (peaks["bf16_sustained"] * 1e12)) * 1e3
    bt.close()
    return {"value": samples / (ms / 1e3), "unit": "samples/s", "ms_per_run": ms,
            "roofline": {"step_T_roof_ms": t_roof, "step_T_meas_ms": ms,
                         "step_frac": t_roof / ms, "gathered_bytes": tby, "gram_flops": tfl,
                         "bound": "hbm" if tby / (peaks["hbm"] * 1e9) >=
                         tfl / (peaks["bf16_sustained"] * 1e12) else "tensor"},
            "problems": cfg["P"], "rows_total": int(sum(p["A"].shape[0] for p in probs)),
            "iters_per_problem": cfg["iters"], "b": cfg["b"], "storage": "bf16",
            "autotuned_s_by_n": choice, "create_and_tune_s": t_create,
            "nonfinite": int(sum(1 for s_ in status if s_)),
            "median_final_loss": float(statistics.median(losses))}


def _ttt(ds, pr, w, s, b, seed, target, horizon, opts, stream, torch, glm):
    """Training time until the full-data loss reaches `target` (segments of
    horizon/16 iterations; loss evaluated between segments, not timed)."""
    res = {}
    seg = max(s, (horizon // 16) // s * s)
    for name in ("ca", "sgd"):
        x = torch.zeros(pr.n, dtype=torch.float32, device="cuda")
        done, train_ms, reached = 0, 0.0, None
        with torch.cuda.stream(stream):
            while done < 4 * horizon:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                o = dict(opts, first_iter=done, use_graph=0, timing=0)
                e0.record(stream)
                if name == "ca":
                    ds.ca_sgd(x, s, b, w["eta"], w["lam"], seg, seed, **o)
                else:
                    ds.sgd(x, b, w["eta"], w["lam"], seg, seed, first_iter=done, use_graph=0)
                e1.record(stream)
                stream.synchronize()
                train_ms += e0.elapsed_time(e1)
                done += seg
                if ds.loss_value(x, w["lam"]) <= target:
                    reached = done
                    break
        res[name] = {"seconds": train_ms / 1e3 if reached else None,
                     "iters": reached, "segment": seg}
    return res


if __name__ == "__main__":
    main()
