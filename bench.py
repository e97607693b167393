"""Benchmark: CA-SGD samples/s on one GB300 (and N independent replicas).

Workload (default): binary logistic regression, dense A 1,048,576 x 512 FP32
with entries N(0, 1/512), planted w*, 5% label flips; CA-SGD with s = 8,
b = 64, eta = 0.5, lambda = 0, 65,536 SGD-equivalent iterations; Gram, margin
and gradient operands in BF16 with FP32 accumulation, FP32 recurrence and
master weights.  One bench step = one full training run (x reset to 0, then
65,536 iterations through the C ABI, replayed as a CUDA graph).

Printed: one JSON line (rank 0) with the whole-job samples/s, the
end-to-end number through the public API with host buffers, the roofline of
the dominant kernel, the FP32 plain-SGD GPU baseline, the CPU oracle and, as
an extra object, the batched workload (256 independent logistic / least-
squares fits of uneven m, n and lambda, BF16 storage, autotuned s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU: one process per GPU (torchrun); each rank runs an independent
replica (the single-fit path is not sharded on this build), value = all
ranks' samples / max-over-ranks time.
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
                "chain": "paper_2606_18463_gb300/csrc/k_chain.cu"}


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
    bounded sample of the same workload: the first T_s iterations."""
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
    return {"value": Ts * w["b"] / dt, "unit": "samples/s", "cores": 1, "kind": "oracle",
            "sample": f"first {Ts} of {w['iters']} iterations (b={w['b']}), FP64 SGD, "
                      "single-threaded C", "seconds": dt, "iters": Ts}, x, Ts


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

    # ---- roofline of the dominant kernel ------------------------------------
    peaks = _peaks()
    names = ["gather", "gram", "chain"]
    dom = max(range(3), key=lambda k: kms[k])
    avg_ms = kms[dom] / max(kl[dom], 1)
    H = (T + s - 1) // s
    per_launch_outer = H / max(kl[dom], 1)
    e_op = {"f32": 4, "tf32": 4, "bf16": 2, "f16": 2}[args.gram]
    if names[dom] == "gram":
        flops = acc.gram_flops(s, b, w["n"]) * per_launch_outer
        achieved = flops / (avg_ms / 1e3) / 1e12
        if args.gram == "f32":
            peak, unit, bound = 152 * 128 * 2 * 2.07e9 / 1e12, "TFLOP/s", "alu"
            psrc = "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"
        else:
            ratio = 0.5 if args.gram == "tf32" else 1.0
            peak, unit, bound = peaks["bf16"] * ratio, "TFLOP/s", "tensor"
            psrc = f"{peaks['src']} bf16 burst" + (" x 0.5 (tf32 nominal ratio)" if ratio < 1 else "")
    else:
        if names[dom] == "gather":
            byts = (acc.gathered_bytes(s, b, w["n"], 4) + acc.staged_bytes(s, b, w["n"], e_op)) * per_launch_outer
        else:
            byts = acc.chain_bytes(s, b, w["n"], e_op) * per_launch_outer
        achieved = byts / (avg_ms / 1e3) / 1e9
        peak, unit, bound = peaks["hbm"], "GB/s", "hbm"
        psrc = f"{peaks['src']} HBM copy"
    roof = {"kernel": names[dom], "bound": bound, "achieved": achieved, "peak": peak,
            "unit": unit, "frac": achieved / peak, "peak_source": psrc,
            "traffic": _traffic(names[dom] if not (names[dom] == "gram" and plan.gram_impl == 1)
                                else "gram_simt", "c2"),
            "avg_launch_ms": avg_ms, "launches_per_step": kl[dom],
            "kernel_ms_per_step": {names[k]: kms[k] for k in range(3)}}

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
                      "includes": "x0 H2D, run, x_T D2H, full-data loss D2H",
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
    if not args.no_extras and not args.no_batch:
        out["batched"] = _batched(args, torch, synth, glm, rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


BATCH = {"P": 256, "b": 64, "iters": 4096, "eta": 0.25, "data_seed": 0}


def _batched(args, torch, synth, glm, rank):
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
    bt.close()
    return {"value": samples / (ms / 1e3), "unit": "samples/s", "ms_per_run": ms,
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
