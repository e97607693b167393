"""Seeded synthetic GLM inputs, shared by the oracle-side tests and the CUDA-side
tests and benchmark.

This module holds data recipes only (planted models, label noise, feature
scales); none of the arithmetic of SGD / CA-SGD lives here.  Every array is a
deterministic function of its arguments (numpy PCG64 streams), so both sides
consume identical bytes.

The paper's own datasets (synth 1e6 x 9984, epsilon, SUSY, HIGGS; Table
"datasets" in Sec. 7.1) are not available; the recipes below stand in for
them with the shapes and distributions of the workloads this library is
measured on:

  logistic_planted  dense N(0, 1/n) features, planted w* ~ N(0, I), labels
                    +-1 drawn from sigmoid(a_i^T w*), optional label flips.
  logistic_wide     N(0,1) features times log-uniform column scales in
                    [0.1, 10] (an epsilon-shaped 400000 x 2048 stand-in).
  lsq_planted       dense N(0, var) features, y = A x* + N(0, noise^2).
  lsq_bf16          as lsq_planted but the BF16-rounded values are the data.
  lsq_bf16_device   the same recipe drawn with torch's CUDA generator, for
                    sizes (4,194,304 x 1024) that a host generator makes slow;
                    its bytes differ from lsq_bf16's (another stream).
  batch_problems    the 256-problem batch: log-uniform m, cycling n, lambda
                    on a log grid, alternating logistic / least squares.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LOGISTIC, LSQ, POISSON = 0, 1, 2


@dataclass
class Problem:
    A: np.ndarray          # float32, row-major m x n
    y: np.ndarray          # float32, m
    loss: int              # LOGISTIC or LSQ
    lam: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]


def _normal_f32(rng, shape, std, chunk_rows=1 << 16):
    """N(0, std^2) float32 matrix, generated in row chunks to bound memory."""
    m, n = shape
    out = np.empty((m, n), dtype=np.float32)
    for i in range(0, m, chunk_rows):
        blk = rng.standard_normal((min(chunk_rows, m - i), n), dtype=np.float32)
        blk *= np.float32(std)
        out[i:i + blk.shape[0]] = blk
    return out


def _planted_labels(rng, A, w, chunk_rows=1 << 16):
    m = A.shape[0]
    y = np.empty(m, dtype=np.float32)
    for i in range(0, m, chunk_rows):
        t = A[i:i + chunk_rows].astype(np.float64) @ w
        p = 1.0 / (1.0 + np.exp(-t))
        U = rng.random(t.shape[0])
        y[i:i + chunk_rows] = np.where(U < p, 1.0, -1.0)
    return y


def logistic_planted(m: int, n: int, seed: int = 0, flip: float = 0.0,
                     lam: float = 0.0) -> Problem:
    """A_ij ~ N(0, 1/n), w* ~ N(0, I_n), y_i = +1 w.p. sigmoid(a_i^T w*),
    then each label flipped independently with probability `flip`."""
    rng = np.random.default_rng([seed, 101, m, n])
    A = _normal_f32(rng, (m, n), 1.0 / math.sqrt(n))
    w = rng.standard_normal(n)
    y = _planted_labels(rng, A, w)
    if flip > 0:
        y[rng.random(m) < flip] *= -1.0
    return Problem(A, y, LOGISTIC, lam, {"recipe": "logistic_planted",
                                          "seed": seed, "flip": flip})


def logistic_wide(m: int, n: int, seed: int = 0, lam: float = 0.0,
                  kappa_lo: float = 0.1, kappa_hi: float = 10.0) -> Problem:
    """A_ij = N(0,1) * kappa_j with kappa_j log-uniform in [kappa_lo, kappa_hi];
    planted w*_j ~ N(0,1) / (kappa_j sqrt(n)) so margins are O(1)."""
    rng = np.random.default_rng([seed, 202, m, n])
    kappa = np.exp(rng.uniform(math.log(kappa_lo), math.log(kappa_hi), n))
    A = _normal_f32(rng, (m, n), 1.0)
    A *= kappa.astype(np.float32)[None, :]
    w = rng.standard_normal(n) / (kappa * math.sqrt(n))
    y = _planted_labels(rng, A, w)
    return Problem(A, y, LOGISTIC, lam, {"recipe": "logistic_wide",
                                          "seed": seed, "kappa": kappa})


def lsq_planted(m: int, n: int, seed: int = 0, noise: float = 0.1,
                lam: float = 0.0, var: float | None = None) -> Problem:
    """A_ij ~ N(0, var) (default 1/n), x* ~ N(0, I), y = A x* + N(0, noise^2)."""
    rng = np.random.default_rng([seed, 303, m, n])
    std = math.sqrt(var) if var is not None else 1.0 / math.sqrt(n)
    A = _normal_f32(rng, (m, n), std)
    xs = rng.standard_normal(n)
    y = np.empty(m, dtype=np.float32)
    for i in range(0, m, 1 << 16):
        blk = A[i:i + (1 << 16)].astype(np.float64) @ xs
        y[i:i + blk.shape[0]] = blk + noise * rng.standard_normal(blk.shape[0])
    return Problem(A, y, LSQ, lam, {"recipe": "lsq_planted", "seed": seed,
                                     "noise": noise, "x_star": xs})


def poisson_planted(m: int, n: int, seed: int = 0, scale: float = 0.5,
                    lam: float = 0.0) -> Problem:
    """Poisson regression with the log link: A_ij ~ N(0, 1/n), x*_j ~ N(0, scale^2),
    y_i ~ Poisson(exp(a_i^T x*)) as float32 counts (margins are O(scale))."""
    rng = np.random.default_rng([seed, 404, m, n])
    A = _normal_f32(rng, (m, n), 1.0 / math.sqrt(n))
    w = rng.normal(0.0, scale, n)
    r = np.zeros(m)
    for i in range(0, m, 1 << 16):
        r[i:i + (1 << 16)] = A[i:i + (1 << 16)].astype(np.float64) @ w
    y = rng.poisson(np.exp(r)).astype(np.float32)
    return Problem(A=A, y=y, loss=POISSON, lam=lam, meta={"w_star": w})


def to_bf16_values(A: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest BF16 value (ties to even); the
    result is float32 holding exactly-representable BF16 values."""
    u = A.view(np.uint32)
    out = np.empty_like(A)
    ov = out.view(np.uint32)
    step = 1 << 20
    flat_u = u.reshape(-1)
    flat_o = ov.reshape(-1)
    for i in range(0, flat_u.size, step):
        x = flat_u[i:i + step].astype(np.uint64)
        x = ((x + 0x7FFF + ((x >> 16) & 1)) >> 16) << 16
        flat_o[i:i + step] = (x & 0xFFFFFFFF).astype(np.uint32)
    return out


def lsq_bf16(m: int, n: int, seed: int = 0, noise: float = 0.01,
             lam: float = 0.0) -> Problem:
    """Least squares whose data ARE BF16 values: A_ij ~ N(0, 1/n) rounded to
    BF16 (kept as float32 holding BF16 values), y = A x* + N(0, noise^2)."""
    rng = np.random.default_rng([seed, 404, m, n])
    A = to_bf16_values(_normal_f32(rng, (m, n), 1.0 / math.sqrt(n)))
    xs = rng.standard_normal(n)
    y = np.empty(m, dtype=np.float32)
    for i in range(0, m, 1 << 16):
        blk = A[i:i + (1 << 16)].astype(np.float64) @ xs
        y[i:i + blk.shape[0]] = blk + noise * rng.standard_normal(blk.shape[0])
    return Problem(A, y, LSQ, lam, {"recipe": "lsq_bf16", "seed": seed,
                                     "noise": noise, "x_star": xs})


def batch_specs(P: int = 256, seed: int = 0, m_lo: int = 4096,
                m_hi: int = 131072, ns=(64, 128, 256, 512, 1024)):
    """Shapes of the batched workload: m_p = floor(exp(U[ln m_lo, ln m_hi])),
    n_p cycling through `ns`, lambda_p = 10^(-6 + 5 p / (P-1)), even p
    logistic, odd p least squares."""
    rng = np.random.default_rng([seed, 505, P])
    specs = []
    for p in range(P):
        m = int(math.floor(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        n = int(ns[p % len(ns)])
        lam = 10.0 ** (-6.0 + 5.0 * p / max(P - 1, 1))
        specs.append({"p": p, "m": m, "n": n, "lam": lam,
                      "loss": LOGISTIC if p % 2 == 0 else LSQ})
    return specs


def batch_problem(spec: dict, seed: int = 0) -> Problem:
    if spec["loss"] == LOGISTIC:
        pr = logistic_planted(spec["m"], spec["n"], seed=seed * 1000 + spec["p"],
                              lam=spec["lam"])
    else:
        pr = lsq_planted(spec["m"], spec["n"], seed=seed * 1000 + spec["p"],
                         noise=0.1, lam=spec["lam"])
    pr.meta["spec"] = spec
    return pr


def ragged(m: int, n: int, seed: int = 0, loss: int = LOGISTIC,
           lam: float = 0.0) -> Problem:
    """Small odd-shaped problem for edge-case tests."""
    if loss == LOGISTIC:
        return logistic_planted(m, n, seed=seed, lam=lam)
    return lsq_planted(m, n, seed=seed, lam=lam)


def lsq_bf16_device(m: int, n: int, seed: int = 0, noise: float = 0.01,
                    chunk_rows: int = 1 << 18):
    """Least squares whose data ARE BF16 values, drawn on the current CUDA
    device: A_ij ~ N(0, 1/n) rounded to BF16, x* ~ N(0, I) (numpy PCG64),
    y = A x* + N(0, noise^2) (FP64 products of the BF16 values, stored FP32).
    Returns (A as a CUDA bfloat16 tensor, y as a CUDA float32 tensor, x*)."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(int(np.random.default_rng([seed, 606, m, n]).integers(1 << 62)))
    xs = np.random.default_rng([seed, 607, m, n]).standard_normal(n)
    xd = torch.from_numpy(xs).cuda()
    A = torch.empty((m, n), dtype=torch.bfloat16, device="cuda")
    y = torch.empty(m, dtype=torch.float32, device="cuda")
    for i in range(0, m, chunk_rows):
        r = min(chunk_rows, m - i)
        blk = torch.randn((r, n), generator=g, device="cuda", dtype=torch.float32)
        blk.mul_(1.0 / math.sqrt(n))
        A[i:i + r] = blk.to(torch.bfloat16)
        e = torch.randn(r, generator=g, device="cuda", dtype=torch.float64)
        y[i:i + r] = (A[i:i + r].double() @ xd + noise * e).float()
    return A, y, xs
