"""Theorem 1 (Sec. 5.2) as an invariant of the GPU path: one CA-SGD outer step
of each precision mode, run through the C ABI from a mid-training FP32
iterate, stays within the theorem's first-order local error budget (times 2,
standing for the unspecified 1 + C_loc Omega) of the exact FP64 outer step
over the same sampled rows, and the theorem's hypotheses omega, tau_G <= 1/2
hold.

Data: 65,536 x 512 planted logistic (5 % label flips) and least-squares
problems with rows scaled to norm at most 1 (Assumption 1); b = 64,
eta = 0.5 (alpha = 2^-7, exact), lambda = 0; the start iterate is the FP64
oracle's after 4,096 SGD iterations, rounded to FP32, and the measured step
draws the stream's next s b indices.

Slots of the library's kernels on one GPU (no all-reduce terms):
  u_A      0 for FP32 storage (the data are the FP32 values), 2^-8 for BF16
           storage (power-of-two column scales keep the relative error).
  gamma_r, gamma_G, gamma_g
           2 u_in + gamma_q(2^-24) with q = n for the margin and the Gram and
           q = s b for the gradient; u_in is the operand rounding (0 for FP32
           operands, 2^-11 TF32 and FP16, 2^-8 BF16), FP32 accumulation.  The
           FP16-accumulate Gram (Recipe F's Gram slot) has gamma_G =
           2 u_in + gamma_n(2^-11).
  u_c      2^-24 for the FP32 recurrence, 2^-53 for the FP64 one.
  u_sigma  2^-24.  C_delta: logistic 10 + 2.35 M, M the largest |y z| of the
           step, from the documented error bounds of the fast exponential
           (2 + 1.173 |t| ulp) and fast division (2 ulp) plus three FP32
           roundings (the IEEE form of the FP64 recurrence, with its FP32
           margin, stays below this); least squares 2 (the FP32 subtraction
           and, in FP64, the margin's rounding to FP32).
  u_x      2^-24 (the FP32 master weights; the update is Kahan-compensated).

One configuration lies outside the theorem: least squares with the
FP16-accumulate Gram.  The least-squares slope L_sigma = 1 and gamma_G of
about 1/3 (FP16 accumulation over n = 512) give tau_G = 0.53 > 1/2, so the
theorem's hypothesis rules it out (the paper's Recipe F accumulates n_loc = 256
per rank).  That case checks that the hypothesis does fail, and reports its
deviation.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import local_error as le

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M, N, B, ETA, K0, SEED = 65536, 512, 64, 0.5, 4096, 5
U32, U64 = 2.0 ** -24, 2.0 ** -53
U_IN = {"f32": 0.0, "tf32": 2.0 ** -11, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}

# (storage, Gram and GEMV operands, s, FP64 recurrence, Gram implementation:
# 0 automatic, 3 FP16 accumulation (SIMT), 4 FP16 accumulation (tcgen05))
MODES = [("f32", "f32", 8, 0, 0), ("f32", "tf32", 8, 0, 0), ("f32", "bf16", 8, 0, 0),
         ("f32", "f16", 8, 0, 0), ("bf16", "bf16", 8, 0, 0), ("f32", "f32", 32, 1, 0),
         ("f32", "bf16", 32, 1, 0), ("f32", "f32", 16, 0, 0),
         pytest.param("f32", "f16", 8, 0, 3, id="f16acc"),
         pytest.param("f32", "f16", 8, 0, 4, id="f16acc-tc")]

# (loss, Gram implementation) the theorem's hypotheses exclude at this shape
EXCLUDED = {("lsq", 3), ("lsq", 4)}


@pytest.fixture(scope="module")
def G():
    from paper_2606_18463_gb300 import glm
    glm.load()
    return glm


def _normalized(pr):
    A = pr.A.astype(np.float64)
    A /= np.maximum(1.0, np.linalg.norm(A, axis=1, keepdims=True))
    return A.astype(np.float32)


@pytest.fixture(scope="module", params=["logistic", "lsq"])
def case(request, G):
    if request.param == "logistic":
        pr = synth.logistic_planted(M, N, seed=21, flip=0.05)
    else:
        pr = synth.lsq_planted(M, N, seed=22, noise=0.1)
    A = _normalized(pr)
    x0 = oracle.sgd(A, pr.y, pr.loss, B, ETA, 0.0, K0, SEED).astype(np.float32)
    dev = {}
    At, yt = torch.from_numpy(A).cuda(), torch.from_numpy(pr.y).cuda()
    ds = {st: G.Dataset(At, yt, pr.loss, st) for st in ("f32", "bf16")}
    del At, yt
    yield request.param, pr.loss, A, pr.y, x0, ds, dev
    for d in ds.values():
        d.close()
    print(f"{request.param}: deviations {dev}")


@pytest.mark.parametrize("storage,op,s,rec,impl", MODES)
def test_one_outer_step_within_theorem_budget(case, storage, op, s, rec, impl):
    name, loss, A, y, x0, ds, devs = case
    x = torch.from_numpy(x0.copy()).cuda()
    ds[storage].ca_sgd(x, s, B, ETA, 0.0, s, SEED, first_iter=K0, gram_dtype=op,
                       recurrence_f64=rec, gram_impl=impl)
    ds[storage].sync()
    xg = x.cpu().numpy().astype(np.float64)

    idx = oracle.sample_indices(SEED, 0, K0 * B, s * B, M)
    Y = A[idx].astype(np.float64)
    yI = y[idx].astype(np.float64)
    z, _, _ = le.exact_step(Y, yI, x0.astype(np.float64), loss, ETA, s, B)
    if loss == le.LOGISTIC:
        C_delta = 10.0 + 2.35 * float(np.max(np.abs(yI * z)))
    else:
        C_delta = 2.0
    u_in = U_IN[op]
    ev = le.local_error(Y, yI, x0.astype(np.float64), loss, ETA, s, B,
                        u_A=2.0 ** -8 if storage == "bf16" else 0.0,
                        gamma_r=le.gamma_mixed(N, u_in, U32),
                        gamma_G=le.gamma_mixed(N, u_in, 2.0 ** -11 if impl in (3, 4) else U32),
                        u_c=U64 if rec else U32, u_sigma=U32,
                        gamma_g=le.gamma_mixed(s * B, u_in, U32), u_x=U32,
                        C_delta=C_delta)
    hyp = ev["omega"] <= 0.5 and ev["tau_G"] <= 0.5
    dev = float(np.linalg.norm(xg - ev["x_s"]))
    devs[(storage, op, s, impl)] = dev
    print(f"{name} storage={storage} op={op} s={s} rec64={rec} impl={impl}: "
          f"|x_gpu - x_s| = {dev:.3e}, "
          f"sum E = {ev['sum']:.3e} (ratio {dev / ev['sum']:.3e}), K_s = {ev['K_s']:.4f}, "
          f"Omega = {ev['Omega']:.2e}, tau_G = {ev['tau_G']:.2e}, "
          f"|x_s| = {np.linalg.norm(ev['x_s']):.3f}")
    if (name, impl) in EXCLUDED:
        assert not hyp and np.isfinite(dev), (ev["omega"], ev["tau_G"], dev)
        return
    assert hyp, (ev["omega"], ev["tau_G"])
    assert 0.0 < dev <= 2.0 * ev["sum"], (dev, ev["sum"])
