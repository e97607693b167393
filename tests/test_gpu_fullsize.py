"""Parity at the full sizes the bench times, in its launch configuration.

c2: logistic 1,048,576 x 512 (FP32 storage, N(0,1/512), planted w*, 5% label
flips), b = 64, eta = 0.5, lambda = 0, 65,536 iterations, seed 0, through the
C ABI with the library's default cluster and chunking.  The FP64 oracle runs
the same index stream (plain SGD: CA-SGD equals SGD in exact arithmetic).
  * FP32 operands and Gram (s = 8): iterate relative error <= 1e-5.
  * BF16 Gram and GEMV operands (the bench's configuration, s = 8) and the
    FP64 recurrence (s = 32): final risk within 1e-3 of the oracle's.
Batched: the bench's 256-problem workload (BF16 storage, autotuned s); a
sample of problems against the oracle on their own streams (key (seed_p, p)),
final risk within 1e-3.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M, N, B, ETA, T, SEED = 1 << 20, 512, 64, 0.5, 65536, 0


@pytest.fixture(scope="module")
def G():
    from paper_2606_18463_gb300 import glm
    glm.load()
    return glm


@pytest.fixture(scope="module")
def c2():
    return synth.logistic_planted(M, N, seed=0, flip=0.05)


@pytest.fixture(scope="module")
def c2_ref(c2):
    return oracle.sgd(c2.A, c2.y, c2.loss, B, ETA, 0.0, T, SEED)


@pytest.fixture(scope="module")
def c2_ds(G, c2):
    ds = G.Dataset(torch.from_numpy(c2.A).cuda(), torch.from_numpy(c2.y).cuda(), c2.loss,
                   "f32")
    yield ds
    ds.close()


def _run(ds, s, **opts):
    x = torch.zeros(N, dtype=torch.float32, device="cuda")
    ds.ca_sgd(x, s, B, ETA, 0.0, T, SEED, **opts)
    ds.sync()
    return x.cpu().numpy().astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_c2_fp32_iterate(c2_ds, c2_ref):
    x = _run(c2_ds, 8, gram_dtype="f32")
    assert _rel(x, c2_ref) <= 1e-5, _rel(x, c2_ref)


@pytest.mark.parametrize("s", [8, 32])
def test_c2_bf16_final_risk(c2, c2_ds, c2_ref, s):
    x = _run(c2_ds, s, gram_dtype="bf16")
    f = oracle.loss(c2.A, c2.y, c2.loss, 0.0, x)
    fr = oracle.loss(c2.A, c2.y, c2.loss, 0.0, c2_ref)
    assert abs(f - fr) <= 1e-3 * fr, (s, f, fr)


def test_c2_plain_sgd_and_one_launch_per_chunk(G, c2_ds, c2_ref):
    x = torch.zeros(N, dtype=torch.float32, device="cuda")
    c2_ds.sgd(x, B, ETA, 0.0, T, SEED)
    c2_ds.sync()
    assert _rel(x.cpu().numpy().astype(np.float64), c2_ref) <= 1e-5
    # the same CA-SGD run without graph capture (launch by launch)
    xg = _run(c2_ds, 8, gram_dtype="f32", use_graph=0)
    assert _rel(xg, c2_ref) <= 1e-5


def test_batched_workload_sampled(G):
    P, b, iters, eta = 256, 64, 4096, 0.25
    specs = synth.batch_specs(P=P, seed=0)
    probs, prs = [], []
    for sp in specs:
        pr = synth.batch_problem(sp, seed=0)
        prs.append(pr)
        probs.append(dict(A=pr.A, y=pr.y, loss=sp["loss"], lam=sp["lam"], eta=eta,
                          iters=iters, seed=1000 + sp["p"], b=b, s=0))
    bt = G.Batch(probs, dtype="bf16")
    try:
        xs = [torch.zeros(p["A"].shape[1], dtype=torch.float32, device="cuda") for p in probs]
        st = bt.run(xs)
        assert st == [G.GLM_OK] * P
        # every shape class and both losses: the first ten problems, the largest
        # and the smallest
        ms = [p["A"].shape[0] for p in probs]
        sample = sorted(set(list(range(10)) + [int(np.argmax(ms)), int(np.argmin(ms))]))
        for p in sample:
            sp = specs[p]
            ref = oracle.sgd(prs[p].A, prs[p].y, sp["loss"], b, eta, sp["lam"], iters,
                             1000 + p, problem=p)
            x = xs[p].cpu().numpy().astype(np.float64)
            f = oracle.loss(prs[p].A, prs[p].y, sp["loss"], sp["lam"], x)
            fr = oracle.loss(prs[p].A, prs[p].y, sp["loss"], sp["lam"], ref)
            assert abs(f - fr) <= 1e-3 * fr, (p, f, fr)
    finally:
        bt.close()
