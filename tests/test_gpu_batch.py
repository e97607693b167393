"""Batched fits (glm_batch_*) through the C ABI against the FP64 oracle.

Problem p of a batch draws from Philox key (seed_p, p), so its oracle is
plain FP64 SGD on that stream (CA-SGD equals SGD in exact arithmetic).
Tolerances as for single problems: FP32 storage and Gram, iterate relative
error <= 1e-5; BF16 storage, final risk within 1e-3 of the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    from paper_2606_18463_gb300 import glm
    glm.load()
    return glm


# (m, n, loss, lambda, s): mixed shapes, s = 1 (plain SGD), odd s and partial
# last outer steps (200 iterations)
SPECS = [(700, 64, oracle.LOGISTIC, 1e-3, 4), (1500, 100, oracle.LSQ, 1e-2, 8),
         (3000, 256, oracle.LOGISTIC, 1e-4, 3), (900, 64, oracle.LSQ, 0.0, 1),
         (2500, 130, oracle.LOGISTIC, 0.0, 16), (400, 33, oracle.LSQ, 1e-3, 5),
         (2000, 72, oracle.POISSON, 1e-3, 4)]
ITERS, B, ETA = 200, 16, 0.25


def _make(specs, seed0=0):
    out = []
    for k, (m, n, loss, lam, s) in enumerate(specs):
        if loss == oracle.LOGISTIC:
            pr = synth.logistic_planted(m, n, seed=seed0 + k, lam=lam)
        elif loss == oracle.POISSON:
            pr = synth.poisson_planted(m, n, seed=seed0 + k, lam=lam)
        else:
            pr = synth.lsq_planted(m, n, seed=seed0 + k, noise=0.1, lam=lam)
        out.append(dict(A=pr.A, y=pr.y, loss=loss, lam=lam, eta=ETA, iters=ITERS,
                        seed=100 + k, b=B, s=s))
    return out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _zeros(probs):
    return [torch.zeros(p["A"].shape[1], dtype=torch.float32, device="cuda") for p in probs]


def test_batch_f32_matches_oracle_and_replays(G):
    probs = _make(SPECS)
    for p in probs:
        p["gram"] = "f32"
    bt = G.Batch(probs, dtype="f32")
    try:
        xs = _zeros(probs)
        assert bt.run(xs) == [G.GLM_OK] * len(probs)
        got = [x.cpu().numpy().astype(np.float64) for x in xs]
        for k, p in enumerate(probs):
            ref = oracle.sgd(p["A"], p["y"], p["loss"], B, ETA, p["lam"], ITERS, p["seed"],
                             problem=k)
            assert _rel(got[k], ref) <= 1e-5, (k, _rel(got[k], ref))
            assert bt.choice(k)[:2] == (p["s"], B)
        xs2 = _zeros(probs)  # new iterate pointers: the captured run is replayed
        bt.run(xs2)
        for k in range(len(probs)):
            assert np.array_equal(xs2[k].cpu().numpy(), got[k].astype(np.float32))
    finally:
        bt.close()


def test_batch_autotuned_s(G):
    probs = _make(SPECS[:4], seed0=10)
    for p in probs:
        p["s"] = 0
        p["gram"] = "f32"
    bt = G.Batch(probs, dtype="f32")
    try:
        for k in range(len(probs)):
            assert bt.choice(k)[0] in (1, 2, 4, 8, 16)
        xs = _zeros(probs)
        bt.run(xs)
        for k, p in enumerate(probs):
            ref = oracle.sgd(p["A"], p["y"], p["loss"], B, ETA, p["lam"], ITERS, p["seed"],
                             problem=k)
            assert _rel(xs[k].cpu().numpy().astype(np.float64), ref) <= 1e-5
    finally:
        bt.close()


def test_batch_bf16_final_loss(G):
    specs = [(3000, 64, oracle.LOGISTIC, 1e-4, 8), (2000, 128, oracle.LSQ, 1e-3, 8),
             (4000, 256, oracle.LOGISTIC, 1e-3, 16), (1000, 64, oracle.LSQ, 1e-2, 4)]
    probs = _make(specs, seed0=20)
    bt = G.Batch(probs, dtype="bf16")
    try:
        xs = _zeros(probs)
        assert bt.run(xs) == [G.GLM_OK] * len(probs)
        losses = bt.loss(xs)
        for k, p in enumerate(probs):
            x = xs[k].cpu().numpy().astype(np.float64)
            ref = oracle.sgd(p["A"], p["y"], p["loss"], B, ETA, p["lam"], ITERS, p["seed"],
                             problem=k)
            f = oracle.loss(p["A"], p["y"], p["loss"], p["lam"], x)
            fr = oracle.loss(p["A"], p["y"], p["loss"], p["lam"], ref)
            assert abs(f - fr) <= 1e-3 * fr, (k, f, fr)
            # glm_batch_loss is the risk of the iterate on the stored (BF16) data
            assert abs(losses[k] - f) <= 2e-2 * f
    finally:
        bt.close()


def test_batch_nonfinite_status(G):
    probs = _make(SPECS[:3], seed0=30)
    bad = synth.lsq_planted(2000, 64, seed=99, var=100.0)
    probs.append(dict(A=bad.A, y=bad.y, loss=oracle.LSQ, lam=0.0, eta=0.9, iters=4000,
                      seed=7, b=8, s=4))
    for p in probs:
        p["gram"] = "f32"
    bt = G.Batch(probs, dtype="f32")
    try:
        st = bt.run(_zeros(probs))
        assert st[:3] == [G.GLM_OK] * 3 and st[3] == G.GLM_ENONFINITE
    finally:
        bt.close()


def test_batch_argument_errors(G):
    probs = _make(SPECS[:2], seed0=40)
    probs[0]["gram"], probs[1]["gram"] = "f32", "bf16"
    with pytest.raises(G.GlmError) as e:
        G.Batch(probs, dtype="f32")
    assert e.value.code == G.GLM_EINVAL
    probs = _make(SPECS[:1], seed0=41)
    probs[0]["b"] = 0
    with pytest.raises(G.GlmError) as e:
        G.Batch(probs, dtype="f32")
    assert e.value.code == G.GLM_EINVAL


def test_batch_tuner_gram_kernel_and_tile(G):
    # BF16 storage: the tuner times the SIMT kernel and both tcgen05 tiles for
    # every s > 1 and reports its choice; results are held to the final-loss bar
    probs = _make([(3000, 64, oracle.LOGISTIC, 1e-4, 0), (2500, 128, oracle.LSQ, 1e-3, 0),
                   (2000, 256, oracle.LOGISTIC, 1e-3, 0), (1800, 512, oracle.LSQ, 1e-3, 0)],
                  seed0=30)
    bt = G.Batch(probs, dtype="bf16")
    try:
        for k in range(len(probs)):
            s, _, _ = bt.choice(k)
            gk, tau = bt.choice_kernel(k)
            assert (s == 1 and gk == 0) or (s > 1 and gk in (1, 2, 3)), (s, gk)
            assert tau == 0.0                   # no bound asked: not estimated
        xs = _zeros(probs)
        assert bt.run(xs) == [G.GLM_OK] * len(probs)
        for k, p in enumerate(probs):
            ref = oracle.sgd(p["A"], p["y"], p["loss"], B, ETA, p["lam"], ITERS, p["seed"],
                             problem=k)
            f = oracle.loss(p["A"], p["y"], p["loss"], p["lam"], xs[k].cpu().numpy())
            fr = oracle.loss(p["A"], p["y"], p["loss"], p["lam"], ref)
            assert abs(f - fr) <= 1e-3 * fr, (k, f, fr)
    finally:
        bt.close()


@pytest.mark.parametrize("bound", [0.5, 1e-12])
def test_batch_tuner_theorem_prior(G, bound):
    # FP32 storage with a bound on tau_G: the tuner may pick a narrower Gram
    # type only where the prior admits it.  Every problem's estimated tau_G at
    # its (s, type) stays within the bound (s = 1 needs no Gram); with an
    # impossible bound every problem runs plain SGD and matches the oracle
    # at 1e-5.
    probs = _make([(3000, 64, oracle.LOGISTIC, 1e-4, 0), (2500, 128, oracle.LSQ, 1e-3, 0),
                   (2000, 256, oracle.LOGISTIC, 1e-3, 0)], seed0=40)
    bt = G.Batch(probs, dtype="f32", tau_bound=bound)
    try:
        gdt = bt.choice(0)[2]
        assert gdt in (G.GLM_F32, G.GLM_TF32, G.GLM_F16, G.GLM_BF16)
        for k in range(len(probs)):
            s, _, g2 = bt.choice(k)
            gk, tau = bt.choice_kernel(k)
            assert g2 == gdt
            assert tau <= bound, (k, s, tau)
            if bound < 1e-9:
                assert s == 1
        xs = _zeros(probs)
        assert bt.run(xs) == [G.GLM_OK] * len(probs)
        for k, p in enumerate(probs):
            ref = oracle.sgd(p["A"], p["y"], p["loss"], B, ETA, p["lam"], ITERS, p["seed"],
                             problem=k)
            got = xs[k].cpu().numpy().astype(np.float64)
            if bound < 1e-9:
                assert _rel(got, ref) <= 1e-5
            f = oracle.loss(p["A"], p["y"], p["loss"], p["lam"], got)
            fr = oracle.loss(p["A"], p["y"], p["loss"], p["lam"], ref)
            assert abs(f - fr) <= 1e-3 * fr
    finally:
        bt.close()
