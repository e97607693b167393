"""Failure paths, provoked without faulting the GPU.

  * Device timeouts: glm_ca_opts.wait_probe_cycles makes one thread of every
    CTA of the chain and tcgen05 Gram kernels wait on a barrier that nothing
    signals.  The wait gives up, the kernels unwind (copies in flight
    drained, TMEM freed, x untouched), glm_sync reports GLM_ETIMEOUT once,
    and the handle stays usable: the next run is bit-identical to a run on a
    fresh handle.  The batch's Gram launches take the same probe.
  * Allocation failure: glm_debug_fail_alloc makes the k-th device
    allocation fail; glm_create_ex and the first run of a shape return
    GLM_ENOMEM and leave nothing half-built.
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
    yield glm
    glm.glm_debug_fail_alloc(-1)


@pytest.fixture(scope="module")
def pr():
    return synth.logistic_planted(8192, 256, seed=0, lam=1e-4)


def _ds(G, pr, dtype="f32"):
    return G.Dataset(torch.from_numpy(pr.A).cuda(), torch.from_numpy(pr.y).cuda(), pr.loss,
                     dtype)


@pytest.mark.parametrize("s,gram,graph", [(4, "f32", 1), (4, "bf16", 1), (4, "bf16", 0),
                                          (1, None, 1), (16, "bf16", 1)])
def test_probe_times_out_and_handle_recovers(G, pr, s, gram, graph):
    ds = _ds(G, pr, "f32" if gram != "bf16" else "bf16")
    rng = np.random.default_rng(1)
    x0 = torch.tensor(rng.standard_normal(pr.n).astype(np.float32), device="cuda")
    x = x0.clone()
    opts = dict(use_graph=graph, wait_probe_cycles=2000)
    if gram:
        opts["gram_dtype"] = gram
    run = ds.sgd if s == 1 else (lambda *a, **k: ds.ca_sgd(a[0], s, *a[1:], **k))
    run(x, 16, 0.5, 1e-4, 512, 0, **opts)
    assert G.glm_sync(ds.h) == G.GLM_ETIMEOUT
    assert G.glm_sync(ds.h) == G.GLM_OK               # reported once, then cleared
    assert torch.equal(x, x0)                           # x left as it was
    # the same handle, normal runs: equal to a fresh handle's, bit for bit
    del opts["wait_probe_cycles"]
    x.copy_(x0)
    run(x, 16, 0.5, 1e-4, 512, 0, **opts)
    ds.sync()
    fresh = _ds(G, pr, "f32" if gram != "bf16" else "bf16")
    y = x0.clone()
    run2 = fresh.sgd if s == 1 else (lambda *a, **k: fresh.ca_sgd(a[0], s, *a[1:], **k))
    run2(y, 16, 0.5, 1e-4, 512, 0, **opts)
    fresh.sync()
    assert torch.equal(x, y)
    if gram != "bf16":
        ref = oracle.sgd(pr.A, pr.y, pr.loss, 16, 0.5, 1e-4, 512, 0,
                         x0=x0.cpu().numpy().astype(np.float64))
        got = x.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    ds.close()
    fresh.close()


def test_batch_gram_probe_reports_timeout(G):
    specs = [dict(p=p, m=3000 + 500 * p, n=128, lam=1e-4, loss=p % 2) for p in range(4)]
    probs = []
    for sp in specs:
        q = synth.batch_problem(sp, seed=3)
        probs.append(dict(A=q.A, y=q.y, loss=sp["loss"], lam=sp["lam"], eta=0.1, iters=256,
                          seed=sp["p"], b=32, s=4))
    bt = G.Batch(probs, dtype="bf16", wait_probe_cycles=2000)
    xs = [torch.zeros(128, device="cuda") for _ in probs]
    with pytest.raises(G.GlmError) as e:
        bt.run(xs)
    assert e.value.code == G.GLM_ETIMEOUT
    bt.close()
    ok = G.Batch(probs, dtype="bf16")
    assert ok.run(xs) == [G.GLM_OK] * 4
    ok.close()


def test_forced_allocation_failure(G, pr):
    A = torch.from_numpy(pr.A).cuda()
    y = torch.from_numpy(pr.y).cuda()
    fails = 0
    for k in range(0, 12):
        G.glm_debug_fail_alloc(k)
        try:
            ds = G.Dataset(A, y, pr.loss, "bf16")
        except G.GlmError as e:
            assert e.code == G.GLM_ENOMEM, str(e)
            fails += 1
            continue
        finally:
            G.glm_debug_fail_alloc(-1)
        break
    assert fails >= 5          # every allocation of the create path was hit once
    # a run's first allocation of scratch fails; the handle stays usable
    x = torch.zeros(pr.n, device="cuda")
    G.glm_debug_fail_alloc(0)
    with pytest.raises(G.GlmError) as e:
        ds.ca_sgd(x, 4, 16, 0.5, 1e-4, 256, 0)
    G.glm_debug_fail_alloc(-1)
    assert e.value.code == G.GLM_ENOMEM
    ds.ca_sgd(x, 4, 16, 0.5, 1e-4, 256, 0)
    ds.sync()
    ref = _ds(G, pr, "bf16")
    xr = torch.zeros(pr.n, device="cuda")
    ref.ca_sgd(xr, 4, 16, 0.5, 1e-4, 256, 0)
    ref.sync()
    assert torch.equal(x, xr)
    ds.close()
    ref.close()
