"""The streaming chain (glm_ca_opts.chain_impl = 2: Y and G streamed through
shared-memory rings, full-width own-row margins, x all-gathered every outer
iteration) against the FP64 oracle, through the C ABI: FP32 iterates at
1e-5 relative (FP32, FP64 and compensated-FP32 recurrences), reduced
precision at the 1e-3 final-loss bar, the failure probe, and the wide /
long-block shapes it exists for (m reduced)."""
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


def _ds(G, pr, dtype="f32", **kw):
    return G.Dataset(torch.from_numpy(pr.A).cuda(), torch.from_numpy(pr.y).cuda(), pr.loss,
                     dtype, **kw)


def _run(G, ds, n, s, b, eta, lam, T, seed, **opts):
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    ds.ca_sgd(x, s, b, eta, lam, T, seed, chain_impl=2, **opts)
    ds.sync()
    return x.cpu().numpy().astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("rec", [0, 1, 2])
@pytest.mark.parametrize("cluster", [1, 4, 16])
def test_stream_fp32_matches_oracle(G, rec, cluster):
    pr = synth.logistic_planted(8192, 256, seed=0, lam=1e-4)
    ds = _ds(G, pr)
    x = _run(G, ds, pr.n, 4, 16, 0.5, 1e-4, 2048, 0, gram_dtype="f32", recurrence_f64=rec,
             cluster=cluster)
    ref = oracle.sgd(pr.A, pr.y, pr.loss, 16, 0.5, 1e-4, 2048, 0)
    assert _rel(x, ref) <= 1e-5, _rel(x, ref)
    plan = G.glm_ca_plan(ds.h, 4, 16, 0.5, 1e-4, 2048,
                         G.default_ca_opts(chain_impl=2, gram_dtype="f32", cluster=cluster))
    assert plan.chain_impl == 2
    ds.close()


@pytest.mark.parametrize("m,n,b,s,T,loss,lam,C", [
    (97, 37, 5, 3, 31, synth.LOGISTIC, 0.0, 1),
    (500, 8, 1, 7, 50, synth.LSQ, 1e-2, 1),
    (2000, 130, 12, 16, 200, synth.LOGISTIC, 1e-3, 2),
    (3000, 64, 32, 8, 100, synth.LSQ, 0.0, 8),
    (1024, 300, 9, 5, 47, synth.LSQ, 5e-3, 2),
    (300, 1, 4, 3, 40, synth.LOGISTIC, 1e-3, 4),
    (4000, 600, 64, 6, 300, synth.LOGISTIC, 1e-4, 16),
])
def test_stream_ragged(G, m, n, b, s, T, loss, lam, C):
    pr = synth.ragged(m, n, seed=m + n, loss=loss, lam=lam)
    ds = _ds(G, pr)
    ref = oracle.sgd(pr.A, pr.y, loss, b, 0.25, lam, T, 11)
    for rec in (0, 2):
        x = _run(G, ds, n, s, b, 0.25, lam, T, 11, gram_dtype="f32", cluster=C,
                 chunk_outer=3, recurrence_f64=rec)
        assert _rel(x, ref) <= 1e-5, (rec, _rel(x, ref))
    ds.close()


def test_stream_poisson_and_graph_off(G):
    pr = synth.poisson_planted(4000, 96, seed=5, lam=1e-3)
    ds = _ds(G, pr)
    x = _run(G, ds, pr.n, 8, 16, 0.05, 1e-3, 1000, 3, gram_dtype="f32", use_graph=0, cluster=8)
    ref = oracle.sgd(pr.A, pr.y, pr.loss, 16, 0.05, 1e-3, 1000, 3)
    assert _rel(x, ref) <= 1e-5
    ds.close()


@pytest.mark.parametrize("storage,gram,s,rec", [("bf16", "bf16", 16, -1), ("bf16", "e4m3", 16, -1),
                                                ("bf16", "bf16", 32, 2), ("bf16", "bf16", 64, 1)])
def test_stream_wide_shape_final_loss(G, storage, gram, s, rec):
    pr = synth.logistic_wide(65536, 2048, seed=0, lam=1e-3)
    ds = _ds(G, pr, storage, fp8_copy=(gram == "e4m3"))
    x = _run(G, ds, pr.n, s, 128, 2.0 ** -10, 1e-3, 2048, 0, gram_dtype=gram, recurrence_f64=rec)
    ref = oracle.sgd(pr.A, pr.y, pr.loss, 128, 2.0 ** -10, 1e-3, 2048, 0)
    f = oracle.loss(pr.A, pr.y, pr.loss, 1e-3, x)
    fr = oracle.loss(pr.A, pr.y, pr.loss, 1e-3, ref)
    assert abs(f - fr) <= 1e-3 * fr
    ds.close()


def test_stream_long_blocks_fp32_parity(G):
    # the large least-squares shape's blocks (s = 64, b = 256, n = 1024) at
    # m = 65,536 with FP32 storage and Gram: the iterate against the oracle
    pr = synth.lsq_planted(65536, 1024, seed=7, noise=0.01, lam=1e-5)
    ds = _ds(G, pr)
    ref = oracle.sgd(pr.A, pr.y, pr.loss, 256, 0.5, 1e-5, 1024, 0)
    for rec in (1, 2):
        x = _run(G, ds, pr.n, 64, 256, 0.5, 1e-5, 1024, 0, gram_dtype="f32", recurrence_f64=rec)
        assert _rel(x, ref) <= 1e-5, (rec, _rel(x, ref))
    ds.close()


def test_stream_probe_and_recovery(G):
    pr = synth.logistic_planted(8192, 256, seed=0, lam=1e-4)
    ds = _ds(G, pr, "bf16")
    x = torch.ones(pr.n, device="cuda")
    ds.ca_sgd(x, 4, 16, 0.5, 1e-4, 512, 0, chain_impl=2, wait_probe_cycles=2000)
    assert G.glm_sync(ds.h) == G.GLM_ETIMEOUT
    assert torch.equal(x, torch.ones(pr.n, device="cuda"))
    y = torch.zeros(pr.n, device="cuda")
    ds.ca_sgd(y, 4, 16, 0.5, 1e-4, 512, 0, chain_impl=2)
    ds.sync()
    z = torch.zeros(pr.n, device="cuda")
    ds.ca_sgd(z, 4, 16, 0.5, 1e-4, 512, 0, chain_impl=2)
    ds.sync()
    assert torch.equal(y, z)
    with pytest.raises(G.GlmError):
        ds.ca_sgd(z, 4, 16, 0.5, 1e-4, 512, 0, chain_impl=1, recurrence_f64=2)
    ds.close()
