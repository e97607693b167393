"""Column-partitioned CA-SGD (paper Algorithm 1 on P ranks, 1D block-column
partition; the grouped sum of {r, G_L} per outer iteration) through the C ABI:
P ranks emulated on one device, each with a dataset handle over its column
slab, glm_sum_buffers in place of the AllReduce.  In exact arithmetic the
partitioned iterate is the SGD iterate, so the FP32 path is held to 1e-5
relative against the FP64 oracle's SGD, like the one-rank path; reduced
precision to the final-loss bar 1e-3."""
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


def _run(G, pr, P, s, b, eta, lam, T, seed, dtype="f32", **opts):
    from paper_2606_18463_gb300 import partition
    y = torch.from_numpy(pr.y).cuda()
    ops, xs = [], []
    for r in range(P):
        c0, c1 = partition.slab_columns(pr.n, P, r)
        A = torch.from_numpy(np.ascontiguousarray(pr.A[:, c0:c1])).cuda()
        ds = G.Dataset(A, y, pr.loss, dtype)
        ops.append(partition.SlabOps(ds, s, b, **opts))
        xs.append(torch.zeros(c1 - c0, dtype=torch.float32, device="cuda"))
    partition.run_emulated(ops, xs, s=s, eta=eta, lam=lam, iters=T, seed=seed)
    for o in ops:
        o.ds.sync()
    x = torch.cat(xs).cpu().numpy().astype(np.float64)
    for o in ops:
        o.ds.close()
    return x


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_partitioned_fp32_equals_sgd(G, P):
    pr = synth.logistic_planted(8192, 256, seed=0, lam=1e-4)
    x = _run(G, pr, P, 4, 16, 0.5, 1e-4, 1024, 0, gram_dtype="f32")
    ref = oracle.sgd(pr.A, pr.y, pr.loss, 16, 0.5, 1e-4, 1024, 0)
    assert _rel(x, ref) <= 1e-5, _rel(x, ref)


@pytest.mark.parametrize("m,n,b,s,T,loss,lam,P", [
    (500, 37, 5, 3, 31, synth.LOGISTIC, 0.0, 3),     # ragged slabs (13, 12, 12), tail
    (700, 8, 16, 7, 100, synth.LSQ, 1e-2, 2),
    (600, 3, 4, 5, 50, synth.LSQ, 0.0, 3),           # one column per rank
])
def test_partitioned_ragged(G, m, n, b, s, T, loss, lam, P):
    pr = synth.ragged(m, n, seed=m + n, loss=loss, lam=lam)
    x = _run(G, pr, P, s, b, 0.25, lam, T, 11, gram_dtype="f32")
    ref = oracle.sgd(pr.A, pr.y, loss, b, 0.25, lam, T, 11)
    assert _rel(x, ref) <= 1e-5, _rel(x, ref)


def test_partitioned_fp64_recurrence_and_poisson(G):
    pr = synth.logistic_planted(4096, 128, seed=2, lam=1e-4)
    x = _run(G, pr, 2, 32, 8, 0.5, 1e-4, 512, 3, gram_dtype="f32", recurrence_f64=1)
    ref = oracle.sgd(pr.A, pr.y, pr.loss, 8, 0.5, 1e-4, 512, 3)
    assert _rel(x, ref) <= 1e-5
    pp = synth.poisson_planted(4000, 96, seed=5, lam=1e-3)
    x = _run(G, pp, 3, 8, 16, 0.05, 1e-3, 400, 3, gram_dtype="f32")
    ref = oracle.sgd(pp.A, pp.y, pp.loss, 16, 0.05, 1e-3, 400, 3)
    assert _rel(x, ref) <= 1e-5


@pytest.mark.parametrize("storage,gram", [("bf16", "bf16"), ("f32", "tf32"), ("f16", "f16")])
def test_partitioned_low_precision_final_loss(G, storage, gram):
    pr = synth.logistic_planted(8192, 256, seed=0, lam=1e-4)
    x = _run(G, pr, 2, 4, 16, 0.5, 1e-4, 2048, 0, dtype=storage, gram_dtype=gram)
    ref = oracle.sgd(pr.A, pr.y, pr.loss, 16, 0.5, 1e-4, 2048, 0)
    f = oracle.loss(pr.A, pr.y, pr.loss, 1e-4, x)
    fr = oracle.loss(pr.A, pr.y, pr.loss, 1e-4, ref)
    assert abs(f - fr) <= 1e-3 * fr


def test_sum_buffers_and_errors(G):
    srcs = [torch.arange(10, dtype=torch.float32, device="cuda") * (p + 1) for p in range(5)]
    dst = torch.empty(10, device="cuda")
    G.glm_sum_buffers(dst, srcs, 10)
    torch.cuda.synchronize()
    assert torch.equal(dst, torch.arange(10, dtype=torch.float32, device="cuda") * 15)
    G.glm_sum_buffers(srcs[0], srcs[:2], 10)    # in place
    torch.cuda.synchronize()
    assert torch.equal(srcs[0], torch.arange(10, dtype=torch.float32, device="cuda") * 3)
    with pytest.raises(G.GlmError):
        G.glm_sum_buffers(dst, [], 10)
    assert G.glm_slab_reduce_floats(4, 16) == 64 + 16 * (16 + 32 + 48)
    with pytest.raises(G.GlmError):
        G.glm_slab_reduce_floats(128, 128)
    pr = synth.logistic_planted(512, 16, seed=1)
    ds = G.Dataset(torch.from_numpy(pr.A).cuda(), torch.from_numpy(pr.y).cuda(), pr.loss)
    x = torch.zeros(16, device="cuda")
    red = torch.zeros(G.glm_slab_reduce_floats(4, 8), device="cuda")
    with pytest.raises(G.GlmError) as e:
        G.glm_slab_partial(ds.h, 4, 8, 5, 0, 0, x, red)    # sh > s
    assert e.value.code == G.GLM_EINVAL
    ds.close()
