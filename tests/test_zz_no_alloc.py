"""glm_sample_indices_noalloc: host-output index draw staged in a fixed device
array.  Called through the C ABI twice in a row, it must give exactly what
glm_sample_indices gives (indices are integers: bit-exact), and it must
reject counts above its static capacity before touching the device.

The file name sorts last so that the module runs after every other GPU test
(and passes when run alone too).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    from paper_2606_18463_gb300 import glm
    glm.load()
    return glm


@pytest.mark.parametrize("seed,problem,first,count,m", [
    (7, 0, 0, 1000, 8192),
    (11, 3, 12345, 777, 400_000),
    (5, 1, 2**40 + 5, 64, 2**31 - 1),
    (3, 2, 99, 1 << 20, 1_048_576),   # the full static capacity
])
def test_noalloc_matches_allocating_path_twice(G, seed, problem, first, count, m):
    ref = np.zeros(count, dtype=np.int32)
    G.glm_sample_indices(seed, problem, first, count, m, ref)
    for _ in range(2):
        got = np.full(count, -1, dtype=np.int32)
        G.glm_sample_indices_noalloc(seed, problem, first, count, m, got)
        assert np.array_equal(got, ref)


def test_noalloc_matches_the_oracle(G):
    import oracle
    ref = oracle.sample_indices(13, 4, 2**33 + 7, 5000, 123_457)
    for _ in range(2):
        got = np.full(5000, -1, dtype=np.int32)
        G.glm_sample_indices_noalloc(13, 4, 2**33 + 7, 5000, 123_457, got)
        assert np.array_equal(got.astype(np.int64), ref)


def test_noalloc_rejects_device_and_short_outputs(G):
    # through the raw C entry point: the binding would refuse a torch tensor
    dev = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = G.load().glm_sample_indices_noalloc(0, 0, 0, 16, 10, dev.data_ptr())
    assert rc == G.GLM_EINVAL and "host memory" in G.glm_last_error()
    with pytest.raises(ValueError):
        G.glm_sample_indices_noalloc(0, 0, 0, 16, 10, np.zeros(8, dtype=np.int32))
    with pytest.raises(ValueError):
        G.glm_sample_indices_noalloc(0, 0, 0, 4, 10, np.zeros(4, dtype=np.int64))


def test_noalloc_smaller_call_after_larger(G):
    big = np.zeros(4096, dtype=np.int32)
    G.glm_sample_indices_noalloc(1, 0, 0, 4096, 1000, big)
    small = np.full(10, -1, dtype=np.int32)
    G.glm_sample_indices_noalloc(1, 0, 5000, 10, 1000, small)
    ref = np.zeros(10, dtype=np.int32)
    G.glm_sample_indices(1, 0, 5000, 10, 1000, ref)
    assert np.array_equal(small, ref)


def test_noalloc_rejects_over_capacity(G):
    out = np.zeros(8, dtype=np.int32)   # never written: rejection comes first
    with pytest.raises(G.GlmError) as ei:
        G.glm_sample_indices_noalloc(0, 0, 0, G.GLM_SAMPLE_NOALLOC_MAX + 1, 10, out)
    assert ei.value.code == G.GLM_EINVAL
    assert "GLM_SAMPLE_NOALLOC_MAX" in str(ei.value)


def test_noalloc_empty_and_bad_args(G):
    G.glm_sample_indices_noalloc(0, 0, 0, 0, 5, None)
    with pytest.raises(G.GlmError) as ei:
        G.glm_sample_indices_noalloc(0, 0, 0, 4, 0, np.zeros(4, dtype=np.int32))
    assert ei.value.code == G.GLM_EINVAL
