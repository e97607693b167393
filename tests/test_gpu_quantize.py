"""Create-time quantisation, byte for byte (storage slot u_A of the paper's
precision table; the FP8 copy with per-row scales).

What glm_create_ex stored is read back through the C ABI
(glm_storage_read) and compared bit-exactly with the oracle's definitions:
  * column scales kappa_j = the power of two nearest the column RMS
    (oracle.column_scales), 1 for all-zero columns and for FP32 storage;
  * stored values round(A / kappa) to BF16 (oracle.round_bf16) or FP16
    (oracle.round_f16), nearest even, padding columns zero;
  * FP8 row scales rho_i (oracle.fp8_row_scales) and bytes
    E4M3(a / rho_i) (oracle.round_e4m3), nearest even, saturating.
The inputs carry exact rounding ties for every format, all-zero rows and
columns, FP16 subnormals and E4M3 subnormals, on ragged shapes.  Column
scales whose log2 falls exactly on a half integer are not constructed: the
RMS would have to be an odd power of sqrt(2), which no input reaches
exactly, and the reading (nearest power of two) leaves that case open.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    from paper_2606_18463_gb300 import glm
    glm.load()
    return glm


def _decode_e4m3(byte_arr):
    """E4M3 (bias 7, 3 mantissa bits; exponent field 0 subnormal, S.1111.111
    NaN) bytes to FP64 values."""
    b = np.asarray(byte_arr, dtype=np.uint8).astype(np.int64)
    sign = np.where(b & 0x80, -1.0, 1.0)
    e = (b >> 3) & 0xF
    mnt = b & 0x7
    val = np.where(e == 0, mnt * 2.0 ** -9, (1.0 + mnt / 8.0) * np.exp2(e - 7.0))
    val = np.where((e == 15) & (mnt == 7), np.nan, val)
    return sign * val


def _tricky(m, n, seed):
    """Dyadic values (few significant bits, so exact ties occur after every
    power-of-two scaling) with zero rows and columns, tiny and huge entries."""
    rng = np.random.default_rng(seed)
    A = rng.integers(-4096, 4097, (m, n)).astype(np.float64) * 2.0 ** -10
    A *= np.exp2(rng.integers(-3, 4, (1, n)))                 # column magnitudes
    if n > 2:
        A[:, 1] = 0.0                                           # all-zero column
    if m > 3:
        A[2, :] = 0.0                                           # all-zero row
    if n > 3:
        # a column of tiny entries beside one large one: after dividing by the
        # column scale (set by the large entry) they are FP16 subnormals
        A[:, 3] = rng.integers(1, 64, m) * 2.0 ** -24
        A[0, 3] = 3.0
    if m > 5:
        # E4M3 subnormals: a row whose maximum sets rho, other entries far below
        A[5, :] = rng.integers(-7, 8, n) * 2.0 ** -12
        A[5, 0] = 448.0 * 2.0 ** -3
    # explicit ties: 1 + k/128 + 1/256 are BF16 ties, 1 + k/1024 + 1/2048 FP16
    # ties, 1 + k/8 + 1/16 E4M3 ties (for unit scales)
    if n > 5 and m > 8:
        A[6:, 4] = 1.0 + rng.integers(0, 40, m - 6) / 128 + 1 / 256
        A[6:, 5] = 1.0 + rng.integers(0, 300, m - 6) / 1024 + 1 / 2048
    if m > 7:
        A[7, :] = np.where(np.arange(n) % 2 == 0, 1.0 + 3 / 8 + 1 / 16, -(1.0 + 1 / 16))
        A[7, 0] = 448.0 / 256.0  # rho = 2^-8 exactly at the boundary (max = 448 rho)
    return A.astype(np.float32)


def _labels(m):
    return np.where(np.arange(m) % 3 == 0, -1.0, 1.0).astype(np.float32)


def _read(G, ds, m):
    dt, lda, lda8 = G.glm_storage_layout(ds.h)
    eb = {G.GLM_F32: 4, G.GLM_BF16: 2, G.GLM_F16: 2}[dt]
    raw = np.zeros(m * lda * eb, dtype=np.uint8)
    cs = np.zeros(ds.n, dtype=np.float32)
    G.glm_storage_read(ds.h, 0, m, raw, cs)
    return dt, lda, lda8, raw, cs


@pytest.mark.parametrize("m,n", [(37, 13), (9, 1), (11, 3), (300, 200), (64, 8)])
@pytest.mark.parametrize("storage", ["bf16", "f16", "f32"])
@pytest.mark.parametrize("where", ["host", "device"])
def test_storage_bit_exact(G, m, n, storage, where):
    A = _tricky(m, n, seed=m * 31 + n)
    y = _labels(m)
    Ai = torch.from_numpy(A) if where == "host" else torch.from_numpy(A).cuda()
    yi = torch.from_numpy(y) if where == "host" else torch.from_numpy(y).cuda()
    ds = G.Dataset(Ai, yi, G.GLM_LOGISTIC, storage)
    dt, lda, lda8, raw, cs = _read(G, ds, m)
    assert lda == (n + 7) // 8 * 8 and lda8 == 0
    if storage == "f32":
        assert np.all(cs == 1.0)
        st = raw.view(np.float32).reshape(m, lda)
        assert np.array_equal(st[:, :n].view(np.uint32), A.view(np.uint32))
        assert np.all(st[:, n:].view(np.uint32) == 0)
        return
    kappa = oracle.column_scales(A)
    assert np.array_equal(cs.astype(np.float64), kappa), (cs, kappa)
    scaled = (A.astype(np.float64) / kappa).astype(np.float32)   # exact: powers of two
    assert np.array_equal(scaled.astype(np.float64) * kappa, A.astype(np.float64))
    bits = raw.view(np.uint16).reshape(m, lda)
    assert np.all(bits[:, n:] == 0)
    if storage == "bf16":
        want = oracle.round_bf16(scaled).view(np.uint32) >> 16
        got = bits[:, :n].astype(np.uint32)
    else:
        want = oracle.round_f16(scaled).astype(np.float16).view(np.uint16)
        got = bits[:, :n]
    bad = np.argwhere(got != want)
    assert bad.size == 0, (bad[:5], got[tuple(bad[0])], want[tuple(bad[0])])
    # the inputs really hold FP16 subnormals
    if storage == "f16" and n > 3 and m > 3:
        assert np.any(((got & 0x7C00) == 0) & ((got & 0x3FF) != 0))
    ds.close()


@pytest.mark.parametrize("m,n", [(37, 13), (9, 1), (11, 3), (300, 200), (40, 16)])
def test_fp8_copy_bit_exact(G, m, n):
    A = _tricky(m, n, seed=m * 17 + n)
    y = _labels(m)
    ds = G.Dataset(torch.from_numpy(A).cuda(), torch.from_numpy(y).cuda(), G.GLM_LOGISTIC,
                   "bf16", fp8_copy=True)
    dt, lda, lda8 = G.glm_storage_layout(ds.h)
    assert lda8 == (n + 15) // 16 * 16
    q = np.zeros(m * lda8, dtype=np.uint8)
    rs = np.zeros(m, dtype=np.float32)
    G.glm_storage_read(ds.h, 0, m, None, None, q, rs)
    rho = oracle.fp8_row_scales(A)
    assert np.array_equal(rs.astype(np.float64), rho), (rs, rho)
    q = q.reshape(m, lda8)
    assert np.all(q[:, n:] == 0)
    want = oracle.round_e4m3(A.astype(np.float64) / rho[:, None])
    got = _decode_e4m3(q[:, :n])
    assert np.array_equal(got, want), np.argwhere(got != want)[:5]
    # signs of zeros: a negative value that rounds to zero keeps its sign
    assert np.array_equal(np.signbit(got), np.signbit(want))
    # exact ties (368 between 352 and 384, 272 between 256 and 288) and
    # subnormals (exponent field 0) occurred
    if m > 7 and n > 1:
        mid = np.abs(A[7, :n].astype(np.float64) / rho[7])
        assert rho[7] == 2.0 ** -8 and np.any(mid == 368.0) and np.any(mid == 272.0)
    if m > 5 and n > 1:
        sub = q[5, :n]
        assert np.any((((sub >> 3) & 0xF) == 0) & ((sub & 7) != 0))
    ds.close()


def test_bf16_input_and_partial_reads(G):
    m, n = 50, 24
    A = _tricky(m, n, seed=3)
    Ab = oracle.round_bf16(A)                             # BF16 values
    bits = (Ab.view(np.uint32) >> 16).astype(np.uint16)
    ds = G.Dataset(torch.from_numpy(bits.view(np.int16)).cuda(),
                   torch.from_numpy(_labels(m)).cuda(), G.GLM_LOGISTIC, "f16",
                   input_dtype="bf16", fp8_copy=True)
    dt, lda, lda8 = G.glm_storage_layout(ds.h)
    raw = np.zeros(7 * lda, dtype=np.uint16)
    cs = np.zeros(n, dtype=np.float32)
    q = np.zeros(7 * lda8, dtype=np.uint8)
    rs = np.zeros(7, dtype=np.float32)
    G.glm_storage_read(ds.h, 20, 7, raw, cs, q, rs)       # rows 20..26 only
    kappa = oracle.column_scales(Ab)
    assert np.array_equal(cs.astype(np.float64), kappa)
    want = oracle.round_f16((Ab[20:27].astype(np.float64) / kappa).astype(np.float32))
    assert np.array_equal(raw.reshape(7, lda)[:, :n], want.astype(np.float16).view(np.uint16))
    rho = oracle.fp8_row_scales(Ab[20:27])
    assert np.array_equal(rs.astype(np.float64), rho)
    want8 = oracle.round_e4m3(Ab[20:27].astype(np.float64) / rho[:, None])
    assert np.array_equal(_decode_e4m3(q.reshape(7, lda8)[:, :n]), want8)
    # argument errors
    with pytest.raises(G.GlmError) as e:
        G.glm_storage_read(ds.h, 45, 10, raw)
    assert e.value.code == G.GLM_EINVAL
    dsn = G.Dataset(torch.from_numpy(_tricky(8, 4, 1)).cuda(),
                    torch.from_numpy(_labels(8)).cuda(), G.GLM_LOGISTIC, "bf16")
    with pytest.raises(G.GlmError) as e:
        G.glm_storage_read(dsn.h, 0, 1, None, None, q)    # no FP8 copy
    assert e.value.code == G.GLM_EINVAL
    dev = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(G.GlmError) as e:
        G.glm_storage_read(dsn.h, 0, 1, None, dev)         # device output
    assert e.value.code == G.GLM_EINVAL
    ds.close()
    dsn.close()
