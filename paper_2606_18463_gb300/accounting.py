"""Algorithmic work per CA-SGD outer iteration (roofline accounting).

Units are per outer iteration of s inner steps with mini-batch b, n columns.
  gathered_bytes  one read of the s b sampled rows plus their labels:
                  s b (n e_A + 4)
  gram_flops      strictly block-lower Gram only (Algorithm 1 reads only
                  G_{j,<j}): b^2 s (s-1) n
  paper_gram_ai   the paper's own convention for its Gram roofline (Sec. 7.6):
                  2 (s b)^2 n flops over e_A s b n + 4 (s b)^2 bytes
  chain_bytes     what the x-dependent chain streams per outer iteration:
                  two passes over the staged Y (margin and update), the
                  strictly block-lower G in FP32, labels: 2 s b n e_v +
                  4 |G_L| + 4 s b
  recurrence_flops  b^2 s (s-1) (paper Table "abg-comparison")
  roof_seconds    the run's roofline time: over every outer iteration (a
                  tail block of T mod s inner steps included) the slower of
                  its gathered bytes at the HBM bandwidth and its Gram flops
                  at the Gram type's peak
"""
from __future__ import annotations


def gram_lower_floats(s: int, b: int) -> int:
    """Stored floats of one outer iteration's strictly block-lower G
    (rows padded to multiples of 4 floats)."""
    return b * sum(((j * b + 3) // 4) * 4 for j in range(1, s))


def gathered_bytes(s: int, b: int, n: int, e_A: int) -> int:
    return s * b * (n * e_A + 4)


def staged_bytes(s: int, b: int, n: int, e_op: int) -> int:
    return s * b * n * e_op


def gram_flops(s: int, b: int, n: int) -> int:
    return b * b * s * (s - 1) * n


def paper_gram_ai(s: int, b: int, n: int, e_A: int) -> float:
    sb = s * b
    return 2.0 * sb * sb * n / (e_A * sb * n + 4.0 * sb * sb)


def chain_bytes(s: int, b: int, n: int, e_v: int) -> int:
    return 2 * s * b * n * e_v + 4 * b * b * s * (s - 1) // 2 + 4 * s * b


def recurrence_flops(s: int, b: int) -> int:
    return b * b * s * (s - 1)


def sgd_flops(b: int, n: int) -> int:
    return 4 * b * n


def outer_blocks(T: int, s: int):
    """Inner-step counts of the outer iterations of a T-iteration run."""
    full, tail = divmod(T, s)
    return [s] * full + ([tail] if tail else [])


def roof_seconds(T: int, s: int, b: int, n: int, e_A: int, hbm_gbs: float,
                 tc_tflops: float) -> float:
    t = 0.0
    for sj in outer_blocks(T, s):
        t += max(gathered_bytes(sj, b, n, e_A) / (hbm_gbs * 1e9),
                 gram_flops(sj, b, n) / (tc_tflops * 1e12))
    return t


def run_bytes_flops(T: int, s: int, b: int, n: int, e_A: int):
    """Total gathered bytes and Gram flops of a T-iteration run."""
    by = fl = 0
    for sj in outer_blocks(T, s):
        by += gathered_bytes(sj, b, n, e_A)
        fl += gram_flops(sj, b, n)
    return by, fl


# nominal dense tensor throughput relative to BF16 (NVIDIA's GB300 figures:
# TF32 1.1, FP16 2.25, FP8 4.5 PFLOP/s against BF16 2.25)
TC_RATIO = {"bf16": 1.0, "f16": 1.0, "tf32": 0.5, "e4m3": 2.0}


def fp32_alu_tflops(sm_mhz: float = 2070.0, sms: int = 152) -> float:
    """FP32 FMA peak of the SIMT Gram: SMs x 128 lanes x 2 flop x clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def gram_peak_tflops(gram: str, bf16_tflops: float, sm_mhz: float = 2070.0) -> float:
    if gram == "f32":
        return fp32_alu_tflops(sm_mhz)
    return bf16_tflops * TC_RATIO[gram]
