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
