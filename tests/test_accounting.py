"""The roofline accounting reproduces the paper's printed arithmetic
intensities (tests/golden/paper_roofline_ai.txt, Sec. 7.6 roofline figure)."""
import os

import pytest

from paper_2606_18463_gb300 import accounting as acc

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_roofline_ai.txt")


def _rows():
    for line in open(GOLD):
        line = line.strip()
        if line and not line.startswith("#"):
            r, e, s, ai = line.split()
            yield r, int(e), int(s), float(ai)


@pytest.mark.parametrize("recipe,e_A,s,ai", list(_rows()))
def test_paper_gram_ai(recipe, e_A, s, ai):
    assert abs(acc.paper_gram_ai(s, 32, 16384, e_A) - ai) <= 0.06


def test_counts_small_cases():
    # s=2, b=1, n=3: one strictly-lower entry, 3 FMAs -> 6 flops
    assert acc.gram_flops(2, 1, 3) == 6
    assert acc.gram_lower_floats(2, 1) == 4          # one row padded to 4
    assert acc.gram_lower_floats(3, 4) == 4 * 4 + 4 * 8
    assert acc.gathered_bytes(4, 16, 256, 4) == 64 * (1024 + 4)
    assert acc.recurrence_flops(16, 64) == 64 * 64 * 16 * 15


def test_roof_seconds_by_hand():
    # T = 10, s = 4: outer blocks of 4, 4 and 2 inner steps; b = 2, n = 3,
    # e_A = 4.  Bytes per block of sj steps: sj * 2 * (12 + 4) = 32 sj;
    # Gram flops: 4 sj (sj - 1) * 3 = 12 sj (sj - 1).
    assert acc.outer_blocks(10, 4) == [4, 4, 2]
    by, fl = acc.run_bytes_flops(10, 4, 2, 3, 4)
    assert by == 32 * 10 and fl == 12 * (12 + 12 + 2)
    # HBM 1 GB/s, 1 TFLOP/s: bytes bind in every block (32 sj ns vs 12 sj (sj-1) ps)
    t = acc.roof_seconds(10, 4, 2, 3, 4, 1.0, 1.0)
    assert t == pytest.approx(320e-9)
    # a slow tensor unit (1e-9 TFLOP/s = 1 kflop/s) makes the Gram bind where sj > 1
    t = acc.roof_seconds(10, 4, 2, 3, 4, 1.0, 1e-9)
    assert t == pytest.approx((144 + 144 + 24) / 1e3)
    assert acc.gram_peak_tflops("tf32", 2000.0) == 1000.0
    assert acc.gram_peak_tflops("e4m3", 2000.0) == 4000.0
    assert acc.gram_peak_tflops("f32", 2000.0, 2070.0) == pytest.approx(80.55, abs=0.01)
