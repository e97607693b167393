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
