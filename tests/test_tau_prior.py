"""The batched autotuner's Theorem 1 prior (paper Sec. 5.2), host arithmetic
through the C ABI (no GPU): its ||H_L||_2 bound is an upper bound of the
oracle's exact norm and within sqrt(s b) of it, K_s's Neumann bound covers
the oracle's exact K_s, so the estimated tau_G covers the oracle's exact
hypothesis figure for the same slots; closed forms in small cases."""
import math
import os

import numpy as np
import pytest

from oracle import local_error as le
from paper_2606_18463_gb300 import glm

pytestmark = pytest.mark.skipif(not os.path.exists(glm.LIB_PATH), reason="libglm.so not built")


@pytest.mark.parametrize("loss", [le.LOGISTIC, le.LSQ])
@pytest.mark.parametrize("s,b,n", [(2, 4, 8), (4, 8, 16), (8, 16, 64), (16, 4, 10)])
def test_prior_covers_exact_theorem_figures(loss, s, b, n):
    rng = np.random.default_rng(s * 100 + b + n)
    for trial in range(4):
        Y = rng.standard_normal((s * b, n)) / math.sqrt(n)
        Y = Y.astype(np.float32).astype(np.float64)
        y = np.where(rng.random(s * b) < 0.5, -1.0, 1.0) if loss == le.LOGISTIC else \
            rng.standard_normal(s * b)
        x = rng.standard_normal(n) * 0.3
        eta = 0.5
        u_A, u_in = 2.0 ** -8, 2.0 ** -11
        q = n * 2.0 ** -24
        gamma_G = 2 * u_in + q / (1 - q)
        ev = le.local_error(Y, y, x, loss, eta, s, b, u_A=u_A, gamma_G=gamma_G)
        hl, tau = glm.glm_tau_prior(Y, s, b, eta / b, loss, u_A, u_in)
        assert hl >= ev["norm_H_L"] * (1 - 1e-12)
        assert hl <= math.sqrt(s * b) * ev["norm_H_L"] * (1 + 1e-12)
        assert tau >= ev["tau_G"] * (1 - 1e-12), (tau, ev["tau_G"])


def test_prior_closed_forms():
    # two blocks of one row each, one column: H_L = [[0, 0], [|a1 a0|, 0]],
    # every norm is |a1 a0| = 6; L alpha ||H_L|| = 1 * 0.1 * 6 = 0.6
    Y = np.array([[2.0], [3.0]], dtype=np.float32)
    hl, tau = glm.glm_tau_prior(Y, 2, 1, 0.1, le.LSQ, 0.0, 0.0)
    assert hl == 6.0
    q = 2.0 ** -24
    assert tau == pytest.approx((1 / (1 - 0.6)) * 1.0 * 0.1 * (q / (1 - q)) * 6.0, rel=1e-12)
    # L alpha ||H_L|| >= 1: the Neumann bound fails, the figure is infinite
    _, tau = glm.glm_tau_prior(Y, 2, 1, 0.2, le.LSQ, 0.0, 0.0)
    assert math.isinf(tau)
    # Poisson: no Lipschitz bound; exact operands give 0, rounded ones infinity
    assert glm.glm_tau_prior(Y, 2, 1, 0.1, 2, 0.0, 0.0)[1] == 0.0
    assert math.isinf(glm.glm_tau_prior(Y, 2, 1, 0.1, 2, 0.0, 2.0 ** -8)[1])
    # one block: no strictly lower part
    assert glm.glm_tau_prior(Y, 1, 2, 0.1, le.LSQ, 0.0, 0.0) == (0.0, 0.0)
