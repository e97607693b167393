"""One-GPU analogue of the paper's recipe check (Sec. "Accuracy gap", the
validation table there): the relative final-loss gap |L_C - L_A| / |L_A|
between the BF16 recipe (BF16 storage with per-column scales, BF16 Gram and
GEMV operands, FP32 accumulation; the recurrence as the library sets it) and
the FP32 recipe, at (m, n) = (65,536, 4,096), b = 32, s in {16, 64}, H = 200
outer iterations, three seeds, for logistic, least-squares and Poisson losses.
The paper's cells (P = 16, its own synthetic data) are at most 3.3e-4 against
a 0.5 % threshold; the bar here is the 1e-3 final-loss target.  The data are
synthetic stand-ins with the paper's shape (rows of about unit norm); both
losses are evaluated on the FP32 data.
"""
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M, N, B, H, LAM = 65536, 4096, 32, 200, 1e-4
# step sizes: stable for unit-norm rows (logistic, least squares) and for the
# exponential link at margins of about 0.5 (Poisson)
CASES = {"logistic": (lambda: synth.logistic_planted(M, N, seed=31, lam=LAM), 0.5),
         "lsq": (lambda: synth.lsq_planted(M, N, seed=32, noise=0.1, lam=LAM), 0.5),
         "poisson": (lambda: synth.poisson_planted(M, N, seed=33, lam=LAM), 0.05)}


@pytest.fixture(scope="module")
def G():
    from paper_2606_18463_gb300 import glm
    glm.load()
    return glm


@pytest.fixture(scope="module", params=list(CASES))
def case(request, G):
    make, eta = CASES[request.param]
    pr = make()
    A = torch.from_numpy(pr.A).cuda()
    y = torch.from_numpy(pr.y).cuda()
    ds_a = G.Dataset(A, y, pr.loss, "f32")
    ds_c = G.Dataset(A, y, pr.loss, "bf16")
    del A, y
    yield request.param, eta, ds_a, ds_c
    ds_a.close()
    ds_c.close()


@pytest.mark.parametrize("s", [16, 64])
def test_recipe_c_vs_a_final_loss_gap(G, case, s):
    name, eta, ds_a, ds_c = case
    for seed in range(3):
        xa = torch.zeros(N, dtype=torch.float32, device="cuda")
        xc = torch.zeros(N, dtype=torch.float32, device="cuda")
        ds_a.ca_sgd(xa, s, B, eta, LAM, H * s, seed, gram_dtype="f32")
        ds_c.ca_sgd(xc, s, B, eta, LAM, H * s, seed, gram_dtype="bf16")
        ds_a.sync()
        ds_c.sync()
        la = ds_a.loss_value(xa, LAM)
        lc = ds_a.loss_value(xc, LAM)
        gap = abs(lc - la) / abs(la)
        print(f"recipe gap {name} s={s} seed={seed}: L_A={la:.8g} L_C={lc:.8g} gap={gap:.2e}")
        assert gap <= 1e-3, (name, s, seed, la, lc, gap)


def test_long_horizon_gap(G):
    # the paper's long-horizon stress run at one GPU: logistic, b = 32, s = 16,
    # H = 320,000 outer iterations (5.12 M SGD steps), eta = 0.1; the two
    # recipes resume in segments and their losses are compared at H = 20,000,
    # 80,000 and 320,000 (the paper's mixed-precision recipes stay within
    # 1.4e-6 of the FP32 one; the bar here is 1e-5)
    pr = synth.logistic_planted(65536, 1024, seed=41, lam=0.0)
    A = torch.from_numpy(pr.A).cuda()
    y = torch.from_numpy(pr.y).cuda()
    ds_a = G.Dataset(A, y, pr.loss, "f32")
    ds_c = G.Dataset(A, y, pr.loss, "bf16")
    del A, y
    s, b, eta = 16, 32, 0.1
    xa = torch.zeros(1024, dtype=torch.float32, device="cuda")
    xc = torch.zeros(1024, dtype=torch.float32, device="cuda")
    done = 0
    try:
        for h_end in (20000, 80000, 320000):
            seg = h_end * s - done
            ds_a.ca_sgd(xa, s, b, eta, 0.0, seg, 7, gram_dtype="f32", first_iter=done)
            ds_c.ca_sgd(xc, s, b, eta, 0.0, seg, 7, gram_dtype="bf16", first_iter=done)
            ds_a.sync()
            ds_c.sync()
            done = h_end * s
            la = ds_a.loss_value(xa, 0.0)
            lc = ds_a.loss_value(xc, 0.0)
            gap = abs(lc - la) / abs(la)
            print(f"long horizon H={h_end}: L_A={la:.8g} L_C={lc:.8g} gap={gap:.2e}")
            assert gap <= 1e-5, (h_end, la, lc, gap)
    finally:
        ds_a.close()
        ds_c.close()
