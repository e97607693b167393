"""One-GPU analogues of the paper's recipe checks (Sec. "Accuracy gap").

Validation table: the relative final-loss gap |L_X - L_A| / |L_A| between a
mixed-precision recipe X and the FP32 recipe A at (m, n) = (65,536, 4,096),
b = 32, s in {16, 64}, H = 200 outer iterations, three seeds, for logistic,
least-squares and Poisson losses.  The paper's cells (Recipe C, P = 16, its
own synthetic data) are at most 3.3e-4 against a 0.5 % threshold; the bar
here is the 1e-3 final-loss target.

Long horizon: logistic, b = 32, s = 16, eta = 0.1, H = 320,000; the paper's
Recipes A-G stay within 1.4e-6 of A; the bar here is 1e-5.

Recipes at P = 1 (precision-symbol table, Sec. 5.3; the all-reduce slots drop
out, so D coincides with C), with FP32 accumulation in every kernel and the
recurrence as the library sets it (FP32, FP64 at s >= 32; finer than G's
TF32 recurrence):
  B  BF16 storage (per-column scales), FP32 Gram and GEMV operands;
  C  BF16 storage, BF16 operands;
  E  FP16 storage (per-column scales), FP16 operands;
  G  FP32 storage, TF32 operands.
The data are synthetic stand-ins with the paper's shape (rows of about unit
norm); every loss is evaluated on the FP32 data.
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


# recipe -> (storage, Gram and GEMV operands)
RECIPES = {"A": ("f32", "f32"), "B": ("bf16", "f32"), "C": ("bf16", "bf16"),
           "E": ("f16", "f16"), "G": ("f32", "tf32")}


def _datasets(G, pr):
    A = torch.from_numpy(pr.A).cuda()
    y = torch.from_numpy(pr.y).cuda()
    ds = {st: G.Dataset(A, y, pr.loss, st) for st in ("f32", "bf16", "f16")}
    del A, y
    return ds


@pytest.fixture(scope="module", params=list(CASES))
def case(request, G):
    make, eta = CASES[request.param]
    ds = _datasets(G, make())
    yield request.param, eta, ds
    for d in ds.values():
        d.close()


@pytest.mark.parametrize("recipe", ["B", "C", "E", "G"])
@pytest.mark.parametrize("s", [16, 64])
def test_recipe_vs_a_final_loss_gap(G, case, s, recipe):
    name, eta, ds = case
    st, op = RECIPES[recipe]
    for seed in range(3):
        xa = torch.zeros(N, dtype=torch.float32, device="cuda")
        xc = torch.zeros(N, dtype=torch.float32, device="cuda")
        ds["f32"].ca_sgd(xa, s, B, eta, LAM, H * s, seed, gram_dtype="f32")
        ds[st].ca_sgd(xc, s, B, eta, LAM, H * s, seed, gram_dtype=op)
        ds["f32"].sync()
        ds[st].sync()
        la = ds["f32"].loss_value(xa, LAM)
        lc = ds["f32"].loss_value(xc, LAM)
        gap = abs(lc - la) / abs(la)
        print(f"recipe {recipe} gap {name} s={s} seed={seed}: L_A={la:.8g} "
              f"L_{recipe}={lc:.8g} gap={gap:.2e}")
        assert gap <= 1e-3, (recipe, name, s, seed, la, lc, gap)


def test_long_horizon_gap(G):
    # the paper's long-horizon stress run at one GPU: logistic, b = 32, s = 16,
    # H = 320,000 outer iterations (5.12 M SGD steps), eta = 0.1; every recipe
    # resumes in segments and its loss is compared with A's at H = 20,000,
    # 80,000 and 320,000 (the paper's Recipes A-G stay within 1.4e-6 of A;
    # the bar here is 1e-5)
    pr = synth.logistic_planted(65536, 1024, seed=41, lam=0.0)
    ds = _datasets(G, pr)
    s, b, eta = 16, 32, 0.1
    xs = {r: torch.zeros(1024, dtype=torch.float32, device="cuda") for r in RECIPES}
    done = 0
    try:
        for h_end in (20000, 80000, 320000):
            seg = h_end * s - done
            for r, (st, op) in RECIPES.items():
                ds[st].ca_sgd(xs[r], s, b, eta, 0.0, seg, 7, gram_dtype=op, first_iter=done)
            for d in ds.values():
                d.sync()
            done = h_end * s
            la = ds["f32"].loss_value(xs["A"], 0.0)
            for r in RECIPES:
                if r == "A":
                    continue
                lr = ds["f32"].loss_value(xs[r], 0.0)
                gap = abs(lr - la) / abs(la)
                print(f"long horizon H={h_end} recipe {r}: L_A={la:.8g} L_{r}={lr:.8g} "
                      f"gap={gap:.2e}")
                assert gap <= 1e-5, (r, h_end, la, lr, gap)
    finally:
        for d in ds.values():
            d.close()
