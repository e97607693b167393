"""First-order local error budget of one CA-SGD outer step (Sec. 5.2: the
amplification factor K_s, the source quantities T_g, T_r, T_G, T_c and the
nine terms of Theorem 1), and a simulator of that outer step in which every
operation is rounded at its own precision.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the product path never
imports it.  Plain FP64 numpy throughout.

Notation (Sec. 5.2).  Y (sb x n) holds the sampled rows in the inner-step
blocks Y_0 .. Y_{s-1} of b rows each, alpha = eta / b, and d = (d_0; ...;
d_{s-1}) is the exact residual history delta = -dL/dr along the s inner steps
that start from the common iterate x.  G = Y Y^T, G_L is its strictly
block-lower part and H_L the strictly block-lower part of |Y| |Y|^T.  The
theorem has no ridge term: the budget is for lambda = 0.  It covers the
Lipschitz-residual losses (logistic with L_sigma = 1/4, least squares with
L_sigma = 1); Poisson lies outside it.

Slots (Sec. 3, the nine operations of an outer step): u_A storage of Y, the
margin GEMV (factor gamma_r), the Gram (gamma_G), the correction recurrence
u_c, the residual u_sigma, the gradient GEMV (gamma_g), the master weights
u_x, and the two all-reduces (C(P) u_AR,r and C(P) u_AR,G; zero on one GPU).
The simulator can split the columns over P ranks to exercise the last two.

Parity status (pins in ``tests/test_oracle_local_error.py``):
  fl .............. pinned (numpy's float32 and float16 casts, the BF16 rounding).
  exact_step ...... pinned (the C oracle's SGD on the same index stream; the
                    residual against the C oracle's loss derivative).
  simulate_step ... pinned (without rounding it equals exact_step: CA-SGD and
                    SGD agree in exact arithmetic; one rank needs no reduction).
  local_error ..... pinned (K_s by the terminating Neumann series and a 2 x 2
                    closed form; H_L, T_g, T_r, T_G, T_c by element loops;
                    each term bounds the deviation the simulator shows with
                    its slot alone rounded, sits within a fixed factor of it
                    under directed rounding, and equals it to first order in
                    cases where every inequality behind the term is tight;
                    all slots together stay within the first-order sum; the
                    two all-reduce terms likewise, against a simulation over
                    P ranks).  The factor K_s in E_sigma, which no case makes
                    tight (the residual's slope reaches L_sigma only near zero
                    margin, its size reaches D_delta only far from it), is
                    pinned by a case with amplifying inner steps (alpha a^2 =
                    3) whose deviation exceeds the term without K_s.
"""
from __future__ import annotations

import math

import numpy as np

LOGISTIC, LSQ = 0, 1

# L_sigma, the Lipschitz constant of the residual in the margin (Assumption 2)
LIPSCHITZ = {LOGISTIC: 0.25, LSQ: 1.0}

SLOTS = ("A", "r", "G", "c", "sigma", "g", "x", "AR_r", "AR_G")


# --------------------------------------------------------------------------
# Rounding model (Sec. 3: fl_u(x op y) = (x op y)(1 + theta), |theta| <= u)
# --------------------------------------------------------------------------
def fl(v, p, mode: str = "nearest"):
    """v rounded to p significant bits with an unbounded exponent range.
    ``mode`` 'nearest' (ties to even; unit roundoff 2^-p) or 'up' (toward
    +infinity; every error at most one ulp, 2^(1-p) relative); 'model' is
    the rounding model's extreme case v (1 + u) with u = 2^-p, every
    operation off by the full unit roundoff in the same direction (Sec. 3).
    p None returns v unchanged (exact FP64)."""
    if p is None:
        return v
    v = np.asarray(v, dtype=np.float64)
    if mode == "model":
        return v * (1.0 + math.ldexp(1.0, -p))
    m, e = np.frexp(v)  # v = m 2^e with 1/2 <= |m| < 1
    q = np.ldexp(m, p)
    q = np.rint(q) if mode == "nearest" else np.ceil(q)
    return np.ldexp(q, e - p)


def unit_roundoff(p: int, mode: str = "nearest") -> float:
    return math.ldexp(1.0, 1 - p if mode == "up" else -p)


def gamma(q: int, u: float) -> float:
    """Higham factor gamma_q = q u / (1 - q u) (Sec. 3); needs q u < 1."""
    qu = q * u
    if qu >= 1.0:
        raise ValueError(f"gamma_{q} outside its domain (q u = {qu})")
    return qu / (1.0 - qu)


def gamma_mixed(q: int, u_in: float, u_acc: float) -> float:
    """Factor of a length-q inner product whose two inputs are rounded at
    u_in and whose accumulation runs at u_acc: 2 u_in + gamma_q(u_acc) (the
    BF16-input / FP32-accumulate factor of Sec. 5.2)."""
    return 2.0 * u_in + gamma(q, u_acc)


# --------------------------------------------------------------------------
# The exact outer step
# --------------------------------------------------------------------------
def residual(loss: int, z, y):
    """delta(r, y) = -dL/dr (Sec. 3.1): y (1 - sigma(y r)) = y sigma(-y r) for
    logistic labels in {-1, +1}, y - r for least squares."""
    z = np.asarray(z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if loss == LOGISTIC:
        t = y * z
        e = np.exp(-np.abs(t))
        return y * np.where(t >= 0, e / (1.0 + e), 1.0 / (1.0 + e))
    if loss == LSQ:
        return y - z
    raise ValueError("the local error budget covers logistic and least-squares losses")


def exact_step(Y, yI, x, loss: int, eta: float, s: int, b: int):
    """The exact outer step from x: s mini-batch SGD steps, step j on the
    rows Y_j (Algorithm 1 in exact arithmetic).  Returns (z, d, xs): the
    stacked margins z_j = Y_j x_j, the residual history d_j = delta(z_j) and
    the inner iterates x_0 .. x_s."""
    Y = np.asarray(Y, dtype=np.float64)
    yI = np.asarray(yI, dtype=np.float64)
    alpha = eta / b
    xj = np.array(x, dtype=np.float64)
    xs = [xj.copy()]
    z = np.empty(s * b)
    d = np.empty(s * b)
    for j in range(s):
        rows = slice(j * b, (j + 1) * b)
        z[rows] = Y[rows] @ xj
        d[rows] = residual(loss, z[rows], yI[rows])
        xj = xj + alpha * (Y[rows].T @ d[rows])
        xs.append(xj.copy())
    return z, d, xs


# --------------------------------------------------------------------------
# The outer step with each operation rounded at its slot's precision
# --------------------------------------------------------------------------
def _dot_rows(U, v, p, mode):
    """U @ v by recursive summation over the columns of U, each product and
    each of the q - 1 partial sums rounded to p bits (p None: the exact FP64
    product; no columns: zeros)."""
    if p is None or U.shape[1] == 0:
        return U @ v
    acc = fl(U[:, 0] * v[0], p, mode)
    for k in range(1, U.shape[1]):
        acc = fl(acc + fl(U[:, k] * v[k], p, mode), p, mode)
    return acc


def _gram(Y, p, mode):
    if p is None:
        return Y @ Y.T
    acc = fl(np.outer(Y[:, 0], Y[:, 0]), p, mode)
    for k in range(1, Y.shape[1]):
        acc = fl(acc + fl(np.outer(Y[:, k], Y[:, k]), p, mode), p, mode)
    return acc


def _allreduce(parts, p, mode):
    """Sum of the ranks' partial arrays, rank by rank, each addition rounded
    to p bits: |error| <= gamma_{P-1} sum_p |part_p| (one rank: no rounding)."""
    acc = parts[0]
    for v in parts[1:]:
        acc = fl(acc + v, p, mode)
    return acc


def simulate_step(Y, yI, x, loss: int, eta: float, s: int, b: int, prec=None,
                  mode: str = "nearest", P: int = 1):
    """One CA-SGD outer step from x in the order of the outer iteration of
    Sec. 4 (Algorithm 1): rows stored (slot A), base margins r = Y x (r),
    Gram G = Y Y^T (G), then for each inner step j the correction
    z_j = r_j + alpha sum_{i<j} G_{j,i} d_i (c) and the residual
    d_j = delta(z_j) (sigma), the gradient Y^T d (g) and the update
    x + alpha Y^T d (x).  ``prec`` maps a slot name to the bits its
    operations keep; a missing slot is exact.  lambda = 0.

    With P > 1 the columns are split into P contiguous slabs, one per rank
    (the paper's 1D block-column partition): each rank forms its partial
    margins and Gram over its slab, and the all-reduces sum them rank by rank
    (slots AR_r and AR_G).  The gradient and the update of each slab stay on
    its rank and need no reduction."""
    prec = dict(prec or {})
    bad = set(prec) - set(SLOTS)
    if bad:
        raise ValueError(f"unknown slots {sorted(bad)}")
    bits = lambda k: prec.get(k)  # noqa: E731
    alpha = eta / b
    Y = fl(np.asarray(Y, dtype=np.float64), bits("A"), mode)
    yI = np.asarray(yI, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    slabs = np.array_split(np.arange(Y.shape[1]), P)
    r = _allreduce([_dot_rows(Y[:, c], x[c], bits("r"), mode) for c in slabs],
                   bits("AR_r"), mode)
    G = _allreduce([_gram(Y[:, c], bits("G"), mode) for c in slabs], bits("AR_G"), mode)
    d = np.zeros(s * b)
    pc = bits("c")
    for j in range(s):
        rows = slice(j * b, (j + 1) * b)
        if j == 0:
            z = r[rows]
        else:
            t = _dot_rows(G[rows, :j * b], d[:j * b], pc, mode)
            z = fl(r[rows] + fl(alpha * t, pc, mode), pc, mode)
        d[rows] = fl(residual(loss, z, yI[rows]), bits("sigma"), mode)
    g = _dot_rows(Y.T, d, bits("g"), mode)
    px = bits("x")
    return fl(x + fl(alpha * g, px, mode), px, mode)


# --------------------------------------------------------------------------
# Theorem 1: the nine first-order terms
# --------------------------------------------------------------------------
def local_error(Y, yI, x, loss: int, eta: float, s: int, b: int, *,
                u_A: float = 0.0, gamma_r: float = 0.0, gamma_G: float = 0.0,
                u_c: float = 0.0, u_sigma: float = 0.0, gamma_g: float = 0.0,
                u_x: float = 0.0, cP_u_AR_r: float = 0.0, cP_u_AR_G: float = 0.0,
                C_delta: float = 1.0, R: float | None = None) -> dict:
    """The nine terms E_* of Theorem 1 for one outer step from x on the rows
    Y with labels yI, with the slot factors given (unit roundoffs u_*, kernel
    factors gamma_*, and C(P) u_AR,* for the two all-reduces), together with
    the quantities they are made of and the hypothesis figures omega, tau_G
    and Omega = max(omega, tau_G) (the theorem asks omega, tau_G <= 1/2; the
    remainder is at most C_loc Omega sum E_*).

    R bounds the iterates of the step (Assumption 5; default: the largest
    norm of the exact inner iterates) and enters D_delta = max|y| + R for
    least squares; D_delta = 1 for logistic (Assumption 2).  C_delta is the
    residual's rounding constant, |fl(delta) - delta| <= C_delta u D_delta."""
    if loss not in LIPSCHITZ:
        raise ValueError("the local error budget covers logistic and least-squares losses")
    Y = np.asarray(Y, dtype=np.float64)
    yI = np.asarray(yI, dtype=np.float64)
    sb = s * b
    if Y.shape[0] != sb or yI.shape[0] != sb:
        raise ValueError("Y and yI must hold s b rows")
    alpha = eta / b
    L = LIPSCHITZ[loss]
    z, d, xs = exact_step(Y, yI, x, loss, eta, s, b)
    x_s = xs[-1]

    blk = np.arange(sb) // b
    lower = blk[:, None] > blk[None, :]  # strictly block-lower
    G = Y @ Y.T
    G_L = np.where(lower, G, 0.0)
    aY = np.abs(Y)
    H_L = np.where(lower, aY @ aY.T, 0.0)
    # K_s (Eq. for the triangular amplification); unit lower triangular
    K_s = float(np.linalg.norm(np.linalg.inv(np.eye(sb) - L * alpha * np.abs(G_L)), 2))
    norm_Y = float(np.linalg.norm(Y, 2))
    norm_H_L = float(np.linalg.norm(H_L, 2))

    ad = np.abs(d)
    T_g = float(np.linalg.norm(aY.T @ ad))
    T_r = float(np.linalg.norm(aY @ np.abs(np.asarray(x, dtype=np.float64))))
    T_G = float(np.linalg.norm(H_L @ ad))
    T_c = math.sqrt(sum((j * b * np.linalg.norm(G[j * b:(j + 1) * b, :j * b])
                         * np.linalg.norm(d[:j * b])) ** 2 for j in range(1, s)))

    if R is None:
        R = max(float(np.linalg.norm(v)) for v in xs)
    D_delta = 1.0 if loss == LOGISTIC else float(np.max(np.abs(yI))) + R

    a = alpha * norm_Y * K_s * L
    E = {
        "E_A": a * u_A * T_r + 2 * alpha * a * u_A * T_G + alpha * u_A * T_g,
        "E_r": a * gamma_r * T_r,
        "E_AR_r": a * cP_u_AR_r * T_r,
        "E_G": alpha * a * gamma_G * T_G,
        "E_AR_G": alpha * a * cP_u_AR_G * T_G,
        "E_c": a * u_c * T_r + 2 * alpha * a * u_c * T_G + alpha * a * u_c * T_c,
        "E_sigma": alpha * norm_Y * K_s * C_delta * u_sigma * D_delta * math.sqrt(sb),
        "E_g": alpha * gamma_g * T_g,
        "E_x": u_x * (float(np.linalg.norm(x_s)) + alpha * float(np.linalg.norm(Y.T @ d))),
    }
    omega = max(u_A, gamma_r, gamma_G, gamma((s - 1) * b, u_c), gamma_g, cP_u_AR_r,
                cP_u_AR_G, u_sigma, u_x)
    tau_G = K_s * L * alpha * (2 * u_A + gamma_G + cP_u_AR_G) * norm_H_L
    out = dict(E)
    out.update(sum=sum(E.values()), K_s=K_s, norm_Y=norm_Y, norm_H_L=norm_H_L, T_g=T_g,
               T_r=T_r, T_G=T_G, T_c=T_c, omega=omega, tau_G=tau_G,
               Omega=max(omega, tau_G), D_delta=D_delta, L_sigma=L, R=R, x_s=x_s, d=d, z=z)
    return out
