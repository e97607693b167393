"""Column-partitioned CA-SGD, host side, on CPU: two gloo ranks each hold a
column slab, run the outer iterations through ``partition.run_rank`` and sum
their packed [r_p | G_p] buffers with ``torch.distributed.all_reduce``.  The
ranks' steps are an FP64 numpy stand-in for libglm's glm_slab_partial /
glm_slab_finish with the same buffer layout (defined in this file, from
Algorithm 1), so the sequencing, the slab split, the buffer layout and the
collective are checked against the FP64 oracle's SGD without a GPU."""
import datetime
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _gram_ld(j, b):
    return (j * b + 3) // 4 * 4


def _gram_off(j, b):
    return sum(b * _gram_ld(t, b) for t in range(1, j))


def _dloss(loss, z, y):
    if loss == 0:
        t = y * z
        return -y / (1.0 + np.exp(t))
    return z - y


class NumpySlabOps:
    """FP64 stand-in for one rank's libglm slab steps (same red layout)."""

    def __init__(self, A_slab, y, loss, s, b, problem=0):
        import torch
        import oracle
        self.oracle, self.torch = oracle, torch
        self.A, self.y, self.loss, self.s, self.b, self.problem = A_slab, y, loss, s, b, problem
        self.sbp = (s * b + 3) // 4 * 4
        self.red = torch.zeros(self.sbp + _gram_off(s, b), dtype=torch.float64)

    def partial(self, x, seed, first_iter, sh):
        b = self.b
        idx = self.oracle.sample_indices(seed, self.problem, first_iter * b, sh * b,
                                         self.A.shape[0])
        self.Y = self.A[idx].astype(np.float64)
        self.lab = self.y[idx].astype(np.float64)
        red = np.zeros(self.red.numel())
        red[:sh * b] = self.Y @ x
        G = self.Y @ self.Y.T
        for j in range(1, sh):
            for l in range(b):
                o = self.sbp + _gram_off(j, b) + l * _gram_ld(j, b)
                red[o:o + j * b] = G[j * b + l, :j * b]
        self.red.copy_(self.torch.from_numpy(red))
        return self.red

    def finish(self, x, red, eta, lam, sh):
        b = self.b
        red = red.numpy()
        alpha, c = eta / b, 1.0 - eta * lam
        u = np.zeros(sh * b)
        for j in range(sh):
            corr = np.zeros(b)
            for l in range(b):
                o = self.sbp + _gram_off(j, b) + l * _gram_ld(j, b)
                g = red[o:o + j * b]
                w = np.array([c ** (j - 1 - i // b) for i in range(j * b)])
                corr[l] = np.dot(g * w, u[:j * b])
            z = c ** j * red[j * b:(j + 1) * b] - alpha * corr
            u[j * b:(j + 1) * b] = _dloss(self.loss, z, self.lab[j * b:(j + 1) * b])
        wts = np.repeat([c ** (sh - 1 - j) for j in range(sh)], b)
        x[:] = c ** sh * x - alpha * self.Y.T @ (wts * u)


def _worker(rank, ws, port, q, cfg):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import synth
    from paper_2606_18463_gb300 import partition
    dist.init_process_group("gloo", rank=rank, world_size=ws,
                            timeout=datetime.timedelta(seconds=30))
    pr = (synth.logistic_planted if cfg["loss"] == 0 else synth.lsq_planted)(
        cfg["m"], cfg["n"], seed=3, lam=cfg["lam"])
    c0, c1 = partition.slab_columns(cfg["n"], ws, rank)
    ops = NumpySlabOps(pr.A[:, c0:c1], pr.y, cfg["loss"], cfg["s"], cfg["b"])
    x = np.zeros(c1 - c0)
    partition.run_rank(ops, x, s=cfg["s"], eta=cfg["eta"], lam=cfg["lam"], iters=cfg["T"],
                       seed=cfg["seed"], allreduce=dist.all_reduce)
    q.put((rank, c0, c1, x))
    dist.destroy_process_group()


@pytest.mark.parametrize("cfg", [
    dict(m=400, n=13, loss=0, lam=1e-3, s=3, b=4, T=40, eta=0.5, seed=5),   # tail block
    dict(m=300, n=8, loss=1, lam=0.0, s=4, b=3, T=24, eta=0.25, seed=1),
])
def test_two_slab_ranks_equal_sgd(cfg):
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q, cfg)) for r in range(2)]
    for p in ps:
        p.start()
    out = {}
    try:
        for _ in range(2):
            item = q.get(timeout=120)
            out[item[0]] = item[1:]
    finally:
        for p in ps:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
                p.join(timeout=10)
    assert [p.exitcode for p in ps] == [0, 0]
    (a0, a1, x0), (b0, b1, x1) = out[0], out[1]
    assert (a0, a1, b0, b1) == (0, (cfg["n"] + 1) // 2, (cfg["n"] + 1) // 2, cfg["n"])
    x = np.concatenate([x0, x1])
    pr = (synth.logistic_planted if cfg["loss"] == 0 else synth.lsq_planted)(
        cfg["m"], cfg["n"], seed=3, lam=cfg["lam"])
    ref = oracle.sgd(pr.A, pr.y, cfg["loss"], cfg["b"], cfg["eta"], cfg["lam"], cfg["T"],
                     cfg["seed"])
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)


def test_slab_columns_and_blocks():
    from paper_2606_18463_gb300 import partition
    for n, P in [(13, 2), (13, 3), (512, 16), (7, 7)]:
        cuts = [partition.slab_columns(n, P, r) for r in range(P)]
        assert cuts[0][0] == 0 and cuts[-1][1] == n
        assert all(cuts[r][1] == cuts[r + 1][0] for r in range(P - 1))
        sizes = [c1 - c0 for c0, c1 in cuts]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        partition.slab_columns(3, 4, 0)
    assert list(partition.outer_blocks(5, 10, 4)) == [(5, 4), (9, 4), (13, 2)]
