"""Host side of column-partitioned CA-SGD (paper Algorithm 1 on P ranks, the
1D block-column partition of Sec. 4 with one grouped AllReduce of the
partial margins and the strictly block-lower Gram per outer iteration).

Argument marshalling and sequencing only: the gather, the partial margins
and Gram, the recurrence and the update run in libglm's kernels
(glm_slab_partial / glm_slab_finish); the sum over ranks is the caller's
collective (``torch.distributed.all_reduce`` of the packed buffer, over NCCL
or gloo) or, for ranks emulated on one device, ``glm_sum_buffers``.
"""
from __future__ import annotations


def slab_columns(n: int, P: int, rank: int):
    """Columns [c0, c1) of rank `rank`: contiguous slabs whose sizes differ by
    at most one, the larger ones first."""
    if not (0 <= rank < P) or n < P:
        raise ValueError("need 0 <= rank < P <= n")
    q, r = divmod(n, P)
    c0 = rank * q + min(rank, r)
    return c0, c0 + q + (1 if rank < r else 0)


def outer_blocks(first_iter: int, iters: int, s: int):
    """(first SGD-equivalent iteration, inner steps) of each outer iteration
    of a run of `iters` iterations starting at `first_iter`."""
    t = first_iter
    end = first_iter + iters
    while t < end:
        sh = min(s, end - t)
        yield t, sh
        t += sh


class SlabOps:
    """One rank's steps on a libglm dataset handle over its column slab."""

    def __init__(self, ds, s: int, b: int, **opts):
        import torch
        from . import glm
        self.glm, self.ds, self.s, self.b = glm, ds, s, b
        self.opts = glm.default_ca_opts(**opts) if opts else None
        self.red = torch.zeros(glm.glm_slab_reduce_floats(s, b), dtype=torch.float32,
                               device="cuda")

    def partial(self, x, seed: int, first_iter: int, sh: int):
        self.glm.glm_slab_partial(self.ds.h, self.s, self.b, sh, seed, first_iter, x, self.red,
                                  self.opts)
        return self.red

    def finish(self, x, red, eta: float, lam: float, sh: int):
        self.glm.glm_slab_finish(self.ds.h, self.s, self.b, sh, eta, lam, red, x, self.opts)


def run_rank(ops, x, *, s: int, eta: float, lam: float, iters: int, seed: int, allreduce,
             first_iter: int = 0):
    """This rank's part of a run: per outer iteration its partial buffer,
    the collective sum `allreduce(red)` (in place), then the recurrence and
    the slab's update."""
    for t, sh in outer_blocks(first_iter, iters, s):
        red = ops.partial(x, seed, t, sh)
        allreduce(red)
        ops.finish(x, red, eta, lam, sh)


def run_emulated(ops_list, xs, *, s: int, eta: float, lam: float, iters: int, seed: int,
                 first_iter: int = 0, stream=None):
    """P ranks on one device: every rank's partial, one summed buffer
    (glm_sum_buffers in rank order), every rank's finish on that sum."""
    glm = ops_list[0].glm
    total = ops_list[0].red.clone()
    for t, sh in outer_blocks(first_iter, iters, s):
        reds = [ops.partial(x, seed, t, sh) for ops, x in zip(ops_list, xs)]
        # the handles may run on different streams: the sum waits for all
        for ops in ops_list:
            ops.ds.stream.synchronize()
        glm.glm_sum_buffers(total, reds, total.numel(),
                            stream.cuda_stream if stream is not None else None)
        if stream is not None:
            stream.synchronize()
        else:
            import torch
            torch.cuda.synchronize()
        for ops, x in zip(ops_list, xs):
            ops.finish(x, total, eta, lam, sh)
        for ops in ops_list:
            ops.ds.stream.synchronize()
