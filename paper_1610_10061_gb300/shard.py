"""Client-sharded evaluation across ranks (one process per GPU).

The cost of an individual is a sum over clients (Eq. 6), and each client's
row of Pi'/Delta' depends on that client alone (the truncation to
L = m - p + 1 columns is per row, Section 2.1).  So rank r of W can hold
only the rows of its client block and evaluate, for every individual, the
partial cost over those clients; one all-reduce (sum) of the int64 partial
costs gives every rank the full costs.  The sums are integers, so the result
does not depend on the reduction order and equals the single-GPU cost bit
for bit.  This is the exchange step of client sharding: one all-reduce of
8 bytes per individual per evaluation, for instances whose tables exceed one
GPU's memory.

The GA itself is not sharded this way (it would need an all-reduce inside
every scan of a generation); the GA runs as independent replicas per rank.
"""

from __future__ import annotations

from typing import Callable, Optional

import numpy as np


def client_block(n: int, rank: int, world: int) -> tuple[int, int]:
    """The clients [lo, hi) of `rank`: contiguous blocks whose sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(int(n), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


class ShardedEvaluator:
    """Evaluate populations on this rank's client block and all-reduce the partial costs.

    d: the full n x m distance matrix (only this rank's rows are used), p: open facilities.
    group: a torch.distributed process group (None: the default group); with a single rank the
    evaluator reduces to the plain evaluation.  Each rank holds an Instance of its rows on its GPU,
    so every step of an evaluation runs in the library's kernels; the collective is torch.distributed's
    (NCCL between GPUs).  `slice_evaluator` replaces the GPU instance with another callable
    masks -> partial costs (used by tests that run the ranks on CPU).
    """

    def __init__(self, d, p: int, group=None, device: int = 0, cumulative: bool = False,
                 slice_evaluator: Optional[Callable] = None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        d = np.ascontiguousarray(d, dtype=np.int32)
        self.n, self.m = d.shape
        self.p = int(p)
        self.lo, self.hi = client_block(self.n, self.rank, self.world)
        if self.hi <= self.lo:
            raise ValueError("more ranks than clients")
        self.rows = d[self.lo:self.hi]
        if slice_evaluator is not None:
            self._eval = slice_evaluator
            self.inst = None
        else:
            from . import pm

            self.inst = pm.Instance(self.rows, self.p, device=device, cumulative=cumulative)
            self._eval = self.inst.eval

    def partial(self, masks):
        """Partial costs over this rank's clients (numpy in -> numpy out, CUDA tensor in -> CUDA tensor out)."""
        return self._eval(masks)

    def eval(self, masks):
        """Full costs of every individual, identical on every rank."""
        import torch

        part = self.partial(masks)
        t = part if isinstance(part, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(part, dtype=np.int64))
        if self.world > 1:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t if isinstance(part, torch.Tensor) else t.numpy()

    def close(self):
        if self.inst is not None:
            self.inst.close()
            self.inst = None
