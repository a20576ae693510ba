"""Data-parallel NBM training: one process per GPU, one exchange per step.

Sec. 3 of the paper makes multi-GPU training of the NBM plain data
parallelism: every step's collocation points are independent, so they are
distributed over the processors and the locally computed gradients are
aggregated.  Here a step's batch of ``n_total`` points is split into
contiguous shards, one per rank (``shard_range``).  Each rank

1. computes its shard's contribution to the loss and gradient on its GPU
   (``nbm_loss_grad_shard``: the points are drawn on the device at the
   counters the whole batch would give them, and both results are already
   scaled by 1/n_total);
2. sums the P-float gradient and the FP64 loss over the ranks (one
   all-reduce each; these are the step's only exchange);
3. applies the same Adam update to its own replica of the parameters
   (``nbm_adam_step``), so the replicas stay identical.

The sums over a partition of the batch are the whole batch's gradient and
loss up to the order of the FP32 additions, and one rank reproduces
``nbm_train_steps`` bitwise.  All arithmetic runs in libnbm; this module only
orders the calls and the collectives.
"""
from __future__ import annotations

import torch


def shard_range(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """(first, n) of rank `rank`'s contiguous shard of an n_total-point batch:
    the first n_total mod world ranks take one point more, and the shards
    partition [0, n_total) in rank order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    if n_total < world:
        raise ValueError("every rank needs at least one point")
    base, extra = divmod(n_total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


class DataParallelTrainer:
    """Adam training of one NBM problem over the ranks of a process group.

    problem      a ``Problem`` on this rank's device (or any object with the
                 same ``loss_grad_shard`` / ``adam_step`` methods)
    params, m, v this rank's replica of the parameters and Adam moments
                 (identical on every rank at the start)
    n_total      points per step over all ranks
    all_reduce   sums a tensor over the ranks in place; None: no exchange
                 (a single rank)

    ``step()`` runs one training step and returns the device tensor that holds
    the step's whole-batch loss (before the update)."""

    def __init__(self, problem, params, m, v, n_total, rank=0, world=1, all_reduce=None,
                 seed=1, step=0, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        if world > 1 and all_reduce is None:
            raise ValueError("more than one rank needs an all_reduce")
        self.problem = problem
        self.params, self.m, self.v = params, m, v
        self.n_total = int(n_total)
        self.rank, self.world = rank, world
        self.first, self.n = shard_range(self.n_total, world, rank)
        self.all_reduce = all_reduce
        self.seed, self.t = seed, int(step)
        self.lr, self.beta1, self.beta2, self.eps = lr, beta1, beta2, eps
        self.grad = torch.empty_like(params)
        self.loss = torch.zeros(1, dtype=torch.float64, device=params.device)

    def step(self, pts=None):
        """One step: this rank's shard (drawn on the device at counter t + 1,
        or `pts`, this shard's [n][3] points), the all-reduce of gradient and
        loss, and the replicated Adam update."""
        self.problem.loss_grad_shard(self.params, self.n_total, self.first, self.n,
                                     seed=self.seed, step=self.t + 1, pts=pts, grad=self.grad,
                                     loss=self.loss)
        if self.all_reduce is not None:
            self.all_reduce(self.grad)
            self.all_reduce(self.loss)
        self.t = self.problem.adam_step(self.params, self.m, self.v, self.grad, self.t,
                                        lr=self.lr, beta1=self.beta1, beta2=self.beta2,
                                        eps=self.eps, loss=self.loss)
        return self.loss


def torch_all_reduce(group=None):
    """An all_reduce (sum) over a torch.distributed process group.  Tensors on
    a GPU go to NCCL directly; a gloo group receives a host copy that is copied
    back after the sum."""
    import torch.distributed as dist

    backend = dist.get_backend(group)

    def reduce(t):
        if t.is_cuda and backend == "gloo":
            h = t.cpu()
            dist.all_reduce(h, group=group)
            t.copy_(h)
        else:
            dist.all_reduce(t, group=group)
    return reduce
