"""Data-parallel training by points across GPUs, one process per GPU (torch.distributed).

Every rank holds a full replica of the tables and the network.  A step of G ranks trains on G
batches of P points, one per rank (the union is one batch of G P points): each rank runs the
encoding forward, the network forward + L2 loss + backward and the encoding backward on its own
points, into one flat binary32 buffer [table gradient | network gradient | squared-residual sum];
one all-reduce averages that buffer over the ranks -- the step's only exchange -- and every rank
then applies the same Adam update to the same gradient, so the replicas stay identical.

Averaging gives exactly the gradient of the union batch: each rank's L2 gradient is
2 (y - t) / (P n_out) over its own P points, and the mean over G ranks of those sums is
2 (y - t) / (G P n_out) summed over all G P points.  The mean of the ranks' squared-residual sums
over P n_out is the union's loss.  On NCCL the average is the collective's own AVG reduction;
where a backend has no AVG (gloo) it is a sum followed by a division by G (exact for G a power of
two).

The table gradient must be one dense array for the exchange, so the tables use the dense layout
(separate binary32 parameter, moment and gradient arrays); the interleaved records would mix the
gradient with state that must not be summed.  Forward-only serving needs no exchange (replicas).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(n: int, rank: int, world: int) -> slice:
    """Rank ``rank``'s contiguous share of n items split over ``world`` ranks (the first n % world
    ranks take one item more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return slice(lo, lo + base + (1 if rank < extra else 0))


def allreduce_mean(buf: torch.Tensor, group=None) -> None:
    """Average ``buf`` over the ranks of ``group`` in place (nothing to do for one rank)."""
    if not dist.is_available() or not dist.is_initialized():
        return
    world = dist.get_world_size(group)
    if world == 1:
        return
    if dist.get_backend(group) == "nccl":
        dist.all_reduce(buf, op=dist.ReduceOp.AVG, group=group)
    else:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
        buf.div_(world)


class DataParallelStep:
    """One data-parallel step, independent of where the per-rank work runs.

    ``local(x, target)`` writes this rank's gradients of its batch into ``flat`` (overwriting the
    squared-residual sum, accumulating into zeroed gradients); ``apply()`` runs the optimiser on
    the averaged ``flat`` and leaves its gradient parts zero for the next step."""

    def __init__(self, flat: torch.Tensor, local, apply, group=None):
        self.flat, self.local, self.apply, self.group = flat, local, apply, group

    def step(self, x, target) -> None:
        self.local(x, target)
        allreduce_mean(self.flat, self.group)
        self.apply()


class DataParallelTrainer:
    """``trainer.Trainer`` replicated across the ranks of ``group``: the same seeded tables and
    network on every rank, ``batch`` points per rank and step, the exchange of
    ``DataParallelStep`` between the backward passes and Adam.  All device work runs in the
    library's kernels on the current stream; the all-reduce runs on torch.distributed's stream
    after the backward's kernels (NCCL orders it after the current stream's work)."""

    def __init__(self, encoder, mlp, batch: int, *, group=None, seed: int = 0, device="cuda", **kw):
        from .trainer import Trainer
        tr = self.tr = Trainer(encoder, mlp, batch, seed=seed, device=device, table_layout="dense", **kw)
        n_tab, n_w = tr.tab.grad.numel(), tr.dW.numel()
        self.flat = torch.zeros((n_tab + n_w + 1,), dtype=torch.float32, device=tr.device)
        tr.tab.grad = self.flat[:n_tab]
        tr.dW = self.flat[n_tab:n_tab + n_w]
        tr.sq_sum = tr.sq_parts = self.flat[n_tab + n_w:]
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
        self._step = DataParallelStep(self.flat, self._local, self._apply, group)

    def _local(self, x, target) -> None:
        tr = self.tr
        tr.t += 1
        tr.adam_tables.advance(tr.t_dev, tr.corrections)
        self.local_grads(x, target)

    def local_grads(self, x, target) -> None:
        """This rank's part of a step: encoding, network + L2 loss + backward, encoding backward,
        into ``flat`` (the squared-residual sum overwritten, the gradients accumulated)."""
        tr = self.tr
        tr.tab.forward(x, tr.enc_out)
        tr.mlp.mlp_train_l2(tr.W_lowp, tr.enc_out, target, tr.dW, tr.sq_sum, din=tr.d_enc,
                            loss_scale=tr.loss_scale, workspace=tr.ws)
        tr.tab.backward(x, tr.d_enc)

    def apply(self) -> None:
        """Adam on the averaged gradients in ``flat`` (identical on every rank); zeroes them."""
        self._apply()

    def _apply(self) -> None:
        tr = self.tr
        tr.tab.adam(tr.adam_tables, tr.corrections)
        tr.adam_mlp.step_dev(tr.corrections, tr.W, tr.mW, tr.vW, tr.dW, lowp=tr.W_lowp)

    def step(self, x: torch.Tensor, target: torch.Tensor) -> None:
        """One step on this rank's batch (x [P, d], target [P, n_out], on this rank's device)."""
        self._step.step(x, target)

    def loss(self) -> float:
        """Mean squared error of the last step over every rank's points (synchronises)."""
        return self.tr.loss()
