"""Shot-parallel CGNR across ranks (one process per GPU).

Shots are independent (Sec. 3: every shot is modelled independently and the
results are reduced across processors), so a survey is split into disjoint
shot sets, one per rank. Model-space vectors are replicated; each rank applies
L and L^T to its own shots only, and the only exchanges are
  * one sum all-reduce of the two-parameter image after every L^T, and
  * sum all-reduces of the FP64 data-space inner products (||q||^2, ||r||^2).
The operator is any object with `born(m) -> d_local` and
`adjoint(d_local) -> g_local` on torch tensors (a `Lsrtm` handle built on the
rank's shots in production)."""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(nshot: int, rank: int, world: int) -> list[int]:
    """Round-robin shot assignment: rank r owns shots r, r + world, ..."""
    return list(range(rank, nshot, world))


def _allreduce(t: torch.Tensor, group=None) -> torch.Tensor:
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def _dot(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    return (a.double() * b.double()).sum().reshape(1)


class ShotParallelCG:
    """CGNR (CGLS form, Sec. 3) over a shot-sharded operator."""

    def __init__(self, op, group=None):
        self.op = op
        self.group = group

    def adjoint(self, d_local: torch.Tensor) -> torch.Tensor:
        """Global image L^T d: local image summed over ranks."""
        return _allreduce(self.op.adjoint(d_local).clone(), self.group)

    def solve(self, d_local: torch.Tensor, niter: int, x0: torch.Tensor | None = None,
              param_mask: int = 3):
        """Returns the (replicated) solution and the normalised misfits
        ||d - L x_k|| / ||d||, k = 0..niter, identical on every rank."""
        g = self.group
        d_local = d_local.float()
        shape = self.op.model_shape
        P = torch.zeros((2,) + tuple(shape), dtype=torch.float32, device=d_local.device)
        if param_mask & 1:
            P[0] = 1
        if param_mask & 2:
            P[1] = 1
        x = torch.zeros_like(P) if x0 is None else x0.float() * P
        r = d_local.clone()
        if x0 is not None:
            r -= self.op.born(x)
        dd = _allreduce(_dot(d_local, d_local), g)
        s = self.adjoint(r) * P
        p = s.clone()
        gamma = float(_dot(s, s))
        mis = [float(torch.sqrt(_allreduce(_dot(r, r), g) / dd))]
        for _ in range(niter):
            q = self.op.born(p)
            qq = float(_allreduce(_dot(q, q), g))
            if qq == 0.0 or gamma == 0.0:
                mis.append(mis[-1])
                continue
            alpha = gamma / qq
            x = x + alpha * p
            r = r - alpha * q
            s = self.adjoint(r) * P
            gnew = float(_dot(s, s))
            p = s + (gnew / gamma) * p
            gamma = gnew
            mis.append(float(torch.sqrt(_allreduce(_dot(r, r), g) / dd)))
        return x, mis
