"""Shot-parallel CGNR / PCGNR across ranks (one process per GPU).

Shots are independent (Sec. 3: every shot is modelled independently and the
results are reduced across processors), so a survey is split into disjoint
shot sets, one per rank. Model-space vectors are replicated; each rank applies
L and L^T to its own shots only, and the only exchanges are
  * one sum all-reduce of the two-parameter image after every L^T,
  * sum all-reduces of the FP64 data-space inner products (||q||^2, ||r||^2),
  * for PCGNR, one sum all-reduce of the pseudo-Hessian diagonal (App. B)
    before the first iteration.
The operator is any object with `born(m) -> d_local`, `adjoint(d_local) ->
g_local` on torch tensors and a `model_shape` (or `shape`) attribute: a
`Lsrtm` handle built on the rank's shots in production.

Failure detection is host-side: before every iteration each rank posts a
heartbeat key in a torch.distributed Store and waits (with a timeout) for the
other ranks' keys of the same iteration. A rank that has left is therefore
reported by the survivors as `RankFailure` before they enter the next
collective, instead of hanging in it."""
from __future__ import annotations

from datetime import timedelta

import torch
import torch.distributed as dist


class RankFailure(RuntimeError):
    """A peer rank did not reach an iteration within the heartbeat timeout."""

    def __init__(self, rank: int, iteration: int, missing: list[int]):
        super().__init__(f"rank {rank}: rank(s) {missing} did not reach CG iteration {iteration}")
        self.rank = rank
        self.iteration = iteration
        self.missing = missing


def shard(nshot: int, rank: int, world: int) -> list[int]:
    """Round-robin shot assignment: rank r owns shots r, r + world, ..."""
    return list(range(rank, nshot, world))


def _world(group=None) -> int:
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(group)
    return 1


def _allreduce(t: torch.Tensor, group=None) -> torch.Tensor:
    if _world(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def _dot(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    return (a.double() * b.double()).sum().reshape(1)


def model_shape(op) -> tuple:
    s = getattr(op, "model_shape", None)
    return tuple(s if s is not None else op.shape)


def pcg_diagonal(op, group=None, eps: float = 1e-3, local_hessian=None) -> torch.Tensor:
    """Inverse of the diagonal preconditioner M = H + eps max(H) of PCGNR,
    with H the pseudo-Hessian diagonal (App. B) summed over every rank's
    shots; replicated, [2, *shape]. `local_hessian` overrides how the rank's
    own H is obtained (default: op.pseudo_hessian())."""
    hl = op.pseudo_hessian() if local_hessian is None else local_hessian
    h = _allreduce(hl.double().clone(), group)
    inv = 1.0 / (h + eps * h.max())
    return torch.stack([inv, inv]).float()


class ShotParallelCG:
    """CGNR (CGLS form, Sec. 3) over a shot-sharded operator; with a diagonal
    preconditioner it is the PCGNR of Sec. 3."""

    def __init__(self, op, group=None, store=None, heartbeat_timeout: float = 60.0, tag: str = "lsrtm_cg"):
        self.op = op
        self.group = group
        self.store = store
        self.timeout = heartbeat_timeout
        self.tag = tag

    def adjoint(self, d_local: torch.Tensor) -> torch.Tensor:
        """Global image L^T d: local image summed over ranks."""
        return _allreduce(self.op.adjoint(d_local).clone(), self.group)

    def _store(self):
        if self.store is not None:
            return self.store
        if _world(self.group) <= 1:
            return None
        try:
            return dist.distributed_c10d._get_default_store()
        except Exception:   # no store reachable: no heartbeats
            return None

    def heartbeat(self, iteration: int):
        """Posts this rank's key for `iteration` and waits for every peer's;
        raises RankFailure naming the ranks that did not arrive in time."""
        st = self._store()
        if st is None:
            return
        rank, world = dist.get_rank(), _world(self.group)
        st.set(f"{self.tag}/{iteration}/{rank}", "1")
        keys = {r: f"{self.tag}/{iteration}/{r}" for r in range(world) if r != rank}
        try:
            st.wait(list(keys.values()), timedelta(seconds=self.timeout))
        except Exception:
            missing = []
            for r, k in keys.items():
                try:
                    st.wait([k], timedelta(milliseconds=1))
                except Exception:
                    missing.append(r)
            raise RankFailure(rank, iteration, missing or sorted(keys)) from None

    def solve(self, d_local: torch.Tensor, niter: int, x0: torch.Tensor | None = None,
              param_mask: int = 3, precond: torch.Tensor | None = None, on_iteration=None):
        """Returns the (replicated) solution and the normalised misfits
        ||d - L x_k|| / ||d||, k = 0..niter, identical on every rank.
        `precond`: replicated inverse diagonal M^-1 [2, *shape] (PCGNR), e.g.
        from pcg_diagonal. `on_iteration(k)` is called after iteration k."""
        g = self.group
        d_local = d_local.float()
        shape = model_shape(self.op)
        P = torch.zeros((2,) + shape, dtype=torch.float32, device=d_local.device)
        if param_mask & 1:
            P[0] = 1
        if param_mask & 2:
            P[1] = 1
        Minv = P if precond is None else P * precond.to(P.device).float()
        x = torch.zeros_like(P) if x0 is None else x0.float() * P
        r = d_local.clone()
        self.heartbeat(0)
        if x0 is not None:
            r -= self.op.born(x)
        dd = _allreduce(_dot(d_local, d_local), g)
        s = self.adjoint(r) * P
        z = s * Minv
        p = z.clone()
        gamma = float(_dot(s, z))
        mis = [float(torch.sqrt(_allreduce(_dot(r, r), g) / dd))]
        for k in range(niter):
            self.heartbeat(k + 1)
            q = self.op.born(p)
            qq = float(_allreduce(_dot(q, q), g))
            if qq == 0.0 or gamma == 0.0:
                mis.append(mis[-1])
            else:
                alpha = gamma / qq
                x = x + alpha * p
                r = r - alpha * q
                s = self.adjoint(r) * P
                z = s * Minv
                gnew = float(_dot(s, z))
                p = z + (gnew / gamma) * p
                gamma = gnew
                mis.append(float(torch.sqrt(_allreduce(_dot(r, r), g) / dd)))
            if on_iteration is not None:
                on_iteration(k + 1)
        return x, mis
