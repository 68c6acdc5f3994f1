"""Shot-parallel CGNR over two gloo ranks on CPU equals the single-process
CGNR over all shots. The operator here is the FP64 oracle restricted to each
rank's shots (test infrastructure); the production operator is a GPU handle
built on the same shot subset."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import lsrtm_inputs as li
import oracle


class _OracleShots:
    def __init__(self, w, shots):
        self.w = w
        self.geom = w.geom.subset(shots)
        self.model_shape = w.shape

    def pseudo_hessian(self):
        return torch.tensor(oracle.pseudo_hessian(self.w, geom=self.geom), dtype=torch.float64)

    def born(self, m):
        return torch.tensor(oracle.born(self.w, m.double().numpy(), geom=self.geom), dtype=torch.float32)

    def adjoint(self, d):
        return torch.tensor(oracle.adjoint(self.w, d.double().numpy(), geom=self.geom), dtype=torch.float32)


def _case():
    return li.small_case(nz=18, nx=22, nt=90, order=4, npml=5, nshot=5, seed=77)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _local(w, rank, world):
    from paper_2508_10405_gb300.distributed import shard
    shots = shard(w.geom.nshot, rank, world)
    d_all = oracle.born(w, w.dm)
    rows = np.concatenate([np.arange(w.geom.rec_ptr[s], w.geom.rec_ptr[s + 1]) for s in shots])
    return _OracleShots(w, shots), torch.tensor(d_all[rows], dtype=torch.float32)


def _worker(rank, world, port, out, precond):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2508_10405_gb300.distributed import ShotParallelCG, pcg_diagonal
    w = _case()
    op, d_local = _local(w, rank, world)
    minv = pcg_diagonal(op) if precond else None
    x, mis = ShotParallelCG(op).solve(d_local, 4, precond=minv)
    out[rank] = (x.numpy(), np.asarray(mis))
    dist.barrier()
    dist.destroy_process_group()


def _leaving_worker(rank, world, port, out):
    """Rank 1 leaves after CG iteration 2 (between iterations, with none of
    its collectives in flight); rank 0 must report it at iteration 3."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2508_10405_gb300.distributed import RankFailure, ShotParallelCG
    w = _case()
    op, d_local = _local(w, rank, world)

    def leave(k):
        if rank == 1 and k == 2:
            out[rank] = ("left", k)
            os._exit(0)

    try:
        ShotParallelCG(op, heartbeat_timeout=5.0).solve(d_local, 5, on_iteration=leave)
        out[rank] = ("finished", None)
    except RankFailure as e:
        out[rank] = ("failure", (e.iteration, list(e.missing)))
    os._exit(0)


def test_shard_is_a_partition():
    from paper_2508_10405_gb300.distributed import shard
    for n in (1, 5, 96):
        for world in (1, 2, 3, 8):
            parts = [shard(n, r, world) for r in range(world)]
            flat = sorted(s for p in parts for s in p)
            assert flat == list(range(n))


def _spawn(target, args, world=2):
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, out) + args) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    return dict(out)


@pytest.mark.parametrize("precond", [False, True])
def test_two_rank_cg_equals_single_process(precond):
    from paper_2508_10405_gb300.distributed import ShotParallelCG, pcg_diagonal
    out = _spawn(_worker, (precond,))
    w = _case()
    op = _OracleShots(w, list(range(w.geom.nshot)))
    d_all = torch.tensor(oracle.born(w, w.dm), dtype=torch.float32)
    x1, mis1 = ShotParallelCG(op).solve(d_all, 4, precond=pcg_diagonal(op) if precond else None)
    # the single-process solve is the oracle's own CGNR / PCGNR in FP32 vectors
    xr, misr = oracle.lsrtm_cg(w, d_all.double().numpy(), 4, precond=precond)
    np.testing.assert_allclose(mis1, misr, rtol=1e-4, atol=1e-6)
    for r in range(2):
        x, mis = out[r]
        np.testing.assert_allclose(mis, mis1, rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(x, x1.numpy(), rtol=0, atol=1e-4 * np.abs(x1.numpy()).max())
    # both ranks hold the same replicated model
    np.testing.assert_array_equal(out[0][0], out[1][0])


def test_rank_leaving_between_iterations_is_reported():
    """Host-side failure detection: a rank that exits between CG iterations
    is reported by the survivor (RankFailure naming it and the iteration)
    before the survivor enters another collective."""
    out = _spawn(_leaving_worker, ())
    assert out[1] == ("left", 2)
    status, info = out[0]
    assert status == "failure", out[0]
    assert info == (3, [1]), info
