"""Multi-GPU host logic on the CPU: column partition and the sharded bisection.

The bisection over ranks runs as world_size-2 ``gloo`` processes whose
per-rank builds are stand-ins computed by the oracle on the rank's block
columns (the CUDA shard itself is covered by a single-GPU test that builds
the shards one after the other).
"""

import os

import numpy as np
import pytest

import oracle as O
from paper_2205_14741_gb300.shard import partition_columns, solve_mu_sharded
from synth import make_workload


def test_partition_is_contiguous_and_balanced():
    rng = np.random.default_rng(0)
    dims = rng.integers(60, 300, 500)
    for world in [1, 2, 3, 7, 152]:
        parts = partition_columns(dims, world)
        assert parts[0][0] == 0 and parts[-1][1] == len(dims)
        assert all(a < b for a, b in parts) and all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
        work = np.array([np.sum(dims[a:b].astype(float) ** 3) for a, b in parts])
        ideal = np.sum(dims.astype(float) ** 3) / world
        assert np.max(work) <= ideal + np.max(dims.astype(float) ** 3) * 1.0001


def test_partition_edge_cases():
    assert partition_columns([5, 5, 5], 3) == [(0, 1), (1, 2), (2, 3)]
    assert partition_columns([100, 1, 1, 1], 2)[0] == (0, 1)  # the heavy column alone
    with pytest.raises(ValueError):
        partition_columns([1, 2], 3)
    with pytest.raises(ValueError):
        partition_columns([1, 2], 0)


class OracleShard:
    """Stand-in for a context restricted to block columns [j0, j1), computed by the oracle."""

    def __init__(self, sysm, eps, j0, j1):
        self.bs = sysm.block_size
        self.cp, self.ri, self.v, _ = O.filter_blocks(sysm.block_size, sysm.col_ptr, sysm.row_idx, sysm.values, eps)
        self.cols = list(range(j0, j1))
        self.mu = None
        self.res = None

    def get_gershgorin_interval(self):
        return O.global_gershgorin(self.bs, self.cp, self.ri, self.v)

    def set_mu(self, mu):
        self.mu = mu

    def build_density(self):
        self.res = O.density_submatrix(self.bs, self.cp, self.ri, self.v, self.mu, columns=self.cols)

    def get_trace(self):
        return self.res.trace, self.res.energy, self.mu


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = make_workload("water32")
    dims = [int(np.sum(s.block_size[s.row_idx[s.col_ptr[j]:s.col_ptr[j + 1]]])) for j in range(s.n_blocks)]
    j0, j1 = partition_columns(dims, world)[rank]
    ctx = OracleShard(s, 0.0, j0, j1)

    def allreduce_sum(x):
        t = torch.from_numpy(x.copy())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()

    mu, tr, en, steps = solve_mu_sharded(ctx, 96.0, allreduce_sum, max_steps=30, tol=0.5)
    np.save(f"{out_path}.{rank}.npy", np.array([mu, tr, en, steps, j0, j1]))
    dist.destroy_process_group()


def test_sharded_bisection_over_two_gloo_ranks(tmp_path):
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = str(tmp_path / "res")
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    r0, r1 = np.load(f"{out}.0.npy"), np.load(f"{out}.1.npy")
    assert r0[:4].tolist() == r1[:4].tolist()  # every rank took the same decisions
    assert r0[5] == r1[4]                      # the shards tile the block columns
    s = make_workload("water32")
    mu, res, hist = O.bisect_mu(s.block_size, s.col_ptr, s.row_idx, s.values, 96.0, max_steps=30, tol=0.5)
    assert r0[0] == mu and int(r0[3]) == len(hist)
    assert abs(r0[1] - res.trace) <= 1e-10 and abs(r0[2] - res.energy) <= 1e-10 * abs(res.energy)
