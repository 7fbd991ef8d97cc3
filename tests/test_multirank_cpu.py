"""Two ranks over gloo on CPU: the host-side sharding of the Coulomb matrix
(balanced item ranges, local offsets, the final all_gather) reproduces the
unsharded result.  The per-rank contraction is played by the oracle here;
on GPUs it is coulomb_matrix on the rank's item slice."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads
from oracle import coulomb as ocoul
from oracle import kernel_vectors as okv
from oracle import sinc as osinc
from paper_1504_06289_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, b, M = 48, 6.0, 10
        basis = workloads.basis_set(5, 2, 4, 0.3, 20.0, 3, 1.2, seed=8)
        items = ocoul.item_list(5)
        _, _, _, off = ocoul.item_pairs(basis, items)
        t, a = osinc.conv_nodes(n, b, M)
        P = okv.conv_kernel_vectors(n, b, t, a)
        ranges = shard.balanced_item_ranges(off, world)
        i0, i1, f0, f1, loc = shard.local_items(off, rank, world)
        assert (i0, i1) == ranges[rank] and loc[0] == 0 and loc[-1] == f1 - f0
        J_local, _ = ocoul.coulomb_items(n, b, basis, P, items[i0:i1])
        J = shard.gather_items(torch.tensor(J_local), ranges)
        if rank == 0:
            J_full, _ = ocoul.coulomb_items(n, b, basis, P, items)
            out_q.put(float(np.max(np.abs(J.numpy() - J_full))))
    finally:
        dist.destroy_process_group()


def test_sharded_coulomb_matrix_gathers_to_the_full_result():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    assert q.get(timeout=5) < 1e-12


def test_balanced_ranges_cover_and_balance_rows():
    rng = np.random.default_rng(0)
    ranks = rng.integers(9, 37, size=3240)          # uneven item ranks as in basis80
    off = np.concatenate([[0], np.cumsum(ranks)])
    for world in (1, 2, 3, 8):
        rs = shard.balanced_item_ranges(off, world)
        assert rs[0][0] == 0 and rs[-1][1] == 3240
        assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
        rows = [off[e] - off[b] for b, e in rs]
        assert max(rows) - min(rows) <= 2 * ranks.max()
    assert shard.column_ranges(600, 8)[-1] == (525, 600)
