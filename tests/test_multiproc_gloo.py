"""The N > 1 host logic on CPU with torch.distributed (gloo, world size 2).

The join shards by query windows with no exchange between ranks: each rank
joins its own run of windows (plus the m - 1 halo samples they reach), and the
profiles concatenate. Timing takes the slowest rank. Both are checked here with
the CPU oracle, without a GPU.
"""
import os
import socket

import numpy as np
import pytest

import bench
import oracle
import synthetic


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q, b, offs, m, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = bench.shard_rows(len(q), m, world, rank)
    d, i, _ = oracle.ab_join(q[lo:hi], b, offs, m)
    np.save(os.path.join(out_dir, f"d{rank}.npy"), d)
    np.save(os.path.join(out_dir, f"i{rank}.npy"), i)
    t = bench.max_over_ranks(1.0 + rank, world)  # rank r "took" 1 + r
    np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([t]))
    dist.destroy_process_group()


def test_shard_rows_cover_every_window_once():
    for n, m, world in [(100, 10, 3), (10, 10, 4), (1000, 7, 8), (5, 6, 2), (64, 1, 5)]:
        nq = max(0, n - m + 1)
        covered = []
        for r in range(world):
            lo, hi = bench.shard_rows(n, m, world, r)
            assert 0 <= lo <= hi <= n
            covered += list(range(lo, max(lo, hi - m + 1)))
        assert covered == list(range(nq))


def test_two_gloo_ranks_concatenate_to_the_whole_profile(tmp_path):
    import torch.multiprocessing as tmp

    m = 24
    q = synthetic.random_walk(700, 8)
    b, offs = synthetic.cut_dictionary(synthetic.random_walk(2000, 9), 4, 300)
    port = _free_port()
    tmp.spawn(_worker, args=(2, port, q, b, offs, m, str(tmp_path)), nprocs=2, join=True)
    d = np.concatenate([np.load(tmp_path / f"d{r}.npy") for r in range(2)])
    i = np.concatenate([np.load(tmp_path / f"i{r}.npy") for r in range(2)])
    fd, fi, _ = oracle.ab_join(q, b, offs, m)
    np.testing.assert_array_equal(d, fd)
    np.testing.assert_array_equal(i, fi)
    for r in range(2):
        assert np.load(tmp_path / f"t{r}.npy")[0] == 2.0  # the slowest rank's time on every rank
