"""The replica bookkeeping of multi-GPU runs (paper_2605_17796_gb300.replicas) on two gloo ranks
(CPU processes): disjoint shot ranges that tile the index space, and the max / sum reductions
that bench.py applies at the end of its timed region."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    from paper_2605_17796_gb300 import replicas
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    steps, n_p, spp = 3, 4, 5
    starts = [replicas.shot_offset(s, rank, world, pi, n_p, spp) for s in range(steps) for pi in range(n_p)]
    t = replicas.max_over_ranks(10.0 + rank, world)
    c = replicas.sum_over_ranks([rank + 1, 100 * rank, 7], world)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array(starts + [t] + c, dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    steps, n_p, spp = 3, 4, 5
    res = [np.load(tmp_path / f"r{r}.npy") for r in range(world)]
    starts = np.concatenate([r[:steps * n_p] for r in res]).astype(np.int64)
    covered = np.concatenate([np.arange(s, s + spp) for s in starts])
    assert np.array_equal(np.sort(covered), np.arange(steps * world * n_p * spp))
    for r in res:
        assert r[steps * n_p] == 11.0                         # max of 10 + rank
        assert list(r[steps * n_p + 1:]) == [3, 100, 14]       # sums over the ranks
