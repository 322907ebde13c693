"""Multi-rank logic of bench.py on the CPU: two gloo ranks, replicas by
realization.  Columns are independent given the shared operator (Sec. 2.4),
so the shards integrated on separate ranks must equal the corresponding
columns of one run over the whole ensemble, and the job time is the slowest
rank's time."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
K, M, N, R, RR = 16, 3, 60, 2, 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2009_11742_gb300 import inputs
    p = inputs.make_problem(K, K, M * world, R, seed=4)
    T = bench.rank_periods(p.T, rank, world)
    Z = np.zeros((K, M))
    V, S, tr = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, N, T=T, r=RR)
    t = bench.max_over_ranks(1.0 + 0.5 * rank, dist, torch.device("cpu"))
    got = [None] * world
    dist.all_gather_object(got, {"rank": rank, "V": V.tolist(), "tr": tr.tolist(), "t": t})
    if rank == 0:
        with open(out, "w") as f:
            json.dump(got, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_by_realization(tmp_path):
    world = 2
    out = str(tmp_path / "ranks.json")
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    got = json.load(open(out))
    assert [g["rank"] for g in got] == [0, 1]
    assert all(g["t"] == 1.5 for g in got)  # every rank sees the slowest rank's time
    import oracle
    from paper_2009_11742_gb300 import inputs
    p = inputs.make_problem(K, K, M * world, R, seed=4)
    Z = np.zeros((K, M * world))
    Vf, _, trf = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, N, T=p.T, r=RR)
    V = np.concatenate([np.array(g["V"]) for g in got], axis=1)
    tr = np.concatenate([np.array(g["tr"]) for g in got], axis=2)
    np.testing.assert_array_equal(V, Vf)
    np.testing.assert_array_equal(tr, trf)


def test_shards_partition_the_ensemble():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    T = np.arange(12.0)
    parts = [bench.rank_periods(T, r, 4) for r in range(4)]
    assert all(len(x) == 3 for x in parts)
    np.testing.assert_array_equal(np.concatenate(parts), T)
    assert bench.max_over_ranks(2.5, None, None) == 2.5
