"""Replica execution over ranks, on CPU with the gloo backend (world size 2).

The multi-GPU path runs independent replicas: the cost partition, the max-over-ranks
timing and the gather of per-circuit results are host logic, checked here with real
process groups.  The per-circuit work is the oracle's Algorithm-1 gradient so that
the gathered results can be compared with a serial evaluation."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2009_02823_gb300 import replicas as R
from paper_2009_02823_gb300 import workloads as W


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _small_batch():
    return W.batched(count=10, nmin=3, nmax=6, dmin=1, dmax=3, seed_cfg=41)


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws = _small_batch()
        costs = [R.circuit_cost(w.n, w.n_gates, len(w.terms)) for w in ws]
        parts = R.partition(costs, world)
        mine = parts[rank]
        es, gs = [], []
        for b in mine:
            w = ws[b]
            e, g = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
            es.append(e)
            gs.append(g)
        e_all, g_all = R.gather_results(mine, es, gs, len(ws), dist)
        t_max = R.max_over_ranks(1.0 + rank, dist)
        dist.barrier()
        np.save(os.path.join(out_dir, f"e{rank}.npy"), e_all)
        np.save(os.path.join(out_dir, f"g{rank}.npy"), np.concatenate(g_all))
        np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([t_max]))
    finally:
        dist.destroy_process_group()


def test_partition_covers_and_balances():
    costs = [5, 9, 1, 1, 7, 3, 3, 8, 2]
    for world in (1, 2, 3, 4, 12):
        parts = R.partition(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: max load <= mean + largest item
        assert max(loads) <= sum(costs) / world + max(costs)
    assert R.partition(costs, 2) == R.partition(list(costs), 2)  # deterministic
    with pytest.raises(ValueError):
        R.partition(costs, 0)


def test_gather_single_process_detects_gaps_and_duplicates():
    e, g = R.gather_results([1, 0], [2.0, 1.0], [[2.0], [1.0]], 2)
    assert list(e) == [1.0, 2.0] and [x[0] for x in g] == [1.0, 2.0]
    with pytest.raises(ValueError):
        R.gather_results([0], [1.0], [[1.0]], 2)
    with pytest.raises(ValueError):
        R.gather_results([0, 0], [1.0, 1.0], [[1.0], [1.0]], 1)


def test_replica_theta_distinct_per_rank():
    th = np.linspace(0, 1, 5)
    assert np.array_equal(R.replica_theta(th, 0), th)
    assert not np.array_equal(R.replica_theta(th, 1), th)


def test_two_rank_gloo_batch_matches_serial(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    ws = _small_batch()
    e_ref = np.array([oracle.energy(w.n, w.gates, w.theta, w.terms) for w in ws])
    g_ref = np.concatenate([oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)[1] for w in ws])
    for r in range(world):
        e = np.load(tmp_path / f"e{r}.npy")
        g = np.load(tmp_path / f"g{r}.npy")
        np.testing.assert_allclose(e, e_ref, rtol=0, atol=1e-12)
        np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-12)
        assert float(np.load(tmp_path / f"t{r}.npy")[0]) == 2.0  # max over ranks of 1 + rank
