"""Replica-parallel execution over ranks (one process per GPU).

One circuit's state vector lives on one GPU, so the reverse-mode gradient
(Algorithm 1) is not split across GPUs here.  Several GPUs run independent
replicas instead:

* the single-circuit step: every rank evaluates the same workload on its own
  parameters (weak scaling, ``replica_theta``);
* a batch of independent circuits: the circuits are partitioned over the ranks by
  their cost (``partition``), each rank runs its share in one batched launch, and
  the per-circuit results are gathered at the end (``gather_results``).

Nothing on the data path is exchanged.  The only collectives are a barrier, the
maximum of the per-rank times (``max_over_ranks``) and the final gather, all of
which run on whatever process group the caller set up (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np


def circuit_cost(n_qubits: int, n_gates: int, n_terms: int = 0) -> int:
    """Amplitude passes of one gradient: forward + reverse gate passes plus one pass
    per Hamiltonian term, each over 2^n amplitudes."""
    return (1 << n_qubits) * (3 * n_gates + n_terms)


def partition(costs, world: int) -> list[list[int]]:
    """Longest-processing-time-first assignment of items to ``world`` ranks.

    Items are taken in decreasing cost (ties by index) and each goes to the rank
    with the least load so far (ties by rank).  Deterministic, so every rank
    computes the same partition without communicating.  Returns, per rank, its
    item indices in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = [int(c) for c in costs]
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += costs[i]
        parts[r].append(i)
    return [sorted(p) for p in parts]


def replica_theta(theta, rank: int, spread: float = 1e-3) -> np.ndarray:
    """Per-rank parameters of a single-circuit replica: the workload's theta moved
    by ``spread * rank`` so that replicas do distinct (but equally costly) work."""
    return np.ascontiguousarray(np.asarray(theta, dtype=np.float64) + spread * rank)


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The maximum of a per-rank scalar (a timed duration) over all ranks."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(local_idx, energies, grads, n_total: int, dist=None):
    """Collect per-circuit results from every rank into global circuit order.

    ``local_idx[k]`` is the global index of this rank's k-th circuit, ``energies[k]``
    its energy and ``grads[k]`` its gradient.  Returns (energies, grads) over all
    ``n_total`` circuits on every rank.  Raises if a circuit is missing or claimed
    by two ranks."""
    local = [(int(i), float(e), np.asarray(g, dtype=np.float64)) for i, e, g in zip(local_idx, energies, grads)]
    if dist is None:
        every = [local]
    else:
        every = [None] * dist.get_world_size()
        dist.all_gather_object(every, local)
    e_out = [None] * n_total
    g_out = [None] * n_total
    for part in every:
        for i, e, g in part:
            if not 0 <= i < n_total:
                raise ValueError(f"circuit index {i} out of range")
            if e_out[i] is not None:
                raise ValueError(f"circuit {i} evaluated by two ranks")
            e_out[i], g_out[i] = e, g
    missing = [i for i in range(n_total) if e_out[i] is None]
    if missing:
        raise ValueError(f"circuits {missing[:8]} evaluated by no rank")
    return np.array(e_out), g_out
