"""Receiver sharding over ranks, tested on CPU ranks (gloo, world size 2).

The per-rank J and gradient come from the oracle here; the host logic under
test (Morton ranges, gather of J, sum of per-element gradients) is the same
that GPU ranks run with the CUDA library.
"""

import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import workloads

NSIDE, THETA = 2, 0.75


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    return workloads.random_case(500, 20, nb=2, seed=61, clumped=True, n_active=151)


def _params():
    return [("kappa", 3, 0), ("kappa", 77, 1), ("kappa", 250, 0), ("lum", 500 + 2, 1),
            ("lum", 500 + 9, 0), ("lum", 120, 1)]


def _inv(ot):
    perm = ot.export()["perm"].astype(np.int64)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    return inv


def _bucket_worker(rank, world, port, queue):
    """Per-bucket beams with p-p absorption and the complex source model: a
    receiver's J depends on its bucket only, so Morton ranges walked on
    different ranks give the rows of one walk over all receivers."""
    import torch.distributed as dist

    import oracle
    from paper_2310_15235_gb300 import shard

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        case = _case()
        ot = oracle.OracleTree.from_case(case)
        act = case["active"]
        order = shard.morton_rank(_inv(ot), act)
        flags = oracle.FLAG_BUCKET | oracle.FLAG_PP | oracle.FLAG_CSM
        J = shard.J_sharded(order, act, lambda a: torch.from_numpy(
            ot.J(a, NSIDE, THETA, flags=flags)))
        queue.put((rank, J.numpy()))
    finally:
        dist.destroy_process_group()


def _worker(rank, world, port, queue):
    import torch.distributed as dist

    import oracle
    from paper_2310_15235_gb300 import shard

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        case = _case()
        ot = oracle.OracleTree.from_case(case)
        act = case["active"]
        order = shard.morton_rank(_inv(ot), act)
        J = shard.J_sharded(order, act, lambda a: torch.from_numpy(ot.J(a, NSIDE, THETA)))
        w = torch.from_numpy(np.random.default_rng(3).uniform(size=(len(act), 2)))

        def backward(a, g):
            out = [float((ot.J_deriv(a, NSIDE, THETA, which, e, b) * g.numpy()).sum())
                   for which, e, b in _params()]
            return (torch.tensor(out, dtype=torch.float64),)

        (grad,) = shard.J_backward_sharded(order, act, w, backward)
        rows = shard.local_rows(order, world, rank)
        queue.put((rank, J.numpy(), grad.numpy(), rows))
    finally:
        dist.destroy_process_group()


def test_shard_ranges_cover_once():
    from paper_2310_15235_gb300 import shard
    for A, world in [(0, 2), (1, 2), (7, 3), (1000, 8), (5, 8)]:
        r = shard.shard_ranges(A, world)
        assert len(r) == world and r[0][0] == 0 and r[-1][1] == A
        sizes = [hi - lo for lo, hi in r]
        assert max(sizes) - min(sizes) <= 1
        assert all(r[i][1] == r[i + 1][0] for i in range(world - 1))


def test_morton_rank_orders_by_tree_position(oracle_mod):
    from paper_2310_15235_gb300 import shard
    case = _case()
    ot = oracle_mod.OracleTree.from_case(case)
    inv = _inv(ot)
    order = shard.morton_rank(inv, case["active"])
    keys = ot.export()["keys"]
    k = keys[case["active"][order]]
    assert np.all(k[1:] >= k[:-1])
    assert sorted(order.tolist()) == list(range(len(case["active"])))


def test_sharded_J_and_gradient_world2(oracle_mod):
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, queue)) for r in range(world)]
    for p in procs:
        p.start()
    results = [queue.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    case = _case()
    ot = oracle_mod.OracleTree.from_case(case)
    act = case["active"]
    J_full = ot.J(act, NSIDE, THETA)
    w = np.random.default_rng(3).uniform(size=(len(act), 2))
    g_full = np.array([float((ot.J_deriv(act, NSIDE, THETA, which, e, b) * w).sum())
                       for which, e, b in _params()])
    rows = sorted(np.concatenate([r[3] for r in results]).tolist())
    assert rows == list(range(len(act)))  # every receiver on exactly one rank
    for rank, J, g, _ in results:
        np.testing.assert_array_equal(J, J_full)  # gathered rows land in place
        np.testing.assert_allclose(g, g_full, rtol=1e-12, atol=1e-15 * np.abs(g_full).max())


def test_sharded_bucket_J_world2(oracle_mod):
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    procs = [ctx.Process(target=_bucket_worker, args=(r, world, port, queue))
             for r in range(world)]
    for p in procs:
        p.start()
    results = [queue.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    case = _case()
    ot = oracle_mod.OracleTree.from_case(case)
    flags = oracle_mod.FLAG_BUCKET | oracle_mod.FLAG_PP | oracle_mod.FLAG_CSM
    J_full = ot.J(case["active"], NSIDE, THETA, flags=flags)
    for _, J in results:
        np.testing.assert_array_equal(J, J_full)
