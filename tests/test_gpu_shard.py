"""Receiver sharding helpers with the CUDA tree (single process): the GPU
tree's Morton order equals the oracle's, and J walked range by range and put
back in place equals J walked at once, bit for bit."""

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def t2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_15235_gb300 import build_lib
    build_lib.build()
    import paper_2310_15235_gb300 as mod
    mod.load_library()
    return mod


@pytest.mark.parametrize("world", [2, 3, 8])
def test_ranges_walked_separately_equal_one_walk(t2, oracle_mod, world):
    from paper_2310_15235_gb300 import shard
    case = workloads.random_case(3000, 40, nb=3, seed=62, clumped=True, n_active=1001)
    tree = t2.build(case["pos"], case["mass"], case["kappa"], case["lum"], case["h"],
                    case["box_lo"], case["box_size"], case["bucket"])
    act = case["active"]
    order = shard.tree_morton_rank(tree, act)
    ot = oracle_mod.OracleTree.from_case(case)
    perm = ot.export()["perm"].astype(np.int64)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    np.testing.assert_array_equal(order, shard.morton_rank(inv, act))
    full = tree.J(act, 2, 0.75).cpu().numpy()
    out = np.full_like(full, np.nan)
    for r in range(world):
        rows = shard.local_rows(order, world, r)
        out[rows] = tree.J(act[rows], 2, 0.75).cpu().numpy()
    np.testing.assert_array_equal(out, full)
    tree.free()
