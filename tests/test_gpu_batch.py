"""Batched walk (many receiver subsets over several trees in one launch)
through the C ABI, against the per-subset walk and the FP64 oracle.

Each batched row must equal trevr2_J's row for the same tree and receiver
bit for bit in the default launch shape (the per-receiver arithmetic is the
same code), and the oracle within the J tolerances in every shape the
autotuner may pick.  Individual timesteps (Sec. 1.2) give the subsets;
independent snapshots (Sec. 3.1) give the trees.
"""

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

J_MEDIAN_TOL = 1e-4
J_MAX_TOL = 1e-3


@pytest.fixture(scope="module")
def t2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_15235_gb300 import build_lib
    build_lib.build()
    import paper_2310_15235_gb300 as mod
    mod.load_library()
    return mod


def _gpu_tree(t2, case):
    return t2.build(case["pos"], case["mass"], case["kappa"], case["lum"], case["h"],
                    case["box_lo"], case["box_size"], case["bucket"])


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    r = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
    r[(a == 0) & (b == 0)] = 0.0
    return r


def _assert_J(J, ref, what=""):
    assert np.all(np.isfinite(J)), what
    r = _rel(J, ref)
    med, mx = float(np.median(r)), float(r.max())
    assert med <= J_MEDIAN_TOL and mx <= J_MAX_TOL, f"{what}: median {med:.3e} max {mx:.3e}"


def _small_cases():
    """Three trees of different depth and size with the same band count."""
    return [
        workloads.random_case(900, 25, nb=2, seed=31, clumped=True),
        workloads.random_case(2500, 40, nb=2, seed=32),
        workloads.random_case(300, 12, nb=2, seed=33, clumped=True, bucket=3),
    ]


def _subsets(cases, seed=7):
    """Ragged subsets: empty, single, duplicated, whole trees and random sizes,
    interleaved over the trees."""
    rng = np.random.default_rng(seed)
    subs = []
    for k in range(14):
        t = int(rng.integers(0, len(cases)))
        n = len(cases[t]["pos"])
        kind = k % 7
        if kind == 0:
            m = np.zeros(0, np.int64)
        elif kind == 1:
            m = np.array([int(rng.integers(0, n))], np.int64)
        elif kind == 2:
            m = np.arange(n, dtype=np.int64)
        elif kind == 3:  # duplicates, unsorted
            m = rng.integers(0, n, size=57).astype(np.int64)
        else:
            m = np.sort(rng.choice(n, size=int(rng.integers(2, n)), replace=False)).astype(np.int64)
        subs.append((t, m))
    return subs


def _layout(subs):
    offsets = np.zeros(len(subs) + 1, np.int64)
    offsets[1:] = np.cumsum([len(m) for _, m in subs])
    tree_of = np.array([t for t, _ in subs], np.int32)
    active = np.concatenate([m for _, m in subs]) if subs else np.zeros(0, np.int64)
    return active, offsets, tree_of


@pytest.mark.parametrize("nside,flags", [(1, 0), (2, 3), (4, 0)])
def test_batch_equals_per_subset_and_oracle(t2, oracle_mod, nside, flags):
    cases = _small_cases()
    trees = [_gpu_tree(t2, c) for c in cases]
    subs = _subsets(cases)
    active, offsets, tree_of = _layout(subs)
    J = t2.J_batched(trees, active, offsets, tree_of, nside, 0.75, flags).cpu().numpy()
    assert J.shape == (offsets[-1], 2)
    oracles = [oracle_mod.OracleTree.from_case(c) for c in cases]
    for s, (t, m) in enumerate(subs):
        rows = J[offsets[s]:offsets[s + 1]]
        if len(m) == 0:
            continue
        single = trees[t].J(m, nside, 0.75, flags=flags).cpu().numpy()
        np.testing.assert_array_equal(rows, single, err_msg=f"subset {s} (tree {t})")
        _assert_J(rows, oracles[t].J(m, nside, 0.75, flags=flags), f"subset {s}")
    for tr in trees:
        tr.free()


@pytest.mark.parametrize("nside,extra", [(2, 0), (1, 3), (2, 34), (2, 64), (4, 96 + 2)])
def test_batch_bucket_equals_per_subset_and_oracle(t2, oracle_mod, nside, extra):
    """Per-bucket plans (TREVR2_BUCKET, Sec. 2.5.1; with SOFT|THICK, with p-p
    absorption and THICK, with the complex source model, with both): every
    distinct (tree, bucket) is walked once for all the receivers the
    subsets ask for, and each subset's rows equal trevr2_J's per-bucket rows
    for that subset bit for bit and the oracle within the J tolerances."""
    flags = t2.BUCKET | extra
    cases = _small_cases()
    trees = [_gpu_tree(t2, c) for c in cases]
    subs = _subsets(cases, seed=21)
    active, offsets, tree_of = _layout(subs)
    J = t2.J_batched(trees, active, offsets, tree_of, nside, 0.75, flags).cpu().numpy()
    oracles = [oracle_mod.OracleTree.from_case(c) for c in cases]
    for s, (t, m) in enumerate(subs):
        rows = J[offsets[s]:offsets[s + 1]]
        if len(m) == 0:
            continue
        single = trees[t].J(m, nside, 0.75, flags=flags).cpu().numpy()
        np.testing.assert_array_equal(rows, single, err_msg=f"subset {s} (tree {t})")
        _assert_J(rows, oracles[t].J(m, nside, 0.75, flags=flags), f"subset {s}")
    for tr in trees:
        tr.free()


def test_batch_bucket_graph_replay_and_autotune(t2, oracle_mod):
    """A per-bucket plan autotuned, recorded into a CUDA graph and replayed
    with other receivers in the same buffer."""
    cases = _small_cases()
    trees = [_gpu_tree(t2, c) for c in cases]
    subs = _subsets(cases, seed=22)
    active, offsets, tree_of = _layout(subs)
    plan = t2.Batch(trees, offsets, tree_of, nside=2, theta=0.6, flags=t2.BUCKET)
    act = torch.as_tensor(active, device="cuda")
    w, m = plan.autotune(act)
    assert w == 4 and m in (512, 1024, 2048)
    out = torch.empty((int(offsets[-1]), 2), dtype=torch.float32, device="cuda")
    plan.run(act, out)
    plan.status()
    ref = out.cpu().numpy().copy()
    for s, (t, mem) in enumerate(subs):
        if len(mem):
            want = oracle_mod.OracleTree.from_case(cases[t]).J(mem, 2, 0.6, flags=t2.BUCKET)
            _assert_J(ref[offsets[s]:offsets[s + 1]], want, f"autotuned bucket subset {s}")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.run(act, out)
    out.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    plan.status()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    rng = np.random.default_rng(4)
    perm = np.arange(len(active))
    for s in range(len(subs)):
        lo, hi = offsets[s], offsets[s + 1]
        perm[lo:hi] = lo + rng.permutation(hi - lo)
    act.copy_(torch.as_tensor(active[perm], device="cuda"))
    g.replay()
    torch.cuda.synchronize()
    plan.status()
    np.testing.assert_array_equal(out.cpu().numpy(), ref[perm])
    plan.free()
    for tr in trees:
        tr.free()


def test_batch_bucket_bad_receiver_reported(t2):
    cases = _small_cases()[:2]
    trees = [_gpu_tree(t2, c) for c in cases]
    n0 = len(cases[0]["pos"])
    subs = [(0, np.array([0, n0, 1], np.int64)), (1, np.array([5, 6], np.int64))]
    active, offsets, tree_of = _layout(subs)
    plan = t2.Batch(trees, offsets, tree_of, nside=2, flags=t2.BUCKET)
    J = plan.run(torch.as_tensor(active, device="cuda"))
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        plan.status()
    J = J.cpu().numpy()
    assert np.all(np.isnan(J[1])) and np.all(np.isfinite(J[[0, 2, 3, 4]]))
    plan.free()
    for tr in trees:
        tr.free()


def test_batch_plan_reuse_and_graph_replay(t2, oracle_mod):
    """One plan run eagerly, then recorded into a CUDA graph and replayed with
    new receivers written into the same input buffer."""
    cases = _small_cases()
    trees = [_gpu_tree(t2, c) for c in cases]
    subs = _subsets(cases, seed=8)
    active, offsets, tree_of = _layout(subs)
    plan = t2.Batch(trees, offsets, tree_of, nside=2, theta=0.6)
    act = torch.as_tensor(active, device="cuda")
    out = torch.empty((int(offsets[-1]), 2), dtype=torch.float32, device="cuda")
    plan.run(act, out)
    plan.status()
    ref = out.cpu().numpy().copy()
    plan.run(act, out)  # a second run of the same plan gives the same rows
    plan.status()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.run(act, out)
    out.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    plan.status()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)

    # new receivers (a permutation inside every subset) in the same buffer
    rng = np.random.default_rng(3)
    perm = np.arange(len(active))
    for s in range(len(subs)):
        lo, hi = offsets[s], offsets[s + 1]
        perm[lo:hi] = lo + rng.permutation(hi - lo)
    act.copy_(torch.as_tensor(active[perm], device="cuda"))
    g.replay()
    torch.cuda.synchronize()
    plan.status()
    np.testing.assert_array_equal(out.cpu().numpy(), ref[perm])
    plan.free()
    for tr in trees:
        tr.free()


def test_batch_autotune(t2, oracle_mod):
    cases = _small_cases()
    trees = [_gpu_tree(t2, c) for c in cases]
    subs = _subsets(cases, seed=9)
    active, offsets, tree_of = _layout(subs)
    plan = t2.Batch(trees, offsets, tree_of, nside=2, theta=0.75)
    act = torch.as_tensor(active, device="cuda")
    w, m = plan.autotune(act)
    assert w in (4, 8) and m in (512, 1024, 2048)
    J = plan.run(act).cpu().numpy()
    plan.status()
    for s, (t, mem) in enumerate(subs):
        if len(mem):
            ref = oracle_mod.OracleTree.from_case(cases[t]).J(mem, 2, 0.75)
            _assert_J(J[offsets[s]:offsets[s + 1]], ref, f"autotuned subset {s}")
    plan.free()
    for tr in trees:
        tr.free()


def test_batch_many_sources_every_staging_depth(t2, oracle_mod):
    """theta -> 0 opens every cell: receivers see more sources than the
    smallest staging depth holds, so the shapes take different numbers of
    passes; all must agree with the oracle."""
    case = workloads.random_case(400, 2600, nb=2, seed=16, clumped=True, n_active=150)
    tree = _gpu_tree(t2, case)
    subs = [(0, case["active"][:70]), (0, case["active"][70:])]
    active, offsets, tree_of = _layout(subs)
    plan = t2.Batch([tree], offsets, tree_of, nside=2, theta=1e-6)
    act = torch.as_tensor(active, device="cuda")
    plan.autotune(act)  # runs every shape once on the whole (small) batch
    J = plan.run(act).cpu().numpy()
    plan.status()
    ref = oracle_mod.OracleTree.from_case(case).J(active, 2, 1e-6)
    _assert_J(J, ref, "many sources")
    plan.free()
    tree.free()


def test_batch_bad_receiver_reported(t2):
    cases = _small_cases()[:2]
    trees = [_gpu_tree(t2, c) for c in cases]
    n0 = len(cases[0]["pos"])
    subs = [(0, np.array([0, n0, 1], np.int64)), (1, np.array([5, 6], np.int64))]
    active, offsets, tree_of = _layout(subs)
    plan = t2.Batch(trees, offsets, tree_of, nside=2)
    J = plan.run(torch.as_tensor(active, device="cuda"))
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        plan.status()
    J = J.cpu().numpy()
    assert np.all(np.isnan(J[1])) and np.all(np.isfinite(J[[0, 2, 3, 4]]))
    plan.status()  # the status word was cleared
    plan.free()
    for tr in trees:
        tr.free()


def test_batch_argument_errors(t2):
    a = _gpu_tree(t2, workloads.random_case(200, 5, nb=2, seed=41))
    b = _gpu_tree(t2, workloads.random_case(200, 5, nb=3, seed=42))
    with pytest.raises(t2.TrevrError, match="EINVAL"):  # band counts differ
        t2.Batch([a, b], [0, 1, 2], [0, 1])
    with pytest.raises(t2.TrevrError, match="EINVAL"):  # offsets[0] != 0
        t2.Batch([a], [1, 2], [0])
    with pytest.raises(t2.TrevrError, match="EINVAL"):  # decreasing offsets
        t2.Batch([a], [0, 5, 3], [0, 0])
    with pytest.raises(t2.TrevrError, match="EINVAL"):  # tree_of out of range
        t2.Batch([a], [0, 5], [1])
    with pytest.raises(t2.TrevrError, match="EINVAL"):  # nside not a power of two
        t2.Batch([a], [0, 5], [0], nside=3)
    with pytest.raises(t2.TrevrError, match="EUNSUPPORTED"):
        t2.Batch([a] * 33, [0, 5], [0])
    with pytest.raises(ValueError):
        t2.Batch([a], [0, 5], [0, 0])
    # an empty batch is valid and its run does nothing
    empty = t2.Batch([a], [0], [])
    assert empty.run(torch.zeros(0, dtype=torch.int64, device="cuda")).shape == (0, 2)
    empty.status()
    empty.free()
    a.free()
    b.free()


@pytest.fixture(scope="module")
def snapshots():
    return workloads.batched_cases()


@pytest.mark.parametrize("flags", [0, 16])
def test_batch_full_size_sampled(t2, oracle_mod, snapshots, flags):
    """The individual-timestep workload at full size: 4 snapshots of the
    2,097,152-element clumpy 3-band field, 64 subsets each of 10^U(2,6)
    receivers, nside 4, theta 0.5, autotuned, one launch (per receiver, and
    per bucket with TREVR2_BUCKET = 16); 512 sampled rows against the
    oracle."""
    snaps, subsets = snapshots
    trees = [_gpu_tree(t2, c) for c in snaps]
    active, offsets, tree_of = _layout(subsets)
    plan = t2.Batch(trees, offsets, tree_of, nside=4, theta=0.5, flags=flags)
    act = torch.as_tensor(active, device="cuda")
    plan.autotune(act)
    J = plan.run(act).cpu().numpy()
    plan.status()
    assert np.all(np.isfinite(J)) and np.all(J >= 0)
    rng = np.random.default_rng(11)
    rows = np.sort(rng.choice(len(active), 512, replace=False))
    sub_of_row = np.searchsorted(offsets, rows, side="right") - 1
    for t in range(len(snaps)):
        pick = rows[tree_of[sub_of_row] == t]
        if len(pick):
            ref = oracle_mod.OracleTree.from_case(snaps[t]).J(active[pick], 4, 0.5, flags=flags)
            _assert_J(J[pick], ref, f"snapshot {t}")
    plan.free()
    for tr in trees:
        tr.free()
