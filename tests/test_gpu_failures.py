"""Failure paths, made on the host side so that no GPU faults.

A testing aid of the library (trevr2_debug_set) makes the n-th device
allocation of a call fail.  For n = 0, 1, ... until the call succeeds, every
failure must come back as ENOMEM with a message, release every temporary
(the library's use of the device memory pool returns to what it was, or to
what the tree legitimately caches), and leave the tree or plan usable: the
call that finally succeeds gives the same result as an undisturbed one.  A
capped source-cut stack must come back as EINTERNAL, not as a wrong J.
"""

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

ENOMEM, EINVAL, EINTERNAL = -2, -1, -6


@pytest.fixture(scope="module")
def t2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_15235_gb300 import build_lib
    build_lib.build()
    import paper_2310_15235_gb300 as mod
    mod.load_library()
    return mod


@pytest.fixture(autouse=True)
def _aids_off(t2):
    yield
    t2.debug_set(t2.DEBUG_FAIL_ALLOC, -1)
    t2.debug_set(t2.DEBUG_SOURCE_STACK, 0)


def _case():
    return workloads.random_case(1500, 60, nb=2, seed=301, clumped=True)


def _gpu_tree(t2, case):
    return t2.build(case["pos"], case["mass"], case["kappa"], case["lum"], case["h"],
                    case["box_lo"], case["box_size"], case["bucket"])


def _each_failure(t2, call, after_failure, max_points=400):
    """call() with its n-th allocation failing for n = 0, 1, ...; checks
    after_failure() after each ENOMEM; returns (failing points, result of the
    call that succeeded)."""
    for n in range(max_points):
        t2.debug_set(t2.DEBUG_FAIL_ALLOC, n)
        try:
            result = call()
        except t2.TrevrError as e:
            assert e.code == ENOMEM, f"allocation {n}: {e}"
            assert "failure requested" in str(e), str(e)
            t2.debug_set(t2.DEBUG_FAIL_ALLOC, -1)
            after_failure(n)
            continue
        t2.debug_set(t2.DEBUG_FAIL_ALLOC, -1)
        return n, result
    raise AssertionError(f"the call still failed after {max_points} allocations")


def test_aids_reject_bad_settings(t2):
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        t2.debug_set(7, 1)
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        t2.debug_set(t2.DEBUG_FAIL_ALLOC, -2)
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        t2.debug_set(t2.DEBUG_SOURCE_STACK, -1)


def test_build_every_allocation_failure(t2):
    """A build that fails at any of its allocations returns ENOMEM and keeps
    no device memory; the build that succeeds gives the undisturbed tree."""
    case = _case()
    base = t2.debug_pool_used()
    ref_tree = _gpu_tree(t2, case)
    ref = ref_tree.J(case["active"], 2, 0.75).cpu().numpy()
    ref_tree.free()
    assert t2.debug_pool_used() == base

    def after(n):
        assert t2.debug_pool_used() == base, f"build failing at allocation {n} kept memory"

    points, tree = _each_failure(t2, lambda: _gpu_tree(t2, case), after)
    assert points >= 20  # the build has many allocations; each was exercised
    np.testing.assert_array_equal(tree.J(case["active"], 2, 0.75).cpu().numpy(), ref)
    tree.free()
    assert t2.debug_pool_used() == base


@pytest.mark.parametrize("flags", [0, 8, 16 | 32 | 64 | 2])
def test_J_every_allocation_failure(t2, flags):
    """The first J of a tree (tables, receiver order, walk buffers, and with
    BUCKET | PP | CSM the complex-source tables) failing at any allocation:
    ENOMEM, the tree stays usable, and after trevr2_free nothing is left."""
    case = _case()
    ref_tree = _gpu_tree(t2, case)
    ref = ref_tree.J(case["active"], 2, 0.75, flags=flags).cpu().numpy()
    ref_tree.free()
    base = t2.debug_pool_used()
    tree = _gpu_tree(t2, case)
    held = t2.debug_pool_used()

    def after(n):
        # anything kept now is a complete cached part of the tree
        assert t2.debug_pool_used() >= held

    points, J = _each_failure(t2, lambda: tree.J(case["active"], 2, 0.75, flags=flags), after)
    assert points >= 3
    np.testing.assert_array_equal(J.cpu().numpy(), ref)
    tree.free()
    assert t2.debug_pool_used() == base


def test_backward_every_allocation_failure(t2):
    """trevr2_J_backward allocates its gradient buffers per call: a failure at
    any allocation returns ENOMEM with the pool as before the call, and the
    gradients of the call that succeeds equal an undisturbed call's."""
    case = _case()
    tree = _gpu_tree(t2, case)
    act = case["active"]
    w = np.random.default_rng(3).uniform(0, 1, (len(act), 2)).astype(np.float32)
    gk0, gl0 = (g.cpu().numpy() for g in tree.J_backward(act, w, 2, 0.75))
    held = t2.debug_pool_used()

    def after(n):
        assert t2.debug_pool_used() == held, f"backward failing at allocation {n} kept memory"

    points, (gk, gl) = _each_failure(t2, lambda: tree.J_backward(act, w, 2, 0.75), after)
    assert points >= 1
    # the gradients are summed with FP32 atomics, whose order varies between
    # calls: equal to FP32 rounding, not bit for bit
    for got, want in ((gk.cpu().numpy(), gk0), (gl.cpu().numpy(), gl0)):
        np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-6 * np.abs(want).max())
    tree.free()


@pytest.mark.parametrize("flags", [0, 16])
def test_batch_every_allocation_failure(t2, flags):
    """Creating a batch plan that fails at any allocation returns ENOMEM and
    keeps no memory beyond the trees' own; the plan that is created gives
    each subset's trevr2_J rows."""
    cases = [_case(), workloads.random_case(900, 30, nb=2, seed=302)]
    trees = [_gpu_tree(t2, c) for c in cases]
    for tr in trees:
        tr.prepare(2)
    subs = [(0, np.arange(0, 1500, 3)), (1, np.arange(900)), (0, np.array([5, 5, 7]))]
    offsets = np.zeros(len(subs) + 1, np.int64)
    offsets[1:] = np.cumsum([len(m) for _, m in subs])
    tree_of = np.array([t for t, _ in subs], np.int32)
    active = np.concatenate([m for _, m in subs]).astype(np.int64)
    # the per-subset rows first: they grow the trees' own walk buffers
    refs = [trees[t].J(m, 2, 0.75, flags=flags).cpu().numpy() for t, m in subs]
    held = t2.debug_pool_used()

    def after(n):
        assert t2.debug_pool_used() == held, f"batch creation failing at allocation {n} kept memory"

    points, plan = _each_failure(
        t2, lambda: t2.Batch(trees, offsets, tree_of, nside=2, theta=0.75, flags=flags), after)
    assert points >= 3
    J = plan.run(torch.as_tensor(active, device="cuda")).cpu().numpy()
    plan.status()
    for s in range(len(subs)):
        np.testing.assert_array_equal(J[offsets[s]:offsets[s + 1]], refs[s])
    plan.free()
    assert t2.debug_pool_used() == held
    for tr in trees:
        tr.free()


def test_failed_autotune_leaves_no_half_plan(t2):
    """An autotune that fails while it times shapes on a prefix of the rows
    must not leave the plan walking only that prefix: runs are refused
    (EINVAL) until an autotune succeeds, and then give the full rows."""
    case = _case()
    tree = _gpu_tree(t2, case)
    rng = np.random.default_rng(5)
    active = rng.integers(0, len(case["pos"]), size=70000).astype(np.int64)  # > 65536 rows
    offsets = np.array([0, 30000, 70000], np.int64)
    tree_of = np.array([0, 0], np.int32)
    plan = t2.Batch([tree], offsets, tree_of, nside=2, theta=0.75)
    act = torch.as_tensor(active, device="cuda")
    ref = plan.run(act).cpu().numpy()
    plan.status()
    t2.debug_set(t2.DEBUG_FAIL_ALLOC, 0)  # the first shape that needs more buffers
    try:
        plan.autotune(act)
        failed = False
    except t2.TrevrError as e:
        assert e.code == ENOMEM, str(e)
        failed = True
    t2.debug_set(t2.DEBUG_FAIL_ALLOC, -1)
    assert failed
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        plan.run(act)
    plan.autotune(act)
    J = plan.run(act).cpu().numpy()
    plan.status()
    # another launch shape may round differently (never more than FP32 noise)
    np.testing.assert_allclose(J, ref, rtol=1e-5)
    plan.free()
    tree.free()


def test_source_stack_overflow_is_reported(t2):
    """With the source cut's stack capped below what a cut at small theta
    needs, the walk reports EINTERNAL ("stack overflow") instead of a wrong
    J, for the forward, per-bucket and adjoint walks; with the cap lifted the
    same tree gives the undisturbed J and a clear status."""
    case = workloads.random_case(1200, 400, nb=2, seed=303, clumped=True)
    tree = _gpu_tree(t2, case)
    act = case["active"][:64]
    ref = tree.J(act, 2, 0.2).cpu().numpy()
    t2.debug_set(t2.DEBUG_SOURCE_STACK, 4)
    for flags in (0, 16):
        with pytest.raises(t2.TrevrError, match="stack overflow") as e:
            tree.J(act, 2, 0.2, flags=flags)
        assert e.value.code == EINTERNAL
    with pytest.raises(t2.TrevrError, match="stack overflow"):
        tree.J_backward(act, np.ones((len(act), 2), np.float32), 2, 0.2)
    t2.debug_set(t2.DEBUG_SOURCE_STACK, 0)
    tree.status()
    np.testing.assert_array_equal(tree.J(act, 2, 0.2).cpu().numpy(), ref)
    tree.free()
