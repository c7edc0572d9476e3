"""The allocation-free entry point trevr2_J_noalloc, called through the C ABI.

It serves callers that cannot let a library allocate device memory; its walk
buffers live in one fixed device array inside the library.  Its output must
match trevr2_J (the allocating entry point) within the tolerances of the
other parity tests, on two calls in a row (the array keeps the previous
call's contents, so the second call checks that nothing stale leaks in).
This file is collected last on purpose.
"""

import ctypes as C

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


def _noalloc(t2, tree, active, nside, theta, nb, flags=0):
    lib = t2.load_library()
    act = torch.as_tensor(np.ascontiguousarray(active), dtype=torch.int64, device=tree.device)
    out = torch.full((act.numel(), nb), -1.0, dtype=torch.float32, device=tree.device)
    rc = lib.trevr2_J_noalloc(tree._h, C.c_void_p(act.data_ptr()), act.numel(), nside,
                              C.c_float(theta), None, nb, flags, C.c_void_p(out.data_ptr()),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    r = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
    r[(a == 0) & (b == 0)] = 0.0
    return r


@pytest.mark.parametrize("theta,n_src", [(0.75, 60), (1e-6, 700)])
def test_noalloc_matches_allocating_entry_point(t2, theta, n_src):
    case = workloads.random_case(3000, n_src, nb=3, seed=31, clumped=True, n_active=1500)
    nside = 2
    tree = t2.build(case["pos"], case["mass"], case["kappa"], case["lum"], case["h"],
                    case["box_lo"], case["box_size"], case["bucket"])
    # without tables for this nside the entry point refuses instead of allocating
    rc, _ = _noalloc(t2, tree, case["active"], nside, theta, 3)
    assert rc == -1 and b"trevr2_prepare" in t2.load_library().trevr2_last_error()
    tree.prepare(nside)
    ref = tree.J(case["active"], nside, theta).cpu().numpy()
    for call in range(2):
        rc, out = _noalloc(t2, tree, case["active"], nside, theta, 3)
        assert rc == 0, t2.load_library().trevr2_last_error()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        r = _rel(got, ref)
        assert np.median(r) <= 1e-4 and r.max() <= 1e-3, (call, np.median(r), r.max())
    tree.free()


def test_noalloc_matches_oracle(t2, oracle_mod):
    """The allocation-free walk against the FP64 oracle directly, on a small
    case with ragged sizes, twice in a row, with and without SOFT | THICK."""
    case = workloads.random_case(700, 35, nb=2, seed=33, clumped=True, n_active=301)
    tree = t2.build(case["pos"], case["mass"], case["kappa"], case["lum"], case["h"],
                    case["box_lo"], case["box_size"], case["bucket"])
    tree.prepare(2)
    ot = oracle_mod.OracleTree.from_case(case)
    for flags in (0, 3):
        ref = ot.J(case["active"], 2, 0.75, flags=flags)
        for call in range(2):
            rc, out = _noalloc(t2, tree, case["active"], 2, 0.75, 2, flags)
            assert rc == 0, t2.load_library().trevr2_last_error()
            r = _rel(out.cpu().numpy(), ref)
            assert np.median(r) <= 1e-4 and r.max() <= 1e-3, (flags, call, np.median(r), r.max())
    tree.free()
