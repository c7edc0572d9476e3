"""TREVR2_BUCKET: per-bucket beams (Sec. 2, Sec. 2.5.1).  One walk per leaf
that holds receivers, from the centre of its box; each receiver scales the
beam optical depth by its own distance over the projected one.  J against
the oracle's per-bucket walk (same bars as the other GPU tests), on ragged
cases, buckets larger than a warp, many staging passes, the benchmark field
and the accuracy geometries.
"""

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

BUCKET, SOFT, THICK, LINEAR = 16, 1, 2, 8


@pytest.fixture(scope="module")
def t2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_15235_gb300 import build_lib
    build_lib.build()
    import paper_2310_15235_gb300 as mod
    mod.load_library()
    assert mod.BUCKET == BUCKET
    return mod


def _gpu_tree(t2, case):
    return t2.build(case["pos"], case["mass"], case["kappa"], case["lum"], case["h"],
                    case["box_lo"], case["box_size"], case["bucket"])


def _assert_J(J, ref, what):
    J = np.asarray(J, np.float64)
    assert np.all(np.isfinite(J)), what
    r = np.abs(J - ref) / np.maximum(np.abs(ref), 1e-300)
    r[(J == 0) & (ref == 0)] = 0.0
    med, mx = float(np.median(r)), float(r.max())
    assert med <= 1e-4 and mx <= 1e-3, f"{what}: median {med:.2e} max {mx:.2e}"


CASES = [
    dict(n_gas=1500, n_src=30, nb=3, seed=101, clumped=True, kappa_scale=30.0),
    dict(n_gas=800, n_src=15, nb=1, seed=102, n_active=300),
    dict(n_gas=1200, n_src=25, nb=2, seed=103, clumped=True, bucket=4, n_active=500),
    dict(n_gas=2000, n_src=40, nb=2, seed=104, clumped=True, bucket=40),  # > 32 per leaf
    dict(n_gas=300, n_src=8, nb=4, seed=105, bucket=1),
]


@pytest.mark.parametrize("kw", CASES)
@pytest.mark.parametrize("nside", [1, 2, 4])
@pytest.mark.parametrize("extra", [0, SOFT | THICK, LINEAR])
def test_bucket_J_matches_oracle(t2, oracle_mod, kw, nside, extra):
    case = workloads.random_case(**kw)
    tree = _gpu_tree(t2, case)
    flags = BUCKET | extra
    J = tree.J(case["active"], nside, 0.75, flags=flags).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"], nside, 0.75, flags=flags)
    _assert_J(J, ref, f"bucket nside={nside} flags={flags}")
    tree.free()


def test_bucket_receivers_in_any_order_with_repeats(t2, oracle_mod):
    """Unsorted receivers, repeated ones and a band subset: rows land in the
    caller's order and a repeated receiver gets the same row."""
    case = workloads.random_case(1000, 20, nb=3, seed=106, clumped=True)
    rng = np.random.default_rng(5)
    act = rng.integers(0, len(case["pos"]), size=700)
    tree = _gpu_tree(t2, case)
    J = tree.J(act, 2, 0.75, bands=[2, 0], flags=BUCKET).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(act, 2, 0.75, flags=BUCKET)[:, [2, 0]]
    _assert_J(J, ref, "unsorted")
    first = {}
    for r, i in enumerate(act):
        if i in first:
            np.testing.assert_array_equal(J[r], J[first[i]])
        else:
            first[i] = r
    tree.free()


def test_bucket_many_sources_many_passes(t2, oracle_mod):
    """theta -> 0 opens every cell: each bucket sees more sources than one
    staging pass holds, with 40-element leaves (two receiver chunks)."""
    case = workloads.random_case(900, 2600, nb=2, seed=107, clumped=True, bucket=40)
    tree = _gpu_tree(t2, case)
    J = tree.J(case["active"], 2, 1e-6, flags=BUCKET).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"], 2, 1e-6, flags=BUCKET)
    _assert_J(J, ref, "many sources")
    tree.free()


def test_bucket_equals_per_receiver_at_leaf_centres(t2, oracle_mod):
    """Elements at the centres of a 16^3 grid, bucket 1: the bucket walk
    starts where the receiver walk does, so the two GPU paths agree."""
    rng = np.random.default_rng(108)
    idx = np.arange(16, dtype=np.float64)
    pos = (np.stack(np.meshgrid(idx, idx, idx, indexing="ij"), -1).reshape(-1, 3) + 0.5) / 16
    n = len(pos)
    lum = np.where(rng.uniform(size=(n, 1)) < 0.05, rng.uniform(0.1, 1.0, (n, 2)), 0.0)
    case = workloads._pack("grid16", pos, rng.uniform(0.5, 1.5, n) / n,
                           rng.uniform(0.0, 40.0, (n, 2)), lum, np.full(n, 1 / 16),
                           np.arange(n), 2, 0.75, bucket=1)
    tree = _gpu_tree(t2, case)
    for flags in (0, SOFT | THICK):
        J0 = tree.J(case["active"], 2, 0.75, flags=flags).cpu().numpy()
        J1 = tree.J(case["active"], 2, 0.75, flags=flags | BUCKET).cpu().numpy()
        np.testing.assert_allclose(J1, J0, rtol=2e-6, atol=0)
    tree.free()


def test_bucket_bad_receiver_and_unsupported_calls(t2):
    case = workloads.random_case(500, 10, nb=2, seed=109)
    tree = _gpu_tree(t2, case)
    n = len(case["pos"])
    act = torch.tensor([3, n + 5, 7, -1, 3], dtype=torch.int64, device="cuda")
    out = torch.empty((5, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        tree.J(act, 2, 0.75, flags=BUCKET, out=out)
    J = out.cpu().numpy()
    assert np.all(np.isnan(J[[1, 3]])) and np.all(np.isfinite(J[[0, 2, 4]]))
    np.testing.assert_array_equal(J[0], J[4])
    tree.status()
    with pytest.raises(t2.TrevrError, match="EUNSUPPORTED"):
        tree.J_backward(case["active"][:10], np.ones((10, 2), np.float32), 2, 0.75,
                        flags=BUCKET)
    # batch plans take BUCKET (tests/test_gpu_batch.py); PP and CSM need it
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        t2.Batch([tree], [0, 5], [0], flags=t2.PP)
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        t2.Batch([tree], [0, 5], [0], flags=t2.CSM)
    assert tree.J(np.zeros(0, np.int64), 2, 0.75, flags=BUCKET).shape == (0, 2)
    tree.free()


def test_bucket_clumpy_2M_sampled(t2, oracle_mod):
    """The benchmark field (2,097,152 receivers, nside 4, theta 0.5) with
    per-bucket beams; 512 sampled receivers against the oracle."""
    case = workloads.clumpy_multiband()
    tree = _gpu_tree(t2, case)
    J = tree.J(case["active"], case["nside"], case["theta"], flags=BUCKET).cpu().numpy()
    assert np.all(np.isfinite(J)) and np.all(J >= 0)
    idx = np.sort(np.random.default_rng(1).choice(len(case["active"]), 512, replace=False))
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"][idx], case["nside"],
                                                  case["theta"], flags=BUCKET)
    _assert_J(J[idx], ref, "bucket clumpy 2M")
    tree.free()


@pytest.mark.parametrize("name", ["two_sources_cloud", "source_two_clouds", "source_wall"])
def test_bucket_accuracy_geometries(t2, oracle_mod, name):
    """The accuracy tests of Sec. 3.3-3.4 with the paper's per-bucket beams:
    the outer-sphere J and its escape/covering figures against the oracle."""
    from oracle import escape as esc
    case = workloads.CASES[name]()
    g = case["geometry"]
    act = case["active"]
    pts = case["pos"][act]
    tree = _gpu_tree(t2, case)
    J = tree.J(act, case["nside"], case["theta"], flags=BUCKET).cpu().numpy()[:, 0]
    ref = oracle_mod.OracleTree.from_case(case).J(act, case["nside"], case["theta"],
                                                  flags=BUCKET)[:, 0]
    J_vac = esc.exact_J(pts, g, absorb=False)
    lit = ref > 1e-30 * J_vac
    assert np.all(J[~lit] <= 1e-29 * J_vac[~lit])
    r = np.abs(J[lit] - ref[lit]) / ref[lit]
    assert np.median(r) <= 1e-4 and r.max() <= 1e-3, (np.median(r), r.max())
    e, c = esc.figures(J, pts, g)
    e_o, c_o = esc.figures(ref, pts, g)
    assert abs(e - e_o) <= 1e-5 * e_o and abs(c - c_o) <= 2.0 / len(act)
    tree.free()


@pytest.mark.parametrize("extra", [0, 32 | 2, 64])
def test_bucket_rows_do_not_depend_on_the_other_receivers(t2, extra):
    """A receiver's J comes from its bucket's walk alone: the rows of any
    subset of receivers, in any order, equal those of the full walk bit for
    bit (what makes Morton-range sharding exact)."""
    case = workloads.random_case(3000, 60, nb=2, seed=111, clumped=True)
    tree = _gpu_tree(t2, case)
    flags = BUCKET | extra
    act = case["active"]
    J = tree.J(act, 2, 0.75, flags=flags).cpu().numpy()
    rng = np.random.default_rng(9)
    for m in (1, 37, 1000):
        sub = rng.choice(len(act), m, replace=False)
        Js = tree.J(act[sub], 2, 0.75, flags=flags).cpu().numpy()
        np.testing.assert_array_equal(Js, J[sub])
    tree.free()
