"""CUDA path (through the C ABI) against the FP64 oracle.

Bars: keys, permutation and topology bit-exact; per-node luminosity, centre,
B and bucket absorption within 1e-6 relative (they are FP64 sums rounded once
to FP32, or FP64); per-direction absorption tables within 1e-5 relative; J
within 1e-4 relative (median) and 1e-3 (max) over all receivers.
"""

import math

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
    den = np.maximum(np.abs(b), 1e-300)
    r = np.abs(a - b) / den
    r[(a == 0) & (b == 0)] = 0.0
    return r


def _assert_J(J, ref, what=""):
    assert np.all(np.isfinite(J)), what
    r = _rel(J, ref)
    med, mx = float(np.median(r)), float(r.max())
    assert med <= J_MEDIAN_TOL and mx <= J_MAX_TOL, f"{what}: median {med:.3e} max {mx:.3e}"
    return med, mx


TOPOLOGY_CASES = [
    ("clumped", dict(n_gas=700, n_src=30, nb=2, seed=1, clumped=True)),
    ("uniform_b1", dict(n_gas=300, n_src=5, nb=1, seed=2, bucket=1)),
    ("ragged", dict(n_gas=2049, n_src=3, nb=3, seed=3, clumped=True, bucket=5)),
    ("tiny", dict(n_gas=1, n_src=1, nb=1, seed=4)),
]


def _case(kind, kw):
    return workloads.random_case(**kw)


@pytest.mark.parametrize("name,kw", TOPOLOGY_CASES)
def test_keys_perm_topology_bit_exact(t2, oracle_mod, name, kw):
    case = _case(name, kw)
    if name == "clumped":  # coincident elements force a depth-63 leaf
        case["pos"][:20] = case["pos"][0]
    tree = _gpu_tree(t2, case)
    ot = oracle_mod.OracleTree.from_case(case)
    e = ot.export()
    assert tree.n_nodes == ot.num_nodes and tree.max_depth == ot.max_depth
    perm = tree.export("perm").cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(perm, e["perm"])
    keys = tree.export("keys").cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(keys, e["keys"][e["perm"]])
    for f in ("prefix", "depth", "first", "count", "child", "parent"):
        got = tree.export(f).cpu().numpy()
        want = e[f]
        if f == "prefix":
            got = got.view(np.uint64)
        np.testing.assert_array_equal(got.astype(want.dtype), want, err_msg=f)
    tree.free()


@pytest.mark.parametrize("name,kw", TOPOLOGY_CASES[:3])
def test_aggregates(t2, oracle_mod, name, kw):
    case = _case(name, kw)
    tree = _gpu_tree(t2, case)
    ag = oracle_mod.OracleTree.from_case(case).aggregates()
    L = tree.export("lum").cpu().numpy()
    np.testing.assert_allclose(L, ag["L"], rtol=1e-6, atol=0)
    np.testing.assert_allclose(tree.export("centre").cpu().numpy(), ag["c"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(tree.export("B").cpu().numpy(), ag["B"], rtol=1e-13, atol=0)
    np.testing.assert_allclose(tree.export("alpha_leaf").cpu().numpy(), ag["alpha_leaf"],
                               rtol=1e-6, atol=0)
    tree.free()


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_alpha_tables(t2, oracle_mod, nside):
    case = workloads.random_case(3000, 10, nb=3, seed=5, clumped=True, kappa_scale=200.0)
    tree = _gpu_tree(t2, case)
    got = tree.alpha_table(nside).cpu().numpy()
    want = oracle_mod.OracleTree.from_case(case).alpha_table(nside)
    assert got.shape == want.shape
    r = _rel(got, want)
    assert r.max() <= 1e-5, r.max()
    tree.free()


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16])
def test_healpix(t2, oracle_mod, nside):
    v = t2.healpix_pix2vec(nside).cpu().numpy()
    np.testing.assert_allclose(v, oracle_mod.pix2vec(nside), rtol=0, atol=2e-15)
    rng = np.random.default_rng(nside)
    u = rng.standard_normal((200_000, 3))
    u[:1000] *= 1e-3  # short vectors stress the FP32 guard band
    u = np.concatenate([u, oracle_mod.pix2vec(nside)])
    got = t2.healpix_vec2pix(nside, u).cpu().numpy()
    np.testing.assert_array_equal(got, oracle_mod.vec2pix(nside, u))


@pytest.mark.parametrize("offset", [False, True])
def test_J_uniform_point_source(t2, oracle_mod, offset):
    case = workloads.uniform_point_source(offset=offset)
    tree = _gpu_tree(t2, case)
    J = tree.J(case["active"], case["nside"], case["theta"]).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"], case["nside"], case["theta"])
    _assert_J(J, ref, "uniform point source")
    # and the closed form L e^{-kappa rho r}/(4 pi r^2)
    r = np.linalg.norm(case["pos"][case["active"]] - case["pos"][-1], axis=1)
    closed = np.exp(-2.0 * r) / (4 * np.pi * r * r)
    assert np.median(_rel(J[:, 0], closed)) <= J_MEDIAN_TOL
    tree.free()


def test_J_stromgren_like(t2, oracle_mod):
    case = workloads.stromgren_like()
    tree = _gpu_tree(t2, case)
    J = tree.J(case["active"], case["nside"], case["theta"]).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"], case["nside"], case["theta"])
    _assert_J(J, ref, "stromgren-like")
    tree.free()


RANDOM_J = [
    dict(n_gas=900, n_src=40, nb=1, seed=10, nside=1, theta=0.3),
    dict(n_gas=1500, n_src=25, nb=2, seed=11, nside=2, theta=0.75, clumped=True),
    dict(n_gas=1200, n_src=60, nb=3, seed=12, nside=4, theta=0.5, clumped=True, bucket=4),
    dict(n_gas=800, n_src=15, nb=4, seed=13, nside=8, theta=1.5, kappa_scale=50.0),
    dict(n_gas=500, n_src=30, nb=3, seed=14, nside=2, theta=0.75, bucket=1, n_active=333),
]


@pytest.mark.parametrize("kw", RANDOM_J)
@pytest.mark.parametrize("flags", [0, 1, 2, 3])
def test_J_random_cases(t2, oracle_mod, kw, flags):
    kw = dict(kw)
    nside, theta = kw.pop("nside"), kw.pop("theta")
    case = workloads.random_case(nside=nside, theta=theta, **kw)
    tree = _gpu_tree(t2, case)
    J = tree.J(case["active"], nside, theta, flags=flags).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"], nside, theta, flags=flags)
    _assert_J(J, ref, f"{kw} flags={flags}")
    tree.free()


def test_J_band_selection_and_order(t2, oracle_mod):
    case = workloads.random_case(700, 20, nb=4, seed=15, clumped=True)
    tree = _gpu_tree(t2, case)
    full = tree.J(case["active"], 2, 0.75).cpu().numpy()
    sel = tree.J(case["active"], 2, 0.75, bands=[3, 0, 2]).cpu().numpy()
    np.testing.assert_array_equal(sel, full[:, [3, 0, 2]])
    tree.free()


def test_J_many_sources_multi_pass(t2, oracle_mod):
    """More sources per receiver than one warp's buffers hold (theta -> 0
    opens everything): the walk takes several passes over the cut."""
    case = workloads.random_case(400, 2600, nb=2, seed=16, clumped=True, n_active=150)
    tree = _gpu_tree(t2, case)
    J = tree.J(case["active"], 2, 1e-6).cpu().numpy()
    ot = oracle_mod.OracleTree.from_case(case)
    ref, st = ot.J(case["active"], 2, 1e-6, stats=True)
    assert st[:, 3].max() > 2048
    _assert_J(J, ref, "multi-pass")
    tree.free()


def test_J_receivers_that_are_sources_and_duplicates(t2, oracle_mod):
    case = workloads.random_case(300, 50, nb=2, seed=17, clumped=True, n_active=200)
    case["pos"][310] = case["pos"][5]  # a source on top of a gas element
    case["pos"][311] = case["pos"][312]
    tree = _gpu_tree(t2, case)
    act = np.concatenate([case["active"], [310, 311, 312, 5]])
    J = tree.J(act, 2, 0.75).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(act, 2, 0.75)
    _assert_J(J, ref, "sources as receivers")
    tree.free()


def test_J_edge_cases(t2, oracle_mod):
    case = workloads.random_case(200, 5, nb=2, seed=18)
    tree = _gpu_tree(t2, case)
    out = tree.J(np.zeros(0, dtype=np.int64), 2, 0.75)
    assert out.shape == (0, 2)
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        tree.J(np.array([0, 205, 3]), 2, 0.75)
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        tree.J(np.array([0]), 3, 0.75)  # nside not a power of two
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        tree.J(np.array([0]), 2, -1.0)
    with pytest.raises(t2.TrevrError, match="EUNSUPPORTED"):
        tree.J(np.array([0]), 32, 0.75)
    tree.free()
    # one element alone sees nothing
    one = workloads.random_case(1, 0, nb=1, seed=19)
    tr = _gpu_tree(t2, one)
    assert tr.J([0], 2, 0.75).cpu().item() == 0.0
    tr.free()
    # coincident positions: automatic cube of edge 1
    same = workloads.random_case(20, 2, nb=1, seed=20)
    same["pos"][:] = 0.25
    tr = t2.build(same["pos"], same["mass"], same["kappa"], same["lum"], same["h"])
    assert tr.box_size == 1.0 and tr.max_depth == 63
    assert np.all(tr.J(np.arange(22), 2, 0.75).cpu().numpy() == 0.0)
    tr.free()
    # invalid inputs are rejected
    bad = workloads.random_case(50, 2, nb=1, seed=21)
    bad["pos"][3, 1] = np.nan
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        _gpu_tree(t2, bad)
    neg = workloads.random_case(50, 2, nb=1, seed=21)
    neg["kappa"][4, 0] = -1.0
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        _gpu_tree(t2, neg)
    out_of_box = workloads.random_case(50, 2, nb=1, seed=22)
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        t2.build(out_of_box["pos"], out_of_box["mass"], out_of_box["kappa"], out_of_box["lum"],
                 None, [0.2, 0.2, 0.2], 0.5)


def test_J_general_box(t2, oracle_mod):
    """A root cube other than the unit box (positions in other units)."""
    case = workloads.random_case(900, 30, nb=2, seed=23, clumped=True)
    case["pos"] = case["pos"] * 3.0e3 - 1.0e3
    case["box_lo"] = np.array([-1.0e3, -1.0e3, -1.0e3])
    case["box_size"] = 3.0e3
    case["h"] = case["h"] * 3.0e3
    for flags in (0, 3):
        tree = _gpu_tree(t2, case)
        J = tree.J(case["active"], 2, 0.75, flags=flags).cpu().numpy()
        ref = oracle_mod.OracleTree.from_case(case).J(case["active"], 2, 0.75, flags=flags)
        _assert_J(J, ref, f"general box flags={flags}")
        tree.free()


@pytest.fixture(scope="module")
def clumpy():
    return workloads.clumpy_multiband()


def test_J_clumpy_2M_sampled(t2, oracle_mod, clumpy):
    """The 2,097,152-receiver clumpy 3-band field (nside 4, theta 0.5), in the
    benchmark's configuration; 768 sampled receivers against the oracle."""
    case = clumpy
    tree = _gpu_tree(t2, case)
    J = tree.J(case["active"], case["nside"], case["theta"]).cpu().numpy()
    assert J.shape == (2_097_152, 3) and np.all(np.isfinite(J)) and np.all(J >= 0)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(len(case["active"]), 768, replace=False))
    ot = oracle_mod.OracleTree.from_case(case)
    ref = ot.J(case["active"][idx], case["nside"], case["theta"])
    _assert_J(J[idx], ref, "clumpy 2M sampled")
    tree.free()


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_J_receivers_on_root_faces(t2, oracle_mod, nside):
    """Receivers exactly on the faces of the root cube, seen along beams with
    zero components (nside 1 and 2 have beams along the axes and in the
    equatorial plane): half-open boxes decide which cells such beams cross."""
    case = workloads.random_case(1200, 30, nb=2, seed=24, clumped=True, n_active=400)
    rng = np.random.default_rng(5)
    for i in rng.choice(1200, 60, replace=False):
        case["pos"][i, rng.integers(0, 3)] = rng.choice([0.0, 1.0])
    act = np.unique(np.concatenate([case["active"], np.flatnonzero(
        ((case["pos"][:1200] == 0.0) | (case["pos"][:1200] == 1.0)).any(1))]))
    tree = _gpu_tree(t2, case)
    J = tree.J(act, nside, 0.75).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(act, nside, 0.75)
    _assert_J(J, ref, f"root faces nside={nside}")
    tree.free()


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_J_receivers_on_split_planes(t2, oracle_mod, nside):
    """Receivers exactly on internal split planes (dyadic coordinates, one or
    two of them), seen along beams with zero components: such a beam lies in
    the plane, and the half-open cells put it in the upper half only."""
    case = workloads.random_case(1200, 30, nb=2, seed=25, clumped=True, n_active=300)
    rng = np.random.default_rng(6)
    planes = np.array([0.5, 0.25, 0.75, 0.125, 0.375, 0.625, 0.875])
    moved = rng.choice(1200, 90, replace=False)
    for j, i in enumerate(moved):
        axes = rng.choice(3, 1 + j % 2, replace=False)
        case["pos"][i, axes] = rng.choice(planes, len(axes))
    act = np.unique(np.concatenate([case["active"], moved])).astype(np.int64)
    tree = _gpu_tree(t2, case)
    J = tree.J(act, nside, 0.75).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(act, nside, 0.75)
    _assert_J(J, ref, f"split planes nside={nside}")
    Jb = tree.J(act, nside, 0.75, flags=16).cpu().numpy()
    refb = oracle_mod.OracleTree.from_case(case).J(act, nside, 0.75, flags=16)
    _assert_J(Jb, refb, f"split planes, per bucket, nside={nside}")
    tree.free()


def test_kernels_run_as_sm103a(t2):
    """The loaded kernels are the sm_103a build (the library is compiled for
    that architecture only)."""
    assert t2.kernel_binary_version() == 103
