"""TREVR2_LINEAR: internal cells take the volume-weighted linear average of
their halves' absorption (the scheme Sec. 2.6 compares Eq. transmissionavg
with) instead of the transmission average.  J, the batched rows and the
adjoint under this flag against the oracle (same bars as the other GPU
tests)."""

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

LINEAR = 8


@pytest.fixture(scope="module")
def t2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_15235_gb300 import build_lib
    build_lib.build()
    import paper_2310_15235_gb300 as mod
    mod.load_library()
    assert mod.LINEAR == LINEAR
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
    dict(n_gas=1500, n_src=30, nb=3, seed=81, clumped=True, kappa_scale=60.0, n_active=300),
    dict(n_gas=800, n_src=15, nb=1, seed=82, n_active=200),
    dict(n_gas=1200, n_src=25, nb=2, seed=83, clumped=True, bucket=4, n_active=250),
]


@pytest.mark.parametrize("kw", CASES)
@pytest.mark.parametrize("nside", [1, 2, 4])
@pytest.mark.parametrize("extra", [0, 1, 2])
def test_linear_J_matches_oracle(t2, oracle_mod, kw, nside, extra):
    case = workloads.random_case(**kw)
    tree = _gpu_tree(t2, case)
    flags = LINEAR | extra
    J = tree.J(case["active"], nside, 0.75, flags=flags).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"], nside, 0.75, flags=flags)
    _assert_J(J, ref, f"linear nside={nside} flags={flags}")
    tree.free()


def test_linear_never_brighter_than_transmission(t2):
    """alpha_lin >= alpha_trans in every cell and direction, so J_lin <= J_trans
    for every receiver (up to FP32 rounding), and clumpy fields differ."""
    case = workloads.random_case(900, 30, nb=2, seed=72, clumped=True, kappa_scale=60.0,
                                 n_active=150)
    tree = _gpu_tree(t2, case)
    Jt = tree.J(case["active"], 2, 0.75).cpu().numpy().astype(np.float64)
    Jl = tree.J(case["active"], 2, 0.75, flags=LINEAR).cpu().numpy().astype(np.float64)
    # both tables are cached side by side: the transmission rows are unchanged
    Jt2 = tree.J(case["active"], 2, 0.75).cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(Jt, Jt2)
    assert np.all(Jl <= Jt * (1 + 1e-5))
    lit = Jt > 0  # some receivers' J underflows FP32 under either average
    assert ((Jt[lit] - Jl[lit]) / Jt[lit]).max() > 1e-2
    tree.free()


def test_linear_batched_rows_equal_plain(t2):
    cases = [workloads.random_case(900, 25, nb=2, seed=84, clumped=True),
             workloads.random_case(600, 20, nb=2, seed=85)]
    trees = [_gpu_tree(t2, c) for c in cases]
    rng = np.random.default_rng(4)
    subs = []
    for k in range(6):
        t = k % 2
        n = len(cases[t]["pos"])
        subs.append((t, np.sort(rng.choice(n, int(rng.integers(1, n)), replace=False))))
    offsets = np.zeros(len(subs) + 1, np.int64)
    offsets[1:] = np.cumsum([len(m) for _, m in subs])
    tree_of = np.array([t for t, _ in subs], np.int32)
    active = np.concatenate([m for _, m in subs])
    J = t2.J_batched(trees, active, offsets, tree_of, 2, 0.75, LINEAR).cpu().numpy()
    for s, (t, m) in enumerate(subs):
        single = trees[t].J(m, 2, 0.75, flags=LINEAR).cpu().numpy()
        np.testing.assert_array_equal(J[offsets[s]:offsets[s + 1]], single)
    for tr in trees:
        tr.free()


@pytest.mark.parametrize("extra", [0, 2])
def test_linear_backward_matches_oracle_gradient(t2, oracle_mod, extra):
    case = workloads.random_case(600, 20, nb=2, seed=86, clumped=True, n_active=120)
    tree = _gpu_tree(t2, case)
    act = case["active"]
    flags = LINEAR | extra
    gJ = np.random.default_rng(7).uniform(0.0, 1.0, size=(len(act), 2)).astype(np.float32)
    gk, gl = tree.J_backward(act, gJ, 2, 0.75, flags=flags)
    gk, gl = gk.cpu().numpy(), gl.cpu().numpy()
    ot = oracle_mod.OracleTree.from_case(case)
    rng = np.random.default_rng(0)
    lit = np.flatnonzero(case["lum"].sum(1) > 0)
    massive = np.flatnonzero(case["mass"] > 0)
    params = [("lum", int(e), b) for e in lit for b in range(2)]
    params += [("kappa", int(e), int(rng.integers(0, 2))) for e in rng.choice(massive, 150, False)]
    want = np.array([float((ot.J_deriv(act, 2, 0.75, w, e, b, flags) * gJ).sum())
                     for w, e, b in params])
    got = np.array([gk[e, b] if w == "kappa" else gl[e, b] for w, e, b in params])
    scale = np.abs(want).max()
    big = np.abs(want) >= 1e-3 * scale
    rel = np.abs(got - want)[big] / np.abs(want[big])
    assert np.median(rel) <= 1e-4 and rel.max() <= 2e-3, (np.median(rel), rel.max())
    assert (np.abs(got - want)[~big] <= 2e-6 * scale).all()
    tree.free()


def test_linear_clumpy_2M_sampled(t2, oracle_mod):
    """The benchmark field (2,097,152 receivers, nside 4, theta 0.5) under
    linear averaging; 512 sampled receivers against the oracle."""
    case = workloads.clumpy_multiband()
    tree = _gpu_tree(t2, case)
    J = tree.J(case["active"], case["nside"], case["theta"], flags=LINEAR).cpu().numpy()
    idx = np.sort(np.random.default_rng(1).choice(len(case["active"]), 512, replace=False))
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"][idx], case["nside"],
                                                  case["theta"], flags=LINEAR)
    _assert_J(J[idx], ref, "linear clumpy 2M")
    tree.free()
