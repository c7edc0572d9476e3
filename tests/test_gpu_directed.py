"""Directed rays (trevr2_J_directed, Sec. 3.4.1) on the per-bucket walk: the
beam holding the target's direction from each bucket centre points at the
target.  J against the oracle (same bars as the other GPU tests) on ragged
cases with several flag sets, the accuracy geometries with the target at
their source, and the argument errors.
"""

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

BUCKET, PP, SOFT, THICK, LINEAR = 16, 32, 1, 2, 8


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


def _assert_J(J, ref, what):
    J = np.asarray(J, np.float64)
    assert np.all(np.isfinite(J)), what
    lit = ref > 1e-30
    assert np.all(J[~lit] <= 1e-29), what
    r = np.abs(J[lit] - ref[lit]) / ref[lit]
    med, mx = float(np.median(r)), float(r.max())
    assert med <= 1e-4 and mx <= 1e-3, f"{what}: median {med:.2e} max {mx:.2e}"


CASES = [
    dict(n_gas=1500, n_src=1, nb=2, seed=151, clumped=True, kappa_scale=30.0),
    dict(n_gas=800, n_src=15, nb=1, seed=152, n_active=300),
    dict(n_gas=1200, n_src=25, nb=3, seed=153, clumped=True, bucket=4, n_active=500),
]


@pytest.mark.parametrize("kw", CASES)
@pytest.mark.parametrize("nside", [1, 2, 4])
@pytest.mark.parametrize("extra", [0, SOFT | THICK, LINEAR, PP | THICK])
@pytest.mark.parametrize("where", ["source", "point"])
def test_directed_J_matches_oracle(t2, oracle_mod, kw, nside, extra, where):
    case = workloads.random_case(**kw)
    if where == "source":  # the brightest source
        target = case["pos"][int(np.argmax(case["lum"].sum(1)))]
    else:
        target = np.array([0.37, 0.61, 0.52])
    tree = _gpu_tree(t2, case)
    flags = BUCKET | extra
    J = tree.J(case["active"], nside, 0.75, flags=flags, target=target).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"], nside, 0.75, flags=flags,
                                                  target=target)
    _assert_J(J, ref, f"directed nside={nside} flags={flags} {where}")
    tree.free()


def test_directed_argument_errors(t2):
    case = workloads.random_case(300, 5, seed=154)
    tree = _gpu_tree(t2, case)
    with pytest.raises(t2.TrevrError, match="EINVAL"):  # needs BUCKET
        tree.J(case["active"], 2, 0.75, target=[0.5, 0.5, 0.5])
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        tree.J(case["active"], 2, 0.75, flags=BUCKET, target=[0.5, np.nan, 0.5])
    J = tree.J(case["active"], 2, 0.75, flags=BUCKET, target=[0.5, 0.5, 0.5]).cpu().numpy()
    assert np.all(np.isfinite(J))
    tree.free()


@pytest.mark.parametrize("name", ["source_two_clouds", "source_wall"])
def test_directed_accuracy_geometries(t2, oracle_mod, name):
    """The one-source tests of Sec. 3.4 with the beam aimed at the source:
    outer-sphere J and the escape/covering figures against the oracle."""
    from oracle import escape as esc
    case = workloads.CASES[name]()
    g = case["geometry"]
    act = case["active"]
    pts = case["pos"][act]
    tgt = g["sources"][0]
    tree = _gpu_tree(t2, case)
    J = tree.J(act, case["nside"], case["theta"], flags=BUCKET, target=tgt).cpu().numpy()[:, 0]
    ref = oracle_mod.OracleTree.from_case(case).J(act, case["nside"], case["theta"],
                                                  flags=BUCKET, target=tgt)[:, 0]
    r = np.abs(J - ref) / ref
    assert np.median(r) <= 1e-4 and r.max() <= 1e-3, (np.median(r), r.max())
    e, c = esc.figures(J, pts, g)
    e_o, c_o = esc.figures(ref, pts, g)
    assert abs(e - e_o) <= 1e-5 * e_o and abs(c - c_o) <= 2.0 / len(act)
    tree.free()
