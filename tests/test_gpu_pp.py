"""TREVR2_PP with TREVR2_BUCKET: particle-particle absorption inside each
bucket's p-p radius (Sec. 2.4) on the per-bucket walk.  J against the
oracle (same bars as the other GPU tests) on ragged cases, the closed form
of one absorber, the benchmark field and the accuracy geometries; the
capacity and flag errors.
"""

import math

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
    assert mod.PP == PP
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
    dict(n_gas=1500, n_src=30, nb=3, seed=131, clumped=True, kappa_scale=30.0),
    dict(n_gas=800, n_src=15, nb=1, seed=132, n_active=300),
    dict(n_gas=1200, n_src=25, nb=2, seed=133, clumped=True, bucket=4, n_active=500),
    dict(n_gas=2000, n_src=40, nb=2, seed=134, clumped=True, bucket=40),
]


@pytest.mark.parametrize("kw", CASES)
@pytest.mark.parametrize("nside", [1, 2, 4])
@pytest.mark.parametrize("extra", [0, SOFT | THICK, LINEAR])
def test_pp_J_matches_oracle(t2, oracle_mod, kw, nside, extra):
    case = workloads.random_case(**kw)
    tree = _gpu_tree(t2, case)
    flags = BUCKET | PP | extra
    J = tree.J(case["active"], nside, 0.75, flags=flags).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"], nside, 0.75, flags=flags)
    _assert_J(J, ref, f"pp nside={nside} flags={flags}")
    tree.free()


def test_pp_lattice_varied_h(t2, oracle_mod):
    """A jittered 24^3 lattice with element sizes varied by 3x and clumpy
    opacity: buckets whose p-p radius grows over several steps."""
    rng = np.random.default_rng(135)
    n = 24
    gpos = workloads.jittered_lattice(n, rng)
    ng = n ** 3
    spos = rng.uniform(0, 1, (60, 3))
    pos = np.concatenate([gpos, spos])
    mass = np.concatenate([np.full(ng, 1.0 / ng), np.zeros(60)])
    kappa = np.concatenate([rng.lognormal(1.0, 1.5, (ng, 2)), np.zeros((60, 2))])
    lum = np.concatenate([np.zeros((ng, 2)), rng.uniform(0.1, 1, (60, 2))])
    h = np.concatenate([rng.uniform(0.5, 1.5, ng) / n, np.full(60, 1.0 / n)])
    act = np.sort(rng.choice(ng, 3000, replace=False))
    case = workloads._pack("lattice_pp", pos, mass, kappa, lum, h, act, 2, 0.75)
    tree = _gpu_tree(t2, case)
    ot = oracle_mod.OracleTree.from_case(case)
    for nside, flags in [(2, BUCKET | PP), (4, BUCKET | PP | THICK)]:
        J = tree.J(act, nside, 0.75, flags=flags).cpu().numpy()
        _assert_J(J, ot.J(act, nside, 0.75, flags=flags), f"lattice nside={nside}")
    tree.free()


def test_pp_single_absorber_closed_form(t2):
    """One absorber at impact parameter b from the receiver-star segment, all
    in the root leaf: J = L e^{-kappa 3 m (1 - b/h) / (pi h^2)} / (4 pi r^2)."""
    J0 = 1.0 / (4 * np.pi * 0.4 ** 2)
    for b in (0.0, 0.03, 0.07, 0.12):
        pos = np.array([[0.3, 0.5, 0.5], [0.7, 0.5, 0.5], [0.5, 0.5 + b, 0.5]])
        case = workloads._pack("pp1", pos, np.array([1e-3, 0.0, 0.002]),
                               np.array([[0.0, 0.0], [0.0, 0.0], [30.0, 7.0]]),
                               np.array([[0.0, 0.0], [1.0, 1.0], [0.0, 0.0]]),
                               np.array([0.05, 0.05, 0.1]), np.array([0]), 2, 0.75)
        h, m = float(case["h"][2]), float(case["mass"][2])
        kap = case["kappa"][2].astype(np.float64)
        tree = _gpu_tree(t2, case)
        J = tree.J([0], 2, 0.75, flags=BUCKET | PP).cpu().numpy()[0]
        tau = kap * 3 * m / (math.pi * h * h) * max(0.0, 1 - b / h)
        np.testing.assert_allclose(J, J0 * np.exp(-tau), rtol=2e-5)
        tree.free()


def test_pp_capacity_and_flag_errors(t2):
    # element sizes far above the spacing: every bucket's sphere holds all
    case = workloads.random_case(10000, 10, nb=1, seed=136, n_active=50)
    case["h"][:] = 0.3
    tree = _gpu_tree(t2, case)
    with pytest.raises(t2.TrevrError, match="EUNSUPPORTED"):
        tree.J(case["active"], 2, 0.75, flags=BUCKET | PP)
    tree.status()
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        tree.J(case["active"], 2, 0.75, flags=PP)
    # the tree stays usable
    J = tree.J(case["active"], 2, 0.75, flags=BUCKET).cpu().numpy()
    assert np.all(np.isfinite(J))
    tree.free()


def test_pp_clumpy_2M_sampled(t2, oracle_mod):
    """The benchmark field (2,097,152 receivers, nside 4, theta 0.5) with
    per-bucket beams and p-p absorption; 512 sampled receivers against the
    oracle."""
    case = workloads.clumpy_multiband()
    tree = _gpu_tree(t2, case)
    flags = BUCKET | PP
    J = tree.J(case["active"], case["nside"], case["theta"], flags=flags).cpu().numpy()
    assert np.all(np.isfinite(J)) and np.all(J >= 0)
    idx = np.sort(np.random.default_rng(1).choice(len(case["active"]), 512, replace=False))
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"][idx], case["nside"],
                                                  case["theta"], flags=flags)
    _assert_J(J[idx], ref, "pp clumpy 2M")
    tree.free()


@pytest.mark.parametrize("name", ["two_sources_cloud", "source_two_clouds", "source_wall"])
def test_pp_accuracy_geometries(t2, oracle_mod, name):
    """The accuracy tests of Sec. 3.3-3.4 with the paper's full near field:
    outer-sphere J and the escape/covering figures against the oracle."""
    from oracle import escape as esc
    case = workloads.CASES[name]()
    g = case["geometry"]
    act = case["active"]
    pts = case["pos"][act]
    flags = BUCKET | PP
    tree = _gpu_tree(t2, case)
    J = tree.J(act, case["nside"], case["theta"], flags=flags).cpu().numpy()[:, 0]
    ref = oracle_mod.OracleTree.from_case(case).J(act, case["nside"], case["theta"],
                                                  flags=flags)[:, 0]
    J_vac = esc.exact_J(pts, g, absorb=False)
    lit = ref > 1e-30 * J_vac
    assert np.all(J[~lit] <= 1e-29 * J_vac[~lit])
    r = np.abs(J[lit] - ref[lit]) / ref[lit]
    assert np.median(r) <= 1e-4 and r.max() <= 1e-3, (np.median(r), r.max())
    e, c = esc.figures(J, pts, g)
    e_o, c_o = esc.figures(ref, pts, g)
    assert abs(e - e_o) <= 1e-5 * e_o and abs(c - c_o) <= 2.0 / len(act)
    tree.free()
