"""Edge cases of the per-bucket modes against the oracle: coincident
elements (depth-63 leaves with more receivers than a warp), luminous gas
(p-p and the complex source model must leave the source element out), a
directed target exactly at a bucket centre, and refinement together with
p-p and the complex source model."""

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

BUCKET, PP, CSM, SOFT, THICK, LINEAR = 16, 32, 64, 1, 2, 8


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


def _coincident_case():
    case = workloads.random_case(900, 30, nb=2, seed=201, clumped=True)
    pos = case["pos"].copy()
    pos[100:160] = pos[99]  # 61 coincident gas elements: one depth-63 leaf
    pos[300:305] = pos[299]
    return workloads._pack("coincident", pos, case["mass"], case["kappa"], case["lum"],
                           case["h"], np.arange(900), 2, 0.75)


def _luminous_gas_case():
    case = workloads.random_case(1200, 10, nb=2, seed=202, clumped=True, kappa_scale=30.0)
    rng = np.random.default_rng(3)
    lit = rng.choice(1200, 80, replace=False)
    case["lum"][lit] = rng.uniform(0.1, 1.0, (80, 2)).astype(np.float32)
    case["active"] = np.arange(1200)
    return case


@pytest.mark.parametrize("make", [_coincident_case, _luminous_gas_case])
@pytest.mark.parametrize("flags", [BUCKET, BUCKET | PP | THICK, BUCKET | CSM,
                                   BUCKET | PP | CSM | SOFT | THICK | LINEAR])
def test_modes_on_edge_fields(t2, oracle_mod, make, flags):
    case = make()
    tree = _gpu_tree(t2, case)
    J = tree.J(case["active"], 2, 0.75, flags=flags).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"], 2, 0.75, flags=flags)
    _assert_J(J, ref, f"{make.__name__} flags={flags}")
    tree.free()


def test_directed_target_at_a_bucket_centre(t2, oracle_mod):
    """The bucket whose centre is the target keeps its pixel-centre beams;
    every other bucket aims one beam at it."""
    case = workloads.random_case(1500, 20, nb=1, seed=203, clumped=True)
    ot = oracle_mod.OracleTree.from_case(case)
    e = ot.export()
    q = int(np.flatnonzero((e["child"] < 0) & (e["count"] > 3))[0])
    target = 0.5 * (e["box"][q, :3] + e["box"][q, 3:])
    tree = _gpu_tree(t2, case)
    for flags in (BUCKET, BUCKET | CSM):
        J = tree.J(case["active"], 2, 0.75, flags=flags, target=target).cpu().numpy()
        _assert_J(J, ot.J(case["active"], 2, 0.75, flags=flags, target=target),
                  f"target at a centre flags={flags}")
    tree.free()


@pytest.mark.parametrize("tau", [0.05, 0.5])
def test_refinement_with_pp_and_csm(t2, oracle_mod, tau):
    case = _luminous_gas_case()
    tree = _gpu_tree(t2, case)
    tree.set_tau_refine(tau)
    ot = oracle_mod.OracleTree.from_case(case)
    ot.set_tau_refine(tau)
    flags = BUCKET | PP | CSM | THICK
    J = tree.J(case["active"], 2, 0.75, flags=flags).cpu().numpy()
    _assert_J(J, ot.J(case["active"], 2, 0.75, flags=flags), f"refine {tau}")
    tree.free()


@pytest.mark.parametrize("nside", [8, 16])
@pytest.mark.parametrize("flags", [BUCKET, BUCKET | PP | THICK, BUCKET | CSM])
def test_modes_at_the_largest_nside(t2, oracle_mod, nside, flags):
    """768 and 3072 beams: the walk's shared-memory layout, the p-p sphere
    (r_pp = h / sqrt(4 pi / N_ray) holds every particle here) and the complex
    source tables at their largest."""
    case = workloads.random_case(600, 20, nb=2, seed=204, clumped=True, n_active=150)
    tree = _gpu_tree(t2, case)
    J = tree.J(case["active"], nside, 0.75, flags=flags).cpu().numpy()
    ref = oracle_mod.OracleTree.from_case(case).J(case["active"], nside, 0.75, flags=flags)
    _assert_J(J, ref, f"nside={nside} flags={flags}")
    tree.free()
