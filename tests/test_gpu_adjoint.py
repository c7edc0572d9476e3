"""Adjoint walk (trevr2_J_backward and the autograd function) against the
oracle's forward-mode gradient.

The oracle differentiates its own FP64 J with dual numbers, one pass per
parameter, holding the cut, the beams and the tree fixed; its derivative is
pinned to FP64 central differences in the CPU suite.  Here the GPU gradient
of Loss = sum_{i,b} gJ_ib J_ib with respect to kappa and L must match it.

Bar (FP32 walk, FP32 atomics, FP64 element sums): over the parameters whose
reference gradient is at least 1e-3 of the largest one, relative error
median <= 1e-4 and max <= 2e-3; the others within 2e-6 of the largest.
"""

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


def _gpu_tree(t2, case):
    return t2.build(case["pos"], case["mass"], case["kappa"], case["lum"], case["h"],
                    case["box_lo"], case["box_size"], case["bucket"])


def _oracle_grad(ot, active, gJ_full, nside, theta, params, flags=0):
    """d(sum gJ_full * J)/d(param) for each (which, elem, band)."""
    out = np.empty(len(params))
    for k, (which, e, b) in enumerate(params):
        dJ = ot.J_deriv(active, nside, theta, which, int(e), int(b), flags)
        out[k] = float((dJ * gJ_full).sum())
    return out


def _check(got, want, what):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert np.all(np.isfinite(got)), what
    scale = float(np.abs(want).max())
    assert scale > 0.0, what
    err = np.abs(got - want)
    big = np.abs(want) >= 1e-3 * scale
    rel = err[big] / np.abs(want[big])
    med, mx = float(np.median(rel)), float(rel.max())
    small = float(err[~big].max()) / scale if (~big).any() else 0.0
    assert med <= 1e-4 and mx <= 2e-3 and small <= 2e-6, (
        f"{what}: median {med:.2e} max {mx:.2e} small-gradient error {small:.2e} "
        f"({int(big.sum())} of {len(want)} parameters above 1e-3 of the largest)")


def _all_params(case, n_kappa=200, n_dark=40, seed=0):
    """Every L of a luminous element, the kappa of n_kappa random (element,
    band) pairs of massive elements and the L of n_dark random dark ones."""
    n, nb = case["lum"].shape
    rng = np.random.default_rng(seed)
    lit = case["lum"].sum(1) > 0
    ps = [("lum", int(e), b) for e in np.flatnonzero(lit) for b in range(nb)]
    massive = np.flatnonzero(case["mass"] > 0)
    for e in rng.choice(massive, min(n_kappa, len(massive)), replace=False):
        ps.append(("kappa", int(e), int(rng.integers(0, nb))))
    dark = np.flatnonzero(~lit)
    for e in rng.choice(dark, min(n_dark, len(dark)), replace=False):
        ps.append(("lum", int(e), int(rng.integers(0, nb))))
    return ps


def _gather(gk, gl, params):
    gk = gk.cpu().numpy()
    gl = gl.cpu().numpy()
    return np.array([gk[e, b] if w == "kappa" else gl[e, b] for w, e, b in params])


SMALL = [
    ("nb2_nside2", dict(n_gas=600, n_src=20, nb=2, seed=51, clumped=True, n_active=120), 2, 0.75),
    ("nb1_nside1", dict(n_gas=500, n_src=12, nb=1, seed=52, n_active=100), 1, 0.6),
    ("nb3_nside4", dict(n_gas=700, n_src=25, nb=3, seed=53, clumped=True, n_active=80,
                        kappa_scale=40.0), 4, 0.5),
]


@pytest.mark.parametrize("name,kw,nside,theta", SMALL)
@pytest.mark.parametrize("flags", [0, 1, 2, 3])
def test_backward_matches_oracle_gradient(t2, oracle_mod, name, kw, nside, theta, flags):
    case = workloads.random_case(**kw)
    tree = _gpu_tree(t2, case)
    act = case["active"]
    rng = np.random.default_rng(7)
    gJ = rng.uniform(0.0, 1.0, size=(len(act), case["nb"]))
    gk, gl = tree.J_backward(act, gJ.astype(np.float32), nside, theta, flags=flags)
    params = _all_params(case)
    ot = oracle_mod.OracleTree.from_case(case)
    want = _oracle_grad(ot, act, gJ.astype(np.float32).astype(np.float64), nside, theta, params,
                        flags)
    _check(_gather(gk, gl, params), want, f"{name} flags={flags}")
    # massless elements have no kappa gradient; gradients of unused bands are 0
    assert np.all(gk.cpu().numpy()[case["mass"] == 0] == 0)
    tree.free()


def test_backward_band_selection_and_duplicates(t2, oracle_mod):
    """gJ over a selection of bands (one repeated) and repeated receivers."""
    case = workloads.random_case(500, 15, nb=3, seed=54, clumped=True, n_active=60)
    act = np.concatenate([case["active"], case["active"][:10]])
    bands = [2, 0, 2]
    tree = _gpu_tree(t2, case)
    rng = np.random.default_rng(8)
    g_sel = rng.uniform(0.0, 1.0, size=(len(act), len(bands))).astype(np.float32)
    gk, gl = tree.J_backward(act, g_sel, 2, 0.75, bands=bands, flags=2)
    full = np.zeros((len(act), 3))
    for j, b in enumerate(bands):
        full[:, b] += g_sel[:, j]
    params = _all_params(case)
    want = _oracle_grad(oracle_mod.OracleTree.from_case(case), act, full, 2, 0.75, params, 2)
    _check(_gather(gk, gl, params), want, "band selection")
    # band 1 has no upstream gradient: no kappa gradient (its luminosity still
    # moves the centres of luminosity, which the other bands see)
    assert np.all(gk.cpu().numpy()[:, 1] == 0)
    tree.free()


def test_backward_many_sources_multi_pass(t2, oracle_mod):
    """More sources per receiver than one warp stages: several passes."""
    case = workloads.random_case(300, 1800, nb=2, seed=55, clumped=True, n_active=40)
    tree = _gpu_tree(t2, case)
    act = case["active"]
    rng = np.random.default_rng(9)
    gJ = rng.uniform(0.0, 1.0, size=(len(act), 2)).astype(np.float32)
    gk, gl = tree.J_backward(act, gJ, 2, 1e-6)
    ot = oracle_mod.OracleTree.from_case(case)
    _, st = ot.J(act, 2, 1e-6, stats=True)
    assert st[:, 3].max() > 1024
    params = [p for p in _all_params(case) if p[0] == "kappa" or rng.uniform() < 0.2]
    want = _oracle_grad(ot, act, gJ.astype(np.float64), 2, 1e-6, params)
    _check(_gather(gk, gl, params), want, "multi-pass")
    tree.free()


def test_backward_zero_upstream_and_bad_index(t2):
    case = workloads.random_case(300, 10, nb=2, seed=56, n_active=50)
    tree = _gpu_tree(t2, case)
    gk, gl = tree.J_backward(case["active"], np.zeros((50, 2), np.float32), 2, 0.75)
    assert float(gk.abs().max()) == 0.0 and float(gl.abs().max()) == 0.0
    bad = case["active"].copy()
    bad[3] = len(case["pos"])
    with pytest.raises(t2.TrevrError, match="EINVAL"):
        tree.J_backward(bad, np.ones((50, 2), np.float32), 2, 0.75)
    tree.free()


def test_autograd_function(t2, oracle_mod):
    """J_fn under torch.autograd: backward gives trevr2_J_backward's result and
    the forward gives trevr2_J's."""
    case = workloads.random_case(400, 12, nb=2, seed=57, clumped=True, n_active=70)
    dev = torch.device("cuda")
    kappa = torch.tensor(case["kappa"], dtype=torch.float32, device=dev, requires_grad=True)
    lum = torch.tensor(case["lum"], dtype=torch.float32, device=dev, requires_grad=True)
    pos = torch.tensor(case["pos"], device=dev)
    mass = torch.tensor(case["mass"], dtype=torch.float32, device=dev)
    h = torch.tensor(case["h"], dtype=torch.float32, device=dev)
    act = torch.tensor(case["active"], device=dev)
    w = torch.rand((70, 2), device=dev, generator=torch.Generator(dev).manual_seed(3))
    J = t2.J_fn(pos, mass, kappa, lum, act, nside=2, theta=0.75, h=h, flags=2,
                box_lo=case["box_lo"], box_size=case["box_size"], bucket=case["bucket"])
    (w * J).sum().backward()
    tree = _gpu_tree(t2, case)
    J2 = tree.J(case["active"], 2, 0.75, flags=2)
    assert torch.equal(J.detach(), J2)
    gk, gl = tree.J_backward(case["active"], w, 2, 0.75, flags=2)
    assert torch.allclose(kappa.grad, gk, rtol=1e-5, atol=1e-6 * float(gk.abs().max()))
    assert torch.allclose(lum.grad, gl, rtol=1e-5, atol=1e-6 * float(gl.abs().max()))
    params = [("kappa", e, b) for e in range(0, 400, 37) for b in range(2)] + \
             [("lum", 400 + e, b) for e in range(12) for b in range(2)]
    want = _oracle_grad(oracle_mod.OracleTree.from_case(case), case["active"],
                        w.cpu().numpy().astype(np.float64), 2, 0.75, params, 2)
    _check(_gather(kappa.grad, lum.grad, params), want, "autograd")
    tree.free()


@pytest.fixture(scope="module")
def adjoint_field():
    return workloads.adjoint_case()


def test_backward_full_size_sampled(t2, oracle_mod, adjoint_field):
    """The adjoint workload at full size (64^3 lognormal gas, sigma 1, 1024
    sources, 2 bands, nside 2, theta 0.75) with Loss = sum_i w_i J_i,
    w ~ U(0,1), over 4096 random receivers; 64 random parameters (32 kappa of
    gas, 32 L of sources) against the oracle."""
    case = adjoint_field
    tree = _gpu_tree(t2, case)
    rng = np.random.default_rng(12)
    act = np.sort(rng.choice(case["active"], 4096, replace=False))
    w = rng.uniform(0.0, 1.0, size=(len(act), 2)).astype(np.float32)
    gk, gl = tree.J_backward(act, w, case["nside"], case["theta"])
    n_gas = int((case["mass"] > 0).sum())
    src = np.flatnonzero(case["lum"].sum(1) > 0)
    params = [("kappa", int(e), int(rng.integers(0, 2))) for e in rng.choice(n_gas, 32, False)]
    params += [("lum", int(e), int(rng.integers(0, 2))) for e in rng.choice(src, 32, False)]
    want = _oracle_grad(oracle_mod.OracleTree.from_case(case), act, w.astype(np.float64),
                        case["nside"], case["theta"], params)
    _check(_gather(gk, gl, params), want, "adjoint full size")
    tree.free()


def _central_differences(oracle_mod, case, act, w, params, step_rel=1e-6):
    """FP64 central differences of the oracle's Loss = sum w J for each
    (which, elem, band), a relative step of step_rel, the tree rebuilt per
    evaluation; a parameter whose two one-sided differences disagree by more
    than 10% (a discrete choice of the walk switched inside the step) is
    returned as NaN."""
    nside, theta = case["nside"], case["theta"]

    def loss(c):
        return float((oracle_mod.OracleTree.from_case(c).J(act, nside, theta) * w).sum())

    base_loss = loss(case)
    out = np.empty(len(params))
    for k, (which, elem, band) in enumerate(params):
        base = float(case[which][elem, band])
        step = step_rel * base
        vals = []
        for sgn in (+1, -1):
            c2 = dict(case)
            a2 = case[which].astype(np.float64).copy()
            a2[elem, band] = base + sgn * step
            c2[which] = a2
            vals.append(loss(c2))
        fwd, bwd = (vals[0] - base_loss) / step, (base_loss - vals[1]) / step
        agree = abs(fwd - bwd) <= 0.1 * max(abs(fwd), abs(bwd)) or max(abs(fwd), abs(bwd)) == 0.0
        out[k] = (vals[0] - vals[1]) / (2 * step) if agree else np.nan
    return out


def test_backward_full_size_against_central_differences(t2, oracle_mod, adjoint_field):
    """The same workload, receivers, weights and 64 parameters as above, with
    the GPU gradient checked directly against FP64 central differences of
    the oracle's loss (relative step 1e-6); parameters whose one-sided
    differences disagree by more than 10% are skipped and counted."""
    case = adjoint_field
    tree = _gpu_tree(t2, case)
    rng = np.random.default_rng(12)
    act = np.sort(rng.choice(case["active"], 4096, replace=False))
    w = rng.uniform(0.0, 1.0, size=(len(act), 2)).astype(np.float32)
    gk, gl = tree.J_backward(act, w, case["nside"], case["theta"])
    n_gas = int((case["mass"] > 0).sum())
    src = np.flatnonzero(case["lum"].sum(1) > 0)
    params = [("kappa", int(e), int(rng.integers(0, 2))) for e in rng.choice(n_gas, 32, False)]
    params += [("lum", int(e), int(rng.integers(0, 2))) for e in rng.choice(src, 32, False)]
    fd = _central_differences(oracle_mod, case, act, w.astype(np.float64), params)
    keep = np.isfinite(fd)
    assert keep.sum() >= 56, f"{int((~keep).sum())} of 64 parameters switched a discrete choice"
    got = _gather(gk, gl, params)
    _check(np.asarray(got)[keep], fd[keep], "adjoint full size vs central differences")
    tree.free()


def _line_case(n=1500, nb=2, seed=58):
    """Absorbing elements on a line along +x (a beam direction of nside 1)
    with a source at its far end: with theta -> 0 every leaf on the line is
    a segment of that beam (far more than the adjoint records per beam)."""
    rng = np.random.default_rng(seed)
    off = 0.5 + 1e-4
    gas = np.stack([(np.arange(n) + 0.5) / n, np.full(n, off), np.full(n, off)], 1)
    src = np.array([[0.9995, off, off], [0.3, 0.8, 0.2], [0.7, 0.1, 0.9]])
    pos = np.concatenate([gas, src])
    N = len(pos)
    mass = np.concatenate([np.full(n, 1.0 / n), np.zeros(3)])
    kappa = np.zeros((N, nb))
    kappa[:n] = 2e-6 * rng.uniform(0.2, 1.0, size=(n, nb))  # tau ~ 1 along the line
    lum = np.zeros((N, nb))
    lum[n:] = rng.uniform(0.5, 1.0, size=(3, nb))
    return dict(pos=pos, mass=mass, kappa=kappa, lum=lum, h=np.full(N, 1.0 / n),
                active=np.arange(0, 40, 4, dtype=np.int64), nb=nb, nside=1, theta=1e-6,
                box_lo=np.zeros(3), box_size=1.0, bucket=1, name="line")


def test_backward_long_beam(t2, oracle_mod):
    case = _line_case()
    tree = _gpu_tree(t2, case)
    act = case["active"]
    ot = oracle_mod.OracleTree.from_case(case)
    J = tree.J(act, 1, 1e-6).cpu().numpy()
    ref, st = ot.J(act, 1, 1e-6, stats=True)
    assert st[:, 2].min() > 1000  # segments per receiver
    r = np.abs(J - ref) / np.abs(ref)
    assert np.median(r) <= 1e-4 and r.max() <= 1e-3, r.max()
    rng = np.random.default_rng(10)
    gJ = rng.uniform(0.0, 1.0, size=(len(act), 2)).astype(np.float32)
    gk, gl = tree.J_backward(act, gJ, 1, 1e-6)
    params = _all_params(case, n_kappa=120, n_dark=10)
    want = _oracle_grad(ot, act, gJ.astype(np.float64), 1, 1e-6, params)
    _check(_gather(gk, gl, params), want, "long beam")
    tree.free()
