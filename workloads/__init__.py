"""Seeded synthetic inputs shaped like the TREVR2 paper's workloads.

This module only draws random numbers and lays them out as arrays.  It holds
none of the method's arithmetic (no keys, no tree, no absorption, no rays), so
both the FP64 CPU oracle and the CUDA path can be fed from it without sharing
any code with each other.

Every case is a dict with
    pos    float64 [N, 3]   element positions (gas first, then star sources)
    mass   float32 [N]      element masses (0 for pure point sources)
    kappa  float32 [N, nb]  opacity per unit mass, per band
    lum    float32 [N, nb]  luminosity per band (0 for gas)
    h      float32 [N]      element size (m/rho)^(1/3)
    active int64   [A]      receiver indices (into the original order)
    nb, nside, theta, box_lo, box_size, bucket, name
The unit box [0,1)^3 is used throughout, as in the recipes below.

Recipes (section numbers are the paper's):
  * jittered lattice: x = (i + 0.5 + U(-1/4, 1/4)) / n per axis;
  * lognormal density: n^3 Gaussian white noise, FFT, multiply by sqrt(P(k))
    with P ~ k^-3 and P(0) = 0, inverse FFT, standardise to g, then
    rho = exp(sigma*g - sigma^2/2); each lattice particle gets its cell's rho,
    m = rho / n^3 and h = 1/n;
  * star sources: m = 0, luminosity equal in every band, drawn from
    dN/dL ~ L^-2 on [1e-3, 1] by inverse CDF L = 1/(1000 - 999 u); placed in
    lattice cells chosen with probability ~ rho, plus U(0, 1/n)^3 (sources
    sit in dense gas, Sec. 5).
The galaxy snapshot of Sec. 3.1 is not available; the clumpy 128^3 field
stands in for its shape.

The three accuracy geometries of Sec. 3.3-3.4 (two sources and a cloud, a
source between two clouds, a source beside a wall) are built from the sizes
the text gives.  A jittered lattice of the stated spacing stands in for the
glass; every gas element has unit density (m = spacing^3, h = spacing) and
kappa equal to the absorption coefficient alpha at its position, so the
bucket absorption sum(kappa m)/V is alpha wherever a leaf is filled evenly.
Their dicts also carry the geometry (sources, absorbing features, shell
radius) so that the exact answer can be evaluated next to the method's.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "jittered_lattice",
    "lognormal_density",
    "powerlaw_luminosity",
    "uniform_point_source",
    "clumpy_multiband",
    "stromgren_like",
    "adjoint_case",
    "batched_cases",
    "random_case",
    "two_sources_cloud",
    "source_two_clouds",
    "source_wall",
    "CASES",
]


def jittered_lattice(n: int, rng: np.random.Generator) -> np.ndarray:
    """n^3 points, one per lattice cell, jittered by U(-1/4, 1/4) cell widths.

    Cell (ix, iy, iz) has flat index (ix*n + iy)*n + iz.
    """
    idx = np.arange(n, dtype=np.float64)
    gx, gy, gz = np.meshgrid(idx, idx, idx, indexing="ij")
    base = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    jit = rng.uniform(-0.25, 0.25, size=base.shape)
    return (base + 0.5 + jit) / n


def lognormal_density(n: int, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """Lognormal density on an n^3 grid with a k^-3 power spectrum (flat index)."""
    white = rng.standard_normal((n, n, n))
    k1 = np.fft.fftfreq(n) * n
    kx, ky, kz = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** -1.5  # sqrt(P), P ~ k^-3
    field = np.fft.ifftn(np.fft.fftn(white) * amp).real
    g = (field - field.mean()) / field.std()
    return np.exp(sigma * g - 0.5 * sigma * sigma).ravel()


def powerlaw_luminosity(ns: int, rng: np.random.Generator) -> np.ndarray:
    """dN/dL ~ L^-2 on [1e-3, 1] by inverse CDF."""
    u = rng.uniform(size=ns)
    return 1.0 / (1000.0 - 999.0 * u)


def _pack(name, pos, mass, kappa, lum, h, active, nside, theta, bucket=12):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[0]
    kappa = np.ascontiguousarray(np.asarray(kappa, dtype=np.float32).reshape(n, -1))
    lum = np.ascontiguousarray(np.asarray(lum, dtype=np.float32).reshape(n, -1))
    assert kappa.shape == lum.shape
    return {
        "name": name,
        "pos": pos,
        "mass": np.ascontiguousarray(mass, dtype=np.float32),
        "kappa": kappa,
        "lum": lum,
        "h": np.ascontiguousarray(h, dtype=np.float32),
        "active": np.ascontiguousarray(active, dtype=np.int64),
        "nb": int(kappa.shape[1]),
        "nside": int(nside),
        "theta": float(theta),
        "box_lo": np.zeros(3),
        "box_size": 1.0,
        "bucket": int(bucket),
    }


def _gas_plus_sources(gpos, gmass, gh, kappa_b, spos, slum):
    ng, ns = gpos.shape[0], spos.shape[0]
    nb = len(kappa_b)
    pos = np.concatenate([gpos, spos], axis=0)
    mass = np.concatenate([gmass, np.zeros(ns)])
    kappa = np.zeros((ng + ns, nb))
    kappa[:ng, :] = np.asarray(kappa_b)[None, :]
    lum = np.zeros((ng + ns, nb))
    lum[ng:, :] = np.asarray(slum)[:, None]
    h = np.concatenate([gh, np.full(ns, gh.mean() if ng else 1.0)])
    return pos, mass, kappa, lum, h


def uniform_point_source(offset: bool = False, seed: int = 1001, n: int = 16):
    """Plain-method case: 16^3 jittered lattice, uniform density, kappa*rho = 2,
    one L = 1 source at the box centre (or at (0.53, 0.51, 0.52), off the root
    split planes, as App. A advises), nside = 2, theta = 0.75."""
    rng = np.random.default_rng(seed)
    gpos = jittered_lattice(n, rng)
    ng = n ** 3
    gmass = np.full(ng, 1.0 / ng)
    gh = np.full(ng, 1.0 / n)
    src = np.array([[0.53, 0.51, 0.52]]) if offset else np.array([[0.5, 0.5, 0.5]])
    pos, mass, kappa, lum, h = _gas_plus_sources(gpos, gmass, gh, [2.0], src, [1.0])
    return _pack("uniform_point_source" + ("_offset" if offset else ""), pos, mass,
                 kappa, lum, h, np.arange(ng), nside=2, theta=0.75)


def stromgren_like(seed: int = 1002, n: int = 32, n_src: int = 64):
    """Uniform medium, kappa*rho = 10, 64 sources at U(0,1)^3 with L
    log-uniform in [1e-2, 1], nside = 2, theta = 0.75, all gas active."""
    rng = np.random.default_rng(seed)
    gpos = jittered_lattice(n, rng)
    ng = n ** 3
    spos = rng.uniform(0.0, 1.0, size=(n_src, 3))
    slum = 10.0 ** rng.uniform(-2.0, 0.0, size=n_src)
    pos, mass, kappa, lum, h = _gas_plus_sources(
        gpos, np.full(ng, 1.0 / ng), np.full(ng, 1.0 / n), [10.0], spos, slum)
    return _pack("stromgren_like", pos, mass, kappa, lum, h, np.arange(ng),
                 nside=2, theta=0.75)


def _clumpy(seed, n, sigma, n_src, kappa_b, nside, theta, name):
    rng = np.random.default_rng(seed)
    gpos = jittered_lattice(n, rng)
    rho = lognormal_density(n, sigma, rng)
    ng = n ** 3
    cells = rng.choice(ng, size=n_src, replace=True, p=rho / rho.sum())
    ix, rem = np.divmod(cells, n * n)
    iy, iz = np.divmod(rem, n)
    corner = np.stack([ix, iy, iz], axis=1).astype(np.float64) / n
    spos = corner + rng.uniform(0.0, 1.0 / n, size=(n_src, 3))
    slum = powerlaw_luminosity(n_src, rng)
    pos, mass, kappa, lum, h = _gas_plus_sources(
        gpos, rho / ng, np.full(ng, 1.0 / n), kappa_b, spos, slum)
    return _pack(name, pos, mass, kappa, lum, h, np.arange(ng), nside=nside, theta=theta)


def clumpy_multiband(seed: int = 1003, n: int = 128, n_src: int = 10_000):
    """Clumpy multi-band forward: 128^3 lognormal (sigma = 1.5) gas, 10^4
    power-law sources, 3 bands with kappa = (10, 3, 0.5) (ratios 1:0.3:0.05),
    nside = 4 (192 directions), theta = 0.5, all gas active."""
    return _clumpy(seed, n, 1.5, n_src, [10.0, 3.0, 0.5], 4, 0.5, f"clumpy_multiband_{n}")


def adjoint_case(seed: int = 1005, n: int = 64, n_src: int = 1024):
    """Adjoint case: 64^3 lognormal (sigma = 1.0) gas, 1024 sources, 2 bands
    with kappa = (10, 3), nside = 2, theta = 0.75."""
    return _clumpy(seed, n, 1.0, n_src, [10.0, 3.0], 2, 0.75, f"adjoint_{n}")


def batched_cases(n: int = 128, n_src: int = 10_000, n_snap: int = 4, n_sub: int = 64,
                  seed0: int = 1040, sub_seed: int = 1004):
    """Individual-timestep batching: n_snap clumpy snapshots (seeds 1040..),
    each with n_sub active subsets of size floor(10^U(2,6)) (capped at the gas
    count), members uniform without replacement."""
    snaps = [_clumpy(seed0 + s, n, 1.5, n_src, [10.0, 3.0, 0.5], 4, 0.5,
                     f"clumpy_multiband_{n}_s{s}") for s in range(n_snap)]
    rng = np.random.default_rng(sub_seed)
    subsets = []
    for s, c in enumerate(snaps):
        ng = n ** 3
        for _ in range(n_sub):
            size = min(int(np.floor(10.0 ** rng.uniform(2.0, 6.0))), ng)
            members = np.sort(rng.choice(ng, size=size, replace=False)).astype(np.int64)
            subsets.append((s, members))
    return snaps, subsets


def random_case(n_gas: int, n_src: int, nb: int = 1, seed: int = 0, nside: int = 2,
                theta: float = 0.75, kappa_scale: float = 10.0, clumped: bool = False,
                bucket: int = 12, n_active: int | None = None):
    """Small irregular case for edge coverage: uniform (or Gaussian-clumped)
    gas, random masses and opacities, random sources; ragged sizes allowed."""
    rng = np.random.default_rng(seed)
    if clumped and n_gas > 0:
        centres = rng.uniform(0.2, 0.8, size=(4, 3))
        which = rng.integers(0, 4, size=n_gas)
        gpos = np.clip(centres[which] + rng.normal(0.0, 0.08, size=(n_gas, 3)), 0.0, 1.0)
    else:
        gpos = rng.uniform(0.0, 1.0, size=(n_gas, 3))
    gmass = rng.uniform(0.5, 1.5, size=n_gas) / max(n_gas, 1)
    spos = rng.uniform(0.0, 1.0, size=(n_src, 3))
    pos = np.concatenate([gpos, spos], axis=0)
    n = n_gas + n_src
    mass = np.concatenate([gmass, np.zeros(n_src)])
    kappa = np.zeros((n, nb))
    kappa[:n_gas] = kappa_scale * rng.uniform(0.2, 1.0, size=(n_gas, nb))
    lum = np.zeros((n, nb))
    lum[n_gas:] = 10.0 ** rng.uniform(-2.0, 0.0, size=(n_src, nb))
    h = np.full(n, (1.0 / max(n_gas, 1)) ** (1.0 / 3.0))
    if n_active is None:
        active = np.arange(n_gas)
    else:
        active = np.sort(rng.choice(n, size=n_active, replace=False))
    return _pack(f"random_{n_gas}_{n_src}_{nb}_{seed}", pos, mass, kappa, lum, h, active,
                 nside=nside, theta=theta, bucket=bucket)


def jittered_block(lo, spacing: float, cells: int, rng: np.random.Generator) -> np.ndarray:
    """cells^3 points, one per cubic cell of side `spacing` starting at `lo`,
    each jittered by U(-1/4, 1/4) of a cell per axis."""
    return np.asarray(lo, dtype=np.float64) + jittered_lattice(cells, rng) * (cells * spacing)


def _accuracy_case(name, gpos, spacing, alpha, spos, slum, box_lo, box_size, shell_centre,
                   shell_radius, shell_width, geometry):
    """Unit-density gas (m = s^3, h = s, kappa = alpha) plus point sources;
    the receivers are the gas elements within shell_width/2 of the sphere of
    radius shell_radius about shell_centre."""
    ng = gpos.shape[0]
    pos, mass, kappa, lum, h = _gas_plus_sources(
        gpos, spacing ** 3, spacing, [1.0], spos, slum)
    kappa[:ng, 0] = alpha
    r = np.linalg.norm(gpos - np.asarray(shell_centre)[None, :], axis=1)
    active = np.flatnonzero(np.abs(r - shell_radius) < 0.5 * shell_width)
    case = _pack(name, pos, mass, kappa, lum, h, active, nside=2, theta=0.75)
    case["box_lo"] = np.asarray(box_lo, dtype=np.float64)
    case["box_size"] = float(box_size)
    case["geometry"] = dict(geometry, sources=np.asarray(spos, dtype=np.float64),
                            L=np.asarray(slum, dtype=np.float64),
                            shell_centre=np.asarray(shell_centre, dtype=np.float64),
                            shell_radius=float(shell_radius))
    return case


def two_sources_cloud(seed: int = 1050):
    """Cloud irradiated by two sources (Sec. 3.3): a sphere of radius 0.5 at
    the origin with alpha = 1e4 (spacing 0.0625) in a medium with alpha =
    1e-4 (spacing 0.25); L = 0.5 sources at (-2, 0, 0) and (0, -2, 0).  The
    volume is a cube of side 17 centred on (-2.1, -2.1, -2.1), so that the
    sources and the cloud share a cell of side 4.25; the receivers are the gas
    elements on the sphere r = 6 about the origin."""
    rng = np.random.default_rng(seed)
    side, s_out, s_in, R = 17.0, 0.25, 0.0625, 0.5
    lo = np.full(3, -2.1 - 0.5 * side)
    outer = jittered_block(lo, s_out, int(round(side / s_out)), rng)
    outer = outer[np.linalg.norm(outer, axis=1) >= R]
    inner = jittered_block(np.full(3, -R), s_in, int(round(2 * R / s_in)), rng)
    inner = inner[np.linalg.norm(inner, axis=1) < R]
    gpos = np.concatenate([outer, inner])
    spacing = np.concatenate([np.full(len(outer), s_out), np.full(len(inner), s_in)])
    alpha = np.concatenate([np.full(len(outer), 1e-4), np.full(len(inner), 1e4)])
    spos = np.array([[-2.0, 0.0, 0.0], [0.0, -2.0, 0.0]])
    geometry = {"alpha_bg": 1e-4,
                "features": [("sphere", np.zeros(3), R, 1e4)]}
    return _accuracy_case("two_sources_cloud", gpos, spacing, alpha, spos, [0.5, 0.5],
                          lo, side, np.zeros(3), 6.0, s_out, geometry)


def _offset_source_gas(rng):
    """Sec. 3.4 particles: a sphere of radius 2.5 about the origin at spacing
    0.0625, refined to 0.8/38 (the text's 0.0209) within 0.4 of the source at
    (0.17, 0.17, 0.17)."""
    src = np.full(3, 0.17)
    R_vol, s_out, r_in = 2.5, 0.0625, 0.4
    n_in = 38
    s_in = 2 * r_in / n_in
    outer = jittered_block(np.full(3, -R_vol), s_out, int(round(2 * R_vol / s_out)), rng)
    outer = outer[(np.linalg.norm(outer, axis=1) < R_vol)
                  & (np.linalg.norm(outer - src, axis=1) >= r_in)]
    inner = jittered_block(src - r_in, s_in, n_in, rng)
    inner = inner[np.linalg.norm(inner - src, axis=1) < r_in]
    gpos = np.concatenate([outer, inner])
    spacing = np.concatenate([np.full(len(outer), s_out), np.full(len(inner), s_in)])
    return src, gpos, spacing, s_out


def source_two_clouds(seed: int = 1051):
    """A source flanked by two clouds (Sec. 3.4.1): alpha = 1 medium, clouds
    of radius 0.1 with alpha = 10 at 0.25 either side of the L = 1 source
    along the main diagonal; receivers on the sphere r = 2 about the source."""
    rng = np.random.default_rng(seed)
    src, gpos, spacing, s_out = _offset_source_gas(rng)
    n = np.full(3, 1.0 / np.sqrt(3.0))
    centres = [src + 0.25 * n, src - 0.25 * n]
    alpha = np.ones(len(gpos))
    for c in centres:
        alpha[np.linalg.norm(gpos - c, axis=1) < 0.1] = 10.0
    geometry = {"alpha_bg": 1.0,
                "features": [("sphere", c, 0.1, 10.0) for c in centres]}
    return _accuracy_case("source_two_clouds", gpos, spacing, alpha, src[None, :], [1.0],
                          np.full(3, -2.5), 5.0, src, 2.0, s_out, geometry)


def source_wall(seed: int = 1051):
    """A source beside a wall (Sec. 3.4.2): the particles of the two-cloud
    case; alpha = 10 in the half-space beyond the plane 0.25 from the source
    along -(1, 1, 1)/sqrt(3), alpha = 1 elsewhere."""
    rng = np.random.default_rng(seed)
    src, gpos, spacing, s_out = _offset_source_gas(rng)
    n = -np.full(3, 1.0 / np.sqrt(3.0))  # from the source towards the wall
    p0 = src + 0.25 * n
    alpha = np.where((gpos - p0) @ n >= 0.0, 10.0, 1.0)
    geometry = {"alpha_bg": 1.0, "features": [("halfspace", p0, n, 10.0)]}
    return _accuracy_case("source_wall", gpos, spacing, alpha, src[None, :], [1.0],
                          np.full(3, -2.5), 5.0, src, 2.0, s_out, geometry)


CASES = {
    "uniform_point_source": uniform_point_source,
    "stromgren_like": stromgren_like,
    "clumpy_multiband": clumpy_multiband,
    "adjoint_case": adjoint_case,
    "two_sources_cloud": two_sources_cloud,
    "source_two_clouds": source_two_clouds,
    "source_wall": source_wall,
}
