"""Exact answers and figures of merit for the accuracy tests of Sec. 3.3-3.4.

TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU
baseline may import it; the product library never does).

The tests' absorbers are analytic: a background absorption coefficient plus
spheres or a half-space of another coefficient.  With no scattering the exact
J at a point is, per point source, L exp(-tau) / (4 pi d^2) with tau the
line integral of alpha along the straight segment from the source (Sec. 1.1:
pure absorption along rays).  tau is the background alpha times d plus, per
feature, (alpha_f - alpha_bg) times the length of the segment inside it.

Escape fraction and covering factor follow the definitions of Table escape:
the escape fraction is the flux that reaches the outer sphere relative to an
unabsorbed source, i.e. the solid-angle mean of J / J_vac with J_vac the J of
the same sources in vacuum; the covering factor is the fraction of the
sphere's solid angle where J is less than half of the J seen without the
features (background absorption only).  On a shell of receivers that sample
solid angle evenly both are plain means over the receivers.
"""

from __future__ import annotations

import numpy as np

FOUR_PI = 4.0 * np.pi


def chord_sphere(a, b, centre, radius):
    """Length of the segments a[i] -> b[i] that lies inside the ball."""
    a = np.atleast_2d(a).astype(np.float64)
    b = np.atleast_2d(b).astype(np.float64)
    d = b - a
    L2 = np.einsum("ij,ij->i", d, d)
    f = a - np.asarray(centre, dtype=np.float64)[None, :]
    # |f + t d|^2 = r^2 for t in [0, 1]
    B = np.einsum("ij,ij->i", f, d)
    C = np.einsum("ij,ij->i", f, f) - radius * radius
    disc = B * B - L2 * C
    out = np.zeros(len(a))
    ok = (disc > 0.0) & (L2 > 0.0)
    sq = np.sqrt(np.where(ok, disc, 0.0))
    t0 = np.clip((-B - sq) / np.where(L2 > 0, L2, 1.0), 0.0, 1.0)
    t1 = np.clip((-B + sq) / np.where(L2 > 0, L2, 1.0), 0.0, 1.0)
    out[ok] = ((t1 - t0) * np.sqrt(L2))[ok]
    return out


def chord_halfspace(a, b, p0, normal):
    """Length of the segments a[i] -> b[i] inside {x : (x - p0) . n >= 0}."""
    a = np.atleast_2d(a).astype(np.float64)
    b = np.atleast_2d(b).astype(np.float64)
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    sa = (a - p0) @ n
    sb = (b - p0) @ n
    length = np.linalg.norm(b - a, axis=1)
    out = np.zeros(len(a))
    both = (sa >= 0) & (sb >= 0)
    out[both] = length[both]
    cross = (sa >= 0) != (sb >= 0)
    # fraction of the segment on the positive side
    frac = np.where(cross, np.maximum(sa, sb) / np.where(cross, np.abs(sa - sb), 1.0), 0.0)
    out[cross] = (frac * length)[cross]
    return out


def optical_depth(src, points, alpha_bg, features):
    """tau from one source to every point through the analytic field."""
    points = np.atleast_2d(points).astype(np.float64)
    a = np.broadcast_to(np.asarray(src, dtype=np.float64), points.shape)
    tau = alpha_bg * np.linalg.norm(points - a, axis=1)
    for kind, p, q, alpha in features:
        if kind == "sphere":
            tau += (alpha - alpha_bg) * chord_sphere(a, points, p, q)
        elif kind == "halfspace":
            tau += (alpha - alpha_bg) * chord_halfspace(a, points, p, q)
        else:
            raise ValueError(kind)
    return tau


def exact_J(points, geometry, features=True, absorb=True):
    """J at each point: sum over sources of L exp(-tau) / (4 pi d^2).
    features=False drops the absorbing features (background only);
    absorb=False is the vacuum answer."""
    points = np.atleast_2d(points).astype(np.float64)
    J = np.zeros(len(points))
    feats = geometry["features"] if features else []
    for s, L in zip(geometry["sources"], geometry["L"]):
        d2 = np.einsum("ij,ij->i", points - s, points - s)
        tau = optical_depth(s, points, geometry["alpha_bg"], feats) if absorb else 0.0
        J += L * np.exp(-tau) / (FOUR_PI * d2)
    return J


def escape_fraction(J, J_vac):
    """Mean of J / J_vac over receivers that sample solid angle evenly."""
    return float(np.mean(np.asarray(J, np.float64) / np.asarray(J_vac, np.float64)))


def covering_factor(J, J_nofeatures):
    """Fraction of receivers where J < J_nofeatures / 2 (less than half of
    the flux without the features arrives)."""
    return float(np.mean(np.asarray(J, np.float64) < 0.5 * np.asarray(J_nofeatures, np.float64)))


def sphere_points(n, centre, radius):
    """n Fibonacci-lattice points on a sphere (even in solid angle)."""
    k = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * k / n
    phi = k * np.pi * (3.0 - np.sqrt(5.0))
    r = np.sqrt(1.0 - z * z)
    u = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return np.asarray(centre, dtype=np.float64)[None, :] + radius * u


def figures(J, points, geometry):
    """(escape fraction, covering factor) of J at the receiver points."""
    J_vac = exact_J(points, geometry, absorb=False)
    J_nof = exact_J(points, geometry, features=False)
    return escape_fraction(J, J_vac), covering_factor(J, J_nof)
