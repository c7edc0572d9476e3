"""FP64 CPU oracle for the TREVR2 reverse ray trace (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may load it.
The product library (``paper_2310_15235_gb300``) never imports, links or runs
anything here, and this package never imports the product: the two share no
code.  The C++ source ``trevr2_oracle.cpp`` restates the method of
Wadsley, Baumschlager & Shen (arXiv:2310.15235) in plain FP64; this module only
compiles it with gcc and marshals numpy arrays through ctypes.

Functions whose result the tests pin against something other than the oracle
itself are listed in the design notes; every function here has at least one
such pin (brute force, closed form, worked example, Monte Carlo geometry or
HEALPix invariants).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "trevr2_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FLAG_SOFT = 1
FLAG_THICK = 2
FLAG_LINEAR = 8
FLAG_BUCKET = 16
FLAG_PP = 32
FLAG_CSM = 64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        i64, i32, f64, u32 = C.c_int64, C.c_int, C.c_double, C.c_uint32
        lib.oracle_tree_build.restype = P
        lib.oracle_tree_build.argtypes = [P, P, P, P, P, i64, i32, P, f64, i32]
        lib.oracle_tree_free.argtypes = [P]
        lib.oracle_tree_num_nodes.restype = i64
        lib.oracle_tree_num_nodes.argtypes = [P]
        lib.oracle_tree_max_depth.restype = i32
        lib.oracle_tree_max_depth.argtypes = [P]
        lib.oracle_tree_box.argtypes = [P, P, P]
        lib.oracle_tree_export.argtypes = [P] + [P] * 9
        lib.oracle_tree_aggregates.argtypes = [P, P, P, P, P, P]
        lib.oracle_alpha_table.restype = i32
        lib.oracle_alpha_table.argtypes = [P, i32, i32, P]
        lib.oracle_pix2vec.argtypes = [i32, P]
        lib.oracle_vec2pix.argtypes = [i32, P, i64, P]
        lib.oracle_pair_of_pixel.restype = i64
        lib.oracle_pair_of_pixel.argtypes = [i32, i64]
        lib.oracle_morton_keys.argtypes = [P, i64, P, f64, P]
        lib.oracle_transmission_alpha.restype = f64
        lib.oracle_transmission_alpha.argtypes = [P, i32, P, f64, f64, P]
        lib.oracle_soft_kernel.restype = f64
        lib.oracle_soft_kernel.argtypes = [f64, f64]
        lib.oracle_thick_factor.restype = f64
        lib.oracle_thick_factor.argtypes = [f64]
        lib.oracle_J.restype = i32
        lib.oracle_J.argtypes = [P, P, i64, i32, f64, u32, P, i32, P]
        lib.oracle_J_deriv.restype = i32
        lib.oracle_J_deriv.argtypes = [P, P, i64, i32, f64, u32, i32, i64, i32, P, i32]
        lib.oracle_cell_opens.restype = i32
        lib.oracle_cell_opens.argtypes = [P, P, P, P, f64, P]
        lib.oracle_beam_tau.restype = f64
        lib.oracle_beam_tau.argtypes = [P, i64, i32, f64, i64, f64, i32]
        lib.oracle_J_directed.restype = i32
        lib.oracle_J_directed.argtypes = [P, P, i64, i32, f64, u32, P, P, i32]
        lib.oracle_csm_tables.restype = i32
        lib.oracle_csm_tables.argtypes = [P, i32, i32, P, P]
        lib.oracle_set_tau_refine.restype = i32
        lib.oracle_set_tau_refine.argtypes = [P, f64, P]
        lib.oracle_pp_sphere.restype = i64
        lib.oracle_pp_sphere.argtypes = [P, i64, i32, P, P]
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def morton_keys(pos, lo, size) -> np.ndarray:
    pos = _f64(pos, (-1, 3))
    out = np.empty(pos.shape[0], dtype=np.uint64)
    _load().oracle_morton_keys(_p(pos), pos.shape[0], _p(_f64(lo, (3,))), float(size), _p(out))
    return out


def pix2vec(nside: int) -> np.ndarray:
    out = np.empty((12 * nside * nside, 3))
    _load().oracle_pix2vec(int(nside), _p(out))
    return out


def vec2pix(nside: int, v) -> np.ndarray:
    v = _f64(v, (-1, 3))
    out = np.empty(v.shape[0], dtype=np.int64)
    _load().oracle_vec2pix(int(nside), _p(v), v.shape[0], _p(out))
    return out


def pair_of_pixel(nside: int, k: int) -> int:
    return int(_load().oracle_pair_of_pixel(int(nside), int(k)))


def transmission_alpha(E, axis, n, a1, a2):
    """alpha of Eq. transmissionavg and the geometry (V1, V2, V12, V, d)."""
    geo = np.zeros(5)
    a = _load().oracle_transmission_alpha(_p(_f64(E, (3,))), int(axis), _p(_f64(n, (3,))),
                                          float(a1), float(a2), _p(geo))
    return a, geo


def cell_opens(lo, hi, c, x, theta):
    """(opens?, B) for one cell with centre of luminosity c seen from x."""
    B = np.zeros(1)
    o = _load().oracle_cell_opens(_p(_f64(lo, (3,))), _p(_f64(hi, (3,))), _p(_f64(c, (3,))),
                                  _p(_f64(x, (3,))), float(theta), _p(B))
    return bool(o), float(B[0])


def soft_kernel(r, h):
    return _load().oracle_soft_kernel(float(r), float(h))


def thick_factor(tau):
    return _load().oracle_thick_factor(float(tau))


class OracleTree:
    """FP64 tree over one set of elements (inputs are copied)."""

    def __init__(self, pos, mass, kappa, lum, h=None, box_lo=None, box_size=0.0, bucket=12):
        lib = _load()
        pos = _f64(pos, (-1, 3))
        n = pos.shape[0]
        kappa = _f64(kappa).reshape(n, -1)
        self.nb = kappa.shape[1]
        lum = _f64(lum, (n, self.nb))
        mass = _f64(mass, (n,))
        hh = None if h is None else _f64(h, (n,))
        lo = None if box_lo is None else _f64(box_lo, (3,))
        self._keep = (pos, mass, kappa, lum, hh, lo)
        self.N = n
        self._h = lib.oracle_tree_build(_p(pos), _p(mass), _p(kappa), _p(lum), _p(hh), n,
                                        self.nb, _p(lo), float(box_size if lo is not None else 0.0),
                                        int(bucket))
        if not self._h:
            raise ValueError("oracle_tree_build rejected its inputs")

    @classmethod
    def from_case(cls, case):
        return cls(case["pos"], case["mass"], case["kappa"], case["lum"], case["h"],
                   case["box_lo"], case["box_size"], case["bucket"])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().oracle_tree_free(h)
            self._h = None

    @property
    def num_nodes(self) -> int:
        return int(_load().oracle_tree_num_nodes(self._h))

    @property
    def max_depth(self) -> int:
        return int(_load().oracle_tree_max_depth(self._h))

    def box(self):
        lo = np.zeros(3)
        size = np.zeros(1)
        _load().oracle_tree_box(self._h, _p(lo), _p(size))
        return lo, float(size[0])

    def export(self) -> dict:
        n = self.num_nodes
        out = {
            "keys": np.empty(self.N, np.uint64), "perm": np.empty(self.N, np.int64),
            "prefix": np.empty(n, np.uint64), "depth": np.empty(n, np.int32),
            "first": np.empty(n, np.int64), "count": np.empty(n, np.int64),
            "child": np.empty(n, np.int64), "parent": np.empty(n, np.int64),
            "box": np.empty((n, 6)),
        }
        o = out
        _load().oracle_tree_export(self._h, _p(o["keys"]), _p(o["perm"]), _p(o["prefix"]),
                                   _p(o["depth"]), _p(o["first"]), _p(o["count"]),
                                   _p(o["child"]), _p(o["parent"]), _p(o["box"]))
        return out

    def aggregates(self) -> dict:
        n, nb = self.num_nodes, self.nb
        o = {"L": np.empty((n, nb)), "Ltot": np.empty(n), "c": np.empty((n, 3)),
             "B": np.empty(n), "alpha_leaf": np.empty((n, nb))}
        _load().oracle_tree_aggregates(self._h, _p(o["L"]), _p(o["Ltot"]), _p(o["c"]),
                                       _p(o["B"]), _p(o["alpha_leaf"]))
        return o

    def alpha_table(self, nside: int, linear: bool = False) -> np.ndarray:
        out = np.empty((self.num_nodes, 6 * nside * nside, self.nb))
        if _load().oracle_alpha_table(self._h, int(nside), int(bool(linear)), _p(out)) != 0:
            raise ValueError("bad nside")
        return out

    def J(self, active, nside, theta, flags=0, nthreads=0, stats=False, target=None):
        active = np.ascontiguousarray(np.asarray(active, dtype=np.int64))
        a = active.shape[0]
        J = np.zeros((a, self.nb))
        if target is not None:  # directed rays (needs FLAG_BUCKET)
            tg = _f64(target, (3,))
            rc = _load().oracle_J_directed(self._h, _p(active), a, int(nside), float(theta),
                                           int(flags), _p(tg), _p(J), int(nthreads))
            if rc != 0:
                raise ValueError("oracle_J_directed rejected its inputs")
            return J
        st = np.zeros((a, 4), dtype=np.int64) if stats else None
        rc = _load().oracle_J(self._h, _p(active), a, int(nside), float(theta), int(flags),
                              _p(J), int(nthreads), _p(st))
        if rc != 0:
            raise ValueError("oracle_J rejected its inputs")
        return (J, st) if stats else J

    def beam_tau(self, i, nside, theta, k, s, band=0):
        """Optical depth along beam k of receiver i up to distance s (no r/s)."""
        return _load().oracle_beam_tau(self._h, int(i), int(nside), float(theta), int(k),
                                       float(s), int(band))

    def csm_tables(self, nside, linear=False):
        """Complex source model (R14): d [nodes][npix] and tau [nodes][npix][nb]."""
        npix = 12 * nside * nside
        d = np.empty((self.num_nodes, npix))
        tau = np.empty((self.num_nodes, npix, self.nb))
        if _load().oracle_csm_tables(self._h, int(nside), int(bool(linear)), _p(d), _p(tau)) != 0:
            raise ValueError("bad nside")
        return d, tau

    def set_tau_refine(self, tau_refine):
        """Refinement for every later call (R13; inf turns it off); returns the
        per-node optical-depth variation it compares with tau_refine."""
        out = np.empty(self.num_nodes)
        if _load().oracle_set_tau_refine(self._h, float(tau_refine), _p(out)) != 0:
            raise ValueError("tau_refine must be positive")
        return out

    def pp_sphere(self, i, nside):
        """(r_pp, sorted original indices of the p-p particles) of the bucket
        that holds element i (FLAG_PP)."""
        rpp = np.zeros(1)
        n = _load().oracle_pp_sphere(self._h, int(i), int(nside), _p(rpp), None)
        if n < 0:
            raise ValueError("bad element or nside")
        out = np.empty(n, np.int64)
        _load().oracle_pp_sphere(self._h, int(i), int(nside), _p(rpp), _p(out))
        return float(rpp[0]), out

    def J_deriv(self, active, nside, theta, which, elem, band, flags=0, nthreads=0):
        """dJ[A][nb]/d(kappa or lum)[elem][band] by forward-mode duals."""
        active = np.ascontiguousarray(np.asarray(active, dtype=np.int64))
        a = active.shape[0]
        dJ = np.zeros((a, self.nb))
        w = {"kappa": 0, "lum": 1}[which] if isinstance(which, str) else int(which)
        rc = _load().oracle_J_deriv(self._h, _p(active), a, int(nside), float(theta), int(flags),
                                    w, int(elem), int(band), _p(dJ), int(nthreads))
        if rc != 0:
            raise ValueError("oracle_J_deriv rejected its inputs")
        return dJ
