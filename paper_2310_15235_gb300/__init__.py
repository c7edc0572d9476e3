"""GB300-native TREVR2 reverse ray trace (Wadsley, Baumschlager & Shen,
arXiv:2310.15235): Python binding of the C ABI in ``include/trevr2.h``.

This module only marshals arguments: every step of the method runs in the
CUDA kernels of ``libtrevr2.so`` (built in-tree by ``build_lib.build()``).
There is no CPU fallback; without the library every call raises.

    tree = build(pos, mass, kappa, lum, h=None)    # Sec. 2.3 / 2.6
    J = tree.J(active, nside=2, theta=0.75)        # Sec. 2.5, [A, nb] float32

The paper's other schemes are flags of J: BUCKET (one walk per bucket from
its centre, Sec. 2.5.1) with PP (p-p absorption inside r_pp, Sec. 2.4) and
CSM (the complex source model, Sec. 2.7); LINEAR (the linear absorption
average of Sec. 2.6); SOFT and THICK (Eq. intint, Eq. taucorr).
``tree.J(..., target=p)`` aims the beam holding p at it (directed rays,
Sec. 3.4.1) and ``tree.set_tau_refine(t)`` turns on absorption refinement.

Tensors may live on the GPU (used in place) or on the host (copied to the
current CUDA device first; the result stays on the device).
"""

from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np
import torch

__all__ = [
    "SOFT", "THICK", "ASYNC", "Tree", "TrevrError", "build", "J", "library_path", "load_library",
    "healpix_pix2vec", "healpix_vec2pix", "exported_symbols", "FIELDS", "kernel_launches",
    "Batch", "J_batched", "J_fn", "LINEAR", "BUCKET", "PP", "CSM", "debug_set",
    "debug_pool_used", "DEBUG_FAIL_ALLOC", "DEBUG_SOURCE_STACK",
]

SOFT = 1
THICK = 2
ASYNC = 4
LINEAR = 8  # linear absorption averaging (Sec. 2.6's comparison scheme)
BUCKET = 16  # per-bucket beams from the bucket centre (Sec. 2.5.1), trevr2_J only
PP = 32  # with BUCKET: particle-particle absorption inside r_pp (Sec. 2.4)
CSM = 64  # with BUCKET: the complex source model (Sec. 2.7)

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libtrevr2.so")
_HEADER = os.path.join(os.path.dirname(_HERE), "include", "trevr2.h")
_lock = threading.Lock()
_lib = None

_CODES = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "EUNSUPPORTED",
          -6: "EINTERNAL"}

FIELDS = {
    "keys": (1, torch.int64, None), "perm": (2, torch.int32, None),
    "prefix": (3, torch.int64, None), "depth": (4, torch.int32, None),
    "first": (5, torch.int32, None), "count": (6, torch.int32, None),
    "child": (7, torch.int32, None), "parent": (8, torch.int32, None),
    "lum": (9, torch.float32, "nb"), "centre": (10, torch.float64, 3),
    "alpha_leaf": (11, torch.float32, "nb"), "B": (12, torch.float64, None),
}
_NODE_FIELDS = {"prefix", "depth", "first", "count", "child", "parent", "lum", "centre",
                "alpha_leaf", "B"}


class TrevrError(RuntimeError):
    """A negative status from libtrevr2 (the code name and the library's message)."""

    def __init__(self, code: int, message: str):
        self.code = code
        super().__init__(f"{_CODES.get(code, code)}: {message}")


class _Info(C.Structure):
    _fields_ = [("n_elements", C.c_int64), ("n_nodes", C.c_int64), ("n_internal", C.c_int64),
                ("n_leaves", C.c_int64), ("nb", C.c_int32), ("bucket", C.c_int32),
                ("max_depth", C.c_int32), ("reserved", C.c_int32),
                ("box_lo", C.c_double * 3), ("box_size", C.c_double)]


def kernel_launches() -> int:
    """Kernels launched by libtrevr2 in this process so far."""
    return int(load_library().trevr2_kernel_launches())


def kernel_binary_version() -> int:
    """Architecture of the loaded kernels on the current device (103 = sm_103a)."""
    v = C.c_int(0)
    _check(load_library().trevr2_kernel_binary_version(C.byref(v)))
    return int(v.value)


DEBUG_FAIL_ALLOC = 1
DEBUG_SOURCE_STACK = 2


def debug_set(what: int, value: int) -> None:
    """Testing aid: DEBUG_FAIL_ALLOC (the n-th device allocation from now on
    fails with ENOMEM; -1 turns it off) or DEBUG_SOURCE_STACK (cap the source
    cut's stack at c entries; 0 restores it)."""
    _check(load_library().trevr2_debug_set(int(what), int(value)))


def debug_pool_used() -> int:
    """Bytes libtrevr2 holds in the current device's default memory pool."""
    v = C.c_uint64(0)
    _check(load_library().trevr2_debug_pool_used(C.byref(v)))
    return int(v.value)


def library_path() -> str:
    return _LIB_PATH


def exported_symbols() -> list[str]:
    """Entry points declared in include/trevr2.h."""
    with open(_HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(trevr2_[A-Za-z0-9_]+)\s*\(", text)))


def load_library():
    """Loads libtrevr2.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                f"{_LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
                f"g.build()\"` (nvcc, sm_103a); there is no CPU fallback")
        lib = C.CDLL(_LIB_PATH)
        P, i64, i32, f32, f64, u32, sz = (C.c_void_p, C.c_int64, C.c_int, C.c_float, C.c_double,
                                          C.c_uint32, C.c_size_t)
        lib.trevr2_build.argtypes = [P, P, P, P, P, i64, i32, P, f64, i32, P, C.POINTER(P)]
        lib.trevr2_J.argtypes = [P, P, i64, i32, f32, P, i32, u32, P, P]
        lib.trevr2_J_directed.argtypes = [P, P, i64, i32, f32, P, i32, u32, P, P, P]
        lib.trevr2_set_tau_refine.argtypes = [P, C.c_double, P]
        lib.trevr2_status.argtypes = [P, P]
        lib.trevr2_prepare.argtypes = [P, i32, P]
        lib.trevr2_J_noalloc.argtypes = [P, P, i64, i32, f32, P, i32, u32, P, P]
        lib.trevr2_free.argtypes = [P]
        lib.trevr2_batch_create.argtypes = [P, i32, P, P, i32, i32, f32, u32, P, C.POINTER(P)]
        lib.trevr2_batch_run.argtypes = [P, P, P, P]
        lib.trevr2_batch_autotune.argtypes = [P, P, P, P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        lib.trevr2_batch_status.argtypes = [P, P]
        lib.trevr2_batch_free.argtypes = [P]
        lib.trevr2_J_batched.argtypes = [P, i32, P, P, P, i32, i32, f32, u32, P, P]
        lib.trevr2_J_backward.argtypes = [P, P, i64, i32, f32, P, i32, u32, P, P, P, P]
        lib.trevr2_last_error.restype = C.c_char_p
        lib.trevr2_tree_info_get.argtypes = [P, C.POINTER(_Info)]
        lib.trevr2_tree_export.argtypes = [P, i32, P, sz, P]
        lib.trevr2_alpha_table.argtypes = [P, i32, P, sz, P]
        lib.trevr2_healpix_pix2vec.argtypes = [i32, P, P]
        lib.trevr2_healpix_vec2pix.argtypes = [i32, P, i64, P, P]
        for name in exported_symbols():
            fn = getattr(lib, name)
            if name not in ("trevr2_last_error", "trevr2_kernel_launches"):
                fn.restype = C.c_int
        lib.trevr2_kernel_launches.restype = C.c_uint64
        lib.trevr2_kernel_launches.argtypes = []
        lib.trevr2_debug_set.argtypes = [i32, i64]
        lib.trevr2_kernel_binary_version.argtypes = [C.POINTER(C.c_int)]
        lib.trevr2_debug_pool_used.argtypes = [C.POINTER(C.c_uint64)]
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        msg = load_library().trevr2_last_error().decode(errors="replace")
        raise TrevrError(rc, msg)


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(x, dtype, device, shape=None):
    """The argument as a contiguous CUDA tensor of `dtype` (copied if needed)."""
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x))
    if not isinstance(x, torch.Tensor):
        x = torch.as_tensor(x)
    if x.dtype != dtype:
        x = x.to(dtype)
    if not x.is_cuda:
        x = x.pin_memory().to(device, non_blocking=True) if x.numel() else x.to(device)
    x = x.contiguous()
    if shape is not None:
        x = x.reshape(shape)
    return x


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


class Tree:
    """A radiation tree on the GPU (owns its device memory until `free`)."""

    def __init__(self, handle, device):
        self._h = handle
        self.device = device
        info = _Info()
        _check(load_library().trevr2_tree_info_get(self._h, C.byref(info)))
        self.N = int(info.n_elements)
        self.nb = int(info.nb)
        self.n_nodes = int(info.n_nodes)
        self.n_internal = int(info.n_internal)
        self.n_leaves = int(info.n_leaves)
        self.max_depth = int(info.max_depth)
        self.bucket = int(info.bucket)
        self.box_lo = tuple(info.box_lo)
        self.box_size = float(info.box_size)

    # -- compute -------------------------------------------------------------
    def J(self, active, nside: int = 2, theta: float = 0.75, bands=None, flags: int = 0,
          out: torch.Tensor | None = None, stream=None, target=None) -> torch.Tensor:
        """Integrated intensity per active receiver and band, [A, nbsel] float32.
        With `target` (a point, caller coordinates; needs BUCKET) the beam that
        holds the target's direction from each bucket centre points at it
        (directed rays, Sec. 3.4.1)."""
        self._alive()
        act = _dev(active, torch.int64, self.device).reshape(-1)
        nbsel = self.nb if bands is None else len(bands)
        if out is None:
            out = torch.empty((act.numel(), nbsel), dtype=torch.float32, device=self.device)
        barr = None
        if bands is not None:
            barr = (C.c_int * len(bands))(*[int(b) for b in bands])
        if target is not None:
            tg = (C.c_double * 3)(*[float(v) for v in np.asarray(target, dtype=np.float64).reshape(3)])
            _check(load_library().trevr2_J_directed(self._h, _ptr(act), act.numel(), int(nside),
                                                    float(theta), barr, int(nbsel), int(flags),
                                                    tg, _ptr(out), _stream_ptr(stream)))
            return out
        _check(load_library().trevr2_J(self._h, _ptr(act), act.numel(), int(nside), float(theta),
                                       barr, int(nbsel), int(flags), _ptr(out),
                                       _stream_ptr(stream)))
        return out

    def J_backward(self, active, gJ, nside: int = 2, theta: float = 0.75, bands=None,
                   flags: int = 0, stream=None) -> tuple[torch.Tensor, torch.Tensor]:
        """Adjoint of `J`: given gJ = dLoss/dJ [A, nbsel], returns
        (dLoss/dkappa [N, nb], dLoss/dlum [N, nb]) in the caller's element order."""
        self._alive()
        act = _dev(active, torch.int64, self.device).reshape(-1)
        nbsel = self.nb if bands is None else len(bands)
        g = _dev(gJ, torch.float32, self.device).reshape(act.numel(), nbsel)
        gk = torch.empty((self.N, self.nb), dtype=torch.float32, device=self.device)
        gl = torch.empty((self.N, self.nb), dtype=torch.float32, device=self.device)
        barr = None
        if bands is not None:
            barr = (C.c_int * len(bands))(*[int(b) for b in bands])
        _check(load_library().trevr2_J_backward(self._h, _ptr(act), act.numel(), int(nside),
                                                float(theta), barr, int(nbsel), int(flags),
                                                _ptr(g), _ptr(gk), _ptr(gl), _stream_ptr(stream)))
        return gk, gl

    def set_tau_refine(self, tau_refine: float, stream=None):
        """Absorption refinement for every later walk on this tree (Sec. 2.5.2):
        cells whose optical depth varies by more than tau_refine inside also
        open; float('inf') turns it off."""
        self._alive()
        _check(load_library().trevr2_set_tau_refine(self._h, float(tau_refine),
                                                    _stream_ptr(stream)))

    def prepare(self, nside: int, stream=None):
        """Builds and caches the per-direction tables for `nside` (no walk)."""
        self._alive()
        _check(load_library().trevr2_prepare(self._h, int(nside), _stream_ptr(stream)))

    def status(self, stream=None):
        self._alive()
        _check(load_library().trevr2_status(self._h, _stream_ptr(stream)))

    # -- introspection --------------------------------------------------------
    def export(self, field: str) -> torch.Tensor:
        self._alive()
        code, dtype, cols = FIELDS[field]
        rows = self.n_nodes if field in _NODE_FIELDS else self.N
        shape = (rows,) if cols is None else (rows, self.nb if cols == "nb" else cols)
        out = torch.empty(shape, dtype=dtype, device=self.device)
        _check(load_library().trevr2_tree_export(self._h, code, _ptr(out),
                                                 out.numel() * out.element_size(),
                                                 _stream_ptr()))
        torch.cuda.current_stream().synchronize()
        return out

    def alpha_table(self, nside: int) -> torch.Tensor:
        self._alive()
        out = torch.empty((self.n_nodes, 6 * nside * nside, self.nb), dtype=torch.float32,
                          device=self.device)
        _check(load_library().trevr2_alpha_table(self._h, int(nside), _ptr(out),
                                                 out.numel() * 4, _stream_ptr()))
        torch.cuda.current_stream().synchronize()
        return out

    # -- lifetime -------------------------------------------------------------
    def _alive(self):
        if not self._h:
            raise ValueError("tree already freed")

    def free(self):
        if getattr(self, "_h", None):
            load_library().trevr2_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _subset_layout(trees, offsets, tree_of):
    """Host arrays of a batch: tree handles, offsets [nsub+1] int64, tree_of [nsub] int32."""
    trees = list(trees)
    for t in trees:
        t._alive()
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64).reshape(-1))
    tof = np.ascontiguousarray(np.asarray(tree_of, dtype=np.int32).reshape(-1))
    if off.size != tof.size + 1:
        raise ValueError("offsets needs one more entry than tree_of")
    handles = (C.c_void_p * max(len(trees), 1))(*[t._h for t in trees])
    return trees, handles, off, tof


class Batch:
    """Many receiver subsets over several trees walked in one persistent launch.

    Subset s owns rows offsets[s]..offsets[s+1]-1 of the concatenated receiver
    list and is walked in trees[tree_of[s]] (individual timesteps, Sec. 1.2;
    independent snapshots, Sec. 3.1).  Rows asking for the same receiver of
    the same tree are walked once; with flags=BUCKET (optionally | PP | CSM)
    every distinct bucket of a tree is walked once for all the receivers the
    subsets ask for.  `run` enqueues a fixed sequence of kernels with no
    allocation or synchronisation, so it can be recorded into a CUDA graph and
    replayed.
    """

    def __init__(self, trees, offsets, tree_of, nside: int = 2, theta: float = 0.75,
                 flags: int = 0, stream=None):
        self.trees, handles, self.offsets, self.tree_of = _subset_layout(trees, offsets, tree_of)
        if not self.trees:
            raise ValueError("a batch needs at least one tree")
        self.device = self.trees[0].device
        self.nb = self.trees[0].nb
        self.total = int(self.offsets[-1]) if self.offsets.size else 0
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(load_library().trevr2_batch_create(
                handles, len(self.trees), self.offsets.ctypes.data_as(C.c_void_p),
                self.tree_of.ctypes.data_as(C.c_void_p), int(self.tree_of.size), int(nside),
                float(theta), int(flags), _stream_ptr(stream), C.byref(self._h)))

    def _io(self, active, out):
        act = _dev(active, torch.int64, self.device).reshape(-1)
        if act.numel() != self.total:
            raise ValueError(f"active has {act.numel()} entries, the batch has {self.total} rows")
        if out is None:
            out = torch.empty((self.total, self.nb), dtype=torch.float32, device=self.device)
        elif out.shape != (self.total, self.nb) or out.dtype != torch.float32 or not (
                out.is_cuda and out.is_contiguous()):
            raise ValueError("out must be a contiguous CUDA float32 tensor [total, nb]")
        return act, out

    def run(self, active, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Enqueues the walk of all rows; returns J [total, nb] (not synchronised)."""
        self._alive()
        act, out = self._io(active, out)
        _check(load_library().trevr2_batch_run(self._h, _ptr(act), _ptr(out), _stream_ptr(stream)))
        return out

    def autotune(self, active, out: torch.Tensor | None = None, stream=None) -> tuple[int, int]:
        """Times the launch shapes on a prefix and keeps the fastest: (warps, staged sources)."""
        self._alive()
        act, out = self._io(active, out)
        w, m = C.c_int(0), C.c_int(0)
        _check(load_library().trevr2_batch_autotune(self._h, _ptr(act), _ptr(out),
                                                    _stream_ptr(stream), C.byref(w), C.byref(m)))
        return int(w.value), int(m.value)

    def status(self, stream=None):
        self._alive()
        _check(load_library().trevr2_batch_status(self._h, _stream_ptr(stream)))

    def _alive(self):
        if not self._h:
            raise ValueError("batch already freed")

    def free(self):
        if getattr(self, "_h", None):
            load_library().trevr2_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def J_batched(trees, active, offsets, tree_of, nside: int = 2, theta: float = 0.75,
              flags: int = 0, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """One-shot batch: J [offsets[-1], nb] for every subset (synchronises unless ASYNC)."""
    trees, handles, off, tof = _subset_layout(trees, offsets, tree_of)
    if not trees:
        raise ValueError("J_batched needs at least one tree")
    dev = trees[0].device
    act = _dev(active, torch.int64, dev).reshape(-1)
    total = int(off[-1]) if off.size else 0
    if act.numel() != total:
        raise ValueError(f"active has {act.numel()} entries, offsets say {total}")
    if out is None:
        out = torch.empty((total, trees[0].nb), dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        _check(load_library().trevr2_J_batched(
            handles, len(trees), _ptr(act), off.ctypes.data_as(C.c_void_p),
            tof.ctypes.data_as(C.c_void_p), int(tof.size), int(nside), float(theta), int(flags),
            _ptr(out), _stream_ptr(stream)))
    return out


def build(pos, mass, kappa, lum, h=None, box_lo=None, box_size: float = 0.0, bucket: int = 12,
          device=None, stream=None) -> Tree:
    """Builds the radiation tree (Sec. 2.3) from element positions [N,3] (float64),
    masses [N], opacities [N,nb], luminosities [N,nb] and optional sizes h [N]."""
    lib = load_library()
    if device is None:
        device = pos.device if isinstance(pos, torch.Tensor) and pos.is_cuda else torch.device(
            "cuda", torch.cuda.current_device())
    p = _dev(pos, torch.float64, device)
    n = p.numel() // 3
    p = p.reshape(n, 3)
    m = _dev(mass, torch.float32, device).reshape(n)
    k = _dev(kappa, torch.float32, device).reshape(n, -1)
    nb = k.shape[1] if n else (k.shape[1] if k.dim() == 2 else 1)
    l_ = _dev(lum, torch.float32, device).reshape(n, nb)
    hh = None if h is None else _dev(h, torch.float32, device).reshape(n)
    lo = None
    if box_lo is not None and box_size > 0:
        lo = (C.c_double * 3)(*[float(v) for v in box_lo])
    handle = C.c_void_p()
    with torch.cuda.device(device):
        _check(lib.trevr2_build(_ptr(p), _ptr(m), _ptr(k), _ptr(l_), _ptr(hh), n, int(nb), lo,
                                float(box_size if lo is not None else 0.0), int(bucket),
                                _stream_ptr(stream), C.byref(handle)))
    return Tree(handle, device)


def J(tree: Tree, active, nside: int = 2, theta: float = 0.75, bands=None, flags: int = 0,
      out=None, stream=None) -> torch.Tensor:
    return tree.J(active, nside, theta, bands, flags, out, stream)


class _JFunction(torch.autograd.Function):
    """J as a differentiable function of the opacities and luminosities.

    Forward builds the tree and walks it; backward walks it again through the
    adjoint (no traversal is stored) and returns dLoss/dkappa and dLoss/dlum.
    Positions, masses and sizes get no gradient.
    """

    @staticmethod
    def forward(ctx, kappa, lum, pos, mass, h, active, opts):
        tree = build(pos, mass, kappa.detach(), lum.detach(), h, opts["box_lo"],
                     opts["box_size"], opts["bucket"])
        act = _dev(active, torch.int64, tree.device).reshape(-1)
        out = tree.J(act, opts["nside"], opts["theta"], opts["bands"], opts["flags"])
        ctx.tree, ctx.act, ctx.opts = tree, act, opts
        ctx.shapes = (kappa.shape, kappa.dtype, lum.shape, lum.dtype)
        return out

    @staticmethod
    def backward(ctx, gJ):
        o = ctx.opts
        gk, gl = ctx.tree.J_backward(ctx.act, gJ.contiguous(), o["nside"], o["theta"], o["bands"],
                                     o["flags"])
        ctx.tree.free()
        ks, kd, ls, ld = ctx.shapes
        return gk.reshape(ks).to(kd), gl.reshape(ls).to(ld), None, None, None, None, None


def J_fn(pos, mass, kappa, lum, active, nside: int = 2, theta: float = 0.75, h=None, bands=None,
         flags: int = 0, box_lo=None, box_size: float = 0.0, bucket: int = 12) -> torch.Tensor:
    """Differentiable J [A, nbsel] (autograd gives dLoss/dkappa and dLoss/dlum)."""
    opts = {"nside": int(nside), "theta": float(theta), "bands": bands, "flags": int(flags),
            "box_lo": box_lo, "box_size": float(box_size), "bucket": int(bucket)}
    return _JFunction.apply(kappa, lum, pos, mass, h, active, opts)


def healpix_pix2vec(nside: int, device=None) -> torch.Tensor:
    device = device or torch.device("cuda", torch.cuda.current_device())
    out = torch.empty((12 * nside * nside, 3), dtype=torch.float64, device=device)
    _check(load_library().trevr2_healpix_pix2vec(int(nside), _ptr(out), _stream_ptr()))
    return out


def healpix_vec2pix(nside: int, v) -> torch.Tensor:
    v = _dev(v, torch.float64, torch.device("cuda", torch.cuda.current_device())).reshape(-1, 3)
    out = torch.empty((v.shape[0],), dtype=torch.int32, device=v.device)
    _check(load_library().trevr2_healpix_vec2pix(int(nside), _ptr(v), v.shape[0], _ptr(out),
                                                 _stream_ptr()))
    return out
