"""CPU FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library in
``paper_1705_04702_gb300``) never imports it, and this package imports
nothing from the product except the seeded input descriptions in
``paper_1705_04702_gb300.workloads`` (which hold none of the method's
arithmetic).

``trace`` wraps the plain C implementation in ``mcrt_oracle.c`` (packet life
cycle); ``emission`` and ``mlp`` hold the NumPy FP64 references of the dust
emission step and of its surrogate network.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmcrt_oracle.so")
_SOURCES = [os.path.join(_HERE, "mcrt_oracle.c")]
_HEADERS = [os.path.join(_HERE, "mcrt_oracle.h")]
_lock = threading.Lock()
_lib = None

REC_FIELDS = 8
ERR_EVENT_CAP, ERR_SOURCE, ERR_NONFINITE, ERR_TREE = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no FMA contraction so that
    x86 and Arm give bit-identical results)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest_src = max(os.path.getmtime(p) for p in _SOURCES + _HEADERS)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest_src:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp] + _SOURCES + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bbox", ctypes.c_double * 6),
        ("kr", ctypes.POINTER(ctypes.c_double)),
        ("src_kind", ctypes.c_int),
        ("src_pos", ctypes.c_double * 3),
        ("src_dir", ctypes.c_double * 3),
        ("h_R", ctypes.c_double), ("h_z", ctypes.c_double),
        ("cell_cdf", ctypes.POINTER(ctypes.c_double)),
        ("nlambda", ctypes.c_int),
        ("kscale", ctypes.POINTER(ctypes.c_double)),
        ("albedo", ctypes.POINTER(ctypes.c_double)),
        ("g", ctypes.POINTER(ctypes.c_double)),
        ("lsrc", ctypes.POINTER(ctypes.c_double)),
        ("npk", ctypes.POINTER(ctypes.c_uint64)),
        ("seed", ctypes.c_uint64),
        ("phase", ctypes.c_uint32),
        ("ninstr", ctypes.c_int),
        ("instr", ctypes.POINTER(ctypes.c_double)),
        ("w_min", ctypes.c_double),
        ("max_events", ctypes.c_int),
        ("peel", ctypes.c_int),
        ("pk_begin", ctypes.c_uint64), ("pk_end", ctypes.c_uint64),
        ("absorbed", ctypes.POINTER(ctypes.c_double)),
        ("images", ctypes.POINTER(ctypes.c_double)),
        ("sed", ctypes.POINTER(ctypes.c_double)),
        ("ledger", ctypes.POINTER(ctypes.c_double)),
        ("counters", ctypes.POINTER(ctypes.c_double)),
        ("nrec", ctypes.c_int),
        ("records", ctypes.POINTER(ctypes.c_double)),
        ("status", ctypes.c_int),
        ("oct_levels", ctypes.c_int),
        ("oct_nleaf", ctypes.c_int64),
        ("oct_leaves", ctypes.POINTER(ctypes.c_int32)),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.og_trace.argtypes = [ctypes.POINTER(_Problem)]
            L.og_trace.restype = ctypes.c_int
            L.og_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
            L.og_philox4x32_10.restype = None
            L.og_uniform.argtypes = [ctypes.c_uint32]
            L.og_uniform.restype = ctypes.c_double
            L.og_path.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int]
            L.og_path.restype = ctypes.c_int
            L.og_hg_mu.argtypes = [ctypes.c_double, ctypes.c_double]
            L.og_hg_mu.restype = ctypes.c_double
            L.og_rotate.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_double)]
            L.og_rotate.restype = None
            L.og_octree_check.argtypes = [ctypes.POINTER(_Problem)]
            L.og_octree_check.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().og_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(x: int) -> float:
    return lib().og_uniform(int(x) & 0xffffffff)


def hg_mu(g: float, u: float) -> float:
    return lib().og_hg_mu(float(g), float(u))


def rotate(k, mu, phi):
    kk = (ctypes.c_double * 3)(*[float(v) for v in k])
    out = (ctypes.c_double * 3)()
    lib().og_rotate(kk, float(mu), float(phi), out)
    return np.array(list(out))


class _Keep:
    """Holds the numpy buffers a ctypes problem points into."""


def _make_problem(prob, keep, pk_begin=0, pk_end=None, nrec=0, peel=True, cell_cdf=None,
                  outputs=True):
    g = prob.grid
    P = _Problem()
    P.nx, P.ny, P.nz = g.nx, g.ny, g.nz
    P.bbox = (ctypes.c_double * 6)(*[float(v) for v in g.bbox])
    keep.kr = np.ascontiguousarray(g.kr, dtype=np.float32).astype(np.float64).ravel()
    P.kr = _dp(keep.kr)
    s = prob.source
    P.src_kind = int(s.kind)
    P.src_pos = (ctypes.c_double * 3)(*[float(v) for v in s.pos])
    P.src_dir = (ctypes.c_double * 3)(*[float(v) for v in s.dir])
    P.h_R, P.h_z = float(s.h_R), float(s.h_z)
    if cell_cdf is not None:
        keep.cdf = np.ascontiguousarray(cell_cdf, dtype=np.float64).ravel()
        P.cell_cdf = _dp(keep.cdf)
    wl = prob.wl
    NL = wl.n
    P.nlambda = NL
    keep.kscale = np.ascontiguousarray(wl.kscale, dtype=np.float64)
    keep.albedo = np.ascontiguousarray(wl.albedo, dtype=np.float64)
    keep.g = np.ascontiguousarray(wl.g, dtype=np.float64)
    keep.lsrc = np.ascontiguousarray(wl.lsrc, dtype=np.float64)
    keep.npk = np.ascontiguousarray(prob.npk, dtype=np.uint64)
    P.kscale, P.albedo, P.g, P.lsrc = _dp(keep.kscale), _dp(keep.albedo), _dp(keep.g), _dp(keep.lsrc)
    P.npk = keep.npk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    P.seed = int(prob.seed) & 0xffffffffffffffff
    P.phase = int(prob.phase)
    P.ninstr = len(prob.instruments)
    keep.instr = np.array([[i.distance, i.inclination, i.azimuth, i.fov, i.npx]
                           for i in prob.instruments], dtype=np.float64).reshape(-1)
    if keep.instr.size == 0:
        keep.instr = np.zeros(5)
    P.instr = _dp(keep.instr)
    P.w_min = float(prob.w_min)
    P.max_events = int(prob.max_events)
    P.peel = 1 if peel else 0
    P.pk_begin = int(pk_begin)
    P.pk_end = int(pk_end) if pk_end is not None else 0xffffffffffffffff
    if outputs:
        npx_tot = sum(i.npx * i.npx for i in prob.instruments)
        keep.absorbed = np.zeros((g.ncell, NL))
        keep.images = np.zeros(max(npx_tot * NL, 1))
        keep.sed = np.zeros((max(P.ninstr, 1), NL))
        keep.ledger = np.zeros((NL, 4))
        keep.counters = np.zeros(4)
        keep.records = np.zeros((NL, max(nrec, 1), REC_FIELDS))
        P.absorbed, P.images, P.sed = _dp(keep.absorbed), _dp(keep.images), _dp(keep.sed)
        P.ledger, P.counters, P.records = _dp(keep.ledger), _dp(keep.counters), _dp(keep.records)
        P.nrec = int(nrec)
    P.status = 0
    leaves = getattr(g, "leaves", None)
    if leaves is not None:
        keep.leaves = np.ascontiguousarray(leaves, dtype=np.int32).reshape(-1)
        P.oct_levels = int(g.max_level)
        P.oct_nleaf = int(g.ncell)
        P.oct_leaves = keep.leaves.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    return P


def trace(prob, pk_begin=0, pk_end=None, nrec=0, peel=True, cell_cdf=None):
    """Run packets [pk_begin, pk_end) of every wavelength of ``prob`` through
    the FP64 life cycle and return the tallies.

    Returns a dict: absorbed [ncell, nlambda], images (list per instrument of
    [npx, npx, nlambda]), sed [ninstr, nlambda], ledger [nlambda, 4]
    (emitted, absorbed, escaped, residual), counters [4] (scatterings,
    deposit segments, locate segments, peel segments), records
    [nlambda, nrec, 8] (scatterings, escaped, absorbed, residual, peeled
    flux, x, y, z of the last interaction), status (OR of ERR_* bits)."""
    keep = _Keep()
    P = _make_problem(prob, keep, pk_begin, pk_end, nrec, peel, cell_cdf)
    status = lib().og_trace(ctypes.byref(P))
    NL = prob.wl.n
    imgs, off = [], 0
    for ins in prob.instruments:
        n = ins.npx * ins.npx * NL
        imgs.append(keep.images[off:off + n].reshape(ins.npx, ins.npx, NL))
        off += n
    return {
        "absorbed": keep.absorbed,
        "images": imgs,
        "images_flat": keep.images[:off],
        "sed": keep.sed[:len(prob.instruments)],
        "ledger": keep.ledger,
        "counters": keep.counters,
        "records": keep.records[:, :nrec] if nrec else keep.records[:, :0],
        "status": int(status),
    }


def octree_valid(grid) -> bool:
    """True when the leaves of an octree description tile its root box."""
    keep = _Keep()
    P = _Problem()
    P.nx = P.ny = P.nz = grid.nx
    P.bbox = (ctypes.c_double * 6)(*[float(v) for v in grid.bbox])
    keep.leaves = np.ascontiguousarray(grid.leaves, dtype=np.int32).reshape(-1)
    P.oct_levels = int(grid.max_level)
    P.oct_nleaf = int(grid.ncell)
    P.oct_leaves = keep.leaves.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    return lib().og_octree_check(ctypes.byref(P)) == 0


def path(prob, p, k):
    """Cells and lengths crossed from p along k (oracle's own geometry)."""
    keep = _Keep()
    P = _make_problem(prob, keep, outputs=False)
    cap = prob.grid.nx + prob.grid.ny + prob.grid.nz + 8
    cells = (ctypes.c_int * cap)()
    lens = (ctypes.c_double * cap)()
    pp = (ctypes.c_double * 3)(*[float(v) for v in p])
    kk = (ctypes.c_double * 3)(*[float(v) for v in k])
    n = lib().og_path(ctypes.byref(P), pp, kk, cells, lens, cap)
    return np.array(cells[:n], dtype=np.int64), np.array(lens[:n])
