"""FP64 CPU oracle for the hashed oct-tree build (test infrastructure only).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark
import this package.  It wraps ``oracle.c`` (plain C, single thread,
compiled with ``-ffp-contract=off``) through ctypes and shares no code with
the CUDA library.  See ``oracle.c`` for what each routine computes and
which passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")

LEVELS = 22
DEPTH_MAX = 21


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, -O2, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        vp, i64, i32, u64, f64 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_double
        L.ora_min_depth.argtypes = [u64, u64]
        L.ora_min_depth.restype = C.c_int
        L.ora_interleave.argtypes = [C.c_uint32] * 3
        L.ora_interleave.restype = u64
        L.ora_quantise.argtypes = [C.c_float, f64, f64]
        L.ora_quantise.restype = C.c_uint32
        L.ora_root.argtypes = [vp, i64, vp, vp]
        L.ora_root.restype = C.c_int
        L.ora_root_mode.argtypes = [vp, i64, vp, vp, C.c_int]
        L.ora_root_mode.restype = C.c_int
        L.ora_keys_root.argtypes = [vp, i64, vp, vp, vp, C.c_int, C.c_int]
        L.ora_keys_root.restype = C.c_int
        L.ora_build_root.argtypes = [vp, i64, i32, C.c_int, C.c_int]
        L.ora_build_root.restype = vp
        L.ora_keys.argtypes = [vp, i64, vp, vp, vp]
        L.ora_keys.restype = C.c_int
        L.ora_keys_ordered.argtypes = [vp, i64, vp, vp, vp, C.c_int]
        L.ora_keys_ordered.restype = C.c_int
        L.ora_hilbert.argtypes = [C.c_uint32] * 3
        L.ora_hilbert.restype = u64
        L.ora_build_ordered.argtypes = [vp, i64, i32, C.c_int]
        L.ora_build_ordered.restype = vp
        L.ora_sort.argtypes = [vp, i64, vp, vp]
        L.ora_sort.restype = None
        L.ora_build.argtypes = [vp, i64, i32]
        L.ora_build.restype = vp
        L.ora_n_cells.argtypes = [vp]
        L.ora_n_cells.restype = i64
        L.ora_status.argtypes = [vp]
        L.ora_status.restype = C.c_int
        L.ora_get.argtypes = [vp] * 13
        L.ora_get.restype = None
        L.ora_free.argtypes = [vp]
        L.ora_free.restype = None
        L.ora_moments.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp]
        L.ora_moments.restype = None
        L.ora_paper_build.argtypes = [vp, i64, i32, i64, vp, vp, vp]
        L.ora_paper_build.restype = i64
        L.ora_direct_acc.argtypes = [vp, vp, i64, f64, vp, i64, vp]
        L.ora_direct_acc.restype = None
        L.ora_tree_walk.argtypes = [vp, vp, vp, vp, vp, vp, f64, f64, C.c_int, vp, i64, vp]
        L.ora_tree_walk.restype = None
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32pos(pos):
    return np.ascontiguousarray(pos, dtype=np.float32).reshape(-1, 3)


def min_depth(a: int, b: int) -> int:
    """Minimum distinguished depth of two 64-bit keys (Sec. 2.3.1)."""
    return lib().ora_min_depth(int(a), int(b))


def interleave(qx: int, qy: int, qz: int) -> int:
    return int(lib().ora_interleave(qx, qy, qz))


def quantise(x: float, lo: float, scale: float) -> int:
    return int(lib().ora_quantise(x, lo, scale))


ORDERS = {"morton": 0, "hilbert": 1}


def hilbert(qx: int, qy: int, qz: int) -> int:
    """Peano-Hilbert key of three 21-bit integers (Sec. 2.2 footnote)."""
    return int(lib().ora_hilbert(qx, qy, qz))


ROOTS = {"tight": 0, "pow2": 1}


def root(pos, root_mode: str = "tight"):
    """(lo float64[3], side) of the root cell: the tight bounding box, or
    (pow2) its side forced to the smallest power of two >= the largest extent
    (Sec. 2.2), the corner staying at the per-axis minimum."""
    pos = _f32pos(pos)
    lo = np.zeros(3)
    side = np.zeros(1)
    if lib().ora_root_mode(_p(pos), pos.shape[0], _p(lo), _p(side), ROOTS[root_mode]):
        raise ValueError("non-finite coordinate")
    return lo, float(side[0])


def keys(pos, order: str = "morton", root_mode: str = "tight"):
    """(keys uint64[n], lo float64[3], side) of the root cell (Sec. 2.2), in
    Morton or Peano-Hilbert order."""
    pos = _f32pos(pos)
    n = pos.shape[0]
    out = np.empty(n, dtype=np.uint64)
    lo = np.zeros(3)
    side = np.zeros(1)
    st = lib().ora_keys_root(_p(pos), n, _p(lo), _p(side), _p(out), ORDERS[order],
                             ROOTS[root_mode])
    if st:
        raise ValueError("non-finite coordinate")
    return out, lo, float(side[0])


def sort(keys_):
    keys_ = np.ascontiguousarray(keys_, dtype=np.uint64)
    n = keys_.shape[0]
    sk = np.empty(n, dtype=np.uint64)
    perm = np.empty(n, dtype=np.int32)
    lib().ora_sort(_p(keys_), n, _p(sk), _p(perm))
    return sk, perm


@dataclass
class Tree:
    """Oracle tree in canonical (level, key) order."""
    n: int
    n_crit: int
    lo: np.ndarray
    side: float
    skeys: np.ndarray
    perm: np.ndarray
    ckey: np.ndarray
    level: np.ndarray
    parent: np.ndarray
    child_first: np.ndarray
    child_end: np.ndarray
    pfirst: np.ndarray
    pend: np.ndarray
    level_offset: np.ndarray
    _handle: int = 0

    @property
    def n_cells(self) -> int:
        return int(self.ckey.shape[0])

    @property
    def max_depth(self) -> int:
        return int(self.level.max()) if self.n_cells else 0


class _Handle:
    def __init__(self, h):
        self.h = h

    def __del__(self):
        try:
            lib().ora_free(self.h)
        except Exception:
            pass


def build_tree(pos, n_crit: int, order: str = "morton", root_mode: str = "tight") -> Tree:
    """Top-down Barnes-Hut build (Sec. 2.1) over sorted keys; canonical order
    (level, then key in the chosen order); root cell as in root()."""
    pos = _f32pos(pos)
    n = pos.shape[0]
    h = lib().ora_build_root(_p(pos), n, int(n_crit), ORDERS[order], ROOTS[root_mode])
    if lib().ora_status(h):
        lib().ora_free(h)
        raise ValueError("non-finite coordinate")
    C_ = lib().ora_n_cells(h)
    t = Tree(n=n, n_crit=int(n_crit), lo=np.zeros(3), side=0.0,
             skeys=np.empty(n, np.uint64), perm=np.empty(n, np.int32),
             ckey=np.empty(C_, np.uint64), level=np.empty(C_, np.uint8),
             parent=np.empty(C_, np.int32), child_first=np.empty(C_, np.int32),
             child_end=np.empty(C_, np.int32), pfirst=np.empty(C_, np.int32),
             pend=np.empty(C_, np.int32), level_offset=np.empty(LEVELS + 1, np.int64))
    side = np.zeros(1)
    lib().ora_get(h, _p(t.skeys), _p(t.perm), _p(t.lo), _p(side), _p(t.ckey), _p(t.level),
                  _p(t.parent), _p(t.child_first), _p(t.child_end), _p(t.pfirst), _p(t.pend),
                  _p(t.level_offset))
    t.side = float(side[0])
    t._handle = _Handle(h)
    return t


def moments(tree: Tree, pos, mass=None, cells=None):
    """Direct FP64 sums over member particles: (M, com[.,3], quad[.,6], aabb[.,6] f32).

    quad order: xx, xy, xz, yy, yz, zz (central, about the FP64 COM);
    aabb: min x, min y, min z, max x, max y, max z.  ``cells`` selects a subset.
    """
    pos = _f32pos(pos)
    mass = None if mass is None else np.ascontiguousarray(mass, dtype=np.float32)
    if cells is not None:
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        nc = cells.shape[0]
    else:
        nc = tree.n_cells
    M = np.empty(nc)
    com = np.empty((nc, 3))
    quad = np.empty((nc, 6))
    aabb = np.empty((nc, 6), dtype=np.float32)
    lib().ora_moments(tree._handle.h, _p(pos), _p(mass), _p(cells), nc, _p(M), _p(com),
                      _p(quad), _p(aabb))
    return M, com, quad, aabb


def paper_build(skeys, n_leaf: int):
    """Alg. 1 leaves + Alg. 2 parents on sorted keys: (level u8, key u64, count i64)."""
    skeys = np.ascontiguousarray(skeys, dtype=np.uint64)
    n = skeys.shape[0]
    cap = max(64, 23 * n + 1)
    lv = np.empty(cap, np.uint8)
    k = np.empty(cap, np.uint64)
    c = np.empty(cap, np.int64)
    w = lib().ora_paper_build(_p(skeys), n, int(n_leaf), cap, _p(lv), _p(k), _p(c))
    if w < 0:
        raise RuntimeError("capacity exceeded")
    return lv[:w].copy(), k[:w].copy(), c[:w].copy()


def direct_acc(pos, mass, targets, eps: float):
    pos = _f32pos(pos)
    mass = None if mass is None else np.ascontiguousarray(mass, dtype=np.float32)
    targets = np.ascontiguousarray(targets, dtype=np.int64)
    acc = np.empty((targets.shape[0], 3))
    lib().ora_direct_acc(_p(pos), _p(mass), pos.shape[0], eps, _p(targets), targets.shape[0],
                         _p(acc))
    return acc


def tree_walk(tree: Tree, pos, mass, M, com, quad, targets, theta: float, eps: float,
              use_quad: bool = True):
    pos = _f32pos(pos)
    mass = None if mass is None else np.ascontiguousarray(mass, dtype=np.float32)
    M = np.ascontiguousarray(M, dtype=np.float64)
    com = np.ascontiguousarray(com, dtype=np.float64)
    quad = np.ascontiguousarray(quad, dtype=np.float64)
    targets = np.ascontiguousarray(targets, dtype=np.int64)
    acc = np.empty((targets.shape[0], 3))
    lib().ora_tree_walk(tree._handle.h, _p(pos), _p(mass), _p(M), _p(com), _p(quad), theta, eps,
                        int(use_quad), _p(targets), targets.shape[0], _p(acc))
    return acc


class PrefixIndex:
    """The oracle's own key order (FP64 keys, stable sort) for locating the
    members of a cell by its key prefix, on sizes where the full top-down
    build is too slow for a test."""

    def __init__(self, pos, order: str = "morton"):
        self.pos = _f32pos(pos)
        self.keys, self.lo, self.side = keys(self.pos, order)
        self.order = np.argsort(self.keys, kind="stable")
        self.skeys = self.keys[self.order]

    def members(self, level: int, ckey: int):
        """Original indices of the particles whose key starts with ckey at depth level."""
        sh = 63 - 3 * int(level)
        lo_k = np.uint64(int(ckey) << sh)
        hi_k = np.uint64((int(ckey) << sh) | ((1 << sh) - 1))
        a = int(np.searchsorted(self.skeys, lo_k, side="left"))
        b = int(np.searchsorted(self.skeys, hi_k, side="right"))
        return self.order[a:b]

    def moments(self, mass, levels, ckeys):
        """Direct FP64 sums over each listed cell's members (Sec. 2.3 footnote):
        (M, com[.,3], quad[.,6] central xx xy xz yy yz zz, aabb[.,6] f32, count)."""
        n = len(levels)
        M = np.empty(n)
        com = np.empty((n, 3))
        quad = np.empty((n, 6))
        aabb = np.empty((n, 6), np.float32)
        cnt = np.empty(n, np.int64)
        m_eq = np.float64(np.float32(1.0 / max(1, self.pos.shape[0])))
        for j, (lv, ck) in enumerate(zip(levels, ckeys)):
            idx = self.members(lv, ck)
            x = self.pos[idx].astype(np.float64)
            m = np.full(len(idx), m_eq) if mass is None else mass[idx].astype(np.float64)
            Mj = m.sum()
            c = (m[:, None] * x).sum(0) / Mj if Mj != 0 else x[0].copy()
            d = x - c
            q = [(m * d[:, a] * d[:, b]).sum() for a, b in ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))]
            M[j], com[j], quad[j] = Mj, c, q
            aabb[j, :3] = self.pos[idx].min(0)
            aabb[j, 3:] = self.pos[idx].max(0)
            cnt[j] = len(idx)
        return M, com, quad, aabb, cnt
