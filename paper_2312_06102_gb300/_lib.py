"""ctypes marshalling for libtb (include/tb.h).  No arithmetic of the build
lives here."""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libtb.so")

LEVELS = 22
MOM_FP32_COMP, MOM_FP32_PLAIN, MOM_FP64 = 0, 1, 2
STATUS = {0: "TB_OK", 1: "TB_EINVAL", 2: "TB_ENOMEM", 3: "TB_ECUDA", 4: "TB_EOVERFLOW",
          5: "TB_ETIMEOUT", 6: "TB_ENONFINITE"}


class TbError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({status_string(code)})")
        self.code = code
        self.name = STATUS.get(code, str(code))


class Params(C.Structure):
    _fields_ = [("n_crit", C.c_int32), ("mom_mode", C.c_int32), ("cell_capacity", C.c_int64),
                ("reorder", C.c_int32), ("radix_bits", C.c_int32), ("sort_threads", C.c_int32),
                ("sort_items", C.c_int32), ("batch_threads", C.c_int32), ("key_order", C.c_int32),
                ("batch_one_launch", C.c_int32), ("root_pow2", C.c_int32)]


_vp = C.c_void_p


class TreeC(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("n_cells", C.c_int64), ("n_leaves", C.c_int64),
                ("max_depth", C.c_int32), ("n_crit", C.c_int32),
                ("level_offset", C.c_int64 * (LEVELS + 1)), ("lo", C.c_double * 3),
                ("side", C.c_double), ("cell_capacity", C.c_int64),
                ("pkey", _vp), ("perm", _vp),
                ("ckey", _vp), ("level", _vp), ("parent", _vp), ("child_first", _vp),
                ("child_end", _vp), ("pfirst", _vp), ("pend", _vp), ("leaf_cell", _vp),
                ("mass", _vp), ("com", _vp), ("com_lo", _vp), ("quad", _vp), ("aabb", _vp),
                ("mass64", _vp), ("com64", _vp), ("quad64", _vp),
                ("pos_sorted", _vp),
                ("n_sets", C.c_int32), ("set_particle_offset", _vp), ("set_cell_offset", _vp),
                ("set_root", _vp), ("internal", _vp)]


_lib = None


def library_path() -> str:
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"CUDA library not built: {_LIB_PATH} (run compile_lib.py or __graft_entry__.build())")
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER
        L.tb_build.argtypes = [_vp, _vp, C.c_int64, P(Params), _vp, P(P(TreeC))]
        L.tb_build.restype = C.c_int
        L.tb_moments.argtypes = [P(TreeC), _vp, _vp, _vp]
        L.tb_moments.restype = C.c_int
        L.tb_build_batched.argtypes = [_vp, _vp, _vp, C.c_int32, C.c_int64, P(Params), _vp,
                                       P(P(TreeC))]
        L.tb_build_batched.restype = C.c_int
        L.tb_free.argtypes = [P(TreeC)]
        L.tb_free.restype = None
        L.tb_tree_status.argtypes = [P(TreeC), _vp]
        L.tb_tree_status.restype = C.c_int
        L.tb_status_string.argtypes = [C.c_int]
        L.tb_status_string.restype = C.c_char_p
        L.tb_default_params.argtypes = []
        L.tb_default_params.restype = Params
        L.tb_kernel_launches.argtypes = []
        L.tb_kernel_launches.restype = C.c_int64
        L.tb_profile.argtypes = [P(TreeC), C.c_int32]
        L.tb_profile.restype = C.c_int
        L.tb_stage_times.argtypes = [P(TreeC), _vp, P(C.c_float), C.c_int32]
        L.tb_stage_times.restype = C.c_int32
        L.tb_stage_name.argtypes = [P(TreeC), C.c_int32]
        L.tb_stage_name.restype = C.c_char_p
        L.tb_sort_variant.argtypes = [C.c_int32, P(C.c_int32), P(C.c_int32), P(C.c_int32)]
        L.tb_sort_variant.restype = C.c_int32
        L.tb_keys_sorted_noalloc.argtypes = [_vp, C.c_int64, _vp, _vp, P(C.c_double), _vp]
        L.tb_keys_sorted_noalloc.restype = C.c_int
        L.tb_walk.argtypes = [P(TreeC), C.c_float, C.c_float, C.c_int32, C.c_int32, _vp, _vp]
        L.tb_walk.restype = C.c_int
        L.tb_reorder.argtypes = [P(TreeC), _vp, _vp, C.c_int64, _vp]
        L.tb_reorder.restype = C.c_int
        L.tb_selftest_wait.argtypes = [C.c_int64, _vp]
        L.tb_selftest_wait.restype = C.c_int
        L.tb_walk_counts.argtypes = [P(TreeC), _vp, P(C.c_int64), P(C.c_int64)]
        L.tb_walk_counts.restype = C.c_int
        L.tb_set_wait_limit.argtypes = [C.c_int64]
        L.tb_set_wait_limit.restype = C.c_int
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().tb_status_string(int(code)).decode()


def kernel_launches() -> int:
    return int(lib().tb_kernel_launches())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class _DevView:
    """__cuda_array_interface__ over library-owned device memory."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None, "stream": None}


_TYPES = {"u8": "|u1", "u64": "<u8", "i32": "<i4", "i64": "<i8", "f32": "<f4", "f64": "<f8"}


def _view(ptr, shape, kind):
    if not ptr or any(s == 0 for s in shape):
        dt = {"u8": torch.uint8, "u64": torch.uint64, "i32": torch.int32, "i64": torch.int64,
              "f32": torch.float32, "f64": torch.float64}[kind]
        return torch.empty(shape, dtype=dt, device="cuda")
    return torch.as_tensor(_DevView(ptr, shape, _TYPES[kind]), device="cuda")


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on the GPU")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


class Tree:
    """A tree owned by the library; array properties are CUDA tensor views
    valid until the tree is rebuilt or freed."""

    def __init__(self):
        self._p = C.POINTER(TreeC)()

    def __del__(self):
        try:
            if self._p:
                lib().tb_free(self._p)
        except Exception:
            pass

    @property
    def c(self) -> TreeC:
        return self._p.contents

    def free(self):
        if self._p:
            lib().tb_free(self._p)
            self._p = C.POINTER(TreeC)()

    def sync(self, stream=None) -> int:
        return int(lib().tb_tree_status(self._p, _stream(stream)))

    def profile(self, on: bool = True):
        lib().tb_profile(self._p, int(on))

    def stage_times(self, stream=None, max_events: int = 1 << 16):
        """(name, ms) of every stage recorded since profiling was enabled or
        last read; reading restarts the accumulation."""
        buf = (C.c_float * max_events)()
        k = lib().tb_stage_times(self._p, _stream(stream), buf, max_events)
        return [(lib().tb_stage_name(self._p, i).decode(), float(buf[i])) for i in range(k)]

    # scalars
    n = property(lambda s: int(s.c.n_particles))
    n_cells = property(lambda s: int(s.c.n_cells))
    n_leaves = property(lambda s: int(s.c.n_leaves))
    # the cell views never reach past the allocated arrays, also after a
    # build that ran out of capacity (n_cells then holds the count needed)
    _nc = property(lambda s: min(int(s.c.n_cells), int(s.c.cell_capacity)))
    max_depth = property(lambda s: int(s.c.max_depth))
    level_offset = property(lambda s: [int(v) for v in s.c.level_offset])
    lo = property(lambda s: [float(v) for v in s.c.lo])
    side = property(lambda s: float(s.c.side))
    n_sets = property(lambda s: int(s.c.n_sets))

    # particle arrays
    pkey = property(lambda s: _view(s.c.pkey, (s.n,), "u64"))
    perm = property(lambda s: _view(s.c.perm, (s.n,), "i32"))
    pos_sorted = property(lambda s: _view(s.c.pos_sorted, (s.n, 4), "f32"))
    # cell arrays
    ckey = property(lambda s: _view(s.c.ckey, (s._nc,), "u64"))
    level = property(lambda s: _view(s.c.level, (s._nc,), "u8"))
    parent = property(lambda s: _view(s.c.parent, (s._nc,), "i32"))
    child_first = property(lambda s: _view(s.c.child_first, (s._nc,), "i32"))
    child_end = property(lambda s: _view(s.c.child_end, (s._nc,), "i32"))
    pfirst = property(lambda s: _view(s.c.pfirst, (s._nc,), "i32"))
    pend = property(lambda s: _view(s.c.pend, (s._nc,), "i32"))
    leaf_cell = property(lambda s: _view(s.c.leaf_cell, (s.n_leaves,), "i32"))
    mass = property(lambda s: _view(s.c.mass, (s._nc,), "f32"))
    com = property(lambda s: _view(s.c.com, (s._nc, 3), "f32"))
    com_lo = property(lambda s: _view(s.c.com_lo, (s._nc, 3), "f32"))
    quad = property(lambda s: _view(s.c.quad, (s._nc, 6), "f32"))
    aabb = property(lambda s: _view(s.c.aabb, (s._nc, 6), "f32"))
    mass64 = property(lambda s: _view(s.c.mass64, (s._nc,), "f64"))
    com64 = property(lambda s: _view(s.c.com64, (s._nc, 3), "f64"))
    quad64 = property(lambda s: _view(s.c.quad64, (s._nc, 6), "f64"))
    set_cell_offset = property(lambda s: _view(s.c.set_cell_offset, (s.n_sets + 1,), "i64"))
    set_particle_offset = property(lambda s: _view(s.c.set_particle_offset, (s.n_sets + 1,), "i64"))
    set_root = property(lambda s: _view(s.c.set_root, (s.n_sets, 4), "f64"))


def sort_variants():
    """(radix_bits, threads, items) of every compiled radix-sort variant."""
    out, i = [], 0
    b, t, k = C.c_int32(), C.c_int32(), C.c_int32()
    while lib().tb_sort_variant(i, C.byref(b), C.byref(t), C.byref(k)):
        out.append((b.value, t.value, k.value))
        i += 1
    return out


def _params(n_crit, mom_mode, cell_capacity, reorder, radix_bits, batch_threads, sort_cfg=None):
    p = lib().tb_default_params()
    p.n_crit = int(n_crit)
    p.mom_mode = int(mom_mode)
    p.cell_capacity = int(cell_capacity)
    p.reorder = int(reorder)
    p.radix_bits = int(radix_bits)
    p.batch_threads = int(batch_threads)
    if sort_cfg:
        p.radix_bits, p.sort_threads, p.sort_items = (int(v) for v in sort_cfg)
    return p


def _check(code, what):
    if code != 0:
        raise TbError(int(code), what)


KEYS_MORTON, KEYS_HILBERT = 0, 1


def build(pos: torch.Tensor, mass: torch.Tensor | None = None, n_crit: int = 16,
          mom_mode: int = MOM_FP32_COMP, cell_capacity: int = 0, reorder: bool = False,
          radix_bits: int = 0, tree: Tree | None = None, stream=None, sort_cfg=None,
          key_order: int = KEYS_MORTON, root_pow2: bool = False) -> Tree:
    """tb_build on a [n,3] float32 CUDA tensor; returns (or rebuilds) a Tree.
    sort_cfg = (radix_bits, threads, items) picks a compiled sort variant;
    key_order is KEYS_MORTON or KEYS_HILBERT; root_pow2 forces the root
    cube's side to a power of two."""
    if pos.dtype != torch.float32 or pos.dim() != 2 or pos.shape[1] != 3:
        raise ValueError("pos must be a [n,3] float32 tensor")
    t = tree if tree is not None else Tree()
    if sort_cfg is None and not radix_bits:
        from . import autotune
        sort_cfg = autotune.cached(pos.shape[0])
    p = _params(n_crit, mom_mode, cell_capacity, reorder, radix_bits, 0, sort_cfg)
    p.key_order = int(key_order)
    p.root_pow2 = int(bool(root_pow2))
    code = lib().tb_build(_ptr(pos), _ptr(mass), pos.shape[0], C.byref(p), _stream(stream),
                          C.byref(t._p))
    _check(code, "tb_build")
    return t


def moments(tree: Tree, pos: torch.Tensor, mass: torch.Tensor | None = None, stream=None) -> Tree:
    code = lib().tb_moments(tree._p, _ptr(pos), _ptr(mass), _stream(stream))
    _check(code, "tb_moments")
    return tree


def build_batched(pos: torch.Tensor, mass: torch.Tensor | None, set_offsets: torch.Tensor,
                  n_crit: int = 16, mom_mode: int = MOM_FP32_COMP, cell_capacity: int = 0,
                  radix_bits: int = 0, batch_threads: int = 0, tree: Tree | None = None,
                  n_total: int | None = None, stream=None, key_order: int = KEYS_MORTON,
                  one_launch: bool = False, root_pow2: bool = False) -> Tree:
    """tb_build_batched: set s holds pos[set_offsets[s]:set_offsets[s+1]];
    one_launch (with cell_capacity > 0) runs it as one cooperative launch."""
    if set_offsets.dtype != torch.int64 or not set_offsets.is_cuda:
        raise ValueError("set_offsets must be an int64 CUDA tensor")
    t = tree if tree is not None else Tree()
    if not batch_threads:
        from . import autotune
        batch_threads = autotune.cached_batched(set_offsets.shape[0] - 1,
                                                pos.shape[0] if n_total is None else n_total) or 0
    p = _params(n_crit, mom_mode, cell_capacity, 0, radix_bits, batch_threads)
    p.key_order = int(key_order)
    p.batch_one_launch = int(bool(one_launch))
    p.root_pow2 = int(bool(root_pow2))
    n_total = pos.shape[0] if n_total is None else n_total
    code = lib().tb_build_batched(_ptr(pos), _ptr(mass), _ptr(set_offsets),
                                  set_offsets.shape[0] - 1, int(n_total), C.byref(p),
                                  _stream(stream), C.byref(t._p))
    _check(code, "tb_build_batched")
    return t


def walk(tree: Tree, theta: float, eps: float, n_group: int = 32, use_quad: bool = True,
         out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """tb_walk: accelerations [n, 3] FP32 (original particle order) from the
    tree; its moments must be current."""
    n = tree.n
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    code = lib().tb_walk(tree._p, float(theta), float(eps), int(n_group), int(bool(use_quad)),
                         _ptr(out), _stream(stream))
    _check(code, "tb_walk")
    return out


def reorder(tree: Tree, src: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """tb_reorder: out[k] = src[perm[k]] for a per-particle CUDA tensor
    (first dimension n_particles, contiguous, rows a multiple of 4 bytes)."""
    if not src.is_cuda or not src.is_contiguous():
        raise ValueError("src must be a contiguous CUDA tensor")
    if out is None:
        out = torch.empty_like(src)
    n = src.shape[0]
    row_bytes = src.numel() * src.element_size() // max(1, n)
    code = lib().tb_reorder(tree._p, _ptr(src), _ptr(out), int(row_bytes), _stream(stream))
    _check(code, "tb_reorder")
    return out


NOALLOC_MAX_N = 524288


def keys_sorted_noalloc(pos: torch.Tensor, pkey_out: torch.Tensor, perm_out: torch.Tensor,
                        stream=None):
    """tb_keys_sorted_noalloc: keys and stable sort into caller-owned outputs
    (uint64 [n], int32 [n]) with no device allocation; returns (status, root
    [lo x, lo y, lo z, side])."""
    root = (C.c_double * 4)()
    code = lib().tb_keys_sorted_noalloc(_ptr(pos), pos.shape[0], _ptr(pkey_out), _ptr(perm_out),
                                        root, _stream(stream))
    return int(code), [float(v) for v in root]


def selftest_wait(spin_limit: int, stream=None) -> int:
    return int(lib().tb_selftest_wait(int(spin_limit), _stream(stream)))


def set_wait_limit(polls: int) -> int:
    """tb_set_wait_limit: polls after which a radix-pass look-back wait gives
    up (0 restores the default)."""
    return int(lib().tb_set_wait_limit(int(polls)))


def walk_counts(tree: Tree, stream=None):
    """tb_walk_counts: (target-cell, target-particle) interactions of the
    tree's last walk."""
    a, b = C.c_int64(), C.c_int64()
    _check(lib().tb_walk_counts(tree._p, _stream(stream), C.byref(a), C.byref(b)),
           "tb_walk_counts")
    return int(a.value), int(b.value)
