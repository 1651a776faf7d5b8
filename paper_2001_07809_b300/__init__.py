"""B300-native depth-based selective blurring (arXiv 2001.07809, Section III).

A thin ctypes binding over the C ABI in ``include/sb.h`` (``libsb.so``,
built in-tree for sm_103a by ``build.py``).  The functions keep the C names
and only marshal arguments: torch tensors supply device memory and streams,
every step of the method runs in the library's CUDA kernels.  There is no
CPU fallback: if the library cannot be loaded, importing this package fails.
With ``SB_LIBRARY=checks`` in the environment the bounds-checked build
(``libsb_checks.so``, see ``sb_check_probe`` in include/sb.h) is loaded
instead.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

from . import build as _build

__all__ = [
    "SbError", "Context", "Pair", "sb_default_params", "make_params", "sb_create", "sb_destroy",
    "sb_rgb_to_lightness", "sb_kmeans_segment", "sb_refine_boundaries", "sb_boundary_sad",
    "sb_reconstruct_disparity", "sb_selective_blur", "sb_run", "sb_synchronize", "sb_launch_count",
    "sb_lr_consistency", "sb_autotune", "sb_set_blur_form", "sb_set_union_limit", "sb_checks_built", "sb_check_probe", "sb_set_host_chunk", "sb_host_io_chunks", "SB_BLUR_AUTO", "SB_BLUR_STRIP", "SB_BLUR_TILES_64",
    "SB_BLUR_TILES_112", "SB_PEEK_SNAPSHOT", "SB_PEEK_INPLACE", "SB_VIEW_LEFT", "SB_VIEW_RIGHT",
    "SB_RUN_PLAIN", "SB_RUN_BATCHED", "SB_RUN_GRAPH", "SB_RUN_HOST_IO", "SB_SAD_AUTO", "SB_SAD_DIRECT",
    "SB_SAD_BOXSUM", "SB_MORPH_FILL_REMOVE", "SB_MORPH_OPEN_CLOSE", "UNDETERMINED", "library_path",
]

SB_OK, SB_ERR_INVALID_ARG, SB_ERR_CUDA, SB_ERR_OOM, SB_ERR_TIMEOUT, SB_ERR_UNSUPPORTED, SB_ERR_CHECK = range(7)
SB_MORPH_FILL_REMOVE, SB_MORPH_OPEN_CLOSE = 0, 1
SB_SAD_AUTO, SB_SAD_DIRECT, SB_SAD_BOXSUM = 0, 1, 2
SB_PEEK_SNAPSHOT, SB_PEEK_INPLACE = 0, 1
SB_VIEW_LEFT, SB_VIEW_RIGHT = 0, 1
SB_RUN_PLAIN, SB_RUN_BATCHED, SB_RUN_GRAPH, SB_RUN_HOST_IO = 0, 1, 2, 4
SB_BLUR_AUTO, SB_BLUR_STRIP, SB_BLUR_TILES_64, SB_BLUR_TILES_112 = 0, 32, 64, 112
SB_AUTOTUNE_CANDIDATES = 7
SB_MAX_RANGES = 8
UNDETERMINED = 0xFFFF
STAGES = ("lightness", "kmeans", "refine", "cca", "sad", "sad_rest", "recon", "blur")
_STATUS = {1: "invalid argument", 2: "CUDA error", 3: "out of memory", 4: "timeout", 5: "unsupported"}


class SbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, "status %d" % status), msg))
        self.status = status


class sb_range(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int32), ("hi", ctypes.c_int32)]


class sb_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("max_disp", ctypes.c_int32), ("block", ctypes.c_int32),
                ("disp_threshold", ctypes.c_int32), ("morph_mode", ctypes.c_int32),
                ("kmeans_max_iter", ctypes.c_int32), ("cc_remove_fraction", ctypes.c_double),
                ("sigma", ctypes.c_float), ("n_ranges", ctypes.c_int32), ("ranges", sb_range * SB_MAX_RANGES),
                ("sad_variant", ctypes.c_int32), ("peek_mode", ctypes.c_int32), ("view", ctypes.c_int32)]


class sb_pair(ctypes.Structure):
    _fields_ = [("left_rgb", ctypes.c_void_p), ("right_rgb", ctypes.c_void_p), ("w", ctypes.c_int32),
                ("h", ctypes.c_int32), ("p", sb_params), ("out_rgb", ctypes.c_void_p), ("out_disp", ctypes.c_void_p)]


def _variant() -> str:
    v = os.environ.get("SB_LIBRARY", "")
    if v not in ("", "checks"):
        raise ImportError("SB_LIBRARY must be unset or 'checks', not %r" % v)
    return v


def library_path() -> str:
    return _build.LIB_CHECKS if _variant() == "checks" else _build.LIB


def _load():
    checks = _variant() == "checks"
    path = library_path()
    if _build.needs_build(checks):
        try:
            _build.build(checks=checks)
        except Exception as e:  # no toolkit: fail loudly, there is no fallback
            if not os.path.exists(path):
                raise ImportError("%s is missing and could not be built: %s" % (os.path.basename(path), e)) from e
    lib = ctypes.CDLL(path)
    V, I32, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32
    sig = {
        "sb_default_params": ([ctypes.POINTER(sb_params)], None),
        "sb_create": ([ctypes.c_int, ctypes.c_size_t, V, ctypes.POINTER(V)], ctypes.c_int),
        "sb_destroy": ([V], None),
        "sb_set_stream": ([V, V], ctypes.c_int),
        "sb_last_error": ([V], ctypes.c_char_p),
        "sb_synchronize": ([V], ctypes.c_int),
        "sb_workspace_bytes": ([V], ctypes.c_size_t),
        "sb_launch_count": ([V], ctypes.c_uint64),
        "sb_rgb_to_lightness": ([V, V, I32, I32, V, V], ctypes.c_int),
        "sb_kmeans_segment": ([V, V, I32, I32, I32, I32, V, V, V, V], ctypes.c_int),
        "sb_refine_boundaries": ([V, V, I32, I32, I32, ctypes.c_double, V, V, V], ctypes.c_int),
        "sb_boundary_sad": ([V, V, V, V, I32, I32, I32, I32, I32, V, V], ctypes.c_int),
        "sb_reconstruct_disparity": ([V, V, I32, I32, I32, I32, I32, I32, V], ctypes.c_int),
        "sb_lr_consistency": ([V, V, V, I32, I32, I32, V, V], ctypes.c_int),
        "sb_autotune": ([V, V, I32, ctypes.c_uint32, V, V, V], ctypes.c_int),
        "sb_set_blur_form": ([V, I32], ctypes.c_int),
        "sb_set_union_limit": ([V, I32], ctypes.c_int),
        "sb_checks_built": ([], ctypes.c_int32),
        "sb_check_probe": ([V, I32], ctypes.c_int),
        "sb_set_host_chunk": ([V, ctypes.c_size_t, ctypes.c_size_t], ctypes.c_int),
        "sb_host_io_chunks": ([V], ctypes.c_int32),
        "sb_selective_blur": ([V, V, V, I32, I32, V, I32, ctypes.c_float, V], ctypes.c_int),
        "sb_run": ([V, ctypes.POINTER(sb_pair), I32, U32], ctypes.c_int),
        "sb_profile_enable": ([V, ctypes.c_int], ctypes.c_int),
        "sb_profile_read": ([V, ctypes.POINTER(ctypes.c_float), I32], I32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def _ptr(t) -> Optional[int]:
    """Device (or host) address of a tensor, None for None."""
    if t is None:
        return None
    return int(t.data_ptr())


def _check(ctx, status: int):
    if status != SB_OK:
        msg = _lib.sb_last_error(ctx.handle if ctx is not None else None)
        raise SbError(status, (msg or b"").decode(errors="replace"))


def sb_default_params() -> sb_params:
    p = sb_params()
    _lib.sb_default_params(ctypes.byref(p))
    return p


def make_params(k=10, max_disp=64, block=9, disp_threshold=1, morph_mode=SB_MORPH_FILL_REMOVE,
                kmeans_max_iter=100, cc_remove_fraction=0.04, sigma=3.0,
                ranges: Sequence[Tuple[int, int]] = (), sad_variant=SB_SAD_AUTO,
                peek_mode=SB_PEEK_SNAPSHOT, view=SB_VIEW_LEFT) -> sb_params:
    p = sb_default_params()
    p.k, p.max_disp, p.block, p.disp_threshold = k, max_disp, block, disp_threshold
    p.morph_mode, p.kmeans_max_iter, p.cc_remove_fraction, p.sigma = morph_mode, kmeans_max_iter, cc_remove_fraction, sigma
    if len(ranges) > SB_MAX_RANGES:
        raise ValueError("at most %d ranges" % SB_MAX_RANGES)
    p.n_ranges = len(ranges)
    for i, (lo, hi) in enumerate(ranges):
        p.ranges[i] = sb_range(int(lo), int(hi))
    p.sad_variant = sad_variant
    p.peek_mode = peek_mode
    p.view = view
    return p


class Context:
    """An sb_context on one device; work is queued on ``stream`` (a
    torch.cuda.Stream, a raw cudaStream_t int, or None for torch's current
    stream at creation)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device)
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        h = ctypes.c_void_p()
        st = _lib.sb_create(int(device), int(mem_budget_bytes), ctypes.c_void_p(raw), ctypes.byref(h))
        if st != SB_OK:
            raise SbError(st, "sb_create(device=%d) failed" % device)
        self.handle = h
        self.device = device

    def set_stream(self, stream):
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(self, _lib.sb_set_stream(self.handle, ctypes.c_void_p(raw)))

    def synchronize(self):
        _check(self, _lib.sb_synchronize(self.handle))

    def set_host_chunk(self, first_bytes: int, max_bytes: int):
        """Input bytes of the first and the largest chunk of host-buffer runs ((0, 0): defaults)."""
        _check(self, _lib.sb_set_host_chunk(self.handle, int(first_bytes), int(max_bytes)))

    def host_io_chunks(self) -> int:
        return int(_lib.sb_host_io_chunks(self.handle))

    def set_union_limit(self, limit: int):
        """Bound of the connected-components union-find (0: the default)."""
        _check(self, _lib.sb_set_union_limit(self.handle, int(limit)))

    def check_probe(self, trip: bool):
        """Enqueue the bounds-check probe (bounds-checked library only)."""
        _check(self, _lib.sb_check_probe(self.handle, 1 if trip else 0))

    def workspace_bytes(self) -> int:
        return int(_lib.sb_workspace_bytes(self.handle))

    def launch_count(self) -> int:
        return int(_lib.sb_launch_count(self.handle))

    def profile_enable(self, on: bool = True):
        _check(self, _lib.sb_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self):
        """Milliseconds per stage of the last run (see STAGES), or None."""
        buf = (ctypes.c_float * 8)()
        n = _lib.sb_profile_read(self.handle, buf, 8)
        return None if n < 0 else [float(buf[i]) for i in range(n)]

    def close(self):
        if getattr(self, "handle", None):
            _lib.sb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def sb_create(device: int = 0, mem_budget_bytes: int = 0, stream=None) -> Context:
    return Context(device, mem_budget_bytes, stream)


def sb_destroy(ctx: Context):
    ctx.close()


def sb_synchronize(ctx: Context):
    ctx.synchronize()


def sb_launch_count(ctx: Context) -> int:
    return ctx.launch_count()


def _hw(t):
    return int(t.shape[0]), int(t.shape[1])


def sb_rgb_to_lightness(ctx: Context, rgb, L, hist=None):
    h, w = _hw(rgb)
    _check(ctx, _lib.sb_rgb_to_lightness(ctx.handle, _ptr(rgb), w, h, _ptr(L), _ptr(hist)))


def sb_kmeans_segment(ctx: Context, L_left, k: int, max_iter: int = 100, labels=None, centroids=None,
                      bin2cluster=None, iters=None):
    h, w = _hw(L_left)
    _check(ctx, _lib.sb_kmeans_segment(ctx.handle, _ptr(L_left), w, h, k, max_iter, _ptr(labels), _ptr(centroids),
                                       _ptr(bin2cluster), _ptr(iters)))


def sb_refine_boundaries(ctx: Context, labels, boundary, morph_mode: int = SB_MORPH_FILL_REMOVE,
                         cc_remove_fraction: float = 0.04, refined=None, cc_labels=None):
    h, w = _hw(labels)
    _check(ctx, _lib.sb_refine_boundaries(ctx.handle, _ptr(labels), w, h, morph_mode, float(cc_remove_fraction),
                                          _ptr(boundary), _ptr(refined), _ptr(cc_labels)))


def sb_boundary_sad(ctx: Context, L_left, L_right, boundary, max_disp: int, block: int, disp, cost=None,
                    variant: int = SB_SAD_AUTO):
    h, w = _hw(L_left)
    _check(ctx, _lib.sb_boundary_sad(ctx.handle, _ptr(L_left), _ptr(L_right), _ptr(boundary), w, h, max_disp, block,
                                     variant, _ptr(disp), _ptr(cost)))


def sb_reconstruct_disparity(ctx: Context, disp, max_disp: int, block: int, disp_threshold: int, filled=None,
                             peek_mode: int = 0):
    h, w = _hw(disp)
    _check(ctx, _lib.sb_reconstruct_disparity(ctx.handle, _ptr(disp), w, h, max_disp, block, disp_threshold,
                                              peek_mode, _ptr(filled)))


def sb_lr_consistency(ctx: Context, disp_left, disp_right, ok, tol: int = 1, count=None):
    """Left-right consistency of a left-view and a right-view disparity map
    (device uint16/int16 [h, w]); ok: device uint8 [h, w]; count: None or a
    device int64 tensor of one element."""
    h, w = _hw(disp_left)
    _check(ctx, _lib.sb_lr_consistency(ctx.handle, _ptr(disp_left), _ptr(disp_right), w, h, tol, _ptr(ok),
                                       _ptr(count)))


def sb_selective_blur(ctx: Context, rgb, disp, ranges: Sequence[Tuple[int, int]], sigma: float, out_rgb):
    h, w = _hw(disp)
    arr = (sb_range * max(1, len(ranges)))(*[sb_range(int(a), int(b)) for a, b in ranges])
    _check(ctx, _lib.sb_selective_blur(ctx.handle, _ptr(rgb), _ptr(disp), w, h, arr if ranges else None, len(ranges),
                                       float(sigma), _ptr(out_rgb)))


class Pair:
    """One stereo pair for sb_run: tensors (device, or pinned host with
    SB_RUN_HOST_IO) of shape [h, w, 3] uint8, outputs out_rgb [h, w, 3] uint8
    and optionally out_disp [h, w] uint16 (torch.uint16) or int16 storage."""

    def __init__(self, left_rgb, right_rgb, params: sb_params, out_rgb, out_disp=None):
        self.left_rgb, self.right_rgb, self.params = left_rgb, right_rgb, params
        self.out_rgb, self.out_disp = out_rgb, out_disp


def _pairs_array(pairs: List[Pair]):
    arr = (sb_pair * len(pairs))()
    for i, q in enumerate(pairs):
        h, w = _hw(q.left_rgb)
        arr[i] = sb_pair(_ptr(q.left_rgb), _ptr(q.right_rgb), w, h, q.params, _ptr(q.out_rgb), _ptr(q.out_disp))
    return arr


def sb_autotune(ctx: Context, pairs: List[Pair], flags: int = SB_RUN_PLAIN):
    """Times the candidate box-sum work splits and blur forms on these pairs
    (running them), keeps the fastest for their shape on this context;
    -> (work items, blur form, [ms per candidate])."""
    arr = _pairs_array(pairs)
    ms = (ctypes.c_float * SB_AUTOTUNE_CANDIDATES)()
    items, rows = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(ctx, _lib.sb_autotune(ctx.handle, arr, len(pairs), flags, ms, ctypes.byref(items), ctypes.byref(rows)))
    return int(items.value), int(rows.value), [float(v) for v in ms]


def sb_set_host_chunk(ctx: Context, first_bytes: int, max_bytes: int):
    ctx.set_host_chunk(first_bytes, max_bytes)


def sb_host_io_chunks(ctx: Context) -> int:
    return ctx.host_io_chunks()


def sb_set_union_limit(ctx: Context, limit: int):
    ctx.set_union_limit(limit)


def sb_checks_built() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return bool(_lib.sb_checks_built())


def sb_check_probe(ctx: Context, trip: bool):
    ctx.check_probe(trip)


def sb_set_blur_form(ctx: Context, form: int):
    """Blur kernel form for later calls on this context (SB_BLUR_*; 0 = the
    tuned form, else tiles of 112 rows)."""
    _check(ctx, _lib.sb_set_blur_form(ctx.handle, int(form)))


def sb_run(ctx: Context, pairs: List[Pair], flags: int = SB_RUN_PLAIN):
    arr = _pairs_array(pairs)
    _check(ctx, _lib.sb_run(ctx.handle, arr, len(pairs), int(flags)))
