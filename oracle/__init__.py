"""ORACLE -- test infrastructure only.

A plain single-threaded CPU restatement of the selective-blurring pipeline of
Mukherjee & Guddeti (arXiv 2001.07809, Section III), written from the paper
in ``sb_oracle.c`` (C, FP64) and driven from here with numpy arrays.  Only
``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import it; the CUDA library never does, and it never loads the CUDA
library.

Stages (each cites the paper section it follows; readings of silent points
are stated in ``sb_oracle.c``):

* ``rgb_to_lightness``      Colour space conversion (Section III, IV)
* ``kmeans_hist``           256-bin histogram K-means (Section III)
* ``boundary``              8-neighbour segment boundary (Section III)
* ``morph_fill`` / ``morph_remove`` / ``morph_open_close``   (Section III)
* ``cca`` / ``cc_filter``   connected components, 4 % removal (Section III)
* ``anchor_mask`` / ``boundary_sad``  SAD at boundary pixels (Section III)
* ``recon_fill``            Algorithm 1
* ``recon_peek``            Algorithm 2 (estimates from the map after Algorithm 1)
* ``recon_peek_inplace``    Algorithm 2, in-place top-down reading
* ``selective_blur``        Eq. 1 and Eq. 2
* ``run``                   the whole pipeline in the paper's order
* ``disp_at_points``        final disparity at chosen pixels, evaluated from
  the same definitions but only for the anchors those pixels depend on, for
  checks of full-size images whose exhaustive SAD would take minutes

Parity status: every function is pinned in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
UNDET = 0xFFFF
_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u16p = ctypes.POINTER(ctypes.c_uint16)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile sb_oracle.c (gcc -O2, no FP contraction, no fast math)."""
    src = os.path.join(_HERE, "sb_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        V, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        sig = {
            "or_lightness_of": ([ctypes.c_uint8] * 3, ctypes.c_uint8),
            "or_rgb_to_lightness": ([V, I64, V], None),
            "or_histogram": ([V, I64, V], None),
            "or_kmeans_hist": ([V, I, I, V, V], I),
            "or_label_pixels": ([V, I64, V, V], None),
            "or_boundary": ([V, I, I, V], None),
            "or_morph_fill": ([V, I, I, V], None),
            "or_morph_remove": ([V, I, I, V], None),
            "or_morph_open_close": ([V, I, I, V], None),
            "or_cca": ([V, I, I, V], I64),
            "or_cc_filter": ([V, V, I, I, ctypes.c_double, V], I64),
            "or_anchor_mask": ([V, I, I, I, I, V], None),
            "or_sad_cost": ([V, V, I, I, I, I, I], ctypes.c_uint32),
            "or_sad_argmin": ([V, V, I, I, I, I, I, V], I),
            "or_boundary_sad": ([V, V, V, I, I, I, I, V, V], None),
            "or_recon_fill": ([V, V, I, I], None),
            "or_recon_peek": ([V, I, I, I, I, I, V], None),
            "or_recon_peek_inplace": ([V, I, I, I, I, I, V], None),
            "or_sad_argmin_right": ([V, V, I, I, I, I, I, V], ctypes.c_int),
            "or_lr_consistency": ([V, V, I, I, I, V], ctypes.c_int64),
            "or_blur_radius": ([ctypes.c_float], I),
            "or_selective_blur": ([V, V, I, I, V, I, ctypes.c_float, V], None),
            "or_blur_at": ([V, I, I, I, I, ctypes.c_float, V], None),
            "or_gauss_kernel": ([ctypes.c_float, V, I], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# --------------------------------------------------------------------- stages
def rgb_to_lightness(rgb: np.ndarray) -> np.ndarray:
    rgb = np.ascontiguousarray(rgb, np.uint8)
    h, w = rgb.shape[:2]
    L = np.empty((h, w), np.uint8)
    lib().or_rgb_to_lightness(_p(rgb), h * w, _p(L))
    return L


def lightness_of(r: int, g: int, b: int) -> int:
    return int(lib().or_lightness_of(r, g, b))


def histogram(L: np.ndarray) -> np.ndarray:
    L = np.ascontiguousarray(L, np.uint8)
    hist = np.empty(256, np.uint32)
    lib().or_histogram(_p(L), L.size, _p(hist))
    return hist


def kmeans_hist(hist: np.ndarray, k: int, max_iter: int = 100):
    """-> (centroids float64[k], bin2cluster uint8[256], iterations)."""
    hist = np.ascontiguousarray(hist, np.uint32)
    c = np.empty(k, np.float64)
    lut = np.empty(256, np.uint8)
    it = lib().or_kmeans_hist(_p(hist), k, max_iter, _p(c), _p(lut))
    return c, lut, it


def label_pixels(L: np.ndarray, lut: np.ndarray) -> np.ndarray:
    L = np.ascontiguousarray(L, np.uint8)
    out = np.empty_like(L)
    lib().or_label_pixels(_p(L), L.size, _p(np.ascontiguousarray(lut, np.uint8)), _p(out))
    return out


def _map2(fname: str, a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, np.uint8)
    h, w = a.shape
    out = np.empty_like(a)
    getattr(lib(), fname)(_p(a), w, h, _p(out))
    return out


def boundary(labels: np.ndarray) -> np.ndarray:
    return _map2("or_boundary", labels)


def morph_fill(b: np.ndarray) -> np.ndarray:
    return _map2("or_morph_fill", b)


def morph_remove(b: np.ndarray) -> np.ndarray:
    return _map2("or_morph_remove", b)


def morph_open_close(b: np.ndarray) -> np.ndarray:
    return _map2("or_morph_open_close", b)


def refine(b: np.ndarray, morph_mode: int = 0) -> np.ndarray:
    """Fill then Remove (mode 0, the paper's order) or open/close (mode 1)."""
    return morph_remove(morph_fill(b)) if morph_mode == 0 else morph_open_close(b)


def cca(b: np.ndarray) -> Tuple[np.ndarray, int]:
    b = np.ascontiguousarray(b, np.uint8)
    h, w = b.shape
    lab = np.empty((h, w), np.int32)
    n = lib().or_cca(_p(b), w, h, _p(lab))
    return lab, int(n)


def cc_filter(b: np.ndarray, lab: np.ndarray, frac: float = 0.04) -> np.ndarray:
    b = np.ascontiguousarray(b, np.uint8)
    lab = np.ascontiguousarray(lab, np.int32)
    h, w = b.shape
    out = np.empty_like(b)
    lib().or_cc_filter(_p(b), _p(lab), w, h, float(frac), _p(out))
    return out


def anchor_mask(b: np.ndarray, max_disp: int, block: int) -> np.ndarray:
    b = np.ascontiguousarray(b, np.uint8)
    h, w = b.shape
    out = np.empty_like(b)
    lib().or_anchor_mask(_p(b), w, h, max_disp, block, _p(out))
    return out


def sad_cost(Ll: np.ndarray, Lr: np.ndarray, x: int, y: int, d: int, block: int) -> int:
    w = Ll.shape[1]
    return int(lib().or_sad_cost(_p(Ll), _p(Lr), w, x, y, d, block))


def sad_argmin(Ll: np.ndarray, Lr: np.ndarray, x: int, y: int, max_disp: int, block: int) -> Tuple[int, int]:
    c = ctypes.c_uint32(0)
    w = Ll.shape[1]
    d = lib().or_sad_argmin(_p(Ll), _p(Lr), w, x, y, max_disp, block, ctypes.byref(c))
    return int(d), int(c.value)


def sad_argmin_right(Ll: np.ndarray, Lr: np.ndarray, x: int, y: int, max_disp: int, block: int) -> Tuple[int, int]:
    """Right-referenced SAD argmin at right-image pixel (x, y), written out directly."""
    Ll = np.ascontiguousarray(Ll, np.uint8)
    Lr = np.ascontiguousarray(Lr, np.uint8)
    c = ctypes.c_uint32(0)
    d = lib().or_sad_argmin_right(_p(Ll), _p(Lr), Ll.shape[1], x, y, max_disp, block, ctypes.byref(c))
    return int(d), int(c.value)


def lr_consistency(dL: np.ndarray, dR: np.ndarray, tol: int = 1):
    """-> (ok uint8 map, number of consistent pixels) of a left- and a right-referenced map."""
    dL = np.ascontiguousarray(dL, np.uint16)
    dR = np.ascontiguousarray(dR, np.uint16)
    h, w = dL.shape
    ok = np.empty((h, w), np.uint8)
    n = lib().or_lr_consistency(_p(dL), _p(dR), w, h, tol, _p(ok))
    return ok, int(n)


def boundary_sad(Ll, Lr, anchor, max_disp: int, block: int):
    """-> (disp uint16 with UNDET off the anchors, cost uint32 (0 off anchors))."""
    Ll = np.ascontiguousarray(Ll, np.uint8)
    Lr = np.ascontiguousarray(Lr, np.uint8)
    anchor = np.ascontiguousarray(anchor, np.uint8)
    h, w = Ll.shape
    disp = np.empty((h, w), np.uint16)
    cost = np.empty((h, w), np.uint32)
    lib().or_boundary_sad(_p(Ll), _p(Lr), _p(anchor), w, h, max_disp, block, _p(disp), _p(cost))
    return disp, cost


def recon_fill(disp: np.ndarray, anchor: np.ndarray) -> np.ndarray:
    out = np.array(disp, np.uint16, copy=True, order="C")
    anchor = np.ascontiguousarray(anchor, np.uint8)
    h, w = out.shape
    lib().or_recon_fill(_p(out), _p(anchor), w, h)
    return out


def recon_peek(det: np.ndarray, max_disp: int, block: int, threshold: int) -> np.ndarray:
    det = np.ascontiguousarray(det, np.uint16)
    h, w = det.shape
    out = np.empty_like(det)
    lib().or_recon_peek(_p(det), w, h, max_disp, block, threshold, _p(out))
    return out


def recon_peek_inplace(det: np.ndarray, max_disp: int, block: int, threshold: int) -> np.ndarray:
    """Algorithm 2, in-place top-down reading (estimates feed the pixel below)."""
    det = np.ascontiguousarray(det, np.uint16)
    h, w = det.shape
    out = np.empty_like(det)
    lib().or_recon_peek_inplace(_p(det), w, h, max_disp, block, threshold, _p(out))
    return out


def blur_radius(sigma: float) -> int:
    return int(lib().or_blur_radius(float(sigma)))


def gauss_kernel(sigma: float) -> np.ndarray:
    R = blur_radius(sigma)
    n = 2 * R + 1
    out = np.empty(n * n, np.float64)
    lib().or_gauss_kernel(float(sigma), _p(out), n * n)
    return out.reshape(n, n)


def _ranges_arr(ranges: Sequence[Tuple[int, int]]) -> np.ndarray:
    return np.ascontiguousarray(np.array(list(ranges), np.int32).reshape(-1, 2))


def selective_blur(rgb: np.ndarray, disp: np.ndarray, ranges, sigma: float) -> np.ndarray:
    rgb = np.ascontiguousarray(rgb, np.uint8)
    disp = np.ascontiguousarray(disp, np.uint16)
    h, w = disp.shape
    out = np.empty_like(rgb)
    rr = _ranges_arr(ranges)
    lib().or_selective_blur(_p(rgb), _p(disp), w, h, _p(rr) if rr.size else None, len(rr), float(sigma), _p(out))
    return out


def blur_at(rgb: np.ndarray, x: int, y: int, sigma: float) -> np.ndarray:
    rgb = np.ascontiguousarray(rgb, np.uint8)
    h, w = rgb.shape[:2]
    o = np.empty(3, np.uint8)
    lib().or_blur_at(_p(rgb), w, h, x, y, float(sigma), _p(o))
    return o


# ------------------------------------------------------------------ pipeline
@dataclasses.dataclass
class Result:
    L_left: np.ndarray
    L_right: np.ndarray
    hist: np.ndarray
    centroids: np.ndarray
    bin2cluster: np.ndarray
    kmeans_iters: int
    labels: np.ndarray
    boundary0: np.ndarray      # after detection
    refined: np.ndarray        # after Fill/Remove (or open/close)
    cc_labels: np.ndarray
    n_components: int
    filtered: np.ndarray       # after small-component removal
    anchor: np.ndarray
    disp_sparse: Optional[np.ndarray] = None
    cost: Optional[np.ndarray] = None
    disp_filled: Optional[np.ndarray] = None
    disp: Optional[np.ndarray] = None
    out_rgb: Optional[np.ndarray] = None


def run_front(left_rgb, right_rgb, p) -> Result:
    """Stages up to the anchor mask (all O(N) and cheap at any size)."""
    Ll = rgb_to_lightness(left_rgb)
    Lr = rgb_to_lightness(right_rgb)
    hist = histogram(Ll)
    c, lut, it = kmeans_hist(hist, p.k, p.kmeans_max_iter)
    labels = label_pixels(Ll, lut)
    b0 = boundary(labels)
    b1 = refine(b0, p.morph_mode)
    lab, ncomp = cca(b1)
    bf = cc_filter(b1, lab, p.cc_remove_fraction)
    anc = anchor_mask(bf, p.max_disp, p.block)
    return Result(Ll, Lr, hist, c, lut, it, labels, b0, b1, lab, ncomp, bf, anc)


def run(left_rgb, right_rgb, p, with_blur: bool = True) -> Result:
    """The whole pipeline of Section III in the paper's order.  With
    ``p.view == 1`` the right image is the reference: the method runs on the
    horizontally mirrored pair with the roles swapped (the mirrored right
    image matched against the mirrored left one, disparities still >= 0), and
    ``disp`` / ``out_rgb`` are mirrored back: the right image's disparity map
    and its selectively blurred copy.  The intermediate maps stay mirrored."""
    if getattr(p, "view", 0) == 1:
        left_m = np.ascontiguousarray(left_rgb[:, ::-1])
        right_m = np.ascontiguousarray(right_rgb[:, ::-1])
        res = _run_left(right_m, left_m, p, with_blur=False)
        res.disp = np.ascontiguousarray(res.disp[:, ::-1])
        if with_blur:
            res.out_rgb = selective_blur(right_rgb, res.disp, p.ranges, p.sigma)
        return res
    return _run_left(left_rgb, right_rgb, p, with_blur)


def _run_left(left_rgb, right_rgb, p, with_blur: bool = True) -> Result:
    res = run_front(left_rgb, right_rgb, p)
    res.disp_sparse, res.cost = boundary_sad(res.L_left, res.L_right, res.anchor, p.max_disp, p.block)
    res.disp_filled = recon_fill(res.disp_sparse, res.anchor)
    peek = recon_peek_inplace if getattr(p, "peek_mode", 0) == 1 else recon_peek
    res.disp = peek(res.disp_filled, p.max_disp, p.block, p.disp_threshold)
    if with_blur:
        res.out_rgb = selective_blur(left_rgb, res.disp, p.ranges, p.sigma)
    return res


def disp_at_points(front: Result, p, points: Iterable[Tuple[int, int]],
                   memo: Optional[Dict[Tuple[int, int], int]] = None) -> List[int]:
    """Final disparity at the given (x, y) pixels, from the same definitions
    as ``run`` but evaluating SAD only at the anchors each answer depends on.

    Algorithm 1 fills a non-anchor pixel exactly when the anchors just left
    and just right of it in its row (the consecutive pair that brackets it)
    have equal disparity; Algorithm 2 then needs, per column, the nearest
    pixel above and below that is an anchor or filled.  Both are evaluated
    lazily here with a memo of anchor disparities."""
    if getattr(p, "view", 0) != 0:
        raise NotImplementedError("disp_at_points evaluates the left view")
    if getattr(p, "peek_mode", 0) != 0:
        raise NotImplementedError("disp_at_points follows the Algorithm 2 reading that uses the map after "
                                  "Algorithm 1 (peek_mode 0)")
    Ll, Lr, anc = front.L_left, front.L_right, front.anchor
    h, w = anc.shape
    r = (p.block - 1) // 2
    x0, x1, y0, y1 = p.max_disp + r, w - 1 - r, r, h - 1 - r
    memo = {} if memo is None else memo
    rows: Dict[int, np.ndarray] = {}

    def anchors_of(y):
        if y not in rows:
            rows[y] = np.flatnonzero(anc[y])
        return rows[y]

    def sad(x, y):
        key = (x, y)
        if key not in memo:
            memo[key] = sad_argmin(Ll, Lr, x, y, p.max_disp, p.block)[0]
        return memo[key]

    def determined(x, y):
        """Value after Algorithm 1, or None when undetermined."""
        if anc[y, x]:
            return sad(x, y)
        a = anchors_of(y)
        i = int(np.searchsorted(a, x))
        if i == 0 or i >= len(a):
            return None
        dl, dr = sad(int(a[i - 1]), y), sad(int(a[i]), y)
        return dl if dl == dr else None

    out = []
    for (x, y) in points:
        if not (y0 <= y <= y1 and x0 <= x <= x1):
            out.append(0)
            continue
        v = determined(x, y)
        if v is None:
            a = c = None
            for yy in range(y - 1, y0 - 1, -1):
                a = determined(x, yy)
                if a is not None:
                    break
            for yy in range(y + 1, y1 + 1):
                c = determined(x, yy)
                if c is not None:
                    break
            if a is None and c is None:
                v = 0
            elif a is None:
                v = c
            elif c is None:
                v = a
            else:
                v = min(a, c) if abs(a - c) > p.disp_threshold else (a + c) // 2
        out.append(int(v))
    return out


def bad_pixel_percent(disp: np.ndarray, gt: np.ndarray, mask: np.ndarray, delta: float = 1.0) -> float:
    """Eq. 3: percentage of pixels (inside ``mask``) whose disparity error exceeds delta."""
    e = np.abs(disp.astype(np.float64) - gt.astype(np.float64)) > delta
    n = int(mask.sum())
    return 100.0 * float(e[mask].sum()) / max(n, 1)
