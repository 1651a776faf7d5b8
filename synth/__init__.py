"""Seeded synthetic rectified stereo pairs shaped like the paper's workloads.

The paper evaluates on Middlebury pairs and times a 4096x2304 stereo video
(Section IV); neither is available, so every input here is generated from a
seed.  This package is input generation only: it contains none of the
selective-blurring method's arithmetic and is imported by the tests and the
benchmark, never by the CUDA path or the oracle.

Scenes are lists of textured layers (fronto-parallel rectangles/ellipses and
slanted planes) rendered by ``synth.c`` with integer-only arithmetic, so the
bytes are identical on every host.  Scene parameters are drawn with a
splitmix64 sequence (pure Python integers).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import shutil
import subprocess
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_SO_GPU = os.path.join(_HERE, "libsynth_gpu.so")
_lib_handle = None
_gpu_handle = None

M64 = (1 << 64) - 1


def _stale(out, srcs):
    return not os.path.exists(out) or any(os.path.getmtime(out) < os.path.getmtime(s) for s in srcs)


def build(force: bool = False, gpu: bool = True) -> str:
    """Compile synth.c into libsynth.so (gcc, -O2, pthreads) and, when nvcc is
    available, synth_gpu.cu into libsynth_gpu.so (sm_103a)."""
    core = os.path.join(_HERE, "synth_core.h")
    src = os.path.join(_HERE, "synth.c")
    if force or _stale(_SO, [src, core]):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, src])
        os.replace(tmp, _SO)
    gsrc = os.path.join(_HERE, "synth_gpu.cu")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if gpu and os.path.exists(nvcc) and (force or _stale(_SO_GPU, [gsrc, core])):
        tmp = _SO_GPU + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC",
                               "-shared", "-cudart", "shared", "-o", tmp, gsrc])
        os.replace(tmp, _SO_GPU)
    return _SO


class _Layer(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "shape", "cx", "cy", "hw", "hh", "vx", "vy", "d0_q8", "gx_q16", "gy_q16",
        "dd_frame", "dmin", "dmax")] + [("tex_seed", ctypes.c_uint32)] + [
        (n, ctypes.c_int32) for n in ("mean", "contrast", "tint_r", "tint_g", "tint_b")]


class _Scene(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int32), ("h", ctypes.c_int32), ("n_layers", ctypes.c_int32),
                ("frame", ctypes.c_int32), ("noise_q8", ctypes.c_int32),
                ("gain_l_q10", ctypes.c_int32), ("gain_r_q10", ctypes.c_int32),
                ("noise_seed", ctypes.c_uint64), ("layers", ctypes.POINTER(_Layer))]


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.synth_render.argtypes = [ctypes.POINTER(_Scene), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int32]
        lib.synth_render.restype = ctypes.c_int
        lib.synth_splitmix64.argtypes = [ctypes.c_uint64]
        lib.synth_splitmix64.restype = ctypes.c_uint64
        _lib_handle = lib
    return _lib_handle


def splitmix64(z: int) -> int:
    """The splitmix64 finaliser (published definition), on Python integers."""
    z = (z + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


class Rng:
    """Sequential splitmix64 stream for drawing scene parameters."""

    def __init__(self, seed: int):
        self.s = (seed * 0x9E3779B97F4A7C15 + 0x1234567) & M64

    def u64(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & M64
        return splitmix64(self.s)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + self.u64() % (hi - lo + 1)

    def uniform_q(self, lo: float, hi: float, q: int) -> int:
        """Uniform value in [lo, hi] returned in fixed point with scale q."""
        a, b = int(round(lo * q)), int(round(hi * q))
        return self.randint(min(a, b), max(a, b))

    def choice(self, seq):
        return seq[self.u64() % len(seq)]


@dataclasses.dataclass
class Layer:
    shape: int
    cx: int
    cy: int
    hw: int
    hh: int
    d0_q8: int
    mean: int
    contrast: int
    tex_seed: int
    tint: Tuple[int, int, int] = (256, 256, 256)
    gx_q16: int = 0
    gy_q16: int = 0
    vx: int = 0
    vy: int = 0
    dd_frame: int = 0
    dmin: int = 0
    dmax: int = 0


@dataclasses.dataclass
class Scene:
    w: int
    h: int
    layers: List[Layer]
    noise_q8: int = 256
    gain_l_q10: int = 1024
    gain_r_q10: int = 1024
    noise_seed: int = 0

    def render(self, frame: int = 0, n_threads: Optional[int] = None, want_gt: bool = True):
        """Render (left_rgb, right_rgb, gt) for one frame.

        left_rgb/right_rgb: uint8 [h, w, 3]; gt: float32 [h, w] disparity of
        the left image (None unless want_gt)."""
        lib = _lib()
        sc, keep = _ctypes_scene(self, frame)
        left = np.empty((self.h, self.w, 3), np.uint8)
        right = np.empty((self.h, self.w, 3), np.uint8)
        gt = np.empty((self.h, self.w), np.float32) if want_gt else None
        if n_threads is None:
            n_threads = min(os.cpu_count() or 1, 64)
        rc = lib.synth_render(ctypes.byref(sc), left.ctypes.data, right.ctypes.data,
                              gt.ctypes.data if gt is not None else None, int(n_threads))
        if rc != 0:
            raise ValueError("synth_render rejected the scene")
        return left, right, gt


def _gpu_lib():
    global _gpu_handle
    if _gpu_handle is None:
        build()
        lib = ctypes.CDLL(_SO_GPU)
        lib.synth_render_device.argtypes = [ctypes.POINTER(_Scene), ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_render_device.restype = ctypes.c_int
        _gpu_handle = lib
    return _gpu_handle


def _ctypes_scene(scene: "Scene", frame: int):
    def cur_d(L: Layer) -> int:
        if L.dd_frame == 0:
            return L.d0_q8
        base = (L.d0_q8 + 128) >> 8
        v = base + L.dd_frame * frame
        lo, hi = L.dmin, L.dmax
        p = 2 * (hi - lo)
        m = (v - lo) % p
        return L.d0_q8 + ((lo + (m if m <= hi - lo else p - m)) - base) * 256
    order = sorted(range(len(scene.layers)),
                   key=lambda i: (0 if scene.layers[i].shape == 0 else 1, cur_d(scene.layers[i]), i))
    arr = (_Layer * len(order))()
    for k, i in enumerate(order):
        L = scene.layers[i]
        arr[k] = _Layer(L.shape, L.cx, L.cy, L.hw, L.hh, L.vx, L.vy, L.d0_q8, L.gx_q16, L.gy_q16,
                        L.dd_frame, L.dmin, L.dmax, L.tex_seed & 0xFFFFFFFF, L.mean, L.contrast,
                        L.tint[0], L.tint[1], L.tint[2])
    sc = _Scene(scene.w, scene.h, len(order), frame, scene.noise_q8, scene.gain_l_q10, scene.gain_r_q10,
                scene.noise_seed & M64, arr)
    return sc, arr


def render_device(scene: "Scene", frame: int, left, right, gt=None, stream=0):
    """Render a frame into device tensors (uint8 [h, w, 3] x2, float32 [h, w]
    or None) with the CUDA build; same bytes as Scene.render."""
    sc, keep = _ctypes_scene(scene, frame)
    rc = _gpu_lib().synth_render_device(ctypes.byref(sc), left.data_ptr(), right.data_ptr(),
                                        gt.data_ptr() if gt is not None else None, stream)
    if rc != 0:
        raise RuntimeError("synth_render_device failed with %d" % rc)


@dataclasses.dataclass
class Params:
    """The method's parameters for one pair (Section III, Table 3)."""
    k: int
    max_disp: int
    block: int
    sigma: float
    ranges: Sequence[Tuple[int, int]]       # disparity ranges of INTEREST (kept sharp)
    disp_threshold: int = 1
    morph_mode: int = 0                     # 0 Fill+Remove (paper), 1 open/close
    kmeans_max_iter: int = 100
    cc_remove_fraction: float = 0.04
    peek_mode: int = 0                      # Algorithm 2: 0 from the map after Algorithm 1, 1 in place
    view: int = 0                           # reference image: 0 left (paper's figures), 1 right


def _tint(r: Rng) -> Tuple[int, int, int]:
    return (r.randint(170, 256), r.randint(170, 256), r.randint(170, 256))


def _means(r: Rng, n: int) -> List[int]:
    """n distinct layer lightness means spread over [35, 220]."""
    base = [35 + (185 * i) // max(n - 1, 1) for i in range(n)]
    for i in range(n - 1, 0, -1):          # shuffle
        j = r.u64() % (i + 1)
        base[i], base[j] = base[j], base[i]
    return [b + r.randint(-6, 6) for b in base]


def scene_c1(seed: int = 0, contrast: int = 80) -> Scene:
    """320x240: background at disparity 2 plus four textured rectangles at
    disparities {6, 11, 16, 22}; noise sigma 1."""
    r = Rng(seed)
    w, h = 320, 240
    means = _means(r, 5)
    layers = [Layer(0, w // 2, h // 2, w, h, 2 * 256, means[0], contrast, r.u64() & 0xFFFFFFFF, _tint(r))]
    for i, d in enumerate((6, 11, 16, 22)):
        hw, hh = r.randint(24, 60), r.randint(18, 48)
        cx, cy = r.randint(40 + hw // 2, w - 10 - hw // 2), r.randint(10 + hh // 2, h - 10 - hh // 2)
        layers.append(Layer(1, cx, cy, hw, hh, d * 256, means[i + 1], contrast, r.u64() & 0xFFFFFFFF, _tint(r)))
    return Scene(w, h, layers, noise_q8=256, noise_seed=r.u64())


def _c2_style_layers(r: Rng, w: int, h: int, dmax: int, contrast: int, n_fronto: int = 5,
                     n_slanted: int = 3) -> List[Layer]:
    means = _means(r, n_fronto + n_slanted)
    layers: List[Layer] = []
    s = min(w, h)
    # background: a slanted full-frame plane at small disparity
    g = r.uniform_q(0.02, 0.08, 65536)
    gd = r.randint(0, 1)
    d_back = max(2.0, 0.12 * dmax)
    span = (w if gd == 0 else h) / 2
    g = min(g, int(65536 * 0.9 * d_back / span))
    layers.append(Layer(0, w // 2, h // 2, w, h, int(d_back * 256 + g * span / 256), means[0], contrast,
                        r.u64() & 0xFFFFFFFF, _tint(r), gx_q16=g if gd == 0 else 0, gy_q16=g if gd == 1 else 0))
    for i in range(n_slanted - 1):
        hw, hh = r.randint(s // 10, s // 4), r.randint(s // 10, s // 4)
        cx, cy = r.randint(hw, w - hw), r.randint(hh, h - hh)
        gx = r.uniform_q(0.02, 0.08, 65536) * (1 if r.randint(0, 1) else -1)
        gy = r.uniform_q(0.0, 0.04, 65536) * (1 if r.randint(0, 1) else -1)
        dspan = (abs(gx) * hw + abs(gy) * hh) / 65536
        lo, hi = 0.2 * dmax + dspan, 0.92 * dmax - dspan
        d0 = r.uniform_q(lo, max(lo, hi), 256)
        layers.append(Layer(1, cx, cy, hw, hh, d0, means[1 + i], contrast, r.u64() & 0xFFFFFFFF, _tint(r),
                            gx_q16=gx, gy_q16=gy))
    for i in range(n_fronto):
        hw, hh = r.randint(s // 16, s // 6), r.randint(s // 16, s // 6)
        cx, cy = r.randint(hw, w - hw), r.randint(hh, h - hh)
        d0 = r.randint(int(0.16 * dmax), int(0.94 * dmax)) * 256
        shape = 1 + r.randint(0, 1)
        layers.append(Layer(shape, cx, cy, hw, hh, d0, means[n_slanted + i], contrast,
                            r.u64() & 0xFFFFFFFF, _tint(r)))
    return layers


def scene_c2(seed: int = 1, contrast: int = 34) -> Scene:
    """1400x1100: 5 fronto-parallel rectangles/ellipses at disparities in
    [20, 120] and 3 slanted planes (gradients 0.02-0.08 px/px), noise sigma 2,
    per-image gain 0.95-1.05."""
    r = Rng(seed)
    w, h = 1400, 1100
    layers = _c2_style_layers(r, w, h, 128, contrast)
    return Scene(w, h, layers, noise_q8=512, gain_l_q10=r.uniform_q(0.95, 1.05, 1024),
                 gain_r_q10=r.uniform_q(0.95, 1.05, 1024), noise_seed=r.u64())


def scene_c3(seed: int = 2, contrast: int = 30) -> Scene:
    """4096x2304 video: 12 textured layers whose disparities drift +-1 px per
    frame within [8, 240] and that translate 0-4 px per frame; noise sigma 2.
    Render frame f with ``scene.render(frame=f)``."""
    r = Rng(seed)
    w, h = 4096, 2304
    means = _means(r, 12)
    layers = [Layer(0, w // 2, h // 2, w, h, 8 * 256 + r.randint(0, 8) * 256, means[0], contrast,
                    r.u64() & 0xFFFFFFFF, _tint(r), dd_frame=1, dmin=8, dmax=24,
                    vx=r.randint(-4, 4), vy=r.randint(-2, 2))]
    for i in range(11):
        hw, hh = r.randint(180, 700), r.randint(140, 520)
        cx, cy = r.randint(hw // 2, w - hw // 2), r.randint(hh // 2, h - hh // 2)
        d0 = r.randint(24, 240)
        layers.append(Layer(1 + r.randint(0, 1), cx, cy, hw, hh, d0 * 256, means[1 + i], contrast,
                            r.u64() & 0xFFFFFFFF, _tint(r), vx=r.randint(-4, 4), vy=r.randint(-4, 4),
                            dd_frame=(1 if r.randint(0, 1) else -1), dmin=8, dmax=240))
    return Scene(w, h, layers, noise_q8=512, noise_seed=r.u64())


C4_SIZES = ((640, 480), (1920, 1080), (2560, 1440), (4096, 2304))


def scene_c4(seed: int) -> Tuple[Scene, Params]:
    """One pair of the uneven batch: resolution, max disparity, block and K
    drawn from the mixed sets; C2-style layered + slanted scene whose texture
    contrast sets the boundary density; own interest range and sigma."""
    r = Rng(seed)
    w, h = r.choice(C4_SIZES)
    D = r.choice((64, 128, 256))
    B = r.choice((9, 15, 25, 41))
    K = r.choice((4, 6, 8))
    contrast = r.randint(14, 60)
    layers = _c2_style_layers(r, w, h, D, contrast)
    sc = Scene(w, h, layers, noise_q8=512, gain_l_q10=r.uniform_q(0.95, 1.05, 1024),
               gain_r_q10=r.uniform_q(0.95, 1.05, 1024), noise_seed=r.u64())
    lo = r.randint(0, D // 2)
    hi = r.randint(lo + D // 8, D)
    sigma = r.uniform_q(2.0, 8.0, 8) / 8.0
    return sc, Params(k=K, max_disp=D, block=B, sigma=sigma, ranges=[(lo, hi)])


# The method parameters of each workload (the interest ranges are the
# complement of the blurred disparities named for each workload).
PARAMS_C1 = Params(k=4, max_disp=32, block=15, sigma=3.0, ranges=[(9, 32)])
PARAMS_C2 = Params(k=6, max_disp=128, block=31, sigma=5.0, ranges=[(40, 128)])
PARAMS_C3 = Params(k=8, max_disp=256, block=41, sigma=8.0, ranges=[(120, 256)])


def workload(name: str, index: int = 0):
    """(scene, params, frame) for a named workload item.

    c1, c2: the single pairs; c3: frame ``index`` of the video; c4: pair
    ``index`` (seed 100+index) of the uneven batch; c5: request ``index`` of
    the serving stream (seed 7), drawn like c4."""
    if name == "c1":
        return scene_c1(), PARAMS_C1, 0
    if name == "c2":
        return scene_c2(), PARAMS_C2, 0
    if name == "c3":
        return scene_c3(), PARAMS_C3, index
    if name == "c4":
        sc, p = scene_c4(100 + index)
        return sc, p, 0
    if name == "c5":
        sc, p = scene_c4(splitmix64(7 * 1000003 + index) & 0xFFFFFFFF)
        return sc, p, 0
    raise KeyError(name)


def poisson_arrivals(n: int, rate: float, seed: int = 7) -> np.ndarray:
    """Arrival times (s) of n requests with exponential gaps at ``rate``/s,
    drawn from splitmix64 uniforms (inverse-CDF)."""
    r = Rng(seed * 7919 + int(rate * 1000))
    t, out = 0.0, np.empty(n)
    for i in range(n):
        u = (r.u64() >> 11) * (1.0 / (1 << 53))
        t += -np.log1p(-u) / rate
        out[i] = t
    return out
