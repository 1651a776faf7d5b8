"""Helpers for the GPU tests: numpy <-> device tensors and one call per stage
of the C ABI through the Python binding."""
import numpy as np
import torch

import paper_2001_07809_b300 as sb


def dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda()
    return torch.from_numpy(a).cuda()


def host(t: torch.Tensor, dtype=None) -> np.ndarray:
    a = t.detach().cpu().numpy()
    if dtype is not None and a.dtype != dtype:
        a = a.view(dtype)
    return a


def empty(shape, dtype) -> torch.Tensor:
    tdt = {np.uint8: torch.uint8, np.uint16: torch.int16, np.uint32: torch.int32, np.int32: torch.int32,
           np.float64: torch.float64}[dtype]
    return torch.empty(shape, dtype=tdt, device="cuda")


def lightness(ctx, rgb: np.ndarray, want_hist=True):
    h, w = rgb.shape[:2]
    L = empty((h, w), np.uint8)
    hist = empty((256,), np.uint32) if want_hist else None
    sb.sb_rgb_to_lightness(ctx, dev(rgb), L, hist)
    return host(L), (host(hist, np.uint32) if want_hist else None)


def kmeans(ctx, L: np.ndarray, k: int, max_iter=100):
    h, w = L.shape
    labels = empty((h, w), np.uint8)
    cent = empty((k,), np.float64)
    lut = empty((256,), np.uint8)
    it = empty((1,), np.int32)
    sb.sb_kmeans_segment(ctx, dev(L), k, max_iter, labels, cent, lut, it)
    return host(cent), host(lut), int(host(it)[0]), host(labels)


def refine(ctx, labels: np.ndarray, mode=0, frac=0.04):
    h, w = labels.shape
    bnd = empty((h, w), np.uint8)
    ref = empty((h, w), np.uint8)
    lab = empty((h, w), np.int32)
    sb.sb_refine_boundaries(ctx, dev(labels), bnd, mode, frac, ref, lab)
    return host(ref), host(lab), host(bnd)


def sad(ctx, Ll, Lr, bmap, D, B, variant):
    h, w = Ll.shape
    disp = empty((h, w), np.uint16)
    cost = empty((h, w), np.uint32)
    sb.sb_boundary_sad(ctx, dev(Ll), dev(Lr), dev(bmap), D, B, disp, cost, variant)
    return host(disp, np.uint16), host(cost, np.uint32)


def recon(ctx, sparse: np.ndarray, D, B, T, peek_mode=0):
    h, w = sparse.shape
    d = dev(sparse.astype(np.uint16))
    filled = empty((h, w), np.uint16)
    sb.sb_reconstruct_disparity(ctx, d, D, B, T, filled, peek_mode)
    return host(filled, np.uint16), host(d, np.uint16)


def blur(ctx, rgb, disp, ranges, sigma):
    out = torch.empty(rgb.shape, dtype=torch.uint8, device="cuda")
    sb.sb_selective_blur(ctx, dev(rgb), dev(disp.astype(np.uint16)), ranges, sigma, out)
    return host(out)


def params_of(p, sad_variant=sb.SB_SAD_AUTO):
    return sb.make_params(k=p.k, max_disp=p.max_disp, block=p.block, disp_threshold=p.disp_threshold,
                          morph_mode=p.morph_mode, kmeans_max_iter=p.kmeans_max_iter,
                          cc_remove_fraction=p.cc_remove_fraction, sigma=p.sigma, ranges=p.ranges,
                          sad_variant=sad_variant, peek_mode=getattr(p, "peek_mode", 0),
                          view=getattr(p, "view", 0))


def run_pairs(ctx, items, flags, sad_variant=sb.SB_SAD_AUTO):
    """items: list of (left, right, params).  Returns [(out_rgb, out_disp)]."""
    pairs, outs = [], []
    for left, right, p in items:
        h, w = left.shape[:2]
        o = torch.empty((h, w, 3), dtype=torch.uint8, device="cuda")
        d = torch.empty((h, w), dtype=torch.int16, device="cuda")
        pairs.append(sb.Pair(dev(left), dev(right), params_of(p, sad_variant), o, d))
        outs.append((o, d))
    sb.sb_run(ctx, pairs, flags)
    ctx.synchronize()
    return [(host(o), host(d, np.uint16)) for o, d in outs]
