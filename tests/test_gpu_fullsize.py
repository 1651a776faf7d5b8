"""Parity at the workloads' full sizes, in the benchmark's launch form
(batched pairs replayed from a CUDA graph).  The oracle runs its O(N) stages
(lightness, K-means, boundary refinement, components, anchors) in full and is
compared element by element with the library's stage outputs; SAD, the final
disparity (Algorithms 1 and 2) and the blur are compared at sampled pixels
that the oracle evaluates one by one from the same definitions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import synth  # noqa: E402
import paper_2001_07809_b300 as sb  # noqa: E402
from gpu_helpers import dev, host, params_of  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def ctx():
    c = sb.Context(0)
    yield c
    c.close()


def _gpu_front(ctx, left, right, p):
    """Library stage outputs: L maps, bin->cluster, refined map, labels, filtered map."""
    h, w = left.shape[:2]
    Ll = torch.empty((h, w), dtype=torch.uint8, device="cuda")
    Lr = torch.empty_like(Ll)
    sb.sb_rgb_to_lightness(ctx, dev(left), Ll)
    sb.sb_rgb_to_lightness(ctx, dev(right), Lr)
    labels = torch.empty_like(Ll)
    cent = torch.empty((p.k,), dtype=torch.float64, device="cuda")
    lut = torch.empty((256,), dtype=torch.uint8, device="cuda")
    sb.sb_kmeans_segment(ctx, Ll, p.k, p.kmeans_max_iter, labels, cent, lut)
    bnd = torch.empty_like(Ll)
    ref = torch.empty_like(Ll)
    lab = torch.empty((h, w), dtype=torch.int32, device="cuda")
    sb.sb_refine_boundaries(ctx, labels, bnd, p.morph_mode, p.cc_remove_fraction, ref, lab)
    disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    cost = torch.empty((h, w), dtype=torch.int32, device="cuda")
    sb.sb_boundary_sad(ctx, Ll, Lr, bnd, p.max_disp, p.block, disp, cost)
    ctx.synchronize()
    return dict(L_left=host(Ll), L_right=host(Lr), centroids=host(cent), lut=host(lut), refined=host(ref),
                cc=host(lab), filtered=host(bnd), sparse=host(disp, np.uint16), cost=host(cost, np.uint32))


def _check_pair(ctx, left, right, p, out_rgb, out_disp, rng, n_sad=150, n_pts=150, n_blur=60):
    fr = oracle.run_front(left, right, p)
    g = _gpu_front(ctx, left, right, p)
    for k in ("L_left", "L_right", "refined", "filtered"):
        assert np.array_equal(g[k], getattr(fr, k)), k
    assert np.array_equal(g["centroids"].view(np.uint64), fr.centroids.view(np.uint64))
    assert np.array_equal(g["lut"], fr.bin2cluster)
    assert np.array_equal(g["cc"], fr.cc_labels)
    anchor = fr.anchor.astype(bool)
    assert np.array_equal(g["sparse"] != oracle.UNDET, anchor)
    ys, xs = np.nonzero(anchor)
    for i in rng.choice(len(ys), size=min(n_sad, len(ys)), replace=False):
        d, c = oracle.sad_argmin(fr.L_left, fr.L_right, int(xs[i]), int(ys[i]), p.max_disp, p.block)
        assert (g["sparse"][ys[i], xs[i]], g["cost"][ys[i], xs[i]]) == (d, c)
    h, w = anchor.shape
    pts = [(int(rng.integers(0, w)), int(rng.integers(0, h))) for _ in range(n_pts)]
    memo = {}
    want = oracle.disp_at_points(fr, p, pts, memo)
    got = [int(out_disp[y, x]) for x, y in pts]
    assert got == want
    # blur at sampled pixels, decided by the oracle's own disparity there
    bpts = [(int(rng.integers(0, w)), int(rng.integers(0, h))) for _ in range(n_blur)]
    bd = oracle.disp_at_points(fr, p, bpts, memo)
    for (x, y), d in zip(bpts, bd):
        focus = any(lo <= d <= hi for lo, hi in p.ranges)
        ref = left[y, x] if focus else oracle.blur_at(left, x, y, p.sigma)
        assert np.abs(out_rgb[y, x].astype(int) - ref.astype(int)).max() <= 1, (x, y)


def _run_batch(ctx, items):
    pairs, outs = [], []
    for left, right, p in items:
        h, w = left.shape[:2]
        o = torch.empty((h, w, 3), dtype=torch.uint8, device="cuda")
        d = torch.empty((h, w), dtype=torch.int16, device="cuda")
        pairs.append(sb.Pair(dev(left), dev(right), params_of(p), o, d))
        outs.append((o, d))
    flags = sb.SB_RUN_BATCHED | sb.SB_RUN_GRAPH
    sb.sb_run(ctx, pairs, flags)
    sb.sb_run(ctx, pairs, flags)    # a replay must give the same result
    ctx.synchronize()
    return [(host(o), host(d, np.uint16)) for o, d in outs]


def test_c2_full_size(ctx):
    sc, p, _ = synth.workload("c2")
    left, right, _ = sc.render()
    (o_rgb, o_disp), = _run_batch(ctx, [(left, right, p)])
    _check_pair(ctx, left, right, p, o_rgb, o_disp, np.random.default_rng(1))


def test_c3_frames_full_size(ctx):
    sc, p, _ = synth.workload("c3")
    frames = (0, 1, 124, 249)
    items = []
    for f in frames:
        left, right, _ = sc.render(frame=f, want_gt=False)
        items.append((left, right, p))
    res = _run_batch(ctx, items)
    rng = np.random.default_rng(3)
    for (left, right, _), (o_rgb, o_disp) in zip(items, res):
        _check_pair(ctx, left, right, p, o_rgb, o_disp, rng, n_sad=60, n_pts=60, n_blur=25)


@pytest.mark.parametrize("part", range(4))
def test_c4_uneven_batch(ctx, part):
    # all 64 pairs of the uneven batch, 16 per batched launch (each launch
    # mixes sizes, disparity ranges, blocks and K)
    items = []
    for i in range(16 * part, 16 * part + 16):
        sc, p, _ = synth.workload("c4", i)
        left, right, _ = sc.render(want_gt=False)
        items.append((left, right, p))
    res = _run_batch(ctx, items)
    rng = np.random.default_rng(40 + part)
    for (left, right, p), (o_rgb, o_disp) in zip(items, res):
        _check_pair(ctx, left, right, p, o_rgb, o_disp, rng, n_sad=30, n_pts=30, n_blur=10)


def test_generator_device_build_matches_host(ctx):
    for name, frame in (("c1", 0), ("c3", 7)):
        sc, _, _ = synth.workload(name, frame)
        left, right, gt = sc.render(frame=frame)
        dl = torch.empty(left.shape, dtype=torch.uint8, device="cuda")
        dr = torch.empty_like(dl)
        dg = torch.empty(gt.shape, dtype=torch.float32, device="cuda")
        synth.render_device(sc, frame, dl, dr, dg, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(host(dl), left) and np.array_equal(host(dr), right)
        assert np.array_equal(host(dg), gt)
