"""Parity of every CUDA stage with the CPU oracle (bit-exact; blur within one
level), on seeded synthetic inputs.  Stage tests feed each kernel the
oracle's own input for that stage; pipeline tests run sb_run end to end and
compare with the oracle's whole pipeline."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import synth  # noqa: E402
import paper_2001_07809_b300 as sb  # noqa: E402
from gpu_helpers import blur, dev, host, kmeans, lightness, params_of, recon, refine, run_pairs, sad  # noqa: E402

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(2024)


@pytest.fixture(scope="module")
def ctx():
    c = sb.Context(0)
    yield c
    c.close()


# ------------------------------------------------------------------ lightness
def test_lightness_every_rgb_triple(ctx):
    r, g, b = np.meshgrid(np.arange(256), np.arange(256), np.arange(256), indexing="ij")
    rgb = np.stack([r, g, b], -1).astype(np.uint8).reshape(4096, 4096, 3)
    L, hist = lightness(ctx, rgb)
    want = oracle.rgb_to_lightness(rgb)
    assert np.array_equal(L, want)
    assert np.array_equal(hist, np.bincount(want.ravel(), minlength=256))


@pytest.mark.parametrize("h,w", [(1, 1), (3, 5), (17, 33), (240, 320), (101, 999)])
def test_lightness_shapes(ctx, h, w):
    rgb = RNG.integers(0, 256, (h, w, 3)).astype(np.uint8)
    L, hist = lightness(ctx, rgb)
    assert np.array_equal(L, oracle.rgb_to_lightness(rgb))
    assert np.array_equal(hist, oracle.histogram(L))


# --------------------------------------------------------------------- kmeans
@pytest.mark.parametrize("K", [1, 2, 4, 6, 8, 10, 33, 255])
def test_kmeans_bit_exact(ctx, K):
    vals = np.concatenate([RNG.normal(m, s, 3000) for m, s in ((30, 8), (90, 20), (160, 5), (215, 12))])
    L = np.clip(np.round(vals), 0, 255).astype(np.uint8).reshape(60, 200)
    c, lut, it, labels = kmeans(ctx, L, K)
    oc, olut, oit = oracle.kmeans_hist(oracle.histogram(L), K, 100)
    assert it == oit
    assert np.array_equal(c.view(np.uint64), oc.view(np.uint64))   # FP64 bits
    assert np.array_equal(lut, olut)
    assert np.array_equal(labels, olut[L])


def test_kmeans_flat_and_single_level(ctx):
    L = np.full((20, 30), 77, np.uint8)
    c, lut, it, _ = kmeans(ctx, L, 3)
    oc, olut, oit = oracle.kmeans_hist(oracle.histogram(L), 3)
    assert np.array_equal(c, oc) and np.array_equal(lut, olut) and it == oit


# ------------------------------------------------------------- refinement + CCA
@pytest.mark.parametrize("shape", [(48, 64), (97, 131), (240, 320), (333, 517)])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("frac", [0.0, 0.04, 0.3])
def test_refine_boundaries_bit_exact(ctx, shape, mode, frac):
    h, w = shape
    K = 4
    raw = RNG.integers(0, K, (h // 4 + 1, w // 4 + 1))
    labels = np.kron(raw, np.ones((4, 4), np.int64))[:h, :w]
    noise = RNG.random((h, w)) < 0.05
    labels = np.where(noise, RNG.integers(0, K, (h, w)), labels).astype(np.uint8)
    ref, lab, bnd = refine(ctx, labels, mode, frac)
    o_b0 = oracle.boundary(labels)
    o_ref = oracle.refine(o_b0, mode)
    o_lab, _ = oracle.cca(o_ref)
    o_bnd = oracle.cc_filter(o_ref, o_lab, frac)
    assert np.array_equal(ref, o_ref)
    assert np.array_equal(lab, o_lab)
    assert np.array_equal(bnd, o_bnd)


@pytest.mark.parametrize("frac", [0.01, 0.04, 0.2])
def test_cc_cut_inside_a_size_class(ctx, frac):
    # many equal-size components: the cut falls inside the size class, so the
    # smallest-label rule decides which of them go
    h, w = 300, 400
    labels = np.zeros((h, w), np.uint8)
    for y in range(2, h - 2, 6):
        for x in range(2, w - 2, 6):
            labels[y, x] = 1 + (x // 6) % 3              # isolated dots -> equal 8-px rings
    labels[100:180, 50:350] = 3                         # and one large ring
    ref, lab, bnd = refine(ctx, labels, 0, frac)
    o_ref = oracle.refine(oracle.boundary(labels), 0)
    o_lab, _ = oracle.cca(o_ref)
    o_bnd = oracle.cc_filter(o_ref, o_lab, frac)
    assert np.array_equal(lab, o_lab)
    removed = int(o_ref.sum() - o_bnd.sum())
    assert 0 < removed < int(o_ref.sum())
    assert np.array_equal(bnd, o_bnd)


@pytest.mark.parametrize("noise", [0.3, 0.7])
def test_cca_dense_noisy_maps(ctx, noise):
    # dense, irregular boundary maps: many runs per tile row, diagonal links,
    # runs touching several runs of the row above, components merging late
    h, w = 211, 389
    labels = RNG.integers(0, 2, (h // 3 + 1, w // 3 + 1))
    labels = np.kron(labels, np.ones((3, 3), np.int64))[:h, :w]
    flip = RNG.random((h, w)) < noise
    labels = np.where(flip, RNG.integers(0, 3, (h, w)), labels).astype(np.uint8)
    ref, lab, bnd = refine(ctx, labels, 1, 0.04)
    o_ref = oracle.refine(oracle.boundary(labels), 1)
    o_lab, _ = oracle.cca(o_ref)
    assert np.array_equal(ref, o_ref)
    assert np.array_equal(lab, o_lab)
    assert np.array_equal(bnd, oracle.cc_filter(o_ref, o_lab, 0.04))


def _merge_pattern(kind, h, w):
    # label maps whose boundary maps hold about 40 runs per row that meet the
    # runs of the rows around them at once: stripes three pixels wide crossed
    # by bars of a third label, concentric rings, and combs (teeth joined by
    # a bar)
    y, x = np.mgrid[0:h, 0:w]
    if kind == "stripes":
        lab = np.where((y % 37) > 33, 2, (x // 3) % 2)
    elif kind == "rings":
        lab = (np.hypot(x - w // 2, y - h // 2) // 4).astype(np.int64) % 3
    else:
        lab = ((x % 4) < 2) | ((y % 37) > 33)
    return lab.astype(np.uint8)


@pytest.mark.parametrize("kind", ["stripes", "rings", "comb"])
def test_cca_merging_patterns(ctx, kind):
    # ragged size over several tiles in both directions
    labels = _merge_pattern(kind, 97, 133)
    o_ref = oracle.refine(oracle.boundary(labels), 0)
    ref, lab, bnd = refine(ctx, labels, 0, 0.04)
    o_lab, _ = oracle.cca(o_ref)
    assert np.array_equal(ref, o_ref)
    assert np.array_equal(lab, o_lab)
    assert np.array_equal(bnd, oracle.cc_filter(o_ref, o_lab, 0.04))


def test_refine_degenerate(ctx):
    # K = 1: no boundary at all; one label row; a single pixel image
    for labels in (np.zeros((40, 50), np.uint8), np.array([[0, 1, 1, 0, 2]], np.uint8), np.zeros((1, 1), np.uint8)):
        ref, lab, bnd = refine(ctx, labels)
        o_ref = oracle.refine(oracle.boundary(labels), 0)
        o_lab, _ = oracle.cca(o_ref)
        assert np.array_equal(ref, o_ref) and np.array_equal(lab, o_lab)
        assert np.array_equal(bnd, oracle.cc_filter(o_ref, o_lab, 0.04))


def test_cca_long_snake_spans_many_tiles(ctx):
    # one 8-connected component winding through every 32x32 tile
    h, w = 130, 200
    b = np.zeros((h, w), np.uint8)
    for y in range(0, h, 4):
        b[y, :] = 1
        b[y:y + 4, (w - 1) if (y // 4) % 2 == 0 else 0] = 1
    labels = b  # two labels -> boundary map from them is irrelevant; test CCA through refine of labels
    o_ref = oracle.refine(oracle.boundary(labels), 0)
    ref, lab, _ = refine(ctx, labels)
    o_lab, n = oracle.cca(o_ref)
    assert np.array_equal(ref, o_ref) and np.array_equal(lab, o_lab)


def _snake_labels():
    h, w = 130, 200
    b = np.zeros((h, w), np.uint8)
    for y in range(0, h, 4):
        b[y, :] = 1
        b[y:y + 4, (w - 1) if (y // 4) % 2 == 0 else 0] = 1
    return b


def test_union_limit_reports_timeout_then_recovers():
    # a union-find bound of one parent link cannot label the snake (its chains
    # cross many tiles): the run is flagged and sb_synchronize reports
    # SB_ERR_TIMEOUT; with the default bound the same context labels it exactly
    labels = _snake_labels()
    with sb.Context(0) as c:
        c.set_union_limit(1)
        refine(c, labels)
        with pytest.raises(sb.SbError) as ei:
            c.synchronize()
        assert ei.value.status == sb.SB_ERR_TIMEOUT and "union" in str(ei.value)
        c.synchronize()                       # the flag was cleared
        c.set_union_limit(0)
        ref, lab, _ = refine(c, labels)
        c.synchronize()
        o_ref = oracle.refine(oracle.boundary(labels), 0)
        assert np.array_equal(ref, o_ref) and np.array_equal(lab, oracle.cca(o_ref)[0])
        with pytest.raises(sb.SbError) as ei:
            c.set_union_limit(-1)
        assert ei.value.status == sb.SB_ERR_INVALID_ARG


def test_workspace_budget_reports_oom_and_context_stays_usable():
    # a 1 MB budget cannot hold a 320x240 pair's workspace (about 18 bytes per
    # pixel): sb_run returns SB_ERR_OOM; a pair that fits
    # then runs on the same context and matches the oracle
    sc, p, _ = synth.workload("c1")
    left, right, _ = sc.render()
    with sb.Context(0, mem_budget_bytes=1 << 20) as c:
        with pytest.raises(sb.SbError) as ei:
            run_pairs(c, [(left, right, p)], sb.SB_RUN_BATCHED)
        assert ei.value.status == sb.SB_ERR_OOM
        r = synth.Rng(321)
        w, h, D = 160, 96, 16
        small = synth.Scene(w, h, synth._c2_style_layers(r, w, h, D, contrast=60), noise_q8=256, noise_seed=r.u64())
        sl, sr, _ = small.render()
        ps = synth.Params(k=4, max_disp=D, block=7, sigma=2.0, ranges=[(8, D)])
        (o_rgb, o_disp), = run_pairs(c, [(sl, sr, ps)], sb.SB_RUN_BATCHED)
        assert c.workspace_bytes() <= 1 << 20
        _compare_full(o_rgb, o_disp, sl, sr, ps)


# ------------------------------------------------------------------------ SAD
SAD_CASES = [
    # (h, w, D, B)
    (40, 60, 0, 1), (40, 60, 5, 3), (61, 97, 31, 9), (61, 97, 32, 9), (61, 97, 33, 9),
    (70, 260, 64, 15), (90, 600, 40, 31), (80, 420, 100, 41), (70, 300, 64, 63), (47, 340, 255, 5),
    (65, 700, 256, 41),
    # around the box sums' chunk of 64 disparities: a whole chunk, then 1 and 2
    # disparities past it for the tail kernel, 8 (its largest), and 9 (a partial chunk)
    (61, 97, 63, 9), (61, 97, 64, 9), (61, 97, 65, 9), (70, 320, 71, 15), (70, 320, 72, 15),
    (55, 330, 39, 11), (70, 360, 71, 63), (50, 300, 98, 1), (66, 520, 135, 25),
    # the largest disparity range the 10-bit key holds (16 whole chunks), a tail
    # of 8 at a large range, partial chunks of 40 and 41 disparities (the last with
    # the largest block); widths that are and are not multiples of 16
    (40, 1100, 1023, 5), (40, 1104, 1023, 5), (45, 1100, 967, 9), (45, 1104, 999, 9), (70, 1200, 1000, 63),
]


@pytest.mark.parametrize("h,w,D,B", SAD_CASES)
@pytest.mark.parametrize("variant", [sb.SB_SAD_BOXSUM, sb.SB_SAD_DIRECT])
def test_sad_bit_exact(ctx, h, w, D, B, variant):
    Ll = RNG.integers(0, 256, (h, w)).astype(np.uint8)
    shift = min(D, 7)
    Lr = np.roll(Ll, -shift, axis=1)
    Lr = np.clip(Lr.astype(int) + RNG.integers(-6, 7, (h, w)), 0, 255).astype(np.uint8)
    bmap = (RNG.random((h, w)) < 0.2).astype(np.uint8)
    disp, cost = sad(ctx, Ll, Lr, bmap, D, B, variant)
    anchor = oracle.anchor_mask(bmap, D, B)
    od, oc = oracle.boundary_sad(Ll, Lr, anchor, D, B)
    assert np.array_equal(disp, od)
    assert np.array_equal(cost, oc)


def test_sad_flat_images_tie_to_smallest_d(ctx):
    h, w, D, B = 30, 120, 20, 7
    Ll = np.full((h, w), 100, np.uint8)
    Lr = np.full((h, w), 100, np.uint8)
    bmap = np.ones((h, w), np.uint8)
    for variant in (sb.SB_SAD_BOXSUM, sb.SB_SAD_DIRECT):
        disp, cost = sad(ctx, Ll, Lr, bmap, D, B, variant)
        anchor = oracle.anchor_mask(bmap, D, B).astype(bool)
        assert np.all(disp[anchor] == 0) and np.all(cost[anchor] == 0)
        assert np.all(disp[~anchor] == sb.UNDETERMINED)


def test_sad_extreme_costs(ctx):
    # maximal per-pixel differences: costs up to 63*63*255 must not overflow the key
    h, w, D, B = 70, 200, 20, 63
    Ll = np.zeros((h, w), np.uint8)
    Lr = np.full((h, w), 255, np.uint8)
    bmap = np.ones((h, w), np.uint8)
    for variant in (sb.SB_SAD_BOXSUM, sb.SB_SAD_DIRECT):
        disp, cost = sad(ctx, Ll, Lr, bmap, D, B, variant)
        anchor = oracle.anchor_mask(bmap, D, B).astype(bool)
        od, oc = oracle.boundary_sad(Ll, Lr, anchor.astype(np.uint8), D, B)
        assert np.array_equal(disp, od) and np.array_equal(cost, oc)
        assert np.all(oc[anchor] == 63 * 63 * 255) and np.all(od[anchor] == 0)


@pytest.mark.parametrize("h,w,D,B", [(60, 700, 40, 9), (50, 500, 71, 21)])
def test_sad_every_anchor_pattern(ctx, h, w, D, B):
    # every 8-bit anchor pattern, in every alignment to the box-sum's blocks of
    # eight outputs: row y, columns 8j .. 8j+7 carry the bits of (y * 37 + j) mod 256
    Ll = RNG.integers(0, 256, (h, w)).astype(np.uint8)
    Lr = np.clip(np.roll(Ll, -3, axis=1).astype(int) + RNG.integers(-9, 10, (h, w)), 0, 255).astype(np.uint8)
    ys, xs = np.mgrid[0:h, 0:w]
    pattern = (ys * 37 + (xs + ys) // 8) % 256
    bmap = ((pattern >> ((xs + ys) % 8)) & 1).astype(np.uint8)
    disp, cost = sad(ctx, Ll, Lr, bmap, D, B, sb.SB_SAD_BOXSUM)
    od, oc = oracle.boundary_sad(Ll, Lr, oracle.anchor_mask(bmap, D, B), D, B)
    assert np.array_equal(disp, od) and np.array_equal(cost, oc)


@pytest.mark.parametrize("density,B", [(0.0, 1), (0.0, 9), (0.01, 3), (0.03, 3), (0.5, 25), (0.2, 41)])
def test_sad_auto_choice_is_exact(ctx, density, B):
    # the automatic choice is taken on the device from the map's own count;
    # whichever kernel serves the map, the result is the oracle's
    h, w, D = 90, 400, 48
    Ll = RNG.integers(0, 256, (h, w)).astype(np.uint8)
    Lr = np.clip(np.roll(Ll, -5, axis=1).astype(int) + RNG.integers(-4, 5, (h, w)), 0, 255).astype(np.uint8)
    bmap = (RNG.random((h, w)) < density).astype(np.uint8)
    disp, cost = sad(ctx, Ll, Lr, bmap, D, B, sb.SB_SAD_AUTO)
    od, oc = oracle.boundary_sad(Ll, Lr, oracle.anchor_mask(bmap, D, B), D, B)
    assert np.array_equal(disp, od) and np.array_equal(cost, oc)


def test_batched_auto_mixes_variants_per_pair(ctx):
    # a boundary-free pair (only the domain's edge columns are anchors: the
    # direct kernel serves it) batched with textured pairs (box sums serve
    # them): every pair equals its forced-variant result and the oracle
    items = []
    flat = np.full((96, 300, 3), 90, np.uint8)
    items.append((flat, flat.copy(), synth.Params(k=4, max_disp=40, block=3, sigma=2.0, ranges=[(10, 20)])))
    for i in range(2):
        r = synth.Rng(700 + i)
        sc = synth.Scene(320, 120, synth._c2_style_layers(r, 320, 120, 48, contrast=50), noise_q8=512,
                         noise_seed=r.u64())
        left, right, _ = sc.render(want_gt=False)
        items.append((left, right, synth.Params(k=6, max_disp=48, block=(25, 9)[i], sigma=3.0, ranges=[(0, 16)])))
    auto = run_pairs(ctx, items, sb.SB_RUN_BATCHED)
    for variant in (sb.SB_SAD_BOXSUM, sb.SB_SAD_DIRECT):
        forced = run_pairs(ctx, items, sb.SB_RUN_BATCHED, sad_variant=variant)
        for (a_rgb, a_disp), (f_rgb, f_disp) in zip(auto, forced):
            assert np.array_equal(a_rgb, f_rgb) and np.array_equal(a_disp, f_disp)
    for (left, right, p), (o_rgb, o_disp) in zip(items, auto):
        _compare_full(o_rgb, o_disp, left, right, p)


# ------------------------------------------------------------ reconstruction
@pytest.mark.parametrize("h,w,D,B,T", [(50, 80, 4, 3, 1), (130, 140, 10, 5, 0), (200, 333, 20, 9, 3),
                                       (257, 64, 0, 1, -1), (300, 50, 8, 7, 1000)])
@pytest.mark.parametrize("peek_mode", [sb.SB_PEEK_SNAPSHOT, sb.SB_PEEK_INPLACE])
def test_recon_bit_exact(ctx, h, w, D, B, T, peek_mode):
    bmap = (RNG.random((h, w)) < 0.15).astype(np.uint8)
    anchor = oracle.anchor_mask(bmap, D, B)
    sparse = np.full((h, w), oracle.UNDET, np.uint16)
    vals = RNG.integers(0, 6 if T < 100 else 200, (h, w)).astype(np.uint16)   # few values: many equal neighbours
    sparse[anchor == 1] = vals[anchor == 1]
    filled, final = recon(ctx, sparse, D, B, T, peek_mode)
    o_filled = oracle.recon_fill(sparse, anchor)
    peek = oracle.recon_peek_inplace if peek_mode == sb.SB_PEEK_INPLACE else oracle.recon_peek
    o_final = peek(o_filled, D, B, T)
    assert np.array_equal(filled, o_filled)
    assert np.array_equal(final, o_final)


def test_recon_inplace_golden_columns(ctx, golden_dir):
    import os
    from test_oracle_pins import _blocks, _parse_row
    for tag, rows in _blocks(os.path.join(golden_dir, "alg2_inplace_columns.txt")):
        T = int(tag.split("T=")[1])
        d = dict(rows)
        col = np.array(_parse_row(d["column"]), np.uint16)
        e = np.array(_parse_row(d["expected"]), np.uint16)
        # D = 0, block 1: Omega is the whole image; the column sits beside an
        # empty one (the smallest legal width), so Algorithm 1 changes nothing
        img = np.full((len(col), 2), oracle.UNDET, np.uint16)
        img[:, 0] = col
        _, final = recon(ctx, img, 0, 1, T, sb.SB_PEEK_INPLACE)
        assert np.array_equal(final[:, 0], e), tag
        assert np.all(final[:, 1] == 0), tag


def test_recon_paper_rows_and_columns(ctx, golden_dir):
    # the hand-worked Algorithm 1 rows, stacked into one image with block 1, D 0
    import os
    from test_oracle_pins import _blocks, _parse_row
    for tag, rows in _blocks(os.path.join(golden_dir, "alg1_rows.txt")):
        d = dict(rows)
        a = np.array([_parse_row(d["anchors"])], np.uint16)
        e = np.array([_parse_row(d["expected"])], np.uint16)
        filled, _ = recon(ctx, a, 0, 1, 1)
        assert np.array_equal(filled, e), tag


# ---------------------------------------------------------------------- blur
@pytest.mark.parametrize("sigma", [0.5, 1.0, 2.0, 3.0, 5.0, 8.0, 13.7, 32.0])
def test_blur_within_one_level(ctx, sigma):
    h, w = (90, 150) if sigma <= 8 else (260, 300)
    rgb = RNG.integers(0, 256, (h, w, 3)).astype(np.uint8)
    disp = RNG.integers(0, 40, (h, w)).astype(np.uint16)
    ranges = [(10, 20), (30, 31)]
    out = blur(ctx, rgb, disp, ranges, sigma)
    want = oracle.selective_blur(rgb, disp, ranges, sigma)
    diff = np.abs(out.astype(int) - want.astype(int))
    assert diff.max() <= 1
    keep = ((disp >= 10) & (disp <= 20)) | ((disp >= 30) & (disp <= 31))
    assert np.array_equal(out[keep], rgb[keep])


@pytest.mark.parametrize("sigma", [2.0, 8.0, 8.6, 9.0])
@pytest.mark.parametrize("offset", [0, 1])
def test_blur_interior_tiles(ctx, sigma, offset):
    # wide enough for tiles whose input run lies inside the image (staged with
    # 16-byte copies at per-row offsets: 3*517 bytes per row is not a multiple
    # of 16); offset 1 makes the RGB base unaligned, which takes the byte path
    h, w = 150, 517
    rgb = RNG.integers(0, 256, (h, w, 3)).astype(np.uint8)
    disp = RNG.integers(0, 40, (h, w)).astype(np.uint16)
    ranges = [(10, 20)]
    buf = torch.empty(h * w * 3 + 16, dtype=torch.uint8, device="cuda")
    d_rgb = buf[offset:offset + h * w * 3].view(h, w, 3)
    d_rgb.copy_(torch.from_numpy(rgb))
    out = torch.empty((h, w, 3), dtype=torch.uint8, device="cuda")
    sb.sb_selective_blur(ctx, d_rgb, dev(disp), ranges, sigma, out)
    want = oracle.selective_blur(rgb, disp, ranges, sigma)
    assert np.abs(host(out).astype(int) - want.astype(int)).max() <= 1


@pytest.mark.parametrize("sigma", [3.0, 8.0])
def test_blur_forms_agree_with_oracle(ctx, sigma):
    # tiles of 112 and 64 rows and the strip form give the same bytes; 1100
    # rows span three 512-row strip bands (the last one ragged), 300 columns
    # end in a ragged 44-column strip; rows 0..399 are all in focus (steps with
    # no blurred pixel are copied and the filtered rows only they read are
    # skipped) and so is the band of rows 512..1023 except one row
    h, w = 1100, 300
    rgb = RNG.integers(0, 256, (h, w, 3)).astype(np.uint8)
    disp = RNG.integers(0, 40, (h, w)).astype(np.uint16)
    disp[:400] = 15
    disp[512:1024] = 12
    disp[700, 17:60] = 3
    ranges = [(10, 20)]
    want = oracle.selective_blur(rgb, disp, ranges, sigma)
    outs = []
    try:
        for form in (sb.SB_BLUR_TILES_112, sb.SB_BLUR_TILES_64, sb.SB_BLUR_STRIP):
            sb.sb_set_blur_form(ctx, form)
            outs.append(blur(ctx, rgb, disp, ranges, sigma))
    finally:
        sb.sb_set_blur_form(ctx, sb.SB_BLUR_AUTO)
    assert np.abs(outs[0].astype(int) - want.astype(int)).max() <= 1
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    keep = (disp >= 10) & (disp <= 20)
    assert np.array_equal(outs[2][keep], rgb[keep])


@pytest.mark.parametrize("sigma", [0.5, 20.0])
def test_blur_strip_small_and_large_radius(ctx, sigma):
    # R = 2 and R = 60 (a ring of 160 filtered rows): two bands, the second
    # ragged, and a ragged last strip; every form gives the oracle's bytes within one level
    h, w = 600, 300
    rgb = RNG.integers(0, 256, (h, w, 3)).astype(np.uint8)
    disp = RNG.integers(0, 40, (h, w)).astype(np.uint16)
    ranges = [(10, 20)]
    want = oracle.selective_blur(rgb, disp, ranges, sigma)
    outs = []
    try:
        for form in (sb.SB_BLUR_TILES_112, sb.SB_BLUR_STRIP):
            sb.sb_set_blur_form(ctx, form)
            outs.append(blur(ctx, rgb, disp, ranges, sigma))
    finally:
        sb.sb_set_blur_form(ctx, sb.SB_BLUR_AUTO)
    assert np.abs(outs[1].astype(int) - want.astype(int)).max() <= 1
    assert np.array_equal(outs[0], outs[1])


def test_blur_form_rejects_unknown_values(ctx):
    with pytest.raises(sb.SbError):
        sb.sb_set_blur_form(ctx, 48)


def test_blur_constant_image_unchanged(ctx):
    rgb = np.full((140, 260, 3), 93, np.uint8)
    rgb[..., 2] = 250
    out = blur(ctx, rgb, np.zeros((140, 260), np.uint16), [], 6.0)
    assert np.array_equal(out, rgb)


# ----------------------------------------------------------- whole pipeline
def _compare_full(res_rgb, res_disp, left, right, p):
    want = oracle.run(left, right, p)
    assert np.array_equal(res_disp, want.disp)
    assert np.abs(res_rgb.astype(int) - want.out_rgb.astype(int)).max() <= 1
    return want


@pytest.mark.parametrize("flags", [sb.SB_RUN_PLAIN, sb.SB_RUN_BATCHED, sb.SB_RUN_BATCHED | sb.SB_RUN_GRAPH])
@pytest.mark.parametrize("variant", [sb.SB_SAD_BOXSUM, sb.SB_SAD_DIRECT])
def test_pipeline_c1_full(ctx, flags, variant):
    sc, p, _ = synth.workload("c1")
    left, right, _ = sc.render()
    (o_rgb, o_disp), = run_pairs(ctx, [(left, right, p)], flags, variant)
    _compare_full(o_rgb, o_disp, left, right, p)


def test_pipeline_ragged_and_open_close(ctx):
    r = synth.Rng(99)
    layers = [synth.Layer(0, 150, 120, 333, 257, 5 * 256, 90, 70, r.u64() & 0xFFFFFFFF)]
    for i, d in enumerate((14, 25, 33)):
        layers.append(synth.Layer(1 + i % 2, r.randint(80, 260), r.randint(40, 200), r.randint(20, 50),
                                  r.randint(20, 40), d * 256, 60 + 50 * i, 70, r.u64() & 0xFFFFFFFF))
    sc = synth.Scene(333, 257, layers, noise_q8=300, noise_seed=7)
    left, right, _ = sc.render()
    for mode, T in ((1, 0), (0, 2)):
        p = synth.Params(k=5, max_disp=40, block=11, sigma=2.5, ranges=[(0, 9), (30, 40)], disp_threshold=T,
                         morph_mode=mode)
        (o_rgb, o_disp), = run_pairs(ctx, [(left, right, p)], sb.SB_RUN_PLAIN)
        _compare_full(o_rgb, o_disp, left, right, p)


def test_pipeline_inplace_peek_and_mixed_batch(ctx):
    # the in-place reading of Algorithm 2 through the whole pipeline, and a
    # batch mixing both readings (one launch per kernel, each job picks its own)
    sc, p, _ = synth.workload("c1")
    left, right, _ = sc.render()
    import dataclasses
    p_ip = dataclasses.replace(p, peek_mode=1)
    (rgb_ip, disp_ip), = run_pairs(ctx, [(left, right, p_ip)], sb.SB_RUN_PLAIN)
    _compare_full(rgb_ip, disp_ip, left, right, p_ip)
    mixed = run_pairs(ctx, [(left, right, p), (left, right, p_ip)], sb.SB_RUN_BATCHED | sb.SB_RUN_GRAPH)
    (rgb_sn, disp_sn), = run_pairs(ctx, [(left, right, p)], sb.SB_RUN_PLAIN)
    assert np.array_equal(mixed[0][1], disp_sn) and np.array_equal(mixed[0][0], rgb_sn)
    assert np.array_equal(mixed[1][1], disp_ip) and np.array_equal(mixed[1][0], rgb_ip)


def test_right_view_pipeline_and_lr_consistency(ctx):
    # the right image as the reference: disparity map and
    # blurred right image equal the oracle's; a batch mixing both views equals
    # the views run alone; the left-right consistency map and count equal the
    # oracle's on the two maps
    import dataclasses
    sc, p, _ = synth.workload("c1")
    left, right, _ = sc.render()
    p_r = dataclasses.replace(p, view=1)
    (rgb_r, disp_r), = run_pairs(ctx, [(left, right, p_r)], sb.SB_RUN_PLAIN)
    want = _compare_full(rgb_r, disp_r, left, right, p_r)
    assert np.abs(rgb_r.astype(int) - want.out_rgb.astype(int)).max() <= 1
    (rgb_l, disp_l), = run_pairs(ctx, [(left, right, p)], sb.SB_RUN_PLAIN)
    mixed = run_pairs(ctx, [(left, right, p_r), (left, right, p)], sb.SB_RUN_BATCHED | sb.SB_RUN_GRAPH)
    assert np.array_equal(mixed[0][1], disp_r) and np.array_equal(mixed[0][0], rgb_r)
    assert np.array_equal(mixed[1][1], disp_l) and np.array_equal(mixed[1][0], rgb_l)
    for tol in (0, 1, 3):
        ok = torch.empty(disp_l.shape, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        sb.sb_lr_consistency(ctx, dev(disp_l), dev(disp_r), ok, tol, cnt)
        ctx.synchronize()
        o_ok, o_n = oracle.lr_consistency(disp_l, disp_r, tol)
        assert np.array_equal(host(ok), o_ok) and int(cnt.item()) == o_n


def test_autotune_keeps_results_and_caches_the_split(ctx):
    # the autotuner times the candidate work splits on real pairs; outputs do
    # not depend on the split, and later runs of the shape use the chosen one
    items = []
    for i in range(3):
        r = synth.Rng(800 + i)
        sc = synth.Scene(360, 140, synth._c2_style_layers(r, 360, 140, 48, contrast=40), noise_q8=512,
                         noise_seed=r.u64())
        left, right, _ = sc.render(want_gt=False)
        items.append((left, right, synth.Params(k=6, max_disp=48, block=(9, 15, 25)[i], sigma=3.0,
                                                ranges=[(0, 16)], morph_mode=0)))
    before = run_pairs(ctx, items, sb.SB_RUN_BATCHED)
    pairs, outs = [], []
    for left, right, p in items:
        h, w = left.shape[:2]
        o = torch.empty((h, w, 3), dtype=torch.uint8, device="cuda")
        d = torch.empty((h, w), dtype=torch.int16, device="cuda")
        pairs.append(sb.Pair(dev(left), dev(right), params_of(p, sb.SB_SAD_BOXSUM), o, d))
        outs.append((o, d))
    for flags in (sb.SB_RUN_BATCHED | sb.SB_RUN_GRAPH, sb.SB_RUN_PLAIN):
        chosen, rows, ms = sb.sb_autotune(ctx, pairs, flags)
        assert chosen in [ctx_sms() * 2 * k for k in (1, 2, 3, 6)] and rows in (32, 64, 112)
        assert len(ms) == sb.SB_AUTOTUNE_CANDIDATES == 7 and all(m > 0 for m in ms)
        ctx.synchronize()
        # the tuner's last run used the strip-form blur: its outputs are checked too
        for (o, d), (b_rgb, b_disp) in zip(outs, before):
            assert np.array_equal(host(o), b_rgb) and np.array_equal(host(d, np.uint16), b_disp)
        sb.sb_run(ctx, pairs, flags)
        ctx.synchronize()
        for (o, d), (b_rgb, b_disp) in zip(outs, before):
            assert np.array_equal(host(o), b_rgb) and np.array_equal(host(d, np.uint16), b_disp)
    with pytest.raises(sb.SbError):
        sb.sb_autotune(ctx, pairs, sb.SB_RUN_BATCHED | sb.SB_RUN_HOST_IO)


def ctx_sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_batched_and_graph_equal_plain_on_uneven_batch(ctx):
    items = []
    for i, (w, h, D, B, K) in enumerate([(200, 120, 24, 7, 3), (321, 203, 48, 13, 5), (150, 150, 16, 5, 4),
                                         (400, 90, 64, 9, 6)]):
        r = synth.Rng(500 + i)
        layers = synth._c2_style_layers(r, w, h, D, contrast=60)
        sc = synth.Scene(w, h, layers, noise_q8=256, noise_seed=r.u64())
        left, right, _ = sc.render()
        items.append((left, right, synth.Params(k=K, max_disp=D, block=B, sigma=1.5 + i, ranges=[(D // 3, D)])))
    plain = run_pairs(ctx, items, sb.SB_RUN_PLAIN)
    batched = run_pairs(ctx, items, sb.SB_RUN_BATCHED)
    graph = run_pairs(ctx, items, sb.SB_RUN_BATCHED | sb.SB_RUN_GRAPH)
    graph2 = run_pairs(ctx, items, sb.SB_RUN_BATCHED | sb.SB_RUN_GRAPH)   # replay
    for a, b, c, d in zip(plain, batched, graph, graph2):
        for u, v, x, y in zip(a, b, c, d):
            assert np.array_equal(u, v) and np.array_equal(u, x) and np.array_equal(u, y)
    for (left, right, p), (o_rgb, o_disp) in zip(items, plain):
        _compare_full(o_rgb, o_disp, left, right, p)


def test_graph_cache_keeps_several_shapes():
    # one context alternating three one-pair shapes in the graph form: each
    # shape keeps its own instantiated graph (a replay, not a re-capture, on
    # the second round) and every replay equals the plain form
    items = []
    for i, (w, h, D, B, K) in enumerate([(200, 120, 24, 7, 3), (321, 203, 48, 13, 5), (150, 150, 16, 5, 4)]):
        r = synth.Rng(700 + i)
        layers = synth._c2_style_layers(r, w, h, D, contrast=60)
        sc = synth.Scene(w, h, layers, noise_q8=256, noise_seed=r.u64())
        left, right, _ = sc.render()
        items.append((left, right, synth.Params(k=K, max_disp=D, block=B, sigma=2.0, ranges=[(D // 3, D)])))
    with sb.Context(0) as c:
        plain = [run_pairs(c, [it], sb.SB_RUN_PLAIN)[0] for it in items]
        counts = []
        for rnd in range(3):
            for it, want in zip(items, plain):
                l0 = c.launch_count()
                got = run_pairs(c, [it], sb.SB_RUN_BATCHED | sb.SB_RUN_GRAPH)[0]
                counts.append(c.launch_count() - l0)
                assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        # every replay of a shape counts the same kernels as its first run
        assert counts[:3] == counts[3:6] == counts[6:9] and min(counts) > 0


def test_host_io_equals_device(ctx):
    sc, p, _ = synth.workload("c1")
    left, right, _ = sc.render()
    (d_rgb, d_disp), = run_pairs(ctx, [(left, right, p)], sb.SB_RUN_BATCHED)
    for flags in (sb.SB_RUN_HOST_IO, sb.SB_RUN_HOST_IO | sb.SB_RUN_BATCHED):
        hl = torch.from_numpy(left).pin_memory()
        hr = torch.from_numpy(right).pin_memory()
        ho = torch.empty(left.shape, dtype=torch.uint8).pin_memory()
        hd = torch.empty(left.shape[:2], dtype=torch.int16).pin_memory()
        from gpu_helpers import params_of
        sb.sb_run(ctx, [sb.Pair(hl, hr, params_of(p), ho, hd)], flags)
        ctx.synchronize()
        assert np.array_equal(ho.numpy(), d_rgb)
        assert np.array_equal(hd.numpy().view(np.uint16), d_disp)


def test_host_io_batched_across_chunks_and_slots(ctx):
    # twelve mixed pairs streamed from pinned host memory in chunks that ramp from
    # 1 MB to 4 MB of inputs: seven chunks, so every one of the three staging slots
    # is used at least twice, with uploads, compute and downloads of different chunks in flight
    # together; every pair equals the device-resident batched run, and two are
    # checked against the oracle
    from gpu_helpers import params_of
    items = []
    for i in range(12):
        w, h = (640, 480) if i % 3 else (320, 240)
        D, B = (32, 9) if i % 2 else (48, 15)
        r = synth.Rng(700 + i)
        sc = synth.Scene(w, h, synth._c2_style_layers(r, w, h, D, contrast=60), noise_q8=256, noise_seed=r.u64())
        left, right, _ = sc.render()
        items.append((left, right, synth.Params(k=4 + i % 3, max_disp=D, block=B, sigma=1.5 + i % 4,
                                                ranges=[(D // 3, D)])))
    want = run_pairs(ctx, items, sb.SB_RUN_BATCHED)
    ctx.set_host_chunk(1 << 20, 4 << 20)
    try:
        pairs, outs = [], []
        for left, right, p in items:
            hl, hr = torch.from_numpy(left).pin_memory(), torch.from_numpy(right).pin_memory()
            ho = torch.empty(left.shape, dtype=torch.uint8).pin_memory()
            hd = torch.empty(left.shape[:2], dtype=torch.int16).pin_memory()
            pairs.append(sb.Pair(hl, hr, params_of(p), ho, hd))
            outs.append((ho, hd))
        sb.sb_run(ctx, pairs, sb.SB_RUN_HOST_IO | sb.SB_RUN_BATCHED)
        ctx.synchronize()
        assert ctx.host_io_chunks() == 7
        for (ho, hd), (w_rgb, w_disp) in zip(outs, want):
            assert np.array_equal(ho.numpy(), w_rgb)
            assert np.array_equal(hd.numpy().view(np.uint16), w_disp)
        for i in (0, 7):
            left, right, p = items[i]
            _compare_full(outs[i][0].numpy(), outs[i][1].numpy().view(np.uint16), left, right, p)
    finally:
        ctx.set_host_chunk(0, 0)
    with pytest.raises(sb.SbError):
        ctx.set_host_chunk(4 << 20, 1 << 20)


def test_invalid_arguments_raise(ctx):
    left = torch.zeros((20, 30, 3), dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(left)
    bad = [sb.make_params(max_disp=40, block=9), sb.make_params(max_disp=4, block=8),
           sb.make_params(max_disp=4, block=5, k=0), sb.make_params(max_disp=4, block=5, sigma=0.0)]
    for p in bad:
        with pytest.raises(sb.SbError) as ei:
            sb.sb_run(ctx, [sb.Pair(left, left, p, out)])
        assert ei.value.status == 1
    ok = sb.make_params(max_disp=4, block=5, k=2)
    sb.sb_run(ctx, [sb.Pair(left, left, ok, out)])    # the context is still usable
    ctx.synchronize()
    disp = torch.zeros((20, 30), dtype=torch.int16, device="cuda")
    with pytest.raises(sb.SbError) as ei:            # Algorithm 1's map must not overlap the in-place one
        sb.sb_reconstruct_disparity(ctx, disp, 4, 5, 1, disp[1:])
    assert ei.value.status == 1


def test_pipeline_large_disparity_range(ctx):
    # D = 600 on a 700-pixel-wide pair: the domain is 92 columns wide, the SAD
    # runs 9 whole chunks of 64 and a partial one (601 = 9 * 64 + 25)
    w, h, D, B, K = 700, 90, 600, 9, 4
    r = synth.Rng(900)
    layers = synth._c2_style_layers(r, w, h, 120, contrast=60)
    sc = synth.Scene(w, h, layers, noise_q8=256, noise_seed=r.u64())
    left, right, _ = sc.render()
    p = synth.Params(k=K, max_disp=D, block=B, sigma=2.0, ranges=[(40, D)])
    (o_rgb, o_disp), = run_pairs(ctx, [(left, right, p)], sb.SB_RUN_BATCHED)
    _compare_full(o_rgb, o_disp, left, right, p)


def test_minimum_sizes(ctx):
    for (D, B) in ((0, 1), (3, 3), (10, 5)):
        w, h = D + B + 1, B
        left = RNG.integers(0, 256, (h, w, 3)).astype(np.uint8)
        right = RNG.integers(0, 256, (h, w, 3)).astype(np.uint8)
        p = synth.Params(k=2, max_disp=D, block=B, sigma=1.0, ranges=[(0, 0)])
        (o_rgb, o_disp), = run_pairs(ctx, [(left, right, p)], sb.SB_RUN_PLAIN)
        _compare_full(o_rgb, o_disp, left, right, p)
