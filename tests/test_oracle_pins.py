"""Pins of the CPU oracle against things other than itself.

Each test ties one oracle function to an independent source of truth: a
value worked by hand from the paper's text (fixtures in tests/golden/), a
published standard value, a library routine that computes the same thing by
another method (scipy.ndimage, scikit-learn), brute force on tiny inputs, a
closed form, or an invariant that a plausible slip (a dropped term, a wrong
sign or index, a transposed operand) would break.
"""
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
import synth

RNG = np.random.default_rng(12345)


def _blocks(path):
    """Parse a golden file into (tag, rows) blocks; '#' lines are comments."""
    out, cur = [], None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tok = line.split()
        if len(tok) >= 1 and not tok[0].lstrip("-").isdigit() and tok[0] != ".":
            if tok[0] in ("anchors", "expected", "column") and cur is not None:
                cur[1].append((tok[0], tok[1:]))
                continue
            cur = (line, [])
            out.append(cur)
        else:
            cur[1].append(("row", tok))
    return out


# ----------------------------------------------------------------- lightness
def test_lightness_black_white_and_published_primaries(golden_dir):
    # CIE 1976 L* of the sRGB primaries and mid grey (standard published values,
    # see tests/golden/lightness_srgb.txt), stored as round(2.55 L*).
    rows = [l.split() for l in open(os.path.join(golden_dir, "lightness_srgb.txt"))
            if l.strip() and not l.startswith("#")]
    for r, g, b, lstar in rows:
        want = int(np.floor(2.55 * float(lstar) + 0.5))
        assert oracle.lightness_of(int(r), int(g), int(b)) == want, (r, g, b, lstar)


def test_lightness_grey_ramp_monotone():
    vals = [oracle.lightness_of(v, v, v) for v in range(256)]
    assert vals[0] == 0 and vals[-1] == 255
    assert all(b >= a for a, b in zip(vals, vals[1:]))


@pytest.mark.slow
def test_lightness_all_rgb_against_fp64_definition():
    """All 2^24 RGB triples against CIE L* computed in FP64 straight from the
    sRGB and CIE 1976 definitions.  The oracle quantises linear RGB and Y to
    16 bits, so it may differ by one level, and only where the exact value is
    within the quantisation error bound of a rounding tie."""
    v = np.arange(256, dtype=np.float64) / 255.0
    lin = np.where(v <= 0.04045, v / 12.92, ((v + 0.055) / 1.055) ** 2.4)
    r, g, b = np.meshgrid(np.arange(256), np.arange(256), np.arange(256), indexing="ij")
    Y = 0.2126 * lin[r] + 0.7152 * lin[g] + 0.0722 * lin[b]
    eps = (6 / 29) ** 3
    Ls = np.where(Y > eps, 116 * np.cbrt(Y) - 16, (29 / 3) ** 3 * Y)
    exact = 2.55 * Ls
    want = np.clip(np.floor(exact + 0.5), 0, 255)
    rgb = np.stack([r, g, b], -1).astype(np.uint8).reshape(-1, 1, 3)
    got = oracle.rgb_to_lightness(rgb).reshape(256, 256, 256).astype(np.float64)
    diff = got - want
    assert np.abs(diff).max() <= 1
    bad = diff != 0
    # error bound on Y: 3 channel roundings of lin (0.5/65535 each, weighted),
    # weight rounding (< 0.5/65536 each) and the final shift (0.5/65536)
    dY = (0.5 + 1.5 + 0.5) / 65535.0
    slope = np.where(Y > eps, 116.0 / 3.0 * np.maximum(Y, eps) ** (-2.0 / 3.0), (29 / 3) ** 3)
    bound = 2.55 * slope * dY * 1.01
    dist_to_tie = np.abs((exact - np.floor(exact)) - 0.5)
    assert np.all(dist_to_tie[bad] <= bound[bad])
    assert bad.mean() < 0.02


# -------------------------------------------------------------------- kmeans
def _init_centres(hist, K):
    occ = np.flatnonzero(hist)
    lo, hi = occ[0], occ[-1]
    return np.array([lo + ((k + 0.5) * (hi - lo)) / K for k in range(K)])


def _pixelwise_lloyd(values, c, max_iter=100):
    """Textbook Lloyd on every pixel value (not on bins)."""
    c = c.copy()
    a = np.argmin(np.abs(values[:, None] - c[None, :]), axis=1)
    for _ in range(max_iter):
        for k in range(len(c)):
            sel = values[a == k]
            if sel.size:
                c[k] = float(np.sum(sel.astype(np.int64))) / float(sel.size)
        a2 = np.argmin(np.abs(values[:, None] - c[None, :]), axis=1)
        if np.array_equal(a, a2):
            break
        a = a2
    return c, a


@pytest.mark.parametrize("K", [1, 2, 4, 7, 10])
def test_kmeans_histogram_equals_pixelwise(K):
    """Section III: clustering the histogram bins gives the same centres and
    per-pixel clusters as clustering every pixel value."""
    vals = np.concatenate([RNG.normal(m, s, 700) for m, s in ((40, 9), (110, 15), (170, 7), (220, 10))])
    L = np.clip(np.round(vals), 0, 255).astype(np.uint8)
    hist = oracle.histogram(L)
    assert np.array_equal(hist, np.bincount(L, minlength=256))
    c, lut, it = oracle.kmeans_hist(hist, K, 100)
    cp, ap = _pixelwise_lloyd(L.astype(np.float64), _init_centres(hist, K))
    assert np.array_equal(c, cp)            # exact: same integer sums, one division
    assert np.array_equal(lut[L], ap)


@pytest.mark.parametrize("K", [2, 3, 5, 8])
def test_kmeans_matches_sklearn_lloyd(K):
    from sklearn.cluster import KMeans
    L = np.clip(RNG.gamma(3.0, 30.0, 5000), 0, 255).astype(np.uint8)
    hist = oracle.histogram(L)
    c, lut, _ = oracle.kmeans_hist(hist, K, 300)
    bins = np.flatnonzero(hist)
    km = KMeans(n_clusters=K, init=_init_centres(hist, K).reshape(-1, 1), n_init=1, max_iter=300,
                tol=0.0, algorithm="lloyd")
    km.fit(bins.reshape(-1, 1).astype(np.float64), sample_weight=hist[bins].astype(np.float64))
    np.testing.assert_allclose(c, km.cluster_centers_[:, 0], rtol=0, atol=1e-9)
    # labels equal except at bins (nearly) equidistant from two centres
    d = np.abs(bins[:, None] - c[None, :])
    ds = np.sort(d, axis=1)
    clear = (ds[:, 1] - ds[:, 0]) > 1e-9 if K > 1 else np.ones(len(bins), bool)
    assert np.array_equal(lut[bins][clear], km.labels_[clear])


def test_kmeans_k1_is_mean_and_flat_levels_are_found():
    L = RNG.integers(0, 256, 3001).astype(np.uint8)
    c, lut, _ = oracle.kmeans_hist(oracle.histogram(L), 1)
    assert c[0] == float(L.astype(np.int64).sum()) / L.size
    assert not lut.any()
    levels = [20, 90, 160, 230]
    L = np.repeat(np.array(levels, np.uint8), [50, 70, 90, 110])
    c, lut, _ = oracle.kmeans_hist(oracle.histogram(L), 4)
    assert sorted(c.tolist()) == [float(v) for v in levels]
    assert len(set(lut[levels].tolist())) == 4


def test_kmeans_empty_image():
    c, lut, it = oracle.kmeans_hist(np.zeros(256, np.uint32), 3)
    assert it == 0 and not lut.any() and not c.any()


# ------------------------------------------------------------------ boundary
def test_boundary_rectangle_is_two_pixel_ring():
    for (w, h, x0, y0, rw, rh) in ((20, 15, 4, 3, 7, 5), (33, 21, 1, 1, 30, 18), (9, 9, 3, 3, 1, 1)):
        lab = np.zeros((h, w), np.uint8)
        lab[y0:y0 + rh, x0:x0 + rw] = 1
        b = oracle.boundary(lab)
        inner = 2 * (rw + rh) - 4 if rw > 1 and rh > 1 else rw * rh
        outer = 2 * (rw + 2) + 2 * (rh + 2) - 4
        assert int(b.sum()) == inner + outer


@pytest.mark.parametrize("K", [2, 3, 6])
def test_boundary_matches_min_max_filters(K):
    lab = RNG.integers(0, K, (37, 51)).astype(np.uint8)
    lab = ndi.median_filter(lab, 3)           # some structure
    b = oracle.boundary(lab)
    mx = ndi.maximum_filter(lab, 3, mode="nearest")
    mn = ndi.minimum_filter(lab, 3, mode="nearest")
    assert np.array_equal(b.astype(bool), (mx != lab) | (mn != lab))


# --------------------------------------------------------------- morphology
def test_fill_remove_paper_pattern(golden_dir):
    blocks = _blocks(os.path.join(golden_dir, "fill_pattern.txt"))
    m = {tag: np.array([[int(v) for v in r] for _, r in rows], np.uint8) for tag, rows in blocks}
    assert np.array_equal(oracle.morph_fill(m["input"]), m["fill"])
    assert np.array_equal(oracle.morph_remove(m["fill"]), m["remove"])


@pytest.mark.parametrize("p", [0.3, 0.5, 0.7, 0.9])
def test_fill_remove_match_scipy(p):
    b = (RNG.random((41, 57)) < p).astype(np.uint8)
    ring = np.ones((3, 3), bool)
    ring[1, 1] = False
    centre = np.zeros((3, 3), bool)
    centre[1, 1] = True
    want_fill = b.astype(bool) | ndi.binary_hit_or_miss(b, structure1=ring, structure2=centre)
    assert np.array_equal(oracle.morph_fill(b).astype(bool), want_fill)
    cross = ndi.generate_binary_structure(2, 1)
    want_rem = b.astype(bool) & ~ndi.binary_erosion(b, structure=cross, border_value=0)
    assert np.array_equal(oracle.morph_remove(b).astype(bool), want_rem)


@pytest.mark.parametrize("p", [0.2, 0.5, 0.8])
def test_open_close_matches_scipy_and_is_idempotent(p):
    b = (RNG.random((40, 45)) < p).astype(np.uint8)
    sq = np.ones((3, 3), bool)
    e = ndi.binary_erosion(b, sq, border_value=1)
    o = ndi.binary_dilation(e, sq, border_value=0)
    d = ndi.binary_dilation(o, sq, border_value=0)
    want = ndi.binary_erosion(d, sq, border_value=1)
    got = oracle.morph_open_close(b)
    assert np.array_equal(got.astype(bool), want)
    assert np.array_equal(oracle.morph_open_close(got), got)


# ----------------------------------------------------------------------- CCA
@pytest.mark.parametrize("p", [0.1, 0.35, 0.5, 0.6])
def test_cca_matches_scipy_label(p):
    b = (RNG.random((63, 77)) < p).astype(np.uint8)
    lab, n = oracle.cca(b)
    sl, sn = ndi.label(b, structure=np.ones((3, 3)))
    assert n == sn
    assert np.array_equal(lab < 0, b == 0)
    # same partition, and each label is its component's smallest linear index
    idx = np.arange(b.size).reshape(b.shape)
    for comp in range(1, sn + 1):
        sel = sl == comp
        assert len(np.unique(lab[sel])) == 1
        assert lab[sel][0] == idx[sel].min()


def test_cc_filter_hand_case():
    # components of sizes 1, 1, 2, 3, 40, 60 (N_b = 107): floor(0.04*107) = 4,
    # so the two singletons and the size-2 component go (total 4) and the
    # size-3 one stays (total would be 7).
    w, h = 40, 12
    b = np.zeros((h, w), np.uint8)
    b[0, 0] = 1                      # size 1, label 0
    b[0, 10] = 1                     # size 1, label 10
    b[2, 5:7] = 1                    # size 2
    b[4, 20:23] = 1                  # size 3
    b[6, 0:40] = 1                   # size 40
    b[8:11, 0:20] = 1                # size 60
    lab, n = oracle.cca(b)
    assert n == 6 and b.sum() == 107
    out = oracle.cc_filter(b, lab, 0.04)
    want = b.copy()
    want[0, 0] = want[0, 10] = 0
    want[2, 5:7] = 0
    assert np.array_equal(out, want)
    # ties in size broken by label: with a limit of 1 only the first singleton goes
    out1 = oracle.cc_filter(b, lab, 1.0 / 107 + 1e-12)
    assert out1[0, 0] == 0 and out1[0, 10] == 1


@pytest.mark.parametrize("frac", [0.02, 0.04, 0.1, 0.3])
def test_cc_filter_properties(frac):
    b = (RNG.random((50, 60)) < 0.3).astype(np.uint8)
    lab, n = oracle.cca(b)
    out = oracle.cc_filter(b, lab, frac)
    nb = int(b.sum())
    limit = int(np.floor(frac * nb))
    sizes = {int(l): int((lab == l).sum()) for l in np.unique(lab[lab >= 0])}
    removed = {l for l in sizes if not out[lab == l].any()}
    kept = set(sizes) - removed
    assert np.array_equal(out.astype(bool), b.astype(bool) & np.isin(lab, list(kept)))
    S = sum(sizes[l] for l in removed)
    assert S <= limit
    if kept:
        nxt = min(kept, key=lambda l: (sizes[l], l))
        assert S + sizes[nxt] > limit
        for l in removed:                       # removed ones come first in (size, label) order
            assert (sizes[l], l) < (sizes[nxt], nxt)


# ------------------------------------------------------------------------ SAD
def _sad_volume(Ll, Lr, D, B):
    """All SAD costs by summed-area tables (an independent formulation)."""
    h, w = Ll.shape
    r = (B - 1) // 2
    vol = np.full((D + 1, h, w), -1, np.int64)
    for d in range(D + 1):
        ad = np.zeros((h, w), np.int64)
        ad[:, d:] = np.abs(Ll[:, d:].astype(np.int64) - Lr[:, :w - d].astype(np.int64))
        I = np.zeros((h + 1, w + 1), np.int64)
        I[1:, 1:] = ad.cumsum(0).cumsum(1)
        s = I[B:, B:] - I[:-B, B:] - I[B:, :-B] + I[:-B, :-B]
        vol[d, r:h - r, r:w - r] = s
    return vol


@pytest.mark.parametrize("D,B", [(4, 3), (7, 5), (12, 9), (0, 1), (3, 1)])
def test_sad_matches_summed_area_brute_force(D, B):
    h, w = 21, 30
    Ll = RNG.integers(0, 256, (h, w)).astype(np.uint8)
    Lr = RNG.integers(0, 256, (h, w)).astype(np.uint8)
    Lr[:, :] = np.roll(Ll, -2, axis=1) // 2 + Lr // 2
    anchor = oracle.anchor_mask(np.ones((h, w), np.uint8), D, B)
    disp, cost = oracle.boundary_sad(Ll, Lr, anchor, D, B)
    vol = _sad_volume(Ll, Lr, D, B)
    ys, xs = np.nonzero(anchor)
    assert len(ys) == (h - (B - 1)) * (w - (B - 1) - D)
    for y, x in zip(ys, xs):
        col = vol[:, y, x]
        assert col.min() >= 0
        assert cost[y, x] == col.min()
        assert disp[y, x] == int(np.argmin(col))   # first minimum = smallest d
    assert np.all(disp[anchor == 0] == oracle.UNDET)


def test_anchor_mask_domain_and_border_columns():
    h, w, D, B = 20, 40, 10, 5
    r = 2
    b = np.zeros((h, w), np.uint8)
    b[5, 20] = 1
    b[0, 20] = 1             # outside Omega (row < r)
    b[6, 5] = 1              # outside Omega (x < D + r)
    a = oracle.anchor_mask(b, D, B)
    want = np.zeros_like(b)
    want[r:h - r, D + r] = 1
    want[r:h - r, w - 1 - r] = 1
    want[5, 20] = 1
    assert np.array_equal(a, want)


def test_sad_recovers_constant_disparity_of_noise_free_texture():
    h, w, D, B, d0 = 30, 60, 12, 7, 5
    Ll = RNG.integers(0, 256, (h, w)).astype(np.uint8)
    Lr = np.zeros_like(Ll)
    Lr[:, :w - d0] = Ll[:, d0:]              # right image = left shifted left by d0
    Lr[:, w - d0:] = RNG.integers(0, 256, (h, d0))
    anchor = oracle.anchor_mask(np.ones((h, w), np.uint8), D, B)
    disp, cost = oracle.boundary_sad(Ll, Lr, anchor, D, B)
    r = (B - 1) // 2
    # windows whose right-image samples all stay inside the copied region
    ok = anchor.astype(bool).copy()
    ok[:, w - d0 - r:] = False
    assert np.all(disp[ok] == d0) and np.all(cost[ok] == 0)


# ------------------------------------------------------------ reconstruction
def _parse_row(tok):
    return [oracle.UNDET if t == "." else int(t) for t in tok]


def test_algorithm1_hand_rows(golden_dir):
    for tag, rows in _blocks(os.path.join(golden_dir, "alg1_rows.txt")):
        d = dict(rows)
        a = np.array([_parse_row(d["anchors"])], np.uint16)
        e = np.array([_parse_row(d["expected"])], np.uint16)
        anchor = (a != oracle.UNDET).astype(np.uint8)
        assert np.array_equal(oracle.recon_fill(a, anchor), e), tag


def test_algorithm2_hand_columns(golden_dir):
    for tag, rows in _blocks(os.path.join(golden_dir, "alg2_columns.txt")):
        T = int(tag.split("T=")[1])
        d = dict(rows)
        col = np.array(_parse_row(d["column"]), np.uint16).reshape(-1, 1)
        e = np.array(_parse_row(d["expected"]), np.uint16).reshape(-1, 1)
        got = oracle.recon_peek(col, 0, 1, T)        # D = 0, block 1: Omega is the whole column
        assert np.array_equal(got, e), tag


def test_algorithm2_inplace_paper_columns(golden_dir):
    for tag, rows in _blocks(os.path.join(golden_dir, "alg2_inplace_columns.txt")):
        T = int(tag.split("T=")[1])
        d = dict(rows)
        col = np.array(_parse_row(d["column"]), np.uint16).reshape(-1, 1)
        e = np.array(_parse_row(d["expected"]), np.uint16).reshape(-1, 1)
        got = oracle.recon_peek_inplace(col, 0, 1, T)
        assert np.array_equal(got, e), tag


def test_algorithm2_inplace_properties():
    # T = -1 (always the minimum): an estimate equals min(above, below) of the
    # snapshot reading, so both readings agree; for any T the in-place
    # estimates between two determined pixels move monotonically from the
    # upper value towards the lower one and stay between them, and the first
    # one equals the snapshot estimate
    h, w, D, B = 60, 30, 4, 5
    r = (B - 1) // 2
    for trial in range(20):
        det = np.full((h, w), oracle.UNDET, np.uint16)
        for x in range(w):
            k = int(RNG.integers(0, 8))
            ys = RNG.choice(h, k, replace=False)
            det[ys, x] = RNG.integers(0, 200, k)
        assert np.array_equal(oracle.recon_peek_inplace(det, D, B, -1), oracle.recon_peek(det, D, B, -1))
        T = int(RNG.integers(0, 40))
        ip, sn = oracle.recon_peek_inplace(det, D, B, T), oracle.recon_peek(det, D, B, T)
        for x in range(D + r, w - r):
            ys = [y for y in range(r, h - r) if det[y, x] != oracle.UNDET]
            for y0, y1 in zip(ys, ys[1:]):
                a, b = int(det[y0, x]), int(det[y1, x])
                run = [int(v) for v in ip[y0 + 1:y1, x]]
                if not run:
                    continue
                assert run[0] == int(sn[y0 + 1, x])
                lo, hi = min(a, b), max(a, b)
                assert all(lo <= v <= hi for v in run)
                prev = a
                for v in run:
                    assert abs(b - v) <= abs(b - prev)
                    prev = v
        outside = np.ones((h, w), bool)
        outside[r:h - r, D + r:w - r] = False
        assert np.all(ip[outside] == 0)
        inside = ~outside & (det != oracle.UNDET)
        assert np.array_equal(ip[inside], det[inside])


def test_algorithm2_threshold_extremes():
    det = np.full((40, 9), oracle.UNDET, np.uint16)
    for x in range(9):
        ys = np.sort(RNG.choice(40, 6, replace=False))
        det[ys, x] = RNG.integers(0, 60, 6)
    hi = oracle.recon_peek(det, 0, 1, 10 ** 6)        # range never above T: floor mean
    lo = oracle.recon_peek(det, 0, 1, -1)             # range always above T: minimum
    for x in range(9):
        ys = np.flatnonzero(det[:, x] != oracle.UNDET)
        for y in range(40):
            if det[y, x] != oracle.UNDET:
                assert hi[y, x] == lo[y, x] == det[y, x]
                continue
            up = [v for v in ys if v < y]
            dn = [v for v in ys if v > y]
            a = int(det[up[-1], x]) if up else None
            c = int(det[dn[0], x]) if dn else None
            if a is not None and c is not None:
                assert hi[y, x] == (a + c) // 2 and lo[y, x] == min(a, c)
            else:
                assert hi[y, x] == lo[y, x] == (a if a is not None else c)


def test_peek_outside_omega_is_zero_and_uses_omega_only():
    h, w, D, B = 12, 20, 4, 3
    det = np.full((h, w), oracle.UNDET, np.uint16)
    det[0, 10] = 50           # outside Omega (row 0 < r = 1): never used
    det[5, 10] = 7
    out = oracle.recon_peek(det, D, B, 1)
    assert out[0, 10] == 0 and out[1, 10] == 7 and out[10, 10] == 7
    assert not out[:, :D + 1].any() and not out[:, w - 1:].any()


# ---------------------------------------------------------------------- blur
@pytest.mark.parametrize("sigma", [0.6, 1.0, 2.0, 3.0, 5.0, 8.0, 2.37])
def test_gaussian_kernel_sums_to_one_and_is_separable(sigma):
    k2 = oracle.gauss_kernel(sigma)
    R = oracle.blur_radius(sigma)
    assert R == int(np.ceil(3 * sigma)) and k2.shape == (2 * R + 1, 2 * R + 1)
    assert abs(k2.sum() - 1.0) < 1e-12
    s = float(np.float32(sigma))                      # sigma crosses the interface as a float
    g = np.exp(-np.arange(-R, R + 1) ** 2 / (2.0 * s * s))
    g /= g.sum()
    np.testing.assert_allclose(k2, np.outer(g, g), rtol=0, atol=1e-15)
    assert np.allclose(k2, k2.T) and k2[R, R] == k2.max()


@pytest.mark.parametrize("sigma", [1.0, 2.5, 4.0])
def test_blur_matches_scipy_gaussian_filter(sigma):
    rgb = RNG.integers(0, 256, (23, 29, 3)).astype(np.uint8)
    disp = np.zeros((23, 29), np.uint16)
    out = oracle.selective_blur(rgb, disp, [], sigma)          # no interest range: blur all
    R = oracle.blur_radius(sigma)
    ref = np.stack([ndi.gaussian_filter(rgb[..., c].astype(np.float64), sigma, mode="nearest",
                                        truncate=R / sigma) for c in range(3)], -1)
    want = np.clip(np.floor(ref + 0.5), 0, 255)
    near_tie = np.abs(ref - np.floor(ref) - 0.5) < 1e-9
    assert np.all((out == want) | near_tie)


def test_blur_constant_image_unchanged_and_in_focus_copied():
    rgb = np.full((17, 19, 3), 77, np.uint8)
    rgb[..., 1] = 200
    disp = np.zeros((17, 19), np.uint16)
    assert np.array_equal(oracle.selective_blur(rgb, disp, [], 3.0), rgb)
    img = RNG.integers(0, 256, (17, 19, 3)).astype(np.uint8)
    disp = RNG.integers(0, 30, (17, 19)).astype(np.uint16)
    out = oracle.selective_blur(img, disp, [(5, 9), (20, 22)], 2.0)
    keep = ((disp >= 5) & (disp <= 9)) | ((disp >= 20) & (disp <= 22))
    assert np.array_equal(out[keep], img[keep])
    blurred = oracle.selective_blur(img, disp, [], 2.0)
    assert np.array_equal(out[~keep], blurred[~keep])


def test_blur_impulse_response_is_kernel():
    sigma, R = 2.0, 6
    img = np.zeros((2 * R + 9, 2 * R + 9, 3), np.uint8)
    c = R + 4
    img[c, c, :] = 255
    out = oracle.selective_blur(img, np.zeros(img.shape[:2], np.uint16), [], sigma)
    k = oracle.gauss_kernel(sigma)
    want = np.floor(255.0 * k + 0.5)
    assert np.array_equal(out[c - R:c + R + 1, c - R:c + R + 1, 0], want.astype(np.uint8))
    for y, x in ((c, c), (c - 3, c + 1)):
        assert np.array_equal(oracle.blur_at(img, x, y, sigma), out[y, x])


def test_right_view_matches_direct_right_referenced_sad():
    # the right view runs the method on the mirrored, swapped pair; its SAD
    # at every anchor must equal the right-referenced SAD written out directly
    # (argmin_d sum |R(x+j) - L(x+j+d)|) at the mirrored position
    import dataclasses
    sc, p, _ = synth.workload("c1")
    left, right, _ = sc.render()
    left, right = left[:64, :160].copy(), right[:64, :160].copy()
    p = dataclasses.replace(p, max_disp=12, block=5, view=1)
    res = oracle.run(left, right, p, with_blur=False)
    Ll, Lr = oracle.rgb_to_lightness(left), oracle.rgb_to_lightness(right)
    h, w = Ll.shape
    ys, xs = np.nonzero(res.anchor)
    assert len(ys) > 50
    for i in RNG.choice(len(ys), 60, replace=False):
        y, xm = int(ys[i]), int(xs[i])
        d, c = oracle.sad_argmin_right(Ll, Lr, w - 1 - xm, y, p.max_disp, p.block)
        assert (int(res.disp_sparse[y, xm]), int(res.cost[y, xm])) == (d, c)
    assert res.disp.shape == (h, w) and np.all(res.disp[:, w - p.max_disp - 2:] == 0)


def test_lr_consistency_hand_worked_row():
    # one row, worked by hand: left pixel x matches right pixel x - dL[x]
    dL = np.array([[0, 1, 2, 2, 5, 1]], np.uint16)
    dR = np.array([[0, 1, 2, 1, 0, 0]], np.uint16)
    ok0, n0 = oracle.lr_consistency(dL, dR, 0)
    ok1, n1 = oracle.lr_consistency(dL, dR, 1)
    assert ok0.tolist() == [[1, 0, 0, 0, 0, 0]] and n0 == 1
    assert ok1.tolist() == [[1, 1, 0, 1, 0, 1]] and n1 == 4

