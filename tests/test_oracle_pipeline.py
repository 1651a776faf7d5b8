"""Oracle pipeline checks: the point evaluator used for sampled full-size
parity agrees with the whole-image pipeline; the pipeline recovers the known
disparities of synthetic scenes; the input generator is deterministic."""
import numpy as np
import pytest

import oracle
import synth


def _small_scene(seed, w=150, h=90, noise=256):
    r = synth.Rng(seed)
    layers = [synth.Layer(0, w // 2, h // 2, w, h, 3 * 256, 60, 70, r.u64() & 0xFFFFFFFF)]
    for i, d in enumerate((7, 12)):
        layers.append(synth.Layer(1, r.randint(40, w - 30), r.randint(25, h - 25), r.randint(12, 25),
                                  r.randint(10, 20), d * 256, 120 + 60 * i, 70, r.u64() & 0xFFFFFFFF))
    return synth.Scene(w, h, layers, noise_q8=noise, noise_seed=r.u64())


@pytest.mark.parametrize("seed,T", [(3, 1), (4, 0), (5, 6)])
def test_point_evaluator_equals_full_pipeline(seed, T):
    sc = _small_scene(seed)
    left, right, _ = sc.render(n_threads=1)
    p = synth.Params(k=4, max_disp=16, block=7, sigma=2.0, ranges=[(8, 16)], disp_threshold=T)
    full = oracle.run(left, right, p, with_blur=False)
    front = oracle.run_front(left, right, p)
    h, w = full.disp.shape
    pts = [(x, y) for y in range(h) for x in range(0, w, 3)]
    got = oracle.disp_at_points(front, p, pts)
    want = [int(full.disp[y, x]) for x, y in pts]
    assert got == want


def test_pipeline_recovers_layer_disparities_noise_free():
    sc = _small_scene(11, w=200, h=120, noise=0)
    left, right, gt = sc.render(n_threads=1)
    p = synth.Params(k=4, max_disp=16, block=7, sigma=2.0, ranges=[(8, 16)])
    res = oracle.run(left, right, p)
    r = 3
    # anchors whose window lies on one fronto-parallel layer that no nearer
    # layer can occlude in the right image (nearer layers shift left by up to
    # max_disp, so the strip up to max_disp right of the window must agree)
    gi = np.rint(gt).astype(int)
    good = 0
    ys, xs = np.nonzero(res.anchor)
    for y, x in zip(ys, xs):
        win = gi[y - r:y + r + 1, x - r:x + r + 1]
        d = gi[y, x]
        if (win == d).all() and (gi[y - r:y + r + 1, x - r:x + r + p.max_disp + 1] == d).all():
            good += 1
            assert res.disp_sparse[y, x] == d
    assert good > 50
    assert res.out_rgb.shape == left.shape


def test_c1_pipeline_statistics():
    sc, p, _ = synth.workload("c1")
    left, right, gt = sc.render()
    res = oracle.run(left, right, p)
    r = (p.block - 1) // 2
    mask = np.zeros(gt.shape, bool)
    mask[r:-r, p.max_disp + r:-r] = True
    density = res.anchor.mean()
    assert 0.10 < density < 0.30                   # the paper reports 16-19 %
    assert oracle.bad_pixel_percent(res.disp, gt, mask) < 25.0
    assert set(np.unique(res.disp[mask])) <= set(range(p.max_disp + 1))


def test_generator_deterministic_and_thread_independent():
    sc = _small_scene(21)
    a = sc.render(n_threads=1)
    b = sc.render(n_threads=5)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    sc3 = synth.scene_c3()
    assert sc3.w == 4096 and len(sc3.layers) == 12
    assert synth.splitmix64(0) == synth._lib().synth_splitmix64(0)
