"""Child process of the bounds-checked library's GPU test (run with
SB_LIBRARY=checks): the probe's failure is reported and cleared, then every
stage runs on ragged and dense inputs and on whole pipelines with no check
failing, and every output equals the oracle's.  Prints "ok" at the end."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import synth  # noqa: E402
import paper_2001_07809_b300 as sb  # noqa: E402
from gpu_helpers import refine, run_pairs, sad  # noqa: E402


def main():
    assert sb.sb_checks_built(), sb.library_path()
    rng = np.random.default_rng(11)
    with sb.Context(0) as ctx:
        # the reporting path: a passing probe, a failing one (site 1), cleared
        ctx.check_probe(False)
        ctx.synchronize()
        ctx.check_probe(True)
        try:
            ctx.synchronize()
            raise AssertionError("the failing probe was not reported")
        except sb.SbError as e:
            assert e.status == sb.SB_ERR_CHECK and "site 1 " in str(e), str(e)
        ctx.synchronize()

        # connected components on dense noisy maps and a ragged image
        for (h, w), noise in (((211, 389), 0.7), ((97, 131), 0.3)):
            lab = rng.integers(0, 2, (h // 3 + 1, w // 3 + 1))
            lab = np.kron(lab, np.ones((3, 3), np.int64))[:h, :w]
            lab = np.where(rng.random((h, w)) < noise, rng.integers(0, 3, (h, w)), lab).astype(np.uint8)
            ref, cc, bnd = refine(ctx, lab, 1, 0.04)
            o_ref = oracle.refine(oracle.boundary(lab), 1)
            o_cc, _ = oracle.cca(o_ref)
            assert np.array_equal(ref, o_ref) and np.array_equal(cc, o_cc)
            assert np.array_equal(bnd, oracle.cc_filter(o_ref, o_cc, 0.04))

        # SAD: box sums with a partial chunk and a tail, and the direct kernel
        for (h, w, D, B, variant) in ((70, 333, 40, 9, sb.SB_SAD_BOXSUM), (64, 400, 128, 15, sb.SB_SAD_BOXSUM),
                                      (50, 300, 64, 11, sb.SB_SAD_DIRECT)):
            Ll = rng.integers(0, 256, (h, w)).astype(np.uint8)
            Lr = np.clip(np.roll(Ll, -5, axis=1).astype(int) + rng.integers(-6, 7, (h, w)), 0, 255).astype(np.uint8)
            bmap = (rng.random((h, w)) < 0.2).astype(np.uint8)
            d, c = sad(ctx, Ll, Lr, bmap, D, B, variant)
            want_d, want_c = oracle.boundary_sad(Ll, Lr, oracle.anchor_mask(bmap, D, B), D, B)
            assert np.array_equal(d, want_d) and np.array_equal(c, want_c), (h, w, D, B)
        ctx.synchronize()

        # whole pipelines, plain and batched
        sc, p, _ = synth.workload("c1")
        left, right, _ = sc.render()
        want = oracle.run(left, right, p)
        for flags in (sb.SB_RUN_PLAIN, sb.SB_RUN_BATCHED):
            (out, disp), = run_pairs(ctx, [(left, right, p)], flags)
            assert np.array_equal(disp, want.disp)
            assert np.abs(out.astype(int) - want.out_rgb.astype(int)).max() <= 1
        ctx.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
