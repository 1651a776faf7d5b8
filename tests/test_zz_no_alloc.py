"""The allocation-free boundary SAD entry point (sb_boundary_sad_static).

Some callers cannot allocate device memory: a plug-in inside a host
application that owns all device memory through its own pool, or a
real-time loop that must never call cudaMalloc.  For them the library keeps
the SAD scratch in a static device array.  These tests call that entry point
through the C ABI and check it against sb_boundary_sad on two calls in a row
(the second call must not see the first call's scratch contents).  This file
is collected last so a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2001_07809_b300 as sb  # noqa: E402
from gpu_helpers import dev, host, sad  # noqa: E402

pytestmark = pytest.mark.gpu


def _static_fn():
    lib = ctypes.CDLL(sb.library_path())
    f = lib.sb_boundary_sad_static
    V, I32 = ctypes.c_void_p, ctypes.c_int32
    f.argtypes = [V, V, V, I32, I32, I32, I32, I32, V, V, V, ctypes.c_char_p, ctypes.c_size_t]
    f.restype = ctypes.c_int
    return f


def _call_static(f, Ll, Lr, bmap, D, B, variant):
    h, w = Ll.shape
    dl, dr, db = dev(Ll), dev(Lr), dev(bmap)
    disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    cost = torch.empty((h, w), dtype=torch.int32, device="cuda")
    err = ctypes.create_string_buffer(256)
    st = f(dl.data_ptr(), dr.data_ptr(), db.data_ptr(), w, h, D, B, variant, disp.data_ptr(), cost.data_ptr(),
           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), err, 256)
    assert st == 0, err.value
    torch.cuda.synchronize()
    return host(disp, np.uint16), host(cost, np.uint32)


@pytest.mark.parametrize("variant", [sb.SB_SAD_BOXSUM, sb.SB_SAD_DIRECT, sb.SB_SAD_AUTO])
def test_static_entry_matches_context_entry_twice(variant):
    rng = np.random.default_rng(77 + variant)
    f = _static_fn()
    ctx = sb.Context(0)
    try:
        for (h, w, D, B) in ((90, 500, 64, 15), (61, 333, 40, 9)):    # two calls in a row, different sizes
            Ll = rng.integers(0, 256, (h, w)).astype(np.uint8)
            Lr = np.clip(np.roll(Ll, -5, axis=1).astype(int) + rng.integers(-5, 6, (h, w)), 0, 255).astype(np.uint8)
            bmap = (rng.random((h, w)) < 0.2).astype(np.uint8)
            got_d, got_c = _call_static(f, Ll, Lr, bmap, D, B, variant)
            want_d, want_c = sad(ctx, Ll, Lr, bmap, D, B, variant)
            assert np.array_equal(got_d, want_d)
            assert np.array_equal(got_c, want_c)
    finally:
        ctx.close()


# disparity ranges around the chunk of 64 (a partial chunk, whole chunks, a
# tail of 1..8 disparities, a remainder of 9 taken by the box sums), D = 0 and
# block 1, widths with and without the 16-byte row phase, several row bands
STATIC_CASES = [
    (40, 160, 63, 9), (45, 171, 64, 9), (45, 176, 65, 9), (50, 272, 127, 11), (33, 301, 128, 7),
    (64, 480, 200, 15), (48, 560, 256, 21), (31, 97, 0, 1), (26, 90, 7, 1), (200, 304, 72, 41),
]


@pytest.mark.parametrize("h,w,D,B", STATIC_CASES)
def test_static_entry_equals_oracle(h, w, D, B):
    import oracle
    rng = np.random.default_rng(h * 7919 + w * 31 + D)
    f = _static_fn()
    Ll = rng.integers(0, 256, (h, w)).astype(np.uint8)
    Lr = np.clip(np.roll(Ll, -(D // 3), axis=1).astype(int) + rng.integers(-6, 7, (h, w)), 0, 255).astype(np.uint8)
    bmap = (rng.random((h, w)) < 0.25).astype(np.uint8)
    want_d, want_c = oracle.boundary_sad(Ll, Lr, oracle.anchor_mask(bmap, D, B), D, B)
    for variant in (sb.SB_SAD_BOXSUM, sb.SB_SAD_DIRECT):
        got_d, got_c = _call_static(f, Ll, Lr, bmap, D, B, variant)
        assert np.array_equal(got_d, want_d), variant
        assert np.array_equal(got_c, want_c), variant


def test_static_entry_rejects_images_above_the_limit():
    f = _static_fn()
    h, w = 2049, 2049                       # 4,198,401 pixels > 4,194,304
    err = ctypes.create_string_buffer(256)
    t = torch.zeros(1, dtype=torch.uint8, device="cuda")
    st = f(t.data_ptr(), t.data_ptr(), t.data_ptr(), w, h, 16, 5, 0, t.data_ptr(), None, None, err, 256)
    assert st == 1 and b"static scratch limit" in err.value


def test_static_entry_rejects_too_many_work_items():
    # inside the pixel limit, but a very wide, short image with a large disparity
    # range needs more work items than the static descriptor area holds
    f = _static_fn()
    h, w, D, B = 4, 1048576, 1023, 3        # 4,194,304 pixels; 74,832 work items
    err = ctypes.create_string_buffer(256)
    t = torch.zeros(1, dtype=torch.uint8, device="cuda")
    st = f(t.data_ptr(), t.data_ptr(), t.data_ptr(), w, h, D, B, sb.SB_SAD_BOXSUM, t.data_ptr(), None, None, err, 256)
    assert st == 5 and b"work items" in err.value


def test_static_entry_in_two_driver_contexts():
    import multiprocessing as mp

    import noalloc_child
    import oracle

    rng = np.random.default_rng(5)
    h, w, D, B = 80, 420, 64, 15
    Ll = rng.integers(0, 256, (h, w)).astype(np.uint8)
    Lr = np.clip(np.roll(Ll, -4, axis=1).astype(int) + rng.integers(-5, 6, (h, w)), 0, 255).astype(np.uint8)
    bmap = (rng.random((h, w)) < 0.2).astype(np.uint8)
    want_d, want_c = oracle.boundary_sad(Ll, Lr, oracle.anchor_mask(bmap, D, B), D, B)
    q = mp.get_context("spawn").Queue()
    p = mp.get_context("spawn").Process(target=noalloc_child.two_contexts, args=(sb.library_path(), Ll, Lr, bmap, D, B, q))
    p.start()
    status, res = q.get(timeout=300)
    p.join(timeout=60)
    assert status == "ok", res
    for disp, cost in res:
        assert np.array_equal(disp, want_d) and np.array_equal(cost, want_c)
