"""The continuous-batching server: every result equals the same pair run
alone, requests that arrive while batches are on the GPU are admitted and
batched, and the device-memory budget is enforced."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import synth  # noqa: E402
import paper_2001_07809_b300 as sb  # noqa: E402
from paper_2001_07809_b300.serve import Server, percentile, request_bytes  # noqa: E402
from gpu_helpers import params_of, run_pairs  # noqa: E402

pytestmark = pytest.mark.gpu


def _requests(n):
    out = []
    for i in range(n):
        r = synth.Rng(900 + i)
        w, h = ((640, 480), (960, 540), (1280, 720))[i % 3]
        D = (64, 96, 128)[i % 3]
        sc = synth.Scene(w, h, synth._c2_style_layers(r, w, h, D, contrast=r.randint(20, 60)), noise_q8=512,
                         noise_seed=r.u64())
        left, right, _ = sc.render(want_gt=False)
        p = synth.Params(k=(4, 6, 8)[i % 3], max_disp=D, block=(9, 15, 25)[i % 3], sigma=2.0 + i % 5,
                         ranges=[(D // 4, D // 2)])
        out.append((left, right, p))
    return out


def test_served_results_equal_alone_and_in_the_mix():
    reqs = _requests(18)
    ctx = sb.Context(0)
    alone = [run_pairs(ctx, [item], sb.SB_RUN_PLAIN)[0] for item in reqs]
    ctx.close()
    pinned = [(torch.from_numpy(l).pin_memory(), torch.from_numpy(r).pin_memory(), params_of(p)) for l, r, p in reqs]
    srv = Server(0, mem_budget_bytes=2 << 30, max_batch=8)
    futs = []
    for i, (hl, hr, p) in enumerate(pinned):
        futs.append(srv.submit(hl, hr, p))
        if i % 6 == 5:
            time.sleep(0.005)           # bursts arrive while earlier batches run
    res = [f.result(timeout=120) for f in futs]
    lat = srv.latencies()
    batches = srv.batches
    srv.close()
    for (o_rgb, o_disp), (a_rgb, a_disp) in zip(res, alone):
        assert np.array_equal(o_rgb.numpy(), a_rgb)
        assert np.array_equal(o_disp.numpy().view(np.uint16), a_disp)
    assert len(lat) == len(reqs) and percentile(lat, 99) >= percentile(lat, 50) > 0
    assert batches < len(reqs)          # requests were batched


def test_budget_rejects_oversized_request_and_keeps_serving():
    srv = Server(0, mem_budget_bytes=request_bytes(480, 640) + 1000, max_batch=4)
    big = torch.zeros((1080, 1920, 3), dtype=torch.uint8).pin_memory()
    f = srv.submit(big, big, sb.make_params(max_disp=64, block=9, k=4, sigma=2.0))
    with pytest.raises(MemoryError):
        f.result(timeout=10)
    (left, right, p), = _requests(1)
    g = srv.submit(torch.from_numpy(left).pin_memory(), torch.from_numpy(right).pin_memory(), params_of(p))
    out_rgb, out_disp = g.result(timeout=60)
    srv.close()
    assert out_rgb.shape == left.shape


def test_cancel_drops_a_waiting_request():
    # a budget that admits one request at a time keeps the later ones queued:
    # the last one is cancelled while it waits, the others complete, and the
    # server keeps serving
    reqs = _requests(4)
    srv = Server(0, mem_budget_bytes=request_bytes(720, 1280) + 1000, max_batch=4)
    pinned = [(torch.from_numpy(l).pin_memory(), torch.from_numpy(r).pin_memory(), params_of(p)) for l, r, p in reqs]
    futs = [srv.submit(*q) for q in pinned]
    assert srv.cancel(futs[-1]) and futs[-1].cancelled()
    for f in futs[:-1]:
        f.result(timeout=120)
    assert not srv.cancel(futs[0])          # already done
    g = srv.submit(*pinned[0])
    g.result(timeout=120)
    srv.close()
    assert srv.cancelled == 1 and len(srv.latencies()) == len(reqs)


@pytest.mark.slow
def test_c5_sample_alone_and_in_the_mix():
    # 50 requests of the serving stream (mixed sizes, disparity ranges,
    # blocks, K; seed 7) submitted in bursts: every served result equals the
    # same pair run alone, and a few are checked against the oracle
    import oracle
    items = []
    for i in range(50):
        sc, p, _ = synth.workload("c5", i)
        left, right, _ = sc.render(want_gt=False)
        items.append((left, right, p))
    ctx = sb.Context(0)
    alone = [run_pairs(ctx, [it], sb.SB_RUN_PLAIN)[0] for it in items]
    ctx.close()
    srv = Server(0, mem_budget_bytes=8 << 30, max_batch=16)
    futs = []
    for i, (l, r, p) in enumerate(items):
        futs.append(srv.submit(torch.from_numpy(l).pin_memory(), torch.from_numpy(r).pin_memory(), params_of(p)))
        if i % 10 == 9:
            time.sleep(0.01)
    res = [f.result(timeout=300) for f in futs]
    batches = srv.batches
    srv.close()
    assert batches < len(items)
    for (o_rgb, o_disp), (a_rgb, a_disp) in zip(res, alone):
        assert np.array_equal(o_rgb.numpy(), a_rgb)
        assert np.array_equal(o_disp.numpy().view(np.uint16), a_disp)
    rng = np.random.default_rng(5)
    for i in (0, 17, 33):
        left, right, p = items[i]
        fr = oracle.run_front(left, right, p)
        h, w = left.shape[:2]
        pts = [(int(rng.integers(0, w)), int(rng.integers(0, h))) for _ in range(40)]
        want = oracle.disp_at_points(fr, p, pts)
        got = [int(alone[i][1][y, x]) for x, y in pts]
        assert got == want

