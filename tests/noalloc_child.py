"""Child process of the allocation-free entry point's two-context test: it
runs the entry point through the C ABI in two driver contexts created one after
the other (a host application's own contexts), with inputs and outputs
allocated in each, and sends both results back.  Kept apart from the test
module so the spawned child imports nothing but numpy, ctypes and the CUDA
driver bindings."""
import numpy as np


def two_contexts(lib_path, Ll, Lr, bmap, D, B, q):
    # each round creates its own driver context: the scratch address the first
    # round looked up belongs to a context that no longer exists in the second
    import ctypes as C

    from cuda.bindings import driver as drv

    f = C.CDLL(lib_path).sb_boundary_sad_static
    V, I32 = C.c_void_p, C.c_int32
    f.argtypes = [V, V, V, I32, I32, I32, I32, I32, V, V, V, C.c_char_p, C.c_size_t]
    f.restype = C.c_int
    h, w = Ll.shape
    out = []
    try:
        assert drv.cuInit(0)[0] == drv.CUresult.CUDA_SUCCESS
        err, dev = drv.cuDeviceGet(0)
        for _ in range(2):
            err, ctx = drv.cuCtxCreate(None, 0, dev)
            assert err == drv.CUresult.CUDA_SUCCESS
            bufs = []
            for a in (Ll, Lr, bmap):
                err, p = drv.cuMemAlloc(a.nbytes)
                assert err == drv.CUresult.CUDA_SUCCESS
                drv.cuMemcpyHtoD(p, a, a.nbytes)
                bufs.append(p)
            err, dd = drv.cuMemAlloc(h * w * 2)
            err, dc = drv.cuMemAlloc(h * w * 4)
            msg = C.create_string_buffer(256)
            st = f(int(bufs[0]), int(bufs[1]), int(bufs[2]), w, h, D, B, 0, int(dd), int(dc), None, msg, 256)
            assert st == 0, msg.value
            assert drv.cuCtxSynchronize()[0] == drv.CUresult.CUDA_SUCCESS
            disp = np.empty((h, w), np.uint16)
            cost = np.empty((h, w), np.uint32)
            drv.cuMemcpyDtoH(disp, dd, disp.nbytes)
            drv.cuMemcpyDtoH(cost, dc, cost.nbytes)
            drv.cuCtxDestroy(ctx)
            out.append((disp, cost))
        q.put(("ok", out))
    except Exception as e:  # report to the parent instead of hanging it
        q.put(("error", repr(e)))
