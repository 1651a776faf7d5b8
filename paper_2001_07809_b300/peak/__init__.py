"""Measured instruction rates of the current GPU (see int_peak.cu).

``measure()`` returns thread-instructions per second for add.u32,
vabsdiff4 (four byte cells each), fma.f32, prmt, fma.f32x2 (two FMAs
each), shf, lop3, mad.lo, mad.hi, redux.sync and the byte-masked vabsdiff4,
measured with CUDA events over a full grid, and the same as warp
instructions per clock and SM at the maximum SM clock.  Used by bench.py
beside the derived peaks."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libsb_peak.so")


def measure() -> dict:
    if not os.path.exists(LIB):
        raise RuntimeError("libsb_peak.so is not built: run paper_2001_07809_b300.build.build()")
    lib = ctypes.CDLL(LIB)
    lib.sb_peak_measure.argtypes = [ctypes.POINTER(ctypes.c_double)]
    lib.sb_peak_measure.restype = ctypes.c_int
    rates = (ctypes.c_double * 11)()
    if lib.sb_peak_measure(rates) != 0:
        raise RuntimeError("sb_peak_measure failed")
    out = {"iadd_tops": rates[0] / 1e12, "vabsdiff4_tinstr_s": rates[1] / 1e12,
           "vabsdiff4_tcell_s": 4 * rates[1] / 1e12, "ffma_tflops": 2 * rates[2] / 1e12,
           "prmt_tinstr_s": rates[3] / 1e12, "ffma2_tinstr_s": rates[4] / 1e12,
           "ffma2_tflops": 4 * rates[4] / 1e12}
    names = ["add.u32", "vabsdiff4", "fma.f32", "prmt", "fma.f32x2", "shf.r.wrap", "lop3", "mad.lo.u32",
             "mad.hi.u32", "redux.sync.min", "vabsdiff4 (byte mask)"]
    try:
        import torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    except Exception:
        sms = 148
    # warp instructions per clock and SM at the part's maximum SM clock (2032 MHz)
    out["warp_instr_per_clk_sm"] = {n: rates[i] / 32 / sms / 2.032e9 for i, n in enumerate(names)}
    return out
