"""The bounds-checked build (libsb_checks.so) and the NVTX stage ranges, on
the GPU.  Both run in child processes: the package loads one library per
process, and NVTX loads its injection library at the first NVTX call."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2001_07809_b300 as sb  # noqa: E402

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _child_env(**extra):
    env = dict(os.environ)
    env["PYTHONPATH"] = os.pathsep.join([ROOT, HERE] + ([env["PYTHONPATH"]] if env.get("PYTHONPATH") else []))
    env.update(extra)
    return env


def test_checks_library_reports_and_stays_clean_on_valid_inputs():
    from paper_2001_07809_b300 import build
    build.build(checks=True)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checks_child.py")], env=_child_env(SB_LIBRARY="checks"),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-4000:]


def test_normal_library_has_no_checks():
    assert not sb.sb_checks_built()
    with sb.Context(0) as c:
        with pytest.raises(sb.SbError) as ei:
            c.check_probe(True)
        assert ei.value.status == sb.SB_ERR_UNSUPPORTED
        c.synchronize()


NVTX_CHILD = r"""
import numpy as np, torch, synth, paper_2001_07809_b300 as sb
from gpu_helpers import run_pairs
sc, p, _ = synth.workload("c1")
left, right, _ = sc.render()
with sb.Context(0) as ctx:
    run_pairs(ctx, [(left, right, p)], sb.SB_RUN_PLAIN)
print("ok")
"""


def test_nvtx_ranges_cover_every_stage(tmp_path):
    rec = str(tmp_path / "librec.so")
    subprocess.check_call(["gcc", "-shared", "-fPIC", "-I", "/usr/local/cuda/include",
                           os.path.join(HERE, "nvtx_recorder.c"), "-o", rec])
    log = tmp_path / "nvtx.log"
    r = subprocess.run([sys.executable, "-c", NVTX_CHILD], capture_output=True, text=True, timeout=600,
                       env=_child_env(NVTX_INJECTION64_PATH=rec, SB_NVTX_LOG=str(log)))
    assert r.returncode == 0, r.stderr[-4000:]
    lines = log.read_text().split("\n")[:-1]
    # balanced pushes and pops, never below zero
    depth = 0
    for ln in lines:
        depth += 1 if ln.startswith("push ") else -1
        assert depth >= 0
    assert depth == 0
    pushed = [ln[5:] for ln in lines if ln.startswith("push sb:")]
    stages = ["sb:" + s for s in sb.STAGES]
    assert pushed[0] == "sb:run"
    # one run: every stage once, in pipeline order, each inside sb:run
    assert [s for s in pushed if s != "sb:run"] == stages
    assert np.all(np.diff([lines.index("push " + s) for s in stages]) > 0)
