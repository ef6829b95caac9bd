"""The tensor-core Walsh-Hadamard probe (tcgen05.mma, BF16 operands, FP32
accumulation in tensor memory): its 2^14-point transform of a {-1, 0, 1}
slice, H128 X H128 as two 128 x 128 x 128 products, equals the exact
transform in every mode, and none of its bounded waits runs out.  On the CPU,
every field of the descriptors it builds is decoded back and compared."""
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_descriptor_fields(tmp_path):
    # every field decoded back out of the header's descriptors (host program, no GPU)
    from paper_2601_09477_gb300 import build
    exe = str(tmp_path / "umma_desc_check")
    cmd = [build.nvcc(), "-std=c++17", "-O1",
           "-I" + os.path.join(ROOT, "paper_2601_09477_gb300", "csrc"),
           "-o", exe, os.path.join(ROOT, "tests", "umma_desc_check.cu")]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "descriptor checks passed" in run.stdout


@pytest.mark.gpu
def test_umma_hadamard_probe_exact():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    out = subprocess.run([sys.executable, "-m", "paper_2601_09477_gb300.probes.run_umma_hadamard",
                          "--iters", "64"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    res = json.loads(out.stdout.strip().splitlines()[-1])
    for mode in ("mode0", "mode1", "mode2"):
        assert res[mode]["wrong"] == 0 and res[mode]["status"] == 0, res
