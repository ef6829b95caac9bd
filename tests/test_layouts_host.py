"""Shared-memory index maps of the register-round transforms (fwht_device.cuh),
checked on the CPU for every instantiation the kernels launch: each round's
(thread, register) -> index map is a bijection, the padded layout is
injective, and the accesses are free of bank conflicts (per warp for 32-bit
words, per half-warp for 64-bit words, per quarter-warp for the 16-byte rows
of the vectorised FP32 round 0).  The checker (tests/layout_check.cu) calls
the header's constexpr host/device functions from a host program built with
nvcc; no GPU is used."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_transform_layouts_are_bijective_and_conflict_free(tmp_path):
    from paper_2601_09477_gb300 import build
    exe = str(tmp_path / "layout_check")
    cmd = [build.nvcc(), "-std=c++17", "-O1",
           "-I" + os.path.join(ROOT, "paper_2601_09477_gb300", "csrc"),
           "-I" + os.path.join(ROOT, "include"),
           "-o", exe, os.path.join(HERE, "layout_check.cu")]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "layout checks passed" in run.stdout
