"""Host-side pins of the tensor-core Gram's shared-memory arithmetic (CPU only).

`tests/layout/gram_tc_layout.cu` includes the kernel header and, without
launching anything, replays the address arithmetic of the operand stores and
of every MMA operand read: a warp's stores must fall in 32 distinct banks, the
reads of both tile parities must stay inside the block's allocation, the odd
tiles' shifted A descriptor must map S rows 0..63 onto D rows 64..127, and the
shared-memory and instruction descriptors must carry the fields the kernel
means (start, leading and stride byte offsets, version 1; FP32 accumulators,
TF32 operands, K-major, N/8 and M/16)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def test_gram_tc_layout(tmp_path):
    if not os.path.exists(NVCC):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "gram_tc_layout")
    src = os.path.join(ROOT, "tests", "layout", "gram_tc_layout.cu")
    subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2109_09534_gb300", "csrc"),
                    src, "-o", exe], check=True, capture_output=True, timeout=600)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=60).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("VT ")]
    assert len(lines) == 2, out
    for ln in lines:
        tok = ln.split()
        f = {tok[i]: int(tok[i + 1]) for i in range(0, len(tok) - 1, 2)}
        assert f["bank_conflicts"] == 0, ln
        assert 0 <= f["read_lo"] and f["read_hi"] <= f["bytes"], ln
        assert f["rows_ok"] == 1 and f["desc_ok"] == 1 and f["idesc_ok"] == 1 and f["idesc64_ok"] == 1, ln
        assert f["epilogue"] <= 2 * f["sb"], ln
        # the resident blocks of an SM: their TMEM columns fit its 512 and their
        # shared memory (plus 1 KB reserved each) its 228 KB
        assert f["blocks"] * f["tcols"] <= 512, ln
        assert f["blocks"] * (f["bytes"] + 1024) <= 228 * 1024, ln
