"""Issue rate of the 4-bit block-scaled tensor-core MMA (`tcgen05.mma
kind::mxf4`, M = 128 x N = 224 x K = 64 on one SM, and the CTA-pair form M =
256 over two SMs) that the tensor-core read is built on: the denominator of
the read's "fraction of the instruction's issue rate".  `mma_rates.cu` times
back-to-back MMAs on every SM; this test compiles it for sm_103a, runs it,
checks both forms run at a sane 0/1 multiply-add rate and that the pair form
keeps the per-SM rate of the single one.  Run with -s to see the rates."""

import os
import re
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.gpu
def test_mxf4_mma_issue_rates():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "mma_rates")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                        os.path.join(HERE, "mma_rates.cu")], check=True, capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    rates = {m.group(1): (float(m.group(2)), float(m.group(3)))
             for m in re.finditer(r"(single|pair) M=\d+: .*?, ([\d.]+) cycles per MMA .*?, ([\d.]+) PFLOP/s",
                                  r.stdout)}
    assert set(rates) == {"single", "pair"}, r.stdout
    for cycles, pflops in rates.values():
        assert 80 <= cycles <= 200, rates      # nominal fp4 rate: ~86 cycles for this shape
        assert pflops > 4.0, rates
    # the pair form splits each MMA over two SMs at the per-SM rate of one
    assert abs(rates["pair"][1] / rates["single"][1] - 1.0) < 0.15, rates
