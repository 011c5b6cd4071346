"""Integer-pipe rates behind two design decisions of the batched read: the
LOP3 roofline of the register-tiled kernel (conditional XOR of a 32-bit word,
`acc = (mask & word) ^ acc`, one LOP3), and the rejection of the 1-bit
AND-POPC tensor form (`mma.sync ... m16n8k256 b1 and.popc`) of the GF(2)
product.  `alu_rates.cu` times both on every SM; this test compiles it for
sm_103a, runs it, and checks that one LOP3 (32 bit-multiply-adds of the GF(2)
product) per lane outpaces the b1 MMA by a wide margin, the premise for not
building the AND-POPC kernel.  Run with -s to see the measured rates."""

import os
import re
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.gpu
def test_lop3_outpaces_b1_and_popc_mma():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "alu_rates")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                        os.path.join(HERE, "alu_rates.cu")], check=True, capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    lop3 = [float(x) for x in re.findall(r"lop3: .*?, ([\d.]+) ops/clk/SM", r.stdout)]
    b1 = [float(x) for x in re.findall(r"b1mma: .*?, (\d+) bit-MAC/clk/SM", r.stdout)]
    assert lop3 and b1
    # per SM and clock: LOP3 ops x 32 bits vs the b1 MMA's bit multiply-adds
    assert max(lop3) * 32 > 4 * max(b1), (lop3, b1)
    assert 32 <= max(lop3) <= 72, lop3  # 4 SM sub-partitions x 16 integer lanes
