"""Host check of the split-precision conversions of the tensor-core path
(``csrc/bf16split.cuh``), no GPU: the header is compiled for the host by nvcc.

* f32_bits_to_f64 equals the host's float-to-double conversion on every float
  bit pattern (NaNs excepted: any NaN is a NaN).
* split3_bf16: each piece is the BF16 value nearest to what the earlier pieces
  leave, ties to even (IEEE 754 rounding, checked here in exact rational
  arithmetic), on random values over the whole BF16 normal range, exact ties,
  zeros and values next to the range edges where the integer path hands over
  to the conversion instruction.
"""
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bf16split_check.cu")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc (host compile only)")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("bf16split") / "bf16split_check")
    subprocess.run(["nvcc", "-O2", "-std=c++17", "-o", exe, SRC], check=True)
    return exe


def test_float_to_double_is_exact_on_every_float(checker):
    out = subprocess.run([checker, "f32"], check=True, capture_output=True, text=True).stdout
    assert int(out.strip()) == 0


def _bf16_float(bits):
    return struct.unpack("<f", struct.pack("<I", int(bits) << 16))[0]


def _bf16_value(bits):
    return Fraction(_bf16_float(bits))


def _nearest_even_ok(r, p_bits):
    """p is the BF16 nearest to the exact rational r, ties to the even pattern."""
    p = _bf16_value(p_bits)
    if r == 0:
        return p == 0
    e = (abs(r).numerator.bit_length() - abs(r).denominator.bit_length())
    # BF16 normal spacing at r's binade: 2^(floor(log2|r|) - 7)
    while Fraction(2) ** e > abs(r):
        e -= 1
    while Fraction(2) ** (e + 1) <= abs(r):
        e += 1
    ulp = Fraction(2) ** (max(e, -126) - 7)
    d = abs(r - p)
    if d > ulp / 2:
        return False
    if d == ulp / 2:
        return (int(p_bits) & 1) == 0
    return True


def _inputs():
    rng = np.random.default_rng(1611)
    xs = []
    # random significands over the normal range and both signs
    e = rng.integers(-120, 120, 4000)
    xs += list(rng.uniform(1.0, 2.0, 4000) * np.ldexp(1.0, e) * rng.choice([-1.0, 1.0], 4000))
    # typical history values and their negatives
    xs += list(rng.standard_normal(2000) * 10.0 ** rng.integers(-4, 4, 2000))
    # exact ties at every piece: 1 + 2^-8 (+ 2^-16 (+ 2^-24)), scaled
    for s in (1.0, -3.0, 2.0 ** -50, 2.0 ** 60):
        for t in (1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7 + 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -16,
                  1 + 2.0 ** -16 + 2.0 ** -24, (2 - 2.0 ** -8) + 2.0 ** -9, 2 - 2.0 ** -9):
            xs.append(s * t)
    # zeros, integers, the edges of the integer path's exponent range
    xs += [0.0, -0.0, 1.0, -2.5, 3.0, 65536.0, 1e-300, -1e-300]
    for k in (-127, -126, -125, 125, 126, 127):
        for f in (1.0, 1.5, 2 - 2.0 ** -52, 1 + 2.0 ** -8):
            xs.append(f * 2.0 ** k)
            xs.append(-f * 2.0 ** k)
    return np.array(xs, dtype=np.float64)


def test_split_pieces_are_nearest_even(checker, tmp_path):
    x = _inputs()
    fin, fout = str(tmp_path / "x.bin"), str(tmp_path / "p.bin")
    x.tofile(fin)
    subprocess.run([checker, "split", fin, fout], check=True)
    rec = np.fromfile(fout, dtype=np.uint16).reshape(-1, 6)
    assert rec.shape[0] == x.size
    int_path = 0
    for xi, row in zip(x, rec):
        r = Fraction(float(xi))
        if np.isinf(_bf16_float(row[0])):
            # rounds past BF16's largest finite value (2 - 2^-7) 2^127
            assert abs(r) >= (2 - Fraction(1, 256)) * Fraction(2) ** 127 and not row[3]
            continue
        for k in range(3):
            tiny = r != 0 and abs(r) < Fraction(2) ** -126
            if row[3 + k]:
                int_path += 1
                assert not tiny
            if not tiny:  # BF16 subnormals go to the conversion instruction
                assert _nearest_even_ok(r, row[k]), (float(xi), k, hex(row[k]))
            r -= _bf16_value(row[k])
        # three 8-bit pieces leave at most 2^-24 of |x| (normal range)
        if 2.0 ** -100 < abs(xi) < 2.0 ** 100:
            assert abs(r) <= Fraction(2) ** -24 * abs(Fraction(float(xi)))
    assert int_path > 0.9 * 3 * x.size
