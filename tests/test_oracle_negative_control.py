"""The LCG as the paper's negative control (Sec. II.B, Fig. 4): a serial test
of the lowest output bits, which the Quick and Dirty LCG fails outright (bit k
has period 2^(k+1)) while Hybrid Taus, Ran2 and Lagged Fibonacci pass it."""
import numpy as np
import pytest

import oracle


def low_bit_pair_chi2(words: np.ndarray, bit: int) -> float:
    """Chi-square (3 dof) of the pairs (b_n, b_{n+1}) of one bit over a stream."""
    b = ((words >> np.uint32(bit)) & np.uint32(1)).astype(np.int64)
    pairs = 2 * b[:-1:2] + b[1::2]
    counts = np.bincount(pairs, minlength=4)
    exp = len(pairs) / 4.0
    return float(((counts - exp) ** 2 / exp).sum())


@pytest.mark.parametrize("kind,fails", [("lcg", True), ("taus", False), ("ran2", False),
                                        ("lagfib", False)])
def test_low_bit_serial_test(kind, fails):
    g = oracle.Gen(kind, 2024, 1)
    words = g.fill_u32(1 << 16)
    if kind == "ran2":
        words = words << np.uint32(1)      # Ran2 words are 31-bit: test bits 1, 2 of the value
    chi = max(low_bit_pair_chi2(words, k) for k in (1, 2))
    # 3 dof: P(chi2 > 30) ~ 1.4e-6
    assert (chi > 30.0) == fails, chi
