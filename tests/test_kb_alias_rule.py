"""The outer-bandwidth rule of the real-exponent bands, checked on the exact
Kaiser-Bessel transform (no GPU).

An NFFT with oversampling 2 (b = 3 pi / 2) covers frequencies up to N/2 = n/4;
a band whose occupied frequencies exceed that by e keeps the half-size grid
only if m pi sqrt(6 e / n) <= 0.2.  The rule rests on the nearest alias of
frequency n/4 + e sitting at |nu| = 3/4 - e/n, where
Phi(nu) = pi I_0(m sqrt(b^2 - (2 pi nu)^2)) ~ pi I_0(m pi sqrt(6 e / n)).
Here the exact ratio Phi(3/4 - e/n) / Phi(3/4) is computed from that formula
and compared with the closed form, which bounds it from above, and the growth
the rule accepts is checked to stay within 1 %.
"""
import math

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")

B = 1.5 * math.pi


def phi_hat(nu, m):
    arg = B * B - (2.0 * math.pi * nu) ** 2
    return math.pi * float(scipy_special.i0(m * math.sqrt(max(arg, 0.0))))


def rule_accepts(m, e, n):
    return m * math.pi * math.sqrt(6.0 * e / n) <= 0.2


@pytest.mark.parametrize("m", [2, 4, 5, 6, 8, 10, 12])
@pytest.mark.parametrize("log2n", [10, 14, 18, 20, 22, 24])
def test_alias_growth_within_one_percent(m, log2n):
    n = 2 ** log2n
    for e in range(1, m + 4):
        growth = phi_hat(0.75 - e / n, m) / phi_hat(0.75, m)
        approx = float(scipy_special.i0(m * math.pi * math.sqrt(6.0 * e / n)))
        # b^2 - (b - 2 pi e/n)^2 = 4 pi b e/n - (2 pi e/n)^2 < 6 pi^2 e/n: the closed
        # form bounds the exact growth from above (and is its first-order term)
        assert growth <= approx * (1 + 1e-12)
        assert growth >= 1.0
        if rule_accepts(m, e, n):
            assert growth <= 1.01


def test_rule_excludes_small_grids():
    # the full margin of m_w + 3 frequencies is never accepted on grids of
    # 2^14 points or fewer, for any window half-width
    for m in range(2, 13):
        for log2n in range(5, 15):
            assert not rule_accepts(m, m + 3, 2 ** log2n)
    # and it is on the large grids of the FP32 form (m_w = 5 or 6)
    assert rule_accepts(5, 8, 2 ** 20) and rule_accepts(6, 9, 2 ** 21)
