"""Host checks of the index arithmetic the FFT passes rely on (no GPU).

* The shared-memory swizzle swz(e) = e ^ ((e >> 4) & (P - 1)) (P = 16 for
  complex64, 8 for complex128) is a permutation of every aligned run of 16.
* The shortcut swz(b0 + r D) = (swz(b0) ^ ((r D >> 4) & (P - 1))) + r D used
  for the butterfly loads (b0 = jj < L/R, D = L/R) and stores
  (b0 = (jj - k) R + k, k = jj mod NS, D = NS) whenever D is a multiple of 16,
  and swz(16 t + r) = swz(16 t) ^ r for the first-stage stores.
* The stage-twiddle table layout: every pair read lies inside its region.
"""
import itertools


def swz(e, P):
    return e ^ ((e >> 4) & (P - 1))


def step(bs, r, D, P):
    return (bs ^ (((r * D) >> 4) & (P - 1))) + r * D


def test_swizzle_is_a_permutation_of_runs():
    for P in (16, 8):
        for base in range(0, 4096, 16):
            assert sorted(swz(base + i, P) for i in range(16)) == list(range(base, base + 16))


def test_swizzle_shortcut_for_every_stage_pattern():
    for P in (16, 8):
        for lg in range(4, 13):
            L = 1 << lg
            for R in (2, 4, 8, 16):
                if R > L:
                    continue
                S = L // R
                if S % 16 == 0:
                    for jj in range(S):
                        bs = swz(jj, P)
                        for r in range(R):
                            assert step(bs, r, S, P) == swz(jj + r * S, P)
                for d in range(4, lg):
                    NS = 1 << d
                    if NS * R > L:
                        continue
                    for jj in range(L // R):
                        k = jj & (NS - 1)
                        b0 = (jj - k) * R + k
                        bs = swz(b0, P)
                        for r in range(R):
                            assert step(bs, r, NS, P) == swz(b0 + r * NS, P)
        for t in range(512):
            bs = swz(16 * t, P)
            assert all((bs ^ r) == swz(16 * t + r, P) for r in range(16))


def _last_log(L, F):
    R = L - F
    return R - 4 * ((R + 3) // 4 - 1)


def _stage_log(L, F, d):
    return _last_log(L, F) if d == L - _last_log(L, F) else 4


def _off(L, F, d):
    o, e = 0, F
    while e < d:
        o += (1 << _stage_log(L, F, e)) << e
        e += 4
    return o


def test_twiddle_pairs_stay_in_their_region():
    region = 2 << 12
    for L, F in itertools.product(range(6, 13), (3, 4)):
        if L <= F:
            continue
        base = ((L - 6) * 2 + (F - 3)) * region
        assert _off(L, F, L) <= region
        for d in range(F, L, 4):
            R, NS = 1 << _stage_log(L, F, d), 1 << d
            for k in range(NS):
                for p in range(R // 2):
                    i = base + _off(L, F, d) + 2 * NS * p + 2 * k
                    assert i % 2 == 0 and i + 1 < base + _off(L, F, d) + R * NS
