"""Arithmetic claims of the exact split product (tensor-core refresh and
flush), checked on the CPU with an independent numpy restatement of the
scheme (Ozaki, Ogita, Oishi and Rump, 2012):

- a vector scaled by 2^-E (|x| < 2^E) and rounded to a multiple of 2^-56 is
  exactly the sum of 7 signed base-256 digits d_t 2^(-8(t+1)), |d_0| <= 256,
  |d_t| <= 128, each exactly representable in BF16 (8 significant bits);
- slice products of level l = t + u + 2 summed over an inner dimension of 64
  stay below 2^23 for levels 2..6, so an FP32 accumulator holds them exactly;
- the combined sum of the five exact levels and the rounded tail fits int64.
"""
import numpy as np
import pytest

S, K = 7, 64


def split(x):
    """Digits of one vector: (E, d[S, len(x)]) with x ~ 2^E sum_t d_t 2^(-8(t+1))."""
    m = np.max(np.abs(x))
    E = int(np.frexp(m)[1]) if m > 0 else 0          # m < 2^E
    X = np.rint(np.ldexp(x, 56 - E)).astype(np.int64)  # |X| < 2^56 (exact in int64)
    d = np.zeros((S, len(x)), np.int64)
    for t in range(S):
        sh = 48 - 8 * t
        q = (X + (1 << (sh - 1))) >> sh if sh > 0 else X
        d[t] = q
        X = X - (q << sh)
    assert np.all(X == 0)
    return E, d


def bf16_exact(v):
    """True where the integers v are exactly representable with 8 significant bits."""
    v = np.abs(v.astype(np.int64))
    out = np.ones(v.shape, bool)
    nz = v > 0
    tz = np.zeros(v.shape, np.int64)
    w = v.copy()
    while np.any(nz & (w % 2 == 0)):
        m = nz & (w % 2 == 0)
        w[m] //= 2
        tz[m] += 1
    out[nz] = w[nz] < 256          # odd part has at most 8 bits
    return out


@pytest.mark.parametrize("seed,spread", [(1, 0.0), (2, 6.0), (3, 30.0)])
def test_split_reconstructs_to_2_pow_minus_56_of_the_maximum(seed, spread):
    g = np.random.Generator(np.random.PCG64(seed))
    x = g.standard_normal(K) * 10.0 ** g.uniform(-spread, spread, K)
    E, d = split(x)
    assert np.all(np.abs(d[0]) <= 256) and np.all(np.abs(d[1:]) <= 128)
    assert np.all(bf16_exact(d))
    rec = sum(np.ldexp(d[t].astype(float), E - 8 * (t + 1)) for t in range(S))
    # |x - rec| <= 2^(E - 57) (the one rounding) up to float64 summation
    assert np.max(np.abs(x - rec)) <= 2.0 ** (E - 57) * 1.01 + 4 * np.finfo(float).eps * np.max(np.abs(x))


def test_level_sums_fit_fp32_exactly_for_levels_2_to_6():
    # worst case: every digit at its bound and every product of one sign
    bound = [256] + [128] * (S - 1)
    for lv in range(2, 7):
        s = sum(bound[t] * bound[lv - 2 - t] for t in range(S) if 0 <= lv - 2 - t < S)
        assert K * s < 2 ** 23, (lv, K * s)
    # random data: the exact integer level sums are recovered from FP32 sums
    g = np.random.Generator(np.random.PCG64(9))
    _, a = split(g.standard_normal(K))
    _, b = split(g.standard_normal(K) * 1e3)
    for lv in range(2, 7):
        exact = sum(int(np.dot(a[t], b[lv - 2 - t])) for t in range(S) if 0 <= lv - 2 - t < S)
        acc = np.float32(0)
        for t in range(S):
            u = lv - 2 - t
            if 0 <= u < S:
                for k in range(K):
                    acc = np.float32(acc + np.float32(a[t, k]) * np.float32(b[u, k]))
        assert int(acc) == exact


def test_combined_sum_fits_int64():
    # F = N2 2^40 + N3 2^32 + N4 2^24 + N5 2^16 + N6 2^8 + tail, |N_l| below their
    # worst-case bounds, |tail| < 2^31
    bound = [256] + [128] * (S - 1)
    N = {lv: K * sum(bound[t] * bound[lv - 2 - t] for t in range(S) if 0 <= lv - 2 - t < S) for lv in range(2, 7)}
    F = N[2] * 2 ** 40 + N[3] * 2 ** 32 + N[4] * 2 ** 24 + N[5] * 2 ** 16 + N[6] * 2 ** 8 + 2 ** 31
    assert F < 2 ** 63
    # the int32 pairs formed on the way: N2 * 256 + N3 and N4 * 256 + N5
    assert N[2] * 256 + N[3] < 2 ** 31 and N[4] * 256 + N[5] < 2 ** 31
