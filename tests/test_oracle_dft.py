"""Pins for the oracle's brute-force weighted DFT (Eq. dft, Sec. 2).

None of these checks re-evaluate the oracle's sum of rotations. They use facts the paper
states about the transform and textbook routines on Python integers:
  * principal root: sum_j omega^{ij} = 0 for 0 < i < L, so the all-ones vector maps to L e_0;
  * outputs come in bit-reversed order, so a single-frequency input a_i = omega^{-k i}
    concentrates on the output index whose bit reversal is k;
  * the weight zeta scales output j by zeta^{j'} (checked on the delta input);
  * Horner evaluation: with zeta = 1, a-hat_j is the polynomial sum a_i X^i at X = omega_L^{j'};
  * the convolution theorem against a schoolbook cyclic convolution.
"""
import random

import numpy as np
import pytest


def bitrev(j, l):
    return int(format(j, f"0{l}b")[::-1], 2) if l else 0


def dft(orc, vals, l, z, n, e, N):
    x = orc.cells_from_ints(vals, N, count=1 << l)
    return orc.cells_to_ints(orc.dft_brute(x, l, z, n, e, N), N, n)


@pytest.mark.parametrize("l,N", [(1, 64), (3, 64), (5, 128), (6, 192)])
def test_all_ones_maps_to_L_delta(orc, l, N):
    L = 1 << l
    out = dft(orc, [1] * L, l, L, L, 0, N)
    assert out == [L] + [0] * (L - 1)


@pytest.mark.parametrize("l,N", [(2, 64), (4, 64), (5, 256)])
def test_single_frequency_lands_on_bitreversed_index(orc, l, N):
    L, p = 1 << l, (1 << N) + 1
    w = 2 * N // L  # omega_L = 2^w
    for k in range(L):
        # a_i = omega^{-k i}; then a-hat_j = sum_i omega^{i (j' - k)} = L [j' == k]
        vals = [pow(2, (-k * i * w) % (2 * N), p) for i in range(L)]
        out = dft(orc, vals, l, L, L, 0, N)
        expect = [L if bitrev(j, l) == k else 0 for j in range(L)]
        assert out == expect, k


@pytest.mark.parametrize("l,N", [(3, 64), (5, 128)])
def test_weight_scales_by_bitreversed_power(orc, l, N):
    L, p = 1 << l, (1 << N) + 1
    rng = random.Random(l)
    for e in (0, 1, 5, N, 2 * N - 1, rng.randrange(2 * N)):
        out = dft(orc, [1], l, 1, L, e, N)  # delta at i = 0
        assert out == [pow(2, e * bitrev(j, l), p) for j in range(L)]


@pytest.mark.parametrize("l,N", [(3, 64), (4, 128), (6, 128)])
def test_horner_evaluation(orc, l, N):
    L, p = 1 << l, (1 << N) + 1
    rng = random.Random(100 + l)
    a = [rng.randrange(p) for _ in range(L)]
    out = dft(orc, a, l, L, L, 0, N)
    for j in range(L):
        X = pow(2, (2 * N // L) * bitrev(j, l), p)
        acc = 0
        for c in reversed(a):
            acc = (acc * X + c) % p
        assert out[j] == acc


@pytest.mark.parametrize("l,N", [(3, 64), (5, 128)])
def test_convolution_theorem(orc, l, N):
    L, p = 1 << l, (1 << N) + 1
    rng = random.Random(200 + l)
    a = [rng.randrange(p) for _ in range(L)]
    b = [rng.randrange(p) for _ in range(L)]
    c = [0] * L
    for i in range(L):
        for j in range(L):
            c[(i + j) % L] = (c[(i + j) % L] + a[i] * b[j]) % p
    A, B, Cc = (dft(orc, v, l, L, L, 0, N) for v in (a, b, c))
    assert [(x * y) % p for x, y in zip(A, B)] == Cc


def test_truncation_takes_prefixes(orc):
    # TFT(L, zeta, z, n) is the first n outputs with inputs beyond z equal to zero (Sec. 2)
    N, l = 128, 5
    L, p = 1 << l, (1 << N) + 1
    rng = random.Random(3)
    a = [rng.randrange(p) for _ in range(11)]
    full = dft(orc, a + [0] * (L - 11), l, L, L, 7, N)
    assert dft(orc, a, l, 11, 20, 7, N) == full[:20]


def test_rejects_invalid(orc):
    x = np.zeros(4 * 2, np.uint64)
    with pytest.raises(ValueError):
        orc.dft_brute(x, 8, 1, 1, 0, 64)  # L = 256 does not divide 2N = 128
