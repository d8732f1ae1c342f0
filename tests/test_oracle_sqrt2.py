"""Pins of the oracle's transforms over Z/(2^N+1) with omega = sqrt2 (the sqrt2 trick; not in
the paper). sqrt2 = 2^{3N/4} - 2^{N/4} squares to 2, so it is a principal 4N-th
root of unity and transforms of length L | 4N exist: rings half the size the paper's L | 2N
rule allows. Pins independent of the oracle's recursion:

  * sqrt2^2 = 2 and sqrt2^{2N} = -1 (Python integers);
  * the DFT by definition against Horner evaluation with Python's pow at omega_L = sqrt2^{4N/L};
  * the principal-root property (all-ones transform at L = 4N);
  * Algorithms 1 and 2 against the DFT and the ITFT's definition, at L = 4N and below;
  * for even exponents (L | 2N) the same outputs as the omega = 2 transforms.
"""
import random

import pytest


def sqrt2(N):
    p = (1 << N) + 1
    return ((1 << (3 * N // 4)) - (1 << (N // 4))) % p


def bitrev(j, l):
    return int(format(j, f"0{l}b")[::-1], 2) if l else 0


def py_dft(a, l, n, e, N):
    p = (1 << N) + 1
    s = sqrt2(N)
    L = 1 << l
    wL = pow(s, 4 * N // L, p)
    out = []
    for j in range(n):
        t = pow(wL, bitrev(j, l), p)
        acc = 0
        for x in reversed(a):
            acc = (acc * t + x) % p
        out.append(acc * pow(s, e * bitrev(j, l), p) % p)
    return out


def cells(orc, vals, N, L):
    return orc.cells_from_ints(vals, N, count=L)


def rand_res(rng, N, k):
    p = (1 << N) + 1
    return [0 if rng.random() < 0.04 else (1 << N) if rng.random() < 0.04 else rng.randrange(p) for _ in range(k)]


@pytest.mark.parametrize("N", [64, 128, 192, 1024])
def test_sqrt2_is_a_principal_root(N):
    p = (1 << N) + 1
    s = sqrt2(N)
    assert s * s % p == 2
    assert pow(s, 2 * N, p) == p - 1 and pow(s, 4 * N, p) == 1


def test_principal_root_all_ones(orc):
    N = 64
    l = 8  # L = 4N
    L = 1 << l
    out = orc.cells_to_ints(orc.sqrt2_dft_brute(cells(orc, [1] * L, N, L), l, L, L, 0, N), N, L)
    assert out[0] == L and all(v == 0 for v in out[1:])


@pytest.mark.parametrize("N,l", [(64, 8), (64, 5), (128, 9), (192, 4)])
def test_dft_matches_horner(orc, N, l):
    rng = random.Random(N + l)
    L = 1 << l
    for e in (0, 1, 4 * N - 1, rng.randrange(4 * N)):
        a = rand_res(rng, N, L)
        z = L if e % 2 == 0 else rng.randint(1, L)
        got = orc.cells_to_ints(orc.sqrt2_dft_brute(cells(orc, a[:z], N, L), l, z, L, e, N), N, L)
        assert got == py_dft(a[:z], l, L, e, N), e


@pytest.mark.parametrize("N,l", [(64, 8), (64, 4), (128, 9)])
def test_tft_itft_against_definition(orc, N, l):
    rng = random.Random(7 * N + l)
    L, p = 1 << l, (1 << N) + 1
    for _ in range(12):
        z = rng.randint(1, L)
        n = rng.randint(1, L)
        e = rng.randrange(4 * N)
        a = rand_res(rng, N, z)
        hat = py_dft(a, l, L, e, N)
        x = cells(orc, a, N, L)
        orc.sqrt2_tft(x, l, z, n, e, N)
        assert orc.cells_to_ints(x, N, n) == hat[:n], (z, n, e)
        nn = rng.randint(0, z)
        f = 1 if nn + 1 <= L and rng.random() < 0.5 else 0
        if nn + f < 1:
            nn = 1
        inp = hat[:nn] + [(L * v) % p for v in a[nn:z]]
        want = [(L * v) % p for v in a[:nn]] + ([hat[nn]] if f else [])
        x = cells(orc, inp, N, L)
        orc.sqrt2_itft(x, l, z, nn, f, e, N)
        assert orc.cells_to_ints(x, N, nn + f) == want, (z, nn, f, e)


def test_even_exponents_match_the_omega_2_transform(orc):
    """For L | 2N and an even weight exponent 2e, the sqrt2 transform is the omega = 2 one with
    weight e (omega_L and zeta are the same ring elements)."""
    N, l = 128, 6
    rng = random.Random(1)
    L = 1 << l
    for _ in range(5):
        z, n, e = rng.randint(1, L), rng.randint(1, L), rng.randrange(2 * N)
        a = rand_res(rng, N, z)
        x1, x2 = cells(orc, a, N, L), cells(orc, a, N, L)
        orc.tft(x1, l, z, n, e, N)
        orc.sqrt2_tft(x2, l, z, n, 2 * e, N)
        assert orc.cells_to_ints(x1, N, n) == orc.cells_to_ints(x2, N, n)
