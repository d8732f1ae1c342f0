"""Pins for the oracle's ring arithmetic in Z/(2^N+1) against Python integers.

Python's built-in integers are an independent arbitrary-precision implementation, so these
checks do not route back into the oracle's own bignum (Sec. 2: R = Z/(2^{M/2}+1), omega = 2).
"""
import random

import pytest


def edge_values(N):
    p = (1 << N) + 1
    return [0, 1, 2, 3, (1 << N) - 1, 1 << N, 1 << (N - 1), (1 << (N - 1)) + 1, p - 2,
            (1 << 64) - 1, 1 << 64]


@pytest.mark.parametrize("N", [64, 128, 192, 1024, 4096])
def test_add_sub_mul(orc, N):
    p = (1 << N) + 1
    rng = random.Random(N)
    vals = edge_values(N) + [rng.randrange(p) for _ in range(40)]
    for a in vals:
        for b in vals[:8] + [rng.randrange(p) for _ in range(3)]:
            a %= p
            b %= p
            assert orc.ring_add(a, b, N) == (a + b) % p
            assert orc.ring_sub(a, b, N) == (a - b) % p
            assert orc.ring_mul(a, b, N) == (a * b) % p


@pytest.mark.parametrize("N", [64, 128, 320, 1024])
def test_mul2exp_div2(orc, N):
    p = (1 << N) + 1
    rng = random.Random(7 * N)
    ks = [0, 1, 2, 31, 32, 63, 64, 65, N - 1, N, N + 1, 2 * N - 1, 2 * N, 2 * N + 5, 5 * N + 3]
    for a in edge_values(N) + [rng.randrange(p) for _ in range(20)]:
        a %= p
        for k in ks + [rng.randrange(4 * N) for _ in range(6)]:
            assert orc.ring_mul2exp(a, k, N) == (a * pow(2, k, p)) % p, (a, k)
        h = orc.ring_div2(a, N)
        assert 0 <= h <= (1 << N) and (2 * h) % p == a


def test_powers_of_two_are_roots_of_unity(orc):
    # 2 has order 2N modulo 2^N + 1: 2^N = -1, so omega = 2 is a principal 2N-th root (Sec. 2)
    for N in (64, 256):
        p = (1 << N) + 1
        assert orc.ring_mul2exp(1, N, N) == p - 1
        assert orc.ring_mul2exp(1, 2 * N, N) == 1


@pytest.mark.parametrize("N", [64, 128, 1024])
def test_reduce(orc, N):
    p = (1 << N) + 1
    rng = random.Random(N + 1)
    for bits in (1, 63, N, N + 1, 2 * N + 7, 3 * N, 5 * N + 13):
        for _ in range(5):
            x = rng.getrandbits(bits)
            assert orc.ring_reduce(x, N) == x % p


def test_rejects_bad_N(orc):
    with pytest.raises(ValueError):
        orc.ring_add(1, 2, 96)
