"""Pins of the oracle over the Schoenhage-Nussbaumer coefficient ring (Sec. 5.2).

R = S[y]/(y^{M/2} + 1), S = Z/mZ with m odd: the paper runs its transforms over this ring
with omega = y, so multiplying by a power of omega is a negacyclic shift of the coefficients.
The pins are independent of the oracle's recursion:

  * the ring operations against polynomial arithmetic written here in Python;
  * y is a principal M-th root of unity (the all-ones transform);
  * the DFT by definition (Eq. dft) against Horner evaluation in Python;
  * Algorithms 1 and 2 against the DFT, exhaustively over (z, n, f) for small L, and the ITFT
    against its definition (mixed input built from a-hat and L a);
  * split independence and the convolution theorem (cyclic convolution in R[x]).
"""
import random

import pytest


def py_mul(a, b, m):
    """Negacyclic product of coefficient lists modulo m (y^H = -1)."""
    H = len(a)
    r = [0] * H
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            if i + j < H:
                r[i + j] = (r[i + j] + x * y) % m
            else:
                r[i + j - H] = (r[i + j - H] - x * y) % m
    return r


def py_ypow(a, k, M, m):
    H = M // 2
    mono = [0] * H
    k %= M
    if k < H:
        mono[k] = 1
    else:
        mono[k - H] = m - 1
    return py_mul(a, mono, m)


def rand_elem(rng, H, m):
    r = rng.random()
    if r < 0.05:
        return [0] * H
    if r < 0.1:
        return [m - 1] * H
    return [rng.randrange(m) for _ in range(H)]


def bitrev(j, l):
    return int(format(j, f"0{l}b")[::-1], 2) if l else 0


def py_dft(a, l, n, e, M, m):
    """a-hat_j = zeta^{j'} sum_i omega_L^{i j'} a_i, omega_L = y^{M/L}, zeta = y^e (Horner)."""
    L, H = 1 << l, M // 2
    w = M // L
    out = []
    for j in range(n):
        jr = bitrev(j, l)
        acc = [0] * H
        for x in reversed(a):  # Horner in t = omega_L^{j'}
            acc = py_ypow(acc, w * jr, M, m)
            acc = [(u + v) % m for u, v in zip(acc, x)]
        out.append(py_ypow(acc, e * jr, M, m))
    return out


@pytest.mark.parametrize("M,m", [(2, 3), (8, 5), (16, 65537), (32, (1 << 61) - 1), (64, (1 << 62) + 3)])
def test_ring_operations_match_polynomial_arithmetic(orc, M, m):
    rng = random.Random(M)
    H = M // 2
    for _ in range(10):
        a, b = rand_elem(rng, H, m), rand_elem(rng, H, m)
        assert orc.sn_add(a, b, M, m) == [(x + y) % m for x, y in zip(a, b)]
        assert orc.sn_sub(a, b, M, m) == [(x - y) % m for x, y in zip(a, b)]
        assert orc.sn_mul(a, b, M, m) == py_mul(a, b, m)
        h = orc.sn_half(a, M, m)
        assert [(2 * v) % m for v in h] == a
        for k in (0, 1, H - 1, H, H + 1, M - 1, rng.randrange(-3 * M, 3 * M)):
            assert orc.sn_ypow(a, k, M, m) == py_ypow(a, k, M, m), k
    # y^{M/2} = -1 and y^M = 1
    one = [1] + [0] * (H - 1)
    assert orc.sn_ypow(one, H, M, m) == [m - 1] + [0] * (H - 1)
    assert orc.sn_ypow(one, M, M, m) == one


@pytest.mark.parametrize("M,m", [(8, 5), (16, 65537), (32, (1 << 61) - 1)])
def test_y_is_a_principal_root(orc, M, m):
    """sum_i omega^{i j} is L for j = 0 and 0 otherwise: the transform of the all-ones vector
    at L = M (zeta = 1) is L at output 0 (j' = 0) and zero elsewhere."""
    l = M.bit_length() - 1
    H = M // 2
    ones = [[1] + [0] * (H - 1)] * M
    out = orc.sn_vals(orc.sn_dft_brute(orc.sn_cells(ones, M), l, M, M, 0, M, m), M, M)
    assert out[0] == [M % m] + [0] * (H - 1)
    assert all(v == [0] * H for v in out[1:])


@pytest.mark.parametrize("M,m,l", [(8, 5, 3), (16, 65537, 3), (16, 3, 4), (32, (1 << 61) - 1, 2)])
def test_dft_matches_horner(orc, M, m, l):
    rng = random.Random(M * 7 + l)
    L, H = 1 << l, M // 2
    for e in (0, 1, M - 1, rng.randrange(M)):
        a = [rand_elem(rng, H, m) for _ in range(L)]
        out = orc.sn_vals(orc.sn_dft_brute(orc.sn_cells(a, M), l, L, L, e, M, m), M, L)
        assert out == py_dft(a, l, L, e, M, m), e


def brute(orc, vals, l, z, n, e, M, m):
    x = orc.sn_cells(vals, M, count=1 << l)
    return orc.sn_vals(orc.sn_dft_brute(x, l, z, n, e, M, m), M, n)


@pytest.mark.parametrize("M,m,l", [(8, 5, 2), (8, 3, 3), (16, 65537, 4), (32, (1 << 61) - 1, 4), (64, (1 << 62) + 3, 3)])
def test_tft_itft_exhaustive(orc, M, m, l):
    """Every (z, n) of Algorithm 1 against the DFT, and every (z, n, f) of Algorithm 2 against
    its definition, over S[y]/(y^{M/2}+1)."""
    rng = random.Random(M + 31 * l)
    L, H = 1 << l, M // 2
    for z in range(1, L + 1):
        e = rng.randrange(M)
        a = [rand_elem(rng, H, m) for _ in range(z)]
        hat = brute(orc, a, l, z, L, e, M, m)
        for n in range(1, L + 1):
            x = orc.sn_cells(a, M, count=L)
            orc.sn_tft(x, l, z, n, e, M, m)
            assert orc.sn_vals(x, M, n) == hat[:n], (z, n, e)
        for n in range(0, z + 1):
            for f in (0, 1):
                if not 1 <= n + f <= L:
                    continue
                inp = hat[:n] + [[(L * v) % m for v in c] for c in a[n:z]]
                want = [[(L * v) % m for v in c] for c in a[:n]] + ([hat[n]] if f else [])
                x = orc.sn_cells(inp, M, count=L)
                orc.sn_itft(x, l, z, n, f, e, M, m)
                assert orc.sn_vals(x, M, n + f) == want, (z, n, f, e)


def test_split_independence(orc):
    M, m, l = 64, (1 << 61) - 1, 5
    rng = random.Random(5)
    L, H = 1 << l, M // 2
    for z, n in ((L, L), (19, 23), (7, 30)):
        a = [rand_elem(rng, H, m) for _ in range(z)]
        ref = None
        for policy, seed in ((orc.SPLIT_BALANCED, 0), (orc.SPLIT_DC, 0), (orc.SPLIT_RANDOM, 3), (orc.SPLIT_RANDOM, 9)):
            x = orc.sn_cells(a, M, count=L)
            orc.sn_tft(x, l, z, n, 3, M, m, policy=policy, seed=seed)
            got = orc.sn_vals(x, M, n)
            ref = ref or got
            assert got == ref, (policy, seed)


def test_convolution_theorem(orc):
    """TFT, pointwise products in R, ITFT, division by L: the cyclic convolution in R[x] of
    length L (zeta = 1), against a schoolbook convolution written here."""
    M, m, l = 16, 65537, 4
    rng = random.Random(9)
    L, H = 1 << l, M // 2
    f = [rand_elem(rng, H, m) for _ in range(L)]
    g = [rand_elem(rng, H, m) for _ in range(L)]
    F, G = orc.sn_cells(f, M), orc.sn_cells(g, M)
    orc.sn_tft(F, l, L, L, 0, M, m)
    orc.sn_tft(G, l, L, L, 0, M, m)
    P = orc.sn_cells([orc.sn_mul(a, b, M, m) for a, b in zip(orc.sn_vals(F, M, L), orc.sn_vals(G, M, L))], M)
    orc.sn_itft(P, l, L, L, 0, 0, M, m)
    inv = pow(L, -1, m)
    got = [[(v * inv) % m for v in c] for c in orc.sn_vals(P, M, L)]
    want = [[0] * H for _ in range(L)]
    for i in range(L):
        for j in range(L):
            t = py_mul(f[i], g[j], m)
            k = (i + j) % L
            want[k] = [(u + v) % m for u, v in zip(want[k], t)]
    assert got == want
