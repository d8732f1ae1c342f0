"""Pins for the oracle's Z[x] products (Sec. 2 R[X] product, Sec. 5.1 Schoenhage-Strassen).

The TFT-based product is checked against a schoolbook product on Python integers (a textbook
routine, independent of the oracle's bignum) and against the oracle's own schoolbook code.
"""
import random

import numpy as np
import pytest

import workloads


def to_ints(arr, length, limbs, signed):
    out = []
    for i in range(length):
        v = 0
        for k in range(limbs):
            v |= int(arr[i * limbs + k]) << (64 * k)
        if signed and v >> (64 * limbs - 1):
            v -= 1 << (64 * limbs)
        out.append(v)
    return out


def py_product(f, g):
    h = [0] * (len(f) + len(g) - 1)
    for i, a in enumerate(f):
        for j, b in enumerate(g):
            h[i + j] += a * b
    return h


@pytest.mark.parametrize("lf,lg,bits,signed", [
    (1, 1, 10, False), (1, 7, 64, False), (5, 3, 100, True), (37, 20, 130, False),
    (64, 64, 64, True), (100, 29, 200, True), (33, 31, 500, False),
])
def test_zx_mul_matches_python(orc, lf, lg, bits, signed):
    limbs = (bits + 1 + 63) // 64
    f = workloads.coefficients(lf * 7 + lg, lf, bits, limbs, signed)
    g = workloads.coefficients(lf * 11 + lg + 1, lg, bits, limbs, signed)
    ref = py_product(to_ints(f, lf, limbs, signed), to_ints(g, lg, limbs, signed))
    limbs_h = (2 * bits + 8 + 64) // 64
    h, l, N = orc.zx_mul(f, lf, limbs, g, lg, limbs, limbs_h, signed, bits, bits)
    assert to_ints(h, lf + lg - 1, limbs_h, signed) == ref
    hs = orc.zx_schoolbook(f, lf, limbs, g, lg, limbs, limbs_h, signed)
    assert to_ints(hs, lf + lg - 1, limbs_h, signed) == ref
    assert (1 << l) >= lf + lg - 1 and (2 * N) % (1 << l) == 0


def test_extreme_coefficients(orc):
    # all-ones coefficients of full width: the largest possible product coefficients
    bits, lf, lg = 128, 40, 50
    f = np.full(lf * 2, 0xFFFFFFFFFFFFFFFF, np.uint64)
    g = np.full(lg * 2, 0xFFFFFFFFFFFFFFFF, np.uint64)
    h, _, _ = orc.zx_mul(f, lf, 2, g, lg, 2, 5, False, bits, bits)
    ref = py_product([(1 << bits) - 1] * lf, [(1 << bits) - 1] * lg)
    assert to_ints(h, lf + lg - 1, 5, False) == ref


def test_eval_mod_spot_check(orc):
    P = (1 << 61) - 1
    rng = random.Random(4)
    f = workloads.coefficients(9, 50, 300, 5, True)
    g = workloads.coefficients(10, 40, 300, 5, True)
    h, _, _ = orc.zx_mul(f, 50, 5, g, 40, 5, 11, True, 300, 300)
    for _ in range(5):
        t = rng.randrange(P)
        lhs = orc.poly_eval_mod(f, 50, 5, True, t, P) * orc.poly_eval_mod(g, 40, 5, True, t, P) % P
        assert lhs == orc.poly_eval_mod(h, 89, 11, True, t, P)


def test_plan_medium_product(orc):
    # 3000 x 2500 product of 2000-bit coefficients: 5499 outputs, L = 2^13, N = 4096
    l, N = orc.zx_plan(3000, 2000, 2500, 2000, False)
    assert (l, N) == (13, 4096)
