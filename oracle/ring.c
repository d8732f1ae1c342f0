/*
 * Oracle: plain multi-limb arithmetic in R = Z/(2^N+1) (Sec. 2: R = Z/(2^{M/2}+1), omega = 2;
 * Sec. 5.1: reduction modulo 2^N+1 and multiplication by powers of omega are cheap).
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * Values are canonical residues in [0, 2^N] stored in W = N/64 + 1 little-endian limbs.
 * Everything here is written for clarity, not speed: rotations are a literal shift
 * followed by the textbook reduction x = sum_i d_i 2^{iN} = sum_i (-1)^i d_i (mod 2^N+1).
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static int n_ok(int64_t N) { return N >= 64 && (N % 64) == 0; }
static int64_t limbs_of(int64_t N) { return N / 64 + 1; }

/* r = a + b over n limbs, returns the carry out */
static uint64_t big_add(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t n)
{
    uint64_t c = 0;
    for (int64_t i = 0; i < n; i++) {
        u128 s = (u128)a[i] + b[i] + c;
        r[i] = (uint64_t)s;
        c = (uint64_t)(s >> 64);
    }
    return c;
}

/* r = a - b over n limbs, returns the borrow out */
static uint64_t big_sub(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t n)
{
    uint64_t br = 0;
    for (int64_t i = 0; i < n; i++) {
        uint64_t ai = a[i], bi = b[i];
        uint64_t d = ai - bi - br;
        br = (ai < bi) || (ai == bi && br) ? 1u : 0u;
        r[i] = d;
    }
    return br;
}

static int big_cmp(const uint64_t *a, const uint64_t *b, int64_t n)
{
    for (int64_t i = n - 1; i >= 0; i--) {
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    }
    return 0;
}

/* p = 2^N + 1 in W limbs */
static void set_p(uint64_t *p, int64_t N)
{
    int64_t W = limbs_of(N);
    memset(p, 0, (size_t)W * 8);
    p[0] = 1;
    p[W - 1] = 1; /* bit N: N is a multiple of 64, so it is bit 0 of limb N/64 = W-1 */
}

int orc_ring_reduce(uint64_t *r, const uint64_t *x, int64_t xn, int64_t N)
{
    if (!n_ok(N) || xn < 0) return -1;
    int64_t W = limbs_of(N), D = N / 64; /* limbs per N-bit digit */
    uint64_t *P = calloc((size_t)(W + 1), 8), *Q = calloc((size_t)(W + 1), 8);
    uint64_t *dig = calloc((size_t)(W + 1), 8), *pp = calloc((size_t)(W + 1), 8);
    /* P = sum of even digits, Q = sum of odd digits; x = sum_i d_i 2^{iN} */
    int64_t ndig = (xn + D - 1) / D;
    for (int64_t i = 0; i < ndig; i++) {
        memset(dig, 0, (size_t)(W + 1) * 8);
        for (int64_t k = 0; k < D && i * D + k < xn; k++) dig[k] = x[i * D + k];
        if (i % 2 == 0) big_add(P, P, dig, W + 1);
        else big_add(Q, Q, dig, W + 1);
    }
    /* v = |P - Q|, remember the sign; 2^N = -1 so x = P - Q (mod p) */
    int neg = big_cmp(P, Q, W + 1) < 0;
    uint64_t *v = neg ? Q : P;
    big_sub(v, v, neg ? P : Q, W + 1);
    /* fold once: v = lo + hi 2^N with hi < 2^128 tiny compared with p; v = lo - hi (mod p) */
    uint64_t lo_hi[2] = { v[D], v[D + 1] }; /* hi = limbs D and D+1 (W+1 = D+2 limbs) */
    memset(dig, 0, (size_t)(W + 1) * 8);
    dig[0] = lo_hi[0];
    dig[1] = lo_hi[1];
    v[D] = 0;
    v[D + 1] = 0;
    if (big_cmp(v, dig, W + 1) >= 0) {
        big_sub(v, v, dig, W + 1);
    } else {
        set_p(pp, N);
        big_add(v, v, pp, W + 1);
        big_sub(v, v, dig, W + 1);
    }
    /* v is now in [0, 2^N]; apply the sign */
    int zero = 1;
    for (int64_t i = 0; i < W; i++) zero &= (v[i] == 0);
    if (neg && !zero) {
        set_p(pp, N);
        big_sub(v, pp, v, W);
    }
    memcpy(r, v, (size_t)W * 8);
    free(P); free(Q); free(dig); free(pp);
    return 0;
}

int orc_ring_add(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t N)
{
    if (!n_ok(N)) return -1;
    int64_t W = limbs_of(N);
    uint64_t *t = malloc((size_t)W * 8), *p = malloc((size_t)W * 8);
    big_add(t, a, b, W); /* a + b <= 2^{N+1}: no overflow out of W limbs */
    set_p(p, N);
    if (big_cmp(t, p, W) >= 0) big_sub(t, t, p, W);
    memcpy(r, t, (size_t)W * 8);
    free(t); free(p);
    return 0;
}

int orc_ring_sub(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t N)
{
    if (!n_ok(N)) return -1;
    int64_t W = limbs_of(N);
    uint64_t *t = malloc((size_t)W * 8), *p = malloc((size_t)W * 8);
    if (big_cmp(a, b, W) >= 0) {
        big_sub(t, a, b, W);
    } else {
        set_p(p, N);
        big_add(t, a, p, W); /* a + p <= 2^{N+1} + 1 fits */
        big_sub(t, t, b, W);
    }
    memcpy(r, t, (size_t)W * 8);
    free(t); free(p);
    return 0;
}

int orc_ring_mul2exp(uint64_t *r, const uint64_t *a, int64_t k, int64_t N)
{
    if (!n_ok(N) || k < 0) return -1;
    int64_t W = limbs_of(N);
    k %= 2 * N;
    /* literal shift a << k into a buffer wide enough, then reduce */
    int64_t q = k / 64, s = k % 64, xn = W + q + 1;
    uint64_t *x = calloc((size_t)xn, 8);
    for (int64_t i = 0; i < W; i++) {
        x[i + q] |= a[i] << s;
        if (s) x[i + q + 1] |= a[i] >> (64 - s);
    }
    int rc = orc_ring_reduce(r, x, xn, N);
    free(x);
    return rc;
}

int orc_ring_div2(uint64_t *r, const uint64_t *a, int64_t N)
{
    if (!n_ok(N)) return -1;
    int64_t W = limbs_of(N);
    uint64_t *t = malloc((size_t)W * 8), *p = malloc((size_t)W * 8);
    memcpy(t, a, (size_t)W * 8);
    if (t[0] & 1) { /* odd: a + p is even and represents the same class */
        set_p(p, N);
        big_add(t, t, p, W);
    }
    for (int64_t i = 0; i < W; i++) t[i] = (t[i] >> 1) | (i + 1 < W ? t[i + 1] << 63 : 0);
    memcpy(r, t, (size_t)W * 8);
    free(t); free(p);
    return 0;
}

int orc_ring_mul(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t N)
{
    if (!n_ok(N)) return -1;
    int64_t W = limbs_of(N);
    uint64_t *x = calloc((size_t)(2 * W), 8);
    for (int64_t i = 0; i < W; i++) {
        uint64_t c = 0;
        for (int64_t j = 0; j < W; j++) {
            u128 t = (u128)a[i] * b[j] + x[i + j] + c;
            x[i + j] = (uint64_t)t;
            c = (uint64_t)(t >> 64);
        }
        x[i + W] = c;
    }
    int rc = orc_ring_reduce(r, x, 2 * W, N);
    free(x);
    return rc;
}
