/*
 * Oracle: the coefficient ring of the Schoenhage-Nussbaumer algorithm (Sec. 5.2),
 * R = S[y]/(y^{M/2} + 1) with S = Z/mZ, m odd. TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * An element is its H = M/2 coefficients in S, each a uint64 in [0, m). y is a principal
 * M-th root of unity in R (y^{M/2} = -1 and 2 is invertible modulo odd m), so multiplying by
 * a power of omega_L = y^{M/L} is a negacyclic shift of the coefficient vector: the
 * coefficients that pass y^{M/2} come back at the bottom negated.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

static int sn_ok(int64_t M, uint64_t m)
{
    return M >= 2 && (M & (M - 1)) == 0 && (m & 1u) && m >= 3 && m < ((uint64_t)1 << 63);
}

static uint64_t addm(uint64_t a, uint64_t b, uint64_t m)
{
    uint64_t s = a + b; /* a, b < m < 2^63: no overflow */
    return s >= m ? s - m : s;
}

static uint64_t subm(uint64_t a, uint64_t b, uint64_t m) { return a >= b ? a - b : a + (m - b); }

static uint64_t negm(uint64_t a, uint64_t m) { return a ? m - a : 0; }

int orc_sn_add(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t M, uint64_t m)
{
    if (!sn_ok(M, m)) return -1;
    for (int64_t t = 0; t < M / 2; t++) r[t] = addm(a[t], b[t], m);
    return 0;
}

int orc_sn_sub(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t M, uint64_t m)
{
    if (!sn_ok(M, m)) return -1;
    for (int64_t t = 0; t < M / 2; t++) r[t] = subm(a[t], b[t], m);
    return 0;
}

/* r = y^k a, k taken mod M; r may alias a */
int orc_sn_ypow(uint64_t *r, const uint64_t *a, int64_t k, int64_t M, uint64_t m)
{
    if (!sn_ok(M, m)) return -1;
    const int64_t H = M / 2;
    k %= M;
    if (k < 0) k += M;
    int neg = 0;
    if (k >= H) { /* y^H = -1 */
        neg = 1;
        k -= H;
    }
    uint64_t *t = malloc((size_t)H * 8);
    for (int64_t i = 0; i < H; i++) {
        int64_t j = i + k; /* coefficient i of a moves to j */
        uint64_t v = a[i];
        if (j >= H) {
            j -= H;
            v = negm(v, m);
        }
        t[j] = neg ? negm(v, m) : v;
    }
    memcpy(r, t, (size_t)H * 8);
    free(t);
    return 0;
}

/* r = a / 2 coefficient-wise (2 is invertible modulo odd m) */
int orc_sn_half(uint64_t *r, const uint64_t *a, int64_t M, uint64_t m)
{
    if (!sn_ok(M, m)) return -1;
    for (int64_t t = 0; t < M / 2; t++) r[t] = (a[t] & 1u) ? (a[t] >> 1) + (m >> 1) + 1 : a[t] >> 1;
    return 0;
}

/* r = a b in R: the negacyclic product of the coefficient vectors, schoolbook, modulo m */
int orc_sn_mul(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t M, uint64_t m)
{
    if (!sn_ok(M, m)) return -1;
    const int64_t H = M / 2;
    uint64_t *t = calloc((size_t)H, 8);
    for (int64_t i = 0; i < H; i++)
        for (int64_t j = 0; j < H; j++) {
            uint64_t p = (uint64_t)(((unsigned __int128)a[i] * b[j]) % m);
            int64_t k = i + j;
            if (k < H)
                t[k] = addm(t[k], p, m);
            else
                t[k - H] = subm(t[k - H], p, m); /* y^H = -1 */
        }
    memcpy(r, t, (size_t)H * 8);
    free(t);
    return 0;
}
