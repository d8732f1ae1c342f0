/*
 * Oracle: the weighted DFT by definition and the paper's two recursive algorithms.
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 *   orc_dft_brute   Eq. (dft), Sec. 2: a-hat_j = zeta^{j'} sum_i omega_L^{i j'} a_i
 *   orc_tft         Algorithm 1 (Sec. 3), recursing as written, on (pointer, stride) views
 *                   of rows and columns (Sec. 2: c_u and r_u), zeta carried as an exponent
 *                   (Sec. 6), with a base-case counter for Theorem 1
 *   orc_itft        Algorithm 2 (Sec. 4), same conventions, counter for Theorem 2
 *
 * Exponent bookkeeping (all mod 2N, because omega = 2 has order 2N in Z/(2^N+1)):
 *   omega_L = 2^{2N/L}; column u of an L1 x L2 split uses zeta * omega_L^u -> e + u * 2N/L;
 *   rows use zeta^{L1} -> e * L1; zeta^{-1} -> 2N - e; doubling -> 1; halving -> 2N - 1.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

typedef struct {
    int kind;       /* 0: Z/(2^N+1) with omega = 2; 1: S[y]/(y^{M/2}+1), S = Z/mZ, omega = y;
                       2: Z/(2^N+1) with omega = sqrt2 = 2^{3N/4} - 2^{N/4} (order 4N) */
    uint64_t m;     /* kind 1: the modulus of S */
    int64_t N, W, twoN; /* kind 1: N = M/2 coefficients, W = M/2 words, twoN = M */
    int policy;
    int top_l1;     /* ORC_SPLIT_TOP: l1 at the outermost level */
    int depth;      /* current recursion depth (0 = outermost) */
    uint64_t rng;   /* ORC_SPLIT_RANDOM state */
    int64_t count;  /* base-case executions */
    uint64_t *tmp;  /* two scratch cells */
} ctx_t;

static int n_ok(int64_t N) { return N >= 64 && (N % 64) == 0; }

static int64_t emod(int64_t a, int64_t m)
{
    int64_t r = a % m;
    return r < 0 ? r + m : r;
}

static uint64_t rng_next(uint64_t *s)
{
    /* splitmix64 step, only used to draw split points */
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* l1 for a sub-transform of length 2^l, l >= 2 (Sec. 2: any 1 < L1 < L is valid by the
 * decomposition; the paper's own choice is L1 = 2^floor(l/2)). */
static int choose_l1(ctx_t *c, int l)
{
    switch (c->policy) {
    case ORC_SPLIT_DC: return 1;
    case ORC_SPLIT_RANDOM: return 1 + (int)(rng_next(&c->rng) % (uint64_t)(l - 1));
    case ORC_SPLIT_TOP:
        if (c->depth == 0 && c->top_l1 >= 1 && c->top_l1 < l) return c->top_l1;
        return l / 2;
    default: return l / 2;
    }
}

/* ring helpers on cells */
static void cp(ctx_t *c, uint64_t *d, const uint64_t *s) { memmove(d, s, (size_t)c->W * 8); }
static void add(ctx_t *c, uint64_t *r, const uint64_t *a, const uint64_t *b)
{
    if (c->kind == 1) orc_sn_add(r, a, b, c->twoN, c->m);
    else orc_ring_add(r, a, b, c->N);
}
static void sub(ctx_t *c, uint64_t *r, const uint64_t *a, const uint64_t *b)
{
    if (c->kind == 1) orc_sn_sub(r, a, b, c->twoN, c->m);
    else orc_ring_sub(r, a, b, c->N);
}
/* r = sqrt2^k a over Z/(2^N+1), k mod 4N: 2^{k/2} a for even k, and for odd k
 * 2^{(k-1)/2} (2^{3N/4} - 2^{N/4}) a, a difference of two rotations */
static void rot_sqrt2(ctx_t *c, uint64_t *r, const uint64_t *a, int64_t k)
{
    k = emod(k, 4 * c->N);
    int64_t h = k >> 1;
    if (!(k & 1)) {
        orc_ring_mul2exp(r, a, emod(h, 2 * c->N), c->N);
        return;
    }
    uint64_t *t = c->tmp + 2 * c->W;
    orc_ring_mul2exp(t, a, emod(h + 3 * c->N / 4, 2 * c->N), c->N);
    orc_ring_mul2exp(r, a, emod(h + c->N / 4, 2 * c->N), c->N);
    orc_ring_sub(r, t, r, c->N);
}

/* r = omega^k a: a rotation by k bits (kind 0), a negacyclic shift by k places (kind 1), or a
 * power of sqrt2 (kind 2) */
static void rot(ctx_t *c, uint64_t *r, const uint64_t *a, int64_t k)
{
    if (c->kind == 1) orc_sn_ypow(r, a, emod(k, c->twoN), c->twoN, c->m);
    else if (c->kind == 2) rot_sqrt2(c, r, a, k);
    else orc_ring_mul2exp(r, a, emod(k, c->twoN), c->N);
}
static void half(ctx_t *c, uint64_t *r, const uint64_t *a)
{
    if (c->kind == 1) orc_sn_half(r, a, c->twoN, c->m);
    else orc_ring_div2(r, a, c->N);
}

static unsigned bitrev(uint64_t j, int l)
{
    uint64_t r = 0;
    for (int i = 0; i < l; i++) r |= ((j >> i) & 1u) << (l - 1 - i);
    return (unsigned)r;
}

/* Eq. (dft) term by term: zeta^{j'} omega_L^{i j'} = omega^{e j' + w i j'} with w = twoN / L */
static void dft_brute(ctx_t *c, uint64_t *out, const uint64_t *in, int64_t stride, int l, int64_t z, int64_t n,
                      int64_t e)
{
    int64_t L = (int64_t)1 << l, W = c->W, twoN = c->twoN;
    int64_t w = twoN / L;
    uint64_t *acc = calloc((size_t)W, 8), *term = calloc((size_t)W, 8);
    for (int64_t j = 0; j < n; j++) {
        int64_t jr = bitrev((uint64_t)j, l);
        memset(acc, 0, (size_t)W * 8);
        for (int64_t i = 0; i < z; i++) {
            int64_t k = emod(emod(e, twoN) * jr + w * emod(i * jr, L), twoN);
            rot(c, term, in + i * stride, k);
            add(c, acc, acc, term);
        }
        memcpy(out + j * stride, acc, (size_t)W * 8);
    }
    free(acc);
    free(term);
}

int orc_dft_brute(uint64_t *out, const uint64_t *in, int64_t stride, int l, int64_t z, int64_t n,
                  int64_t e, int64_t N)
{
    if (!n_ok(N) || l < 1 || l > 30) return -1;
    int64_t L = (int64_t)1 << l, W = N / 64 + 1, twoN = 2 * N;
    if (twoN % L != 0 || z < 0 || z > L || n < 0 || n > L || stride < W) return -1;
    ctx_t c;
    memset(&c, 0, sizeof c);
    c.N = N;
    c.W = W;
    c.twoN = twoN;
    dft_brute(&c, out, in, stride, l, z, n, e);
    return 0;
}

/* ------------------------------------------------------------------ Algorithm 1 */

static void tft_rec(ctx_t *c, uint64_t *x, int64_t s, int l, int64_t e, int64_t z, int64_t n)
{
    if (l == 1) {
        /* base case L = 2: (a0, a1) -> (a0 + a1, zeta (a0 - a1)), pruned by z and n */
        c->count++;
        if (!x) return;
        uint64_t *x0 = x, *x1 = x + s, *t = c->tmp;
        if (n == 2 && z == 2) {
            sub(c, t, x0, x1);
            add(c, x0, x0, x1);
            rot(c, x1, t, e);
        } else if (n == 2 && z == 1) {
            rot(c, x1, x0, e);
        } else if (n == 1 && z == 2) {
            add(c, x0, x0, x1);
        }
        return;
    }
    int l1 = choose_l1(c, l), l2 = l - l1;
    int64_t L = (int64_t)1 << l, L1 = (int64_t)1 << l1, L2 = (int64_t)1 << l2;
    int64_t w = c->twoN / L;
    int64_t n2 = n % L2, n1 = n / L2, n1p = (n + L2 - 1) / L2;
    int64_t z2 = z % L2, z1 = z / L2, z2p = z1 > 0 ? L2 : z2;
    c->depth++;
    /* column transforms: column u is x_u, x_{u+L2}, ... (stride L2 cells) */
    for (int64_t u = 0; u < z2; u++)
        tft_rec(c, x ? x + u * s : NULL, s * L2, l1, emod(e + u * w, c->twoN), z1 + 1, n1p);
    for (int64_t u = z2; u < z2p; u++)
        tft_rec(c, x ? x + u * s : NULL, s * L2, l1, emod(e + u * w, c->twoN), z1, n1p);
    /* row transforms: row u is x_{u L2} .. x_{u L2 + L2 - 1} (stride 1 cell) */
    for (int64_t u = 0; u < n1; u++)
        tft_rec(c, x ? x + u * L2 * s : NULL, s, l2, emod(e * L1, c->twoN), z2p, L2);
    if (n2 > 0)
        tft_rec(c, x ? x + n1 * L2 * s : NULL, s, l2, emod(e * L1, c->twoN), z2p, n2);
    c->depth--;
}

/* ------------------------------------------------------------------ Algorithm 2 */

static void itft_rec(ctx_t *c, uint64_t *x, int64_t s, int l, int64_t e, int64_t z, int64_t n, int f)
{
    if (l == 1) {
        c->count++;
        if (!x) return;
        uint64_t *x0 = x, *x1 = x + s, *t = c->tmp, *t2 = c->tmp + c->W;
        if (n == 2) {
            /* (x0 + zeta^{-1} x1, x0 - zeta^{-1} x1) */
            rot(c, t, x1, -e);
            sub(c, x1, x0, t);
            add(c, x0, x0, t);
        } else if (n == 1 && f == 1 && z == 2) {
            /* cross butterfly: (2 x0 - x1, zeta (x0 - x1)) */
            sub(c, t, x0, x1);
            add(c, t2, x0, t); /* x0 + (x0 - x1) = 2 x0 - x1 */
            rot(c, x1, t, e);
            cp(c, x0, t2);
        } else if (n == 1 && f == 1 && z == 1) {
            /* (2 x0, zeta x0) */
            rot(c, x1, x0, e);
            add(c, x0, x0, x0);
        } else if (n == 1 && f == 0 && z == 2) {
            sub(c, t, x0, x1);
            add(c, x0, x0, t);
        } else if (n == 1 && f == 0 && z == 1) {
            add(c, x0, x0, x0);
        } else if (n == 0 && z == 2) {
            add(c, t, x0, x1);
            half(c, x0, t);
        } else if (n == 0 && z == 1) {
            half(c, x0, x0);
        }
        return;
    }
    int l1 = choose_l1(c, l), l2 = l - l1;
    int64_t L = (int64_t)1 << l, L1 = (int64_t)1 << l1, L2 = (int64_t)1 << l2;
    int64_t w = c->twoN / L;
    int64_t n2 = n % L2, n1 = n / L2;
    int64_t z2 = z % L2, z1 = z / L2;
    int fp = (n2 + f > 0) ? 1 : 0;
    int64_t z2p = z1 > 0 ? L2 : z2;
    int64_t m = n2 < z2 ? n2 : z2, mp = n2 > z2 ? n2 : z2;
    int64_t er = emod(e * L1, c->twoN);
    c->depth++;
    /* rows that are complete on input */
    for (int64_t u = 0; u < n1; u++)
        itft_rec(c, x ? x + u * L2 * s : NULL, s, l2, er, L2, L2, 0);
    /* rightmost columns */
    for (int64_t u = n2; u < mp; u++)
        itft_rec(c, x ? x + u * s : NULL, s * L2, l1, emod(e + u * w, c->twoN), z1 + 1, n1, fp);
    for (int64_t u = mp; u < z2p; u++)
        itft_rec(c, x ? x + u * s : NULL, s * L2, l1, emod(e + u * w, c->twoN), z1, n1, fp);
    /* the last (partial) row */
    if (fp)
        itft_rec(c, x ? x + n1 * L2 * s : NULL, s, l2, er, z2p, n2, f);
    /* leftmost columns */
    for (int64_t u = 0; u < m; u++)
        itft_rec(c, x ? x + u * s : NULL, s * L2, l1, emod(e + u * w, c->twoN), z1 + 1, n1 + 1, 0);
    for (int64_t u = m; u < n2; u++)
        itft_rec(c, x ? x + u * s : NULL, s * L2, l1, emod(e + u * w, c->twoN), z1, n1 + 1, 0);
    c->depth--;
}

static int setup(ctx_t *c, int64_t N, int64_t stride, int l, int policy, int top_l1, uint64_t seed,
                 int need_x)
{
    memset(c, 0, sizeof *c);
    if (!n_ok(N) || l < 1 || l > 30) return -1;
    c->N = N;
    c->W = N / 64 + 1;
    c->twoN = 2 * N;
    if (c->twoN % ((int64_t)1 << l) != 0) return -1; /* omega_L must exist: L | 2N */
    if (need_x && stride < c->W) return -1;
    c->policy = policy;
    c->top_l1 = top_l1;
    c->rng = seed;
    c->tmp = calloc((size_t)(3 * c->W), 8);
    return 0;
}

int orc_tft(uint64_t *x, int64_t stride, int l, int64_t z, int64_t n, int64_t e, int64_t N,
            int policy, int top_l1, uint64_t seed, int64_t *count)
{
    ctx_t c;
    if (setup(&c, N, stride, l, policy, top_l1, seed, x != NULL)) return -1;
    int64_t L = (int64_t)1 << l;
    if (z < 1 || z > L || n < 1 || n > L) { free(c.tmp); return -1; }
    tft_rec(&c, x, stride, l, emod(e, c.twoN), z, n);
    if (count) *count += c.count;
    free(c.tmp);
    return 0;
}

int orc_itft(uint64_t *x, int64_t stride, int l, int64_t z, int64_t n, int f, int64_t e, int64_t N,
             int policy, int top_l1, uint64_t seed, int64_t *count)
{
    ctx_t c;
    if (setup(&c, N, stride, l, policy, top_l1, seed, x != NULL)) return -1;
    int64_t L = (int64_t)1 << l;
    if ((f != 0 && f != 1) || z < 1 || z > L || n < 0 || n + f < 1 || n + f > L || z < n) {
        free(c.tmp);
        return -1;
    }
    itft_rec(&c, x, stride, l, emod(e, c.twoN), z, n, f);
    if (count) *count += c.count;
    free(c.tmp);
    return 0;
}

/* ------------------------------------------------------------------ phase stepping */

int orc_tft_phases(uint64_t *x, int64_t s, int l, int l1, int64_t z, int64_t n, int64_t e, int64_t N,
                   int stop_after)
{
    ctx_t c;
    if (setup(&c, N, s, l, ORC_SPLIT_BALANCED, 0, 0, 1)) return -1;
    int64_t L = (int64_t)1 << l;
    if (l < 2 || l1 < 1 || l1 >= l || z < 1 || z > L || n < 1 || n > L) { free(c.tmp); return -1; }
    int l2 = l - l1;
    int64_t L1 = (int64_t)1 << l1, L2 = (int64_t)1 << l2, w = c.twoN / L;
    e = emod(e, c.twoN);
    int64_t n2 = n % L2, n1 = n / L2, n1p = (n + L2 - 1) / L2;
    int64_t z2 = z % L2, z1 = z / L2, z2p = z1 > 0 ? L2 : z2;
    c.depth = 1;
    if (stop_after >= 1) {
        for (int64_t u = 0; u < z2; u++) tft_rec(&c, x + u * s, s * L2, l1, emod(e + u * w, c.twoN), z1 + 1, n1p);
        for (int64_t u = z2; u < z2p; u++) tft_rec(&c, x + u * s, s * L2, l1, emod(e + u * w, c.twoN), z1, n1p);
    }
    if (stop_after >= 2) {
        for (int64_t u = 0; u < n1; u++) tft_rec(&c, x + u * L2 * s, s, l2, emod(e * L1, c.twoN), z2p, L2);
        if (n2 > 0) tft_rec(&c, x + n1 * L2 * s, s, l2, emod(e * L1, c.twoN), z2p, n2);
    }
    free(c.tmp);
    return 0;
}

int orc_itft_phases(uint64_t *x, int64_t s, int l, int l1, int64_t z, int64_t n, int f, int64_t e,
                    int64_t N, int stop_after)
{
    ctx_t c;
    if (setup(&c, N, s, l, ORC_SPLIT_BALANCED, 0, 0, 1)) return -1;
    int64_t L = (int64_t)1 << l;
    if (l < 2 || l1 < 1 || l1 >= l || (f != 0 && f != 1) || z < 1 || z > L || n < 0 ||
        n + f < 1 || n + f > L || z < n) {
        free(c.tmp);
        return -1;
    }
    int l2 = l - l1;
    int64_t L1 = (int64_t)1 << l1, L2 = (int64_t)1 << l2, w = c.twoN / L;
    e = emod(e, c.twoN);
    int64_t n2 = n % L2, n1 = n / L2, z2 = z % L2, z1 = z / L2;
    int fp = (n2 + f > 0) ? 1 : 0;
    int64_t z2p = z1 > 0 ? L2 : z2;
    int64_t m = n2 < z2 ? n2 : z2, mp = n2 > z2 ? n2 : z2;
    int64_t er = emod(e * L1, c.twoN);
    c.depth = 1;
    if (stop_after >= 1)
        for (int64_t u = 0; u < n1; u++) itft_rec(&c, x + u * L2 * s, s, l2, er, L2, L2, 0);
    if (stop_after >= 2) {
        for (int64_t u = n2; u < mp; u++) itft_rec(&c, x + u * s, s * L2, l1, emod(e + u * w, c.twoN), z1 + 1, n1, fp);
        for (int64_t u = mp; u < z2p; u++) itft_rec(&c, x + u * s, s * L2, l1, emod(e + u * w, c.twoN), z1, n1, fp);
    }
    if (stop_after >= 3 && fp) itft_rec(&c, x + n1 * L2 * s, s, l2, er, z2p, n2, f);
    if (stop_after >= 4) {
        for (int64_t u = 0; u < m; u++) itft_rec(&c, x + u * s, s * L2, l1, emod(e + u * w, c.twoN), z1 + 1, n1 + 1, 0);
        for (int64_t u = m; u < n2; u++) itft_rec(&c, x + u * s, s * L2, l1, emod(e + u * w, c.twoN), z1, n1 + 1, 0);
    }
    free(c.tmp);
    return 0;
}

/* ------------------------------------------------------------------ the ring S[y]/(y^{M/2}+1) */

static int setup_sn(ctx_t *c, int64_t M, uint64_t m, int64_t stride, int l, int policy, int top_l1,
                    uint64_t seed, int need_x)
{
    memset(c, 0, sizeof *c);
    if (M < 2 || (M & (M - 1)) != 0 || !(m & 1u) || m < 3 || m >= ((uint64_t)1 << 63)) return -1;
    if (l < 1 || l > 30 || M % ((int64_t)1 << l) != 0) return -1; /* omega_L = y^{M/L}: L | M */
    c->kind = 1;
    c->m = m;
    c->N = M / 2;
    c->W = M / 2;
    c->twoN = M;
    if (need_x && stride < c->W) return -1;
    c->policy = policy;
    c->top_l1 = top_l1;
    c->rng = seed;
    c->tmp = calloc((size_t)(3 * c->W), 8);
    return 0;
}

int orc_sn_dft_brute(uint64_t *out, const uint64_t *in, int64_t stride, int l, int64_t z, int64_t n,
                     int64_t e, int64_t M, uint64_t m)
{
    ctx_t c;
    if (setup_sn(&c, M, m, stride, l, ORC_SPLIT_BALANCED, 0, 0, 1)) return -1;
    int64_t L = (int64_t)1 << l;
    if (z < 0 || z > L || n < 0 || n > L) { free(c.tmp); return -1; }
    dft_brute(&c, out, in, stride, l, z, n, e);
    free(c.tmp);
    return 0;
}

int orc_sn_tft(uint64_t *x, int64_t stride, int l, int64_t z, int64_t n, int64_t e, int64_t M, uint64_t m,
               int policy, int top_l1, uint64_t seed, int64_t *count)
{
    ctx_t c;
    if (setup_sn(&c, M, m, stride, l, policy, top_l1, seed, x != NULL)) return -1;
    int64_t L = (int64_t)1 << l;
    if (z < 1 || z > L || n < 1 || n > L) { free(c.tmp); return -1; }
    tft_rec(&c, x, stride, l, emod(e, c.twoN), z, n);
    if (count) *count += c.count;
    free(c.tmp);
    return 0;
}

int orc_sn_itft(uint64_t *x, int64_t stride, int l, int64_t z, int64_t n, int f, int64_t e, int64_t M,
                uint64_t m, int policy, int top_l1, uint64_t seed, int64_t *count)
{
    ctx_t c;
    if (setup_sn(&c, M, m, stride, l, policy, top_l1, seed, x != NULL)) return -1;
    int64_t L = (int64_t)1 << l;
    if ((f != 0 && f != 1) || z < 1 || z > L || n < 0 || n + f < 1 || n + f > L || z < n) {
        free(c.tmp);
        return -1;
    }
    itft_rec(&c, x, stride, l, emod(e, c.twoN), z, n, f);
    if (count) *count += c.count;
    free(c.tmp);
    return 0;
}

/* ------------------------------------------------------------------ Z/(2^N+1) with omega = sqrt2 */

static int setup_sqrt2(ctx_t *c, int64_t N, int64_t stride, int l, int policy, int top_l1, uint64_t seed,
                       int need_x)
{
    if (setup(c, N, stride, 1, policy, top_l1, seed, need_x)) return -1; /* L | 4N is checked here */
    if (l < 1 || l > 30 || (4 * N) % ((int64_t)1 << l) != 0) { free(c->tmp); return -1; } /* L | 4N */
    c->kind = 2;
    c->twoN = 4 * N; /* the order of omega */
    return 0;
}

int orc_sqrt2_dft_brute(uint64_t *out, const uint64_t *in, int64_t stride, int l, int64_t z, int64_t n,
                        int64_t e, int64_t N)
{
    ctx_t c;
    if (setup_sqrt2(&c, N, stride, l, ORC_SPLIT_BALANCED, 0, 0, 1)) return -1;
    int64_t L = (int64_t)1 << l;
    if (z < 0 || z > L || n < 0 || n > L) { free(c.tmp); return -1; }
    dft_brute(&c, out, in, stride, l, z, n, e);
    free(c.tmp);
    return 0;
}

int orc_sqrt2_tft(uint64_t *x, int64_t stride, int l, int64_t z, int64_t n, int64_t e, int64_t N, int policy,
                  int top_l1, uint64_t seed, int64_t *count)
{
    ctx_t c;
    if (setup_sqrt2(&c, N, stride, l, policy, top_l1, seed, x != NULL)) return -1;
    int64_t L = (int64_t)1 << l;
    if (z < 1 || z > L || n < 1 || n > L) { free(c.tmp); return -1; }
    tft_rec(&c, x, stride, l, emod(e, c.twoN), z, n);
    if (count) *count += c.count;
    free(c.tmp);
    return 0;
}

int orc_sqrt2_itft(uint64_t *x, int64_t stride, int l, int64_t z, int64_t n, int f, int64_t e, int64_t N,
                   int policy, int top_l1, uint64_t seed, int64_t *count)
{
    ctx_t c;
    if (setup_sqrt2(&c, N, stride, l, policy, top_l1, seed, x != NULL)) return -1;
    int64_t L = (int64_t)1 << l;
    if ((f != 0 && f != 1) || z < 1 || z > L || n < 0 || n + f < 1 || n + f > L || z < n) {
        free(c.tmp);
        return -1;
    }
    itft_rec(&c, x, stride, l, emod(e, c.twoN), z, n, f);
    if (count) *count += c.count;
    free(c.tmp);
    return 0;
}
