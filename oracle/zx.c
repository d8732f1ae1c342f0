/*
 * Oracle: products in Z[x].
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 *   orc_zx_mul        Sec. 5.1 (Schoenhage-Strassen in Z[x]) carried out with the TFT route of
 *                     Sec. 2 (R[X] multiplication): TFT(g), TFT(h), n pointwise products,
 *                     ITFT(L, 1, n, n, 0), which returns L u_i, then division by L and lift.
 *   orc_zx_schoolbook the textbook O(len_f len_g) product, an independent check
 *   orc_poly_eval_mod evaluation at a point modulo a prime, for spot checks of big products
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static int64_t ceil_log2(int64_t v)
{
    int64_t l = 0;
    while (((int64_t)1 << l) < v) l++;
    return l;
}

static int64_t coef_bits(const orc_poly *p) { return p->bits > 0 ? p->bits : 64 * p->limbs; }

int orc_zx_plan(int64_t len_f, int64_t bits_f, int64_t len_g, int64_t bits_g, int is_signed,
                int *l_out, int64_t *N_out)
{
    if (len_f < 1 || len_g < 1 || bits_f < 1 || bits_g < 1) return -1;
    int64_t n = len_f + len_g - 1;
    int64_t l = ceil_log2(n);
    if (l < 1) l = 1;
    if (l > 30) return -1;
    int64_t L = (int64_t)1 << l;
    /* |h_k| < min(len) 2^{bits_f + bits_g}; one more bit separates the signs */
    int64_t mn = len_f < len_g ? len_f : len_g;
    int64_t need = bits_f + bits_g + ceil_log2(mn) + (is_signed ? 1 : 0);
    /* omega_L = 2^{2N/L} must exist, so L | 2N; limbs are 64 bits */
    int64_t q = L / 2 > 64 ? L / 2 : 64;
    int64_t N = ((need + q - 1) / q) * q;
    *l_out = (int)l;
    *N_out = N;
    return 0;
}

/* residue of coefficient c (two's complement if sgn) in [0, 2^N], W limbs */
static void pack_coef(uint64_t *r, const uint64_t *c, int64_t limbs, int sgn, int64_t N)
{
    int64_t W = N / 64 + 1;
    uint64_t *buf = calloc((size_t)(limbs > W ? limbs : W) + 1, 8);
    int neg = sgn && (c[limbs - 1] >> 63);
    if (!neg) {
        memcpy(buf, c, (size_t)limbs * 8);
        memset(r, 0, (size_t)W * 8);
        for (int64_t i = 0; i < W && i < limbs; i++) r[i] = buf[i];
        r[W - 1] = 0; /* |c| < 2^N by the plan, so limbs from N/64 up are zero */
    } else {
        /* |c| = -c, then p - |c| */
        uint64_t carry = 1;
        for (int64_t i = 0; i < limbs; i++) {
            u128 t = (u128)(~c[i]) + carry;
            buf[i] = (uint64_t)t;
            carry = (uint64_t)(t >> 64);
        }
        uint64_t *mag = calloc((size_t)W, 8), *p = calloc((size_t)W, 8);
        for (int64_t i = 0; i < W && i < limbs; i++) mag[i] = buf[i];
        mag[W - 1] = 0;
        p[0] = 1;
        p[W - 1] = 1;
        orc_ring_sub(r, p, mag, N); /* p - |c| with |c| < 2^N: canonical */
        free(mag);
        free(p);
    }
    free(buf);
}

/* two's complement (or unsigned) value of residue r, truncated to `limbs` limbs */
static void lift_coef(uint64_t *out, int64_t limbs, const uint64_t *r, int sgn, int64_t N)
{
    int64_t W = N / 64 + 1;
    memset(out, 0, (size_t)limbs * 8);
    /* r > 2^{N-1} means a negative coefficient when signed */
    int neg = 0;
    if (sgn) {
        int64_t hl = (N - 1) / 64; /* limb holding bit N-1 */
        uint64_t hb = (uint64_t)1 << ((N - 1) % 64);
        int gt = 0, decided = 0;
        /* compare r with 2^{N-1} */
        for (int64_t i = W - 1; i >= 0 && !decided; i--) {
            uint64_t ref = (i == hl) ? hb : 0;
            if (r[i] != ref) { gt = r[i] > ref; decided = 1; }
        }
        neg = gt;
    }
    if (!neg) {
        for (int64_t i = 0; i < limbs && i < W; i++) out[i] = r[i];
        return;
    }
    /* value = r - p = -(p - r); magnitude p - r, then negate in `limbs` limbs */
    uint64_t *p = calloc((size_t)W, 8), *m = calloc((size_t)W, 8);
    p[0] = 1;
    p[W - 1] = 1;
    orc_ring_sub(m, p, r, N);
    uint64_t *mag = calloc((size_t)limbs, 8);
    for (int64_t i = 0; i < limbs && i < W; i++) mag[i] = m[i];
    uint64_t carry = 1;
    for (int64_t i = 0; i < limbs; i++) {
        u128 t = (u128)(~mag[i]) + carry;
        out[i] = (uint64_t)t;
        carry = (uint64_t)(t >> 64);
    }
    free(p);
    free(m);
    free(mag);
}

int orc_zx_mul(orc_poly *h, const orc_poly *f, const orc_poly *g, int *l_out, int64_t *N_out)
{
    if (!h || !f || !g || f->len < 1 || g->len < 1 || h->len != f->len + g->len - 1) return -1;
    if (f->limbs < 1 || g->limbs < 1 || h->limbs < 1) return -1;
    int sgn = f->is_signed || g->is_signed;
    int l;
    int64_t N;
    if (orc_zx_plan(f->len, coef_bits(f), g->len, coef_bits(g), sgn, &l, &N)) return -1;
    int64_t L = (int64_t)1 << l, W = N / 64 + 1, n = h->len;
    uint64_t *F = calloc((size_t)(L * W), 8), *G = calloc((size_t)(L * W), 8);
    for (int64_t i = 0; i < f->len; i++) pack_coef(F + i * W, f->data + i * f->limbs, f->limbs, f->is_signed, N);
    for (int64_t i = 0; i < g->len; i++) pack_coef(G + i * W, g->data + i * g->limbs, g->limbs, g->is_signed, N);
    /* forward transforms with zeta = 1, n = deg(u) + 1 outputs */
    orc_tft(F, W, l, f->len, n, 0, N, ORC_SPLIT_BALANCED, 0, 0, NULL);
    orc_tft(G, W, l, g->len, n, 0, N, ORC_SPLIT_BALANCED, 0, 0, NULL);
    for (int64_t i = 0; i < n; i++) orc_ring_mul(F + i * W, F + i * W, G + i * W, N);
    /* inverse: returns L u_i for i < n */
    orc_itft(F, W, l, n, n, 0, 0, N, ORC_SPLIT_BALANCED, 0, 0, NULL);
    for (int64_t i = 0; i < n; i++) {
        orc_ring_mul2exp(F + i * W, F + i * W, 2 * N - l, N); /* 1/L = 2^{-l} = 2^{2N-l} */
        lift_coef(h->data + i * h->limbs, h->limbs, F + i * W, sgn, N);
    }
    h->is_signed = sgn;
    if (l_out) *l_out = l;
    if (N_out) *N_out = N;
    free(F);
    free(G);
    return 0;
}

/* sign- or zero-extend coefficient c (limbs) into w limbs */
static void extend(uint64_t *d, int64_t w, const uint64_t *c, int64_t limbs, int sgn)
{
    uint64_t fill = (sgn && (c[limbs - 1] >> 63)) ? ~(uint64_t)0 : 0;
    for (int64_t i = 0; i < w; i++) d[i] = i < limbs ? c[i] : fill;
}

int orc_zx_schoolbook(orc_poly *h, const orc_poly *f, const orc_poly *g)
{
    if (!h || !f || !g || f->len < 1 || g->len < 1 || h->len != f->len + g->len - 1) return -1;
    int64_t w = h->limbs;
    uint64_t *a = calloc((size_t)w, 8), *b = calloc((size_t)w, 8), *pr = calloc((size_t)w, 8);
    memset(h->data, 0, (size_t)(h->len * w) * 8);
    for (int64_t i = 0; i < f->len; i++) {
        extend(a, w, f->data + i * f->limbs, f->limbs, f->is_signed);
        for (int64_t j = 0; j < g->len; j++) {
            extend(b, w, g->data + j * g->limbs, g->limbs, g->is_signed);
            /* product mod 2^{64 w}: exact two's complement arithmetic when the result fits */
            memset(pr, 0, (size_t)w * 8);
            for (int64_t x = 0; x < w; x++) {
                if (!a[x]) continue;
                uint64_t c = 0;
                for (int64_t y = 0; x + y < w; y++) {
                    u128 t = (u128)a[x] * b[y] + pr[x + y] + c;
                    pr[x + y] = (uint64_t)t;
                    c = (uint64_t)(t >> 64);
                }
            }
            uint64_t *acc = h->data + (i + j) * w, c = 0;
            for (int64_t x = 0; x < w; x++) {
                u128 t = (u128)acc[x] + pr[x] + c;
                acc[x] = (uint64_t)t;
                c = (uint64_t)(t >> 64);
            }
        }
    }
    h->is_signed = f->is_signed || g->is_signed;
    free(a);
    free(b);
    free(pr);
    return 0;
}

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t P) { return (uint64_t)(((u128)a * b) % P); }

uint64_t orc_poly_eval_mod(const orc_poly *f, uint64_t t, uint64_t P)
{
    /* 2^64 mod P */
    uint64_t r64 = (uint64_t)(((u128)1 << 64) % P);
    uint64_t acc = 0;
    for (int64_t i = f->len - 1; i >= 0; i--) {
        const uint64_t *c = f->data + i * f->limbs;
        uint64_t v = 0;
        for (int64_t k = f->limbs - 1; k >= 0; k--) v = (uint64_t)(((u128)mulmod(v, r64, P) + (c[k] % P)) % P);
        if (f->is_signed && (c[f->limbs - 1] >> 63)) {
            /* subtract 2^{64 limbs} mod P */
            uint64_t big = 1;
            for (int64_t k = 0; k < f->limbs; k++) big = mulmod(big, r64, P);
            v = (uint64_t)(((u128)v + P - big) % P);
        }
        acc = (uint64_t)(((u128)mulmod(acc, t, P) + v) % P);
    }
    return acc;
}
