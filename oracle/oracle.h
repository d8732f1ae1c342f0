/*
 * Reference oracle for the truncated Fourier transform over R = Z/(2^N+1).
 *
 * TEST INFRASTRUCTURE ONLY. This plain, slow C code is the ground truth that the
 * GPU library is checked against. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it. It shares no code with the
 * GPU library: it has its own bignum, its own recursion and its own planning.
 *
 * Paper: D. Harvey, "A cache-friendly truncated FFT" (arXiv 0810.3203).
 *   Sec. 2   ring R, root of unity omega, weighted DFT (Eq. dft), TFT/ITFT definitions,
 *            R[X] multiplication, Bailey decomposition (Eqs. b-cols / b-rows)
 *   Sec. 3   Algorithm 1 (CacheFriendlyTFT) and Theorem 1
 *   Sec. 4   Algorithm 2 (CacheFriendlyITFT) and Theorem 2
 *   Sec. 5.1 Schoenhage-Strassen multiplication in Z[x]
 *   Sec. 6   zeta carried as an exponent (zeta = omega^s stored as the integer s)
 *
 * Representation: an element of R is W = N/64 + 1 little-endian uint64 limbs
 * holding its canonical residue in [0, 2^N]. N must be a positive multiple of 64.
 * omega = 2 is a principal 2N-th root of unity (2^N = -1), so M = 2N and
 * omega_L = 2^(2N/L); zeta = 2^e is carried as e (mod 2N).
 *
 * Parity status: every function here is pinned by tests that do not call back
 * into this code (closed forms, Python integers, schoolbook products, the
 * paper's worked cell diagrams, theorem bounds); none is "parity unpinned".
 *
 * Every function returns 0 on success and -1 on a violated precondition.
 */
#ifndef TFT_ORACLE_H
#define TFT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Split policies for the recursive algorithms (Sec. 2, last paragraphs; Sec. 3 split line):
 *   ORC_SPLIT_BALANCED  L1 = 2^floor(l/2), L2 = 2^ceil(l/2) as the paper prescribes
 *   ORC_SPLIT_DC        L1 = 2 (van der Hoeven's divide-and-conquer special case)
 *   ORC_SPLIT_RANDOM    l1 drawn uniformly from [1, l-1] with a seeded generator
 *   ORC_SPLIT_TOP       top level uses the given l1, every deeper level is balanced */
enum { ORC_SPLIT_BALANCED = 0, ORC_SPLIT_DC = 1, ORC_SPLIT_RANDOM = 2, ORC_SPLIT_TOP = 3 };

/* ---- ring arithmetic in Z/(2^N+1) on canonical W-limb values ---- */
int orc_ring_add(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t N);
int orc_ring_sub(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t N);
/* r = a * 2^k for any k >= 0 (k is reduced mod 2N). */
int orc_ring_mul2exp(uint64_t *r, const uint64_t *a, int64_t k, int64_t N);
/* r = a / 2, i.e. a * 2^(2N-1). */
int orc_ring_div2(uint64_t *r, const uint64_t *a, int64_t N);
/* r = a * b mod 2^N+1 (schoolbook product, then reduction by 2^N = -1). */
int orc_ring_mul(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t N);
/* r = x mod 2^N+1 for an arbitrary non-negative integer x of xn limbs. */
int orc_ring_reduce(uint64_t *r, const uint64_t *x, int64_t xn, int64_t N);

/* ---- transforms; x holds cells of stride_limbs >= W limbs ---- */

/* Weighted DFT by its definition (Eq. dft): out_j = zeta^{j'} sum_{i<z} omega_L^{i j'} a_i
 * for j < n, with a_i = in[i] for i < z and a_i = 0 beyond. out and in must not overlap. */
int orc_dft_brute(uint64_t *out, const uint64_t *in, int64_t stride_limbs, int l,
                  int64_t z, int64_t n, int64_t e, int64_t N);

/* Algorithm 1, in place: cells 0..z-1 hold a_i on entry, cells 0..n-1 hold a-hat_i on exit.
 * x == NULL runs the recursion without arithmetic (base-case counting only).
 * *count (if non-NULL) is incremented once per base-case execution (Theorem 1). */
int orc_tft(uint64_t *x, int64_t stride_limbs, int l, int64_t z, int64_t n, int64_t e,
            int64_t N, int policy, int top_l1, uint64_t seed, int64_t *count);

/* Algorithm 2, in place: cells hold a-hat_0..a-hat_{n-1}, L a_n .. L a_{z-1} on entry and
 * L a_0 .. L a_{n-1} (then a-hat_n if f = 1) on exit. Same conventions as orc_tft. */
int orc_itft(uint64_t *x, int64_t stride_limbs, int l, int64_t z, int64_t n, int f, int64_t e,
             int64_t N, int policy, int top_l1, uint64_t seed, int64_t *count);

/* Top-level phases of Algorithm 1 / 2 with a forced top split l1 (deeper levels balanced),
 * stopping after `stop_after` phases, to check the intermediate cell states of Figs. 3-10.
 *   TFT phases:  0 nothing, 1 column transforms, 2 row transforms (complete)
 *   ITFT phases: 0 nothing, 1 full rows, 2 right columns, 3 last row, 4 left columns */
int orc_tft_phases(uint64_t *x, int64_t stride_limbs, int l, int l1, int64_t z, int64_t n,
                   int64_t e, int64_t N, int stop_after);
int orc_itft_phases(uint64_t *x, int64_t stride_limbs, int l, int l1, int64_t z, int64_t n,
                    int f, int64_t e, int64_t N, int stop_after);

/* ---- Z[x] products ---- */

/* Polynomials: len coefficients, each `limbs` little-endian uint64 limbs, two's complement
 * when is_signed, unsigned otherwise. `bits` bounds |coefficient| (0: use 64*limbs). */
typedef struct {
    int64_t len;
    int64_t limbs;
    int is_signed;
    int64_t bits;
    uint64_t *data;
} orc_poly;

/* Schoenhage-Strassen product (Sec. 5.1 with the TFT/ITFT route of Sec. 2):
 * pack, TFT(f), TFT(g), n pointwise products in R, ITFT, scale by 1/L, lift.
 * h->len must be f->len + g->len - 1; the result is reduced to h->limbs limbs (two's
 * complement if either input is signed). *l_out / *N_out report the chosen ring. */
int orc_zx_mul(orc_poly *h, const orc_poly *f, const orc_poly *g, int *l_out, int64_t *N_out);
/* The ring size the oracle's own plan picks for a product (Sec. 5.1 sizing rule). */
int orc_zx_plan(int64_t len_f, int64_t bits_f, int64_t len_g, int64_t bits_g, int is_signed,
                int *l_out, int64_t *N_out);
/* Schoolbook Z[x] product on the same coefficient format (independent check). */
int orc_zx_schoolbook(orc_poly *h, const orc_poly *f, const orc_poly *g);
/* sum_i c_i t^i mod P for a 61-bit prime P (Schwartz-Zippel spot checks of big products). */
uint64_t orc_poly_eval_mod(const orc_poly *f, uint64_t t, uint64_t P);

/* ------------------------------------------------------------------ Schoenhage-Nussbaumer ring
 * R = S[y]/(y^{M/2}+1), S = Z/mZ (Sec. 5.2): M a power of two >= 2, m odd with 3 <= m < 2^63.
 * An element is M/2 coefficients in [0, m), stored as uint64; omega = y is a principal M-th
 * root of unity, omega_L = y^{M/L} (L | M), and zeta = y^e. */
int orc_sn_add(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t M, uint64_t m);
int orc_sn_sub(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t M, uint64_t m);
/* r = y^k a (negacyclic shift), k mod M; r may alias a */
int orc_sn_ypow(uint64_t *r, const uint64_t *a, int64_t k, int64_t M, uint64_t m);
int orc_sn_half(uint64_t *r, const uint64_t *a, int64_t M, uint64_t m);
/* r = a b in R (negacyclic schoolbook product modulo m); test use only */
int orc_sn_mul(uint64_t *r, const uint64_t *a, const uint64_t *b, int64_t M, uint64_t m);
/* Eq. (dft), Algorithm 1 and Algorithm 2 over R, same conventions as the Z/(2^N+1) versions
 * (cells of stride >= M/2 words). */
int orc_sn_dft_brute(uint64_t *out, const uint64_t *in, int64_t stride, int l, int64_t z, int64_t n,
                     int64_t e, int64_t M, uint64_t m);
int orc_sn_tft(uint64_t *x, int64_t stride, int l, int64_t z, int64_t n, int64_t e, int64_t M, uint64_t m,
               int policy, int top_l1, uint64_t seed, int64_t *count);
int orc_sn_itft(uint64_t *x, int64_t stride, int l, int64_t z, int64_t n, int f, int64_t e, int64_t M,
                uint64_t m, int policy, int top_l1, uint64_t seed, int64_t *count);

/* ------------------------------------------------------------------ omega = sqrt2 over Z/(2^N+1)
 * sqrt2 = 2^{3N/4} - 2^{N/4} squares to 2 and is a principal 4N-th root of unity, so transforms
 * of any length L | 4N exist. Exponents (e, and those of omega_L = sqrt2^{4N/L}) are in units of
 * sqrt2, mod 4N; otherwise as orc_dft_brute / orc_tft / orc_itft. Not in the paper. */
int orc_sqrt2_dft_brute(uint64_t *out, const uint64_t *in, int64_t stride, int l, int64_t z, int64_t n,
                        int64_t e, int64_t N);
int orc_sqrt2_tft(uint64_t *x, int64_t stride, int l, int64_t z, int64_t n, int64_t e, int64_t N, int policy,
                  int top_l1, uint64_t seed, int64_t *count);
int orc_sqrt2_itft(uint64_t *x, int64_t stride, int l, int64_t z, int64_t n, int f, int64_t e, int64_t N,
                   int policy, int top_l1, uint64_t seed, int64_t *count);

#ifdef __cplusplus
}
#endif
#endif
