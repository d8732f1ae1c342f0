/* The oracle (oracle/*.c) under AddressSanitizer and UBSan: every entry point on small random
 * inputs, over several ring sizes, lengths, weights and split policies. The transforms are also
 * checked against the DFT by its definition on the same inputs (Algorithm 1; Algorithm 2 on the
 * mixed input of Sec. 4), so a clean run is a correctness run as well. Built and run by
 * tests/test_sanitizers.py; any sanitizer report or mismatch fails it. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../../oracle/oracle.h"

static uint64_t state = 0x243F6A8885A308D3ull;
static uint64_t next(void) { /* splitmix64 */
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static int64_t below(int64_t n) { return (int64_t)(next() % (uint64_t)n); }

static int failures = 0;
#define CHECK(c, ...)                  \
  do {                                 \
    if (!(c)) {                        \
      fprintf(stderr, __VA_ARGS__);    \
      fputc('\n', stderr);             \
      failures++;                      \
    }                                  \
  } while (0)

/* a canonical residue in [0, 2^N]: random limbs below bit N, sometimes 0, 1 or 2^N = -1 */
static void residue(uint64_t *x, int64_t N) {
  const int64_t W = N / 64 + 1;
  const int64_t r = below(16);
  memset(x, 0, (size_t)W * 8);
  if (r == 0) return;
  if (r == 1) { x[0] = 1; return; }
  if (r == 2) { x[W - 1] = 1; return; }
  for (int64_t i = 0; i < W - 1; i++) x[i] = next();
}

static uint64_t *cells(int64_t count, int64_t stride) {
  uint64_t *p = calloc((size_t)(count * stride), 8);
  if (!p) { fprintf(stderr, "out of memory\n"); exit(2); }
  return p;
}

static int64_t ring_checks = 0, transform_checks = 0, product_checks = 0, sn_checks = 0;

static void ring_ops(int64_t N) {
  const int64_t W = N / 64 + 1;
  uint64_t a[W], b[W], r[W], s[W], t[W], x2[2 * W];
  for (int it = 0; it < 40; it++) {
    residue(a, N);
    residue(b, N);
    CHECK(orc_ring_add(r, a, b, N) == 0 && orc_ring_sub(s, r, b, N) == 0 && !memcmp(s, a, W * 8),
          "add/sub N=%lld", (long long)N);
    const int64_t k = below(4 * N);
    CHECK(orc_ring_mul2exp(r, a, k, N) == 0 && orc_ring_mul2exp(s, r, 2 * N - k % (2 * N), N) == 0 &&
              !memcmp(s, a, W * 8),
          "mul2exp N=%lld k=%lld", (long long)N, (long long)k);
    CHECK(orc_ring_div2(r, a, N) == 0 && orc_ring_add(s, r, r, N) == 0 && !memcmp(s, a, W * 8),
          "div2 N=%lld", (long long)N);
    /* a b by the product routine and by reducing the double-length product */
    CHECK(orc_ring_mul(r, a, b, N) == 0, "mul N=%lld", (long long)N);
    memset(x2, 0, sizeof x2);
    memcpy(x2, a, W * 8);
    CHECK(orc_ring_reduce(t, x2, 2 * W, N) == 0 && !memcmp(t, a, W * 8), "reduce N=%lld", (long long)N);
    /* a 2 = a + a */
    CHECK(orc_ring_mul2exp(s, a, 1, N) == 0 && orc_ring_add(t, a, a, N) == 0 && !memcmp(s, t, W * 8),
          "double N=%lld", (long long)N);
    ring_checks++;
  }
}

/* Algorithm 1 and 2 against the DFT by definition for one (l, z, n, f, e, policy) */
static void transform_case(int64_t N, int l, int64_t z, int64_t n, int f, int64_t e, int policy, int sqrt2) {
  const int64_t W = N / 64 + 1, L = (int64_t)1 << l, st = W + below(3);
  uint64_t *a = cells(L, st), *x = cells(L, st), *hat = cells(L, st), *mixed = cells(L, st);
  for (int64_t i = 0; i < z; i++) residue(a + i * st, N);
  /* Algorithm 1 */
  memcpy(x, a, (size_t)(L * st) * 8);
  int rc = sqrt2 ? orc_sqrt2_tft(x, st, l, z, n, e, N, policy, 1, 5, NULL)
                 : orc_tft(x, st, l, z, n, e, N, policy, 1, 5, NULL);
  int rd = sqrt2 ? orc_sqrt2_dft_brute(hat, a, st, l, z, L, e, N) : orc_dft_brute(hat, a, st, l, z, L, e, N);
  CHECK(rc == 0 && rd == 0, "tft rc N=%lld l=%d", (long long)N, l);
  for (int64_t j = 0; j < n; j++)
    CHECK(!memcmp(x + j * st, hat + j * st, W * 8), "tft N=%lld l=%d z=%lld n=%lld j=%lld sqrt2=%d",
          (long long)N, l, (long long)z, (long long)n, (long long)j, sqrt2);
  /* Algorithm 2 on hat_0..hat_{m-1}, L a_m .. L a_{z-1}: L a_i for i < m, then hat_m if f */
  const int64_t m = n <= z ? n : z;
  const int ff = (f && m < L) ? 1 : 0;
  for (int64_t i = 0; i < L; i++) {
    if (i < m)
      memcpy(mixed + i * st, hat + i * st, W * 8);
    else if (i < z)
      orc_ring_mul2exp(mixed + i * st, a + i * st, l, N); /* L a_i, L = 2^l in either mode */
  }
  rc = sqrt2 ? orc_sqrt2_itft(mixed, st, l, z, m, ff, e, N, policy, 1, 7, NULL)
             : orc_itft(mixed, st, l, z, m, ff, e, N, policy, 1, 7, NULL);
  CHECK(rc == 0, "itft rc N=%lld l=%d", (long long)N, l);
  uint64_t La[W];
  for (int64_t i = 0; i < m; i++) {
    orc_ring_mul2exp(La, a + i * st, l, N);
    CHECK(!memcmp(mixed + i * st, La, W * 8), "itft N=%lld l=%d z=%lld n=%lld i=%lld sqrt2=%d", (long long)N, l,
          (long long)z, (long long)m, (long long)i, sqrt2);
  }
  if (ff) CHECK(!memcmp(mixed + m * st, hat + m * st, W * 8), "itft f output N=%lld l=%d", (long long)N, l);
  free(a);
  free(x);
  free(hat);
  free(mixed);
  transform_checks++;
}

/* S[y]/(y^{M/2}+1): ring identities, and Algorithm 1 against the DFT by definition */
static void sn_case(int64_t M, uint64_t m, int l) {
  const int64_t H = M / 2, L = (int64_t)1 << l, st = H + below(2);
  uint64_t a[H], b[H], r[H], s[H];
  for (int it = 0; it < 10; it++) {
    for (int64_t i = 0; i < H; i++) a[i] = next() % m, b[i] = next() % m;
    CHECK(orc_sn_add(r, a, b, M, m) == 0 && orc_sn_sub(s, r, b, M, m) == 0 && !memcmp(s, a, H * 8), "sn add/sub");
    const int64_t k = below(3 * M);
    CHECK(orc_sn_ypow(r, a, k, M, m) == 0 && orc_sn_ypow(s, r, M - k % M, M, m) == 0 && !memcmp(s, a, H * 8),
          "sn ypow M=%lld k=%lld", (long long)M, (long long)k);
    CHECK(orc_sn_half(r, a, M, m) == 0 && orc_sn_add(s, r, r, M, m) == 0 && !memcmp(s, a, H * 8), "sn half");
    CHECK(orc_sn_mul(r, a, b, M, m) == 0 && orc_sn_mul(s, b, a, M, m) == 0 && !memcmp(r, s, H * 8), "sn mul");
  }
  const int64_t z = 1 + below(L), n = 1 + below(L), e = below(M);
  uint64_t *x = cells(L, st), *in = cells(L, st), *hat = cells(L, st);
  for (int64_t i = 0; i < z; i++)
    for (int64_t c = 0; c < H; c++) in[i * st + c] = next() % m;
  memcpy(x, in, (size_t)(L * st) * 8);
  CHECK(orc_sn_tft(x, st, l, z, n, e, M, m, ORC_SPLIT_RANDOM, 1, 3, NULL) == 0 &&
            orc_sn_dft_brute(hat, in, st, l, z, L, e, M, m) == 0,
        "sn rc");
  for (int64_t j = 0; j < n; j++)
    CHECK(!memcmp(x + j * st, hat + j * st, H * 8), "sn tft M=%lld l=%d j=%lld", (long long)M, l, (long long)j);
  /* Algorithm 2 on the mixed input: L a_i for i < n' back */
  const int64_t nn = n <= z ? n : z;
  for (int64_t i = nn; i < z; i++)
    for (int64_t c = 0; c < H; c++) hat[i * st + c] = (uint64_t)(((unsigned __int128)in[i * st + c] * (uint64_t)L) % m);
  for (int64_t i = z; i < L; i++) memset(hat + i * st, 0, (size_t)st * 8);
  CHECK(orc_sn_itft(hat, st, l, z, nn, 0, e, M, m, ORC_SPLIT_BALANCED, 0, 0, NULL) == 0, "sn itft rc");
  for (int64_t i = 0; i < nn; i++)
    for (int64_t c = 0; c < H; c++)
      CHECK(hat[i * st + c] == (uint64_t)(((unsigned __int128)in[i * st + c] * (uint64_t)L) % m),
            "sn itft M=%lld l=%d i=%lld", (long long)M, l, (long long)i);
  free(x);
  free(in);
  free(hat);
  sn_checks++;
}

/* Z[x] products: the transform route against schoolbook, signed and unsigned */
static void product_case(int64_t lf, int64_t lg, int64_t bits, int is_signed) {
  const int64_t limbs = (bits + 63) / 64 + (is_signed ? 1 : 0), lh = lf + lg - 1;
  const int64_t hl = 2 * limbs + 2;
  orc_poly f = {lf, limbs, is_signed, bits, cells(lf, limbs)};
  orc_poly g = {lg, limbs, is_signed, bits, cells(lg, limbs)};
  orc_poly h = {lh, hl, is_signed, 0, cells(lh, hl)};
  orc_poly s = {lh, hl, is_signed, 0, cells(lh, hl)};
  for (int64_t i = 0; i < lf + lg; i++) {
    orc_poly *p = i < lf ? &f : &g;
    uint64_t *c = p->data + (i < lf ? i : i - lf) * limbs;
    for (int64_t k = 0; k < bits / 64; k++) c[k] = next();
    if (bits % 64) c[bits / 64] = next() & ((1ull << (bits % 64)) - 1);
    if (is_signed && (next() & 1)) { /* negate: two's complement over all limbs */
      int carry = 1;
      for (int64_t k = 0; k < limbs; k++) {
        c[k] = ~c[k] + (uint64_t)carry;
        carry = carry && c[k] == 0;
      }
    }
  }
  int lo = 0;
  int64_t No = 0;
  CHECK(orc_zx_mul(&h, &f, &g, &lo, &No) == 0 && orc_zx_schoolbook(&s, &f, &g) == 0, "zx rc");
  CHECK(!memcmp(h.data, s.data, (size_t)(lh * hl) * 8), "zx lf=%lld lg=%lld bits=%lld signed=%d", (long long)lf,
        (long long)lg, (long long)bits, is_signed);
  const uint64_t P = 2305843009213693951ull; /* 2^61 - 1 */
  (void)orc_poly_eval_mod(&h, next() % P, P);
  free(f.data);
  free(g.data);
  free(h.data);
  free(s.data);
  product_checks++;
}

int main(void) {
  const int64_t Ns[] = {64, 128, 256, 1024};
  for (size_t k = 0; k < sizeof Ns / sizeof Ns[0]; k++) {
    const int64_t N = Ns[k];
    ring_ops(N);
    for (int l = 1; ((int64_t)1 << l) <= 2 * N && l <= 8; l++)
      for (int t = 0; t < 3; t++) {
        const int64_t L = (int64_t)1 << l;
        transform_case(N, l, 1 + below(L), 1 + below(L), (int)(next() & 1), below(2 * N), (int)below(3), 0);
      }
    for (int l = 2; ((int64_t)1 << l) <= 4 * N && l <= 8; l += 2) {
      const int64_t L = (int64_t)1 << l;
      transform_case(N, l, 1 + below(L), 1 + below(L), (int)(next() & 1), below(4 * N), ORC_SPLIT_BALANCED, 1);
    }
  }
  for (int l = 1; l <= 5; l++) sn_case(32, 65537, l);
  sn_case(64, (1ull << 61) - 1, 6);
  sn_case(16, 3, 4);
  product_case(1, 1, 64, 0);
  product_case(37, 29, 200, 0);
  product_case(50, 70, 130, 1);
  product_case(300, 200, 64, 1);
  product_case(120, 130, 700, 0);
  printf("ring %lld transforms %lld sn %lld products %lld failures %d\n", (long long)ring_checks,
         (long long)transform_checks, (long long)sn_checks, (long long)product_checks, failures);
  return failures ? 1 : 0;
}
