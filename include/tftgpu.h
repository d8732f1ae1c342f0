/*
 * tftgpu: truncated Fourier transforms over R = Z/(2^N+1) and Schoenhage-Strassen products in
 * Z[x] on one GB300 GPU (sm_103a). C ABI of libtftgpu.so.
 *
 * Method: D. Harvey, "A cache-friendly truncated FFT" (arXiv 0810.3203).
 *   Sec. 2    the ring R, omega = 2, the weighted DFT (Eq. dft), the TFT and ITFT definitions,
 *             polynomial products in R[X] through TFT/ITFT
 *   Sec. 3    Algorithm 1 (cache-friendly TFT); Sec. 4 Algorithm 2 (cache-friendly ITFT)
 *   Sec. 5.1  Schoenhage-Strassen multiplication in Z[x]
 *
 * Conventions shared by every entry point
 *   Ring element ("cell"): W = N/64 + 1 little-endian uint64 limbs holding the canonical residue
 *     in [0, 2^N] (the top limb is 0, or 1 only for 2^N = -1). Consecutive cells are
 *     stride_limbs >= W limbs apart, and a buffer of k cells spans k * stride_limbs limbs. Limbs
 *     past W in a cell are never written; when stride_limbs > W, the limb after a cell's top limb
 *     may be read (loads move 16-byte vectors) and its value is ignored.
 *   omega = 2 (a principal 2N-th root of unity), so omega_L = 2^(2N/L) and L = 2^l must divide
 *     2N. A weight zeta = 2^e is passed as its exponent e (taken mod 2N), as in Sec. 6.
 *   Supported ring sizes: N a multiple of 64 with N <= 1024, or a multiple of 1024 up to 32768.
 *   Buffers passed as uint64_t* to the transform calls are DEVICE memory owned by the caller.
 *   `stream` is a cudaStream_t (NULL = the legacy default stream). All work is enqueued on it;
 *     the calls return without synchronising unless stated. They are safe to call from several
 *     host threads on different streams.
 *   Errors: every call returns a status code (below) and never throws or aborts. On error no
 *     kernel of the failing call has been enqueued, except for ZX_ECUDA from a launch, after
 *     which the contents of the caller's buffer are unspecified. zx_last_error() describes
 *     the most recent failure of the calling thread.
 */
#ifndef TFTGPU_H
#define TFTGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define ZX_OK 0
#define ZX_EINVAL 1       /* a size, index or flag violates the stated preconditions */
#define ZX_ENOMEM 2       /* device or pinned-host allocation failed */
#define ZX_ECUDA 3        /* a CUDA runtime call or kernel launch failed */
#define ZX_ETIMEOUT 4     /* a bounded wait gave up (server drain; device waits, zx_wait_status) */
#define ZX_EBUFSIZE 5     /* an output buffer is too small; the needed size is reported */
#define ZX_EUNSUPPORTED 6 /* valid for the paper, but outside this library's supported sizes */

#define ZX_HOST 0   /* zx_poly.where: data lives in host memory (pageable or pinned) */
#define ZX_DEVICE 1 /* zx_poly.where: data lives in device memory of the current device */

/*
 * TFT(L, zeta, z, n) of Sec. 2 computed in place by the cache-friendly order of Algorithm 1.
 *   x            device buffer of L = 2^l cells. On entry cells 0..z-1 hold a_0..a_{z-1}
 *                (a_i = 0 for i >= z is implied; those cells are not read). On exit cells
 *                0..n-1 hold a-hat_0..a-hat_{n-1} of Eq. (dft), i.e. outputs in bit-reversed
 *                order. All L cells are scratch (Sec. 2: every cell may be used); cells >= n
 *                are unspecified on exit.
 *   l            1 <= l <= 16, with 2^l dividing 2N.
 *   z, n         1 <= z <= L, 1 <= n <= L.
 *   N            ring size as above.  e  the weight exponent (zeta = 2^e), any int64.
 *   stride_limbs distance between cells in limbs, >= N/64 + 1.
 * Returns ZX_EINVAL on bad arguments, ZX_EUNSUPPORTED for an unsupported N, ZX_ECUDA on a
 * launch failure.
 */
int tft_ex(uint64_t *x, int l, int64_t z, int64_t n, int64_t N, int64_t e,
           int64_t stride_limbs, void *stream);

/* tft_ex with z = n, e = 0 (zeta = 1) and stride_limbs = N/64 + 1: n inputs, n outputs. */
int tft(uint64_t *x, int l, int64_t n, int64_t N, void *stream);

/*
 * ITFT(L, zeta, z, n, f) of Sec. 2 computed in place by Algorithm 2 (Sec. 4).
 *   x      device buffer of L cells. On entry cells 0..n-1 hold a-hat_0..a-hat_{n-1} and cells
 *          n..z-1 hold L a_n .. L a_{z-1} (a_i = 0 for i >= z implied). On exit cells 0..n-1
 *          hold L a_0 .. L a_{n-1} when scale = 0, or a_0 .. a_{n-1} when scale = 1 (the
 *          outputs multiplied by L^{-1} = 2^{2N-l}); if f = 1, cell n holds a-hat_n (never
 *          scaled). Other cells are unspecified on exit.
 *   f      0 or 1.  Preconditions: 1 <= z <= L, 0 <= n <= z, 1 <= n + f <= L.
 *   Other arguments and errors as for tft_ex.
 */
int itft_ex(uint64_t *x, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e,
            int64_t stride_limbs, int scale, void *stream);

/* itft_ex with z = n, f = 0, e = 0, stride N/64 + 1 and scale = 1: returns a_i, so that
 * itft(tft(x)) restores x literally. */
int itft(uint64_t *x, int l, int64_t n, int64_t N, void *stream);

/*
 * The same transforms with omega = sqrt2 = 2^(3N/4) - 2^(N/4), a principal 4N-th root of unity
 * in Z/(2^N+1) (the sqrt2 trick; not in the paper): L = 2^l only has to divide 4N, so a product
 * of length L can use a ring of L/4 bits instead of L/2. omega_L = sqrt2^(4N/L), zeta = sqrt2^e
 * with e taken mod 4N; otherwise as tft_ex / itft_ex (itft_sqrt2 with scale = 1 divides by L).
 */
int tft_sqrt2(uint64_t *x, int l, int64_t z, int64_t n, int64_t N, int64_t e, int64_t stride_limbs, void *stream);
int itft_sqrt2(uint64_t *x, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e, int64_t stride_limbs,
               int scale, void *stream);

/* A polynomial in Z[x] with `len` coefficients of `limbs` little-endian uint64 limbs each,
 * two's complement when is_signed != 0, unsigned otherwise. `bits` > 0 promises
 * |coefficient| < 2^bits (0: no promise, 64 * limbs is assumed); the ring size is chosen from
 * it, and a coefficient that breaks the promise gives an unspecified result. */
typedef struct {
    int64_t len;
    int64_t limbs;
    int32_t is_signed;
    int32_t where; /* ZX_HOST or ZX_DEVICE */
    int64_t bits;
    uint64_t *data;
} zx_poly;

/* What zx_mul does for a product (filled by zx_plan). */
typedef struct {
    int32_t l;             /* transform length L = 2^l >= len_f + len_g - 1 */
    int32_t K;             /* 32-bit words per lane of a warp-wide ring element */
    int64_t N;             /* ring Z/(2^N+1) */
    int64_t n;             /* number of product coefficients, len_f + len_g - 1 */
    int64_t stride_limbs;  /* cell stride of the library's ring buffers */
    int64_t limbs_h;       /* minimum h->limbs that holds every product coefficient */
    int64_t scratch_bytes; /* device scratch the product needs (two ring buffers) */
    int32_t tft_passes;    /* kernel passes of one forward transform */
    int32_t itft_passes;   /* kernel passes of the inverse transform */
    int64_t n_fft;         /* transform outputs computed: n rounded up to whole rows of the
                              top-level row/column split (the zero padding of Sec. 6), and of
                              the column jobs' own split when that adds at most n/32; n when
                              one CTA holds the whole transform */
    int32_t sqrt2;         /* 1: the transforms use omega = sqrt2 (L | 4N), which allowed a
                              ring half the size of the L | 2N rule; 0: omega = 2 */
    int32_t pad;
} zx_plan_info;

/*
 * Ring and transform plan for f * g following the sizing of Sec. 5.1: n = len_f + len_g - 1,
 * L = 2^ceil(log2 n), N >= bits_f + bits_g + ceil(log2 min(len_f, len_g)) (+1 if signed),
 * rounded up so that L | 2N and N is a supported size. bits_* are the |coefficient| bounds.
 * Host only. Returns ZX_EINVAL or ZX_EUNSUPPORTED when no supported ring exists.
 */
int zx_plan(int64_t len_f, int64_t bits_f, int64_t len_g, int64_t bits_g, int is_signed,
            zx_plan_info *out);

/*
 * h = f * g in Z[x] by Schoenhage-Strassen with truncated transforms (Sec. 2 R[X] product and
 * Sec. 5.1): pack into R, TFT(f), TFT(g), n_fft pointwise products in R, ITFT, division by L,
 * lift to Z. The product's n coefficients are padded with known zeros to n_fft (zx_plan) so
 * that the ITFT has no partial row (Sec. 6); the padded coefficients are not returned.
 *   f, g   inputs, host or device (each independently); not modified.
 *   h      caller-allocated output with h->len == f->len + g->len - 1 (else ZX_EINVAL) and
 *          h->limbs >= zx_plan(...).limbs_h (else ZX_EBUFSIZE and h->limbs is overwritten
 *          with the needed count). h->is_signed is set to f->is_signed || g->is_signed.
 *   The library owns its scratch (two ring buffers of L cells each), taken from the device's
 *   stream-ordered memory pool on `stream` and returned to it before the call's work ends.
 *   Host operands are copied with cudaMemcpyAsync on `stream` (pinned host memory makes those
 *   copies asynchronous); when any operand is on the host the call synchronises `stream`
 *   before returning, otherwise it is asynchronous. g's packing and TFT run on an internal
 *   stream of the calling thread, forked from `stream` and joined back into it with events,
 *   so all of the call's work is ordered after the work already on `stream` and before
 *   anything enqueued on `stream` later. When the pointwise method for N is the recursive one
 *   (zx_pointwise_plan), its scratch also comes from the pool on `stream`.
 */
int zx_mul(const zx_poly *f, const zx_poly *g, zx_poly *h, void *stream);

/*
 * count independent products hs[i] = fs[i] * gs[i], each with its own ring and length, all
 * operands in device memory. The products run concurrently. A product whose transforms have
 * 2^13 cells or more fills the GPU on its own: it runs as its own launch chain (as zx_mul), the
 * largest first, on one of 4 streams of the calling thread forked from `stream`. The smaller
 * products share merged launches, where every pass of every product is one job of a shared
 * per-pass launch, so short products share SMs instead of leaving them idle. All of the call's
 * work is ordered after the work already on `stream` and before anything enqueued on it later,
 * also when the call fails. Same per-product rules as zx_mul (the first failing index is
 * reported by zx_last_error()).
 */
int zx_mul_batch(const zx_poly *fs, const zx_poly *gs, zx_poly *hs, int count, void *stream);

/*
 * zx_mul without any memory allocation. The paper has no counterpart; this entry point serves
 * callers that cannot call cudaMalloc, e.g. code whose device memory is entirely reserved by
 * another allocator, or a loop that must not pay an allocation's latency and implicit
 * synchronisation. Same product, same rules for h as zx_mul, with these differences:
 *   - f, g and h must all be in device memory (ZX_EINVAL otherwise);
 *   - the ring buffers live in a fixed 20 MiB device array of the library (16 MiB for the two
 *     ring buffers, 4 MiB for launch plans), held by every GPU that loads the library until the
 *     process exits; a product whose two ring buffers (2 L stride_limbs 8 bytes, see zx_plan)
 *     exceed 16 MiB is rejected with ZX_EUNSUPPORTED, and ZX_ENOMEM reports a full plan region;
 *   - the first call on a device looks up that array's address (cudaGetSymbolAddress) with the
 *     device current, so make the first call on each device before any stream capture;
 *   - the first call for each product shape (lengths, bit sizes, signedness) writes that shape's
 *     launch plans into the array from host memory, which a stream capture cannot record for
 *     later replays: such a call returns ZX_EINVAL while `stream` is capturing. Make one call
 *     per shape (and one after changing the ring's launch configuration with zx_config_set or
 *     zx_tune) before capturing; captured calls of known shapes replay correctly;
 *   - the pointwise products use the schoolbook kernel (zx_mul's default method);
 *   - all calls share the array: calls whose GPU work overlaps (different streams or threads
 *     without ordering between them) race. Order them on one stream.
 * It calls no cudaMalloc, cudaFree or other allocating routine; the call is asynchronous.
 */
int zx_mul_noalloc(const zx_poly *f, const zx_poly *g, zx_poly *h, void *stream);

/*
 * Serving loop: continuous batching of Z[x] products on the current device (no counterpart in
 * the paper; it schedules the zx_mul_batch path). zx_server_create reserves a device arena of
 * arena_bytes (<= 0: half of the free device memory) and `slots` streams (1..8) and starts a
 * worker thread. zx_server_submit queues h = f * g (every operand in device memory, same rules
 * as zx_mul; h->is_signed is set) and returns at once with a request id; a product whose ring
 * buffers exceed the arena is refused with ZX_ENOMEM. The worker admits the longest prefix of
 * the queue whose ring buffers fit the free arena into a free slot as one batch, up to about
 * 20 ms of estimated work (a batch completes as a whole, so this bounds the latency it adds).
 * Requests that arrive while others run start as soon as a slot and memory are free and overlap
 * with them on the GPU. f, g and h must stay valid until the request is returned by zx_server_poll.
 * zx_server_poll returns up to `max` finished requests (id, status, seconds from submission to
 * completion; status and latency_s may be NULL). zx_server_drain waits until nothing is queued
 * or running (timeout_s < 0: no limit; ZX_ETIMEOUT otherwise). zx_server_destroy finishes the
 * queued work, stops the worker and frees everything; unpolled results are dropped.
 */
typedef struct zx_server zx_server;

typedef struct {
    int64_t submitted, completed, pending;
    int64_t waves;             /* batches launched */
    int64_t max_wave_products; /* largest batch */
    int32_t slots;
    int32_t max_waves_in_flight;
    int64_t arena_bytes, arena_peak_bytes;
    double time_scale;         /* running average of measured batch time (enqueue to
                                  completion) over the cost model's estimate */
} zx_server_info;

int zx_server_create(int64_t arena_bytes, int slots, zx_server **out);
int zx_server_submit(zx_server *srv, const zx_poly *f, const zx_poly *g, zx_poly *h, int64_t *id);
int zx_server_poll(zx_server *srv, int64_t *ids, int32_t *status, double *latency_s, int max, int *count);
int zx_server_drain(zx_server *srv, double timeout_s);
int zx_server_stats(zx_server *srv, zx_server_info *out);
int zx_server_destroy(zx_server *srv);

/*
 * Autotuner for the launch configuration of ring N (no counterpart in the paper, which fixes
 * the split L1 = 2^floor(l/2) for cache reasons; every configuration computes the same
 * outputs). Candidates: cells per CTA of a cluster job (2^3 .. 2^6), the largest job held by one
 * CTA (the shared-memory limit, or the size at which three CTAs share an SM), warps per CTA
 * (8 or 16) and, for odd l, the top-level split floor or ceil(l/2); and the split with the fewest
 * passes with clusters capped at 2 or 4 CTAs (for l = 16 at N = 32768: three passes, columns of 64
 * cells on 4-CTA clusters, then rows of 32 cells on 2-CTA clusters). The setting `fused` is kept as
 * it is: single round trips cannot show its cost when transforms run on concurrent streams. The
 * round trips use
 * omega = 2 when L | 2N, else omega = sqrt2 (L | 4N), the transforms products use. For each candidate the call
 * times `reps` TFT + ITFT round trips (Algorithm 1, then Algorithm 2 with the division by L)
 * of length n over the caller's device buffer x (L = 2^l cells of stride_limbs >= N/64 + 1
 * limbs holding canonical residues; the round trips restore it), and keeps for every later plan
 * over ring N in this process the default configuration, or a candidate at least 3 % faster than
 * the configuration kept before it (configurations that single round trips cannot tell apart
 * differ in batches and concurrent use, so noise does not decide), and reports it.
 * Synchronises `stream`.
 */
typedef struct {
    int32_t ls_max;     /* log2 of the largest job one CTA holds */
    int32_t ls_c;       /* log2 of the cells per CTA of a cluster job */
    int32_t max_warps;  /* warps per CTA */
    int32_t split;      /* 0: L1 = 2^floor(l/2), 1: L1 = 2^ceil(l/2), 2: at every level the
                           split with the fewest global-memory passes below it */
    int32_t candidates; /* configurations timed */
    float best_ms;      /* round-trip time of the chosen configuration */
    float default_ms;   /* round-trip time of the default configuration */
    int32_t fused;      /* launch form of plans whose jobs all run on single CTAs (rings of
                           N = 2^k >= 4096): 0 one launch per global-memory pass; 1 one
                           persistent launch per transform (zx_transform_schedule), 2 the same
                           for the ITFT only; 3 one launch per pass as a persistent loop that
                           prefetches a CTA's next job into L2; 4 one launch per pass with one
                           CTA per job through the persistent kernels' job body (the
                           default). A persistent launch holds every CTA slot of the GPU until
                           it finishes, so transforms on concurrent streams stop overlapping;
                           it pays for a transform that runs alone */
    int32_t max_cluster_log2; /* cluster jobs use at most 2^max_cluster_log2 CTAs (0 .. 4) */
    int32_t tma;        /* 1 (default): launches of the forms 3 and 4 move each cell with one
                           tensor (TMA) copy for rings of 8 or more words per lane (N = 8192,
                           16384, 32768) when the buffer is 16-byte aligned with an even
                           stride_limbs >= W + 1; 0: row copies and 16-byte stores. Kept as it is
                           by zx_tune */
} zx_tune_info;

int zx_tune(uint64_t *x, int l, int64_t n, int64_t N, int64_t stride_limbs, int reps, void *stream,
            zx_tune_info *out);

/* The launch configuration used for ring N (ls_max, ls_c, max_warps, split, fused,
 * max_cluster_log2, tma; the other fields are zero; a tuned configuration is kept as zx_tune chose it), and pinning one, e.g. a result of zx_tune saved from an earlier process. zx_config_set
 * returns ZX_EINVAL for a configuration the ring cannot run (shared memory, warps, split); with
 * cfg == NULL it restores the default. Host only. */
int zx_config_get(int64_t N, zx_tune_info *out);
int zx_config_set(int64_t N, const zx_tune_info *cfg);

/*
 * Truncated transforms over the Schoenhage-Nussbaumer coefficient ring (Sec. 5.2):
 * R = S[y]/(y^(M/2) + 1), S = Z/mZ, with omega = y a principal M-th root of unity, so the
 * twiddles are negacyclic shifts of the coefficients. Same semantics as tft_ex / itft_ex with
 * omega_L = y^(M/L) and zeta = y^e:
 *   x       device buffer of L = 2^l cells, cell i at x + i * stride (stride >= M/2 uint64);
 *           a cell is the M/2 coefficients of an element, each in [0, m) (canonical)
 *   M       a power of two, 2 <= M <= 2048 (ZX_EUNSUPPORTED above), with L | M
 *   m       odd modulus, 3 <= m < 2^63
 *   sn_itft returns L a_i (scale = 0) or a_i (scale = 1: multiplied by L^-1 mod m), then
 *           a-hat_n when f = 1.
 * The products of the Schoenhage-Nussbaumer algorithm (Kronecker substitution or
 * Nussbaumer's method on the pointwise step) are outside this library.
 */
int sn_tft(uint64_t *x, int l, int64_t z, int64_t n, int64_t M, uint64_t m, int64_t e, int64_t stride,
           void *stream);
int sn_itft(uint64_t *x, int l, int64_t z, int64_t n, int f, int64_t M, uint64_t m, int64_t e, int64_t stride,
            int scale, void *stream);

/* Shape of the launch plan of one transform (host only, no device needed); the same for omega = 2
 * (L | 2N) and omega = sqrt2 (L | 4N), so only L | 4N is required. */
typedef struct {
    int32_t passes;    /* passes over global memory */
    int32_t launches;  /* kernel launches */
    int64_t jobs;      /* on-chip sub-transforms (one CTA each) */
    int32_t onchip_l;  /* log2 of the largest sub-transform held on chip by one job */
    int32_t K;         /* 32-bit words per lane of a ring element */
    int32_t cluster_l; /* log2 of the CTAs per job (thread-block cluster; 0: single CTA) */
    int32_t pad;
} zx_transform_info;

/* Launch plan of tft_ex (kind = 0) or itft_ex (kind = 1) for these sizes; the weight and
 * stride do not change it. Same argument checks and status codes as the transform calls. */
int zx_transform_plan(int kind, int l, int64_t z, int64_t n, int f, int64_t N, zx_transform_info *out);

/*
 * Pointwise products in Z/(2^N+1) (the step between the forward and inverse transforms of a
 * product, Sec. 5.1): a_i <- a_i * b_i mod 2^N + 1 for i < n, over canonical cells (N/64 + 1
 * limbs, little-endian, value in [0, 2^N]) spaced stride_limbs apart in device memory; a and b
 * are caller-owned and must not overlap (a may equal b only for squaring, a == b exactly).
 * method 1: one warp per product, schoolbook product scanning with a negacyclic fold.
 * method 2: a second Schoenhage-Strassen level on the transform kernels: 2^k pieces of
 *   M = N / 2^k bits, weighted by theta^t (theta = 2^{N'/2^k}, theta^{2^k} = -1) in the inner
 *   ring Z/(2^{N'}+1) with N' >= 2M + k + 1, a TFT and ITFT of length 2^k, the inner products
 *   by method 1, and the negacyclic recombination. Device scratch comes from the stream's
 *   memory pool, in chunks of at most 256 MB.
 * method 0: whichever zx_pointwise_plan reports for N.
 * Both methods give the same canonical residues. Returns ZX_EINVAL on bad arguments,
 * ZX_EUNSUPPORTED when N has no recursive plan (method 2), ZX_ENOMEM, ZX_ECUDA. Asynchronous
 * on `stream`.
 */
typedef struct {
    int32_t method;       /* 1 (schoolbook) or 2 (recursive): the resolved method */
    int32_t k;            /* log2 of the pieces per product (method 2; else 0) */
    int64_t N_inner;      /* N' of the inner ring (method 2; else 0) */
    int64_t stride_inner; /* limbs per inner cell in the scratch (method 2; else 0) */
    double cost_recursive;  /* estimated word operations per product, method 2 (0: no plan) */
    double cost_schoolbook; /* estimated word operations per product, method 1 */
} zx_pointwise_info;

int zx_pointwise_plan(int64_t N, int method, zx_pointwise_info *out);
int zx_pointwise(uint64_t *a, const uint64_t *b, int64_t n, int64_t N, int64_t stride_limbs, int method,
                 void *stream);

/*
 * The on-chip schedule of one job (host only): a sub-transform of 2^ls cells (TFT: kind 0,
 * ITFT: kind 1) with the given z, n, f, spread over 2^lc CTAs of a cluster, over
 * Z/(2^N+1) with omega = 2 (mode 0), S[y]/(y^N+1) with omega = y (mode 1: rotations mod 2N,
 * the ITFT's doublings and halvings as scalar flags) or Z/(2^N+1) with omega = sqrt2 (mode 2:
 * rotations mod 4N).
 * Writes the job image -- header [nstages, C, load layout, store layout], per stage
 * [type, arg, per-CTA program offsets], then per-CTA programs of leveled base-case butterflies
 * of Algorithms 1 and 2 (see paper_0810_3203_gb300/csrc/common.h for the word layout) -- into
 * buf (cap_words uint32 words) and its length into *size_words. ZX_EBUFSIZE when buf is too
 * small (the needed length is still written), ZX_EINVAL on bad sizes. For inspection and tests.
 */
int zx_job_program(int kind, int ls, int lc, int64_t z, int64_t n, int f, int64_t N, int mode, uint32_t *buf,
                   int64_t cap_words, int64_t *size_words);

/*
 * The whole plan of one transform (host only, no device needed): the launches tft_ex / itft_ex
 * make for these arguments under the ring's current launch configuration, in stream order,
 * with every job's descriptor and the job images they run (mode 0: omega = 2, mode 2:
 * omega = sqrt2). For inspection and tests.
 *   jobs (int64 words): [passes, launches, jobs, images], then per launch
 *     [ls, lc, warps, program_words, count] followed by `count` jobs of 9 words
 *     [cell0, mstride, e, nload, nstore, nscale, escale, pad, image]: the job reads its cells
 *     m < nload at cell0 + m mstride (the others are zero), runs image `image` with weight
 *     exponent e, stores its cells m < nstore there, those with m < nscale times omega^escale;
 *     pad bits 0-7 hold the job's log2 size when it differs from the launch's ls, bit 8 that
 *     its stores stay in the kernel's internal form (a later launch stores them again).
 *   images (uint32 words): images + 1 offsets, then the images (zx_job_program's format)
 *     back to back, image k at words [offset k, offset k+1) after the offsets.
 * The lengths go to *jobs_words and *images_words; ZX_EBUFSIZE when either buffer is too small.
 */
int zx_transform_jobs(int kind, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e, int scale, int mode,
                      int64_t *jobs, int64_t cap_jobs, int64_t *jobs_words, uint32_t *images, int64_t cap_images,
                      int64_t *images_words);

/*
 * The persistent form of the same plan (host only, no device needed; no counterpart in the
 * paper, which runs the passes one after the other). When every job of the plan runs on a
 * single CTA, tft_ex / itft_ex enqueue one launch whose CTAs claim the jobs in a fixed order from
 * a counter; a claimed job first waits (bounded) until the jobs it depends on have finished: the
 * last job that stored a cell it reads or stores, and every job that read a cell it stores since
 * that cell was last stored. Every dependency comes earlier in the claim order, so the earliest
 * unfinished job can always run. The order is a list schedule over `slots` concurrent CTAs
 * (0: 456, three per SM of a GB300) that takes the deepest ready pass first, so that a pass
 * re-reads the cells the previous pass has just written from L2.
 *   out (int64 words): [count], then per claim position k: [job, ndeps, deps...] where job is the
 *   position of the job in zx_transform_jobs' list (launches in order, their jobs in order) and
 *   deps are claim positions below k. count = 0 when the plan runs as one launch per pass.
 * The length goes to *words; ZX_EBUFSIZE when out is too small (the length is still written).
 */
int zx_transform_schedule(int kind, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e, int scale, int mode,
                          int slots, int64_t *out, int64_t cap, int64_t *words);

/*
 * Bounded device-side waits. The transform kernel stages the cells of single-CTA jobs in
 * shared memory with bulk (TMA) copies and waits for their completion on an mbarrier with a
 * time limit of one second. A wait that runs out waits once more (also bounded) for the copies
 * still in flight, then stops that CTA and sets a status word of the device; the outputs of
 * the call it belonged to are then unspecified. In a persistent launch (zx_transform_schedule)
 * a job's wait for the jobs it depends on is bounded too (two seconds); one that runs out sets
 * the same status word, and later waits of any launch on the device then return at once. Launches do not synchronise, so the status is
 * read on request:
 *   zx_wait_status  synchronises `stream`, then reads and clears the status word of the current
 *                   device (atomically). ZX_OK when no wait gave up since the last read,
 *                   ZX_ETIMEOUT when one did (or when a job that moves cells by tensor copies
 *                   found its shared memory misaligned and ran nothing, which the kernel's
 *                   declaration rules out), ZX_ECUDA on a CUDA error.
 *   zx_wait_probe   enqueues one warp that waits on an mbarrier that nothing completes until
 *                   limit_us microseconds (1 .. 10^6, else ZX_EINVAL) have passed, and reports
 *                   it as the transform kernel does: the error path, taken without a fault.
 *                   Asynchronous; for tests.
 */
int zx_wait_status(void *stream);
int zx_wait_probe(int64_t limit_us, void *stream);

/* Human-readable name of a status code (static storage). */
const char *zx_strerror(int code);

/* Description of the calling thread's most recent failure (static per-thread storage). */
const char *zx_last_error(void);

/* Library version string, e.g. "tftgpu 0.1 sm_103a". */
const char *zx_version(void);

#ifdef __cplusplus
}
#endif
#endif
