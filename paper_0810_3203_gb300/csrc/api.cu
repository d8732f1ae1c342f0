// C ABI of libtftgpu (declared in include/tftgpu.h): argument checks, planning, staging of
// host operands, and the order of kernel launches. No arithmetic of the method runs here.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tftgpu.h"
#include "common.h"
#include "host.h"

namespace tftgpu {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

static int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

static int cuda_fail(cudaError_t e, const char *where) {
  return fail(ZX_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static int64_t ceil_log2(int64_t v) {
  int64_t l = 0;
  while ((int64_t(1) << l) < v) l++;
  return l;
}

static int check_ring(int l, int64_t N, int mode = RING_FERMAT) {
  if (N < 64 || N % 64 != 0) return fail(ZX_EINVAL, "N must be a positive multiple of 64");
  if (l < 1 || l > 30) return fail(ZX_EINVAL, "l out of range");
  if (omega_order(N, mode) % (int64_t(1) << l) != 0)
    return fail(ZX_EINVAL, mode == RING_SQRT2 ? "L = 2^l must divide 4N (omega_L = sqrt2^(4N/L))"
                                              : "L = 2^l must divide 2N (omega_L = 2^(2N/L))");
  if (!ring_supported(N))
    return fail(ZX_EUNSUPPORTED, "N must be <= 1024 (multiple of 64) or a multiple of 1024 up to 32768");
  return ZX_OK;
}

static int check_sizes(int kind, int l, int64_t z, int64_t n, int f) {
  int64_t L = int64_t(1) << l;
  if (kind == KIND_TFT) {
    if (z < 1 || z > L || n < 1 || n > L) return fail(ZX_EINVAL, "TFT needs 1 <= z, n <= L");
  } else {
    if ((f != 0 && f != 1) || z < 1 || z > L || n < 0 || n > z || n + f < 1 || n + f > L)
      return fail(ZX_EINVAL, "ITFT needs 1 <= z <= L, 0 <= n <= z, 1 <= n + f <= L, f in {0,1}");
  }
  return ZX_OK;
}

static int transform(int kind, uint64_t *x, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e,
                     int64_t stride_limbs, int scale, void *stream, int mode = RING_FERMAT) {
  int rc = check_ring(l, N, mode);
  if (rc) return rc;
  if (!x) return fail(ZX_EINVAL, "x is NULL");
  if (stride_limbs < N / 64 + 1) return fail(ZX_EINVAL, "stride_limbs < N/64 + 1");
  if ((rc = check_sizes(kind, l, z, n, f))) return rc;
  int err = ZX_OK;
  const TransformPlan *p = get_transform_plan(kind, l, z, n, f, N, e, stride_limbs, scale, &err, mode);
  if (!p) return err ? fail(err, "planning failed") : fail(ZX_ECUDA, "planning failed");
  cudaError_t ce = run_transform(*p, x, stride_limbs, cudaStream_t(stream));
  if (ce != cudaSuccess) return cuda_fail(ce, "transform launch");
  return ZX_OK;
}

struct ZxPlan {
  int l;
  int mode;  // RING_FERMAT, or RING_SQRT2 when omega = sqrt2 allows a smaller ring
  int64_t N, n, nf, stride, limbs_h, L;
  Ring ring;
};

static int make_zx_plan(int64_t lf, int64_t bf, int64_t lg, int64_t bg, int sgn, ZxPlan *zp) {
  if (lf < 1 || lg < 1) return fail(ZX_EINVAL, "polynomial length must be >= 1");
  if (bf < 1 || bg < 1) return fail(ZX_EINVAL, "coefficient bit bound must be >= 1");
  int64_t n = lf + lg - 1;
  int64_t l = std::max<int64_t>(1, ceil_log2(n));
  if (l > 16) return fail(ZX_EUNSUPPORTED, "product length above 65536");
  int64_t L = int64_t(1) << l;
  int64_t need = bf + bg + ceil_log2(std::min(lf, lg)) + (sgn ? 1 : 0);
  // omega = 2 needs L | 2N; omega = sqrt2 (4 | N) needs only L | 4N, a ring up to half the size
  const int64_t unit = need <= 1024 ? 64 : 1024;
  const int64_t align = std::max<int64_t>(unit, L / 2), align4 = std::max<int64_t>(unit, L / 4);
  int64_t N = (need + align - 1) / align * align;
  const int64_t N4 = (need + align4 - 1) / align4 * align4;
  int mode = RING_FERMAT;
  if (N4 < N && ring_supported(N4)) {
    N = N4;
    mode = RING_SQRT2;
  }
  if (!ring_supported(N)) return fail(ZX_EUNSUPPORTED, "product needs a ring above 2^32768 + 1");
  zp->l = int(l);
  zp->mode = mode;
  zp->N = N;
  zp->n = n;
  zp->nf = zero_padded_outputs(int(l), n, N);
  zp->L = L;
  int64_t W = N / 64 + 1;
  zp->stride = W + (W & 1);  // even stride keeps every cell 16-byte aligned
  zp->limbs_h = (need + 63) / 64;
  zp->ring = make_ring(N);
  return ZX_OK;
}

static int64_t poly_bits(const zx_poly *p) { return p->bits > 0 ? p->bits : 64 * p->limbs; }

static int check_poly(const zx_poly *p, const char *name) {
  if (!p) return fail(ZX_EINVAL, std::string(name) + " is NULL");
  if (p->len < 1 || p->limbs < 1 || !p->data) return fail(ZX_EINVAL, std::string(name) + ": bad len/limbs/data");
  if (p->where != ZX_HOST && p->where != ZX_DEVICE) return fail(ZX_EINVAL, std::string(name) + ": bad where");
  return ZX_OK;
}

// device pointer to the operand's coefficients, staging host data through `tmp`
static int stage_in(const zx_poly *p, uint64_t **dptr, uint64_t **tmp, cudaStream_t s) {
  *tmp = nullptr;
  if (p->where == ZX_DEVICE) {
    *dptr = p->data;
    return ZX_OK;
  }
  size_t bytes = size_t(p->len) * size_t(p->limbs) * 8;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(tmp), bytes, s);
  if (e != cudaSuccess) return fail(ZX_ENOMEM, "staging allocation");
  e = cudaMemcpyAsync(*tmp, p->data, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
  *dptr = *tmp;
  return ZX_OK;
}

int device_product(const zx_poly *f, const zx_poly *g, zx_poly *h, BatchProduct *b) {
  int rc;
  if ((rc = check_poly(f, "f")) || (rc = check_poly(g, "g")) || (rc = check_poly(h, "h"))) return rc;
  if (f->where != ZX_DEVICE || g->where != ZX_DEVICE || h->where != ZX_DEVICE)
    return fail(ZX_EINVAL, "operands must be in device memory");
  if (h->len != f->len + g->len - 1) return fail(ZX_EINVAL, "h->len must be f->len + g->len - 1");
  const int sgn = (f->is_signed || g->is_signed) ? 1 : 0;
  ZxPlan zp;
  if ((rc = make_zx_plan(f->len, poly_bits(f), g->len, poly_bits(g), sgn, &zp))) return rc;
  if (h->limbs < zp.limbs_h) {
    h->limbs = zp.limbs_h;
    return fail(ZX_EBUFSIZE, "h->limbs too small (needed count written to h->limbs)");
  }
  b->f = f->data;
  b->g = g->data;
  b->h = h->data;
  b->len_f = f->len;
  b->len_g = g->len;
  b->limbs_f = f->limbs;
  b->limbs_g = g->limbs;
  b->limbs_h = h->limbs;
  b->signed_f = f->is_signed ? 1 : 0;
  b->signed_g = g->is_signed ? 1 : 0;
  b->sgn = sgn;
  b->l = zp.l;
  b->N = zp.N;
  b->n = zp.n;
  b->nf = zp.nf;
  b->stride = zp.stride;
  b->mode = zp.mode;
  return ZX_OK;
}

// A non-blocking stream of the calling thread on the current device, with two events, for
// work that forks from a caller's stream and joins it again (events order it both ways, so a
// helper shared by successive calls is always correct).
cudaError_t helper_stream(cudaStream_t *s, cudaEvent_t *fork, cudaEvent_t *join) {
  struct Helper {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
  };
  static thread_local Helper per_dev[16];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  Helper &h = per_dev[dev];
  if (!h.s) {
    if ((e = cudaStreamCreateWithFlags(&h.s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&h.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&h.join, cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  *s = h.s;
  *fork = h.fork;
  *join = h.join;
  return cudaSuccess;
}

// zx_mul_batch: a product with a transform of 2^13 cells or more (at least 512 jobs of 16 cells
// a pass, more than the 456 CTA slots of a GB300) fills the GPU on its own, so it runs as its own
// launch chain (zx_mul) on one of kChainStreams streams forked from the caller's; the smaller
// ones share merged launches. On 512 mixed products (lengths 200-20000, 64-1024 bits), dealing
// every product onto 4 streams measured 4.5 % faster than merging all of them (1738 against
// 1662 products/s).
constexpr int kChainMinL = 13;
constexpr int kChainStreams = 4;

static cudaError_t chain_streams(cudaStream_t (&out)[kChainStreams]) {
  static thread_local cudaStream_t per_dev[16][kChainStreams] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  for (int k = 0; k < kChainStreams; k++) {
    if (!per_dev[dev][k] && (e = cudaStreamCreateWithFlags(&per_dev[dev][k], cudaStreamNonBlocking)) != cudaSuccess)
      return e;
    out[k] = per_dev[dev][k];
  }
  return cudaSuccess;
}

// Pointwise method for ring N: 1 (schoolbook) or 2 (recursive, with *rp filled). Auto picks the
// recursion when its estimated word operations fall below kRecAutoRatio of the schoolbook's
// NW^2 word products. Measured on GB300 (10^4 products at N = 32768: 9.27 ms recursive, 1.38 ms
// schoolbook, estimates 158720 and 1048576 operations), one estimated operation of the
// recursion costs about 44 times one of the schoolbook kernel, so no ring up to N = 32768
// crosses over.
constexpr double kRecAutoRatio = 1.0 / 44.0;

int resolve_pointwise(int64_t N, int method, RecPlan *rp, int *resolved) {
  if (method < 0 || method > 2) return fail(ZX_EINVAL, "method must be 0 (auto), 1 or 2");
  if (!ring_supported(N)) return fail(ZX_EUNSUPPORTED, "unsupported N");
  const bool have = rec_plan_auto(N, rp);
  if (method == 2 && !have) return fail(ZX_EUNSUPPORTED, "no recursive plan for this N");
  const double nw = double(N / 32);
  if (method == 0) method = (have && rp->cost < kRecAutoRatio * nw * nw) ? 2 : 1;
  *resolved = method;
  return ZX_OK;
}

cudaError_t pointwise_products(uint64_t *a, const uint64_t *b, int64_t n, int64_t stride, const Ring &r,
                               cudaStream_t s, int *err) {
  RecPlan rp;
  int m = 1;
  *err = resolve_pointwise(r.N, 0, &rp, &m);
  if (*err) return cudaErrorInvalidValue;
  if (m == 2) return run_rec_pointwise(a, b, n, stride, r, rp, s, err);
  return launch_pointwise(a, b, n, stride, r, s);
}

}  // namespace tftgpu

using namespace tftgpu;

extern "C" {

int tft_ex(uint64_t *x, int l, int64_t z, int64_t n, int64_t N, int64_t e, int64_t stride_limbs, void *stream) {
  return transform(KIND_TFT, x, l, z, n, 0, N, e, stride_limbs, 0, stream);
}

int tft(uint64_t *x, int l, int64_t n, int64_t N, void *stream) {
  return transform(KIND_TFT, x, l, n, n, 0, N, 0, N / 64 + 1, 0, stream);
}

int itft_ex(uint64_t *x, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e, int64_t stride_limbs,
            int scale, void *stream) {
  if (scale != 0 && scale != 1) return fail(ZX_EINVAL, "scale must be 0 or 1");
  return transform(KIND_ITFT, x, l, z, n, f, N, e, stride_limbs, scale, stream);
}

int tft_sqrt2(uint64_t *x, int l, int64_t z, int64_t n, int64_t N, int64_t e, int64_t stride_limbs, void *stream) {
  return transform(KIND_TFT, x, l, z, n, 0, N, e, stride_limbs, 0, stream, RING_SQRT2);
}

int itft_sqrt2(uint64_t *x, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e, int64_t stride_limbs,
               int scale, void *stream) {
  if (scale != 0 && scale != 1) return fail(ZX_EINVAL, "scale must be 0 or 1");
  return transform(KIND_ITFT, x, l, z, n, f, N, e, stride_limbs, scale, stream, RING_SQRT2);
}

int itft(uint64_t *x, int l, int64_t n, int64_t N, void *stream) {
  return transform(KIND_ITFT, x, l, n, n, 0, N, 0, N / 64 + 1, 1, stream);
}

int zx_transform_plan(int kind, int l, int64_t z, int64_t n, int f, int64_t N, zx_transform_info *out) {
  if (!out) return fail(ZX_EINVAL, "out is NULL");
  if (kind != KIND_TFT && kind != KIND_ITFT) return fail(ZX_EINVAL, "kind must be 0 (TFT) or 1 (ITFT)");
  int rc = check_ring(l, N, RING_SQRT2);  // the shape is the same for omega = 2 and sqrt2
  if (rc) return rc;
  if ((rc = check_sizes(kind, l, z, n, f))) return rc;
  std::memset(out, 0, sizeof *out);
  int passes = 0, launches = 0, onchip = 0, cl = 0;
  int64_t jobs = 0;
  plan_shape(kind, l, z, n, f, N, &passes, &launches, &jobs, &onchip, &cl);
  out->cluster_l = cl;
  out->passes = passes;
  out->launches = launches;
  out->jobs = jobs;
  out->onchip_l = onchip;
  out->K = make_ring(N).K;
  return ZX_OK;
}

int zx_pointwise_plan(int64_t N, int method, zx_pointwise_info *out) {
  if (!out) return fail(ZX_EINVAL, "out is NULL");
  RecPlan rp;
  int m = 1;
  int rc = resolve_pointwise(N, method, &rp, &m);
  if (rc) return rc;
  std::memset(out, 0, sizeof *out);
  out->method = m;
  const double nw = double(N / 32);
  out->cost_schoolbook = nw * nw;
  if (rec_plan_auto(N, &rp)) {
    out->cost_recursive = rp.cost;
    if (m == 2) {
      out->k = rp.k;
      out->N_inner = rp.Ni;
      out->stride_inner = rp.stride_i;
    }
  }
  return ZX_OK;
}

int zx_pointwise(uint64_t *a, const uint64_t *b, int64_t n, int64_t N, int64_t stride_limbs, int method,
                 void *stream) {
  if (n < 0) return fail(ZX_EINVAL, "n < 0");
  if (n > 0 && (!a || !b)) return fail(ZX_EINVAL, "a or b is NULL");
  if (stride_limbs < N / 64 + 1) return fail(ZX_EINVAL, "stride_limbs < N/64 + 1");
  RecPlan rp;
  int m = 1;
  int rc = resolve_pointwise(N, method, &rp, &m);
  if (rc) return rc;
  if (n == 0) return ZX_OK;
  if (a != b && a < b + n * stride_limbs && b < a + n * stride_limbs)
    return fail(ZX_EINVAL, "a and b overlap");
  const Ring r = make_ring(N);
  cudaError_t ce;
  if (m == 2) {
    int err = ZX_OK;
    ce = run_rec_pointwise(a, b, n, stride_limbs, r, rp, cudaStream_t(stream), &err);
    if (ce != cudaSuccess) return err == ZX_ENOMEM ? fail(ZX_ENOMEM, "scratch") : cuda_fail(ce, "recursive pointwise");
  } else {
    ce = launch_pointwise(a, b, n, stride_limbs, r, cudaStream_t(stream));
    if (ce != cudaSuccess) return cuda_fail(ce, "pointwise");
  }
  return ZX_OK;
}

int zx_job_program(int kind, int ls, int lc, int64_t z, int64_t n, int f, int64_t N, int mode, uint32_t *buf,
                   int64_t cap_words, int64_t *size_words) {
  if (!size_words) return fail(ZX_EINVAL, "size_words is NULL");
  if (kind != KIND_TFT && kind != KIND_ITFT) return fail(ZX_EINVAL, "kind must be 0 (TFT) or 1 (ITFT)");
  if (mode != RING_FERMAT && mode != RING_SN && mode != RING_SQRT2) return fail(ZX_EINVAL, "mode must be 0, 1 or 2");
  if (lc < 0 || lc > kMaxClusterLog2 || ls < 1 || ls - lc < lc || ls - lc < 1 || ls > 16)
    return fail(ZX_EINVAL, "need 1 <= ls <= 16 and 0 <= lc <= 4 with 2 lc <= ls");
  if (mode == RING_SN ? (N < 1 || (N & (N - 1)) != 0) : (N < 64 || N % 64 != 0))
    return fail(ZX_EINVAL, "N must be a multiple of 64 (a power of two for mode 1)");
  if (omega_order(N, mode) % (int64_t(1) << ls) != 0) return fail(ZX_EINVAL, "2^ls must divide the order of omega");
  int rc = check_sizes(kind, ls, z, n, f);
  if (rc) return rc;
  std::vector<uint32_t> img = build_job_image(kind, ls, lc, z, n, f, N, nullptr, mode);
  *size_words = int64_t(img.size());
  if (!buf || cap_words < int64_t(img.size())) return fail(ZX_EBUFSIZE, "buffer too small for the job image");
  std::memcpy(buf, img.data(), img.size() * 4);
  return ZX_OK;
}

int zx_plan(int64_t len_f, int64_t bits_f, int64_t len_g, int64_t bits_g, int is_signed, zx_plan_info *out) {
  if (!out) return fail(ZX_EINVAL, "out is NULL");
  ZxPlan zp;
  int rc = make_zx_plan(len_f, bits_f, len_g, bits_g, is_signed ? 1 : 0, &zp);
  if (rc) return rc;
  std::memset(out, 0, sizeof *out);
  out->l = zp.l;
  out->K = zp.ring.K;
  out->N = zp.N;
  out->n = zp.n;
  out->stride_limbs = zp.stride;
  out->limbs_h = zp.limbs_h;
  out->scratch_bytes = 2 * zp.L * zp.stride * 8;
  out->tft_passes = count_passes(KIND_TFT, zp.l, zp.nf, zp.nf, 0, zp.N);
  out->itft_passes = count_passes(KIND_ITFT, zp.l, zp.nf, zp.nf, 0, zp.N);
  out->n_fft = zp.nf;
  out->sqrt2 = zp.mode == RING_SQRT2 ? 1 : 0;
  return ZX_OK;
}

int zx_mul(const zx_poly *f, const zx_poly *g, zx_poly *h, void *stream) {
  int rc;
  if ((rc = check_poly(f, "f")) || (rc = check_poly(g, "g")) || (rc = check_poly(h, "h"))) return rc;
  if (h->len != f->len + g->len - 1) return fail(ZX_EINVAL, "h->len must be f->len + g->len - 1");
  int sgn = (f->is_signed || g->is_signed) ? 1 : 0;
  ZxPlan zp;
  if ((rc = make_zx_plan(f->len, poly_bits(f), g->len, poly_bits(g), sgn, &zp))) return rc;
  if (h->limbs < zp.limbs_h) {
    h->limbs = zp.limbs_h;
    return fail(ZX_EBUFSIZE, "h->limbs too small (needed count written to h->limbs)");
  }
  cudaStream_t s = cudaStream_t(stream);
  h->is_signed = sgn;
  uint64_t *df = nullptr, *dg = nullptr, *tf = nullptr, *tg = nullptr, *F = nullptr, *Gb = nullptr, *hd = nullptr;
  auto cleanup = [&]() {
    if (tf) cudaFreeAsync(tf, s);
    if (tg) cudaFreeAsync(tg, s);
    if (F) cudaFreeAsync(F, s);
    if (Gb) cudaFreeAsync(Gb, s);
    if (hd && hd != h->data) cudaFreeAsync(hd, s);
  };
  if ((rc = stage_in(f, &df, &tf, s)) || (rc = stage_in(g, &dg, &tg, s))) {
    cleanup();
    return rc;
  }
  size_t ring_bytes = size_t(zp.L) * size_t(zp.stride) * 8;
  if (cudaMallocAsync(reinterpret_cast<void **>(&F), ring_bytes, s) != cudaSuccess ||
      cudaMallocAsync(reinterpret_cast<void **>(&Gb), ring_bytes, s) != cudaSuccess) {
    cleanup();
    return fail(ZX_ENOMEM, "ring buffers");
  }
  size_t hbytes = size_t(h->len) * size_t(h->limbs) * 8;
  if (h->where == ZX_DEVICE) {
    hd = h->data;
  } else if (cudaMallocAsync(reinterpret_cast<void **>(&hd), hbytes, s) != cudaSuccess) {
    cleanup();
    return fail(ZX_ENOMEM, "output staging");
  }
  cudaError_t ce;
  int err = ZX_OK;
  const TransformPlan *pf = get_transform_plan(KIND_TFT, zp.l, f->len, zp.nf, 0, zp.N, 0, zp.stride, 0, &err, zp.mode);
  const TransformPlan *pg =
      pf ? get_transform_plan(KIND_TFT, zp.l, g->len, zp.nf, 0, zp.N, 0, zp.stride, 0, &err, zp.mode) : nullptr;
  const TransformPlan *pi =
      pg ? get_transform_plan(KIND_ITFT, zp.l, zp.nf, zp.nf, 0, zp.N, 0, zp.stride, 1, &err, zp.mode) : nullptr;
  if (!pi) {
    cleanup();
    return fail(err ? err : ZX_ECUDA, "planning failed");
  }
  // the two forward transforms are independent: g's runs on a helper stream forked from s
  cudaStream_t s2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  if ((ce = helper_stream(&s2, &fork, &join)) != cudaSuccess || (ce = cudaEventRecord(fork, s)) != cudaSuccess ||
      (ce = cudaStreamWaitEvent(s2, fork, 0)) != cudaSuccess ||
      (ce = launch_pack(dg, g->len, g->limbs, g->is_signed, Gb, zp.stride, zp.ring, s2)) != cudaSuccess ||
      (ce = run_transform(*pg, Gb, zp.stride, s2)) != cudaSuccess || (ce = cudaEventRecord(join, s2)) != cudaSuccess ||
      (ce = launch_pack(df, f->len, f->limbs, f->is_signed, F, zp.stride, zp.ring, s)) != cudaSuccess ||
      (ce = run_transform(*pf, F, zp.stride, s)) != cudaSuccess || (ce = cudaStreamWaitEvent(s, join, 0)) != cudaSuccess ||
      (ce = pointwise_products(F, Gb, zp.nf, zp.stride, zp.ring, s, &err)) != cudaSuccess ||
      (ce = run_transform(*pi, F, zp.stride, s)) != cudaSuccess ||
      (ce = launch_lift(F, zp.n, zp.stride, sgn, hd, h->limbs, zp.ring, s)) != cudaSuccess) {
    if (s2 && join && cudaEventRecord(join, s2) == cudaSuccess) cudaStreamWaitEvent(s, join, 0);  // before the frees
    cleanup();
    return cuda_fail(ce, "zx_mul launch");
  }
  if (h->where == ZX_HOST) {
    if ((ce = cudaMemcpyAsync(h->data, hd, hbytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess) {
      cleanup();
      return cuda_fail(ce, "device-to-host copy");
    }
  }
  cleanup();
  if (f->where == ZX_HOST || g->where == ZX_HOST || h->where == ZX_HOST) {
    if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ce, "stream synchronize");
  }
  return ZX_OK;
}

int zx_mul_batch(const zx_poly *fs, const zx_poly *gs, zx_poly *hs, int count, void *stream) {
  if (count < 0 || (count > 0 && (!fs || !gs || !hs))) return fail(ZX_EINVAL, "bad batch arguments");
  std::vector<BatchProduct> items(static_cast<size_t>(count));
  for (int i = 0; i < count; i++) {
    int rc = device_product(fs + i, gs + i, hs + i, &items[size_t(i)]);
    if (rc) {
      set_error("product " + std::to_string(i) + ": " + g_last_error);
      return rc;
    }
  }
  for (int i = 0; i < count; i++) hs[i].is_signed = items[size_t(i)].sgn;
  // products whose transforms fill the GPU on their own run as their own launch chains, dealt
  // largest first onto forked streams; the others share the merged launches
  std::vector<BatchProduct> merged;
  std::vector<int> chained;
  for (int i = 0; i < count; i++) {
    if (items[size_t(i)].l >= kChainMinL)
      chained.push_back(i);
    else
      merged.push_back(items[size_t(i)]);
  }
  std::stable_sort(chained.begin(), chained.end(), [&](int a, int b) {
    const BatchProduct &x = items[size_t(a)], &y = items[size_t(b)];
    return (x.stride << x.l) > (y.stride << y.l);
  });
  cudaStream_t s = cudaStream_t(stream);
  cudaStream_t cs[kChainStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaError_t ce = cudaSuccess;
  if (!chained.empty()) {
    if ((ce = chain_streams(cs)) != cudaSuccess || (ce = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming)) != cudaSuccess ||
        (ce = cudaEventRecord(fork, s)) != cudaSuccess) {
      if (fork) cudaEventDestroy(fork);
      return cuda_fail(ce, "batch streams");
    }
    for (int k = 0; k < kChainStreams; k++) cudaStreamWaitEvent(cs[k], fork, 0);
    cudaEventDestroy(fork);
  }
  std::string msg;
  int rc = run_mul_batch(merged, s, &msg);
  std::string chain_msg;
  for (size_t j = 0; j < chained.size() && rc == ZX_OK; j++) {
    const int i = chained[j];
    if ((rc = zx_mul(fs + i, gs + i, hs + i, cs[j % kChainStreams])) != ZX_OK)
      chain_msg = "product " + std::to_string(i) + ": " + g_last_error;
  }
  if (!chained.empty()) {
    // the caller's stream waits for every chain, also after an error (before the caller frees)
    for (int k = 0; k < kChainStreams; k++) {
      cudaEvent_t join = nullptr;
      if (cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess) {
        if (cudaEventRecord(join, cs[k]) == cudaSuccess) cudaStreamWaitEvent(s, join, 0);
        cudaEventDestroy(join);
      } else {
        cudaStreamSynchronize(cs[k]);
      }
    }
  }
  if (rc) return fail(rc, chain_msg.empty() ? msg : chain_msg);
  return ZX_OK;
}

// fraction of the kept configuration's time another must reach to replace it
static constexpr float kTuneMargin = 0.97f;

int zx_tune(uint64_t *x, int l, int64_t n, int64_t N, int64_t stride_limbs, int reps, void *stream,
            zx_tune_info *out) {
  if (!out || !x) return fail(ZX_EINVAL, "x or out is NULL");
  // the round trips use omega = 2 when L | 2N, else omega = sqrt2 (L | 4N), as products do
  const int mode = (2 * N) % (int64_t(1) << (l < 1 ? 1 : l)) == 0 ? RING_FERMAT : RING_SQRT2;
  int rc = check_ring(l, N, mode);
  if (rc) return rc;
  if ((rc = check_sizes(KIND_TFT, l, n, n, 0))) return rc;
  if (stride_limbs < N / 64 + 1) return fail(ZX_EINVAL, "stride_limbs < N/64 + 1");
  if (reps < 1 || reps > 100) return fail(ZX_EINVAL, "reps must be in [1, 100]");
  const Ring r = make_ring(N);
  const PlanConfig before = plan_config(N), def = default_config(r);
  // the largest job that still lets three CTAs share an SM
  int ls3 = 1;
  while (ls3 < 16 && (size_t(2) << ls3) * (size_t(r.pitch) + 1) * 4 <= size_t(72) * 1024) ls3++;
  std::vector<PlanConfig> cands;
  PlanConfig def_kept = def;
  def_kept.fused = before.fused;
  def_kept.tma = before.tma;
  cands.push_back(def_kept);
  for (int ls_max : {def.ls_max, ls3})
    for (int ls_c = 3; ls_c <= 6; ls_c++)
      for (int mw : {8, 16})
        for (int sp = 0; sp <= 2; sp++) {
          if (sp == 1 && !(l & 1)) continue;  // the ceil split differs for odd l only
          for (int mlc : {1, 2, 4}) {
            if ((sp == 2) != (mlc < 4)) continue;  // capped clusters go with the fewest-pass split
            PlanConfig c;
            c.ls_max = ls_max;
            c.ls_c = ls_c;
            c.max_warps = mw;
            c.split = sp;
            c.max_lc = mlc;
            c.fused = before.fused;  // kept as it is (see PlanConfig)
            c.tma = before.tma;
            if (!config_valid(r, c)) continue;
            bool dup = false;
            for (const PlanConfig &o : cands)
              dup = dup || (o.ls_max == c.ls_max && o.ls_c == c.ls_c && o.max_warps == c.max_warps &&
                            o.split == c.split && o.max_lc == c.max_lc);
            if (!dup) cands.push_back(c);
          }
        }
  cudaStream_t s = cudaStream_t(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return fail(ZX_ECUDA, "event");
  auto round_trip = [&]() {
    int q = transform(KIND_TFT, x, l, n, n, 0, N, 0, stride_limbs, 0, stream, mode);
    return q ? q : transform(KIND_ITFT, x, l, n, n, 0, N, 0, stride_limbs, 1, stream, mode);
  };
  float best = 1e30f, def_ms = -1.0f;
  PlanConfig chosen = before;
  // mean round-trip time under configuration c (plans and job images are built in the warm-up)
  auto time_cfg = [&](const PlanConfig &c, float *ms) {
    set_plan_config(N, c);
    int q = round_trip();
    if (q) return q;
    cudaEventRecord(e0, s);
    for (int k = 0; k < reps && !q; k++) q = round_trip();
    cudaEventRecord(e1, s);
    if (q) return q;
    if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_fail(cudaGetLastError(), "tuning run");
    cudaEventElapsedTime(ms, e0, e1);
    *ms /= float(reps);
    return ZX_OK;
  };
  for (const PlanConfig &c : cands) {
    float ms = 0.0f;
    if ((rc = time_cfg(c, &ms))) break;
    if (c.ls_max == def.ls_max && c.ls_c == def.ls_c && c.max_warps == def.max_warps && c.split == def.split &&
        c.max_lc == def.max_lc)
      def_ms = ms;
    // the default is timed first; another configuration replaces the one kept so far only when
    // it is at least 3 % faster, so that timing noise between configurations that round trips
    // alone cannot tell apart does not decide (their cost differs in batches and concurrent use)
    if (best >= 1e29f || ms < kTuneMargin * best) {
      best = ms;
      chosen = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  set_plan_config(N, rc ? before : chosen);
  if (rc) return rc;
  std::memset(out, 0, sizeof *out);
  out->ls_max = chosen.ls_max;
  out->ls_c = chosen.ls_c;
  out->max_warps = chosen.max_warps;
  out->split = chosen.split;
  out->fused = chosen.fused;
  out->max_cluster_log2 = chosen.max_lc;
  out->tma = chosen.tma;
  out->candidates = int32_t(cands.size());
  out->best_ms = best;
  out->default_ms = def_ms;
  return ZX_OK;
}

static int sn_transform(int kind, uint64_t *x, int l, int64_t z, int64_t n, int f, int64_t M, uint64_t m, int64_t e,
                        int64_t stride, int scale, void *stream) {
  if (!x) return fail(ZX_EINVAL, "x is NULL");
  if (M < 2 || (M & (M - 1)) != 0) return fail(ZX_EINVAL, "M must be a power of two >= 2");
  if (M > 2048) return fail(ZX_EUNSUPPORTED, "M above 2048 (elements of more than 1024 coefficients)");
  if (l < 1 || l > 11 || M % (int64_t(1) << l) != 0) return fail(ZX_EINVAL, "L = 2^l must divide M (omega_L = y^(M/L))");
  if (!(m & 1u) || m < 3 || m >= (uint64_t(1) << 63)) return fail(ZX_EINVAL, "m must be odd with 3 <= m < 2^63");
  if (stride < M / 2) return fail(ZX_EINVAL, "stride < M/2");
  int rc = check_sizes(kind, l, z, n, f);
  if (rc) return rc;
  int err = ZX_OK;
  const TransformPlan *p = get_sn_plan(kind, l, z, n, f, M / 2, e, scale, &err);
  if (!p) return err ? fail(err, "planning failed") : fail(ZX_ECUDA, "planning failed");
  cudaError_t ce = run_sn_transform(*p, x, stride, M / 2, m, cudaStream_t(stream));
  if (ce != cudaSuccess) return cuda_fail(ce, "transform launch");
  return ZX_OK;
}

int sn_tft(uint64_t *x, int l, int64_t z, int64_t n, int64_t M, uint64_t m, int64_t e, int64_t stride,
           void *stream) {
  return sn_transform(KIND_TFT, x, l, z, n, 0, M, m, e, stride, 0, stream);
}

int sn_itft(uint64_t *x, int l, int64_t z, int64_t n, int f, int64_t M, uint64_t m, int64_t e, int64_t stride,
            int scale, void *stream) {
  if (scale != 0 && scale != 1) return fail(ZX_EINVAL, "scale must be 0 or 1");
  return sn_transform(KIND_ITFT, x, l, z, n, f, M, m, e, stride, scale, stream);
}

int zx_config_get(int64_t N, zx_tune_info *out) {
  if (!out) return fail(ZX_EINVAL, "out is NULL");
  if (!ring_supported(N)) return fail(ZX_EUNSUPPORTED, "unsupported ring size N");
  const PlanConfig c = plan_config(N);
  std::memset(out, 0, sizeof *out);
  out->ls_max = c.ls_max;
  out->ls_c = c.ls_c;
  out->max_warps = c.max_warps;
  out->split = c.split;
  out->fused = c.fused;
  out->max_cluster_log2 = c.max_lc;
  out->tma = c.tma;
  return ZX_OK;
}

int zx_config_set(int64_t N, const zx_tune_info *cfg) {
  if (!ring_supported(N)) return fail(ZX_EUNSUPPORTED, "unsupported ring size N");
  const Ring r = make_ring(N);
  if (!cfg) {
    set_plan_config(N, default_config(r));
    return ZX_OK;
  }
  PlanConfig c;
  c.ls_max = cfg->ls_max;
  c.ls_c = cfg->ls_c;
  c.max_warps = cfg->max_warps;
  c.split = cfg->split;
  c.fused = cfg->fused;
  c.max_lc = cfg->max_cluster_log2;
  c.tma = cfg->tma;
  if (!config_valid(r, c)) return fail(ZX_EINVAL, "configuration not valid for this ring");
  set_plan_config(N, c);
  return ZX_OK;
}

const char *zx_strerror(int code) {
  switch (code) {
    case ZX_OK: return "ok";
    case ZX_EINVAL: return "invalid argument";
    case ZX_ENOMEM: return "out of memory";
    case ZX_ECUDA: return "CUDA error";
    case ZX_ETIMEOUT: return "device wait timed out";
    case ZX_EBUFSIZE: return "output buffer too small";
    case ZX_EUNSUPPORTED: return "unsupported size";
    default: return "unknown status";
  }
}

const char *zx_last_error(void) { return g_last_error.c_str(); }

int zx_transform_jobs(int kind, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e, int scale, int mode,
                      int64_t *jobs, int64_t cap_jobs, int64_t *jobs_words, uint32_t *images, int64_t cap_images,
                      int64_t *images_words) {
  if (!jobs_words || !images_words) return fail(ZX_EINVAL, "jobs_words or images_words is NULL");
  if (kind != KIND_TFT && kind != KIND_ITFT) return fail(ZX_EINVAL, "kind must be 0 (TFT) or 1 (ITFT)");
  if (mode != RING_FERMAT && mode != RING_SQRT2) return fail(ZX_EINVAL, "mode must be 0 or 2");
  int rc = check_ring(l, N, mode);
  if (rc) return rc;
  if ((rc = check_sizes(kind, l, z, n, f))) return rc;
  HostPlan hp;
  build_host_plan(kind, l, z, n, f, N, e, scale, &hp, mode);
  std::vector<int64_t> J = {hp.npasses, int64_t(hp.groups.size()), 0, int64_t(hp.programs.size())};
  for (const HostPlan::Group &g : hp.groups) {
    J.insert(J.end(), {g.ls, g.lc, g.nwarps, g.prog_words, int64_t(g.jobs.size())});
    for (size_t i = 0; i < g.jobs.size(); i++) {
      const JobDesc &d = g.jobs[i];
      J.insert(J.end(), {d.cell0, d.mstride, d.e, d.nload, d.nstore, d.nscale, d.escale, d.pad, g.prog_index[i]});
    }
    J[2] += int64_t(g.jobs.size());
  }
  std::vector<uint32_t> I(hp.programs.size() + 1, 0u);
  for (size_t k = 0; k < hp.programs.size(); k++) {
    I[k + 1] = I[k] + uint32_t(hp.programs[k].size());
  }
  for (const auto &img : hp.programs) I.insert(I.end(), img.begin(), img.end());
  *jobs_words = int64_t(J.size());
  *images_words = int64_t(I.size());
  if (!jobs || !images || cap_jobs < int64_t(J.size()) || cap_images < int64_t(I.size()))
    return fail(ZX_EBUFSIZE, "buffers too small for the plan");
  std::memcpy(jobs, J.data(), J.size() * sizeof(int64_t));
  std::memcpy(images, I.data(), I.size() * sizeof(uint32_t));
  return ZX_OK;
}

int zx_transform_schedule(int kind, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e, int scale, int mode,
                          int slots, int64_t *out, int64_t cap, int64_t *words) {
  if (!words) return fail(ZX_EINVAL, "words is NULL");
  if (kind != KIND_TFT && kind != KIND_ITFT) return fail(ZX_EINVAL, "kind must be 0 (TFT) or 1 (ITFT)");
  if (mode != RING_FERMAT && mode != RING_SQRT2) return fail(ZX_EINVAL, "mode must be 0 or 2");
  if (slots < 0) return fail(ZX_EINVAL, "slots must be >= 0");
  int rc = check_ring(l, N, mode);
  if (rc) return rc;
  if ((rc = check_sizes(kind, l, z, n, f))) return rc;
  FusedSchedule fs;
  build_host_schedule(kind, l, z, n, f, N, e, scale, &fs, mode, slots);
  std::vector<int64_t> W = {int64_t(fs.order.size())};
  for (size_t k = 0; k < fs.order.size(); k++) {
    W.push_back(fs.order[k]);
    W.push_back(fs.dep_off[k + 1] - fs.dep_off[k]);
    for (int32_t t = fs.dep_off[k]; t < fs.dep_off[k + 1]; t++) W.push_back(fs.deps[size_t(t)]);
  }
  *words = int64_t(W.size());
  if (!out || cap < int64_t(W.size())) return fail(ZX_EBUFSIZE, "buffer too small for the schedule");
  std::memcpy(out, W.data(), W.size() * sizeof(int64_t));
  return ZX_OK;
}

int zx_wait_status(void *stream) {
  uint32_t fault = 0;
  const cudaError_t ce = read_wait_status(&fault, cudaStream_t(stream));
  if (ce != cudaSuccess) return cuda_fail(ce, "reading the wait status");
  if (fault)
    return fail(ZX_ETIMEOUT, (fault & 4u) ? "a tensor-copy job found its shared memory misaligned (outputs unspecified)"
                                          : "a bounded device-side wait gave up (outputs of that call are unspecified)");
  return ZX_OK;
}

int zx_wait_probe(int64_t limit_us, void *stream) {
  if (limit_us < 1 || limit_us > 1000000) return fail(ZX_EINVAL, "limit_us must be in [1, 10^6]");
  const cudaError_t ce = run_wait_probe(uint64_t(limit_us) * 1000u, cudaStream_t(stream));
  if (ce != cudaSuccess) return cuda_fail(ce, "wait probe launch");
  return ZX_OK;
}

const char *zx_version(void) { return "tftgpu 0.1 sm_103a"; }

}  // extern "C"
