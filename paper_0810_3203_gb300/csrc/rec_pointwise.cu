// Pointwise products by recursion: a_i <- a_i b_i mod 2^N + 1 for i < n, computed by a second
// Schoenhage-Strassen level (Sec. 5.1 applied to the coefficient ring itself) on the same
// transform kernels instead of the register-window schoolbook kernel.
//
// With K' = 2^k pieces of M = N / K' bits, a = sum_t a_t 2^{M t} and 2^{M K'} = 2^N = -1, so
//   a b = sum_t c_t 2^{M t},  c_t = sum_{i+j=t} a_i b_j - sum_{i+j=t+K'} a_i b_j,
// a negacyclic convolution with |c_t| < K' 2^{2M}. It is computed exactly in the inner ring
// R' = Z/(2^{N'}+1), N' >= 2M + k + 1, where theta = 2^{N'/K'} has theta^{K'} = -1: the pieces
// are weighted by theta^t, transformed (TFT of length K' with z = n = K', Algorithm 1),
// multiplied pointwise in R', transformed back (ITFT, Algorithm 2, divided by K'), and
// unweighted by theta^{-t}. Each c_t is then recovered from its residue and the c_t are added
// at their offsets M t, modulo 2^N + 1.
//
// Kernels: split (one thread per inner cell), the transforms (one replicated launch per pass
// over every inner sequence of a chunk of products), the inner pointwise products, final
// (one thread per inner cell: unweight and add the bias B = 2^{k+2M}, so that every piece is
// the non-negative c_t + B), combine (one warp per product: add the pieces, remove the bias,
// reduce mod 2^N + 1).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.h"
#include "host.h"
#include "ring_warp.cuh"

namespace tftgpu {

namespace {

constexpr int kRecMaxInnerWords = 128;  // N' <= 4096

// y = x 2^E mod 2^{Ni} + 1 on per-thread words (x canonical: words [0, nw) plus xtop for the
// value 2^{Ni}), E in [0, 2 Ni); returns the top bit of y. x 2^E for E >= Ni is -(x 2^{E-Ni});
// 2^{Ni} = -1 reads as -1; for x < 2^{Ni} and E < Ni, x 2^E = lo - hi with lo = (x << E) mod
// 2^{Ni} and hi = x >> (Ni - E), plus p' = 2^{Ni} + 1 when that is negative.
__device__ uint32_t small_mul2exp(uint32_t *y, const uint32_t *x, uint32_t xtop, int E, int nw) {
  const int Ni = 32 * nw;
  bool neg = false;
  if (E >= Ni) {
    E -= Ni;
    neg = true;
  }
  uint32_t top = 0;
  if (xtop) {
    // -2^E
    for (int w = 0; w < nw; w++) y[w] = 0u;
    if (E == 0) {
      top = 1u;  // 2^{Ni} = -1 itself
    } else {
      y[E >> 5] = 1u << (E & 31);
      neg = !neg;
    }
  } else {
    const int q = E >> 5, r = E & 31;
    uint32_t borrow = 0;
    for (int w = 0; w < nw; w++) {
      // lo word w = bits [32 w - E, 32 w - E + 32) of x; hi word w = bits [Ni - E + 32 w, ..) of x
      const int u = w - q;
      const uint32_t cur = (u >= 0 && u < nw) ? x[u] : 0u, prv = (u - 1 >= 0 && u - 1 < nw) ? x[u - 1] : 0u;
      const uint32_t lo = r ? __funnelshift_l(prv, cur, r) : cur;
      const int v = nw + w - q;  // hi word w = word (nw + w) of x << E
      const uint32_t hc = (v >= 0 && v < nw) ? x[v] : 0u, hp = (v - 1 >= 0 && v - 1 < nw) ? x[v - 1] : 0u;
      const uint32_t hi = r ? __funnelshift_l(hp, hc, r) : hc;
      const uint64_t d = uint64_t(lo) - hi - borrow;
      y[w] = uint32_t(d);
      borrow = uint32_t(d >> 63);
    }
    if (borrow) {
      // + 2^{Ni} + 1: the borrow cancels 2^{Ni}, then + 1
      uint32_t c = 1u;
      for (int w = 0; w < nw && c; w++) {
        y[w] += 1u;
        c = y[w] == 0u;
      }
      top = c;
    }
  }
  if (neg) {
    // p' - y for y != 0
    bool nz = top != 0;
    for (int w = 0; w < nw; w++) nz = nz || y[w] != 0u;
    if (nz) {
      if (top) {
        // p' - 2^{Ni} = 1
        for (int w = 0; w < nw; w++) y[w] = 0u;
        y[0] = 1u;
        top = 0;
      } else {
        // 2^{Ni} + 1 - y = (~y + 1) + 1 over nw words, y in [1, 2^{Ni} - 1]: ~y + 2 <= 2^{Ni}
        uint32_t c = 2u;
        for (int w = 0; w < nw; w++) {
          const uint32_t t = ~y[w];
          y[w] = t + c;
          c = (y[w] < t) ? 1u : 0u;
        }
        top = c;
      }
    }
  }
  return top;
}

// Inner cell idx of the chunk: side (0: a, 1: b), product i, piece t. Piece t of the outer value
// is the M-bit slice at bit M t, times theta^t = 2^{t Ni / K'}: with the shift s = t Ni / K',
// lo = (slice << s) mod 2^{Ni}, hi = slice >> (Ni - s), value lo - hi (+ p' when negative). An
// outer value 2^N (= -1) gives zero pieces; combine handles its product.
__global__ void rec_split_kernel(const uint64_t *__restrict__ a, const uint64_t *__restrict__ b, int64_t stride,
                                 int64_t count, int N, int M, int Ni, int k, uint64_t *__restrict__ X,
                                 int64_t stride_i) {
  const int64_t Ki = int64_t(1) << k, per_side = count * Ki;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= 2 * per_side) return;
  const int side = idx >= per_side ? 1 : 0;
  const int64_t rem = idx - side * per_side, i = rem >> k;
  const int t = int(rem & (Ki - 1));
  const uint32_t *src = reinterpret_cast<const uint32_t *>((side ? b : a) + i * stride);
  uint32_t *dst = reinterpret_cast<uint32_t *>(X + idx * stride_i);
  const int NW = N / 32, nwi = Ni / 32, MW = M / 32;
  if (src[NW] & 1u) {
    for (int w = 0; w < nwi + 2; w++) dst[w] = 0u;
    return;
  }
  const uint32_t *p = src + int64_t(t) * MW;
  const int s = t * (Ni >> k), q = s >> 5, r = s & 31;
  auto P = [&](int u) -> uint32_t { return (u >= 0 && u < MW) ? p[u] : 0u; };
  auto shifted = [&](int w) -> uint32_t {  // word w of slice << s
    const int u = w - q;
    return r ? __funnelshift_l(P(u - 1), P(u), r) : P(u);
  };
  uint32_t borrow = 0;
  for (int w = 0; w < nwi; w++) {
    const uint64_t d = uint64_t(shifted(w)) - shifted(nwi + w) - borrow;
    dst[w] = uint32_t(d);
    borrow = uint32_t(d >> 63);
  }
  uint32_t top = 0;
  if (borrow) {
    uint32_t c = 1u;
    for (int w = 0; w < nwi && c; w++) {
      const uint32_t v = dst[w] + 1u;
      dst[w] = v;
      c = v == 0u;
    }
    top = c;
  }
  dst[nwi] = top;
  dst[nwi + 1] = 0u;
}

// Inner cell (i, t) of the a side after the inverse transform holds theta^t c_t: multiply by
// theta^{-t} = 2^{2 Ni - t Ni / K'} and add B = 2^{k + 2M}, giving c_t + B in [0, 2B), 2B <= 2^{Ni}.
__global__ void rec_final_kernel(uint64_t *__restrict__ X, int64_t count, int Ni, int k, int M, int64_t stride_i) {
  const int64_t Ki = int64_t(1) << k;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= count * Ki) return;
  const int t = int(idx & (Ki - 1));
  uint32_t *cell = reinterpret_cast<uint32_t *>(X + idx * stride_i);
  const int nwi = Ni / 32;
  uint32_t x[kRecMaxInnerWords], y[kRecMaxInnerWords];
  for (int w = 0; w < nwi; w++) x[w] = cell[w];
  const uint32_t xtop = cell[nwi] & 1u;
  int E = 2 * Ni - t * (Ni >> k);
  if (E >= 2 * Ni) E -= 2 * Ni;
  uint32_t top = small_mul2exp(y, x, xtop, E, nwi);
  // + B; the sum stays below p' for a legitimate c_t, else reduce by p' = 2^{Ni} + 1
  const int bb = k + 2 * M;
  uint32_t c = 1u << (bb & 31);
  for (int w = bb >> 5; w < nwi && c; w++) {
    const uint32_t v = y[w] + c;
    c = v < c ? 1u : 0u;
    y[w] = v;
  }
  top += c;
  if (top) {
    // value 2^{Ni} + rest >= p': subtract p', i.e. drop 2^{Ni} and subtract 1
    uint32_t bo = 1u;
    for (int w = 0; w < nwi && bo; w++) {
      const uint32_t v = y[w];
      y[w] = v - 1u;
      bo = v == 0u;
    }
    top = top - 1u - bo;
  }
  for (int w = 0; w < nwi; w++) cell[w] = y[w];
  cell[nwi] = top;
  cell[nwi + 1] = 0u;
}

// add the piece words into this lane's chunk [w0, w0 + K) (piece word u sits at word o + u, u <
// nwp) with one carry chain; returns the carry out of the chunk
template <int K>
__device__ __forceinline__ uint32_t add_piece(uint32_t (&acc)[K], const uint32_t *piece, int o, int nwp, int w0) {
  uint32_t pw[K];
#pragma unroll
  for (int s = 0; s < K; s++) {
    const int u = w0 + s - o;
    pw[s] = (u >= 0 && u < nwp) ? piece[u] : 0u;
  }
  return add_chain<K>(acc, acc, pw, 0u);
}

// carries c (small counts, one per lane) out of each lane's chunk moved up through the lanes;
// returns the total carried out of the top lane (bit N)
template <int K>
__device__ __forceinline__ int settle_counts(uint32_t (&acc)[K], uint32_t c, const Geo &g) {
  int out = 0;
  for (int round = 0; round < 64 && __any_sync(TFT_FULL, c != 0u); round++) {
    out += int(__shfl_sync(TFT_FULL, c, g.G - 1));
    uint32_t cin = __shfl_up_sync(TFT_FULL, c, 1);
    if (g.lane == 0 || g.lane >= g.G) cin = 0u;
    c = ripple_add<K>(acc, cin);
    if (g.lane >= g.G) c = 0u;
  }
  return out;
}

// One product per warp: S' = sum_t (c_t + B) 2^{M t} = acc + 2^N ovr (acc: bits below N, ovr:
// bits from N up), the bias B sum_t 2^{M t} = sum_t 2^{P_t} with P_t = M t + 2M + k is Cpos -
// Cn mod 2^N + 1 (Cpos: the P_t < N, Cn: 2^{P_t - N} for the others), so
// a b = (acc + Cn) - (ovr + Cpos) mod 2^N + 1.
template <int K>
__global__ void __launch_bounds__(128) rec_combine_kernel(uint64_t *__restrict__ a, const uint64_t *__restrict__ b,
                                                          int64_t stride, const uint64_t *__restrict__ X,
                                                          int64_t stride_i, int64_t count, int N, int M, int k,
                                                          int nwp) {
  Geo g;
  g.N = N;
  g.NW = N / 32;
  g.G = g.NW / K;
  g.lane = threadIdx.x & 31;
  g.twoN = 2 * N;
  const int NW = g.NW, MW = M / 32, Ki = 1 << k, wi2 = int(2 * stride_i);
  const int w0 = K * g.lane;
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < count; i += nwarps) {
    uint64_t *ac = a + i * stride;
    const uint64_t *bc = b + i * stride;
    const uint32_t Ta = reinterpret_cast<const uint32_t *>(ac)[NW] & 1u;
    const uint32_t Tb = reinterpret_cast<const uint32_t *>(bc)[NW] & 1u;
    uint32_t r[K];
    uint32_t top = 0;
    if (Ta | Tb) {
      // 2^N = -1: the product is 1, -b or -a
#pragma unroll
      for (int s = 0; s < K; s++) r[s] = 0u;
      if (Ta & Tb) {
        if (g.lane == 0) r[0] = 1u;
      } else {
        uint32_t o[K], zero[K];
        gmem_load_x<K>(o, Ta ? bc : ac, g);
#pragma unroll
        for (int s = 0; s < K; s++) zero[s] = 0u;
        const uint32_t bo = g.lane < g.G ? sub_chain<K>(r, zero, o, 0u) : 0u;
        const uint32_t T = resolve_sub<K>(r, bo, g);
        top = canon_x<K>(r, int(T), g);
      }
    } else {
      uint32_t acc[K], ovr[K];
#pragma unroll
      for (int s = 0; s < K; s++) acc[s] = ovr[s] = 0u;
      uint32_t pa = 0, po = 0;
      const uint32_t *Xi = reinterpret_cast<const uint32_t *>(X + i * int64_t(Ki) * stride_i);
      if (g.lane < g.G) {
        // pieces overlapping words [w0, w0 + K) of acc and [NW + w0, NW + w0 + K) of the sum
        int tlo = (w0 - nwp + 1 + MW - 1) / MW;
        if (w0 - nwp + 1 <= 0) tlo = 0;
        const int thi = min(Ki - 1, (w0 + K - 1) / MW);
        for (int t = tlo; t <= thi; t++) pa += add_piece<K>(acc, Xi + t * wi2, t * MW, nwp, w0);
        int ulo = (NW + w0 - nwp + 1 + MW - 1) / MW;
        if (NW + w0 - nwp + 1 <= 0) ulo = 0;
        const int uhi = min(Ki - 1, (NW + w0 + K - 1) / MW);
        for (int t = ulo; t <= uhi; t++) po += add_piece<K>(ovr, Xi + t * wi2, t * MW - NW, nwp, w0);
        // the bias bits: bit k of word t MW + 2 MW (into ovr when below N, else of word - NW into acc)
        uint32_t cp[K], cn[K];
#pragma unroll
        for (int s = 0; s < K; s++) {
          const int w = w0 + s;
          const int dp = w - 2 * MW, dn = w + NW - 2 * MW;
          cp[s] = (dp >= 0 && dp % MW == 0 && dp / MW < Ki) ? (1u << k) : 0u;
          cn[s] = (dn >= 0 && dn % MW == 0 && dn / MW < Ki) ? (1u << k) : 0u;
        }
        po += add_chain<K>(ovr, ovr, cp, 0u);
        pa += add_chain<K>(acc, acc, cn, 0u);
      }
      int v = -settle_counts<K>(acc, pa, g);  // carries out of bit N of acc: 2^N = -1
      v += settle_counts<K>(ovr, po, g);      // ovr is subtracted
      const uint32_t bo = g.lane < g.G ? sub_chain<K>(r, acc, ovr, 0u) : 0u;
      if (g.lane >= g.G) {
#pragma unroll
        for (int s = 0; s < K; s++) r[s] = 0u;
      }
      v += int(resolve_sub<K>(r, bo, g));  // r - T 2^N = r + T
      top = canon_x<K>(r, v, g);
    }
    gmem_store_x<K>(ac, r, top, g);
  }
}

}  // namespace

bool rec_plan_for(int64_t N, int k, RecPlan *out) {
  // k >= 2 keeps a piece's 2M + k + 1 bits below N, so the part of a piece past bit N is short
  if (k < 2 || k > 12 || !ring_supported(N)) return false;
  const int64_t Ki = int64_t(1) << k;
  if (N % (32 * Ki) != 0) return false;  // pieces of whole 32-bit words
  const int64_t M = N / Ki, need = 2 * M + k + 1;
  int64_t Ni = 0;
  for (int64_t c = 64; c <= 32 * kRecMaxInnerWords; c += 64) {
    if (c >= need && c % Ki == 0 && ring_supported(c)) {
      Ni = c;
      break;
    }
  }
  if (!Ni) return false;
  RecPlan p;
  p.N = N;
  p.k = k;
  p.M = M;
  p.Ni = Ni;
  p.nwp = int((need + 31) / 32);
  const Ring ri = make_ring(Ni);
  p.stride_i = (Ni / 64 + 1 + 1) & ~int64_t(1);
  // work estimate: inner products (NW'^2 word products each) and three transforms (about
  // 2k word operations per cell and level pair), per outer product
  p.cost = double(Ki) * (double(ri.NW) * ri.NW + 6.0 * k * ri.NW);
  *out = p;
  return true;
}

bool rec_plan_auto(int64_t N, RecPlan *out) {
  bool any = false;
  RecPlan best;
  for (int k = 2; k <= 12; k++) {
    RecPlan p;
    if (rec_plan_for(N, k, &p) && (!any || p.cost < best.cost)) {
      best = p;
      any = true;
    }
  }
  if (any) *out = best;
  return any;
}

cudaError_t run_rec_pointwise(uint64_t *a, const uint64_t *b, int64_t n, int64_t stride, const Ring &ro,
                              const RecPlan &rp, cudaStream_t s, int *err) {
  *err = ZX_OK;
  if (n <= 0) return cudaSuccess;
  const Ring ri = make_ring(rp.Ni);
  const int64_t Ki = int64_t(1) << rp.k;
  const TransformPlan *pt = get_transform_plan(KIND_TFT, rp.k, Ki, Ki, 0, rp.Ni, 0, rp.stride_i, 0, err, RING_FERMAT, true);
  const TransformPlan *pi =
      pt ? get_transform_plan(KIND_ITFT, rp.k, Ki, Ki, 0, rp.Ni, 0, rp.stride_i, 1, err, RING_FERMAT, true) : nullptr;
  if (!pi) {
    if (*err == ZX_OK) *err = ZX_ECUDA;
    return cudaErrorInvalidValue;
  }
  const size_t cell_bytes = size_t(rp.stride_i) * 8;
  const size_t budget = size_t(256) << 20;
  int64_t chunk = int64_t(budget / (2 * size_t(Ki) * cell_bytes));
  chunk = std::max<int64_t>(1, std::min<int64_t>(chunk, n));
  uint64_t *X = nullptr;
  cudaError_t ce = cudaMallocAsync(reinterpret_cast<void **>(&X), size_t(2 * chunk * Ki) * cell_bytes, s);
  if (ce != cudaSuccess) {
    *err = ZX_ENOMEM;
    return ce;
  }
  for (int64_t off = 0; off < n && ce == cudaSuccess; off += chunk) {
    const int64_t c = std::min(chunk, n - off);
    uint64_t *ca = a + off * stride;
    const uint64_t *cb = b + off * stride;
    const int64_t cells = 2 * c * Ki;
    rec_split_kernel<<<unsigned((cells + 255) / 256), 256, 0, s>>>(ca, cb, stride, c, int(ro.N), int(rp.M), int(rp.Ni),
                                                                   rp.k, X, rp.stride_i);
    if ((ce = cudaGetLastError()) != cudaSuccess) break;
    if ((ce = run_transform_reps(*pt, X, rp.stride_i, 2 * c, Ki, s)) != cudaSuccess) break;
    if ((ce = launch_pointwise(X, X + c * Ki * rp.stride_i, c * Ki, rp.stride_i, ri, s)) != cudaSuccess) break;
    if ((ce = run_transform_reps(*pi, X, rp.stride_i, c, Ki, s)) != cudaSuccess) break;
    rec_final_kernel<<<unsigned((c * Ki + 127) / 128), 128, 0, s>>>(X, c, int(rp.Ni), rp.k, int(rp.M), rp.stride_i);
    if ((ce = cudaGetLastError()) != cudaSuccess) break;
    const int blocks = int(std::min<int64_t>((c + 3) / 4, 152 * 16));
#define TFT_RC(KK)                                                                                        \
  rec_combine_kernel<KK><<<blocks, 128, 0, s>>>(ca, cb, stride, X, rp.stride_i, c, int(ro.N), int(rp.M), \
                                                rp.k, rp.nwp)
    switch (ro.K) {
      case 1: TFT_RC(1); break;
      case 2: TFT_RC(2); break;
      case 4: TFT_RC(4); break;
      case 8: TFT_RC(8); break;
      case 16: TFT_RC(16); break;
      case 32: TFT_RC(32); break;
      default: ce = cudaErrorInvalidValue;
    }
#undef TFT_RC
    if (ce == cudaSuccess) ce = cudaGetLastError();
  }
  const cudaError_t fe = cudaFreeAsync(X, s);
  if (ce == cudaSuccess) ce = fe;
  if (ce != cudaSuccess && *err == ZX_OK) *err = ZX_ECUDA;
  return ce;
}

}  // namespace tftgpu
