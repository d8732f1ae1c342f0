// Kernels of the Schoenhage-Strassen product in Z[x] (Sec. 5.1) around the transforms:
//   pack      coefficient in Z -> residue in [0, 2^N] (negatives become 2^N + 1 - |c|)
//   pointwise n products in R = Z/(2^N+1) (the n pointwise multiplications of Sec. 2)
//   lift      residue -> coefficient in Z (residues above 2^{N-1} are negative when signed)
// One warp handles one ring element in the lane-chunked layout of ring_warp.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "common.h"
#include "host.h"
#include "ring_warp.cuh"

namespace tftgpu {

namespace {

__device__ __forceinline__ Geo make_geo(int N, int K) {
  Geo g;
  g.N = N;
  g.NW = N / 32;
  g.G = g.NW / K;
  g.lane = threadIdx.x & 31;
  g.twoN = 2 * N;
  return g;
}

template <int K>
__device__ __forceinline__ void pack_one(const uint64_t *coef, int64_t limbs, int sgn, uint64_t *cell,
                                         const Geo &g) {
  const uint32_t *c32 = reinterpret_cast<const uint32_t *>(coef);
  const int64_t cw = 2 * limbs;
  const bool neg = sgn && (c32[cw - 1] >> 31);
  const uint32_t fill = neg ? 0xffffffffu : 0u;
  uint32_t r[K];
#pragma unroll
  for (int s = 0; s < K; s++) {
    int64_t w = int64_t(K) * g.lane + s;
    r[s] = (g.lane < g.G) ? (w < cw ? c32[w] : fill) : 0u;
  }
  // negative c: residue = (c mod 2^N) + 1, i.e. c + 2^N + 1
  uint32_t top = neg ? add_small<K>(r, 1u, g) : 0u;
  gmem_store_x<K>(cell, r, top, g);
}

template <int K>
__global__ void pack_kernel(const uint64_t *__restrict__ coef, int64_t len, int64_t limbs, int sgn,
                            uint64_t *__restrict__ cells, int64_t stride, int N) {
  grid_dependency_enter();
  const Geo g = make_geo(N, K);
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < len; i += nwarps)
    pack_one<K>(coef + i * limbs, limbs, sgn, cells + i * stride, g);
}

template <int K>
__global__ void pack_batch_kernel(const PackItem *__restrict__ items, int64_t stride, int N,
                                  uint64_t *__restrict__ pool) {
  grid_dependency_enter();
  const Geo g = make_geo(N, K);
  const PackItem it = items[blockIdx.y];
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < it.len; i += nwarps)
    pack_one<K>(it.coef + i * it.limbs, it.limbs, it.is_signed, pool + it.cells + i * stride, g);
}

template <int K>
__device__ __forceinline__ void lift_one(const uint64_t *cell, int sgn, uint64_t *out, int64_t limbs_out,
                                         const Geo &g) {
  uint32_t r[K];
  uint32_t T = gmem_load_x<K>(r, cell, g);
  bool negative = false;
  if (sgn) {
    // x > 2^{N-1}: x = 2^N, or bit N-1 set and some other bit set
    uint32_t hb = 0, other = 0;
#pragma unroll
    for (int s = 0; s < K; s++) {
      int w = K * g.lane + s;
      if (w == g.NW - 1 && g.lane < g.G) {
        hb = r[s] >> 31;
        other |= r[s] & 0x7fffffffu;
      } else {
        other |= r[s];
      }
    }
    bool any_hb = __any_sync(TFT_FULL, hb != 0), any_other = __any_sync(TFT_FULL, other != 0);
    negative = T != 0 || (any_hb && any_other);
  }
  uint32_t fill = 0u;
  if (negative) {
    // x - (2^N + 1) = (x - 1) - 2^N: the N-bit value x - 1, ones above bit N
    sub_small<K>(r, 1u, g);
    fill = 0xffffffffu;
  } else {
    fill = 0u;
  }
  uint32_t *o32 = reinterpret_cast<uint32_t *>(out);
  const int64_t ow = 2 * limbs_out;
  if (g.lane < g.G) {
#pragma unroll
    for (int s = 0; s < K; s++) {
      int64_t w = int64_t(K) * g.lane + s;
      if (w < ow) o32[w] = r[s];
    }
  }
  // words from bit N upward: the top bit of an unsigned 2^N, or the sign fill
  for (int64_t w = g.NW + g.lane; w < ow; w += 32) {
    uint32_t v = fill;
    if (!negative && w == g.NW) v = T;
    o32[w] = v;
  }
}

template <int K>
__global__ void lift_kernel(const uint64_t *__restrict__ cells, int64_t n, int64_t stride, int sgn,
                            uint64_t *__restrict__ out, int64_t limbs_out, int N) {
  grid_dependency_enter();
  const Geo g = make_geo(N, K);
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nwarps)
    lift_one<K>(cells + i * stride, sgn, out + i * limbs_out, limbs_out, g);
}

template <int K>
__global__ void lift_batch_kernel(const LiftItem *__restrict__ items, int64_t stride, int N,
                                  const uint64_t *__restrict__ pool) {
  grid_dependency_enter();
  const Geo g = make_geo(N, K);
  const LiftItem it = items[blockIdx.y];
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < it.n; i += nwarps)
    lift_one<K>(pool + it.cells + i * stride, it.is_signed, it.out + i * it.limbs_out, it.limbs_out, g);
}

// One multiply-accumulate of column sums: (c2:c1:c0) += a * w (96-bit column accumulator).
__device__ __forceinline__ void mac96(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t a, uint32_t w) {
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
      "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
      "addc.u32 %2, %2, 0;"
      : "+r"(c0), "+r"(c1), "+r"(c2)
      : "r"(a), "r"(w));
}

// out word w = in word w - D (zero below D) of a lane-chunked number, D = 1 or 2; the words
// shifted past the top are dropped
template <int K, int D>
__device__ __forceinline__ void shift_words_up(uint32_t (&out)[K], const uint32_t (&in)[K], const Geo &g) {
  const bool act = g.lane < g.G;
  if (K >= D) {
    uint32_t from[D];
#pragma unroll
    for (int d = 0; d < D; d++) {
      from[d] = __shfl_up_sync(TFT_FULL, in[K - D + d], 1);
      if (g.lane == 0) from[d] = 0u;
    }
#pragma unroll
    for (int q = K - 1; q >= D; q--) out[q] = in[q - D];
#pragma unroll
    for (int d = 0; d < D; d++) out[d] = act ? from[d] : 0u;
  } else {  // K = 1, D = 2
    uint32_t v = __shfl_up_sync(TFT_FULL, in[0], 2);
    out[0] = (act && g.lane >= 2) ? v : 0u;
  }
}

// a <- a * b mod 2^N + 1 for one product (one warp), by product scanning with a negacyclic fold:
// lane l owns the K column sums p = K l + q of
//   X = sum_{i+j=p} A_i B_j - sum_{i+j=p+NW} A_i B_j    (2^{32 NW} = 2^N = -1),
// each a 96-bit accumulator. B sits in registers as a window that turns by one word per step
// i (window word at column p = B_{(p - i) mod NW}); A_i is a broadcast shared-memory read. A
// word that wraps from the top column to column 0 enters complemented (~w = 2^32 - 1 - w), which
// turns the subtraction into a multiply-add; the surplus (2^32 - 1) A_i per wrapped word adds up
// to (2^32 - 1) SA_p per column, SA_p = sum_{i > p} A_i, and is taken off at the end.
// `As` is this warp's NW words of shared memory.
template <int K>
__device__ __forceinline__ void pointwise_one(uint64_t *acell, const uint64_t *bcell, uint32_t *As,
                                              const Geo &g) {
  constexpr int U = K < 4 ? K : 4;  // steps per unrolled block
  const int NW = g.NW;
  const uint32_t *a32 = reinterpret_cast<const uint32_t *>(acell);
  const uint32_t Ta = __ldg(a32 + NW) & 1u;
  uint32_t win[K + U];
  uint32_t rb[K];
  const uint32_t Tb = gmem_load_x<K>(rb, bcell, g) & 1u;
  // 2^N = -1: use magnitude 1 and remember the sign
  const uint32_t neg = Ta ^ Tb;
  for (int w = g.lane; w < NW; w += 32) As[w] = Ta ? (w == 0 ? 1u : 0u) : __ldg(a32 + w);
  if (Tb) {
#pragma unroll
    for (int q = 0; q < K; q++) rb[q] = 0u;
    if (g.lane == 0) rb[0] = 1u;
  }
#pragma unroll
  for (int q = 0; q < K; q++) win[U + q] = rb[q];
  __syncwarp();

  uint32_t c0[K], c1[K], c2[K];
#pragma unroll
  for (int q = 0; q < K; q++) c0[q] = c1[q] = c2[q] = 0u;
  const int src = g.lane >= g.G ? g.lane : (g.lane == 0 ? g.G - 1 : g.lane - 1);
  for (int i0 = 0; i0 < NW; i0 += U) {
    uint32_t a[U];
    if (U == 4) {
      const uint4 v = *reinterpret_cast<const uint4 *>(As + i0);
      a[0] = v.x;
      a[1 % U] = v.y;
      a[2 % U] = v.z;
      a[3 % U] = v.w;
    } else {
#pragma unroll
      for (int s = 0; s < U; s++) a[s] = As[i0 + s];
    }
#pragma unroll
    for (int s = 0; s < U; s++) {
#pragma unroll
      for (int q = 0; q < K; q++) mac96(c0[q], c1[q], c2[q], a[s], win[U - s + q]);
      const uint32_t x = __shfl_sync(TFT_FULL, win[U - s + K - 1], src);
      win[U - s - 1] = g.lane == 0 ? ~x : x;
    }
#pragma unroll
    for (int q = K - 1; q >= 0; q--) win[U + q] = win[q];
  }

  // SA_p = sum_{i > p} A_i for this lane's columns (below 2^42: two words sa0, sa1)
  uint32_t sa0[K], sa1[K];
  {
    uint64_t own = 0;
    if (g.lane < g.G) {
#pragma unroll
      for (int q = 0; q < K; q++) own += As[K * g.lane + q];
    }
    uint64_t above = own;  // inclusive suffix over lanes
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t t = __shfl_down_sync(TFT_FULL, above, d);
      if (g.lane + d < 32) above += t;
    }
    uint64_t run = above - own;  // lanes above this one
#pragma unroll
    for (int q = K - 1; q >= 0; q--) {
      const bool act = g.lane < g.G;
      sa0[q] = act ? uint32_t(run) : 0u;
      sa1[q] = act ? uint32_t(run >> 32) : 0u;
      if (act) run += As[K * g.lane + q];
    }
  }
  // the words past the top that wrap (negated): c1 of column NW-1, c2 of columns NW-2, NW-1
  const uint32_t h_c1 = __shfl_sync(TFT_FULL, c1[K - 1], g.G - 1);
  const uint32_t h_c2b = __shfl_sync(TFT_FULL, c2[K - 1], g.G - 1);
  uint32_t h_c2a;
  if (K >= 2)
    h_c2a = __shfl_sync(TFT_FULL, c2[K >= 2 ? K - 2 : 0], g.G - 1);
  else
    h_c2a = __shfl_sync(TFT_FULL, c2[0], g.G - 2);

  // X = V0 + V1 + V2 + Qa + Qb - Qc - Qd - H, with V0 = c0, V1 = c1 one word up, V2 = c2 two
  // words up, Qa = sa0, Qb = sa1 one word up (= SA), Qc = sa0 one word up, Qd = sa1 two words
  // up (= SA 2^32), H = the wrapped words
  uint32_t R[K], t[K];
  int v = 0;
  shift_words_up<K, 1>(t, c1, g);
  v -= int(resolve_add<K>(R, add_chain<K>(R, c0, t, 0u), g));
  shift_words_up<K, 2>(t, c2, g);
  v -= int(resolve_add<K>(R, add_chain<K>(R, R, t, 0u), g));
  v -= int(resolve_add<K>(R, add_chain<K>(R, R, sa0, 0u), g));
  shift_words_up<K, 1>(t, sa1, g);
  v -= int(resolve_add<K>(R, add_chain<K>(R, R, t, 0u), g));
  shift_words_up<K, 1>(t, sa0, g);
  v += int(resolve_sub<K>(R, sub_chain<K>(R, R, t, 0u), g));
  shift_words_up<K, 2>(t, sa1, g);
  v += int(resolve_sub<K>(R, sub_chain<K>(R, R, t, 0u), g));
  {
    const uint64_t h0 = uint64_t(h_c1) + h_c2a;
    const uint32_t hw0 = uint32_t(h0), hw1 = uint32_t(h0 >> 32) + h_c2b;
#pragma unroll
    for (int q = 0; q < K; q++) {
      const int w = K * g.lane + q;
      t[q] = w == 0 ? hw0 : (w == 1 ? hw1 : 0u);
    }
  }
  v += int(resolve_sub<K>(R, sub_chain<K>(R, R, t, 0u), g));
  uint32_t T = canon_x<K>(R, v, g);
  if (neg) {
    // -x: 2^N -> 1, 0 -> 0, else ~x + 2 (N bits)
    if (T) {
#pragma unroll
      for (int q = 0; q < K; q++) R[q] = 0u;
      if (g.lane == 0) R[0] = 1u;
      T = 0u;
    } else if (!is_zero<K>(R)) {
#pragma unroll
      for (int q = 0; q < K; q++) R[q] = g.lane < g.G ? ~R[q] : 0u;
      T = add_small<K>(R, 2u, g);
    }
  }
  __syncwarp();
  gmem_store_x<K>(acell, R, T, g);
  __syncwarp();
}

// Launch with programmatic dependent launch (every kernel of this file calls grid_dependency_enter
// first), so that the launches of a product's chain (pack, transforms, pointwise, lift) start
// their CTAs as the previous launch's last wave finishes.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute a[1];
  a[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  a[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = a;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

constexpr int kPointwiseWarps = 4;

__host__ __device__ constexpr int pointwise_warp_words(int NW) { return (NW + 3) & ~3; }

template <int K>
__global__ void __launch_bounds__(kPointwiseWarps * 32)
    pointwise_kernel(uint64_t *__restrict__ a, const uint64_t *__restrict__ b, int64_t n, int64_t stride, int N,
                     int warps_per_block) {
  grid_dependency_enter();
  extern __shared__ uint4 sm4[];
  uint32_t *sm = reinterpret_cast<uint32_t *>(sm4);
  const Geo g = make_geo(N, K);
  const int warp = threadIdx.x >> 5;
  uint32_t *ws = sm + size_t(warp) * pointwise_warp_words(g.NW);
  const int64_t nwarps = int64_t(gridDim.x) * warps_per_block;
  for (int64_t i = int64_t(blockIdx.x) * warps_per_block + warp; i < n; i += nwarps)
    pointwise_one<K>(a + i * stride, b + i * stride, ws, g);
}

// The pointwise products of a batch group as one sequence of `total` products (item p holds
// products first .. first + n - 1 of it): warps take them in a grid-stride loop, so a group's
// longest product is spread over the whole grid instead of a per-item share of it. A warp's index
// only grows, so its item cursor only moves forward.
template <int K>
__global__ void __launch_bounds__(kPointwiseWarps * 32)
    pointwise_batch_kernel(const PointwiseItem *__restrict__ items, int count, int64_t total, int64_t stride, int N,
                           int warps_per_block, uint64_t *__restrict__ pool) {
  grid_dependency_enter();
  extern __shared__ uint4 sm4[];
  uint32_t *sm = reinterpret_cast<uint32_t *>(sm4);
  const Geo g = make_geo(N, K);
  const int warp = threadIdx.x >> 5;
  uint32_t *ws = sm + size_t(warp) * pointwise_warp_words(g.NW);
  const int64_t nwarps = int64_t(gridDim.x) * warps_per_block;
  int p = 0;
  for (int64_t t = int64_t(blockIdx.x) * warps_per_block + warp; t < total; t += nwarps) {
    while (p + 1 < count && items[p + 1].first <= t) p++;
    const int64_t i = t - items[p].first;
    pointwise_one<K>(pool + items[p].a + i * stride, pool + items[p].b + i * stride, ws, g);
  }
}

template <int K>
cudaError_t pointwise_k(uint64_t *a, const uint64_t *b, int64_t n, int64_t stride, const Ring &r,
                        cudaStream_t s) {
  const int wpb = kPointwiseWarps;
  const size_t smem = size_t(pointwise_warp_words(r.NW)) * 4 * wpb;
  int64_t blocks = (n + wpb - 1) / wpb;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  return launch_pdl(pointwise_kernel<K>, dim3(unsigned(blocks)), dim3(unsigned(wpb * 32)), smem, s, a, b, n, stride,
                    int(r.N), wpb);
}

int grid_for(int64_t items, int warps_per_block) {
  int64_t b = (items + warps_per_block - 1) / warps_per_block;
  if (b > 152 * 32) b = 152 * 32;
  return int(b < 1 ? 1 : b);
}

}  // namespace

#define TFT_DISPATCH_K(K_, CALL)                 \
  switch (K_) {                                  \
    case 1: { constexpr int KK = 1; CALL; } break;  \
    case 2: { constexpr int KK = 2; CALL; } break;  \
    case 4: { constexpr int KK = 4; CALL; } break;  \
    case 8: { constexpr int KK = 8; CALL; } break;  \
    case 16: { constexpr int KK = 16; CALL; } break; \
    case 32: { constexpr int KK = 32; CALL; } break; \
    default: return cudaErrorInvalidValue;       \
  }

cudaError_t launch_pack(const uint64_t *coef, int64_t len, int64_t limbs, int is_signed, uint64_t *cells,
                        int64_t stride_limbs, const Ring &r, cudaStream_t s) {
  if (len <= 0) return cudaSuccess;
  const dim3 grid(unsigned(grid_for(len, 8)));
  TFT_DISPATCH_K(r.K, return launch_pdl(pack_kernel<KK>, grid, dim3(256), 0, s, coef, len, limbs, is_signed, cells,
                                        stride_limbs, int(r.N)));
  return cudaSuccess;
}

cudaError_t launch_lift(const uint64_t *cells, int64_t n, int64_t stride_limbs, int is_signed, uint64_t *out,
                        int64_t limbs_out, const Ring &r, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const dim3 grid(unsigned(grid_for(n, 8)));
  TFT_DISPATCH_K(r.K, return launch_pdl(lift_kernel<KK>, grid, dim3(256), 0, s, cells, n, stride_limbs, is_signed, out,
                                        limbs_out, int(r.N)));
  return cudaSuccess;
}

template <int K>
cudaError_t pointwise_batch_k(const PointwiseItem *items, int count, int64_t total, int64_t stride,
                              const Ring &r, uint64_t *pool, cudaStream_t s) {
  const int wpb = kPointwiseWarps;
  const size_t smem = size_t(pointwise_warp_words(r.NW)) * 4 * wpb;
  int64_t blocks = (total + wpb - 1) / wpb;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  return launch_pdl(pointwise_batch_kernel<K>, dim3(unsigned(blocks)), dim3(unsigned(wpb * 32)), smem, s, items, count,
                    total, stride, int(r.N), wpb, pool);
}

int grid_x_for(int64_t max_items, int count, int warps_per_block) {
  int64_t b = (max_items + warps_per_block - 1) / warps_per_block;
  int64_t cap = std::max<int64_t>(1, (152 * 32) / std::max(1, count));
  if (b > cap) b = cap;
  return int(b < 1 ? 1 : b);
}

cudaError_t launch_pack_batch(const PackItem *d_items, int count, int64_t max_len, int64_t stride_limbs,
                              const Ring &r, uint64_t *pool, cudaStream_t s) {
  if (count <= 0 || max_len <= 0) return cudaSuccess;
  const dim3 grid(unsigned(grid_x_for(max_len, count, 8)), unsigned(count));
  TFT_DISPATCH_K(r.K, return launch_pdl(pack_batch_kernel<KK>, grid, dim3(256), 0, s, d_items, stride_limbs, int(r.N),
                                        pool));
  return cudaSuccess;
}

cudaError_t launch_lift_batch(const LiftItem *d_items, int count, int64_t max_n, int64_t stride_limbs,
                              const Ring &r, uint64_t *pool, cudaStream_t s) {
  if (count <= 0 || max_n <= 0) return cudaSuccess;
  const dim3 grid(unsigned(grid_x_for(max_n, count, 8)), unsigned(count));
  TFT_DISPATCH_K(r.K, return launch_pdl(lift_batch_kernel<KK>, grid, dim3(256), 0, s, d_items, stride_limbs, int(r.N),
                                        pool));
  return cudaSuccess;
}

cudaError_t launch_pointwise_batch(const PointwiseItem *d_items, int count, int64_t total, int64_t stride_limbs,
                                   const Ring &r, uint64_t *pool, cudaStream_t s) {
  if (count <= 0 || total <= 0) return cudaSuccess;
  TFT_DISPATCH_K(r.K, return pointwise_batch_k<KK>(d_items, count, total, stride_limbs, r, pool, s));
  return cudaSuccess;
}

cudaError_t launch_pointwise(uint64_t *a, const uint64_t *b, int64_t n, int64_t stride_limbs, const Ring &r,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  TFT_DISPATCH_K(r.K, return pointwise_k<KK>(a, b, n, stride_limbs, r, s));
  return cudaSuccess;
}

}  // namespace tftgpu
