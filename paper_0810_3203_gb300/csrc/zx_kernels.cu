// Kernels of the Schoenhage-Strassen product in Z[x] (Sec. 5.1) around the transforms:
//   pack      coefficient in Z -> residue in [0, 2^N] (negatives become 2^N + 1 - |c|)
//   pointwise n products in R = Z/(2^N+1) (the n pointwise multiplications of Sec. 2)
//   lift      residue -> coefficient in Z (residues above 2^{N-1} are negative when signed)
// One warp handles one ring element in the lane-chunked layout of ring_warp.cuh.
#include <cuda_runtime.h>

#include <algorithm>

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
  const Geo g = make_geo(N, K);
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < len; i += nwarps)
    pack_one<K>(coef + i * limbs, limbs, sgn, cells + i * stride, g);
}

template <int K>
__global__ void pack_batch_kernel(const PackItem *__restrict__ items, int64_t stride, int N,
                                  uint64_t *__restrict__ pool) {
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
  const Geo g = make_geo(N, K);
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nwarps)
    lift_one<K>(cells + i * stride, sgn, out + i * limbs_out, limbs_out, g);
}

template <int K>
__global__ void lift_batch_kernel(const LiftItem *__restrict__ items, int64_t stride, int N,
                                  const uint64_t *__restrict__ pool) {
  const Geo g = make_geo(N, K);
  const LiftItem it = items[blockIdx.y];
  const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < it.n; i += nwarps)
    lift_one<K>(pool + it.cells + i * stride, it.is_signed, it.out + i * it.limbs_out, it.limbs_out, g);
}

// a <- a * b mod 2^N + 1 for one product, by a schoolbook column product and the reduction
// P = P_lo + P_hi 2^N = P_lo - P_hi. `ws` is this warp's shared-memory scratch of 8 NW + 8 words.
template <int K>
__device__ __forceinline__ void pointwise_one(uint64_t *acell, const uint64_t *bcell, uint32_t *ws,
                                              const Geo &g) {
  const int NW = g.NW;
  uint32_t *A = ws;
  uint32_t *B = A + NW;
  uint32_t *C0 = B + NW;       // column sums, low words (2NW)
  uint32_t *C1 = C0 + 2 * NW;  // middle words
  uint32_t *C2 = C1 + 2 * NW;  // high words
  uint32_t ra[K], rb[K];
  uint32_t Ta = gmem_load_x<K>(ra, acell, g);
  uint32_t Tb = gmem_load_x<K>(rb, bcell, g);
  // 2^N = -1: use magnitude 1 and remember the sign
  const uint32_t neg = (Ta ^ Tb) & 1u;
  if (Ta) {
#pragma unroll
    for (int s = 0; s < K; s++) ra[s] = 0u;
    if (g.lane == 0) ra[0] = 1u;
  }
  if (Tb) {
#pragma unroll
    for (int s = 0; s < K; s++) rb[s] = 0u;
    if (g.lane == 0) rb[0] = 1u;
  }
  if (g.lane < g.G) {
#pragma unroll
    for (int s = 0; s < K; s++) {
      A[K * g.lane + s] = ra[s];
      B[K * g.lane + s] = rb[s];
    }
  }
  __syncwarp();
  // column k = lane + 32 t, t = 0 .. 2K-1 (k < 2NW - 1); groups of 4 columns per sweep
  for (int t0 = 0; t0 < 2 * K; t0 += 4) {
    uint32_t c0[4] = {0, 0, 0, 0}, c1[4] = {0, 0, 0, 0}, c2[4] = {0, 0, 0, 0};
    int kmin = g.lane + 32 * t0;
    int ilo = kmin - (NW - 1);
    if (ilo < 0) ilo = 0;
    int ihi = kmin + 32 * 3;
    if (ihi > NW - 1) ihi = NW - 1;
    for (int ii = ilo; ii <= ihi; ii++) {
      uint32_t av = A[ii];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        int j = kmin + 32 * u - ii;
        if (j >= 0 && j < NW) {
          uint32_t bv = B[j];
          asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
              "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
              "addc.u32 %2, %2, 0;"
              : "+r"(c0[u]), "+r"(c1[u]), "+r"(c2[u])
              : "r"(av), "r"(bv));
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      int k = kmin + 32 * u;
      if (k < 2 * NW) {
        C0[k] = c0[u];
        C1[k] = c1[u];
        C2[k] = c2[u];
      }
    }
  }
  __syncwarp();
  // P = L + H 2^N + extra 2^{2N} with L = sum_{w<NW} (C0[w] + C1[w-1] + C2[w-2]) 2^{32w},
  // H the same sum over words NW .. 2NW-1, and extra = C2[2NW-2] (word 2NW); 2^N = -1.
  uint32_t L[K], H[K], t1[K], t2[K];
#pragma unroll
  for (int s = 0; s < K; s++) {
    int w = K * g.lane + s;
    bool act = g.lane < g.G;
    L[s] = act ? C0[w] : 0u;
    t1[s] = (act && w >= 1) ? C1[w - 1] : 0u;
    t2[s] = (act && w >= 2) ? C2[w - 2] : 0u;
  }
  uint32_t c = add_chain<K>(L, L, t1, 0u);
  uint32_t Lt = resolve_add<K>(L, c, g);
  c = add_chain<K>(L, L, t2, 0u);
  Lt += resolve_add<K>(L, c, g);
#pragma unroll
  for (int s = 0; s < K; s++) {
    int w = NW + K * g.lane + s;
    bool act = g.lane < g.G;
    H[s] = act ? C0[w] : 0u;
    t1[s] = act ? C1[w - 1] : 0u;
    t2[s] = act ? C2[w - 2] : 0u;
  }
  c = add_chain<K>(H, H, t1, 0u);
  uint32_t Ht = resolve_add<K>(H, c, g);
  c = add_chain<K>(H, H, t2, 0u);
  Ht += resolve_add<K>(H, c, g);
  uint32_t extra = C2[2 * NW - 2];
  // X = L + Lt 2^N - H - Ht 2^N + extra 2^{2N} = L - H - Lt + Ht + extra (mod p)
  uint32_t bo = sub_chain<K>(L, L, H, 0u);
  uint32_t Bd = resolve_sub<K>(L, bo, g);
  int v = int(Bd) - int(Lt) + int(Ht) + int(extra);
  uint32_t T = canon_x<K>(L, v, g);
  if (neg) {
    // -x: 2^N -> 1, 0 -> 0, else ~x + 2 (N bits)
    if (T) {
#pragma unroll
      for (int s = 0; s < K; s++) L[s] = 0u;
      if (g.lane == 0) L[0] = 1u;
      T = 0u;
    } else if (!is_zero<K>(L)) {
#pragma unroll
      for (int s = 0; s < K; s++) L[s] = g.lane < g.G ? ~L[s] : 0u;
      T = add_small<K>(L, 2u, g);
    }
  }
  __syncwarp();
  gmem_store_x<K>(acell, L, T, g);
  __syncwarp();
}

template <int K>
__global__ void pointwise_kernel(uint64_t *__restrict__ a, const uint64_t *__restrict__ b, int64_t n,
                                 int64_t stride, int N, int warps_per_block) {
  extern __shared__ uint32_t sm[];
  const Geo g = make_geo(N, K);
  const int warp = threadIdx.x >> 5;
  uint32_t *ws = sm + size_t(warp) * (8 * g.NW + 8);
  const int64_t nwarps = int64_t(gridDim.x) * warps_per_block;
  for (int64_t i = int64_t(blockIdx.x) * warps_per_block + warp; i < n; i += nwarps)
    pointwise_one<K>(a + i * stride, b + i * stride, ws, g);
}

template <int K>
__global__ void pointwise_batch_kernel(const PointwiseItem *__restrict__ items, int64_t stride, int N,
                                       int warps_per_block, uint64_t *__restrict__ pool) {
  extern __shared__ uint32_t sm[];
  const Geo g = make_geo(N, K);
  const int warp = threadIdx.x >> 5;
  uint32_t *ws = sm + size_t(warp) * (8 * g.NW + 8);
  const PointwiseItem it = items[blockIdx.y];
  const int64_t nwarps = int64_t(gridDim.x) * warps_per_block;
  for (int64_t i = int64_t(blockIdx.x) * warps_per_block + warp; i < it.n; i += nwarps)
    pointwise_one<K>(pool + it.a + i * stride, pool + it.b + i * stride, ws, g);
}

template <int K>
cudaError_t pointwise_k(uint64_t *a, const uint64_t *b, int64_t n, int64_t stride, const Ring &r,
                        cudaStream_t s) {
  size_t per_warp = size_t(8 * r.NW + 8) * 4;
  int wpb = int(std::min<size_t>(8, std::max<size_t>(1, (96 * 1024) / per_warp)));
  size_t smem = per_warp * wpb;
  cudaError_t e = cudaFuncSetAttribute(pointwise_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  int64_t blocks = (n + wpb - 1) / wpb;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  pointwise_kernel<K><<<int(blocks), wpb * 32, smem, s>>>(a, b, n, stride, int(r.N), wpb);
  return cudaGetLastError();
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
  TFT_DISPATCH_K(r.K, (pack_kernel<KK><<<grid_for(len, 8), 256, 0, s>>>(coef, len, limbs, is_signed, cells,
                                                                         stride_limbs, int(r.N))));
  return cudaGetLastError();
}

cudaError_t launch_lift(const uint64_t *cells, int64_t n, int64_t stride_limbs, int is_signed, uint64_t *out,
                        int64_t limbs_out, const Ring &r, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  TFT_DISPATCH_K(r.K, (lift_kernel<KK><<<grid_for(n, 8), 256, 0, s>>>(cells, n, stride_limbs, is_signed, out,
                                                                       limbs_out, int(r.N))));
  return cudaGetLastError();
}

template <int K>
cudaError_t pointwise_batch_k(const PointwiseItem *items, int count, int64_t max_n, int64_t stride,
                              const Ring &r, uint64_t *pool, cudaStream_t s) {
  size_t per_warp = size_t(8 * r.NW + 8) * 4;
  int wpb = int(std::min<size_t>(8, std::max<size_t>(1, (96 * 1024) / per_warp)));
  size_t smem = per_warp * wpb;
  cudaError_t e = cudaFuncSetAttribute(pointwise_batch_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e != cudaSuccess) return e;
  int64_t bx = (max_n + wpb - 1) / wpb;
  int64_t cap = std::max<int64_t>(1, (152 * 16) / std::max(1, count));
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  pointwise_batch_kernel<K><<<dim3(unsigned(bx), unsigned(count)), wpb * 32, smem, s>>>(items, stride, int(r.N), wpb, pool);
  return cudaGetLastError();
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
  TFT_DISPATCH_K(r.K, (pack_batch_kernel<KK><<<grid, 256, 0, s>>>(d_items, stride_limbs, int(r.N), pool)));
  return cudaGetLastError();
}

cudaError_t launch_lift_batch(const LiftItem *d_items, int count, int64_t max_n, int64_t stride_limbs,
                              const Ring &r, uint64_t *pool, cudaStream_t s) {
  if (count <= 0 || max_n <= 0) return cudaSuccess;
  const dim3 grid(unsigned(grid_x_for(max_n, count, 8)), unsigned(count));
  TFT_DISPATCH_K(r.K, (lift_batch_kernel<KK><<<grid, 256, 0, s>>>(d_items, stride_limbs, int(r.N), pool)));
  return cudaGetLastError();
}

cudaError_t launch_pointwise_batch(const PointwiseItem *d_items, int count, int64_t max_n, int64_t stride_limbs,
                                   const Ring &r, uint64_t *pool, cudaStream_t s) {
  if (count <= 0 || max_n <= 0) return cudaSuccess;
  TFT_DISPATCH_K(r.K, return pointwise_batch_k<KK>(d_items, count, max_n, stride_limbs, r, pool, s));
  return cudaSuccess;
}

cudaError_t launch_pointwise(uint64_t *a, const uint64_t *b, int64_t n, int64_t stride_limbs, const Ring &r,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  TFT_DISPATCH_K(r.K, return pointwise_k<KK>(a, b, n, stride_limbs, r, s));
  return cudaSuccess;
}

}  // namespace tftgpu
