// The on-chip sub-transform kernel: one CTA runs one job (a TFT or ITFT of 2^ls cells that
// sits in shared memory), following a program of base-case butterflies generated from
// Algorithm 1 or 2 (program.cpp). Global memory is touched once per cell on the way in and
// once on the way out; every butterfly in between works on shared memory.
#include <cuda_runtime.h>

#include <cstdio>

#include "common.h"
#include "host.h"
#include "ring_warp.cuh"

namespace tftgpu {

__device__ __forceinline__ int rot_amount(RotA a, int e, int twoN) {
  long long v = (long long)a.mul * e + a.add;
  v %= twoN;
  return int(v < 0 ? v + twoN : v);
}

template <int K>
__device__ __forceinline__ void write_cell(uint32_t *cell, uint32_t *meta, const uint32_t (&r)[K],
                                           int zflag, int tag, const Geo &g) {
  if (!zflag) smem_store_plain<K>(cell, r, g);
  if (g.lane == 0) *meta = (uint32_t(tag) << 1) | uint32_t(zflag);
}

template <int K>
__device__ void exec_op(const OpDesc &op, uint32_t *cells, uint32_t *meta, int P, int e, const Geo &g) {
  uint32_t *ci = cells + op.i * P, *cj = cells + op.j * P;
  uint32_t mi = meta[op.i], mj = meta[op.j];
  if (op.kind == OP_TAG) {
    int ra = rot_amount(op.ra, e, g.twoN);
    int ti = int(mi >> 1);
    if (op.flags & OPF_COPY) {
      uint32_t v[K];
      smem_load_plain<K>(v, ci, g);
      int tj = ti + rot_amount(op.rb, e, g.twoN);
      if (tj >= g.twoN) tj -= g.twoN;
      __syncwarp();
      write_cell<K>(cj, meta + op.j, v, int(mi & 1u), tj, g);
    }
    int tn = ti + ra;
    if (tn >= g.twoN) tn -= g.twoN;
    __syncwarp();
    if (g.lane == 0) meta[op.i] = (uint32_t(tn) << 1) | (mi & 1u);
    return;
  }
  uint32_t A[K], B[K];
  int za = smem_read_raw<K>(A, ci, mi, rot_amount(op.ra, e, g.twoN), g);
  int zb = (op.kind == OP_BF || op.kind == OP_CROSS)
               ? smem_read_raw<K>(B, cj, mj, rot_amount(op.rb, e, g.twoN), g)
               : 0;
  __syncwarp();
  const uint32_t c0 = g.lane == 0 ? 1u : 0u;
  if (op.kind == OP_BF) {
    if (op.flags & OPF_S) {
      // S - 1 = rawA + rawB + 1 - (za + zb) 2^N
      uint32_t S[K];
      uint32_t c = add_chain<K>(S, A, B, c0);
      uint32_t C = resolve_add<K>(S, c, g);
      int zs = canon_m<K>(S, za + zb - int(C), g);
      bool toj = op.flags & OPF_S_TO_J;
      write_cell<K>(toj ? cj : ci, meta + (toj ? op.j : op.i), S, zs, rot_amount(op.p0, e, g.twoN), g);
    }
    if (op.flags & OPF_D) {
      // D - 1 = rawA - rawB - 1 - (za - zb) 2^N
      uint32_t b = sub_chain<K>(B, A, B, c0);
      uint32_t Bo = resolve_sub<K>(B, b, g);
      int zd = canon_m<K>(B, int(Bo) + za - zb, g);
      bool toi = op.flags & OPF_D_TO_I;
      write_cell<K>(toi ? ci : cj, meta + (toi ? op.i : op.j), B, zd, rot_amount(op.p1, e, g.twoN), g);
    }
    return;
  }
  // OP_CROSS: D = x_i - x_j -> x_j (pending p1); then x_i <- x_i + D
  {
    uint32_t b = sub_chain<K>(B, A, B, c0);
    uint32_t Bo = resolve_sub<K>(B, b, g);
    int zd = canon_m<K>(B, int(Bo) + za - zb, g);
    write_cell<K>(cj, meta + op.j, B, zd, rot_amount(op.p1, e, g.twoN), g);
    if (zd) set_ones<K>(B, g);
    uint32_t S[K];
    uint32_t c = add_chain<K>(S, A, B, c0);
    uint32_t C = resolve_add<K>(S, c, g);
    int zs = canon_m<K>(S, za + zd - int(C), g);
    write_cell<K>(ci, meta + op.i, S, zs, 0, g);
  }
}

template <int K>
__global__ void __launch_bounds__(512) job_kernel(uint64_t *__restrict__ x, int64_t stride_limbs,
                                                  const JobDesc *__restrict__ jobs, int N, int ls) {
  extern __shared__ uint32_t smem[];
  const JobDesc jd = jobs[blockIdx.x];
  Geo g;
  g.N = N;
  g.NW = N / 32;
  g.G = g.NW / K;
  g.lane = threadIdx.x & 31;
  g.twoN = 2 * N;
  const int Ls = 1 << ls;
  const int P = cell_pitch_words(g.NW);
  uint32_t *cells = smem;
  uint32_t *meta = smem + Ls * P;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;

  // cells never loaded read as the implicit zero inputs
  for (int m = threadIdx.x; m < Ls; m += blockDim.x)
    if (m >= jd.nload) meta[m] = 1u;

  // load: m = x - 1 into shared memory
  for (int m = warp; m < jd.nload; m += nw) {
    const uint64_t *gc = x + (jd.cell0 + int64_t(m) * jd.mstride) * stride_limbs;
    uint32_t r[K];
    uint32_t T = gmem_load_x<K>(r, gc, g);
    uint32_t b = sub_small<K>(r, 1u, g);
    int z = canon_m<K>(r, int(b) - int(T), g);
    write_cell<K>(cells + m * P, meta + m, r, z, 0, g);
  }
  __syncthreads();

  // program
  const uint32_t *pg = jd.prog;
  const int nlev = int(pg[0]);
  const OpDesc *ops = reinterpret_cast<const OpDesc *>(pg + prog_ops_offset_words(nlev));
  for (int v = 0; v < nlev; v++) {
    const int a = int(pg[2 + v]), b = int(pg[3 + v]);
    for (int o = a + warp; o < b; o += nw) {
      OpDesc op = ops[o];
      exec_op<K>(op, cells, meta, P, jd.e, g);
    }
    __syncthreads();
  }

  // store: x = rotc(m, t) + 1, with the final scaling where requested
  for (int m = warp; m < jd.nstore; m += nw) {
    uint32_t r[K];
    int E = m < jd.nscale ? jd.escale : 0;
    int z = smem_read_raw<K>(r, cells + m * P, meta[m], E, g);
    uint32_t top = 0;
    if (z) {
#pragma unroll
      for (int s = 0; s < K; s++) r[s] = 0u;
    } else {
      top = add_small<K>(r, 1u, g);
    }
    uint64_t *gc = x + (jd.cell0 + int64_t(m) * jd.mstride) * stride_limbs;
    gmem_store_x<K>(gc, r, top, g);
  }
}

namespace {

template <int K>
cudaError_t launch_k(const Launch &L, uint64_t *x, int64_t stride_limbs, const Ring &r, cudaStream_t s) {
  size_t smem = size_t(1 << L.ls) * size_t(r.pitch) * 4 + size_t(1 << L.ls) * 4;
  static thread_local int configured_dev[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 8 && configured_dev[dev] != 1) {
    cudaError_t e = cudaFuncSetAttribute(job_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    configured_dev[dev] = 1;
  }
  job_kernel<K><<<L.njobs, L.nwarps * 32, smem, s>>>(x, stride_limbs, L.d_jobs, int(r.N), L.ls);
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_transform(const TransformPlan &p, uint64_t *x, int64_t stride_limbs, cudaStream_t s) {
  for (const Launch &L : p.launches) {
    cudaError_t e;
    switch (p.ring.K) {
      case 1: e = launch_k<1>(L, x, stride_limbs, p.ring, s); break;
      case 2: e = launch_k<2>(L, x, stride_limbs, p.ring, s); break;
      case 4: e = launch_k<4>(L, x, stride_limbs, p.ring, s); break;
      case 8: e = launch_k<8>(L, x, stride_limbs, p.ring, s); break;
      case 16: e = launch_k<16>(L, x, stride_limbs, p.ring, s); break;
      case 32: e = launch_k<32>(L, x, stride_limbs, p.ring, s); break;
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace tftgpu
