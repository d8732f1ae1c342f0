// Sub-transform kernel over the Schoenhage-Nussbaumer coefficient ring (Sec. 5.2):
// R = S[y]/(y^H + 1), H = M/2, S = Z/mZ with m odd and below 2^63. omega = y, so a twiddle is
// a negacyclic shift of the H coefficients (those that pass y^H come back negated), and
// addition and subtraction work coefficient by coefficient modulo m, with no carries.
//
// One job (a TFT or ITFT of Ls = 2^ls elements, Algorithm 1 or 2 as a leveled program from
// program.cpp in S[y] mode) runs on one CTA; every element sits in shared memory for the whole
// job. One warp runs one butterfly; lane l holds coefficients l, l + 32, l + 64, ... so that a
// warp's accesses, shifted or not, touch consecutive addresses. Pending rotations (a cell's tag,
// in units of y, mod M) are merged into the next read, as in the Z/(2^N+1) kernel; the ITFT's
// factors 2 and 1/2 are scalar flags of the ops.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.h"
#include "host.h"

namespace tftgpu {

namespace {

struct SnGeo {
  int H;       // coefficients per element
  int M;       // 2H: order of y
  int lane;
  uint64_t m;  // modulus of S
};

__device__ __forceinline__ uint64_t add_m(uint64_t a, uint64_t b, uint64_t m) {
  const uint64_t s = a + b;  // a, b < m < 2^63
  return s >= m ? s - m : s;
}
__device__ __forceinline__ uint64_t sub_m(uint64_t a, uint64_t b, uint64_t m) { return a >= b ? a - b : a + (m - b); }
__device__ __forceinline__ uint64_t neg_m(uint64_t a, uint64_t m) { return a ? m - a : 0; }
__device__ __forceinline__ uint64_t half_m(uint64_t a, uint64_t m) {
  return (a & 1u) ? (a >> 1) + (m >> 1) + 1 : (a >> 1);  // (a + m) / 2 for odd a
}

// coefficient t of y^E x (E in [0, M)): x_{t-E} with the sign of the wrap
__device__ __forceinline__ uint64_t read_shifted(const uint64_t *cell, int t, int E, const SnGeo &g) {
  const bool neg0 = E >= g.H;
  const int k = neg0 ? E - g.H : E;
  int u = t - k;
  bool neg = neg0;
  if (u < 0) {
    u += g.H;
    neg = !neg;
  }
  const uint64_t v = cell[u];
  return neg ? neg_m(v, g.m) : v;
}

__device__ __forceinline__ int rot_of(RotA a, int e, const SnGeo &g) {
  long long v = ((long long)a.mul * e + a.add) % g.M;
  return int(v < 0 ? v + g.M : v);
}

// one op; KC = coefficients per lane (H / 32, or 1 when H < 32 and lanes >= H are idle)
template <int KC>
__device__ __forceinline__ void sn_exec_op(const OpDesc &op, uint64_t *cells, uint32_t *meta, int e,
                                           const SnGeo &g) {
  uint64_t *ci = cells + size_t(op.i) * g.H, *cj = cells + size_t(op.j) * g.H;
  const int ti = int(meta[op.i]), tj = int(meta[op.j]);
  const bool act = g.lane < g.H;
  if (op.kind == OP_TAG) {
    if (op.flags & OPF_COPY) {
      // x_j <- x_i (old) y^rb: data copied, the rotation pending
      int tn = ti + rot_of(op.rb, e, g);
      if (tn >= g.M) tn -= g.M;
      if (act)
        for (int s = 0; s < KC; s++) cj[g.lane + 32 * s] = ci[g.lane + 32 * s];
      if (g.lane == 0) meta[op.j] = uint32_t(tn);
    }
    if (op.pad & (OPS_A_DOUBLE | OPS_A_HALVE)) {
      if (act)
        for (int s = 0; s < KC; s++) {
          const uint64_t v = ci[g.lane + 32 * s];
          ci[g.lane + 32 * s] = (op.pad & OPS_A_DOUBLE) ? add_m(v, v, g.m) : half_m(v, g.m);
        }
    }
    int tn = ti + rot_of(op.ra, e, g);
    if (tn >= g.M) tn -= g.M;
    __syncwarp();
    if (g.lane == 0) meta[op.i] = uint32_t(tn);
    return;
  }
  // x_i y^Ei (+-) x_j y^Ej = y^Ei (x_i (+-) x_j y^(Ej - Ei)): x_i read plain, x_j shifted, the
  // outputs take Ei more pending rotation
  int Ei = ti + rot_of(op.ra, e, g);
  if (Ei >= g.M) Ei -= g.M;
  int Ej = tj + rot_of(op.rb, e, g);
  if (Ej >= g.M) Ej -= g.M;
  int Er = Ej - Ei;
  if (Er < 0) Er += g.M;
  uint64_t B[KC];
#pragma unroll
  for (int s = 0; s < KC; s++) B[s] = act ? read_shifted(cj, g.lane + 32 * s, Er, g) : 0;
  __syncwarp();  // every lane has read x_j before any lane writes it
  auto pend = [&](RotA p) {
    int t = rot_of(p, e, g) + Ei;
    return t >= g.M ? t - g.M : t;
  };
  const bool adbl = op.pad & OPS_A_DOUBLE, ahalf = op.pad & OPS_A_HALVE, shalf = op.pad & OPS_S_HALVE;
  if (op.kind == OP_BF) {
    const bool wantS = op.flags & OPF_S, wantD = op.flags & OPF_D;
    uint64_t *sdst = (op.flags & OPF_S_TO_J) ? cj : ci;
    uint64_t *ddst = (op.flags & OPF_D_TO_I) ? ci : cj;
    if (act) {
#pragma unroll
      for (int s = 0; s < KC; s++) {
        const int t = g.lane + 32 * s;
        uint64_t a = ci[t];
        if (adbl) a = add_m(a, a, g.m);
        if (ahalf) a = half_m(a, g.m);
        uint64_t sv = add_m(a, B[s], g.m);
        if (shalf) sv = half_m(sv, g.m);
        const uint64_t dv = sub_m(a, B[s], g.m);
        if (wantS) sdst[t] = sv;
        if (wantD) ddst[t] = dv;
      }
    }
    __syncwarp();
    if (g.lane == 0) {
      if (wantS) meta[(op.flags & OPF_S_TO_J) ? op.j : op.i] = uint32_t(pend(op.p0));
      if (wantD) meta[(op.flags & OPF_D_TO_I) ? op.i : op.j] = uint32_t(pend(op.p1));
    }
    return;
  }
  // OP_CROSS: D = x_i - x_j -> x_j (pending p1); x_i <- x_i + D = 2 x_i - x_j (pending Ei)
  if (act) {
#pragma unroll
    for (int s = 0; s < KC; s++) {
      const int t = g.lane + 32 * s;
      const uint64_t a = ci[t];
      const uint64_t dv = sub_m(a, B[s], g.m);
      cj[t] = dv;
      ci[t] = add_m(a, dv, g.m);
    }
  }
  __syncwarp();
  if (g.lane == 0) {
    meta[op.j] = uint32_t(pend(op.p1));
    meta[op.i] = uint32_t(Ei);
  }
}

template <int KC>
__global__ void __launch_bounds__(256, 2)
    sn_job_kernel(uint64_t *__restrict__ x, int64_t stride, const JobDesc *__restrict__ jobs, int H, uint64_t m,
                  int ls, int prog_cap) {
  extern __shared__ uint64_t sn_smem[];
  const JobDesc jd = jobs[blockIdx.x];
  SnGeo g;
  g.H = H;
  g.M = 2 * H;
  g.lane = threadIdx.x & 31;
  g.m = m;
  const int nslots = 1 << job_ls(jd.pad, ls);
  uint64_t *cells = sn_smem;
  uint32_t *meta = reinterpret_cast<uint32_t *>(cells + size_t(nslots) * H);
  uint32_t *pstage = meta + ((nslots + 1) & ~1);  // 8-byte aligned
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool act = g.lane < H;

  // load; cells that are not inputs are the implicit zeros
  for (int s = warp; s < nslots; s += nw) {
    uint64_t *c = cells + size_t(s) * H;
    if (s < jd.nload) {
      const uint64_t *gc = x + (jd.cell0 + int64_t(s) * jd.mstride) * stride;
      if (act)
        for (int q = 0; q < KC; q++) c[g.lane + 32 * q] = __ldg(gc + g.lane + 32 * q);
    } else if (act) {
      for (int q = 0; q < KC; q++) c[g.lane + 32 * q] = 0;
    }
    if (g.lane == 0) meta[s] = 0;
  }
  __syncthreads();

  const uint32_t *img = jd.image;
  const uint32_t off = img[job_header_words() + 2];  // the single stage's program (C = 1)
  if (off) {
    const uint32_t *pg = img + off;
    const int words = prog_ops_offset_words(int(pg[0])) + int(pg[1]) * int(sizeof(OpDesc) / 4);
    const bool staged = words <= prog_cap;
    if (staged) {
      const uint2 *src = reinterpret_cast<const uint2 *>(pg);
      uint2 *dst = reinterpret_cast<uint2 *>(pstage);
      for (int w = threadIdx.x; w < (words + 1) / 2; w += blockDim.x) dst[w] = __ldg(src + w);
      __syncthreads();
    }
    const uint32_t *p = staged ? pstage : pg;
    const int nlev = int(p[0]);
    const OpDesc *ops = reinterpret_cast<const OpDesc *>(p + prog_ops_offset_words(nlev));
    for (int v = 0; v < nlev; v++) {
      const int a = int(p[2 + v]), b = int(p[3 + v]);
      for (int o = a + warp; o < b; o += nw) {
        const OpDesc op = ops[o];
        sn_exec_op<KC>(op, cells, meta, jd.e, g);
      }
      __syncthreads();
    }
  }

  // store: y^tag x, then the final halvings of the scaled outputs
  for (int s = warp; s < nslots; s += nw) {
    if (s >= jd.nstore) continue;
    const uint64_t *c = cells + size_t(s) * H;
    const int E = int(meta[s]);
    const int halvings = s < jd.nscale ? jd.escale : 0;
    uint64_t *gc = x + (jd.cell0 + int64_t(s) * jd.mstride) * stride;
    if (act)
      for (int q = 0; q < KC; q++) {
        uint64_t v = read_shifted(c, g.lane + 32 * q, E, g);
        for (int h = 0; h < halvings; h++) v = half_m(v, g.m);
        gc[g.lane + 32 * q] = v;
      }
  }
}

template <int KC>
cudaError_t sn_launch(const Launch &L, uint64_t *x, int64_t stride, int64_t H, uint64_t m, cudaStream_t s) {
  const int nslots = 1 << L.ls;
  const size_t base = size_t(nslots) * size_t(H) * 8 + size_t((nslots + 1) & ~1) * 4;
  const size_t max_bytes = 227 * 1024;
  const int prog_cap = int(std::min<size_t>(size_t(L.prog_words), max_bytes > base ? (max_bytes - base) / 4 : 0));
  const size_t smem = base + size_t(prog_cap) * 4;
  cudaError_t e = cudaFuncSetAttribute(sn_job_kernel<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  sn_job_kernel<KC><<<unsigned(L.njobs), unsigned(L.nwarps * 32), smem, s>>>(x, stride, L.d_jobs, int(H), m, L.ls,
                                                                            prog_cap);
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_sn_transform(const TransformPlan &p, uint64_t *x, int64_t stride, int64_t H, uint64_t m,
                             cudaStream_t s) {
  for (const Launch &L : p.launches) {
    cudaError_t e;
    const int64_t kc = H >= 32 ? H / 32 : 1;
    switch (kc) {
      case 1: e = sn_launch<1>(L, x, stride, H, m, s); break;
      case 2: e = sn_launch<2>(L, x, stride, H, m, s); break;
      case 4: e = sn_launch<4>(L, x, stride, H, m, s); break;
      case 8: e = sn_launch<8>(L, x, stride, H, m, s); break;
      case 16: e = sn_launch<16>(L, x, stride, H, m, s); break;
      case 32: e = sn_launch<32>(L, x, stride, H, m, s); break;
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace tftgpu
