// Device code of the sub-transform kernel, shared by the translation unit of the per-pass
// launches (transform_kernel.cu) and that of the persistent launches (transform_fused.cu).
//
// The sub-transform kernel. One job (a TFT or ITFT of Ls = 2^ls cells) runs on a cluster of
// C = 2^lc CTAs; every CTA keeps Ls / C cells in shared memory for the whole job, so global
// memory is read once and written once per cell. Inside a CTA the base-case butterflies of
// Algorithm 1 or 2 run as a program of dependency levels (program.cpp), one warp per
// butterfly. When C > 1 the cells move between the column layout and the row layout of the
// job's own C x (Ls / C) split through distributed shared memory (STAGE_XCHG / STAGE_SWAP).
#pragma once

#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "common.h"
#include "host.h"
#include "ring_warp.cuh"

namespace cg = cooperative_groups;

namespace tftgpu {

struct KGeo {
  Geo g;
  int ord;        // order of omega: 2N (omega = 2) or 4N (omega = sqrt2); exponents are mod ord
  uint32_t mask;  // ord - 1 when ord is a power of two, else 0
};

__device__ __forceinline__ int rot_amount(RotA a, int e, const KGeo &k) {
  if (k.mask) return int((uint32_t(a.mul) * uint32_t(e) + uint32_t(a.add)) & k.mask);
  long long v = ((long long)a.mul * e + a.add) % k.ord;
  return int(v);
}

// raw form of x omega^E (E in [0, ord)): a rotation for omega = 2, a power of sqrt2 otherwise
template <int K, bool SQ>
__device__ __forceinline__ int read_omega_pow(uint32_t (&r)[K], const uint32_t *cell, int zflag, int E,
                                              const Geo &g) {
  if (SQ) return smem_read_pow<K>(r, cell, zflag, E, g);
  return smem_read_abs<K>(r, cell, zflag, E, g);
}

template <int K>
__device__ __forceinline__ void write_cell(uint32_t *cell, uint32_t *meta, const uint32_t (&r)[K],
                                           int zflag, int tag, const Geo &g) {
  if (!zflag) smem_store_plain<K>(cell, r, g);
  if (g.lane == 0) *meta = (uint32_t(tag) << 1) | uint32_t(zflag);
}

// chunk of this lane inside a shared-memory cell
template <int K>
__device__ __forceinline__ uint32_t *lane_chunk(uint32_t *cell, const Geo &g) {
  return cell + phys<K>(K * (g.lane < g.G ? g.lane : 0));
}

template <int K>
__device__ __forceinline__ void set_meta(uint32_t *meta, int zflag, int tag, const Geo &g) {
  if (g.lane == 0) *meta = (uint32_t(tag) << 1) | uint32_t(zflag);
}

// S - 1 = rawA + rawB + 1 - (za + zb) 2^N, written to `dst` in storage form; rawA is the
// unrotated cell `acell` (all ones when za), rawB is in registers
template <int K>
__device__ __forceinline__ int sum_to(uint32_t *dst, const uint32_t *acell, const uint32_t (&B)[K], int za,
                                      int zb, const Geo &g) {
  uint32_t *ch = lane_chunk<K>(dst, g);
  uint32_t c = 0;
  if (g.lane < g.G) c = chain_stream<K, false>(ch, lane_chunk<K>(const_cast<uint32_t *>(acell), g), za != 0, B,
                                                 g.lane == 0 ? 1u : 0u);
  return settle_smem<K>(ch, int(c), za + zb, g);
}

// D - 1 = rawA - rawB - 1 - (za - zb) 2^N, written to `dst` in storage form
template <int K>
__device__ __forceinline__ int diff_to(uint32_t *dst, const uint32_t *acell, const uint32_t (&B)[K], int za,
                                       int zb, const Geo &g) {
  uint32_t *ch = lane_chunk<K>(dst, g);
  uint32_t bo = 0;
  if (g.lane < g.G) bo = chain_stream<K, true>(ch, lane_chunk<K>(const_cast<uint32_t *>(acell), g), za != 0, B,
                                                 g.lane == 0 ? 1u : 0u);
  return settle_smem<K>(ch, -int(bo), za - zb, g);
}

// S (to dS) and D (to dD) of one butterfly from one pass over the cell `acell` (K >= 4); dS or
// dD may be acell. Sets the zero flags of both outputs.
template <int K>
__device__ __forceinline__ void sum_diff_to(uint32_t *dS, uint32_t *dD, const uint32_t *acell, const uint32_t (&B)[K],
                                            int za, int zb, const Geo &g, int &zs, int &zd) {
  uint32_t *chS = lane_chunk<K>(dS, g), *chD = lane_chunk<K>(dD, g);
  uint32_t c = 0, bo = 0;
  if (g.lane < g.G)
    bf_stream<K>(chS, chD, lane_chunk<K>(const_cast<uint32_t *>(acell), g), za != 0, B, g.lane == 0 ? 1u : 0u, c, bo);
  zd = settle_smem<K>(chD, -int(bo), za - zb, g);
  zs = settle_smem<K>(chS, int(c), za + zb, g);
}

template <int K, bool SQ>
__device__ __forceinline__ void exec_op(const OpDesc &op, uint32_t *cells, uint32_t *meta, int P, int e,
                                        const KGeo &kg) {
  const Geo &g = kg.g;
  uint32_t *ci = cells + op.i * P, *cj = cells + op.j * P;
  const uint32_t mi = meta[op.i], mj = meta[op.j];
  if (op.kind == OP_TAG) {
    const int ti = int(mi >> 1);
    if (op.flags & OPF_COPY) {
      uint32_t v[K];
      smem_load_plain<K>(v, ci, g);
      int tj = ti + rot_amount(op.rb, e, kg);
      if (tj >= kg.ord) tj -= kg.ord;
      __syncwarp();
      write_cell<K>(cj, meta + op.j, v, int(mi & 1u), tj, g);
    }
    int tn = ti + rot_amount(op.ra, e, kg);
    if (tn >= kg.ord) tn -= kg.ord;
    __syncwarp();
    if (g.lane == 0) meta[op.i] = (uint32_t(tn) << 1) | (mi & 1u);
    return;
  }
  // x_i 2^Ei (+-) x_j 2^Ej = 2^Ei (x_i (+-) x_j 2^(Ej - Ei)): read x_i without rotation and
  // x_j with the difference, and give the outputs Ei more pending rotation
  int Ei = int(mi >> 1) + rot_amount(op.ra, e, kg);
  if (Ei >= kg.ord) Ei -= kg.ord;
  int Ej = int(mj >> 1) + rot_amount(op.rb, e, kg);
  if (Ej >= kg.ord) Ej -= kg.ord;
  int Er = Ej - Ei;
  if (Er < 0) Er += kg.ord;
  const int za = int(mi & 1u), zb = int(mj & 1u);
  uint32_t B[K];
  read_omega_pow<K, SQ>(B, cj, zb, Er, g);
  __syncwarp();
  auto pend = [&](RotA p) {
    int t = rot_amount(p, e, kg) + Ei;
    return t >= kg.ord ? t - kg.ord : t;
  };
  if (op.kind == OP_BF) {
    // x_i is streamed from its cell: the difference goes first when it is written to cell j,
    // so that x_i is still intact for the sum, which then rewrites cell i word by word
    const bool wantS = op.flags & OPF_S, wantD = op.flags & OPF_D;
    const bool toj = op.flags & OPF_S_TO_J, toi = op.flags & OPF_D_TO_I;
    if constexpr (K >= 4) {
      if (wantS && wantD && toj == toi) {
        // S and D from one pass over x_i (S to i and D to j, or S to j and D to i)
        int zs, zd;
        sum_diff_to<K>(toj ? cj : ci, toi ? ci : cj, ci, B, za, zb, g, zs, zd);
        set_meta<K>(meta + (toi ? op.i : op.j), zd, pend(op.p1), g);
        set_meta<K>(meta + (toj ? op.j : op.i), zs, pend(op.p0), g);
        return;
      }
    }
    if (wantD && !toi) {
      const int zd = diff_to<K>(cj, ci, B, za, zb, g);
      set_meta<K>(meta + op.j, zd, pend(op.p1), g);
    }
    if (wantS) {
      const int zs = sum_to<K>(toj ? cj : ci, ci, B, za, zb, g);
      set_meta<K>(meta + (toj ? op.j : op.i), zs, pend(op.p0), g);
    }
    if (wantD && toi) {
      const int zd = diff_to<K>(ci, ci, B, za, zb, g);
      set_meta<K>(meta + op.i, zd, pend(op.p1), g);
    }
    return;
  }
  // OP_CROSS: D = x_i - x_j -> x_j (pending p1); then x_i <- x_i + D
  const int zd = diff_to<K>(cj, ci, B, za, zb, g);
  set_meta<K>(meta + op.j, zd, pend(op.p1), g);
  __syncwarp();
  if (zd)
    set_ones<K>(B, g);
  else
    smem_load_plain<K>(B, cj, g);
  const int zs = sum_to<K>(ci, ci, B, za, zd, g);
  set_meta<K>(meta + op.i, zs, Ei, g);
}

// Copy the N-bit part of a cell between global memory (16-byte aligned when vec16) and a
// shared-memory cell, with consecutive lanes on consecutive addresses (coalesced); returns the
// top limb on loads. Cell loads go through L2 only (ld.global.cg): in a persistent launch
// another CTA of the same kernel may have written the cell. Groups of 4 words never straddle a 32-word row, so for K >= 4 both sides
// move 16-byte vectors.
template <int K>
__device__ __forceinline__ uint64_t gmem_to_smem_cell(uint32_t *scell, const uint64_t *gcell, bool vec16,
                                                      const Geo &g) {
  const uint32_t *w32 = reinterpret_cast<const uint32_t *>(gcell);
  if (vec16 && (g.NW & 3) == 0) {
    const uint4 *src = reinterpret_cast<const uint4 *>(w32);
    for (int q = g.lane; q < g.NW / 4; q += 32) {
      const uint4 v = __ldcg(src + q);
      const int pw = phys<K>(4 * q);
      if constexpr (K >= 4) {
        *reinterpret_cast<uint4 *>(scell + pw) = v;
      } else {
        scell[pw] = v.x;
        scell[pw + 1] = v.y;
        scell[pw + 2] = v.z;
        scell[pw + 3] = v.w;
      }
    }
  } else {
    const uint2 *src = reinterpret_cast<const uint2 *>(w32);
    for (int q = g.lane; q < g.NW / 2; q += 32) {
      const uint2 v = __ldcg(src + q);
      const int pw = phys<K>(2 * q);
      scell[pw] = v.x;
      scell[pw + 1] = v.y;
    }
  }
  return __ldcg(gcell + g.NW / 2);
}

template <int K>
__device__ __forceinline__ void smem_to_gmem_cell(uint64_t *gcell, const uint32_t *scell, uint64_t top, bool vec16,
                                                  const Geo &g) {
  uint32_t *w32 = reinterpret_cast<uint32_t *>(gcell);
  if (vec16 && (g.NW & 3) == 0) {
    uint4 *dst = reinterpret_cast<uint4 *>(w32);
    for (int q = g.lane; q < g.NW / 4; q += 32) {
      const int pw = phys<K>(4 * q);
      if constexpr (K >= 4)
        dst[q] = *reinterpret_cast<const uint4 *>(scell + pw);
      else
        dst[q] = make_uint4(scell[pw], scell[pw + 1], scell[pw + 2], scell[pw + 3]);
    }
  } else {
    uint2 *dst = reinterpret_cast<uint2 *>(w32);
    for (int q = g.lane; q < g.NW / 2; q += 32) {
      const int pw = phys<K>(2 * q);
      dst[q] = make_uint2(scell[pw], scell[pw + 1]);
    }
  }
  if (g.lane == 0) gcell[g.NW / 2] = top;
}

// The status word of the bounded waits (one per device, defined in transform_kernel.cu): a
// kernel that gives up on a wait sets bit 1 (a bulk load) or bit 2 (a dependency of a
// persistent launch); the host reads and clears it through read_wait_status. Kernels receive
// its device address as a parameter, so every translation unit sets the same word.

// Wait limit of a bulk-copy completion (the copies of one job land within microseconds).
constexpr uint64_t kBulkWaitNs = 1000000000ull;

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the given phase parity of an mbarrier; false when limit_ns passed first.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mb, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mb), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// Bulk (TMA) load of the N-bit parts of a job's first nl cells, one 128-byte row per lane and
// cell, into the padded shared-memory rows, and of each cell's top limb with the limb after it
// (16 bytes at byte 4 NW of the cell, inside its stride) into tops[4 s ..]; completion is
// counted on the mbarrier mb (one arrival, by thread 0, announcing all the bytes). Needs
// 16-byte aligned cells of an even stride and NW a multiple of 32 (rows of 32 words); cell s is
// read from gcell(s).
__device__ __forceinline__ void bulk_copy(uint32_t dst_smem, const void *src_gen, uint32_t bytes, uint32_t mb) {
  uint64_t src;
  asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(src) : "l"(src_gen));
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst_smem),
               "l"(src), "r"(bytes), "r"(mb)
               : "memory");
}

template <typename CellAddr>
__device__ __forceinline__ void bulk_load_cells(uint32_t *cells, uint32_t *tops, int P, int nl, uint32_t mb, int NW,
                                                int warp, int nw, int lane, CellAddr gcell) {
  if (threadIdx.x == 0) {
    const uint32_t bytes = uint32_t(nl) * (uint32_t(NW) * 4u + 16u);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
  }
  const int rows = NW >> 5;
  for (int s = warp; s < nl; s += nw) {
    const char *gc = reinterpret_cast<const char *>(gcell(s));
    if (lane < rows) bulk_copy(uint32_t(__cvta_generic_to_shared(cells + s * P + 36 * lane)), gc + 128 * lane, 128u, mb);
    if (lane == 0) bulk_copy(uint32_t(__cvta_generic_to_shared(tops + 4 * s)), gc + 4 * NW, 16u, mb);
  }
}

// Tensor (TMA) copies of whole cells, for rings of 8 or more 32-word rows (K >= 8) whose cells
// are 16-byte aligned with room for the top limb and the limb after it (stride >= W + 1). The
// maps (CellMaps, built per transform call by make_cell_maps) view the call's buffer as
// [cell][row][word] with 32-word rows. The load map's rows are 36 words long, so they overlap
// the next row by 4 words: one copy fills a cell's padded shared-memory rows (36-word pitch)
// directly, and the pad of its last row receives the top limb and the limb after it. The store
// map's rows are 32 words long and its box 36: the pad words fall outside the map and are not
// written, so a copy stores exactly the N-bit part; the top limb is stored separately.
struct CellMaps {
  CUtensorMap ld, st;
  int mode;  // bit 0: load map valid, bit 1: store map valid
};

// words of a cell's box (rows of 36 words)
__host__ __device__ __forceinline__ int cell_box_words(int NW) { return (NW >> 5) * 36; }

__device__ __forceinline__ void tensor_load_cell(uint32_t dst_smem, const CUtensorMap *tm, int cell, uint32_t mb) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst_smem),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(0), "r"(cell), "r"(mb)
      : "memory");
}

// one cell from shared memory to the caller's buffer as its own bulk group
__device__ __forceinline__ void tensor_store_cell(const CUtensorMap *tm, int cell, uint32_t src_smem) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(0), "r"(0), "r"(cell), "r"(src_smem)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// orders this thread's generic shared-memory accesses with later bulk (async proxy) copies
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// cell index of the job held at `slot` of CTA `rank` in the given layout
__device__ __forceinline__ int job_cell(uint32_t layout, int rank, int slot, int C, int L2, int b) {
  if (C == 1) return slot;
  if (layout == LAYOUT_ROW) return rank * L2 + slot;
  return (slot / b) * L2 + rank * b + (slot % b);
}

// one op descriptor from shared memory (8-byte aligned) or, when the program did not fit
// there, from global memory through the read-only path
__device__ __forceinline__ OpDesc load_op_shared(const uint32_t *p) {
  const uint2 *q = reinterpret_cast<const uint2 *>(p);
  uint2 w0 = q[0], w1 = q[1], w2 = q[2], w3 = q[3], w4 = q[4];
  OpDesc o;
  uint2 *d = reinterpret_cast<uint2 *>(&o);
  d[0] = w0;
  d[1] = w1;
  d[2] = w2;
  d[3] = w3;
  d[4] = w4;
  return o;
}

__device__ __forceinline__ OpDesc load_op_global(const uint32_t *p) {
  const uint2 *q = reinterpret_cast<const uint2 *>(p);
  OpDesc o;
  uint2 *d = reinterpret_cast<uint2 *>(&o);
#pragma unroll
  for (int k = 0; k < 5; k++) d[k] = __ldg(q + k);
  return o;
}

template <int K, bool STAGED, bool SQ>
__device__ __forceinline__ void run_program(const uint32_t *pg, uint32_t *cells, uint32_t *meta, int P, int e,
                                            const KGeo &kg, int warp, int nw) {
  const int nlev = int(pg[0]);
  const uint32_t *ops = pg + prog_ops_offset_words(nlev);
  const int ow = int(sizeof(OpDesc) / 4);
  for (int v = 0; v < nlev; v++) {
    const int a = int(pg[2 + v]), b = int(pg[3 + v]);
    for (int o = a + warp; o < b; o += nw) {
      const OpDesc op = STAGED ? load_op_shared(ops + o * ow) : load_op_global(ops + o * ow);
      exec_op<K, SQ>(op, cells, meta, P, e, kg);
    }
    __syncthreads();
  }
}

// Cells of CTA `rank` that arrive from partner `y` in a layout exchange: local slots
// [y b, y b + b) take the partner's slots [rank b, rank b + b). A cell is one block of P words
// in either CTA, copied whole with 16-byte loads from the partner's shared memory (consecutive
// lanes on consecutive addresses). The (partner distance r, block offset i) items go in chunks
// of one cell per warp: read into registers, cluster barrier, write locally. Pairs are
// symmetric (y = rank ^ r), so when a chunk's barrier is passed every block it touches has
// been read by its partner, and later chunks touch other blocks. All CTAs run the same number
// of chunks and barriers.
constexpr int kXchgVec = 9;  // 16-byte vectors per lane: cells of up to 9 * 32 * 4 = 1152 words

template <int K>
__device__ __forceinline__ void exchange(uint32_t *cells, uint32_t *meta, int P, int rank, int C, int b, int only,
                                         const Geo &g, int warp, int nw) {
  cg::cluster_group cluster = cg::this_cluster();
  const int items = (C - 1) * b;
  const int nvec = P / 4;
  cluster.sync();  // partners finished writing the cells we are about to read
  for (int base = 0; base < items; base += nw) {
    const int t = base + warp;
    const int r = 1 + t / b, i = t % b, y = rank ^ r;
    const bool mine = t < items && y < C && (only < 0 || rank == only || y == only);
    uint4 buf[kXchgVec];
    uint32_t m = 0;
    if (mine) {
      const uint4 *src = reinterpret_cast<const uint4 *>(cluster.map_shared_rank(cells, y) + (rank * b + i) * P);
#pragma unroll
      for (int k = 0; k < kXchgVec; k++) {
        const int v = g.lane + 32 * k;
        if (v < nvec) buf[k] = src[v];
      }
      m = *(cluster.map_shared_rank(meta, y) + (rank * b + i));
    }
    cluster.sync();
    if (mine) {
      uint4 *dst = reinterpret_cast<uint4 *>(cells + (y * b + i) * P);
#pragma unroll
      for (int k = 0; k < kXchgVec; k++) {
        const int v = g.lane + 32 * k;
        if (v < nvec) dst[v] = buf[k];
      }
      if (g.lane == 0) meta[y * b + i] = m;
    }
  }
  __syncthreads();
}

// Arguments of a persistent launch that runs every job of a plan (njobs > 0): the CTAs claim
// jobs in the order of `jobs` from a counter, wait until the jobs listed for a claimed job have
// finished (their done flags), run it and set its own flag. Every job a job waits for comes
// earlier in the claim order and was claimed by a CTA that is running, so the earliest
// unfinished job can always proceed; the waits are bounded all the same.
struct FusedArgs {
  const JobDesc *jobs;     // in claim order
  const int32_t *dep_off;  // job k waits for deps[dep_off[k] .. dep_off[k + 1])
  const int32_t *deps;     // claim positions, all below k
  uint32_t *sync;          // [0] claim counter, [1 + k] done flag of job k (zero on entry)
  int njobs;               // 0: one job per CTA (plain or merged launch)
};

// Wait limit of a dependency (a job finishes within microseconds; a whole plan within
// milliseconds).
constexpr uint64_t kDepWaitNs = 2000000000ull;

// Dynamic shared memory a job kernel may take: the 227 KB of a block less the persistent
// kernel's static claim word, which the 128-byte alignment of the dynamic cells (tensor copies)
// rounds up to 128 bytes.
constexpr size_t kJobStaticSmem = 128;
constexpr size_t kJobDynSmem = 227 * 1024 - kJobStaticSmem;

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One warp waits until every job job k depends on has set its done flag, polling with a short
// sleep. It gives up when the limit passes (bit 2 of the status word) or when an earlier wait
// has given up, so that no CTA waits twice on a plan that already failed.
__device__ __forceinline__ void wait_deps(const FusedArgs &fa, int k, int lane, uint32_t *fault) {
  const int a = fa.dep_off[k], b = fa.dep_off[k + 1];
  const uint64_t t0 = globaltimer_ns();
  for (int base = a; base < b; base += 32) {
    const int d = base + lane < b ? fa.deps[base + lane] : -1;
    for (;;) {
      const uint32_t done = d >= 0 ? ld_acquire_u32(fa.sync + 1 + d) : 1u;
      if (__all_sync(TFT_FULL, done != 0)) break;
      if (*reinterpret_cast<volatile uint32_t *>(fault) & 2u) return;
      if (globaltimer_ns() - t0 > kDepWaitNs) {
        if (lane == 0) atomicOr(fault, 2u);
        return;
      }
      __nanosleep(256);
    }
  }
}

// Shared-memory layout of a job of nslots cells (in 32-bit words): the cells (pitch words each),
// one metadata word per cell, the load's mbarrier (8-byte aligned, 4 words), the top limbs of
// bulk-loaded cells (16 bytes per cell: the top limb and the limb after it, 16-byte aligned),
// then the program staging area.
TFT_HD inline int job_mbar_word(int nslots, int pitch) { return (nslots * pitch + nslots + 1) & ~1; }
TFT_HD inline int job_tops_word(int nslots, int pitch) { return (job_mbar_word(nslots, pitch) + 4 + 3) & ~3; }
TFT_HD inline int job_stage_word(int nslots, int pitch) { return job_tops_word(nslots, pitch) + 4 * nslots; }

// One job (see the file comment): load its cells into shared memory, run the stages of its
// image, store. Returns false when its bulk load did not land in time (the status word of the
// device is set; its outputs are then unspecified).
//
// SINGLE: the launch runs single-CTA jobs only (lc = 0 at compile time), which drops the cluster
// exchange and its registers from the kernel.
// TM = 3: the cells move through the call's tensor maps tm_ld / tm_st (CellMaps, kernel
// parameters) and nothing else is compiled; the host launches it only where make_cell_maps
// succeeded, and the shared-memory alignment the copies need is that of the declaration below
// (a CTA that finds it otherwise sets bit 4 of the status word and runs nothing). TM = 0: row
// copies and 16-byte stores. The two are separate instantiations: carrying both paths in one
// body costs the three-CTAs-per-SM job its spill-free register budget.
template <int K, bool SQ, bool SINGLE, int TM = 0>
__device__ __forceinline__ bool run_job(const JobDesc &jd, uint64_t *__restrict__ x, int64_t stride_limbs, int ls,
                                        int lc, const KGeo &kg, int prog_cap, uint32_t *fault,
                                        const CUtensorMap *tm_ld = nullptr, const CUtensorMap *tm_st = nullptr) {
  extern __shared__ __align__(128) uint32_t smem[];
  if (SINGLE) lc = 0;
  const int C = 1 << lc;
  const int rank = int(blockIdx.x) & (C - 1);
  const Geo &g = kg.g;
  const int nslots = 1 << (job_ls(jd.pad, ls) - lc);
  const int L2 = nslots, b = nslots / C;
  const int P = cell_pitch_words(g.NW);
  uint32_t *cells = smem;
  uint32_t *meta = smem + nslots * P;
  uint32_t *mbar = smem + job_mbar_word(nslots, P);
  uint32_t *tops = smem + job_tops_word(nslots, P);
  uint32_t *pstage = smem + job_stage_word(nslots, P);
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t *img = jd.image;
  const int nstages = int(img[0]);
  const uint32_t load_layout = img[2], store_layout = img[3];

  // the program of the first stage is copied into shared memory (when it fits) while the cells
  // load (after the loads are issued); the other stages copy theirs when they start
  bool staged0 = false;
  auto stage_first_program = [&]() {
    if (nstages == 0) return;
    const uint32_t *ent = img + job_header_words();
    const uint32_t off = ent[2 + rank];
    if (ent[0] != STAGE_PROG || !off) return;
    const uint32_t *pg = img + off;
    const int words = prog_ops_offset_words(int(pg[0])) + int(pg[1]) * int(sizeof(OpDesc) / 4);
    if (words > prog_cap) return;
    const uint2 *src = reinterpret_cast<const uint2 *>(pg);
    uint2 *dst = reinterpret_cast<uint2 *>(pstage);
    for (int w = threadIdx.x; w < (words + 1) / 2; w += blockDim.x) dst[w] = __ldg(src + w);
    staged0 = true;
  };

  // slots whose cells are not inputs read as the implicit zeros
  for (int s = threadIdx.x; s < nslots; s += blockDim.x)
    if (job_cell(load_layout, rank, s, C, L2, b) >= jd.nload) meta[s] = 1u;

  // load into shared memory, then the storage form m = x - 1
  const bool vec16 = ((reinterpret_cast<uintptr_t>(x) & 15) == 0) && ((stride_limbs & 1) == 0);
  if constexpr (TM != 0) {
    // tensor copies need 128-byte aligned cells: rows of 36 words in multiples of 8 rows
    if (!(C == 1 && vec16 && ((g.NW >> 5) & 7) == 0 && (uint32_t(__cvta_generic_to_shared(cells)) & 127u) == 0)) {
      if (threadIdx.x == 0) atomicOr(fault, 4u);
      return false;
    }
  }
  if (TM != 0 || (K >= 4 && vec16 && C == 1 && (g.NW & 31) == 0 && stride_limbs > g.NW / 2 + 1)) {
    // single-CTA job (slot s holds cell s): one tensor copy per cell (its top limb lands in the
    // pad of its last row), or bulk copies of whole rows and of each cell's top limb
    const int nl = jd.nload < nslots ? jd.nload : nslots;
    const uint32_t mb = uint32_t(__cvta_generic_to_shared(mbar));
    constexpr bool tens = TM != 0;
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if constexpr (tens) {
      if (threadIdx.x == 0) {
        const uint32_t bytes = uint32_t(nl) * uint32_t(cell_box_words(g.NW)) * 4u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
        for (int s = 0; s < nl; s++)
          tensor_load_cell(uint32_t(__cvta_generic_to_shared(cells + s * P)), tm_ld,
                           int(jd.cell0 + int64_t(s) * jd.mstride), mb);
      }
    } else {
      const uint64_t *x0 = x + jd.cell0 * stride_limbs;
      const int64_t cstep = jd.mstride * stride_limbs;
      bulk_load_cells(cells, tops, P, nl, mb, g.NW, warp, nw, g.lane,
                      [&](int s) { return x0 + int64_t(s) * cstep; });
    }
    stage_first_program();
    // One thread waits for the copies; the others wait at the barrier, which takes no issue
    // slots from the butterflies of the other CTAs on the SM (the waiting thread polls without
    // sleeping: a sleep's wake-up delay shows on the short loads of small jobs). The barrier
    // orders every thread's reads of the copied cells after the observed completion.
    bool landed = true;
    if (threadIdx.x == 0) landed = mbar_wait_bounded(mb, 0, kBulkWaitNs);
    if (__syncthreads_or(!landed)) {
      // the copies did not all land in time: wait once more for those in flight, report, stop
      if (!landed) mbar_wait_bounded(mb, 0, kBulkWaitNs);
      __syncthreads();
      if (threadIdx.x == 0) atomicOr(fault, 1u);
      return false;
    }
    for (int s = warp; s < nl; s += nw) {
      const uint64_t T = *reinterpret_cast<const uint64_t *>(tens ? cells + s * P + P - 4 : tops + 4 * s);
      if (T & kRawTopMark) {
        // written by an earlier pass in internal form: the words are m, the top limb the metadata
        if (g.lane == 0) meta[s] = uint32_t(T);
      } else {
        const int z = settle_smem<K>(lane_chunk<K>(cells + s * P, g), 0, -1 - int(T & 1u), g);
        set_meta<K>(meta + s, z, 0, g);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mb) : "memory");
  } else {
    // coalesced plain loads
    stage_first_program();
    for (int s = warp; s < nslots; s += nw) {
      const int m = job_cell(load_layout, rank, s, C, L2, b);
      if (m >= jd.nload) continue;
      const uint64_t *gc = x + (jd.cell0 + int64_t(m) * jd.mstride) * stride_limbs;
      const uint64_t T = gmem_to_smem_cell<K>(cells + s * P, gc, vec16, g);
      if (T & kRawTopMark) {
        // written by an earlier pass in internal form: the words are m, the top limb the metadata
        if (g.lane == 0) meta[s] = uint32_t(T);
      } else {
        __syncwarp();
        const int z = settle_smem<K>(lane_chunk<K>(cells + s * P, g), 0, -1 - int(T & 1u), g);
        set_meta<K>(meta + s, z, 0, g);
      }
    }
  }
  __syncthreads();

  for (int st = 0; st < nstages; st++) {
    const uint32_t *ent = img + job_header_words() + st * job_stage_words(C);
    const uint32_t type = ent[0];
    if (type == STAGE_PROG) {
      const uint32_t off = ent[2 + rank];
      if (off) {
        // copy this CTA's program into shared memory when it fits (ops are then read from there)
        const uint32_t *pg = img + off;
        const int words = prog_ops_offset_words(int(pg[0])) + int(pg[1]) * int(sizeof(OpDesc) / 4);
        if (words <= prog_cap) {
          if (!(st == 0 && staged0)) {
            const uint2 *src = reinterpret_cast<const uint2 *>(pg);
            uint2 *dst = reinterpret_cast<uint2 *>(pstage);
            for (int w = threadIdx.x; w < (words + 1) / 2; w += blockDim.x) dst[w] = __ldg(src + w);
            __syncthreads();
          }
          run_program<K, true, SQ>(pstage, cells, meta, P, jd.e, kg, warp, nw);
        } else {
          run_program<K, false, SQ>(pg, cells, meta, P, jd.e, kg, warp, nw);
        }
      }
    } else {
      if (!SINGLE) exchange<K>(cells, meta, P, rank, C, b, type == STAGE_SWAP ? int(ent[1]) : -1, g, warp, nw);
    }
  }

  // store: x = rotc(m, t) + 1, with the final scaling where requested; or, when a later pass
  // stores these cells again, m as it is with the rotation and zero flag in the top limb.
  // TM: each warp leaves its cells' final form in their slots and stores their top limbs, then one
  // thread issues a tensor copy per cell. Else each warp stores its cells with coalesced 16-byte
  // stores, through the cell's own slot (no longer needed) when the value changes form.
  const bool raw = (jd.pad & JOB_RAW_STORE) != 0;
  for (int s = warp; s < nslots; s += nw) {
    const int m = job_cell(store_layout, rank, s, C, L2, b);
    if (m >= jd.nstore) continue;
    uint32_t r[K];
    int E = int(meta[s] >> 1) + (m < jd.nscale ? jd.escale : 0);
    if (E >= kg.ord) E -= kg.ord;
    uint64_t *gc = x + (jd.cell0 + int64_t(m) * jd.mstride) * stride_limbs;
    if (raw) {
      const uint64_t T = kRawTopMark | (uint64_t(E) << 1) | (meta[s] & 1u);
      if constexpr (TM != 0) {
        if (g.lane == 0) gc[g.NW / 2] = T;
      } else {
        smem_to_gmem_cell<K>(gc, cells + s * P, T, vec16, g);
      }
      continue;
    }
    const int z = read_omega_pow<K, SQ>(r, cells + s * P, int(meta[s] & 1u), E, g);
    uint32_t top = 0;
    if (z) {
#pragma unroll
      for (int q = 0; q < K; q++) r[q] = 0u;
    } else {
      top = add_small<K>(r, 1u, g);
    }
    __syncwarp();
    smem_store_plain<K>(cells + s * P, r, g);
    if constexpr (TM != 0) {
      if (g.lane == 0) gc[g.NW / 2] = top;
    } else {
      __syncwarp();
      smem_to_gmem_cell<K>(gc, cells + s * P, top, vec16, g);
    }
  }
  if constexpr (TM != 0) {
    // the cells written in shared memory become visible to the tensor copies, which have read
    // them before shared memory is reused or released
    fence_async_shared();
    __syncthreads();
    if (threadIdx.x == 0) {
      const int ns = jd.nstore < nslots ? jd.nstore : nslots;
      for (int s = 0; s < ns; s++)
        tensor_store_cell(tm_st, int(jd.cell0 + int64_t(s) * jd.mstride), uint32_t(__cvta_generic_to_shared(cells + s * P)));
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
  }
  return true;
}

// MINB = 3: jobs of at most 8 warps and 75 KB of shared memory, three CTAs per SM (registers
// capped at 85 per thread); MINB = 1: up to 16 warps, one CTA per SM. FULL: all 32 lanes hold
// words (NW = 32 K), which lets the compiler drop the idle-lane cases.
template <int K, bool FULL, bool SQ>
__device__ __forceinline__ KGeo make_kgeo(int N, uint32_t mask) {
  KGeo kg;
  // a FULL ring has N = 1024 K: its geometry is compile-time
  if (FULL) N = 1024 * K;
  kg.g.N = N;
  kg.g.NW = N / 32;
  kg.g.G = FULL ? 32 : kg.g.NW / K;
  kg.g.lane = threadIdx.x & 31;
  kg.g.twoN = 2 * N;
  kg.ord = SQ ? 4 * N : 2 * N;
  kg.mask = FULL ? uint32_t(kg.ord - 1) : mask;
  return kg;
}

// One job per CTA (per cluster): a plain launch, a replicated one or a merged one. TM = 3 (single-CTA
// launches only): the cells move through the tensor maps tm_ld / tm_st (see run_job).
template <int K, int MINB, bool FULL, bool SQ, bool SINGLE, int TM>
__global__ void __launch_bounds__(MINB == 3 ? 256 : 512, MINB) job_kernel(uint64_t *__restrict__ x, int64_t stride_limbs,
                                                  const JobDesc *__restrict__ jobs, int N, int ls, int lc,
                                                  uint32_t mask, int prog_cap,
                                                  const Segment *__restrict__ segs, int nsegs, int64_t rep_cells,
                                                  int rep_ctas, uint32_t *fault,
                                                  const __grid_constant__ CUtensorMap tm_ld,
                                                  const __grid_constant__ CUtensorMap tm_st) {
  grid_dependency_enter();  // signalling at the end instead measured 0.9 % slower on the batch leg
  const KGeo kg = make_kgeo<K, FULL, SQ>(N, mask);
  JobDesc jd;
  if (nsegs == 0) {
    // replicated launch: rep_ctas CTAs per replica, replica r shifted by r * rep_cells cells
    int b = int(blockIdx.x);
    int64_t shift = 0;
    if (rep_ctas > 0) {
      const int r = b / rep_ctas;
      b -= r * rep_ctas;
      shift = int64_t(r) * rep_cells;
    }
    jd = jobs[b >> lc];
    jd.cell0 += shift;
  } else {
    // merged launch: the last segment that starts at or before this CTA (segments hold whole
    // clusters, so the CTAs of one cluster agree)
    int lo = 0, hi = nsegs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (segs[mid].first_cta <= int(blockIdx.x)) lo = mid;
      else hi = mid - 1;
    }
    const Segment sg = segs[lo];
    jd = sg.jobs[(int(blockIdx.x) - sg.first_cta) >> lc];
    jd.cell0 += sg.cell_off;
  }
  run_job<K, SQ, SINGLE, TM>(jd, x, stride_limbs, ls, lc, kg, prog_cap, fault, &tm_ld, &tm_st);
}

// L2 prefetch of the input cells of a job (bulk prefetch, no shared memory): one cell per lane
// of the calling warp, 4 NW bytes each, when the cells are 16-byte aligned.
__device__ __forceinline__ void prefetch_job_l2(const JobDesc &jd, const uint64_t *x, int64_t stride_limbs, int NW,
                                                int lane) {
  const uint64_t *x0 = x + jd.cell0 * stride_limbs;
  for (int m = lane; m < jd.nload; m += 32) {
    const void *p = x0 + int64_t(m) * jd.mstride * stride_limbs;
    uint64_t a;
    asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(a) : "l"(p));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(uint32_t(NW) * 4u) : "memory");
  }
}

// A plain launch of independent single-CTA jobs as a persistent loop: CTA b runs jobs b, b + G,
// b + 2 G, ... (G CTAs) and, while it works on one, prefetches the cells of its next one into L2,
// so that the next job's loads overlap the current job's butterflies.
// TM = 3: cells move through the tensor maps tm_ld / tm_st (CellMaps); TM = 0: the maps are
// unused (see run_job).
template <int K, int MINB, bool FULL, bool SQ, int TM>
__global__ void __launch_bounds__(MINB == 3 ? 256 : 512, MINB) job_kernel_stream(uint64_t *__restrict__ x,
                                                  int64_t stride_limbs, const JobDesc *__restrict__ jobs, int njobs,
                                                  int N, int ls, uint32_t mask, int prog_cap, uint32_t *fault,
                                                  const __grid_constant__ CUtensorMap tm_ld,
                                                  const __grid_constant__ CUtensorMap tm_st) {
  grid_dependency_wait();  // dependents are signalled at the end: measured 0.35 % ahead on the benchmark
  const KGeo kg = make_kgeo<K, FULL, SQ>(N, mask);
  const bool vec16 = ((reinterpret_cast<uintptr_t>(x) & 15) == 0) && ((stride_limbs & 1) == 0);
  for (int k = int(blockIdx.x); k < njobs; k += int(gridDim.x)) {
    const int nk = k + int(gridDim.x);
    if (vec16 && nk < njobs && threadIdx.x < 32) prefetch_job_l2(jobs[nk], x, stride_limbs, kg.g.NW, kg.g.lane);
    // the descriptor goes to registers first: passed as a reference into global memory, its fields
    // would be loaded again wherever the job body uses them
    const JobDesc jd = jobs[k];
    run_job<K, SQ, true, TM>(jd, x, stride_limbs, ls, 0, kg, prog_cap, fault, &tm_ld, &tm_st);
    fence_async_shared();  // this job's shared-memory reads come before the next job's bulk copies
    __syncthreads();       // the job is done with shared memory
  }
  grid_dependents_launch();
}

// The persistent form (FusedArgs): single-CTA jobs claimed in order until none is left.
template <int K, int MINB, bool FULL, bool SQ>
__global__ void __launch_bounds__(MINB == 3 ? 256 : 512, MINB) job_kernel_fused(uint64_t *__restrict__ x,
                                                  int64_t stride_limbs, int N, int ls, uint32_t mask, int prog_cap,
                                                  FusedArgs fa, uint32_t *fault) {
  const KGeo kg = make_kgeo<K, FULL, SQ>(N, mask);
  // A job's done flag is set at the top of the CTA's next iteration by one thread of warp 1 (all
  // of the job's stores were issued before the barrier there), while thread 0 claims the next job
  // and warp 0 checks its dependencies: the fence overlaps the claim and the check, and no flag
  // waits on a check.
  __shared__ int s_claim;
  const int publisher = blockDim.x > 32 ? 32 : 0;
  uint32_t *done = nullptr;  // done flag of this CTA's previous job, not yet set
  for (;;) {
    fence_async_shared();  // the previous job's shared-memory reads come before the next bulk copies
    __syncthreads();       // the previous job is done with shared memory and with s_claim
    if (int(threadIdx.x) == publisher && done) {
      __threadfence();
      st_release_u32(done, 1u);
    }
    if (threadIdx.x == 0) s_claim = int(atomicAdd(fa.sync, 1u));
    __syncthreads();
    const int k = s_claim;
    if (k >= fa.njobs) return;
    if (threadIdx.x < 32) wait_deps(fa, k, kg.g.lane, fault);
    __syncthreads();
    // the cells written by the jobs waited for are read by bulk copies (async proxy) below
    asm volatile("fence.proxy.async.global;" ::: "memory");
    const JobDesc jd = fa.jobs[k];  // in registers (see job_kernel_stream)
    run_job<K, SQ, true>(jd, x, stride_limbs, ls, 0, kg, prog_cap, fault);
    done = fa.sync + 1 + k;
  }
}

// launchers (internal to each translation unit)
template <int K, int MINB, bool FULL, bool SQ, bool FUSED>
static cudaError_t launch_km(const Launch &L, uint64_t *x, int64_t stride_limbs, const Ring &r, cudaStream_t s,
                      size_t smem, int prog_cap, uint32_t mask, int64_t reps, int64_t rep_cells, const FusedArgs &fa,
                      uint32_t *fault, const CellMaps *cm) {
  static thread_local int configured[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 8 || !configured[dev]) {
    cudaError_t e;
    if constexpr (FUSED) {
      e = cudaFuncSetAttribute(job_kernel_fused<K, MINB, FULL, SQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(kJobDynSmem));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(job_kernel_stream<K, MINB, FULL, SQ, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(kJobDynSmem));
      if constexpr (K >= 8)
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(job_kernel_stream<K, MINB, FULL, SQ, 3>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(kJobDynSmem));
    } else {
      e = cudaFuncSetAttribute(job_kernel<K, MINB, FULL, SQ, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(kJobDynSmem));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(job_kernel<K, MINB, FULL, SQ, false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(kJobDynSmem));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(job_kernel<K, MINB, FULL, SQ, false, 0>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if constexpr (K >= 8 && FULL)
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(job_kernel<K, MINB, FULL, SQ, true, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(kJobDynSmem));
    }
    if (e != cudaSuccess) return e;
    if (dev < 8) configured[dev] = 1;
  }
  cudaLaunchConfig_t cfg = {};
  const int64_t per_rep = int64_t(L.njobs) << L.lc;
  if (per_rep * reps > int64_t(0x7fffffff)) return cudaErrorInvalidConfiguration;
  cfg.gridDim = dim3(unsigned(per_rep * reps));
  if constexpr (FUSED) {
    cfg.blockDim = dim3(unsigned(L.nwarps * 32));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    // persistent: as many CTAs as the SMs hold at once, at most one per job
    int per_sm = 0;
    cudaError_t e = fa.sync ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, job_kernel_fused<K, MINB, FULL, SQ>,
                                                                           L.nwarps * 32, smem)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, job_kernel_stream<K, MINB, FULL, SQ, 0>,
                                                                           L.nwarps * 32, smem);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    cfg.gridDim = dim3(unsigned(std::max(1, std::min(fa.njobs, std::max(1, per_sm) * sms))));
    if (!fa.sync) {
      // one CTA per job (njobs < 0): the streaming kernel's loop runs once and prefetches nothing
      const int nj = fa.njobs < 0 ? -fa.njobs : fa.njobs;
      if (fa.njobs < 0) cfg.gridDim = dim3(unsigned(nj));
      cudaLaunchAttribute pdl[1];
      pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      pdl[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = pdl;
      cfg.numAttrs = 1;
      if constexpr (K >= 8)
        if (cm && cm->mode == 3)
          return cudaLaunchKernelEx(&cfg, job_kernel_stream<K, MINB, FULL, SQ, 3>, x, stride_limbs, fa.jobs, nj,
                                    int(r.N), L.ls, mask, prog_cap, fault, cm->ld, cm->st);
      static const CellMaps no_maps = {};
      return cudaLaunchKernelEx(&cfg, job_kernel_stream<K, MINB, FULL, SQ, 0>, x, stride_limbs, fa.jobs, nj,
                                int(r.N), L.ls, mask, prog_cap, fault, no_maps.ld, no_maps.st);
    }
    return cudaLaunchKernelEx(&cfg, job_kernel_fused<K, MINB, FULL, SQ>, x, stride_limbs, int(r.N), L.ls, mask,
                              prog_cap, fa, fault);
  } else {
    cfg.blockDim = dim3(unsigned(L.nwarps * 32));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (L.lc > 0) {
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 1u << L.lc;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
    } else {
      // single-CTA jobs: programmatic dependent launch (griddepcontrol in the kernels)
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static const CellMaps no_maps = {};
    if constexpr (K >= 8 && FULL)
      if (L.lc == 0 && cm && cm->mode == 3)
        return cudaLaunchKernelEx(&cfg, job_kernel<K, MINB, FULL, SQ, true, 3>, x, stride_limbs,
                                  (const JobDesc *)L.d_jobs, int(r.N), L.ls, 0, mask, prog_cap, L.d_segs, L.nsegs,
                                  rep_cells, reps > 1 ? int(per_rep) : 0, fault, cm->ld, cm->st);
    if (L.lc == 0)
      return cudaLaunchKernelEx(&cfg, job_kernel<K, MINB, FULL, SQ, true, 0>, x, stride_limbs, (const JobDesc *)L.d_jobs,
                                int(r.N), L.ls, 0, mask, prog_cap, L.d_segs, L.nsegs, rep_cells,
                                reps > 1 ? int(per_rep) : 0, fault, no_maps.ld, no_maps.st);
    return cudaLaunchKernelEx(&cfg, job_kernel<K, MINB, FULL, SQ, false, 0>, x, stride_limbs, (const JobDesc *)L.d_jobs,
                              int(r.N), L.ls, L.lc, mask, prog_cap, L.d_segs, L.nsegs, rep_cells,
                              reps > 1 ? int(per_rep) : 0, fault, no_maps.ld, no_maps.st);
  }
}

// SMs of the current device (cached per host thread and device)
static int sm_count() {
  static thread_local int dev_cached = -1, count = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (dev != dev_cached) {
    if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || count <= 0) count = 152;
    dev_cached = dev;
  }
  return count;
}

template <int K, bool SQ, bool FUSED>
static cudaError_t launch_k(const Launch &L, uint64_t *x, int64_t stride_limbs, const Ring &r, cudaStream_t s,
                     int64_t reps, int64_t rep_cells, const FusedArgs &fa, uint32_t *fault,
                     const CellMaps *cm = nullptr) {
  const int nslots = 1 << (L.ls - L.lc);
  // cells, their metadata, the load's mbarrier and the top limbs (job_stage_word)
  const size_t base_words = size_t(job_stage_word(nslots, r.pitch));
  const uint32_t ord = uint32_t((SQ ? 4 : 2) * r.N);
  const uint32_t mask = (ord & (ord - 1)) == 0 ? ord - 1 : 0u;
  // three CTAs per SM of at most 8 warps when the cells fit in 75 KB and the launch has the
  // CTAs to fill the SMs three deep (a smaller launch gives each CTA all of its warps instead);
  // the program is staged in shared memory only if it fits beside the cells (else its ops are
  // read through the read-only path)
  // three CTAs per SM: 228 KB less 1 KB reserved per CTA, beside the static claim word
  const size_t small_words = (75 * 1024 - kJobStaticSmem) / 4;
  const int64_t ctas = (int64_t(L.njobs) << L.lc) * reps;
  if (base_words <= small_words && (L.nwarps <= 8 || ctas >= 3 * int64_t(sm_count()))) {
    Launch L8 = L;
    L8.nwarps = std::min(L.nwarps, 8);
    const int cap = size_t(L.prog_words) <= small_words - base_words ? L.prog_words : 0;
    const size_t smem = (base_words + size_t(cap)) * 4;
    // (the persistent form is built for rings that fill all 32 lanes only)
    if constexpr (FUSED) {
      if (r.G != 32) return cudaErrorInvalidValue;
      return launch_km<K, 3, true, SQ, FUSED>(L8, x, stride_limbs, r, s, smem, cap, mask, reps, rep_cells, fa, fault, cm);
    } else {
      if (r.G == 32) return launch_km<K, 3, true, SQ, FUSED>(L8, x, stride_limbs, r, s, smem, cap, mask, reps, rep_cells, fa, fault, cm);
      return launch_km<K, 3, false, SQ, FUSED>(L8, x, stride_limbs, r, s, smem, cap, mask, reps, rep_cells, fa, fault, cm);
    }
  }
  const size_t max_words = kJobDynSmem / 4;
  const int prog_cap = int(std::min<size_t>(size_t(L.prog_words), max_words > base_words ? max_words - base_words : 0));
  const size_t smem = (base_words + size_t(prog_cap)) * 4;
  if constexpr (FUSED) {
    if (r.G != 32) return cudaErrorInvalidValue;
    return launch_km<K, 1, true, SQ, FUSED>(L, x, stride_limbs, r, s, smem, prog_cap, mask, reps, rep_cells, fa, fault, cm);
  } else {
    if (r.G == 32) return launch_km<K, 1, true, SQ, FUSED>(L, x, stride_limbs, r, s, smem, prog_cap, mask, reps, rep_cells, fa, fault, cm);
    return launch_km<K, 1, false, SQ, FUSED>(L, x, stride_limbs, r, s, smem, prog_cap, mask, reps, rep_cells, fa, fault, cm);
  }
}

// Launch entry points, one translation unit per group of rings so that they compile in
// parallel (transform_k*.cu: one launch of a plan's per-pass form; transform_fused*.cu: the
// persistent form, rings of four or more words per lane). fault is the device address of the
// status word of the bounded waits.
#define TFT_DECLARE_LAUNCHES(KK, SQN)                                                                       \
  cudaError_t launch_plain_k##KK##_##SQN(const TransformPlan &p, const Launch &L, uint64_t *x, int64_t stride_limbs, \
                                        cudaStream_t s, int64_t reps, int64_t rep_cells, uint32_t *fault,       \
                                        const CellMaps *cm)
TFT_DECLARE_LAUNCHES(1, w2);
TFT_DECLARE_LAUNCHES(1, sq);
TFT_DECLARE_LAUNCHES(2, w2);
TFT_DECLARE_LAUNCHES(2, sq);
TFT_DECLARE_LAUNCHES(4, w2);
TFT_DECLARE_LAUNCHES(4, sq);
TFT_DECLARE_LAUNCHES(8, w2);
TFT_DECLARE_LAUNCHES(8, sq);
TFT_DECLARE_LAUNCHES(16, w2);
TFT_DECLARE_LAUNCHES(16, sq);
TFT_DECLARE_LAUNCHES(32, w2);
TFT_DECLARE_LAUNCHES(32, sq);
#undef TFT_DECLARE_LAUNCHES
// fa.sync null: the plain launch *plain (single-CTA jobs, no segments or replicas) in the
// persistent streaming form (job_kernel_stream)
// (cm: the call's tensor maps, or null)
cudaError_t launch_fused_small(const TransformPlan &p, uint64_t *x, int64_t stride_limbs, cudaStream_t s,
                               const FusedArgs &fa, uint32_t *fault, const Launch *plain = nullptr,
                               const CellMaps *cm = nullptr);  // K = 4, 8, 16
cudaError_t launch_fused_k32(const TransformPlan &p, uint64_t *x, int64_t stride_limbs, cudaStream_t s,
                             const FusedArgs &fa, uint32_t *fault, const Launch *plain = nullptr,
                             const CellMaps *cm = nullptr);
// Tensor maps of cells [0, ext) of the buffer x (CellMaps) for plan p's ring; false (mode 0) when
// the plan asks for none (tma), the ring or the buffer does not qualify, or the driver cannot encode
// them.
bool make_cell_maps(const TransformPlan &p, uint64_t *x, int64_t stride_limbs, int64_t ext, CellMaps *cm);

// Definitions for the translation units above.
// SQN: w2 for omega = 2, sq for omega = sqrt2 (SQ = false / true)
#define TFT_DEFINE_PLAIN(KK, SQN, SQB)                                                                      \
  cudaError_t launch_plain_k##KK##_##SQN(const TransformPlan &p, const Launch &L, uint64_t *x, int64_t stride_limbs, \
                                        cudaStream_t s, int64_t reps, int64_t rep_cells, uint32_t *fault,       \
                                        const CellMaps *cm) {                                                   \
    const FusedArgs none = {nullptr, nullptr, nullptr, nullptr, 0};                                           \
    return launch_k<KK, SQB, false>(L, x, stride_limbs, p.ring, s, reps, rep_cells, none, fault, cm);         \
  }

template <int K>
cudaError_t launch_fused_as(const TransformPlan &p, uint64_t *x, int64_t stride_limbs, cudaStream_t s,
                            const FusedArgs &fa, uint32_t *fault, const Launch *plain, const CellMaps *cm) {
  Launch L;
  if (plain) {
    L = *plain;
  } else {
    L.ls = p.f_ls;
    L.lc = 0;
    L.nwarps = p.f_nwarps;
    L.njobs = p.f_njobs;
    L.prog_words = p.f_prog_words;
  }
  return p.mode == RING_SQRT2 ? launch_k<K, true, true>(L, x, stride_limbs, p.ring, s, 1, 0, fa, fault, cm)
                              : launch_k<K, false, true>(L, x, stride_limbs, p.ring, s, 1, 0, fa, fault, cm);
}

}  // namespace tftgpu
