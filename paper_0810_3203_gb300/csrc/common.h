// Internal definitions shared by the host planner and the CUDA kernels of libtftgpu.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define TFT_HD __host__ __device__
#else
#define TFT_HD
#endif

namespace tftgpu {

#ifdef __CUDACC__
// Programmatic dependent launch (the job kernels' launches of single-CTA jobs and the launches of
// a product's pack, pointwise and lift kernels carry the attribute): the grid lets the stream's
// next launch place its CTAs as this grid's CTAs finish, and waits until the launch before it has
// completed, its writes visible, before it touches a cell (the plan's job lists and programs were
// written long before). For a launch without the attribute, or after a predecessor that does not
// signal, the wait returns at once or the stream order holds as usual. Every kernel launched with
// the attribute calls this first. (The S[y] kernel's single-wave launches measured 5 % slower with
// it and do without.)
__device__ __forceinline__ void grid_dependency_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
// The two halves, for a kernel that signals late: the next launch's CTAs then take SM slots
// only as this grid's last CTAs end, instead of waiting there from the start of the grid's last
// wave while CTAs of launches on other streams could have used the slots.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

// ---------------------------------------------------------------- on-chip programs
//
// A sub-transform held on chip is executed as a "program": the base-case butterflies of
// Algorithm 1 or 2 (recursing down to L = 2) listed in dependency levels. Ops of one level
// touch disjoint cells and run on different warps; a block barrier separates levels.
// Rotation amounts are affine in the weight exponent e of the job that runs the program:
// amount = (mul * e + add) mod 2N, because the recursion turns zeta into zeta * omega^u
// (e + u w) or zeta^{L1} (e L1), both affine in e.

enum OpKind : uint8_t {
  OP_BF = 1,     // A = x_i 2^ra, B = x_j 2^rb; outputs S = A + B and/or D = A - B
  OP_CROSS = 2,  // D = x_i - x_j -> x_j (pending p1); x_i <- x_i + D = 2 x_i - x_j
  OP_TAG = 3,    // x_i <- x_i 2^ra (metadata only); with OPF_COPY also x_j <- x_i(old) 2^rb
};

enum OpFlags : uint8_t {
  OPF_S = 1,       // compute S
  OPF_D = 2,       // compute D
  OPF_S_TO_J = 4,  // S is written to cell j (default cell i)
  OPF_D_TO_I = 8,  // D is written to cell i (default cell j)
  OPF_COPY = 16,   // OP_TAG: copy x_i into x_j
};

// Rings of a program: Z/(2^N+1) with omega = 2 (order 2N), S[y]/(y^N+1) with omega = y (order
// M = 2N), Z/(2^N+1) with omega = sqrt2 = 2^{3N/4} - 2^{N/4} (order 4N). Rotation amounts of
// programs, jobs and cell tags are exponents of omega.
enum RingMode : int { RING_FERMAT = 0, RING_SN = 1, RING_SQRT2 = 2 };
TFT_HD inline int64_t omega_order(int64_t N, int mode) { return mode == RING_SQRT2 ? 4 * N : 2 * N; }

// Scalar flags of an op (OpDesc::pad), used over S[y]/(y^{M/2}+1) only, where the ITFT base
// case's factors 2 and 1/2 are not powers of omega: A (x_i, or the tagged cell of OP_TAG) is
// doubled or halved as it is read, S is halved as it is written.
enum OpScalar : uint16_t {
  OPS_A_DOUBLE = 1,
  OPS_A_HALVE = 2,
  OPS_S_HALVE = 4,
};

struct RotA {  // affine rotation amount: (mul * e + add) mod 2N
  int32_t mul, add;
};

struct OpDesc {
  uint16_t i, j;
  uint8_t kind, flags;
  uint16_t pad;  // OpScalar flags (S[y]/(y^{M/2}+1) programs), else 0
  RotA ra, rb, p0, p1;  // read rotations of x_i, x_j; pending rotations of the S and D outputs
};
static_assert(sizeof(OpDesc) == 40, "OpDesc layout");

// Program image (uint32 words):
//   [0] nlevels  [1] nops  [2 .. 2+nlevels] level starts (op indices)  then OpDesc[nops]
// (the op array starts at word 4 + nlevels rounded up to a multiple of 2 for 8-byte alignment)
TFT_HD inline int prog_ops_offset_words(int nlevels) { return (3 + nlevels + 1) & ~1; }

// ---------------------------------------------------------------- jobs and stages
//
// A job transforms Ls = 2^ls cells of the caller's buffer: cell m of the job is buffer cell
// (cell0 + m * mstride). It runs on a cluster of C = 2^lc CTAs (C = 1: a single CTA); each CTA
// holds Ls / C cells in shared memory. For C > 1 the job's sub-transform is split once more
// into C x (Ls / C) (Eqs. b-cols / b-rows with L1 = C): in "row layout" CTA r holds row r
// (cells r L2 + k), in "column layout" CTA c holds columns [c b, c b + b) with b = L2 / C
// (cell j L2 + c b + i at slot j b + i). A job image lists the stages the CTAs run:
//   STAGE_PROG  every CTA runs its own program (word offset per CTA, 0 = nothing to do)
//   STAGE_XCHG  switch between row and column layout: CTA x swaps its slots [y b, y b + b)
//               with CTA y's slots [x b, x b + b) through distributed shared memory
//   STAGE_SWAP  the same swap restricted to pairs that involve CTA `arg` (brings row `arg`
//               of the column layout into CTA `arg`, or back)
//
// Job image (uint32 words):
//   [0] nstages [1] C [2] load layout [3] store layout (0 row, 1 column)
//   then per stage: type, arg, offset[C]; then the program images (8-byte aligned)
enum StageType : uint32_t { STAGE_PROG = 0, STAGE_XCHG = 1, STAGE_SWAP = 2 };
enum Layout : uint32_t { LAYOUT_ROW = 0, LAYOUT_COL = 1 };

TFT_HD inline int job_stage_words(int C) { return 2 + C; }
TFT_HD inline int job_header_words() { return 4; }

// Cells [0, nload) are read on entry (the others are implicit zeros), cells [0, nstore) are
// written back; of those, [0, nscale) are multiplied by 2^escale on the way out (the ITFT's
// final division by L).
struct JobDesc {
  int64_t cell0;
  int64_t mstride;
  const uint32_t *image;
  int32_t e;
  int32_t nload;
  int32_t nstore;
  int32_t nscale;
  int32_t escale;
  int32_t pad;  // bits 0-7: log2 of the job's cells (0: the launch's ls; single-CTA launches
                // mix sizes); JOB_RAW_STORE: the job's stored cells stay in internal form
};
static_assert(sizeof(JobDesc) == 48, "JobDesc layout");

// A later pass of the same transform stores every cell this job stores, so the job may write
// them in the kernel's internal form: the N-bit storage word m = x - 1 (unrotated) and, in the
// top limb, bit 63 set with the cell's metadata word (pending rotation << 1 | zero flag) below.
// A canonical top limb is 0 or 1, so loads tell the two forms apart.
constexpr int32_t JOB_RAW_STORE = 1 << 8;
constexpr uint64_t kRawTopMark = uint64_t(1) << 63;
TFT_HD inline int job_ls(int32_t pad, int ls) { return (pad & 0xff) > 0 ? (pad & 0xff) : ls; }

// One segment of a merged launch: the jobs of one cached plan launch, applied to a buffer that
// starts `cell_off` cells after the launch's base pointer. Segment s covers the CTAs
// [first_cta, first_cta + (njobs << lc)) of the launch.
struct Segment {
  const JobDesc *jobs;
  int64_t cell_off;
  int32_t njobs;
  int32_t first_cta;
};
static_assert(sizeof(Segment) == 24, "Segment layout");

// shared-memory geometry of one cell: NW = N/32 words. Rings of more than 64 words (4 or more
// words per lane; NW is then a multiple of 32) pad each 32-word row to 36 words, which keeps
// 16-byte vector accesses aligned and free of bank conflicts; smaller rings pad one word per
// 32 (scalar accesses of a warp on 32 different banks), rounded up to 16 bytes so that every
// cell can be copied as a block of 16-byte vectors.
TFT_HD inline int cell_pitch_words(int NW) { return NW > 64 ? (NW / 32) * 36 : (NW + NW / 32 + 1 + 3) & ~3; }

// words per lane (K) for a ring of NW 32-bit words: 1 for NW <= 32, else NW/32 rounded up to
// a power of two (NW is a multiple of 32 then)
inline int words_per_lane(int NW) {
  if (NW <= 32) return 1;
  int k = (NW + 31) / 32, p = 1;
  while (p < k) p <<= 1;
  return p;
}

}  // namespace tftgpu
