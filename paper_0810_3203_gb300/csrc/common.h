// Internal definitions shared by the host planner and the CUDA kernels of libtftgpu.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define TFT_HD __host__ __device__
#else
#define TFT_HD
#endif

namespace tftgpu {

// ---------------------------------------------------------------- on-chip programs
//
// A sub-transform that fits in one CTA's shared memory is executed as a "program": the
// butterflies of Algorithm 1 or 2 (recursing down to the L = 2 base cases) listed in
// dependency levels. Ops of one level touch disjoint cells and run on different warps; a
// block barrier separates levels. Rotation amounts are affine in the weight exponent e of
// the job that runs the program: amount = (mul * e + add) mod 2N, because the recursion
// turns zeta into zeta * omega^u (e + u w) or zeta^{L1} (e L1), both affine in e.

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

struct RotA {  // affine rotation amount: (mul * e + add) mod 2N
  int32_t mul, add;
};

struct OpDesc {
  uint16_t i, j;
  uint8_t kind, flags;
  uint16_t pad;
  RotA ra, rb, p0, p1;  // read rotations of x_i, x_j; pending rotations of the S and D outputs
};
static_assert(sizeof(OpDesc) == 40, "OpDesc layout");

// Program image in device memory (uint32 words):
//   [0] nlevels  [1] nops  [2 .. 2+nlevels] level starts (op indices)  then OpDesc[nops]
// (the op array starts at word 4 + nlevels rounded up to a multiple of 2 for 8-byte alignment)
TFT_HD inline int prog_ops_offset_words(int nlevels) { return (3 + nlevels + 1) & ~1; }

// ---------------------------------------------------------------- jobs
//
// A job runs one program on Ls = 2^ls cells of the caller's buffer: cell m of the job is
// cell (cell0 + m * mstride) of the buffer. Cells [0, nload) are read on entry (the others
// are implicit zeros), cells [0, nstore) are written back; of those, [0, nscale) are
// multiplied by 2^escale on the way out (the ITFT's final division by L).
struct JobDesc {
  int64_t cell0;
  int64_t mstride;
  const uint32_t *prog;
  int32_t e;
  int32_t nload;
  int32_t nstore;
  int32_t nscale;
  int32_t escale;
  int32_t pad;
};
static_assert(sizeof(JobDesc) == 48, "JobDesc layout");

// shared-memory geometry of one cell: NW = N/32 words, one padding word per 32 so that the
// lane-chunked accesses of a warp hit 32 different banks
TFT_HD inline int cell_pitch_words(int NW) { return NW + NW / 32 + 1; }

// words per lane (K) for a ring of NW 32-bit words: 1 for NW <= 32, else NW/32 rounded up to
// a power of two (NW is a multiple of 32 then)
inline int words_per_lane(int NW) {
  if (NW <= 32) return 1;
  int k = (NW + 31) / 32, p = 1;
  while (p < k) p <<= 1;
  return p;
}

}  // namespace tftgpu
