// Warp-wide arithmetic in R = Z/(2^N+1) (Sec. 2: R = Z/(2^{M/2}+1) with omega = 2).
//
// One ring element is spread over one warp: lane l holds the K consecutive 32-bit words
// [K l, K l + K) of its N-bit part (lanes >= G = NW/K hold zeros). Additions run a carry
// chain inside each lane and then pass the lane carry to the next lane with shuffles; a
// carry that has to cross a lane again is rare for random data, so the cross-lane step loops
// only while some lane still has one.
//
// Storage form of a cell (shared memory): m = x - 1 (an N-bit number, so 2^N = -1 is all
// ones) plus a zero flag for x = 0, plus a pending rotation t: the cell stands for
// x 2^t. With that form, multiplying by 2^E needs no correction step except the final +1:
//   x 2^E = rotc(m, E) + 1  for x in [1, 2^N],  0 <= E < N,
// where rotc rotates the N bits of m left by E and complements the E bits that wrapped
// around (2^N = -1). For N <= E < 2N the complement applies to the bits that did not wrap
// (x 2^E = -(x 2^{E-N}) and -(y + 1) = ~y + 1). This is the "multiplication by powers of
// omega is cheap" of Sec. 5.1 written for lane-distributed words.
#pragma once

#include <cstdint>

namespace tftgpu {

#define TFT_FULL 0xffffffffu

struct Geo {
  int N;     // ring bits
  int NW;    // words of the N-bit part
  int G;     // lanes holding words
  int lane;  // this thread's lane
  int twoN;
};

// ------------------------------------------------------------------ carry chains (PTX)
template <int K>
__device__ __forceinline__ uint32_t add_chain(uint32_t (&r)[K], const uint32_t (&a)[K],
                                              const uint32_t (&b)[K], uint32_t cin) {
  uint32_t cout, d;
  asm volatile("add.cc.u32 %0, %1, 0xffffffff;" : "=r"(d) : "r"(cin));
#pragma unroll
  for (int s = 0; s < K; s++) asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(r[s]) : "r"(a[s]), "r"(b[s]));
  asm volatile("addc.u32 %0, 0, 0;" : "=r"(cout));
  return cout;
}

// r = a - b - bin over the chunk; returns the borrow out (0/1)
template <int K>
__device__ __forceinline__ uint32_t sub_chain(uint32_t (&r)[K], const uint32_t (&a)[K],
                                              const uint32_t (&b)[K], uint32_t bin) {
  uint32_t bout, d;
  asm volatile("sub.cc.u32 %0, 0, %1;" : "=r"(d) : "r"(bin));
#pragma unroll
  for (int s = 0; s < K; s++) asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(r[s]) : "r"(a[s]), "r"(b[s]));
  asm volatile("subc.u32 %0, 0, 0;" : "=r"(bout));
  return bout & 1u;
}

// ------------------------------------------------------------------ ripples
// add c at slot 0 of the lane's chunk (c may exceed 1), propagate; returns the carry out
template <int K>
__device__ __forceinline__ uint32_t ripple_add(uint32_t (&r)[K], uint32_t c) {
#pragma unroll
  for (int s = 0; s < K; s++) {
    if (!__any_sync(TFT_FULL, c)) return 0u;
    uint32_t t = r[s] + c;
    c = t < c ? 1u : 0u;
    r[s] = t;
  }
  return c;
}

// subtract c at slot 0 of the lane's chunk, propagate; returns the borrow out
template <int K>
__device__ __forceinline__ uint32_t ripple_sub(uint32_t (&r)[K], uint32_t c) {
#pragma unroll
  for (int s = 0; s < K; s++) {
    if (!__any_sync(TFT_FULL, c)) return 0u;
    uint32_t v = r[s];
    r[s] = v - c;
    c = v < c ? 1u : 0u;
  }
  return c;
}

// Carry lookahead across the lanes of a warp. Lane l emits a carry out of its chunk (gen) or
// lets an incoming one through (pass: its chunk is all ones for carries, all zeros for
// borrows; gen and pass never hold together, since a chunk that has just emitted a carry cannot
// be all ones). The carry entering lane l is c_l = gen_{l-1} | (pass_{l-1} & c_{l-1}), c_0 = 0,
// which are the carries of the binary sum A + B with A = gen and B = gen | pass as lane masks:
// c_l = bit l of (A + B) ^ A ^ B. Returns c_l of this lane and sets *top to the carry out of
// lane G - 1, which is bit G: when G < 32 the idle lane G sees it as its c_l and must not
// apply it. O(1) warp operations, however far a carry travels.
__device__ __forceinline__ uint32_t lookahead_in(bool gen, bool pass, const Geo &g, uint32_t *top) {
  const uint32_t A = __ballot_sync(TFT_FULL, gen);
  const uint32_t B = A | __ballot_sync(TFT_FULL, pass);
  const uint64_t c = (uint64_t(A) + uint64_t(B)) ^ uint64_t(A) ^ uint64_t(B);
  *top = uint32_t(c >> g.G) & 1u;
  return uint32_t(c >> g.lane) & 1u;
}

// Lane carries cout (0/1, out of each lane's chunk) moved into the following lanes. Returns the
// carry out of bit N.
template <int K>
__device__ __forceinline__ uint32_t resolve_add(uint32_t (&r)[K], uint32_t cout, const Geo &g) {
  const bool gen = g.lane < g.G && cout != 0;
  if (!__any_sync(TFT_FULL, gen)) return 0u;
  bool pass = g.lane < g.G && !gen;
#pragma unroll
  for (int s = 0; s < K; s++) pass = pass && r[s] == TFT_FULL;
  uint32_t top;
  if (lookahead_in(gen, pass, g, &top) && g.lane < g.G) {
    uint32_t c = 1u;
#pragma unroll
    for (int s = 0; s < K; s++) {
      r[s] += c;
      c = (c && r[s] == 0u) ? 1u : 0u;
    }
  }
  return top;
}

// Lane borrows bout (0/1) moved into the following lanes. Returns the borrow out of bit N.
template <int K>
__device__ __forceinline__ uint32_t resolve_sub(uint32_t (&r)[K], uint32_t bout, const Geo &g) {
  const bool gen = g.lane < g.G && bout != 0;
  if (!__any_sync(TFT_FULL, gen)) return 0u;
  bool pass = g.lane < g.G && !gen;
#pragma unroll
  for (int s = 0; s < K; s++) pass = pass && r[s] == 0u;
  uint32_t top;
  if (lookahead_in(gen, pass, g, &top) && g.lane < g.G) {
    uint32_t c = 1u;
#pragma unroll
    for (int s = 0; s < K; s++) {
      const uint32_t old = r[s];
      r[s] = old - c;
      c = (c && old == 0u) ? 1u : 0u;
    }
  }
  return top;
}

// r += v at bit 0 (v >= 0, warp-uniform); returns the carry out of bit N
template <int K>
__device__ __forceinline__ uint32_t add_small(uint32_t (&r)[K], uint32_t v, const Geo &g) {
  uint32_t co = ripple_add<K>(r, g.lane == 0 ? v : 0u);
  return resolve_add<K>(r, co, g);
}

template <int K>
__device__ __forceinline__ uint32_t sub_small(uint32_t (&r)[K], uint32_t v, const Geo &g) {
  uint32_t bo = ripple_sub<K>(r, g.lane == 0 ? v : 0u);
  return resolve_sub<K>(r, bo, g);
}

template <int K>
__device__ __forceinline__ bool is_zero(const uint32_t (&r)[K]) {
  uint32_t o = 0;
#pragma unroll
  for (int s = 0; s < K; s++) o |= r[s];
  return !__any_sync(TFT_FULL, o);
}

template <int K>
__device__ __forceinline__ void set_ones(uint32_t (&r)[K], const Geo &g) {
#pragma unroll
  for (int s = 0; s < K; s++) r[s] = g.lane < g.G ? TFT_FULL : 0u;
}

// Canonical value: x = R + v (mod 2^N+1) with x in [0, 2^N]; returns the top bit (1 only for
// x = 2^N, then r is zero).
template <int K>
__device__ __forceinline__ uint32_t canon_x(uint32_t (&r)[K], int v, const Geo &g) {
  while (v != 0) {
    if (v > 0) {
      uint32_t o = add_small<K>(r, uint32_t(v), g);
      v = -int(o);
    } else {
      if (v == -1 && is_zero<K>(r)) return 1u;  // x = -1 = 2^N
      uint32_t b = sub_small<K>(r, uint32_t(-v), g);
      v = b ? 1 : 0;
    }
  }
  return 0u;
}

// ------------------------------------------------------------------ chains into shared memory
// dst = a + b + cin (ADD) or a - b - cin (SUB) over this lane's chunk, where a is read from
// the shared-memory chunk `asrc` (or is all ones when a_ones: the zero cell's raw form) and b
// sits in registers. Works in groups of up to 8 words: the group's loads issued together, then
// its chained add/sub and stores, so a needs no register array. Each group's accesses use one
// base address and immediate offsets. asrc and dst may be the same chunk. Returns the carry
// (ADD) or borrow (SUB) out of the chunk.
template <int K, bool SUB>
__device__ __forceinline__ uint32_t chain_stream(uint32_t *dst, const uint32_t *asrc, bool a_ones,
                                                 const uint32_t (&b)[K], uint32_t cin) {
  const uint32_t da = (uint32_t)__cvta_generic_to_shared(dst);
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(asrc);
  uint32_t d, cout;
  if (SUB)
    asm volatile("sub.cc.u32 %0, 0, %1;" : "=r"(d) : "r"(cin));
  else
    asm volatile("add.cc.u32 %0, %1, 0xffffffff;" : "=r"(d) : "r"(cin));
  if (K >= 8) {
#pragma unroll
    for (int g0 = 0; g0 < K; g0 += 8) {
      const uint32_t sg = sa + 4u * g0, dg = da + 4u * g0;
      uint32_t a0, a1, a2, a3, a4, a5, a6, a7;
      if (a_ones) {
        a0 = a1 = a2 = a3 = a4 = a5 = a6 = a7 = 0xffffffffu;
      } else {
        asm volatile(
            "ld.shared.u32 %0, [%8];\n\t"
            "ld.shared.u32 %1, [%8+4];\n\t"
            "ld.shared.u32 %2, [%8+8];\n\t"
            "ld.shared.u32 %3, [%8+12];\n\t"
            "ld.shared.u32 %4, [%8+16];\n\t"
            "ld.shared.u32 %5, [%8+20];\n\t"
            "ld.shared.u32 %6, [%8+24];\n\t"
            "ld.shared.u32 %7, [%8+28];"
            : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3), "=r"(a4), "=r"(a5), "=r"(a6), "=r"(a7)
            : "r"(sg));
      }
      if (SUB)
        asm volatile(
            "{\n\t.reg .u32 w;\n\t"
            "subc.cc.u32 w, %0, %8;\n\tst.shared.u32 [%16], w;\n\t"
            "subc.cc.u32 w, %1, %9;\n\tst.shared.u32 [%16+4], w;\n\t"
            "subc.cc.u32 w, %2, %10;\n\tst.shared.u32 [%16+8], w;\n\t"
            "subc.cc.u32 w, %3, %11;\n\tst.shared.u32 [%16+12], w;\n\t"
            "subc.cc.u32 w, %4, %12;\n\tst.shared.u32 [%16+16], w;\n\t"
            "subc.cc.u32 w, %5, %13;\n\tst.shared.u32 [%16+20], w;\n\t"
            "subc.cc.u32 w, %6, %14;\n\tst.shared.u32 [%16+24], w;\n\t"
            "subc.cc.u32 w, %7, %15;\n\tst.shared.u32 [%16+28], w;\n\t}"
            ::"r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(a4), "r"(a5), "r"(a6), "r"(a7), "r"(b[g0]), "r"(b[g0 + 1]),
            "r"(b[g0 + 2]), "r"(b[g0 + 3]), "r"(b[g0 + 4]), "r"(b[g0 + 5]), "r"(b[g0 + 6]), "r"(b[g0 + 7]), "r"(dg)
            : "memory");
      else
        asm volatile(
            "{\n\t.reg .u32 w;\n\t"
            "addc.cc.u32 w, %0, %8;\n\tst.shared.u32 [%16], w;\n\t"
            "addc.cc.u32 w, %1, %9;\n\tst.shared.u32 [%16+4], w;\n\t"
            "addc.cc.u32 w, %2, %10;\n\tst.shared.u32 [%16+8], w;\n\t"
            "addc.cc.u32 w, %3, %11;\n\tst.shared.u32 [%16+12], w;\n\t"
            "addc.cc.u32 w, %4, %12;\n\tst.shared.u32 [%16+16], w;\n\t"
            "addc.cc.u32 w, %5, %13;\n\tst.shared.u32 [%16+20], w;\n\t"
            "addc.cc.u32 w, %6, %14;\n\tst.shared.u32 [%16+24], w;\n\t"
            "addc.cc.u32 w, %7, %15;\n\tst.shared.u32 [%16+28], w;\n\t}"
            ::"r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(a4), "r"(a5), "r"(a6), "r"(a7), "r"(b[g0]), "r"(b[g0 + 1]),
            "r"(b[g0 + 2]), "r"(b[g0 + 3]), "r"(b[g0 + 4]), "r"(b[g0 + 5]), "r"(b[g0 + 6]), "r"(b[g0 + 7]), "r"(dg)
            : "memory");
    }
  } else {
    uint32_t a[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      if (a_ones)
        a[k] = 0xffffffffu;
      else
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(a[k]) : "r"(sa + 4u * k));
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
      uint32_t w;
      if (SUB)
        asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(w) : "r"(a[k]), "r"(b[k]));
      else
        asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(w) : "r"(a[k]), "r"(b[k]));
      asm volatile("st.shared.u32 [%0], %1;" ::"r"(da + 4u * k), "r"(w) : "memory");
    }
  }
  if (SUB) {
    asm volatile("subc.u32 %0, 0, 0;" : "=r"(cout));
    return cout & 1u;
  }
  asm volatile("addc.u32 %0, 0, 0;" : "=r"(cout));
  return cout;
}

// Rest of settle_smem once some carry has survived the first word of a chunk: c (-1, 0 or +1)
// is pending at word `start` of this lane's chunk. Each round ripples the pending carries
// through the lanes' own chunks, moves the carries that leave a chunk across lanes with the
// lookahead (one sign at a time, each over whole chunks that pass it on), and puts the net
// carry out of bit N back in at bit 0 with the opposite sign (2^N = -1). A legitimate result
// settles within two rounds; carries that still circulate after six mean the value is -1 (the
// zero cell), reported by returning 1.
template <int K>
__device__ __noinline__ int settle_smem_slow(uint32_t *chunk, int c, const Geo &g) {
  int start = 1;
  for (int round = 0; round < 6; round++) {
    for (int s = start; s < K && c != 0; s++) {
      const uint32_t old = chunk[s];
      const uint32_t t = old + uint32_t(c);
      c = c > 0 ? int(t < old) : -int(t > old);
      chunk[s] = t;
    }
    if (!__any_sync(TFT_FULL, c != 0)) return 0;
    // Lanes above 0 carry the chain's sign, lane 0 may carry the other one. That sign goes
    // first: its emitters are then untouched when they emit, so no lane ever has to pass on
    // two carries of one sign (which the lookahead cannot express); in the second phase only
    // lane 0 emits, and nothing enters lane 0.
    int wrap = 0;
    const bool plus_first = __any_sync(TFT_FULL, g.lane > 0 && c > 0);
    for (int ph = 0; ph < 2; ph++) {
      const bool plus = (ph == 0) == plus_first;
      const bool gen = plus ? c > 0 : c < 0;
      if (!__any_sync(TFT_FULL, gen)) continue;
      const uint32_t pattern = plus ? TFT_FULL : 0u;  // a chunk that passes the carry on
      bool pass = g.lane < g.G && !gen;
      for (int s = 0; s < K && pass; s++) pass = chunk[s] == pattern;
      uint32_t top;
      if (lookahead_in(gen, pass, g, &top) && g.lane < g.G) {
        for (int s = 0; s < K; s++) {
          const uint32_t old = chunk[s];
          chunk[s] = plus ? old + 1u : old - 1u;
          if (old != pattern) break;
        }
      }
      wrap += plus ? -int(top) : int(top);
    }
    if (wrap == 0) return 0;
    c = g.lane == 0 ? wrap : 0;
    start = 0;
  }
  return 1;
}

// settle() for a result that sits in this lane's chunk `chunk` of a shared-memory cell: cout is
// each lane's carry out of its chunk (all of one sign); it enters the next lane, and the carry
// out of bit N re-enters lane 0 negated (2^N = -1) together with v0. Leaves m in [0, 2^N - 1]
// and returns 0, or returns 1 when m = -1 (the cell value x is zero). Carries are applied to
// the first word of each chunk without a loop; for random data none survives that, and the
// rest (long runs of ones or zeros, common in structured data) goes to the lookahead path.
template <int K>
__device__ __forceinline__ int settle_smem(uint32_t *chunk, int cout, int v0, const Geo &g) {
  const int top = __shfl_sync(TFT_FULL, cout, g.G - 1);
  int c = __shfl_up_sync(TFT_FULL, cout, 1);
  if (g.lane == 0) c = v0 - top;
  if (g.lane >= g.G) c = 0;
  if (c != 0) {
    const uint32_t old = chunk[0];
    const uint32_t t = old + uint32_t(c);
    c = c > 0 ? int(t < old) : -int(t > old);
    chunk[0] = t;
  }
  if (!__any_sync(TFT_FULL, c != 0)) return 0;
  return settle_smem_slow<K>(chunk, c, g);
}

// ------------------------------------------------------------------ shared-memory cells
// word w of a cell sits at w + w/32 (one pad word per 32 keeps lane chunks on distinct banks)
__device__ __forceinline__ int phys(int w) { return w + (w >> 5); }

template <int K>
__device__ __forceinline__ void smem_store_plain(uint32_t *cell, const uint32_t (&r)[K], const Geo &g) {
  if (g.lane < g.G) {
    int b = phys(K * g.lane);
#pragma unroll
    for (int s = 0; s < K; s++) cell[b + s] = r[s];
  }
}

template <int K>
__device__ __forceinline__ void smem_load_plain(uint32_t (&r)[K], const uint32_t *cell, const Geo &g) {
  if (g.lane < g.G) {
    int b = phys(K * g.lane);
#pragma unroll
    for (int s = 0; s < K; s++) r[s] = cell[b + s];
  } else {
#pragma unroll
    for (int s = 0; s < K; s++) r[s] = 0u;
  }
}

// raw = rotc(m, E) for the cell (see the file comment); E in [0, 2N). The zero cell reads as
// all ones with the returned flag set (then x 2^E = raw + 1 - 2^N = 0).
//
// Output word j of lane l (j = K l + s) is the funnel shift of source words j - q - 1 and
// j - q (q = E' / 32 words, sh = E' mod 32 bits), each complemented when its logical index
// is negative (it wrapped past 2^N = -1). A lane's K + 1 source words form one window that
// crosses at most one 32-word row of the padded cell (or the end of the cell), so the window
// is two runs of consecutive addresses, each with a lane-uniform complement mask.
template <int K>
__device__ __forceinline__ int smem_read_raw(uint32_t (&r)[K], const uint32_t *cell, uint32_t meta,
                                             int Ereq, const Geo &g);

// raw = rotc(m, E) with E in [0, 2N) taken as the whole rotation (the cell's pending rotation
// is ignored: the caller has accounted for it); zflag is the cell's zero flag
template <int K>
__device__ __forceinline__ int smem_read_abs(uint32_t (&r)[K], const uint32_t *cell, int zflag, int E,
                                             const Geo &g) {
  return smem_read_raw<K>(r, cell, uint32_t(zflag), E, g);
}

template <int K>
__device__ __forceinline__ int smem_read_raw(uint32_t (&r)[K], const uint32_t *cell, uint32_t meta,
                                             int Ereq, const Geo &g) {
  if (meta & 1u) {
    set_ones<K>(r, g);
    return 1;
  }
  int E = int(meta >> 1) + Ereq;
  if (E >= g.twoN) E -= g.twoN;
  if (E == 0) {
    smem_load_plain<K>(r, cell, g);
    return 0;
  }
  if (g.lane >= g.G) {
#pragma unroll
    for (int s = 0; s < K; s++) r[s] = 0u;
    return 0;
  }
  const bool low_wrapped = E < g.N;  // complement the wrapped bits (else the others)
  const int Ep = low_wrapped ? E : E - g.N;
  const int q = Ep >> 5, sh = Ep & 31;
  const int lam0 = K * g.lane - q - 1;  // logical index of window word 0 (negative: wrapped)
  const int i0 = lam0 < 0 ? lam0 + g.NW : lam0;
  int tb, baseA, baseB;
  if (g.NW >= 32) {
    const int c0 = i0 & 31, r0 = i0 >> 5, rows = g.NW >> 5;
    const int r1 = (r0 + 1 == rows) ? 0 : r0 + 1;
    tb = 31 - c0;
    baseA = 33 * r0 + c0;
    baseB = 33 * r1 + c0 - 32;
  } else {
    tb = g.NW - 1 - i0;
    baseA = i0;
    baseB = i0 - g.NW;
  }
  const uint32_t flip = low_wrapped ? 0u : TFT_FULL;
  const uint32_t mA = (lam0 < 0 ? TFT_FULL : 0u) ^ flip;
  const uint32_t mB = (lam0 + tb + 1 < 0 ? TFT_FULL : 0u) ^ flip;
  if (sh == 0) {
    // word-aligned rotation: output word j is source word j - q, no funnel shift
#pragma unroll
    for (int s = 0; s < K; s++) {
      const int t = s + 1;
      const bool inA = t <= tb;
      r[s] = cell[(inA ? baseA : baseB) + t] ^ (inA ? mA : mB);
    }
    return 0;
  }
  uint32_t prev = cell[0 <= tb ? baseA : baseB] ^ (0 <= tb ? mA : mB);
#pragma unroll
  for (int s = 0; s < K; s++) {
    const int t = s + 1;
    const bool inA = t <= tb;
    uint32_t cur = cell[(inA ? baseA : baseB) + t] ^ (inA ? mA : mB);
    r[s] = __funnelshift_l(prev, cur, sh);  // (cur:prev) << sh, high word
    prev = cur;
  }
  return 0;
}

// r = r - rotc(m, E) - bin over this lane's chunk, as one borrow chain (E in [0, 2N), m the
// cell's N-bit storage form): the rotated words come out of the same two-run window as in
// smem_read_raw and feed subc directly, so the second operand needs no register array.
// Returns the borrow out of the chunk. Lanes >= G subtract nothing.
template <int K>
__device__ __forceinline__ uint32_t smem_sub_rotated(uint32_t (&r)[K], const uint32_t *cell, int E, uint32_t bin,
                                                     const Geo &g) {
  if (g.lane >= g.G) return 0u;
  uint32_t d, bout;
  asm volatile("sub.cc.u32 %0, 0, %1;" : "=r"(d) : "r"(bin));
  if (E == 0) {
    const int b = phys(K * g.lane);
#pragma unroll
    for (int s = 0; s < K; s++) asm volatile("subc.cc.u32 %0, %0, %1;" : "+r"(r[s]) : "r"(cell[b + s]));
  } else {
    const bool low_wrapped = E < g.N;
    const int Ep = low_wrapped ? E : E - g.N;
    const int q = Ep >> 5, sh = Ep & 31;
    const int lam0 = K * g.lane - q - 1;
    const int i0 = lam0 < 0 ? lam0 + g.NW : lam0;
    int tb, baseA, baseB;
    if (g.NW >= 32) {
      const int c0 = i0 & 31, r0 = i0 >> 5, rows = g.NW >> 5;
      const int r1 = (r0 + 1 == rows) ? 0 : r0 + 1;
      tb = 31 - c0;
      baseA = 33 * r0 + c0;
      baseB = 33 * r1 + c0 - 32;
    } else {
      tb = g.NW - 1 - i0;
      baseA = i0;
      baseB = i0 - g.NW;
    }
    const uint32_t flip = low_wrapped ? 0u : TFT_FULL;
    const uint32_t mA = (lam0 < 0 ? TFT_FULL : 0u) ^ flip;
    const uint32_t mB = (lam0 + tb + 1 < 0 ? TFT_FULL : 0u) ^ flip;
    uint32_t prev = cell[0 <= tb ? baseA : baseB] ^ (0 <= tb ? mA : mB);
#pragma unroll
    for (int s = 0; s < K; s++) {
      const int t = s + 1;
      const bool inA = t <= tb;
      const uint32_t cur = cell[(inA ? baseA : baseB) + t] ^ (inA ? mA : mB);
      const uint32_t w = sh ? __funnelshift_l(prev, cur, sh) : cur;
      asm volatile("subc.cc.u32 %0, %0, %1;" : "+r"(r[s]) : "r"(w));
      prev = cur;
    }
  }
  asm volatile("subc.u32 %0, 0, 0;" : "=r"(bout));
  return bout & 1u;
}

// raw form of x sqrt2^E over Z/(2^N+1), E in [0, 4N) (sqrt2 = 2^{3N/4} - 2^{N/4}): for even E
// the rotation rotc(m, E/2); for odd E = 2h + 1, x 2^h sqrt2 = x 2^{h+3N/4} - x 2^{h+N/4}, whose
// storage form is rotc(m, h + 3N/4) - rotc(m, h + N/4) - 1 (the +1 of x = m + 1 cancels), made
// canonical. Returns 1 for the zero cell (r all ones), like smem_read_abs.
template <int K>
__device__ __forceinline__ int smem_read_pow(uint32_t (&r)[K], const uint32_t *cell, int zflag, int E,
                                             const Geo &g) {
  if (zflag) {
    set_ones<K>(r, g);
    return 1;
  }
  const int h = E >> 1;
  if (!(E & 1)) return smem_read_abs<K>(r, cell, 0, h, g);
  int e1 = h + 3 * (g.N >> 2), e2 = h + (g.N >> 2);
  if (e1 >= g.twoN) e1 -= g.twoN;
  if (e2 >= g.twoN) e2 -= g.twoN;
  smem_read_abs<K>(r, cell, 0, e1, g);
  const uint32_t bo = smem_sub_rotated<K>(r, cell, e2, g.lane == 0 ? 1u : 0u, g);
  // r - T 2^N = r + T (mod 2^N + 1), T the borrow out of bit N
  const uint32_t T = resolve_sub<K>(r, bo, g);
  if (T && add_small<K>(r, 1u, g)) {  // r + 1 = 2^N would be the value 0: not for x != 0
    set_ones<K>(r, g);
    return 1;
  }
  return 0;
}

// ------------------------------------------------------------------ global memory cells
// canonical x: words [0, NW) and the top limb (word NW holds its low half)
template <int K>
__device__ __forceinline__ uint32_t gmem_load_x(uint32_t (&r)[K], const uint64_t *cell, const Geo &g) {
  const uint32_t *w32 = reinterpret_cast<const uint32_t *>(cell);
  if (g.lane < g.G) {
    if (K == 1) {
      r[0] = __ldg(w32 + g.lane);
    } else {
      const uint2 *p = reinterpret_cast<const uint2 *>(w32 + K * g.lane);
#pragma unroll
      for (int s = 0; s < K / 2; s++) {
        uint2 v = __ldg(p + s);
        r[2 * s] = v.x;
        r[2 * s + 1] = v.y;
      }
    }
  } else {
#pragma unroll
    for (int s = 0; s < K; s++) r[s] = 0u;
  }
  return __ldg(w32 + g.NW);
}

template <int K>
__device__ __forceinline__ void gmem_store_x(uint64_t *cell, const uint32_t (&r)[K], uint32_t top,
                                             const Geo &g) {
  uint32_t *w32 = reinterpret_cast<uint32_t *>(cell);
  if (g.lane < g.G) {
    if (K == 1) {
      w32[g.lane] = r[0];
    } else {
      uint2 *p = reinterpret_cast<uint2 *>(w32 + K * g.lane);
#pragma unroll
      for (int s = 0; s < K / 2; s++) p[s] = make_uint2(r[2 * s], r[2 * s + 1]);
    }
  }
  if (g.lane == 0) cell[g.NW / 2] = uint64_t(top);
}

}  // namespace tftgpu
