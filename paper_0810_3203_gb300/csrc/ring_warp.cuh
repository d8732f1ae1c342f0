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
// One group of GW (4 or 8) words of a carry (ADD) or borrow (SUB) chain, o = a +- b[g0 ..] +- c,
// as one asm block: the chain's carry is kept in the register c between groups (c enters as
// zero / nonzero and leaves as the carry 0/1, or the borrow 0 / all ones), so that two chains
// can advance in turns. The outputs are early-clobber: each is written while later inputs of
// the block are still to be read.
template <int GW, bool SUB, int K>
__device__ __forceinline__ void chain_group(uint32_t (&o)[GW], const uint32_t (&a)[GW], const uint32_t (&b)[K],
                                            int g0, uint32_t &c) {
  if constexpr (GW == 8) {
    if (SUB)
      asm volatile(
          "{\n\t.reg .u32 t;\n\tsub.cc.u32 t, 0, %8;\n\t"
          "subc.cc.u32 %0, %9, %17;\n\tsubc.cc.u32 %1, %10, %18;\n\t"
          "subc.cc.u32 %2, %11, %19;\n\tsubc.cc.u32 %3, %12, %20;\n\t"
          "subc.cc.u32 %4, %13, %21;\n\tsubc.cc.u32 %5, %14, %22;\n\t"
          "subc.cc.u32 %6, %15, %23;\n\tsubc.cc.u32 %7, %16, %24;\n\t"
          "subc.u32 %8, 0, 0;\n\t}"
          : "=&r"(o[0]), "=&r"(o[1]), "=&r"(o[2]), "=&r"(o[3]), "=&r"(o[4]), "=&r"(o[5]), "=&r"(o[6]), "=&r"(o[7]), "+r"(c)
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(b[g0]),
            "r"(b[g0 + 1]), "r"(b[g0 + 2]), "r"(b[g0 + 3]), "r"(b[g0 + 4]), "r"(b[g0 + 5]), "r"(b[g0 + 6]),
            "r"(b[g0 + 7]));
    else
      asm volatile(
          "{\n\t.reg .u32 t;\n\tadd.cc.u32 t, %8, 0xffffffff;\n\t"
          "addc.cc.u32 %0, %9, %17;\n\taddc.cc.u32 %1, %10, %18;\n\t"
          "addc.cc.u32 %2, %11, %19;\n\taddc.cc.u32 %3, %12, %20;\n\t"
          "addc.cc.u32 %4, %13, %21;\n\taddc.cc.u32 %5, %14, %22;\n\t"
          "addc.cc.u32 %6, %15, %23;\n\taddc.cc.u32 %7, %16, %24;\n\t"
          "addc.u32 %8, 0, 0;\n\t}"
          : "=&r"(o[0]), "=&r"(o[1]), "=&r"(o[2]), "=&r"(o[3]), "=&r"(o[4]), "=&r"(o[5]), "=&r"(o[6]), "=&r"(o[7]), "+r"(c)
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(b[g0]),
            "r"(b[g0 + 1]), "r"(b[g0 + 2]), "r"(b[g0 + 3]), "r"(b[g0 + 4]), "r"(b[g0 + 5]), "r"(b[g0 + 6]),
            "r"(b[g0 + 7]));
  } else {
    if (SUB)
      asm volatile(
          "{\n\t.reg .u32 t;\n\tsub.cc.u32 t, 0, %4;\n\t"
          "subc.cc.u32 %0, %5, %9;\n\tsubc.cc.u32 %1, %6, %10;\n\t"
          "subc.cc.u32 %2, %7, %11;\n\tsubc.cc.u32 %3, %8, %12;\n\t"
          "subc.u32 %4, 0, 0;\n\t}"
          : "=&r"(o[0]), "=&r"(o[1]), "=&r"(o[2]), "=&r"(o[3]), "+r"(c)
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[g0]), "r"(b[g0 + 1]), "r"(b[g0 + 2]), "r"(b[g0 + 3]));
    else
      asm volatile(
          "{\n\t.reg .u32 t;\n\tadd.cc.u32 t, %4, 0xffffffff;\n\t"
          "addc.cc.u32 %0, %5, %9;\n\taddc.cc.u32 %1, %6, %10;\n\t"
          "addc.cc.u32 %2, %7, %11;\n\taddc.cc.u32 %3, %8, %12;\n\t"
          "addc.u32 %4, 0, 0;\n\t}"
          : "=&r"(o[0]), "=&r"(o[1]), "=&r"(o[2]), "=&r"(o[3]), "+r"(c)
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[g0]), "r"(b[g0 + 1]), "r"(b[g0 + 2]), "r"(b[g0 + 3]));
  }
}

// GW words of a 16-byte aligned shared-memory chunk (all ones for a_ones)
template <int GW>
__device__ __forceinline__ void load_group(uint32_t (&a)[GW], const uint32_t *src, bool a_ones) {
#pragma unroll
  for (int v = 0; v < GW / 4; v++) {
    const uint4 q = a_ones ? make_uint4(TFT_FULL, TFT_FULL, TFT_FULL, TFT_FULL)
                           : reinterpret_cast<const uint4 *>(src)[v];
    a[4 * v] = q.x;
    a[4 * v + 1] = q.y;
    a[4 * v + 2] = q.z;
    a[4 * v + 3] = q.w;
  }
}

template <int GW>
__device__ __forceinline__ void store_group(uint32_t *dst, const uint32_t (&o)[GW]) {
#pragma unroll
  for (int v = 0; v < GW / 4; v++)
    reinterpret_cast<uint4 *>(dst)[v] = make_uint4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
}

// dst = a + b + cin (ADD) or a - b - cin (SUB) over this lane's chunk, where a is read from
// the shared-memory chunk `asrc` (or is all ones when a_ones: the zero cell's raw form) and b
// sits in registers. K >= 4: groups of 8 words (4 for K = 4) read and written as 16-byte
// vectors, so a needs no register array; K <= 2: scalar words. asrc and dst may be the same
// chunk. Returns the carry (ADD) or borrow (SUB) out of the chunk.
template <int K, bool SUB>
__device__ __forceinline__ uint32_t chain_stream(uint32_t *dst, const uint32_t *asrc, bool a_ones,
                                                 const uint32_t (&b)[K], uint32_t cin) {
  if constexpr (K >= 4) {
    constexpr int GW = K >= 8 ? 8 : 4;
    uint32_t c = cin;
#pragma unroll
    for (int g0 = 0; g0 < K; g0 += GW) {
      uint32_t a[GW], o[GW];
      load_group<GW>(a, asrc + g0, a_ones);
      chain_group<GW, SUB, K>(o, a, b, g0, c);
      store_group<GW>(dst + g0, o);
    }
    return SUB ? (c & 1u) : c;
  } else {
    const uint32_t da = (uint32_t)__cvta_generic_to_shared(dst);
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(asrc);
    uint32_t d, cout;
    if (SUB)
      asm volatile("sub.cc.u32 %0, 0, %1;" : "=r"(d) : "r"(cin));
    else
      asm volatile("add.cc.u32 %0, %1, 0xffffffff;" : "=r"(d) : "r"(cin));
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
    if (SUB) {
      asm volatile("subc.u32 %0, 0, 0;" : "=r"(cout));
      return cout & 1u;
    }
    asm volatile("addc.u32 %0, 0, 0;" : "=r"(cout));
    return cout;
  }
}

// Both outputs of a butterfly in one pass over a (K >= 4): per group of words, the group of a is
// read once, then D = a - b - cin and S = a + b + cin each advance by one group and are stored
// (the two chains take turns on the one carry flag). dS or dD may be the chunk of a: each group
// is read before it is written. Sets the carry out of S and the borrow out of D.
template <int K>
__device__ __forceinline__ void bf_stream(uint32_t *dS, uint32_t *dD, const uint32_t *asrc, bool a_ones,
                                          const uint32_t (&b)[K], uint32_t cin, uint32_t &cS, uint32_t &bD) {
  constexpr int GW = K >= 8 ? 8 : 4;
  uint32_t c = cin, d = cin;
#pragma unroll
  for (int g0 = 0; g0 < K; g0 += GW) {
    uint32_t a[GW], o[GW];
    load_group<GW>(a, asrc + g0, a_ones);
    chain_group<GW, true, K>(o, a, b, g0, d);
    store_group<GW>(dD + g0, o);
    chain_group<GW, false, K>(o, a, b, g0, c);
    store_group<GW>(dS + g0, o);
  }
  cS = c;
  bD = d & 1u;
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
// Rings of K >= 4 words per lane: word w of a cell sits at w + 4 (w / 32) (rows of 32 words
// padded to 36), so every lane chunk and every aligned group of 4 words starts on a 16-byte
// boundary, and the 8 lanes of a quarter warp that touch one 16-byte vector each in 8
// consecutive rows hit 8 distinct groups of banks: all cell accesses are 16-byte vectors.
// Rings of K <= 2 words per lane: w + w / 32 (one pad word per 32 keeps the scalar accesses of
// a warp on 32 distinct banks).
template <int K>
__device__ __forceinline__ int phys(int w) {
  return K >= 4 ? w + ((w >> 5) << 2) : w + (w >> 5);
}

template <int K>
__device__ __forceinline__ void smem_store_plain(uint32_t *cell, const uint32_t (&r)[K], const Geo &g) {
  if (g.lane < g.G) {
    const int b = phys<K>(K * g.lane);
    if constexpr (K >= 4) {
      uint4 *p = reinterpret_cast<uint4 *>(cell + b);
#pragma unroll
      for (int v = 0; v < K / 4; v++) p[v] = make_uint4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
    } else {
#pragma unroll
      for (int s = 0; s < K; s++) cell[b + s] = r[s];
    }
  }
}

template <int K>
__device__ __forceinline__ void smem_load_plain(uint32_t (&r)[K], const uint32_t *cell, const Geo &g) {
  if (g.lane < g.G) {
    const int b = phys<K>(K * g.lane);
    if constexpr (K >= 4) {
      const uint4 *p = reinterpret_cast<const uint4 *>(cell + b);
#pragma unroll
      for (int v = 0; v < K / 4; v++) {
        const uint4 q = p[v];
        r[4 * v] = q.x;
        r[4 * v + 1] = q.y;
        r[4 * v + 2] = q.z;
        r[4 * v + 3] = q.w;
      }
    } else {
#pragma unroll
      for (int s = 0; s < K; s++) r[s] = cell[b + s];
    }
  } else {
#pragma unroll
    for (int s = 0; s < K; s++) r[s] = 0u;
  }
}

// The rotated window of this lane for rotc(m, E') (K >= 4, E' = Ep + flip N with Ep in [0, N)):
// output word s (word K lane + s of the result) is the funnel shift of window words s and
// s + 1, where window word 0 has logical index lam0 = K lane - q - 1 (q = Ep / 32; a negative
// index wrapped past 2^N = -1 and is complemented, and for flip all the others are instead).
// The window starts u = lam0 mod 4 words into an aligned 16-byte vector; u is the same in
// every lane (K and NW are multiples of 4), so the window is read as K/4 + 1 aligned vectors
// and u picks one of four unrolled copies of the shift loop. The vectors lie in at most two
// 32-word rows, tA of them in the first; the wrap point (logical index 0) falls on a vector
// boundary, so each vector has a single complement mask. emit(s, word) receives the output
// words in order s = 0 .. K-1.
template <int K, int U, class Emit>
__device__ __forceinline__ void rot_window_u(const uint32_t *cell, int baseA, int baseB, int tA, int lamA,
                                             uint32_t flip, int sh, Emit &emit) {
  constexpr int V = K / 4 + 1;
  uint32_t w[4 * V];
#pragma unroll
  for (int t = 0; t < V; t++) {
    const uint4 v = *reinterpret_cast<const uint4 *>(cell + (t < tA ? baseA : baseB) + 4 * t);
    const uint32_t m = (lamA + 4 * t < 0 ? TFT_FULL : 0u) ^ flip;
    w[4 * t] = v.x ^ m;
    w[4 * t + 1] = v.y ^ m;
    w[4 * t + 2] = v.z ^ m;
    w[4 * t + 3] = v.w ^ m;
    // the outputs whose upper source word is in this vector
#pragma unroll
    for (int s = 0; s < K; s++)
      if (U + s + 1 >= 4 * t && U + s + 1 < 4 * t + 4) emit(s, __funnelshift_l(w[U + s], w[U + s + 1], sh));
  }
}

template <int K, class Emit>
__device__ __forceinline__ void rot_window(const uint32_t *cell, int E, const Geo &g, Emit &emit) {
  const bool low_wrapped = E < g.N;  // complement the wrapped bits (else the others)
  const int Ep = low_wrapped ? E : E - g.N;
  const int q = Ep >> 5, sh = Ep & 31;
  const int lam0 = K * g.lane - q - 1;
  const int u = lam0 & 3;
  const int a = (lam0 < 0 ? lam0 + g.NW : lam0) - u;  // aligned start, in [0, NW)
  const int r0 = a >> 5, c0 = a & 31, rows = g.NW >> 5;
  const int r1 = (r0 + 1 == rows) ? 0 : r0 + 1;
  const int tA = (32 - c0) >> 2;
  const int baseA = 36 * r0 + c0, baseB = 36 * r1 - 4 * tA;
  const uint32_t flip = low_wrapped ? 0u : TFT_FULL;
  switch (u) {
    case 0: rot_window_u<K, 0>(cell, baseA, baseB, tA, lam0, flip, sh, emit); break;
    case 1: rot_window_u<K, 1>(cell, baseA, baseB, tA, lam0 - 1, flip, sh, emit); break;
    case 2: rot_window_u<K, 2>(cell, baseA, baseB, tA, lam0 - 2, flip, sh, emit); break;
    default: rot_window_u<K, 3>(cell, baseA, baseB, tA, lam0 - 3, flip, sh, emit); break;
  }
}

// The same window for K <= 2 (rows of 33 words, scalar reads): a lane's K + 1 source words
// cross at most one 32-word row of the padded cell (or the end of the cell), so the window is
// two runs of consecutive addresses, each with a lane-uniform complement mask.
template <int K, class Emit>
__device__ __forceinline__ void rot_window_scalar(const uint32_t *cell, int E, const Geo &g, Emit &emit) {
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
  uint32_t prev = cell[0 <= tb ? baseA : baseB] ^ (0 <= tb ? mA : mB);
#pragma unroll
  for (int s = 0; s < K; s++) {
    const int t = s + 1;
    const bool inA = t <= tb;
    const uint32_t cur = cell[(inA ? baseA : baseB) + t] ^ (inA ? mA : mB);
    emit(s, __funnelshift_l(prev, cur, sh));  // (cur:prev) << sh, high word (cur for sh = 0)
    prev = cur;
  }
}

// raw = rotc(m, E) for the cell (see the file comment); E in [0, 2N). The zero cell reads as
// all ones with the returned flag set (then x 2^E = raw + 1 - 2^N = 0).
//
// Output word j of lane l (j = K l + s) is the funnel shift of source words j - q - 1 and
// j - q (q = E' / 32 words, sh = E' mod 32 bits), each complemented when its logical index
// is negative (it wrapped past 2^N = -1). K >= 4: the window is read as 16-byte vectors
// (rot_window). K <= 2: a lane's K + 1 source words cross at most one 32-word row of the padded
// cell (or the end of the cell), so the window is two runs of consecutive addresses, each with
// a lane-uniform complement mask.
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
  auto put = [&](int s, uint32_t w) { r[s] = w; };
  if constexpr (K >= 4)
    rot_window<K>(cell, E, g, put);
  else
    rot_window_scalar<K>(cell, E, g, put);
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
  auto sub = [&](int s, uint32_t w) { asm volatile("subc.cc.u32 %0, %0, %1;" : "+r"(r[s]) : "r"(w)); };
  if (E == 0) {
    const int b = phys<K>(K * g.lane);
#pragma unroll
    for (int s = 0; s < K; s++) sub(s, cell[b + s]);
  } else if constexpr (K >= 4) {
    rot_window<K>(cell, E, g, sub);
  } else {
    rot_window_scalar<K>(cell, E, g, sub);
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
