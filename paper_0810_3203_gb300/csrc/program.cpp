// Host-side generation of on-chip butterfly programs and job images.
//
// A program lists the base-case butterflies that Algorithm 1 (TFT, Sec. 3) or Algorithm 2
// (ITFT, Sec. 4) executes for a sub-transform, in the order the recursion produces them, then
// groups them into dependency levels. The weight is symbolic: every rotation is
// (mul * e + add) mod 2N where e is the weight exponent of the job that runs it.
//
// Any split 1 < L1 < L computes the same outputs (Sec. 2, the decomposition into Eqs. b-cols
// and b-rows); programs use the split that gives the fewest dependency levels. A job spread
// over a cluster of C CTAs takes one more split with L1 = C at its top: column transforms of
// length C in column layout and row transforms of length Ls / C in row layout, in the order of
// Algorithm 1 or 2, with layout exchanges between the phases.
#include <algorithm>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <stdexcept>
#include <tuple>
#include <vector>

#include "common.h"
#include "host.h"

namespace tftgpu {

namespace {

struct SymE {
  int64_t mul, add;  // exponent = mul * e + add (mod 2N)
};

// Emits the base cases of Algorithm 1 / 2 on cell indices base + i * stride.
class ProgGen {
 public:
  // mode RING_SN: the ring is S[y]/(y^{M/2}+1) (twoN = M, omega = y); there 2 is not a power of
  // omega, so the ITFT base case's doublings and halvings become scalar flags (OPS_*) instead of
  // rotations. RING_SQRT2: omega = sqrt2 over Z/(2^N+1) (twoN = 4N), so 2 = omega^2.
  ProgGen(int64_t twoN, int policy, int mode = RING_FERMAT) : twoN_(twoN), policy_(policy), mode_(mode) {}

  std::vector<OpDesc> ops;

  SymE zero() const { return {0, 0}; }
  SymE cst(int64_t a) const { return {0, md(a)}; }
  SymE neg(SymE a) const { return {md(-a.mul), md(-a.add)}; }
  SymE plus(SymE a, int64_t c) const { return {a.mul, md(a.add + c)}; }
  SymE times(SymE a, int64_t c) const { return {md(a.mul * c), md(a.add * c)}; }

  void tft(int base, int stride, int l, SymE E, int64_t z, int64_t n) {
    if (l == 1) {
      int c0 = base, c1 = base + stride;
      if (n == 2 && z == 2) {
        push(OP_BF, c0, c1, OPF_S | OPF_D, zero(), zero(), zero(), E);
      } else if (n == 2 && z == 1) {
        push(OP_TAG, c0, c1, OPF_COPY, zero(), E, zero(), zero());
      } else if (n == 1 && z == 2) {
        push(OP_BF, c0, c1, OPF_S, zero(), zero(), zero(), zero());
      }
      return;
    }
    int l1 = split(l), l2 = l - l1;
    int64_t L = int64_t(1) << l, L1 = int64_t(1) << l1, L2 = int64_t(1) << l2;
    int64_t w = twoN_ / L;
    int64_t n2 = n % L2, n1 = n / L2, n1p = (n + L2 - 1) / L2;
    int64_t z2 = z % L2, z1 = z / L2, z2p = z1 > 0 ? L2 : z2;
    for (int64_t u = 0; u < z2; u++)
      tft(base + int(u) * stride, stride * int(L2), l1, plus(E, u * w), z1 + 1, n1p);
    for (int64_t u = z2; u < z2p; u++)
      tft(base + int(u) * stride, stride * int(L2), l1, plus(E, u * w), z1, n1p);
    SymE Er = times(E, L1);
    for (int64_t u = 0; u < n1; u++) tft(base + int(u * L2) * stride, stride, l2, Er, z2p, L2);
    if (n2 > 0) tft(base + int(n1 * L2) * stride, stride, l2, Er, z2p, n2);
  }

  void itft(int base, int stride, int l, SymE E, int64_t z, int64_t n, int f) {
    if (l == 1) {
      int c0 = base, c1 = base + stride;
      // doubling / halving: 2 = omega and 1/2 = omega^{2N-1} over Z/(2^N+1); scalar flags
      // over S[y]/(y^{M/2}+1)
      const bool sn = mode_ == RING_SN;
      const int64_t u = mode_ == RING_SQRT2 ? 2 : 1;  // the exponent of 2 in powers of omega
      const SymE two = sn ? zero() : cst(u), half = sn ? zero() : cst(twoN_ - u);
      const uint16_t a2 = sn ? OPS_A_DOUBLE : 0, ah = sn ? OPS_A_HALVE : 0, sh = sn ? OPS_S_HALVE : 0;
      if (n == 2) {
        push(OP_BF, c0, c1, OPF_S | OPF_D, zero(), neg(E), zero(), zero());
      } else if (n == 1 && f == 1 && z == 2) {
        push(OP_CROSS, c0, c1, 0, zero(), zero(), zero(), E);
      } else if (n == 1 && f == 1 && z == 1) {
        push(OP_TAG, c0, c1, OPF_COPY, two, E, zero(), zero(), a2);
      } else if (n == 1 && f == 0 && z == 2) {
        push(OP_BF, c0, c1, OPF_D | OPF_D_TO_I, two, zero(), zero(), zero(), a2);
      } else if (n == 1 && f == 0 && z == 1) {
        push(OP_TAG, c0, c0, 0, two, zero(), zero(), zero(), a2);
      } else if (n == 0 && z == 2) {
        push(OP_BF, c0, c1, OPF_S, zero(), zero(), half, zero(), sh);
      } else if (n == 0 && z == 1) {
        push(OP_TAG, c0, c0, 0, half, zero(), zero(), zero(), ah);
      }
      return;
    }
    int l1 = split(l), l2 = l - l1;
    int64_t L = int64_t(1) << l, L1 = int64_t(1) << l1, L2 = int64_t(1) << l2;
    int64_t w = twoN_ / L;
    int64_t n2 = n % L2, n1 = n / L2, z2 = z % L2, z1 = z / L2;
    int fp = (n2 + f > 0) ? 1 : 0;
    int64_t z2p = z1 > 0 ? L2 : z2;
    int64_t m = std::min(n2, z2), mp = std::max(n2, z2);
    SymE Er = times(E, L1);
    int cs = stride * int(L2);
    for (int64_t u = 0; u < n1; u++) itft(base + int(u * L2) * stride, stride, l2, Er, L2, L2, 0);
    for (int64_t u = n2; u < mp; u++) itft(base + int(u) * stride, cs, l1, plus(E, u * w), z1 + 1, n1, fp);
    for (int64_t u = mp; u < z2p; u++) itft(base + int(u) * stride, cs, l1, plus(E, u * w), z1, n1, fp);
    if (fp) itft(base + int(n1 * L2) * stride, stride, l2, Er, z2p, n2, f);
    for (int64_t u = 0; u < m; u++) itft(base + int(u) * stride, cs, l1, plus(E, u * w), z1 + 1, n1 + 1, 0);
    for (int64_t u = m; u < n2; u++) itft(base + int(u) * stride, cs, l1, plus(E, u * w), z1, n1 + 1, 0);
  }

 private:
  int64_t twoN_;
  int policy_;
  int mode_;

  int split(int l) const { return policy_ == 0 ? 1 : l / 2; }
  int64_t md(int64_t a) const {
    int64_t r = a % twoN_;
    return r < 0 ? r + twoN_ : r;
  }
  RotA ra(SymE a) const { return RotA{int32_t(a.mul), int32_t(a.add)}; }

  void push(uint8_t kind, int i, int j, uint8_t flags, SymE r_a, SymE r_b, SymE p0, SymE p1, uint16_t scal = 0) {
    OpDesc o;
    std::memset(&o, 0, sizeof o);
    o.i = uint16_t(i);
    o.j = uint16_t(j);
    o.kind = kind;
    o.flags = flags;
    o.pad = scal;
    o.ra = ra(r_a);
    o.rb = ra(r_b);
    o.p0 = ra(p0);
    o.p1 = ra(p1);
    ops.push_back(o);
  }
};

// group ops into levels: an op goes one level after the last op that touched one of its cells
std::vector<uint32_t> level_and_pack(const std::vector<OpDesc> &ops, int nslots, int *nlevels_out) {
  std::vector<int> last(nslots, -1), lvl(ops.size());
  int nlev = 0;
  for (size_t k = 0; k < ops.size(); k++) {
    const OpDesc &o = ops[k];
    int a = last[o.i], b = (o.j != o.i) ? last[o.j] : -1;
    int v = std::max(a, b) + 1;
    lvl[k] = v;
    last[o.i] = v;
    last[o.j] = v;
    nlev = std::max(nlev, v + 1);
  }
  std::vector<std::vector<int>> byl(nlev);
  for (size_t k = 0; k < ops.size(); k++) byl[lvl[k]].push_back(int(k));
  int off = prog_ops_offset_words(nlev);
  std::vector<uint32_t> img(off + ops.size() * (sizeof(OpDesc) / 4), 0);
  img[0] = uint32_t(nlev);
  img[1] = uint32_t(ops.size());
  uint32_t start = 0;
  OpDesc *dst = reinterpret_cast<OpDesc *>(img.data() + off);
  size_t w = 0;
  for (int v = 0; v < nlev; v++) {
    img[2 + v] = start;
    for (int k : byl[v]) dst[w++] = ops[k];
    start += uint32_t(byl[v].size());
  }
  img[2 + nlev] = start;
  *nlevels_out = nlev;
  return img;
}

// Generate with both split policies (through `emit`) and keep the image with fewer levels.
// `slot` maps a generated cell index to the local slot of the CTA that runs the program.
std::vector<uint32_t> best_program(int64_t twoN, int nslots, const std::function<void(ProgGen &)> &emit,
                                   const std::function<int(int)> &slot, ProgramStats *stats, int mode = RING_FERMAT) {
  std::vector<uint32_t> best;
  int best_lev = -1;
  for (int policy = 0; policy < 2; policy++) {
    ProgGen g(twoN, policy, mode);
    emit(g);
    if (g.ops.empty()) return {};
    for (OpDesc &o : g.ops) {
      o.i = uint16_t(slot(o.i));
      o.j = uint16_t(slot(o.j));
    }
    int nlev = 0;
    std::vector<uint32_t> img = level_and_pack(g.ops, nslots, &nlev);
    if (best_lev < 0 || nlev < best_lev) {
      best_lev = nlev;
      best = std::move(img);
    }
  }
  if (stats) {
    stats->nlevels += best_lev;
    stats->nops += int(best[1]);
  }
  return best;
}

}  // namespace

std::vector<uint32_t> build_program(int kind, int ls, int64_t z, int64_t n, int f, int64_t N,
                                    ProgramStats *stats, int mode) {
  const int64_t twoN = omega_order(N, mode);
  auto emit = [&](ProgGen &g) {
    if (kind == KIND_TFT)
      g.tft(0, 1, ls, {1, 0}, z, n);
    else
      g.itft(0, 1, ls, {1, 0}, z, n, f);
  };
  return best_program(twoN, 1 << ls, emit, [](int c) { return c; }, stats, mode);
}

std::vector<uint32_t> build_job_image(int kind, int ls, int lc, int64_t z, int64_t n, int f, int64_t N,
                                      ProgramStats *stats, int mode) {
  const int64_t twoN = omega_order(N, mode);
  const int C = 1 << lc;
  struct Stage {
    uint32_t type, arg;
    std::vector<std::vector<uint32_t>> progs;  // per CTA (empty: nothing to run)
  };
  std::vector<Stage> stages;
  uint32_t load_layout = LAYOUT_ROW, store_layout = LAYOUT_ROW;
  if (lc == 0) {
    Stage s{STAGE_PROG, 0, {build_program(kind, ls, z, n, f, N, stats, mode)}};
    stages.push_back(std::move(s));
  } else {
    const int l2 = ls - lc;
    const int64_t L2 = int64_t(1) << l2, Ls = int64_t(1) << ls, b = L2 / C;
    const int64_t w = twoN / Ls;
    const int nslots = int(Ls / C);
    // cell -> slot in row layout (CTA r holds cells r L2 + k at slot k)
    auto row_slot = [=](int cell) { return int(cell % L2); };
    // cell -> slot in column layout (CTA c holds cell j L2 + c b + i at slot j b + i)
    auto col_slot = [=](int cell) { return int((cell / L2) * b + (cell % L2) % b); };
    auto prog_stage = [&](const std::function<void(ProgGen &, int)> &emit, bool cols) {
      Stage s{STAGE_PROG, 0, {}};
      for (int c = 0; c < C; c++) {
        auto e = [&](ProgGen &g) { emit(g, c); };
        s.progs.push_back(best_program(twoN, nslots, e, cols ? std::function<int(int)>(col_slot)
                                                              : std::function<int(int)>(row_slot),
                                       stats, mode));
      }
      stages.push_back(std::move(s));
    };
    auto xchg = [&](uint32_t type, uint32_t arg) {
      Stage s{type, arg, std::vector<std::vector<uint32_t>>(C)};
      stages.push_back(std::move(s));
    };
    if (kind == KIND_TFT) {
      const int64_t n2 = n % L2, n1 = n / L2, n1p = (n + L2 - 1) / L2;
      const int64_t z2 = z % L2, z1 = z / L2, z2p = z1 > 0 ? L2 : z2;
      load_layout = LAYOUT_COL;
      store_layout = LAYOUT_ROW;
      prog_stage([&](ProgGen &g, int c) {
        for (int64_t u = c * b; u < std::min<int64_t>((c + 1) * b, z2p); u++)
          g.tft(int(u), int(L2), lc, g.plus({1, 0}, u * w), u < z2 ? z1 + 1 : z1, n1p);
      }, true);
      xchg(STAGE_XCHG, 0);
      prog_stage([&](ProgGen &g, int c) {
        if (c < n1p) g.tft(int(c * L2), 1, l2, g.times({1, 0}, C), z2p, c < n1 ? L2 : n2);
      }, false);
    } else {
      const int64_t n2 = n % L2, n1 = n / L2, z2 = z % L2, z1 = z / L2;
      const int fp = (n2 + f > 0) ? 1 : 0;
      const int64_t z2p = z1 > 0 ? L2 : z2;
      const int64_t m = std::min(n2, z2), mp = std::max(n2, z2);
      load_layout = LAYOUT_ROW;
      store_layout = LAYOUT_COL;
      prog_stage([&](ProgGen &g, int c) {
        if (c < n1) g.itft(int(c * L2), 1, l2, g.times({1, 0}, C), L2, L2, 0);
      }, false);
      xchg(STAGE_XCHG, 0);
      prog_stage([&](ProgGen &g, int c) {
        for (int64_t u = std::max<int64_t>(n2, c * b); u < std::min<int64_t>(z2p, (c + 1) * b); u++)
          g.itft(int(u), int(L2), lc, g.plus({1, 0}, u * w), u < mp ? z1 + 1 : z1, n1, fp);
      }, true);
      if (fp) {
        xchg(STAGE_SWAP, uint32_t(n1));
        prog_stage([&](ProgGen &g, int c) {
          if (c == n1) g.itft(int(c * L2), 1, l2, g.times({1, 0}, C), z2p, n2, f);
        }, false);
        xchg(STAGE_SWAP, uint32_t(n1));
      }
      prog_stage([&](ProgGen &g, int c) {
        for (int64_t u = c * b; u < std::min<int64_t>(n2, (c + 1) * b); u++)
          g.itft(int(u), int(L2), lc, g.plus({1, 0}, u * w), u < m ? z1 + 1 : z1, n1 + 1, 0);
      }, true);
    }
  }
  // assemble: header, stage table, program images
  const int sw = job_stage_words(C);
  std::vector<uint32_t> img(job_header_words() + stages.size() * sw, 0);
  img[0] = uint32_t(stages.size());
  img[1] = uint32_t(C);
  img[2] = load_layout;
  img[3] = store_layout;
  for (size_t s = 0; s < stages.size(); s++) {
    uint32_t *e = &img[job_header_words() + s * sw];
    e[0] = stages[s].type;
    e[1] = stages[s].arg;
  }
  for (size_t s = 0; s < stages.size(); s++) {
    for (int c = 0; c < int(stages[s].progs.size()); c++) {
      const std::vector<uint32_t> &p = stages[s].progs[c];
      if (p.empty()) continue;
      if (img.size() & 1) img.push_back(0);
      uint32_t off = uint32_t(img.size());
      img.insert(img.end(), p.begin(), p.end());
      img[job_header_words() + s * sw + 2 + c] = off;
    }
  }
  return img;
}

int image_max_program_words(const std::vector<uint32_t> &img) {
  const int nst = int(img[0]), C = int(img[1]);
  int best = 0;
  for (int s = 0; s < nst; s++) {
    const uint32_t *e = &img[job_header_words() + s * job_stage_words(C)];
    if (e[0] != STAGE_PROG) continue;
    for (int c = 0; c < C; c++) {
      const uint32_t off = e[2 + c];
      if (!off) continue;
      const int words = prog_ops_offset_words(int(img[off])) + int(img[off + 1]) * int(sizeof(OpDesc) / 4);
      best = std::max(best, words);
    }
  }
  return best;
}

}  // namespace tftgpu
