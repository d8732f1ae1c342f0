// Batched Z[x] products (zx_mul_batch): many independent products of uneven lengths and rings.
//
// Products are sorted by ring size N and cut into sub-batches whose ring buffers fit a memory
// budget. Inside a sub-batch the products of one ring form a group that runs as one sequence
// of launches: one pack launch for every operand of the group, then pass k of every
// operand's TFT plan (Algorithm 1 over global memory) as the jobs of shared launches, one
// pointwise launch, pass k of every product's ITFT plan (Algorithm 2), and one lift launch.
// A short product thus fills SMs next to long ones instead of paying a launch sequence of its
// own. Groups of different rings run on forked streams so that they overlap too.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/tftgpu.h"
#include "common.h"
#include "host.h"

namespace tftgpu {

namespace {

constexpr int kForkStreams = 4;
constexpr size_t kGroupProducts = 96;  // products per group at most

struct DeviceStreams {
  bool ready = false;
  cudaStream_t s[kForkStreams] = {};
};

std::mutex g_batch_mu;  // guards the fork streams while a call enqueues its work

DeviceStreams &fork_streams(int dev) {
  static DeviceStreams per_dev[64];
  return per_dev[dev & 63];
}

// Byte image of the descriptors a sub-batch uploads in one copy.
struct DescImage {
  std::vector<unsigned char> bytes;
  size_t add(const void *p, size_t n) {
    size_t off = (bytes.size() + 15) & ~size_t(15);
    bytes.resize(off + n);
    if (n) std::memcpy(bytes.data() + off, p, n);
    return off;
  }
};

// Launches of many transforms over one ring buffer pool, merged by (pass, ls, lc): each
// product's transform uses its cached plan (job lists stay in device memory), and a merged
// launch is a table of segments, one per product launch, with the product's cell offset.
struct MergedSegs {
  struct Acc {
    std::vector<Segment> segs;
    int nwarps = 0, prog_words = 0, ctas = 0, njobs = 0;
  };
  std::map<std::tuple<int, int, int>, Acc> m;
  int add(int kind, int l, int64_t z, int64_t n, int64_t N, int64_t stride, int64_t cell_off, int scale, int mode) {
    int err = ZX_OK;
    const TransformPlan *p = get_transform_plan(kind, l, z, n, 0, N, 0, stride, scale, &err, mode);
    if (!p) return err ? err : ZX_ECUDA;
    for (const Launch &L : p->launches) {
      Acc &a = m[std::make_tuple(L.pass, L.ls, L.lc)];
      a.segs.push_back(Segment{L.d_jobs, cell_off, int32_t(L.njobs), int32_t(a.ctas)});
      a.ctas += L.njobs << L.lc;
      a.njobs += L.njobs;
      a.nwarps = L.nwarps;
      a.prog_words = std::max(a.prog_words, L.prog_words);
    }
    return ZX_OK;
  }
};

void to_launches(const MergedSegs &m, DescImage *img, std::vector<Launch> *out) {
  for (const auto &kv : m.m) {
    const MergedSegs::Acc &a = kv.second;
    Launch L;
    L.pass = std::get<0>(kv.first);
    L.ls = std::get<1>(kv.first);
    L.lc = std::get<2>(kv.first);
    L.nwarps = a.nwarps;
    L.njobs = a.njobs;
    L.prog_words = a.prog_words;
    L.d_jobs = nullptr;
    L.nsegs = int(a.segs.size());
    L.d_segs = reinterpret_cast<const Segment *>(img->add(a.segs.data(), a.segs.size() * sizeof(Segment)));
    out->push_back(L);
  }
}

template <class T>
const T *rebase(const T *off, unsigned char *base) {
  return reinterpret_cast<const T *>(base + reinterpret_cast<size_t>(off));
}

}  // namespace

size_t product_pool_bytes(const BatchProduct &p) { return 2 * size_t(p.stride) * 8 * (size_t(1) << p.l); }

int layout_batch(const std::vector<BatchProduct> &items, const std::vector<int> &idx_in,
                 std::vector<unsigned char> *desc, BatchLayout *out, std::string *msg) {
  std::vector<int> idx(idx_in);
  // by ring (size, then omega), largest rings first, then by transform length
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
    if (items[a].N != items[b].N) return items[a].N > items[b].N;
    if (items[a].mode != items[b].mode) return items[a].mode < items[b].mode;
    return items[a].l > items[b].l;
  });
  DescImage img;
  img.bytes.swap(*desc);
  out->groups.clear();
  int64_t cell_off = 0;  // in cells of the current group's stride, from the pool's start
  size_t byte_off = 0;
  // the products of one ring, dealt round-robin into groups of at most kGroupProducts, so that
  // a ring with many products runs as several groups on the forked streams (one group's
  // pointwise products then overlap another's transforms)
  std::vector<std::vector<int>> subs;
  for (size_t a = 0; a < idx.size();) {
    size_t b = a;
    while (b < idx.size() && items[idx[b]].N == items[idx[a]].N && items[idx[b]].mode == items[idx[a]].mode) b++;
    const size_t ng = (b - a + kGroupProducts - 1) / kGroupProducts;
    for (size_t g = 0; g < ng; g++) {
      subs.emplace_back();
      for (size_t t = a + g; t < b; t += ng) subs.back().push_back(idx[t]);
    }
    a = b;
  }
  for (const std::vector<int> &sub : subs) {
    BatchGroup gd;
    const BatchProduct &p0 = items[sub[0]];
    gd.ring = make_ring(p0.N);
    gd.mode = p0.mode;
    gd.stride = p0.stride;
    gd.count = int(sub.size());
    std::vector<PackItem> pk;
    std::vector<PointwiseItem> pw;
    std::vector<LiftItem> lf;
    MergedSegs mt, mi;
    const size_t cell_bytes = size_t(gd.stride) * 8;
    cell_off = int64_t((byte_off + cell_bytes - 1) / cell_bytes);  // first whole cell after the last group
    for (size_t t = 0; t < sub.size(); t++) {
      const BatchProduct &p = items[sub[t]];
      const int64_t L = int64_t(1) << p.l;
      const int64_t cf = cell_off, cg = cell_off + L;
      cell_off += 2 * L;
      const int64_t F = cf * p.stride, G = cg * p.stride;  // limb offsets in the pool
      pk.push_back(PackItem{p.f, F, p.len_f, p.limbs_f, p.signed_f, 0});
      pk.push_back(PackItem{p.g, G, p.len_g, p.limbs_g, p.signed_g, 0});
      pw.push_back(PointwiseItem{F, G, p.nf, gd.pw_total});
      gd.pw_total += p.nf;
      lf.push_back(LiftItem{F, p.h, p.n, p.limbs_h, p.sgn, 0});
      gd.max_len = std::max(gd.max_len, std::max(p.len_f, p.len_g));
      gd.max_n = std::max(gd.max_n, p.nf);
      int rc;
      if ((rc = mt.add(KIND_TFT, p.l, p.len_f, p.nf, p.N, p.stride, cf, 0, p.mode)) ||
          (rc = mt.add(KIND_TFT, p.l, p.len_g, p.nf, p.N, p.stride, cg, 0, p.mode)) ||
          (rc = mi.add(KIND_ITFT, p.l, p.nf, p.nf, p.N, p.stride, cf, 1, p.mode))) {
        *msg = "planning failed for product " + std::to_string(sub[t]);
        img.bytes.swap(*desc);
        return rc;
      }
    }
    byte_off = size_t(cell_off) * cell_bytes;
    gd.cell_end = cell_off;
    gd.pack_off = img.add(pk.data(), pk.size() * sizeof(PackItem));
    gd.pw_off = img.add(pw.data(), pw.size() * sizeof(PointwiseItem));
    gd.lift_off = img.add(lf.data(), lf.size() * sizeof(LiftItem));
    to_launches(mt, &img, &gd.tft);
    to_launches(mi, &img, &gd.itft);
    out->groups.push_back(std::move(gd));
  }
  out->pool_bytes = byte_off;
  img.bytes.swap(*desc);
  return ZX_OK;
}

cudaError_t enqueue_group(const BatchGroup &gd, unsigned char *d_desc, unsigned char *pool, cudaStream_t s) {
  uint64_t *x = reinterpret_cast<uint64_t *>(pool);
  TransformPlan tp, ip;
  tp.ring = ip.ring = gd.ring;
  tp.mode = ip.mode = gd.mode;
  // the merged launches touch the group's cells only; tensor copies as the ring's configuration says
  tp.cell_extent = ip.cell_extent = gd.cell_end;
  tp.tma = ip.tma = plan_config(gd.ring.N).tma != 0;
  for (Launch L : gd.tft) {
    L.d_segs = rebase(L.d_segs, d_desc);
    tp.launches.push_back(L);
  }
  for (Launch L : gd.itft) {
    L.d_segs = rebase(L.d_segs, d_desc);
    ip.launches.push_back(L);
  }
  const PackItem *pk = reinterpret_cast<const PackItem *>(d_desc + gd.pack_off);
  const PointwiseItem *pw = reinterpret_cast<const PointwiseItem *>(d_desc + gd.pw_off);
  const LiftItem *lf = reinterpret_cast<const LiftItem *>(d_desc + gd.lift_off);
  cudaError_t ce;
  if ((ce = launch_pack_batch(pk, 2 * gd.count, gd.max_len, gd.stride, gd.ring, x, s)) != cudaSuccess) return ce;
  if ((ce = run_transform(tp, x, gd.stride, s)) != cudaSuccess) return ce;
  if ((ce = launch_pointwise_batch(pw, gd.count, gd.pw_total, gd.stride, gd.ring, x, s)) != cudaSuccess) return ce;
  if ((ce = run_transform(ip, x, gd.stride, s)) != cudaSuccess) return ce;
  return launch_lift_batch(lf, gd.count, gd.max_n, gd.stride, gd.ring, x, s);
}

int run_mul_batch(const std::vector<BatchProduct> &items, cudaStream_t s, std::string *msg) {
  if (items.empty()) return ZX_OK;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    *msg = "cudaMemGetInfo failed";
    return ZX_ECUDA;
  }
  const size_t budget = free_b / 2;
  // cut into sub-batches under the memory budget, largest rings first
  std::vector<int> order(items.size());
  for (size_t i = 0; i < order.size(); i++) order[i] = int(i);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (items[a].N != items[b].N) return items[a].N > items[b].N;
    return items[a].l > items[b].l;
  });
  std::vector<std::vector<int>> parts(1);
  size_t acc = 0;
  for (int i : order) {
    const size_t need = product_pool_bytes(items[i]);
    if (!parts.back().empty() && acc + need > budget) {
      parts.emplace_back();
      acc = 0;
    }
    parts.back().push_back(i);
    acc += need;
  }
  std::vector<unsigned char> desc;
  std::vector<BatchLayout> lays(parts.size());
  for (size_t k = 0; k < parts.size(); k++) {
    int rc = layout_batch(items, parts[k], &desc, &lays[k], msg);
    if (rc) return rc;
  }

  std::lock_guard<std::mutex> lk(g_batch_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  DeviceStreams &fs = fork_streams(dev);
  if (!fs.ready) {
    for (int k = 0; k < kForkStreams; k++)
      if (cudaStreamCreateWithFlags(&fs.s[k], cudaStreamNonBlocking) != cudaSuccess) {
        *msg = "stream creation failed";
        return ZX_ECUDA;
      }
    fs.ready = true;
  }
  unsigned char *d_desc = nullptr;
  cudaError_t ce = cudaMallocAsync(reinterpret_cast<void **>(&d_desc), desc.size(), s);
  if (ce != cudaSuccess) {
    *msg = "descriptor allocation failed";
    return ZX_ENOMEM;
  }
  ce = cudaMemcpyAsync(d_desc, desc.data(), desc.size(), cudaMemcpyHostToDevice, s);
  if (ce != cudaSuccess) {
    cudaFreeAsync(d_desc, s);
    *msg = std::string("descriptor upload: ") + cudaGetErrorString(ce);
    return ZX_ECUDA;
  }
  int rc = ZX_OK;
  std::vector<cudaEvent_t> events;
  auto new_event = [&](cudaEvent_t *ev) {
    if (cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess) return false;
    events.push_back(*ev);
    return true;
  };
  for (const BatchLayout &lay : lays) {
    unsigned char *pool = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&pool), lay.pool_bytes, s) != cudaSuccess) {
      *msg = "ring buffer pool of " + std::to_string(lay.pool_bytes) + " bytes";
      rc = ZX_ENOMEM;
      break;
    }
    const bool fork = lay.groups.size() > 1;
    const int nstreams = std::min<int>(kForkStreams, int(lay.groups.size()));
    if (fork) {
      cudaEvent_t ev;
      if (!new_event(&ev) || cudaEventRecord(ev, s) != cudaSuccess) {
        cudaFreeAsync(pool, s);
        *msg = "event record failed";
        rc = ZX_ECUDA;
        break;
      }
      for (int k = 0; k < nstreams; k++) cudaStreamWaitEvent(fs.s[k], ev, 0);
    }
    for (size_t gi = 0; gi < lay.groups.size() && rc == ZX_OK; gi++) {
      cudaStream_t gs = fork ? fs.s[gi % kForkStreams] : s;
      if ((ce = enqueue_group(lay.groups[gi], d_desc, pool, gs)) != cudaSuccess) {
        *msg = std::string("batch launch: ") + cudaGetErrorString(ce);
        rc = ZX_ECUDA;
      }
    }
    if (fork) {
      for (int k = 0; k < nstreams; k++) {
        cudaEvent_t join;
        if (!new_event(&join)) {
          rc = ZX_ECUDA;
          break;
        }
        cudaEventRecord(join, fs.s[k]);
        cudaStreamWaitEvent(s, join, 0);
      }
    }
    cudaFreeAsync(pool, s);
    if (rc) break;
  }
  cudaFreeAsync(d_desc, s);
  for (cudaEvent_t ev : events) cudaEventDestroy(ev);
  return rc;
}

}  // namespace tftgpu
