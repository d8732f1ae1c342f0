// Transform planning: Algorithms 1 and 2 applied at the level of global memory.
//
// A transform of length L = 2^l whose cells fit in the shared memory of one CTA, or of a
// cluster of up to 8 CTAs, is a single job. Otherwise the array is viewed as an L1 x L2 matrix
// (L1 = 2^floor(l/2), L2 = 2^ceil(l/2), the paper's split) and the column and row
// sub-transforms are planned recursively, exactly in the order of Algorithm 1 (columns, then
// rows) or Algorithm 2 (full rows, rightmost columns, last row, leftmost columns). Each
// recursion level is one pass over global memory; all sub-transforms of a pass are
// independent and become the jobs of one kernel launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <tuple>
#include <vector>

#include "../../include/tftgpu.h"
#include "common.h"
#include "host.h"

namespace tftgpu {

bool ring_supported(int64_t N) {
  if (N < 64 || N % 64 != 0) return false;
  if (N <= 1024) return true;
  return N % 1024 == 0 && N <= 32768;
}

Ring make_ring(int64_t N) {
  Ring r;
  r.N = N;
  r.NW = int(N / 32);
  r.K = words_per_lane(r.NW);
  r.G = r.NW / r.K;
  r.pitch = cell_pitch_words(r.NW);
  return r;
}

static const size_t kSmemBudget = 200 * 1024;

int max_onchip_ls(const Ring &r) {
  int ls = 1;
  while (ls < 16 && size_t(2 << ls) * (size_t(r.pitch) + 1) * 4 <= kSmemBudget) ls++;
  return ls;
}

int cluster_cta_ls(const Ring &r) {
  int ls = 1;
  while (ls < 16 && size_t(2 << ls) * (size_t(r.pitch) + 1) * 4 <= kSmemBudget / 2) ls++;
  return ls;
}

// Default: the largest single-CTA job the shared memory allows, eight cells per CTA of a cluster
// job, up to sixteen warps per CTA, the paper's split. Measured on GB300 (zx_tune): small
// clusters and CTAs that three or more share an SM beat fewer, larger jobs with fewer passes,
// because a job's time is set by the latency of its dependency levels.
PlanConfig default_config(const Ring &r) {
  PlanConfig c;
  c.ls_max = max_onchip_ls(r);
  c.ls_c = std::min(3, cluster_cta_ls(r));
  // up to 16 warps per CTA; a launch with enough CTAs to fill the SMs three deep runs jobs
  // that fit three to an SM with 8 (launch_k)
  c.max_warps = 16;
  c.split = 0;
  return c;
}

bool config_valid(const Ring &r, const PlanConfig &c) {
  auto fits = [&](int ls) { return ls >= 1 && ls <= 16 && size_t(1) << ls <= 65536 &&
                                   (size_t(1) << ls) * (size_t(r.pitch) + 1) * 4 <= kSmemBudget; };
  return fits(c.ls_max) && fits(c.ls_c) && c.ls_c <= c.ls_max + 1 && (c.max_warps == 8 || c.max_warps == 16) &&
         (c.split >= 0 && c.split <= 2) && (c.fused >= FUSED_NONE && c.fused <= FUSED_DIRECT) && c.max_lc >= 0 &&
         c.max_lc <= kMaxClusterLog2 && (c.tma == 0 || c.tma == 1);
}

namespace {

std::mutex g_config_mu;
std::map<int64_t, PlanConfig> &config_table() {
  static std::map<int64_t, PlanConfig> *t = new std::map<int64_t, PlanConfig>();
  return *t;
}

}  // namespace

PlanConfig plan_config(int64_t N) {
  std::lock_guard<std::mutex> lk(g_config_mu);
  auto it = config_table().find(N);
  return it != config_table().end() ? it->second : default_config(make_ring(N));
}

void set_plan_config(int64_t N, const PlanConfig &c) {
  std::lock_guard<std::mutex> lk(g_config_mu);
  config_table()[N] = c;
}

int warps_for_job(int ls, int lc, int max_warps) {
  const int nslots = 1 << (ls - lc);
  return std::max(1, std::min(max_warps, nslots / 2));
}



namespace {

int64_t md(int64_t a, int64_t m) {
  int64_t r = a % m;
  return r < 0 ? r + m : r;
}

// Device memory of the plan caches (job lists, job images, persistent schedules). Plans are made
// while other streams run (a serving loop plans each new product shape as it arrives), and a
// device allocation or a copy on the legacy default stream between two launches of different
// streams keeps those launches from overlapping. So plans take their memory from chunks
// allocated ahead (64 MiB at a time per device; the caches keep every plan, so nothing is
// freed) and upload on a non-blocking stream of their own, synchronising only that stream.
struct PlanMemory {
  std::mutex mu;
  struct Chunk {
    unsigned char *base = nullptr;
    size_t size = 0, used = 0;
  };
  std::map<int, Chunk> chunk;         // per device: the chunk plans are taken from
  std::map<int, cudaStream_t> stream;  // per device: the upload stream
};

PlanMemory &plan_memory() {
  static PlanMemory *m = new PlanMemory();
  return *m;
}

// 256-byte aligned device memory for a cached plan; nullptr when the device has none left
void *plan_alloc(size_t bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  PlanMemory &pm = plan_memory();
  std::lock_guard<std::mutex> lk(pm.mu);
  PlanMemory::Chunk &c = pm.chunk[dev];
  bytes = std::max<size_t>(256, (bytes + 255) & ~size_t(255));
  if (!c.base || c.used + bytes > c.size) {
    const size_t size = std::max<size_t>(size_t(64) << 20, bytes);
    unsigned char *p = nullptr;
    if (cudaMalloc(reinterpret_cast<void **>(&p), size) != cudaSuccess) return nullptr;
    c = PlanMemory::Chunk{p, size, 0};  // the previous chunk keeps the plans it holds
  }
  void *r = c.base + c.used;
  c.used += bytes;
  return r;
}

// Host -> device copy of a plan on the upload stream; returns when the copy has landed.
cudaError_t plan_upload(void *dst, const void *src, size_t bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  PlanMemory &pm = plan_memory();
  cudaStream_t s = nullptr;
  {
    std::lock_guard<std::mutex> lk(pm.mu);
    auto it = pm.stream.find(dev);
    if (it == pm.stream.end()) {
      const cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
      pm.stream[dev] = s;
    } else {
      s = it->second;
    }
  }
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

// device copies of job images, keyed by (device, kind, ls, lc, z, n, f, N)
struct ImageCache {
  std::mutex mu;
  std::map<std::tuple<int, int, int, int, int64_t, int64_t, int, int64_t, int>, uint32_t *> images;
  std::map<const uint32_t *, int> prog_words;  // largest per-CTA program of each image

  int max_prog(const uint32_t *d) {
    std::lock_guard<std::mutex> lk(mu);
    auto it = prog_words.find(d);
    return it == prog_words.end() ? 0 : it->second;
  }

  const uint32_t *get(int kind, int ls, int lc, int64_t z, int64_t n, int f, int64_t N, int *err,
                      int mode = RING_FERMAT) {
    int dev = 0;
    cudaGetDevice(&dev);
    auto key = std::make_tuple(dev, kind, ls, lc, z, n, f, N, mode);
    std::lock_guard<std::mutex> lk(mu);
    auto it = images.find(key);
    if (it != images.end()) return it->second;
    std::vector<uint32_t> img = build_job_image(kind, ls, lc, z, n, f, N, nullptr, mode);
    uint32_t *d = static_cast<uint32_t *>(plan_alloc(img.size() * 4));
    if (!d) {
      *err = ZX_ENOMEM;
      return nullptr;
    }
    if (plan_upload(d, img.data(), img.size() * 4) != cudaSuccess) {
      *err = ZX_ECUDA;
      return nullptr;
    }
    images[key] = d;
    prog_words[d] = image_max_program_words(img);
    return d;
  }
};

ImageCache &image_cache() {
  static ImageCache *c = new ImageCache();
  return *c;
}

struct JobRec {
  int pass;
  int ls;
  int lc;
  int kind;
  int64_t z, n;
  int f;
  JobDesc d;
};

// Job lists and the planner's scratch arrays run to hundreds of kilobytes; allocated afresh for
// every plan, their pages fault in again each time (most of a plan's host time). Each thread
// keeps its largest buffers for the next plan instead.
thread_local std::vector<JobRec> t_jobs_spare, t_jobs_sorted;
thread_local std::vector<int32_t> t_cells_scratch;

struct Planner {
  Ring ring;
  int64_t twoN;
  int ls_max;  // largest job held by one CTA
  int ls_c;    // cells (log2) per CTA of a cluster job
  int split;   // 0: L1 = 2^floor(l/2) (the paper's split), 1: L1 = 2^ceil(l/2)
  PlanConfig cfg;
  std::vector<JobRec> jobs;

  int mode;   // RingMode: twoN is the order of omega (2N, or 4N for sqrt2)

  explicit Planner(int64_t N, const PlanConfig *c = nullptr, int mode_ = RING_FERMAT) {
    ring = make_ring(N);
    mode = mode_;
    twoN = omega_order(N, mode_);
    cfg = c ? *c : plan_config(N);
    ls_max = cfg.ls_max;
    ls_c = cfg.ls_c;
    split = cfg.split;
    jobs.swap(t_jobs_spare);
    jobs.clear();
  }
  ~Planner() {
    if (jobs.capacity() > t_jobs_spare.capacity()) jobs.swap(t_jobs_spare);
  }
  Planner(const Planner &) = delete;
  Planner &operator=(const Planner &) = delete;
  int top_l1(int l) const {
    if (split == 2) return fewest_pass_l1(l);
    return split ? l - l / 2 : l / 2;
  }

  // single CTA up to ls_max; a cluster of up to 2^max_lc CTAs of 2^ls_c cells above that, as
  // long as every CTA row of the job's split holds at least one cell per CTA (2 lc <= l)
  int cluster_log2(int l) const { return l <= ls_max ? 0 : l - ls_c; }
  bool leaf_below_top(int l) const {
    const int lc = cluster_log2(l);
    return lc == 0 || (lc > 0 && lc <= cfg.max_lc && 2 * lc <= l);
  }
  bool leaf(int l) const {
    // a whole transform of more than 64 cells takes the two-pass split: as one job it would run
    // on a single CTA (one SM) for l levels, as two passes its jobs spread over the SMs
    if (whole_split && depth == 0 && l > kTopSingleJobMax) return false;
    return leaf_below_top(l);
  }
  // global-memory passes of a sub-transform of 2^l cells below the top under split 2, and the
  // split that achieves them (memoised; l <= 30)
  int min_passes(int l) const {
    if (l <= 1 || leaf_below_top(l)) return 1;
    if (memo_passes[l]) return memo_passes[l];
    int best = 1 << 20;
    for (int l1 = 1; l1 < l; l1++) best = std::min(best, min_passes(l1) + min_passes(l - l1));
    memo_passes[l] = best;
    return best;
  }
  int fewest_pass_l1(int l) const {
    int best = -1, bp = 1 << 20;
    for (int l1 = 1; l1 < l; l1++) {
      const int p = min_passes(l1) + min_passes(l - l1);
      // ties: nearest to the balanced split l / 2, then the smaller column length
      if (p < bp || (p == bp && std::abs(2 * l1 - l) < std::abs(2 * best - l))) {
        bp = p;
        best = l1;
      }
    }
    return best;
  }
  mutable int memo_passes[32] = {0};
  static constexpr int kTopSingleJobMax = 6;
  bool whole_split = true;  // false for plans that run on many sequences at once
  int depth = 0;  // recursion depth of the current tft / itft call (0: the whole transform)

  void job(int pass, int kind, int64_t cell0, int64_t ms, int l, int64_t e, int64_t z, int64_t n,
           int f, int64_t nscale, int64_t escale) {
    JobRec j;
    std::memset(&j, 0, sizeof j);
    j.pass = pass;
    j.ls = l;
    j.lc = cluster_log2(l);
    j.kind = kind;
    j.z = z;
    j.n = n;
    j.f = f;
    j.d.cell0 = cell0;
    j.d.mstride = ms;
    j.d.e = int32_t(md(e, twoN));
    j.d.nload = int32_t(z);
    j.d.nstore = int32_t(n + f);
    j.d.nscale = int32_t(nscale);
    j.d.escale = int32_t(escale);
    j.d.pad = l;  // the job's own size (launches mix single-CTA jobs of different sizes)
    jobs.push_back(j);
  }

  // Algorithm 1 over global memory; returns the number of passes used
  int tft(int pass, int64_t cell0, int64_t ms, int l, int64_t e, int64_t z, int64_t n) {
    if (leaf(l)) {
      job(pass, KIND_TFT, cell0, ms, l, e, z, n, 0, 0, 0);
      return 1;
    }
    int l1 = top_l1(l), l2 = l - l1;
    int64_t L = int64_t(1) << l, L1 = int64_t(1) << l1, L2 = int64_t(1) << l2, w = twoN / L;
    int64_t n2 = n % L2, n1 = n / L2, n1p = (n + L2 - 1) / L2;
    int64_t z2 = z % L2, z1 = z / L2, z2p = z1 > 0 ? L2 : z2;
    int dc = 0, dr = 0;
    depth++;
    for (int64_t u = 0; u < z2p; u++)
      dc = std::max(dc, tft(pass, cell0 + u * ms, ms * L2, l1, e + u * w, u < z2 ? z1 + 1 : z1, n1p));
    for (int64_t u = 0; u < n1p; u++)
      dr = std::max(dr, tft(pass + dc, cell0 + u * L2 * ms, ms, l2, e * L1, z2p, u < n1 ? L2 : n2));
    depth--;
    return dc + dr;
  }

  // Algorithm 2 over global memory; outputs L a_i (i < n) are multiplied by 2^escale when
  // escale >= 0; the f = 1 output a-hat_n never is.
  int itft(int pass, int64_t cell0, int64_t ms, int l, int64_t e, int64_t z, int64_t n, int f,
           int64_t escale) {
    if (leaf(l)) {
      job(pass, KIND_ITFT, cell0, ms, l, e, z, n, f, escale >= 0 ? n : 0, escale >= 0 ? escale : 0);
      return 1;
    }
    int l1 = top_l1(l), l2 = l - l1;
    int64_t L = int64_t(1) << l, L1 = int64_t(1) << l1, L2 = int64_t(1) << l2, w = twoN / L;
    int64_t n2 = n % L2, n1 = n / L2, z2 = z % L2, z1 = z / L2;
    int fp = (n2 + f > 0) ? 1 : 0;
    int64_t z2p = z1 > 0 ? L2 : z2;
    int64_t m = std::min(n2, z2), mp = std::max(n2, z2);
    int p = pass, d = 0;
    depth++;
    for (int64_t u = 0; u < n1; u++) d = std::max(d, itft(p, cell0 + u * L2 * ms, ms, l2, e * L1, L2, L2, 0, -1));
    p += d;
    d = 0;
    for (int64_t u = n2; u < z2p; u++)
      d = std::max(d, itft(p, cell0 + u * ms, ms * L2, l1, e + u * w, u < mp ? z1 + 1 : z1, n1, fp, escale));
    p += d;
    if (fp) p += itft(p, cell0 + n1 * L2 * ms, ms, l2, e * L1, z2p, n2, f, -1);
    d = 0;
    for (int64_t u = 0; u < n2; u++)
      d = std::max(d, itft(p, cell0 + u * ms, ms * L2, l1, e + u * w, u < m ? z1 + 1 : z1, n1 + 1, 0, escale));
    p += d;
    depth--;
    return p - pass;
  }

  // The recursions number passes in the order Algorithms 1 and 2 take their steps, one step
  // after another. Steps that touch no common cell need not wait for each other (in Algorithm 2
  // the last row's sub-transforms, for example, only need the rows and columns that feed them).
  // relevel() renumbers the passes as levels of the dependency graph between them: a pass goes
  // one level above every earlier pass that wrote a cell it reads or writes, and every earlier
  // pass that read a cell it writes since that cell was last written. Running the levels in order
  // keeps every such pair in order, and the passes of one level touch disjoint cells, so they
  // share launches. Returns the number of levels.
  //
  // A plan of Algorithm 1 alone is already levelled: a sub-transform reads all of its inputs in
  // its first pass (a leaf loads its z cells; the columns of a split share the first pass and
  // load the inputs between them), so the rows' first pass reads the deepest column's last
  // output, and every pass reads a cell the pass before it wrote.
  int relevel() {
    if (jobs.empty()) return 0;
    int maxp = 0;
    int64_t ncells = 0;
    bool all_tft = true;
    for (const JobRec &j : jobs) {
      maxp = std::max(maxp, j.pass);
      all_tft = all_tft && j.kind == KIND_TFT;
      const int32_t m = std::max(j.d.nload, j.d.nstore);
      if (m > 0) ncells = std::max(ncells, j.d.cell0 + int64_t(m - 1) * j.d.mstride + 1);
    }
    if (all_tft) return maxp + 1;
    // job indices grouped by pass
    std::vector<int32_t> first(size_t(maxp) + 2, 0), order(jobs.size());
    for (const JobRec &j : jobs) first[size_t(j.pass) + 1]++;
    for (int p = 0; p <= maxp; p++) first[size_t(p) + 1] += first[size_t(p)];
    {
      std::vector<int32_t> at(first.begin(), first.end() - 1);
      for (size_t i = 0; i < jobs.size(); i++) order[size_t(at[size_t(jobs[i].pass)]++)] = int32_t(i);
    }
    // per cell: the level of its last store, the highest level that read it since
    std::vector<int32_t> &seen = t_cells_scratch;
    seen.assign(size_t(2 * ncells), 0);
    std::vector<int> level(size_t(maxp) + 1, 0);
    int32_t *lw = seen.data(), *lr = seen.data() + 1;  // cell c at 2c
    int top = 0;
    for (int p = 0; p <= maxp; p++) {
      const int32_t b = first[size_t(p)], en = first[size_t(p) + 1];
      int lev = 1;
      for (int32_t t = b; t < en; t++) {
        const JobDesc &d = jobs[size_t(order[size_t(t)])].d;
        const int64_t c0 = d.cell0, ms = d.mstride;
        const int32_t ns = d.nstore, span = std::max(d.nload, d.nstore);
        int32_t m = 0;
        for (; m < ns; m++) lev = std::max(lev, std::max(lw[2 * (c0 + m * ms)], lr[2 * (c0 + m * ms)]) + 1);  // stored
        for (; m < span; m++) lev = std::max(lev, lw[2 * (c0 + m * ms)] + 1);                           // loaded only
      }
      for (int32_t t = b; t < en; t++) {
        const JobDesc &d = jobs[size_t(order[size_t(t)])].d;
        const int64_t c0 = d.cell0, ms = d.mstride;
        const int32_t ns = d.nstore, span = std::max(d.nload, d.nstore);
        int32_t m = 0;
        for (; m < ns; m++) {
          lw[2 * (c0 + m * ms)] = lev;
          lr[2 * (c0 + m * ms)] = 0;
        }
        for (; m < span; m++) lr[2 * (c0 + m * ms)] = std::max(lr[2 * (c0 + m * ms)], lev);
      }
      level[size_t(p)] = lev;
      if (en > b) top = std::max(top, lev);
    }
    for (JobRec &j : jobs) j.pass = level[size_t(j.pass)] - 1;
    return top;
  }
};

struct PlanCache {
  std::mutex mu;
  std::map<std::tuple<int, int, int, int64_t, int64_t, int, int64_t, int64_t, int, int>, std::unique_ptr<TransformPlan>>
      plans;
};

PlanCache &plan_cache() {
  static PlanCache *c = new PlanCache();
  return *c;
}

}  // namespace

namespace {

// Jobs of one pass share a launch: single-CTA jobs of every size together (each job carries its
// own size, the launch is sized for the largest), cluster jobs by size.
bool same_launch(const JobRec &a, const JobRec &b) {
  return a.pass == b.pass && a.lc == b.lc && (a.lc == 0 || a.ls == b.ls);
}
bool launch_order(const JobRec &a, const JobRec &b) {
  if (a.pass != b.pass) return a.pass < b.pass;
  if (a.lc != b.lc) return a.lc < b.lc;
  return a.ls < b.ls;
}

// the largest job of the launch jobs[i .. k)
int launch_ls(const std::vector<JobRec> &jobs, size_t i, size_t k) {
  int ls = 0;
  for (size_t t = i; t < k; t++) ls = std::max(ls, jobs[t].ls);
  return ls;
}

// Every other launch takes its jobs in reverse order. Jobs of one launch touch disjoint cells,
// so any order is correct; CTAs start roughly in job order, and a pass that reads what the one
// before it stored then begins with the cells stored last, the ones most likely still in L2.
// Only plans whose cells outgrow half of the 129 MB L2 take it: there it made the l = 16
// transforms at N = 32768 about 3 % faster alone, while the products' transforms, which fit in
// L2, came out 1.8 % slower with it.
constexpr int64_t kSnakeBytes = int64_t(64) << 20;
bool wants_snake(const std::vector<JobRec> &jobs, int64_t N) {
  int64_t extent = 0;
  for (const JobRec &j : jobs) {
    const int32_t m = std::max(j.d.nload, j.d.nstore);
    if (m > 0) extent = std::max(extent, j.d.cell0 + int64_t(m - 1) * j.d.mstride + 1);
  }
  return extent * 8 * (N / 64 + 1) > kSnakeBytes;
}

void snake_launches(std::vector<JobRec> &jobs) {
  int launch = 0;
  for (size_t i = 0; i < jobs.size();) {
    size_t k = i + 1;
    while (k < jobs.size() && same_launch(jobs[k], jobs[i])) k++;
    if (launch & 1) std::reverse(jobs.begin() + i, jobs.begin() + k);
    launch++;
    i = k;
  }
}

// Reorder into launch order: a counting sort over the packed key (pass, lc, ls), whose range the
// plans keep small (a comparison sort otherwise), then, for snake, every other launch reversed.
// Within a launch the job sizes are therefore not in order: take the largest with launch_ls.
void sort_launch_order(std::vector<JobRec> &jobs, bool snake) {
  if (jobs.size() < 2) return;
  int maxp = 0;
  bool small = true;
  for (const JobRec &j : jobs) {
    maxp = std::max(maxp, j.pass);
    small = small && j.pass >= 0 && j.lc >= 0 && j.lc < 8 && j.ls >= 0 && j.ls < 32;
  }
  const size_t range = (size_t(maxp) + 1) * 256;
  if (!small || range > 4 * jobs.size() + 65536) {
    std::stable_sort(jobs.begin(), jobs.end(), launch_order);
    if (snake) snake_launches(jobs);
    return;
  }
  auto key = [](const JobRec &j) { return (size_t(j.pass) * 8 + size_t(j.lc)) * 32 + size_t(j.ls); };
  std::vector<int32_t> at(range + 1, 0);
  for (const JobRec &j : jobs) at[key(j) + 1]++;
  for (size_t k = 0; k < range; k++) at[k + 1] += at[k];
  std::vector<JobRec> &out = t_jobs_sorted;
  out.resize(jobs.size());
  for (const JobRec &j : jobs) out[size_t(at[key(j)]++)] = j;
  jobs.swap(out);  // the scratch keeps the old list's buffer
  if (snake) snake_launches(jobs);
}

}  // namespace

// Flag the jobs whose every stored cell is stored again by a later pass (JOB_RAW_STORE): they
// may leave their cells in internal form, which a later load recognises by the top limb. The
// last store of every cell stays canonical. Passes are the unit: jobs of one pass touch
// disjoint cells, and merged launches keep the pass order.
static void mark_raw_stores(std::vector<JobRec> &jobs, int l) {
  if (l > 22 || jobs.empty()) return;
  const int64_t L = int64_t(1) << l;
  std::vector<int32_t> &last = t_cells_scratch;
  last.assign(size_t(L), -1);
  int32_t *lp = last.data();
  for (const JobRec &j : jobs) {
    const int64_t c0 = j.d.cell0, ms = j.d.mstride, ns = j.d.nstore;
    if (ns <= 0) continue;
    if (c0 < 0 || c0 >= L || c0 + (ns - 1) * ms < 0 || c0 + (ns - 1) * ms >= L)
      return;  // not a plan over [0, L): leave every store canonical
    const int pass = j.pass;
    for (int64_t m = 0; m < ns; m++) lp[c0 + m * ms] = std::max(lp[c0 + m * ms], pass);
  }
  for (JobRec &j : jobs) {
    const int64_t c0 = j.d.cell0, ms = j.d.mstride, ns = j.d.nstore;
    const int pass = j.pass;
    bool raw = ns > 0;
    for (int64_t m = 0; m < ns && raw; m++) raw = lp[c0 + m * ms] > pass;
    if (raw) j.d.pad |= JOB_RAW_STORE;
  }
}

bool build_fused_schedule(const std::vector<JobDesc> &jobs, const std::vector<int> &pass, int64_t L, int slots,
                          FusedSchedule *out) {
  *out = FusedSchedule();
  const int nj = int(jobs.size());
  if (nj == 0 || L > (int64_t(1) << 22) || slots < 1) return false;
  // dependencies, taking the jobs in pass order (jobs of one pass touch disjoint cells)
  const size_t ncells = size_t(L);
  std::vector<int32_t> last_store(ncells, -1);
  std::vector<std::vector<int32_t>> readers(ncells);
  std::vector<std::vector<int32_t>> deps(nj);
  for (int j = 0; j < nj; j++) {
    const JobDesc &d = jobs[j];
    const int64_t span = std::max(d.nload, d.nstore);
    for (int64_t m = 0; m < span; m++) {
      const int64_t c = d.cell0 + m * d.mstride;
      if (c < 0 || c >= L) return false;
    }
    std::vector<int32_t> &dj = deps[j];
    for (int64_t m = 0; m < span; m++) {
      const size_t c = size_t(d.cell0 + m * d.mstride);
      if (last_store[c] >= 0) dj.push_back(last_store[c]);
      if (m < d.nstore) dj.insert(dj.end(), readers[c].begin(), readers[c].end());
    }
    std::sort(dj.begin(), dj.end());
    dj.erase(std::unique(dj.begin(), dj.end()), dj.end());
    for (int64_t m = 0; m < span; m++) {
      const size_t c = size_t(d.cell0 + m * d.mstride);
      if (m < d.nstore) {
        last_store[c] = j;
        readers[c].clear();
      } else if (m < d.nload) {
        readers[c].push_back(j);
      }
    }
  }
  // list schedule: rounds of `slots` jobs; a job is ready once every job it depends on ran in an
  // earlier round; among ready jobs the deepest pass goes first, then the plan order
  std::vector<std::vector<int32_t>> users(nj);
  std::vector<int32_t> pending(nj);
  for (int j = 0; j < nj; j++) {
    pending[j] = int32_t(deps[j].size());
    for (int32_t d : deps[j]) users[d].push_back(j);
  }
  auto later = [&](int32_t a, int32_t b) { return pass[a] != pass[b] ? pass[a] < pass[b] : a > b; };
  std::priority_queue<int32_t, std::vector<int32_t>, decltype(later)> ready(later);
  for (int j = 0; j < nj; j++)
    if (!pending[j]) ready.push(j);
  std::vector<int32_t> pos(nj, -1), round;
  out->order.reserve(nj);
  while (!ready.empty()) {
    round.clear();
    while (!ready.empty() && int(round.size()) < slots) {
      const int32_t j = ready.top();
      ready.pop();
      pos[j] = int32_t(out->order.size());
      out->order.push_back(j);
      round.push_back(j);
    }
    for (int32_t j : round)
      for (int32_t u : users[j])
        if (--pending[u] == 0) ready.push(u);
  }
  if (int(out->order.size()) != nj) {  // a cycle cannot occur; keep the per-pass launches if it did
    *out = FusedSchedule();
    return false;
  }
  out->dep_off.push_back(0);
  for (int k = 0; k < nj; k++) {
    for (int32_t d : deps[out->order[k]]) out->deps.push_back(pos[d]);
    out->dep_off.push_back(int32_t(out->deps.size()));
  }
  return true;
}

// Concurrent CTAs of a fused launch, for the list schedule (the launch uses the occupancy of its
// kernel; this only shapes the order): three single-CTA jobs per SM.
static int schedule_slots() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 152;
  }
  return 3 * sms;
}

int64_t zero_padded_outputs(int l, int64_t n, int64_t N) {
  Planner P(N);
  const int64_t L = int64_t(1) << l;
  auto up = [](int64_t v, int64_t m) { return (v + m - 1) / m * m; };
  // Granularities that make the rows of one more recursion level whole: the top split's rows
  // (L2), then the rows of the column sub-transforms' own split (their n is n / L2), and so on
  // down to the jobs (a cluster job's in-job rows; a single CTA needs nothing).
  std::vector<int64_t> grains;
  int64_t g = 1;
  for (int ll = l;;) {
    if (P.leaf(ll)) {
      const int lc = P.cluster_log2(ll);
      if (lc > 0) grains.push_back(g << (ll - lc));
      break;
    }
    const int l1 = P.top_l1(ll);
    g <<= (ll - l1);
    grains.push_back(g);
    ll = l1;
    P.depth = 1;  // below the whole transform
  }
  if (grains.empty()) return n;
  // the top level's whole rows always (they remove a pass); finer ones while they add at most n/32
  int64_t best = std::min(L, up(n, grains[0]));
  for (size_t k = 1; k < grains.size(); k++) {
    const int64_t c = up(n, grains[k]);
    if (c <= L && (c - n) * 32 <= n) best = c;
  }
  return best;
}

int count_passes(int kind, int l, int64_t z, int64_t n, int f, int64_t N) {
  Planner P(N);
  if (kind == KIND_TFT)
    P.tft(0, 0, 1, l, 0, z, n);
  else
    P.itft(0, 0, 1, l, 0, z, n, f, -1);
  return P.relevel();
}

void plan_shape(int kind, int l, int64_t z, int64_t n, int f, int64_t N, int *passes, int *launches,
                int64_t *jobs, int *onchip_l, int *cluster_l) {
  Planner P(N);
  if (kind == KIND_TFT)
    P.tft(0, 0, 1, l, 0, z, n);
  else
    P.itft(0, 0, 1, l, 0, z, n, f, -1);
  *passes = P.relevel();
  sort_launch_order(P.jobs, false);
  int nl = 0, lcmax = 0, lsmax = 0;
  for (size_t i = 0; i < P.jobs.size(); i++) {
    if (i == 0 || !same_launch(P.jobs[i], P.jobs[i - 1])) nl++;
    lcmax = std::max(lcmax, P.jobs[i].lc);
    lsmax = std::max(lsmax, P.jobs[i].ls);
  }
  *launches = nl;
  *jobs = int64_t(P.jobs.size());
  *onchip_l = lsmax;
  *cluster_l = lcmax;
}

// the exponent of 1/L in powers of omega (2^{-l} = omega^{-l u}, u = 1, or 2 for sqrt2)
static int64_t inv_l_exponent(int l, int64_t twoN, int mode) {
  return md(twoN - int64_t(l) * (mode == RING_SQRT2 ? 2 : 1), twoN);
}

void build_host_plan(int kind, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e, int scale,
                     HostPlan *out, int mode) {
  const int64_t twoN = omega_order(N, mode);
  e = md(e, twoN);
  Planner P(N, nullptr, mode);
  out->ring = P.ring;
  if (kind == KIND_TFT)
    P.tft(0, 0, 1, l, e, z, n);
  else
    P.itft(0, 0, 1, l, e, z, n, f, scale ? inv_l_exponent(l, twoN, mode) : -1);
  out->npasses = P.relevel();
  std::map<std::tuple<int, int, int, int64_t, int64_t, int>, int> index;
  mark_raw_stores(P.jobs, l);
  sort_launch_order(P.jobs, wants_snake(P.jobs, N));
  for (size_t i = 0; i < P.jobs.size();) {
    size_t k = i;
    while (k < P.jobs.size() && same_launch(P.jobs[k], P.jobs[i])) k++;
    HostPlan::Group g;
    g.ls = launch_ls(P.jobs, i, k);
    g.lc = P.jobs[i].lc;
    g.nwarps = warps_for_job(g.ls, g.lc, P.cfg.max_warps);
    g.prog_words = 0;
    for (size_t t = i; t < k; t++) {
      const JobRec &j = P.jobs[t];
      auto key = std::make_tuple(j.kind, j.ls, j.lc, j.z, j.n, j.f);
      auto it = index.find(key);
      int pi;
      if (it == index.end()) {
        pi = int(out->programs.size());
        out->programs.push_back(build_job_image(j.kind, j.ls, j.lc, j.z, j.n, j.f, N, nullptr, mode));
        index[key] = pi;
      } else {
        pi = it->second;
      }
      g.jobs.push_back(j.d);
      g.prog_index.push_back(pi);
      g.prog_words = std::max(g.prog_words, image_max_program_words(out->programs[pi]));
    }
    out->groups.push_back(std::move(g));
    i = k;
  }
}

void build_host_schedule(int kind, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e, int scale,
                         FusedSchedule *out, int mode, int slots) {
  *out = FusedSchedule();
  const int64_t twoN = omega_order(N, mode);
  e = md(e, twoN);
  Planner P(N, nullptr, mode);
  if (kind == KIND_TFT)
    P.tft(0, 0, 1, l, e, z, n);
  else
    P.itft(0, 0, 1, l, e, z, n, f, scale ? inv_l_exponent(l, twoN, mode) : -1);
  P.relevel();
  mark_raw_stores(P.jobs, l);
  sort_launch_order(P.jobs, wants_snake(P.jobs, N));
  int nl = 0;
  bool single = true;
  for (size_t i = 0; i < P.jobs.size(); i++) {
    if (i == 0 || !same_launch(P.jobs[i], P.jobs[i - 1])) nl++;
    single = single && P.jobs[i].lc == 0;
  }
  if (!fused_for(P.cfg.fused, kind) || !single || nl < 2 || P.ring.K < 4 || P.ring.G != 32) return;
  std::vector<JobDesc> flat;
  std::vector<int> passes;
  for (const JobRec &j : P.jobs) {
    flat.push_back(j.d);
    passes.push_back(j.pass);
  }
  build_fused_schedule(flat, passes, int64_t(1) << l, slots > 0 ? slots : 456, out);
}

const TransformPlan *get_transform_plan(int kind, int l, int64_t z, int64_t n, int f, int64_t N,
                                        int64_t e, int64_t stride_limbs, int scale, int *err, int mode,
                                        bool replicated) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int64_t twoN = omega_order(N, mode);
  e = md(e, twoN);
  const PlanConfig cfg = plan_config(N);
  // ls_max, ls_c, max_warps 5 bits each; split, mode, fused, max_lc 3 bits each
  const int cfg_key = cfg.ls_max | (cfg.ls_c << 5) | (cfg.max_warps << 10) | (cfg.split << 15) | (mode << 18) |
                      (replicated ? 1 << 21 : 0) | (cfg.fused << 22) | (cfg.max_lc << 25) | (cfg.tma << 28);
  auto key = std::make_tuple(dev, kind, l, z, n, f, N, e, scale, cfg_key);
  PlanCache &pc = plan_cache();
  {
    std::lock_guard<std::mutex> lk(pc.mu);
    auto it = pc.plans.find(key);
    if (it != pc.plans.end()) return it->second.get();
  }
  Planner P(N, &cfg, mode);
  P.whole_split = !replicated;
  if (kind == KIND_TFT)
    P.tft(0, 0, 1, l, e, z, n);
  else
    P.itft(0, 0, 1, l, e, z, n, f, scale ? inv_l_exponent(l, twoN, mode) : -1);
  const int npass = P.relevel();

  std::unique_ptr<TransformPlan> plan(new TransformPlan());
  plan->ring = P.ring;
  plan->mode = mode;
  plan->npasses = npass;
  plan->njobs = int64_t(P.jobs.size());
  // resolve job images, then group jobs by (pass, ls, lc) in pass order
  // neighbouring jobs mostly share a shape: look an image up once per run of equal shapes
  const JobRec *prev = nullptr;
  for (JobRec &j : P.jobs) {
    if (prev && prev->kind == j.kind && prev->ls == j.ls && prev->lc == j.lc && prev->z == j.z &&
        prev->n == j.n && prev->f == j.f) {
      j.d.image = prev->d.image;
    } else {
      j.d.image = image_cache().get(j.kind, j.ls, j.lc, j.z, j.n, j.f, N, err, mode);
      if (!j.d.image) return nullptr;
    }
    prev = &j;
  }
  mark_raw_stores(P.jobs, l);
  sort_launch_order(P.jobs, wants_snake(P.jobs, N));
  std::vector<JobDesc> flat;
  std::vector<std::pair<size_t, Launch>> groups;
  for (size_t i = 0; i < P.jobs.size();) {
    size_t k = i;
    while (k < P.jobs.size() && same_launch(P.jobs[k], P.jobs[i])) k++;
    Launch L;
    L.pass = P.jobs[i].pass;
    L.ls = launch_ls(P.jobs, i, k);
    L.lc = P.jobs[i].lc;
    L.njobs = int(k - i);
    L.nwarps = warps_for_job(L.ls, L.lc, P.cfg.max_warps);
    for (size_t t = i; t < k; t++)
      if (t == i || P.jobs[t].d.image != P.jobs[t - 1].d.image)
        L.prog_words = std::max(L.prog_words, image_cache().max_prog(P.jobs[t].d.image));
    groups.push_back({flat.size(), L});
    for (size_t t = i; t < k; t++) flat.push_back(P.jobs[t].d);
    i = k;
  }
  JobDesc *d = static_cast<JobDesc *>(plan_alloc(std::max<size_t>(1, flat.size()) * sizeof(JobDesc)));
  if (!d) {
    *err = ZX_ENOMEM;
    return nullptr;
  }
  if (plan_upload(d, flat.data(), flat.size() * sizeof(JobDesc)) != cudaSuccess) {
    *err = ZX_ECUDA;
    return nullptr;
  }
  for (auto &g : groups) {
    g.second.d_jobs = d + g.first;
    plan->launches.push_back(g.second);
  }
  for (const JobDesc &jd : flat) {
    const int32_t m = std::max(jd.nload, jd.nstore);
    if (m > 0) plan->cell_extent = std::max(plan->cell_extent, jd.cell0 + int64_t(m - 1) * jd.mstride + 1);
  }
  (void)stride_limbs;
  // the fused form: every job single-CTA, more than one launch, not replicated
  plan->stream = (cfg.fused == FUSED_STREAM || cfg.fused == FUSED_DIRECT) && !replicated && P.ring.K >= 4 &&
                 P.ring.G == 32;
  plan->direct = cfg.fused == FUSED_DIRECT;
  plan->tma = cfg.tma != 0;
  // (the persistent kernel is built for rings whose words fill all 32 lanes, four or more words
  // per lane: N a power of two from 4096 on)
  bool fusable = fused_for(cfg.fused, kind) && !replicated && plan->launches.size() > 1 && P.ring.K >= 4 &&
                 P.ring.G == 32;
  for (const Launch &L : plan->launches) fusable = fusable && L.lc == 0;
  FusedSchedule fs;
  std::vector<int> passes;
  for (const JobRec &j : P.jobs) passes.push_back(j.pass);
  if (fusable && build_fused_schedule(flat, passes, int64_t(1) << l, schedule_slots(), &fs)) {
    const size_t nj = fs.order.size();
    const size_t bytes = nj * sizeof(JobDesc) + (fs.dep_off.size() + fs.deps.size()) * sizeof(int32_t);
    std::vector<unsigned char> blob(bytes);
    JobDesc *hj = reinterpret_cast<JobDesc *>(blob.data());
    for (size_t k = 0; k < nj; k++) hj[k] = flat[size_t(fs.order[k])];
    int32_t *ho = reinterpret_cast<int32_t *>(hj + nj);
    std::memcpy(ho, fs.dep_off.data(), fs.dep_off.size() * sizeof(int32_t));
    std::memcpy(ho + fs.dep_off.size(), fs.deps.data(), fs.deps.size() * sizeof(int32_t));
    unsigned char *dblob = static_cast<unsigned char *>(plan_alloc(bytes));
    if (!dblob) {
      *err = ZX_ENOMEM;
      return nullptr;
    }
    if (plan_upload(dblob, blob.data(), bytes) != cudaSuccess) {
      *err = ZX_ECUDA;
      return nullptr;
    }
    plan->f_njobs = int(nj);
    plan->f_jobs = reinterpret_cast<const JobDesc *>(dblob);
    plan->f_dep_off = reinterpret_cast<const int32_t *>(dblob + nj * sizeof(JobDesc));
    plan->f_deps = plan->f_dep_off + fs.dep_off.size();
    for (const Launch &L : plan->launches) {
      plan->f_ls = std::max(plan->f_ls, L.ls);
      plan->f_prog_words = std::max(plan->f_prog_words, L.prog_words);
    }
    plan->f_nwarps = warps_for_job(plan->f_ls, 0, P.cfg.max_warps);
  }
  std::lock_guard<std::mutex> lk(pc.mu);
  auto &slot = pc.plans[key];
  if (!slot) slot = std::move(plan);
  return slot.get();
}

// ---------------------------------------------------------------- S[y]/(y^{M/2}+1) plans
// Algorithms 1 and 2 over global memory exactly as for Z/(2^N+1), with omega = y (rotations
// mod M = 2H) and single-CTA jobs only: an element is H = M/2 coefficients of 8 bytes.

int sn_max_onchip_ls(int64_t H) {
  int ls = 1;
  while (ls < 16 && (size_t(2) << ls) * (size_t(H) * 8 + 4) <= size_t(72) * 1024) ls++;
  return ls;
}

namespace {
struct SnPlanCache {
  std::mutex mu;
  std::map<std::tuple<int, int, int, int64_t, int64_t, int, int64_t, int64_t, int>, std::unique_ptr<TransformPlan>> plans;
};
SnPlanCache &sn_plan_cache() {
  static SnPlanCache *c = new SnPlanCache();
  return *c;
}
}  // namespace

const TransformPlan *get_sn_plan(int kind, int l, int64_t z, int64_t n, int f, int64_t H, int64_t e, int scale,
                                 int *err) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int64_t M = 2 * H;
  e = md(e, M);
  auto key = std::make_tuple(dev, kind, l, z, n, f, H, e, scale);
  SnPlanCache &pc = sn_plan_cache();
  {
    std::lock_guard<std::mutex> lk(pc.mu);
    auto it = pc.plans.find(key);
    if (it != pc.plans.end()) return it->second.get();
  }
  PlanConfig cfg;
  cfg.ls_max = sn_max_onchip_ls(H);
  cfg.ls_c = -64;  // no cluster jobs: sub-transforms above ls_max recurse
  cfg.max_warps = 8;
  cfg.split = 0;
  Planner P(H, &cfg);
  // the final division by L: l halvings of every coefficient (escale counts them)
  if (kind == KIND_TFT)
    P.tft(0, 0, 1, l, e, z, n);
  else
    P.itft(0, 0, 1, l, e, z, n, f, scale ? l : -1);
  const int npass = P.relevel();
  std::unique_ptr<TransformPlan> plan(new TransformPlan());
  plan->ring = make_ring(64);
  plan->ring.N = H;
  plan->npasses = npass;
  plan->njobs = int64_t(P.jobs.size());
  for (JobRec &j : P.jobs) {
    if (j.lc != 0) {
      *err = ZX_EUNSUPPORTED;
      return nullptr;
    }
    j.d.image = image_cache().get(j.kind, j.ls, j.lc, j.z, j.n, j.f, H, err, RING_SN);
    if (!j.d.image) return nullptr;
  }
  sort_launch_order(P.jobs, false);
  std::vector<JobDesc> flat;
  std::vector<std::pair<size_t, Launch>> groups;
  for (size_t i = 0; i < P.jobs.size();) {
    size_t k = i;
    while (k < P.jobs.size() && same_launch(P.jobs[k], P.jobs[i])) k++;
    Launch L;
    L.pass = P.jobs[i].pass;
    L.ls = launch_ls(P.jobs, i, k);
    L.lc = 0;
    L.njobs = int(k - i);
    L.nwarps = warps_for_job(L.ls, 0, cfg.max_warps);
    for (size_t t = i; t < k; t++)
      if (t == i || P.jobs[t].d.image != P.jobs[t - 1].d.image)
        L.prog_words = std::max(L.prog_words, image_cache().max_prog(P.jobs[t].d.image));
    groups.push_back({flat.size(), L});
    for (size_t t = i; t < k; t++) flat.push_back(P.jobs[t].d);
    i = k;
  }
  JobDesc *d = static_cast<JobDesc *>(plan_alloc(std::max<size_t>(1, flat.size()) * sizeof(JobDesc)));
  if (!d) {
    *err = ZX_ENOMEM;
    return nullptr;
  }
  if (plan_upload(d, flat.data(), flat.size() * sizeof(JobDesc)) != cudaSuccess) {
    *err = ZX_ECUDA;
    return nullptr;
  }
  for (auto &g : groups) {
    g.second.d_jobs = d + g.first;
    plan->launches.push_back(g.second);
  }
  std::lock_guard<std::mutex> lk(pc.mu);
  auto &slot = pc.plans[key];
  if (!slot) slot = std::move(plan);
  return slot.get();
}

void sn_plan_shape(int kind, int l, int64_t z, int64_t n, int f, int64_t H, int *passes, int *launches,
                   int64_t *jobs) {
  PlanConfig cfg;
  cfg.ls_max = sn_max_onchip_ls(H);
  cfg.ls_c = -64;
  cfg.max_warps = 8;
  cfg.split = 0;
  Planner P(H, &cfg);
  if (kind == KIND_TFT)
    P.tft(0, 0, 1, l, 0, z, n);
  else
    P.itft(0, 0, 1, l, 0, z, n, f, -1);
  *passes = P.relevel();
  sort_launch_order(P.jobs, false);
  int nl = 0;
  for (size_t i = 0; i < P.jobs.size(); i++)
    if (i == 0 || !same_launch(P.jobs[i], P.jobs[i - 1])) nl++;
  *launches = nl;
  *jobs = int64_t(P.jobs.size());
}

}  // namespace tftgpu
