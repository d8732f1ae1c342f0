// zx_mul_noalloc: the Z[x] product of zx_mul for callers that must not allocate memory.
//
// The paper has no counterpart to this entry point; it exists for callers that cannot call
// cudaMalloc: code whose device memory is entirely reserved by another allocator (a framework
// that pre-allocates the whole GPU and forbids foreign allocations), or loops that must not
// pay the latency and implicit synchronisation of an allocation. It runs the same kernels as
// zx_mul, but its two ring buffers and its launch plans live in one file-scope device array of
// fixed size instead of memory obtained from an allocator.
//
// The array (20 MiB per GPU that loads the library, held until the process exits):
//   limbs [0, 2^21)           the two ring buffers of L cells each (16 MiB)
//   the remaining 4 MiB       job lists and butterfly programs of the plans used so far
// The first call on a device looks up the array's device address with cudaGetSymbolAddress
// (with that device current); make that first call before any stream capture. Plans are
// written into the array the first time a product shape is seen (under the ring's launch
// configuration at that time) and kept for later calls; that first call for a shape is refused
// while the stream is capturing, since a capture cannot record the upload of host data for later
// replays. The pointwise products use the schoolbook kernel (zx_mul's default method).
// Nothing in the ring buffers needs to start at zero: the transforms read only cells that
// the pack step of the same call has written. All calls share the array, so calls whose work
// overlaps on the GPU (different streams or host threads without ordering) race.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/tftgpu.h"
#include "common.h"
#include "host.h"

namespace tftgpu {

namespace {

constexpr size_t kRingLimbs = size_t(1) << 21;            // 16 MiB of ring buffers
constexpr size_t kPlanLimbs = size_t(1) << 19;            // 4 MiB of plans
constexpr size_t kScratchLimbs = kRingLimbs + kPlanLimbs;  // 20 MiB in total

static __device__ __align__(256) uint64_t g_noalloc_scratch[kScratchLimbs];

// plans of one device, keyed by the transform and the ring's launch configuration when planned
using PlanKey = std::tuple<int, int, int64_t, int64_t, int, int64_t, int64_t, int, int, int, int, int, int>;

struct NoAllocDevice {
  uint64_t *base = nullptr;  // device address of g_noalloc_scratch on this device
  size_t plan_used = 0;      // limbs of the plan region in use
  std::map<PlanKey, std::unique_ptr<TransformPlan>> plans;
};

std::mutex g_mu;
std::map<int, NoAllocDevice> g_devices;

int na_fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

// device state for the current device, looking up the array address on first use
int device_state(NoAllocDevice **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(ZX_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  NoAllocDevice &st = g_devices[dev];
  if (!st.base) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return na_fail(ZX_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    st.base = static_cast<uint64_t *>(p);
  }
  *out = &st;
  return ZX_OK;
}

// place `bytes` in the plan region (16-byte aligned); nullptr when the region is full
uint64_t *plan_space(NoAllocDevice &st, size_t bytes) {
  size_t limbs = (bytes + 15) / 16 * 2;
  if (st.plan_used + limbs > kPlanLimbs) return nullptr;
  uint64_t *p = st.base + kRingLimbs + st.plan_used;
  st.plan_used += limbs;
  return p;
}

// The plan of one transform in the plan region: found in the cache, or built and uploaded. The
// upload copies host memory to the device, which a stream capture cannot record for later
// replays, so a plan that is not cached yet is refused while `s` is capturing.
int plan_in_scratch(NoAllocDevice &st, int kind, int l, int64_t z, int64_t n, int f, int64_t N, int scale,
                    int mode, cudaStream_t s, const TransformPlan **out) {
  const PlanConfig cfg = plan_config(N);
  const PlanKey key(kind, l, z, n, f, N, int64_t(mode), scale, cfg.ls_max, cfg.ls_c, cfg.max_warps, cfg.split,
                    cfg.fused);
  auto it = st.plans.find(key);
  if (it != st.plans.end()) {
    *out = it->second.get();
    return ZX_OK;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(s, &cap);
  if (ce != cudaSuccess) return na_fail(ZX_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
  if (cap != cudaStreamCaptureStatusNone)
    return na_fail(ZX_EINVAL,
                   "zx_mul_noalloc: the first call for a product shape (or after a change of the ring's launch "
                   "configuration) uploads its launch plan and cannot be captured; make it once before capturing");
  HostPlan hp;
  build_host_plan(kind, l, z, n, f, N, 0, scale, &hp, mode);
  size_t need = 0;
  for (const auto &img : hp.programs) need += (img.size() * 4 + 15) / 16 * 16;
  for (const auto &g : hp.groups) need += (g.jobs.size() * sizeof(JobDesc) + 15) / 16 * 16;
  if (st.plan_used * 8 + need > kPlanLimbs * 8)
    return na_fail(ZX_ENOMEM, "zx_mul_noalloc: the 4 MiB plan region is full (too many distinct product shapes)");
  // on a failed upload the region taken so far is given back
  const size_t used_before = st.plan_used;
  auto upload_fail = [&](cudaError_t e) {
    st.plan_used = used_before;
    return na_fail(ZX_ECUDA, std::string("plan upload: ") + cudaGetErrorString(e));
  };
  std::vector<const uint32_t *> dprog;
  for (const auto &img : hp.programs) {
    uint64_t *d = plan_space(st, img.size() * 4);
    cudaError_t e = cudaMemcpyAsync(d, img.data(), img.size() * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return upload_fail(e);
    dprog.push_back(reinterpret_cast<const uint32_t *>(d));
  }
  std::unique_ptr<TransformPlan> plan(new TransformPlan());
  plan->ring = hp.ring;
  plan->mode = mode;
  plan->npasses = hp.npasses;
  for (auto &g : hp.groups) {
    for (size_t i = 0; i < g.jobs.size(); i++) g.jobs[i].image = dprog[g.prog_index[i]];
    uint64_t *d = plan_space(st, g.jobs.size() * sizeof(JobDesc));
    cudaError_t e = cudaMemcpyAsync(d, g.jobs.data(), g.jobs.size() * sizeof(JobDesc), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return upload_fail(e);
    Launch L;
    L.ls = g.ls;
    L.lc = g.lc;
    L.nwarps = g.nwarps;
    L.prog_words = g.prog_words;
    L.njobs = int(g.jobs.size());
    L.d_jobs = reinterpret_cast<JobDesc *>(d);
    plan->launches.push_back(L);
    plan->njobs += L.njobs;
  }
  *out = plan.get();
  st.plans[key] = std::move(plan);
  return ZX_OK;
}

}  // namespace

}  // namespace tftgpu

using namespace tftgpu;

extern "C" int zx_mul_noalloc(const zx_poly *f, const zx_poly *g, zx_poly *h, void *stream) {
  const zx_poly *ps[3] = {f, g, h};
  for (const zx_poly *p : ps) {
    if (!p || p->len < 1 || p->limbs < 1 || !p->data)
      return na_fail(ZX_EINVAL, "zx_mul_noalloc: bad polynomial (NULL, len or limbs < 1)");
    if (p->where != ZX_DEVICE)
      return na_fail(ZX_EINVAL, "zx_mul_noalloc: every operand must be in device memory");
  }
  if (h->len != f->len + g->len - 1) return na_fail(ZX_EINVAL, "zx_mul_noalloc: h->len must be f->len + g->len - 1");
  zx_plan_info info;
  int sgn = (f->is_signed || g->is_signed) ? 1 : 0;
  int64_t bf = f->bits > 0 ? f->bits : 64 * f->limbs, bg = g->bits > 0 ? g->bits : 64 * g->limbs;
  int rc = zx_plan(f->len, bf, g->len, bg, sgn, &info);
  if (rc) return rc;
  if (h->limbs < info.limbs_h) {
    h->limbs = info.limbs_h;
    return na_fail(ZX_EBUFSIZE, "zx_mul_noalloc: h->limbs too small (needed count written to h->limbs)");
  }
  const int64_t L = int64_t(1) << info.l;
  const size_t ring = size_t(L) * size_t(info.stride_limbs);
  if (2 * ring > kRingLimbs)
    return na_fail(ZX_EUNSUPPORTED, "zx_mul_noalloc: the product needs " + std::to_string(2 * ring * 8) +
                                        " bytes of ring buffers; the fixed scratch holds 16 MiB");
  cudaStream_t s = cudaStream_t(stream);
  std::lock_guard<std::mutex> lk(g_mu);
  NoAllocDevice *st = nullptr;
  if ((rc = device_state(&st))) return rc;
  const TransformPlan *pf = nullptr, *pg = nullptr, *pi = nullptr;
  const int mode = info.sqrt2 ? RING_SQRT2 : RING_FERMAT;
  if ((rc = plan_in_scratch(*st, KIND_TFT, info.l, f->len, info.n_fft, 0, info.N, 0, mode, s, &pf)) ||
      (rc = plan_in_scratch(*st, KIND_TFT, info.l, g->len, info.n_fft, 0, info.N, 0, mode, s, &pg)) ||
      (rc = plan_in_scratch(*st, KIND_ITFT, info.l, info.n_fft, info.n_fft, 0, info.N, 1, mode, s, &pi)))
    return rc;
  uint64_t *F = st->base, *G = st->base + ring;
  const Ring &r = pf->ring;
  h->is_signed = sgn;
  cudaError_t ce;
  if ((ce = launch_pack(f->data, f->len, f->limbs, f->is_signed, F, info.stride_limbs, r, s)) != cudaSuccess ||
      (ce = launch_pack(g->data, g->len, g->limbs, g->is_signed, G, info.stride_limbs, r, s)) != cudaSuccess ||
      (ce = run_transform(*pf, F, info.stride_limbs, s, false)) != cudaSuccess ||
      (ce = run_transform(*pg, G, info.stride_limbs, s, false)) != cudaSuccess ||
      (ce = launch_pointwise(F, G, info.n_fft, info.stride_limbs, r, s)) != cudaSuccess ||
      (ce = run_transform(*pi, F, info.stride_limbs, s, false)) != cudaSuccess ||
      (ce = launch_lift(F, info.n, info.stride_limbs, sgn, h->data, h->limbs, r, s)) != cudaSuccess)
    return na_fail(ZX_ECUDA, std::string("zx_mul_noalloc launch: ") + cudaGetErrorString(ce));
  return ZX_OK;
}
