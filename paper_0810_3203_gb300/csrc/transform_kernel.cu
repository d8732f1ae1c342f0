// Per-pass launches of the sub-transform kernel (job_kernel.cuh) and the host entry points that
// enqueue a plan: one launch per pass, or the plan's persistent form (transform_fused.cu).
#include <cudaTypedefs.h>

#include <climits>

#include "job_kernel.cuh"

namespace tftgpu {

// The status word of the bounded waits on each device (see job_kernel.cuh).
__device__ uint32_t g_wait_fault;

// Its device address on the current device (looked up once per device and host thread).
static uint32_t *fault_word() {
  static thread_local uint32_t *addr[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if (dev < 8 && addr[dev]) return addr[dev];
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_wait_fault) != cudaSuccess) return nullptr;
  if (dev < 8) addr[dev] = static_cast<uint32_t *>(p);
  return static_cast<uint32_t *>(p);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link-time dependency on
// the driver library); null when the driver does not provide it
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

bool make_cell_maps(const TransformPlan &p, uint64_t *x, int64_t stride_limbs, int64_t ext_cells, CellMaps *cm) {
  cm->mode = 0;
  const int NW = p.ring.NW, rows = NW / 32;
  // rings of 8, 16 or 32 words per lane that fill all 32 lanes (rows of 36 words in multiples of
  // 8 rows keep every cell 128-byte aligned in shared memory); 16-byte aligned cells whose stride
  // leaves the limb after the top limb inside the cell's stride (the load box reads it)
  if (!p.tma || p.ring.G != 32 || p.ring.K < 8 || (rows & 7) != 0 || ext_cells <= 0 || ext_cells > INT32_MAX)
    return false;
  if ((reinterpret_cast<uintptr_t>(x) & 15) != 0 || (stride_limbs & 1) != 0 || stride_limbs < NW / 2 + 2) return false;
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t ext = cuuint64_t(ext_cells);
  const cuuint64_t dims_ld[3] = {36, cuuint64_t(rows), ext}, dims_st[3] = {32, cuuint64_t(rows), ext};
  const cuuint64_t strides[2] = {128, cuuint64_t(stride_limbs) * 8};
  const cuuint32_t box[3] = {36, cuuint32_t(rows), 1}, elem[3] = {1, 1, 1};
  if (enc(&cm->ld, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, x, dims_ld, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  if (enc(&cm->st, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, x, dims_st, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  cm->mode = 3;
  return true;
}

// one launch of a plan's per-pass form, by the ring's words per lane
static cudaError_t launch_any(const TransformPlan &p, const Launch &L, uint64_t *x, int64_t stride_limbs,
                              cudaStream_t s, int64_t reps, int64_t rep_cells, uint32_t *fault, const CellMaps *cm) {
  const bool sq = p.mode == RING_SQRT2;
#define TFT_PL(KK) (sq ? launch_plain_k##KK##_sq(p, L, x, stride_limbs, s, reps, rep_cells, fault, cm) \
                       : launch_plain_k##KK##_w2(p, L, x, stride_limbs, s, reps, rep_cells, fault, cm))
  switch (p.ring.K) {
    case 1: return TFT_PL(1);
    case 2: return TFT_PL(2);
    case 4: return TFT_PL(4);
    case 8: return TFT_PL(8);
    case 16: return TFT_PL(16);
    case 32: return TFT_PL(32);
    default: return cudaErrorInvalidValue;
  }
#undef TFT_PL
}

cudaError_t run_transform_reps(const TransformPlan &p, uint64_t *x, int64_t stride_limbs, int64_t reps,
                               int64_t rep_cells, cudaStream_t s) {
  if (reps < 1) return cudaSuccess;
  uint32_t *fault = fault_word();
  if (!fault) return cudaErrorInvalidSymbol;
  // tensor maps over every cell the launches touch (replicas included)
  CellMaps cm;
  const bool maps = make_cell_maps(p, x, stride_limbs, (reps - 1) * rep_cells + p.cell_extent, &cm);
  for (const Launch &L : p.launches) {
    if (reps > 1 && L.nsegs != 0) return cudaErrorInvalidValue;
    cudaError_t e;
    if (p.stream && reps == 1 && L.nsegs == 0 && L.lc == 0 && p.ring.K >= 4 && p.ring.G == 32) {
      // direct: sync is null and njobs negative, one CTA per job (see launch_km)
      const FusedArgs plain = {L.d_jobs, nullptr, nullptr, nullptr, p.direct ? -L.njobs : L.njobs};
      e = p.ring.K == 32 ? launch_fused_k32(p, x, stride_limbs, s, plain, fault, &L, maps ? &cm : nullptr)
                         : launch_fused_small(p, x, stride_limbs, s, plain, fault, &L, maps ? &cm : nullptr);
    } else {
      e = launch_any(p, L, x, stride_limbs, s, reps, rep_cells, fault, maps ? &cm : nullptr);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t run_transform(const TransformPlan &p, uint64_t *x, int64_t stride_limbs, cudaStream_t s,
                          bool allow_fused) {
  if (!allow_fused || p.f_njobs == 0 || p.ring.K < 4 || p.ring.G != 32)
    return run_transform_reps(p, x, stride_limbs, 1, 0, s);
  uint32_t *fault = fault_word();
  if (!fault) return cudaErrorInvalidSymbol;
  // claim counter and done flags, zeroed, for this call only (two calls of one plan may overlap
  // on different streams)
  uint32_t *sync = nullptr;
  const size_t bytes = (size_t(p.f_njobs) + 1) * sizeof(uint32_t);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&sync), bytes, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(sync, 0, bytes, s);
  if (e == cudaSuccess) {
    const FusedArgs fa = {p.f_jobs, p.f_dep_off, p.f_deps, sync, p.f_njobs};
    CellMaps cm;
    const CellMaps *pm = make_cell_maps(p, x, stride_limbs, p.cell_extent, &cm) ? &cm : nullptr;
    e = p.ring.K == 32 ? launch_fused_k32(p, x, stride_limbs, s, fa, fault, nullptr, pm)
                       : launch_fused_small(p, x, stride_limbs, s, fa, fault, nullptr, pm);
  }
  const cudaError_t ef = cudaFreeAsync(sync, s);
  return e != cudaSuccess ? e : ef;
}

namespace {

// One warp waits on an mbarrier that nothing completes until limit_ns passes, and reports it
// as the job kernel reports a bulk load that did not land.
__global__ void wait_probe_kernel(uint64_t limit_ns) {
  __shared__ alignas(8) uint64_t bar;
  const uint32_t mb = uint32_t(__cvta_generic_to_shared(&bar));
  if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
  __syncthreads();
  const bool landed = mbar_wait_bounded(mb, 0, limit_ns);
  if (__syncthreads_or(!landed) && threadIdx.x == 0) atomicOr(&g_wait_fault, 1u);
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mb) : "memory");
}

__global__ void take_wait_fault_kernel(uint32_t *out) { *out = atomicExch(&g_wait_fault, 0u); }

}  // namespace

cudaError_t run_wait_probe(uint64_t limit_ns, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(limit_ns);
  return cudaGetLastError();
}

cudaError_t read_wait_status(uint32_t *fault, cudaStream_t s) {
  uint32_t *d = nullptr, v = 0;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d), sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  take_wait_fault_kernel<<<1, 1, 0, s>>>(d);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  const cudaError_t ef = cudaFreeAsync(d, s);
  if (e == cudaSuccess) e = ef;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) *fault = v;
  return e;
}

}  // namespace tftgpu
