// Host-side internals of libtftgpu: program generation, transform planning and launches.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tftgpu.h"
#include "common.h"

namespace tftgpu {

enum { KIND_TFT = 0, KIND_ITFT = 1 };

struct ProgramStats {
  int nops = 0;
  int nlevels = 0;
};

// Program image for a sub-transform of length 2^ls held entirely on chip (see common.h).
// mode (RingMode): RING_SN programs are for S[y]/(y^{N}+1) (2N = M), where doublings and
// halvings are scalar flags; RING_SQRT2 programs take exponents of sqrt2 (mod 4N).
std::vector<uint32_t> build_program(int kind, int ls, int64_t z, int64_t n, int f, int64_t N,
                                    ProgramStats *stats, int mode = RING_FERMAT);

// Job image (stage table plus per-CTA programs, see common.h) for a job of 2^ls cells on a
// cluster of 2^lc CTAs.
// Largest per-CTA program (words) in a job image.
int image_max_program_words(const std::vector<uint32_t> &img);
std::vector<uint32_t> build_job_image(int kind, int ls, int lc, int64_t z, int64_t n, int f, int64_t N,
                                      ProgramStats *stats, int mode = RING_FERMAT);

// Ring geometry used by the kernels.
struct Ring {
  int64_t N = 0;
  int NW = 0;     // 32-bit words of an N-bit value
  int K = 0;      // words per lane
  int G = 0;      // lanes holding words (NW / K)
  int pitch = 0;  // shared-memory words per cell
};
bool ring_supported(int64_t N);
Ring make_ring(int64_t N);

// Launch configuration of the plans over one ring: the largest job one CTA holds (ls_max),
// the cells per CTA of a cluster job (ls_c, both log2), the warps per CTA (8 or 16) and the
// top-level split (0: L1 = 2^floor(l/2) as in the paper, 1: L1 = 2^ceil(l/2)). Every choice
// computes the same outputs; they differ in speed. zx_tune measures the candidates.
// fused, the launch form of plans whose jobs all run on single CTAs (rings that fill all 32
// lanes; other plans always launch job_kernel once per pass):
//   0 one launch per pass of job_kernel (segment and replica logic included);
//   1 one persistent launch per transform that claims the jobs in dependency order
//     (FusedSchedule), 2 the same for the ITFT only;
//   3 one launch per pass as a persistent loop over its jobs that prefetches a CTA's next job into
//     L2 while it computes the current one;
//   4 one launch per pass, one CTA per job, through the persistent kernels' instantiation: the
//     default. With row copies that job body fit the registers of three CTAs per SM without
//     spilling where job_kernel spilled (46 bytes a thread, which the L1 beside 225 KB of shared
//     memory could not hold), and it ran 4 % faster on GB300; with tensor copies (tma) the two
//     measure within 1 %.
// Measured at l = 16, N = 32768: alone, the persistent ITFT is faster from n = 40000 on, the TFT
// slower; with several transforms on concurrent streams, persistent launches hold every CTA slot
// until they finish and the transforms stop overlapping (the five-stream benchmark step went from
// 4.74 to 5.18 ms). zx_tune times single round trips and therefore leaves this setting as it is;
// zx_config_set chooses it.
enum { FUSED_NONE = 0, FUSED_ALL = 1, FUSED_ITFT = 2, FUSED_STREAM = 3, FUSED_DIRECT = 4 };
inline bool fused_for(int fused, int kind) { return fused == FUSED_ALL || (fused == FUSED_ITFT && kind == KIND_ITFT); }
// max_lc caps cluster jobs at 2^max_lc CTAs (at most kMaxClusterLog2). split 2: at every level,
// the split with the fewest global-memory passes below it (ties: the one nearest to balanced).
// tma 1: the per-pass launches of single-CTA jobs (fused 3 and 4) move whole cells with one
// tensor copy each (CellMaps) where the ring and the buffer allow it; 0: row copies and 16-byte
// stores everywhere.
struct PlanConfig {
  int ls_max = 0, ls_c = 0, max_warps = 16, split = 0, fused = FUSED_DIRECT, max_lc = 4, tma = 1;
};
PlanConfig default_config(const Ring &r);
bool config_valid(const Ring &r, const PlanConfig &c);
// The configuration used for ring N: the tuned one when set, else the default.
PlanConfig plan_config(int64_t N);
void set_plan_config(int64_t N, const PlanConfig &c);
// Warps per CTA of a job of 2^ls cells on 2^lc CTAs: one per butterfly of a full level, at most
// max_warps.
int warps_for_job(int ls, int lc, int max_warps);

// Largest sub-transform (log2 of its cell count) one CTA holds in shared memory.
int max_onchip_ls(const Ring &r);
// Cells (log2) per CTA of a cluster job: small enough that two CTAs share an SM, so that the
// stages of one job overlap with those of another.
int cluster_cta_ls(const Ring &r);
// Largest cluster (log2 of its CTA count) a job may use (16 CTAs: a non-portable size).
constexpr int kMaxClusterLog2 = 4;

// One kernel launch: jobs of equal ls.
struct Launch {
  int pass = 0;  // global-memory pass of the plan this launch belongs to
  int ls = 0;
  int lc = 0;  // cluster of 2^lc CTAs per job
  int nwarps = 0;
  int njobs = 0;       // jobs of the launch (all segments together when d_segs is set)
  int prog_words = 0;  // largest per-CTA program of the launch (shared-memory staging size)
  JobDesc *d_jobs = nullptr;         // device copy (owned by the plan cache)
  const Segment *d_segs = nullptr;   // merged launch: segments in device memory (d_jobs unused)
  int nsegs = 0;
};

// One persistent launch over every job of a plan whose jobs are all single-CTA jobs. Jobs are
// claimed in `order` (positions in the plan's pass-ordered job list); claimed job k waits for
// the jobs at claim positions deps[dep_off[k] .. dep_off[k + 1]): the last job that stored a
// cell k reads or stores, and every job that read a cell k stores since it was last stored.
// The order is a list schedule over `slots` concurrent CTAs that prefers the deepest pass among
// the jobs whose dependencies are done, so a pass re-reads what the previous one just wrote
// while it is still in L2.
struct FusedSchedule {
  std::vector<int32_t> order;
  std::vector<int32_t> dep_off;
  std::vector<int32_t> deps;
};
// jobs in pass order with their pass numbers; L cells; false (and an empty schedule) when the
// plan does not qualify (a job outside [0, L), or L above 2^22)
bool build_fused_schedule(const std::vector<JobDesc> &jobs, const std::vector<int> &pass, int64_t L, int slots,
                          FusedSchedule *out);

struct TransformPlan {
  Ring ring;
  int mode = RING_FERMAT;  // RingMode of the rotation amounts
  std::vector<Launch> launches;  // in stream order
  int npasses = 0;
  int64_t njobs = 0;
  // the fused form (used when f_njobs > 0 and the caller allows it): one launch of f_ls-sized
  // single-CTA jobs in claim order with their dependency lists, all in device memory
  int f_njobs = 0, f_ls = 0, f_nwarps = 0, f_prog_words = 0;
  const JobDesc *f_jobs = nullptr;
  const int32_t *f_dep_off = nullptr, *f_deps = nullptr;
  // launches of single-CTA jobs run as persistent loops with L2 prefetch (FUSED_STREAM), or
  // through the same kernel with one CTA per job (FUSED_DIRECT)
  bool stream = false, direct = false;
  bool tma = false;  // PlanConfig::tma
  // one more than the largest cell index a job of the plan reads or writes (the extent of the
  // tensor maps of a call's buffer)
  int64_t cell_extent = 0;
};

// Cached plan of TFT (kind = KIND_TFT) or ITFT for the given parameters; nullptr with *err set
// on failure. escale < 0 means no final scaling. `replicated`: the plan runs on many sequences
// at once (run_transform_reps), so a transform that fits one job stays one job (alone, one
// that has more than 64 cells takes two passes to spread over the SMs).
const TransformPlan *get_transform_plan(int kind, int l, int64_t z, int64_t n, int f, int64_t N,
                                        int64_t e, int64_t stride_limbs, int scale, int *err,
                                        int mode = RING_FERMAT, bool replicated = false);

// Outputs a product's transforms compute when the product length n is padded with known zero
// coefficients up to a whole number of rows of the top-level split (Sec. 6): the ITFT then has
// no partial row and is the TFT's steps reversed. Where the column sub-transforms run on
// clusters, n is padded to whole rows of their in-job split too when that costs at most n/32.
// n itself when one CTA holds the transform.
int64_t zero_padded_outputs(int l, int64_t n, int64_t N);

// Number of global-memory passes of a transform (host only; no device needed).
int count_passes(int kind, int l, int64_t z, int64_t n, int f, int64_t N);
// passes, launches and jobs of a transform's plan (host only)
void plan_shape(int kind, int l, int64_t z, int64_t n, int f, int64_t N, int *passes, int *launches,
                int64_t *jobs, int *onchip_l, int *cluster_l);

// Host-side image of a transform plan: the launches with their job lists and the distinct
// program images they use (JobDesc::prog is left null; prog_index names the image).
struct HostPlan {
  struct Group {
    int ls = 0, lc = 0, nwarps = 0, prog_words = 0;
    std::vector<JobDesc> jobs;
    std::vector<int> prog_index;
  };
  Ring ring;
  int npasses = 0;
  std::vector<Group> groups;
  std::vector<std::vector<uint32_t>> programs;
};
void build_host_plan(int kind, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e, int scale,
                     HostPlan *out, int mode = RING_FERMAT);
// The fused schedule of the same plan (empty when it has none), with `order` given as positions
// in HostPlan's launch-major job list.
void build_host_schedule(int kind, int l, int64_t z, int64_t n, int f, int64_t N, int64_t e, int scale,
                         FusedSchedule *out, int mode = RING_FERMAT, int slots = 0);

// Plans over S[y]/(y^{M/2}+1), H = M/2 coefficients per element (single-CTA jobs; the ITFT's
// final division by L is escale = l halvings). nullptr with *err set on failure.
int sn_max_onchip_ls(int64_t H);
const TransformPlan *get_sn_plan(int kind, int l, int64_t z, int64_t n, int f, int64_t H, int64_t e, int scale,
                                 int *err);
void sn_plan_shape(int kind, int l, int64_t z, int64_t n, int f, int64_t H, int *passes, int *launches,
                   int64_t *jobs);
// Enqueue an S[y]/(y^{M/2}+1) plan (sn_kernel.cu).
cudaError_t run_sn_transform(const TransformPlan &p, uint64_t *x, int64_t stride, int64_t H, uint64_t m,
                             cudaStream_t s);

// Enqueue a plan on a stream. A plan with a fused form runs as one persistent launch, whose
// claim counter and done flags come from the stream-ordered allocator; allow_fused = false
// keeps one launch per pass and allocates nothing.
cudaError_t run_transform(const TransformPlan &p, uint64_t *x, int64_t stride_limbs,
                          cudaStream_t s, bool allow_fused = true);
// The same plan applied to `reps` buffers of rep_cells cells each, back to back from x: every
// launch covers all of them (replica r shifts each job by r * rep_cells cells).
cudaError_t run_transform_reps(const TransformPlan &p, uint64_t *x, int64_t stride_limbs, int64_t reps,
                               int64_t rep_cells, cudaStream_t s);

// Bounded device waits (transform_kernel.cu). A job kernel whose bulk load did not land within
// its limit stops and sets a per-device status word; read_wait_status synchronises s, then
// returns that word in *fault and clears it (atomically on the device). run_wait_probe enqueues
// one warp that waits limit_ns on a barrier nothing completes and reports it the same way.
cudaError_t read_wait_status(uint32_t *fault, cudaStream_t s);
cudaError_t run_wait_probe(uint64_t limit_ns, cudaStream_t s);

// Pointwise products by a second Schoenhage-Strassen level (rec_pointwise.cu): 2^k pieces of
// M = N / 2^k bits, inner ring Z/(2^Ni + 1) with Ni >= 2M + k + 1 and 2^k | Ni.
struct RecPlan {
  int64_t N = 0, M = 0, Ni = 0, stride_i = 0;
  int k = 0;
  int nwp = 0;        // 32-bit words of a recovered piece c_t + 2^{k+2M}
  double cost = 0.0;  // word operations per outer product (estimate)
};
bool rec_plan_for(int64_t N, int k, RecPlan *out);
bool rec_plan_auto(int64_t N, RecPlan *out);
// a_i <- a_i b_i mod 2^N + 1 for i < n (canonical cells of stride limbs); *err gets a ZX_ code
cudaError_t run_rec_pointwise(uint64_t *a, const uint64_t *b, int64_t n, int64_t stride, const Ring &ro,
                              const RecPlan &rp, cudaStream_t s, int *err);

// Kernels of the Z[x] path (zx_kernels.cu).
cudaError_t launch_pack(const uint64_t *coef, int64_t len, int64_t limbs, int is_signed,
                        uint64_t *cells, int64_t stride_limbs, const Ring &r, cudaStream_t s);
cudaError_t launch_pointwise(uint64_t *a, const uint64_t *b, int64_t n, int64_t stride_limbs,
                             const Ring &r, cudaStream_t s);
cudaError_t launch_lift(const uint64_t *cells, int64_t n, int64_t stride_limbs, int is_signed,
                        uint64_t *out, int64_t limbs_out, const Ring &r, cudaStream_t s);

// Batched forms over many products of one ring (item descriptors in device memory). Cell
// arrays are given as limb offsets from `pool`; operands and outputs as device pointers.
struct PackItem {
  const uint64_t *coef;
  int64_t cells;  // limb offset of the first cell in the pool
  int64_t len, limbs;
  int32_t is_signed, pad;
};
struct PointwiseItem {
  int64_t a, b;   // limb offsets of the two cell arrays (a <- a * b)
  int64_t n;
  int64_t first;  // the group's products before this item's (items in order, first ascending)
};
struct LiftItem {
  int64_t cells;  // limb offset
  uint64_t *out;
  int64_t n, limbs_out;
  int32_t is_signed, pad;
};
cudaError_t launch_pack_batch(const PackItem *d_items, int count, int64_t max_len, int64_t stride_limbs,
                              const Ring &r, uint64_t *pool, cudaStream_t s);
cudaError_t launch_pointwise_batch(const PointwiseItem *d_items, int count, int64_t total, int64_t stride_limbs,
                                   const Ring &r, uint64_t *pool, cudaStream_t s);
cudaError_t launch_lift_batch(const LiftItem *d_items, int count, int64_t max_n, int64_t stride_limbs,
                              const Ring &r, uint64_t *pool, cudaStream_t s);

// One product of a batch (operands and output in device memory; ring chosen by the caller).
struct BatchProduct {
  const uint64_t *f = nullptr, *g = nullptr;
  uint64_t *h = nullptr;
  int64_t len_f = 0, len_g = 0, limbs_f = 0, limbs_g = 0, limbs_h = 0;
  int32_t signed_f = 0, signed_g = 0, sgn = 0, l = 0;
  int64_t N = 0, n = 0, nf = 0, stride = 0;  // nf: zero-padded transform outputs
  int mode = RING_FERMAT;                      // omega = 2, or sqrt2 (RING_SQRT2)
};
// Checks one product of device operands and fills *b (api.cu); ZX_* status with the error
// text set on failure. h->limbs is overwritten with the needed count on ZX_EBUFSIZE.
int device_product(const zx_poly *f, const zx_poly *g, zx_poly *h, BatchProduct *b);

// Enqueue the products on `s` (zx_batch.cu). Returns ZX_OK or a ZX_* status with *msg set.
int run_mul_batch(const std::vector<BatchProduct> &items, cudaStream_t s, std::string *msg);

// Products of one ring laid out in a pool: item arrays and merged per-pass job lists, all as
// byte offsets into a descriptor image that is copied to the device as one block.
struct BatchGroup {
  Ring ring;
  int mode = RING_FERMAT;
  int64_t stride = 0;
  int count = 0;
  int64_t max_len = 0, max_n = 0;
  int64_t pw_total = 0;  // pointwise products of the group (the sum of its items' n)
  size_t pack_off = 0, pw_off = 0, lift_off = 0;
  std::vector<Launch> tft, itft;  // merged launches; d_segs hold descriptor-image byte offsets
  int64_t cell_end = 0;           // the group's cells end here (cells of `stride` from the pool's start)
};
struct BatchLayout {
  size_t pool_bytes = 0;
  std::vector<BatchGroup> groups;
};
// Ring buffer bytes of one product (two buffers of L cells).
size_t product_pool_bytes(const BatchProduct &p);
// Lay out the products idx (any order; grouped by ring inside) in one pool, appending their
// descriptors to *desc (16-byte aligned). ZX_* status with *msg set on failure.
int layout_batch(const std::vector<BatchProduct> &items, const std::vector<int> &idx,
                 std::vector<unsigned char> *desc, BatchLayout *out, std::string *msg);
// Enqueue one ring group: descriptors at d_desc on the device, ring buffers at pool.
cudaError_t enqueue_group(const BatchGroup &g, unsigned char *d_desc, unsigned char *pool, cudaStream_t s);

// per-thread error text
void set_error(const std::string &msg);

}  // namespace tftgpu
