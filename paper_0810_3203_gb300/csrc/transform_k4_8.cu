// Per-pass launches of the sub-transform kernel (job_kernel.cuh) for rings of four or eight words per lane (N = 4096 .. 8192).
#include "job_kernel.cuh"

namespace tftgpu {

TFT_DEFINE_PLAIN(4, w2, false)
TFT_DEFINE_PLAIN(4, sq, true)
TFT_DEFINE_PLAIN(8, w2, false)
TFT_DEFINE_PLAIN(8, sq, true)

}  // namespace tftgpu
