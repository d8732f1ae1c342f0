// The host planner and job-image builder under AddressSanitizer and UBSan: transform plans over
// a sweep of rings, lengths, weights and both omega modes, and job images of every single-CTA
// and cluster shape. Built and run by tests/test_sanitizers.py; any report fails it.
#include <cstdio>
#include <random>
#include <vector>
#include "../../paper_0810_3203_gb300/csrc/common.h"
#include "../../paper_0810_3203_gb300/csrc/host.h"
using namespace tftgpu;
int main() {
  std::mt19937_64 rng(7);
  long plans = 0, images = 0;
  const int modes[2] = {RING_FERMAT, RING_SQRT2};
  for (int64_t N : {64, 128, 1024, 2048, 4096, 8192, 16384, 32768}) {
    for (int mode : modes) {
      const int64_t ord = (mode == RING_SQRT2 ? 4 : 2) * N;
      for (int l = 1; (int64_t(1) << l) <= ord && l <= 17; l++) {
        const int64_t L = int64_t(1) << l;
        for (int t = 0; t < (l >= 15 ? 2 : 6); t++) {
          const int64_t n = 1 + int64_t(rng() % L);
          const int64_t z = 1 + int64_t(rng() % L);
          HostPlan a;
          build_host_plan(KIND_TFT, l, z, n, 0, N, int64_t(rng() % ord), 0, &a, mode);
          const int f = n < L ? int(rng() & 1) : 0;
          const int64_t zi = n + int64_t(rng() % (L - n + 1));
          HostPlan b;
          build_host_plan(KIND_ITFT, l, zi, n, f, N, int64_t(rng() % ord), 1, &b, mode);
          plans += 2;
          (void)zero_padded_outputs(l, n, N);
        }
      }
    }
  }
  for (int ls = 1; ls <= 8; ls++)
    for (int lc = 0; 2 * lc <= ls && lc <= 4; lc++)
      for (int t = 0; t < 20; t++) {
        const int64_t L = int64_t(1) << ls;
        const int64_t n = 1 + int64_t(rng() % L), z = 1 + int64_t(rng() % L);
        (void)build_job_image(KIND_TFT, ls, lc, z, n, 0, 1024, nullptr, RING_FERMAT);
        const int f = n < L ? int(rng() & 1) : 0;
        (void)build_job_image(KIND_ITFT, ls, lc, n + int64_t(rng() % (L - n + 1)), n, f, 1024, nullptr, RING_SQRT2);
        images += 2;
      }
  std::printf("plans %ld images %ld\n", plans, images);
  return 0;
}
