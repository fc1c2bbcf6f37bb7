// The exact line search's step (Sec. 3.2) for a batch of cubics, through the two device solvers
// the iteration runs: one thread per cubic (the per-column cubics of TriOFM, Eqs. (16)/(18)) and
// one warp per cubic (the single cubic of OFM, Eqs. (15)/(17)), so that the root choice can be
// checked on its own against the FP64 oracle and the two solvers against each other.
#include <algorithm>

#include "common.cuh"
#include "cubic.cuh"

namespace ofsc {
namespace {

constexpr int kStepThreads = 256;

__global__ void __launch_bounds__(kStepThreads) k_step_thread(int64_t n, const double* __restrict__ coef,
                                                              double* __restrict__ steps, int* __restrict__ bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int b = 0;
    const double* c = coef + 4 * i;
    steps[i] = pick_step(c[0], c[1], c[2], c[3], &b);
    if (bad) bad[i] = b;
  }
}

// One warp per cubic; the loop index is the same in every lane of a warp, as pick_step_warp needs.
__global__ void __launch_bounds__(kStepThreads) k_step_warp(int64_t n, const double* __restrict__ coef,
                                                            double* __restrict__ steps, int* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    int b = 0;
    const double* c = coef + 4 * i;
    const double s = pick_step_warp(c[0], c[1], c[2], c[3], &b);
    if (lane == 0) {
      steps[i] = s;
      if (bad) bad[i] = b;
    }
  }
}

}  // namespace
}  // namespace ofsc

using namespace ofsc;

extern "C" ofsc_status ofsc_line_search_step(int64_t n, const double* coef, int32_t solver, double* steps,
                                             int32_t* bad, void* stream_) {
  clear_error();
  if (n < 0) return fail(OFSC_ERR_INVALID_ARG, "ofsc_line_search_step: n=%lld < 0", (long long)n);
  if (solver != 0 && solver != 1)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_line_search_step: solver must be 0 (thread) or 1 (warp), not %d", solver);
  if (n == 0) return OFSC_OK;
  if (!coef || !steps) return fail(OFSC_ERR_INVALID_ARG, "ofsc_line_search_step: coef or steps is NULL");
  cudaStream_t s = (cudaStream_t)stream_;
  const int64_t threads = solver == 0 ? n : 32 * n;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(threads, kStepThreads), 8 * kNumSMs));
  if (solver == 0)
    k_step_thread<<<grid, kStepThreads, 0, s>>>(n, coef, steps, bad);
  else
    k_step_warp<<<grid, kStepThreads, 0, s>>>(n, coef, steps, bad);
  OFSC_LAUNCH_CHECK("ofsc_line_search_step");
  return OFSC_OK;
}
