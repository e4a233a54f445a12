// k_sumfact32_alt.cu -- the persistent FP32 / BF16 sum-factorization kernels in
// their non-default variants, timed by the batch autotuner against the default
// ones (k_sumfact32.cu, k_stream32.cu) and against the warp-per-element form
// (k_warp32.cu):
//   MODE_ALT_FORM: p = 3: stage 3 on warp-level mma.sync instead of tcgen05;
//                  p = 4, 5: the other of the two forms there -- the
//                  CTA-per-element form with symmetric operand rows and a
//                  staged element matrix (mma.sync for FP32 and at p = 5,
//                  tcgen05 for BF16 at p = 4), and the streamed form of
//                  k_stream32.cu (the default except at p = 4 with a general map);
//   MODE_ALT_CTA:  that staged form with the other CTA size (512 threads at
//                  p = 4, 256 at p = 5; identity geometry, where 512 threads fit
//                  the registers).
// A separate translation unit, so that these instantiations compile in
// parallel with the default ones.
#include "k_sumfact32.cuh"

namespace iga {
namespace {

// FLAG: the MODE flags of the instantiation (MODE_ALT_FORM at p >= 4 selects
// the staged form, which is that class's flagless instantiation).
template <int P, int QG, bool BF, int FLAG0>
cudaError_t runq_alt(const QueueArgs& b, int mode, int grid, cudaStream_t st, int* max_grid) {
  constexpr int FLAG = (P >= 4 && FLAG0 == MODE_ALT_FORM) ? 0 : FLAG0;
  if (b.jac) {
    if constexpr (FLAG0 == MODE_ALT_CTA) {
      return cudaErrorInvalidValue;   // general maps keep 256 threads (registers)
    } else {
      if (mode == 0) return run_queue<P, QG, true, 0 | FLAG, BF>(b, grid, st, max_grid);
      if (mode == 1) return run_queue<P, QG, true, 1 | FLAG, BF>(b, grid, st, max_grid);
      return run_queue<P, QG, true, 2 | FLAG, BF>(b, grid, st, max_grid);
    }
  }
  if (mode == 0) return run_queue<P, QG, false, 0 | FLAG, BF>(b, grid, st, max_grid);
  if (mode == 1) return run_queue<P, QG, false, 1 | FLAG, BF>(b, grid, st, max_grid);
  return run_queue<P, QG, false, 2 | FLAG, BF>(b, grid, st, max_grid);
}

}  // namespace

bool f32_variant_supported(int p, int q, bool bf16, int variant) {
  if (variant == MODE_ALT_FORM)
    return (p == 3 && (q == 4 || q == 5)) || (p == 4 && (q == 5 || q == 6)) || (p == 5 && q == 6);
  // BF16 at p = 4 has no 512-thread staged form (its staged form is tcgen05)
  if (variant == MODE_ALT_CTA) return (!bf16 && p == 4 && (q == 5 || q == 6)) || (p == 5 && q == 6);
  return false;
}

cudaError_t launch_sumfact_f32_queue_alt(const QueueArgs& b, int p, int q, bool bf16, int mode,
                                         int variant, int grid, cudaStream_t st, int* max_grid) {
  if (!f32_variant_supported(p, q, bf16, variant)) return cudaErrorInvalidValue;
  // p = 4 with a general map defaults to the staged form: its other form is the
  // streamed one
  if (variant == MODE_ALT_FORM && p == 4 && b.jac)
    return launch_sumfact_f32_stream_queue(b, p, q, bf16, mode, grid, st, max_grid);
  if (variant == MODE_ALT_FORM) {
    if (p == 3 && q == 4) return bf16 ? runq_alt<3, 4, true, MODE_ALT_FORM>(b, mode, grid, st, max_grid)
                                      : runq_alt<3, 4, false, MODE_ALT_FORM>(b, mode, grid, st, max_grid);
    if (p == 3 && q == 5) return bf16 ? runq_alt<3, 5, true, MODE_ALT_FORM>(b, mode, grid, st, max_grid)
                                      : runq_alt<3, 5, false, MODE_ALT_FORM>(b, mode, grid, st, max_grid);
    if (p == 4 && q == 5) return bf16 ? runq_alt<4, 5, true, MODE_ALT_FORM>(b, mode, grid, st, max_grid)
                                      : runq_alt<4, 5, false, MODE_ALT_FORM>(b, mode, grid, st, max_grid);
    if (p == 4 && q == 6) return bf16 ? runq_alt<4, 6, true, MODE_ALT_FORM>(b, mode, grid, st, max_grid)
                                      : runq_alt<4, 6, false, MODE_ALT_FORM>(b, mode, grid, st, max_grid);
    return bf16 ? runq_alt<5, 6, true, MODE_ALT_FORM>(b, mode, grid, st, max_grid)
                : runq_alt<5, 6, false, MODE_ALT_FORM>(b, mode, grid, st, max_grid);
  }
  if (p == 4 && q == 5) return bf16 ? runq_alt<4, 5, true, MODE_ALT_CTA>(b, mode, grid, st, max_grid)
                                    : runq_alt<4, 5, false, MODE_ALT_CTA>(b, mode, grid, st, max_grid);
  if (p == 4 && q == 6) return bf16 ? runq_alt<4, 6, true, MODE_ALT_CTA>(b, mode, grid, st, max_grid)
                                    : runq_alt<4, 6, false, MODE_ALT_CTA>(b, mode, grid, st, max_grid);
  return bf16 ? runq_alt<5, 6, true, MODE_ALT_CTA>(b, mode, grid, st, max_grid)
              : runq_alt<5, 6, false, MODE_ALT_CTA>(b, mode, grid, st, max_grid);
}

}  // namespace iga
