// k_sumfact32.cu -- launchers of the FP32 / BF16 sum-factorized element
// matrices (kernels in k_sumfact32.cuh).
#include "k_sumfact32.cuh"

namespace iga {

bool sumfact_f32_supported(int dim, int p, int q) {
  return dim == 3 && p >= 1 && p <= 5 && (q == p + 1 || (q == p + 2 && p <= 4));
}

bool queue_both_fit(int p, int q, bool bf16) {
  if (stream_form_supported(p, q)) return stream_both_fit(p, q, bf16);
#define F(PP, QQ)                                                           \
  if (p == PP && q == QQ)                                                   \
    return bf16 ? (SF3F<PP, QQ, true, 0, true>::smem <= 227 * 1024 &&       \
                   SF3F<PP, QQ, false, 0, true>::smem <= 227 * 1024)        \
                : (SF3F<PP, QQ, true, 0, false>::smem <= 227 * 1024 &&      \
                   SF3F<PP, QQ, false, 0, false>::smem <= 227 * 1024);
  F(1, 2) F(1, 3) F(2, 3) F(2, 4) F(3, 4) F(3, 5)
#undef F
  return false;
}

cudaError_t launch_sumfact_f32(const ElemArgs& a, int dim, int p, int q, bool bf16,
                               cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  if (dim != 3) return cudaErrorInvalidValue;
  // p = 5, and p = 4 with the identity map: the streamed tcgen05 form.  With a
  // general map at p = 4 its doubled stage 2 (all n^4 operand rows, with the
  // off-diagonal terms) costs more than the staged form's scatter: measured on
  // GB300, 48^3 curved FP32 8.3 ms streamed against 4.5 ms staged.
  if (stream_form_supported(p, q) && !(p == 4 && a.jac))
    return launch_sumfact_f32_stream(a, p, q, bf16, st);
  // the stiffness alone with a general map at p = 4, q = 5: k_curved32.cu
  if (curved_form_supported(p, q) && a.jac && a.K_out && !a.M_out)
    return launch_sumfact_f32_curved(a, bf16, st);
  const int dq = q - p;
#define C3(PP)                                                                                  \
  if (p == PP && dq == 1) return bf16 ? runm<PP, PP + 1, true>(a, st) : runm<PP, PP + 1, false>(a, st); \
  if (p == PP && dq == 2) return bf16 ? runm<PP, PP + 2, true>(a, st) : runm<PP, PP + 2, false>(a, st);
  C3(1) C3(2) C3(3) C3(4)
#undef C3
  return cudaErrorInvalidValue;
}

cudaError_t launch_sumfact_f32_queue(const QueueArgs& b, int p, int q, bool bf16, int mode,
                                     int grid, cudaStream_t st, int* max_grid) {
  // the same form choice as the per-patch launch (so that the default
  // persistent schedules reproduce it bit for bit)
  if (stream_form_supported(p, q) && !(p == 4 && b.jac))
    return launch_sumfact_f32_stream_queue(b, p, q, bf16, mode, grid, st, max_grid);
  if (curved_form_supported(p, q) && b.jac && mode == 1)
    return launch_sumfact_f32_curved_queue(b, bf16, grid, st, max_grid);
  const int dq = q - p;
#define C3(PP)                                                                                \
  if (p == PP && dq == 1) return bf16 ? runq<PP, PP + 1, true>(b, mode, grid, st, max_grid)   \
                                      : runq<PP, PP + 1, false>(b, mode, grid, st, max_grid); \
  if (p == PP && dq == 2) return bf16 ? runq<PP, PP + 2, true>(b, mode, grid, st, max_grid)   \
                                      : runq<PP, PP + 2, false>(b, mode, grid, st, max_grid);
  C3(1) C3(2) C3(3) C3(4)
#undef C3
  return cudaErrorInvalidValue;
}

}  // namespace iga
