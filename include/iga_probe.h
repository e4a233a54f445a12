/*
 * iga_probe.h -- measurement probes of the GB300 arithmetic rates that the
 * rooflines of the integration kernels divide by.  They are not part of the
 * integration path of iga.h: the paper (arxiv 2207.00280) states its cost in
 * operation counts (Sec. 1.2, the O(p^9) classical and O(p^6)-per-stage sum
 * factorization counts; Sec. 3.2), and a roofline turns such a count into a
 * time only through the rate of the unit that executes it.  GB300's FP64 rate
 * is not in the measured peaks (a copy bandwidth and a BF16 GEMM), so
 * the library measures it itself.
 *
 * iga_probe_rate runs one throughput kernel on `cuda_stream` (a cudaStream_t,
 * NULL = legacy default stream), times it with CUDA events recorded on that
 * stream around the launch, synchronizes, and returns:
 *   *ms_out     the kernel's device time in milliseconds;
 *   *flops_out  the floating-point operations it executed (multiply-add = 2).
 * kind:
 *   IGA_PROBE_DFMA  independent FP64 fused multiply-add chains on the CUDA cores;
 *   IGA_PROBE_DMMA  FP64 warp-level matrix multiply-accumulate (mma.sync
 *                   m8n8k4 f64, 512 flops per warp instruction);
 *   IGA_PROBE_FFMA  independent FP32 fused multiply-add chains (context for the
 *                   float-float and FP32 kernels).
 * iters: multiply-adds per chain (DFMA/FFMA) or MMAs per warp (DMMA), >= 1.
 * ctas_per_sm: CTAs of 256 threads per SM (grid = SM count x ctas_per_sm), 1..8.
 * Both output pointers are host pointers and must be non-NULL.  Returns an
 * iga_status code (IGA_ERR_ARG for bad arguments, IGA_ERR_CUDA if a CUDA call
 * failed).  So that the compiler cannot drop the arithmetic, each thread
 * compares its result with a value the chains cannot produce and would store
 * it to a file-scope device word if they did; no device memory is allocated.
 * Not for use while other work runs on the GPU: the rate is the whole GPU's.
 */
#ifndef IGA_PROBE_H
#define IGA_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { IGA_PROBE_DFMA = 0, IGA_PROBE_DMMA = 1, IGA_PROBE_FFMA = 2 };

int iga_probe_rate(int kind, int64_t iters, int ctas_per_sm, double* ms_out, double* flops_out,
                   void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* IGA_PROBE_H */
