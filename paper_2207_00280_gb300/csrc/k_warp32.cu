// k_warp32.cu -- warp-per-element schedule of the FP32 sum-factorized element
// matrices (3D, p <= 2), for the persistent batched launch.
//
// The paper's concurrency levels (Sec. 3.3) put elements on level 2 and the
// entries of one element matrix on level 3.  The CTA-per-element kernel of
// k_sumfact32.cu spreads one element over a whole CTA (thread per entry);
// at p <= 2 an element matrix has at most 27 x 27 entries, so most of its
// threads wait at the barriers between the stages.  Here every warp pops its
// own work items from the class's queue and integrates its elements alone,
// with __syncwarp between the stages of Algorithm 2 (z, then y, then x) and
// no CTA-wide barrier, so the warps of an SM are always at different stages.
// The autotuner of the batched schedule times both forms per (p, q) class.
//
// Arithmetic: the Jacobian cofactors and determinant in FP64 (as the CTA
// form), everything else in FP32 on the CUDA cores.  There is no tensor-core
// stage: for BF16 plans this form is therefore more accurate than the BF16
// CTA form (its last contraction is FP32, not BF16).
#include "iga_internal.h"

namespace iga {
namespace {

__device__ __forceinline__ unsigned long long wq_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int kWarps = 4;   // warps per CTA (128 threads)

template <int P, int QG, bool GEN, int MODE>
struct W32 {
  static constexpr bool DK = MODE != 2, DM = MODE != 1;
  static constexpr int n = P + 1, q = QG, n2 = n * n, N = n2 * n, Q = q * q * q;
  static constexpr int REC = 2 * q * n + q;
  static constexpr int NI = GEN ? 9 : 3, NC = GEN ? 7 : 2;
  static constexpr int S = N * (N + 1) / 2;
  // per-warp shared memory, floats
  static constexpr int f_rec = 3 * REC;
  static constexpr int f_pat = 3 * 4 * n2 * q;     // [dir][pattern][a][b][k]
  static constexpr int f_coef = NC * Q;
  static constexpr int f_T1 = NI * n2 * q * q;     // [item][a3][b3][k1][k2]
  static constexpr int f_C = 5 * n2 * n2 * q;      // [X][a'][b'][k1], a' = a2 + n a3
  static constexpr int per_warp = (f_rec + f_pat + f_coef + f_T1 + f_C + 3) / 4 * 4;
  static constexpr size_t smem = (size_t)kWarps * per_warp * 4;
};

// Stage-1 items (z pattern, coefficient) and stage-2 terms per C buffer
// (x pattern 11, 10, 01, 00, mass): (y pattern, item); patterns 0 = (v, v),
// 1 = (d, d), 2 = (d, v), 3 = (v, d), test factor first.  Stiffness term
// (i, j) differentiates the test function in direction i and the trial
// function in direction j.  General map, coefficients {D00, D11, D01, DM,
// D22, D02, D12}:
//   items (00,D00) (00,D01) (00,D11) (11,D22) (10,D02) (10,D12) (01,D02) (01,D12) (00,DM);
//   C0 = (00,I0); C1 = (01,I1) + (00,I6); C2 = (10,I1) + (00,I4);
//   C3 = (11,I2) + (10,I7) + (01,I5) + (00,I3); C4 = (00,I8).
// Identity map, coefficients {W kappa, W rho}: items (00,Dk) (11,Dk) (00,DM);
//   C0 = (00,J0); C3 = (11,J0) + (00,J1); C4 = (00,J2).
__device__ __constant__ int wItemGen[9][2] = {{0, 0}, {0, 2}, {0, 1}, {1, 4}, {2, 5},
                                              {2, 6}, {3, 5}, {3, 6}, {0, 3}};
__device__ __constant__ int wItemId[3][2] = {{0, 0}, {1, 0}, {0, 1}};
__device__ __constant__ int wTermGen[5][4][2] = {
    {{0, 0}, {-1, -1}, {-1, -1}, {-1, -1}},
    {{3, 1}, {0, 6}, {-1, -1}, {-1, -1}},
    {{2, 1}, {0, 4}, {-1, -1}, {-1, -1}},
    {{1, 2}, {2, 7}, {3, 5}, {0, 3}},
    {{0, 8}, {-1, -1}, {-1, -1}, {-1, -1}}};
__device__ __constant__ int wTermId[5][4][2] = {
    {{0, 0}, {-1, -1}, {-1, -1}, {-1, -1}},
    {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}},
    {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}},
    {{1, 0}, {0, 1}, {-1, -1}, {-1, -1}},
    {{0, 2}, {-1, -1}, {-1, -1}, {-1, -1}}};
__device__ __constant__ int wXPat[5] = {1, 2, 3, 0, 0};

// One element, by one warp.  All buffers are the warp's own slice of shared
// memory; __syncwarp orders the stages.
template <int P, int QG, bool GEN, int MODE>
__device__ __forceinline__ void w32_element(const PatchDev& pd, const QueueArgs& B, int64_t e,
                                            float* base, int lane) {
  using C = W32<P, QG, GEN, MODE>;
  constexpr int n = C::n, q = C::q, n2 = C::n2, N = C::N, Q = C::Q, REC = C::REC;
  constexpr int NI = C::NI, NC = C::NC;
  float* rec = base;
  float* pat = rec + C::f_rec;
  float* coef = pat + C::f_pat;
  float* T1 = coef + C::f_coef;
  float* Cb = T1 + C::f_T1;
  const int e1 = (int)(e % pd.K[0]);
  const int e2 = (int)((e / pd.K[0]) % pd.K[1]);
  const int e3 = (int)(e / ((int64_t)pd.K[0] * pd.K[1]));
  // basis records of the three directions (FP64 tables -> FP32); the offsets
  // are selected, not indexed, so that the patch record stays in registers
  const int64_t to0 = pd.tab_offset[0] + (int64_t)e1 * REC, to1 = pd.tab_offset[1] + (int64_t)e2 * REC,
                to2 = pd.tab_offset[2] + (int64_t)e3 * REC;
  for (int i = lane; i < 3 * REC; i += 32) {
    const int d = i / REC, j = i - d * REC;
    rec[i] = (float)B.tables[(d == 0 ? to0 : (d == 1 ? to1 : to2)) + j];
  }
  __syncwarp();
  // 1D factor patterns of every direction: pat[d][pt][a][b][k]
  for (int i = lane; i < C::f_pat; i += 32) {
    const int k = i % q, b = (i / q) % n, a = (i / (q * n)) % n, pt = (i / (q * n2)) % 4,
              d = i / (4 * q * n2);
    const float* v = rec + d * REC;
    const float* dv = v + q * n;
    const int sa = (pt == 1 || pt == 2), sb = (pt == 1 || pt == 3);
    pat[i] = (sa ? dv : v)[k * n + a] * (sb ? dv : v)[k * n + b];
  }
  // coefficients at the quadrature points
  const int64_t g0 = pd.qp_offset + e * Q;
  for (int k = lane; k < Q; k += 32) {
    const int k1 = k % q, k2 = (k / q) % q, k3 = k / (q * q);
    const float* w0 = rec + 2 * q * n;
    const float W = w0[k1] * (w0 + REC)[k2] * (w0 + 2 * REC)[k3];
    const float kp = B.kappa ? (float)B.kappa[g0 + k] : 1.f;
    const float rh = B.rho ? (float)B.rho[g0 + k] : 1.f;
    if (GEN) {
      const double* G = B.jac + (g0 + k) * 9;
      const double g00 = G[0], g01 = G[1], g02 = G[2], g10 = G[3], g11 = G[4], g12 = G[5],
                   g20 = G[6], g21 = G[7], g22 = G[8];
      const double d00 = g11 * g22 - g12 * g21, d01 = g12 * g20 - g10 * g22,
                   d02 = g10 * g21 - g11 * g20;
      const double det = g00 * d00 + g01 * d01 + g02 * d02;
      const float c00 = (float)d00, c01 = (float)d01, c02 = (float)d02;
      const float c10 = (float)(g02 * g21 - g01 * g22), c11 = (float)(g00 * g22 - g02 * g20),
                  c12 = (float)(g01 * g20 - g00 * g21);
      const float c20 = (float)(g01 * g12 - g02 * g11), c21 = (float)(g02 * g10 - g00 * g12),
                  c22 = (float)(g00 * g11 - g01 * g10);
      const float adet = (float)fabs(det);
      const float s = W * kp / adet;
      coef[0 * Q + k] = s * (c00 * c00 + c10 * c10 + c20 * c20);
      coef[1 * Q + k] = s * (c01 * c01 + c11 * c11 + c21 * c21);
      coef[2 * Q + k] = s * (c00 * c01 + c10 * c11 + c20 * c21);
      coef[3 * Q + k] = W * adet * rh;
      coef[4 * Q + k] = s * (c02 * c02 + c12 * c12 + c22 * c22);
      coef[5 * Q + k] = s * (c00 * c02 + c10 * c12 + c20 * c22);
      coef[6 * Q + k] = s * (c01 * c02 + c11 * c12 + c21 * c22);
    } else {
      coef[0 * Q + k] = W * kp;
      coef[1 * Q + k] = W * rh;
    }
  }
  __syncwarp();
  const float* PX = pat;
  const float* PY = pat + 4 * n2 * q;
  const float* PZ = pat + 8 * n2 * q;
  // stage 1 (z): T1[item][a3][b3][k1][k2] = sum_k3 Z(item)[a3][b3][k3] D(item)[k1,k2,k3]
  for (int i = lane; i < NI * n2 * q * q; i += 32) {
    const int k2 = i % q, k1 = (i / q) % q, ab = (i / (q * q)) % n2, it = i / (q * q * n2);
    const int zp = GEN ? wItemGen[it][0] : wItemId[it][0];
    const int ci = GEN ? wItemGen[it][1] : wItemId[it][1];
    const float* z = PZ + (zp * n2 + ab) * q;
    const float* D = coef + ci * Q + k1 + q * k2;
    float acc = 0.f;
#pragma unroll
    for (int k3 = 0; k3 < q; ++k3) acc = fmaf(z[k3], D[q * q * k3], acc);
    T1[i] = acc;
  }
  __syncwarp();
  // stage 2 (y): C[X][a'][b'][k1] = sum over the terms of X of
  //              sum_k2 Y(pattern)[a2][b2][k2] T1[item][a3][b3][k1][k2]
  for (int i = lane; i < 5 * n2 * n2 * q; i += 32) {
    const int k1 = i % q, bp = (i / q) % n2, ap = (i / (q * n2)) % n2, X = i / (q * n2 * n2);
    if ((X < 4 && !C::DK) || (X == 4 && !C::DM) || (!GEN && (X == 1 || X == 2))) continue;
    const int a2 = ap % n, a3 = ap / n, b2 = bp % n, b3 = bp / n;
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int yp = GEN ? wTermGen[X][m][0] : wTermId[X][m][0];
      if (yp < 0) break;
      const int it = GEN ? wTermGen[X][m][1] : wTermId[X][m][1];
      const float* y = PY + (yp * n2 + a2 * n + b2) * q;
      const float* t = T1 + ((it * n2 + a3 * n + b3) * q + k1) * q;
#pragma unroll
      for (int k2 = 0; k2 < q; ++k2) acc = fmaf(y[k2], t[k2], acc);
    }
    Cb[i] = acc;
  }
  __syncwarp();
  // stage 3 (x): the upper triangle of the element matrices, stored at (a, b)
  // and (b, a)
  float* Ke = C::DK ? (float*)B.K_out + pd.mat_offset + e * (int64_t)N * N : nullptr;
  float* Me = C::DM ? (float*)B.M_out + pd.mat_offset + e * (int64_t)N * N : nullptr;
  for (int it = lane; it < C::S; it += 32) {
    // row a of the upper triangle: it = a N - a (a - 1) / 2 + (b - a)
    int a = (int)((2.0f * N + 1.0f - sqrtf((2.0f * N + 1.0f) * (2.0f * N + 1.0f) - 8.0f * it)) * 0.5f);
    a = a < 0 ? 0 : (a > N - 1 ? N - 1 : a);
    while (a > 0 && a * N - a * (a - 1) / 2 > it) --a;
    while (a + 1 < N && (a + 1) * N - (a + 1) * a / 2 <= it) ++a;
    const int b = a + (it - (a * N - a * (a - 1) / 2));
    const int a1 = a % n, ap = a / n, b1 = b % n, bp = b / n;
    if (C::DK) {
      float acc = 0.f;
#pragma unroll
      for (int X = 0; X < 4; ++X) {
        if (!GEN && (X == 1 || X == 2)) continue;
        const float* x = PX + (wXPat[X] * n2 + a1 * n + b1) * q;
        const float* c = Cb + ((X * n2 + ap) * n2 + bp) * q;
#pragma unroll
        for (int k1 = 0; k1 < q; ++k1) acc = fmaf(x[k1], c[k1], acc);
      }
      Ke[(int64_t)a * N + b] = acc;
      Ke[(int64_t)b * N + a] = acc;
    }
    if (C::DM) {
      float acc = 0.f;
      const float* x = PX + (a1 * n + b1) * q;
      const float* c = Cb + ((4 * n2 + ap) * n2 + bp) * q;
#pragma unroll
      for (int k1 = 0; k1 < q; ++k1) acc = fmaf(x[k1], c[k1], acc);
      Me[(int64_t)a * N + b] = acc;
      Me[(int64_t)b * N + a] = acc;
    }
  }
  __syncwarp();
}

// Persistent warp-per-element kernel: every warp pops work items from the
// class's device queue until it is empty.  Checks, budget and error reporting
// as in the CTA form: a bad item sets IGA_ERR_DEVICE and is skipped; a spent
// time budget sets IGA_ERR_TIMEOUT and the warp stops; no warp waits on another.
template <int P, int QG, bool GEN, int MODE>
__global__ void __launch_bounds__(32 * kWarps) k_sf3_warp_queue(const QueueArgs B) {
  using C = W32<P, QG, GEN, MODE>;
  extern __shared__ __align__(16) float smw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* base = smw + warp * C::per_warp;
  const unsigned long long t0 = wq_timer_ns();
  for (;;) {
    int it = -1;
    if (lane == 0) {
      if (B.budget_ns != 0 && wq_timer_ns() - t0 + 1 >= B.budget_ns)
        atomicCAS(B.err, 0, (int)IGA_ERR_TIMEOUT);
      else
        it = atomicAdd(B.counter, 1);
    }
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it < 0 || it >= B.n_items) break;
    const WorkItem w = B.items[it];
    if (w.patch < 0 || w.patch >= B.n_patches) {
      if (lane == 0) atomicCAS(B.err, 0, (int)IGA_ERR_DEVICE);
      continue;
    }
    const PatchDev pd = B.patches[w.patch];
    const int64_t E = (int64_t)pd.K[0] * pd.K[1] * pd.K[2];
    if (w.e0 < 0 || w.count <= 0 || w.e0 + w.count > E || pd.p != P || pd.q != QG || !pd.iso) {
      if (lane == 0) atomicCAS(B.err, 0, (int)IGA_ERR_DEVICE);
      continue;
    }
    for (int64_t e = w.e0; e < w.e0 + w.count; ++e) w32_element<P, QG, GEN, MODE>(pd, B, e, base, lane);
  }
}

template <int P, int QG, bool GEN, int MODE>
cudaError_t run_warp(const QueueArgs& b, int grid, cudaStream_t st, int* max_grid) {
  using C = W32<P, QG, GEN, MODE>;
  static_assert(C::smem <= 227 * 1024, "shared memory");
  auto k = k_sf3_warp_queue<P, QG, GEN, MODE>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
  if (e != cudaSuccess) return e;
  if (max_grid) {
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * kWarps, C::smem);
    if (e != cudaSuccess) return e;
    // a CTA holds kWarps queue consumers
    *max_grid = sms * (per_sm > 0 ? per_sm : 1) * kWarps;
    return cudaSuccess;
  }
  const int ctas = (grid + kWarps - 1) / kWarps;
  k<<<(unsigned)(ctas > 0 ? ctas : 1), 32 * kWarps, C::smem, st>>>(b);
  return cudaGetLastError();
}

template <int P, int QG>
cudaError_t run_warp_m(const QueueArgs& b, int mode, int grid, cudaStream_t st, int* max_grid) {
  if (b.jac) {
    if (mode == 0) return run_warp<P, QG, true, 0>(b, grid, st, max_grid);
    if (mode == 1) return run_warp<P, QG, true, 1>(b, grid, st, max_grid);
    return run_warp<P, QG, true, 2>(b, grid, st, max_grid);
  }
  if (mode == 0) return run_warp<P, QG, false, 0>(b, grid, st, max_grid);
  if (mode == 1) return run_warp<P, QG, false, 1>(b, grid, st, max_grid);
  return run_warp<P, QG, false, 2>(b, grid, st, max_grid);
}

}  // namespace

bool warp_schedule_supported(int p, int q) { return p >= 1 && p <= 2 && (q == p + 1 || q == p + 2); }

cudaError_t launch_sumfact_warp_queue(const QueueArgs& b, int p, int q, int mode, int grid,
                                      cudaStream_t st, int* max_grid) {
  if (p == 1 && q == 2) return run_warp_m<1, 2>(b, mode, grid, st, max_grid);
  if (p == 1 && q == 3) return run_warp_m<1, 3>(b, mode, grid, st, max_grid);
  if (p == 2 && q == 3) return run_warp_m<2, 3>(b, mode, grid, st, max_grid);
  if (p == 2 && q == 4) return run_warp_m<2, 4>(b, mode, grid, st, max_grid);
  return cudaErrorInvalidValue;
}

}  // namespace iga
