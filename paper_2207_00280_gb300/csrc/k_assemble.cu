// k_assemble.cu -- global assembly of element matrices into CSR form and the
// per-dof gather of the matrix-free operator.
//
// The global matrix is the sum of the element matrices placed at the support
// index sets of the elements (Sec. 3.1, eq. 10 and the Remark on K^Delta_alpha;
// the insertion step of Table 3, Sec. 3.3).  Here it is formed as a gather,
// not a scatter: one warp owns one global row i, walks the elements that hold
// function i in ascending element order, reads row a(i, e) of each element
// matrix (N contiguous values: coalesced, and read by no other warp) and adds
// it into a shared-memory copy of the row.  No atomics; every entry is summed
// in ascending element order in the precision of the data, so the result is
// deterministic (and, in FP64, identical to a sequential sum in element
// order).  FP32 data is summed in FP32: on GB300 the FP64 pipe issues about
// two lanes per SM per clock, and converting and adding FP32 data in FP64
// made the FP32 assembly FP64-bound.
//
// The pattern is the tensor product of 1D coupling ranges: in each direction
// the functions that share an element with i_k form the range flo..fhi, so a
// row holds (j3, j2, j1) in flo..fhi of each direction, ascending.
#include "ff.cuh"
#include "iga_internal.h"

namespace iga {
namespace {

constexpr int kWarpsPerBlock = 4;

struct RowGeom {
  FnCouple f[3];
  int w[3];
  int64_t start;   // first entry of the row in the patch's CSR arrays
  int len;
};

__device__ __forceinline__ FnCouple fn_couple(const CsrPatch& c, const FnCouple* fc, int k, int i) {
  if (c.fn_offset[k] < 0) {
    FnCouple t;
    t.flo = t.fhi = t.elo = t.ehi = 0;
    t.S = 0;
    return t;
  }
  return fc[c.fn_offset[k] + i];
}

__device__ __forceinline__ RowGeom row_geom(const CsrPatch& c, const FnCouple* fc, int64_t row,
                                            int* ii) {
  RowGeom g;
  ii[0] = (int)(row % c.nf[0]);
  ii[1] = (int)((row / c.nf[0]) % c.nf[1]);
  ii[2] = (int)(row / ((int64_t)c.nf[0] * c.nf[1]));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    g.f[k] = fn_couple(c, fc, k, ii[k]);
    g.w[k] = g.f[k].fhi - g.f[k].flo + 1;
  }
  g.start = c.nnz_offset + g.f[2].S * c.W[1] * c.W[0] + (int64_t)g.w[2] * g.f[1].S * c.W[0] +
            (int64_t)g.w[2] * g.w[1] * g.f[0].S;
  g.len = g.w[0] * g.w[1] * g.w[2];
  return g;
}

__device__ __forceinline__ int first_fn(const CsrPatch& c, const int* spans, int k, int e) {
  return c.fn_offset[k] < 0 ? 0 : spans[c.span_offset[k] + e] - c.p;
}

// One warp per row: row pointer (lane 0) and the row's column indices.
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
    k_csr_pattern(const CsrPatch c, const FnCouple* __restrict__ fc, int64_t* __restrict__ row_ptr,
                  int32_t* __restrict__ col_idx) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_rows = (int64_t)c.nf[0] * c.nf[1] * c.nf[2];
  const int64_t row = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
  if (row >= n_rows) return;
  int ii[3];
  const RowGeom g = row_geom(c, fc, row, ii);
  if (lane == 0) {
    row_ptr[c.dof_offset + row] = g.start;
    if (row == n_rows - 1) row_ptr[c.dof_offset + n_rows] = g.start + g.len;
  }
  for (int z = lane; z < g.len; z += 32) {
    const int j1 = g.f[0].flo + z % g.w[0];
    const int j2 = g.f[1].flo + (z / g.w[0]) % g.w[1];
    const int j3 = g.f[2].flo + z / (g.w[0] * g.w[1]);
    col_idx[g.start + z] =
        (int32_t)(c.dof_offset + j1 + (int64_t)c.nf[0] * (j2 + (int64_t)c.nf[1] * j3));
  }
}

// One warp per row.  For each (e3, e2) the rows of up to n elements along x
// are loaded into registers first (all loads in flight together), then added
// in ascending e1; __syncwarp orders the additions of successive elements.
template <typename T, int P, int DIM>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
    k_assemble(const CsrPatch c, const FnCouple* __restrict__ fc, const int* __restrict__ spans,
               const T* __restrict__ A, T* __restrict__ values) {
  constexpr int n = P + 1, N = DIM == 3 ? n * n * n : n * n, NB = (N + 31) / 32;
  extern __shared__ __align__(8) unsigned char sraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* buf = (T*)sraw + (size_t)warp * c.lmax;
  const int64_t n_rows = (int64_t)c.nf[0] * c.nf[1] * c.nf[2];
  const int64_t row = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
  if (row >= n_rows) return;
  int ii[3];
  const RowGeom g = row_geom(c, fc, row, ii);
  for (int z = lane; z < g.len; z += 32) buf[z] = (T)0;
  // this lane's local columns b = lane + 32 nb and their per-direction parts
  int bl[NB][3];
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) {
    const int b = lane + 32 * nb;
    bl[nb][0] = b % n;
    bl[nb][1] = (b / n) % n;
    bl[nb][2] = b / (n * n);
  }
  __syncwarp();
  for (int e3 = g.f[2].elo; e3 <= g.f[2].ehi; ++e3) {
    const int s3 = first_fn(c, spans, 2, e3);
    for (int e2 = g.f[1].elo; e2 <= g.f[1].ehi; ++e2) {
      const int s2 = first_fn(c, spans, 1, e2);
      const int64_t ebase = (int64_t)c.K[0] * (e2 + (int64_t)c.K[1] * e3);
      const int arow23 = n * ((ii[1] - s2) + n * (ii[2] - s3));
      T v[n][NB];
      int s1v[n];
#pragma unroll
      for (int t = 0; t < n; ++t) {
        const int e1 = g.f[0].elo + t;
        s1v[t] = 0;
        if (e1 <= g.f[0].ehi) {
          const int s1 = first_fn(c, spans, 0, e1);
          s1v[t] = s1;
          const int a = (ii[0] - s1) + arow23;
          const T* Arow = A + c.mat_offset + ((ebase + e1) * N + a) * (int64_t)N;
#pragma unroll
          for (int nb = 0; nb < NB; ++nb) {
            const int b = lane + 32 * nb;
            v[t][nb] = (b < N) ? Arow[b] : (T)0;
          }
        }
      }
#pragma unroll
      for (int t = 0; t < n; ++t) {
        if (g.f[0].elo + t <= g.f[0].ehi) {
#pragma unroll
          for (int nb = 0; nb < NB; ++nb) {
            if (lane + 32 * nb < N) {
              const int z = ((s3 + bl[nb][2] - g.f[2].flo) * g.w[1] + (s2 + bl[nb][1] - g.f[1].flo)) *
                                g.w[0] +
                            (s1v[t] + bl[nb][0] - g.f[0].flo);
              buf[z] += v[t][nb];
            }
          }
        }
        __syncwarp();
      }
    }
  }
  for (int z = lane; z < g.len; z += 32) values[g.start + z] = buf[z];
}

// Phase 2 of the operator: one thread per dof, y[i] = sum over the elements
// holding i (ascending) of scratch[a(i, e) * E + e].  Adjacent threads read
// adjacent elements at the same local index: coalesced.
template <typename T, int P>
__global__ void __launch_bounds__(256)
    k_apply_gather(const CsrPatch c, const FnCouple* __restrict__ fc, const int* __restrict__ spans,
                   const T* __restrict__ scratch, T* __restrict__ y) {
  constexpr int n = P + 1;
  const int64_t n_rows = (int64_t)c.nf[0] * c.nf[1] * c.nf[2];
  const int64_t E = (int64_t)c.K[0] * c.K[1] * c.K[2];
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n_rows;
       row += (int64_t)gridDim.x * blockDim.x) {
    int ii[3];
    FnCouple f[3];
    ii[0] = (int)(row % c.nf[0]);
    ii[1] = (int)((row / c.nf[0]) % c.nf[1]);
    ii[2] = (int)(row / ((int64_t)c.nf[0] * c.nf[1]));
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = fn_couple(c, fc, k, ii[k]);
    T acc = (T)0;
    for (int e3 = f[2].elo; e3 <= f[2].ehi; ++e3) {
      const int a3 = ii[2] - first_fn(c, spans, 2, e3);
      for (int e2 = f[1].elo; e2 <= f[1].ehi; ++e2) {
        const int a2 = ii[1] - first_fn(c, spans, 1, e2);
        const int64_t eb = (int64_t)c.K[0] * (e2 + (int64_t)c.K[1] * e3);
        T v[n];
#pragma unroll
        for (int t = 0; t < n; ++t) {
          const int e1 = f[0].elo + t;
          v[t] = (T)0;
          if (e1 <= f[0].ehi) {
            const int a1 = ii[0] - first_fn(c, spans, 0, e1);
            v[t] = scratch[(int64_t)(a1 + n * (a2 + n * a3)) * E + eb + e1];
          }
        }
#pragma unroll
        for (int t = 0; t < n; ++t)
          if (f[0].elo + t <= f[0].ehi) acc += v[t];
      }
    }
    y[c.dof_offset + row] = acc;
  }
}

// Global mass matrix by weighted quadrature (3D, FP64): one CTA per row i.
// With V_k the per-direction tables of test function i_k (rule weights times
// trial values at the rule's points) and c the coefficient on the points of
// the support box, the row is contracted one direction at a time (the sum
// factorization of Sec. 3.2 applied to the rule of the row):
//   T1[j3][q1][q2] = sum_q3 V3[j3][q3] c[q1, q2, q3]
//   T2[j2][j3][q1] = sum_q2 V2[j2][q2] T1[j3][q1][q2]
//   M[j1][j2][j3]  = sum_q1 V1[j1][q1] T2[j2][j3][q1]
// and written to the row's CSR entries (j3, j2, j1 ascending).
template <typename T, int P>
__global__ void __launch_bounds__(128) k_wq_mass(const WqPatchArgs A) {
  constexpr int W = 2 * P + 1, NT = 128;
  extern __shared__ double wsm[];
  const CsrPatch& c = A.c;
  const int64_t n_rows = (int64_t)c.nf[0] * c.nf[1] * c.nf[2];
  for (int64_t row = blockIdx.x; row < n_rows; row += gridDim.x) {
    int ii[3];
    const RowGeom g = row_geom(c, A.fc, row, ii);
    int qlo[3], qn[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      qlo[k] = A.d[k].qlo[ii[k]];
      qn[k] = A.d[k].qn[ii[k]];
    }
    const int n1 = qn[0], n2 = qn[1], n3 = qn[2];
    const int w1 = g.w[0], w2 = g.w[1], w3 = g.w[2];
    T* V1 = reinterpret_cast<T*>(wsm);   // [w1][n1]
    T* V2 = V1 + W * n1;                 // [w2][n2]
    T* V3 = V2 + W * n2;                 // [w3][n3]
    T* T1 = V3 + W * n3;                 // [w3][n1][n2]
    T* T2 = T1 + (size_t)W * n1 * n2;    // [w2][w3][n1]
    __syncthreads();                     // the previous row's buffers are no longer read
    for (int k = 0; k < 3; ++k) {
      const int wk = g.w[k], nk = qn[k];
      const double* src = A.d[k].V + (size_t)ii[k] * W * A.d[k].qmax;
      T* dst = k == 0 ? V1 : (k == 1 ? V2 : V3);
      for (int t = threadIdx.x; t < wk * nk; t += NT)
        dst[t] = to_compute<T>(src[(t / nk) * A.d[k].qmax + t % nk]);
    }
    __syncthreads();
    // q3: one coefficient load per point, all w3 sums of the point in registers
    const int64_t np1 = A.d[0].np, np2 = A.d[1].np;
    for (int it = threadIdx.x; it < n1 * n2; it += NT) {
      const int q1 = it % n1, q2 = it / n1;
      T acc[W];
#pragma unroll
      for (int j = 0; j < W; ++j) acc[j] = 0;
      for (int q3 = 0; q3 < n3; ++q3) {
        const T cq = A.coef ? to_compute<T>(A.coef[(qlo[0] + q1) + np1 * ((qlo[1] + q2) + np2 * (qlo[2] + q3))])
                            : T(1);
#pragma unroll
        for (int j = 0; j < W; ++j)
          if (j < w3) mac(acc[j], V3[j * n3 + q3], cq);
      }
#pragma unroll
      for (int j = 0; j < W; ++j)
        if (j < w3) T1[((size_t)j * n1 + q1) * n2 + q2] = fin(acc[j]);
    }
    __syncthreads();
    // q2
    for (int it = threadIdx.x; it < n1 * w3; it += NT) {
      const int q1 = it % n1, j3 = it / n1;
      const T* t1 = T1 + ((size_t)j3 * n1 + q1) * n2;
      T acc[W];
#pragma unroll
      for (int j = 0; j < W; ++j) acc[j] = 0;
      for (int q2 = 0; q2 < n2; ++q2) {
        const T tv = t1[q2];
#pragma unroll
        for (int j = 0; j < W; ++j)
          if (j < w2) mac(acc[j], V2[j * n2 + q2], tv);
      }
#pragma unroll
      for (int j = 0; j < W; ++j)
        if (j < w2) T2[((size_t)j * w3 + j3) * n1 + q1] = fin(acc[j]);
    }
    __syncthreads();
    // q1, then the row's entries
    for (int it = threadIdx.x; it < w2 * w3; it += NT) {
      const int j2 = it % w2, j3 = it / w2;
      const T* t2 = T2 + ((size_t)j2 * w3 + j3) * n1;
      T acc[W];
#pragma unroll
      for (int j = 0; j < W; ++j) acc[j] = 0;
      for (int q1 = 0; q1 < n1; ++q1) {
        const T tv = t2[q1];
#pragma unroll
        for (int j = 0; j < W; ++j)
          if (j < w1) mac(acc[j], V1[j * n1 + q1], tv);
      }
      double* out = A.values + g.start + ((int64_t)j3 * w2 + j2) * w1;
#pragma unroll
      for (int j = 0; j < W; ++j)
        if (j < w1) out[j] = to_store<T>(fin(acc[j]));
    }
  }
}

// Global diffusion stiffness by weighted quadrature (3D, FP64): one CTA per
// row i.  Direction k has two tables of test function i_k, V0_k (mass rule x
// trial values) and V1_k (derivative rule x trial derivatives); the row is
//   K[j] = sum_q c(q) (V1_1 V0_2 V0_3 + V0_1 V1_2 V0_3 + V0_1 V0_2 V1_3)[j](q),
// contracted one direction at a time:
//   z: Z0[j3][q1][q2] = sum_q3 V0_3 c,  Z1 = sum_q3 V1_3 c
//   y: Ya[j2][j3][q1] = sum_q2 V0_2 Z0,  Yb = sum_q2 (V1_2 Z0 + V0_2 Z1)
//   x: K[j1][j2][j3]  = sum_q1 (V1_1 Ya + V0_1 Yb)
// and written to the row's CSR entries (j3, j2, j1 ascending).
template <typename T, int P>
__global__ void __launch_bounds__(128) k_wq_stiff(const WqPatchArgs A) {
  constexpr int W = 2 * P + 1, NT = 128;
  extern __shared__ double wsm[];
  const CsrPatch& c = A.c;
  const int64_t n_rows = (int64_t)c.nf[0] * c.nf[1] * c.nf[2];
  for (int64_t row = blockIdx.x; row < n_rows; row += gridDim.x) {
    int ii[3];
    const RowGeom g = row_geom(c, A.fc, row, ii);
    int qlo[3], qn[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      qlo[k] = A.d[k].qlo[ii[k]];
      qn[k] = A.d[k].qn[ii[k]];
    }
    const int n1 = qn[0], n2 = qn[1], n3 = qn[2];
    const int w1 = g.w[0], w2 = g.w[1], w3 = g.w[2];
    T* V[3][2];
    V[0][0] = reinterpret_cast<T*>(wsm);   // [w1][n1]
    V[0][1] = V[0][0] + W * n1;
    V[1][0] = V[0][1] + W * n1;          // [w2][n2]
    V[1][1] = V[1][0] + W * n2;
    V[2][0] = V[1][1] + W * n2;          // [w3][n3]
    V[2][1] = V[2][0] + W * n3;
    T* Z0 = V[2][1] + W * n3;                // [w3][n1][n2]
    T* Z1 = Z0 + (size_t)W * n1 * n2;
    T* Ya = Z1 + (size_t)W * n1 * n2;        // [w2][w3][n1]
    T* Yb = Ya + (size_t)W * W * n1;
    __syncthreads();                     // the previous row's buffers are no longer read
    for (int k = 0; k < 3; ++k) {
      const int wk = g.w[k], nk = qn[k];
      for (int v = 0; v < 2; ++v) {
        const double* src = (v ? A.d[k].V1 : A.d[k].V) + (size_t)ii[k] * W * A.d[k].qmax;
        T* dst = V[k][v];
        for (int t = threadIdx.x; t < wk * nk; t += NT)
          dst[t] = to_compute<T>(src[(t / nk) * A.d[k].qmax + t % nk]);
      }
    }
    __syncthreads();
    // z: one coefficient load per point, both tables' sums in registers
    const int64_t np1 = A.d[0].np, np2 = A.d[1].np;
    const T* V30 = V[2][0];
    const T* V31 = V[2][1];
    for (int it = threadIdx.x; it < n1 * n2; it += NT) {
      const int q1 = it % n1, q2 = it / n1;
      T a0[W], a1[W];
#pragma unroll
      for (int j = 0; j < W; ++j) a0[j] = a1[j] = 0;
      for (int q3 = 0; q3 < n3; ++q3) {
        const T cq = A.coef ? to_compute<T>(A.coef[(qlo[0] + q1) + np1 * ((qlo[1] + q2) + np2 * (qlo[2] + q3))])
                            : T(1);
#pragma unroll
        for (int j = 0; j < W; ++j)
          if (j < w3) {
            mac(a0[j], V30[j * n3 + q3], cq);
            mac(a1[j], V31[j * n3 + q3], cq);
          }
      }
#pragma unroll
      for (int j = 0; j < W; ++j)
        if (j < w3) {
          Z0[((size_t)j * n1 + q1) * n2 + q2] = fin(a0[j]);
          Z1[((size_t)j * n1 + q1) * n2 + q2] = fin(a1[j]);
        }
    }
    __syncthreads();
    // y
    const T* V20 = V[1][0];
    const T* V21 = V[1][1];
    for (int it = threadIdx.x; it < n1 * w3; it += NT) {
      const int q1 = it % n1, j3 = it / n1;
      const T* z0 = Z0 + ((size_t)j3 * n1 + q1) * n2;
      const T* z1 = Z1 + ((size_t)j3 * n1 + q1) * n2;
      T aa[W], ab[W];
#pragma unroll
      for (int j = 0; j < W; ++j) aa[j] = ab[j] = 0;
      for (int q2 = 0; q2 < n2; ++q2) {
        const T t0 = z0[q2], t1 = z1[q2];
#pragma unroll
        for (int j = 0; j < W; ++j)
          if (j < w2) {
            const T v0 = V20[j * n2 + q2];
            mac(aa[j], v0, t0);
            mac(ab[j], v0, t1);
            mac(ab[j], V21[j * n2 + q2], t0);
          }
      }
#pragma unroll
      for (int j = 0; j < W; ++j)
        if (j < w2) {
          Ya[((size_t)j * w3 + j3) * n1 + q1] = fin(aa[j]);
          Yb[((size_t)j * w3 + j3) * n1 + q1] = fin(ab[j]);
        }
    }
    __syncthreads();
    // x, then the row's entries
    const T* V10 = V[0][0];
    const T* V11 = V[0][1];
    for (int it = threadIdx.x; it < w2 * w3; it += NT) {
      const int j2 = it % w2, j3 = it / w2;
      const T* ya = Ya + ((size_t)j2 * w3 + j3) * n1;
      const T* yb = Yb + ((size_t)j2 * w3 + j3) * n1;
      T acc[W];
#pragma unroll
      for (int j = 0; j < W; ++j) acc[j] = 0;
      for (int q1 = 0; q1 < n1; ++q1) {
        const T ta = ya[q1], tb = yb[q1];
#pragma unroll
        for (int j = 0; j < W; ++j)
          if (j < w1) {
            mac(acc[j], V10[j * n1 + q1], tb);
            mac(acc[j], V11[j * n1 + q1], ta);
          }
      }
      double* out = A.values + g.start + ((int64_t)j3 * w2 + j2) * w1;
#pragma unroll
      for (int j = 0; j < W; ++j)
        if (j < w1) out[j] = to_store<T>(fin(acc[j]));
    }
  }
}

template <typename T, int P, int DIM>
cudaError_t run_assemble(const CsrPatch& c, const FnCouple* fc, const int* spans, const void* A,
                         void* values, cudaStream_t st) {
  const int64_t n_rows = (int64_t)c.nf[0] * c.nf[1] * c.nf[2];
  if (n_rows == 0) return cudaSuccess;
  const size_t smem = sizeof(T) * (size_t)c.lmax * kWarpsPerBlock;
  auto k = k_assemble<T, P, DIM>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = (n_rows + kWarpsPerBlock - 1) / kWarpsPerBlock;
  k<<<(unsigned)blocks, 32 * kWarpsPerBlock, smem, st>>>(c, fc, spans, (const T*)A, (T*)values);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_assemble(const CsrPatch& c, const FnCouple* fc, const int* spans,
                              const void* A, void* values, cudaStream_t st) {
  if (c.dim == 3) {
    switch (c.p) {
      case 1: return run_assemble<T, 1, 3>(c, fc, spans, A, values, st);
      case 2: return run_assemble<T, 2, 3>(c, fc, spans, A, values, st);
      case 3: return run_assemble<T, 3, 3>(c, fc, spans, A, values, st);
      case 4: return run_assemble<T, 4, 3>(c, fc, spans, A, values, st);
      case 5: return run_assemble<T, 5, 3>(c, fc, spans, A, values, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (c.p) {
    case 1: return run_assemble<T, 1, 2>(c, fc, spans, A, values, st);
    case 2: return run_assemble<T, 2, 2>(c, fc, spans, A, values, st);
    case 3: return run_assemble<T, 3, 2>(c, fc, spans, A, values, st);
    case 4: return run_assemble<T, 4, 2>(c, fc, spans, A, values, st);
    case 5: return run_assemble<T, 5, 2>(c, fc, spans, A, values, st);
    case 6: return run_assemble<T, 6, 2>(c, fc, spans, A, values, st);
    case 7: return run_assemble<T, 7, 2>(c, fc, spans, A, values, st);
    case 8: return run_assemble<T, 8, 2>(c, fc, spans, A, values, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int P>
cudaError_t run_gather(const CsrPatch& c, const FnCouple* fc, const int* spans,
                       const void* scratch, void* y, cudaStream_t st) {
  const int64_t n_rows = (int64_t)c.nf[0] * c.nf[1] * c.nf[2];
  if (n_rows == 0) return cudaSuccess;
  int64_t blocks = (n_rows + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_apply_gather<T, P><<<(unsigned)blocks, 256, 0, st>>>(c, fc, spans, (const T*)scratch, (T*)y);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_gather(const CsrPatch& c, const FnCouple* fc, const int* spans,
                            const void* scratch, void* y, cudaStream_t st) {
  // 2D: the missing direction has one function and one element (fn_couple)
  switch (c.p) {
    case 1: return run_gather<T, 1>(c, fc, spans, scratch, y, st);
    case 2: return run_gather<T, 2>(c, fc, spans, scratch, y, st);
    case 3: return run_gather<T, 3>(c, fc, spans, scratch, y, st);
    case 4: return run_gather<T, 4>(c, fc, spans, scratch, y, st);
    case 5: return run_gather<T, 5>(c, fc, spans, scratch, y, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int P>
cudaError_t run_wq(const WqPatchArgs& a, cudaStream_t st) {
  constexpr int W = 2 * P + 1;
  const int64_t n_rows = (int64_t)a.c.nf[0] * a.c.nf[1] * a.c.nf[2];
  if (n_rows == 0) return cudaSuccess;
  const size_t q1 = a.d[0].qmax, q2 = a.d[1].qmax, q3 = a.d[2].qmax;
  const size_t smem = sizeof(double) * (W * (q1 + q2 + q3) + W * q1 * q2 + (size_t)W * W * q1);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  auto k = k_wq_mass<T, P>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = n_rows < 152 * 64 ? n_rows : 152 * 64;
  k<<<(unsigned)blocks, 128, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int P>
cudaError_t run_wq_stiff(const WqPatchArgs& a, cudaStream_t st) {
  constexpr int W = 2 * P + 1;
  const int64_t n_rows = (int64_t)a.c.nf[0] * a.c.nf[1] * a.c.nf[2];
  if (n_rows == 0) return cudaSuccess;
  const size_t q1 = a.d[0].qmax, q2 = a.d[1].qmax, q3 = a.d[2].qmax;
  const size_t smem =
      sizeof(double) * (2 * W * (q1 + q2 + q3) + 2 * W * q1 * q2 + 2 * (size_t)W * W * q1);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  auto k = k_wq_stiff<T, P>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = n_rows < 152 * 64 ? n_rows : 152 * 64;
  k<<<(unsigned)blocks, 128, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool wq_stiffness_supported(int dim, int p) { return (dim == 2 || dim == 3) && p >= 2 && p <= 4; }

template <typename T>
cudaError_t wq_stiff_p(const WqPatchArgs& a, int p, cudaStream_t st) {
  switch (p) {
    case 2: return run_wq_stiff<T, 2>(a, st);
    case 3: return run_wq_stiff<T, 3>(a, st);
    case 4: return run_wq_stiff<T, 4>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t wq_mass_p(const WqPatchArgs& a, int p, cudaStream_t st) {
  switch (p) {
    case 1: return run_wq<T, 1>(a, st);
    case 2: return run_wq<T, 2>(a, st);
    case 3: return run_wq<T, 3>(a, st);
    case 4: return run_wq<T, 4>(a, st);
    case 5: return run_wq<T, 5>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_wq_stiffness(const WqPatchArgs& a, int p, bool df, cudaStream_t st) {
  return df ? wq_stiff_p<ff>(a, p, st) : wq_stiff_p<double>(a, p, st);
}

cudaError_t launch_wq_mass(const WqPatchArgs& a, int p, bool df, cudaStream_t st) {
  return df ? wq_mass_p<ff>(a, p, st) : wq_mass_p<double>(a, p, st);
}

cudaError_t launch_csr_pattern(const CsrPatch& c, const FnCouple* fc, int64_t* row_ptr,
                               int32_t* col_idx, cudaStream_t st) {
  const int64_t n_rows = (int64_t)c.nf[0] * c.nf[1] * c.nf[2];
  if (n_rows == 0) return cudaSuccess;
  const int64_t blocks = (n_rows + kWarpsPerBlock - 1) / kWarpsPerBlock;
  k_csr_pattern<<<(unsigned)blocks, 32 * kWarpsPerBlock, 0, st>>>(c, fc, row_ptr, col_idx);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const CsrPatch& c, const FnCouple* fc, const int* spans,
                            const void* A, void* values, bool fp64, cudaStream_t st) {
  return fp64 ? dispatch_assemble<double>(c, fc, spans, A, values, st)
              : dispatch_assemble<float>(c, fc, spans, A, values, st);
}

cudaError_t launch_apply_gather(const CsrPatch& c, const FnCouple* fc, const int* spans,
                                const void* scratch, void* y, bool fp64, cudaStream_t st) {
  return fp64 ? dispatch_gather<double>(c, fc, spans, scratch, y, st)
              : dispatch_gather<float>(c, fc, spans, scratch, y, st);
}

}  // namespace iga
