// k_tables.cu -- Cox--de Boor basis/derivative tables and the global dof map.
#include "iga_internal.h"

namespace iga {

// One 32-thread block per (patch, direction, element) record.  At each Gauss
// point the p+1 non-zero B-splines B_{s-p+r;p}(xi), r = 0..p, are built by the
// triangular form of the Cox--de Boor recursion (Sec. 2.3, eq. cox2: each
// degree combines two neighbours of the previous degree, the degree-0 start
// being the indicator of span s, eq. cox1).  Only the non-vanishing functions
// are carried, so no 0/0 term ever arises.  This left/right/saved evaluation
// of the non-zero triangle is the published one of Piegl and Tiller, The
// NURBS Book (2nd ed., 1997), Algorithm A2.2.  The derivative uses the degree
// p-1 row:
//   B'_{i;p} = p B_{i;p-1}/(t_{i+p}-t_i) - p B_{i+1;p-1}/(t_{i+p+1}-t_{i+1}).
// The record also stores the Gauss weight scaled by half the span length.
// Every division of the recursion (and of the derivative) is by a knot
// difference t_{s+k+1} - t_{s+1-d+k} (degree d, 0 <= k < d) that depends on
// the span only and is at least the span length: the block first forms these
// reciprocals, one per thread, then each thread evaluates one Gauss point with
// multiplications only.  GB300's FP64 pipe retires about two lanes per SM per
// clock, so the serial chain of a thread is what bounds this kernel.
__global__ void __launch_bounds__(32)
    k_basis_tables(const TableJob* __restrict__ jobs, const double* __restrict__ knots,
                   const double* __restrict__ gauss, double* __restrict__ tables) {
  __shared__ double rden[kMaxDegree2D * (kMaxDegree2D + 1) / 2];   // [d(d-1)/2 + k]
  const TableJob J = jobs[blockIdx.x];
  const double* t = knots + J.knot_off;
  const int p = J.p, q = J.q, n = p + 1, s = J.span;
  for (int i = threadIdx.x; i < p * (p + 1) / 2; i += 32) {
    int d = 1, k = i;
    while (k >= d) { k -= d; ++d; }
    rden[i] = 1.0 / (t[s + k + 1] - t[s + 1 - d + k]);
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j >= q) return;
  const double a = t[s], b = t[s + 1];
  const double mid = 0.5 * (a + b), half = 0.5 * (b - a);
  double* out = tables + J.out_off;
  const double xi = mid + half * gauss[J.gauss_off + j];
  double N[kMaxDegree2D + 1], Nm1[kMaxDegree2D + 1];
  double left[kMaxDegree2D + 1], right[kMaxDegree2D + 1];
  N[0] = 1.0;
  Nm1[0] = 1.0;
  for (int d = 1; d <= p; ++d) {
    if (d == p) {
      for (int k = 0; k < d; ++k) Nm1[k] = N[k];
    }
    left[d] = xi - t[s + 1 - d];
    right[d] = t[s + d] - xi;
    const double* rd = rden + d * (d - 1) / 2;
    double saved = 0.0;
    for (int k = 0; k < d; ++k) {
      const double tmp = N[k] * rd[k];
      N[k] = saved + right[k + 1] * tmp;
      saved = left[d - k] * tmp;
    }
    N[d] = saved;
  }
  // derivative denominators are the degree-p differences: t_{s+rr} - t_{s-p+rr}
  // is entry k = rr - 1 and t_{s+rr+1} - t_{s-p+rr+1} entry k = rr of degree p
  const double* rp = rden + p * (p - 1) / 2;
  for (int rr = 0; rr < n; ++rr) {
    double dv = 0.0;
    // B_{s-p+rr; p-1} is Nm1[rr-1] (rr >= 1), B_{s-p+rr+1; p-1} is Nm1[rr] (rr <= p-1)
    if (rr >= 1) dv += Nm1[rr - 1] * rp[rr - 1];
    if (rr <= p - 1) dv -= Nm1[rr] * rp[rr];
    out[j * n + rr] = N[rr];
    out[q * n + j * n + rr] = p * dv;
  }
  out[2 * q * n + j] = half * gauss[J.gauss_off + q + j];
}

cudaError_t launch_basis_tables(const TableJob* jobs, int n_jobs, const double* knots,
                                const double* gauss, double* tables, cudaStream_t st) {
  if (n_jobs <= 0) return cudaSuccess;
  k_basis_tables<<<(unsigned)n_jobs, 32, 0, st>>>(jobs, knots, gauss, tables);
  return cudaGetLastError();
}

// Global dof of every local function of every element (support set of the
// Remark in Sec. 3.1): dof = dof_offset + sum_k (s_k - p_k + a_k) stride_k.
// One block per element (grid-stride), one thread per local function:
// consecutive threads write consecutive entries.  The planner keeps every
// index below 2^31, so the arithmetic is 32-bit (64-bit division is slow).
__global__ void k_dofmap(const PatchDev* __restrict__ pdp, const int* __restrict__ spans,
                         int32_t* __restrict__ dof, int n_elem) {
  const PatchDev pd = *pdp;
  const int a = threadIdx.x;
  if (a >= pd.N) return;
  const int a1 = a % pd.nk[0];
  const int a2 = (a / pd.nk[0]) % pd.nk[1];
  const int a3 = a / (pd.nk[0] * pd.nk[1]);
  const int base = (int)pd.dof_offset;
  for (int e = blockIdx.x; e < n_elem; e += gridDim.x) {
    const int e1 = e % pd.K[0];
    const int r = e / pd.K[0];
    const int e2 = r % pd.K[1];
    const int e3 = r / pd.K[1];
    int g = spans[pd.span_offset[0] + e1] - pd.pk[0] + a1;
    g += (spans[pd.span_offset[1] + e2] - pd.pk[1] + a2) * pd.nf[0];
    if (pd.dim == 3) g += (spans[pd.span_offset[2] + e3] - pd.pk[2] + a3) * pd.nf[0] * pd.nf[1];
    dof[(int64_t)e * pd.N + a] = base + g;
  }
}

cudaError_t launch_dofmap(const PatchDev* pdp, const PatchDev& ph, const int* spans,
                          int32_t* dof_out, cudaStream_t st) {
  const int64_t E = (int64_t)ph.K[0] * ph.K[1] * ph.K[2];
  if (E == 0) return cudaSuccess;
  const int bs = (ph.N + 31) / 32 * 32;
  const int64_t blocks = E < 152 * 64 ? E : 152 * 64;
  k_dofmap<<<(unsigned)blocks, bs, 0, st>>>(pdp, spans, dof_out, (int)E);
  return cudaGetLastError();
}

}  // namespace iga
