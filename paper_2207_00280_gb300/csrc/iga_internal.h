// iga_internal.h -- plan layout and kernel launchers shared by the CUDA
// translation units of the library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "iga.h"

namespace iga {

// Degrees and Gauss orders accepted by iga_plan (per direction).  Degrees
// above the specialised kernels' range, a different degree or Gauss order per
// direction, and Gauss orders other than p+1 / p+2 run on the runtime-sized
// FP64 kernels of k_generic64.cu.
constexpr int kMaxDegree = 8;
constexpr int kMaxDegree2D = kMaxDegree;   // size of the per-point Cox--de Boor arrays
constexpr int kMaxGauss = 16;

// Per-patch description, uploaded to the device.  Offsets index the plan's
// concatenated arrays.  p, q, n are direction 0's values; pk, qk, nk hold
// every direction's (1 beyond dim for nk and qk), iso = 1 when all directions
// of the patch share p and q.
struct PatchDev {
  int dim, p, q, n, N, Q;
  int pk[3], qk[3], nk[3];
  int iso;
  int K[3];              // elements per direction
  int nf[3];             // functions per direction (global 1D dofs)
  int64_t elem_offset;   // first global element
  int64_t qp_offset;     // first global quadrature point
  int64_t dof_offset;    // first global dof
  int64_t mat_offset;    // first entry of K_out / M_out
  int64_t dofmap_offset; // first entry of dof_out
  int64_t tab_offset[3]; // first double of direction k's basis records
  int span_offset[3];    // first entry of direction k's spans
  int knot_offset[3];    // first knot of direction k
  int gauss_offset[3];   // first reference node / weight of direction k's rule
};

// Basis record of one element of one direction: val[q][n], der[q][n], w[q]
// (w = reference weight times half the span length).
__host__ __device__ constexpr int record_size(int n, int q) { return 2 * q * n + q; }

// One table job = one (patch, direction, element) record.
struct TableJob {
  int knot_off;   // first knot of the direction
  int span;       // knot span index s of the element
  int p, q;
  int gauss_off;  // reference nodes at gauss[gauss_off], weights at gauss[gauss_off + q]
  int64_t out_off;
};

// Device error word values are iga_status codes; 0 = OK.

// ---- launchers (each returns a cudaError_t of the launch) ----------------
cudaError_t launch_basis_tables(const TableJob* jobs, int n_jobs, const double* knots,
                                const double* gauss, double* tables, cudaStream_t st);

cudaError_t launch_dofmap(const PatchDev* patches_dev, const PatchDev& ph, const int* spans,
                          int32_t* dof_out, cudaStream_t st);

struct ElemArgs {
  const PatchDev* pd;     // device copy of the patch
  int64_t n_elem;         // elements of this patch
  int K1, K2, K3;
  const double* tab[3];   // first record of each direction
  const double* kappa;    // patch-local (already offset), [E][Q] or null
  const double* rho;
  const double* jac;
  void* K_out;            // patch-local, or null
  void* M_out;
  int* err;
};

#ifdef __CUDACC__
// Coordinates (e1, e2, e3) of element e = e1 + K1 (e2 + K2 e3).  Element
// indices below 2^31 (every patch in practice) take two 32-bit unsigned
// divisions; a 64-bit division by a runtime divisor is a long instruction
// sequence that each thread would otherwise run once per element.
template <class Args>   // any launch-argument record with K1, K2
__device__ __forceinline__ void elem_coords(const Args& A, int64_t e, int& e1, int& e2, int& e3) {
  if (e < 0x7fffffffLL) {
    const unsigned u = (unsigned)e, k1 = (unsigned)A.K1, k2 = (unsigned)A.K2;
    const unsigned r1 = u / k1, r2 = r1 / k2;
    e1 = (int)(u - r1 * k1);
    e2 = (int)(r1 - r2 * k2);
    e3 = (int)r2;
  } else {
    e1 = (int)(e % A.K1);
    e2 = (int)((e / A.K1) % A.K2);
    e3 = (int)(e / ((int64_t)A.K1 * A.K2));
  }
}
// 2D: element e = e1 + K1 e2.
template <class Args>
__device__ __forceinline__ void elem_coords2(const Args& A, int64_t e, int& e1, int& e2) {
  if (e < 0x7fffffffLL) {
    const unsigned u = (unsigned)e, k1 = (unsigned)A.K1, r1 = u / k1;
    e1 = (int)(u - r1 * k1);
    e2 = (int)r1;
  } else {
    e1 = (int)(e % A.K1);
    e2 = (int)(e / A.K1);
  }
}
#endif

// FP64 sum factorization (Algorithm 2 generalised to the stiffness terms).
cudaError_t launch_sumfact_f64(const ElemArgs& a, int dim, int p, int q, cudaStream_t st);
// FP64 classical integration (Algorithm 1).
cudaError_t launch_classical_f64(const ElemArgs& a, int dim, int p, int q, cudaStream_t st);

// Runtime-sized FP64 forms for any patch (degree 1..8 and Gauss order 1..16
// per direction, 2D and 3D): sum factorization tiled over the (a3, b3) blocks
// of the element matrix, classical integration tiled over quadrature points,
// and the matrix-free adjoint.  ph is the host copy of the patch.
cudaError_t launch_sumfact_gen(const ElemArgs& a, const PatchDev& ph, cudaStream_t st);
cudaError_t launch_classical_gen(const ElemArgs& a, const PatchDev& ph, cudaStream_t st);

// Persistent batched form: one work item = `count` consecutive elements of one
// patch; CTAs pop items from a device counter.
struct WorkItem {
  int patch;
  int count;
  int64_t e0;
};
struct QueueArgs {
  const PatchDev* patches;
  int n_patches;
  const double* tables;
  const double* kappa;   // global [n_qp] or null
  const double* rho;
  const double* jac;     // global [n_qp][9] or null
  void* K_out;           // global, float
  void* M_out;
  const WorkItem* items;
  int n_items;
  int* counter;          // zeroed before the launch
  int* err;
  unsigned long long budget_ns;  // 0 = no time budget
};
cudaError_t launch_sumfact_f32_queue(const QueueArgs& b, int p, int q, bool bf16, int mode,
                                     int grid, cudaStream_t st, int* max_grid);
bool queue_both_fit(int p, int q, bool bf16);

// Schedules of one (p, q) class of the persistent batched launch, chosen by
// the autotuner: the default CTA-per-element kernel, its variants (stage 3 on
// mma.sync where the default is tcgen05; the other CTA size), and the
// warp-per-element kernel (p <= 2).  The variant values are the MODE flags of
// k_sumfact32.cuh.
enum { kSchedCta = 0, kSchedCtaAltForm = 4, kSchedCtaAltSize = 8, kSchedWarp = 16 };
bool f32_variant_supported(int p, int q, bool bf16, int variant);
cudaError_t launch_sumfact_f32_queue_alt(const QueueArgs& b, int p, int q, bool bf16, int mode,
                                         int variant, int grid, cudaStream_t st, int* max_grid);
bool warp_schedule_supported(int p, int q);
// The streamed tcgen05 form of p = 4, 5 (k_stream32.cu): the default FP32/BF16
// form there, per patch and in the persistent queue.
bool stream_form_supported(int p, int q);
bool stream_both_fit(int p, int q, bool bf16);
cudaError_t launch_sumfact_f32_stream(const ElemArgs& a, int p, int q, bool bf16, cudaStream_t st);
cudaError_t launch_sumfact_f32_stream_queue(const QueueArgs& b, int p, int q, bool bf16, int mode,
                                            int grid, cudaStream_t st, int* max_grid);
// Stiffness of 3D patches with a general map at p = 4, q = 5 in FP32 / BF16
// (k_curved32.cu): the default form of that class, per patch and in the
// persistent queue (stiffness-only launches).
bool curved_form_supported(int p, int q);
cudaError_t launch_sumfact_f32_curved(const ElemArgs& a, bool bf16, cudaStream_t st);
cudaError_t launch_sumfact_f32_curved_queue(const QueueArgs& b, bool bf16, int grid, cudaStream_t st,
                                            int* max_grid);
// max_grid reports the number of queue consumers (warps) that fit; grid is a
// number of warps.
cudaError_t launch_sumfact_warp_queue(const QueueArgs& b, int p, int q, int mode, int grid,
                                      cudaStream_t st, int* max_grid);

// FP32 sum factorization (3D): FP64 cofactors/determinant, FP32 contractions;
// with bf16 = true the last contraction runs on the tensor cores in BF16.
cudaError_t launch_sumfact_f32(const ElemArgs& a, int dim, int p, int q, bool bf16,
                               cudaStream_t st);

// Matrix-free adjoint (3D; 2D for FP64 plans): grad[e*Q + k] = dJ/dkappa, partial[partial_offset + e]
// = per-element sum of kappa * grad.  All array pointers are patch-local except
// u, v (global dof vectors) and partial.
struct AdjArgs {
  int64_t n_elem;
  int K1, K2, K3;
  const double* tab[3];
  const int* span[3];
  int nf0, nf1;
  int64_t dof_offset;
  const double* kappa;   // patch-local [E][Q] or null (= 1)
  const double* jac;     // patch-local [E][Q][d*d] or null
  const void* u;         // global [n_dofs], double or float
  const void* v;
  void* grad;            // patch-local [E][Q] or null
  double* partial;       // [n_elements] or null
  int64_t partial_offset;
};
cudaError_t launch_adjoint(const AdjArgs& a, int dim, int p, int q, bool fp64, bool df,
                           cudaStream_t st);
// FP64 adjoint for any patch (u, v double); ph gives the per-direction sizes.
cudaError_t launch_adjoint_gen(const AdjArgs& a, const PatchDev& ph, cudaStream_t st);
cudaError_t launch_reduce_fixed(const double* partial, int64_t n, double* out, cudaStream_t st);
bool adjoint_supported(int dim, int p, int q);

// FP64-accurate sum factorization in float-float arithmetic (3D).
cudaError_t launch_sumfact_df(const ElemArgs& a, int dim, int p, int q, cudaStream_t st);
bool sumfact_df_supported(int dim, int p, int q);

bool sumfact_f64_supported(int dim, int p, int q);
bool sumfact_f32_supported(int dim, int p, int q);
bool classical_f64_supported(int dim, int p, int q);

// ---- assembled (CSR) form and operator application -------------------------
// Coupling data of one global 1D function of one direction: the elements that
// hold it (elo..ehi, indices into the direction's element list), the functions
// it shares an element with (flo..fhi, a contiguous range) and the prefix sum S
// of the widths fhi - flo + 1 over the functions before it.
struct FnCouple {
  int flo, fhi, elo, ehi;
  int64_t S;
};

// One patch of the assembled form.  Rows (and columns) are global dofs
// i = i1 + nf0 (i2 + nf1 i3); the pattern is the tensor product of the 1D
// coupling ranges, so the row start of i is
//   nnz_offset + S3(i3) W1 W0 + w3(i3) S2(i2) W0 + w3(i3) w2(i2) S1(i1).
struct CsrPatch {
  int dim, p, n, N;
  int K[3], nf[3];
  int64_t dof_offset, mat_offset, nnz_offset, elem_offset;
  int64_t W[3];          // sum of the widths per direction (1 for a missing direction)
  int fn_offset[3];      // first FnCouple of direction k (-1: missing direction)
  int span_offset[3];
  int lmax;              // longest row
};

// CSR row pointers (int64, n_dofs + 1) and column indices (int32) of one patch.
cudaError_t launch_csr_pattern(const CsrPatch& c, const FnCouple* fc, int64_t* row_ptr,
                               int32_t* col_idx, cudaStream_t st);
// values[nnz of the patch] = sum over elements (ascending) of the element
// matrices A (patch block of a [E][N][N] array), in the data's precision.
cudaError_t launch_assemble(const CsrPatch& c, const FnCouple* fc, const int* spans,
                            const void* A, void* values, bool fp64, cudaStream_t st);

// y = alpha K(kappa) x + beta M(rho) x, matrix-free (3D; 2D for FP64 plans).  Phase 1 writes each
// element's local result to scratch[a * E + e]; phase 2 sums them per dof in
// ascending element order.
struct ApplyArgs {
  int64_t n_elem;
  int K1, K2, K3;
  const double* tab[3];
  const int* span[3];
  int nf0, nf1;
  int64_t dof_offset;
  const double* kappa;   // patch-local [E][Q] or null (= 1)
  const double* rho;     // patch-local [E][Q] or null (= 1)
  const double* jac;     // patch-local [E][Q][d*d] or null
  const void* x;         // global [n_dofs], double or float
  double alpha, beta;
  void* scratch;         // patch-local [N][E], double or float
};
cudaError_t launch_apply(const ApplyArgs& a, int dim, int p, int q, bool fp64, bool df,
                         cudaStream_t st);
cudaError_t launch_apply_gather(const CsrPatch& c, const FnCouple* fc, const int* spans,
                                const void* scratch, void* y, bool fp64, cudaStream_t st);
bool apply_supported(int dim, int p, int q);

// Backward of the element matrices with respect to the coefficients (2D, 3D):
// grad_kappa[e*Q + k] = sum_ab GK[e][a][b] dK_ab/dkappa_k and grad_rho[e*Q + k]
// = sum_ab GM[e][a][b] dM_ab/drho_k.  All pointers are patch-local; GK, GM
// and the gradients are double (fp64) or float.
struct GradArgs {
  int64_t n_elem;
  int K1, K2, K3;
  const double* tab[3];
  const double* jac;     // [E][Q][d*d] or null (= identity)
  const void* GK;        // [E][N][N] or null (skip grad_kappa)
  const void* GM;        // [E][N][N] or null (skip grad_rho)
  void* grad_kappa;      // [E][Q]
  void* grad_rho;        // [E][Q]
  bool two_buffers;      // set by the launcher
};
// fp64: double arrays; df (with fp64): float-float arithmetic where supported
cudaError_t launch_grad(const GradArgs& a, int dim, int p, int q, bool fp64, bool df,
                        cudaStream_t st);
bool grad_supported(int dim, int p, int q, bool fp64);

// ---- weighted quadrature (mass matrix, 3D, FP64) -------------------------------
// One direction of one patch: the rule of test function i covers the points
// qlo[i] .. qlo[i] + qn[i] - 1 of the direction's global point list, and
// V[(i * W + jj) * QMAX + qq] = w_{i, qlo + qq} B_{flo(i) + jj}(x_{qlo + qq})
// (W = 2p + 1 columns, zero-padded).
struct WqDirDev {
  const int* qlo;
  const int* qn;
  const double* V;
  const double* V1;   // derivative rule x trial derivatives, same layout (p >= 2), or null
  int np;      // points of the direction
  int qmax;    // padding of the point index in V
};
struct WqPatchArgs {
  CsrPatch c;            // rows, coupling ranges, CSR offsets
  const FnCouple* fc;
  WqDirDev d[3];
  const double* coef;    // patch block of the coefficient grid [np3][np2][np1], or null = 1
  double* values;        // global CSR values
};
// df: float-float arithmetic (FP64_DF plans), else FP64
cudaError_t launch_wq_mass(const WqPatchArgs& a, int p, bool df, cudaStream_t st);
// Diffusion stiffness by weighted quadrature (3D, FP64, 2 <= p <= 4): values of
// the rows of one patch, sum over the three derivative directions.
cudaError_t launch_wq_stiffness(const WqPatchArgs& a, int p, bool df, cudaStream_t st);
bool wq_stiffness_supported(int dim, int p);

}  // namespace iga
