/*
 * iga.h -- C ABI of the GB300 (sm_103a) library for batched integration of
 * IGA-FEM element matrices over tensor-product B-spline bases
 * (arxiv 2207.00280, "A study of efficient concurrent integration methods of
 * B-Spline basis functions in IGA-FEM").
 *
 * What is computed (per element E of a patch, N local functions):
 *   mass       M_ab = sum_q w_q |det G_q| rho_q   phi_a(x_q) phi_b(x_q)
 *   stiffness  K_ab = sum_q w_q |det G_q| kappa_q (G_q^{-T} grad phi_a).(G_q^{-T} grad phi_b)
 * The mass is the element Gram matrix of Sec. 3.1 (eqs. 88 and 10); the
 * stiffness is the diffusion term of the weak form of Sec. 2.2 (eq. Euler)
 * with a coefficient per quadrature point (not integrated in the paper).
 * phi_a are tensor products of 1D B-splines (Sec. 2.3, eqs. cox1, cox2,
 * basis_construction) on open knot vectors (eq. knot_vector).  The quadrature
 * is Gauss--Legendre with q points per direction ("a proper exact
 * quadrature", Sec. 3.1).  Two methods give the same sums up to rounding:
 * the classical loop (Sec. 3.2, Algorithm 1) and sum factorization
 * (Sec. 3.2, Algorithm 2, eqs. finalsum and bufferC).
 *
 * Each direction k of a patch has its own degree p_k and number of Gauss
 * points q_k: the paper uses one degree for every direction and notes that the
 * method extends to bases of different degrees (Sec. 2.3), and its element sum
 * (eq. 10) has P_1 P_2 P_3 points.  N = n_1 n_2 (n_3) with n_k = p_k + 1 and
 * Q = q_1 q_2 (q_3).
 *
 * Conventions (all indices 0-based, x fastest in every multi-index):
 *   element   e = e1 + K1*(e2 + K2*e3), elements = non-empty knot spans;
 *   local fn  a = a1 + n_1*(a2 + n_2*a3) (the support set of the Remark in
 *             Sec. 3.1, global 1D index s_k - p_k + a_k for span s_k);
 *   global dof = i1 + f1*(i2 + f2*i3), f_k = functions in direction k,
 *             patches concatenated in batch order;
 *   quad pt   k = k1 + q_1*(k2 + q_2*k3);
 *   kappa, rho: [n_qp] doubles, element-major: index = qp_offset(patch) +
 *             e*Q + k;
 *   jac:      [n_qp][d][d] doubles, jac[..][i][j] = d x_i / d xi_j with xi
 *             the knot (parametric) coordinate; |det| is the J(x^n) of eq. 10;
 *   K_out, M_out: per patch [E][N][N] row-major, patches concatenated
 *             (offsets in iga_plan_info.mat_offset), double for IGA_FP64 and
 *             IGA_FP64_DF, float for IGA_FP32 and IGA_BF16;
 *   dof_out:  per patch [E][N] int32, concatenated (iga_plan_info.dofmap_offset).
 *
 * Ownership: every array pointer passed to an entry point below (except the
 * host knot vectors of iga_patch_desc and the host x_out of iga_wq_points) is
 * owned by the caller and must be device memory of the device that was
 * current at iga_plan (no copies are made; some kernels write their outputs
 * with bulk asynchronous copies, which need device memory).  The plan owns its device tables
 * and the arrays that iga_plan_info points to; iga_destroy frees them.
 *
 * Errors: argument and knot errors are returned synchronously and nothing is
 * launched.  Device-side errors set a plan-owned error word; with
 * opts.blocking = 1 the call synchronizes the stream and returns it, otherwise
 * it is sticky and reported by the next call or by iga_destroy.  No device
 * code traps or asserts; device waits are bounded and end in IGA_ERR_TIMEOUT.
 */
#ifndef IGA_H
#define IGA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct iga_plan_s* iga_plan_t;

typedef enum {
  IGA_OK = 0,
  IGA_ERR_ARG = 1,          /* null/negative/out-of-range argument */
  IGA_ERR_KNOTS = 2,        /* knot vector not open, decreasing, or multiplicity > p */
  IGA_ERR_UNSUPPORTED = 3,  /* valid but not built (degree, Gauss order, mixed dims) */
  IGA_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  IGA_ERR_OOM = 5,          /* device allocation failed */
  IGA_ERR_TIMEOUT = 6,      /* a bounded device wait expired */
  IGA_ERR_DEVICE = 7,       /* the device reported an inconsistency (bad work item) */
  IGA_ERR_TOO_LARGE = 8     /* beyond the fixed scratch of iga_adjoint_noalloc */
} iga_status;

enum { IGA_CLASSICAL = 0, IGA_SUMFACT = 1 };
/* Precisions.  IGA_FP64: FP64 arithmetic.  IGA_FP32: FP64 Jacobian cofactors
 * and determinant, FP32 contractions (stage 3 as 3xTF32 on the tensor cores).
 * IGA_BF16: as FP32 with the last contraction in BF16 on the tensor cores (FP32
 * accumulation).  IGA_FP64_DF: FP64-accurate results (double outputs, tested
 * to <= 1e-12 per element like IGA_FP64) computed in float-float arithmetic
 * (pairs of FP32 numbers) on the FP32 pipes; sum factorization in 3D only. */
enum { IGA_FP64 = 0, IGA_FP32 = 1, IGA_BF16 = 2, IGA_FP64_DF = 3 };
enum { IGA_MASS = 1, IGA_STIFF = 2 };

/* Schedules (iga_plan_opts.schedule).  AUTO picks PERSISTENT_GRAPH for FP32 or
 * BF16 sum factorization of a batch of several patches, PER_PATCH otherwise,
 * and lets the autotuner choose the work-item size of every degree class.
 *   PER_PATCH:        one grid launch (one CTA per element) per patch;
 *   PERSISTENT:       one persistent kernel per (degree, Gauss order) class,
 *                     CTAs pop work items (consecutive elements of one patch)
 *                     from a device queue;
 *   PERSISTENT_GRAPH: the same kernels plus the table and dof-map kernels
 *                     captured once into a CUDA graph (classes on parallel
 *                     branches) and replayed while the pointers are unchanged.
 * The persistent schedules exist for FP32/BF16 sum factorization only.
 * Within them the autotuner chooses, per (degree, Gauss order) class, among
 * the CTA-per-element kernel (one thread per element-matrix entry; at p = 4, 5
 * the streamed tcgen05 form), its variants where the class has them (p = 3:
 * stage 3 on warp-level mma.sync instead of tcgen05; p = 4, 5: the staged form
 * with symmetric operand rows, and that form with 512 instead of 256 threads
 * at FP32 p = 4 and 256 instead of 512 at p = 5, identity geometry), and a
 * warp-per-element kernel (p <= 2, all contractions in FP32), each with work
 * items of 1, 2, 4 or 8 elements, by timing every candidate (median of three
 * launches).  The environment variable IGA_BATCH_SCHED, read by iga_plan,
 * forces one schedule (0 CTA, 4 mma.sync form, 8 other CTA size, 16 warp) for
 * the classes that have it and disables the tuning; IGA_AUTOTUNE_CACHE names a
 * JSON file that keeps the choices ({key: schedule * 100 + work-item size}). */
enum { IGA_SCHED_AUTO = 0, IGA_SCHED_PER_PATCH = 1, IGA_SCHED_PERSISTENT = 2,
       IGA_SCHED_PERSISTENT_GRAPH = 3 };

/* One tensor-product patch.  Knot vectors are host arrays, copied by
 * iga_plan.  Knot vector k must be non-decreasing and open (first and last
 * p_k+1 knots equal) with interior multiplicity <= p_k (Sec. 2.3,
 * eq. knot_vector).  1 <= degree[k] <= 8 and 1 <= n_gauss[k] <= 16 for each of
 * the dim directions (IGA_ERR_ARG otherwise); entries beyond dim are ignored.
 *
 * Which forms take which patches:
 *   IGA_FP64 (classical and sum factorization), iga_integrate_backward on
 *     IGA_FP64 plans, iga_basis_tables, iga_csr_pattern: every patch.  Patches
 *     with one degree p <= 5 and one Gauss order q in {p+1, p+2} (2D: p <= 8)
 *     run on kernels specialised for that (p, q); the others on runtime-sized
 *     FP64 kernels.
 *   IGA_FP32, IGA_BF16, IGA_FP64_DF (sum factorization only), and the other
 *     entry points (iga_apply, iga_assemble, iga_integrate_grad, the weighted
 *     quadrature): patches with one degree and one Gauss order in every
 *     direction, within the limits each entry states; otherwise
 *     IGA_ERR_UNSUPPORTED. */
typedef struct {
  int dim;                  /* 2 or 3 */
  int degree[3];            /* p_k per direction */
  int n_gauss[3];           /* q_k, Gauss points per direction */
  int n_knots[3];           /* knots per direction (dim entries used) */
  const double* knots[3];   /* host pointers */
} iga_patch_desc;

typedef struct {
  int method;     /* IGA_CLASSICAL or IGA_SUMFACT */
  int precision;  /* IGA_FP64, IGA_FP32, IGA_BF16 or IGA_FP64_DF (the last three
                     for sum factorization only) */
  int matrices;   /* bitmask of IGA_MASS | IGA_STIFF */
  int schedule;   /* IGA_SCHED_*; 0 = automatic (autotuned) */
  int blocking;   /* 1 = synchronize the stream and return the device status */
  int profile;    /* 1 = record CUDA events around the element-matrix kernels */
} iga_plan_opts;

typedef struct {
  int64_t n_elements;       /* all patches */
  int64_t n_qp;             /* length of kappa / rho, and of jac in d*d units */
  int64_t n_dofs;           /* length of u, v */
  int64_t n_mat_entries;    /* length of K_out / M_out */
  int64_t n_dofmap_entries; /* length of dof_out */
  int64_t n_table_entries;  /* length of the output of iga_basis_tables */
  int dim;
  int n_patches;
  int local_n;              /* N of the first patch (all patches if uniform) */
  /* per-patch arrays of n_patches+1 prefix offsets, owned by the plan */
  const int64_t* elem_offset;
  const int64_t* qp_offset;
  const int64_t* dof_offset;
  const int64_t* mat_offset;
  const int64_t* dofmap_offset;
  int64_t n_csr_nnz;        /* entries of the assembled (CSR) global matrix */
} iga_plan_info;

/* Validate the patches, build the element spans, Gauss rules and dof strides
 * on the host, allocate the plan's device tables on the current device.
 * A batch (n_patches > 1) may mix degrees and sizes but not dimensions.
 * info_out may be NULL.  Returns IGA_OK and *out, or an error and *out = NULL. */
int iga_plan(iga_plan_t* out, const iga_patch_desc* patches, int n_patches,
             const iga_plan_opts* opts, iga_plan_info* info_out);

/* Integrate every element of every patch on `cuda_stream` (a cudaStream_t,
 * NULL = legacy default stream): the Cox--de Boor basis/derivative tables,
 * the dof map, then mass and/or stiffness by the plan's method.
 *   kappa  [n_qp] or NULL (= 1); required values > 0 are not checked.
 *   rho    [n_qp] or NULL (= 1); used by the mass only.
 *   jac    [n_qp][d][d] or NULL (= identity).
 *   K_out, M_out: NULL skips that matrix; must be non-NULL if the plan's
 *          `matrices` includes it and the other is NULL.
 *   dof_out: [n_dofmap_entries] or NULL (skip). */
int iga_integrate(iga_plan_t plan, const double* kappa, const double* rho,
                  const double* jac, void* K_out, void* M_out, int32_t* dof_out,
                  void* cuda_stream);

/* Matrix-free adjoint of J(kappa) = u^T K(kappa) v (not in the paper; 3D,
 * or 2D on IGA_FP64 plans):
 *   grad_kappa[k] = dJ/dkappa_k = w_k |det G_k| (G_k^{-T} grad u).(G_k^{-T} grad v)
 * at every quadrature point, computed by sum-factorized interpolation of u and
 * v from the basis tables (no element matrix is formed), and
 *   J_out = sum_k kappa_k grad_kappa[k]   (deterministic fixed-order reduction).
 * u, v: [n_dofs] global vectors; double for IGA_FP64 and IGA_FP64_DF plans,
 * float otherwise.  IGA_FP64 computes in FP64, IGA_FP64_DF in float-float
 * on the FP32 pipes (FP64-accurate), the others in FP32 with FP64 Jacobian
 * cofactors and determinant.
 * grad_kappa: [n_qp], same dtype as u.  J_out: one double, may be NULL.
 * kappa may be NULL only if J_out is NULL.  jac as for iga_integrate. */
int iga_integrate_backward(iga_plan_t plan, const double* kappa, const double* jac,
                           const void* u, const void* v, void* grad_kappa,
                           double* J_out, void* cuda_stream);

/* Evaluate the 1D basis tables (Sec. 2.3, eqs. cox1/cox2; derivatives by the
 * de Boor identity) into `out` (device, n_table_entries doubles) on
 * `cuda_stream`.  Order: patches, then directions, then elements of that
 * direction; one record per element of direction k: val[q_k][p_k+1],
 * der[q_k][p_k+1] of the p_k+1 functions non-zero on the element at its Gauss
 * points, then w[q_k], the Gauss weights times half the element length.  iga_integrate computes the same
 * tables internally; this entry exposes them for inspection. */
int iga_basis_tables(iga_plan_t plan, double* out, void* cuda_stream);

/* Sparsity pattern of the assembled global matrix (Sec. 3.1: the global
 * matrix sums the element matrices over the support index sets of the
 * elements, eq. 10 and the Remark on K^Delta_alpha; the insertion step of
 * Table 3, Sec. 3.3).  Entry (i, j) is present iff some element holds both
 * global functions i and j; patches are independent diagonal blocks.
 *   row_ptr: device, [n_dofs + 1] int64, row_ptr[n_dofs] = info.n_csr_nnz;
 *   col_idx: device, [n_csr_nnz] int32, ascending within each row.
 * Both are written on `cuda_stream` (caller-owned buffers; the pattern
 * depends on the plan only, so it needs computing once). */
int iga_csr_pattern(iga_plan_t plan, int64_t* row_ptr, int32_t* col_idx, void* cuda_stream);

/* Global assembly of element matrices into the values of the CSR pattern of
 * iga_csr_pattern (same Sec. 3.1 sum, the paper's insert-into-global step of
 * Table 3): values[z] of entry (i, j) is the sum, over the elements e that
 * hold both i and j in ascending element order, of A_elem[e][a][b] with
 * dof(e, a) = i and dof(e, b) = j.  A_elem is any per-element [E][N][N]
 * array laid out like K_out/M_out of iga_integrate ([n_mat_entries], device);
 * values is [n_csr_nnz], device.  Both are double for IGA_FP64/IGA_FP64_DF
 * plans and float otherwise; each entry is summed in that precision in
 * ascending element order.  No atomics: the result does not depend on
 * scheduling. */
int iga_assemble(iga_plan_t plan, const void* A_elem, void* values, void* cuda_stream);

/* Matrix-free operator application (3D, or 2D on IGA_FP64 plans; every patch):
 *   y = alpha K(kappa) x + beta M(rho) x,
 * the products K u and M u of the forward-Euler step of Sec. 2.2 (eq. Euler)
 * for the stiffness and mass of iga_integrate, without forming a global or
 * an element matrix: per element, x is interpolated at the quadrature points
 * by sum factorization (one direction at a time, as in Algorithm 2 of
 * Sec. 3.2), multiplied by the coefficient and geometry factors, and
 * integrated back against the test functions; the element results are then
 * summed per dof in ascending element order (deterministic, no atomics).
 *   kappa, rho: [n_qp] or NULL (= 1);  jac: [n_qp][d][d] or NULL (= identity);
 *   x, y: [n_dofs] device vectors, double for IGA_FP64/IGA_FP64_DF plans,
 *         float otherwise (FP32 arithmetic with FP64 Jacobian cofactors and
 *         determinant; IGA_FP64_DF computes in float-float on the FP32 pipes,
 *         FP64-accurate); y is overwritten and must not alias x.
 * The first call allocates plan-owned scratch of n_dofmap_entries values
 * (freed by iga_destroy). */
int iga_apply(iga_plan_t plan, const double* kappa, const double* rho, const double* jac,
              const void* x, double alpha, double beta, void* y, void* cuda_stream);

/* Backward of the element matrices with respect to the coefficients (not in
 * the paper).  3D: p <= 4 with q = p+1 or p+2, and p = 5 with q = 6 on FP32
 * plans; 2D (FP64 plans): p <= 5 with q = p+1 or p+2.  The
 * element matrices are linear in kappa and rho, so for upstream gradients
 * GK = dL/dK_e and GM = dL/dM_e (layout and dtype of iga_integrate's K_out):
 *   grad_kappa[k] = w_k |det G_k| sum_ab GK_ab (G_k^{-T} grad phi_a).(G_k^{-T} grad phi_b)
 *   grad_rho[k]   = w_k |det G_k| sum_ab GM_ab phi_a(x_k) phi_b(x_k)
 * at every quadrature point.  The double sum over (a, b) is evaluated by sum
 * factorization run backwards (x, then y, then z factors), one CTA per
 * element, in FP64 for IGA_FP64 plans, in float-float on the FP32 pipes for
 * IGA_FP64_DF plans (3D p <= 3; FP64 otherwise) and in FP32 (FP64 cofactors
 * and determinant) for the others.
 *   jac: [n_qp][d][d] or NULL (= identity).
 *   GK, GM: device, NULL skips that gradient (not both NULL).
 *   grad_kappa, grad_rho: device [n_qp], dtype of GK; required where the
 *   matching upstream gradient is given, overwritten. */
int iga_integrate_grad(iga_plan_t plan, const double* jac, const void* GK, const void* GM,
                       void* grad_kappa, void* grad_rho, void* cuda_stream);

/* Weighted quadrature for the mass matrix (2D and 3D, p <= 5; the variant Sec. 1.2
 * names as a further reduction of the integration cost, which the paper does
 * not define).  Each direction has one global point list: every element's
 * left end and midpoint, p+1 points in the p boundary elements at each end,
 * and the right end of the domain.  Test function B_i integrates with the
 * least-norm weights w_{i,q} on the points of its closed support that make
 * sum_q w_{i,q} B_j(x_q) = int B_i B_j exact for every spline B_j; the global
 * matrix is formed row by row,
 *   M_ij = sum_q w1_{i1,q1} w2_{i2,q2} w3_{i3,q3} c(x_q) B_j(x_q),
 * so no element matrix exists.  With c = 1 it is the exact Gram matrix.
 * iga_wq_points: number (n_out) and, if x_out != NULL (host, n_out
 * doubles), the parametric coordinates of the points of direction `dir` of
 * patch `patch`; dir = -1 gives the patch's grid size (x_out NULL), patch = -1
 * (with dir = -1) the total over patches.  The first call of either entry
 * builds the plan's tables (host least-norm solves, device upload).
 * iga_wq_mass: FP64 plans only (IGA_FP64_DF computes in float-float on the
 * FP32 pipes, FP64-accurate).  c: device, the coefficient (rho |det G| for
 * a mass) at every grid point, patches concatenated, each [n3][n2][n1] with x
 * fastest; NULL = 1.  values: device [n_csr_nnz] doubles on the pattern of
 * iga_csr_pattern, overwritten. */
int iga_wq_points(iga_plan_t plan, int patch, int dir, double* x_out, int64_t* n_out);
int iga_wq_mass(iga_plan_t plan, const double* c, double* values, void* cuda_stream);

/* Weighted quadrature for the diffusion stiffness (2D and 3D, 2 <= p <= 4; the same
 * variant extended to derivatives, not defined in the paper).  Besides the
 * mass rule above, each test function B_i has a derivative rule w'_{i,q} on
 * the same points: least-norm among the rules with sum_q w'_{i,q} B'_j(x_q) =
 * int B'_i B'_j for every spline B_j (the B'_j sum to zero on the support, so
 * one of these equations is dependent and is left out of the solve; B' at the
 * right end of the domain is the left limit).  The global matrix is formed
 * row by row,
 *   K_ij = sum_q c(x_q) sum_k prod_l R^{(l == k)}_{i_l}(x_{q_l}) B^{(l == k)}_{j_l}(x_{q_l}),
 * R^(0) the mass rule, R^(1) the derivative rule, B^(0) = B, B^(1) = B': the
 * reference-gradient form int c grad B_i . grad B_j (c = kappa for the
 * identity map).  With c = 1 it is the exact stiffness.  FP64 plans only;
 * c and values as for iga_wq_mass.  IGA_ERR_UNSUPPORTED for p < 2 or p > 4,
 * or rule tables beyond shared memory. */
int iga_wq_stiffness(iga_plan_t plan, const double* c, double* values, void* cuda_stream);

/* With opts.profile = 1: synchronize on the last recorded event and return
 * the summed device time (ms) of the element-matrix kernel launches since the
 * previous call, timed by CUDA events recorded on the caller's stream
 * immediately before and after them, and the number of such launches; then
 * reset the counters.  Returns IGA_ERR_ARG if profiling is off. */
int iga_profile_read(iga_plan_t plan, double* kernel_ms, int64_t* launches);

/* iga_integrate_backward without any device allocation.  The paper has no
 * counterpart: this entry exists for callers that cannot call cudaMalloc --
 * code that runs inside a memory pool or arena it does not own, an embedding
 * host whose allocator forbids foreign allocations, or a latency-critical loop
 * that must never enter the allocator -- and so cannot create a plan, which
 * allocates its tables.
 * It computes dJ/dkappa and J = u^T K(kappa) v (FP64) for one 3D patch whose
 * knot vectors are host arrays, with kappa, jac, u, v, grad_kappa and J_out
 * in device memory as for a FP64 plan's iga_integrate_backward (jac may be
 * NULL; kappa may be NULL only if J_out is NULL).  The patch must have one
 * degree (1..8) and one Gauss order (1..16) in all three directions
 * (IGA_ERR_UNSUPPORTED otherwise).  Its working memory is one file-scope
 * device array of 3.7 MiB that every GPU which loads the library holds until
 * the process exits: at most 1024 knots per direction, 262144 elements and
 * 196608 doubles of basis tables; larger patches return IGA_ERR_TOO_LARGE
 * before anything is launched.  The first call in a CUDA context (the
 * runtime's primary context of a device, or one the caller made current)
 * looks up the array's device address in that context, so make that first
 * call before any stream capture; the address is cached per context (by its
 * unique id), so a context created later, e.g. after cudaDeviceReset, gets
 * its own lookup.  All calls share the array: calls whose work overlaps on
 * the GPU (different streams, or different host threads on one device) race
 * and must be serialized by the caller.  Nothing in the array needs clearing:
 * each call overwrites what it reads.  The patch description (knots and the
 * Gauss rule, about 25 KB) travels to the device as a kernel parameter, which
 * needs the large kernel parameters of CUDA 12.1 or later.  Launch errors are
 * returned; the call does not synchronize. */
int iga_adjoint_noalloc(const iga_patch_desc* patch, const double* kappa, const double* jac,
                        const double* u, const double* v, double* grad_kappa, double* J_out,
                        void* cuda_stream);

/* Free the plan and its device memory; NULL-safe.  Returns the sticky device
 * status of the plan (IGA_OK if none). */
int iga_destroy(iga_plan_t plan);

/* Static, human-readable name of a status code. */
const char* iga_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif /* IGA_H */
