/*
 * iga_oracle.h -- plain, slow, FP64 CPU oracle for IGA-FEM element-matrix
 * integration over tensor-product B-spline bases (arxiv 2207.00280).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library and must never be used as a
 * fallback for it.
 *
 * Conventions (0-based everywhere, x fastest in every multi-index):
 *   knots t[0..m-1] per direction, degree p_k, number of functions m-p_k-1;
 *   elements per direction = non-empty knot spans [t_s, t_{s+1});
 *   element e = e1 + K1*(e2 + K2*e3);
 *   local function a = a1 + n_1*(a2 + n_2*a3), n_k = p_k+1, global 1D index
 *   s_k-p_k+a_k;
 *   quadrature point k = k1 + q_1*(k2 + q_2*k3);
 *   kappa[E][Q], rho[E][Q], G[E][Q][d][d] with G[i][j] = dx_i/dxi_j (row-major);
 *   element matrices [n_sel][N][N] row-major, N = n_1 n_2 (n_3), Q = q_1 q_2 (q_3).
 * The paper takes one degree for every direction and notes that the method
 * extends to bases of different degrees (Sec. 2.3); its element sum (eq. 10)
 * already has P_1, P_2, P_3 quadrature points per direction.  Each patch
 * therefore has a degree and a number of Gauss points per direction.
 *
 * Every function cites the passage of the paper it follows.  Items with no
 * counterpart in the paper (derivatives, stiffness, the adjoint) are written
 * from their textbook definitions and say so.
 */
#ifndef IGA_ORACLE_H
#define IGA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Gauss--Legendre rule on [-1,1] by Golub--Welsch: eigen-decomposition of the
 * symmetric tridiagonal Jacobi matrix of the Legendre recurrence, done with
 * cyclic Jacobi rotations.  Nodes ascending.  Returns 0 on success. */
int ora_gauss_legendre(int q, double* x, double* w);

/* B_{i;p}(xi), literally recursive Cox--de Boor (Sec. 2.3, eqs. cox1/cox2;
 * 0/0 := 0). */
double ora_bspline(const double* t, int i, int p, double xi);

/* dB_{i;p}/dxi by the de Boor derivative identity (not in the paper). */
double ora_bspline_deriv(const double* t, int i, int p, double xi);

/* Non-empty knot spans s (t_s < t_{s+1}, s = p..m-p-2) -> spans[], returns
 * their count (Sec. 2.3 knot vector; Sec. 3.1 element decomposition). */
int ora_spans(const double* t, int m, int p, int* spans);

/* One direction of one element: mapped Gauss nodes xi[q], mapped weights w[q]
 * (reference weight times half the span length), values val[q][n] and
 * derivatives der[q][n] of B_{s-p+r}, r = 0..p, by the recursive functions. */
void ora_basis_1d(const double* t, int p, int s, int q, double* xi, double* w,
                  double* val, double* der);

/* Description of one patch for the element-matrix routines. */
typedef struct {
  int dim;                 /* 2 or 3 */
  int p;                   /* degree of every direction whose pd[k] is 0 */
  int q;                   /* Gauss points of every direction whose qd[k] is 0 */
  int m[3];                /* knots per direction */
  const double* t[3];      /* knot vectors */
  int pd[3];               /* degree of direction k, or 0 (= p) */
  int qd[3];               /* Gauss points of direction k, or 0 (= q) */
} ora_patch;

/* Classical integration (Sec. 3.2, Algorithm 1; element integral eq. 10),
 * extended with the variable-coefficient stiffness:
 *   M_ab = sum_q w_q |det G_q| rho_q phi_a phi_b,
 *   K_ab = sum_q w_q |det G_q| kappa_q (G_q^{-T} grad phi_a).(G_q^{-T} grad phi_b).
 * elems[n_sel] are global element ids; kappa/rho/G are indexed by global id.
 * rho or G may be NULL (1 / identity); K or M may be NULL (skip).
 * Returns 0, or -1 on bad arguments. */
int ora_classical(const ora_patch* pt, const int64_t* elems, int64_t n_sel,
                  const double* kappa, const double* rho, const double* G,
                  double* K, double* M);

/* Sum factorization (Sec. 3.2, Algorithm 2; eqs. finalsum/bufferC): per
 * element and per derivative term, contract the last direction first, then
 * the middle, then x, with per-direction weights applied in their own stage.
 * Same arguments and result as ora_classical (up to rounding order). */
int ora_sumfact(const ora_patch* pt, const int64_t* elems, int64_t n_sel,
                const double* kappa, const double* rho, const double* G,
                double* K, double* M);

/* Global dof of each local function of each selected element (Remark on the
 * support set K^Delta_alpha, Sec. 3.1): dof = sum_k (s_k - p_k + a_k) * stride_k,
 * stride = 1, f_1, f_1 f_2 with f_k = m_k - p_k - 1 functions in direction k. */
int ora_dofmap(const ora_patch* pt, const int64_t* elems, int64_t n_sel,
               int32_t* dof);

/* Adjoint of J(kappa) = u^T K(kappa) v (not in the paper): for each selected
 * element and quadrature point
 *   g_q = w_q |det G_q| (G_q^{-T} grad u)(x_q) . (G_q^{-T} grad v)(x_q),
 * with grad u = sum_a u[dof(e,a)] grad phi_a.  Writes g[n_sel][Q] and
 * *J = sum over the selected elements of sum_q kappa_q g_q (if J != NULL). */
int ora_adjoint(const ora_patch* pt, const int64_t* elems, int64_t n_sel,
                const double* kappa, const double* G, const double* u,
                const double* v, double* g, double* J);

/* Sparsity pattern of the assembled global matrix.  The global matrix sums
 * the element matrices over the support index sets of the elements (Sec. 3.1,
 * eq. 10 and the Remark on K^Delta_alpha; the insertion step of Table 3,
 * Sec. 3.3), so entry (i, j) is present iff at least one element holds both
 * functions i and j.  Rows in global dof order, columns ascending.
 * row_ptr[n_dofs + 1] is always written; col_idx[row_ptr[n_dofs]] only if
 * non-NULL.  Returns 0, or -1 on bad arguments. */
int ora_csr_pattern(const ora_patch* pt, int64_t* row_ptr, int32_t* col_idx);

/* Global assembly of element matrices Ae[E][N][N] (every element of the
 * patch, in element order) into CSR values on the pattern of
 * ora_csr_pattern: values[z] of entry (i, j) is the sum over elements e, in
 * ascending e, of Ae[e][a][b] with dof(e,a) = i and dof(e,b) = j.  Returns 0,
 * -1 on bad arguments, -2 if an entry is missing from the pattern. */
int ora_assemble(const ora_patch* pt, const int64_t* row_ptr, const int32_t* col_idx,
                 const double* Ae, double* values);

/* Application of the assembled operators to a global vector x[n_dofs] (not in
 * the paper as such: the products K u and M u of the forward-Euler step of
 * Sec. 2.2, eq. Euler):
 *   yK = sum_e P_e^T K_e P_e x,   yM = sum_e P_e^T M_e P_e x,
 * with K_e, M_e the element matrices of ora_classical and P_e the gather
 * through the dof map; elements in ascending order.  kappa may be NULL (= 1)
 * only for the mass; yK or yM may be NULL (skip).  Returns 0, or -1. */
int ora_apply(const ora_patch* pt, const double* kappa, const double* rho, const double* G,
              const double* x, double* yK, double* yM);

/* Weighted quadrature for the mass matrix (named in Sec. 1.2 as a further
 * reduction of the integration cost; not defined in the paper -- the reading
 * below is written from the method's defining property).  For each test
 * function B_i, a rule sum_q w_{i,q} f(x_q) over global points x_q in the
 * closed support of B_i that integrates B_i f exactly for every spline f of
 * the space, i.e. sum_q w_{i,q} B_j(x_q) = int B_i B_j for all j; among such
 * rules the one of least Euclidean norm.
 * ora_wq_points: the global points of one direction, ascending: each
 * element's left end and midpoint, plus the right end of the last element; in
 * the first p and the last p elements instead the left end and p interior
 * points at fractions r/(p+1), r = 1..p.  Writes at most cap points to x,
 * returns their number (or -1). */
int ora_wq_points(const double* t, int m, int p, double* x, int cap);

/* The weights of one direction: W[nf][np] (row i = test function i, zero
 * outside the closed support), from the point set of ora_wq_points.  The
 * exact integrals int B_i B_j come from Gauss--Legendre with p+1 points per
 * element; the least-norm solution is W_i = A^T (A A^T)^{-1} r_i with
 * A[j][q] = B_j(x_q) restricted to the support, solved by Gaussian elimination
 * with partial pivoting.  Returns 0, or -1 (bad arguments or a singular
 * system). */
int ora_wq_weights(const double* t, int m, int p, const double* x, int np, double* W);

/* Global mass matrix by weighted quadrature, on the CSR pattern of
 * ora_csr_pattern: values[z] of entry (i, j) = sum over the points x_q of the
 * tensor grid (q = q1 + n1 (q2 + n2 q3)) of W1[i1][q1] W2[i2][q2] W3[i3][q3]
 * c[q] B_j1(x_q1) B_j2(x_q2) B_j3(x_q3) (2D: two factors).  c holds the
 * coefficient (for the mass: rho |det G|) at every grid point, or NULL = 1.
 * Returns 0, or -1. */
int ora_wq_mass(const ora_patch* pt, const double* c, const int64_t* row_ptr,
                const int32_t* col_idx, double* values);

/* The derivative rule of one direction (p >= 2, where the B'_j are
 * continuous at the points): W[nf][np] with sum_q W[i][q] B'_j(x_q) =
 * int B'_i B'_j for every j, least-norm, zero outside the closed support of
 * B_i; B' at the right end of the domain is the left limit.  The B'_j sum to
 * zero on every support, so one equation of each system is dependent (with a
 * consistent right-hand side) and is dropped before the solve.  Returns 0,
 * or -1. */
int ora_wq_weights_deriv(const double* t, int m, int p, const double* x, int np, double* W);

/* Global diffusion stiffness by weighted quadrature (p >= 2), on the CSR
 * pattern of ora_csr_pattern:
 *   values[z] of (i, j) = sum_k sum_q c[q] prod_l R^(k,l)_{i_l}(x_{q_l}) D^(k,l)_{j_l}(x_{q_l})
 * where for direction l = k the derivative rule and B'_{j_l}, for l != k the
 * mass rule and B_{j_l}: the reference-gradient form int c grad B_i . grad B_j
 * with c the coefficient (kappa for the identity map) at every grid
 * point (layout of ora_wq_mass), or NULL = 1.  Returns 0, or -1. */
int ora_wq_stiffness(const ora_patch* pt, const double* c, const int64_t* row_ptr,
                     const int32_t* col_idx, double* values);

/* Backward of the element matrices with respect to the coefficients (not in
 * the paper; the element integrals of eq. 10 and of the stiffness are linear
 * in kappa and rho): given upstream gradients GK[n_sel][N][N] = dL/dK_e and
 * GM[n_sel][N][N] = dL/dM_e (either may be NULL),
 *   gk[s][q] = dL/dkappa_q = w_q |det G_q| sum_ab GK_ab (G^{-T} grad phi_a).(G^{-T} grad phi_b)
 *   gr[s][q] = dL/drho_q   = w_q |det G_q| sum_ab GM_ab phi_a phi_b
 * at every quadrature point of every selected element, by the plain double
 * sum.  Returns 0, or -1. */
int ora_integrate_grad(const ora_patch* pt, const int64_t* elems, int64_t n_sel, const double* G,
                       const double* GK, const double* GM, double* gk, double* gr);

#ifdef __cplusplus
}
#endif
#endif
