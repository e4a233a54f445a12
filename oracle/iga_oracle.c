/*
 * iga_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for IGA-FEM
 * element-matrix integration (arxiv 2207.00280).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark, never by the CUDA library.  Nothing here is
 * shared with the GPU path.  Built with -O2 -ffp-contract=off so every product
 * and sum is rounded exactly as written.
 *
 * Pins (what fixes each function independently of itself) live in
 * tests/test_oracle_*.py: closed-form Gauss rules and polynomial exactness,
 * scipy's B-spline evaluation, partition of unity, exact rational integrals of
 * the piecewise polynomials, p = 1 Kronecker closed forms, K 1 = 0, mass sum =
 * element volume, classical == sum factorization, Greville identities and
 * finite differences for the adjoint, brute-force support sets for the dofs.
 */
#include "iga_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Gauss--Legendre by Golub--Welsch.                                         */
/* The paper only asks for "a proper exact quadrature" (Sec. 3.1, eq. 10).   */
/* Nodes are the eigenvalues of the Jacobi matrix of the Legendre three-term */
/* recurrence (zero diagonal, off-diagonal k / sqrt(4k^2-1)); the weight of a */
/* node is 2 v_0^2 from its normalised eigenvector.  The eigenproblem is     */
/* solved by cyclic Jacobi rotations (Golub & Van Loan, "Matrix              */
/* Computations", Sec. 8.5: each rotation zeroes one off-diagonal pair).     */
/* ------------------------------------------------------------------------ */
int ora_gauss_legendre(int q, double* x, double* w) {
  if (q < 1 || q > 64 || !x || !w) return -1;
  double* A = (double*)calloc((size_t)q * q, sizeof(double));
  double* V = (double*)calloc((size_t)q * q, sizeof(double));
  if (!A || !V) { free(A); free(V); return -1; }
  for (int i = 0; i < q; ++i) V[i * q + i] = 1.0;
  for (int k = 1; k < q; ++k) {
    double beta = (double)k / sqrt(4.0 * k * k - 1.0);
    A[k * q + (k - 1)] = beta;
    A[(k - 1) * q + k] = beta;
  }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j)
        if (i != j) off += A[i * q + j] * A[i * q + j];
    if (off < 1e-60) break;
    for (int pp = 0; pp < q - 1; ++pp) {
      for (int r = pp + 1; r < q; ++r) {
        double apr = A[pp * q + r];
        if (apr == 0.0) continue;
        double tau = (A[r * q + r] - A[pp * q + pp]) / (2.0 * apr);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        for (int k = 0; k < q; ++k) { /* A <- A J */
          double akp = A[k * q + pp], akr = A[k * q + r];
          A[k * q + pp] = c * akp - s * akr;
          A[k * q + r] = s * akp + c * akr;
        }
        for (int k = 0; k < q; ++k) { /* A <- J^T A */
          double apk = A[pp * q + k], ark = A[r * q + k];
          A[pp * q + k] = c * apk - s * ark;
          A[r * q + k] = s * apk + c * ark;
        }
        for (int k = 0; k < q; ++k) { /* V <- V J */
          double vkp = V[k * q + pp], vkr = V[k * q + r];
          V[k * q + pp] = c * vkp - s * vkr;
          V[k * q + r] = s * vkp + c * vkr;
        }
      }
    }
  }
  for (int i = 0; i < q; ++i) {
    x[i] = A[i * q + i];
    w[i] = 2.0 * V[0 * q + i] * V[0 * q + i];
  }
  /* insertion sort by node, ascending */
  for (int i = 1; i < q; ++i) {
    double xi = x[i], wi = w[i];
    int j = i - 1;
    while (j >= 0 && x[j] > xi) { x[j + 1] = x[j]; w[j + 1] = w[j]; --j; }
    x[j + 1] = xi; w[j + 1] = wi;
  }
  free(A); free(V);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Cox--de Boor, literally recursive (Sec. 2.3, eqs. cox1 and cox2).         */
/* Degree 0 is the indicator of the half-open span [t_i, t_{i+1}); a term    */
/* whose knot-difference denominator vanishes is 0 ("0/0 := 0").             */
/* ------------------------------------------------------------------------ */
double ora_bspline(const double* t, int i, int p, double xi) {
  if (p == 0) return (t[i] <= xi && xi < t[i + 1]) ? 1.0 : 0.0;
  double left = 0.0, right = 0.0;
  double d1 = t[i + p] - t[i];
  double d2 = t[i + p + 1] - t[i + 1];
  if (d1 != 0.0) left = (xi - t[i]) / d1 * ora_bspline(t, i, p - 1, xi);
  if (d2 != 0.0) right = (t[i + p + 1] - xi) / d2 * ora_bspline(t, i + 1, p - 1, xi);
  return left + right;
}

/* Derivative (not in the paper; de Boor, "A Practical Guide to Splines",
 * ch. X):  B'_{i;p} = p/(t_{i+p}-t_i) B_{i;p-1} - p/(t_{i+p+1}-t_{i+1}) B_{i+1;p-1},
 * zero-denominator terms taken as 0. */
double ora_bspline_deriv(const double* t, int i, int p, double xi) {
  if (p == 0) return 0.0;
  double a = 0.0, b = 0.0;
  double d1 = t[i + p] - t[i];
  double d2 = t[i + p + 1] - t[i + 1];
  if (d1 != 0.0) a = (double)p / d1 * ora_bspline(t, i, p - 1, xi);
  if (d2 != 0.0) b = (double)p / d2 * ora_bspline(t, i + 1, p - 1, xi);
  return a - b;
}

/* Elements = non-empty spans of the knot vector (Sec. 2.3 knot vector with
 * p+1 repeated end knots; Sec. 3.1 element decomposition). */
int ora_spans(const double* t, int m, int p, int* spans) {
  int c = 0;
  for (int s = p; s <= m - p - 2; ++s)
    if (t[s] < t[s + 1]) spans[c++] = s;
  return c;
}

/* Quadrature nodes and weights mapped to the span, and the p+1 non-zero
 * functions B_{s-p+r} and their derivatives at each node. */
void ora_basis_1d(const double* t, int p, int s, int q, double* xi, double* w,
                  double* val, double* der) {
  double xr[64], wr[64];
  ora_gauss_legendre(q, xr, wr);
  double a = t[s], b = t[s + 1];
  double mid = 0.5 * (a + b), half = 0.5 * (b - a);
  for (int j = 0; j < q; ++j) {
    xi[j] = mid + half * xr[j];
    w[j] = half * wr[j];
    for (int r = 0; r <= p; ++r) {
      val[j * (p + 1) + r] = ora_bspline(t, s - p + r, p, xi[j]);
      der[j * (p + 1) + r] = ora_bspline_deriv(t, s - p + r, p, xi[j]);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Shared bookkeeping for the element routines.                              */
/* ------------------------------------------------------------------------ */
/* Per direction k: degree p[k], n[k] = p[k]+1 functions per element, q[k]
 * Gauss points (eq. 10 takes P_k points in direction k).  A direction beyond
 * the patch's dimension has n = q = 1 so that the index products hold. */
typedef struct {
  int d, p[3], n[3], q[3], N, Q;
  int K[3];           /* elements per direction */
  int* spans[3];
} layout;

static int make_layout(const ora_patch* pt, layout* L) {
  for (int k = 0; k < 3; ++k) { L->spans[k] = NULL; L->K[k] = 1; L->p[k] = 0; L->n[k] = 1; L->q[k] = 1; }
  if (!pt || (pt->dim != 2 && pt->dim != 3)) return -1;
  L->d = pt->dim;
  L->N = 1; L->Q = 1;
  for (int k = 0; k < L->d; ++k) {
    const int p = pt->pd[k] ? pt->pd[k] : pt->p;
    const int q = pt->qd[k] ? pt->qd[k] : pt->q;
    if (p < 1 || p > 16 || q < 1 || q > 64) return -1;
    L->p[k] = p; L->n[k] = p + 1; L->q[k] = q;
    if (!pt->t[k] || pt->m[k] < 2 * p + 2) return -1;
    L->spans[k] = (int*)malloc(sizeof(int) * (size_t)pt->m[k]);
    L->K[k] = ora_spans(pt->t[k], pt->m[k], p, L->spans[k]);
    L->N *= L->n[k]; L->Q *= L->q[k];
  }
  return 0;
}

/* 1 if every direction of the patch has the same degree. */
static int same_degree(const layout* L) {
  for (int k = 1; k < L->d; ++k)
    if (L->p[k] != L->p[0]) return 0;
  return 1;
}

static void free_layout(layout* L) {
  for (int k = 0; k < 3; ++k) free(L->spans[k]);
}

static int64_t n_elements(const layout* L) {
  return (int64_t)L->K[0] * L->K[1] * (L->d == 3 ? L->K[2] : 1);
}

/* element id -> per-direction element index */
static void split_elem(const layout* L, int64_t e, int* ek) {
  ek[0] = (int)(e % L->K[0]);
  int64_t r = e / L->K[0];
  ek[1] = (int)(r % L->K[1]);
  ek[2] = (L->d == 3) ? (int)(r / L->K[1]) : 0;
}

/* |det G| and G^{-1} of a d x d row-major matrix by cofactors. */
static double geom_inverse(int d, const double* G, double* Ginv) {
  if (d == 2) {
    double det = G[0] * G[3] - G[1] * G[2];
    Ginv[0] = G[3] / det; Ginv[1] = -G[1] / det;
    Ginv[2] = -G[2] / det; Ginv[3] = G[0] / det;
    return fabs(det);
  }
  double c00 = G[4] * G[8] - G[5] * G[7];
  double c01 = G[5] * G[6] - G[3] * G[8];
  double c02 = G[3] * G[7] - G[4] * G[6];
  double det = G[0] * c00 + G[1] * c01 + G[2] * c02;
  /* inverse = adjugate / det, adjugate = cofactor matrix transposed */
  Ginv[0] = c00 / det;
  Ginv[1] = (G[2] * G[7] - G[1] * G[8]) / det;
  Ginv[2] = (G[1] * G[5] - G[2] * G[4]) / det;
  Ginv[3] = c01 / det;
  Ginv[4] = (G[0] * G[8] - G[2] * G[6]) / det;
  Ginv[5] = (G[2] * G[3] - G[0] * G[5]) / det;
  Ginv[6] = c02 / det;
  Ginv[7] = (G[1] * G[6] - G[0] * G[7]) / det;
  Ginv[8] = (G[0] * G[4] - G[1] * G[3]) / det;
  return fabs(det);
}

/* Per-element 1D data for every direction. */
typedef struct {
  double xi[3][64], w[3][64];
  double val[3][64 * 17], der[3][64 * 17];
} elem1d;

static void element_1d(const ora_patch* pt, const layout* L, const int* ek, elem1d* B) {
  for (int k = 0; k < L->d; ++k)
    ora_basis_1d(pt->t[k], L->p[k], L->spans[k][ek[k]], L->q[k], B->xi[k], B->w[k],
                 B->val[k], B->der[k]);
}

/* Quadrature point k -> per-direction indices (k = k1 + q_1 (k2 + q_2 k3)). */
static void split_qp(const layout* L, int k, int* kk) {
  kk[0] = k % L->q[0];
  kk[1] = (k / L->q[0]) % L->q[1];
  kk[2] = (L->d == 3) ? k / (L->q[0] * L->q[1]) : 0;
}

/* Local function a -> per-direction indices (a = a1 + n_1 (a2 + n_2 a3)). */
static void split_local(const layout* L, int a, int* aa) {
  aa[0] = a % L->n[0];
  aa[1] = (a / L->n[0]) % L->n[1];
  aa[2] = (L->d == 3) ? a / (L->n[0] * L->n[1]) : 0;
}

/* Value (s = 0) or derivative (s = 1) of local function r of direction j at
 * its Gauss point k. */
#define B1D(B, L, j, s, r, k) \
  ((s) ? (B)->der[j][(k) * (L)->n[j] + (r)] : (B)->val[j][(k) * (L)->n[j] + (r)])

/* Weights, |det G| and G^{-T}-mapped reference gradients at every quadrature
 * point of one element: the J(x^n) of eq. 10 is |det G| with G the derivative
 * of the geometry map with respect to the knot coordinates; the factor from
 * the reference interval to the span sits in the mapped weights. */
static void element_geometry(const layout* L, int64_t e, const elem1d* B,
                             const double* G, double* W, double* Ginv) {
  int d = L->d;
  for (int k = 0; k < L->Q; ++k) {
    int kk[3];
    split_qp(L, k, kk);
    double wq = 1.0;
    for (int j = 0; j < d; ++j) wq *= B->w[j][kk[j]];
    double Gid[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    double G2[4] = {1, 0, 0, 1};
    const double* Gq;
    if (G) Gq = G + ((size_t)e * L->Q + k) * d * d;
    else Gq = (d == 3) ? Gid : G2;
    double det = geom_inverse(d, Gq, Ginv + (size_t)k * d * d);
    W[k] = wq * det;
  }
}

/* ------------------------------------------------------------------------ */
/* Classical integration: Algorithm 1 (Sec. 3.2) on the sum of eq. 10.       */
/* ------------------------------------------------------------------------ */
int ora_classical(const ora_patch* pt, const int64_t* elems, int64_t n_sel,
                  const double* kappa, const double* rho, const double* G,
                  double* K, double* M) {
  layout L;
  if (make_layout(pt, &L)) { free_layout(&L); return -1; }
  if (K && !kappa) { free_layout(&L); return -1; }
  int d = L.d, N = L.N, Q = L.Q;
  const int n1 = L.n[0], n2 = L.n[1], n3 = L.n[2];
  int64_t E = n_elements(&L);
  elem1d* B = (elem1d*)malloc(sizeof(elem1d));
  double* W = (double*)malloc(sizeof(double) * Q);
  double* Ginv = (double*)malloc(sizeof(double) * Q * 9);
  double* phi = (double*)malloc(sizeof(double) * (size_t)N * Q);
  double* grad = (double*)malloc(sizeof(double) * (size_t)N * Q * 3);
  for (int64_t s = 0; s < n_sel; ++s) {
    int64_t e = elems[s];
    if (e < 0 || e >= E) { free(B); free(W); free(Ginv); free(phi); free(grad); free_layout(&L); return -1; }
    int ek[3];
    split_elem(&L, e, ek);
    element_1d(pt, &L, ek, B);
    element_geometry(&L, e, B, G, W, Ginv);
    /* basis values and physical gradients of the tensor functions (eq.
     * basis_construction) at every quadrature point */
    for (int a = 0; a < N; ++a) {
      int aa[3];
      split_local(&L, a, aa);
      for (int k = 0; k < Q; ++k) {
        int kk[3];
        split_qp(&L, k, kk);
        double v = 1.0, gr[3];
        for (int j = 0; j < d; ++j) v *= B1D(B, &L, j, 0, aa[j], kk[j]);
        for (int i = 0; i < d; ++i) {
          double g = 1.0;
          for (int j = 0; j < d; ++j) g *= B1D(B, &L, j, i == j, aa[j], kk[j]);
          gr[i] = g;
        }
        phi[(size_t)a * Q + k] = v;
        const double* Gi = Ginv + (size_t)k * d * d;
        for (int i = 0; i < d; ++i) { /* (G^{-T} gr)_i = sum_j Ginv[j][i] gr_j */
          double s2 = 0.0;
          for (int j = 0; j < d; ++j) s2 += Gi[j * d + i] * gr[j];
          grad[((size_t)a * Q + k) * 3 + i] = s2;
        }
      }
    }
    double* Ke = K ? K + (size_t)s * N * N : NULL;
    double* Me = M ? M + (size_t)s * N * N : NULL;
    /* the six nested test/trial loops of Algorithm 1, then the quadrature
     * loop (n3 = 1 in 2D) */
    for (int i1 = 0; i1 < n1; ++i1)
      for (int j1 = 0; j1 < n1; ++j1)
        for (int i2 = 0; i2 < n2; ++i2)
          for (int j2 = 0; j2 < n2; ++j2)
            for (int i3 = 0; i3 < n3; ++i3)
              for (int j3 = 0; j3 < n3; ++j3) {
                int a = i1 + n1 * (i2 + n2 * i3);
                int b = j1 + n1 * (j2 + n2 * j3);
                double mab = 0.0, kab = 0.0;
                for (int k = 0; k < Q; ++k) {
                  if (Me) {
                    double r = rho ? rho[(size_t)e * Q + k] : 1.0;
                    mab += phi[(size_t)a * Q + k] * phi[(size_t)b * Q + k] * W[k] * r;
                  }
                  if (Ke) {
                    double dot = 0.0;
                    for (int i = 0; i < d; ++i)
                      dot += grad[((size_t)a * Q + k) * 3 + i] * grad[((size_t)b * Q + k) * 3 + i];
                    kab += dot * W[k] * kappa[(size_t)e * Q + k];
                  }
                }
                if (Me) Me[(size_t)a * N + b] = mab;
                if (Ke) Ke[(size_t)a * N + b] = kab;
              }
  }
  free(B); free(W); free(Ginv); free(phi); free(grad);
  free_layout(&L);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Sum factorization: Algorithm 2 (Sec. 3.2, eqs. finalsum and bufferC).     */
/* Each term of the integrand is a product of one factor per direction       */
/* (value or derivative of the test and of the trial function) and a        */
/* coefficient J^t at the quadrature point.  The mass has one term; the      */
/* stiffness has d*d terms (alpha, beta) = (direction differentiated in the  */
/* test function, in the trial function) with coefficient                    */
/* |det G| kappa (G^{-1} G^{-T})_{alpha beta}.  Buffers follow Algorithm 2:  */
/* D(i3,j3,k1,k2) sums over k3 with w_z, C(i2,i3,j2,j3,k1) over k2 with w_y, */
/* A(a,b) over k1 with w_x.  In 2D the last-direction stage is the y stage.  */
/* ------------------------------------------------------------------------ */
static void sf_term(const layout* L, const elem1d* B, const double* coef,
                    int sa[3], int sb[3], double* Dbuf, double* Cbuf, double* A) {
  const int n1 = L->n[0], n2 = L->n[1], n3 = L->n[2];
  const int q1 = L->q[0], q2 = L->q[1], q3 = L->q[2], N = L->N;
  /* factor of direction j for the test (s = sa[j]) or trial (s = sb[j]) function */
#define FAC(j, s, r, k) B1D(B, L, j, s, r, k)
  if (L->d == 3) {
    /* D(i3,j3,k1,k2) = sum_k3 Bz_i3 Bz_j3 w_z J */
    for (int i3 = 0; i3 < n3; ++i3)
      for (int j3 = 0; j3 < n3; ++j3)
        for (int k1 = 0; k1 < q1; ++k1)
          for (int k2 = 0; k2 < q2; ++k2) {
            double acc = 0.0;
            for (int k3 = 0; k3 < q3; ++k3)
              acc += FAC(2, sa[2], i3, k3) * FAC(2, sb[2], j3, k3) * B->w[2][k3] *
                     coef[k1 + q1 * (k2 + q2 * k3)];
            Dbuf[((i3 * n3 + j3) * q1 + k1) * q2 + k2] = acc;
          }
    /* C(i2,i3,j2,j3,k1) = sum_k2 By_i2 By_j2 D(i3,j3,k1,k2) w_y */
    for (int i2 = 0; i2 < n2; ++i2)
      for (int j2 = 0; j2 < n2; ++j2)
        for (int i3 = 0; i3 < n3; ++i3)
          for (int j3 = 0; j3 < n3; ++j3)
            for (int k1 = 0; k1 < q1; ++k1) {
              double acc = 0.0;
              for (int k2 = 0; k2 < q2; ++k2)
                acc += FAC(1, sa[1], i2, k2) * FAC(1, sb[1], j2, k2) *
                       Dbuf[((i3 * n3 + j3) * q1 + k1) * q2 + k2] * B->w[1][k2];
              Cbuf[(((i2 * n3 + i3) * n2 + j2) * n3 + j3) * q1 + k1] = acc;
            }
    /* A((i1,i2,i3),(j1,j2,j3)) += sum_k1 Bx_i1 Bx_j1 C(i2,i3,j2,j3,k1) w_x */
    for (int i1 = 0; i1 < n1; ++i1)
      for (int j1 = 0; j1 < n1; ++j1)
        for (int i2 = 0; i2 < n2; ++i2)
          for (int j2 = 0; j2 < n2; ++j2)
            for (int i3 = 0; i3 < n3; ++i3)
              for (int j3 = 0; j3 < n3; ++j3) {
                double acc = 0.0;
                for (int k1 = 0; k1 < q1; ++k1)
                  acc += FAC(0, sa[0], i1, k1) * FAC(0, sb[0], j1, k1) *
                         Cbuf[(((i2 * n3 + i3) * n2 + j2) * n3 + j3) * q1 + k1] * B->w[0][k1];
                int a = i1 + n1 * (i2 + n2 * i3);
                int b = j1 + n1 * (j2 + n2 * j3);
                A[(size_t)a * N + b] += acc;
              }
  } else {
    /* D(i2,j2,k1) = sum_k2 By_i2 By_j2 w_y J */
    for (int i2 = 0; i2 < n2; ++i2)
      for (int j2 = 0; j2 < n2; ++j2)
        for (int k1 = 0; k1 < q1; ++k1) {
          double acc = 0.0;
          for (int k2 = 0; k2 < q2; ++k2)
            acc += FAC(1, sa[1], i2, k2) * FAC(1, sb[1], j2, k2) * B->w[1][k2] *
                   coef[k1 + q1 * k2];
          Dbuf[(i2 * n2 + j2) * q1 + k1] = acc;
        }
    /* A((i1,i2),(j1,j2)) += sum_k1 Bx_i1 Bx_j1 D(i2,j2,k1) w_x */
    for (int i1 = 0; i1 < n1; ++i1)
      for (int j1 = 0; j1 < n1; ++j1)
        for (int i2 = 0; i2 < n2; ++i2)
          for (int j2 = 0; j2 < n2; ++j2) {
            double acc = 0.0;
            for (int k1 = 0; k1 < q1; ++k1)
              acc += FAC(0, sa[0], i1, k1) * FAC(0, sb[0], j1, k1) *
                     Dbuf[(i2 * n2 + j2) * q1 + k1] * B->w[0][k1];
            A[(size_t)(i1 + n1 * i2) * N + (j1 + n1 * j2)] += acc;
          }
  }
#undef FAC
}

int ora_sumfact(const ora_patch* pt, const int64_t* elems, int64_t n_sel,
                const double* kappa, const double* rho, const double* G,
                double* K, double* M) {
  layout L;
  if (make_layout(pt, &L)) { free_layout(&L); return -1; }
  if (K && !kappa) { free_layout(&L); return -1; }
  int d = L.d, N = L.N, Q = L.Q;
  int64_t E = n_elements(&L);
  elem1d* B = (elem1d*)malloc(sizeof(elem1d));
  double* coef = (double*)malloc(sizeof(double) * Q);
  /* stage buffers: D [n_last^2][q1][q2], C [n2^2 n3^2][q1] (sizes of the 3D
   * case, which cover the 2D one) */
  const size_t nl = (size_t)L.n[d - 1];
  double* Dbuf = (double*)malloc(sizeof(double) * nl * nl * L.q[0] * L.q[1]);
  double* Cbuf = (double*)malloc(sizeof(double) * (size_t)L.n[1] * L.n[1] * L.n[2] * L.n[2] * L.q[0]);
  for (int64_t s = 0; s < n_sel; ++s) {
    int64_t e = elems[s];
    if (e < 0 || e >= E) { free(B); free(coef); free(Dbuf); free(Cbuf); free_layout(&L); return -1; }
    int ek[3];
    split_elem(&L, e, ek);
    element_1d(pt, &L, ek, B);
    /* J(x^n) of eq. 10 without the weights, which Algorithm 2 applies one
     * direction per stage. */
    double* Ke = K ? K + (size_t)s * N * N : NULL;
    double* Me = M ? M + (size_t)s * N * N : NULL;
    if (Me) {
      memset(Me, 0, sizeof(double) * (size_t)N * N);
      for (int k = 0; k < Q; ++k) {
        double Gid[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, G2[4] = {1, 0, 0, 1}, tmp[9];
        const double* Gq = G ? G + ((size_t)e * Q + k) * d * d : (d == 3 ? Gid : G2);
        double det = geom_inverse(d, Gq, tmp);
        coef[k] = det * (rho ? rho[(size_t)e * Q + k] : 1.0);
      }
      int sa[3] = {0, 0, 0}, sb[3] = {0, 0, 0};
      sf_term(&L, B, coef, sa, sb, Dbuf, Cbuf, Me);
    }
    if (Ke) {
      memset(Ke, 0, sizeof(double) * (size_t)N * N);
      for (int al = 0; al < d; ++al)
        for (int be = 0; be < d; ++be) {
          for (int k = 0; k < Q; ++k) {
            double Gid[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, G2[4] = {1, 0, 0, 1}, Gi[9];
            const double* Gq = G ? G + ((size_t)e * Q + k) * d * d : (d == 3 ? Gid : G2);
            double det = geom_inverse(d, Gq, Gi);
            double gg = 0.0; /* (G^{-1} G^{-T})_{al be} = sum_l Ginv[al][l] Ginv[be][l] */
            for (int l = 0; l < d; ++l) gg += Gi[al * d + l] * Gi[be * d + l];
            coef[k] = det * kappa[(size_t)e * Q + k] * gg;
          }
          int sa[3] = {al == 0, al == 1, al == 2};
          int sb[3] = {be == 0, be == 1, be == 2};
          sf_term(&L, B, coef, sa, sb, Dbuf, Cbuf, Ke);
        }
    }
  }
  free(B); free(coef); free(Dbuf); free(Cbuf);
  free_layout(&L);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Dof map (Remark on K^Delta_alpha, Sec. 3.1; ordering x fastest).          */
/* ------------------------------------------------------------------------ */
int ora_dofmap(const ora_patch* pt, const int64_t* elems, int64_t n_sel, int32_t* dof) {
  layout L;
  if (make_layout(pt, &L)) { free_layout(&L); return -1; }
  int64_t E = n_elements(&L);
  int64_t nf[3] = {1, 1, 1};
  for (int k = 0; k < L.d; ++k) nf[k] = pt->m[k] - L.p[k] - 1;
  for (int64_t s = 0; s < n_sel; ++s) {
    int64_t e = elems[s];
    if (e < 0 || e >= E) { free_layout(&L); return -1; }
    int ek[3];
    split_elem(&L, e, ek);
    for (int a = 0; a < L.N; ++a) {
      int aa[3];
      split_local(&L, a, aa);
      int64_t g = 0, stride = 1;
      for (int k = 0; k < L.d; ++k) {
        g += (int64_t)(L.spans[k][ek[k]] - L.p[k] + aa[k]) * stride;
        stride *= nf[k];
      }
      dof[(size_t)s * L.N + a] = (int32_t)g;
    }
  }
  free_layout(&L);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of J(kappa) = u^T K(kappa) v (not in the paper): J is linear in    */
/* kappa, J = sum_q kappa_q g_q, so dJ/dkappa_q = g_q.                        */
/* ------------------------------------------------------------------------ */
int ora_adjoint(const ora_patch* pt, const int64_t* elems, int64_t n_sel,
                const double* kappa, const double* G, const double* u,
                const double* v, double* g, double* J) {
  layout L;
  if (make_layout(pt, &L)) { free_layout(&L); return -1; }
  int d = L.d, N = L.N, Q = L.Q;
  int64_t E = n_elements(&L);
  elem1d* B = (elem1d*)malloc(sizeof(elem1d));
  double* W = (double*)malloc(sizeof(double) * Q);
  double* Ginv = (double*)malloc(sizeof(double) * Q * 9);
  int32_t* dof = (int32_t*)malloc(sizeof(int32_t) * N);
  double Jsum = 0.0;
  for (int64_t s = 0; s < n_sel; ++s) {
    int64_t e = elems[s];
    if (e < 0 || e >= E) { free(B); free(W); free(Ginv); free(dof); free_layout(&L); return -1; }
    int ek[3];
    split_elem(&L, e, ek);
    element_1d(pt, &L, ek, B);
    element_geometry(&L, e, B, G, W, Ginv);
    ora_dofmap(pt, &e, 1, dof);
    for (int k = 0; k < Q; ++k) {
      int kk[3];
      split_qp(&L, k, kk);
      double gu[3] = {0, 0, 0}, gv[3] = {0, 0, 0};
      for (int a = 0; a < N; ++a) {
        int aa[3];
        split_local(&L, a, aa);
        for (int i = 0; i < d; ++i) {
          double f = 1.0;
          for (int j = 0; j < d; ++j) f *= B1D(B, &L, j, i == j, aa[j], kk[j]);
          gu[i] += u[dof[a]] * f;
          gv[i] += v[dof[a]] * f;
        }
      }
      const double* Gi = Ginv + (size_t)k * d * d;
      double dot = 0.0;
      for (int i = 0; i < d; ++i) {
        double pu = 0.0, pv = 0.0;
        for (int j = 0; j < d; ++j) { pu += Gi[j * d + i] * gu[j]; pv += Gi[j * d + i] * gv[j]; }
        dot += pu * pv;
      }
      double gq = W[k] * dot;
      g[(size_t)s * Q + k] = gq;
      if (kappa) Jsum += kappa[(size_t)e * Q + k] * gq;
    }
  }
  if (J) *J = Jsum;
  free(B); free(W); free(Ginv); free(dof);
  free_layout(&L);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Global assembly: the global matrix is the sum of the element matrices     */
/* placed at their support index sets (Sec. 3.1, eq. 10 and the Remark on    */
/* K^Delta_alpha; the insertion step of Table 3).                            */
/* ------------------------------------------------------------------------ */
static int64_t n_global_dofs(const ora_patch* pt, const layout* L) {
  int64_t nd = 1;
  for (int k = 0; k < L->d; ++k) nd *= pt->m[k] - L->p[k] - 1;
  return nd;
}

static int cmp_i32(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

int ora_csr_pattern(const ora_patch* pt, int64_t* row_ptr, int32_t* col_idx) {
  layout L;
  if (!row_ptr || make_layout(pt, &L)) { free_layout(&L); return -1; }
  const int64_t E = n_elements(&L), nd = n_global_dofs(pt, &L);
  const int N = L.N;
  /* the elements that hold each dof: counts, prefix sums, lists */
  int64_t* first = (int64_t*)calloc((size_t)nd + 1, sizeof(int64_t));
  int64_t* fill = (int64_t*)calloc((size_t)nd, sizeof(int64_t));
  int64_t* owner = (int64_t*)malloc(sizeof(int64_t) * (size_t)(E * N > 0 ? E * N : 1));
  int32_t* dof = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nd > 0 ? nd : 1));
  int32_t* row = NULL;
  int64_t row_cap = 0;
  for (int64_t e = 0; e < E; ++e) {
    ora_dofmap(pt, &e, 1, dof);
    for (int a = 0; a < N; ++a) first[dof[a] + 1]++;
  }
  for (int64_t i = 0; i < nd; ++i) first[i + 1] += first[i];
  for (int64_t e = 0; e < E; ++e) {
    ora_dofmap(pt, &e, 1, dof);
    for (int a = 0; a < N; ++a) owner[first[dof[a]] + fill[dof[a]]++] = e;
  }
  for (int64_t i = 0; i < nd; ++i) mark[i] = -1;
  row_ptr[0] = 0;
  for (int64_t i = 0; i < nd; ++i) {
    int64_t cnt = 0;
    const int64_t need = (first[i + 1] - first[i]) * N;
    if (need > row_cap) {
      row_cap = need;
      row = (int32_t*)realloc(row, sizeof(int32_t) * (size_t)row_cap);
    }
    for (int64_t o = first[i]; o < first[i + 1]; ++o) {
      ora_dofmap(pt, &owner[o], 1, dof);
      for (int b = 0; b < N; ++b)
        if (mark[dof[b]] != i) { mark[dof[b]] = i; row[cnt++] = dof[b]; }
    }
    qsort(row, (size_t)cnt, sizeof(int32_t), cmp_i32);
    if (col_idx) memcpy(col_idx + row_ptr[i], row, sizeof(int32_t) * (size_t)cnt);
    row_ptr[i + 1] = row_ptr[i] + cnt;
  }
  free(first); free(fill); free(owner); free(dof); free(mark); free(row);
  free_layout(&L);
  return 0;
}

int ora_assemble(const ora_patch* pt, const int64_t* row_ptr, const int32_t* col_idx,
                 const double* Ae, double* values) {
  layout L;
  if (!row_ptr || !col_idx || !Ae || !values || make_layout(pt, &L)) { free_layout(&L); return -1; }
  const int64_t E = n_elements(&L), nd = n_global_dofs(pt, &L);
  const int N = L.N;
  int32_t* dof = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  int rc = 0;
  for (int64_t z = 0; z < row_ptr[nd]; ++z) values[z] = 0.0;
  for (int64_t e = 0; e < E && rc == 0; ++e) {
    ora_dofmap(pt, &e, 1, dof);
    for (int a = 0; a < N && rc == 0; ++a) {
      const int64_t lo = row_ptr[dof[a]], hi = row_ptr[dof[a] + 1];
      for (int b = 0; b < N; ++b) {
        /* binary search of column dof[b] in row dof[a] */
        int64_t l = lo, h = hi;
        while (l < h) {
          int64_t mid = l + (h - l) / 2;
          if (col_idx[mid] < dof[b]) l = mid + 1; else h = mid;
        }
        if (l >= hi || col_idx[l] != dof[b]) { rc = -2; break; }
        values[l] += Ae[((size_t)e * N + a) * N + b];
      }
    }
  }
  free(dof);
  free_layout(&L);
  return rc;
}

int ora_apply(const ora_patch* pt, const double* kappa, const double* rho, const double* G,
              const double* x, double* yK, double* yM) {
  layout L;
  if (!x || (!yK && !yM) || make_layout(pt, &L)) { free_layout(&L); return -1; }
  const int64_t E = n_elements(&L), nd = n_global_dofs(pt, &L);
  const int N = L.N, Q = L.Q;
  double* ones = NULL;
  if (yK && !kappa) {
    ones = (double*)malloc(sizeof(double) * (size_t)(E * Q));
    for (int64_t i = 0; i < E * Q; ++i) ones[i] = 1.0;
    kappa = ones;
  }
  double* Ke = yK ? (double*)malloc(sizeof(double) * (size_t)N * N) : NULL;
  double* Me = yM ? (double*)malloc(sizeof(double) * (size_t)N * N) : NULL;
  int32_t* dof = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  for (int64_t i = 0; i < nd; ++i) {
    if (yK) yK[i] = 0.0;
    if (yM) yM[i] = 0.0;
  }
  for (int64_t e = 0; e < E; ++e) {
    ora_classical(pt, &e, 1, kappa, rho, G, Ke, Me);
    ora_dofmap(pt, &e, 1, dof);
    for (int a = 0; a < N; ++a) {
      double sK = 0.0, sM = 0.0;
      for (int b = 0; b < N; ++b) {
        if (Ke) sK += Ke[(size_t)a * N + b] * x[dof[b]];
        if (Me) sM += Me[(size_t)a * N + b] * x[dof[b]];
      }
      if (yK) yK[dof[a]] += sK;
      if (yM) yM[dof[a]] += sM;
    }
  }
  free(ones); free(Ke); free(Me); free(dof);
  free_layout(&L);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Weighted quadrature for the mass matrix (Sec. 1.2 names it; the rule is   */
/* defined in iga_oracle.h).                                                 */
/* ------------------------------------------------------------------------ */

/* B_{i;p}(x) with the right end of the domain included: an open knot vector
 * makes the last function 1 there and every other one 0 (the half-open
 * recursion alone would give 0 for all). */
static double wq_bspline(const double* t, int m, int i, int p, double x) {
  if (x >= t[m - 1]) return (i == m - p - 2) ? 1.0 : 0.0;
  return ora_bspline(t, i, p, x);
}

/* B'_{i;p}(x), the right end of the domain taken as the left limit: there
 * the degree p-1 function of the last non-empty span is 1 and every other one
 * 0, so the derivative formula (de Boor) reduces to its two end terms. */
static double wq_bspline_deriv(const double* t, int m, int i, int p, double x) {
  if (x < t[m - 1]) return ora_bspline_deriv(t, i, p, x);
  const int s = m - p - 2;   /* last non-empty span */
  double d = 0.0;
  if (i == s && t[i + p] > t[i]) d += (double)p / (t[i + p] - t[i]);
  if (i + 1 == s && t[i + p + 1] > t[i + 1]) d -= (double)p / (t[i + p + 1] - t[i + 1]);
  return d;
}

int ora_wq_points(const double* t, int m, int p, double* x, int cap) {
  if (!t || !x || m < 2 * p + 2 || p < 1) return -1;
  int* sp = (int*)malloc(sizeof(int) * (size_t)m);
  const int K = ora_spans(t, m, p, sp);
  int n = 0;
  for (int e = 0; e < K; ++e) {
    const double a = t[sp[e]], b = t[sp[e] + 1];
    if (n >= cap) { free(sp); return -1; }
    x[n++] = a;
    if (e < p || e >= K - p) {
      for (int r = 1; r <= p; ++r) {
        if (n >= cap) { free(sp); return -1; }
        x[n++] = a + (b - a) * (double)r / (double)(p + 1);
      }
    } else {
      if (n >= cap) { free(sp); return -1; }
      x[n++] = 0.5 * (a + b);
    }
  }
  if (n >= cap) { free(sp); return -1; }
  x[n++] = t[sp[K - 1] + 1];
  free(sp);
  return n;
}

/* Solve the dense system G y = r (n x n, row-major, overwritten) by Gaussian
 * elimination with partial pivoting.  Returns 0, or -1 if a pivot vanishes. */
static int wq_solve(double* G, double* r, int n) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(G[i * n + k]) > fabs(G[piv * n + k])) piv = i;
    if (!(fabs(G[piv * n + k]) > 0.0)) return -1;
    if (piv != k) {
      for (int j = 0; j < n; ++j) { double tmp = G[k * n + j]; G[k * n + j] = G[piv * n + j]; G[piv * n + j] = tmp; }
      double tmp = r[k]; r[k] = r[piv]; r[piv] = tmp;
    }
    for (int i = k + 1; i < n; ++i) {
      const double f = G[i * n + k] / G[k * n + k];
      for (int j = k; j < n; ++j) G[i * n + j] -= f * G[k * n + j];
      r[i] -= f * r[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = r[k];
    for (int j = k + 1; j < n; ++j) s -= G[k * n + j] * r[j];
    r[k] = s / G[k * n + k];
  }
  return 0;
}

/* The rule of every test function; der = 0: exact against the values of the
 * trial functions with the test function's value (the mass rule), der = 1:
 * exact against the trial derivatives with the test derivative.  The
 * derivatives sum to zero on every support (the B_j sum to 1), so with
 * der = 1 the system has exactly one dependent equation and a consistent
 * right-hand side; the last equation is dropped, which leaves the solution
 * set, and so its least-norm member, unchanged. */
static int wq_weights_impl(const double* t, int m, int p, const double* x, int np, double* W,
                           int der) {
  if (!t || !x || !W || np < 1 || (der && p < 2)) return -1;
  const int nf = m - p - 1;
  double gx[64], gw[64];
  if (ora_gauss_legendre(p + 1, gx, gw)) return -1;
  int* sp = (int*)malloc(sizeof(int) * (size_t)m);
  const int K = ora_spans(t, m, p, sp);
  const int cap = 2 * p + 1;
  double* A = (double*)malloc(sizeof(double) * (size_t)cap * np);
  double* G = (double*)malloc(sizeof(double) * (size_t)cap * cap);
  double* r = (double*)malloc(sizeof(double) * (size_t)cap);
  int js[64];
  int rc = 0;
  for (int i = 0; i < nf * np; ++i) W[i] = 0.0;
  for (int i = 0; i < nf && rc == 0; ++i) {
    const double lo = t[i], hi = t[i + p + 1];
    /* points in the closed support */
    int qlo = 0;
    while (qlo < np && x[qlo] < lo) ++qlo;
    int qhi = qlo;
    while (qhi < np && x[qhi] <= hi) ++qhi;
    const int nq = qhi - qlo;
    /* test-trial pairs with a support overlap of positive length */
    int nj = 0;
    for (int j = 0; j < nf; ++j) {
      const double olo = t[i] > t[j] ? t[i] : t[j];
      const double ohi = t[i + p + 1] < t[j + p + 1] ? t[i + p + 1] : t[j + p + 1];
      if (ohi > olo && nj < 64) js[nj++] = j;
    }
    const int ns = der ? nj - 1 : nj;   /* equations kept */
    if (nj > cap || nq < ns) { rc = -1; break; }
    for (int a = 0; a < nj; ++a) {
      for (int q = 0; q < nq; ++q)
        A[a * nq + q] = der ? wq_bspline_deriv(t, m, js[a], p, x[qlo + q])
                            : wq_bspline(t, m, js[a], p, x[qlo + q]);
      /* exact int B_i B_j (or B'_i B'_j): Gauss with p + 1 points on every element */
      double s = 0.0;
      for (int e = 0; e < K; ++e) {
        const double ea = t[sp[e]], eb = t[sp[e] + 1];
        if (eb <= lo || ea >= hi) continue;
        for (int g = 0; g < p + 1; ++g) {
          const double xi = 0.5 * (ea + eb) + 0.5 * (eb - ea) * gx[g];
          s += der ? 0.5 * (eb - ea) * gw[g] * ora_bspline_deriv(t, i, p, xi) *
                         ora_bspline_deriv(t, js[a], p, xi)
                   : 0.5 * (eb - ea) * gw[g] * ora_bspline(t, i, p, xi) * ora_bspline(t, js[a], p, xi);
        }
      }
      r[a] = s;
    }
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < ns; ++b) {
        double s = 0.0;
        for (int q = 0; q < nq; ++q) s += A[a * nq + q] * A[b * nq + q];
        G[a * ns + b] = s;
      }
    if (wq_solve(G, r, ns)) { rc = -1; break; }
    for (int q = 0; q < nq; ++q) {
      double s = 0.0;
      for (int a = 0; a < ns; ++a) s += A[a * nq + q] * r[a];
      W[(size_t)i * np + qlo + q] = s;
    }
  }
  free(sp); free(A); free(G); free(r);
  return rc;
}

int ora_wq_weights(const double* t, int m, int p, const double* x, int np, double* W) {
  return wq_weights_impl(t, m, p, x, np, W, 0);
}

int ora_wq_weights_deriv(const double* t, int m, int p, const double* x, int np, double* W) {
  return wq_weights_impl(t, m, p, x, np, W, 1);
}

int ora_wq_mass(const ora_patch* pt, const double* c, const int64_t* row_ptr,
                const int32_t* col_idx, double* values) {
  layout L;
  if (!row_ptr || !col_idx || !values || make_layout(pt, &L) || !same_degree(&L)) {
    free_layout(&L);
    return -1;
  }
  const int d = L.d, p = L.p[0];
  double* x[3] = {NULL, NULL, NULL};
  double* W[3] = {NULL, NULL, NULL};
  double* Bv[3] = {NULL, NULL, NULL};
  int np[3] = {1, 1, 1}, nf[3] = {1, 1, 1};
  int rc = 0;
  for (int k = 0; k < d && rc == 0; ++k) {
    const int m = pt->m[k];
    nf[k] = m - p - 1;
    const int cap = 4 * m + 8;
    x[k] = (double*)malloc(sizeof(double) * (size_t)cap);
    np[k] = ora_wq_points(pt->t[k], m, p, x[k], cap);
    if (np[k] < 1) { rc = -1; break; }
    W[k] = (double*)malloc(sizeof(double) * (size_t)nf[k] * np[k]);
    Bv[k] = (double*)malloc(sizeof(double) * (size_t)nf[k] * np[k]);
    if (ora_wq_weights(pt->t[k], m, p, x[k], np[k], W[k])) { rc = -1; break; }
    for (int j = 0; j < nf[k]; ++j)
      for (int q = 0; q < np[k]; ++q) Bv[k][(size_t)j * np[k] + q] = wq_bspline(pt->t[k], m, j, p, x[k][q]);
  }
  if (rc == 0) {
    const int64_t nd = (int64_t)nf[0] * nf[1] * nf[2];
    for (int64_t i = 0; i < nd; ++i) {
      const int i1 = (int)(i % nf[0]), i2 = (int)((i / nf[0]) % nf[1]), i3 = (int)(i / ((int64_t)nf[0] * nf[1]));
      for (int64_t z = row_ptr[i]; z < row_ptr[i + 1]; ++z) {
        const int64_t j = col_idx[z];
        const int j1 = (int)(j % nf[0]), j2 = (int)((j / nf[0]) % nf[1]), j3 = (int)(j / ((int64_t)nf[0] * nf[1]));
        double s = 0.0;
        for (int q3 = 0; q3 < np[2]; ++q3) {
          const double f3 = (d == 3) ? W[2][(size_t)i3 * np[2] + q3] * Bv[2][(size_t)j3 * np[2] + q3] : 1.0;
          if (f3 == 0.0) continue;
          for (int q2 = 0; q2 < np[1]; ++q2) {
            const double f2 = W[1][(size_t)i2 * np[1] + q2] * Bv[1][(size_t)j2 * np[1] + q2];
            if (f2 == 0.0) continue;
            for (int q1 = 0; q1 < np[0]; ++q1) {
              const double f1 = W[0][(size_t)i1 * np[0] + q1] * Bv[0][(size_t)j1 * np[0] + q1];
              if (f1 == 0.0) continue;
              const double cq = c ? c[q1 + (int64_t)np[0] * (q2 + (int64_t)np[1] * q3)] : 1.0;
              s += f1 * f2 * f3 * cq;
            }
          }
        }
        values[z] = s;
      }
    }
  }
  for (int k = 0; k < 3; ++k) { free(x[k]); free(W[k]); free(Bv[k]); }
  free_layout(&L);
  return rc;
}

int ora_wq_stiffness(const ora_patch* pt, const double* c, const int64_t* row_ptr,
                     const int32_t* col_idx, double* values) {
  layout L;
  if (!row_ptr || !col_idx || !values || make_layout(pt, &L) || !same_degree(&L)) {
    free_layout(&L);
    return -1;
  }
  const int d = L.d, p = L.p[0];
  /* per direction: R[0] mass rule, R[1] derivative rule; B[0] values, B[1] derivatives */
  double* x[3] = {NULL, NULL, NULL};
  double* R[3][2] = {{NULL, NULL}, {NULL, NULL}, {NULL, NULL}};
  double* B[3][2] = {{NULL, NULL}, {NULL, NULL}, {NULL, NULL}};
  int np[3] = {1, 1, 1}, nf[3] = {1, 1, 1};
  int rc = p < 2 ? -1 : 0;
  for (int k = 0; k < d && rc == 0; ++k) {
    const int m = pt->m[k];
    nf[k] = m - p - 1;
    const int cap = 4 * m + 8;
    x[k] = (double*)malloc(sizeof(double) * (size_t)cap);
    np[k] = ora_wq_points(pt->t[k], m, p, x[k], cap);
    if (np[k] < 1) { rc = -1; break; }
    for (int v = 0; v < 2; ++v) {
      R[k][v] = (double*)malloc(sizeof(double) * (size_t)nf[k] * np[k]);
      B[k][v] = (double*)malloc(sizeof(double) * (size_t)nf[k] * np[k]);
    }
    if (ora_wq_weights(pt->t[k], m, p, x[k], np[k], R[k][0]) ||
        ora_wq_weights_deriv(pt->t[k], m, p, x[k], np[k], R[k][1])) { rc = -1; break; }
    for (int j = 0; j < nf[k]; ++j)
      for (int q = 0; q < np[k]; ++q) {
        B[k][0][(size_t)j * np[k] + q] = wq_bspline(pt->t[k], m, j, p, x[k][q]);
        B[k][1][(size_t)j * np[k] + q] = wq_bspline_deriv(pt->t[k], m, j, p, x[k][q]);
      }
  }
  if (rc == 0) {
    const int64_t nd = (int64_t)nf[0] * nf[1] * nf[2];
    for (int64_t i = 0; i < nd; ++i) {
      const int i1 = (int)(i % nf[0]), i2 = (int)((i / nf[0]) % nf[1]), i3 = (int)(i / ((int64_t)nf[0] * nf[1]));
      for (int64_t z = row_ptr[i]; z < row_ptr[i + 1]; ++z) {
        const int64_t j = col_idx[z];
        const int j1 = (int)(j % nf[0]), j2 = (int)((j / nf[0]) % nf[1]), j3 = (int)(j / ((int64_t)nf[0] * nf[1]));
        double s = 0.0;
        /* term k: derivatives in direction k, values in the others */
        for (int k = 0; k < d; ++k) {
          const int v1 = k == 0, v2 = k == 1, v3 = k == 2;
          for (int q3 = 0; q3 < np[2]; ++q3) {
            const double f3 = (d == 3) ? R[2][v3][(size_t)i3 * np[2] + q3] * B[2][v3][(size_t)j3 * np[2] + q3] : 1.0;
            if (f3 == 0.0) continue;
            for (int q2 = 0; q2 < np[1]; ++q2) {
              const double f2 = R[1][v2][(size_t)i2 * np[1] + q2] * B[1][v2][(size_t)j2 * np[1] + q2];
              if (f2 == 0.0) continue;
              for (int q1 = 0; q1 < np[0]; ++q1) {
                const double f1 = R[0][v1][(size_t)i1 * np[0] + q1] * B[0][v1][(size_t)j1 * np[0] + q1];
                if (f1 == 0.0) continue;
                const double cq = c ? c[q1 + (int64_t)np[0] * (q2 + (int64_t)np[1] * q3)] : 1.0;
                s += f1 * f2 * f3 * cq;
              }
            }
          }
        }
        values[z] = s;
      }
    }
  }
  for (int k = 0; k < 3; ++k) {
    free(x[k]);
    for (int v = 0; v < 2; ++v) { free(R[k][v]); free(B[k][v]); }
  }
  free_layout(&L);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Backward of the element matrices with respect to kappa and rho.           */
/* ------------------------------------------------------------------------ */
int ora_integrate_grad(const ora_patch* pt, const int64_t* elems, int64_t n_sel, const double* G,
                       const double* GK, const double* GM, double* gk, double* gr) {
  layout L;
  if ((!GK && !GM) || (GK && !gk) || (GM && !gr) || make_layout(pt, &L)) { free_layout(&L); return -1; }
  const int d = L.d, N = L.N, Q = L.Q;
  const int64_t E = n_elements(&L);
  elem1d* B = (elem1d*)malloc(sizeof(elem1d));
  double* W = (double*)malloc(sizeof(double) * Q);
  double* Ginv = (double*)malloc(sizeof(double) * Q * 9);
  double* phi = (double*)malloc(sizeof(double) * (size_t)N);
  double* grad = (double*)malloc(sizeof(double) * (size_t)N * 3);
  int rc = 0;
  for (int64_t s = 0; s < n_sel && rc == 0; ++s) {
    const int64_t e = elems[s];
    if (e < 0 || e >= E) { rc = -1; break; }
    int ek[3];
    split_elem(&L, e, ek);
    element_1d(pt, &L, ek, B);
    element_geometry(&L, e, B, G, W, Ginv);
    for (int k = 0; k < Q; ++k) {
      int kk[3];
      split_qp(&L, k, kk);
      const double* Gi = Ginv + (size_t)k * d * d;
      for (int a = 0; a < N; ++a) {
        int aa[3];
        split_local(&L, a, aa);
        double v = 1.0, gref[3];
        for (int j = 0; j < d; ++j) v *= B1D(B, &L, j, 0, aa[j], kk[j]);
        for (int i = 0; i < d; ++i) {
          double g = 1.0;
          for (int j = 0; j < d; ++j) g *= B1D(B, &L, j, i == j, aa[j], kk[j]);
          gref[i] = g;
        }
        phi[a] = v;
        for (int i = 0; i < d; ++i) {
          double s2 = 0.0;
          for (int j = 0; j < d; ++j) s2 += Gi[j * d + i] * gref[j];
          grad[(size_t)a * 3 + i] = s2;
        }
      }
      double sk = 0.0, sm = 0.0;
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
          if (GK) {
            double dot = 0.0;
            for (int i = 0; i < d; ++i) dot += grad[(size_t)a * 3 + i] * grad[(size_t)b * 3 + i];
            sk += GK[((size_t)s * N + a) * N + b] * dot;
          }
          if (GM) sm += GM[((size_t)s * N + a) * N + b] * phi[a] * phi[b];
        }
      if (GK) gk[(size_t)s * Q + k] = W[k] * sk;
      if (GM) gr[(size_t)s * Q + k] = W[k] * sm;
    }
  }
  free(B); free(W); free(Ginv); free(phi); free(grad);
  free_layout(&L);
  return rc;
}
