// k_apply.cu -- matrix-free operator application y = alpha K(kappa) x +
// beta M(rho) x, 3D and (k_apply2, below) 2D (the products K u and M u of the forward-Euler step of
// Sec. 2.2, eq. Euler; no global matrix and no element matrix is formed).
//
// Per element (one CTA): gather x_e through the dof map, interpolate the
// reference gradient and the value of x at every quadrature point by sum
// factorization (contract a1, then a2, then a3: the one-direction-at-a-time
// order of Algorithm 2, Sec. 3.2), form the reference flux
//   f = alpha w kappa |det G| G^{-1} G^{-T} grad x,   m = beta w rho |det G| x,
// and integrate it back against the test functions with the transposed
// contractions (q3, then q2, then q1):
//   y_e[a] = sum_q (d1 phi_a f_1 + d2 phi_a f_2 + d3 phi_a f_3 + phi_a m).
// The element result goes to scratch[a * E + e]; k_apply_gather then sums the
// contributions of every dof in ascending element order (deterministic, no
// atomics).  T = double is FP64 throughout; T = float keeps the Jacobian
// cofactors and determinant in FP64 and the rest in FP32; T = ff (FP64_DF
// plans) is float-float on the FP32 pipes with double inputs and results.
#include "ff.cuh"
#include "iga_internal.h"

namespace iga {
namespace {

template <typename T, int P, int QG>
struct APL {
  static constexpr int n = P + 1, q = QG, Q = q * q * q, n2 = n * n, N = n2 * n;
  static constexpr int NT = 128;
  static constexpr int REC = 2 * q * n + q;
};

template <typename T, int P, int QG, bool GEN>
__global__ void __launch_bounds__(128) k_apply3(const ApplyArgs A) {
  using C = APL<T, P, QG>;
  constexpr int n = C::n, q = C::q, Q = C::Q, n2 = C::n2, N = C::N, NT = C::NT, REC = C::REC;
  __shared__ double rec[3 * REC];
  __shared__ T tb[3][2][q * n];          // [direction][value, derivative][q][n]
  __shared__ T xe[N];
  __shared__ T U1[2][n2 * q];            // [x factor][a2 + n a3][q1]
  __shared__ T U2[3][n * q * q];         // [vv, dv, vd][a3][q1 + q q2]
  __shared__ T F[4][Q];                  // f1, f2, f3, m at every quadrature point
  __shared__ T R[3][n * q * q];          // [a3][q1 + q q2]: z-contracted f1, f2, f3 + m
  __shared__ T S[2][n2 * q];             // [a2 + n a3][q1]: pairs with d_x, with v_x
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  int e1, e2, e3;
  elem_coords(A, e, e1, e2, e3);
  for (int i = tid; i < 3 * REC; i += NT) {
    const int d = i / REC, j = i - d * REC;
    const int ek = d == 0 ? e1 : (d == 1 ? e2 : e3);
    rec[i] = A.tab[d][(int64_t)ek * REC + j];
  }
  const int s1 = A.span[0][e1] - P, s2 = A.span[1][e2] - P, s3 = A.span[2][e3] - P;
  for (int a = tid; a < N; a += NT) {
    const int a1 = a % n, a2 = (a / n) % n, a3 = a / n2;
    const int64_t g =
        A.dof_offset + (s1 + a1) + (int64_t)A.nf0 * ((s2 + a2) + (int64_t)A.nf1 * (s3 + a3));
    xe[a] = to_compute<T>(((const store_t<T>*)A.x)[g]);
  }
  __syncthreads();
  for (int i = tid; i < 3 * 2 * q * n; i += NT) {
    const int d = i / (2 * q * n), j = i % (2 * q * n);
    (&tb[0][0][0])[i] = from_double<T>(rec[d * REC + j]);
  }
  __syncthreads();
  // interpolation, a1: U1[s][a23][q1] = sum_a1 x[a1, a23] B^s_x(q1)[a1]
  for (int it = tid; it < 2 * n2 * q; it += NT) {
    const int s = it / (n2 * q), r = it % (n2 * q), a23 = r / q, q1 = r % q;
    const T* B = &tb[0][s][q1 * n];
    T acc = 0;
#pragma unroll
    for (int a1 = 0; a1 < n; ++a1) mac(acc, xe[a1 + n * a23], B[a1]);
    U1[s][r] = fin(acc);
  }
  __syncthreads();
  // a2: U2[c][a3][q1 q2], c = vv (x value, y value), dv (x der), vd (y der)
  for (int it = tid; it < 3 * n * q * q; it += NT) {
    const int c = it / (n * q * q), r = it % (n * q * q), a3 = r / (q * q), qq = r % (q * q);
    const int q1 = qq % q, q2 = qq / q;
    const T* U = U1[c == 1 ? 1 : 0];
    const T* B = &tb[1][c == 2 ? 1 : 0][q2 * n];
    T acc = 0;
#pragma unroll
    for (int a2 = 0; a2 < n; ++a2) mac(acc, U[(a2 + n * a3) * q + q1], B[a2]);
    U2[c][r] = fin(acc);
  }
  __syncthreads();
  // a3 at every quadrature point, then the flux
  for (int k = tid; k < Q; k += NT) {
    const int qq = k % (q * q), q3 = k / (q * q);
    const int q1 = qq % q, q2 = qq / q;
    T g0 = 0, g1 = 0, g2 = 0, u = 0;
#pragma unroll
    for (int a3 = 0; a3 < n; ++a3) {
      const T vz = tb[2][0][q3 * n + a3], dz = tb[2][1][q3 * n + a3];
      const int o = a3 * q * q + qq;
      mac(g0, U2[1][o], vz);
      mac(g1, U2[2][o], vz);
      mac(g2, U2[0][o], dz);
      mac(u, U2[0][o], vz);
    }
    g0 = fin(g0);
    g1 = fin(g1);
    g2 = fin(g2);
    u = fin(u);
    const double wq = rec[2 * q * n + q1] * rec[REC + 2 * q * n + q2] * rec[2 * REC + 2 * q * n + q3];
    const double kap = A.kappa ? A.kappa[e * Q + k] : 1.0;
    const double rh = A.rho ? A.rho[e * Q + k] : 1.0;
    T f0, f1, f2, m;
    if (GEN) {
      // G^{-T} = c / det with c the cofactor matrix; reference flux
      // f = (w kappa / |det|) c^T (c g), mass weight w rho |det|
      const double* G = A.jac + (e * Q + k) * 9;
      const double g00 = G[0], g01 = G[1], g02 = G[2], g10 = G[3], g11 = G[4], g12 = G[5],
                   g20 = G[6], g21 = G[7], g22 = G[8];
      const double c00 = g11 * g22 - g12 * g21, c01 = g12 * g20 - g10 * g22, c02 = g10 * g21 - g11 * g20;
      const double c10 = g02 * g21 - g01 * g22, c11 = g00 * g22 - g02 * g20, c12 = g01 * g20 - g00 * g21;
      const double c20 = g01 * g12 - g02 * g11, c21 = g02 * g10 - g00 * g12, c22 = g00 * g11 - g01 * g10;
      const double det = g00 * c00 + g01 * c01 + g02 * c02;
      const double adet = fabs(det);
      const T sK = from_double<T>(A.alpha * wq * kap / adet);
      const T C00 = from_double<T>(c00), C01 = from_double<T>(c01), C02 = from_double<T>(c02);
      const T C10 = from_double<T>(c10), C11 = from_double<T>(c11), C12 = from_double<T>(c12);
      const T C20 = from_double<T>(c20), C21 = from_double<T>(c21), C22 = from_double<T>(c22);
      const T h0 = C00 * g0 + C01 * g1 + C02 * g2;
      const T h1 = C10 * g0 + C11 * g1 + C12 * g2;
      const T h2 = C20 * g0 + C21 * g1 + C22 * g2;
      f0 = sK * (C00 * h0 + C10 * h1 + C20 * h2);
      f1 = sK * (C01 * h0 + C11 * h1 + C21 * h2);
      f2 = sK * (C02 * h0 + C12 * h1 + C22 * h2);
      m = from_double<T>(A.beta * wq * adet * rh) * u;
    } else {
      const T sK = from_double<T>(A.alpha * wq * kap);
      f0 = sK * g0;
      f1 = sK * g1;
      f2 = sK * g2;
      m = from_double<T>(A.beta * wq * rh) * u;
    }
    F[0][k] = f0;
    F[1][k] = f1;
    F[2][k] = f2;
    F[3][k] = m;
  }
  __syncthreads();
  // test side, q3: R0 = sum v_z f1, R1 = sum v_z f2, R2 = sum (d_z f3 + v_z m)
  for (int it = tid; it < 3 * n * q * q; it += NT) {
    const int c = it / (n * q * q), r = it % (n * q * q), a3 = r / (q * q), qq = r % (q * q);
    T acc = 0;
#pragma unroll
    for (int q3 = 0; q3 < q; ++q3) {
      const T vz = tb[2][0][q3 * n + a3];
      const int k = qq + q * q * q3;
      if (c == 0) mac(acc, vz, F[0][k]);
      else if (c == 1) mac(acc, vz, F[1][k]);
      else {
        mac(acc, tb[2][1][q3 * n + a3], F[2][k]);
        mac(acc, vz, F[3][k]);
      }
    }
    R[c][r] = fin(acc);
  }
  __syncthreads();
  // q2: S0 = sum v_y R0 (pairs with d_x), S1 = sum (d_y R1 + v_y R2) (pairs with v_x)
  for (int it = tid; it < 2 * n2 * q; it += NT) {
    const int c = it / (n2 * q), r = it % (n2 * q), a23 = r / q, q1 = r % q;
    const int a2 = a23 % n, a3 = a23 / n;
    T acc = 0;
#pragma unroll
    for (int q2 = 0; q2 < q; ++q2) {
      const T vy = tb[1][0][q2 * n + a2];
      const int o = a3 * q * q + q1 + q * q2;
      if (c == 0) mac(acc, vy, R[0][o]);
      else {
        mac(acc, tb[1][1][q2 * n + a2], R[1][o]);
        mac(acc, vy, R[2][o]);
      }
    }
    S[c][r] = fin(acc);
  }
  __syncthreads();
  // q1: y[a] = sum (d_x S0 + v_x S1); one value per local function
  store_t<T>* out = (store_t<T>*)A.scratch;
  for (int a = tid; a < N; a += NT) {
    const int a1 = a % n, a23 = a / n;
    T acc = 0;
#pragma unroll
    for (int q1 = 0; q1 < q; ++q1) {
      mac(acc, tb[0][1][q1 * n + a1], S[0][a23 * q + q1]);
      mac(acc, tb[0][0][q1 * n + a1], S[1][a23 * q + q1]);
    }
    out[(int64_t)a * A.n_elem + e] = to_store<T>(fin(acc));
  }
}

// 2D (FP64 plans): the same steps with two directions.  Interpolation
// U[s][a2][q1] = sum_a1 x[a1 + n a2] B^s_x(q1)[a1] (value and derivative), at
// every point g0 = d_x x, g1 = d_y x, u = x; flux f = alpha w kappa |det G|
// G^{-1} G^{-T} g through the 2x2 cofactors, m = beta w rho |det G| u; back:
// S0[a2][q1] = sum_q2 v_y f0, S1[a2][q1] = sum_q2 (d_y f1 + v_y m),
// y_e[a1 + n a2] = sum_q1 (d_x S0 + v_x S1).
template <typename T, int P, int QG, bool GEN>
__global__ void __launch_bounds__(64) k_apply2(const ApplyArgs A) {
  constexpr int n = P + 1, q = QG, N = n * n, Q = q * q, NT = 64, REC = 2 * q * n + q;
  __shared__ double rec[2 * REC];
  __shared__ T tb[2][2][q * n];          // [direction][value, derivative][q][n]
  __shared__ T xe[N];
  __shared__ T U[2][n * q];              // [value, derivative in x][a2][q1]
  __shared__ T F[3][Q];                  // f0, f1, m at every quadrature point
  __shared__ T S[2][n * q];              // [a2][q1]: pairs with d_x, with v_x
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  int e1, e2;
  elem_coords2(A, e, e1, e2);
  for (int i = tid; i < 2 * REC; i += NT) {
    const int d = i / REC, j = i - d * REC;
    rec[i] = (d == 0 ? A.tab[0] + (int64_t)e1 * REC : A.tab[1] + (int64_t)e2 * REC)[j];
  }
  const int s1 = A.span[0][e1] - P, s2 = A.span[1][e2] - P;
  for (int a = tid; a < N; a += NT) {
    const int64_t g = A.dof_offset + (s1 + a % n) + (int64_t)A.nf0 * (s2 + a / n);
    xe[a] = to_compute<T>(((const store_t<T>*)A.x)[g]);
  }
  __syncthreads();
  for (int i = tid; i < 2 * 2 * q * n; i += NT) {
    const int d = i / (2 * q * n), j = i % (2 * q * n);
    (&tb[0][0][0])[i] = from_double<T>(rec[d * REC + j]);
  }
  __syncthreads();
  for (int it = tid; it < 2 * n * q; it += NT) {
    const int sd = it / (n * q), r = it % (n * q), a2 = r / q, q1 = r % q;
    const T* B = &tb[0][sd][q1 * n];
    T acc = 0;
#pragma unroll
    for (int a1 = 0; a1 < n; ++a1) mac(acc, xe[a1 + n * a2], B[a1]);
    U[sd][r] = fin(acc);
  }
  __syncthreads();
  for (int k = tid; k < Q; k += NT) {
    const int q1 = k % q, q2 = k / q;
    T g0 = 0, g1 = 0, u = 0;
#pragma unroll
    for (int a2 = 0; a2 < n; ++a2) {
      const T vy = tb[1][0][q2 * n + a2], dy = tb[1][1][q2 * n + a2];
      mac(g0, U[1][a2 * q + q1], vy);
      mac(g1, U[0][a2 * q + q1], dy);
      mac(u, U[0][a2 * q + q1], vy);
    }
    g0 = fin(g0);
    g1 = fin(g1);
    u = fin(u);
    const double wq = rec[2 * q * n + q1] * rec[REC + 2 * q * n + q2];
    const double kap = A.kappa ? A.kappa[e * Q + k] : 1.0;
    const double rh = A.rho ? A.rho[e * Q + k] : 1.0;
    if (GEN) {
      // cofactors c = [[g11, -g10], [-g01, g00]]: G^{-T} = c / det; reference
      // flux f = (w kappa / |det|) c^T (c g), mass weight w rho |det|
      const double* G = A.jac + (e * Q + k) * 4;
      const double g00 = G[0], g01 = G[1], g10 = G[2], g11 = G[3];
      const double adet = fabs(g00 * g11 - g01 * g10);
      const T c00 = from_double<T>(g11), c01 = from_double<T>(-g10);
      const T c10 = from_double<T>(-g01), c11 = from_double<T>(g00);
      const T sK = from_double<T>(A.alpha * wq * kap / adet);
      const T h0 = c00 * g0 + c01 * g1, h1 = c10 * g0 + c11 * g1;
      F[0][k] = sK * (c00 * h0 + c10 * h1);
      F[1][k] = sK * (c01 * h0 + c11 * h1);
      F[2][k] = from_double<T>(A.beta * wq * adet * rh) * u;
    } else {
      const T sK = from_double<T>(A.alpha * wq * kap);
      F[0][k] = sK * g0;
      F[1][k] = sK * g1;
      F[2][k] = from_double<T>(A.beta * wq * rh) * u;
    }
  }
  __syncthreads();
  for (int it = tid; it < 2 * n * q; it += NT) {
    const int c = it / (n * q), r = it % (n * q), a2 = r / q, q1 = r % q;
    T acc = 0;
#pragma unroll
    for (int q2 = 0; q2 < q; ++q2) {
      const T vy = tb[1][0][q2 * n + a2];
      const int k = q1 + q * q2;
      if (c == 0) {
        mac(acc, vy, F[0][k]);
      } else {
        mac(acc, tb[1][1][q2 * n + a2], F[1][k]);
        mac(acc, vy, F[2][k]);
      }
    }
    S[c][r] = fin(acc);
  }
  __syncthreads();
  store_t<T>* out = (store_t<T>*)A.scratch;
  for (int a = tid; a < N; a += NT) {
    const int a1 = a % n, a2 = a / n;
    T acc = 0;
#pragma unroll
    for (int q1 = 0; q1 < q; ++q1) {
      mac(acc, tb[0][1][q1 * n + a1], S[0][a2 * q + q1]);
      mac(acc, tb[0][0][q1 * n + a1], S[1][a2 * q + q1]);
    }
    out[(int64_t)a * A.n_elem + e] = to_store<T>(fin(acc));
  }
}

template <int P, int QG>
cudaError_t run2(const ApplyArgs& a, cudaStream_t st) {
  if (a.jac) k_apply2<double, P, QG, true><<<(unsigned)a.n_elem, 64, 0, st>>>(a);
  else k_apply2<double, P, QG, false><<<(unsigned)a.n_elem, 64, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t dispatch2(const ApplyArgs& a, int p, int q, cudaStream_t st) {
  const int dq = q - p;
#define C2(PP)                                                \
  if (p == PP && dq == 1) return run2<PP, PP + 1>(a, st);     \
  if (p == PP && dq == 2) return run2<PP, PP + 2>(a, st);
  C2(1) C2(2) C2(3) C2(4) C2(5)
#undef C2
  return cudaErrorInvalidValue;
}

template <typename T, int P, int QG>
cudaError_t run(const ApplyArgs& a, cudaStream_t st) {
  if (a.jac) k_apply3<T, P, QG, true><<<(unsigned)a.n_elem, 128, 0, st>>>(a);
  else k_apply3<T, P, QG, false><<<(unsigned)a.n_elem, 128, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(const ApplyArgs& a, int p, int q, cudaStream_t st) {
  const int dq = q - p;
#define C3(PP)                                               \
  if (p == PP && dq == 1) return run<T, PP, PP + 1>(a, st);  \
  if (p == PP && dq == 2) return run<T, PP, PP + 2>(a, st);
  C3(1) C3(2) C3(3) C3(4)
  if (p == 5 && dq == 1) return run<T, 5, 6>(a, st);
#undef C3
  return cudaErrorInvalidValue;
}

}  // namespace

bool apply_supported(int dim, int p, int q) {
  if (dim == 2) return p >= 1 && p <= 5 && (q == p + 1 || q == p + 2);
  return dim == 3 && p >= 1 && p <= 5 && (q == p + 1 || (q == p + 2 && p <= 4));
}

cudaError_t launch_apply(const ApplyArgs& a, int dim, int p, int q, bool fp64, bool df,
                         cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  if (dim == 2) return fp64 ? dispatch2(a, p, q, st) : cudaErrorInvalidValue;
  if (df) return dispatch<ff>(a, p, q, st);
  return fp64 ? dispatch<double>(a, p, q, st) : dispatch<float>(a, p, q, st);
}

}  // namespace iga
