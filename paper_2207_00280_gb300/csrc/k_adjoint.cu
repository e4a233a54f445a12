// k_adjoint.cu -- matrix-free adjoint of J(kappa) = u^T K(kappa) v, 3D and 2D (not
// in the paper; it differentiates the stiffness of the weak form, Sec. 2.2).
//
// J is linear in kappa:  J = sum_q kappa_q g_q  with
//   g_q = w_q |det G_q| (G_q^{-T} grad u)(x_q) . (G_q^{-T} grad v)(x_q),
// so dJ/dkappa_q = g_q.  No element matrix is formed: per element, u and v
// are gathered through the dof map and their reference gradients at every
// quadrature point are interpolated by sum factorization from the 1D basis
// tables (contract a1 against x factors, then a2, then a3), the same
// one-direction-at-a-time order as Algorithm 2 of Sec. 3.2.
// J is reduced deterministically: a fixed-order per-element sum written to
// scratch (one double per element), then one block sums the scratch array in
// a fixed order.  No floating-point atomics.  T = double (FP64), float (FP32
// with FP64 cofactors and determinant) or ff (float-float on the FP32 pipes
// with double inputs and results, FP64_DF plans).
#include "ff.cuh"
#include "iga_internal.h"

namespace iga {
namespace {

template <typename T, int P, int QG, bool GEN>
struct ADJ {
  static constexpr int n = P + 1, q = QG, Q = q * q * q, n2 = n * n, N = n2 * n;
  static constexpr int NT = (Q + 31) / 32 * 32 < 64 ? 64 : (Q + 31) / 32 * 32;
  static constexpr int REC = 2 * q * n + q;
};

template <typename T, int P, int QG, bool GEN>
__global__ void __launch_bounds__(ADJ<T, P, QG, GEN>::NT) k_adjoint3(const AdjArgs A) {
  using C = ADJ<T, P, QG, GEN>;
  constexpr int n = C::n, q = C::q, Q = C::Q, n2 = C::n2, N = C::N, NT = C::NT, REC = C::REC;
  __shared__ double rec[3 * REC];
  __shared__ T tabT[3 * 2 * q * n];            // [dir][val/der][q][n] in T
  __shared__ T ue[N], ve[N];
  __shared__ T U1[2][2][n2 * q];               // [vec][x factor][a2 a3][q1]
  __shared__ T U2[2][3][n * q * q];            // [vec][vv, dv, vd][a3][q1 q2]
  __shared__ double red[NT / 32];
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  int e1, e2, e3;
  elem_coords(A, e, e1, e2, e3);
  for (int i = tid; i < 3 * REC; i += NT) {
    const int d = i / REC, j = i - d * REC;
    const int ek = d == 0 ? e1 : (d == 1 ? e2 : e3);
    const double* tb = d == 0 ? A.tab[0] : (d == 1 ? A.tab[1] : A.tab[2]);
    rec[i] = tb[(int64_t)ek * REC + j];
  }
  // gather u_e, v_e through the dof map (support set of the element)
  const int s1 = A.span[0][e1] - P, s2 = A.span[1][e2] - P, s3 = A.span[2][e3] - P;
  for (int a = tid; a < N; a += NT) {
    const int a1 = a % n, a2 = (a / n) % n, a3 = a / n2;
    const int64_t g = A.dof_offset + (s1 + a1) + (int64_t)A.nf0 * ((s2 + a2) + (int64_t)A.nf1 * (s3 + a3));
    ue[a] = to_compute<T>(((const store_t<T>*)A.u)[g]);
    ve[a] = to_compute<T>(((const store_t<T>*)A.v)[g]);
  }
  __syncthreads();
  for (int i = tid; i < 3 * 2 * q * n; i += NT) {
    const int d = i / (2 * q * n), j = i % (2 * q * n);
    tabT[i] = from_double<T>(rec[d * REC + j]);
  }
  __syncthreads();
  const T* vx = tabT;               const T* dx = tabT + q * n;
  const T* vy = tabT + 2 * q * n;   const T* dy = vy + q * n;
  const T* vz = tabT + 4 * q * n;   const T* dz = vz + q * n;
  // contract a1: U1[vec][s][a2 + n a3][q1] = sum_a1 u[a1,a2,a3] F^s_x(q1)[a1]
  for (int it = tid; it < 2 * n2 * q; it += NT) {
    const int s = it / (n2 * q), r = it % (n2 * q), a23 = r / q, q1 = r % q;
    const T* F = (s ? dx : vx) + q1 * n;
    T au = 0, av = 0;
#pragma unroll
    for (int a1 = 0; a1 < n; ++a1) {
      mac(au, ue[a1 + n * a23], F[a1]);
      mac(av, ve[a1 + n * a23], F[a1]);
    }
    U1[0][s][a23 * q + q1] = fin(au);
    U1[1][s][a23 * q + q1] = fin(av);
  }
  __syncthreads();
  // contract a2: U2[vec][c][a3][q1 + q q2], c = vv (s=0,t=0), dv (s=1,t=0), vd (s=0,t=1)
  for (int it = tid; it < 3 * n * q * q; it += NT) {
    const int c = it / (n * q * q), r = it % (n * q * q), a3 = r / (q * q), qq = r % (q * q);
    const int q1 = qq % q, q2 = qq / q;
    const int s = (c == 1), t = (c == 2);
    const T* F = (t ? dy : vy) + q2 * n;
    T au = 0, av = 0;
#pragma unroll
    for (int a2 = 0; a2 < n; ++a2) {
      mac(au, U1[0][s][(a2 + n * a3) * q + q1], F[a2]);
      mac(av, U1[1][s][(a2 + n * a3) * q + q1], F[a2]);
    }
    U2[0][c][a3 * q * q + qq] = fin(au);
    U2[1][c][a3 * q * q + qq] = fin(av);
  }
  __syncthreads();
  // contract a3 at every quadrature point, then the geometry and the product
  double part = 0.0;
  for (int k = tid; k < Q; k += NT) {
    const int qq = k % (q * q), q3 = k / (q * q);
    const int q1 = qq % q, q2 = qq / q;
    T gu[3] = {0, 0, 0}, gv[3] = {0, 0, 0};
#pragma unroll
    for (int a3 = 0; a3 < n; ++a3) {
      const T fz = vz[q3 * n + a3], dfz = dz[q3 * n + a3];
      const int o = a3 * q * q + qq;
      mac(gu[0], U2[0][1][o], fz);
      mac(gu[1], U2[0][2][o], fz);
      mac(gu[2], U2[0][0][o], dfz);
      mac(gv[0], U2[1][1][o], fz);
      mac(gv[1], U2[1][2][o], fz);
      mac(gv[2], U2[1][0][o], dfz);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      gu[i] = fin(gu[i]);
      gv[i] = fin(gv[i]);
    }
    const double* w0 = rec + 2 * q * n;
    const double Wd = w0[q1] * (w0 + REC)[q2] * (w0 + 2 * REC)[q3];
    T gq;
    if (GEN) {
      // g = (W / |det|) (c gu) . (c gv),  c = cofactor matrix: G^{-T} = c / det
      const double* G = A.jac + (e * Q + k) * 9;
      const double g00 = G[0], g01 = G[1], g02 = G[2], g10 = G[3], g11 = G[4], g12 = G[5],
                   g20 = G[6], g21 = G[7], g22 = G[8];
      const double d00 = g11 * g22 - g12 * g21, d01 = g12 * g20 - g10 * g22,
                   d02 = g10 * g21 - g11 * g20;
      const double det = g00 * d00 + g01 * d01 + g02 * d02;
      const T c00 = from_double<T>(d00), c01 = from_double<T>(d01), c02 = from_double<T>(d02);
      const T c10 = from_double<T>(g02 * g21 - g01 * g22), c11 = from_double<T>(g00 * g22 - g02 * g20),
              c12 = from_double<T>(g01 * g20 - g00 * g21);
      const T c20 = from_double<T>(g01 * g12 - g02 * g11), c21 = from_double<T>(g02 * g10 - g00 * g12),
              c22 = from_double<T>(g00 * g11 - g01 * g10);
      const T pu0 = c00 * gu[0] + c01 * gu[1] + c02 * gu[2];
      const T pu1 = c10 * gu[0] + c11 * gu[1] + c12 * gu[2];
      const T pu2 = c20 * gu[0] + c21 * gu[1] + c22 * gu[2];
      const T pv0 = c00 * gv[0] + c01 * gv[1] + c02 * gv[2];
      const T pv1 = c10 * gv[0] + c11 * gv[1] + c12 * gv[2];
      const T pv2 = c20 * gv[0] + c21 * gv[1] + c22 * gv[2];
      gq = from_double<T>(Wd / fabs(det)) * (pu0 * pv0 + pu1 * pv1 + pu2 * pv2);
    } else {
      gq = from_double<T>(Wd) * (gu[0] * gv[0] + gu[1] * gv[1] + gu[2] * gv[2]);
    }
    const store_t<T> gs = to_store_int<T>(gq);
    if (A.grad) ((store_t<T>*)A.grad)[e * Q + k] = gs;
    if (A.partial) part += (A.kappa ? A.kappa[e * Q + k] : 1.0) * (double)gs;
  }
  if (A.partial) {
    // fixed-order block reduction: warp tree, then warp 0 over the warp sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red[w];
      A.partial[A.partial_offset + e] = s;
    }
  }
}

// 2D (FP64 plans): u_e and v_e gathered, U[vec][s][a2][q1] = sum_a1 x[a1 + n a2]
// B^s_x(q1)[a1] (value and derivative), at every point the reference
// gradients (d_x: derivative in x with the y value; d_y: value in x with the
// y derivative), g = w (G^{-T} grad u).(G^{-T} grad v) through the 2x2
// cofactors, and the same fixed-order partial of kappa g as in 3D.
template <int P, int QG, bool GEN>
__global__ void __launch_bounds__(64) k_adjoint2(const AdjArgs A) {
  constexpr int n = P + 1, q = QG, N = n * n, Q = q * q, NT = 64, REC = 2 * q * n + q;
  __shared__ double rec[2 * REC];
  __shared__ double ue[N], ve[N];
  __shared__ double U[2][2][n * q];     // [vec][value, derivative in x][a2][q1]
  __shared__ double red[NT / 32];
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
    ue[a] = ((const double*)A.u)[g];
    ve[a] = ((const double*)A.v)[g];
  }
  __syncthreads();
  const double* vx = rec;               const double* dx = rec + q * n;
  const double* vy = rec + REC;         const double* dy = vy + q * n;
  for (int it = tid; it < 2 * n * q; it += NT) {
    const int sd = it / (n * q), r = it % (n * q), a2 = r / q, q1 = r % q;
    const double* F = (sd ? dx : vx) + q1 * n;
    double au = 0.0, av = 0.0;
#pragma unroll
    for (int a1 = 0; a1 < n; ++a1) {
      au = fma(ue[a1 + n * a2], F[a1], au);
      av = fma(ve[a1 + n * a2], F[a1], av);
    }
    U[0][sd][r] = au;
    U[1][sd][r] = av;
  }
  __syncthreads();
  double part = 0.0;
  for (int k = tid; k < Q; k += NT) {
    const int q1 = k % q, q2 = k / q;
    double gu0 = 0.0, gu1 = 0.0, gv0 = 0.0, gv1 = 0.0;
#pragma unroll
    for (int a2 = 0; a2 < n; ++a2) {
      const double fy = vy[q2 * n + a2], dfy = dy[q2 * n + a2];
      gu0 = fma(U[0][1][a2 * q + q1], fy, gu0);
      gu1 = fma(U[0][0][a2 * q + q1], dfy, gu1);
      gv0 = fma(U[1][1][a2 * q + q1], fy, gv0);
      gv1 = fma(U[1][0][a2 * q + q1], dfy, gv1);
    }
    const double W = rec[2 * q * n + q1] * rec[REC + 2 * q * n + q2];
    double gq;
    if (GEN) {
      // g = (W / |det|) (c gu) . (c gv),  c = [[g11, -g10], [-g01, g00]]: G^{-T} = c / det
      const double* G = A.jac + (e * Q + k) * 4;
      const double g00 = G[0], g01 = G[1], g10 = G[2], g11 = G[3];
      const double adet = fabs(g00 * g11 - g01 * g10);
      const double pu0 = g11 * gu0 - g10 * gu1, pu1 = -g01 * gu0 + g00 * gu1;
      const double pv0 = g11 * gv0 - g10 * gv1, pv1 = -g01 * gv0 + g00 * gv1;
      gq = W / adet * (pu0 * pv0 + pu1 * pv1);
    } else {
      gq = W * (gu0 * gv0 + gu1 * gv1);
    }
    if (A.grad) ((double*)A.grad)[e * Q + k] = gq;
    if (A.partial) part += (A.kappa ? A.kappa[e * Q + k] : 1.0) * gq;
  }
  if (A.partial) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red[w];
      A.partial[A.partial_offset + e] = s;
    }
  }
}

// One block sums partial[0..n) in a fixed order (strided per thread, then a
// fixed tree) and writes the double result.
__global__ void __launch_bounds__(1024) k_reduce_fixed(const double* __restrict__ partial,
                                                       int64_t n, double* out) {
  __shared__ double sm[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 1024) s += partial[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

template <typename T, int P, int QG, bool GEN>
cudaError_t run(const AdjArgs& a, cudaStream_t st) {
  using C = ADJ<T, P, QG, GEN>;
  k_adjoint3<T, P, QG, GEN><<<(unsigned)a.n_elem, C::NT, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int P, int QG>
cudaError_t rung(const AdjArgs& a, cudaStream_t st) {
  return a.jac ? run<T, P, QG, true>(a, st) : run<T, P, QG, false>(a, st);
}

template <typename T>
cudaError_t dispatch(const AdjArgs& a, int p, int q, cudaStream_t st) {
  const int dq = q - p;
#define C3(PP)                                                 \
  if (p == PP && dq == 1) return rung<T, PP, PP + 1>(a, st);   \
  if (p == PP && dq == 2) return rung<T, PP, PP + 2>(a, st);
  C3(1) C3(2) C3(3) C3(4)
  if (p == 5 && dq == 1) return rung<T, 5, 6>(a, st);
#undef C3
  return cudaErrorInvalidValue;
}

}  // namespace

bool adjoint_supported(int dim, int p, int q) {
  if (dim == 2) return p >= 1 && p <= 5 && (q == p + 1 || q == p + 2);
  return dim == 3 && p >= 1 && p <= 5 && (q == p + 1 || (q == p + 2 && p <= 4));
}

template <int P, int QG>
cudaError_t run2(const AdjArgs& a, cudaStream_t st) {
  if (a.jac) k_adjoint2<P, QG, true><<<(unsigned)a.n_elem, 64, 0, st>>>(a);
  else k_adjoint2<P, QG, false><<<(unsigned)a.n_elem, 64, 0, st>>>(a);
  return cudaGetLastError();
}

static cudaError_t dispatch2(const AdjArgs& a, int p, int q, cudaStream_t st) {
  const int dq = q - p;
#define C2(PP)                                              \
  if (p == PP && dq == 1) return run2<PP, PP + 1>(a, st);   \
  if (p == PP && dq == 2) return run2<PP, PP + 2>(a, st);
  C2(1) C2(2) C2(3) C2(4) C2(5)
#undef C2
  return cudaErrorInvalidValue;
}

cudaError_t launch_adjoint(const AdjArgs& a, int dim, int p, int q, bool fp64, bool df,
                           cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  if (dim == 2) return fp64 ? dispatch2(a, p, q, st) : cudaErrorInvalidValue;
  if (df) return dispatch<ff>(a, p, q, st);
  return fp64 ? dispatch<double>(a, p, q, st) : dispatch<float>(a, p, q, st);
}

cudaError_t launch_reduce_fixed(const double* partial, int64_t n, double* out, cudaStream_t st) {
  k_reduce_fixed<<<1, 1024, 0, st>>>(partial, n, out);
  return cudaGetLastError();
}

}  // namespace iga
