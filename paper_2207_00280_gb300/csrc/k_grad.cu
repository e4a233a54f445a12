// k_grad.cu -- backward of the element matrices with respect to the
// coefficients (3D; not in the paper: the element integrals are linear in
// kappa and rho, eq. 10 and the stiffness of Sec. 2.2).  Given upstream
// gradients GK = dL/dK_e and GM = dL/dM_e:
//   dL/dkappa_q = w_q |det G_q| sum_ij (G^{-1} G^{-T})_ij H_ij(q),
//   H_ij(q)     = sum_ab GK_ab d_i phi_a(q) d_j phi_b(q)   (reference derivatives)
//   dL/drho_q   = w_q |det G_q| sum_ab GM_ab phi_a(q) phi_b(q).
// H is formed by sum factorization run backwards (the transpose of Algorithm
// 2's stage order): for each Gauss point q1 of x, contract (a1, b1) against
// the x factors, then (a2, b2) against the y factors at every q2, then (a3,
// b3) against the z factors at every q3.  A term (i, j) uses the derivative
// factor in direction i on the test side and in direction j on the trial
// side; identity geometry needs the three terms i = j, a general Jacobian all
// nine.  One CTA per element; T = double (FP64) or float (FP32 with FP64
// cofactors and determinant).
#include "iga_internal.h"

namespace iga {
namespace {

template <typename T, int P, int QG, bool GEN>
struct GRD {
  static constexpr int n = P + 1, q = QG, n2 = n * n, n4 = n2 * n2, N = n2 * n, Q = q * q * q;
  static constexpr int NT = 128;
  static constexpr int REC = 2 * q * n + q;
  static constexpr int NTERM = GEN ? 9 : 3;       // stiffness terms (i, j)
  static constexpr int NXP = GEN ? 4 : 2;         // x factor pairs of the stiffness
  // term t -> (i, j): GEN t = 3 i + j; identity t -> (t, t)
  static constexpr int ti(int t) { return GEN ? t / 3 : t; }
  static constexpr int tj(int t) { return GEN ? t % 3 : t; }
  // x pair index of (s, t): GEN 0 (1,1) 1 (1,0) 2 (0,1) 3 (0,0); identity 0 (1,1) 1 (0,0)
  static constexpr int xp(int s, int t) {
    return GEN ? (s ? (t ? 0 : 1) : (t ? 2 : 3)) : (s ? 0 : 1);
  }
};

template <typename T, int P, int QG, bool GEN>
__global__ void __launch_bounds__(128) k_grad3(const GradArgs A) {
  using C = GRD<T, P, QG, GEN>;
  constexpr int n = C::n, q = C::q, n2 = C::n2, n4 = C::n4, N = C::N, Q = C::Q, NT = C::NT,
                REC = C::REC, NTERM = C::NTERM, NXP = C::NXP;
  __shared__ double rec[3 * REC];
  __shared__ T f[3][2][q * n];          // [direction][value, derivative][q][n]
  __shared__ T UX[NXP + 1][n4];         // x-contracted pairs of GK, then the mass pair of GM
  __shared__ T UY[NTERM + 1][n2 * q];   // [term][a3 n + b3][q2], the mass last
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  const int e1 = (int)(e % A.K1);
  const int e2 = (int)((e / A.K1) % A.K2);
  const int e3 = (int)(e / ((int64_t)A.K1 * A.K2));
  for (int i = tid; i < 3 * REC; i += NT) {
    const int d = i / REC, j = i - d * REC;
    const int ek = d == 0 ? e1 : (d == 1 ? e2 : e3);
    const double* tb = d == 0 ? A.tab[0] : (d == 1 ? A.tab[1] : A.tab[2]);
    rec[i] = tb[(int64_t)ek * REC + j];
  }
  __syncthreads();
  for (int i = tid; i < 3 * 2 * q * n; i += NT) {
    const int d = i / (2 * q * n), j = i % (2 * q * n);
    (&f[0][0][0])[i] = (T)rec[d * REC + j];
  }
  __syncthreads();
  const T* GK = (const T*)A.GK;
  const T* GM = (const T*)A.GM;
  const bool doK = GK != nullptr, doM = GM != nullptr;
#pragma unroll 1
  for (int q1 = 0; q1 < q; ++q1) {
    // x: every (a2 a3, b2 b3) block of the upstream matrices against the x factors
    for (int it = tid; it < n4; it += NT) {
      const int a23 = it / n2, b23 = it % n2;
      if (doK) {
        T v[2][n];
#pragma unroll
        for (int a1 = 0; a1 < n; ++a1) {
          const T* row = GK + ((int64_t)e * N + a1 + n * a23) * N + n * b23;
          T s0 = 0, s1 = 0;
#pragma unroll
          for (int b1 = 0; b1 < n; ++b1) {
            const T g = row[b1];
            s0 += g * f[0][0][q1 * n + b1];
            s1 += g * f[0][1][q1 * n + b1];
          }
          v[0][a1] = s0;
          v[1][a1] = s1;
        }
#pragma unroll
        for (int pi = 0; pi < NXP; ++pi) {
          const int s = GEN ? (pi <= 1) : (pi == 0);
          const int t = GEN ? (pi == 0 || pi == 2) : (pi == 0);
          T acc = 0;
#pragma unroll
          for (int a1 = 0; a1 < n; ++a1) acc += f[0][s][q1 * n + a1] * v[t][a1];
          UX[pi][it] = acc;
        }
      }
      if (doM) {
        T acc = 0;
#pragma unroll
        for (int a1 = 0; a1 < n; ++a1) {
          const T* row = GM + ((int64_t)e * N + a1 + n * a23) * N + n * b23;
          T s0 = 0;
#pragma unroll
          for (int b1 = 0; b1 < n; ++b1) s0 += row[b1] * f[0][0][q1 * n + b1];
          acc += f[0][0][q1 * n + a1] * s0;
        }
        UX[NXP][it] = acc;
      }
    }
    __syncthreads();
    // y: every (term, a3 b3, q2)
    for (int it = tid; it < (NTERM + 1) * n2 * q; it += NT) {
      const int term = it / (n2 * q), r = it % (n2 * q), ab3 = r / q, q2 = r % q;
      if ((term < NTERM && !doK) || (term == NTERM && !doM)) continue;
      const int a3 = ab3 / n, b3 = ab3 % n;
      int px, sy, ty;
      if (term < NTERM) {
        const int i = C::ti(term), j = C::tj(term);
        px = C::xp(i == 0, j == 0);
        sy = i == 1;
        ty = j == 1;
      } else {
        px = NXP;
        sy = ty = 0;
      }
      T acc = 0;
#pragma unroll
      for (int a2 = 0; a2 < n; ++a2) {
        T s0 = 0;
#pragma unroll
        for (int b2 = 0; b2 < n; ++b2) s0 += f[1][ty][q2 * n + b2] * UX[px][(a2 + n * a3) * n2 + b2 + n * b3];
        acc += f[1][sy][q2 * n + a2] * s0;
      }
      UY[term][ab3 * q + q2] = acc;
    }
    __syncthreads();
    // z and the geometry at every (q2, q3) of this q1
    for (int it = tid; it < q * q; it += NT) {
      const int q2 = it % q, q3 = it / q;
      const int k = q1 + q * (q2 + q * q3);
      T H[NTERM + 1];
#pragma unroll
      for (int term = 0; term <= NTERM; ++term) {
        H[term] = 0;
        if ((term < NTERM && !doK) || (term == NTERM && !doM)) continue;
        int sz = 0, tz = 0;
        if (term < NTERM) {
          sz = C::ti(term) == 2;
          tz = C::tj(term) == 2;
        }
        T acc = 0;
#pragma unroll
        for (int a3 = 0; a3 < n; ++a3) {
          T s0 = 0;
#pragma unroll
          for (int b3 = 0; b3 < n; ++b3) s0 += f[2][tz][q3 * n + b3] * UY[term][(a3 * n + b3) * q + q2];
          acc += f[2][sz][q3 * n + a3] * s0;
        }
        H[term] = acc;
      }
      const double W = rec[2 * q * n + q1] * rec[REC + 2 * q * n + q2] * rec[2 * REC + 2 * q * n + q3];
      double wk = W, wm = W;
      T D[NTERM];
      if (GEN) {
        const double* G = A.jac + (e * Q + k) * 9;
        const double g00 = G[0], g01 = G[1], g02 = G[2], g10 = G[3], g11 = G[4], g12 = G[5],
                     g20 = G[6], g21 = G[7], g22 = G[8];
        const double c[3][3] = {{g11 * g22 - g12 * g21, g12 * g20 - g10 * g22, g10 * g21 - g11 * g20},
                                {g02 * g21 - g01 * g22, g00 * g22 - g02 * g20, g01 * g20 - g00 * g21},
                                {g01 * g12 - g02 * g11, g02 * g10 - g00 * g12, g00 * g11 - g01 * g10}};
        const double det = g00 * c[0][0] + g01 * c[0][1] + g02 * c[0][2];
        const double adet = fabs(det);
        // w |det| (G^{-1} G^{-T})_ij = (w / |det|) sum_m c_mi c_mj
        wk = W / adet;
        wm = W * adet;
#pragma unroll
        for (int term = 0; term < NTERM; ++term) {
          const int i = C::ti(term), j = C::tj(term);
          D[term] = (T)(wk * (c[0][i] * c[0][j] + c[1][i] * c[1][j] + c[2][i] * c[2][j]));
        }
      } else {
#pragma unroll
        for (int term = 0; term < NTERM; ++term) D[term] = (T)W;
      }
      if (doK) {
        T g = 0;
#pragma unroll
        for (int term = 0; term < NTERM; ++term) g += D[term] * H[term];
        ((T*)A.grad_kappa)[e * Q + k] = g;
      }
      if (doM) ((T*)A.grad_rho)[e * Q + k] = (T)wm * H[NTERM];
    }
    __syncthreads();
  }
}

template <typename T, int P, int QG>
cudaError_t run(const GradArgs& a, cudaStream_t st) {
  if (a.jac) k_grad3<T, P, QG, true><<<(unsigned)a.n_elem, 128, 0, st>>>(a);
  else k_grad3<T, P, QG, false><<<(unsigned)a.n_elem, 128, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(const GradArgs& a, int p, int q, cudaStream_t st) {
  const int dq = q - p;
#define C3(PP)                                               \
  if (p == PP && dq == 1) return run<T, PP, PP + 1>(a, st);  \
  if (p == PP && dq == 2) return run<T, PP, PP + 2>(a, st);
  C3(1) C3(2) C3(3)
  if (p == 4 && dq == 1) return run<T, 4, 5>(a, st);
#undef C3
  return cudaErrorInvalidValue;
}

}  // namespace

bool grad_supported(int dim, int p, int q) {
  return dim == 3 && p >= 1 && ((p <= 3 && (q == p + 1 || q == p + 2)) || (p == 4 && q == 5));
}

cudaError_t launch_grad(const GradArgs& a, int p, int q, bool fp64, cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  return fp64 ? dispatch<double>(a, p, q, st) : dispatch<float>(a, p, q, st);
}

}  // namespace iga
