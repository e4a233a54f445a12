// k_classical64.cu -- FP64 classical element matrices (Sec. 3.2, Algorithm 1;
// the triple Gauss sum of eq. 10), with the paper's level-3 concurrency
// (Sec. 3.3: one thread per element-matrix entry).  One CTA per element; the
// quadrature points are processed in tiles whose tensor-product basis values
// and gradients sit in shared memory:
//   phi_a(x_k) = prod_j B_{a_j}(x_kj),   g_a = G^{-T} grad_xi phi_a,
//   M_ab += (w |det G| rho phi_b) phi_a,   K_ab += sum_i (w |det G| kappa g_b)_i (g_a)_i.
// Only a <= b is accumulated; both triangles are stored.
#include "iga_internal.h"

namespace iga {
namespace {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <int DIM, int P, int QG>
struct CL {
  static constexpr int n = P + 1, q = QG, N = ipow(n, DIM), Q = ipow(q, DIM);
  static constexpr int S = N * (N + 1) / 2;
  static constexpr int NT = 256;
  static constexpr int EPT_ALL = (S + NT - 1) / NT;
  static constexpr int EPT = EPT_ALL <= 16 ? EPT_ALL : 16;    // entries per thread per pass
  static constexpr int PASS = NT * EPT;
  static constexpr int REC = 2 * q * n + q;
  // quadrature tile: (2 + 2 DIM) N QT doubles of tables + 2 QT + 9 QT geometry
  static constexpr int qt_fit(int t) {
    return ((2 + 2 * DIM) * N * t + 11 * t + DIM * REC) * 8 <= 100 * 1024 ? t : qt_fit(t - 1);
  }
  static constexpr int QT = qt_fit(Q < 64 ? Q : 64);
  static constexpr size_t smem = (size_t)8 * ((2 + 2 * DIM) * N * QT + 11 * QT + DIM * REC);
};

template <int DIM, int P, int QG, bool GEN>
__global__ void __launch_bounds__(256) k_classical_f64(const ElemArgs A) {
  using C = CL<DIM, P, QG>;
  constexpr int n = C::n, q = C::q, N = C::N, Q = C::Q, S = C::S, NT = C::NT, EPT = C::EPT,
                QT = C::QT, REC = C::REC;
  extern __shared__ __align__(16) double sm[];
  double* rec = sm;                       // [DIM][REC]
  double* phi = rec + DIM * REC;          // [N][QT]
  double* g = phi + N * QT;               // [DIM][N][QT]   physical gradients
  double* wphi = g + DIM * N * QT;        // [N][QT]        W rho phi
  double* wg = wphi + N * QT;             // [DIM][N][QT]   W kappa g
  double* geo = wg + DIM * N * QT;        // [11][QT]: Wk, Wr, Ginv (row-major)
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  int e1, e2, e3;
  elem_coords(A, e, e1, e2, e3);
  for (int i = tid; i < DIM * REC; i += NT) {
    const int d = i / REC, j = i - d * REC;
    const int ek = d == 0 ? e1 : (d == 1 ? e2 : e3);
    const double* tb = d == 0 ? A.tab[0] : (d == 1 ? A.tab[1] : A.tab[2]);
    rec[i] = tb[(int64_t)ek * REC + j];
  }
  double* Ke = A.K_out ? (double*)A.K_out + e * (int64_t)N * N : nullptr;
  double* Me = A.M_out ? (double*)A.M_out + e * (int64_t)N * N : nullptr;

  for (int pass0 = 0; pass0 < S; pass0 += C::PASS) {
    int ea[EPT], eb[EPT];
    double accK[EPT], accM[EPT];
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      const int it = pass0 + tid + j * NT;
      int a = -1, b = -1;
      if (it < S) {
        // row a of the upper triangle: it = a N - a (a - 1) / 2 + (b - a)
        const float fN = 2.0f * N + 1.0f;
        a = (int)((fN - sqrtf(fN * fN - 8.0f * (float)it)) * 0.5f);
        if (a < 0) a = 0;
        if (a > N - 1) a = N - 1;
        while (a > 0 && a * N - a * (a - 1) / 2 > it) --a;
        while (a + 1 < N && (a + 1) * N - (a + 1) * a / 2 <= it) ++a;
        b = a + (it - (a * N - a * (a - 1) / 2));
      }
      ea[j] = a; eb[j] = b;
      accK[j] = 0.0; accM[j] = 0.0;
    }
    for (int k0 = 0; k0 < Q; k0 += QT) {
      __syncthreads();
      // geometry of the tile
      for (int t = tid; t < QT; t += NT) {
        const int k = k0 + t;
        if (k >= Q) continue;
        int kk[3] = {k % q, (k / q) % q, DIM == 3 ? k / (q * q) : 0};
        double W = 1.0;
        for (int d = 0; d < DIM; ++d) W *= rec[d * REC + 2 * q * n + kk[d]];
        const double kap = A.kappa ? A.kappa[e * Q + k] : 1.0;
        const double rh = A.rho ? A.rho[e * Q + k] : 1.0;
        double adet = 1.0;
        if (GEN) {
          const double* G = A.jac + (e * Q + k) * DIM * DIM;
          double inv[9];
          if (DIM == 3) {
            const double c00 = G[4] * G[8] - G[5] * G[7], c01 = G[5] * G[6] - G[3] * G[8],
                         c02 = G[3] * G[7] - G[4] * G[6];
            const double det = G[0] * c00 + G[1] * c01 + G[2] * c02;
            const double r = 1.0 / det;
            inv[0] = c00 * r; inv[3] = c01 * r; inv[6] = c02 * r;
            inv[1] = (G[2] * G[7] - G[1] * G[8]) * r;
            inv[4] = (G[0] * G[8] - G[2] * G[6]) * r;
            inv[7] = (G[1] * G[6] - G[0] * G[7]) * r;
            inv[2] = (G[1] * G[5] - G[2] * G[4]) * r;
            inv[5] = (G[2] * G[3] - G[0] * G[5]) * r;
            inv[8] = (G[0] * G[4] - G[1] * G[3]) * r;
            adet = fabs(det);
          } else {
            const double det = G[0] * G[3] - G[1] * G[2];
            const double r = 1.0 / det;
            inv[0] = G[3] * r; inv[1] = -G[1] * r; inv[2] = -G[2] * r; inv[3] = G[0] * r;
            adet = fabs(det);
          }
          for (int i = 0; i < DIM * DIM; ++i) geo[(2 + i) * QT + t] = inv[i];
        }
        geo[0 * QT + t] = W * adet * kap;
        geo[1 * QT + t] = W * adet * rh;
      }
      __syncthreads();
      // tensor-product values and physical gradients of every local function
      for (int i = tid; i < N * QT; i += NT) {
        const int a = i / QT, t = i % QT;
        const int k = k0 + t;
        if (k >= Q) {
          phi[i] = 0.0; wphi[i] = 0.0;
          for (int d = 0; d < DIM; ++d) { g[d * N * QT + i] = 0.0; wg[d * N * QT + i] = 0.0; }
          continue;
        }
        int kk[3] = {k % q, (k / q) % q, DIM == 3 ? k / (q * q) : 0};
        int aa[3] = {a % n, (a / n) % n, DIM == 3 ? a / (n * n) : 0};
        double v[3], dv[3];
        for (int d = 0; d < DIM; ++d) {
          v[d] = rec[d * REC + kk[d] * n + aa[d]];
          dv[d] = rec[d * REC + q * n + kk[d] * n + aa[d]];
        }
        double ph, gr[3];
        if (DIM == 3) {
          ph = v[0] * v[1] * v[2];
          gr[0] = dv[0] * v[1] * v[2];
          gr[1] = v[0] * dv[1] * v[2];
          gr[2] = v[0] * v[1] * dv[2];
        } else {
          ph = v[0] * v[1];
          gr[0] = dv[0] * v[1];
          gr[1] = v[0] * dv[1];
        }
        double pg[3];
        if (GEN) {
          for (int d = 0; d < DIM; ++d) {  // (G^{-T} gr)_d = sum_j Ginv[j][d] gr_j
            double s = 0.0;
            for (int j = 0; j < DIM; ++j) s = fma(geo[(2 + j * DIM + d) * QT + t], gr[j], s);
            pg[d] = s;
          }
        } else {
          for (int d = 0; d < DIM; ++d) pg[d] = gr[d];
        }
        const double wk = geo[t], wr = geo[QT + t];
        phi[i] = ph;
        wphi[i] = wr * ph;
        for (int d = 0; d < DIM; ++d) {
          g[d * N * QT + i] = pg[d];
          wg[d * N * QT + i] = wk * pg[d];
        }
      }
      __syncthreads();
      // Algorithm 1's innermost loop: accumulate over the quadrature tile
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        if (ea[j] < 0) continue;
        const int a = ea[j], b = eb[j];
        double sk = accK[j], smm = accM[j];
        const double* pa = phi + a * QT;
        const double* pb = wphi + b * QT;
#pragma unroll 4
        for (int t = 0; t < QT; ++t) {
          if (Ke) {
#pragma unroll
            for (int d = 0; d < DIM; ++d)
              sk = fma(g[d * N * QT + a * QT + t], wg[d * N * QT + b * QT + t], sk);
          }
          if (Me) smm = fma(pa[t], pb[t], smm);
        }
        accK[j] = sk; accM[j] = smm;
      }
    }
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      if (ea[j] < 0) continue;
      const int a = ea[j], b = eb[j];
      if (Ke) { Ke[(int64_t)a * N + b] = accK[j]; Ke[(int64_t)b * N + a] = accK[j]; }
      if (Me) { Me[(int64_t)a * N + b] = accM[j]; Me[(int64_t)b * N + a] = accM[j]; }
    }
  }
}

template <int DIM, int P, int QG, bool GEN>
cudaError_t runc(const ElemArgs& a, cudaStream_t st) {
  using C = CL<DIM, P, QG>;
  static_assert(C::smem <= 227 * 1024, "shared memory");
  auto k = k_classical_f64<DIM, P, QG, GEN>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)a.n_elem, C::NT, C::smem, st>>>(a);
  return cudaGetLastError();
}

template <int DIM, int P, int QG>
cudaError_t runcg(const ElemArgs& a, cudaStream_t st) {
  return a.jac ? runc<DIM, P, QG, true>(a, st) : runc<DIM, P, QG, false>(a, st);
}

}  // namespace

bool classical_f64_supported(int dim, int p, int q) {
  if (dim == 3) return p >= 1 && p <= 5 && (q == p + 1 || (q == p + 2 && p <= 4));
  if (dim == 2) return p >= 1 && p <= 8 && (q == p + 1 || q == p + 2);
  return false;
}

cudaError_t launch_classical_f64(const ElemArgs& a, int dim, int p, int q, cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  const int dq = q - p;
  if (dim == 3) {
#define C3(PP)                                              \
  if (p == PP && dq == 1) return runcg<3, PP, PP + 1>(a, st); \
  if (p == PP && dq == 2) return runcg<3, PP, PP + 2>(a, st);
    C3(1) C3(2) C3(3) C3(4)
    if (p == 5 && dq == 1) return runcg<3, 5, 6>(a, st);
#undef C3
  } else {
#define C2(PP)                                              \
  if (p == PP && dq == 1) return runcg<2, PP, PP + 1>(a, st); \
  if (p == PP && dq == 2) return runcg<2, PP, PP + 2>(a, st);
    C2(1) C2(2) C2(3) C2(4) C2(5) C2(6) C2(7) C2(8)
#undef C2
  }
  return cudaErrorInvalidValue;
}

}  // namespace iga
