// k_generic64.cu -- FP64 element matrices and adjoint with runtime sizes: a
// degree 1 <= p_k <= 8 and a Gauss order 1 <= q_k <= 16 per direction, in 2D
// and 3D.  The paper takes one degree for all directions and notes that the
// method extends to bases of different degrees (Sec. 2.3); its element sum
// (eq. 10) already has P_1 P_2 P_3 quadrature points, and its experiments run
// degrees up to 9 (Sec. 4).  The templated kernels of k_sumfact64.cu and
// k_classical64.cu cover the isotropic patches with p <= 5 and q = p+1, p+2,
// where an element matrix fits in shared memory; these kernels cover the rest.
//
// A 2D patch runs as a 3D one whose third direction has one function (value 1,
// derivative 0) and one quadrature point of weight 1.
//
// Sum factorization (Algorithm 2: contract z, then y, then x) with the
// element matrix produced one (a3, b3) block at a time: for each pair
// a3 <= b3 the stage-1 buffers T1 (z contracted, [item][q1][q2]), the stage-2
// buffers C (y contracted, [x pattern][a2][b2][q1]) and the block
// K[(a1,a2,a3), (b1,b2,b3)] (x contracted) are formed; the block is written to
// HBM straight from the registers, and its transpose into block (b3, a3)
// (the matrices are symmetric).  Per-point coefficients
//   D = w |det G| kappa G^{-1} G^{-T} (6 unique),  D_M = w |det G| rho
// sit in shared memory when they fit, otherwise they are recomputed from
// kappa, rho and G at every use (Gauss orders far above p+1).
#include "iga_internal.h"

namespace iga {
namespace {

constexpr int kGenThreads = 256;
constexpr size_t kGenSmemMax = 227 * 1024;   // the opt-in maximum per CTA

struct Shape {
  int dim;
  int n[3], q[3];   // functions and Gauss points per direction (1 beyond dim)
  int N, Q;
  int rs[3];        // record size per direction in shared memory
  int roff[3];      // record offset per direction in shared memory
  int rsum;
};

Shape make_shape(const PatchDev& ph) {
  Shape S{};
  S.dim = ph.dim;
  S.N = 1;
  S.Q = 1;
  S.rsum = 0;
  for (int k = 0; k < 3; ++k) {
    S.n[k] = k < ph.dim ? ph.nk[k] : 1;
    S.q[k] = k < ph.dim ? ph.qk[k] : 1;
    S.N *= S.n[k];
    S.Q *= S.q[k];
    S.rs[k] = record_size(S.n[k], S.q[k]);   // 3 for a missing direction
    S.roff[k] = S.rsum;
    S.rsum += S.rs[k];
  }
  return S;
}

// Value (s = 0) or derivative (s = 1) of local function a of direction k at
// its Gauss point j, and the mapped Gauss weight.
__device__ __forceinline__ double fval(const double* R, const Shape& S, int k, int s, int a, int j) {
  return R[S.roff[k] + (s ? S.q[k] * S.n[k] : 0) + j * S.n[k] + a];
}
__device__ __forceinline__ double fw(const double* R, const Shape& S, int k, int j) {
  return R[S.roff[k] + 2 * S.q[k] * S.n[k] + j];
}

// Basis records of element e into shared memory (a synthetic record for the
// missing direction of a 2D patch).
// (Per-direction values are selected, not indexed with a runtime direction,
// so that the argument records stay out of local memory.)
__device__ void load_records(double* R, const Shape& S, const double* const* tab, int e1, int e2,
                             int e3) {
  const double* t0 = tab[0] + (int64_t)e1 * S.rs[0];
  const double* t1 = tab[1] + (int64_t)e2 * S.rs[1];
  const double* t2 = tab[2] + (int64_t)e3 * S.rs[2];
  for (int i = threadIdx.x; i < S.rsum; i += blockDim.x) {
    const int k = i < S.roff[1] ? 0 : (i < S.roff[2] ? 1 : 2);
    const int j = i - (k == 0 ? 0 : (k == 1 ? S.roff[1] : S.roff[2]));
    if (k < S.dim) {
      R[i] = (k == 0 ? t0 : (k == 1 ? t1 : t2))[j];
    } else {
      R[i] = j == 1 ? 0.0 : 1.0;   // val = 1, der = 0, w = 1
    }
  }
}

// c[i] for a runtime i < 7 by selects (c stays in registers).
__device__ __forceinline__ double pick7(const double* c, int i) {
  return i == 0 ? c[0] : i == 1 ? c[1] : i == 2 ? c[2] : i == 3 ? c[3] : i == 4 ? c[4]
       : i == 5 ? c[5] : c[6];
}

// Coefficients at quadrature point k of element e.  GEN: {D00, D11, D01, DM,
// D22, D02, D12} with D = W kappa |det G| G^{-1} G^{-T} (2D: D22 = D02 = D12 = 0);
// identity map: {W kappa, W rho}.
template <bool GEN>
__device__ __forceinline__ void point_coefs(const ElemArgs& A, const double* R, const Shape& S,
                                            int64_t e, int k, double* c) {
  const int k1 = k % S.q[0], k2 = (k / S.q[0]) % S.q[1], k3 = k / (S.q[0] * S.q[1]);
  const double W = fw(R, S, 0, k1) * fw(R, S, 1, k2) * fw(R, S, 2, k3);
  const int64_t g = e * S.Q + k;
  const double kap = A.kappa ? A.kappa[g] : 1.0;
  const double rh = A.rho ? A.rho[g] : 1.0;
  if (!GEN) {
    c[0] = W * kap;
    c[1] = W * rh;
    return;
  }
  if (S.dim == 3) {
    const double* G = A.jac + g * 9;
    const double c00 = G[4] * G[8] - G[5] * G[7], c01 = G[5] * G[6] - G[3] * G[8],
                 c02 = G[3] * G[7] - G[4] * G[6];
    const double c10 = G[2] * G[7] - G[1] * G[8], c11 = G[0] * G[8] - G[2] * G[6],
                 c12 = G[1] * G[6] - G[0] * G[7];
    const double c20 = G[1] * G[5] - G[2] * G[4], c21 = G[2] * G[3] - G[0] * G[5],
                 c22 = G[0] * G[4] - G[1] * G[3];
    const double det = G[0] * c00 + G[1] * c01 + G[2] * c02;
    const double adet = fabs(det);
    // G^{-1} = cof^T / det, so (G^{-1} G^{-T})_ij = sum_l cof_li cof_lj / det^2
    const double s = W * kap / adet;
    c[0] = s * (c00 * c00 + c10 * c10 + c20 * c20);
    c[1] = s * (c01 * c01 + c11 * c11 + c21 * c21);
    c[2] = s * (c00 * c01 + c10 * c11 + c20 * c21);
    c[3] = W * adet * rh;
    c[4] = s * (c02 * c02 + c12 * c12 + c22 * c22);
    c[5] = s * (c00 * c02 + c10 * c12 + c20 * c22);
    c[6] = s * (c01 * c02 + c11 * c12 + c21 * c22);
  } else {
    const double* G = A.jac + g * 4;
    const double det = G[0] * G[3] - G[1] * G[2];
    const double adet = fabs(det);
    // G^{-1} = cof^T / det with cof = [[g11, -g10], [-g01, g00]], so
    // (G^{-1} G^{-T})_ij = sum_l cof_li cof_lj / det^2
    const double s = W * kap / adet;
    c[0] = s * (G[3] * G[3] + G[1] * G[1]);
    c[1] = s * (G[2] * G[2] + G[0] * G[0]);
    c[2] = s * (-G[3] * G[2] - G[1] * G[0]);
    c[3] = W * adet * rh;
    c[4] = 0.0;
    c[5] = 0.0;
    c[6] = 0.0;
  }
}

// 1D factor patterns: 0 = (v, v), 1 = (d, d), 2 = (d, v), 3 = (v, d), the first
// factor belonging to the test function a, the second to the trial function b.
__device__ __forceinline__ double pattern(const double* R, const Shape& S, int k, int pt, int a,
                                          int b, int j) {
  const int sa = (pt == 1 || pt == 2), sb = (pt == 1 || pt == 3);
  return fval(R, S, k, sa, a, j) * fval(R, S, k, sb, b, j);
}

// Stage-1 items (z pattern, coefficient index).  Stiffness term (i, j) has the
// derivative of the test function in direction i and of the trial function in
// direction j; its pattern in direction k is (i == k, j == k).
//   GEN:  (00,D00) (00,D01) (00,D11) (11,D22) (10,D02) (10,D12) (01,D02) (01,D12) (00,DM)
//   identity: (00,Dk) (11,Dk) (00,DM)
__device__ __constant__ int kItemGen[9][2] = {{0, 0}, {0, 2}, {0, 1}, {1, 4}, {2, 5},
                                              {2, 6}, {3, 5}, {3, 6}, {0, 3}};
__device__ __constant__ int kItemId[3][2] = {{0, 0}, {1, 0}, {0, 1}};
// Stage-2 terms per C buffer (x pattern 11, 10, 01, 00, mass): (y pattern, item).
//   GEN:  C0 = (00, I0); C1 = (01, I1) + (00, I6); C2 = (10, I1) + (00, I4);
//         C3 = (11, I2) + (10, I7) + (01, I5) + (00, I3); C4 = (00, I8)
//   identity: C0 = (00, J0); C3 = (11, J0) + (00, J1); C4 = (00, J2)
__device__ __constant__ int kTermGen[5][4][2] = {
    {{0, 0}, {-1, -1}, {-1, -1}, {-1, -1}},
    {{3, 1}, {0, 6}, {-1, -1}, {-1, -1}},
    {{2, 1}, {0, 4}, {-1, -1}, {-1, -1}},
    {{1, 2}, {2, 7}, {3, 5}, {0, 3}},
    {{0, 8}, {-1, -1}, {-1, -1}, {-1, -1}}};
__device__ __constant__ int kTermId[5][4][2] = {
    {{0, 0}, {-1, -1}, {-1, -1}, {-1, -1}},
    {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}},
    {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}},
    {{1, 0}, {0, 1}, {-1, -1}, {-1, -1}},
    {{0, 2}, {-1, -1}, {-1, -1}, {-1, -1}}};
// x pattern of each C buffer
__device__ __constant__ int kXPat[5] = {1, 2, 3, 0, 0};

struct SfLayout {
  int XP, YP, ZF, T1, CB, D, total;   // offsets in doubles
};

SfLayout sf_layout(const Shape& S, bool gen, bool dsmem) {
  const int NI = gen ? 9 : 3, NC = gen ? 7 : 2;
  SfLayout L{};
  int o = S.rsum;
  L.XP = o; o += 4 * S.n[0] * S.n[0] * S.q[0];
  L.YP = o; o += 4 * S.n[1] * S.n[1] * S.q[1];
  L.ZF = o; o += 4 * S.q[2];
  L.T1 = o; o += NI * S.q[0] * S.q[1];
  L.CB = o; o += 5 * S.n[1] * S.n[1] * S.q[0];
  L.D = o;  o += dsmem ? NC * S.Q : 0;
  L.total = o;
  return L;
}

template <bool GEN, bool DSMEM>
__global__ void __launch_bounds__(kGenThreads)
    k_sf_gen(const ElemArgs A, const Shape S, const SfLayout L) {
  constexpr int NI = GEN ? 9 : 3, NC = GEN ? 7 : 2;
  extern __shared__ __align__(16) double sm[];
  double* R = sm;
  double* XP = sm + L.XP;
  double* YP = sm + L.YP;
  double* ZF = sm + L.ZF;
  double* T1 = sm + L.T1;
  double* CB = sm + L.CB;
  double* Dc = sm + L.D;
  const int tid = threadIdx.x;
  const int n1 = S.n[0], n2 = S.n[1], n3 = S.n[2], q1 = S.q[0], q2 = S.q[1], q3 = S.q[2];
  const int N = S.N, Q = S.Q;
  const int64_t e = blockIdx.x;
  int e1, e2, e3;
  elem_coords(A, e, e1, e2, e3);
  const bool wantK = A.K_out != nullptr, wantM = A.M_out != nullptr;
  double* Ke = wantK ? (double*)A.K_out + e * (int64_t)N * N : nullptr;
  double* Me = wantM ? (double*)A.M_out + e * (int64_t)N * N : nullptr;

  load_records(R, S, A.tab, e1, e2, e3);
  __syncthreads();
  for (int i = tid; i < 4 * n1 * n1 * q1; i += kGenThreads) {
    const int j = i % q1, b = (i / q1) % n1, a = (i / (q1 * n1)) % n1, pt = i / (q1 * n1 * n1);
    XP[i] = pattern(R, S, 0, pt, a, b, j);
  }
  for (int i = tid; i < 4 * n2 * n2 * q2; i += kGenThreads) {
    const int j = i % q2, b = (i / q2) % n2, a = (i / (q2 * n2)) % n2, pt = i / (q2 * n2 * n2);
    YP[i] = pattern(R, S, 1, pt, a, b, j);
  }
  if (DSMEM) {
    for (int k = tid; k < Q; k += kGenThreads) {
      double c[7];
      point_coefs<GEN>(A, R, S, e, k, c);
#pragma unroll
      for (int t = 0; t < NC; ++t) Dc[t * Q + k] = c[t];
    }
  }
  __syncthreads();

  const int n12 = n1 * n2;
  for (int a3 = 0; a3 < n3; ++a3) {
    for (int b3 = a3; b3 < n3; ++b3) {
      // z factors of the pair (a3, b3) at every z Gauss point
      for (int i = tid; i < 4 * q3; i += kGenThreads) ZF[i] = pattern(R, S, 2, i / q3, a3, b3, i % q3);
      __syncthreads();
      // stage 1 (Algorithm 2, z): T1[item][q1][q2] = sum_k3 Z(item)[k3] D(item)[q1,q2,k3]
      for (int t = tid; t < q1 * q2; t += kGenThreads) {
        const int k1 = t % q1, k2 = t / q1;
        double acc[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) acc[i] = 0.0;
        for (int k3 = 0; k3 < q3; ++k3) {
          const int k = k1 + q1 * (k2 + q2 * k3);
          double c[7];
          if (DSMEM) {
#pragma unroll
            for (int j = 0; j < NC; ++j) c[j] = Dc[j * Q + k];
          } else {
            point_coefs<GEN>(A, R, S, e, k, c);
          }
#pragma unroll
          for (int i = 0; i < NI; ++i) {
            const int zp = GEN ? kItemGen[i][0] : kItemId[i][0];
            const int ci = GEN ? kItemGen[i][1] : kItemId[i][1];
            acc[i] = fma(ZF[zp * q3 + k3], pick7(c, ci), acc[i]);
          }
        }
#pragma unroll
        for (int i = 0; i < NI; ++i) T1[(i * q1 + k1) * q2 + k2] = acc[i];
      }
      __syncthreads();
      // stage 2 (y): C[X][a2][b2][q1] = sum over the terms of X of
      //              sum_k2 Y(pattern)[a2][b2][k2] T1[item][q1][k2]
      for (int t = tid; t < 5 * n2 * n2 * q1; t += kGenThreads) {
        const int k1 = t % q1, b2 = (t / q1) % n2, a2 = (t / (q1 * n2)) % n2, X = t / (q1 * n2 * n2);
        if ((X < 4 && !wantK) || (X == 4 && !wantM)) continue;
        double acc = 0.0;
        for (int m = 0; m < 4; ++m) {
          const int yp = GEN ? kTermGen[X][m][0] : kTermId[X][m][0];
          if (yp < 0) break;
          const int it = GEN ? kTermGen[X][m][1] : kTermId[X][m][1];
          const double* y = YP + ((yp * n2 + a2) * n2 + b2) * q2;
          const double* tt = T1 + (it * q1 + k1) * q2;
          for (int k2 = 0; k2 < q2; ++k2) acc = fma(y[k2], tt[k2], acc);
        }
        CB[t] = acc;
      }
      __syncthreads();
      // stage 3 (x): block (a3, b3) of the element matrices; a diagonal block
      // (a3 = b3) is symmetric, so only its upper triangle is formed and every
      // entry is stored at (row, col) and (col, row)
      for (int t = tid; t < n12 * n12; t += kGenThreads) {
        const int r = t / n12, c = t % n12;
        if (a3 == b3 && r > c) continue;
        const int a1 = r % n1, a2 = r / n1, b1 = c % n1, b2 = c / n1;
        const int64_t row = r + (int64_t)n12 * a3, col = c + (int64_t)n12 * b3;
        if (wantK) {
          double acc = 0.0;
          for (int X = 0; X < 4; ++X) {
            if (!GEN && (X == 1 || X == 2)) continue;
            const double* x = XP + ((kXPat[X] * n1 + a1) * n1 + b1) * q1;
            const double* cb = CB + ((X * n2 + a2) * n2 + b2) * q1;
            for (int k1 = 0; k1 < q1; ++k1) acc = fma(x[k1], cb[k1], acc);
          }
          Ke[row * N + col] = acc;
          if (row != col) Ke[col * N + row] = acc;
        }
        if (wantM) {
          double acc = 0.0;
          const double* x = XP + (a1 * n1 + b1) * q1;
          const double* cb = CB + ((4 * n2 + a2) * n2 + b2) * q1;
          for (int k1 = 0; k1 < q1; ++k1) acc = fma(x[k1], cb[k1], acc);
          Me[row * N + col] = acc;
          if (row != col) Me[col * N + row] = acc;
        }
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Classical integration (Algorithm 1) with runtime sizes: one CTA per element,
// one thread per upper-triangle entry (EPT entries per thread per pass), the
// quadrature points in tiles of QT whose tensor-product values and physical
// gradients sit in shared memory.
// ---------------------------------------------------------------------------
constexpr int kClEpt = 16;

template <bool GEN>
__global__ void __launch_bounds__(kGenThreads)
    k_cl_gen(const ElemArgs A, const Shape S, int QT) {
  extern __shared__ __align__(16) double sm[];
  const int tid = threadIdx.x;
  const int N = S.N, Q = S.Q, S2 = N * (N + 1) / 2, dim = S.dim;
  double* R = sm;
  double* phi = R + S.rsum;               // [N][QT]
  double* g = phi + N * QT;               // [3][N][QT]  physical gradients
  double* wphi = g + 3 * N * QT;          // [N][QT]     W |det| rho phi
  double* wg = wphi + N * QT;             // [3][N][QT]  W |det| kappa g
  double* geo = wg + 3 * N * QT;          // [11][QT]    W|det|kappa, W|det|rho, G^{-1}
  const int64_t e = blockIdx.x;
  int e1, e2, e3;
  elem_coords(A, e, e1, e2, e3);
  load_records(R, S, A.tab, e1, e2, e3);
  double* Ke = A.K_out ? (double*)A.K_out + e * (int64_t)N * N : nullptr;
  double* Me = A.M_out ? (double*)A.M_out + e * (int64_t)N * N : nullptr;
  const int PASS = kGenThreads * kClEpt;
  for (int pass0 = 0; pass0 < S2; pass0 += PASS) {
    int ea[kClEpt], eb[kClEpt];
    double accK[kClEpt], accM[kClEpt];
#pragma unroll
    for (int j = 0; j < kClEpt; ++j) {
      const int it = pass0 + tid + j * kGenThreads;
      int a = -1, b = -1;
      if (it < S2) {
        // row a of the upper triangle: it = a N - a (a - 1) / 2 + (b - a)
        const double fN = 2.0 * N + 1.0;
        a = (int)((fN - sqrt(fN * fN - 8.0 * (double)it)) * 0.5);
        if (a < 0) a = 0;
        if (a > N - 1) a = N - 1;
        while (a > 0 && a * N - a * (a - 1) / 2 > it) --a;
        while (a + 1 < N && (a + 1) * N - (a + 1) * a / 2 <= it) ++a;
        b = a + (it - (a * N - a * (a - 1) / 2));
      }
      ea[j] = a;
      eb[j] = b;
      accK[j] = 0.0;
      accM[j] = 0.0;
    }
    for (int k0 = 0; k0 < Q; k0 += QT) {
      __syncthreads();
      for (int t = tid; t < QT; t += kGenThreads) {
        const int k = k0 + t;
        if (k >= Q) continue;
        const int k1 = k % S.q[0], k2 = (k / S.q[0]) % S.q[1], k3 = k / (S.q[0] * S.q[1]);
        const double W = fw(R, S, 0, k1) * fw(R, S, 1, k2) * fw(R, S, 2, k3);
        const double kap = A.kappa ? A.kappa[e * Q + k] : 1.0;
        const double rh = A.rho ? A.rho[e * Q + k] : 1.0;
        double adet = 1.0;
        double inv[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        if (GEN) {
          if (dim == 3) {
            const double* G = A.jac + (e * Q + k) * 9;
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
            const double* G = A.jac + (e * Q + k) * 4;
            const double det = G[0] * G[3] - G[1] * G[2];
            const double r = 1.0 / det;
            // 2x2 inverse, stored in the 3x3 slots (row-major, third row/column identity)
            inv[0] = G[3] * r; inv[1] = -G[1] * r; inv[3] = -G[2] * r; inv[4] = G[0] * r;
            adet = fabs(det);
          }
        }
        for (int i = 0; i < 9; ++i) geo[(2 + i) * QT + t] = inv[i];
        geo[t] = W * adet * kap;
        geo[QT + t] = W * adet * rh;
      }
      __syncthreads();
      for (int i = tid; i < N * QT; i += kGenThreads) {
        const int a = i / QT, t = i % QT;
        const int k = k0 + t;
        if (k >= Q) {
          phi[i] = 0.0;
          wphi[i] = 0.0;
          for (int d = 0; d < 3; ++d) { g[d * N * QT + i] = 0.0; wg[d * N * QT + i] = 0.0; }
          continue;
        }
        const int kk[3] = {k % S.q[0], (k / S.q[0]) % S.q[1], k / (S.q[0] * S.q[1])};
        const int aa[3] = {a % S.n[0], (a / S.n[0]) % S.n[1], a / (S.n[0] * S.n[1])};
        double v[3], dv[3];
        for (int d = 0; d < 3; ++d) {
          v[d] = fval(R, S, d, 0, aa[d], kk[d]);
          dv[d] = fval(R, S, d, 1, aa[d], kk[d]);
        }
        const double ph = v[0] * v[1] * v[2];
        const double gr[3] = {dv[0] * v[1] * v[2], v[0] * dv[1] * v[2], v[0] * v[1] * dv[2]};
        double pg[3];
        for (int d = 0; d < 3; ++d) {   // (G^{-T} gr)_d = sum_j Ginv[j][d] gr_j
          double s = 0.0;
          for (int j = 0; j < 3; ++j) s = fma(geo[(2 + j * 3 + d) * QT + t], gr[j], s);
          pg[d] = s;
        }
        const double wk = geo[t], wr = geo[QT + t];
        phi[i] = ph;
        wphi[i] = wr * ph;
        for (int d = 0; d < 3; ++d) {
          g[d * N * QT + i] = pg[d];
          wg[d * N * QT + i] = wk * pg[d];
        }
      }
      __syncthreads();
      const int nt = (Q - k0) < QT ? (Q - k0) : QT;
#pragma unroll
      for (int j = 0; j < kClEpt; ++j) {
        if (ea[j] < 0) continue;
        const int a = ea[j], b = eb[j];
        double sk = accK[j], smm = accM[j];
        for (int t = 0; t < nt; ++t) {
          if (Ke) {
            for (int d = 0; d < dim; ++d)
              sk = fma(g[d * N * QT + a * QT + t], wg[d * N * QT + b * QT + t], sk);
          }
          if (Me) smm = fma(phi[a * QT + t], wphi[b * QT + t], smm);
        }
        accK[j] = sk;
        accM[j] = smm;
      }
    }
#pragma unroll
    for (int j = 0; j < kClEpt; ++j) {
      if (ea[j] < 0) continue;
      const int a = ea[j], b = eb[j];
      if (Ke) { Ke[(int64_t)a * N + b] = accK[j]; Ke[(int64_t)b * N + a] = accK[j]; }
      if (Me) { Me[(int64_t)a * N + b] = accM[j]; Me[(int64_t)b * N + a] = accM[j]; }
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint (not in the paper): g_k = w |det G| (G^{-T} grad u).(G^{-T} grad v)
// at every quadrature point, the reference gradients of u and v interpolated
// by sum factorization (contract a1, then a2, then a3), and the element's
// fixed-order sum of kappa g.
// ---------------------------------------------------------------------------
struct AdjLayout {
  int ue, ve, A1, A2, part, total;
};

AdjLayout adj_layout(const Shape& S) {
  AdjLayout L{};
  int o = S.rsum;
  L.ue = o; o += S.N;
  L.ve = o; o += S.N;
  L.A1 = o; o += 2 * 2 * S.n[1] * S.n[2] * S.q[0];           // [vec][s][a2 a3][q1]
  L.A2 = o; o += 2 * 3 * S.n[2] * S.q[0] * S.q[1];           // [vec][c][a3][q1 q2]
  L.part = o; o += S.Q;
  L.total = o;
  return L;
}

__global__ void __launch_bounds__(kGenThreads)
    k_adj_gen(const AdjArgs A, const Shape S, const AdjLayout L, int p1, int p2, int p3) {
  extern __shared__ __align__(16) double sm[];
  double* R = sm;
  double* ue = sm + L.ue;
  double* ve = sm + L.ve;
  double* A1 = sm + L.A1;
  double* A2 = sm + L.A2;
  double* part = sm + L.part;
  const int tid = threadIdx.x;
  const int n1 = S.n[0], n2 = S.n[1], n3 = S.n[2], q1 = S.q[0], q2 = S.q[1];
  const int N = S.N, Q = S.Q;
  const int64_t e = blockIdx.x;
  int e1, e2, e3;
  elem_coords(A, e, e1, e2, e3);
  load_records(R, S, A.tab, e1, e2, e3);
  // gather u_e, v_e through the dof map (support set of the element)
  const int s1 = A.span[0][e1] - p1, s2 = A.span[1][e2] - p2;
  const int s3 = S.dim == 3 ? A.span[2][e3] - p3 : 0;
  const double* u = (const double*)A.u;
  const double* v = (const double*)A.v;
  for (int a = tid; a < N; a += kGenThreads) {
    const int a1 = a % n1, a2 = (a / n1) % n2, a3 = a / (n1 * n2);
    const int64_t gi = A.dof_offset + (s1 + a1) +
                       (int64_t)A.nf0 * ((s2 + a2) + (int64_t)A.nf1 * (s3 + a3));
    ue[a] = u[gi];
    ve[a] = v[gi];
  }
  __syncthreads();
  const int n23 = n2 * n3;
  // contract a1: A1[vec][s][a23][q1] = sum_a1 u[a1 + n1 a23] F^s_x(q1)[a1]
  for (int t = tid; t < 2 * n23 * q1; t += kGenThreads) {
    const int k1 = t % q1, a23 = (t / q1) % n23, s = t / (q1 * n23);
    double au = 0.0, av = 0.0;
    for (int a1 = 0; a1 < n1; ++a1) {
      const double f = fval(R, S, 0, s, a1, k1);
      au = fma(ue[a1 + n1 * a23], f, au);
      av = fma(ve[a1 + n1 * a23], f, av);
    }
    A1[(s * n23 + a23) * q1 + k1] = au;
    A1[((2 + s) * n23 + a23) * q1 + k1] = av;
  }
  __syncthreads();
  // contract a2: A2[vec][c][a3][q1 q2], c = 0: (x derivative, y value),
  // 1: (x value, y derivative), 2: (x value, y value)
  const int q12 = q1 * q2;
  for (int t = tid; t < 3 * n3 * q12; t += kGenThreads) {
    const int k12 = t % q12, a3 = (t / q12) % n3, c = t / (q12 * n3);
    const int k1 = k12 % q1, k2 = k12 / q1;
    const int sx = c == 0, sy = c == 1;
    double au = 0.0, av = 0.0;
    for (int a2 = 0; a2 < n2; ++a2) {
      const double f = fval(R, S, 1, sy, a2, k2);
      au = fma(A1[(sx * n23 + a2 + n2 * a3) * q1 + k1], f, au);
      av = fma(A1[((2 + sx) * n23 + a2 + n2 * a3) * q1 + k1], f, av);
    }
    A2[(c * n3 + a3) * q12 + k12] = au;
    A2[((3 + c) * n3 + a3) * q12 + k12] = av;
  }
  __syncthreads();
  // contract a3 at every point, then the metric
  for (int k = tid; k < Q; k += kGenThreads) {
    const int k12 = k % q12, k3 = k / q12;
    const int k1 = k12 % q1, k2 = k12 / q1;
    double gu[3] = {0.0, 0.0, 0.0}, gv[3] = {0.0, 0.0, 0.0};
    for (int a3 = 0; a3 < n3; ++a3) {
      const double z = fval(R, S, 2, 0, a3, k3), dz = fval(R, S, 2, 1, a3, k3);
      gu[0] = fma(A2[(0 * n3 + a3) * q12 + k12], z, gu[0]);
      gu[1] = fma(A2[(1 * n3 + a3) * q12 + k12], z, gu[1]);
      gu[2] = fma(A2[(2 * n3 + a3) * q12 + k12], dz, gu[2]);
      gv[0] = fma(A2[(3 * n3 + a3) * q12 + k12], z, gv[0]);
      gv[1] = fma(A2[(4 * n3 + a3) * q12 + k12], z, gv[1]);
      gv[2] = fma(A2[(5 * n3 + a3) * q12 + k12], dz, gv[2]);
    }
    const double W = fw(R, S, 0, k1) * fw(R, S, 1, k2) * fw(R, S, 2, k3);
    double gq;
    if (A.jac) {
      double inv[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, adet;
      if (S.dim == 3) {
        const double* G = A.jac + (e * Q + k) * 9;
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
        const double* G = A.jac + (e * Q + k) * 4;
        const double det = G[0] * G[3] - G[1] * G[2];
        const double r = 1.0 / det;
        inv[0] = G[3] * r; inv[1] = -G[1] * r; inv[3] = -G[2] * r; inv[4] = G[0] * r;
        adet = fabs(det);
      }
      double dot = 0.0;
      for (int d = 0; d < 3; ++d) {   // (G^{-T} g)_d = sum_j Ginv[j][d] g_j
        double pu = 0.0, pv = 0.0;
        for (int j = 0; j < 3; ++j) {
          pu = fma(inv[j * 3 + d], gu[j], pu);
          pv = fma(inv[j * 3 + d], gv[j], pv);
        }
        dot = fma(pu, pv, dot);
      }
      gq = W * adet * dot;
    } else {
      gq = W * (gu[0] * gv[0] + gu[1] * gv[1] + gu[2] * gv[2]);
    }
    if (A.grad) ((double*)A.grad)[e * Q + k] = gq;
    part[k] = (A.kappa ? A.kappa[e * Q + k] : 1.0) * gq;
  }
  if (A.partial) {
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int k = 0; k < Q; ++k) s += part[k];   // fixed order
      A.partial[A.partial_offset + e] = s;
    }
  }
}

template <typename K>
cudaError_t set_smem(K kern, size_t smem) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

cudaError_t launch_sumfact_gen(const ElemArgs& a, const PatchDev& ph, cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  const Shape S = make_shape(ph);
  const bool gen = a.jac != nullptr;
  SfLayout L = sf_layout(S, gen, true);
  bool dsmem = (size_t)L.total * 8 <= kGenSmemMax;
  if (!dsmem) L = sf_layout(S, gen, false);
  const size_t smem = (size_t)L.total * 8;
  if (smem > kGenSmemMax) return cudaErrorInvalidValue;
  cudaError_t e;
#define RUN_SF(G, DS)                                                        \
  {                                                                          \
    auto k = k_sf_gen<G, DS>;                                                \
    e = set_smem(k, smem);                   \
    if (e != cudaSuccess) return e;                                          \
    k<<<(unsigned)a.n_elem, kGenThreads, smem, st>>>(a, S, L);               \
  }
  if (gen && dsmem) RUN_SF(true, true)
  else if (gen) RUN_SF(true, false)
  else if (dsmem) RUN_SF(false, true)
  else RUN_SF(false, false)
#undef RUN_SF
  return cudaGetLastError();
}

cudaError_t launch_classical_gen(const ElemArgs& a, const PatchDev& ph, cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  const Shape S = make_shape(ph);
  // quadrature tile: 8 N QT doubles of tables, 11 QT of geometry
  int QT = S.Q < 64 ? S.Q : 64;
  while (QT > 1 && (size_t)8 * (S.rsum + 8 * (size_t)S.N * QT + 11 * QT) > kGenSmemMax) --QT;
  const size_t smem = (size_t)8 * (S.rsum + 8 * (size_t)S.N * QT + 11 * QT);
  if (smem > kGenSmemMax) return cudaErrorInvalidValue;
  cudaError_t e;
  if (a.jac) {
    e = set_smem(k_cl_gen<true>, smem);
    if (e != cudaSuccess) return e;
    k_cl_gen<true><<<(unsigned)a.n_elem, kGenThreads, smem, st>>>(a, S, QT);
  } else {
    e = set_smem(k_cl_gen<false>, smem);
    if (e != cudaSuccess) return e;
    k_cl_gen<false><<<(unsigned)a.n_elem, kGenThreads, smem, st>>>(a, S, QT);
  }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_gen(const AdjArgs& a, const PatchDev& ph, cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  const Shape S = make_shape(ph);
  const AdjLayout L = adj_layout(S);
  const size_t smem = (size_t)L.total * 8;
  if (smem > kGenSmemMax) return cudaErrorInvalidValue;
  cudaError_t e = set_smem(k_adj_gen, smem);
  if (e != cudaSuccess) return e;
  k_adj_gen<<<(unsigned)a.n_elem, kGenThreads, smem, st>>>(a, S, L, ph.pk[0], ph.pk[1],
                                                           ph.dim == 3 ? ph.pk[2] : 0);
  return cudaGetLastError();
}

}  // namespace iga
