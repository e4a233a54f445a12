// k_sumfact64.cu -- FP64 sum-factorized element matrices (Sec. 3.2,
// Algorithm 2; eqs. finalsum and bufferC), generalised from the Gram matrix
// to the variable-coefficient stiffness.
//
// Each integrand term is a product of one 1D factor per direction (value or
// derivative of the test function a_k and of the trial function b_k at the
// Gauss point) and a coefficient at the quadrature point.  With
//   D = w |det G| kappa G^{-1} G^{-T}  (symmetric),  D_M = w |det G| rho,
// the stiffness is sum_{i,j} D_ij d_i phi_a d_j phi_b and the mass D_M phi_a phi_b.
// Per direction and pair (a_k, b_k) the four 1D factor patterns are
//   P00 = v_a v_b, P11 = d_a d_b, P10 = d_a v_b, P01 = v_a d_b = P10^T.
// Algorithm 2's order is kept: contract the last direction first (stage 1,
// buffer D of the paper, here T1), then the middle one (stage 2, buffer C),
// then x (stage 3, the element matrix).  Exact symmetries are used to skip
// work that the paper's loops would repeat:
//   * D_ij = D_ji, so the (1,2)/(2,1) and (0,2)/(2,0) stage-1 buffers are
//     transposes of one another (one is computed);
//   * stage-1 buffers of symmetric patterns are symmetric in (a3,b3), and the
//     stage-2 buffers C11, C00 and C_M are symmetric in (a',b'), a' = (a2,a3);
//   * the x-pattern (0,1) buffer is the transpose of the (1,0) one;
//   * the element matrices are symmetric: only a <= b is computed and both
//     (a,b) and (b,a) are stored.
// With identity geometry (jac == NULL) D is diagonal with D00 = D11 = D22,
// so the off-diagonal terms vanish identically and are not formed.
#include <cstdio>

#include "iga_internal.h"

namespace iga {
namespace {

template <int P, int QG, bool GEN>
struct SF3 {
  static constexpr int n = P + 1, q = QG, Q = q * q * q, n2 = n * n, N = n2 * n;
  static constexpr int NS1 = n * (n + 1) / 2;   // symmetric (a3<=b3) pairs
  static constexpr int Np = n2;                  // a' = a2 + n a3
  static constexpr int NSp = Np * (Np + 1) / 2;  // symmetric (a'<=b') pairs
  static constexpr int NT = (N >= 64) ? 256 : 128;
  // stage-1 buffers: GEN: z00*{D00,D11,D01,DM}, z11*D22 (symmetric), z01*{D02,D12}
  //                  identity: z00*Dk, z00*DM, z11*Dk
  static constexpr int NSYM = GEN ? 5 : 3;
  static constexpr int NFULL = GEN ? 2 : 0;
  static constexpr int NT1 = NSYM + NFULL;
  static constexpr int NCOEF = GEN ? 7 : 2;
  static constexpr int T_00 = 0, T_11 = GEN ? 1 : 0, T_01 = 2, T_M = GEN ? 3 : 1,
                       T_22 = GEN ? 4 : 2, T_02 = 5, T_12 = 6;
  static constexpr int REC = 2 * q * n + q;
  static constexpr size_t doubles(int qc) {
    return (size_t)3 * REC + 3 * 3 * n2 * q + (size_t)NCOEF * Q + (size_t)NT1 * n2 * qc * q +
           (size_t)3 * NSp * q + (GEN ? (size_t)Np * Np * q : 0);
  }
  static constexpr int QC = (doubles(q) * 8 <= 112 * 1024) ? q : 1;
  static constexpr size_t smem = doubles(QC) * 8 + (size_t)(NSp + NS1) * 4;
};

// term -> (z pattern, coefficient) of stage 1; z pattern 0 = P00, 1 = P11, 2 = P01
template <bool GEN>
__device__ __forceinline__ void t1_term(int t, int& zp, int& c) {
  if (GEN) {
    zp = t < 4 ? 0 : (t == 4 ? 1 : 2);
    c = t;
  } else {
    zp = t == 2 ? 1 : 0;
    c = t == 1 ? 1 : 0;
  }
}

template <int P, int QG, bool GEN>
__global__ void __launch_bounds__(SF3<P, QG, GEN>::NT)
    k_sf3_f64(const ElemArgs A) {
  using C = SF3<P, QG, GEN>;
  constexpr int n = C::n, q = C::q, Q = C::Q, n2 = C::n2, N = C::N, NS1 = C::NS1,
                Np = C::Np, NSp = C::NSp, NT = C::NT, QC = C::QC, REC = C::REC;
  extern __shared__ __align__(16) double sm[];
  double* rec = sm;                          // [3][REC]
  double* pat = rec + 3 * REC;               // [dir][3 patterns][n][n][q]
  double* coef = pat + 3 * 3 * n2 * q;       // [NCOEF][Q]
  double* T1 = coef + C::NCOEF * Q;          // [NT1][n][n][QC][q]
  double* Cs = T1 + C::NT1 * n2 * QC * q;    // [3: C11,C00,CM][NSp][q]
  double* C10 = Cs + 3 * NSp * q;            // [Np][Np][q]   (GEN only)
  int* pairs = (int*)(C10 + (GEN ? Np * Np * q : 0));  // [NSp] packed (a'<<16 | b')
  int* pairs1 = pairs + NSp;                 // [NS1] packed (a3<<8 | b3)

  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  int e1, e2, e3;
  elem_coords(A, e, e1, e2, e3);

  // ---- basis records of the three directions, pair tables ----------------
  for (int i = tid; i < 3 * REC; i += NT) {
    const int d = i / REC, j = i - d * REC;
    const int ek = d == 0 ? e1 : (d == 1 ? e2 : e3);
    const double* tb = d == 0 ? A.tab[0] : (d == 1 ? A.tab[1] : A.tab[2]);
    rec[i] = tb[(int64_t)ek * REC + j];
  }
  for (int i = tid; i < NSp; i += NT) {
    int a = 0, r = i;
    while (r >= Np - a) { r -= Np - a; ++a; }
    pairs[i] = (a << 16) | (a + r);
  }
  for (int i = tid; i < NS1; i += NT) {
    int a = 0, r = i;
    while (r >= n - a) { r -= n - a; ++a; }
    pairs1[i] = (a << 8) | (a + r);
  }
  __syncthreads();

  // ---- per-direction 1D factor patterns: P00, P11, P10 ----------------------
  for (int i = tid; i < 3 * 3 * n2 * q; i += NT) {
    const int k = i % q;
    const int b = (i / q) % n;
    const int a = (i / (q * n)) % n;
    const int pt = (i / (q * n2)) % 3;
    const int d = i / (3 * q * n2);
    const double* v = rec + d * REC;
    const double* dv = v + q * n;
    double x;
    if (pt == 0) x = v[k * n + a] * v[k * n + b];
    else if (pt == 1) x = dv[k * n + a] * dv[k * n + b];
    else x = dv[k * n + a] * v[k * n + b];
    pat[i] = x;
  }

  // ---- coefficients at the quadrature points (the J(x^n) of eq. 10) -------
  for (int k = tid; k < Q; k += NT) {
    const int k1 = k % q, k2 = (k / q) % q, k3 = k / (q * q);
    const double* w0 = rec + 2 * q * n;
    const double W = w0[k1] * (w0 + REC)[k2] * (w0 + 2 * REC)[k3];
    const double kap = A.kappa ? A.kappa[e * Q + k] : 1.0;
    const double rh = A.rho ? A.rho[e * Q + k] : 1.0;
    if (GEN) {
      const double* G = A.jac + (e * Q + k) * 9;
      const double g00 = G[0], g01 = G[1], g02 = G[2], g10 = G[3], g11 = G[4], g12 = G[5],
                   g20 = G[6], g21 = G[7], g22 = G[8];
      // cofactors c_ij of G; G^{-1} = c^T / det
      const double c00 = g11 * g22 - g12 * g21, c01 = g12 * g20 - g10 * g22,
                   c02 = g10 * g21 - g11 * g20;
      const double c10 = g02 * g21 - g01 * g22, c11 = g00 * g22 - g02 * g20,
                   c12 = g01 * g20 - g00 * g21;
      const double c20 = g01 * g12 - g02 * g11, c21 = g02 * g10 - g00 * g12,
                   c22 = g00 * g11 - g01 * g10;
      const double det = g00 * c00 + g01 * c01 + g02 * c02;
      const double adet = fabs(det);
      // D = W kappa |det| G^{-1} G^{-T} = (W kappa / |det|) c^T c
      const double s = W * kap / adet;
      coef[0 * Q + k] = s * (c00 * c00 + c10 * c10 + c20 * c20);  // D00
      coef[1 * Q + k] = s * (c01 * c01 + c11 * c11 + c21 * c21);  // D11
      coef[2 * Q + k] = s * (c00 * c01 + c10 * c11 + c20 * c21);  // D01
      coef[3 * Q + k] = W * adet * rh;                             // DM
      coef[4 * Q + k] = s * (c02 * c02 + c12 * c12 + c22 * c22);  // D22
      coef[5 * Q + k] = s * (c00 * c02 + c10 * c12 + c20 * c22);  // D02
      coef[6 * Q + k] = s * (c01 * c02 + c11 * c12 + c21 * c22);  // D12
    } else {
      coef[0 * Q + k] = W * kap;
      coef[1 * Q + k] = W * rh;
    }
  }
  __syncthreads();

  const double* Pz = pat + 2 * 3 * n2 * q;
  const double* Py = pat + 1 * 3 * n2 * q;
  const double* Px = pat;

  for (int c0 = 0; c0 < q; c0 += QC) {
    // ---- stage 1: T1[t][a3][b3][q1][q2] = sum_k3 Z[a3][b3][k3] D_t[q1,q2,k3] ----
    constexpr int nsym_items = C::NSYM * NS1 * QC * q;
    constexpr int n_items1 = nsym_items + C::NFULL * n2 * QC * q;
    for (int it = tid; it < n_items1; it += NT) {
      int t, a3, b3, r;
      if (it < nsym_items) {
        t = it / (NS1 * QC * q);
        r = it - t * (NS1 * QC * q);
        const int pr = pairs1[r / (QC * q)];
        a3 = pr >> 8; b3 = pr & 255;
        r %= QC * q;
      } else {
        const int j = it - nsym_items;
        t = C::NSYM + j / (n2 * QC * q);
        r = j % (n2 * QC * q);
        const int ab = r / (QC * q);
        a3 = ab / n; b3 = ab % n;
        r %= QC * q;
      }
      const int q1c = r / q, q2 = r % q;
      int zp, ci;
      t1_term<GEN>(t, zp, ci);
      const double* D = coef + ci * Q + (c0 + q1c) + q * q2;
      double acc = 0.0;
      if (zp < 2) {
        const double* Z = Pz + zp * n2 * q + (a3 * n + b3) * q;
#pragma unroll
        for (int k3 = 0; k3 < q; ++k3) acc = fma(Z[k3], D[q * q * k3], acc);
      } else {  // P01[a3][b3] = P10[b3][a3]
        const double* Z = Pz + 2 * n2 * q + (b3 * n + a3) * q;
#pragma unroll
        for (int k3 = 0; k3 < q; ++k3) acc = fma(Z[k3], D[q * q * k3], acc);
      }
      T1[((t * n2 + a3 * n + b3) * QC + q1c) * q + q2] = acc;
      if (t < C::NSYM && a3 != b3) T1[((t * n2 + b3 * n + a3) * QC + q1c) * q + q2] = acc;
    }
    __syncthreads();

    // ---- stage 2: C^X[a'][b'][q1] = sum_k2 (y factors) T1 ----------------------
    constexpr int n_sym2 = 3 * NSp * QC;
    constexpr int n_items2 = n_sym2 + (GEN ? Np * Np * QC : 0);
    for (int it = tid; it < n_items2; it += NT) {
      if (it < n_sym2) {
        const int X = it / (NSp * QC);
        const int r = it - X * (NSp * QC);
        const int pp = r / QC, q1c = r % QC;
        const int pr = pairs[pp];
        const int ap = pr >> 16, bp = pr & 0xffff;
        const int a2 = ap % n, a3 = ap / n, b2 = bp % n, b3 = bp / n;
        const double* y00 = Py + (a2 * n + b2) * q;
        const double* y11 = Py + n2 * q + (a2 * n + b2) * q;
        auto t1 = [&](int t, int x3, int y3) -> const double* {
          return T1 + ((t * n2 + x3 * n + y3) * QC + q1c) * q;
        };
        double acc = 0.0;
        if (X == 0) {  // C11: x pattern (1,1) <- term (0,0)
          const double* T = t1(C::T_00, a3, b3);
#pragma unroll
          for (int k2 = 0; k2 < q; ++k2) acc = fma(y00[k2], T[k2], acc);
        } else if (X == 1) {  // C00: terms (1,1), (2,2), (1,2), (2,1)
          const double* Ta = t1(C::T_11, a3, b3);
          const double* Tb = t1(C::T_22, a3, b3);
#pragma unroll
          for (int k2 = 0; k2 < q; ++k2) {
            acc = fma(y11[k2], Ta[k2], acc);
            acc = fma(y00[k2], Tb[k2], acc);
          }
          if (GEN) {
            const double* y10 = Py + 2 * n2 * q + (a2 * n + b2) * q;
            const double* y01 = Py + 2 * n2 * q + (b2 * n + a2) * q;
            const double* Tc = t1(C::T_12, a3, b3);
            const double* Td = t1(C::T_12, b3, a3);
#pragma unroll
            for (int k2 = 0; k2 < q; ++k2) {
              acc = fma(y10[k2], Tc[k2], acc);
              acc = fma(y01[k2], Td[k2], acc);
            }
          }
        } else {  // CM: mass
          const double* T = t1(C::T_M, a3, b3);
#pragma unroll
          for (int k2 = 0; k2 < q; ++k2) acc = fma(y00[k2], T[k2], acc);
        }
        Cs[(X * NSp + pp) * q + c0 + q1c] = acc;
      } else if (GEN) {
        // C10: x pattern (1,0) <- terms (0,1) [y01, z00, D01] and (0,2) [y00, z01, D02]
        const int r = it - n_sym2;
        const int ab = r / QC, q1c = r % QC;
        const int ap = ab / Np, bp = ab % Np;
        const int a2 = ap % n, a3 = ap / n, b2 = bp % n, b3 = bp / n;
        const double* y00 = Py + (a2 * n + b2) * q;
        const double* y01 = Py + 2 * n2 * q + (b2 * n + a2) * q;
        const double* Ta = T1 + ((C::T_01 * n2 + a3 * n + b3) * QC + q1c) * q;
        const double* Tb = T1 + ((C::T_02 * n2 + a3 * n + b3) * QC + q1c) * q;
        double acc = 0.0;
#pragma unroll
        for (int k2 = 0; k2 < q; ++k2) {
          acc = fma(y01[k2], Ta[k2], acc);
          acc = fma(y00[k2], Tb[k2], acc);
        }
        C10[(ap * Np + bp) * q + c0 + q1c] = acc;
      }
    }
    __syncthreads();
  }

  // ---- stage 3: element matrices, a <= b, both triangles stored -------------
  double* Ke = A.K_out ? (double*)A.K_out + e * (int64_t)N * N : nullptr;
  double* Me = A.M_out ? (double*)A.M_out + e * (int64_t)N * N : nullptr;
  const double* x00 = Px;
  const double* x11 = Px + n2 * q;
  const double* x10 = Px + 2 * n2 * q;
  for (int it = tid; it < NSp * n; it += NT) {
    const int pp = it / n, a1 = it % n;
    const int pr = pairs[pp];
    const int ap = pr >> 16, bp = pr & 0xffff;
    double c11[q], c00[q], cM[q], c10[q], c01[q];
#pragma unroll
    for (int k = 0; k < q; ++k) {
      c11[k] = Cs[(0 * NSp + pp) * q + k];
      c00[k] = Cs[(1 * NSp + pp) * q + k];
      cM[k] = Cs[(2 * NSp + pp) * q + k];
      if (GEN) {
        c10[k] = C10[(ap * Np + bp) * q + k];
        c01[k] = C10[(bp * Np + ap) * q + k];
      }
    }
    const int b1s = (ap == bp) ? a1 : 0;
    const int64_t rowa = (int64_t)(a1 + n * ap) * N;
    for (int b1 = b1s; b1 < n; ++b1) {
      const int64_t rowb = (int64_t)(b1 + n * bp) * N;
      if (Ke) {
        const double* p11 = x11 + (a1 * n + b1) * q;
        const double* p00 = x00 + (a1 * n + b1) * q;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < q; ++k) {
          acc = fma(p11[k], c11[k], acc);
          acc = fma(p00[k], c00[k], acc);
        }
        if (GEN) {
          const double* p10 = x10 + (a1 * n + b1) * q;
          const double* p01 = x10 + (b1 * n + a1) * q;
#pragma unroll
          for (int k = 0; k < q; ++k) {
            acc = fma(p10[k], c10[k], acc);
            acc = fma(p01[k], c01[k], acc);
          }
        }
        Ke[rowa + b1 + n * bp] = acc;
        Ke[rowb + a1 + n * ap] = acc;
      }
      if (Me) {
        const double* p00 = x00 + (a1 * n + b1) * q;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < q; ++k) acc = fma(p00[k], cM[k], acc);
        Me[rowa + b1 + n * bp] = acc;
        Me[rowb + a1 + n * ap] = acc;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// 2D: stage 1 contracts y, stage 2 contracts x.
// ---------------------------------------------------------------------------
template <int P, int QG, bool GEN>
struct SF2 {
  static constexpr int n = P + 1, q = QG, Q = q * q, n2 = n * n, N = n2;
  static constexpr int NS1 = n * (n + 1) / 2;
  static constexpr int NT = 128;
  static constexpr int REC = 2 * q * n + q;
  // T: [0] y00*D00 (C11), [1] y11*D11 (C00), [2] y00*DM (CM), [3] y01*D01 (C10, GEN)
  static constexpr int NTB = GEN ? 4 : 3;
  static constexpr int NCOEF = GEN ? 4 : 2;
  static constexpr size_t smem =
      8 * ((size_t)2 * REC + 2 * 3 * n2 * q + (size_t)NCOEF * Q + (size_t)NTB * n2 * q) +
      4 * (size_t)NS1;
};

template <int P, int QG, bool GEN>
__global__ void __launch_bounds__(SF2<P, QG, GEN>::NT) k_sf2_f64(const ElemArgs A) {
  using C = SF2<P, QG, GEN>;
  constexpr int n = C::n, q = C::q, Q = C::Q, n2 = C::n2, N = C::N, NS1 = C::NS1, NT = C::NT,
                REC = C::REC;
  extern __shared__ __align__(16) double sm[];
  double* rec = sm;
  double* pat = rec + 2 * REC;          // [dir][3][n][n][q]
  double* coef = pat + 2 * 3 * n2 * q;  // [NCOEF][Q]: D00, D11, DM, D01
  double* T = coef + C::NCOEF * Q;      // [NTB][n][n][q]
  int* pairs1 = (int*)(T + C::NTB * n2 * q);
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  int e1, e2;
  elem_coords2(A, e, e1, e2);
  for (int i = tid; i < 2 * REC; i += NT) {
    const int d = i / REC, j = i - d * REC;
    const double* tb = d == 0 ? A.tab[0] : A.tab[1];
    rec[i] = tb[(int64_t)(d == 0 ? e1 : e2) * REC + j];
  }
  for (int i = tid; i < NS1; i += NT) {
    int a = 0, r = i;
    while (r >= n - a) { r -= n - a; ++a; }
    pairs1[i] = (a << 8) | (a + r);
  }
  __syncthreads();
  for (int i = tid; i < 2 * 3 * n2 * q; i += NT) {
    const int k = i % q, b = (i / q) % n, a = (i / (q * n)) % n, pt = (i / (q * n2)) % 3,
              d = i / (3 * q * n2);
    const double* v = rec + d * REC;
    const double* dv = v + q * n;
    pat[i] = pt == 0 ? v[k * n + a] * v[k * n + b]
                     : (pt == 1 ? dv[k * n + a] * dv[k * n + b] : dv[k * n + a] * v[k * n + b]);
  }
  for (int k = tid; k < Q; k += NT) {
    const int k1 = k % q, k2 = k / q;
    const double* w0 = rec + 2 * q * n;
    const double W = w0[k1] * (w0 + REC)[k2];
    const double kap = A.kappa ? A.kappa[e * Q + k] : 1.0;
    const double rh = A.rho ? A.rho[e * Q + k] : 1.0;
    if (GEN) {
      const double* G = A.jac + (e * Q + k) * 4;
      const double det = G[0] * G[3] - G[1] * G[2];
      const double adet = fabs(det);
      // G^{-1} = [[g11, -g01], [-g10, g00]] / det; D = (W kappa / |det|) adj adj^T
      const double s = W * kap / adet;
      coef[0 * Q + k] = s * (G[3] * G[3] + G[1] * G[1]);
      coef[1 * Q + k] = s * (G[2] * G[2] + G[0] * G[0]);
      coef[2 * Q + k] = W * adet * rh;
      coef[3 * Q + k] = -s * (G[3] * G[2] + G[1] * G[0]);
    } else {
      coef[0 * Q + k] = W * kap;
      coef[1 * Q + k] = W * rh;
    }
  }
  __syncthreads();
  const double* Py = pat + 3 * n2 * q;
  const double* Px = pat;
  // stage 1: T[t][a2][b2][q1] = sum_k2 Y[a2][b2][k2] D_t[q1 + q k2]
  constexpr int nsym = 3 * NS1 * q;
  constexpr int nitems = nsym + (GEN ? n2 * q : 0);
  for (int it = tid; it < nitems; it += NT) {
    if (it < nsym) {
      const int t = it / (NS1 * q);
      const int r = it - t * NS1 * q;
      const int pr = pairs1[r / q];
      const int a2 = pr >> 8, b2 = pr & 255, q1 = r % q;
      const double* Y = Py + (t == 1 ? n2 * q : 0) + (a2 * n + b2) * q;
      const int ci = GEN ? t : (t == 1 ? 0 : (t == 2 ? 1 : 0));
      const double* D = coef + ci * Q + q1;
      double acc = 0.0;
#pragma unroll
      for (int k2 = 0; k2 < q; ++k2) acc = fma(Y[k2], D[q * k2], acc);
      T[(t * n2 + a2 * n + b2) * q + q1] = acc;
      T[(t * n2 + b2 * n + a2) * q + q1] = acc;
    } else {
      const int r = it - nsym;
      const int ab = r / q, q1 = r % q;
      const int a2 = ab / n, b2 = ab % n;
      const double* Y = Py + 2 * n2 * q + (b2 * n + a2) * q;  // P01 = P10^T
      const double* D = coef + 3 * Q + q1;
      double acc = 0.0;
#pragma unroll
      for (int k2 = 0; k2 < q; ++k2) acc = fma(Y[k2], D[q * k2], acc);
      T[(3 * n2 + a2 * n + b2) * q + q1] = acc;
    }
  }
  __syncthreads();
  // stage 2: K[a][b], a <= b
  double* Ke = A.K_out ? (double*)A.K_out + e * (int64_t)N * N : nullptr;
  double* Me = A.M_out ? (double*)A.M_out + e * (int64_t)N * N : nullptr;
  for (int it = tid; it < NS1 * n; it += NT) {
    const int pp = it / n, a1 = it % n;
    const int pr = pairs1[pp];
    const int a2 = pr >> 8, b2 = pr & 255;
    const int b1s = (a2 == b2) ? a1 : 0;
    for (int b1 = b1s; b1 < n; ++b1) {
      const int a = a1 + n * a2, b = b1 + n * b2;
      if (Ke) {
        const double* p11 = Px + n2 * q + (a1 * n + b1) * q;
        const double* p00 = Px + (a1 * n + b1) * q;
        const double* c11 = T + (0 * n2 + a2 * n + b2) * q;
        const double* c00 = T + (1 * n2 + a2 * n + b2) * q;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < q; ++k) {
          acc = fma(p11[k], c11[k], acc);
          acc = fma(p00[k], c00[k], acc);
        }
        if (GEN) {
          const double* p10 = Px + 2 * n2 * q + (a1 * n + b1) * q;
          const double* p01 = Px + 2 * n2 * q + (b1 * n + a1) * q;
          const double* c10 = T + (3 * n2 + a2 * n + b2) * q;
          const double* c01 = T + (3 * n2 + b2 * n + a2) * q;
#pragma unroll
          for (int k = 0; k < q; ++k) {
            acc = fma(p10[k], c10[k], acc);
            acc = fma(p01[k], c01[k], acc);
          }
        }
        Ke[(int64_t)a * N + b] = acc;
        Ke[(int64_t)b * N + a] = acc;
      }
      if (Me) {
        const double* p00 = Px + (a1 * n + b1) * q;
        const double* cM = T + (2 * n2 + a2 * n + b2) * q;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < q; ++k) acc = fma(p00[k], cM[k], acc);
        Me[(int64_t)a * N + b] = acc;
        Me[(int64_t)b * N + a] = acc;
      }
    }
  }
}

template <int P, int QG, bool GEN>
cudaError_t run3(const ElemArgs& a, cudaStream_t st) {
  using C = SF3<P, QG, GEN>;
  static_assert(C::smem <= 227 * 1024, "shared memory");
  auto k = k_sf3_f64<P, QG, GEN>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)a.n_elem, C::NT, C::smem, st>>>(a);
  return cudaGetLastError();
}

template <int P, int QG, bool GEN>
cudaError_t run2(const ElemArgs& a, cudaStream_t st) {
  using C = SF2<P, QG, GEN>;
  auto k = k_sf2_f64<P, QG, GEN>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)a.n_elem, C::NT, C::smem, st>>>(a);
  return cudaGetLastError();
}

template <int P, int QG>
cudaError_t run3g(const ElemArgs& a, cudaStream_t st) {
  return a.jac ? run3<P, QG, true>(a, st) : run3<P, QG, false>(a, st);
}
template <int P, int QG>
cudaError_t run2g(const ElemArgs& a, cudaStream_t st) {
  return a.jac ? run2<P, QG, true>(a, st) : run2<P, QG, false>(a, st);
}

}  // namespace

bool sumfact_f64_supported(int dim, int p, int q) {
  if (dim == 3) return p >= 1 && p <= 5 && (q == p + 1 || (q == p + 2 && p <= 4));
  if (dim == 2) return p >= 1 && p <= 8 && (q == p + 1 || q == p + 2);
  return false;
}

cudaError_t launch_sumfact_f64(const ElemArgs& a, int dim, int p, int q, cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  const int dq = q - p;
  if (dim == 3) {
#define C3(PP)                                          \
  if (p == PP && dq == 1) return run3g<PP, PP + 1>(a, st); \
  if (p == PP && dq == 2) return run3g<PP, PP + 2>(a, st);
    C3(1) C3(2) C3(3) C3(4)
    if (p == 5 && dq == 1) return run3g<5, 6>(a, st);
#undef C3
  } else {
#define C2(PP)                                          \
  if (p == PP && dq == 1) return run2g<PP, PP + 1>(a, st); \
  if (p == PP && dq == 2) return run2g<PP, PP + 2>(a, st);
    C2(1) C2(2) C2(3) C2(4) C2(5) C2(6) C2(7) C2(8)
#undef C2
  }
  return cudaErrorInvalidValue;
}

}  // namespace iga
