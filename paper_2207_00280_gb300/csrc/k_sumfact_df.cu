// k_sumfact_df.cu -- FP64-accurate sum factorization in float-float
// arithmetic, 3D (precision IGA_FP64_DF).
//
// Same terms, stages and symmetries as the FP64 kernel (Sec. 3.2, Algorithm 2
// generalised to the stiffness; see k_sumfact64.cu), but every working value
// is an unevaluated sum hi + lo of two FP32 numbers (about 48 significant
// bits) and every multiply-add runs on the FP32 pipes:
//   product a*b: p = a.hi*b.hi, its rounding error fma(a.hi, b.hi, -p) is
//   exact, plus the cross terms a.hi*b.lo + a.lo*b.hi (Dekker/Kahan with FMA);
//   sum: Knuth's two-sum of the high parts plus the low parts, renormalised.
// GB300 issues FP32 FMAs 64 times faster than FP64 ones, so this trades 12
// FP32 operations for one FP64 multiply-add.  The Jacobian cofactors and
// determinant, the weights times kappa and the conversions of the inputs and
// of the outputs (exact) use the otherwise idle FP64 pipe.
#include <cstdint>

#include "iga_internal.h"

namespace iga {
namespace {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = p + e;
  return {s, e - (s - p)};
}

// hi + lo as a double.  Both halves convert exactly and their sum has at most
// 48 significant bits, so the double addition is exact: three FP64-pipe
// instructions per warp of entries, on a pipe this kernel otherwise leaves idle.
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// Dot-product accumulator: the running sum s of the high products (kept exact
// by two-sum) and the running sum e of all low-order terms; one
// renormalisation at the end (12 FP32 operations per multiply-add).
struct dacc {
  float s, e;
};

__device__ __forceinline__ void acc_fma(dacc& A, df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = A.s + p;
  const float bb = s - A.s;
  const float err = (A.s - (s - bb)) + (p - bb);
  A.s = s;
  A.e += err + e;
}

__device__ __forceinline__ df acc_value(dacc A) {
  const float hi = A.s + A.e;
  return {hi, A.e - (hi - A.s)};
}

template <int P, int QG, bool GEN>
struct SFD {
  static constexpr int n = P + 1, q = QG, Q = q * q * q, n2 = n * n, N = n2 * n;
  static constexpr int NS1 = n * (n + 1) / 2;
  static constexpr int Np = n2;
  static constexpr int NSp = Np * (Np + 1) / 2;
  static constexpr int NT = (N >= 64) ? 256 : 128;
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

template <int P, int QG, bool GEN>
__global__ void __launch_bounds__(SFD<P, QG, GEN>::NT) k_sf3_df(const ElemArgs A) {
  using C = SFD<P, QG, GEN>;
  constexpr int n = C::n, q = C::q, Q = C::Q, n2 = C::n2, N = C::N, NS1 = C::NS1,
                Np = C::Np, NSp = C::NSp, NT = C::NT, QC = C::QC, REC = C::REC;
  extern __shared__ __align__(16) df smd[];
  df* rec = smd;                          // [3][REC]
  df* pat = rec + 3 * REC;                // [dir][3 patterns][n][n][q]
  df* coef = pat + 3 * 3 * n2 * q;        // [NCOEF][Q]
  df* T1 = coef + C::NCOEF * Q;           // [NT1][n][n][QC][q]
  df* Cs = T1 + C::NT1 * n2 * QC * q;     // [3: C11,C00,CM][NSp][q]
  df* C10 = Cs + 3 * NSp * q;             // [Np][Np][q]   (GEN only)
  int* pairs = (int*)(C10 + (GEN ? Np * Np * q : 0));
  int* pairs1 = pairs + NSp;

  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  int e1, e2, e3;
  elem_coords(A, e, e1, e2, e3);

  for (int i = tid; i < 3 * REC; i += NT) {
    const int d = i / REC, j = i - d * REC;
    const int ek = d == 0 ? e1 : (d == 1 ? e2 : e3);
    const double* tb = d == 0 ? A.tab[0] : (d == 1 ? A.tab[1] : A.tab[2]);
    rec[i] = df_make(tb[(int64_t)ek * REC + j]);
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

  // 1D factor patterns P00, P11, P10 in float-float
  for (int i = tid; i < 3 * 3 * n2 * q; i += NT) {
    const int k = i % q, b = (i / q) % n, a = (i / (q * n)) % n, pt = (i / (q * n2)) % 3,
              d = i / (3 * q * n2);
    const df* v = rec + d * REC;
    const df* dv = v + q * n;
    pat[i] = pt == 0 ? df_mul(v[k * n + a], v[k * n + b])
                     : (pt == 1 ? df_mul(dv[k * n + a], dv[k * n + b]) : df_mul(dv[k * n + a], v[k * n + b]));
  }
  // coefficients: weights times kappa (and the geometry) in FP64, then split
  for (int k = tid; k < Q; k += NT) {
    const int k1 = k % q, k2 = (k / q) % q, k3 = k / (q * q);
    const double W = A.tab[0][(int64_t)e1 * REC + 2 * q * n + k1] *
                     A.tab[1][(int64_t)e2 * REC + 2 * q * n + k2] *
                     A.tab[2][(int64_t)e3 * REC + 2 * q * n + k3];
    const double kap = A.kappa ? A.kappa[e * Q + k] : 1.0;
    const double rh = A.rho ? A.rho[e * Q + k] : 1.0;
    if (GEN) {
      const double* G = A.jac + (e * Q + k) * 9;
      const double g00 = G[0], g01 = G[1], g02 = G[2], g10 = G[3], g11 = G[4], g12 = G[5],
                   g20 = G[6], g21 = G[7], g22 = G[8];
      const double c00 = g11 * g22 - g12 * g21, c01 = g12 * g20 - g10 * g22,
                   c02 = g10 * g21 - g11 * g20;
      const double c10 = g02 * g21 - g01 * g22, c11 = g00 * g22 - g02 * g20,
                   c12 = g01 * g20 - g00 * g21;
      const double c20 = g01 * g12 - g02 * g11, c21 = g02 * g10 - g00 * g12,
                   c22 = g00 * g11 - g01 * g10;
      const double det = g00 * c00 + g01 * c01 + g02 * c02;
      const double adet = fabs(det);
      const double s = W * kap / adet;
      coef[0 * Q + k] = df_make(s * (c00 * c00 + c10 * c10 + c20 * c20));
      coef[1 * Q + k] = df_make(s * (c01 * c01 + c11 * c11 + c21 * c21));
      coef[2 * Q + k] = df_make(s * (c00 * c01 + c10 * c11 + c20 * c21));
      coef[3 * Q + k] = df_make(W * adet * rh);
      coef[4 * Q + k] = df_make(s * (c02 * c02 + c12 * c12 + c22 * c22));
      coef[5 * Q + k] = df_make(s * (c00 * c02 + c10 * c12 + c20 * c22));
      coef[6 * Q + k] = df_make(s * (c01 * c02 + c11 * c12 + c21 * c22));
    } else {
      coef[0 * Q + k] = df_make(W * kap);
      coef[1 * Q + k] = df_make(W * rh);
    }
  }
  __syncthreads();

  const df* Pz = pat + 2 * 3 * n2 * q;
  const df* Py = pat + 1 * 3 * n2 * q;
  const df* Px = pat;
  
  for (int c0 = 0; c0 < q; c0 += QC) {
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
      if (GEN) { zp = t < 4 ? 0 : (t == 4 ? 1 : 2); ci = t; }
      else { zp = t == 2 ? 1 : 0; ci = t == 1 ? 1 : 0; }
      const df* D = coef + ci * Q + (c0 + q1c) + q * q2;
      const df* Z = zp < 2 ? Pz + zp * n2 * q + (a3 * n + b3) * q : Pz + 2 * n2 * q + (b3 * n + a3) * q;
      dacc acc = {0.f, 0.f};
#pragma unroll
      for (int k3 = 0; k3 < q; ++k3) acc_fma(acc, Z[k3], D[q * q * k3]);
      const df v = acc_value(acc);
      T1[((t * n2 + a3 * n + b3) * QC + q1c) * q + q2] = v;
      if (t < C::NSYM && a3 != b3) T1[((t * n2 + b3 * n + a3) * QC + q1c) * q + q2] = v;
    }
    __syncthreads();
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
        const df* y00 = Py + (a2 * n + b2) * q;
        const df* y11 = Py + n2 * q + (a2 * n + b2) * q;
        auto t1 = [&](int t, int x3, int y3) -> const df* {
          return T1 + ((t * n2 + x3 * n + y3) * QC + q1c) * q;
        };
        dacc acc = {0.f, 0.f};
        if (X == 0) {
          const df* T = t1(C::T_00, a3, b3);
#pragma unroll
          for (int k2 = 0; k2 < q; ++k2) acc_fma(acc, y00[k2], T[k2]);
        } else if (X == 1) {
          const df* Ta = t1(C::T_11, a3, b3);
          const df* Tb = t1(C::T_22, a3, b3);
#pragma unroll
          for (int k2 = 0; k2 < q; ++k2) {
            acc_fma(acc, y11[k2], Ta[k2]);
            acc_fma(acc, y00[k2], Tb[k2]);
          }
          if (GEN) {
            const df* y10 = Py + 2 * n2 * q + (a2 * n + b2) * q;
            const df* y01 = Py + 2 * n2 * q + (b2 * n + a2) * q;
            const df* Tc = t1(C::T_12, a3, b3);
            const df* Td = t1(C::T_12, b3, a3);
#pragma unroll
            for (int k2 = 0; k2 < q; ++k2) {
              acc_fma(acc, y10[k2], Tc[k2]);
              acc_fma(acc, y01[k2], Td[k2]);
            }
          }
        } else {
          const df* T = t1(C::T_M, a3, b3);
#pragma unroll
          for (int k2 = 0; k2 < q; ++k2) acc_fma(acc, y00[k2], T[k2]);
        }
        Cs[(X * NSp + pp) * q + c0 + q1c] = acc_value(acc);
      } else if (GEN) {
        const int r = it - n_sym2;
        const int ab = r / QC, q1c = r % QC;
        const int ap = ab / Np, bp = ab % Np;
        const int a2 = ap % n, a3 = ap / n, b2 = bp % n, b3 = bp / n;
        const df* y00 = Py + (a2 * n + b2) * q;
        const df* y01 = Py + 2 * n2 * q + (b2 * n + a2) * q;
        const df* Ta = T1 + ((C::T_01 * n2 + a3 * n + b3) * QC + q1c) * q;
        const df* Tb = T1 + ((C::T_02 * n2 + a3 * n + b3) * QC + q1c) * q;
        dacc acc = {0.f, 0.f};
#pragma unroll
        for (int k2 = 0; k2 < q; ++k2) {
          acc_fma(acc, y01[k2], Ta[k2]);
          acc_fma(acc, y00[k2], Tb[k2]);
        }
        C10[(ap * Np + bp) * q + c0 + q1c] = acc_value(acc);
      }
    }
    __syncthreads();
  }

  double* Ke = A.K_out ? (double*)A.K_out + e * (int64_t)N * N : nullptr;
  double* Me = A.M_out ? (double*)A.M_out + e * (int64_t)N * N : nullptr;
  const df* x00 = Px;
  const df* x11 = Px + n2 * q;
  const df* x10 = Px + 2 * n2 * q;
  for (int it = tid; it < NSp * n; it += NT) {
    const int pp = it / n, a1 = it % n;
    const int pr = pairs[pp];
    const int ap = pr >> 16, bp = pr & 0xffff;
    df c11[q], c00[q], cM[q], c10[q], c01[q];
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
        const df* p11 = x11 + (a1 * n + b1) * q;
        const df* p00 = x00 + (a1 * n + b1) * q;
        dacc acc = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < q; ++k) {
          acc_fma(acc, p11[k], c11[k]);
          acc_fma(acc, p00[k], c00[k]);
        }
        if (GEN) {
          const df* p10 = x10 + (a1 * n + b1) * q;
          const df* p01 = x10 + (b1 * n + a1) * q;
#pragma unroll
          for (int k = 0; k < q; ++k) {
            acc_fma(acc, p10[k], c10[k]);
            acc_fma(acc, p01[k], c01[k]);
          }
        }
        const double v = df_to_double(acc_value(acc));
        Ke[rowa + b1 + n * bp] = v;
        Ke[rowb + a1 + n * ap] = v;
      }
      if (Me) {
        const df* p00 = x00 + (a1 * n + b1) * q;
        dacc acc = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < q; ++k) acc_fma(acc, p00[k], cM[k]);
        const double v = df_to_double(acc_value(acc));
        Me[rowa + b1 + n * bp] = v;
        Me[rowb + a1 + n * ap] = v;
      }
    }
  }
}

template <int P, int QG, bool GEN>
cudaError_t run3(const ElemArgs& a, cudaStream_t st) {
  using C = SFD<P, QG, GEN>;
  static_assert(C::smem <= 227 * 1024, "shared memory");
  auto k = k_sf3_df<P, QG, GEN>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)a.n_elem, C::NT, C::smem, st>>>(a);
  return cudaGetLastError();
}

template <int P, int QG>
cudaError_t run3g(const ElemArgs& a, cudaStream_t st) {
  return a.jac ? run3<P, QG, true>(a, st) : run3<P, QG, false>(a, st);
}

}  // namespace

bool sumfact_df_supported(int dim, int p, int q) {
  return dim == 3 && p >= 1 && p <= 5 && (q == p + 1 || (q == p + 2 && p <= 4));
}

cudaError_t launch_sumfact_df(const ElemArgs& a, int dim, int p, int q, cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  if (dim != 3) return cudaErrorInvalidValue;
  const int dq = q - p;
#define C3(PP)                                             \
  if (p == PP && dq == 1) return run3g<PP, PP + 1>(a, st); \
  if (p == PP && dq == 2) return run3g<PP, PP + 2>(a, st);
  C3(1) C3(2) C3(3) C3(4)
  if (p == 5 && dq == 1) return run3g<5, 6>(a, st);
#undef C3
  return cudaErrorInvalidValue;
}

}  // namespace iga
