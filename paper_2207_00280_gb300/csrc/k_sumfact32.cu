// k_sumfact32.cu -- FP32 and BF16 sum-factorized element matrices, 3D.
//
// Same integrand terms and stage order as the FP64 kernel (Sec. 3.2,
// Algorithm 2 generalised to the stiffness; see k_sumfact64.cu): stage 1
// contracts the last direction (k3), stage 2 the middle one (k2), stage 3 the
// first (k1).  Precision: the Jacobian cofactors and determinant are formed in
// FP64; D = w kappa / |det| c^T c, the 1D factor patterns and the three
// contractions run in FP32.  In the BF16 form the stage-3 contraction is a
// dense GEMM per element on the tensor cores (bf16 operands, FP32
// accumulation): rows (a',b'), columns (a1,b1), depth (x pattern, k1); the
// x-pattern operand is split into bf16 hi + lo parts.
//
// The FP32 stages are register-blocked: each thread keeps the operand that is
// reused (quadrature-point coefficients in stage 1, stage-1 buffers in stage
// 2, stage-2 buffers in stage 3) in registers and streams the 1D factor
// patterns from shared memory, laid out [a][b][pattern][k] so that stage 3
// reads them as broadcast float4 loads (one load feeds four FMAs).  Each
// element matrix is assembled in shared memory (upper triangle computed,
// mirrored there) and written with coalesced stores when it fits, else stored
// directly.  MODE: 0 = stiffness and mass, 1 = stiffness only, 2 = mass only.
#include <cuda_bf16.h>

#include "iga_internal.h"

namespace iga {
namespace {

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int P, int QG, bool GEN, int MODE, bool BF>
struct SF3F {
  static constexpr bool DK = MODE != 2, DM = MODE != 1;
  static constexpr int n = P + 1, q = QG, Q = q * q * q, n2 = n * n, N = n2 * n;
  static constexpr int NS1 = n * (n + 1) / 2;
  static constexpr int Np = n2;
  static constexpr int NSp = Np * (Np + 1) / 2;
  static constexpr int NT = 256;
  static constexpr int REC = 2 * q * n + q;
  static constexpr size_t al4(size_t x) { return (x + 3) / 4 * 4; }
  // pattern records, floats: x [a1][b1][4][q] (11, 00, 10, 01); y [a2][b2][4][q]
  // (00, 11, 10, 01); z [a3][b3][3][q] (00, 11, 01)
  static constexpr int RW = 4 * q;
  static constexpr size_t f_px = (size_t)n2 * RW, f_py = (size_t)n2 * RW, f_pz = al4((size_t)n2 * 3 * q);
  // coefficients [7][Q]: 0 D00, 1 D11, 2 D01, 3 DM, 4 D22, 5 D02, 6 D12 (identity: 0 = W kappa, 3 = W rho)
  static constexpr size_t f_coef = al4((size_t)7 * Q);
  // stage-1 buffers T[7][a3][b3][k1][k2] (same indices as the coefficients)
  static constexpr size_t f_T1 = al4((size_t)7 * n2 * q * q);
  // stage-2 buffers: FP32 form Cs [3: C11, C00, CM][NSp][q] and C10 [Np][Np][q]
  static constexpr size_t f_Cs32 = al4((size_t)3 * NSp * q);
  static constexpr size_t f_C10 = (GEN && !BF) ? al4((size_t)Np * Np * q) : 0;
  // BF16 form: GEMM operands A_K [MP][LDK], A_M [MP][LDM], B_K and B_M hi/lo
  static constexpr int al16i(int x) { return (x + 15) / 16 * 16; }
  static constexpr int NXK = GEN ? 4 : 2;
  static constexpr int KK = al16i(NXK * q), KM = al16i(q);
  static constexpr int LDK = KK + 8, LDM = KM + 8;
  static constexpr int MP = al16i(Np * Np);
  static constexpr int NPAD = (n2 + 7) / 8 * 8;
  static constexpr size_t h_A = (size_t)MP * ((DK ? LDK : 0) + (DM ? LDM : 0));
  static constexpr size_t h_B = (size_t)2 * NPAD * ((DK ? LDK : 0) + (DM ? LDM : 0));
  static constexpr size_t f_Cs = BF ? al4((h_A + h_B + 1) / 2) : f_Cs32;
  static constexpr size_t f_out = al4((size_t)N * N);
  static constexpr size_t d_geo = 3 * REC + 2 * (size_t)Q + (GEN ? 9 * (size_t)Q : 0);
  static constexpr size_t f_recf = al4(3 * REC);
  // aliased region: {T1, coef, geometry staging, FP32 records} until stage 2
  // ends, then the output stage
  static constexpr size_t f_alias = f_T1 + f_coef + 2 * d_geo + f_recf;
  static constexpr size_t f_fixed = f_px + f_py + f_pz + f_Cs + f_C10;
  static constexpr size_t f_pairs = al4((size_t)NSp);
  static constexpr bool STAGE =
      4 * (f_fixed + (f_alias > f_out ? f_alias : f_out) + f_pairs) <= 200 * 1024;
  static constexpr size_t f_region = al4((STAGE && f_out > f_alias) ? f_out : f_alias);
  static constexpr size_t smem = 4 * (f_fixed + f_region + f_pairs);
};

__device__ __forceinline__ void mma_bf16_16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Stage 3 of the BF16 form on the tensor cores: for one element,
//   OUT[(a',b')][(a1,b1)] = sum_k A[(a',b')][k] * (Bhi + Blo)[(a1,b1)][k],
// k = (x pattern, k1), FP32 accumulation, scattered to K[a1 + n a'][b1 + n b'].
// Warp w takes the 16-row tiles w, w+8, ...; the fragments follow the
// m16n8k16 register layout (row g = lane/4, column pair 2*(lane%4)).
template <class C, int LD, int KS>
__device__ __forceinline__ void gemm_scatter(const __nv_bfloat16* Am, const __nv_bfloat16* Bm,
                                             float* dst_stage, float* dst_global) {
  constexpr int n = C::n, N = C::N, Np = C::Np, NTN = C::NPAD / 8, MT = C::MP / 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  uint32_t bh[NTN][KS][2], bl[NTN][KS][2];
#pragma unroll
  for (int nt = 0; nt < NTN; ++nt)
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const __nv_bfloat16* r0 = Bm + (nt * 8 + g) * LD + ks * 16 + t * 2;
      const __nv_bfloat16* r1 = Bm + (C::NPAD + nt * 8 + g) * LD + ks * 16 + t * 2;
      bh[nt][ks][0] = *(const uint32_t*)r0;
      bh[nt][ks][1] = *(const uint32_t*)(r0 + 8);
      bl[nt][ks][0] = *(const uint32_t*)r1;
      bl[nt][ks][1] = *(const uint32_t*)(r1 + 8);
    }
  for (int mt = warp; mt < MT; mt += C::NT / 32) {
    uint32_t a[KS][4];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const __nv_bfloat16* r0 = Am + (mt * 16 + g) * LD + ks * 16 + t * 2;
      const __nv_bfloat16* r1 = r0 + 8 * LD;
      a[ks][0] = *(const uint32_t*)r0;
      a[ks][1] = *(const uint32_t*)r1;
      a[ks][2] = *(const uint32_t*)(r0 + 8);
      a[ks][3] = *(const uint32_t*)(r1 + 8);
    }
#pragma unroll
    for (int nt = 0; nt < NTN; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        mma_bf16_16816(c, a[ks], bh[nt][ks]);
        mma_bf16_16816(c, a[ks], bl[nt][ks]);
      }
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int m = mt * 16 + g + (h >> 1) * 8;
        const int nn = nt * 8 + t * 2 + (h & 1);
        if (m < Np * Np && nn < n * n) {
          const int ap = m / Np, bp = m % Np, a1 = nn / n, b1 = nn % n;
          const int idx = (a1 + n * ap) * N + b1 + n * bp;
          if (C::STAGE) dst_stage[idx] = c[h];
          else dst_global[idx] = c[h];
        }
      }
    }
  }
}

// packed index of (a', b'), a' <= b', in the upper triangle of an Np x Np matrix
template <int Np>
__device__ __forceinline__ int upper_index(int ap, int bp) {
  return ap * Np - (ap * (ap - 1)) / 2 + (bp - ap);
}

// One element, all stages.  Called by the per-patch kernel (e = blockIdx.x)
// and by the persistent queue kernel.
template <int P, int QG, bool GEN, int MODE, bool BF>
__device__ __forceinline__ void sf3_f32_element(const ElemArgs& A, int64_t e, float* smf) {
  using C = SF3F<P, QG, GEN, MODE, BF>;
  constexpr int n = C::n, q = C::q, Q = C::Q, n2 = C::n2, N = C::N, NS1 = C::NS1,
                Np = C::Np, NSp = C::NSp, NT = C::NT, REC = C::REC, RW = C::RW;
  constexpr bool DK = C::DK, DM = C::DM;
  float* px = smf;                                   // [n2][4][q]
  float* py = px + C::f_px;                          // [n2][4][q]
  float* pz = py + C::f_py;                          // [n2][3][q]
  float* Cs = pz + C::f_pz;                          // [3][NSp][q]  (or the BF16 operands)
  float* C10 = Cs + C::f_Cs;                         // [Np][Np][q]
  float* region = C10 + C::f_C10;
  float* T1 = region;                                // [7][n2][q][q]
  float* coef = T1 + C::f_T1;                        // [7][Q]
  double* geo = (double*)(coef + C::f_coef);
  double* rec = geo;                                 // [3][REC]
  double* kap = rec + 3 * REC;                       // [Q]
  double* rho = kap + Q;                             // [Q]
  double* jac = rho + Q;                             // [Q][9]
  float* recf = (float*)(geo + C::d_geo);            // [3][REC]
  float* outs = region;                              // [N][N] after stage 2
  int* pairs = (int*)(region + C::f_region);         // [NSp] packed (a' << 16 | b')
  __nv_bfloat16* AK = (__nv_bfloat16*)Cs;
  __nv_bfloat16* AM = AK + (DK ? (size_t)C::MP * C::LDK : 0);
  __nv_bfloat16* BK = AM + (DM ? (size_t)C::MP * C::LDM : 0);
  __nv_bfloat16* BM = BK + (DK ? (size_t)2 * C::NPAD * C::LDK : 0);

  const int tid = threadIdx.x;
  const int e1 = (int)(e % A.K1);
  const int e2 = (int)((e / A.K1) % A.K2);
  const int e3 = (int)(e / ((int64_t)A.K1 * A.K2));
  __syncthreads();  // shared memory of the previous element is no longer read

  // ---- coalesced staging of this element's inputs --------------------------
  for (int i = tid; i < 3 * REC; i += NT) {
    const int d = i / REC, j = i - d * REC;
    const int ek = d == 0 ? e1 : (d == 1 ? e2 : e3);
    const double* tb = d == 0 ? A.tab[0] : (d == 1 ? A.tab[1] : A.tab[2]);
    rec[i] = tb[(int64_t)ek * REC + j];
  }
  for (int k = tid; k < Q; k += NT) {
    kap[k] = A.kappa ? A.kappa[e * Q + k] : 1.0;
    rho[k] = A.rho ? A.rho[e * Q + k] : 1.0;
  }
  if (GEN) {
    const double* G = A.jac + e * Q * 9;
    for (int i = tid; i < 9 * Q; i += NT) jac[i] = G[i];
  }
  for (int i = tid; i < NSp; i += NT) {
    int a = 0, r = i;
    while (r >= Np - a) { r -= Np - a; ++a; }
    pairs[i] = (a << 16) | (a + r);
  }
  __syncthreads();
  for (int i = tid; i < 3 * REC; i += NT) recf[i] = (float)rec[i];
  __syncthreads();

  // ---- 1D factor pattern records in FP32 ---------------------------------------
  for (int i = tid; i < n2 * q; i += NT) {
    const int a = i / (n * q), b = (i / q) % n, k = i % q;
    const int ab = a * n + b;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float* v = recf + d * REC;
      const float* dv = v + q * n;
      const float va = v[k * n + a], vb = v[k * n + b], da = dv[k * n + a], db = dv[k * n + b];
      if (d == 0) {
        float* r = px + ab * RW;
        r[0 * q + k] = da * db; r[1 * q + k] = va * vb; r[2 * q + k] = da * vb; r[3 * q + k] = va * db;
      } else if (d == 1) {
        float* r = py + ab * RW;
        r[0 * q + k] = va * vb; r[1 * q + k] = da * db; r[2 * q + k] = da * vb; r[3 * q + k] = va * db;
      } else {
        float* r = pz + ab * 3 * q;
        r[0 * q + k] = va * vb; r[1 * q + k] = da * db; r[2 * q + k] = va * db;
      }
    }
  }
  // ---- coefficients: cofactors and determinant in FP64, the rest in FP32 ------
  for (int k = tid; k < Q; k += NT) {
    const int k1 = k % q, k2 = (k / q) % q, k3 = k / (q * q);
    const float* w0 = recf + 2 * q * n;
    const float W = w0[k1] * (w0 + REC)[k2] * (w0 + 2 * REC)[k3];
    const float kp = (float)kap[k], rh = (float)rho[k];
    if (GEN) {
      const double* G = jac + 9 * k;
      const double g00 = G[0], g01 = G[1], g02 = G[2], g10 = G[3], g11 = G[4], g12 = G[5],
                   g20 = G[6], g21 = G[7], g22 = G[8];
      const double d00 = g11 * g22 - g12 * g21, d01 = g12 * g20 - g10 * g22,
                   d02 = g10 * g21 - g11 * g20;
      const double det = g00 * d00 + g01 * d01 + g02 * d02;
      const float c00 = (float)d00, c01 = (float)d01, c02 = (float)d02;
      const float c10 = (float)(g02 * g21 - g01 * g22), c11 = (float)(g00 * g22 - g02 * g20),
                  c12 = (float)(g01 * g20 - g00 * g21);
      const float c20 = (float)(g01 * g12 - g02 * g11), c21 = (float)(g02 * g10 - g00 * g12),
                  c22 = (float)(g00 * g11 - g01 * g10);
      const float adet = (float)fabs(det);
      const float s = W * kp / adet;
      coef[0 * Q + k] = s * (c00 * c00 + c10 * c10 + c20 * c20);
      coef[1 * Q + k] = s * (c01 * c01 + c11 * c11 + c21 * c21);
      coef[2 * Q + k] = s * (c00 * c01 + c10 * c11 + c20 * c21);
      coef[3 * Q + k] = W * adet * rh;
      coef[4 * Q + k] = s * (c02 * c02 + c12 * c12 + c22 * c22);
      coef[5 * Q + k] = s * (c00 * c02 + c10 * c12 + c20 * c22);
      coef[6 * Q + k] = s * (c01 * c02 + c11 * c12 + c21 * c22);
    } else {
      coef[0 * Q + k] = W * kp;
      coef[3 * Q + k] = W * rh;
    }
  }
  if constexpr (BF) {
    // zero every GEMM operand (padding rows and columns must be zero)
    uint32_t* z = (uint32_t*)Cs;
    for (size_t i = tid; i < (C::h_A + C::h_B) / 2; i += NT) z[i] = 0u;
  }
  __syncthreads();

  if constexpr (BF) {
    // B operand: x patterns split into bf16 hi + lo, B[(a1,b1)][X q + k1]
    if (DK) {
      for (int i = tid; i < n2 * C::NXK * q; i += NT) {
        const int nn = i / (C::NXK * q), kx = i % (C::NXK * q);
        const float v = px[nn * RW + kx];  // record order 11, 00, 10, 01 matches X
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        BK[nn * C::LDK + kx] = hi;
        BK[(C::NPAD + nn) * C::LDK + kx] = __float2bfloat16_rn(v - __bfloat162float(hi));
      }
    }
    if (DM) {
      for (int i = tid; i < n2 * q; i += NT) {
        const int nn = i / q, k1 = i % q;
        const float v = px[nn * RW + q + k1];
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        BM[nn * C::LDM + k1] = hi;
        BM[(C::NPAD + nn) * C::LDM + k1] = __float2bfloat16_rn(v - __bfloat162float(hi));
      }
    }
  }

  // ---- stage 1: T_t[a3][b3][k1][k2] = sum_k3 Z_t[a3][b3][k3] D_t[k1,k2,k3] -------
  // item = (k1, k2, a3), coefficients of the item in registers, loop over b3
  for (int it = tid; it < q * q * n; it += NT) {
    const int a3 = it % n, kk = it / n;  // kk = k1 + q k2
    float d0[q], d1[q], d2[q], d3[q], d4[q], d5[q], d6[q];
#pragma unroll
    for (int k3 = 0; k3 < q; ++k3) {
      const int o = kk + q * q * k3;
      d0[k3] = coef[0 * Q + o];
      d3[k3] = coef[3 * Q + o];
      if (GEN) {
        d1[k3] = coef[1 * Q + o]; d2[k3] = coef[2 * Q + o]; d4[k3] = coef[4 * Q + o];
        d5[k3] = coef[5 * Q + o]; d6[k3] = coef[6 * Q + o];
      }
    }
#pragma unroll 1
    for (int b3 = 0; b3 < n; ++b3) {
      const float* z = pz + (a3 * n + b3) * 3 * q;
      float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f, t4 = 0.f, t5 = 0.f, t6 = 0.f;
#pragma unroll
      for (int k3 = 0; k3 < q; ++k3) {
        const float z00 = z[k3], z11 = z[q + k3], z01 = z[2 * q + k3];
        if (DK) {
          t0 = fmaf(z00, d0[k3], t0);
          t4 = fmaf(z11, GEN ? d4[k3] : d0[k3], t4);
          if (GEN) {
            t1 = fmaf(z00, d1[k3], t1);
            t2 = fmaf(z00, d2[k3], t2);
            t5 = fmaf(z01, d5[k3], t5);
            t6 = fmaf(z01, d6[k3], t6);
          }
        }
        if (DM) t3 = fmaf(z00, d3[k3], t3);
      }
      const int o = (a3 * n + b3) * q * q + kk;
      constexpr int S = n2 * q * q;
      if (DK) {
        T1[0 * S + o] = t0; T1[4 * S + o] = t4;
        if (GEN) { T1[1 * S + o] = t1; T1[2 * S + o] = t2; T1[5 * S + o] = t5; T1[6 * S + o] = t6; }
      }
      if (DM) T1[3 * S + o] = t3;
    }
  }
  __syncthreads();

  // ---- stage 2 ----------------------------------------------------------------
  {
    constexpr int S = n2 * q * q;
    constexpr int T11 = GEN ? 1 : 0;
    // (a) symmetric buffers C11, C00, CM for a' <= b': item = (a3 <= b3, k1, a2)
    for (int it = tid; it < NS1 * q * n; it += NT) {
      const int a2 = it % n, r = it / n, k1 = r % q, ps = r / q;
      int a3 = 0, rr = ps;
      while (rr >= n - a3) { rr -= n - a3; ++a3; }
      const int b3 = a3 + rr;
      // T layout [t][a3][b3][k1][k2] with k1 + q k2 = kk: element (k1, k2) at k1 + q k2
      const int ab3 = (a3 * n + b3) * q * q + k1, ba3 = (b3 * n + a3) * q * q + k1;
      float t00[q], t11[q], t22[q], tab[q], tba[q], tm[q];
#pragma unroll
      for (int k2 = 0; k2 < q; ++k2) {
        if (DK) {
          t00[k2] = T1[0 * S + ab3 + q * k2];
          t11[k2] = T1[T11 * S + ab3 + q * k2];
          t22[k2] = T1[4 * S + ab3 + q * k2];
          if (GEN) { tab[k2] = T1[6 * S + ab3 + q * k2]; tba[k2] = T1[6 * S + ba3 + q * k2]; }
        }
        if (DM) tm[k2] = T1[3 * S + ab3 + q * k2];
      }
      const int ap = a2 + n * a3;
#pragma unroll 1
      for (int b2 = (a3 == b3 ? a2 : 0); b2 < n; ++b2) {
        const float* y = py + (a2 * n + b2) * RW;  // 00, 11, 10, 01
        float c11 = 0.f, c00a = 0.f, c00b = 0.f, cm = 0.f;
#pragma unroll
        for (int k2 = 0; k2 < q; ++k2) {
          const float y00 = y[k2], y11 = y[q + k2], y10 = y[2 * q + k2], y01 = y[3 * q + k2];
          if (DK) {
            c11 = fmaf(y00, t00[k2], c11);
            c00a = fmaf(y11, t11[k2], c00a);
            c00b = fmaf(y00, t22[k2], c00b);
            if (GEN) {
              c00a = fmaf(y10, tab[k2], c00a);
              c00b = fmaf(y01, tba[k2], c00b);
            }
          }
          if (DM) cm = fmaf(y00, tm[k2], cm);
        }
        const int bp = b2 + n * b3;
        if constexpr (BF) {
          if (DK) {
            const __nv_bfloat16 h11 = __float2bfloat16_rn(c11), h00 = __float2bfloat16_rn(c00a + c00b);
            AK[(ap * Np + bp) * C::LDK + 0 * q + k1] = h11;
            AK[(bp * Np + ap) * C::LDK + 0 * q + k1] = h11;
            AK[(ap * Np + bp) * C::LDK + 1 * q + k1] = h00;
            AK[(bp * Np + ap) * C::LDK + 1 * q + k1] = h00;
          }
          if (DM) {
            const __nv_bfloat16 hm = __float2bfloat16_rn(cm);
            AM[(ap * Np + bp) * C::LDM + k1] = hm;
            AM[(bp * Np + ap) * C::LDM + k1] = hm;
          }
        } else {
          const int pp = upper_index<Np>(ap, bp);
          if (DK) {
            Cs[(0 * NSp + pp) * q + k1] = c11;
            Cs[(1 * NSp + pp) * q + k1] = c00a + c00b;
          }
          if (DM) Cs[(2 * NSp + pp) * q + k1] = cm;
        }
      }
    }
    // (b) C10[a'][b'][k1] for all (a', b'): item = (a3, b3, k1, a2)
    if (GEN && DK) {
      for (int it = tid; it < n2 * q * n; it += NT) {
        const int a2 = it % n, r = it / n, k1 = r % q, ab = r / q;
        const int a3 = ab / n, b3 = ab % n;
        const int o = (a3 * n + b3) * q * q + k1;
        float t01[q], t02[q];
#pragma unroll
        for (int k2 = 0; k2 < q; ++k2) {
          t01[k2] = T1[2 * S + o + q * k2];
          t02[k2] = T1[5 * S + o + q * k2];
        }
        const int ap = a2 + n * a3;
#pragma unroll 1
        for (int b2 = 0; b2 < n; ++b2) {
          const float* y = py + (a2 * n + b2) * RW;
          float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
          for (int k2 = 0; k2 < q; ++k2) {
            acc0 = fmaf(y[3 * q + k2], t01[k2], acc0);  // y01 with z00 D01 (term (0,1))
            acc1 = fmaf(y[k2], t02[k2], acc1);          // y00 with z01 D02 (term (0,2))
          }
          const int bp = b2 + n * b3;
          if constexpr (BF) {
            const __nv_bfloat16 h = __float2bfloat16_rn(acc0 + acc1);
            AK[(ap * Np + bp) * C::LDK + 2 * q + k1] = h;  // C10[a'][b']
            AK[(bp * Np + ap) * C::LDK + 3 * q + k1] = h;  // C01[b'][a'] = C10[a'][b']
          } else {
            C10[(ap * Np + bp) * q + k1] = acc0 + acc1;
          }
        }
      }
    }
  }
  __syncthreads();

  if constexpr (BF) {
#pragma unroll 1
    for (int mat = 0; mat < 2; ++mat) {
      const bool isK = mat == 0;
      if ((isK && !DK) || (!isK && !DM)) continue;
      float* dst = (float*)(isK ? A.K_out : A.M_out);
      if (!dst) continue;
      float* g = dst + e * (int64_t)N * N;
      if (isK) gemm_scatter<C, C::LDK, C::KK / 16>(AK, BK, outs, g);
      else gemm_scatter<C, C::LDM, C::KM / 16>(AM, BM, outs, g);
      if (C::STAGE) {
        __syncthreads();
        for (int i = tid; i < N * N; i += NT) g[i] = outs[i];
        __syncthreads();
      }
    }
  } else {

  // ---- stage 3 (FP32): item = (a', b'), a' <= b'; its stage-2 values in
  // registers, the x pattern record of (a1, b1) streamed as float4 -------------
#pragma unroll 1
  for (int mat = 0; mat < 2; ++mat) {
    const bool isK = (mat == 0);
    if ((isK && !DK) || (!isK && !DM)) continue;
    float* dst = (float*)(isK ? A.K_out : A.M_out);
    if (!dst) continue;
    float* g = dst + e * (int64_t)N * N;
    for (int pp = tid; pp < NSp; pp += NT) {
      const int pr = pairs[pp];
      const int ap = pr >> 16, bp = pr & 0xffff;
      float c0[q], c1[q], c2[q], c3[q];
#pragma unroll
      for (int k = 0; k < q; ++k) {
        if (isK) {
          c0[k] = Cs[(0 * NSp + pp) * q + k];
          c1[k] = Cs[(1 * NSp + pp) * q + k];
          if (GEN) {
            c2[k] = C10[(ap * Np + bp) * q + k];
            c3[k] = C10[(bp * Np + ap) * q + k];
          }
        } else {
          c1[k] = Cs[(2 * NSp + pp) * q + k];
        }
      }
#pragma unroll 1
      for (int a1 = 0; a1 < n; ++a1) {
        const int ra = a1 + n * ap;
#pragma unroll
        for (int b1 = 0; b1 < n; ++b1) {
          const float4* x4 = (const float4*)(px + (a1 * n + b1) * RW);
          float xr[RW];
#pragma unroll
          for (int v = 0; v < RW / 4; ++v) {
            const float4 t4 = x4[v];
            xr[4 * v] = t4.x; xr[4 * v + 1] = t4.y; xr[4 * v + 2] = t4.z; xr[4 * v + 3] = t4.w;
          }
          float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
          for (int k = 0; k < q; ++k) {
            if (isK) {
              acc0 = fmaf(xr[k], c0[k], acc0);          // x11 * C11
              acc1 = fmaf(xr[q + k], c1[k], acc1);      // x00 * C00
              if (GEN) {
                acc0 = fmaf(xr[2 * q + k], c2[k], acc0);  // x10 * C10
                acc1 = fmaf(xr[3 * q + k], c3[k], acc1);  // x01 * C01
              }
            } else {
              acc1 = fmaf(xr[q + k], c1[k], acc1);      // x00 * CM
            }
          }
          const float val = acc0 + acc1;
          const int rb = b1 + n * bp;
          if (C::STAGE) {
            outs[ra * N + rb] = val;
            if (ap != bp) outs[rb * N + ra] = val;
          } else {
            g[(int64_t)ra * N + rb] = val;
            if (ap != bp) g[(int64_t)rb * N + ra] = val;
          }
        }
      }
    }
    if (C::STAGE) {
      __syncthreads();
      for (int i = tid; i < N * N; i += NT) g[i] = outs[i];
      __syncthreads();
    }
  }
  }
}

template <int P, int QG, bool GEN, int MODE, bool BF>
__global__ void __launch_bounds__(256) k_sf3_f32(const ElemArgs A) {
  extern __shared__ __align__(16) float smf[];
  sf3_f32_element<P, QG, GEN, MODE, BF>(A, blockIdx.x, smf);
}

// Persistent form: every CTA pops work items (patch, first element, count)
// from the class's device queue until it is empty.  A work item is checked
// against its patch before use (IGA_ERR_DEVICE otherwise).  With a non-zero
// time budget, a CTA stops popping once the budget since its start has passed
// and records IGA_ERR_TIMEOUT; no CTA ever waits on another.
template <int P, int QG, bool GEN, int MODE, bool BF>
__global__ void __launch_bounds__(256) k_sf3_f32_queue(const QueueArgs B) {
  extern __shared__ __align__(16) float smf[];
  __shared__ int s_item;
  const unsigned long long t0 = global_timer_ns();
  for (;;) {
    if (threadIdx.x == 0) {
      int it = -1;
      if (B.budget_ns != 0 && global_timer_ns() - t0 + 1 >= B.budget_ns)
        atomicCAS(B.err, 0, (int)IGA_ERR_TIMEOUT);
      else
        it = atomicAdd(B.counter, 1);
      s_item = it;
    }
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it < 0 || it >= B.n_items) break;
    const WorkItem w = B.items[it];
    if (w.patch < 0 || w.patch >= B.n_patches) {
      if (threadIdx.x == 0) atomicCAS(B.err, 0, (int)IGA_ERR_DEVICE);
      continue;
    }
    const PatchDev pd = B.patches[w.patch];
    const int64_t E = (int64_t)pd.K[0] * pd.K[1] * pd.K[2];
    if (w.e0 < 0 || w.count <= 0 || w.e0 + w.count > E || pd.p != P || pd.q != QG) {
      if (threadIdx.x == 0) atomicCAS(B.err, 0, (int)IGA_ERR_DEVICE);
      continue;
    }
    ElemArgs A;
    A.pd = B.patches + w.patch;
    A.n_elem = E;
    A.K1 = pd.K[0]; A.K2 = pd.K[1]; A.K3 = pd.K[2];
    A.tab[0] = B.tables + pd.tab_offset[0];
    A.tab[1] = B.tables + pd.tab_offset[1];
    A.tab[2] = B.tables + pd.tab_offset[2];
    A.kappa = B.kappa ? B.kappa + pd.qp_offset : nullptr;
    A.rho = B.rho ? B.rho + pd.qp_offset : nullptr;
    A.jac = B.jac ? B.jac + pd.qp_offset * 9 : nullptr;
    A.K_out = B.K_out ? (void*)((float*)B.K_out + pd.mat_offset) : nullptr;
    A.M_out = B.M_out ? (void*)((float*)B.M_out + pd.mat_offset) : nullptr;
    A.err = B.err;
    for (int64_t e = w.e0; e < w.e0 + w.count; ++e)
      sf3_f32_element<P, QG, GEN, MODE, BF>(A, e, smf);
  }
}

template <int P, int QG, bool GEN, int MODE, bool BF>
cudaError_t run(const ElemArgs& a, cudaStream_t st) {
  using C = SF3F<P, QG, GEN, MODE, BF>;
  if constexpr (MODE == 0 && C::smem > 227 * 1024) {
    // both matrices do not fit one CTA: stiffness and mass in two launches
    ElemArgs ak = a, am = a;
    ak.M_out = nullptr;
    am.K_out = nullptr;
    cudaError_t e = run<P, QG, GEN, 1, BF>(ak, st);
    if (e != cudaSuccess) return e;
    return run<P, QG, GEN, 2, BF>(am, st);
  } else {
    static_assert(C::smem <= 227 * 1024, "shared memory");
    auto k = k_sf3_f32<P, QG, GEN, MODE, BF>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)a.n_elem, C::NT, C::smem, st>>>(a);
    return cudaGetLastError();
  }
}

// Queue launch; with max_grid != null only report the resident-CTA capacity.
template <int P, int QG, bool GEN, int MODE, bool BF>
cudaError_t run_queue(const QueueArgs& b, int grid, cudaStream_t st, int* max_grid) {
  using C = SF3F<P, QG, GEN, MODE, BF>;
  if constexpr (C::smem > 227 * 1024) {
    return cudaErrorNotSupported;  // the planner splits such classes by matrix
  } else {
    auto k = k_sf3_f32_queue<P, QG, GEN, MODE, BF>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (e != cudaSuccess) return e;
    if (max_grid) {
      int dev = 0, sms = 0, per_sm = 0;
      e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, C::NT, C::smem);
      if (e != cudaSuccess) return e;
      *max_grid = sms * (per_sm > 0 ? per_sm : 1);
      return cudaSuccess;
    }
    k<<<(unsigned)grid, C::NT, C::smem, st>>>(b);
    return cudaGetLastError();
  }
}

template <int P, int QG, bool BF>
cudaError_t runm(const ElemArgs& a, cudaStream_t st) {
  const int mode = (a.K_out && a.M_out) ? 0 : (a.K_out ? 1 : 2);
  if (a.jac) {
    if (mode == 0) return run<P, QG, true, 0, BF>(a, st);
    if (mode == 1) return run<P, QG, true, 1, BF>(a, st);
    return run<P, QG, true, 2, BF>(a, st);
  }
  if (mode == 0) return run<P, QG, false, 0, BF>(a, st);
  if (mode == 1) return run<P, QG, false, 1, BF>(a, st);
  return run<P, QG, false, 2, BF>(a, st);
}

template <int P, int QG, bool BF>
cudaError_t runq(const QueueArgs& b, int mode, int grid, cudaStream_t st, int* max_grid) {
  if (b.jac) {
    if (mode == 0) return run_queue<P, QG, true, 0, BF>(b, grid, st, max_grid);
    if (mode == 1) return run_queue<P, QG, true, 1, BF>(b, grid, st, max_grid);
    return run_queue<P, QG, true, 2, BF>(b, grid, st, max_grid);
  }
  if (mode == 0) return run_queue<P, QG, false, 0, BF>(b, grid, st, max_grid);
  if (mode == 1) return run_queue<P, QG, false, 1, BF>(b, grid, st, max_grid);
  return run_queue<P, QG, false, 2, BF>(b, grid, st, max_grid);
}

}  // namespace

bool sumfact_f32_supported(int dim, int p, int q) {
  return dim == 3 && p >= 1 && p <= 5 && (q == p + 1 || (q == p + 2 && p <= 4));
}

bool queue_both_fit(int p, int q, bool bf16) {
#define F(PP, QQ)                                                           \
  if (p == PP && q == QQ)                                                   \
    return bf16 ? (SF3F<PP, QQ, true, 0, true>::smem <= 227 * 1024 &&       \
                   SF3F<PP, QQ, false, 0, true>::smem <= 227 * 1024)        \
                : (SF3F<PP, QQ, true, 0, false>::smem <= 227 * 1024 &&      \
                   SF3F<PP, QQ, false, 0, false>::smem <= 227 * 1024);
  F(1, 2) F(1, 3) F(2, 3) F(2, 4) F(3, 4) F(3, 5) F(4, 5) F(4, 6) F(5, 6)
#undef F
  return false;
}

cudaError_t launch_sumfact_f32(const ElemArgs& a, int dim, int p, int q, bool bf16,
                               cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  if (dim != 3) return cudaErrorInvalidValue;
  const int dq = q - p;
#define C3(PP)                                                                                  \
  if (p == PP && dq == 1) return bf16 ? runm<PP, PP + 1, true>(a, st) : runm<PP, PP + 1, false>(a, st); \
  if (p == PP && dq == 2) return bf16 ? runm<PP, PP + 2, true>(a, st) : runm<PP, PP + 2, false>(a, st);
  C3(1) C3(2) C3(3) C3(4)
  if (p == 5 && dq == 1) return bf16 ? runm<5, 6, true>(a, st) : runm<5, 6, false>(a, st);
#undef C3
  return cudaErrorInvalidValue;
}

cudaError_t launch_sumfact_f32_queue(const QueueArgs& b, int p, int q, bool bf16, int mode,
                                     int grid, cudaStream_t st, int* max_grid) {
  const int dq = q - p;
#define C3(PP)                                                                                \
  if (p == PP && dq == 1) return bf16 ? runq<PP, PP + 1, true>(b, mode, grid, st, max_grid)   \
                                      : runq<PP, PP + 1, false>(b, mode, grid, st, max_grid); \
  if (p == PP && dq == 2) return bf16 ? runq<PP, PP + 2, true>(b, mode, grid, st, max_grid)   \
                                      : runq<PP, PP + 2, false>(b, mode, grid, st, max_grid);
  C3(1) C3(2) C3(3) C3(4)
  if (p == 5 && dq == 1) return bf16 ? runq<5, 6, true>(b, mode, grid, st, max_grid)
                                     : runq<5, 6, false>(b, mode, grid, st, max_grid);
#undef C3
  return cudaErrorInvalidValue;
}

}  // namespace iga
