// k_curved32.cu -- FP32 and BF16 sum-factorized stiffness matrices of 3D
// patches with a general geometry map, degree 4 and 5 Gauss points per
// direction (the curved-map workload of the FP32/BF16 forms).
//
// Same stage order as the other sum-factorization kernels (Sec. 3.2,
// Algorithm 2 generalised to the stiffness): stage 1 contracts z (k3), stage 2
// y (k2), stage 3 x (k1).  A general map makes D = (w kappa / |det G|) c^T c a
// full symmetric 3x3 matrix at every point (c: the cofactors of G, formed in
// FP64), so every stage carries the off-diagonal terms:
//   stage 1 (6 terms):  T_t(a3,b3)[k1][k2] = sum_k3 Z_t[a3,b3,k3] D_t[k1,k2,k3]
//     T0 = z00 D00, T1 = z00 D11, T2 = z00 D01, T4 = z11 D22, T5 = z01 D02, T6 = z01 D12
//     (z00 = B_a3 B_b3, z11 = B'_a3 B'_b3, z01 = B_a3 B'_b3; T0, T1, T2, T4 are
//     symmetric in (a3, b3), T5 and T6 are not);
//   stage 2, for the row (a', b') = ((a2, a3), (b2, b3)) and k1, over k2:
//     C11 = y00 T0
//     C00 = y11 T1 + y00 T4 + y10 T6(a3,b3) + y01 T6(b3,a3)
//     C10 = y01 T2 + y00 T5(a3,b3)
//     C01 = y10 T2 + y00 T5(b3,a3)
//     (y00 = B_a2 B_b2, y11 = B'_a2 B'_b2, y10 = B'_a2 B_b2, y01 = B_a2 B'_b2);
//   stage 3 (tcgen05): K[a1 + n a'][b1 + n b'] = sum_{k1, X} C^X[(a',b')][k1] P^X_x[(a1,b1)][k1].
// C11 and C00 are symmetric under (a', b') <-> (b', a') and C10, C01 trade
// places, so only the rows a' <= b' are formed (325 of 625); each result is
// written to (a, b) and mirrored to (b, a).
//
// Data layout:
//  - the operand columns are ordered (k1, X), so that the four x patterns of
//    one (row, k1) form one 16-byte chunk of the K-major operand: stage 2
//    writes whole chunks (FP32 hi and lo: two 16-byte stores; BF16: one 8-byte
//    store), and the B operand (x patterns) is a plain copy of its records;
//  - z pairs are ranked: P = 0..9 the off-diagonal pairs a3 < b3, 10..14 the
//    diagonal ones, 15..24 the off-diagonal pairs transposed (a3 > b3); the
//    stage-1 buffers are T_t[k2][k1][P] (P fastest), so that lanes of
//    consecutive P touch consecutive words;
//  - stage 2 lanes: (row chunk c, k1, z pair P) with P fastest -- 250 lanes of
//    at most 8 rows (an off-diagonal pair's 25 rows in chunks of 7, 6, 6, 6, a
//    diagonal pair's 15 in chunks of 8, 7).  The lanes of one chunk class walk
//    the same (a2, b2) sequence, so a warp's y loads are broadcasts.  A lane
//    keeps its eight stage-1 arrays (40 values) in registers and reads one
//    16-byte y record (y00, y11, y10, y01) per k2 and row: 45 FMAs per 5
//    shared-memory loads.  The operand rows of off-diagonal pair P are
//    25 P .. 25 P + 24 (so the rows that a quarter-warp writes at once fall in
//    different 16-byte bank groups), those of diagonal pair d 250 + 15 d ..;
//  - stage 3 stacks B_hi and B_lo along N (N = 64): FP32 A_hi [B_hi; B_lo] +
//    A_lo B_hi (3xTF32), BF16 A [B_hi; B_lo]; FP32 accumulation in TMEM, the
//    epilogue adds the two halves; the element matrix is staged in shared
//    memory (entries and mirrors) and leaves by one bulk asynchronous copy.
//
// Two kernels share these stages (same arithmetic, bit for bit):
//  - k_sf3_curved (per-patch launch): one CTA per SM, warp-specialised, three
//    elements in flight -- warps 12-15 (geometry) load the inputs of the next
//    element by bulk asynchronous copies and form the coefficients (FP64
//    cofactors) of element i+1; warps 4-11 form the patterns, the B operand
//    and stages 1 and 2 of element i; warps 0-3 (epilogue) issue the MMAs of each
//    element into one of two TMEM buffers, then stage and copy it out.  They
//    meet at mbarriers (inputs loaded, buffers full/empty, operand ready, MMA
//    done), double-buffered by element parity; every wait is
//    bounded (1 s) and a timed-out wait raises a CTA-wide abort flag that
//    every role checks;
//  - k_sf3_curved_queue (persistent batch queue): the same stages run one
//    element after another by a 256-thread CTA, two CTAs per SM.
// On an expired wait the CTA records IGA_ERR_TIMEOUT, stops, waits for its own
// copies and frees its TMEM.
#include "k_sumfact32.cuh"

namespace iga {
namespace {

template <bool BF>
struct CV {
  static constexpr int n = 5, q = 5, n2 = 25, N = 125, Q = 125;
  static constexpr int NROW = 325;                 // operand rows a' <= b'
  static constexpr int MU = 384;                   // three 128-row MMA tiles
  static constexpr int NL2 = 250;                  // stage-2 lanes
  static constexpr int NL1 = 250;                  // stage-1 lanes
  static constexpr int REC = 2 * q * n + q;        // basis record (doubles)
  static constexpr int EB = BF ? 2 : 4;            // operand bytes per element
  static constexpr int KA = BF ? 32 : 24;          // K columns 4 k1 + X (20 used), padded
  static constexpr int NU = 32;                    // (a1, b1) columns, 25 used
  static constexpr int NS = 2 * NU;                // MMA N: [B_hi; B_lo]
  static constexpr int NAU = BF ? 1 : 2;           // A arrays: BF16 one, FP32 hi + lo
  static constexpr uint32_t SBO = KA * EB * 8;     // bytes between 8-row groups
  static constexpr size_t A_BYTES = (size_t)MU * KA * EB;
  static constexpr size_t B_BYTES = (size_t)NU * KA * EB;
  // stage-1 buffers T_t[k2][k1][P]: the symmetric terms T0, T1, T2, T4 for
  // the 15 pairs a3 <= b3, T5 and T6 for all 25 ordered pairs
  static constexpr int TS = q * n * 15, TA = q * n * 25;
  static constexpr int T5OFF = 4 * TS, T6OFF = 4 * TS + TA;
  static constexpr size_t T_FLOATS = (size_t)4 * TS + 2 * TA;
  static constexpr size_t STAGE_FLOATS = (size_t)N * N + 4;
  static constexpr size_t IN_DOUBLES = 3 * REC + Q + 9 * Q;   // records, kappa, Jacobians
  static constexpr size_t r128(size_t x) { return (x + 127) / 128 * 128; }
  static constexpr size_t mx(size_t a, size_t b) { return a > b ? a : b; }
  static_assert(A_BYTES % 1024 == 0 && B_BYTES % 128 == 0, "operand alignment");
};

// ---------------------------------------------------------------------------
// Stages.  t = thread index within the threads running the stage, nt = their
// number.  Every value is computed by one thread with a fixed formula, so the
// result does not depend on (t, nt).

// z pair of rank P: off-diagonal P = 0..9 in the order (0,1), (0,2), (0,3),
// (0,4), (1,2), (1,3), (1,4), (2,3), (2,4), (3,4); diagonal P = 10 + d;
// transposed off-diagonal P = 15 + o.
__device__ __forceinline__ void cv_pair(int P, int& a3, int& b3) {
  if (P >= 10 && P < 15) { a3 = b3 = P - 10; return; }
  int rem = P < 10 ? P : P - 15, x = 0;
  while (rem >= 4 - x) { rem -= 4 - x; ++x; }
  a3 = x;
  b3 = x + 1 + rem;
  if (P >= 15) { const int t = a3; a3 = b3; b3 = t; }
}

// The table of operand rows: R -> (a' << 8 | b').  Rows 25 P + 5 a2 + b2 of
// off-diagonal pair P, rows 250 + 15 d + (a2 <= b2 in row order) of diagonal
// pair d.
template <bool BF>
__device__ __forceinline__ void cv_rows(uint16_t* rows, int t, int nt) {
  for (int R = t; R < CV<BF>::NROW; R += nt) {
    int a3, b3, a2, b2;
    if (R < 250) {
      cv_pair(R / 25, a3, b3);
      a2 = (R % 25) / 5;
      b2 = R % 5;
    } else {
      const int d = (R - 250) / 15;
      int loc = (R - 250) % 15;
      a3 = b3 = d;
      a2 = 0;
      while (loc >= 5 - a2) { loc -= 5 - a2; ++a2; }
      b2 = a2 + loc;
    }
    rows[R] = (uint16_t)(((a2 + 5 * a3) << 8) | (b2 + 5 * b3));
  }
}

// cp.async copies of element e's inputs into rec / kap / jac: its three basis
// records, kappa (1 where kappa is null) and the Jacobians.
template <bool BF>
__device__ __forceinline__ void cv_issue_inputs(const ElemArgs& A, int64_t e, double* rec, double* kap,
                                                double* jac, int t, int nt) {
  using C = CV<BF>;
  constexpr int REC = C::REC, Q = C::Q;
  int e1, e2, e3;
  elem_coords(A, e, e1, e2, e3);
  for (int i = t; i < 3 * REC; i += nt) {
    const int d = i / REC, j = i - d * REC;
    const int ek = d == 0 ? e1 : (d == 1 ? e2 : e3);
    const double* tb = d == 0 ? A.tab[0] : (d == 1 ? A.tab[1] : A.tab[2]);
    cp_async8(rec + i, tb + (int64_t)ek * REC + j);
  }
  for (int k = t; k < Q; k += nt) {
    if (A.kappa) cp_async8(kap + k, A.kappa + e * Q + k);
    else kap[k] = 1.0;
  }
  const double* G = A.jac + e * Q * 9;
  for (int i = t; i < 9 * Q; i += nt) cp_async8(jac + i, G + i);
}

// Double -> float, rounded toward zero, by integer operations on the IEEE
// 754 encodings (sign; exponent rebiased from 1023 to 127; the 52-bit
// fraction cut to its top 23 bits): on GB300 a conversion instruction would
// take the FP64 pipe, which the cofactors need.  Values outside the normal
// float range (zero included) take the conversion instruction.
__device__ __forceinline__ float cv_d2f(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex - 897u > 253u) return (float)x;
  return __uint_as_float((hi & 0x80000000u) | ((ex - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// FP32 copies of the records (each thread converts the values it copied
// itself: visible to it after its cp.async wait).
template <bool BF>
__device__ __forceinline__ void cv_recf(const double* rec, float* recf, int t, int nt) {
  for (int i = t; i < 3 * CV<BF>::REC; i += nt) recf[i] = cv_d2f(rec[i]);
}

// Coefficients of the quadrature points, D_t[k] (k = k1 + q k2 + q^2 k3):
// slots 0 D00, 1 D11, 2 D01, 3 D22, 4 D02, 5 D12.  Cofactors and determinant
// of the Jacobian in FP64, the rest in FP32.
template <bool BF>
__device__ __forceinline__ void cv_coef(const float* recf, const double* kap, const double* jac,
                                        float* coef, int t, int nt) {
  using C = CV<BF>;
  constexpr int n = C::n, q = C::q, Q = C::Q, REC = C::REC;
  for (int k = t; k < Q; k += nt) {
    const int k1 = k % q, k2 = (k / q) % q, k3 = k / (q * q);
    const float* w0 = recf + 2 * q * n;
    const float W = w0[k1] * (w0 + REC)[k2] * (w0 + 2 * REC)[k3];
    const double* G = jac + 9 * k;
    const double g00 = G[0], g01 = G[1], g02 = G[2], g10 = G[3], g11 = G[4], g12 = G[5],
                 g20 = G[6], g21 = G[7], g22 = G[8];
    const double d00 = g11 * g22 - g12 * g21, d01 = g12 * g20 - g10 * g22,
                 d02 = g10 * g21 - g11 * g20;
    const double det = g00 * d00 + g01 * d01 + g02 * d02;
    const float c00 = cv_d2f(d00), c01 = cv_d2f(d01), c02 = cv_d2f(d02);
    const float c10 = cv_d2f(g02 * g21 - g01 * g22), c11 = cv_d2f(g00 * g22 - g02 * g20),
                c12 = cv_d2f(g01 * g20 - g00 * g21);
    const float c20 = cv_d2f(g01 * g12 - g02 * g11), c21 = cv_d2f(g02 * g10 - g00 * g12),
                c22 = cv_d2f(g00 * g11 - g01 * g10);
    const float s = W * cv_d2f(kap[k]) / fabsf(cv_d2f(det));
    coef[0 * Q + k] = s * (c00 * c00 + c10 * c10 + c20 * c20);
    coef[1 * Q + k] = s * (c01 * c01 + c11 * c11 + c21 * c21);
    coef[2 * Q + k] = s * (c00 * c01 + c10 * c11 + c20 * c21);
    coef[3 * Q + k] = s * (c02 * c02 + c12 * c12 + c22 * c22);
    coef[4 * Q + k] = s * (c00 * c02 + c10 * c12 + c20 * c22);
    coef[5 * Q + k] = s * (c01 * c02 + c11 * c12 + c21 * c22);
  }
}

// 1D factor patterns, records [(a,b)][k][4]: x (11, 00, 10, 01) -- the order
// of the operand columns X; y (00, 11, 10, 01); z (00, 11, 01, 0).
template <bool BF>
__device__ __forceinline__ void cv_patterns(const float* recf, float* px, float* py, float* pz, int t,
                                            int nt) {
  using C = CV<BF>;
  constexpr int n = C::n, q = C::q, REC = C::REC;
  for (int it = t; it < 3 * C::n2 * q; it += nt) {
    const int d = it / (C::n2 * q), i = it % (C::n2 * q);
    const int a = i / (n * q), b = (i / q) % n, k = i % q;
    const float* v = recf + d * REC;
    const float* dv = v + q * n;
    const float va = v[k * n + a], vb = v[k * n + b], da = dv[k * n + a], db = dv[k * n + b];
    float4 r;
    if (d == 0) r = make_float4(da * db, va * vb, da * vb, va * db);
    else if (d == 1) r = make_float4(va * vb, da * db, da * vb, va * db);
    else r = make_float4(va * vb, da * db, va * db, 0.f);
    float* dst = d == 0 ? px : (d == 1 ? py : pz);
    *(float4*)(dst + (a * n + b) * 20 + 4 * k) = r;
  }
}

// B operand (x patterns): rows (a1, b1), columns 4 k1 + X; FP32 as TF32 hi +
// lo, BF16 as bf16 hi + lo.  B_lo follows B_hi (rows 32..63 of one operand).
template <bool BF>
__device__ __forceinline__ void cv_bop(const float* px, unsigned char* Bh, int t, int nt) {
  using C = CV<BF>;
  unsigned char* Bl = Bh + C::B_BYTES;
  for (int it = t; it < C::n2 * C::q; it += nt) {
    const int ab = it / C::q, k1 = it % C::q;
    const float4 v = *(const float4*)(px + ab * 20 + 4 * k1);
    if constexpr (BF) {
      const float h[4] = {__bfloat162float(__float2bfloat16_rn(v.x)), __bfloat162float(__float2bfloat16_rn(v.y)),
                          __bfloat162float(__float2bfloat16_rn(v.z)), __bfloat162float(__float2bfloat16_rn(v.w))};
      const uint32_t o = (ab >> 3) * C::SBO + (k1 >> 1) * 128 + (ab & 7) * 16 + (k1 & 1) * 8;
      *(uint2*)(Bh + o) = make_uint2(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]));
      *(uint2*)(Bl + o) = make_uint2(pack_bf16x2(v.x - h[0], v.y - h[1]), pack_bf16x2(v.z - h[2], v.w - h[3]));
    } else {
      const uint32_t o = (ab >> 3) * C::SBO + k1 * 128 + (ab & 7) * 16;
      const uint4 hi = make_uint4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
      const uint4 lo = make_uint4(to_tf32(v.x - __uint_as_float(hi.x)), to_tf32(v.y - __uint_as_float(hi.y)),
                                  to_tf32(v.z - __uint_as_float(hi.z)), to_tf32(v.w - __uint_as_float(hi.w)));
      *(uint4*)(Bh + o) = hi;
      *(uint4*)(Bl + o) = lo;
    }
  }
}

// Stage 1: T_t[k2][k1][P].  Lane = (pair chunk h, k1, k2): h takes the pairs
// P = h, h + 10, h + 20; the symmetric terms for P < 15 only.
template <bool BF>
__device__ __forceinline__ void cv_stage1(const float* coef, const float* pz, float* T, int t, int nt) {
  using C = CV<BF>;
  constexpr int n = C::n, q = C::q, Q = C::Q;
#pragma unroll 1
  for (int ln = t; ln < C::NL1; ln += nt) {
    const int h = ln % 10, kk = ln / 10, k1 = kk % 5, k2 = kk / 5;
    float d[6][q];
#pragma unroll
    for (int s = 0; s < 6; ++s)
#pragma unroll
      for (int k3 = 0; k3 < q; ++k3) d[s][k3] = coef[s * Q + k1 + q * k2 + q * q * k3];
#pragma unroll 1
    for (int P = h; P < 25; P += 10) {
      int a3, b3;
      cv_pair(P, a3, b3);
      const float4* z4 = (const float4*)(pz + (a3 * n + b3) * 20);
      float t0 = 0.f, t1 = 0.f, t2 = 0.f, t4 = 0.f, t5 = 0.f, t6 = 0.f;
#pragma unroll
      for (int k3 = 0; k3 < q; ++k3) {
        const float4 z = z4[k3];   // z00, z11, z01
        t0 = fmaf(z.x, d[0][k3], t0);
        t1 = fmaf(z.x, d[1][k3], t1);
        t2 = fmaf(z.x, d[2][k3], t2);
        t4 = fmaf(z.y, d[3][k3], t4);
        t5 = fmaf(z.z, d[4][k3], t5);
        t6 = fmaf(z.z, d[5][k3], t6);
      }
      if (P < 15) {
        const int o = (k2 * n + k1) * 15 + P;
        T[0 * C::TS + o] = t0; T[1 * C::TS + o] = t1; T[2 * C::TS + o] = t2; T[3 * C::TS + o] = t4;
      }
      const int oa = (k2 * n + k1) * 25 + P;
      T[C::T5OFF + oa] = t5; T[C::T6OFF + oa] = t6;
    }
  }
}

// Stage 2 of one lane (ls < 250): its eight stage-1 arrays are loaded into
// registers first (load), then its rows are formed and written to the
// operand (run), so that the caller can place a barrier in between.
// Lanes 0..199: off-diagonal pair P = 0..9, chunk c of rows 7, 6, 6, 6;
// lanes 200..249: diagonal pair d, chunk c of rows 8, 7 (rows a2 <= b2);
// lane = (c, k1, pair) with the pair fastest.
template <bool BF>
struct CvLane2 {
  using C = CV<BF>;
  float T0[5], T1[5], T2[5], T4[5], T5a[5], T5b[5], T6a[5], T6b[5];
  int R0, al2, be2, k1, cnt;
  bool diag;
  __device__ __forceinline__ void load(const float* T, int ls) {
    int P, Pt;
    if (ls < 200) {
      const int c = ls / 50, r = ls % 50;
      k1 = r / 10;
      P = r % 10;
      Pt = 15 + P;
      const int l0 = c == 0 ? 0 : 7 + 6 * (c - 1);
      cnt = c == 0 ? 7 : 6;
      al2 = l0 / 5;
      be2 = l0 % 5;
      R0 = 25 * P + l0;
      diag = false;
    } else {
      const int c = (ls - 200) / 25, r = (ls - 200) % 25;
      k1 = r / 5;
      const int dd = r % 5;
      P = Pt = 10 + dd;
      diag = true;
      cnt = c == 0 ? 8 : 7;
      al2 = c == 0 ? 0 : 1;   // local row 8 = (a2, b2) = (1, 4)
      be2 = c == 0 ? 0 : 4;
      R0 = 250 + 15 * dd + (c == 0 ? 0 : 8);
    }
#pragma unroll
    for (int k2 = 0; k2 < 5; ++k2) {
      const int os = (k2 * C::n + k1) * 15 + P, oa = (k2 * C::n + k1) * 25;
      T0[k2] = T[0 * C::TS + os];
      T1[k2] = T[1 * C::TS + os];
      T2[k2] = T[2 * C::TS + os];
      T4[k2] = T[3 * C::TS + os];
      T5a[k2] = T[C::T5OFF + oa + P];
      T5b[k2] = T[C::T5OFF + oa + Pt];
      T6a[k2] = T[C::T6OFF + oa + P];
      T6b[k2] = T[C::T6OFF + oa + Pt];
    }
  }
  __device__ __forceinline__ void run(const float* py, unsigned char* Ah) {
    unsigned char* Al = Ah + C::A_BYTES;
#pragma unroll 1
    for (int s = 0; s < cnt; ++s) {
      const int R = R0 + s;
      const float4* y4 = (const float4*)(py + (al2 * C::n + be2) * 20);
      float c11 = 0.f, c00 = 0.f, c00b = 0.f, c10 = 0.f, c01 = 0.f;
#pragma unroll
      for (int k2 = 0; k2 < 5; ++k2) {
        const float4 y = y4[k2];   // y00, y11, y10, y01
        c11 = fmaf(y.x, T0[k2], c11);
        c00 = fmaf(y.y, T1[k2], c00);
        c00b = fmaf(y.x, T4[k2], c00b);
        c00 = fmaf(y.z, T6a[k2], c00);
        c00b = fmaf(y.w, T6b[k2], c00b);
        c10 = fmaf(y.w, T2[k2], c10);
        c10 = fmaf(y.x, T5a[k2], c10);
        c01 = fmaf(y.z, T2[k2], c01);
        c01 = fmaf(y.x, T5b[k2], c01);
      }
      c00 += c00b;
      // columns 4 k1 + X, X = 11, 00, 10, 01 (the x-pattern order of B)
      if constexpr (BF) {
        const uint32_t o = (R >> 3) * C::SBO + (k1 >> 1) * 128 + (R & 7) * 16 + (k1 & 1) * 8;
        const uint2 w = make_uint2(pack_bf16x2(c11, c00), pack_bf16x2(c10, c01));
        if (k1 == 4) {
          // the chunk's other half and the last chunk are K padding
          *(uint4*)(Ah + o) = make_uint4(w.x, w.y, 0u, 0u);
          *(uint4*)(Ah + o + 128) = make_uint4(0u, 0u, 0u, 0u);
        } else {
          *(uint2*)(Ah + o) = w;
        }
      } else {
        const uint32_t o = (R >> 3) * C::SBO + k1 * 128 + (R & 7) * 16;
        *(float4*)(Ah + o) = make_float4(c11, c00, c10, c01);
        *(float4*)(Al + o) = make_float4(c11 - tf32_trunc(c11), c00 - tf32_trunc(c00),
                                         c10 - tf32_trunc(c10), c01 - tf32_trunc(c01));
        if (k1 == 4) {   // the K padding chunk
          *(float4*)(Ah + o + 128) = make_float4(0.f, 0.f, 0.f, 0.f);
          *(float4*)(Al + o + 128) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      // next row: (a2, b2) in row order, a2 <= b2 for a diagonal pair
      if (++be2 == 5) { ++al2; be2 = diag ? al2 : 0; }
    }
  }
};

// Stage 3 (one thread): the three 128-row tiles into TMEM columns d .. d + 191.
template <bool BF>
__device__ __forceinline__ void cv_mma(uint32_t d, const unsigned char* Ah, const unsigned char* Bh) {
  using C = CV<BF>;
  constexpr uint32_t ID64 = umma_idesc(BF ? 1u : 2u, 128, C::NS);
  constexpr uint32_t ID32 = umma_idesc(BF ? 1u : 2u, 128, C::NU);
  constexpr int KS = C::KA * C::EB / 32;
  const uint32_t ah = smem_u32(Ah), bh = smem_u32(Bh);
  const uint32_t al = BF ? 0u : ah + (uint32_t)C::A_BYTES;
#pragma unroll 1
  for (int t = 0; t < 3; ++t) {
    const uint32_t dt = d + (uint32_t)(t * C::NS);
    const uint32_t ta = (uint32_t)t * 16u * C::SBO;
#pragma unroll
    for (int s = 0; s < KS; ++s) {
      const uint64_t dAh = umma_desc(ah + ta + 256u * s, 128, C::SBO);
      const uint64_t dB = umma_desc(bh + 256u * s, 128, C::SBO);   // [B_hi; B_lo]
      if constexpr (BF) {
        umma_f16(dt, dAh, dB, ID64, s > 0 ? 1u : 0u);
      } else {
        const uint64_t dAl = umma_desc(al + ta + 256u * s, 128, C::SBO);
        umma_tf32(dt, dAh, dB, ID64, s > 0 ? 1u : 0u);
        umma_tf32(dt, dAl, dB, ID32, 1u);
      }
    }
  }
}

// Epilogue of one TMEM row: the accumulators of tile t, lanes 32 wq .. + 31
// (this warp), row R = 128 t + 32 wq + lane; entry and mirror into the staged
// matrix.  Columns 0..31: A B_hi (+ A_lo B_hi), 32..63: A_hi B_lo.
template <bool BF>
__device__ __forceinline__ void cv_epi_tile(uint32_t d, int t, int wq, int lane, const uint16_t* rows,
                                            float* stage) {
  using C = CV<BF>;
  constexpr int n = C::n, N = C::N;
  const int R = 128 * t + 32 * wq + lane;
  float v[32], w[16];
  const uint32_t ta = d + (uint32_t)(t * C::NS) + ((uint32_t)(32 * wq) << 16);
  tmem_ld16(ta, v);
  tmem_ld16(ta + 32, w);
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] += w[i];
  tmem_ld16(ta + 16, v + 16);
  tmem_ld16(ta + 48, w);
#pragma unroll
  for (int i = 16; i < C::n2; ++i) v[i] += w[i - 16];
  if (R < C::NROW) {
    const int pr = rows[R];
    const int ap = pr >> 8, bp = pr & 0xff;
    float* dd = stage + (n * ap) * N + n * bp;
    float* dm = stage + (n * bp) * N + n * ap;
#pragma unroll
    for (int a1 = 0; a1 < n; ++a1)
#pragma unroll
      for (int b1 = 0; b1 < n; ++b1) dd[a1 * N + b1] = v[a1 * n + b1];
    if (ap != bp) {
#pragma unroll
      for (int a1 = 0; a1 < n; ++a1)
#pragma unroll
        for (int b1 = 0; b1 < n; ++b1) dm[b1 * N + a1] = v[a1 * n + b1];
    }
  }
}

// Copy a staged element matrix to g: the 16-byte-aligned middle by one bulk
// asynchronous copy (issued by t == 0, committed, not awaited), the scalar
// head and tail by the threads.  The staged matrix starts stage_offset(g)
// floats into its buffer.
__device__ __forceinline__ void cv_copy_out(float* g, const float* stage, int t, int nt) {
  constexpr int nn = 125 * 125;
  const int head = (int)((4 - (((uintptr_t)g >> 2) & 3)) & 3);
  const int nv = (nn - head) / 4;
  for (int i = t; i < head; i += nt) g[i] = stage[i];
  for (int i = head + 4 * nv + t; i < nn; i += nt) g[i] = stage[i];
  if (t == 0) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n"
                 ::"l"(g + head), "r"(smem_u32(stage + head)), "r"(nv * 16) : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
  }
}

// ---------------------------------------------------------------------------
// Serial form (queue kernel): 256 threads run every stage of one element,
// two CTAs per SM.

template <bool BF>
struct CvS {
  using C = CV<BF>;
  static constexpr int NT = 256;
  // the stage-3 operand and the staged matrix share one region
  static constexpr size_t o_region = 0;
  static constexpr size_t region_bytes = C::r128(C::mx(C::NAU * C::A_BYTES, 4 * C::STAGE_FLOATS));
  static constexpr size_t o_T = o_region + region_bytes;
  static constexpr size_t o_B = o_T + C::r128(4 * C::T_FLOATS);
  static constexpr size_t o_in = o_B + C::r128(2 * C::B_BYTES);
  static constexpr size_t o_recf = o_in + C::r128(8 * C::IN_DOUBLES);
  static constexpr size_t o_coef = o_recf + C::r128(4 * 3 * C::REC);
  static constexpr size_t o_px = o_coef + C::r128(4 * 6 * C::Q);
  static constexpr size_t o_py = o_px + 4 * C::n2 * 20;
  static constexpr size_t o_pz = o_py + 4 * C::n2 * 20;
  static constexpr size_t o_rows = o_pz + 4 * C::n2 * 20;
  static constexpr size_t o_mbar = o_rows + C::r128(2 * C::NROW);
  static constexpr size_t smem = o_mbar + 16 + 128;
  static constexpr int TCOLS = 256;
};

template <bool BF>
struct CvSPtrs {
  using L = CvS<BF>;
  unsigned char* b;
  __device__ __forceinline__ explicit CvSPtrs(unsigned char* sm)
      : b((unsigned char*)(((uintptr_t)sm + 127) & ~(uintptr_t)127)) {}
  __device__ __forceinline__ unsigned char* region() const { return b + L::o_region; }
  __device__ __forceinline__ float* T() const { return (float*)(b + L::o_T); }
  __device__ __forceinline__ unsigned char* Bh() const { return b + L::o_B; }
  __device__ __forceinline__ double* rec() const { return (double*)(b + L::o_in); }
  __device__ __forceinline__ double* kap() const { return rec() + 3 * CV<BF>::REC; }
  __device__ __forceinline__ double* jac() const { return kap() + CV<BF>::Q; }
  __device__ __forceinline__ float* recf() const { return (float*)(b + L::o_recf); }
  __device__ __forceinline__ float* coef() const { return (float*)(b + L::o_coef); }
  __device__ __forceinline__ float* px() const { return (float*)(b + L::o_px); }
  __device__ __forceinline__ float* py() const { return (float*)(b + L::o_py); }
  __device__ __forceinline__ float* pz() const { return (float*)(b + L::o_pz); }
  __device__ __forceinline__ uint16_t* rows() const { return (uint16_t*)(b + L::o_rows); }
  __device__ __forceinline__ uint64_t* mbar() const { return (uint64_t*)(b + L::o_mbar); }
  __device__ __forceinline__ uint32_t* tslot() const { return (uint32_t*)(b + L::o_mbar + 8); }
};

// One element.  The inputs of e were issued before the call; those of the
// next element en of the same patch (when has_next) are issued once this
// element's coefficients are formed.  `copy_pending`: a bulk copy of the
// previous element may still read the region (stage 2 waits for it).
// Returns false only on a timed-out MMA wait (IGA_ERR_TIMEOUT recorded).
template <bool BF>
__device__ __forceinline__ bool cv_element(const ElemArgs& A, int64_t e, bool has_next, int64_t en,
                                           const CvSPtrs<BF>& S, uint32_t& phase, bool& copy_pending) {
  using C = CV<BF>;
  constexpr int NT = CvS<BF>::NT;
  const int tid = threadIdx.x;
  cp_async_wait_all();
  cv_recf<BF>(S.rec(), S.recf(), tid, NT);
  __syncthreads();
  cv_coef<BF>(S.recf(), S.kap(), S.jac(), S.coef(), NT - 1 - tid, NT);
  cv_patterns<BF>(S.recf(), S.px(), S.py(), S.pz(), tid, NT);
  __syncthreads();
  if (has_next) cv_issue_inputs<BF>(A, en, S.rec(), S.kap(), S.jac(), tid, NT);
  cv_bop<BF>(S.px(), S.Bh(), tid, NT);
  cv_stage1<BF>(S.coef(), S.pz(), S.T(), tid, NT);
  __syncthreads();
  CvLane2<BF> L;
  const bool act2 = tid < C::NL2;
  if (act2) L.load(S.T(), tid);
  // the previous element's staged matrix has been read by its bulk copy: the
  // region takes the operand
  if (tid == 0 && copy_pending) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
  copy_pending = false;
  __syncthreads();
  if (act2) L.run(S.py(), S.region());
  fence_proxy_async_smem();   // the operands are read by the tensor core
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *S.tslot();
  if (tid == 0) {
    cv_mma<BF>(tmem, S.region(), S.Bh());
    umma_commit(smem_u32(S.mbar()));
  }
  const bool done = mbar_wait_bounded(smem_u32(S.mbar()), phase, 1000000000ull);
  phase ^= 1u;
  if (!__syncthreads_and(done)) {
    if (tid == 0) atomicCAS(A.err, 0, (int)IGA_ERR_TIMEOUT);
    return false;
  }
  fence_after_sync();
  float* g = (float*)A.K_out + e * (int64_t)C::N * C::N;
  float* stage = (float*)S.region() + stage_offset(g);
  {
    // warps 0-3: tiles 0 and 2, warps 4-7: tile 1
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll 1
    for (int t = warp >> 2; t < 3; t += 2) cv_epi_tile<BF>(tmem, t, warp & 3, lane, S.rows(), stage);
  }
  fence_before_sync();          // the TMEM reads precede the next element's MMAs
  fence_proxy_async_smem();     // the staged matrix is read by the bulk copy
  __syncthreads();
  cv_copy_out(g, stage, tid, NT);
  copy_pending = true;
  return true;
}

template <bool BF>
__device__ __forceinline__ void cv_serial_setup(unsigned char* sm) {
  using C = CV<BF>;
  CvSPtrs<BF> S(sm);
  for (int i = threadIdx.x; i < (int)(2 * C::B_BYTES / 4); i += CvS<BF>::NT) ((uint32_t*)S.Bh())[i] = 0u;
  cv_rows<BF>(S.rows(), threadIdx.x, CvS<BF>::NT);
  if (threadIdx.x < 32) {
    tmem_alloc(smem_u32(S.tslot()), CvS<BF>::TCOLS);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(S.mbar()), 1);
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}

template <bool BF>
__device__ __forceinline__ void cv_serial_teardown(unsigned char* sm) {
  CvSPtrs<BF> S(sm);
  cp_async_wait_all();   // a prefetch issued before an early stop
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (threadIdx.x < 32) tmem_dealloc(*S.tslot(), CvS<BF>::TCOLS);
}

// Persistent form: CTAs pop work items (patch, first element, count) from a
// device counter, as the other queue kernels; within an item the next
// element's inputs are prefetched.
template <bool BF>
__global__ void __launch_bounds__(256, 2) k_sf3_curved_queue(const QueueArgs B) {
  extern __shared__ __align__(16) unsigned char sms[];
  __shared__ int s_item;
  const unsigned long long t0 = global_timer_ns();
  cv_serial_setup<BF>(sms);
  const CvSPtrs<BF> S(sms);
  uint32_t phase = 0;
  bool copy_pending = false;
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
    if (w.e0 < 0 || w.count <= 0 || w.e0 + w.count > E || pd.p != 4 || pd.q != 5 || !pd.iso ||
        !B.jac || !B.K_out) {
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
    A.rho = nullptr;
    A.jac = B.jac + pd.qp_offset * 9;
    A.K_out = (void*)((float*)B.K_out + pd.mat_offset);
    A.M_out = nullptr;
    A.err = B.err;
    cv_issue_inputs<BF>(A, w.e0, S.rec(), S.kap(), S.jac(), threadIdx.x, CvS<BF>::NT);
    bool ok = true;
    const int64_t e1 = w.e0 + w.count;
    for (int64_t e = w.e0; e < e1 && ok; ++e)
      ok = cv_element<BF>(A, e, e + 1 < e1, e + 1, S, phase, copy_pending);
    if (!ok) break;
  }
  cv_serial_teardown<BF>(sms);
}

// ---------------------------------------------------------------------------
// Warp-specialised form (per-patch launch): one CTA of 512 threads per SM.
//   warps 0-3   E (epilogue): thread 0 issues the MMAs of each element into
//                             TMEM buffer i mod 2; TMEM -> staged matrix ->
//                             bulk copy
//   warps 4-11  S: patterns, B operand, stages 1 and 2 of element i
//   warps 12-15 G (geometry): inputs (bulk copies), FP32 records and
//                             coefficients (FP64 cofactors) of element i+1
// Buffers by element parity b = i mod 2: inputs, FP32 records,
// coefficients, B operand, TMEM (3 tiles x 64 columns); one set of patterns
// and stage-1 buffers, one stage-3 operand, one staged matrix.  mbarriers
// (b = 0, 1):
//   in[b]    bulk copies of input buffer b complete (1 + transaction bytes)
//   full[b]  G -> S  records and coefficients of b written (128)
//   empty[b] S -> G  S has read them (256)
//   mma[b]   tcgen05.commit of the MMAs that used b (1): their operands are
//            read (B operand b, the stage-3 operand) and TMEM buffer b holds
//            the element's accumulators
//   ready    S -> E  the operands of the next element are written (256)
// A role waiting for element j's event on a barrier of parity b waits for the
// phase (j / 2) mod 2: no barrier can run a phase ahead of any of its waiters,
// because each next phase needs an arrival that follows the wait.

template <bool BF>
struct CvP {
  using C = CV<BF>;
  static constexpr int NT = 512;
  static constexpr size_t o_A = 0;                                              // stage-3 operand
  static constexpr size_t o_stage = o_A + C::r128(C::NAU * C::A_BYTES);          // staged matrix
  static constexpr size_t o_T = o_stage + C::r128(4 * C::STAGE_FLOATS);          // stage-1 buffers
  static constexpr size_t o_B = o_T + C::r128(4 * C::T_FLOATS);                  // [2] B operands
  static constexpr size_t B_STRIDE = C::r128(2 * C::B_BYTES);
  // [2] inputs, each array in a 16-byte-aligned slot with 16 bytes of slack
  // (it starts at the slot + (its global address mod 16)): 3 records, kappa,
  // Jacobians
  static constexpr size_t SL_REC = (8 * C::REC + 16 + 15) / 16 * 16;
  static constexpr size_t SL_KAP = (8 * C::Q + 16 + 15) / 16 * 16;
  static constexpr size_t SL_JAC = (8 * 9 * C::Q + 16 + 15) / 16 * 16;
  static constexpr size_t o_in = o_B + 2 * B_STRIDE;
  static constexpr size_t IN_STRIDE = C::r128(3 * SL_REC + SL_KAP + SL_JAC);
  static constexpr size_t PAT = C::r128(4 * C::n2 * 20);
  static constexpr size_t o_px = o_in + 2 * IN_STRIDE;                           // x, y, z patterns
  static constexpr size_t o_py = o_px + PAT;
  static constexpr size_t o_pz = o_py + PAT;
  static constexpr size_t o_coef = o_pz + PAT;                                   // [2] coefficients
  static constexpr size_t COEF_STRIDE = C::r128(4 * 6 * C::Q);
  static constexpr size_t o_recf = o_coef + 2 * COEF_STRIDE;                     // [2] FP32 records
  static constexpr size_t RECF_STRIDE = C::r128(4 * 3 * C::REC);
  static constexpr size_t o_rows = o_recf + 2 * RECF_STRIDE;
  static constexpr size_t o_mbar = o_rows + C::r128(2 * C::NROW);   // 10 mbarriers, TMEM slot, abort flag
  static constexpr size_t smem = o_mbar + 128 + 128;
  static constexpr int TCOLS = 512;                                  // 2 buffers x 192 columns
  static constexpr int TBUF = 256;                                   // column offset of buffer 1
};

template <bool BF>
struct CvPPtrs {
  using L = CvP<BF>;
  unsigned char* b;
  __device__ __forceinline__ explicit CvPPtrs(unsigned char* sm)
      : b((unsigned char*)(((uintptr_t)sm + 127) & ~(uintptr_t)127)) {}
  __device__ __forceinline__ unsigned char* A() const { return b + L::o_A; }
  __device__ __forceinline__ float* stage() const { return (float*)(b + L::o_stage); }
  __device__ __forceinline__ float* T() const { return (float*)(b + L::o_T); }
  __device__ __forceinline__ unsigned char* Bh(int k) const { return b + L::o_B + k * L::B_STRIDE; }
  // input slots of buffer k: record d (0..2), kappa (3), Jacobians (4)
  __device__ __forceinline__ unsigned char* slot(int k, int which) const {
    return b + L::o_in + k * L::IN_STRIDE + (which < 3 ? which * L::SL_REC
                                             : which == 3 ? 3 * L::SL_REC : 3 * L::SL_REC + L::SL_KAP);
  }
  __device__ __forceinline__ float* px() const { return (float*)(b + L::o_px); }
  __device__ __forceinline__ float* py() const { return (float*)(b + L::o_py); }
  __device__ __forceinline__ float* pz() const { return (float*)(b + L::o_pz); }
  __device__ __forceinline__ float* coef(int k) const { return (float*)(b + L::o_coef + k * L::COEF_STRIDE); }
  __device__ __forceinline__ float* recf(int k) const { return (float*)(b + L::o_recf + k * L::RECF_STRIDE); }
  __device__ __forceinline__ uint16_t* rows() const { return (uint16_t*)(b + L::o_rows); }
  // mbarriers: 0-1 full, 2-3 empty, 4-5 mma, 6 operand ready, 8-9 inputs
  __device__ __forceinline__ uint32_t mb(int which, int k) const {
    return smem_u32(b + L::o_mbar + 8 * (2 * which + k));
  }
  __device__ __forceinline__ uint32_t* tslot() const { return (uint32_t*)(b + L::o_mbar + 96); }
  __device__ __forceinline__ volatile int* abort_flag() const { return (volatile int*)(b + L::o_mbar + 104); }
};

// Global source ranges of element e = e1 + K1 (e2 + K2 e3): records d = 0..2,
// kappa (3), Jacobians (4) -- the first double of each.
struct CvSrc {
  const double* p[5];
  __device__ __forceinline__ CvSrc(const ElemArgs& A, int64_t e, int e1, int e2, int e3) {
    constexpr int REC = CV<false>::REC, Q = CV<false>::Q;
    p[0] = A.tab[0] + (int64_t)e1 * REC;
    p[1] = A.tab[1] + (int64_t)e2 * REC;
    p[2] = A.tab[2] + (int64_t)e3 * REC;
    p[3] = A.kappa ? A.kappa + e * Q : nullptr;
    p[4] = A.jac + e * Q * 9;
  }
};
// (e1, e2, e3) of element e, and the step to element e + s (s >= 0).
struct CvCoord {
  int e1, e2, e3;
  __device__ __forceinline__ CvCoord(const ElemArgs& A, int64_t e) { elem_coords(A, e, e1, e2, e3); }
  __device__ __forceinline__ void step(const ElemArgs& A, int s1, int s2, int s3) {
    // s = s1 + K1 (s2 + K2 s3) with s1 < K1, s2 < K2: add with carries
    e1 += s1;
    if (e1 >= A.K1) { e1 -= A.K1; ++e2; }
    e2 += s2;
    if (e2 >= A.K2) { e2 -= A.K2; ++e3; }
    e3 += s3;
  }
};

__device__ __forceinline__ int cv_len(int which) {
  return which < 3 ? CV<false>::REC : (which == 3 ? CV<false>::Q : 9 * CV<false>::Q);
}

// Where a range's first double lands in its slot: the slot + (address mod 16),
// so that the 16-byte-aligned middle of the range maps to 16-byte-aligned
// shared memory.
__device__ __forceinline__ double* cv_dst(unsigned char* slot, const double* src) {
  return (double*)(slot + ((uintptr_t)src & 15u));
}

// Issue the loads of element e's inputs (ranges R) into input buffer k: the
// 16-byte-aligned middle of each range by one bulk asynchronous copy that
// completes on the buffer's mbarrier (thread t == 0 announces their bytes,
// arrives and issues them), a head or tail double outside it by cp.async
// (threads t = 32..41).  Kappa == null: the slot is filled with ones.
template <bool BF>
__device__ __forceinline__ void cv_tma_inputs(const CvSrc& R, const CvPPtrs<BF>& S, int k, int t) {
  constexpr int Q = CV<BF>::Q;
  const uint32_t mb = S.mb(4, k);
  if (t == 0) {
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < 5; ++w) {
      const double* src = R.p[w];
      if (!src) continue;
      const uintptr_t a = (uintptr_t)src, z = a + 8 * (uintptr_t)cv_len(w);
      const uintptr_t a16 = (a + 15) & ~(uintptr_t)15, z16 = z & ~(uintptr_t)15;
      if (z16 > a16) total += (uint32_t)(z16 - a16);
    }
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(total) : "memory");
#pragma unroll
    for (int w = 0; w < 5; ++w) {
      const double* src = R.p[w];
      if (!src) continue;
      const uintptr_t a = (uintptr_t)src, z = a + 8 * (uintptr_t)cv_len(w);
      const uintptr_t a16 = (a + 15) & ~(uintptr_t)15, z16 = z & ~(uintptr_t)15;
      if (z16 > a16) {
        unsigned char* d = (unsigned char*)cv_dst(S.slot(k, w), src) + (a16 - a);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            ::"r"(smem_u32(d)), "l"((const void*)a16), "r"((uint32_t)(z16 - a16)), "r"(mb) : "memory");
      }
    }
  } else if (t >= 32 && t < 42) {
    // thread 32 + 2 which + (0: head, 1: tail) (another warp than the issuer's)
    const int which = (t - 32) >> 1, tail = (t - 32) & 1;
    const double* src = which == 0 ? R.p[0] : which == 1 ? R.p[1] : which == 2 ? R.p[2]
                       : which == 3 ? R.p[3] : R.p[4];
    if (src) {
      const int len = cv_len(which);
      const uintptr_t a = (uintptr_t)src, z = a + 8 * (uintptr_t)len;
      double* d = cv_dst(S.slot(k, which), src);
      if (!tail && (a & 15u)) cp_async8(d, src);
      if (tail && (z & 15u)) cp_async8(d + len - 1, src + len - 1);
    }
  }
  if (!R.p[3]) {
    double* kp = (double*)S.slot(k, 3);
    for (int i = t; i < Q; i += 128) kp[i] = 1.0;
  }
}

// Bounded wait for the given phase parity of an mbarrier that also gives up
// once the CTA's abort flag is raised.
__device__ __forceinline__ bool cv_wait(uint32_t mbar, uint32_t parity, volatile int* abort_flag) {
  const unsigned long long t0 = gtimer_ns();
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (mbar_try_wait(mbar, parity)) return true;
    if ((it & 63u) == 63u && (*abort_flag || gtimer_ns() - t0 > 1000000000ull)) return false;
  }
  return false;
}

// Barrier of one role (named barrier id, cnt threads) that returns whether
// every participating thread passed ok (and the abort flag is clear).
__device__ __forceinline__ bool cv_role_sync(int id, int cnt, bool ok, volatile int* abort_flag) {
  const int mine = (ok && !*abort_flag) ? 1 : 0;
  int all;
  asm volatile("{\n.reg .pred p, q;\nsetp.ne.s32 p, %1, 0;\nbar.red.and.pred q, %2, %3, p;\nselp.s32 %0, 1, 0, q;\n}\n"
               : "=r"(all) : "r"(mine), "r"(id), "r"(cnt) : "memory");
  return all != 0;
}
__device__ __forceinline__ void cv_bar(int id, int cnt) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(cnt) : "memory");
}

template <bool BF>
__global__ void __launch_bounds__(512, 1) k_sf3_curved(const ElemArgs A) {
  using C = CV<BF>;
  using L = CvP<BF>;
  extern __shared__ __align__(16) unsigned char sms[];
  const CvPPtrs<BF> S(sms);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // ---- set-up ----------------------------------------------------------------
  for (int k = 0; k < 2; ++k)
    for (int i = tid; i < (int)(2 * C::B_BYTES / 4); i += L::NT) ((uint32_t*)S.Bh(k))[i] = 0u;
  cv_rows<BF>(S.rows(), tid, L::NT);
  if (warp == 0) {
    tmem_alloc(smem_u32(S.tslot()), L::TCOLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int k = 0; k < 2; ++k) {
      mbar_init(S.mb(0, k), 128);
      mbar_init(S.mb(1, k), 256);
      mbar_init(S.mb(2, k), 1);
      mbar_init(S.mb(4, k), 1);
    }
    mbar_init(S.mb(3, 0), 256);
    *S.abort_flag() = 0;
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *S.tslot();
  volatile int* abort_flag = S.abort_flag();
  // elements of this CTA: e_i = blockIdx.x + i gridDim.x, i < ne
  const int64_t ne = A.n_elem > blockIdx.x ? (A.n_elem - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (warp >= 12) {
    // ---- G: inputs, FP32 records, coefficients --------------------------------
    const int t = tid - 384;
    // element coordinates of this CTA's first element and of the stride
    CvCoord cur(A, blockIdx.x), nxt = cur;
    const CvCoord stp(A, gridDim.x);
    nxt.step(A, stp.e1, stp.e2, stp.e3);
    if (ne > 0) cv_tma_inputs<BF>(CvSrc(A, blockIdx.x, cur.e1, cur.e2, cur.e3), S, 0, t);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
#pragma unroll 1
    for (int64_t i = 0; i < ne; ++i) {
      const int b = (int)(i & 1);
      const int64_t e = blockIdx.x + i * gridDim.x;
      if (i + 1 < ne) cv_tma_inputs<BF>(CvSrc(A, e + gridDim.x, nxt.e1, nxt.e2, nxt.e3), S, b ^ 1, t);
      asm volatile("cp.async.commit_group;\n" ::: "memory");
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // this element's heads and tails
      bool ok = cv_wait(S.mb(4, b), (uint32_t)(i >> 1) & 1u, abort_flag);
      // element i - 2 released the records and coefficients of parity b
      if (ok && i >= 2) ok = cv_wait(S.mb(1, b), (uint32_t)((i - 2) >> 1) & 1u, abort_flag);
      if (!cv_role_sync(1, 128, ok, abort_flag)) { *abort_flag = 1; break; }
      const CvSrc R(A, e, cur.e1, cur.e2, cur.e3);
      const double* r0 = cv_dst(S.slot(b, 0), R.p[0]);
      const double* r1 = cv_dst(S.slot(b, 1), R.p[1]);
      const double* r2 = cv_dst(S.slot(b, 2), R.p[2]);
      for (int x = t; x < 3 * C::REC; x += 128) {
        const int d = x / C::REC;
        S.recf(b)[x] = cv_d2f((d == 0 ? r0 : (d == 1 ? r1 : r2))[x - d * C::REC]);
      }
      const double* kap = R.p[3] ? cv_dst(S.slot(b, 3), R.p[3]) : (const double*)S.slot(b, 3);
      const double* jac = cv_dst(S.slot(b, 4), R.p[4]);
      cv_bar(1, 128);
      cv_coef<BF>(S.recf(b), kap, jac, S.coef(b), t, 128);
      mbar_arrive(S.mb(0, b));
      cv_bar(1, 128);             // input buffer b is reloaded for element i + 2
      cur = nxt;
      nxt.step(A, stp.e1, stp.e2, stp.e3);
    }
    cp_async_wait_all();
  } else if (warp >= 4) {
    // ---- S: patterns, B operand, stages 1 and 2 -----------------------------------
    const int ls = tid - 128;
#pragma unroll 1
    for (int64_t i = 0; i < ne; ++i) {
      const int b = (int)(i & 1);
      bool ok = cv_wait(S.mb(0, b), (uint32_t)(i >> 1) & 1u, abort_flag);
      if (!cv_role_sync(2, 256, ok, abort_flag)) { *abort_flag = 1; break; }
      cv_patterns<BF>(S.recf(b), S.px(), S.py(), S.pz(), ls, 256);
      cv_bar(2, 256);
      // (B operand b was last read by the MMAs of element i - 2, awaited by the
      // previous iteration)
      cv_bop<BF>(S.px(), S.Bh(b), ls, 256);
      cv_stage1<BF>(S.coef(b), S.pz(), S.T(), ls, 256);
      cv_bar(2, 256);
      mbar_arrive(S.mb(1, b));    // records and coefficients of b are free
      CvLane2<BF> L2;
      const bool act = ls < C::NL2;
      if (act) L2.load(S.T(), ls);
      // the MMAs of element i - 1 have read the stage-3 operand
      ok = true;
      if (i >= 1) ok = cv_wait(S.mb(2, b ^ 1), (uint32_t)((i - 1) >> 1) & 1u, abort_flag);
      if (!cv_role_sync(2, 256, ok, abort_flag)) { *abort_flag = 1; break; }
      if (act) L2.run(S.py(), S.A());
      fence_proxy_async_smem();   // the operands are read by the tensor core
      fence_before_sync();
      cv_bar(2, 256);
      mbar_arrive(S.mb(3, 0));    // the operands of element i are written
    }
  } else {
    // ---- E: MMA issue, epilogue, copy-out ------------------------------------
    bool copy_pending = false;
    int64_t issued = -1;   // (thread 0) the last element whose MMAs it issued
#pragma unroll 1
    for (int64_t i = 0; i < ne; ++i) {
      const int b = (int)(i & 1);
      // thread 0 issues the MMAs of element i once its operand is written
      // (TMEM buffer b was read by this role's epilogue of element i - 2)
      if (tid == 0) {
        if (cv_wait(S.mb(3, 0), (uint32_t)(i & 1), abort_flag)) {
          fence_after_sync();
          cv_mma<BF>(tmem + (uint32_t)(b * L::TBUF), S.A(), S.Bh(b));
          umma_commit(S.mb(2, b));
          issued = i;
        } else {
          *abort_flag = 1;
        }
      }
      bool ok = cv_wait(S.mb(2, b), (uint32_t)(i >> 1) & 1u, abort_flag);
      // the staged matrix of element i - 1 has been read by its bulk copy
      if (tid == 0 && copy_pending) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
      if (!cv_role_sync(3, 128, ok, abort_flag)) { *abort_flag = 1; break; }
      fence_after_sync();
      const int64_t e = blockIdx.x + i * gridDim.x;
      float* g = (float*)A.K_out + e * (int64_t)C::N * C::N;
      float* stage = S.stage() + stage_offset(g);
#pragma unroll 1
      for (int t = 0; t < 3; ++t)
        cv_epi_tile<BF>(tmem + (uint32_t)(b * L::TBUF), t, warp, lane, S.rows(), stage);
      fence_before_sync();        // the TMEM reads precede the MMAs of element i + 2
      fence_proxy_async_smem();   // the staged matrix is read by the bulk copy
      cv_bar(3, 128);
      cv_copy_out(g, stage, tid, 128);
      copy_pending = true;
    }
    if (tid == 0) {
      // after an early stop, MMAs that were issued complete before the TMEM
      // is released
      if (issued >= 0) mbar_wait_bounded(S.mb(2, (int)(issued & 1)), (uint32_t)(issued >> 1) & 1u, 1000000000ull);
      asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
    }
  }
  // ---- teardown --------------------------------------------------------------
  if (*abort_flag && tid == 0) atomicCAS(A.err, 0, (int)IGA_ERR_TIMEOUT);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, L::TCOLS);
}

template <class K>
cudaError_t cv_prepare(K k, int nt, size_t smem, int tcols, int* cap_out) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  int dev = 0, sms = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = resident_ctas_tmem((const void*)k, nt, smem, tcols, &per_sm);
  if (e != cudaSuccess) return e;
  *cap_out = sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

template <bool BF>
cudaError_t cv_run(const ElemArgs& a, cudaStream_t st) {
  using L = CvP<BF>;
  static_assert(L::smem <= 227 * 1024, "shared memory");
  auto k = k_sf3_curved<BF>;
  static int capacity = 0;   // resident CTAs on this GPU, looked up once
  if (capacity == 0) {
    cudaError_t e = cv_prepare(k, L::NT, L::smem, L::TCOLS, &capacity);
    if (e != cudaSuccess) return e;
  }
  const int64_t grid = a.n_elem < capacity ? a.n_elem : capacity;
  k<<<(unsigned)grid, L::NT, L::smem, st>>>(a);
  return cudaGetLastError();
}

template <bool BF>
cudaError_t cv_run_queue(const QueueArgs& b, int grid, cudaStream_t st, int* max_grid) {
  using L = CvS<BF>;
  static_assert(L::smem <= 227 * 1024, "shared memory");
  auto k = k_sf3_curved_queue<BF>;
  int cap = 0;
  cudaError_t e = cv_prepare(k, L::NT, L::smem, L::TCOLS, &cap);
  if (e != cudaSuccess) return e;
  if (max_grid) {
    *max_grid = cap;
    return cudaSuccess;
  }
  k<<<(unsigned)grid, L::NT, L::smem, st>>>(b);
  return cudaGetLastError();
}

}  // namespace

bool curved_form_supported(int p, int q) { return p == 4 && q == 5; }

cudaError_t launch_sumfact_f32_curved(const ElemArgs& a, bool bf16, cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  if (!a.jac || !a.K_out || a.M_out) return cudaErrorInvalidValue;
  return bf16 ? cv_run<true>(a, st) : cv_run<false>(a, st);
}

cudaError_t launch_sumfact_f32_curved_queue(const QueueArgs& b, bool bf16, int grid, cudaStream_t st,
                                            int* max_grid) {
  if (!b.jac || !b.K_out || b.M_out) return cudaErrorInvalidValue;
  return bf16 ? cv_run_queue<true>(b, grid, st, max_grid) : cv_run_queue<false>(b, grid, st, max_grid);
}

}  // namespace iga
