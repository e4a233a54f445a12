#pragma once
// k_sumfact32.cuh -- FP32 and BF16 sum-factorized element matrices, 3D: the
// templated kernels, included by k_sumfact32.cu (the per-patch launches and
// the default persistent form) and k_sumfact32_alt.cu (the persistent forms
// with the other stage-3 form or CTA size, which the batch autotuner times).
//
// Same integrand terms and stage order as the FP64 kernel (Sec. 3.2,
// Algorithm 2 generalised to the stiffness; see k_sumfact64.cu): stage 1
// contracts the last direction (k3), stage 2 the middle one (k2), stage 3 the
// first (k1).  Precision: the Jacobian cofactors and determinant are formed in
// FP64; D = w kappa / |det| c^T c, the 1D factor patterns and stages 1-2 run
// in FP32 FFMA (register-blocked: the reused operand in registers, the 1D
// factor patterns streamed from shared memory as float4 records).
//
// Stage 3 is a dense GEMM per element on the tensor cores:
//   K[(a1 + n a')][(b1 + n b')] = sum_{X,k1} C^X[(a',b')][k1] P^X_x[(a1,b1)][k1]
// with rows (a',b') over the symmetric pairs a' <= b' only, columns (a1,b1)
// and depth (x pattern X, k1); every result is written to (a,b) and, off the
// diagonal blocks, mirrored to (b,a).  FP32 form: 3xTF32 (operands split into
// TF32 hi + lo; hi*hi + hi*lo + lo*hi, FP32 accumulation) with
// mma.sync.m16n8k8.tf32.  BF16 form: bf16 stage-2 operand, x patterns split
// into bf16 hi + lo, mma.sync.m16n8k16.bf16, FP32 accumulation.  Each element
// matrix is assembled in shared memory and written with coalesced 16-byte
// stores when it fits, else scattered to HBM directly.
//
// For p <= 3 (and p = 4 in BF16) stage 3 runs on the 5th-generation tensor
// cores instead (tcgen05.mma, accumulators in tensor memory).  p <= 3: stage
// 2 writes every row (a', b') -- the symmetric half computed once and written
// to both (a', b') and (b', a') with the x patterns 10 and 01 exchanged -- in
// the K-major core-matrix layout of umma.cuh; one thread issues the MMAs
// (3xTF32, or BF16 x (hi + lo) for the BF16 form) into TMEM and commits them
// to an mbarrier; after a bounded wait every warp reads its 32 TMEM lanes (one
// row (a', b') per thread, its n^2 columns (a1, b1)) and stores the row's
// entries K[a1 + n a'][b1 + n b'] straight to HBM: consecutive threads hold
// consecutive b', so the stores are coalesced and need no staging.  p = 4:
// the rows a' <= b' only; the epilogue writes each entry and its mirror into a
// staged copy of the element matrix (over the operands, dead by then) and
// copies it to HBM with aligned 16-byte stores.
// MODE: 0 = stiffness and mass, 1 = stiffness only, 2 = mass only; plus
// MODE_ALT_FORM (4): stage 3 on mma.sync where the default is tcgen05, and
// MODE_ALT_CTA (8): the other CTA size (256 <-> 512 threads, identity map, p >= 4).
// The two flags select the variants the batch autotuner times.
#include <cuda_bf16.h>

#include "iga_internal.h"
#include "umma.cuh"

namespace iga {
namespace {

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int MODE_ALT_FORM = 4, MODE_ALT_CTA = 8;

template <int P, int QG, bool GEN, int MODE, bool BF>
struct SF3F {
  static constexpr int MD = MODE & 3;
  static constexpr bool DK = MD != 2, DM = MD != 1;
  static constexpr int n = P + 1, q = QG, Q = q * q * q, n2 = n * n, N = n2 * n;
  static constexpr int NS1 = n * (n + 1) / 2;
  static constexpr int Np = n2;
  static constexpr int NSp = Np * (Np + 1) / 2;
  // threads per CTA: one CTA per SM at p = 5 (its operands and row block fill
  // shared memory), so there 16 warps instead of 8 hide the latency of the
  // dependent stages (identity geometry; the general-map variants need more
  // than the 128 registers a 512-thread CTA allows)
  static constexpr bool NT512 = P >= 5 && !GEN;
  static constexpr int NT = (NT512 != ((MODE & MODE_ALT_CTA) != 0)) ? 512 : 256;
  static constexpr int REC = 2 * q * n + q;
  static constexpr size_t al4(size_t x) { return (x + 3) / 4 * 4; }
  static constexpr int rup(int x, int m) { return (x + m - 1) / m * m; }
  // pattern records, floats: x [a1][b1][4][q] (11, 00, 10, 01); y [a2][b2][4][q]
  // (00, 11, 10, 01); z [a3][b3][3][q] (00, 11, 01)
  static constexpr int RW = 4 * q;
  // z-pattern records and stage-1 rows are padded to an odd number of words
  // when their natural length is even, so that threads indexing consecutive
  // (a3, b3) hit different shared-memory banks
  static constexpr int RZ = (3 * q) % 2 == 0 ? 3 * q + 1 : 3 * q;       // z record stride
  // p = 3, q = 4 with identity geometry: stage 2 of the tcgen05 form writes
  // whole 16-byte operand chunks (all k1 of a row at once, VEC2 below) and
  // reads the stage-1 rows as float4, so their stride is a multiple of 4
  // words (20: the stage-1 writes of consecutive b3 still spread over banks)
  static constexpr bool VEC2 = !GEN && P == 3 && QG == 4;
  static constexpr int TS = VEC2 ? 20 : ((q * q) % 2 == 0 ? q * q + 1 : q * q);  // stage-1 row stride
  static constexpr size_t f_px = (size_t)n2 * RW, f_py = (size_t)n2 * RW, f_pz = al4((size_t)n2 * RZ);
  // coefficients [7][Q]: 0 D00, 1 D11, 2 D01, 3 DM, 4 D22, 5 D02, 6 D12 (identity: 0 = W kappa, 3 = W rho)
  // stage-1 terms and coefficients held: all seven with a general Jacobian;
  // with identity geometry only D00 (= D11 = D22), the mass weight and the
  // z-derivative term (slots 0, 1, 2 for terms 0, 3, 4)
  static constexpr int NTERM = GEN ? 7 : 3, NCOEF = GEN ? 7 : 2;
  static constexpr int ts(int t) { return GEN ? t : (t == 0 ? 0 : (t == 3 ? 1 : 2)); }
  static constexpr int cs(int t) { return GEN ? t : (t == 0 ? 0 : 1); }
  static constexpr size_t f_coef = al4((size_t)NCOEF * Q);
  // stage-1 buffers T[7][a3][b3][k1][k2] (same indices as the coefficients)
  static constexpr size_t f_T1 = al4((size_t)NTERM * n2 * TS);
  // stage-3 GEMM: A rows = symmetric pairs (padded to 16), depth padded to the k-step
  static constexpr int NXK = GEN ? 4 : 2;
  static constexpr int KSTEP = BF ? 16 : 8;
  static constexpr int KA = rup(NXK * q, KSTEP), KAM = rup(q, KSTEP);
  static constexpr int LDA = KA + 4, LDAM = KAM + 4;          // FP32 A row strides (words)
  static constexpr int MPs = rup(NSp, 16);
  static constexpr int NPAD = rup(n2, 8);
  static constexpr int LDB = BF ? (KA + 8) / 2 : KA + 4;        // B row strides (words)
  static constexpr int LDBM = BF ? (KAM + 8) / 2 : KAM + 4;
  static constexpr size_t f_A = (size_t)MPs * ((DK ? LDA : 0) + (DM ? LDAM : 0));
  static constexpr size_t f_B = (size_t)2 * NPAD * ((DK ? LDB : 0) + (DM ? LDBM : 0));
  static constexpr size_t f_out = al4((size_t)N * N + 4);
  static constexpr size_t d_geo = 3 * REC + 2 * (size_t)Q + (GEN ? 9 * (size_t)Q : 0);
  static constexpr size_t f_recf = al4(3 * REC);
  // aliased region: {T1, coef, geometry staging, FP32 records} until stage 2
  // ends, then the output stage
  static constexpr size_t f_alias = f_T1 + f_coef + 2 * d_geo + f_recf;
  static constexpr size_t f_A4 = al4(f_A), f_B4 = al4(f_B);
  static constexpr size_t f_fixed = f_px + f_py + f_pz + f_A4 + f_B4;
  static constexpr size_t f_pairs = al4((size_t)NSp);
  // the staged element matrix: whole, or in NSPLIT blocks of RB rows when the
  // whole one does not fit beside the operands (the stage-3 GEMM then runs
  // once per block and keeps the entries of the block's rows)
  static constexpr int rows_of(int s) { return (N + s - 1) / s; }
  static constexpr size_t f_outb_of(int s) { return al4((size_t)rows_of(s) * N + 4); }
  static constexpr bool fits(int s) {
    return 4 * (f_fixed + (f_alias > f_outb_of(s) ? f_alias : f_outb_of(s)) + f_pairs) <= 216 * 1024;
  }
  static constexpr int NSPLIT = fits(1) ? 1 : fits(2) ? 2 : fits(3) ? 3 : fits(4) ? 4 : 0;
  static constexpr bool STAGE = NSPLIT > 0;
  static constexpr int RB = STAGE ? rows_of(NSPLIT) : N;
  static constexpr size_t f_outb = f_outb_of(STAGE ? NSPLIT : 1);
  static constexpr size_t f_region_mma = al4((STAGE && f_outb > f_alias) ? f_outb : f_alias);
  static constexpr size_t smem_mma = 4 * (f_fixed + f_region_mma + f_pairs);
  // ---- stage 3 on tcgen05: p <= 3, and p = 4 in BF16 ----
  // (FP32 at p = 4 needs hi and lo operands of 74 KB: two CTAs per SM, where
  // the mma.sync form below is faster)
  static constexpr bool UM = !(MODE & MODE_ALT_FORM) && (P <= 3 || (P == 4 && BF));
  // p <= 3: A holds every row (a', b') and the epilogue stores rows straight to
  // HBM; p = 4: A holds the rows a' <= b' and the epilogue stages the element
  // matrix (both triangles) in shared memory over the dead operands
  static constexpr bool FULLR = P <= 3;
  static constexpr int EB = BF ? 2 : 4;                 // bytes per operand element
  static constexpr int MU = rup(FULLR ? n2 * n2 : NSp, 128);   // A rows, whole tiles
  static constexpr int MTU = MU / 128;                  // 128-row MMA tiles
  static constexpr int NU = rup(n2, 16);                // B rows (a1, b1) = MMA N
  static constexpr int NAU = BF ? 1 : 2;                // A arrays: BF16 one, FP32 hi + lo
  static constexpr size_t uAK = DK ? (size_t)MU * KA * EB : 0, uAM = DM ? (size_t)MU * KAM * EB : 0;
  static constexpr size_t uBK = DK ? (size_t)NU * KA * EB : 0, uBM = DM ? (size_t)NU * KAM * EB : 0;
  static constexpr size_t u_ops = NAU * (uAK + uAM) + 2 * (uBK + uBM);   // bytes
  static constexpr size_t f_uops = (u_ops + 127) / 128 * 32;             // floats, 128-B multiple
  static constexpr int TC_NEED = (DK ? MTU * NU : 0) + (DM ? MTU * NU : 0);
  static constexpr int TCOLS = TC_NEED <= 32 ? 32 : TC_NEED <= 64 ? 64 : TC_NEED <= 128 ? 128
                               : TC_NEED <= 256 ? 256 : 512;
  static constexpr size_t f_base = f_px + f_py + f_pz;
  // tcgen05 region: the geometry staging and the FP32 records are dead once
  // the coefficients are formed, before stage 1 writes T1, so they share its
  // space; then the coefficients
  static constexpr size_t f_geo_u = 2 * d_geo + f_recf;
  static constexpr size_t f_T1u = al4(f_T1 > f_geo_u ? f_T1 : f_geo_u);
  static constexpr size_t f_region_u = al4(f_T1u + f_coef);
  // p = 4: the staged element matrix covers the operands and the region
  static constexpr size_t f_span_u = (FULLR || f_uops + f_region_u >= f_out + 4)
                                         ? f_uops + f_region_u : al4(f_out + 4);
  static constexpr size_t f_region = UM ? f_region_u : f_region_mma;
  // UM: [px py pz][operands][region (or the staged matrix)][mbarrier + TMEM slot]
  static constexpr size_t smem = UM ? 4 * (f_base + f_span_u + 4) + 128 : smem_mma;
};

template <int EB, int KDIM>
__device__ __forceinline__ int uoff(int r, int k) {
  // byte offset of element (r, k) of a K-major operand with KDIM elements per row
  return (r >> 3) * (KDIM * EB * 8) + ((k * EB) >> 4) * 128 + (r & 7) * 16 + ((k * EB) & 15);
}

// Physical operand row of (a', b') in the tcgen05 form.  For n^2 = 16 the
// rows of one a' form one block of 16 (which keeps the epilogue's global
// stores coalesced), permuted within the block so that stage 2's writes
// spread over the shared-memory banks.  A permutation of A's rows only
// permutes the TMEM rows of the product; the epilogue inverts it (urow_inv).
//   V = false (stage 2 writes one value per thread and row): the low three
//     bits of the row are rotated by a', so that the threads of a warp writing
//     rows (a', b') for consecutive a' -- and the mirrored rows (b', a') --
//     land on different banks;
//   V = true (p = 3, q = 4, identity map: stage 2 writes whole 16-byte
//     chunks, eight consecutive threads = four b2 by two a2 of one (a3, b3)
//     pair): with b' = y2 + 4 y3 (y2 = b' mod 4) the row within the block is
//       8 (y3 >> 1) + 4 ((y3 + a') mod 2) + ((y2 + a') mod 4),
//     which puts the chunks of those eight threads in eight different 16-byte
//     bank groups, for the rows (a', b') and for their mirrors (b', a').
template <int n2, bool V>
__device__ __forceinline__ int urow(int x, int y) {
  if constexpr (n2 == 16 && V) {
    const int y3 = y >> 2;
    return 16 * x + 8 * (y3 >> 1) + 4 * ((y3 + x) & 1) + ((y + x) & 3);
  } else if constexpr (n2 == 16) {
    return 16 * x + ((y & 8) | ((x + y) & 7));
  } else {
    return x * n2 + y;
  }
}
template <int n2, bool V>
__device__ __forceinline__ void urow_inv(int r, int& x, int& y) {
  if constexpr (n2 == 16 && V) {
    x = r >> 4;
    const int lo = r & 15;
    const int y3 = 2 * (lo >> 3) + (((lo >> 2) - x) & 1);
    y = 4 * y3 + ((lo - x) & 3);
  } else if constexpr (n2 == 16) {
    x = r >> 4;
    const int lo = r & 15;
    y = (lo & 8) | ((lo - x) & 7);
  } else {
    x = r / n2;
    y = r % n2;
  }
}

__device__ __forceinline__ float tf32_trunc(float v) {
  return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
}

// Store v at element (r, k) of an A or B operand: FP32 as hi (the word
// itself; the tensor core reads its top 19 bits) and lo = v - hi; BF16 as one
// rounded value (A) or hi + lo (B, when lo != nullptr).
template <bool BF, int KDIM>
__device__ __forceinline__ void uput(unsigned char* hi, unsigned char* lo, int r, int k, float v) {
  if (BF) {
    const int o = uoff<2, KDIM>(r, k);
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    *(__nv_bfloat16*)(hi + o) = h;
    if (lo) *(__nv_bfloat16*)(lo + o) = __float2bfloat16_rn(v - __bfloat162float(h));
  } else {
    const int o = uoff<4, KDIM>(r, k);
    *(float*)(hi + o) = v;
    if (lo) *(float*)(lo + o) = v - tf32_trunc(v);
  }
}

__device__ __forceinline__ void mma_bf16_16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_tf32_1688(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Asynchronous 8-byte global -> shared copy (cp.async); all of a thread's
// copies are in flight together and complete at cp_async_wait_all().
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *(const uint32_t*)&v;
}

// packed index of (a', b'), a' <= b', in the upper triangle of an Np x Np matrix
template <int Np>
__device__ __forceinline__ int upper_index(int ap, int bp) {
  return ap * Np - (ap * (ap - 1)) / 2 + (bp - ap);
}

// Stage 3 on the tensor cores for one matrix.  A: [MPs][LDA_] FP32 (rows =
// symmetric pairs), B: hi and lo [2][NPAD][LDB_] (tf32 bit patterns or bf16x2
// words).  Warp w takes the 16-row tiles w, w+8, ...; fragments follow the
// m16n8k8 (TF32) / m16n8k16 (BF16) register layouts: row g = lane/4, column
// pair 2*(lane%4).
// Only the entries whose row lies in [r0, r1) are written, at (row - r0) N + col
// of dst (the staged row block, or the element matrix itself when r0 = 0).
template <class C, int LDA_, int LDB_, int KS>
__device__ __forceinline__ void gemm_sym(const float* Am, const uint32_t* Bm, const int* pairs,
                                         float* dst_stage, float* dst_global, int r0, int r1) {
  constexpr int n = C::n, N = C::N, NSp = C::NSp, NTN = C::NPAD / 8, MT = C::MPs / 16;
  constexpr bool BF = C::KSTEP == 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  uint32_t bh[NTN][KS][2], bl[NTN][KS][2];
#pragma unroll
  for (int nt = 0; nt < NTN; ++nt)
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const uint32_t* r0 = Bm + (nt * 8 + g) * LDB_;
      const uint32_t* r1 = Bm + (C::NPAD + nt * 8 + g) * LDB_;
      if (BF) {  // k pairs: word index = k / 2
        bh[nt][ks][0] = r0[ks * 8 + t];
        bh[nt][ks][1] = r0[ks * 8 + t + 4];
        bl[nt][ks][0] = r1[ks * 8 + t];
        bl[nt][ks][1] = r1[ks * 8 + t + 4];
      } else {
        bh[nt][ks][0] = r0[ks * 8 + t];
        bh[nt][ks][1] = r0[ks * 8 + t + 4];
        bl[nt][ks][0] = r1[ks * 8 + t];
        bl[nt][ks][1] = r1[ks * 8 + t + 4];
      }
    }
  // column offsets of this lane's two columns in every N tile: direct (a1 N + b1)
  // and mirrored (b1 N + a1); -1 marks padding columns
  int cd[NTN][2], cm[NTN][2], ca[NTN][2], cb[NTN][2];
#pragma unroll
  for (int nt = 0; nt < NTN; ++nt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int nn = nt * 8 + 2 * t + h;
      const int a1 = nn / n, b1 = nn % n;
      cd[nt][h] = nn < n * n ? a1 * N + b1 : -1;
      cm[nt][h] = b1 * N + a1;
      ca[nt][h] = a1;   // row offset of the direct entry
      cb[nt][h] = b1;   // row offset of the mirrored entry
    }
  float* dst = C::STAGE ? dst_stage : dst_global;
  const int off0 = r0 * N;
  for (int mt = warp; mt < MT; mt += C::NT / 32) {
    uint32_t ah[KS][4], al[KS][4];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const float* r0 = Am + (mt * 16 + g) * LDA_;
      const float* r1 = r0 + 8 * LDA_;
      if (BF) {
        const float2 x0 = *(const float2*)(r0 + ks * 16 + 2 * t);
        const float2 x1 = *(const float2*)(r1 + ks * 16 + 2 * t);
        const float2 x2 = *(const float2*)(r0 + ks * 16 + 2 * t + 8);
        const float2 x3 = *(const float2*)(r1 + ks * 16 + 2 * t + 8);
        ah[ks][0] = pack_bf16x2(x0.x, x0.y);
        ah[ks][1] = pack_bf16x2(x1.x, x1.y);
        ah[ks][2] = pack_bf16x2(x2.x, x2.y);
        ah[ks][3] = pack_bf16x2(x3.x, x3.y);
      } else {
        const float x[4] = {r0[ks * 8 + t], r1[ks * 8 + t], r0[ks * 8 + t + 4], r1[ks * 8 + t + 4]};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          ah[ks][i] = to_tf32(x[i]);
          al[ks][i] = to_tf32(x[i] - __uint_as_float(ah[ks][i]));
        }
      }
    }
    // row bases of this lane's two rows: direct n (a' N + b'), mirrored n (b' N + a');
    // the entry rows are n a' + a1 (direct) and n b' + b1 (mirrored)
    int rd[2], rm[2], ra[2], rb[2];
    bool rv[2], off[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = mt * 16 + g + 8 * h;
      rv[h] = m < NSp;
      const int pr = rv[h] ? pairs[m] : 0;
      const int ap = pr >> 16, bp = pr & 0xffff;
      rd[h] = n * (ap * N + bp);
      rm[h] = n * (bp * N + ap);
      ra[h] = n * ap;
      rb[h] = n * bp;
      off[h] = ap != bp;
    }
    float c[NTN][4];
#pragma unroll
    for (int nt = 0; nt < NTN; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.f;
    // the N tiles' accumulation chains are independent: interleave them
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      if (BF) {
#pragma unroll
        for (int nt = 0; nt < NTN; ++nt) mma_bf16_16816(c[nt], ah[ks], bh[nt][ks]);
#pragma unroll
        for (int nt = 0; nt < NTN; ++nt) mma_bf16_16816(c[nt], ah[ks], bl[nt][ks]);
      } else {
#pragma unroll
        for (int nt = 0; nt < NTN; ++nt) mma_tf32_1688(c[nt], ah[ks], bh[nt][ks]);
#pragma unroll
        for (int nt = 0; nt < NTN; ++nt) mma_tf32_1688(c[nt], ah[ks], bl[nt][ks]);
#pragma unroll
        for (int nt = 0; nt < NTN; ++nt) mma_tf32_1688(c[nt], al[ks], bh[nt][ks]);
      }
    }
#pragma unroll
    for (int nt = 0; nt < NTN; ++nt) {
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int r = h >> 1, cc = h & 1;
        if (rv[r] && cd[nt][cc] >= 0) {
          if constexpr (C::NSPLIT > 1) {
            const int rowd = ra[r] + ca[nt][cc], rowm = rb[r] + cb[nt][cc];
            if (rowd >= r0 && rowd < r1) dst[rd[r] + cd[nt][cc] - off0] = c[nt][h];
            if (off[r] && rowm >= r0 && rowm < r1) dst[rm[r] + cm[nt][cc] - off0] = c[nt][h];
          } else {
            dst[rd[r] + cd[nt][cc]] = c[nt][h];
            if (off[r]) dst[rm[r] + cm[nt][cc]] = c[nt][h];
          }
        }
      }
    }
  }
}

// The staged matrix starts stage_offset(g) floats into the stage buffer, so
// that entry i sits on a 16-byte shared-memory boundary exactly when g + i
// sits on a 16-byte global boundary.
__device__ __forceinline__ int stage_offset(const float* g) {
  const int head = (int)((4 - (((uintptr_t)g >> 2) & 3)) & 3);
  return (4 - head) & 3;
}

// Copy nn floats of a staged element matrix (or row block) to HBM: the
// 16-byte-aligned middle by one bulk asynchronous copy (the untiled form of
// the tensor memory accelerator, issued by thread 0; the callers fence the
// staging writes to the async proxy before their barrier), the scalar head
// and tail by the threads.  Returns once the copy has read shared memory, so
// the caller's next barrier releases the buffer.
template <int NT>
__device__ __forceinline__ void copy_out_bulk(const float* __restrict__ s, float* __restrict__ g,
                                              int nn) {
  const int head = (int)((4 - (((uintptr_t)g >> 2) & 3)) & 3);
  const int h = head < nn ? head : nn;
  const int nv = (nn - h) / 4;
  for (int i = threadIdx.x; i < h; i += NT) g[i] = s[i];
  for (int i = h + 4 * nv + threadIdx.x; i < nn; i += NT) g[i] = s[i];
  if (threadIdx.x == 0 && nv > 0) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n"
                 ::"l"(g + h), "r"(smem_u32(s + h)), "r"(nv * 16) : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
  }
}

// Once per CTA, before its first element: the table of symmetric pairs
// (a',b'), and zeros in the GEMM operands (their padding rows and columns are
// never written by the element stages).
// Stage 3 of one matrix on tcgen05 (called by one thread): for every 128-row
// tile of A, D = A B^T over the K steps of 32 bytes, accumulated in TMEM
// columns d0 + t NU.  FP32: 3xTF32 (A_hi B_hi + A_hi B_lo + A_lo B_hi); BF16:
// A (B_hi + B_lo).
template <class C, int KD>
__device__ __forceinline__ void sf3_issue_um(uint32_t d0, const unsigned char* Ah,
                                             const unsigned char* Al, const unsigned char* Bh,
                                             const unsigned char* Bl) {
  constexpr int EB = C::EB;
  constexpr uint32_t SBO = KD * EB * 8, LBO = 128;
  constexpr uint32_t IDESC = umma_idesc(EB == 2 ? 1u : 2u, 128, C::NU);
  constexpr int KS = KD * EB / 32;
  const uint32_t ah = smem_u32(Ah), bh = smem_u32(Bh), bl = smem_u32(Bl);
  const uint32_t al = Al ? smem_u32(Al) : 0u;
#pragma unroll 1
  for (int t = 0; t < C::MTU; ++t) {
    const uint32_t d = d0 + (uint32_t)(t * C::NU);
    const uint32_t ta = (uint32_t)t * 16u * SBO;   // 128 rows = 16 groups of 8
#pragma unroll
    for (int s = 0; s < KS; ++s) {
      const uint64_t dAh = umma_desc(ah + ta + 256u * s, LBO, SBO);
      const uint64_t dBh = umma_desc(bh + 256u * s, LBO, SBO);
      const uint64_t dBl = umma_desc(bl + 256u * s, LBO, SBO);
      if (EB == 2) {
        umma_f16(d, dAh, dBh, IDESC, s > 0 ? 1u : 0u);
        umma_f16(d, dAh, dBl, IDESC, 1u);
      } else {
        const uint64_t dAl = umma_desc(al + ta + 256u * s, LBO, SBO);
        umma_tf32(d, dAh, dBh, IDESC, s > 0 ? 1u : 0u);
        umma_tf32(d, dAh, dBl, IDESC, 1u);
        umma_tf32(d, dAl, dBh, IDESC, 1u);
      }
    }
  }
}

// Entries K[a1 + n a'][b1 + n b'] = v[a1 n + b1] of one TMEM row (a', b'):
// n contiguous floats per a1, vectorised when the element matrix is aligned.
template <int n, int N>
__device__ __forceinline__ void sf3_store_row_um(float* g, int ap, int bp, const float* v) {
  float* row = g + (int64_t)(n * ap) * N + n * bp;
  if constexpr (n == 4) {
    if ((((uintptr_t)g) & 15u) == 0) {
#pragma unroll
      for (int a1 = 0; a1 < 4; ++a1)
        *(float4*)(row + a1 * N) = make_float4(v[4 * a1], v[4 * a1 + 1], v[4 * a1 + 2], v[4 * a1 + 3]);
      return;
    }
  } else if constexpr (n == 2) {
    if ((((uintptr_t)g) & 7u) == 0) {
#pragma unroll
      for (int a1 = 0; a1 < 2; ++a1) *(float2*)(row + a1 * N) = make_float2(v[2 * a1], v[2 * a1 + 1]);
      return;
    }
  }
#pragma unroll
  for (int a1 = 0; a1 < n; ++a1)
#pragma unroll
    for (int b1 = 0; b1 < n; ++b1) row[a1 * N + b1] = v[a1 * n + b1];
}

// Shared-memory carve-up of the tcgen05 form.
template <class C>
struct UPtrs {
  unsigned char *AKh, *AKl, *AMh, *AMl, *BKh, *BKl, *BMh, *BMl;
  float* region;
  uint64_t* mbar;
  uint32_t* tslot;
  __device__ __forceinline__ explicit UPtrs(float* smf) {
    // operands start on a 128-byte boundary (the size reserves the slack)
    uintptr_t o = (uintptr_t)(smf + C::f_base);
    o = (o + 127) & ~(uintptr_t)127;
    unsigned char* ops = (unsigned char*)o;
    AKh = ops;
    AKl = C::NAU == 2 ? AKh + C::uAK : nullptr;
    AMh = ops + C::NAU * C::uAK;
    AMl = C::NAU == 2 ? AMh + C::uAM : nullptr;
    BKh = ops + C::NAU * (C::uAK + C::uAM);
    BKl = BKh + C::uBK;
    BMh = BKh + 2 * C::uBK;
    BMl = BMh + C::uBM;
    region = (float*)(ops + C::f_uops * 4);
    mbar = (uint64_t*)((float*)ops + C::f_span_u);
    tslot = (uint32_t*)(mbar + 1);
  }
};

// tcgen05 form, once per CTA: zero the operands (padding rows and K columns
// are never written by the element stages), allocate the CTA's TMEM columns
// (warp 0) and initialise the MMA-completion mbarrier.
template <int P, int QG, bool GEN, int MODE, bool BF>
__device__ __forceinline__ void sf3_f32_cta_setup_um(float* smf) {
  using C = SF3F<P, QG, GEN, MODE, BF>;
  UPtrs<C> U(smf);
  uint32_t* ops = (uint32_t*)U.AKh;
  for (int i = threadIdx.x; i < (int)(C::f_uops); i += C::NT) ops[i] = 0u;
  if (threadIdx.x < 32) {
    tmem_alloc(smem_u32(U.tslot), C::TCOLS);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(U.mbar), 1);
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}

// tcgen05 form, once per CTA after its last element: free the TMEM columns.
template <int P, int QG, bool GEN, int MODE, bool BF>
__device__ __forceinline__ void sf3_f32_cta_teardown_um(float* smf) {
  using C = SF3F<P, QG, GEN, MODE, BF>;
  UPtrs<C> U(smf);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (threadIdx.x < 32) tmem_dealloc(*U.tslot, C::TCOLS);
}

template <int P, int QG, bool GEN, int MODE, bool BF>
__device__ __forceinline__ void sf3_f32_cta_setup(float* smf) {
  using C = SF3F<P, QG, GEN, MODE, BF>;
  if constexpr (C::UM) {
    sf3_f32_cta_setup_um<P, QG, GEN, MODE, BF>(smf);
    return;
  }
  constexpr int Np = C::Np, NSp = C::NSp, NT = C::NT;
  float* AK = smf + C::f_px + C::f_py + C::f_pz;
  float* region = AK + C::f_A4 + C::f_B4;
  int* pairs = (int*)(region + C::f_region);
  for (int i = threadIdx.x; i < NSp; i += NT) {
    int a = 0, r = i;
    while (r >= Np - a) { r -= Np - a; ++a; }
    pairs[i] = (a << 16) | (a + r);
  }
  for (int i = threadIdx.x; i < (int)C::f_A; i += NT) AK[i] = 0.f;
  __syncthreads();
}

// One element, all stages.  Called by the per-patch kernel (e = blockIdx.x)
// and by the persistent queue kernel.
// Issue the cp.async copies of element e's inputs: its three 1D basis
// records, kappa, rho and (curved geometry) the Jacobians.
template <class C, bool GEN>
__device__ __forceinline__ void sf3_f32_stage_inputs(const ElemArgs& A, int64_t e, double* rec,
                                                     double* kap, double* rho, double* jac) {
  constexpr int REC = C::REC, Q = C::Q, NT = C::NT;
  const int tid = threadIdx.x;
  int e1, e2, e3;
  elem_coords(A, e, e1, e2, e3);
  for (int i = tid; i < 3 * REC; i += NT) {
    const int d = i / REC, j = i - d * REC;
    const int ek = d == 0 ? e1 : (d == 1 ? e2 : e3);
    const double* tb = d == 0 ? A.tab[0] : (d == 1 ? A.tab[1] : A.tab[2]);
    cp_async8(rec + i, tb + (int64_t)ek * REC + j);
  }
  for (int k = tid; k < Q; k += NT) {
    if (A.kappa) cp_async8(kap + k, A.kappa + e * Q + k);
    else kap[k] = 1.0;
    if (A.rho) cp_async8(rho + k, A.rho + e * Q + k);
    else rho[k] = 1.0;
  }
  if (GEN) {
    const double* G = A.jac + e * Q * 9;
    for (int i = tid; i < 9 * Q; i += NT) cp_async8(jac + i, G + i);
  }
}

// Coefficients of quadrature point k: cofactors and determinant of the
// Jacobian in FP64, the rest in FP32.  General geometry:
//   D = (w kappa / |det G|) c^T c  (c = cofactor matrix, G^{-T} = c / det G),
// the six distinct entries in slots 0 D00, 1 D11, 2 D01, 4 D22, 5 D02, 6 D12,
// and slot 3 the mass weight w |det G| rho; identity geometry: w kappa, w rho.
// Kept out of line: inlined, its FP64 temporaries raise the register count of
// the whole element kernel (64 instead of 40 at p = 3), which costs resident CTAs.
template <class C, bool GEN>
__device__ __noinline__ void sf3_f32_coef(int k, const float* recf, const double* kap,
                                             const double* rho, const double* jac, float* coef) {
  constexpr int q = C::q, n = C::n, Q = C::Q, REC = C::REC;
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
    coef[C::cs(0) * Q + k] = s * (c00 * c00 + c10 * c10 + c20 * c20);
    coef[C::cs(1) * Q + k] = s * (c01 * c01 + c11 * c11 + c21 * c21);
    coef[C::cs(2) * Q + k] = s * (c00 * c01 + c10 * c11 + c20 * c21);
    coef[C::cs(3) * Q + k] = W * adet * rh;
    coef[C::cs(4) * Q + k] = s * (c02 * c02 + c12 * c12 + c22 * c22);
    coef[C::cs(5) * Q + k] = s * (c00 * c02 + c10 * c12 + c20 * c22);
    coef[C::cs(6) * Q + k] = s * (c01 * c02 + c11 * c12 + c21 * c22);
  } else {
    coef[C::cs(0) * Q + k] = W * kp;
    coef[C::cs(3) * Q + k] = W * rh;
  }
}

// Returns false only if the tcgen05 form gave up waiting for its MMAs (the
// error word then holds IGA_ERR_TIMEOUT and the caller stops).  `phase` is the
// parity of the MMA-completion mbarrier (one phase per element).
template <int P, int QG, bool GEN, int MODE, bool BF>
__device__ __forceinline__ bool sf3_f32_element(const ElemArgs& A, int64_t e, float* smf,
                                                uint32_t& phase) {
  using C = SF3F<P, QG, GEN, MODE, BF>;
  constexpr int n = C::n, q = C::q, Q = C::Q, n2 = C::n2, N = C::N, NS1 = C::NS1,
                Np = C::Np, NSp = C::NSp, NT = C::NT, REC = C::REC, RW = C::RW;
  constexpr bool DK = C::DK, DM = C::DM, UM = C::UM;
  float* px = smf;                                   // [n2][4][q]
  float* py = px + C::f_px;                          // [n2][4][q]
  float* pz = py + C::f_py;                          // [n2][3][q]
  float* AK = pz + C::f_pz;                          // [MPs][LDA]   stiffness GEMM operand
  float* AM = AK + (DK ? (size_t)C::MPs * C::LDA : 0);  // [MPs][LDAM]  mass GEMM operand
  uint32_t* BK = (uint32_t*)(AK + C::f_A4);   // [2][NPAD][LDB]
  uint32_t* BM = BK + (DK ? (size_t)2 * C::NPAD * C::LDB : 0);  // [2][NPAD][LDBM]
  const UPtrs<C> U(smf);                             // tcgen05 form
  float* region = UM ? U.region : (float*)BK + C::f_B4;
  float* T1 = region;                                // [NTERM][n2][TS]
  float* coef = T1 + (UM ? C::f_T1u : C::f_T1);      // [NCOEF][Q]
  // tcgen05 form: the staging lives in T1's space (dead before stage 1)
  double* geo = UM ? (double*)T1 : (double*)(coef + C::f_coef);
  double* rec = geo;                                 // [3][REC]
  double* kap = rec + 3 * REC;                       // [Q]
  double* rho = kap + Q;                             // [Q]
  double* jac = rho + Q;                             // [Q][9]
  float* recf = (float*)(geo + C::d_geo);            // [3][REC]
  float* outs = region;                              // [N][N] after stage 2
  int* pairs = (int*)(region + C::f_region);         // [NSp] packed (a' << 16 | b')

  const int tid = threadIdx.x;
  int e1, e2, e3;
  elem_coords(A, e, e1, e2, e3);
  __syncthreads();  // shared memory of the previous element is no longer read

  // ---- coalesced staging of this element's inputs -------------------------------
  // every copy of this thread is issued before any completes (cp.async)
  sf3_f32_stage_inputs<C, GEN>(A, e, rec, kap, rho, jac);
  cp_async_wait_all();
  // each thread converts the records it copied itself (visible to it after the
  // wait), so one barrier serves both
  for (int i = tid; i < 3 * REC; i += NT) recf[i] = (float)rec[i];
  __syncthreads();

  // ---- quadrature-point coefficients (taken from the last threads down) and ------
  // ---- the 1D factor pattern records in FP32 (from the first threads up) --------
  for (int k = NT - 1 - tid; k < Q; k += NT) sf3_f32_coef<C, GEN>(k, recf, kap, rho, jac, coef);
  for (int it = tid; it < 3 * n2 * q; it += NT) {
    const int d = it / (n2 * q), i = it % (n2 * q);
    const int a = i / (n * q), b = (i / q) % n, k = i % q;
    const int ab = a * n + b;
    {
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
        float* r = pz + ab * C::RZ;
        r[0 * q + k] = va * vb; r[1 * q + k] = da * db; r[2 * q + k] = va * db;
      }
    }
  }
  __syncthreads();

  // ---- B operands: x patterns split into hi + lo (TF32 bits or bf16 pairs) ------
  // B[(a1,b1)][X q + k1] = P^X_x[a1][b1][k1] in the record order 11, 00, 10, 01
  // (the same X order as the A columns); mass: B[(a1,b1)][k1] = P^00_x
  if constexpr (UM) {
    // B[(a1,b1)][X q + k1] in the core-matrix layout, hi + lo
    if (DK) {
      for (int i = tid; i < C::NU * C::KA; i += NT) {
        const int nn = i / C::KA, k = i % C::KA;
        const float v = (nn < n2 && k < C::NXK * q) ? px[nn * RW + k] : 0.f;
        uput<BF, C::KA>(U.BKh, U.BKl, nn, k, v);
      }
    }
    if (DM) {
      for (int i = tid; i < C::NU * C::KAM; i += NT) {
        const int nn = i / C::KAM, k = i % C::KAM;
        const float v = (nn < n2 && k < q) ? px[nn * RW + q + k] : 0.f;
        uput<BF, C::KAM>(U.BMh, U.BMl, nn, k, v);
      }
    }
  }
#pragma unroll 1
  for (int mat = 0; mat < (UM ? 0 : 2); ++mat) {
    if ((mat == 0 && !DK) || (mat == 1 && !DM)) continue;
    uint32_t* Bm = mat == 0 ? BK : BM;
    const int ld = mat == 0 ? C::LDB : C::LDBM;
    const int kdepth = mat == 0 ? C::KA : C::KAM;
    const int kvalid = mat == 0 ? C::NXK * q : q;
    const int kofs = mat == 0 ? 0 : q;
    if (BF) {
      for (int i = tid; i < C::NPAD * (kdepth / 2); i += NT) {
        const int nn = i / (kdepth / 2), kw = i % (kdepth / 2);
        float v[2], hv[2];
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
          const int k = 2 * kw + s2;
          v[s2] = (nn < n2 && k < kvalid) ? px[nn * RW + kofs + k] : 0.f;
          hv[s2] = __bfloat162float(__float2bfloat16_rn(v[s2]));
        }
        Bm[nn * ld + kw] = pack_bf16x2(hv[0], hv[1]);
        Bm[(C::NPAD + nn) * ld + kw] = pack_bf16x2(v[0] - hv[0], v[1] - hv[1]);
      }
    } else {
      for (int i = tid; i < C::NPAD * kdepth; i += NT) {
        const int nn = i / kdepth, k = i % kdepth;
        const float v = (nn < n2 && k < kvalid) ? px[nn * RW + kofs + k] : 0.f;
        const uint32_t hi = to_tf32(v);
        Bm[nn * ld + k] = hi;
        Bm[(C::NPAD + nn) * ld + k] = to_tf32(v - __uint_as_float(hi));
      }
    }
  }

  const float* Pz = pz;
  const float* Py = py;
  // ---- stage 1: T_t[a3][b3][k1][k2] = sum_k3 Z_t[a3][b3][k3] D_t[k1,k2,k3] -------
  // item = (k1, k2, a3, part of the b3 range), coefficients of the item in
  // registers, loop over its b3
  constexpr int S1 = (q * q * n >= NT) ? 1 : ((NT / (q * q * n)) < n ? (NT / (q * q * n)) : n);
  constexpr int CH = (n + S1 - 1) / S1;
  for (int it = tid; it < q * q * n * S1; it += NT) {
    const int part = it % S1, rest = it / S1;
    const int a3 = rest % n, kk = rest / n;  // kk = k1 + q k2
    float d0[q], d1[q], d2[q], d3[q], d4[q], d5[q], d6[q];
#pragma unroll
    for (int k3 = 0; k3 < q; ++k3) {
      const int o = kk + q * q * k3;
      d0[k3] = coef[C::cs(0) * Q + o];
      d3[k3] = coef[C::cs(3) * Q + o];
      if (GEN) {
        d1[k3] = coef[C::cs(1) * Q + o]; d2[k3] = coef[C::cs(2) * Q + o]; d4[k3] = coef[C::cs(4) * Q + o];
        d5[k3] = coef[C::cs(5) * Q + o]; d6[k3] = coef[C::cs(6) * Q + o];
      }
    }
    const int b3e = (part + 1) * CH < n ? (part + 1) * CH : n;
#pragma unroll
    for (int bo = 0; bo < CH; ++bo) {
      const int b3 = part * CH + bo;
      if (b3 >= b3e) break;
      const float* z = Pz + (a3 * n + b3) * C::RZ;
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
      const int o = (a3 * n + b3) * C::TS + kk;
      constexpr int S = n2 * C::TS;
      if (DK) {
        T1[C::ts(0) * S + o] = t0; T1[C::ts(4) * S + o] = t4;
        if (GEN) { T1[C::ts(1) * S + o] = t1; T1[C::ts(2) * S + o] = t2; T1[C::ts(5) * S + o] = t5; T1[C::ts(6) * S + o] = t6; }
      }
      if (DM) T1[C::ts(3) * S + o] = t3;
    }
  }
  __syncthreads();

  // ---- stage 2: the GEMM operand rows (a',b'), a' <= b' --------------------------
  {
    constexpr int S = n2 * C::TS;
    constexpr int T11 = GEN ? 1 : 0;
    if constexpr (UM && C::FULLR && C::VEC2) {
      // p = 3, q = 4, identity geometry: item = (a3 <= b3, a2, b2), all four
      // k1 at once, so that each operand row receives whole 16-byte chunks:
      // FP32 A[m][X q + k1], k1 = 0..3, is one chunk per pattern X (hi and
      // lo), BF16 holds both patterns of K in one chunk and the mass in half
      // of one.  Threads: b2 fastest, then a2, then the (a3, b3) pair.
      static_assert(n == 4 && q == 4 && !GEN, "VEC2 is the p = 3, q = 4 identity form");
      const float4* T4 = (const float4*)T1;
      constexpr int S4 = S / 4, TS4 = C::TS / 4;
      for (int it = tid; it < NS1 * n2; it += NT) {
        const int b2 = it & 3, a2 = (it >> 2) & 3, ps = it >> 4;
        int a3 = 0, rr = ps;
        while (rr >= n - a3) { rr -= n - a3; ++a3; }
        const int b3 = a3 + rr;
        const float4* y4 = (const float4*)(Py + (a2 * n + b2) * RW);  // 00, 11, 10, 01
        const float4 y00 = y4[0], y11 = y4[1];
        const float ya[4] = {y00.x, y00.y, y00.z, y00.w}, yb[4] = {y11.x, y11.y, y11.z, y11.w};
        const int ab3 = (a3 * n + b3) * TS4;
        float4 c11 = make_float4(0.f, 0.f, 0.f, 0.f), c00 = c11, cm = c11;
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          if (DK) {
            const float4 t0 = T4[C::ts(0) * S4 + ab3 + k2], t4 = T4[C::ts(4) * S4 + ab3 + k2];
            c11.x = fmaf(ya[k2], t0.x, c11.x); c11.y = fmaf(ya[k2], t0.y, c11.y);
            c11.z = fmaf(ya[k2], t0.z, c11.z); c11.w = fmaf(ya[k2], t0.w, c11.w);
            c00.x = fmaf(yb[k2], t0.x, fmaf(ya[k2], t4.x, c00.x));
            c00.y = fmaf(yb[k2], t0.y, fmaf(ya[k2], t4.y, c00.y));
            c00.z = fmaf(yb[k2], t0.z, fmaf(ya[k2], t4.z, c00.z));
            c00.w = fmaf(yb[k2], t0.w, fmaf(ya[k2], t4.w, c00.w));
          }
          if (DM) {
            const float4 t3 = T4[C::ts(3) * S4 + ab3 + k2];
            cm.x = fmaf(ya[k2], t3.x, cm.x); cm.y = fmaf(ya[k2], t3.y, cm.y);
            cm.z = fmaf(ya[k2], t3.z, cm.z); cm.w = fmaf(ya[k2], t3.w, cm.w);
          }
        }
        const int ap = a2 + n * a3, bp = b2 + n * b3;
        const int m1 = urow<n2, C::VEC2>(ap, bp), m2 = urow<n2, C::VEC2>(bp, ap);
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          if (side == 1 && m2 == m1) break;
          const int m = side == 0 ? m1 : m2;
          // K-major core matrices: 8-row groups (8 rows x 16 bytes per K chunk)
          const int base = (m >> 3) * (8 * 8 * C::EB * (C::KA / 8)) + (m & 7) * 16;
          if constexpr (BF) {
            if (DK) {
              uint4 w;
              w.x = pack_bf16x2(c11.x, c11.y); w.y = pack_bf16x2(c11.z, c11.w);
              w.z = pack_bf16x2(c00.x, c00.y); w.w = pack_bf16x2(c00.z, c00.w);
              *(uint4*)(U.AKh + base) = w;
            }
            if (DM) {
              const int bm = (m >> 3) * (8 * 8 * C::EB * (C::KAM / 8)) + (m & 7) * 16;
              *(uint2*)(U.AMh + bm) = make_uint2(pack_bf16x2(cm.x, cm.y), pack_bf16x2(cm.z, cm.w));
            }
          } else {
            if (DK) {
              *(float4*)(U.AKh + base) = c11;
              *(float4*)(U.AKh + base + 128) = c00;
              *(float4*)(U.AKl + base) = make_float4(c11.x - tf32_trunc(c11.x), c11.y - tf32_trunc(c11.y),
                                                     c11.z - tf32_trunc(c11.z), c11.w - tf32_trunc(c11.w));
              *(float4*)(U.AKl + base + 128) = make_float4(c00.x - tf32_trunc(c00.x), c00.y - tf32_trunc(c00.y),
                                                           c00.z - tf32_trunc(c00.z), c00.w - tf32_trunc(c00.w));
            }
            if (DM) {
              const int bm = (m >> 3) * (8 * 8 * C::EB * (C::KAM / 8)) + (m & 7) * 16;
              *(float4*)(U.AMh + bm) = cm;
              *(float4*)(U.AMl + bm) = make_float4(cm.x - tf32_trunc(cm.x), cm.y - tf32_trunc(cm.y),
                                                   cm.z - tf32_trunc(cm.z), cm.w - tf32_trunc(cm.w));
            }
          }
        }
      }
    } else {
      // (a) C11, C00, CM: item = (a3 <= b3, k1, a2)
      for (int it = tid; it < NS1 * q * n; it += NT) {
        const int a2 = it % n, r = it / n, k1 = r % q, ps = r / q;
        int a3 = 0, rr = ps;
        while (rr >= n - a3) { rr -= n - a3; ++a3; }
        const int b3 = a3 + rr;
        // T layout [t][a3][b3][k1 + q k2]
        const int ab3 = (a3 * n + b3) * C::TS + k1, ba3 = (b3 * n + a3) * C::TS + k1;
        float t00[q], t11[q], t22[q], tab[q], tba[q], tm[q];
  #pragma unroll
        for (int k2 = 0; k2 < q; ++k2) {
          if (DK) {
            t00[k2] = T1[C::ts(0) * S + ab3 + q * k2];
            t11[k2] = T1[C::ts(T11) * S + ab3 + q * k2];
            t22[k2] = T1[C::ts(4) * S + ab3 + q * k2];
            if (GEN) { tab[k2] = T1[C::ts(6) * S + ab3 + q * k2]; tba[k2] = T1[C::ts(6) * S + ba3 + q * k2]; }
          }
          if (DM) tm[k2] = T1[C::ts(3) * S + ab3 + q * k2];
        }
        const int ap = a2 + n * a3;
        const int b2s = (a3 == b3 ? a2 : 0);
        const int pp0 = upper_index<Np>(ap, b2s + n * b3) - b2s;  // rows are consecutive in b2
  #pragma unroll
        for (int b2 = 0; b2 < n; ++b2) {
          if (b2 < b2s) continue;
          const int pp = pp0 + b2;
          const float4* y4 = (const float4*)(Py + (a2 * n + b2) * RW);  // 00, 11, 10, 01
          float y[RW];
  #pragma unroll
          for (int v = 0; v < RW / 4; ++v) {
            const float4 w4 = y4[v];
            y[4 * v] = w4.x; y[4 * v + 1] = w4.y; y[4 * v + 2] = w4.z; y[4 * v + 3] = w4.w;
          }
          float c11 = 0.f, c00a = 0.f, c00b = 0.f, cm = 0.f;
  #pragma unroll
          for (int k2 = 0; k2 < q; ++k2) {
            if (DK) {
              c11 = fmaf(y[k2], t00[k2], c11);
              c00a = fmaf(y[q + k2], t11[k2], c00a);
              c00b = fmaf(y[k2], t22[k2], c00b);
              if (GEN) {
                c00a = fmaf(y[2 * q + k2], tab[k2], c00a);
                c00b = fmaf(y[3 * q + k2], tba[k2], c00b);
              }
            }
            if (DM) cm = fmaf(y[k2], tm[k2], cm);
          }
          if constexpr (UM && !C::FULLR) {
            // rows a' <= b' only; the K columns past the data are rewritten with
            // zeros (the staged matrix of the previous element covered them)
            if (DK) {
              uput<BF, C::KA>(U.AKh, U.AKl, pp, 0 * q + k1, c11);
              uput<BF, C::KA>(U.AKh, U.AKl, pp, 1 * q + k1, c00a + c00b);
              if (k1 == 0)
                for (int kz = C::NXK * q; kz < C::KA; ++kz) uput<BF, C::KA>(U.AKh, U.AKl, pp, kz, 0.f);
            }
            if (DM) {
              uput<BF, C::KAM>(U.AMh, U.AMl, pp, k1, cm);
              if (k1 == 0)
                for (int kz = q; kz < C::KAM; ++kz) uput<BF, C::KAM>(U.AMh, U.AMl, pp, kz, 0.f);
            }
          } else if constexpr (UM) {
            // rows (a', b') and (b', a'): the patterns 11, 00 and the mass are
            // symmetric under the exchange
            const int bp = b2 + n * b3;
            const int m1 = urow<n2, C::VEC2>(ap, bp), m2 = urow<n2, C::VEC2>(bp, ap);
            if (DK) {
              uput<BF, C::KA>(U.AKh, U.AKl, m1, 0 * q + k1, c11);
              uput<BF, C::KA>(U.AKh, U.AKl, m1, 1 * q + k1, c00a + c00b);
              if (m2 != m1) {
                uput<BF, C::KA>(U.AKh, U.AKl, m2, 0 * q + k1, c11);
                uput<BF, C::KA>(U.AKh, U.AKl, m2, 1 * q + k1, c00a + c00b);
              }
            }
            if (DM) {
              uput<BF, C::KAM>(U.AMh, U.AMl, m1, k1, cm);
              if (m2 != m1) uput<BF, C::KAM>(U.AMh, U.AMl, m2, k1, cm);
            }
          } else {
            if (DK) {
              AK[pp * C::LDA + 0 * q + k1] = c11;
              AK[pp * C::LDA + 1 * q + k1] = c00a + c00b;
            }
            if (DM) AM[pp * C::LDAM + k1] = cm;
          }
        }
      }
    }
    // (b) C10[a'][b'] for all (a', b'): row pp(a',b') column 2q+k1 when a' <= b'
    // and, as C01 of the row pp(b',a'), column 3q+k1 when b' <= a'
    if (GEN && DK) {
      for (int it = tid; it < n2 * q * n; it += NT) {
        const int a2 = it % n, r = it / n, k1 = r % q, ab = r / q;
        const int a3 = ab / n, b3 = ab % n;
        const int o = (a3 * n + b3) * C::TS + k1;
        float t01[q], t02[q];
#pragma unroll
        for (int k2 = 0; k2 < q; ++k2) {
          t01[k2] = T1[C::ts(2) * S + o + q * k2];
          t02[k2] = T1[C::ts(5) * S + o + q * k2];
        }
        const int ap = a2 + n * a3;
#pragma unroll
        for (int b2 = 0; b2 < n; ++b2) {
          const float4* y4 = (const float4*)(Py + (a2 * n + b2) * RW);
          float y[RW];
#pragma unroll
          for (int v = 0; v < RW / 4; ++v) {
            const float4 w4 = y4[v];
            y[4 * v] = w4.x; y[4 * v + 1] = w4.y; y[4 * v + 2] = w4.z; y[4 * v + 3] = w4.w;
          }
          float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
          for (int k2 = 0; k2 < q; ++k2) {
            acc0 = fmaf(y[3 * q + k2], t01[k2], acc0);  // y01 with z00 D01 (term (0,1))
            acc1 = fmaf(y[k2], t02[k2], acc1);          // y00 with z01 D02 (term (0,2))
          }
          const float val = acc0 + acc1;
          const int bp = b2 + n * b3;
          if constexpr (UM && !C::FULLR) {
            if (ap <= bp) uput<BF, C::KA>(U.AKh, U.AKl, upper_index<Np>(ap, bp), 2 * q + k1, val);
            if (bp <= ap) uput<BF, C::KA>(U.AKh, U.AKl, upper_index<Np>(bp, ap), 3 * q + k1, val);
          } else if constexpr (UM) {
            // C10 of row (a', b') is C01 of row (b', a')
            uput<BF, C::KA>(U.AKh, U.AKl, urow<n2, C::VEC2>(ap, bp), 2 * q + k1, val);
            uput<BF, C::KA>(U.AKh, U.AKl, urow<n2, C::VEC2>(bp, ap), 3 * q + k1, val);
          } else {
            if (ap <= bp) AK[upper_index<Np>(ap, bp) * C::LDA + 2 * q + k1] = val;
            if (bp <= ap) AK[upper_index<Np>(bp, ap) * C::LDA + 3 * q + k1] = val;
          }
        }
      }
    }
  }
  __syncthreads();

  if constexpr (UM) {
    // ---- stage 3 on tcgen05: MMAs into TMEM, then TMEM rows straight to HBM -----
    fence_proxy_async_smem();  // the operands written above are read by the tensor core
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *U.tslot;
    constexpr uint32_t colM = DK ? C::MTU * C::NU : 0;
    if (tid == 0) {
      if (DK) sf3_issue_um<C, C::KA>(tmem, U.AKh, U.AKl, U.BKh, U.BKl);
      if (DM) sf3_issue_um<C, C::KAM>(tmem + colM, U.AMh, U.AMl, U.BMh, U.BMl);
      umma_commit(smem_u32(U.mbar));
    }
    const bool done = mbar_wait_bounded(smem_u32(U.mbar), phase, 1000000000ull);
    phase ^= 1u;
    if (!__syncthreads_and(done)) {
      if (tid == 0) atomicCAS(A.err, 0, (int)IGA_ERR_TIMEOUT);
      return false;
    }
    fence_after_sync();
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll 1
    for (int mat = 0; mat < 2; ++mat) {
      if ((mat == 0 && !DK) || (mat == 1 && !DM)) continue;
      float* g = (float*)(mat == 0 ? A.K_out : A.M_out) + e * (int64_t)N * N;
      const uint32_t col0 = mat == 0 ? 0u : colM;
      if constexpr (C::FULLR) {
#pragma unroll 1
        for (int t = warp >> 2; t < C::MTU; t += NT / 128) {
          float v[16];
          tmem_ld16(tmem + col0 + (uint32_t)(t * C::NU) + ((uint32_t)(32 * (warp & 3)) << 16), v);
          const int m = t * 128 + 32 * (warp & 3) + lane;
          if (m < n2 * n2) {
            int ap, bp;
            urow_inv<n2, C::VEC2>(m, ap, bp);
            sf3_store_row_um<n, N>(g, ap, bp, v);
          }
        }
      } else {
        // rows a' <= b': entry (a1 + n a', b1 + n b') and its mirror into the
        // staged matrix (over the operands, all read by now), then one
        // coalesced copy to HBM
        float* stage = (float*)U.AKh + stage_offset(g);
#pragma unroll 1
        for (int t = warp >> 2; t < C::MTU; t += NT / 128) {
          float v[C::NU];
          const uint32_t ta = tmem + col0 + (uint32_t)(t * C::NU) + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll
          for (int c = 0; c < C::NU; c += 16) tmem_ld16(ta + c, v + c);
          const int m = t * 128 + 32 * (warp & 3) + lane;
          if (m < NSp) {
            int ap = 0, r = m;
            while (r >= Np - ap) { r -= Np - ap; ++ap; }
            const int bp = ap + r;
#pragma unroll
            for (int a1 = 0; a1 < n; ++a1)
#pragma unroll
              for (int b1 = 0; b1 < n; ++b1) {
                const float x = v[a1 * n + b1];
                stage[(a1 + n * ap) * N + n * bp + b1] = x;
                if (ap != bp) stage[(b1 + n * bp) * N + n * ap + a1] = x;
              }
          }
        }
        fence_proxy_async_smem();
        __syncthreads();
        copy_out_bulk<NT>(stage, g, N * N);
        __syncthreads();
      }
    }
    fence_before_sync();
    return true;
  }

  // ---- stage 3 on the tensor cores, one matrix at a time ---------------------------
#pragma unroll 1
  for (int mat = 0; mat < 2; ++mat) {
    const bool isK = mat == 0;
    if ((isK && !DK) || (!isK && !DM)) continue;
    float* dst = (float*)(isK ? A.K_out : A.M_out);
    if (!dst) continue;
    float* g = dst + e * (int64_t)N * N;
#pragma unroll 1
    for (int blk = 0; blk < (C::STAGE ? C::NSPLIT : 1); ++blk) {
      const int r0 = blk * C::RB, r1 = (r0 + C::RB < N) ? r0 + C::RB : N;
      float* gb = g + (int64_t)r0 * N;
      float* stage = outs + stage_offset(gb);
      if (isK) gemm_sym<C, C::LDA, C::LDB, C::KA / C::KSTEP>(AK, BK, pairs, stage, g, r0, r1);
      else gemm_sym<C, C::LDAM, C::LDBM, C::KAM / C::KSTEP>(AM, BM, pairs, stage, g, r0, r1);
      if (C::STAGE) {
        fence_proxy_async_smem();
        __syncthreads();
        copy_out_bulk<NT>(stage, gb, (r1 - r0) * N);
        __syncthreads();
      }
    }
  }
  return true;
}

template <int P, int QG, bool GEN, int MODE, bool BF>
__global__ void __launch_bounds__(SF3F<P, QG, GEN, MODE, BF>::NT) k_sf3_f32(const ElemArgs A) {
  extern __shared__ __align__(16) float smf[];
  sf3_f32_cta_setup<P, QG, GEN, MODE, BF>(smf);
  uint32_t phase = 0;
  for (int64_t e = blockIdx.x; e < A.n_elem; e += gridDim.x)
    if (!sf3_f32_element<P, QG, GEN, MODE, BF>(A, e, smf, phase)) break;
  if constexpr (SF3F<P, QG, GEN, MODE, BF>::UM) sf3_f32_cta_teardown_um<P, QG, GEN, MODE, BF>(smf);
}

// Persistent form: every CTA pops work items (patch, first element, count)
// from the class's device queue until it is empty.  A work item is checked
// against its patch before use (IGA_ERR_DEVICE otherwise).  With a non-zero
// time budget, a CTA stops popping once the budget since its start has passed
// and records IGA_ERR_TIMEOUT; no CTA ever waits on another.
template <int P, int QG, bool GEN, int MODE, bool BF>
__global__ void __launch_bounds__(SF3F<P, QG, GEN, MODE, BF>::NT) k_sf3_f32_queue(const QueueArgs B) {
  extern __shared__ __align__(16) float smf[];
  __shared__ int s_item;
  const unsigned long long t0 = global_timer_ns();
  sf3_f32_cta_setup<P, QG, GEN, MODE, BF>(smf);
  uint32_t phase = 0;
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
    bool ok = true;
    for (int64_t e = w.e0; e < w.e0 + w.count && ok; ++e)
      ok = sf3_f32_element<P, QG, GEN, MODE, BF>(A, e, smf, phase);
    if (!ok) break;
  }
  if constexpr (SF3F<P, QG, GEN, MODE, BF>::UM) sf3_f32_cta_teardown_um<P, QG, GEN, MODE, BF>(smf);
}

// Resident CTAs per SM of a kernel using TMEM.  The runtime's occupancy query
// answers 1 for such kernels (it cannot see how many TMEM columns a CTA
// takes), so the count comes from the kernel's registers and shared memory,
// the SM's limits, and the 512 TMEM columns of an SM.
cudaError_t resident_ctas_tmem(const void* kernel, int nt, size_t smem, int tcols, int* out) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  int dev = 0, smem_sm = 0, res_blk = 0, regs_sm = 0, thr_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&res_blk, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  if (e != cudaSuccess) return e;
  const size_t per_block = (smem + fa.sharedSizeBytes + res_blk + 127) / 128 * 128;
  int n = (int)(smem_sm / per_block);
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
  const int by_regs = regs_sm / (regs_warp * (nt / 32));
  if (by_regs < n) n = by_regs;
  if (thr_sm / nt < n) n = thr_sm / nt;
  if (512 / tcols < n) n = 512 / tcols;
  *out = n > 0 ? n : 1;
  return cudaSuccess;
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
    static int capacity = 0;  // resident CTAs on this GPU, looked up once
    cudaError_t e = cudaSuccess;
    if (capacity == 0) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
      int dev = 0, sms = 0, per_sm = 0;
      if (e == cudaSuccess) e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      // the tcgen05 form sizes its grid from the full shared-memory carveout
      if (e == cudaSuccess && C::UM)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
      if (e == cudaSuccess) {
        if (C::UM) e = resident_ctas_tmem((const void*)k, C::NT, C::smem, C::TCOLS, &per_sm);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, C::NT, C::smem);
      }
      if (e != cudaSuccess) return e;
      capacity = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int64_t grid = a.n_elem < capacity ? a.n_elem : capacity;
    k<<<(unsigned)grid, C::NT, C::smem, st>>>(a);
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
    if (e == cudaSuccess && C::UM)
      e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if (max_grid) {
      int dev = 0, sms = 0, per_sm = 0;
      e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) {
        if (C::UM) e = resident_ctas_tmem((const void*)k, C::NT, C::smem, C::TCOLS, &per_sm);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, C::NT, C::smem);
      }
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
}  // namespace iga
