// k_stream32.cu -- FP32 and BF16 sum-factorized element matrices for 3D
// p = 4 and 5: stage 3 on tcgen05 in 128-row tiles, streamed.
//
// Algorithm 2 (Sec. 3.2) as in k_sumfact32.cuh -- stage 1 contracts z, stage 2
// y, stage 3 x -- with the last stage a GEMM per element:
//   K[a1 + n a'][b1 + n b'] = sum_{X,k1} C^X[(a',b')][k1] P^X_x[(a1,b1)][k1].
// At p >= 4 the operand of all n^4 rows (a', b') does not fit in shared memory
// beside the other stages, so the CTA-per-element kernel there kept only the
// symmetric rows a' <= b' and scattered every result and its mirror into a
// staged copy of the element matrix before writing it out.  This form instead
// produces all of the rows, in tiles of whole a' blocks: APT = floor(128 / n^2)
// values of a' (5 at p = 4, 3 at p = 5) and all n^2 values of b' per 128-row
// MMA tile.  The entries of such a tile, K[a1 + n a'][b1 + n b'], fill the
// complete output rows n a'_0 .. n (a'_0 + APT) - 1: one contiguous block of
// the element matrix.
// The warps of a CTA split the tile loop (warp specialisation):
//   producers (warps 4-11): stage 2 writes the rows of tile t into the operand
//            buffer (once the MMAs of tile t-1 have read it); one thread
//            issues the tile's MMAs into TMEM buffer t mod 2 (once the
//            consumers have read that buffer's tile t-2) and commits them to
//            the MMA mbarrier of the buffer;
//   consumers (warps 0-3, one per TMEM lane quarter): wait for the MMAs of
//            tile t, read the accumulators (tcgen05.ld, one TMEM lane = one
//            row (a', b') per thread), release the TMEM buffer (its "free"
//            mbarrier), place the entries in a shared-memory copy of the
//            tile's output block (thread (a', b') writes n floats per a1 at
//            stride n from its neighbours: no bank conflicts at odd n; 8-byte
//            stores at even n), and move the block to HBM with one bulk
//            asynchronous copy; three or four staging buffers rotate, so two
//            copies can be in flight while the next block is filled (with four,
//            the K and M blocks of a tile are staged between one pair of group
//            barriers).
// Stage 2 for the identity map takes one thread per operand row and value
// group, all q values k1 at once (st_stage2_rows); the general map one value
// per thread (st_stage2).
// Producers and consumers meet only at these mbarriers and at the start of
// an element; every wait is bounded.
// The symmetric half of stage 2 is computed twice (once per row order), which
// costs FP32 FMAs but no mirrored scatter.  FP32: 3xTF32 (A_hi B_hi + A_hi B_lo + A_lo B_hi);
// BF16: A (B_hi + B_lo); FP32 accumulation in TMEM.  The Jacobian cofactors
// and determinant are formed in FP64 (sf3_f32_coef).
#include "k_sumfact32.cuh"

namespace iga {
namespace {

template <int P, int QG, bool GEN, int MODE, bool BF>
struct ST {
  static constexpr bool DK = (MODE & 3) != 2, DM = (MODE & 3) != 1;
  static constexpr int n = P + 1, q = QG, Q = q * q * q, n2 = n * n, N = n2 * n;
  static constexpr int NR = n2 * n2;                  // A rows (a', b'), all orders
  static constexpr int APT = 128 / n2;                // values of a' per tile
  static constexpr int RT = APT * n2;                 // rows used of a 128-row tile
  static constexpr int MT = (n2 + APT - 1) / APT;     // tiles
  // one output block, + alignment slack; a multiple of 4 floats, so that the
  // second staging buffer starts on a 16-byte boundary like the first (the
  // bulk copies read both from 16-byte-aligned addresses)
  static constexpr size_t f_stage = ((size_t)n * APT * N + 8 + 3) / 4 * 4;
  static constexpr int NT = 384;                      // 4 consumer + 8 producer warps
  static constexpr int NP = NT - 128;                 // producer threads
  static constexpr int REC = 2 * q * n + q;
  static constexpr int RW = 4 * q;                    // x, y pattern records: 4 patterns
  static constexpr int RZ = (3 * q) % 2 == 0 ? 3 * q + 1 : 3 * q;
  // stage-1 row stride: identity map, a multiple of 4 (stage 2 reads the q
  // values k1 of one k2 as 16- and 8-byte vectors); general map, odd (its
  // stage 2 reads one value per thread, consecutive threads along k1)
  static constexpr int TS = !GEN ? (q * q + 3) / 4 * 4 : ((q * q) % 2 == 0 ? q * q + 1 : q * q);
  static constexpr int NTERM = GEN ? 7 : 3, NCOEF = GEN ? 7 : 2;
  // stage-1 term and coefficient slots (the identity map keeps terms 0, 3, 4
  // and coefficients W kappa, W rho)
  static constexpr int ts(int t) { return GEN ? t : (t == 0 ? 0 : (t == 3 ? 1 : 2)); }
  static constexpr int cs(int t) { return GEN ? t : (t == 0 ? 0 : 1); }
  static constexpr int NXK = GEN ? 4 : 2;
  static constexpr int EB = BF ? 2 : 4;
  static constexpr int KSTEP = 32 / EB;
  static constexpr int rup(int x, int m) { return (x + m - 1) / m * m; }
  static constexpr int KA = rup(NXK * q, KSTEP), KAM = rup(q, KSTEP);
  static constexpr int NU = rup(n2, 16);              // MMA N: columns (a1, b1)
  static constexpr int NAU = BF ? 1 : 2;              // A arrays: hi (+ lo)
  // bytes
  static constexpr size_t tAK = DK ? (size_t)128 * KA * EB : 0, tAM = DM ? (size_t)128 * KAM * EB : 0;
  static constexpr size_t tile_bytes = NAU * (tAK + tAM);              // one A buffer
  static constexpr size_t bBK = DK ? (size_t)NU * KA * EB : 0, bBM = DM ? (size_t)NU * KAM * EB : 0;
  static constexpr size_t b_bytes = 2 * (bBK + bBM);                     // B hi + lo
  static constexpr size_t al128(size_t x) { return (x + 127) / 128 * 128; }
  static constexpr size_t o_A0 = 0, o_B = al128(tile_bytes);
  static constexpr size_t ops_bytes = o_B + al128(b_bytes);
  // floats after the operands
  static constexpr size_t f_px = (size_t)n2 * RW, f_py = (size_t)n2 * RW, f_pz = (size_t)n2 * RZ + 1;
  static constexpr size_t f_T1 = (size_t)NTERM * n2 * TS;
  static constexpr size_t f_coef = (size_t)NCOEF * Q;
  static constexpr size_t d_geo = 3 * REC + 2 * (size_t)Q + (GEN ? 9 * (size_t)Q : 0);  // doubles
  static constexpr size_t f_geo = 2 * d_geo + 3 * REC;   // the FP64 staging + FP32 records
  // the staging is dead once the coefficients exist, before stage 1 writes T1
  static constexpr size_t f_T1g = (f_T1 > f_geo ? f_T1 : f_geo) + 4;
  static constexpr size_t floats_for(int nb) { return f_px + f_py + f_pz + f_T1g + f_coef + nb * f_stage + 8; }
  static constexpr size_t smem_for(int nb) { return ops_bytes + 4 * floats_for(nb) + 96 + 128; }
  // output staging buffers: four where they fit beside the CTAs per SM of the
  // form (two of at most 112 KB for the identity map, one for the general
  // map) -- the K and M blocks of one tile then share one pair of group
  // barriers, with the two copies of the previous tile still in flight --
  // else three (one matrix per step, two copies in flight)
  static constexpr int NSTG = smem_for(4) <= (GEN ? 227 * 1024 : 112 * 1024) ? 4 : 3;
  static constexpr size_t floats = floats_for(NSTG);
  static constexpr size_t smem = smem_for(NSTG);   // + mbarriers, slot, align
  static_assert(f_stage % 4 == 0, "staging buffers must stay 16-byte aligned");
  static constexpr int CPB = (DK ? NU : 0) + (DM ? NU : 0);          // TMEM columns per buffer
  static constexpr int TCOLS = 2 * CPB <= 32 ? 32 : 2 * CPB <= 64 ? 64 : 2 * CPB <= 128 ? 128
                               : 2 * CPB <= 256 ? 256 : 512;
};

template <class C>
struct SPtrs {
  unsigned char* A0;       // the operand tile: K hi, K lo, M hi, M lo
  unsigned char *BKh, *BKl, *BMh, *BMl;
  float *px, *py, *pz, *T1, *coef, *recf, *stage0, *stage1, *stage2, *stage3;
  double *rec, *kap, *rho, *jac;
  uint64_t* mbar;          // [4]: MMA done (buffer 0, 1), TMEM free (buffer 0, 1)
  uint32_t* tslot;
  __device__ __forceinline__ explicit SPtrs(unsigned char* sm) {
    uintptr_t o = ((uintptr_t)sm + 127) & ~(uintptr_t)127;
    unsigned char* ops = (unsigned char*)o;
    A0 = ops + C::o_A0;
    BKh = ops + C::o_B;
    BKl = BKh + C::bBK;
    BMh = BKh + 2 * C::bBK;
    BMl = BMh + C::bBM;
    float* f = (float*)(ops + C::ops_bytes);
    px = f;
    py = px + C::f_px;
    pz = py + C::f_py;
    T1 = pz + C::f_pz;
    // 16-byte alignment: the vector reads of stage 2 and the FP64 staging
    // that shares T1's space
    T1 = (float*)(((uintptr_t)T1 + 15) & ~(uintptr_t)15);
    rec = (double*)T1;
    kap = rec + 3 * C::REC;
    rho = kap + C::Q;
    jac = rho + C::Q;
    recf = (float*)(rec + C::d_geo);
    coef = T1 + C::f_T1g;
    stage0 = (float*)(((uintptr_t)(coef + C::f_coef) + 15) & ~(uintptr_t)15);
    stage1 = stage0 + C::f_stage;
    stage2 = stage1 + C::f_stage;
    stage3 = stage2 + C::f_stage;   // (NSTG = 4 only)
    uintptr_t mb = ((uintptr_t)(stage0 + C::NSTG * C::f_stage) + 15) & ~(uintptr_t)15;
    mbar = (uint64_t*)mb;
    tslot = (uint32_t*)(mbar + 4);
  }
  // staging buffer sb (a select, not an indexed array: an index into a
  // member array would put the pointer record in local memory)
  __device__ __forceinline__ float* stage(int sb) const {
    return sb == 0 ? stage0 : (sb == 1 ? stage1 : (sb == 2 || C::NSTG == 3 ? stage2 : stage3));
  }
  // operand arrays of the tile
  __device__ __forceinline__ unsigned char* AKh() const { return A0; }
  __device__ __forceinline__ unsigned char* AKl() const { return C::NAU == 2 ? A0 + C::tAK : nullptr; }
  __device__ __forceinline__ unsigned char* AMh() const { return A0 + C::NAU * C::tAK; }
  __device__ __forceinline__ unsigned char* AMl() const {
    return C::NAU == 2 ? A0 + C::NAU * C::tAK + C::tAM : nullptr;
  }
};

// Once per CTA: zero the operand buffers (their padding rows and K columns
// are never written by the element stages), allocate the TMEM columns of the
// two accumulator buffers (warp 0), initialise the two MMA-completion mbarriers.
template <class C>
__device__ __forceinline__ void st_cta_setup(unsigned char* sm) {
  SPtrs<C> S(sm);
  uint32_t* ops = (uint32_t*)S.A0;
  for (int i = threadIdx.x; i < (int)(C::ops_bytes / 4); i += C::NT) ops[i] = 0u;
  if (threadIdx.x < 32) {
    tmem_alloc(smem_u32(S.tslot), C::TCOLS);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(S.mbar), 1);          // MMA done: one tcgen05.commit
    mbar_init(smem_u32(S.mbar + 1), 1);
    mbar_init(smem_u32(S.mbar + 2), 128);    // TMEM free: the 128 consumer threads
    mbar_init(smem_u32(S.mbar + 3), 128);
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}

template <class C>
__device__ __forceinline__ void st_cta_teardown(unsigned char* sm) {
  SPtrs<C> S(sm);
  // the bulk copies of the last output blocks (issued by thread 0) complete
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (threadIdx.x < 32) tmem_dealloc(*S.tslot, C::TCOLS);
}

// The MMAs of one 128-row tile and one matrix (one thread): D = A B^T over the
// K steps of 32 bytes.
template <class C, int KD>
__device__ __forceinline__ void st_issue(uint32_t d, const unsigned char* Ah, const unsigned char* Al,
                                         const unsigned char* Bh, const unsigned char* Bl) {
  constexpr int EB = C::EB;
  constexpr uint32_t SBO = KD * EB * 8, LBO = 128;
  constexpr uint32_t IDESC = umma_idesc(EB == 2 ? 1u : 2u, 128, C::NU);
  constexpr int KS = KD * EB / 32;
  const uint32_t ah = smem_u32(Ah), bh = smem_u32(Bh), bl = smem_u32(Bl);
  const uint32_t al = Al ? smem_u32(Al) : 0u;
#pragma unroll
  for (int s = 0; s < KS; ++s) {
    const uint64_t dAh = umma_desc(ah + 256u * s, LBO, SBO);
    const uint64_t dBh = umma_desc(bh + 256u * s, LBO, SBO);
    const uint64_t dBl = umma_desc(bl + 256u * s, LBO, SBO);
    if (EB == 2) {
      umma_f16(d, dAh, dBh, IDESC, s > 0 ? 1u : 0u);
      umma_f16(d, dAh, dBl, IDESC, 1u);
    } else {
      const uint64_t dAl = umma_desc(al + 256u * s, LBO, SBO);
      umma_tf32(d, dAh, dBh, IDESC, s > 0 ? 1u : 0u);
      umma_tf32(d, dAh, dBl, IDESC, 1u);
      umma_tf32(d, dAl, dBh, IDESC, 1u);
    }
  }
}

// The L consecutive floats base[OFF .. OFF + L) into v (base 16-byte
// aligned; OFF and L fixed at compile time): 16-byte loads where the offset
// allows, then 8-byte, then single words.
template <int OFF, int L, int J = 0>
__device__ __forceinline__ void ld_run(const float* __restrict__ base, float* v) {
  if constexpr (J < L) {
    constexpr int c = OFF + J;
    if constexpr (c % 4 == 0 && J + 4 <= L) {
      const float4 w = *(const float4*)(base + c);
      v[J] = w.x; v[J + 1] = w.y; v[J + 2] = w.z; v[J + 3] = w.w;
      ld_run<OFF, L, J + 4>(base, v);
    } else if constexpr (c % 2 == 0 && J + 2 <= L) {
      const float2 w = *(const float2*)(base + c);
      v[J] = w.x; v[J + 1] = w.y;
      ld_run<OFF, L, J + 2>(base, v);
    } else {
      v[J] = base[c];
      ld_run<OFF, L, J + 1>(base, v);
    }
  }
}

// v[0 .. L) into the columns C0 .. C0 + L - 1 of one row of a K-major
// operand (rb = the row's byte offset, (r >> 3) KDIM EB 8 + (r & 7) 16; one
// 16-byte chunk per row and 16 / EB columns, the chunks 128 bytes apart), as
// uput does it value by value: FP32 hi = the value, lo = value - its TF32
// truncation; BF16 the rounded value (lo == nullptr: the A operand).  Runs
// within a chunk go out as one 16-, 8- or 4-byte store.
template <bool BF, int C0, int L, int J = 0>
__device__ __forceinline__ void uput_run(unsigned char* hi, unsigned char* lo, int rb, const float* v) {
  if constexpr (J < L) {
    constexpr int c = C0 + J;
    constexpr int EB = BF ? 2 : 4, PER = 16 / EB;
    constexpr int o = (c / PER) * 128 + (c % PER) * EB;
    if constexpr (!BF) {
      if constexpr (c % 4 == 0 && J + 4 <= L) {
        *(float4*)(hi + rb + o) = make_float4(v[J], v[J + 1], v[J + 2], v[J + 3]);
        *(float4*)(lo + rb + o) = make_float4(v[J] - tf32_trunc(v[J]), v[J + 1] - tf32_trunc(v[J + 1]),
                                              v[J + 2] - tf32_trunc(v[J + 2]), v[J + 3] - tf32_trunc(v[J + 3]));
        uput_run<BF, C0, L, J + 4>(hi, lo, rb, v);
      } else if constexpr (c % 2 == 0 && J + 2 <= L) {
        *(float2*)(hi + rb + o) = make_float2(v[J], v[J + 1]);
        *(float2*)(lo + rb + o) = make_float2(v[J] - tf32_trunc(v[J]), v[J + 1] - tf32_trunc(v[J + 1]));
        uput_run<BF, C0, L, J + 2>(hi, lo, rb, v);
      } else {
        *(float*)(hi + rb + o) = v[J];
        *(float*)(lo + rb + o) = v[J] - tf32_trunc(v[J]);
        uput_run<BF, C0, L, J + 1>(hi, lo, rb, v);
      }
    } else {
      if constexpr (c % 8 == 0 && J + 8 <= L) {
        *(uint4*)(hi + rb + o) = make_uint4(pack_bf16x2(v[J], v[J + 1]), pack_bf16x2(v[J + 2], v[J + 3]),
                                            pack_bf16x2(v[J + 4], v[J + 5]), pack_bf16x2(v[J + 6], v[J + 7]));
        uput_run<BF, C0, L, J + 8>(hi, lo, rb, v);
      } else if constexpr (c % 4 == 0 && J + 4 <= L) {
        *(uint2*)(hi + rb + o) = make_uint2(pack_bf16x2(v[J], v[J + 1]), pack_bf16x2(v[J + 2], v[J + 3]));
        uput_run<BF, C0, L, J + 4>(hi, lo, rb, v);
      } else if constexpr (c % 2 == 0 && J + 2 <= L) {
        *(uint32_t*)(hi + rb + o) = pack_bf16x2(v[J], v[J + 1]);
        uput_run<BF, C0, L, J + 2>(hi, lo, rb, v);
      } else {
        *(__nv_bfloat16*)(hi + rb + o) = __float2bfloat16_rn(v[J]);
        uput_run<BF, C0, L, J + 1>(hi, lo, rb, v);
      }
    }
  }
}

// f(ic<0>{}), ..., f(ic<N - 1>{}): a loop whose index is a compile-time
// constant in the body (the vector widths of ld_run depend on it).
template <int V>
struct ic {
  static constexpr int value = V;
};
template <int I, int N, class F>
__device__ __forceinline__ void unroll_ic(F&& f) {
  if constexpr (I < N) {
    f(ic<I>{});
    unroll_ic<I + 1, N>(f);
  }
}

// Stage 2 of tile t for the identity map: one thread per operand row and
// value group, all q values k1 at once (role 0, producer threads 0-127: C11
// and CM; role 1, threads 128-255: C00), so that each row receives whole
// vector stores and the stage-1 rows T_t[a3][b3][k1 + q k2] (16-byte aligned,
// TS a multiple of 4) are read as vectors.  Same sums, same order of the
// terms as st_stage2.
template <class C, bool BF>
__device__ __forceinline__ void st_stage2_rows(const SPtrs<C>& S, int t, int ptid) {
  constexpr int n = C::n, q = C::q, n2 = C::n2, RW = C::RW, TS = C::TS;
  constexpr int SZ = n2 * TS;
  static_assert(TS % 4 == 0 && RW % 4 == 0 && C::NP == 256 && C::RT <= 128, "row-vector stage 2");
  const int role = ptid >> 7, r = ptid & 127;
  if (r >= C::RT) return;
  const int ap = C::APT * t + r / n2, bp = r - (r / n2) * n2;
  if (ap >= n2) return;
  const int a2 = ap % n, a3 = ap / n, b2 = bp % n, b3 = bp / n;
  const float* y = S.py + (a2 * n + b2) * RW;   // 00, 11, 10, 01
  const float* T = S.T1 + (a3 * n + b3) * TS;
  float y00[q];
  ld_run<0, q>(y, y00);
  if (role == 0) {
    float c11[q], cm[q];
#pragma unroll
    for (int k1 = 0; k1 < q; ++k1) { c11[k1] = 0.f; cm[k1] = 0.f; }
    unroll_ic<0, q>([&](auto K2) {
      constexpr int k2 = decltype(K2)::value;
      float tv[q];
      if constexpr (C::DK) {
        ld_run<q * k2, q>(T + C::ts(0) * SZ, tv);
#pragma unroll
        for (int k1 = 0; k1 < q; ++k1) c11[k1] = fmaf(y00[k2], tv[k1], c11[k1]);
      }
      if constexpr (C::DM) {
        ld_run<q * k2, q>(T + C::ts(3) * SZ, tv);
#pragma unroll
        for (int k1 = 0; k1 < q; ++k1) cm[k1] = fmaf(y00[k2], tv[k1], cm[k1]);
      }
    });
    if constexpr (C::DK) uput_run<BF, 0, q>(S.AKh(), S.AKl(), (r >> 3) * (C::KA * C::EB * 8) + (r & 7) * 16, c11);
    if constexpr (C::DM) uput_run<BF, 0, q>(S.AMh(), S.AMl(), (r >> 3) * (C::KAM * C::EB * 8) + (r & 7) * 16, cm);
  } else if constexpr (C::DK) {
    float y11[q], c00[q];
    ld_run<q, q>(y, y11);
#pragma unroll
    for (int k1 = 0; k1 < q; ++k1) c00[k1] = 0.f;
    unroll_ic<0, q>([&](auto K2) {
      constexpr int k2 = decltype(K2)::value;
      float t0[q], t4[q];
      ld_run<q * k2, q>(T + C::ts(0) * SZ, t0);
      ld_run<q * k2, q>(T + C::ts(4) * SZ, t4);
#pragma unroll
      for (int k1 = 0; k1 < q; ++k1) c00[k1] = fmaf(y00[k2], t4[k1], fmaf(y11[k2], t0[k1], c00[k1]));
    });
    uput_run<BF, q, q>(S.AKh(), S.AKl(), (r >> 3) * (C::KA * C::EB * 8) + (r & 7) * 16, c00);
  }
}

// Stage 2 of tile t (the producer threads, ptid = 0..NP-1): the operand
// rows r < RT, (a', b') = (APT t + r / n^2, r mod n^2), a' = a2 + n a3,
// b' = b2 + n b3.  Columns
// of the stiffness operand X q + k1 in the x-pattern order 11, 00, 10, 01 of
// the B operand; the mass operand has the 00 pattern only.
//   C11 = sum_k2 Y00 T0;   C00 = sum_k2 Y11 T1' + Y00 T4 (+ Y10 T6(a3,b3) + Y01 T6(b3,a3));
//   C10 = sum_k2 Y01 T2 + Y00 T5(a3,b3);   C01 = sum_k2 Y10 T2 + Y00 T5(b3,a3);
//   CM  = sum_k2 Y00 T3,
// with T_t the stage-1 buffers of the terms (z00 D00, z00 D11, z00 D01, z00 DM,
// z11 D22, z01 D02, z01 D12; T1' = T0 for the identity map, whose D is kappa W I).
template <class C, bool GEN, bool BF>
__device__ __forceinline__ void st_stage2(const SPtrs<C>& S, int t, int ptid) {
  constexpr int n = C::n, q = C::q, n2 = C::n2, RW = C::RW, TS = C::TS;
  constexpr int SZ = n2 * TS;
  constexpr int T11 = GEN ? 1 : 0;
  for (int it = ptid; it < C::RT * q; it += C::NP) {
    const int r = it / q, k1 = it - r * q;
    const int ap = C::APT * t + r / n2, bp = r % n2;
    if (ap >= n2) continue;
    const int a2 = ap % n, a3 = ap / n, b2 = bp % n, b3 = bp / n;
    const float* y = S.py + (a2 * n + b2) * RW;   // 00, 11, 10, 01
    const int oab = (a3 * n + b3) * TS + k1, oba = (b3 * n + a3) * TS + k1;
    float c11 = 0.f, c00 = 0.f, cm = 0.f, c10 = 0.f, c01 = 0.f;
#pragma unroll
    for (int k2 = 0; k2 < q; ++k2) {
      const float y00 = y[k2], y11 = y[q + k2], y10 = y[2 * q + k2], y01 = y[3 * q + k2];
      const int o = oab + q * k2;
      if (C::DK) {
        c11 = fmaf(y00, S.T1[C::ts(0) * SZ + o], c11);
        c00 = fmaf(y11, S.T1[C::ts(T11) * SZ + o], c00);
        c00 = fmaf(y00, S.T1[C::ts(4) * SZ + o], c00);
        if (GEN) {
          const int ob = oba + q * k2;
          c00 = fmaf(y10, S.T1[C::ts(6) * SZ + o], c00);
          c00 = fmaf(y01, S.T1[C::ts(6) * SZ + ob], c00);
          const float t2 = S.T1[C::ts(2) * SZ + o];
          c10 = fmaf(y01, t2, c10);
          c10 = fmaf(y00, S.T1[C::ts(5) * SZ + o], c10);
          c01 = fmaf(y10, t2, c01);
          c01 = fmaf(y00, S.T1[C::ts(5) * SZ + ob], c01);
        }
      }
      if (C::DM) cm = fmaf(y00, S.T1[C::ts(3) * SZ + o], cm);
    }
    if (C::DK) {
      uput<BF, C::KA>(S.AKh(), S.AKl(), r, 0 * q + k1, c11);
      uput<BF, C::KA>(S.AKh(), S.AKl(), r, 1 * q + k1, c00);
      if (GEN) {
        uput<BF, C::KA>(S.AKh(), S.AKl(), r, 2 * q + k1, c10);
        uput<BF, C::KA>(S.AKh(), S.AKl(), r, 3 * q + k1, c01);
      }
    }
    if (C::DM) uput<BF, C::KAM>(S.AMh(), S.AMl(), r, k1, cm);
  }
}

// Named barrier of a warp group (id 1: the producers, 2: the consumers).
__device__ __forceinline__ void bar_group(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// The accumulators v of operand row (a', b') of a tile whose first a' is ap0:
// entries K[a1 + n a'][b1 + n b'] into the tile's staged output block stg
// (output rows n ap0 .., mirroring g's alignment).
template <class C>
__device__ __forceinline__ void st_stage_row(float* stg, const float* g, int ap, int ap0, int bp,
                                             const float* v) {
  constexpr int n = C::n, N = C::N;
  float* row = stg + (n * (ap - ap0)) * N + n * bp;
  if constexpr (n % 2 == 0) {
    // even n: every run of n entries starts on an 8-byte boundary when g is
    // 8-byte aligned
    if ((stage_offset(g) & 1) == 0) {
#pragma unroll
      for (int a1 = 0; a1 < n; ++a1)
#pragma unroll
        for (int b1 = 0; b1 < n; b1 += 2)
          *(float2*)(row + a1 * N + b1) = make_float2(v[a1 * n + b1], v[a1 * n + b1 + 1]);
      return;
    }
  }
#pragma unroll
  for (int a1 = 0; a1 < n; ++a1)
#pragma unroll
    for (int b1 = 0; b1 < n; ++b1) row[a1 * N + b1] = v[a1 * n + b1];
}

// A staged block of nn floats to g: the 16-byte-aligned middle by one bulk
// copy (consumer thread 0; one bulk group per block, committed even when
// empty, so that the group count per staging step is fixed), the scalar head
// and tail by the consumer threads.
__device__ __forceinline__ void st_copy_block(float* g, const float* stg, int nn, int ctid) {
  const int head = (int)((4 - (((uintptr_t)g >> 2) & 3)) & 3);
  const int h = head < nn ? head : nn;
  const int nv = (nn - h) / 4;
  for (int i = ctid; i < h; i += 128) g[i] = stg[i];
  for (int i = h + 4 * nv + ctid; i < nn; i += 128) g[i] = stg[i];
  if (ctid == 0) {
    if (nv > 0)
      asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n"
                   ::"l"(g + h), "r"(smem_u32(stg + h)), "r"(nv * 16) : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
  }
}

// Epilogue of tile t from TMEM buffer b (the 128 consumer threads, ctid =
// TMEM lane = operand row r; warp w reads lanes 32 w .. 32 w + 31): the
// accumulators of the row are read and the entries K[a1 + n a'][b1 + n b'] go
// into a staging buffer laid out as the output rows n APT t .. n APT (t + 1) - 1,
// which consumer thread 0 moves to HBM with one bulk asynchronous copy.  The
// NSTG buffers rotate (`sc` counts the staging steps); before one is refilled,
// the copy issued from it NSTG steps earlier must have read it.  Four buffers
// (both matrices): one step per matrix, both in one pair of group barriers,
// two copies of the previous tile in flight.  Three buffers (or one matrix):
// one step and one barrier pair per matrix, two copies in flight.  The TMEM
// buffer is released after its last read.
template <class C>
__device__ __forceinline__ void st_epilogue(const SPtrs<C>& S, uint32_t tmem, int t, int b,
                                            float* gK, float* gM, int ctid, uint32_t& sc) {
  constexpr int n = C::n, n2 = C::n2, N = C::N, NU = C::NU;
  const int warp = ctid >> 5;
  const int r = ctid;
  const int ap0 = C::APT * t;
  const int na = (n2 - ap0) < C::APT ? (n2 - ap0) : C::APT;   // a' values in this tile
  const int ap = ap0 + r / n2, bp = r % n2;
  const bool valid = r < C::RT && ap < n2;
  const uint32_t ta = tmem + (uint32_t)(b * C::CPB) + ((uint32_t)(32 * warp) << 16);
  const int nn = n * na * N;
  if constexpr (C::NSTG == 4 && C::DK && C::DM) {
    float* g0 = gK + (int64_t)(n * ap0) * N;
    float* g1 = gM + (int64_t)(n * ap0) * N;
    float* st0 = S.stage((int)(sc & 3u)) + stage_offset(g0);
    float* st1 = S.stage((int)((sc + 1u) & 3u)) + stage_offset(g1);
    sc += 2u;
    // the copies issued from these two buffers (the previous tile's but one)
    // have read them; the previous tile's two may still be in flight
    if (ctid == 0) asm volatile("cp.async.bulk.wait_group.read 2;\n" ::: "memory");
    bar_group(2, 128);
    float v[NU];
#pragma unroll
    for (int c = 0; c < NU; c += 16) tmem_ld16(ta + (uint32_t)c, v + c);
    if (valid) st_stage_row<C>(st0, g0, ap, ap0, bp, v);
#pragma unroll
    for (int c = 0; c < NU; c += 16) tmem_ld16(ta + (uint32_t)(NU + c), v + c);
    // the last read of this TMEM buffer: it may take the MMAs of tile t + 2
    fence_before_sync();
    mbar_arrive(smem_u32(S.mbar + 2 + b));
    if (valid) st_stage_row<C>(st1, g1, ap, ap0, bp, v);
    fence_proxy_async_smem();  // the staged blocks are read by the bulk copies
    bar_group(2, 128);
    st_copy_block(g0, st0, nn, ctid);
    st_copy_block(g1, st1, nn, ctid);
  } else {
#pragma unroll
    for (int mat = 0; mat < 2; ++mat) {
      if ((mat == 0 && !C::DK) || (mat == 1 && !C::DM)) continue;
      float v[NU];
      const uint32_t col = (mat == 1 && C::DK) ? (uint32_t)NU : 0u;
#pragma unroll
      for (int c = 0; c < NU; c += 16) tmem_ld16(ta + col + (uint32_t)c, v + c);
      if (mat == 1 || !C::DM) {
        fence_before_sync();
        mbar_arrive(smem_u32(S.mbar + 2 + b));
      }
      float* g = (mat == 0 ? gK : gM) + (int64_t)(n * ap0) * N;
      float* stg = S.stage((int)(sc % (uint32_t)C::NSTG)) + stage_offset(g);
      ++sc;
      // the copy issued from this buffer NSTG steps ago has read it (the
      // NSTG - 1 later ones may still be in flight)
      if (ctid == 0) {
        if constexpr (C::NSTG == 4) asm volatile("cp.async.bulk.wait_group.read 3;\n" ::: "memory");
        else asm volatile("cp.async.bulk.wait_group.read 2;\n" ::: "memory");
      }
      bar_group(2, 128);
      if (valid) st_stage_row<C>(stg, g, ap, ap0, bp, v);
      fence_proxy_async_smem();  // the staged block is read by the bulk copy
      bar_group(2, 128);
      st_copy_block(g, stg, nn, ctid);
    }
  }
}

// One element, all stages.  Returns false only if a bounded wait expired
// (IGA_ERR_TIMEOUT recorded; the caller stops).  `tc` counts the tiles this
// CTA has processed (it fixes the buffers and mbarrier parities), `sc` the
// staging steps of its consumer threads.
template <int P, int QG, bool GEN, int MODE, bool BF>
__device__ __forceinline__ bool st_element(const ElemArgs& A, int64_t e, unsigned char* sm,
                                           uint32_t& tc, uint32_t& sc) {
  using C = ST<P, QG, GEN, MODE, BF>;
  constexpr int n = C::n, q = C::q, Q = C::Q, n2 = C::n2, N = C::N, NT = C::NT, REC = C::REC,
                RW = C::RW, TS = C::TS;
  const SPtrs<C> S(sm);
  const int tid = threadIdx.x;
  __syncthreads();  // the previous element's shared memory is no longer read

  // inputs (cp.async), FP32 records, coefficients and 1D factor patterns
  sf3_f32_stage_inputs<C, GEN>(A, e, S.rec, S.kap, S.rho, S.jac);
  cp_async_wait_all();
  for (int i = tid; i < 3 * REC; i += NT) S.recf[i] = (float)S.rec[i];
  __syncthreads();
  for (int k = NT - 1 - tid; k < Q; k += NT) sf3_f32_coef<C, GEN>(k, S.recf, S.kap, S.rho, S.jac, S.coef);
  for (int it = tid; it < 3 * n2 * q; it += NT) {
    const int d = it / (n2 * q), i = it % (n2 * q);
    const int a = i / (n * q), b = (i / q) % n, k = i % q;
    const float* v = S.recf + d * REC;
    const float* dv = v + q * n;
    const float va = v[k * n + a], vb = v[k * n + b], da = dv[k * n + a], db = dv[k * n + b];
    if (d == 0) {          // x: 11, 00, 10, 01 (the order of the GEMM's K columns)
      float* r = S.px + (a * n + b) * RW;
      r[k] = da * db; r[q + k] = va * vb; r[2 * q + k] = da * vb; r[3 * q + k] = va * db;
    } else if (d == 1) {   // y: 00, 11, 10, 01
      float* r = S.py + (a * n + b) * RW;
      r[k] = va * vb; r[q + k] = da * db; r[2 * q + k] = da * vb; r[3 * q + k] = va * db;
    } else {               // z: 00, 11, 01
      float* r = S.pz + (a * n + b) * C::RZ;
      r[k] = va * vb; r[q + k] = da * db; r[2 * q + k] = va * db;
    }
  }
  __syncthreads();

  // B operands (x patterns, hi + lo) and stage 1 (z):
  //   T_t[a3][b3][k1 + q k2] = sum_k3 Z_t[a3][b3][k3] D_t[k1, k2, k3]
  if (C::DK) {
    for (int i = tid; i < C::NU * C::KA; i += NT) {
      const int nn = i / C::KA, k = i % C::KA;
      const float v = (nn < n2 && k < C::NXK * q) ? S.px[nn * RW + k] : 0.f;
      uput<BF, C::KA>(S.BKh, S.BKl, nn, k, v);
    }
  }
  if (C::DM) {
    for (int i = tid; i < C::NU * C::KAM; i += NT) {
      const int nn = i / C::KAM, k = i % C::KAM;
      const float v = (nn < n2 && k < q) ? S.px[nn * RW + q + k] : 0.f;
      uput<BF, C::KAM>(S.BMh, S.BMl, nn, k, v);
    }
  }
  {
    constexpr int SZ = n2 * TS;
    for (int it = tid; it < q * q * n; it += NT) {
      // consecutive threads take consecutive kk = k1 + q k2 (their T writes
      // fall on consecutive words, their z reads are shared)
      const int kk = it % (q * q), a3 = it / (q * q);
      float d0[q], d1[q], d2[q], d3[q], d4[q], d5[q], d6[q];
#pragma unroll
      for (int k3 = 0; k3 < q; ++k3) {
        const int o = kk + q * q * k3;
        d0[k3] = S.coef[C::cs(0) * Q + o];
        d3[k3] = S.coef[C::cs(3) * Q + o];
        if (GEN) {
          d1[k3] = S.coef[C::cs(1) * Q + o]; d2[k3] = S.coef[C::cs(2) * Q + o];
          d4[k3] = S.coef[C::cs(4) * Q + o]; d5[k3] = S.coef[C::cs(5) * Q + o];
          d6[k3] = S.coef[C::cs(6) * Q + o];
        }
      }
#pragma unroll 1
      for (int b3 = 0; b3 < n; ++b3) {
        const float* z = S.pz + (a3 * n + b3) * C::RZ;
        float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f, t4 = 0.f, t5 = 0.f, t6 = 0.f;
#pragma unroll
        for (int k3 = 0; k3 < q; ++k3) {
          const float z00 = z[k3], z11 = z[q + k3], z01 = z[2 * q + k3];
          if (C::DK) {
            t0 = fmaf(z00, d0[k3], t0);
            t4 = fmaf(z11, GEN ? d4[k3] : d0[k3], t4);
            if (GEN) {
              t1 = fmaf(z00, d1[k3], t1);
              t2 = fmaf(z00, d2[k3], t2);
              t5 = fmaf(z01, d5[k3], t5);
              t6 = fmaf(z01, d6[k3], t6);
            }
          }
          if (C::DM) t3 = fmaf(z00, d3[k3], t3);
        }
        const int o = (a3 * n + b3) * TS + kk;
        if (C::DK) {
          S.T1[C::ts(0) * SZ + o] = t0;
          S.T1[C::ts(4) * SZ + o] = t4;
          if (GEN) {
            S.T1[C::ts(1) * SZ + o] = t1; S.T1[C::ts(2) * SZ + o] = t2;
            S.T1[C::ts(5) * SZ + o] = t5; S.T1[C::ts(6) * SZ + o] = t6;
          }
        }
        if (C::DM) S.T1[C::ts(3) * SZ + o] = t3;
      }
    }
  }
  fence_proxy_async_smem();  // every thread's B-operand writes are read by the tensor core
  __syncthreads();

  // stages 2 and 3, tile by tile, producers and consumers in parallel.  The
  // global tile number g = tc + t picks the TMEM buffer b = g mod 2; use
  // u = g / 2 of buffer b's mbarriers completes with parity u mod 2.
  const uint32_t tmem = *S.tslot;
  float* gK = C::DK ? (float*)A.K_out + e * (int64_t)N * N : nullptr;
  float* gM = C::DM ? (float*)A.M_out + e * (int64_t)N * N : nullptr;
  constexpr unsigned long long kWait = 1000000000ull;   // 1 s of global time
  bool ok = true;
  const int warp = tid >> 5;
  if (warp >= 4) {
    const int ptid = tid - 128;
#pragma unroll 1
    for (int t = 0; t < C::MT; ++t) {
      const uint32_t g = tc + (uint32_t)t, b = g & 1u;
      // the operand tile is free once the MMAs of the previous tile have read it
      if (g >= 1) ok &= mbar_wait_bounded(smem_u32(S.mbar + ((g - 1) & 1u)), ((g - 1) >> 1) & 1u, kWait);
      if constexpr (GEN) st_stage2<C, GEN, BF>(S, t, ptid);
      else st_stage2_rows<C, BF>(S, t, ptid);
      fence_proxy_async_smem();  // the operand rows are read by the tensor core
      bar_group(1, C::NP);
      if (ptid == 0) {
        // TMEM buffer b is free once the consumers have read tile g - 2
        if (g >= 2) ok &= mbar_wait_bounded(smem_u32(S.mbar + 2 + b), ((g - 2) >> 1) & 1u, kWait);
        fence_after_sync();
        const uint32_t d = tmem + b * (uint32_t)C::CPB;
        if (ok) {
          if (C::DK) st_issue<C, C::KA>(d, S.AKh(), S.AKl(), S.BKh, S.BKl);
          if (C::DM) st_issue<C, C::KAM>(d + (C::DK ? C::NU : 0), S.AMh(), S.AMl(), S.BMh, S.BMl);
          umma_commit(smem_u32(S.mbar + b));
        }
      }
    }
    // the last tile's MMAs have read the operand before the next element
    // rewrites it (and the B operands)
    const uint32_t gl = tc + (uint32_t)(C::MT - 1);
    ok &= mbar_wait_bounded(smem_u32(S.mbar + (gl & 1u)), (gl >> 1) & 1u, kWait);
  } else {
#pragma unroll 1
    for (int t = 0; t < C::MT; ++t) {
      const uint32_t g = tc + (uint32_t)t, b = g & 1u;
      ok &= mbar_wait_bounded(smem_u32(S.mbar + b), (g >> 1) & 1u, kWait);
      fence_after_sync();
      st_epilogue<C>(S, tmem, t, (int)b, gK, gM, tid, sc);
    }
  }
  tc += (uint32_t)C::MT;
  fence_before_sync();
  if (!__syncthreads_and(ok)) {
    if (tid == 0) atomicCAS(A.err, 0, (int)IGA_ERR_TIMEOUT);
    return false;
  }
  fence_after_sync();
  return true;
}

template <int P, int QG, bool GEN, int MODE, bool BF>
__global__ void __launch_bounds__(384, GEN ? 1 : 2) k_sf3_stream(const ElemArgs A) {
  extern __shared__ __align__(16) unsigned char sms[];
  using C = ST<P, QG, GEN, MODE, BF>;
  st_cta_setup<C>(sms);
  uint32_t tc = 0, sc = 0;
  for (int64_t e = blockIdx.x; e < A.n_elem; e += gridDim.x)
    if (!st_element<P, QG, GEN, MODE, BF>(A, e, sms, tc, sc)) break;
  st_cta_teardown<C>(sms);
}

// Persistent form: CTAs pop work items (patch, first element, count) from the
// class's device queue; checks and time budget as in k_sumfact32.cuh.
template <int P, int QG, bool GEN, int MODE, bool BF>
__global__ void __launch_bounds__(384, GEN ? 1 : 2) k_sf3_stream_queue(const QueueArgs B) {
  extern __shared__ __align__(16) unsigned char sms[];
  using C = ST<P, QG, GEN, MODE, BF>;
  __shared__ int s_item;
  const unsigned long long t0 = global_timer_ns();
  st_cta_setup<C>(sms);
  uint32_t tc = 0, sc = 0;
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
    if (w.e0 < 0 || w.count <= 0 || w.e0 + w.count > E || pd.p != P || pd.q != QG || !pd.iso) {
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
    for (int64_t e = w.e0; e < w.e0 + w.count && ok; ++e) ok = st_element<P, QG, GEN, MODE, BF>(A, e, sms, tc, sc);
    if (!ok) break;
  }
  st_cta_teardown<C>(sms);
}

template <class C, class K>
cudaError_t st_prepare(K k, int* per_sm_out) {
  static_assert(C::smem <= 227 * 1024, "shared memory");
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  int dev = 0, sms = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = resident_ctas_tmem((const void*)k, C::NT, C::smem, C::TCOLS, &per_sm);
  if (e != cudaSuccess) return e;
  *per_sm_out = sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

template <int P, int QG, bool GEN, int MODE, bool BF>
cudaError_t st_run(const ElemArgs& a, cudaStream_t st) {
  using C = ST<P, QG, GEN, MODE, BF>;
  if constexpr (MODE == 0 && C::smem > 227 * 1024) {
    // both matrices do not fit one CTA: stiffness and mass in two launches
    ElemArgs ak = a, am = a;
    ak.M_out = nullptr;
    am.K_out = nullptr;
    cudaError_t e = st_run<P, QG, GEN, 1, BF>(ak, st);
    if (e != cudaSuccess) return e;
    return st_run<P, QG, GEN, 2, BF>(am, st);
  } else {
    auto k = k_sf3_stream<P, QG, GEN, MODE, BF>;
    static int capacity = 0;   // resident CTAs on this GPU, looked up once
    if (capacity == 0) {
      cudaError_t e = st_prepare<C>(k, &capacity);
      if (e != cudaSuccess) return e;
    }
    const int64_t grid = a.n_elem < capacity ? a.n_elem : capacity;
    k<<<(unsigned)grid, C::NT, C::smem, st>>>(a);
    return cudaGetLastError();
  }
}

template <int P, int QG, bool GEN, int MODE, bool BF>
cudaError_t st_run_queue(const QueueArgs& b, int grid, cudaStream_t st, int* max_grid) {
  using C = ST<P, QG, GEN, MODE, BF>;
  if constexpr (C::smem > 227 * 1024) {
    return cudaErrorNotSupported;   // the planner splits such classes by matrix
  } else {
    auto k = k_sf3_stream_queue<P, QG, GEN, MODE, BF>;
    int cap = 0;
    cudaError_t e = st_prepare<C>(k, &cap);
    if (e != cudaSuccess) return e;
    if (max_grid) {
      *max_grid = cap;
      return cudaSuccess;
    }
    k<<<(unsigned)grid, C::NT, C::smem, st>>>(b);
    return cudaGetLastError();
  }
}

template <int P, int QG, bool BF>
cudaError_t st_runm(const ElemArgs& a, cudaStream_t st) {
  const int mode = (a.K_out && a.M_out) ? 0 : (a.K_out ? 1 : 2);
  if (a.jac) {
    if (mode == 0) return st_run<P, QG, true, 0, BF>(a, st);
    if (mode == 1) return st_run<P, QG, true, 1, BF>(a, st);
    return st_run<P, QG, true, 2, BF>(a, st);
  }
  if (mode == 0) return st_run<P, QG, false, 0, BF>(a, st);
  if (mode == 1) return st_run<P, QG, false, 1, BF>(a, st);
  return st_run<P, QG, false, 2, BF>(a, st);
}

template <int P, int QG, bool BF>
cudaError_t st_runq(const QueueArgs& b, int mode, int grid, cudaStream_t st, int* max_grid) {
  if (b.jac) {
    if (mode == 0) return st_run_queue<P, QG, true, 0, BF>(b, grid, st, max_grid);
    if (mode == 1) return st_run_queue<P, QG, true, 1, BF>(b, grid, st, max_grid);
    return st_run_queue<P, QG, true, 2, BF>(b, grid, st, max_grid);
  }
  if (mode == 0) return st_run_queue<P, QG, false, 0, BF>(b, grid, st, max_grid);
  if (mode == 1) return st_run_queue<P, QG, false, 1, BF>(b, grid, st, max_grid);
  return st_run_queue<P, QG, false, 2, BF>(b, grid, st, max_grid);
}

}  // namespace

bool stream_form_supported(int p, int q) { return (p == 4 && (q == 5 || q == 6)) || (p == 5 && q == 6); }

bool stream_both_fit(int p, int q, bool bf16) {
#define F(PP, QQ)                                                                        \
  if (p == PP && q == QQ)                                                                \
    return bf16 ? (ST<PP, QQ, true, 0, true>::smem <= 227 * 1024 &&                     \
                   ST<PP, QQ, false, 0, true>::smem <= 227 * 1024)                       \
                : (ST<PP, QQ, true, 0, false>::smem <= 227 * 1024 &&                     \
                   ST<PP, QQ, false, 0, false>::smem <= 227 * 1024);
  F(4, 5) F(4, 6) F(5, 6)
#undef F
  return false;
}

cudaError_t launch_sumfact_f32_stream(const ElemArgs& a, int p, int q, bool bf16, cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  if (p == 4 && q == 5) return bf16 ? st_runm<4, 5, true>(a, st) : st_runm<4, 5, false>(a, st);
  if (p == 4 && q == 6) return bf16 ? st_runm<4, 6, true>(a, st) : st_runm<4, 6, false>(a, st);
  if (p == 5 && q == 6) return bf16 ? st_runm<5, 6, true>(a, st) : st_runm<5, 6, false>(a, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_sumfact_f32_stream_queue(const QueueArgs& b, int p, int q, bool bf16, int mode,
                                            int grid, cudaStream_t st, int* max_grid) {
  if (p == 4 && q == 5) return bf16 ? st_runq<4, 5, true>(b, mode, grid, st, max_grid)
                                    : st_runq<4, 5, false>(b, mode, grid, st, max_grid);
  if (p == 4 && q == 6) return bf16 ? st_runq<4, 6, true>(b, mode, grid, st, max_grid)
                                    : st_runq<4, 6, false>(b, mode, grid, st, max_grid);
  if (p == 5 && q == 6) return bf16 ? st_runq<5, 6, true>(b, mode, grid, st, max_grid)
                                    : st_runq<5, 6, false>(b, mode, grid, st, max_grid);
  return cudaErrorInvalidValue;
}

}  // namespace iga
