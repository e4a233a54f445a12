// k_grad.cu -- backward of the element matrices with respect to the
// coefficients (3D; not in the paper: the element integrals are linear in
// kappa and rho, eq. 10 and the stiffness of Sec. 2.2; 3D below, 2D in
// k_grad2).  Given upstream
// gradients GK = dL/dK_e and GM = dL/dM_e:
//   dL/dkappa_q = w_q |det G_q| sum_ij (G^{-1} G^{-T})_ij H_ij(q),
//   H_ij(q)     = sum_ab GK_ab d_i phi_a(q) d_j phi_b(q)   (reference derivatives)
//   dL/drho_q   = w_q |det G_q| sum_ab GM_ab phi_a(q) phi_b(q).
// The metric G^{-1} G^{-T} and phi_a phi_b are symmetric, so only the
// symmetric parts of GK and GM matter; with a symmetric upstream matrix H is
// symmetric too (6 distinct terms i <= j instead of 9, 3 for the identity
// map) and every diagonal stage below is a symmetric matrix, formed on its
// upper triangle and mirrored.
//
// H is formed by sum factorization run backwards (the transpose of Algorithm
// 2's stage order).  One CTA per element and one pass per upstream matrix:
// the element's block is read once from HBM into shared memory (padded rows,
// cp.async; the mass block streams in during the stiffness pass where both
// fit), and S = G + G^T is formed; then for each Gauss point q1 of x,
//   x: UX_st[a2 a3][b2 b3] = sum_{a1 b1} f^s_x(q1)[a1] S[a][b] f^t_x(q1)[b1], S = G + G^T,
//      for the factor pairs (s, t) the terms need (in FP64 on the upper
//      triangle of (a2 a3, b2 b3), the pair (derivative, value) giving both
//      halves);
//   y: UY_ij[a3][b3][q2] = sum_{a2 b2} f_y(q2)[a2] f_y(q2)[b2] UX[a2 a3][b2 b3];
//   z: H_ij[q2][q3]      = sum_{a3 b3} f_z(q3)[a3] f_z(q3)[b3] UY_ij[a3][b3][q2];
// then the geometry at the q^2 points of the slice.  T = double (FP64) or
// float (FP32 with FP64 cofactors and determinant).
#include "ff.cuh"
#include "iga_internal.h"

namespace iga {
namespace {

// stiffness terms (i, j), i <= j: the diagonal first
__host__ __device__ constexpr int term_i(int t) { return t < 3 ? t : (t == 5 ? 1 : 0); }
__host__ __device__ constexpr int term_j(int t) { return t < 3 ? t : (t == 3 ? 1 : 2); }

template <typename T, int P, int QG, bool GEN>
struct GRD {
  static constexpr int n = P + 1, q = QG, n2 = n * n, n4 = n2 * n2, N = n2 * n, Q = q * q * q;
  static constexpr int GS = N + 1;               // padded row stride of the staged block
  static constexpr size_t dyn_bytes = sizeof(store_t<T>) * (size_t)N * GS;   // one block
  // room for both upstream blocks (the mass block loads during the stiffness pass)
  // (FP32 only: the FP64 kernel is bound by its pipe and wants more CTAs per SM)
  static constexpr bool TWO = sizeof(T) == 4 && 2 * dyn_bytes <= 80 * 1024;
  // one CTA per SM when the block is large: give it 8 warps
  static constexpr int NT = dyn_bytes > 48 * 1024 ? 256 : 128;
  static constexpr int REC = 2 * q * n + q;
  static constexpr int T3 = n * (n + 1) / 2;      // upper triangle of (a3, b3)
  // x items: the upper triangle of (a2 a3, b2 b3) in FP64 (bound by the FP64
  // pipe: fewer operations); every pair in FP32 (balanced over the threads)
  static constexpr bool TRI = sizeof(T) == 8;
  static constexpr int TX = TRI ? n2 * (n2 + 1) / 2 : n4;
  static constexpr int ITX = (TX + NT - 1) / NT;  // x items per thread
  static constexpr int NPX = GEN ? 3 : 2;         // x pairs: (d, d), (v, v), (d, v)
  static constexpr int NTY = GEN ? 6 : 3;         // stiffness terms
  // the x blocks of a thread's items stay in registers across q1 when small
  static constexpr bool HOLD = n2 * ITX * (int)sizeof(T) <= 256;
};

__device__ __forceinline__ void tri_decode(int t, int m, int& a, int& b) {
  a = 0;
  while (t >= m - a) {
    t -= m - a;
    ++a;
  }
  b = a + t;
}

// [N][N] block from HBM into rows of stride GS = N + 1 (the transposed
// accesses of the symmetrization then hit distinct banks) by cp.async of one
// value per thread and step: coalesced, any alignment, the whole block in
// flight at once without passing through registers.
template <typename T, int N, int GS, int NT>
__device__ __forceinline__ void issue_block(const T* __restrict__ src, T* G) {
  for (int i = threadIdx.x; i < N * N; i += NT) {
    const int r = i / N;
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(G + r * GS + i - r * N));
    if (sizeof(T) == 8)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src + i) : "memory");
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src + i) : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int PENDING>
__device__ __forceinline__ void wait_blocks() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
  __syncthreads();
}

// One upstream matrix: MASS = GM -> grad_rho, else GK -> grad_kappa.
template <typename T, int P, int QG, bool GEN, bool MASS>
__device__ __forceinline__ void grad_pass(const GradArgs& A, int64_t e, store_t<T>* __restrict__ out,
                                          store_t<T>* G, const T (*f)[2][QG * (P + 1)],
                                          const double* rec, const T* wts, const unsigned char* tri3,
                                          T* UX, T* UY, T* HZ) {
  using C = GRD<T, P, QG, GEN>;
  constexpr int n = C::n, q = C::q, n2 = C::n2, n4 = C::n4, N = C::N, Q = C::Q, NT = C::NT,
                REC = C::REC, T3 = C::T3, TX = C::TX, ITX = C::ITX, GS = C::GS;
  constexpr bool TRI = C::TRI;
  constexpr int ND = MASS ? 1 : 3;                  // diagonal terms
  constexpr int NO = MASS ? 0 : C::NTY - 3;         // off-diagonal terms
  constexpr bool HOLD = C::HOLD;
  const int tid = threadIdx.x;
  // The caller has waited for this pass's block and synchronized.  S = G + G^T
  // (twice the symmetric part; the 1/2 goes into the weights): formed while
  // loading the register blocks, else in place.
  if constexpr (!HOLD) {
    for (int idx = tid; idx < N * N; idx += NT) {
      const int a = idx / N, b = idx - a * N;
      if (a <= b) {
        const store_t<T> s = G[a * GS + b] + G[b * GS + a];
        G[a * GS + b] = s;
        G[b * GS + a] = s;
      }
    }
    __syncthreads();
  }
  int ia[ITX], ib[ITX];
  T Gr[HOLD ? ITX : 1][HOLD ? n2 : 1];
#pragma unroll
  for (int k = 0; k < ITX; ++k) {
    const int t = tid + k * NT;
    ia[k] = ib[k] = -1;
    if (t < TX) {
      if (TRI) {
        tri_decode(t, n2, ia[k], ib[k]);
      } else {
        ia[k] = t / n2;
        ib[k] = t - ia[k] * n2;
      }
    }
    if (HOLD && t < TX) {
#pragma unroll
      for (int a1 = 0; a1 < n; ++a1)
#pragma unroll
        for (int b1 = 0; b1 < n; ++b1)
          Gr[HOLD ? k : 0][HOLD ? a1 * n + b1 : 0] =
              to_compute<T>(G[(a1 + n * ia[k]) * GS + n * ib[k] + b1]) +
              to_compute<T>(G[(b1 + n * ib[k]) * GS + n * ia[k] + a1]);
    }
  }
#pragma unroll 1
  for (int q1 = 0; q1 < q; ++q1) {
    const T* fx0 = &f[0][0][q1 * n];
    const T* fx1 = &f[0][1][q1 * n];
    // x
#pragma unroll
    for (int k = 0; k < ITX; ++k) {
      if (ia[k] < 0) continue;
      const int a23 = ia[k], b23 = ib[k];
      T v0[n], v1[n];
#pragma unroll
      for (int a1 = 0; a1 < n; ++a1) {
        T s0 = 0, s1 = 0;
#pragma unroll
        for (int b1 = 0; b1 < n; ++b1) {
          T g;
          if constexpr (HOLD) g = Gr[k][a1 * n + b1];
          else g = to_compute<T>(G[(a1 + n * a23) * GS + n * b23 + b1]);
          mac(s0, g, fx0[b1]);
          if (!MASS) mac(s1, g, fx1[b1]);
        }
        v0[a1] = fin(s0);
        v1[a1] = fin(s1);
      }
      T p00 = 0, p11 = 0, p10 = 0, p01 = 0;
#pragma unroll
      for (int a1 = 0; a1 < n; ++a1) {
        mac(p00, fx0[a1], v0[a1]);
        if (!MASS) {
          mac(p11, fx1[a1], v1[a1]);
          if (GEN) {
            mac(p10, fx1[a1], v0[a1]);
            if (TRI) mac(p01, fx0[a1], v1[a1]);
          }
        }
      }
      p00 = fin(p00);
      p11 = fin(p11);
      p10 = fin(p10);
      p01 = fin(p01);
      const int u = a23 * n2 + b23, l = b23 * n2 + a23;
      if (MASS) {
        UX[u] = p00;
        if (TRI) UX[l] = p00;
      } else {
        UX[u] = p11;
        UX[n4 + u] = p00;
        if (GEN) UX[2 * n4 + u] = p10;
        if (TRI) {
          UX[l] = p11;
          UX[n4 + l] = p00;
          if (GEN) UX[2 * n4 + l] = p01;
        }
      }
    }
    __syncthreads();
    // y: diagonal terms on the (a3 <= b3) triangle, then the off-diagonal ones
    for (int it = tid; it < (ND * T3 + NO * n2) * q; it += NT) {
      int term, a3, b3, q2;
      bool mirror;
      if (it < ND * T3 * q) {
        term = it / (T3 * q);
        const int r = it - term * (T3 * q);
        q2 = r % q;
        const int ab = tri3[r / q];
        a3 = ab >> 4;
        b3 = ab & 15;
        mirror = true;
      } else {
        const int r0 = it - ND * T3 * q;
        term = ND + r0 / (n2 * q);
        const int r = r0 % (n2 * q);
        q2 = r % q;
        a3 = (r / q) / n;
        b3 = (r / q) % n;
        mirror = false;
      }
      int px, sy, ty;
      if (MASS) {
        px = 0;
        sy = ty = 0;
      } else {
        const int i = term_i(term), j = term_j(term);
        px = (i == 0 && j == 0) ? 0 : (i == 0 ? 2 : 1);
        sy = i == 1;
        ty = j == 1;
      }
      const T* U = UX + px * n4;
      const T* fa = &f[1][sy][q2 * n];
      const T* fb = &f[1][ty][q2 * n];
      T acc = 0;
#pragma unroll
      for (int a2 = 0; a2 < n; ++a2) {
        T s0 = 0;
#pragma unroll
        for (int b2 = 0; b2 < n; ++b2) mac(s0, fb[b2], U[(a2 + n * a3) * n2 + b2 + n * b3]);
        mac(acc, fa[a2], fin(s0));
      }
      acc = fin(acc);
      UY[(term * n2 + a3 * n + b3) * q + q2] = acc;
      if (mirror) UY[(term * n2 + b3 * n + a3) * q + q2] = acc;
    }
    __syncthreads();
    // z: every (term, q2, q3)
    for (int it = tid; it < (ND + NO) * q * q; it += NT) {
      const int term = it / (q * q), r = it - term * (q * q), q2 = r % q, q3 = r / q;
      int sz = 0, tz = 0;
      if (!MASS) {
        sz = term_i(term) == 2;
        tz = term_j(term) == 2;
      }
      const T* fa = &f[2][sz][q3 * n];
      const T* fb = &f[2][tz][q3 * n];
      const T* U = UY + term * n2 * q + q2;
      T acc = 0;
#pragma unroll
      for (int a3 = 0; a3 < n; ++a3) {
        T s0 = 0;
#pragma unroll
        for (int b3 = 0; b3 < n; ++b3) mac(s0, fb[b3], U[(a3 * n + b3) * q]);
        mac(acc, fa[a3], fin(s0));
      }
      HZ[term * q * q + r] = fin(acc);
    }
    __syncthreads();
    // geometry at the q^2 points of this slice
    for (int it = tid; it < q * q; it += NT) {
      const int q2 = it % q, q3 = it / q;
      const int k = q1 + q * (q2 + q * q3);
      T g;
      if (GEN) {
        const double W =
            0.5 * rec[2 * q * n + q1] * rec[REC + 2 * q * n + q2] * rec[2 * REC + 2 * q * n + q3];
        const double* Gq = A.jac + (e * Q + k) * 9;
        const double g00 = Gq[0], g01 = Gq[1], g02 = Gq[2], g10 = Gq[3], g11 = Gq[4], g12 = Gq[5],
                     g20 = Gq[6], g21 = Gq[7], g22 = Gq[8];
        const double c[3][3] = {{g11 * g22 - g12 * g21, g12 * g20 - g10 * g22, g10 * g21 - g11 * g20},
                                {g02 * g21 - g01 * g22, g00 * g22 - g02 * g20, g01 * g20 - g00 * g21},
                                {g01 * g12 - g02 * g11, g02 * g10 - g00 * g12, g00 * g11 - g01 * g10}};
        const double adet = fabs(g00 * c[0][0] + g01 * c[0][1] + g02 * c[0][2]);
        if (MASS) {
          g = (T)(W * adet) * HZ[it];
        } else {
          // w |det| (G^{-1} G^{-T})_ij = (w / |det|) sum_m c_mi c_mj; off-diagonal terms twice
          const double wk = W / adet;
          g = 0;
#pragma unroll
          for (int term = 0; term < C::NTY; ++term) {
            const int i = term_i(term), j = term_j(term);
            const double d = (term < 3 ? wk : 2.0 * wk) *
                             (c[0][i] * c[0][j] + c[1][i] * c[1][j] + c[2][i] * c[2][j]);
            mac(g, (T)d, HZ[term * q * q + it]);
          }
          g = fin(g);
        }
      } else {
        // identity map: the weight in the kernel's precision
        const T Wt = (T)0.5 * wts[q1] * wts[q + q2] * wts[2 * q + q3];
        g = MASS ? Wt * HZ[it] : Wt * (HZ[it] + HZ[q * q + it] + HZ[2 * q * q + it]);
      }
      out[e * Q + k] = to_store<T>(g);
    }
  }
}

template <typename T, int P, int QG, bool GEN>
__global__ void __launch_bounds__(GRD<T, P, QG, GEN>::NT) k_grad3(const GradArgs A) {
  using C = GRD<T, P, QG, GEN>;
  constexpr int n = C::n, q = C::q, n2 = C::n2, n4 = C::n4, NT = C::NT, REC = C::REC;
  extern __shared__ __align__(16) unsigned char grad_dyn[];
  __shared__ double rec[3 * REC];
  __shared__ T f[3][2][q * n];            // [direction][value, derivative][q][n]
  __shared__ T UX[C::NPX * n4];
  __shared__ T UY[C::NTY * n2 * q];
  __shared__ T HZ[C::NTY * q * q];
  __shared__ unsigned char tri3[C::T3];   // (a3 << 4 | b3) of the (a3 <= b3) triangle
  __shared__ T wts[3 * q];                // Gauss weights per direction
  using S = store_t<T>;
  S* G = reinterpret_cast<S*>(grad_dyn);
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
  __syncthreads();
  for (int i = tid; i < 3 * 2 * q * n; i += NT) {
    const int d = i / (2 * q * n), j = i % (2 * q * n);
    (&f[0][0][0])[i] = from_double<T>(rec[d * REC + j]);
  }
  if (tid < 3 * q) wts[tid] = from_double<T>(rec[(tid / q) * REC + 2 * q * n + tid % q]);
  if (tid < C::T3) {
    int a3, b3;
    tri_decode(tid, n, a3, b3);
    tri3[tid] = (unsigned char)(a3 << 4 | b3);
  }
  // both blocks in flight at once when the launch gave two buffers
  constexpr int64_t NN = (int64_t)C::N * C::N;
  const bool two = A.GK && A.GM && A.two_buffers;
  S* G1 = two ? G + C::N * C::GS : G;
  if (A.GK) issue_block<S, C::N, C::GS, NT>((const S*)A.GK + e * NN, G);
  if (A.GM && (two || !A.GK)) issue_block<S, C::N, C::GS, NT>((const S*)A.GM + e * NN, G1);
  if (A.GK) {
    if (two) wait_blocks<1>();
    else wait_blocks<0>();
    grad_pass<T, P, QG, GEN, false>(A, e, (S*)A.grad_kappa, G, f, rec, wts, tri3, UX, UY, HZ);
  }
  if (A.GM) {
    if (A.GK && !two) {
      __syncthreads();   // the stiffness pass is done with the buffer
      issue_block<S, C::N, C::GS, NT>((const S*)A.GM + e * NN, G1);
    }
    wait_blocks<0>();
    grad_pass<T, P, QG, GEN, true>(A, e, (S*)A.grad_rho, G1, f, rec, wts, tri3, UX, UY, HZ);
  }
}

// 2D: one CTA per element, both upstream blocks in shared memory (padded rows,
// cp.async) and replaced by S = G + G^T; for each Gauss point q1 of x the x
// stage UX_st[a2][b2] = sum_{a1 b1} f^s_x(q1)[a1] S[a][b] f^t_x(q1)[b1] for the
// pairs the terms need, then one thread per q2 forms every term
// H_ij(q1, q2) = sum_{a2 b2} f_y(q2)[a2] f_y(q2)[b2] UX[a2][b2] and the
// geometry: terms (0,0), (1,1) and, for a general map, (0,1) twice.
template <typename T, int P, int QG, bool GEN>
__global__ void __launch_bounds__(64) k_grad2(const GradArgs A) {
  constexpr int n = P + 1, q = QG, N = n * n, GS = N + 1, NT = 64, REC = 2 * q * n + q;
  constexpr int NP = GEN ? 3 : 2;              // x pairs (d, d), (v, v), (d, v)
  __shared__ __align__(16) T Gs[2][N * GS];
  __shared__ double rec[2 * REC];
  __shared__ T f[2][2][q * n];
  __shared__ T UX[NP + 1][N];                  // the stiffness pairs, then the mass pair
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  int e1, e2;
  elem_coords2(A, e, e1, e2);
  const int64_t NN = (int64_t)N * N;
  if (A.GK) issue_block<T, N, GS, NT>((const T*)A.GK + e * NN, Gs[0]);
  if (A.GM) issue_block<T, N, GS, NT>((const T*)A.GM + e * NN, Gs[1]);
  for (int i = tid; i < 2 * REC; i += NT) {
    const int d = i / REC, j = i - d * REC;
    rec[i] = (d == 0 ? A.tab[0] + (int64_t)e1 * REC : A.tab[1] + (int64_t)e2 * REC)[j];
  }
  wait_blocks<0>();
  for (int i = tid; i < 2 * 2 * q * n; i += NT) {
    const int d = i / (2 * q * n), j = i % (2 * q * n);
    (&f[0][0][0])[i] = (T)rec[d * REC + j];
  }
  for (int m = 0; m < 2; ++m) {
    if ((m == 0 && !A.GK) || (m == 1 && !A.GM)) continue;
    T* G = Gs[m];
    for (int idx = tid; idx < N * N; idx += NT) {
      const int a = idx / N, b = idx - a * N;
      if (a <= b) {
        const T s = G[a * GS + b] + G[b * GS + a];
        G[a * GS + b] = s;
        G[b * GS + a] = s;
      }
    }
  }
  __syncthreads();
  const bool doK = A.GK != nullptr, doM = A.GM != nullptr;
#pragma unroll 1
  for (int q1 = 0; q1 < q; ++q1) {
    const T* fx0 = &f[0][0][q1 * n];
    const T* fx1 = &f[0][1][q1 * n];
    for (int it = tid; it < 2 * N; it += NT) {
      const int m = it / N, ab = it - m * N, a2 = ab / n, b2 = ab % n;
      if ((m == 0 && !doK) || (m == 1 && !doM)) continue;
      const T* G = Gs[m];
      T v0[n], v1[n];
#pragma unroll
      for (int a1 = 0; a1 < n; ++a1) {
        T s0 = 0, s1 = 0;
#pragma unroll
        for (int b1 = 0; b1 < n; ++b1) {
          const T g = G[(a1 + n * a2) * GS + n * b2 + b1];
          s0 += g * fx0[b1];
          s1 += g * fx1[b1];
        }
        v0[a1] = s0;
        v1[a1] = s1;
      }
      T p00 = 0, p11 = 0, p10 = 0;
#pragma unroll
      for (int a1 = 0; a1 < n; ++a1) {
        p00 += fx0[a1] * v0[a1];
        p11 += fx1[a1] * v1[a1];
        p10 += fx1[a1] * v0[a1];
      }
      if (m == 1) {
        UX[NP][ab] = p00;
      } else {
        UX[0][ab] = p11;
        UX[1][ab] = p00;
        if (GEN) UX[2][ab] = p10;
      }
    }
    __syncthreads();
    for (int q2 = tid; q2 < q; q2 += NT) {
      const T* fy0 = &f[1][0][q2 * n];
      const T* fy1 = &f[1][1][q2 * n];
      // H00: x pair (d, d) with y values; H11: (v, v) with y derivatives;
      // H01: (d, v) with y (value, derivative); the mass: (v, v) with y values
      T h00 = 0, h11 = 0, h01 = 0, hm = 0;
#pragma unroll
      for (int a2 = 0; a2 < n; ++a2) {
        T s00 = 0, s11 = 0, s01 = 0, sm = 0;
#pragma unroll
        for (int b2 = 0; b2 < n; ++b2) {
          const int ab = a2 * n + b2;
          if (doK) {
            s00 += fy0[b2] * UX[0][ab];
            s11 += fy1[b2] * UX[1][ab];
            if (GEN) s01 += fy1[b2] * UX[2][ab];
          }
          if (doM) sm += fy0[b2] * UX[NP][ab];
        }
        h00 += fy0[a2] * s00;
        h11 += fy1[a2] * s11;
        h01 += fy0[a2] * s01;
        hm += fy0[a2] * sm;
      }
      const int k = q1 + q * q2;
      const double W = 0.5 * rec[2 * q * n + q1] * rec[REC + 2 * q * n + q2];
      if (GEN) {
        const double* Gq = A.jac + (e * q * q + k) * 4;
        const double g00 = Gq[0], g01 = Gq[1], g10 = Gq[2], g11 = Gq[3];
        // cofactors c = [[g11, -g10], [-g01, g00]]; w |det| (G^{-1} G^{-T})_ij
        // = (w / |det|) sum_m c_mi c_mj
        const double adet = fabs(g00 * g11 - g01 * g10);
        const double wk = W / adet;
        const double d00 = wk * (g11 * g11 + g01 * g01);
        const double d11 = wk * (g10 * g10 + g00 * g00);
        const double d01 = wk * (-g11 * g10 - g01 * g00);
        if (doK)
          ((T*)A.grad_kappa)[e * q * q + k] = (T)d00 * h00 + (T)d11 * h11 + (T)(2.0 * d01) * h01;
        if (doM) ((T*)A.grad_rho)[e * q * q + k] = (T)(W * adet) * hm;
      } else {
        if (doK) ((T*)A.grad_kappa)[e * q * q + k] = (T)W * (h00 + h11);
        if (doM) ((T*)A.grad_rho)[e * q * q + k] = (T)W * hm;
      }
    }
    __syncthreads();
  }
}

template <typename T, int P, int QG, bool GEN>
cudaError_t run2(const GradArgs& a, cudaStream_t st) {
  k_grad2<T, P, QG, GEN><<<(unsigned)a.n_elem, 64, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int P, int QG, bool GEN>
cudaError_t run1(GradArgs a, cudaStream_t st) {
  using C = GRD<T, P, QG, GEN>;
  a.two_buffers = a.GK && a.GM && C::TWO;
  const size_t dyn = C::dyn_bytes * (a.two_buffers ? 2 : 1);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_grad3<T, P, QG, GEN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(C::dyn_bytes * (C::TWO ? 2 : 1)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_grad3<T, P, QG, GEN>,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_grad3<T, P, QG, GEN><<<(unsigned)a.n_elem, C::NT, dyn, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int P, int QG>
cudaError_t run(const GradArgs& a, cudaStream_t st) {
  return a.jac ? run1<T, P, QG, true>(a, st) : run1<T, P, QG, false>(a, st);
}

template <typename T>
cudaError_t dispatch(const GradArgs& a, int dim, int p, int q, cudaStream_t st) {
  const int dq = q - p;
  if (dim == 2) {
    if constexpr (sizeof(T) == 8) {   // 2D plans are FP64 (the FP32 forms are 3D)
#define C2(PP)                                                                             \
  if (p == PP && dq == 1)                                                                  \
    return a.jac ? run2<T, PP, PP + 1, true>(a, st) : run2<T, PP, PP + 1, false>(a, st);   \
  if (p == PP && dq == 2)                                                                  \
    return a.jac ? run2<T, PP, PP + 2, true>(a, st) : run2<T, PP, PP + 2, false>(a, st);
      C2(1) C2(2) C2(3) C2(4) C2(5)
#undef C2
    }
    return cudaErrorInvalidValue;
  }
#define C3(PP)                                               \
  if (p == PP && dq == 1) return run<T, PP, PP + 1>(a, st);  \
  if (p == PP && dq == 2) return run<T, PP, PP + 2>(a, st);
  C3(1) C3(2) C3(3)
#undef C3
  if (p == 4 && dq == 1) return run<T, 4, 5>(a, st);
  if (p == 4 && dq == 2) return run<T, 4, 6>(a, st);
  if constexpr (sizeof(T) == 4) {
    // the FP32 block of p = 5 (187.5 KB padded) fits one CTA; the FP64 one does not
    if (p == 5 && dq == 1) return run<T, 5, 6>(a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t dispatch_ff(const GradArgs& a, int p, int q, cudaStream_t st) {
  const int dq = q - p;
#define CF(PP)                                                \
  if (p == PP && dq == 1) return run<ff, PP, PP + 1>(a, st);  \
  if (p == PP && dq == 2) return run<ff, PP, PP + 2>(a, st);
  CF(1) CF(2) CF(3)
#undef CF
  return cudaErrorInvalidValue;
}

}  // namespace

bool grad_supported(int dim, int p, int q, bool fp64) {
  const bool q_ok = q == p + 1 || q == p + 2;
  if (dim == 2) return fp64 && p >= 1 && p <= 5 && q_ok;
  if (dim != 3 || p < 1) return false;
  if (p <= 4) return q_ok;
  return p == 5 && q == 6 && !fp64;
}

cudaError_t launch_grad(const GradArgs& a, int dim, int p, int q, bool fp64, bool df,
                        cudaStream_t st) {
  if (a.n_elem <= 0) return cudaSuccess;
  // float-float where the blocks stay in registers (3D p <= 3), else FP64
  if (df && dim == 3 && p <= 3) return dispatch_ff(a, p, q, st);
  return fp64 ? dispatch<double>(a, dim, p, q, st) : dispatch<float>(a, dim, p, q, st);
}

}  // namespace iga
