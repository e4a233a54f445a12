// iga_capi.cu -- host side of the C ABI declared in include/iga.h: argument
// and knot validation, element spans, Gauss--Legendre rules, plan layout,
// device tables and kernel launches.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "iga_batch.h"
#include "iga_internal.h"

using namespace iga;

struct iga_plan_s {
  int device = 0;
  iga_plan_opts opts{};
  int dim = 0;
  int n_patches = 0;
  std::vector<PatchDev> ph;          // host copy of the patch descriptions
  std::vector<std::vector<int>> spans_h;  // [patch*dim + k]
  PatchDev* d_patches = nullptr;
  double* d_knots = nullptr;
  int* d_spans = nullptr;
  double* d_gauss = nullptr;
  double* d_tables = nullptr;
  TableJob* d_jobs = nullptr;
  int n_jobs = 0;
  int* d_err = nullptr;
  double* d_partial = nullptr;   // adjoint scratch: one double per element
  int sticky = IGA_OK;
  // batched schedules (FP32/BF16 sum factorization)
  bool use_batch = false;
  bool use_graph = false;
  BatchState batch;
  // profiling: event pairs around the element-matrix kernels
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
  size_t prof_used = 0;
  int64_t prof_launches = 0;
  std::vector<int64_t> elem_off, qp_off, dof_off, mat_off, dofmap_off;
  // assembled form: per-patch coupling data (host) and the 1D records (device)
  std::vector<CsrPatch> csr;
  FnCouple* d_fc = nullptr;
  // operator application: per-element results [N][E] per patch, allocated by
  // the first iga_apply call
  void* d_apply_scratch = nullptr;
  // weighted quadrature: per patch and direction, built by the first call
  struct WqDir {
    std::vector<double> x;      // global points
    int qmax = 0;
    int* d_qlo = nullptr;
    int* d_qn = nullptr;
    double* d_V = nullptr;
    double* d_V1 = nullptr;     // derivative rule x trial derivatives (p >= 2)
  };
  std::vector<WqDir> wq;        // [patch * 3 + k]
  std::vector<int64_t> wq_coef_off;  // [n_patches + 1] prefix of the grid sizes
  std::vector<double> knots_host;    // all knot vectors, as uploaded
  std::vector<FnCouple> fc_host;     // all coupling records, as uploaded
  int wq_status = -1;           // -1 not built, else the build's iga_status
  iga_plan_info info{};
};

namespace {

bool g_log = false;

// NVTX range around a public call (visible in Nsight timelines; a no-op
// without a profiler attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

void log_msg(const char* msg) {
  if (g_log) fprintf(stderr, "[iga] %s\n", msg);
}

// Gauss--Legendre on [-1,1] by Newton's method on the Legendre polynomial
// P_q (three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1});
// weight 2 / ((1 - x^2) P_q'(x)^2).  Symmetric nodes are mirrored exactly.
void gauss_legendre_newton(int q, double* x, double* w) {
  for (int i = 0; i < (q + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < q; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) { p1 = z; p0 = 1.0; }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    // final derivative at the converged node
    {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < q; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) { p1 = z; p0 = 1.0; }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
    }
    double wi = 2.0 / ((1.0 - z * z) * dp * dp);
    x[q - 1 - i] = z;   // z > 0 for the first half: largest nodes first
    x[i] = -z;
    w[i] = w[q - 1 - i] = wi;
  }
  if (q % 2 == 1) x[q / 2] = 0.0;
}

int validate_knots(const double* t, int m, int p) {
  if (!t || m < 2 * p + 2) return IGA_ERR_KNOTS;
  for (int i = 0; i < m; ++i)
    if (!std::isfinite(t[i])) return IGA_ERR_KNOTS;
  for (int i = 1; i < m; ++i)
    if (t[i] < t[i - 1]) return IGA_ERR_KNOTS;
  for (int i = 1; i <= p; ++i)
    if (t[i] != t[0] || t[m - 1 - i] != t[m - 1]) return IGA_ERR_KNOTS;
  if (!(t[m - 1] > t[0])) return IGA_ERR_KNOTS;
  // open: exactly p+1 repeated end knots; interior multiplicity <= p
  if (t[p + 1] == t[0] || t[m - p - 2] == t[m - 1]) return IGA_ERR_KNOTS;
  int run = 1;
  for (int i = p + 2; i < m - p - 1; ++i) {
    run = (t[i] == t[i - 1]) ? run + 1 : 1;
    if (run > p) return IGA_ERR_KNOTS;
  }
  return IGA_OK;
}

std::vector<int> knot_spans(const double* t, int m, int p) {
  std::vector<int> s;
  for (int i = p; i <= m - p - 2; ++i)
    if (t[i] < t[i + 1]) s.push_back(i);
  return s;
}

// Coupling records of the nf functions of one direction.  Function i is
// non-zero on the elements whose span s satisfies s - p <= i <= s (Sec. 3.1,
// Remark on the support set), a contiguous run of elements because the spans
// increase; the functions sharing an element with i are then
// s(elo) - p .. s(ehi).
std::vector<FnCouple> couple_1d(const std::vector<int>& spans, int p, int nf) {
  std::vector<FnCouple> out(nf);
  int64_t S = 0;
  for (int i = 0; i < nf; ++i) {
    FnCouple f;
    f.elo = (int)(std::lower_bound(spans.begin(), spans.end(), i) - spans.begin());
    f.ehi = (int)(std::upper_bound(spans.begin(), spans.end(), i + p) - spans.begin()) - 1;
    f.flo = spans[f.elo] - p;
    f.fhi = spans[f.ehi];
    f.S = S;
    S += f.fhi - f.flo + 1;
    out[i] = f;
  }
  return out;
}

// Values of the p+1 B-splines non-zero on span s at x (triangular Cox--de Boor
// of Sec. 2.3, the polynomial piece of span s, so x at the span's right end
// gives the left limit): N[r] = B_{s-p+r;p}(x).  The left/right/saved
// evaluation is Piegl and Tiller's, The NURBS Book (2nd ed.), Algorithm A2.2.
void host_basis(const double* t, int p, int s, double x, double* N) {
  double left[kMaxDegree2D + 1], right[kMaxDegree2D + 1];
  N[0] = 1.0;
  for (int d = 1; d <= p; ++d) {
    left[d] = x - t[s + 1 - d];
    right[d] = t[s + d] - x;
    double saved = 0.0;
    for (int r = 0; r < d; ++r) {
      const double tmp = N[r] / (right[r + 1] + left[d - r]);
      N[r] = saved + right[r + 1] * tmp;
      saved = left[d - r] * tmp;
    }
    N[d] = saved;
  }
}

// B_{j;p}(x) for x in [t_p, t_end]: the span holding x (the last non-empty span
// for the right end), then the triangular values.
double host_bspline(const double* t, const std::vector<int>& spans, int p, int j, double x) {
  size_t e = std::upper_bound(spans.begin(), spans.end(), 0, [&](int, int s) { return x < t[s]; }) -
             spans.begin();
  e = e == 0 ? 0 : e - 1;
  const int s = spans[e];
  if (j < s - p || j > s) return 0.0;
  double N[kMaxDegree2D + 1];
  host_basis(t, p, s, x, N);
  return N[j - (s - p)];
}

// Derivatives of the p+1 B-splines non-zero on span s at x (de Boor's
// formula from the degree p-1 values of the span, so the right end of the
// span gives the left limit): dN[r] = B'_{s-p+r;p}(x).
void host_basis_deriv(const double* t, int p, int s, double x, double* dN) {
  double Nm[kMaxDegree2D + 1];
  host_basis(t, p - 1, s, x, Nm);   // Nm[r] = B_{s-p+1+r;p-1}(x), r = 0..p-1
  for (int r = 0; r <= p; ++r) {
    const int j = s - p + r;
    double d = 0.0;
    if (r >= 1) d += Nm[r - 1] / (t[j + p] - t[j]);
    if (r <= p - 1) d -= Nm[r] / (t[j + p + 1] - t[j + 1]);
    dN[r] = p * d;
  }
}

double host_bspline_deriv(const double* t, const std::vector<int>& spans, int p, int j, double x) {
  size_t e = std::upper_bound(spans.begin(), spans.end(), 0, [&](int, int s) { return x < t[s]; }) -
             spans.begin();
  e = e == 0 ? 0 : e - 1;
  const int s = spans[e];
  if (j < s - p || j > s) return 0.0;
  double dN[kMaxDegree2D + 1];
  host_basis_deriv(t, p, s, x, dN);
  return dN[j - (s - p)];
}

// Least-norm w = A^T y with (A A^T) y = r for the first ns rows of A [nj][nq]
// (Cholesky of the Gram matrix); V[(i W + jj) qmax + qq] = w_q A[jj][q] for
// every jj < nj.  Returns IGA_OK, or IGA_ERR_UNSUPPORTED if the Gram matrix is
// not positive definite.
int wq_least_norm(const std::vector<double>& A, std::vector<double> r, int nj, int ns, int nq,
                  int i, int W, int qmax, std::vector<double>* V_out) {
  std::vector<double> G((size_t)ns * ns, 0.0);
  for (int u = 0; u < ns; ++u)
    for (int v = 0; v <= u; ++v) {
      double acc = 0.0;
      for (int qq = 0; qq < nq; ++qq) acc += A[(size_t)u * nq + qq] * A[(size_t)v * nq + qq];
      G[(size_t)u * ns + v] = acc;
    }
  // Cholesky G = L L^T (lower triangle in place), then L L^T y = r
  for (int u = 0; u < ns; ++u) {
    for (int v = 0; v <= u; ++v) {
      double acc = G[(size_t)u * ns + v];
      for (int k = 0; k < v; ++k) acc -= G[(size_t)u * ns + k] * G[(size_t)v * ns + k];
      if (u == v) {
        if (!(acc > 0.0)) return IGA_ERR_UNSUPPORTED;
        G[(size_t)u * ns + u] = std::sqrt(acc);
      } else {
        G[(size_t)u * ns + v] = acc / G[(size_t)v * ns + v];
      }
    }
  }
  for (int u = 0; u < ns; ++u) {
    double acc = r[u];
    for (int k = 0; k < u; ++k) acc -= G[(size_t)u * ns + k] * r[k];
    r[u] = acc / G[(size_t)u * ns + u];
  }
  for (int u = ns - 1; u >= 0; --u) {
    double acc = r[u];
    for (int k = u + 1; k < ns; ++k) acc -= G[(size_t)k * ns + u] * r[k];
    r[u] = acc / G[(size_t)u * ns + u];
  }
  std::vector<double>& V = *V_out;
  for (int qq = 0; qq < nq; ++qq) {
    double w = 0.0;
    for (int jj = 0; jj < ns; ++jj) w += A[(size_t)jj * nq + qq] * r[jj];
    for (int jj = 0; jj < nj; ++jj) V[((size_t)i * W + jj) * qmax + qq] = w * A[(size_t)jj * nq + qq];
  }
  return IGA_OK;
}

// One direction of the weighted quadrature of the mass matrix: the global
// points (each element's left end and midpoint, p+1 points in the p boundary
// elements at each end, the right end), and for each test function i the
// least-norm weights on the points of its closed support that integrate
// B_i B_j exactly for every coupled j (G y = r with G = A A^T by Cholesky,
// w = A^T y; A[j][q] = B_j(x_q), r_j = int B_i B_j by Gauss--Legendre with
// p+1 points per element).  Output: V[(i W + jj) qmax + qq] = w_q B_j(x_q).
int wq_build_direction(const double* t, int p, const std::vector<int>& spans,
                       const std::vector<FnCouple>& fc, std::vector<double>* x_out,
                       std::vector<int>* qlo_out, std::vector<int>* qn_out,
                       std::vector<double>* V_out, std::vector<double>* V1_out, int* qmax_out) {
  const int K = (int)spans.size(), nf = (int)fc.size(), W = 2 * p + 1;
  std::vector<double>& x = *x_out;
  x.clear();
  for (int e = 0; e < K; ++e) {
    const double a = t[spans[e]], b = t[spans[e] + 1];
    x.push_back(a);
    if (e < p || e >= K - p) {
      for (int r = 1; r <= p; ++r) x.push_back(a + (b - a) * r / (double)(p + 1));
    } else {
      x.push_back(0.5 * (a + b));
    }
  }
  x.push_back(t[spans[K - 1] + 1]);
  std::vector<double> gx(p + 1), gw(p + 1);
  gauss_legendre_newton(p + 1, gx.data(), gw.data());
  std::vector<int>& qlo = *qlo_out;
  std::vector<int>& qn = *qn_out;
  qlo.assign(nf, 0);
  qn.assign(nf, 0);
  int qmax = 0;
  for (int i = 0; i < nf; ++i) {
    const double lo = t[i], hi = t[i + p + 1];
    const int a = (int)(std::lower_bound(x.begin(), x.end(), lo) - x.begin());
    const int b = (int)(std::upper_bound(x.begin(), x.end(), hi) - x.begin());
    qlo[i] = a;
    qn[i] = b - a;
    qmax = std::max(qmax, b - a);
  }
  std::vector<double>& V = *V_out;
  V.assign((size_t)nf * W * qmax, 0.0);
  if (V1_out) V1_out->assign((size_t)nf * W * qmax, 0.0);
  for (int i = 0; i < nf; ++i) {
    const int nj = fc[i].fhi - fc[i].flo + 1, nq = qn[i];
    if (nj > W || nq < nj) return IGA_ERR_UNSUPPORTED;
    std::vector<double> A((size_t)nj * nq), r(nj, 0.0);
    for (int jj = 0; jj < nj; ++jj)
      for (int qq = 0; qq < nq; ++qq)
        A[(size_t)jj * nq + qq] = host_bspline(t, spans, p, fc[i].flo + jj, x[qlo[i] + qq]);
    for (int e = fc[i].elo; e <= fc[i].ehi; ++e) {
      const int s = spans[e];
      const double ea = t[s], eb = t[s + 1];
      double N[kMaxDegree2D + 1];
      for (int g = 0; g <= p; ++g) {
        const double xi = 0.5 * (ea + eb) + 0.5 * (eb - ea) * gx[g];
        host_basis(t, p, s, xi, N);
        const double bi = N[i - (s - p)], wg = 0.5 * (eb - ea) * gw[g];
        for (int jj = 0; jj < nj; ++jj) {
          const int j = fc[i].flo + jj;
          if (j >= s - p && j <= s) r[jj] += wg * bi * N[j - (s - p)];
        }
      }
    }
    int rc = wq_least_norm(A, r, nj, nj, nq, i, W, qmax, &V);
    if (rc != IGA_OK) return rc;
    if (V1_out) {
      // the derivative rule: exact against B'_j with B'_i; the B'_j sum to zero
      // on the support, so the last equation is dependent and is dropped
      std::vector<double> A1((size_t)nj * nq), r1(nj, 0.0);
      for (int jj = 0; jj < nj; ++jj)
        for (int qq = 0; qq < nq; ++qq)
          A1[(size_t)jj * nq + qq] = host_bspline_deriv(t, spans, p, fc[i].flo + jj, x[qlo[i] + qq]);
      for (int e = fc[i].elo; e <= fc[i].ehi; ++e) {
        const int s = spans[e];
        const double ea = t[s], eb = t[s + 1];
        double dN[kMaxDegree2D + 1];
        for (int g = 0; g <= p; ++g) {
          const double xi = 0.5 * (ea + eb) + 0.5 * (eb - ea) * gx[g];
          host_basis_deriv(t, p, s, xi, dN);
          const double di = dN[i - (s - p)], wg = 0.5 * (eb - ea) * gw[g];
          for (int jj = 0; jj < nj; ++jj) {
            const int j = fc[i].flo + jj;
            if (j >= s - p && j <= s) r1[jj] += wg * di * dN[j - (s - p)];
          }
        }
      }
      rc = wq_least_norm(A1, r1, nj, nj - 1, nq, i, W, qmax, V1_out);
      if (rc != IGA_OK) return rc;
    }
  }
  *qmax_out = qmax;
  return IGA_OK;
}

// Whether the plan's method and precision can integrate patch pd: FP64 takes
// every patch (specialised kernels where they exist, the runtime-sized ones
// otherwise); the other precisions need a specialised kernel.
bool method_supported(const iga_plan_opts& o, const PatchDev& pd) {
  if (o.precision == IGA_FP64) return true;
  if (!pd.iso) return false;
  const int dim = pd.dim, p = pd.p, q = pd.q;
  if (o.precision == IGA_FP32 || o.precision == IGA_BF16)
    return o.method == IGA_SUMFACT && sumfact_f32_supported(dim, p, q);
  if (o.precision == IGA_FP64_DF) return o.method == IGA_SUMFACT && sumfact_df_supported(dim, p, q);
  return false;
}

// A specialised (compile-time sized) FP64 kernel exists for the patch.
bool fp64_specialised(const iga_plan_opts& o, const PatchDev& pd) {
  if (!pd.iso) return false;
  if (o.method == IGA_SUMFACT) return sumfact_f64_supported(pd.dim, pd.p, pd.q);
  return classical_f64_supported(pd.dim, pd.p, pd.q);
}

template <class T>
cudaError_t upload(T** dst, const T* src, size_t n) {
  *dst = nullptr;
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
}

void free_plan_memory(iga_plan_s* P) {
  batch_free(&P->batch);
  for (auto& pr : P->prof_events) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  P->prof_events.clear();
  cudaFree(P->d_patches);
  cudaFree(P->d_knots);
  cudaFree(P->d_spans);
  cudaFree(P->d_gauss);
  cudaFree(P->d_tables);
  cudaFree(P->d_jobs);
  cudaFree(P->d_err);
  cudaFree(P->d_partial);
  cudaFree(P->d_fc);
  cudaFree(P->d_apply_scratch);
  for (auto& w : P->wq) {
    cudaFree(w.d_qlo);
    cudaFree(w.d_qn);
    cudaFree(w.d_V);
    cudaFree(w.d_V1);
  }
}

int map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return IGA_OK;
  if (e == cudaErrorMemoryAllocation) return IGA_ERR_OOM;
  return IGA_ERR_CUDA;
}

}  // namespace

extern "C" const char* iga_status_str(int s) {
  switch (s) {
    case IGA_OK: return "IGA_OK";
    case IGA_ERR_ARG: return "IGA_ERR_ARG: invalid argument";
    case IGA_ERR_KNOTS: return "IGA_ERR_KNOTS: knot vector not open/non-decreasing or multiplicity > p";
    case IGA_ERR_UNSUPPORTED: return "IGA_ERR_UNSUPPORTED: configuration not built";
    case IGA_ERR_CUDA: return "IGA_ERR_CUDA: CUDA runtime error";
    case IGA_ERR_OOM: return "IGA_ERR_OOM: device allocation failed";
    case IGA_ERR_TIMEOUT: return "IGA_ERR_TIMEOUT: bounded device wait expired";
    case IGA_ERR_DEVICE: return "IGA_ERR_DEVICE: device-side consistency check failed";
    case IGA_ERR_TOO_LARGE:
      return "IGA_ERR_TOO_LARGE: the patch exceeds the fixed scratch of the allocation-free entry "
             "point (at most 1024 knots per direction, 262144 elements, 196608 table doubles)";
    default: return "unknown iga status";
  }
}

extern "C" int iga_plan(iga_plan_t* out, const iga_patch_desc* patches, int n_patches,
                        const iga_plan_opts* opts, iga_plan_info* info_out) {
  if (out) *out = nullptr;
  const char* lg = getenv("IGA_LOG");
  g_log = lg && lg[0] == '1';
  if (!out || !patches || n_patches < 1 || !opts) return IGA_ERR_ARG;
  const iga_plan_opts o = *opts;
  if (o.method != IGA_CLASSICAL && o.method != IGA_SUMFACT) return IGA_ERR_ARG;
  if (o.precision < IGA_FP64 || o.precision > IGA_FP64_DF) return IGA_ERR_ARG;
  if (o.matrices < 1 || o.matrices > 3) return IGA_ERR_ARG;
  if (o.method == IGA_CLASSICAL && o.precision != IGA_FP64) return IGA_ERR_UNSUPPORTED;
  if (o.schedule < IGA_SCHED_AUTO || o.schedule > IGA_SCHED_PERSISTENT_GRAPH) return IGA_ERR_ARG;
  const bool lowprec_sf =
      o.method == IGA_SUMFACT && (o.precision == IGA_FP32 || o.precision == IGA_BF16);
  if (!lowprec_sf && o.schedule > IGA_SCHED_PER_PATCH) return IGA_ERR_UNSUPPORTED;
  const int dim = patches[0].dim;
  if (dim != 2 && dim != 3) return IGA_ERR_ARG;

  iga_plan_s* P = new (std::nothrow) iga_plan_s();
  if (!P) return IGA_ERR_OOM;
  P->opts = o;
  P->dim = dim;
  P->n_patches = n_patches;

  std::vector<double> knots_all, gauss_all;
  std::vector<int> spans_all;
  std::vector<TableJob> jobs;
  int64_t e_off = 0, qp_off = 0, dof_off = 0, mat_off = 0, dm_off = 0, tab_off = 0;
  for (int ip = 0; ip < n_patches; ++ip) {
    const iga_patch_desc& d = patches[ip];
    if (d.dim != dim) { delete P; return IGA_ERR_UNSUPPORTED; }
    PatchDev pd{};
    pd.dim = dim;
    pd.iso = 1;
    for (int k = 0; k < 3; ++k) {
      if (k >= dim) { pd.pk[k] = 0; pd.qk[k] = 1; pd.nk[k] = 1; continue; }
      const int p = d.degree[k], q = d.n_gauss[k];
      if (p < 1 || p > kMaxDegree || q < 1 || q > kMaxGauss) { delete P; return IGA_ERR_ARG; }
      pd.pk[k] = p; pd.qk[k] = q; pd.nk[k] = p + 1;
      if (p != d.degree[0] || q != d.n_gauss[0]) pd.iso = 0;
    }
    for (int k = 0; k < dim; ++k) {
      int rc = validate_knots(d.knots[k], d.n_knots[k], pd.pk[k]);
      if (rc != IGA_OK) { delete P; return rc; }
    }
    pd.p = pd.pk[0]; pd.q = pd.qk[0]; pd.n = pd.nk[0];
    if (!method_supported(o, pd)) { delete P; return IGA_ERR_UNSUPPORTED; }
    pd.N = 1; pd.Q = 1;
    int64_t E = 1, nd = 1;
    for (int k = 0; k < 3; ++k) {
      if (k >= dim) { pd.K[k] = 1; pd.nf[k] = 1; continue; }
      const int p = pd.pk[k], q = pd.qk[k];
      pd.gauss_offset[k] = (int)gauss_all.size();
      std::vector<double> xr(q), wr(q);
      gauss_legendre_newton(q, xr.data(), wr.data());
      gauss_all.insert(gauss_all.end(), xr.begin(), xr.end());
      gauss_all.insert(gauss_all.end(), wr.begin(), wr.end());
      const double* t = d.knots[k];
      const int m = d.n_knots[k];
      std::vector<int> s = knot_spans(t, m, p);
      pd.K[k] = (int)s.size();
      pd.nf[k] = m - p - 1;
      pd.knot_offset[k] = (int)knots_all.size();
      pd.span_offset[k] = (int)spans_all.size();
      pd.tab_offset[k] = tab_off;
      for (int ek = 0; ek < pd.K[k]; ++ek) {
        TableJob j;
        j.knot_off = pd.knot_offset[k];
        j.span = s[ek];
        j.p = p; j.q = q;
        j.gauss_off = pd.gauss_offset[k];
        j.out_off = tab_off;
        jobs.push_back(j);
        tab_off += record_size(p + 1, q);
      }
      knots_all.insert(knots_all.end(), t, t + m);
      spans_all.insert(spans_all.end(), s.begin(), s.end());
      P->spans_h.push_back(s);
      E *= pd.K[k];
      nd *= pd.nf[k];
      pd.N *= pd.nk[k];
      pd.Q *= q;
    }
    pd.elem_offset = e_off; pd.qp_offset = qp_off; pd.dof_offset = dof_off;
    pd.mat_offset = mat_off; pd.dofmap_offset = dm_off;
    P->elem_off.push_back(e_off); P->qp_off.push_back(qp_off); P->dof_off.push_back(dof_off);
    P->mat_off.push_back(mat_off); P->dofmap_off.push_back(dm_off);
    e_off += E;
    qp_off += E * pd.Q;
    dof_off += nd;
    mat_off += E * (int64_t)pd.N * pd.N;
    dm_off += E * (int64_t)pd.N;
    if (dm_off > INT32_MAX || dof_off > INT32_MAX || E > INT32_MAX) {
      delete P;
      return IGA_ERR_UNSUPPORTED;
    }
    P->ph.push_back(pd);
  }
  P->elem_off.push_back(e_off); P->qp_off.push_back(qp_off); P->dof_off.push_back(dof_off);
  P->mat_off.push_back(mat_off); P->dofmap_off.push_back(dm_off);
  P->n_jobs = (int)jobs.size();

  // coupling data of the assembled form (tensor product of 1D ranges)
  std::vector<FnCouple> fc_all;
  int64_t nnz_off = 0;
  for (int ip = 0; ip < n_patches; ++ip) {
    const PatchDev& pd = P->ph[ip];
    CsrPatch c{};
    c.dim = pd.dim; c.p = pd.p; c.n = pd.n; c.N = pd.N;
    c.dof_offset = pd.dof_offset; c.mat_offset = pd.mat_offset; c.elem_offset = pd.elem_offset;
    c.nnz_offset = nnz_off;
    int64_t nnz = 1;
    int64_t lmax = 1;
    for (int k = 0; k < 3; ++k) {
      c.K[k] = pd.K[k]; c.nf[k] = pd.nf[k];
      c.span_offset[k] = pd.span_offset[k];
      if (k >= pd.dim) { c.fn_offset[k] = -1; c.W[k] = 1; continue; }
      std::vector<FnCouple> f = couple_1d(P->spans_h[(size_t)ip * dim + k], pd.pk[k], pd.nf[k]);
      c.fn_offset[k] = (int)fc_all.size();
      c.W[k] = f.back().S + (f.back().fhi - f.back().flo + 1);
      int wmax = 0;
      for (const FnCouple& x : f) wmax = std::max(wmax, x.fhi - x.flo + 1);
      lmax *= wmax;
      nnz *= c.W[k];
      fc_all.insert(fc_all.end(), f.begin(), f.end());
    }
    c.lmax = (int)lmax;
    nnz_off += nnz;
    P->csr.push_back(c);
  }

  cudaError_t ce = cudaGetDevice(&P->device);
  if (ce == cudaSuccess) ce = upload(&P->d_patches, P->ph.data(), P->ph.size());
  if (ce == cudaSuccess) ce = upload(&P->d_knots, knots_all.data(), knots_all.size());
  if (ce == cudaSuccess) ce = upload(&P->d_spans, spans_all.data(), spans_all.size());
  if (ce == cudaSuccess) ce = upload(&P->d_gauss, gauss_all.data(), gauss_all.size());
  if (ce == cudaSuccess) ce = upload(&P->d_jobs, jobs.data(), jobs.size());
  if (ce == cudaSuccess) ce = upload(&P->d_fc, fc_all.data(), fc_all.size());
  P->knots_host = knots_all;
  P->fc_host = fc_all;
  if (ce == cudaSuccess) ce = cudaMalloc((void**)&P->d_tables, sizeof(double) * (size_t)tab_off);
  if (ce == cudaSuccess) ce = cudaMalloc((void**)&P->d_err, sizeof(int));
  if (ce == cudaSuccess) ce = cudaMemset(P->d_err, 0, sizeof(int));
  if (ce == cudaSuccess && e_off > 0)
    ce = cudaMalloc((void**)&P->d_partial, sizeof(double) * (size_t)e_off);
  if (ce != cudaSuccess) {
    free_plan_memory(P);
    delete P;
    cudaGetLastError();
    return map_cuda(ce);
  }
  if (lowprec_sf) {
    const int sched = o.schedule == IGA_SCHED_AUTO
                          ? (n_patches > 1 ? IGA_SCHED_PERSISTENT_GRAPH : IGA_SCHED_PER_PATCH)
                          : o.schedule;
    if (sched != IGA_SCHED_PER_PATCH) {
      P->use_batch = true;
      P->use_graph = sched == IGA_SCHED_PERSISTENT_GRAPH;
      const int rc = batch_plan(&P->batch, P->ph, o.precision, o.schedule);
      if (rc != IGA_OK) {
        free_plan_memory(P);
        delete P;
        cudaGetLastError();
        return rc;
      }
    }
  }
  iga_plan_info& I = P->info;
  I.n_elements = e_off; I.n_qp = qp_off; I.n_dofs = dof_off;
  I.n_mat_entries = mat_off; I.n_dofmap_entries = dm_off; I.n_table_entries = tab_off;
  I.dim = dim; I.n_patches = n_patches; I.local_n = P->ph[0].N;
  I.elem_offset = P->elem_off.data(); I.qp_offset = P->qp_off.data();
  I.dof_offset = P->dof_off.data(); I.mat_offset = P->mat_off.data();
  I.dofmap_offset = P->dofmap_off.data();
  I.n_csr_nnz = nnz_off;
  if (info_out) *info_out = I;
  log_msg("plan built");
  *out = P;
  return IGA_OK;
}

namespace {
struct ProCtx {
  iga_plan_s* P;
  int32_t* dof_out;
};

// Basis tables of every patch, then the dof maps (when requested).
cudaError_t run_prologue(void* c, cudaStream_t st) {
  ProCtx* x = (ProCtx*)c;
  iga_plan_s* P = x->P;
  cudaError_t e = launch_basis_tables(P->d_jobs, P->n_jobs, P->d_knots, P->d_gauss,
                                      P->d_tables, st);
  if (e == cudaSuccess && x->dof_out) {
    for (int ip = 0; ip < P->n_patches && e == cudaSuccess; ++ip)
      e = launch_dofmap(P->d_patches + ip, P->ph[ip], P->d_spans,
                        x->dof_out + P->ph[ip].dofmap_offset, st);
  }
  return e;
}
}  // namespace

static int finish(iga_plan_s* P, cudaStream_t st, cudaError_t launch_err) {
  if (launch_err != cudaSuccess) {
    P->sticky = map_cuda(launch_err);
    return P->sticky;
  }
  if (!P->opts.blocking) return IGA_OK;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { P->sticky = map_cuda(e); return P->sticky; }
  int h = 0;
  e = cudaMemcpy(&h, P->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) { P->sticky = map_cuda(e); return P->sticky; }
  if (h != 0) P->sticky = h;
  return h;
}

extern "C" int iga_integrate(iga_plan_t P, const double* kappa, const double* rho,
                             const double* jac, void* K_out, void* M_out, int32_t* dof_out,
                             void* cuda_stream) {
  NvtxRange range("iga_integrate");
  if (!P) return IGA_ERR_ARG;
  if (P->sticky != IGA_OK) return P->sticky;
  const bool want_K = (P->opts.matrices & IGA_STIFF) && K_out;
  const bool want_M = (P->opts.matrices & IGA_MASS) && M_out;
  if (!want_K && !want_M && !dof_out) return IGA_ERR_ARG;
  if ((K_out && !(P->opts.matrices & IGA_STIFF)) || (M_out && !(P->opts.matrices & IGA_MASS)))
    return IGA_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return IGA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  ProCtx pctx{P, dof_out};
  cudaError_t e = cudaSuccess;
  if (P->use_batch && (want_K || want_M)) {
    QueueArgs b{};
    b.patches = P->d_patches;
    b.n_patches = P->n_patches;
    b.tables = P->d_tables;
    b.kappa = kappa; b.rho = rho; b.jac = jac;
    b.K_out = want_K ? K_out : nullptr;
    b.M_out = want_M ? M_out : nullptr;
    b.err = P->d_err;
    const int mode = (want_K && want_M) ? 0 : (want_K ? 1 : 2);
    BatchPrologue pro{run_prologue, &pctx, dof_out};
    std::pair<cudaEvent_t, cudaEvent_t>* evb = nullptr;
    if (P->opts.profile) {
      if (P->prof_used == P->prof_events.size()) {
        cudaEvent_t a0, b0;
        e = cudaEventCreate(&a0);
        if (e == cudaSuccess) e = cudaEventCreate(&b0);
        if (e == cudaSuccess) P->prof_events.push_back({a0, b0});
      }
      if (e == cudaSuccess) {
        evb = &P->prof_events[P->prof_used++];
        e = cudaEventRecord(evb->first, st);
      }
    }
    if (e == cudaSuccess) e = batch_integrate(&P->batch, b, mode, st, pro, P->use_graph);
    if (e == cudaSuccess && evb) {
      e = cudaEventRecord(evb->second, st);
      P->prof_launches += 1;
    }
    return finish(P, st, e);
  }
  e = run_prologue(&pctx, st);
  const bool dbl_out = P->opts.precision == IGA_FP64 || P->opts.precision == IGA_FP64_DF;
  const size_t esz = dbl_out ? sizeof(double) : sizeof(float);
  std::pair<cudaEvent_t, cudaEvent_t>* ev = nullptr;
  if (e == cudaSuccess && P->opts.profile && (want_K || want_M)) {
    if (P->prof_used == P->prof_events.size()) {
      cudaEvent_t a, b;
      e = cudaEventCreate(&a);
      if (e == cudaSuccess) e = cudaEventCreate(&b);
      if (e == cudaSuccess) P->prof_events.push_back({a, b});
    }
    if (e == cudaSuccess) {
      ev = &P->prof_events[P->prof_used++];
      e = cudaEventRecord(ev->first, st);
    }
  }
  int64_t n_launch = 0;
  for (int ip = 0; ip < P->n_patches && e == cudaSuccess && (want_K || want_M); ++ip) {
    const PatchDev& pd = P->ph[ip];
    ElemArgs a{};
    a.pd = P->d_patches + ip;
    a.n_elem = (int64_t)pd.K[0] * pd.K[1] * pd.K[2];
    a.K1 = pd.K[0]; a.K2 = pd.K[1]; a.K3 = pd.K[2];
    for (int k = 0; k < 3; ++k) a.tab[k] = P->d_tables + pd.tab_offset[k];
    a.kappa = kappa ? kappa + pd.qp_offset : nullptr;
    a.rho = rho ? rho + pd.qp_offset : nullptr;
    a.jac = jac ? jac + pd.qp_offset * pd.dim * pd.dim : nullptr;
    a.K_out = want_K ? (char*)K_out + esz * pd.mat_offset : nullptr;
    a.M_out = want_M ? (char*)M_out + esz * pd.mat_offset : nullptr;
    a.err = P->d_err;
    const bool spec = fp64_specialised(P->opts, pd);
    if (P->opts.method == IGA_SUMFACT && P->opts.precision == IGA_FP64_DF)
      e = launch_sumfact_df(a, pd.dim, pd.p, pd.q, st);
    else if (P->opts.method == IGA_SUMFACT && P->opts.precision != IGA_FP64)
      e = launch_sumfact_f32(a, pd.dim, pd.p, pd.q, P->opts.precision == IGA_BF16, st);
    else if (P->opts.method == IGA_SUMFACT)
      e = spec ? launch_sumfact_f64(a, pd.dim, pd.p, pd.q, st) : launch_sumfact_gen(a, pd, st);
    else
      e = spec ? launch_classical_f64(a, pd.dim, pd.p, pd.q, st) : launch_classical_gen(a, pd, st);
    ++n_launch;
  }
  if (ev && e == cudaSuccess) {
    e = cudaEventRecord(ev->second, st);
    P->prof_launches += n_launch;
  }
  return finish(P, st, e);
}

extern "C" int iga_integrate_backward(iga_plan_t P, const double* kappa, const double* jac,
                                      const void* u, const void* v, void* grad_kappa,
                                      double* J_out, void* cuda_stream) {
  NvtxRange range("iga_integrate_backward");
  if (!P) return IGA_ERR_ARG;
  if (P->sticky != IGA_OK) return P->sticky;
  if (!u || !v || (!grad_kappa && !J_out) || (J_out && !kappa)) return IGA_ERR_ARG;
  // FP64 plans take every patch (the runtime-sized adjoint where no
  // specialised one exists); the others need a specialised kernel
  for (const PatchDev& pd : P->ph)
    if (P->opts.precision != IGA_FP64 && !(pd.iso && adjoint_supported(pd.dim, pd.p, pd.q)))
      return IGA_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return IGA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const bool fp64 = P->opts.precision == IGA_FP64 || P->opts.precision == IGA_FP64_DF;
  const size_t gsz = fp64 ? sizeof(double) : sizeof(float);
  cudaError_t e = launch_basis_tables(P->d_jobs, P->n_jobs, P->d_knots, P->d_gauss,
                                      P->d_tables, st);
  for (int ip = 0; ip < P->n_patches && e == cudaSuccess; ++ip) {
    const PatchDev& pd = P->ph[ip];
    AdjArgs a{};
    a.n_elem = (int64_t)pd.K[0] * pd.K[1] * pd.K[2];
    a.K1 = pd.K[0]; a.K2 = pd.K[1]; a.K3 = pd.K[2];
    for (int k = 0; k < 3; ++k) {
      a.tab[k] = P->d_tables + pd.tab_offset[k];
      a.span[k] = P->d_spans + pd.span_offset[k];
    }
    a.nf0 = pd.nf[0]; a.nf1 = pd.nf[1];
    a.dof_offset = pd.dof_offset;
    a.kappa = kappa ? kappa + pd.qp_offset : nullptr;
    a.jac = jac ? jac + pd.qp_offset * pd.dim * pd.dim : nullptr;
    a.u = u; a.v = v;
    a.grad = grad_kappa ? (char*)grad_kappa + gsz * pd.qp_offset : nullptr;
    a.partial = J_out ? P->d_partial : nullptr;
    a.partial_offset = pd.elem_offset;
    if (pd.iso && adjoint_supported(pd.dim, pd.p, pd.q))
      e = launch_adjoint(a, pd.dim, pd.p, pd.q, fp64, P->opts.precision == IGA_FP64_DF, st);
    else
      e = launch_adjoint_gen(a, pd, st);
  }
  if (e == cudaSuccess && J_out) e = launch_reduce_fixed(P->d_partial, P->info.n_elements, J_out, st);
  return finish(P, st, e);
}

extern "C" int iga_integrate_grad(iga_plan_t P, const double* jac, const void* GK,
                                  const void* GM, void* grad_kappa, void* grad_rho,
                                  void* cuda_stream) {
  NvtxRange range("iga_integrate_grad");
  if (!P) return IGA_ERR_ARG;
  if (P->sticky != IGA_OK) return P->sticky;
  if ((!GK && !GM) || (GK && !grad_kappa) || (GM && !grad_rho)) return IGA_ERR_ARG;
  const bool fp64 = P->opts.precision == IGA_FP64 || P->opts.precision == IGA_FP64_DF;
  for (const PatchDev& pd : P->ph)
    if (!pd.iso || !grad_supported(pd.dim, pd.p, pd.q, fp64)) return IGA_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return IGA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t esz = fp64 ? sizeof(double) : sizeof(float);
  cudaError_t e = launch_basis_tables(P->d_jobs, P->n_jobs, P->d_knots, P->d_gauss,
                                      P->d_tables, st);
  for (int ip = 0; ip < P->n_patches && e == cudaSuccess; ++ip) {
    const PatchDev& pd = P->ph[ip];
    GradArgs a{};
    a.n_elem = (int64_t)pd.K[0] * pd.K[1] * pd.K[2];
    a.K1 = pd.K[0]; a.K2 = pd.K[1]; a.K3 = pd.K[2];
    for (int k = 0; k < 3; ++k) a.tab[k] = P->d_tables + pd.tab_offset[k];
    a.jac = jac ? jac + pd.qp_offset * pd.dim * pd.dim : nullptr;
    a.GK = GK ? (const char*)GK + esz * pd.mat_offset : nullptr;
    a.GM = GM ? (const char*)GM + esz * pd.mat_offset : nullptr;
    a.grad_kappa = GK ? (char*)grad_kappa + esz * pd.qp_offset : nullptr;
    a.grad_rho = GM ? (char*)grad_rho + esz * pd.qp_offset : nullptr;
    e = launch_grad(a, pd.dim, pd.p, pd.q, fp64, P->opts.precision == IGA_FP64_DF, st);
  }
  return finish(P, st, e);
}

extern "C" int iga_basis_tables(iga_plan_t P, double* out, void* cuda_stream) {
  if (!P || !out) return IGA_ERR_ARG;
  if (P->sticky != IGA_OK) return P->sticky;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return IGA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e = launch_basis_tables(P->d_jobs, P->n_jobs, P->d_knots, P->d_gauss, out, st);
  return finish(P, st, e);
}

extern "C" int iga_csr_pattern(iga_plan_t P, int64_t* row_ptr, int32_t* col_idx,
                               void* cuda_stream) {
  NvtxRange range("iga_csr_pattern");
  if (!P || !row_ptr || !col_idx) return IGA_ERR_ARG;
  if (P->sticky != IGA_OK) return P->sticky;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return IGA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSuccess;
  for (int ip = 0; ip < P->n_patches && e == cudaSuccess; ++ip)
    e = launch_csr_pattern(P->csr[ip], P->d_fc, row_ptr, col_idx, st);
  return finish(P, st, e);
}

extern "C" int iga_assemble(iga_plan_t P, const void* A_elem, void* values, void* cuda_stream) {
  NvtxRange range("iga_assemble");
  if (!P || !A_elem || !values) return IGA_ERR_ARG;
  if (P->sticky != IGA_OK) return P->sticky;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return IGA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const bool fp64 = P->opts.precision == IGA_FP64 || P->opts.precision == IGA_FP64_DF;
  // the gather kernels are specialised per degree (3D: p <= 5, 2D: p <= 8)
  for (const PatchDev& pd : P->ph)
    if (!pd.iso || (pd.dim == 3 && pd.p > 5)) return IGA_ERR_UNSUPPORTED;
  cudaError_t e = cudaSuccess;
  for (int ip = 0; ip < P->n_patches && e == cudaSuccess; ++ip)
    e = launch_assemble(P->csr[ip], P->d_fc, P->d_spans, A_elem, values, fp64, st);
  return finish(P, st, e);
}

extern "C" int iga_apply(iga_plan_t P, const double* kappa, const double* rho, const double* jac,
                         const void* x, double alpha, double beta, void* y, void* cuda_stream) {
  NvtxRange range("iga_apply");
  if (!P || !x || !y) return IGA_ERR_ARG;
  if (P->sticky != IGA_OK) return P->sticky;
  for (const PatchDev& pd : P->ph)
    if (!pd.iso || !apply_supported(pd.dim, pd.p, pd.q)) return IGA_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return IGA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const bool fp64 = P->opts.precision == IGA_FP64 || P->opts.precision == IGA_FP64_DF;
  const size_t esz = fp64 ? sizeof(double) : sizeof(float);
  if (!P->d_apply_scratch) {
    // one value per (element, local function): the size of the dof map
    cudaError_t ae = cudaMalloc(&P->d_apply_scratch, esz * (size_t)P->info.n_dofmap_entries);
    if (ae != cudaSuccess) {
      P->d_apply_scratch = nullptr;
      cudaGetLastError();
      return map_cuda(ae);
    }
  }
  cudaError_t e = launch_basis_tables(P->d_jobs, P->n_jobs, P->d_knots, P->d_gauss,
                                      P->d_tables, st);
  for (int ip = 0; ip < P->n_patches && e == cudaSuccess; ++ip) {
    const PatchDev& pd = P->ph[ip];
    ApplyArgs a{};
    a.n_elem = (int64_t)pd.K[0] * pd.K[1] * pd.K[2];
    a.K1 = pd.K[0]; a.K2 = pd.K[1]; a.K3 = pd.K[2];
    for (int k = 0; k < 3; ++k) {
      a.tab[k] = P->d_tables + pd.tab_offset[k];
      a.span[k] = P->d_spans + pd.span_offset[k];
    }
    a.nf0 = pd.nf[0]; a.nf1 = pd.nf[1];
    a.dof_offset = pd.dof_offset;
    a.kappa = kappa ? kappa + pd.qp_offset : nullptr;
    a.rho = rho ? rho + pd.qp_offset : nullptr;
    a.jac = jac ? jac + pd.qp_offset * pd.dim * pd.dim : nullptr;
    a.x = x;
    a.alpha = alpha; a.beta = beta;
    a.scratch = (char*)P->d_apply_scratch + esz * pd.dofmap_offset;
    e = launch_apply(a, pd.dim, pd.p, pd.q, fp64, P->opts.precision == IGA_FP64_DF, st);
    if (e == cudaSuccess)
      e = launch_apply_gather(P->csr[ip], P->d_fc, P->d_spans, a.scratch, y, fp64, st);
  }
  return finish(P, st, e);
}

namespace {
// Build the weighted-quadrature tables of every patch (host) and upload them.
int wq_ensure(iga_plan_s* P) {
  if (P->wq_status >= 0) return P->wq_status;
  int rc = IGA_OK;
  P->wq.assign((size_t)P->n_patches * 3, iga_plan_s::WqDir{});
  P->wq_coef_off.assign(1, 0);
  for (int ip = 0; ip < P->n_patches && rc == IGA_OK; ++ip) {
    const PatchDev& pd = P->ph[ip];
    if (!pd.iso || pd.p > 5) { rc = IGA_ERR_UNSUPPORTED; break; }
    int64_t grid = 1;
    for (int k = 0; k < 3 && rc == IGA_OK; ++k) {
      iga_plan_s::WqDir& w = P->wq[(size_t)ip * 3 + k];
      if (k >= pd.dim) {
        // the missing direction of a 2D patch: one function, one point, a
        // mass-rule product w B = 1 and a derivative-rule product 0, so the
        // 3D row kernels give the 2D matrices
        const int W = 2 * pd.p + 1;
        w.x.assign(1, 0.0);
        w.qmax = 1;
        std::vector<int> qlo(1, 0), qn(1, 1);
        std::vector<double> V(W, 0.0), V1(W, 0.0);
        V[0] = 1.0;
        cudaError_t e = upload(&w.d_qlo, qlo.data(), qlo.size());
        if (e == cudaSuccess) e = upload(&w.d_qn, qn.data(), qn.size());
        if (e == cudaSuccess) e = upload(&w.d_V, V.data(), V.size());
        if (e == cudaSuccess) e = upload(&w.d_V1, V1.data(), V1.size());
        if (e != cudaSuccess) { cudaGetLastError(); rc = map_cuda(e); }
        continue;
      }
      const CsrPatch& c = P->csr[ip];
      // the coupling records of this direction (the planner's host copy)
      std::vector<FnCouple> all(P->fc_host.begin() + c.fn_offset[k],
                                P->fc_host.begin() + c.fn_offset[k] + pd.nf[k]);
      std::vector<int> qlo, qn;
      std::vector<double> V, V1;
      const double* t = P->knots_host.data() + pd.knot_offset[k];
      rc = wq_build_direction(t, pd.p, P->spans_h[(size_t)ip * P->dim + k], all, &w.x, &qlo, &qn, &V,
                              pd.p >= 2 ? &V1 : nullptr, &w.qmax);
      if (rc != IGA_OK) break;
      cudaError_t e = upload(&w.d_qlo, qlo.data(), qlo.size());
      if (e == cudaSuccess) e = upload(&w.d_qn, qn.data(), qn.size());
      if (e == cudaSuccess) e = upload(&w.d_V, V.data(), V.size());
      if (e == cudaSuccess && pd.p >= 2) e = upload(&w.d_V1, V1.data(), V1.size());
      if (e != cudaSuccess) { cudaGetLastError(); rc = map_cuda(e); }
      grid *= (int64_t)w.x.size();
    }
    P->wq_coef_off.push_back(P->wq_coef_off.back() + grid);
  }
  P->wq_status = rc;
  return rc;
}
}  // namespace

extern "C" int iga_wq_points(iga_plan_t P, int patch, int dir, double* x_out, int64_t* n_out) {
  if (!P || !n_out || patch < -1 || patch >= P->n_patches || dir < -1 || dir > 2) return IGA_ERR_ARG;
  if (P->sticky != IGA_OK) return P->sticky;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return IGA_ERR_ARG;
  const int rc = wq_ensure(P);
  if (rc != IGA_OK) return rc;
  if (patch == -1) {
    if (dir != -1 || x_out) return IGA_ERR_ARG;
    *n_out = P->wq_coef_off.back();
    return IGA_OK;
  }
  if (dir == -1) {
    if (x_out) return IGA_ERR_ARG;
    *n_out = P->wq_coef_off[patch + 1] - P->wq_coef_off[patch];
    return IGA_OK;
  }
  if (dir >= P->ph[patch].dim) return IGA_ERR_ARG;
  const std::vector<double>& x = P->wq[(size_t)patch * 3 + dir].x;
  *n_out = (int64_t)x.size();
  if (x_out) std::memcpy(x_out, x.data(), sizeof(double) * x.size());
  return IGA_OK;
}

extern "C" int iga_wq_mass(iga_plan_t P, const double* c, double* values, void* cuda_stream) {
  NvtxRange range("iga_wq_mass");
  if (!P || !values) return IGA_ERR_ARG;
  if (P->sticky != IGA_OK) return P->sticky;
  if (P->opts.precision != IGA_FP64 && P->opts.precision != IGA_FP64_DF) return IGA_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return IGA_ERR_ARG;
  const int rc = wq_ensure(P);
  if (rc != IGA_OK) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSuccess;
  for (int ip = 0; ip < P->n_patches && e == cudaSuccess; ++ip) {
    WqPatchArgs a{};
    a.c = P->csr[ip];
    a.fc = P->d_fc;
    for (int k = 0; k < 3; ++k) {
      const iga_plan_s::WqDir& w = P->wq[(size_t)ip * 3 + k];
      a.d[k].qlo = w.d_qlo;
      a.d[k].qn = w.d_qn;
      a.d[k].V = w.d_V;
      a.d[k].V1 = w.d_V1;
      a.d[k].np = (int)w.x.size();
      a.d[k].qmax = w.qmax;
    }
    a.coef = c ? c + P->wq_coef_off[ip] : nullptr;
    a.values = values;
    e = launch_wq_mass(a, P->ph[ip].p, P->opts.precision == IGA_FP64_DF, st);
  }
  return finish(P, st, e);
}

extern "C" int iga_wq_stiffness(iga_plan_t P, const double* c, double* values, void* cuda_stream) {
  NvtxRange range("iga_wq_stiffness");
  if (!P || !values) return IGA_ERR_ARG;
  if (P->sticky != IGA_OK) return P->sticky;
  if (P->opts.precision != IGA_FP64 && P->opts.precision != IGA_FP64_DF) return IGA_ERR_UNSUPPORTED;
  for (const PatchDev& pd : P->ph)
    if (!pd.iso || !wq_stiffness_supported(pd.dim, pd.p)) return IGA_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return IGA_ERR_ARG;
  const int rc = wq_ensure(P);
  if (rc != IGA_OK) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSuccess;
  for (int ip = 0; ip < P->n_patches && e == cudaSuccess; ++ip) {
    WqPatchArgs a{};
    a.c = P->csr[ip];
    a.fc = P->d_fc;
    for (int k = 0; k < 3; ++k) {
      const iga_plan_s::WqDir& w = P->wq[(size_t)ip * 3 + k];
      a.d[k].qlo = w.d_qlo;
      a.d[k].qn = w.d_qn;
      a.d[k].V = w.d_V;
      a.d[k].V1 = w.d_V1;
      a.d[k].np = (int)w.x.size();
      a.d[k].qmax = w.qmax;
    }
    a.coef = c ? c + P->wq_coef_off[ip] : nullptr;
    a.values = values;
    e = launch_wq_stiffness(a, P->ph[ip].p, P->opts.precision == IGA_FP64_DF, st);
    // a patch whose rule tables exceed shared memory (very short knot vectors)
    if (e == cudaErrorInvalidValue) {
      cudaGetLastError();
      return IGA_ERR_UNSUPPORTED;
    }
  }
  return finish(P, st, e);
}

extern "C" int iga_profile_read(iga_plan_t P, double* kernel_ms, int64_t* launches) {
  if (!P || !P->opts.profile) return IGA_ERR_ARG;
  double total = 0.0;
  for (size_t i = 0; i < P->prof_used; ++i) {
    cudaError_t e = cudaEventSynchronize(P->prof_events[i].second);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, P->prof_events[i].first, P->prof_events[i].second);
    if (e != cudaSuccess) return map_cuda(e);
    total += ms;
  }
  if (kernel_ms) *kernel_ms = total;
  if (launches) *launches = P->prof_launches;
  P->prof_used = 0;
  P->prof_launches = 0;
  return IGA_OK;
}

extern "C" int iga_destroy(iga_plan_t P) {
  if (!P) return IGA_OK;
  int rc = P->sticky;
  int h = 0;
  if (P->d_err && cudaMemcpy(&h, P->d_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
      h != 0 && rc == IGA_OK)
    rc = h;
  free_plan_memory(P);
  delete P;
  return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free adjoint for callers that cannot allocate device memory.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNaMaxKnots = 1024;            // knots per direction
constexpr int64_t kNaMaxElements = 262144;   // elements of the patch
constexpr int64_t kNaTableDoubles = 196608;  // basis-table records
// scratch layout, in doubles
constexpr int64_t kNaKnots = 0;                                   // [3][kNaMaxKnots]
constexpr int64_t kNaGauss = kNaKnots + 3 * kNaMaxKnots;          // [2][kMaxGauss]
constexpr int64_t kNaSpans = kNaGauss + 2 * kMaxGauss;            // int [3][kNaMaxKnots]
constexpr int64_t kNaJobs = kNaSpans + 3 * kNaMaxKnots / 2;       // TableJob [3][kNaMaxKnots]
constexpr int64_t kNaTables = kNaJobs + 3 * kNaMaxKnots * (int64_t)sizeof(TableJob) / 8;
constexpr int64_t kNaPartials = kNaTables + kNaTableDoubles;      // [kNaMaxElements]
constexpr int64_t kNaDoubles = kNaPartials + kNaMaxElements;      // 3.7 MiB in total

// The scratch of iga_adjoint_noalloc: one fixed array per GPU that loads the
// library, kept until the process exits and shared by every call.
static __device__ __align__(256) double g_noalloc_scratch[kNaDoubles];

// Device address of g_noalloc_scratch per CUDA context.  The address belongs
// to the context that loaded the module: a cudaDeviceReset, or a context the
// caller created through the driver API, gets a new one.  The cache is keyed by
// the context's process-unique id (cuCtxGetId), which is never reused, so a
// stale address is never handed to a kernel.  The two driver calls are reached
// through cudaGetDriverEntryPointByVersion, so the library does not link libcuda.
typedef int (*PfnCtxGetCurrent)(void** ctx);
typedef int (*PfnCtxGetId)(void* ctx, unsigned long long* id);
std::mutex g_na_mu;
PfnCtxGetCurrent g_ctx_current = nullptr;
PfnCtxGetId g_ctx_id = nullptr;
std::vector<std::pair<unsigned long long, double*>> g_na_ptr;

// Id of the context current on this thread (created by the runtime if none
// is); false if the driver entry points are unavailable.
bool current_context_id(unsigned long long* id) {
  if (!g_ctx_current || !g_ctx_id) {
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0, q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) !=
            cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
      return false;
    g_ctx_current = (PfnCtxGetCurrent)f0;
    g_ctx_id = (PfnCtxGetId)f1;
  }
  void* ctx = nullptr;
  if (g_ctx_current(&ctx) != 0) return false;
  if (!ctx) {
    // no context yet on this thread: cudaSetDevice makes the runtime's
    // primary context of the current device current (CUDA >= 12)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess ||
        g_ctx_current(&ctx) != 0 || !ctx)
      return false;
  }
  return g_ctx_id(ctx, id) == 0;
}

struct NaParams {
  double knots[3][kNaMaxKnots];
  int m[3];
  int p, q;
  double gx[kMaxGauss], gw[kMaxGauss];
};

// Writes the knots, the Gauss rule, the element spans and the table jobs of
// one 3D patch into the scratch (one thread per (direction, element)).
__global__ void k_noalloc_setup(const NaParams P, double* scratch, int K0, int K1, int K2) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double* knots = scratch + kNaKnots;
  double* gauss = scratch + kNaGauss;
  int* spans = (int*)(scratch + kNaSpans);
  TableJob* jobs = (TableJob*)(scratch + kNaJobs);
  for (int i = tid; i < 3 * kNaMaxKnots; i += gridDim.x * blockDim.x) {
    const int d = i / kNaMaxKnots, j = i % kNaMaxKnots;
    knots[i] = j < P.m[d] ? P.knots[d][j] : 0.0;
  }
  for (int i = tid; i < P.q; i += gridDim.x * blockDim.x) {
    gauss[i] = P.gx[i];
    gauss[P.q + i] = P.gw[i];
  }
  const int Ks[3] = {K0, K1, K2};
  const int rec = 2 * P.q * (P.p + 1) + P.q;
  for (int i = tid; i < K0 + K1 + K2; i += gridDim.x * blockDim.x) {
    int d = 0, ek = i;
    while (ek >= Ks[d]) { ek -= Ks[d]; ++d; }
    // the ek-th non-empty span of direction d
    int s = P.p, c = -1;
    for (; s <= P.m[d] - P.p - 2; ++s) {
      if (P.knots[d][s] < P.knots[d][s + 1]) ++c;
      if (c == ek) break;
    }
    spans[d * kNaMaxKnots + ek] = s;
    TableJob j;
    j.knot_off = d * kNaMaxKnots;
    j.span = s;
    j.p = P.p;
    j.q = P.q;
    j.gauss_off = 0;
    int64_t before = 0;
    for (int dd = 0; dd < d; ++dd) before += Ks[dd];
    j.out_off = (before + ek) * rec;
    jobs[i] = j;
  }
}

}  // namespace

extern "C" int iga_adjoint_noalloc(const iga_patch_desc* patch, const double* kappa,
                                   const double* jac, const double* u, const double* v,
                                   double* grad_kappa, double* J_out, void* cuda_stream) {
  if (!patch || !u || !v || (!grad_kappa && !J_out) || (J_out && !kappa)) return IGA_ERR_ARG;
  const iga_patch_desc& d = *patch;
  if (d.dim != 3) return IGA_ERR_UNSUPPORTED;
  const int p = d.degree[0], q = d.n_gauss[0];
  for (int k = 0; k < 3; ++k)
    if (d.degree[k] < 1 || d.degree[k] > kMaxDegree || d.n_gauss[k] < 1 || d.n_gauss[k] > kMaxGauss)
      return IGA_ERR_ARG;
  for (int k = 1; k < 3; ++k)
    if (d.degree[k] != p || d.n_gauss[k] != q) return IGA_ERR_UNSUPPORTED;
  int K[3], nf[3];
  int64_t E = 1, tab = 0;
  for (int k = 0; k < 3; ++k) {
    const int rc = validate_knots(d.knots[k], d.n_knots[k], p);
    if (rc != IGA_OK) return rc;
    if (d.n_knots[k] > kNaMaxKnots) return IGA_ERR_TOO_LARGE;
    K[k] = (int)knot_spans(d.knots[k], d.n_knots[k], p).size();
    nf[k] = d.n_knots[k] - p - 1;
    E *= K[k];
    tab += (int64_t)K[k] * record_size(p + 1, q);
  }
  if (E > kNaMaxElements || tab > kNaTableDoubles) return IGA_ERR_TOO_LARGE;

  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    unsigned long long id = 0;
    if (!current_context_id(&id)) return IGA_ERR_CUDA;
    for (const auto& kv : g_na_ptr)
      if (kv.first == id) scratch = kv.second;
    if (!scratch) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) return IGA_ERR_CUDA;
      scratch = (double*)ptr;
      g_na_ptr.push_back({id, scratch});
    }
  }
  NaParams P;
  for (int k = 0; k < 3; ++k) {
    P.m[k] = d.n_knots[k];
    for (int j = 0; j < kNaMaxKnots; ++j) P.knots[k][j] = j < d.n_knots[k] ? d.knots[k][j] : 0.0;
  }
  P.p = p;
  P.q = q;
  gauss_legendre_newton(q, P.gx, P.gw);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_noalloc_setup<<<8, 256, 0, st>>>(P, scratch, K[0], K[1], K[2]);
  cudaError_t e = cudaGetLastError();
  const int n_jobs = K[0] + K[1] + K[2];
  double* tables = scratch + kNaTables;
  if (e == cudaSuccess)
    e = launch_basis_tables((const TableJob*)(scratch + kNaJobs), n_jobs, scratch + kNaKnots,
                            scratch + kNaGauss, tables, st);
  if (e == cudaSuccess) {
    AdjArgs a{};
    a.n_elem = E;
    a.K1 = K[0]; a.K2 = K[1]; a.K3 = K[2];
    const int rec = record_size(p + 1, q);
    a.tab[0] = tables;
    a.tab[1] = tables + (int64_t)K[0] * rec;
    a.tab[2] = tables + (int64_t)(K[0] + K[1]) * rec;
    const int* spans = (const int*)(scratch + kNaSpans);
    for (int k = 0; k < 3; ++k) a.span[k] = spans + k * kNaMaxKnots;
    a.nf0 = nf[0]; a.nf1 = nf[1];
    a.dof_offset = 0;
    a.kappa = kappa;
    a.jac = jac;
    a.u = u; a.v = v;
    a.grad = grad_kappa;
    a.partial = J_out ? scratch + kNaPartials : nullptr;
    a.partial_offset = 0;
    if (adjoint_supported(3, p, q)) {
      e = launch_adjoint(a, 3, p, q, true, false, st);
    } else {
      PatchDev ph{};
      ph.dim = 3;
      ph.p = p; ph.q = q; ph.n = p + 1;
      for (int k = 0; k < 3; ++k) { ph.pk[k] = p; ph.qk[k] = q; ph.nk[k] = p + 1; }
      e = launch_adjoint_gen(a, ph, st);
    }
  }
  if (e == cudaSuccess && J_out) e = launch_reduce_fixed(scratch + kNaPartials, E, J_out, st);
  if (e != cudaSuccess) return map_cuda(e);
  return IGA_OK;
}
