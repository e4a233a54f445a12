// iga_batch.cu -- host side of the batched schedules: degree classes, work
// items, the persistent queue launches, CUDA-graph capture and the autotuner.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "iga_batch.h"

namespace iga {
namespace {

constexpr int kEpiCandidates[] = {1, 2, 4, 8};
constexpr int kNumEpi = 4;

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;  // tuning key -> schedule * 100 + elements per work item
bool g_tune_loaded = false;

int tune_value(int sched, int epi) { return sched * 100 + epi; }

const char* cache_path() {
  const char* p = getenv("IGA_AUTOTUNE_CACHE");
  return (p && p[0]) ? p : nullptr;
}

// The cache file is a flat JSON object {"key": epi, ...}; keys contain no quotes.
void load_cache_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = cache_path();
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  std::string s;
  char buf[4096];
  size_t r;
  while ((r = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, r);
  fclose(f);
  size_t i = 0;
  while ((i = s.find('"', i)) != std::string::npos) {
    size_t j = s.find('"', i + 1);
    if (j == std::string::npos) break;
    std::string key = s.substr(i + 1, j - i - 1);
    size_t c = s.find(':', j);
    if (c == std::string::npos) break;
    int v = atoi(s.c_str() + c + 1);
    if (v > 0) g_tune[key] = v;
    i = c + 1;
  }
}

void save_cache_locked() {
  const char* path = cache_path();
  if (!path) return;
  std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t k = 0;
  for (auto& kv : g_tune)
    fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++k < g_tune.size() ? "," : "");
  fprintf(f, "}\n");
  fclose(f);
  rename(tmp.c_str(), path);
}

std::string device_key() {
  int dev = 0, drv = 0;
  cudaGetDevice(&dev);
  cudaDriverGetVersion(&drv);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  std::string name = prop.name;
  for (auto& c : name)
    if (c == '"' || c == ' ') c = '_';
  return name + "/drv" + std::to_string(drv);
}

int epi_index(int epi) {
  for (int i = 0; i < kNumEpi; ++i)
    if (kEpiCandidates[i] == epi) return i;
  return 0;
}

}  // namespace

int batch_plan(BatchState* B, const std::vector<PatchDev>& ph, int precision, int schedule) {
  B->bf16 = (precision == IGA_BF16);
  B->schedule = schedule;
  const char* bud = getenv("IGA_QUEUE_BUDGET_NS");
  B->budget_ns = bud ? strtoull(bud, nullptr, 10) : 0ull;
  const char* fs = getenv("IGA_BATCH_SCHED");
  const int forced = (fs && fs[0]) ? atoi(fs) : -1;
  const char* corrupt = getenv("IGA_TEST_CORRUPT_QUEUE");
  const bool corrupt_items = corrupt && corrupt[0] == '1';
  // classes keyed by (p, q), patches of a class in decreasing size
  std::map<std::pair<int, int>, std::vector<int>> cls;
  for (int i = 0; i < (int)ph.size(); ++i) cls[{ph[i].p, ph[i].q}].push_back(i);
  std::vector<WorkItem> all;
  for (auto it = cls.rbegin(); it != cls.rend(); ++it) {  // highest degree first
    BatchClass c;
    c.p = it->first.first;
    c.q = it->first.second;
    std::vector<int> pl = it->second;
    std::stable_sort(pl.begin(), pl.end(), [&](int a, int b) {
      return (int64_t)ph[a].K[0] * ph[a].K[1] * ph[a].K[2] > (int64_t)ph[b].K[0] * ph[b].K[1] * ph[b].K[2];
    });
    c.elements = 0;
    for (int pi : pl) c.elements += (int64_t)ph[pi].K[0] * ph[pi].K[1] * ph[pi].K[2];
    for (int ci = 0; ci < kNumEpi; ++ci) {
      const int epi = kEpiCandidates[ci];
      c.item_offset[ci] = (int64_t)all.size();
      for (int pi : pl) {
        const int64_t E = (int64_t)ph[pi].K[0] * ph[pi].K[1] * ph[pi].K[2];
        for (int64_t e0 = 0; e0 < E; e0 += epi) {
          WorkItem w;
          w.patch = pi;
          w.e0 = e0;
          w.count = (int)std::min<int64_t>(epi, E - e0);
          all.push_back(w);
        }
      }
      c.n_items[ci] = (int)((int64_t)all.size() - c.item_offset[ci]);
    }
    c.epi = c.p >= 3 ? 1 : (c.p == 2 ? 2 : 4);  // default until tuned
    c.sched = kSchedCta;
    c.tuned = false;
    c.split = !queue_both_fit(c.p, c.q, B->bf16);
    if (forced >= 0) {
      // a schedule forced by the caller (tests): the classes that have it use
      // it, the others keep the default; no tuning
      const bool has = forced == kSchedCta ||
                       (forced == kSchedWarp && warp_schedule_supported(c.p, c.q)) ||
                       ((forced == kSchedCtaAltForm || forced == kSchedCtaAltSize) &&
                        f32_variant_supported(c.p, c.q, B->bf16, forced));
      if (has) c.sched = forced;
      c.tuned = true;
    }
    B->classes.push_back(c);
  }
  if (corrupt_items)  // host-made fault: the first item of every list names a missing patch
    for (auto& c : B->classes)
      for (int ci = 0; ci < kNumEpi; ++ci)
        if (c.n_items[ci] > 0) all[c.item_offset[ci]].patch = (int)ph.size() + 7;
  const size_t nc = B->classes.size();
  cudaError_t e = cudaMalloc((void**)&B->d_items, sizeof(WorkItem) * std::max<size_t>(all.size(), 1));
  if (e == cudaSuccess && !all.empty())
    e = cudaMemcpy(B->d_items, all.data(), sizeof(WorkItem) * all.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_counters, sizeof(int) * 2 * std::max<size_t>(nc, 1));
  for (size_t i = 0; i < nc && e == cudaSuccess; ++i) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) B->streams.push_back(s);
    cudaEvent_t ev;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) B->join.push_back(ev);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->cap_done, cudaEventDisableTiming);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? IGA_ERR_OOM : IGA_ERR_CUDA;
  B->gen_key = device_key();
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_cache_locked();
  }
  return IGA_OK;
}

void batch_free(BatchState* B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  B->exec = nullptr;
  for (auto s : B->streams) cudaStreamDestroy(s);
  for (auto ev : B->join) cudaEventDestroy(ev);
  B->streams.clear();
  B->join.clear();
  if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->cap_done) cudaEventDestroy(B->cap_done);
  cudaFree(B->d_items);
  cudaFree(B->d_counters);
  B->d_items = nullptr;
  B->d_counters = nullptr;
}

// One queue launch of class c in schedule `sched` (grid <= 0: the resident
// capacity, capped by the items).
static cudaError_t launch_sched(const BatchState* B, const BatchClass& c, const QueueArgs& a,
                                int mode, int sched, cudaStream_t s) {
  int cap = 0;
  cudaError_t e;
  if (sched == kSchedWarp) {
    e = launch_sumfact_warp_queue(a, c.p, c.q, mode, 0, s, &cap);
    if (e != cudaSuccess) return e;
    return launch_sumfact_warp_queue(a, c.p, c.q, mode, std::max(1, std::min(cap, a.n_items)), s,
                                     nullptr);
  }
  if (sched == kSchedCta) {
    e = launch_sumfact_f32_queue(a, c.p, c.q, B->bf16, mode, 0, s, &cap);
    if (e != cudaSuccess) return e;
    return launch_sumfact_f32_queue(a, c.p, c.q, B->bf16, mode, std::max(1, std::min(cap, a.n_items)),
                                    s, nullptr);
  }
  e = launch_sumfact_f32_queue_alt(a, c.p, c.q, B->bf16, mode, sched, 0, s, &cap);
  if (e == cudaErrorNotSupported && !B->tuning) {
    // the variant does not fit this matrix mode: the default form
    return launch_sched(B, c, a, mode, kSchedCta, s);
  }
  if (e != cudaSuccess) return e;
  return launch_sumfact_f32_queue_alt(a, c.p, c.q, B->bf16, mode, sched,
                                      std::max(1, std::min(cap, a.n_items)), s, nullptr);
}

// Launch one class (both matrix modes as needed) on stream s, in its chosen
// schedule or the given one (sched_override >= 0, epi_override > 0).
static cudaError_t launch_class(BatchState* B, size_t ci, const QueueArgs& base, int mode,
                                cudaStream_t s, int epi_override, int sched_override = -1) {
  BatchClass& c = B->classes[ci];
  const int ei = epi_index(epi_override > 0 ? epi_override : c.epi);
  int sched = sched_override >= 0 ? sched_override : c.sched;
  // the 512-thread variant exists for the identity map only
  if (sched == kSchedCtaAltSize && base.jac) sched = kSchedCta;
  QueueArgs a = base;
  a.items = B->d_items + c.item_offset[ei];
  a.n_items = c.n_items[ei];
  a.budget_ns = B->budget_ns;
  // the warp form holds both matrices; the CTA forms split them when they do not fit
  const bool split = c.split && mode == 0 && sched != kSchedWarp;
  const int modes[2] = {split ? 1 : mode, 2};
  const int n_launch = split ? 2 : 1;
  for (int m = 0; m < n_launch; ++m) {
    QueueArgs am = a;
    am.counter = B->d_counters + 2 * ci + m;
    if (modes[m] == 1) am.M_out = nullptr;
    if (modes[m] == 2) am.K_out = nullptr;
    cudaError_t e = launch_sched(B, c, am, modes[m], sched, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static std::string tune_key(const BatchState* B, const BatchClass& c, int mode, bool gen) {
  int64_t bucket = 1;
  while (bucket < c.elements) bucket *= 4;
  return B->gen_key + "/sf3v2/" + (B->bf16 ? "bf16" : "fp32") + "/p" + std::to_string(c.p) + "q" +
         std::to_string(c.q) + "/m" + std::to_string(mode) + (gen ? "/jac" : "/id") + "/E" +
         std::to_string(bucket);
}

// Autotuner: for every untuned class, time every candidate schedule (the
// CTA-per-element kernel, its variants where the class has them, the
// warp-per-element kernel for p <= 2) with every work-item size, each
// candidate alone on stream st with CUDA events: one warm-up launch, then
// three timed launches of which the median counts.  The fastest candidate is
// kept, but a candidate replaces the current best only when it is at least 3%
// faster, so that timing noise does not flip the choice between nearly equal
// candidates.  Results are cached per GPU, driver and class shape (in memory,
// and in the file named by IGA_AUTOTUNE_CACHE if set).
static cudaError_t autotune(BatchState* B, const QueueArgs& base, int mode, cudaStream_t st) {
  const bool gen = base.jac != nullptr;
  B->tuning = true;
  struct Reset { BatchState* b; ~Reset() { b->tuning = false; } } reset{B};
  cudaEvent_t t0, t1;
  cudaError_t e = cudaEventCreate(&t0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&t1);
  if (e != cudaSuccess) { cudaEventDestroy(t0); return e; }
  for (size_t ci = 0; ci < B->classes.size() && e == cudaSuccess; ++ci) {
    BatchClass& c = B->classes[ci];
    if (c.tuned) continue;
    const std::string key = tune_key(B, c, mode, gen);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) {
        c.sched = it->second / 100;
        c.epi = it->second % 100;
        c.tuned = true;
        continue;
      }
    }
    std::vector<int> scheds = {kSchedCta};
    for (int v : {kSchedCtaAltForm, kSchedCtaAltSize})
      if (f32_variant_supported(c.p, c.q, B->bf16, v) && !(v == kSchedCtaAltSize && gen))
        scheds.push_back(v);
    if (warp_schedule_supported(c.p, c.q)) scheds.push_back(kSchedWarp);
    float best = 1e30f;
    int best_epi = c.epi, best_sched = c.sched;
    for (int sched : scheds) {
      for (int k = 0; k < kNumEpi && e == cudaSuccess; ++k) {
        const int epi = kEpiCandidates[k];
        if (k > 0 && c.n_items[k] < 152) break;  // keep every SM busy
        float ts[4];
        bool ok = true;
        for (int rep = 0; rep < 4 && ok; ++rep) {
          e = cudaMemsetAsync(B->d_counters + 2 * ci, 0, 2 * sizeof(int), st);
          if (e == cudaSuccess) e = cudaEventRecord(t0, st);
          if (e == cudaSuccess) {
            const cudaError_t el = launch_class(B, ci, base, mode, st, epi, sched);
            if (el == cudaErrorNotSupported || el == cudaErrorInvalidValue) {
              ok = false;          // this variant does not fit the class: skip it
              cudaGetLastError();
              break;
            }
            e = el;
          }
          if (e == cudaSuccess) e = cudaEventRecord(t1, st);
          if (e == cudaSuccess) e = cudaEventSynchronize(t1);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
          if (e != cudaSuccess) { ok = false; break; }
          ts[rep] = ms;
        }
        if (e != cudaSuccess) break;
        if (!ok) break;
        std::sort(ts + 1, ts + 4);   // ts[0] is the warm-up
        const float med = ts[2];
        if (med < 0.97f * best || best >= 1e29f) {
          best = med;
          best_epi = epi;
          best_sched = sched;
        }
      }
      if (e != cudaSuccess) break;
    }
    if (e != cudaSuccess) break;
    c.epi = best_epi;
    c.sched = best_sched;
    c.tuned = true;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = tune_value(best_sched, best_epi);
    save_cache_locked();
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  return e;
}

cudaError_t batch_integrate(BatchState* B, const QueueArgs& base, int mode, cudaStream_t st,
                            const BatchPrologue& pro, bool graph) {
  cudaError_t e = cudaSuccess;
  if (B->schedule == IGA_SCHED_AUTO) {
    bool need = false;
    for (auto& c : B->classes) need |= !c.tuned;
    if (need) {
      // the autotuner needs the basis tables of this call
      e = pro.run(pro.ctx, st);
      if (e == cudaSuccess) e = autotune(B, base, mode, st);
      if (e != cudaSuccess) return e;
      if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    }
  }
  auto body = [&](cudaStream_t s0) -> cudaError_t {
    cudaError_t r = pro.run(pro.ctx, s0);
    if (r == cudaSuccess)
      r = cudaMemsetAsync(B->d_counters, 0, sizeof(int) * 2 * B->classes.size(), s0);
    if (r != cudaSuccess) return r;
    if (!graph) {
      for (size_t ci = 0; ci < B->classes.size() && r == cudaSuccess; ++ci)
        r = launch_class(B, ci, base, mode, s0, 0);
      return r;
    }
    r = cudaEventRecord(B->fork, s0);
    for (size_t ci = 0; ci < B->classes.size() && r == cudaSuccess; ++ci) {
      r = cudaStreamWaitEvent(B->streams[ci], B->fork, 0);
      if (r == cudaSuccess) r = launch_class(B, ci, base, mode, B->streams[ci], 0);
      if (r == cudaSuccess) r = cudaEventRecord(B->join[ci], B->streams[ci]);
      if (r == cudaSuccess) r = cudaStreamWaitEvent(s0, B->join[ci], 0);
    }
    return r;
  };
  if (!graph) return body(st);
  const bool same = B->exec && B->key_mode == mode && B->key_kappa == base.kappa &&
                    B->key_rho == base.rho && B->key_jac == base.jac && B->key_K == base.K_out &&
                    B->key_M == base.M_out && B->key_dof == pro.dof_out;
  if (!same) {
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    // the capture stream must start after the caller's prior work only at launch
    // time; capture records no dependency on st
    e = cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t eb = body(B->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(B->cap_stream, &g);
    if (eb != cudaSuccess) { if (g) cudaGraphDestroy(g); return eb; }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&B->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { B->exec = nullptr; return e; }
    B->key_mode = mode; B->key_kappa = base.kappa; B->key_rho = base.rho; B->key_jac = base.jac;
    B->key_K = base.K_out; B->key_M = base.M_out; B->key_dof = pro.dof_out;
  }
  return cudaGraphLaunch(B->exec, st);
}

}  // namespace iga
