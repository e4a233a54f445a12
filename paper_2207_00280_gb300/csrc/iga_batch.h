// iga_batch.h -- plan state of the batched (persistent / CUDA-graph) schedules.
#pragma once

#include <string>
#include <vector>

#include "iga_internal.h"

namespace iga {

struct BatchClass {
  int p, q;
  int64_t elements;
  int64_t item_offset[4];   // one item list per work-item size candidate
  int n_items[4];
  int epi;                  // chosen elements per work item
  int sched;                // chosen schedule (kSched*)
  bool tuned;
  bool split;               // stiffness and mass in separate launches
};

// Launches that precede the element kernels (basis tables, dof map).
struct BatchPrologue {
  cudaError_t (*run)(void* ctx, cudaStream_t s);
  void* ctx;
  const void* dof_out;
};

struct BatchState {
  bool bf16 = false;
  bool tuning = false;      // inside the autotuner: a variant that does not fit is skipped
  int schedule = IGA_SCHED_AUTO;
  unsigned long long budget_ns = 0;
  std::vector<BatchClass> classes;
  WorkItem* d_items = nullptr;
  int* d_counters = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t fork = nullptr, cap_done = nullptr;
  cudaGraphExec_t exec = nullptr;
  int key_mode = -1;
  const void *key_kappa = nullptr, *key_rho = nullptr, *key_jac = nullptr, *key_K = nullptr,
             *key_M = nullptr, *key_dof = nullptr;
  std::string gen_key;
};

int batch_plan(BatchState* B, const std::vector<PatchDev>& ph, int precision, int schedule);
void batch_free(BatchState* B);
cudaError_t batch_integrate(BatchState* B, const QueueArgs& base, int mode, cudaStream_t st,
                            const BatchPrologue& pro, bool graph);

}  // namespace iga
