// Host-side launch interface of the chemistry kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rde_chem.h"

namespace rde {

struct LaunchArgs {
  const unsigned char* mech;      // device image (mech_layout.h), 16-byte aligned
  int mech_bytes;
  int K;
  rde_block cells;                // used when blocks == nullptr
  const rde_block* blocks;        // device table or nullptr
  int n_blocks;
  long long n_total;
  const long long* order;         // device permutation or nullptr
  double dt;
  rde_chem_options opt;
  unsigned long long* queue;      // device counter (reset by the caller)
  long long* stats;               // device [5]: cells, accepted, rejected, failed, max attempts
  int schedule;                   // RDE_SCHED_PLAIN or RDE_SCHED_QUEUE
  int threads;                    // threads per CTA
  int ctas_per_sm;
  int num_sms;
};

// true if a kernel is compiled for K species
bool kernel_supports(int K);

// Launches on `stream`; returns cudaSuccess or the launch error.
cudaError_t launch_advance(const LaunchArgs& a, cudaStream_t stream);

// Test hook: y = exp(x) (fn 0) or log(x) (fn 1) with the library's table-driven
// functions; tabs = exp table (1024) followed by the log table (256), device memory.
cudaError_t launch_selftest_math(int fn, long long n, const double* x, double* y, const double* tabs,
                                 cudaStream_t stream);

}  // namespace rde
