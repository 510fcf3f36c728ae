// Host-side launch interface of the chemistry kernels (internal to the library).
#pragma once
#if !defined(__CUDACC_RTC__)  /* run-time compilation: device code only */
#include <cuda_runtime.h>
#include <stdint.h>
#endif

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
  int fit;                        // CTAs per SM that fit (from prepare_advance)
  double* jscratch;               // extrapolation method: [N^2][lanes] Jacobian scratch, else null
  int jscratch_ctas;              // CTAs (of 128 lanes) the scratch holds
  double* park;                   // wide kernels: [4 N][lanes] state and stage vectors, else null
  long long park_lanes;           // lanes the park area holds
  // CTA-per-cell kernel only
  const unsigned char* plan;      // device gather plan (large_plan.h)
  int R;                          // reactions
  int large_fit;                  // CTAs per SM that fit (from prepare_large)
};

#if !defined(__CUDACC_RTC__)
// true if a kernel is compiled for K species
bool kernel_supports(int K);

// Once per mechanism, outside any stream capture: raise the kernels' dynamic
// shared-memory limit for this mechanism and report how many queue CTAs fit per SM.
cudaError_t prepare_advance(int K, int mech_bytes, int* fit);

// Threads per CTA and dynamic shared bytes per CTA (no block table) for K species.
int kernel_threads();
size_t kernel_shared_bytes(int K, int mech_bytes);

// Launches on `stream` (stream work only: capture-safe); returns the launch error.
cudaError_t launch_advance(const LaunchArgs& a, cudaStream_t stream);

// ---- CTA-per-cell kernel (any species count; chem_large.cu) ----
// Dynamic shared bytes per CTA (n_blocks = 0: no block table).
size_t large_shared_bytes(int K, int R, int n_blocks);
// Once per mechanism, outside any stream capture; fails if a cell's arrays exceed shared memory.
cudaError_t prepare_large(int K, int R, int* fit);
// Launches on `stream` (capture-safe); PLAIN: one CTA per cell, otherwise persistent CTAs on the queue.
cudaError_t launch_large(const LaunchArgs& a, cudaStream_t stream);
int large_threads();

// ---- batched small LU, DMMA or DFMA trailing update (lu_compare.cu) ----
int lu_compare_max_order();
cudaError_t launch_batched_lu(int dmma, long long batch, int n, double* A, int32_t* piv, int32_t* info,
                              cudaStream_t stream);

// Test hook: y = exp(x) (fn 0) or log(x) (fn 1) with the library's table-driven
// functions; tabs = exp table (1024) followed by the log table (256), device memory.
cudaError_t launch_selftest_math(int fn, long long n, const double* x, double* y, const double* tabs,
                                 cudaStream_t stream);

#endif  // !__CUDACC_RTC__

// ---- discrete adjoint ----
struct AdjointLaunch {
  const unsigned char* mech;
  const unsigned char* plan;   // gather plan (CTA-per-cell adjoint)
  bool large;                  // the CTA-per-cell adjoint (any K up to 63) instead of thread per cell
  int mech_bytes, K, R;
  long long n;
  const double *p, *T0, *Y0;
  long long ldY;
  double dt;
  rde_chem_options opt;
  const int* n_steps;
  long long total_steps;   // records the pool (and stages) hold
  long long* offsets;
  long long* order;        // [n] workspace: the cells by accepted steps, most first
  double* pool;
  double* stages;   // stage checkpoints ([sum n_steps][adjoint_stage_doubles(K)]) or null: recompute
  int* rec;
  const double *gT, *gY;
  double *gT0, *gY0, *g_lnA, *g_E;
  double* lane_scratch;
  double* rows;
  unsigned long long* queue;
  int* status;
  int num_sms;
  // kernels specialised to the mechanism (cudaKernel_t as pointers) or null for the generic ones
  const void* jit_record;
  const void* jit_reverse;
  const void* jit_reverse_self;
  int jit_fit_record;
  // self-checkpointing mode (n_steps == null): checkpoints per cell (or per CTA for the
  // CTA-per-cell adjoint), the largest stride, and the workspace regions
  int ckpt_S;
  int seg_max;
  double* ckpt;
  double* seg;
  double* replay;
};

#if !defined(__CUDACC_RTC__)
// persistent lanes of the reverse kernel (size of its per-lane scratch)
long long adjoint_lanes(int num_sms);

// Checkpoint entries per cell of the self-checkpointing adjoint: a power of two in
// [kCkptMin, kCkptMax]; the workspace query sizes for kCkptDefault.
constexpr int kCkptMin = 16, kCkptDefault = 512, kCkptMax = 1024;
// Largest checkpoint stride the options allow: a cell takes at most max_substeps steps.
inline int ckpt_seg_max(int max_substeps, int S) {
  int s = 1;
  while ((long long)S * s < (long long)max_substeps) s <<= 1;
  return s;
}

// doubles of one accepted step's stage checkpoint: the LU factors of
// I/(gamma h) - J (1/U_kk on the diagonal), the pivot word and u_1 .. u_4
inline long long adjoint_stage_doubles(int K) { return (long long)(K + 1) * (K + 1) + 4LL * (K + 1) + 1; }

// scan, record, reverse and reduce kernels on `stream`
cudaError_t launch_adjoint(const AdjointLaunch& a, cudaStream_t stream);

// CTA-per-cell adjoint: shared memory of its kernel and its per-device set-up
size_t large_adjoint_shared_bytes(int K, int R);
cudaError_t prepare_large_adjoint(int K, int R);
#endif  // !__CUDACC_RTC__

}  // namespace rde
