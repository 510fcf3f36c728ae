// Generic per-cell chemistry kernels for sm_103a: plain (one pass, one cell per
// thread) and queue (persistent CTAs, substep-granular refill from a device work
// queue), compiled for 2, 3 and 9 species and for both integrators (RODAS3 and
// ROS2); the body is in chem_kernel_body.cuh.
#include <cuda_runtime.h>

#include "chem_kernel_body.cuh"

namespace rde {

namespace {

template <int K, bool QUEUE, int METHOD>
__global__ void __launch_bounds__(kThreads, 1) chem_advance_kernel(const LaunchArgs a) {
  advance_body<K, QUEUE, GenericRhs, METHOD>(a);
}

template <int K>
size_t smem_bytes(int mech_bytes, int n_blocks) {
  return (size_t)mech_bytes + Slots<K>::bytes(kThreads) + (n_blocks > 0 ? sizeof(long long) * (n_blocks + 1) : 0);
}

template <int K, bool QUEUE, int METHOD>
cudaError_t set_smem(size_t smax) {
  return cudaFuncSetAttribute(chem_advance_kernel<K, QUEUE, METHOD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smax);
}

template <int K>
cudaError_t prepare_k(int mech_bytes, int* fit) {
  const size_t smax = smem_bytes<K>(mech_bytes, kMaxBlocks);
  cudaError_t e = set_smem<K, true, kMethodRodas3>(smax);
  if (e == cudaSuccess) e = set_smem<K, false, kMethodRodas3>(smax);
  if (e == cudaSuccess) e = set_smem<K, true, kMethodRos2>(smax);
  if (e == cudaSuccess) e = set_smem<K, false, kMethodRos2>(smax);
  if (e == cudaSuccess) e = set_smem<K, true, kMethodExtrap>(smax);
  // one resident CTA per SM for every instance (launch bounds and shared memory);
  // the fit of the RODAS3 queue kernel sizes the persistent grid of both methods
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(fit, chem_advance_kernel<K, true, kMethodRodas3>, kThreads,
                                                      smax);
  if (e == cudaSuccess && *fit < 1) e = cudaErrorInvalidConfiguration;
  return e;
}

template <int K, bool QUEUE, int METHOD>
cudaError_t launch_one(const LaunchArgs& a, cudaStream_t stream) {
  const size_t smem = smem_bytes<K>(a.mech_bytes, a.blocks ? a.n_blocks : 0);
  const long long blocks_needed = (a.n_total + kThreads - 1) / kThreads;
  long long grid = blocks_needed;
  if (QUEUE) {
    const int fit = a.fit > 0 ? a.fit : 1;
    const int per_sm = a.ctas_per_sm > 0 ? min(a.ctas_per_sm, fit) : fit;
    grid = min(blocks_needed, (long long)a.num_sms * per_sm);
  }
  if (grid < 1) grid = 1;
  chem_advance_kernel<K, QUEUE, METHOD><<<(unsigned)grid, kThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_k(const LaunchArgs& a, cudaStream_t stream) {
  const bool plain = a.schedule == RDE_SCHED_PLAIN;
  if (a.opt.method == RDE_METHOD_ROS2)
    return plain ? launch_one<K, false, kMethodRos2>(a, stream) : launch_one<K, true, kMethodRos2>(a, stream);
  if (a.opt.method == RDE_METHOD_EXTRAP)   // queue schedule only: the Jacobian scratch is per resident lane
    return plain ? cudaErrorInvalidValue : launch_one<K, true, kMethodExtrap>(a, stream);
  return plain ? launch_one<K, false, kMethodRodas3>(a, stream) : launch_one<K, true, kMethodRodas3>(a, stream);
}

}  // namespace

bool kernel_supports(int K) { return K == 2 || K == 3 || K == 9; }

int kernel_threads() { return kThreads; }

size_t kernel_shared_bytes(int K, int mech_bytes) {
  switch (K) {
    case 2: return smem_bytes<2>(mech_bytes, 0);
    case 3: return smem_bytes<3>(mech_bytes, 0);
    case 9: return smem_bytes<9>(mech_bytes, 0);
    default: return 0;
  }
}

cudaError_t prepare_advance(int K, int mech_bytes, int* fit) {
  switch (K) {
    case 2: return prepare_k<2>(mech_bytes, fit);
    case 3: return prepare_k<3>(mech_bytes, fit);
    case 9: return prepare_k<9>(mech_bytes, fit);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_advance(const LaunchArgs& a, cudaStream_t stream) {
  if (a.blocks && a.n_blocks > kMaxBlocks) return cudaErrorInvalidValue;
  switch (a.K) {
    case 2: return launch_k<2>(a, stream);
    case 3: return launch_k<3>(a, stream);
    case 9: return launch_k<9>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rde

// ---- test hook: the library's exp / log on device arrays ----
namespace rde {
namespace {
__global__ void selftest_math_kernel(int fn, long long n, const double* x, double* y, const double* tabs) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = fn == 0 ? exp_tab(x[i], tabs) : log_tab(x[i], tabs + kExpTabSize);
}
}  // namespace

cudaError_t launch_selftest_math(int fn, long long n, const double* x, double* y, const double* tabs,
                                 cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  selftest_math_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(fn, n, x, y, tabs);
  return cudaGetLastError();
}
}  // namespace rde
