// Discrete adjoint of the per-cell chemistry step: generic kernels (2, 3 and 9
// species) and their launch; the device code is in chem_adjoint_body.cuh.
#include <cuda_runtime.h>
#include <stdint.h>

#include "chem_adjoint_body.cuh"

namespace rde {

// the CTA-per-cell adjoint kernel (chem_large_adjoint.cu)
cudaError_t launch_large_adjoint_kernel(const AdjArgs& a, cudaStream_t stream);

namespace {

template <int K>
__global__ void __launch_bounds__(kThreadsA, 1) record_kernel(const AdjArgs a) {
  record_body<K, GenericReactions>(a);
}

template <int K, bool SELF>
__global__ void __launch_bounds__(kThreadsA, 1) reverse_kernel(const AdjArgs a) {
  reverse_body<K, GenericReactions, 1, SELF>(a);   // one dual evaluation per stage
}

// ---------------------------------------------------------------------------
// exclusive scan of the step counts (one CTA) and the parameter reduction
// ---------------------------------------------------------------------------
__global__ void scan_kernel(const int* counts, long long n, long long* offsets) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const long long chunk = (n + blockDim.x - 1) / blockDim.x;
  const long long lo = min(n, t * chunk), hi = min(n, lo + chunk);
  long long sum = 0;
  for (long long i = lo; i < hi; ++i) sum += max(counts[i], 0);
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    long long acc = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      const long long v = part[i];
      part[i] = acc;
      acc += v;
    }
    offsets[n] = acc;
  }
  __syncthreads();
  long long acc = part[t];
  for (long long i = lo; i < hi; ++i) {
    offsets[i] = acc;
    acc += max(counts[i], 0);
  }
}

// order[0..n) = the cells by accepted-step count, most first (one CTA): cells whose
// counts share a power of two form one bucket, buckets in descending order, cells in
// a bucket in any order (the per-cell results do not depend on it).  The queues of the
// record and reverse passes hand cells out in this order, so the last cells a lane
// takes are short ones.
__global__ void order_kernel(const int* counts, long long n, long long* order) {
  __shared__ unsigned long long cnt[33], start[33];
  const int t = threadIdx.x;
  if (t < 33) cnt[t] = 0ull;
  __syncthreads();
  auto bucket = [](int c) { return c <= 0 ? 0 : 32 - __clz(c); };   // 0 .. 32
  for (long long i = t; i < n; i += blockDim.x) atomicAdd(&cnt[bucket(counts[i])], 1ull);
  __syncthreads();
  if (t == 0) {
    unsigned long long acc = 0;
    for (int b = 32; b >= 0; --b) {
      start[b] = acc;
      acc += cnt[b];
    }
  }
  __syncthreads();
  for (long long i = t; i < n; i += blockDim.x) {
    const unsigned long long pos = atomicAdd(&start[bucket(counts[i])], 1ull);
    order[pos] = i;
  }
}

// out[j] = sum_i rows[j*n + i], in a fixed order (one CTA per j)
__global__ void reduce_rows_kernel(const double* rows, long long n, double* outA, double* outE, int R) {
  __shared__ double part[256];
  const int j = blockIdx.x;
  const double* row = rows + (long long)j * n;
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += row[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (j < R) outA[j] = part[0];
    else outE[j - R] = part[0];
  }
}

// scan, record and reverse with the given kernels and their CTAs per SM.  In the
// self-checkpointing mode (a.ckpt_S > 0) the record pass finds each cell's step count
// itself, in index order, and the cost order is taken from its counts before the reverse
// sweep.
cudaError_t adjoint_run(const AdjArgs& a0, const void* rec, const void* rev, int fit_rec, size_t smem_rec,
                        size_t smem_rev, cudaStream_t stream) {
  AdjArgs a = a0;
  if (fit_rec < 1) return cudaErrorInvalidConfiguration;
  const long long need = (a.n + kThreadsA - 1) / kThreadsA;
  const long long g_rec = max(1LL, min(need, (long long)a.num_sms * fit_rec));
  // the reverse kernel's per-lane scratch is sized for one CTA per SM (adjoint_lanes)
  const long long g_rev = max(1LL, min(need, (long long)a.num_sms));
  cudaError_t e;
  if (a.ckpt_S > 0) {
    AdjArgs r = a;
    r.order = nullptr;
    void* prec[] = {&r};
    e = cudaLaunchKernel(rec, dim3((unsigned)g_rec), dim3(kThreadsA), prec, smem_rec, stream);
    if (e != cudaSuccess) return e;
    order_kernel<<<1, 1024, 0, stream>>>(a.rec, a.n, const_cast<long long*>(a.order));
  } else {
    scan_kernel<<<1, 1024, 0, stream>>>(a.n_steps, a.n, a.offsets);
    order_kernel<<<1, 1024, 0, stream>>>(a.n_steps, a.n, const_cast<long long*>(a.order));
    void* params[] = {&a};
    e = cudaLaunchKernel(rec, dim3((unsigned)g_rec), dim3(kThreadsA), params, smem_rec, stream);
    if (e != cudaSuccess) return e;
  }
  void* params[] = {&a};
  e = cudaLaunchKernel(rev, dim3((unsigned)g_rev), dim3(kThreadsA), params, smem_rev, stream);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int K>
cudaError_t adjoint_k(const AdjArgs& a, cudaStream_t stream) {
  const size_t smem_rec = (size_t)a.mech_bytes + Slots<K>::bytes(kThreadsA);
  const size_t smem_rev = (size_t)a.mech_bytes + AdjSlots<K>::bytes(kThreadsA);
  const bool self = a.ckpt_S > 0;
  const void* rev = self ? reinterpret_cast<const void*>(reverse_kernel<K, true>)
                         : reinterpret_cast<const void*>(reverse_kernel<K, false>);
  cudaError_t e = cudaFuncSetAttribute(record_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rec);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(rev, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rev);
  if (e != cudaSuccess) return e;
  int fit_rec = 0, fit_rev = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit_rec, record_kernel<K>, kThreadsA, smem_rec);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit_rev, rev, kThreadsA, smem_rev);
  if (e != cudaSuccess) return e;
  if (fit_rev < 1) return cudaErrorInvalidConfiguration;
  return adjoint_run(a, reinterpret_cast<const void*>(record_kernel<K>), rev, fit_rec, smem_rec, smem_rev, stream);
}

}  // namespace

long long adjoint_lanes(int num_sms) { return (long long)num_sms * kThreadsA * 1; }

cudaError_t launch_adjoint(const AdjointLaunch& L, cudaStream_t stream) {
  AdjArgs a;
  a.mech = L.mech;
  a.plan = L.plan;
  a.mech_bytes = L.mech_bytes;
  a.K = L.K;
  a.R = L.R;
  a.n = L.n;
  a.p = L.p;
  a.T0 = L.T0;
  a.Y0 = L.Y0;
  a.ldY = L.ldY;
  a.dt = L.dt;
  a.opt = L.opt;
  a.n_steps = L.n_steps;
  a.order = L.order;
  a.offsets = L.offsets;
  a.pool = L.pool;
  a.stages = L.stages;
  a.total_steps = L.total_steps;
  a.rec = L.rec;
  a.gT = L.gT;
  a.gY = L.gY;
  a.gT0 = L.gT0;
  a.gY0 = L.gY0;
  a.lane_scratch = L.lane_scratch;
  a.rows = L.rows;
  a.queue = L.queue;
  a.status = L.status;
  a.num_sms = L.num_sms;
  a.ckpt_S = L.ckpt_S;
  a.seg_max = L.seg_max;
  a.ckpt = L.ckpt;
  a.seg = L.seg;
  a.replay = L.replay;
  const bool self = L.ckpt_S > 0;
  cudaError_t e;
  if (L.large) {
    if (self) {
      a.order = nullptr;   // the counts are not known before the cells are integrated
    } else {
      scan_kernel<<<1, 1024, 0, stream>>>(a.n_steps, a.n, a.offsets);
      order_kernel<<<1, 1024, 0, stream>>>(a.n_steps, a.n, const_cast<long long*>(a.order));
    }
    e = launch_large_adjoint_kernel(a, stream);
  } else if (L.jit_record && (self ? L.jit_reverse_self != nullptr : L.jit_reverse != nullptr)) {
    const size_t N = (size_t)L.K + 1;
    const size_t smem_rec = (size_t)L.mech_bytes + sizeof(double) * (N * N + 6 * (size_t)L.K + 2 * N) * kThreadsA;   // Slots<K>
    const size_t head = N * N + 9 * (size_t)L.K, dual = 18 * (size_t)L.K;
    const size_t smem_rev = (size_t)L.mech_bytes + sizeof(double) * ((head > dual ? head : dual) + 2 * N) * kThreadsA;
    e = adjoint_run(a, L.jit_record, self ? L.jit_reverse_self : L.jit_reverse, L.jit_fit_record, smem_rec, smem_rev,
                    stream);
  } else {
    switch (L.K) {
      case 2: e = adjoint_k<2>(a, stream); break;
      case 3: e = adjoint_k<3>(a, stream); break;
      case 9: e = adjoint_k<9>(a, stream); break;
      default: return cudaErrorInvalidValue;
    }
  }
  if (e != cudaSuccess) return e;
  reduce_rows_kernel<<<2 * L.R, 256, 0, stream>>>(L.rows, L.n, L.g_lnA, L.g_E, L.R);
  return cudaGetLastError();
}

}  // namespace rde
