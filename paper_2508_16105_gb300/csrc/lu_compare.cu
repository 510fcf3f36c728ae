// Batched small dense LU with partial pivoting, two trailing-update paths:
// FP64 tensor cores (DMMA, mma.sync m8n8k4 f64) and CUDA-core DFMA.
//
// The large-mechanism step factorises one 54 x 54 matrix I/(gamma h) - J per
// attempt and cell.  This file measures whether the FP64 tensor-core path helps
// that factorisation on GB300.  Both variants run the same right-looking blocked
// LU (panel width 4, the k of one m8n8k4 MMA): one warp per matrix, the matrix
// padded to 64 x 64 in shared memory; per panel the warp factorises the panel
// with partial pivoting (the first largest |a_ij| wins, as a serial scan picks),
// solves for the U12 block row and updates the trailing block in 8 x 8 tiles.
// Only the tile update differs: one DMMA per tile, or eight DFMA per lane
// producing the same two elements of the tile.  Results are P A = L U with unit
// lower L below the diagonal and U on and above it, as LAPACK's getrf stores them.
#include <cuda_runtime.h>
#include <stdint.h>

namespace rde {

namespace {

constexpr int kNP = 64;            // padded order
constexpr int kLD = 65;            // shared-memory row stride (odd: column walks hit distinct banks)
constexpr int kWarpsPerCta = 2;
constexpr unsigned kFullM = 0xffffffffu;

__device__ __forceinline__ void dmma_8x8x4(double a, double b, double& c0, double& c1) {
  // D = A B + C for an 8x4 A (row), 4x8 B (col); lane l holds A[l/4][l%4], B[l%4][l/4],
  // C/D[l/4][2(l%4)], C/D[l/4][2(l%4)+1]
  double d0, d1;
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%4, %5};\n"
               : "=d"(d0), "=d"(d1)
               : "d"(a), "d"(b), "d"(c0), "d"(c1));
  c0 = d0;
  c1 = d1;
}

template <bool DMMA>
__global__ void __launch_bounds__(32 * kWarpsPerCta) batched_lu_kernel(double* A, int32_t* piv, long long batch, int n,
                                                                         int32_t* info) {
  extern __shared__ double lu_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long b = (long long)blockIdx.x * kWarpsPerCta + warp;
  if (b >= batch) return;   // whole warp; the kernel uses warp-level synchronisation only
  double* M = lu_smem + (size_t)warp * kNP * kLD;
  double* g = A + b * (long long)n * n;
  for (int e = lane; e < kNP * kNP; e += 32) {
    const int i = e >> 6, j = e & 63;
    M[i * kLD + j] = (i < n && j < n) ? g[i * n + j] : 0.0;
  }
  __syncwarp();
  int singular = 0;
  const int gq = lane >> 2, tq = lane & 3;
  for (int p0 = 0; p0 < n; p0 += 4) {
    const int pe = min(p0 + 4, n);
    // 1. panel columns p0..pe-1, rows j..n-1
    for (int j = p0; j < pe; ++j) {
      double best = -1.0;
      int bi = n;
      for (int i = j + lane; i < n; i += 32) {
        const double v = fabs(M[i * kLD + j]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(kFullM, best, off);
        const int oi = __shfl_down_sync(kFullM, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      const int p = __shfl_sync(kFullM, bi < n ? bi : j, 0);
      if (__shfl_sync(kFullM, best, 0) == 0.0 && !singular) singular = j + 1;
      if (lane == 0) piv[b * n + j] = p;
      if (p != j)
        for (int c = lane; c < kNP; c += 32) {
          const double t = M[j * kLD + c];
          M[j * kLD + c] = M[p * kLD + c];
          M[p * kLD + c] = t;
        }
      __syncwarp();
      const double inv = 1.0 / M[j * kLD + j];
      for (int i = j + 1 + lane; i < n; i += 32) {
        const double l = M[i * kLD + j] * inv;
        M[i * kLD + j] = l;
        for (int c = j + 1; c < pe; ++c) M[i * kLD + c] -= l * M[j * kLD + c];
      }
      __syncwarp();
    }
    if (pe >= n) break;
    // 2. U12: rows p0+1..pe-1, columns pe..n-1 (unit lower triangle of the panel)
    for (int c = pe + lane; c < n; c += 32)
      for (int r = p0 + 1; r < pe; ++r) {
        double acc = M[r * kLD + c];
        for (int s = p0; s < r; ++s) acc -= M[r * kLD + s] * M[s * kLD + c];
        M[r * kLD + c] = acc;
      }
    __syncwarp();
    // 3. trailing block A22 -= L21 U12 in 8 x 8 tiles (k = 4; padding rows/columns are zero)
    for (int i0 = pe; i0 < n; i0 += 8)
      for (int j0 = pe; j0 < n; j0 += 8) {
        double* crow = M + (i0 + gq) * kLD + j0 + 2 * tq;
        double c0 = crow[0], c1 = crow[1];
        if (DMMA) {
          dmma_8x8x4(-M[(i0 + gq) * kLD + p0 + tq], M[(p0 + tq) * kLD + j0 + gq], c0, c1);
        } else {
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const double l = M[(i0 + gq) * kLD + p0 + s];
            c0 -= l * M[(p0 + s) * kLD + j0 + 2 * tq];
            c1 -= l * M[(p0 + s) * kLD + j0 + 2 * tq + 1];
          }
        }
        crow[0] = c0;
        crow[1] = c1;
      }
    __syncwarp();
  }
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e - (e / n) * n;
    g[e] = M[i * kLD + j];
  }
  if (lane == 0 && info) info[b] = singular;
}

}  // namespace

int lu_compare_max_order() { return 56; }   // tiles of the trailing block stay inside the 64 x 64 padding

cudaError_t launch_batched_lu(int dmma, long long batch, int n, double* A, int32_t* piv, int32_t* info,
                              cudaStream_t stream) {
  const size_t smem = sizeof(double) * kNP * kLD * kWarpsPerCta;
  const long long grid = (batch + kWarpsPerCta - 1) / kWarpsPerCta;
  if (grid < 1) return cudaSuccess;
  cudaError_t e;
  if (dmma) {
    e = cudaFuncSetAttribute(batched_lu_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      batched_lu_kernel<true><<<(unsigned)grid, 32 * kWarpsPerCta, smem, stream>>>(A, piv, batch, n, info);
  } else {
    e = cudaFuncSetAttribute(batched_lu_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      batched_lu_kernel<false><<<(unsigned)grid, 32 * kWarpsPerCta, smem, stream>>>(A, piv, batch, n, info);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace rde
