// Per-cell chemistry step for large mechanisms (tens of species): one CTA of 128
// threads cooperates on one cell.
//
// With N = K + 1 ~ 54 unknowns a cell's matrix alone is 23 KB, so the thread-per-
// cell layout of chem_kernels.cu does not fit on chip.  Here the cell's matrix,
// species arrays, stage vectors and per-reaction values live in the CTA's shared
// memory and the 128 threads split every phase: species loops, reactions, the
// analytic Jacobian (each matrix entry gathered from a host-built plan of its
// contributions, in a fixed order, so results are reproducible), the dense LU
// with partial pivoting (block-wide pivot / swap / multiplier / update phases)
// and the error norm; one warp performs the triangular solves.  All threads take
// the same step-size decisions (the controller runs on block-reduced values).
// The arithmetic is that of chem_device.cuh written for a cooperating block.
#include <cuda_runtime.h>
#include <stdint.h>

#include "chem_large_block.cuh"

namespace rde {
namespace {

constexpr int kLargeMaxBlocks = 1024;
constexpr int kLargeCtasPerSm = 3;   // register budget per thread: 65536 / (3 x 128) = 170

__global__ void __launch_bounds__(kLT, kLargeCtasPerSm) chem_large_kernel(const LaunchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const MechHeader* H = reinterpret_cast<const MechHeader*>(a.mech);
  const int K = a.K, N = K + 1, R = H->R, LD = N | 1;
  // only the exp/log tables (random access) are staged; the species records (read by the
  // species loops, 53 threads) and the reaction table (consecutive threads read consecutive
  // reactions: coalesced) are read through L1, which leaves room for three CTAs per SM
  const int tab_bytes = (int)(sizeof(double) * (kExpTabSize + 2 * kLogTabSize));
  {
    const int4* src2 = reinterpret_cast<const int4*>(a.mech + H->tab_offset);
    int4* dst2 = reinterpret_cast<int4*>(smem);
    for (int i = threadIdx.x; i < tab_bytes / 16; i += blockDim.x) dst2[i] = src2[i];
  }
  MechView m;
  m.hdr = H;
  m.sp = reinterpret_cast<const SpecPacked*>(a.mech + sizeof(MechHeader));
  m.rx = reinterpret_cast<const RxnPacked*>(a.mech + sizeof(MechHeader) + sizeof(SpecPacked) * K);
  m.eff = reinterpret_cast<const EffEntry*>(a.mech + sizeof(MechHeader) + sizeof(SpecPacked) * K +
                                            sizeof(RxnPacked) * R);
  m.exptab = reinterpret_cast<const double*>(smem);
  m.logtab = m.exptab + kExpTabSize;
  const PlanView pl = plan_view(a.plan);
  double* d = reinterpret_cast<double*>(smem + tab_bytes);
  Cell c;
  {
    const PlanHeader* PH = reinterpret_cast<const PlanHeader*>(a.plan);
    const double* rx = reinterpret_cast<const double*>(a.plan + PH->o_rx);
    const int st = PH->rx_stride;
    c.rlnA = rx;
    c.rb = rx + st;
    c.rEaR = rx + 2 * st;
    c.rdnu = rx + 3 * st;
    c.rmeta = reinterpret_cast<const int4*>(rx + 4 * st);
  }
  c.N = N;
  c.LD = LD;
  c.K = K;
  c.R = R;
  c.MX = d;
  d += N * LD;
  c.C = d; d += K;
  c.G = d; d += K;
  c.HRT = d; d += K;
  c.CPR = d; d += K;
  c.WDOT = d; d += K;
  c.WT = d; d += K;
  c.BK = d; d += K;
  c.Yv = d; d += N;
  c.ARG = d; d += N;
  c.VEC = d; d += N;
  c.F0 = d; d += N;
  c.U1 = d; d += N;
  c.U2 = d; d += N;
  c.U3 = d; d += N;
  c.U4 = d; d += N;
  c.INVD = d; d += N;
  c.RS = d; d += 9 * R;
  c.red = d; d += 8;
  long long* cellidx = reinterpret_cast<long long*>(c.red + 6);   // red[0..3] serve block_sum
  long long* offs = reinterpret_cast<long long*>(d);               // block table prefix sums
  if (a.blocks) d += a.n_blocks + 1;
  c.perm = reinterpret_cast<int*>(d);
  c.ired = c.perm + N;
  if (a.blocks && threadIdx.x == 0) {
    long long acc = 0;
    for (int b = 0; b < a.n_blocks; ++b) {
      offs[b] = acc;
      const long long nb = (long long)a.blocks[b].n;
      acc += nb > 0 ? nb : 0;   // a block with n < 0 is empty
    }
    offs[a.n_blocks] = acc;
  }
  __syncthreads();
  // with a block table, never hand out positions beyond the cells the table holds
  const long long n_total = a.blocks ? min(a.n_total, offs[a.n_blocks]) : a.n_total;
  const int tid = threadIdx.x;
  const Opts o{a.opt.rtol, a.opt.atol, a.opt.h_min, a.opt.facmax, a.opt.facmin, a.opt.safety, a.opt.max_substeps, 0};
  const double dt = a.dt;
  const bool queue = (a.schedule != RDE_SCHED_PLAIN);
  long long st_cells = 0, st_acc = 0, st_rej = 0, st_fail = 0, st_max = 0;
  bool plain_taken = false;
  for (;;) {
    // ---- take a cell ----
    if (tid == 0) {
      long long g;
      if (queue) g = (long long)atomicAdd(a.queue, 1ull);
      else g = plain_taken ? n_total : (long long)blockIdx.x;
      cellidx[0] = g;
    }
    plain_taken = true;
    __syncthreads();
    const long long g = cellidx[0];
    __syncthreads();
    if (g >= n_total) break;
    const long long gc = a.order ? a.order[g] : g;
    if (gc < 0 || gc >= n_total) continue;   // invalid permutation entry: nothing to do
    // single block or block table: resolve (block, i)
    rde_block blk = a.cells;
    long long i = gc;
    if (a.blocks) {
      int lo = 0, hi = a.n_blocks - 1;
      while (lo < hi) {  // last block whose first global index is <= gc
        const int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= gc) lo = mid;
        else hi = mid - 1;
      }
      blk = a.blocks[lo];
      i = gc - offs[lo];
      if (i >= blk.n) continue;   // unreachable while offsets are monotone; never index past a block
    }
    const long long t_take = clock64();   // the cell's measured cost starts (thread 0's clock)
    const double p = blk.p[i];
    for (int k = tid; k < N; k += kLT) c.Yv[k] = (k < K) ? blk.Y[k * blk.ldY + i] : blk.T[i];
    __syncthreads();
    int good = 1;
    for (int k = tid; k < N; k += kLT) good &= isfinite(c.Yv[k]) ? 1 : 0;
    good = block_and(good, c.ired) && isfinite(p) && p > 0.0 && c.Yv[K] > 0.0;
    const double invp = 1.0 / p;
    double t = 0.0, h = dt;
    if (blk.h_hint) {
      const double hh = blk.h_hint[i];
      if (hh > 0.0) h = fmin(dt, hh);
    }
    int attempts = 0, nacc = 0, nrej = 0, status = RDE_CELL_OK;
    bool reject_prev = false;
    if (!good) status = RDE_CELL_BAD_STATE;
    while (status == RDE_CELL_OK && dt - t > 1e-14 * dt) {
      if (attempts >= o.max_substeps) {
        status = RDE_CELL_MAX_SUBSTEPS;
        break;
      }
      ++attempts;
      h = fmin(h, dt - t);
      double err;
      int fin;
      if (!large_attempt(m, pl, c, invp, h, o, err, fin)) {
        status = RDE_CELL_LU_SINGULAR;
        break;
      }
      if (fin && err <= 1.0) {
        for (int k = tid; k < N; k += kLT) c.Yv[k] = c.U4[k];
        __syncthreads();
        t += h;
        ++nacc;
        h *= fmin(reject_prev ? 1.0 : o.facmax, fmax(o.facmin, o.safety / cbrt(err)));
        reject_prev = false;
      } else {
        ++nrej;
        h *= (fin && isfinite(err)) ? fmax(o.facmin, o.safety / cbrt(err)) : o.facmin;
        reject_prev = true;
        if (h < o.hmin) status = RDE_CELL_H_UNDERFLOW;
      }
    }
    __syncthreads();
    // ---- outputs ----
    if (status != RDE_CELL_BAD_STATE)
      for (int k = tid; k < N; k += kLT) {
        if (k < K) blk.Y[k * blk.ldY + i] = c.Yv[k];
        else blk.T[i] = c.Yv[k];
      }
    if (tid == 0) {
      if (blk.status) blk.status[i] = status;
      if (blk.n_acc) blk.n_acc[i] = nacc;
      if (blk.n_rej) blk.n_rej[i] = nrej;
      if (blk.h_hint && status == RDE_CELL_OK) blk.h_hint[i] = h;
      if (blk.cycles) blk.cycles[i] = clock64() - t_take;
      ++st_cells;
      st_acc += nacc;
      st_rej += nrej;
      st_fail += (status != RDE_CELL_OK);
      st_max = max(st_max, (long long)(nacc + nrej));
    }
    __syncthreads();
  }
  if (tid == 0 && st_cells > 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 0), (unsigned long long)st_cells);
    atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 1), (unsigned long long)st_acc);
    atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 2), (unsigned long long)st_rej);
    atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 3), (unsigned long long)st_fail);
    atomicMax(a.stats + 4, st_max);
  }
}

}  // namespace

size_t large_shared_bytes(int K, int R, int n_blocks) {
  const int N = K + 1, LD = N | 1;
  const size_t tab = sizeof(double) * (kExpTabSize + 2 * kLogTabSize);
  size_t dbl = (size_t)N * LD + 7 * (size_t)K + 9 * (size_t)N + 9 * (size_t)R + 8;
  if (n_blocks > 0) dbl += (size_t)n_blocks + 1;
  const size_t ints = (size_t)N + 8;   // permutation, reduction flags
  return tab + sizeof(double) * dbl + sizeof(int) * ints;
}

cudaError_t prepare_large(int K, int R, int* fit) {
  if (K < 1 || K + 1 > kLargeMaxN) return cudaErrorInvalidConfiguration;   // register solves hold N <= 64
  const size_t smax = large_shared_bytes(K, R, kLargeMaxBlocks);
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (smax > (size_t)optin) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(chem_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(fit, chem_large_kernel, kLT, smax);
  if (e == cudaSuccess && *fit < 1) e = cudaErrorInvalidConfiguration;
  return e;
}

cudaError_t launch_large(const LaunchArgs& a, cudaStream_t stream) {
  if (a.blocks && a.n_blocks > kLargeMaxBlocks) return cudaErrorInvalidValue;
  const size_t smem = large_shared_bytes(a.K, a.R, a.blocks ? a.n_blocks : 0);
  long long grid = a.n_total;
  if (a.schedule != RDE_SCHED_PLAIN) {
    const int fit = a.large_fit > 0 ? a.large_fit : 1;
    const int per_sm = a.ctas_per_sm > 0 ? min(a.ctas_per_sm, fit) : fit;
    grid = min(a.n_total, (long long)a.num_sms * per_sm);
  }
  if (grid < 1) grid = 1;
  if (grid > 0x7fffffffLL) grid = 0x7fffffffLL;
  chem_large_kernel<<<(unsigned)grid, kLT, smem, stream>>>(a);
  return cudaGetLastError();
}

int large_threads() { return kLT; }

}  // namespace rde
