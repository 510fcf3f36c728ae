// Body of the thread-per-cell chemistry kernels (plain and queue schedules),
// templated on the f evaluation so that the generic kernels (reactions read from
// the mechanism image) and mechanism-specialised kernels (reactions generated as
// straight-line code at load time) share every other line.
//
// Both schedules run the same per-lane attempt code, so a cell's result does not
// depend on the schedule.  In the queue schedule a lane whose cell finishes takes
// the next queue position at the next substep boundary, so the lanes of a warp
// stay busy while neighbouring cells need 100 or 1000 substeps; this is the
// single-GPU counterpart of the paper's time-weighted load balancing of CPU ranks
// (Section 3.3.1) for cost that is uneven across the front (Section 1).
#pragma once
#include "chem_device.cuh"
#include "chem_launch.h"

namespace rde {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 128;     // threads per CTA (one lane slot each)
constexpr int kMaxBlocks = 1024;  // block-table entries per launch

struct LaneCell {
  const double* p;
  double* T;
  double* Y;
  double* h_hint;
  int32_t* status;
  int32_t* n_acc;
  int32_t* n_rej;
  long long* cycles;
  long long i;
  long long ldY;
  long long t0;   // clock64 when the lane took the cell
};

// Maps queue position g to its cell; returns false (cell skipped) if a caller-supplied
// permutation entry lies outside [0, n_total).
__device__ __forceinline__ bool locate(const LaunchArgs& a, const long long* offs, long long n_total, long long g,
                                       LaneCell& c) {
  if (a.order) {
    g = a.order[g];
    if (g < 0 || g >= n_total) return false;
  }
  rde_block blk;
  long long i = g;
  if (!a.blocks) {
    blk = a.cells;
  } else {
    int lo = 0, hi = a.n_blocks - 1;
    while (lo < hi) {  // last block whose first global index is <= g
      const int mid = (lo + hi + 1) >> 1;
      if (offs[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    blk = a.blocks[lo];
    i = g - offs[lo];
    if (i >= blk.n) return false;   // unreachable while offsets are monotone; never index past a block
  }
  c.p = blk.p;
  c.T = blk.T;
  c.Y = blk.Y;
  c.h_hint = blk.h_hint;
  c.status = blk.status;
  c.n_acc = blk.n_acc;
  c.n_rej = blk.n_rej;
  c.cycles = reinterpret_cast<long long*>(blk.cycles);
  c.i = i;
  c.ldY = blk.ldY;
  c.t0 = clock64();
  return true;
}

template <bool B, class T, class F>
struct PickType {
  using type = T;
};
template <class T, class F>
struct PickType<false, T, F> {
  using type = F;
};

// THREADS = kThreads: every lane slot in shared memory (Lane).  THREADS = 256 (the
// wide queue kernel, mechanism-specialised RODAS3 only): the matrix in shared memory,
// the species and vector slots in registers (RegLane) and the cell state and stage
// vectors in the park area, so that two warps share each SM sub-partition; the same
// operations, agreeing with the 128-thread kernels to rounding.
template <int K, bool QUEUE, class RHS, int METHOD = kMethodRodas3, int THREADS = kThreads>
__device__ __forceinline__ void advance_body(const LaunchArgs& a) {
  using S = Slots<K>;
  constexpr int N = K + 1;
  constexpr bool WIDE = THREADS != kThreads;
  using LaneT = typename PickType<WIDE, RegLane<K, THREADS>, Lane>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  {
    const int4* src = reinterpret_cast<const int4*>(a.mech);
    int4* dst = reinterpret_cast<int4*>(smem);
    for (int i = threadIdx.x; i < a.mech_bytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  double* lanes = reinterpret_cast<double*>(smem + a.mech_bytes);
  long long* offs = reinterpret_cast<long long*>(lanes + (WIDE ? N * N : S::TOTAL) * THREADS);
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
  const MechView m = mech_view(smem);
  LaneT L;
  L.base = lanes + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const double dt = a.dt;
  const Opts o{a.opt.rtol, a.opt.atol, a.opt.h_min, a.opt.facmax, a.opt.facmin, a.opt.safety, a.opt.max_substeps, METHOD};
  // the extrapolation method's per-lane Jacobian scratch (queue schedule: one lane per
  // thread of the persistent grid); a grid the scratch does not cover does no work
  const long long nl = (long long)gridDim.x * blockDim.x;
  double* Jg = a.jscratch ? a.jscratch + (long long)blockIdx.x * blockDim.x + threadIdx.x : nullptr;
  if (METHOD == kMethodExtrap && (!QUEUE || !a.jscratch || (long long)gridDim.x > a.jscratch_ctas)) return;
  // the wide kernels keep the cell state and stage vectors in the park area (queue
  // schedule: one lane per thread of the persistent grid); a grid it does not cover does
  // no work
  static_assert(!WIDE || METHOD == kMethodRodas3, "the wide kernels integrate with RODAS3");
  if (WIDE && (!QUEUE || !a.park || (long long)gridDim.x * THREADS > a.park_lanes)) return;
  const Park P{WIDE ? a.park + (long long)blockIdx.x * THREADS + threadIdx.x : nullptr,
               (long long)gridDim.x * THREADS};

  // lane state
  bool active = false, exhausted = false, plain_taken = false;
  LaneCell cell{};
  double y[N];
  double invp = 0.0, t = 0.0, h = 0.0;
  int attempts = 0, nacc = 0, nrej = 0;
  bool reject_prev = false;
  long long st_cells = 0, st_acc = 0, st_rej = 0, st_fail = 0, st_max = 0;

  auto finish = [&](int status) {
    if (status != RDE_CELL_BAD_STATE) {
      if constexpr (WIDE) {
#pragma unroll
        for (int k = 0; k < K; ++k) cell.Y[k * cell.ldY + cell.i] = P.ld(k);
        cell.T[cell.i] = P.ld(K);
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) cell.Y[k * cell.ldY + cell.i] = y[k];
        cell.T[cell.i] = y[K];
      }
    }
    if (cell.status) cell.status[cell.i] = status;
    if (cell.n_acc) cell.n_acc[cell.i] = nacc;
    if (cell.n_rej) cell.n_rej[cell.i] = nrej;
    if (cell.h_hint && status == RDE_CELL_OK) cell.h_hint[cell.i] = h;
    if (cell.cycles) cell.cycles[cell.i] = clock64() - cell.t0;
    ++st_cells;
    st_acc += nacc;
    st_rej += nrej;
    st_fail += (status != RDE_CELL_OK);
    st_max = max(st_max, (long long)(nacc + nrej));
    active = false;
  };

  for (;;) {
    // ---- refill: lanes without a cell take the next queue position ----
    bool need = !active && !exhausted;
    while (__any_sync(kFull, need)) {
      long long g = n_total;
      if (QUEUE) {
        const unsigned mask = __ballot_sync(kFull, need);
        const int leader = __ffs(mask) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(a.queue, (unsigned long long)__popc(mask));
        base = __shfl_sync(kFull, base, leader);
        if (need) g = (long long)(base + __popc(mask & ((1u << lane) - 1u)));
      } else if (need && !plain_taken) {
        g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        plain_taken = true;
      }
      if (need) {
        if (g >= n_total) {
          exhausted = true;
          need = false;
        } else if (!locate(a, offs, n_total, g, cell)) {
          // invalid permutation entry: nothing to do for this position
        } else {
          const double p = cell.p[cell.i];
          bool good = isfinite(p) && p > 0.0;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            y[k] = cell.Y[k * cell.ldY + cell.i];
            good = good && isfinite(y[k]);
          }
          y[K] = cell.T[cell.i];
          good = good && isfinite(y[K]) && y[K] > 0.0;
          nacc = nrej = attempts = 0;
          reject_prev = false;
          t = 0.0;
          h = dt;
          if (cell.h_hint) {
            const double hh = cell.h_hint[cell.i];
            if (hh > 0.0) h = fmin(dt, hh);
          }
          invp = 1.0 / p;
          if constexpr (WIDE) {
#pragma unroll
            for (int i = 0; i < N; ++i) P.st(i, y[i]);
          }
          if (good) {
            active = true;
            need = false;
          } else {
            finish(RDE_CELL_BAD_STATE);
          }
        }
      }
    }
    // the wide kernel keeps its warps in step: every thread of the CTA passes this
    // barrier once per attempt (and all leave the loop together), so the warps run the
    // same stretch of the long attempt code at the same time and share the instruction
    // cache; the 128-thread kernels let each warp leave on its own
    if constexpr (WIDE) {
      if (!__syncthreads_or(active ? 1 : 0)) break;
    } else {
      if (!__any_sync(kFull, active)) break;
    }

    // ---- one Rosenbrock attempt on every active lane ----
    if (active) {
      if (attempts >= o.max_substeps) {
        finish(RDE_CELL_MAX_SUBSTEPS);
      } else {
        ++attempts;
        h = fmin(h, dt - t);
        double yn[N], err, unused[4][N];
        bool finite, ok;
        unsigned long long swaps;
        if constexpr (WIDE)
          ok = rodas3_attempt_parked<K, RHS>(m, L, invp, P, h, o, yn, err, finite);
        else if constexpr (METHOD == kMethodExtrap)
          ok = extrapolation_attempt<K, RHS>(m, L, invp, y, h, o, yn, err, finite, Jg, nl);
        else
          ok = rosenbrock_attempt<K, RHS, METHOD>(m, L, invp, y, h, o, yn, err, finite, swaps, unused);
        if (!ok) {
          finish(RDE_CELL_LU_SINGULAR);
        } else if (finite && err <= 1.0) {
          if constexpr (WIDE) {
#pragma unroll
            for (int i = 0; i < N; ++i) P.st(i, yn[i]);
          } else {
#pragma unroll
            for (int i = 0; i < N; ++i) y[i] = yn[i];
          }
          t += h;
          ++nacc;
          h *= step_factor<METHOD>(err, finite, true, reject_prev, o);
          reject_prev = false;
          if (dt - t <= 1e-14 * dt) finish(RDE_CELL_OK);
        } else {
          ++nrej;
          h *= step_factor<METHOD>(err, finite, false, reject_prev, o);
          reject_prev = true;
          if (h < o.hmin) finish(RDE_CELL_H_UNDERFLOW);
        }
      }
    }
  }

  // ---- statistics: warp sums, one atomic per warp ----
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    st_cells += __shfl_down_sync(kFull, st_cells, off);
    st_acc += __shfl_down_sync(kFull, st_acc, off);
    st_rej += __shfl_down_sync(kFull, st_rej, off);
    st_fail += __shfl_down_sync(kFull, st_fail, off);
    st_max = max(st_max, __shfl_down_sync(kFull, st_max, off));
  }
  if (lane == 0 && st_cells > 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 0), (unsigned long long)st_cells);
    atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 1), (unsigned long long)st_acc);
    atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 2), (unsigned long long)st_rej);
    atomicAdd(reinterpret_cast<unsigned long long*>(a.stats + 3), (unsigned long long)st_fail);
    atomicMax(a.stats + 4, st_max);
  }
}

}  // namespace rde
