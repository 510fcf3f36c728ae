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

#include "chem_device.cuh"
#include "chem_launch.h"
#include "large_plan.h"

namespace rde {
namespace {

constexpr int kLT = 128;
constexpr int kLargeMaxBlocks = 1024;
constexpr int kLargeMaxN = 64;
constexpr int kLargeCtasPerSm = 3;   // register budget per thread: 65536 / (3 x 128) = 170
constexpr unsigned kFullL = 0xffffffffu;

// deterministic block sum (fixed shuffle pattern, fixed order across warps); all threads get it
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(kFullL, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  return red[0] + red[1] + red[2] + red[3];
}

__device__ __forceinline__ int block_and(int v, int* ired) {
  v = __all_sync(kFullL, v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) ired[threadIdx.x >> 5] = v;
  __syncthreads();
  return ired[0] & ired[1] & ired[2] & ired[3];
}

// a reaction order (1, 2 or 3) as a double, without an integer conversion
__device__ __forceinline__ double ord_d(int o) { return o == 1 ? 1.0 : (o == 2 ? 2.0 : 3.0); }

// shared-memory arrays of one cell
struct Cell {
  double* MX;   // N x LD
  double *C, *G, *HRT, *CPR, *WDOT, *WT, *BK;  // K each
  double *Yv, *ARG, *VEC, *F0, *U1, *U2, *U3, *U4, *INVD;  // N each
  double* RS;   // R x 9 per-reaction values
  double* red;  // 4 (+4) reduction slots
  int* perm;    // N: row i of P b is b[perm[i]] (the LU's row interchanges composed)
  int* ired;    // 4 + bookkeeping
  // reaction table staged from the plan (structure of arrays)
  const double *rlnA, *rb, *rEaR, *rdnu;
  const int4* rmeta;
  int N, LD, K, R;
};

// f at ARG into VEC; with JAC also D (K x K block of MX), WT, CPR.  Returns mixture state.
template <bool JAC>
__device__ MixState rhs_block(const MechView& m, const PlanView& pl, const Cell& c, double invp) {
  const int K = c.K, R = c.R, tid = threadIdx.x;
  const double T = c.ARG[K];
  const double invT = 1.0 / T;
  const double lnT = log_tab(T, m.logtab);
  const SpecPacked* sp = m.sp;
  double part = 0.0;
  for (int k = tid; k < K; k += kLT) {
    const double yw = c.ARG[k] * sp[k].Winv;
    c.C[k] = yw;
    part += yw;
  }
  const double sumYW = block_sum(part, c.red);
  const double RT = kRu * T;
  const double invrho = RT * sumYW * invp;
  const double rho = 1.0 / invrho;
  double pM = 0.0, pcp = 0.0, pdcp = 0.0;
  for (int k = tid; k < K; k += kLT) {
    const double yw = c.C[k];
    const double cc = yw * rho;
    c.C[k] = cc;
    pM += cc;
    const int r = (T >= sp[k].Tmid) ? 1 : 0;
    const double* a = sp[k].cp[r];
    const double cp = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    const double* hh = sp[k].h[r];
    c.HRT[k] = hh[0] + T * (hh[1] + T * (hh[2] + T * (hh[3] + T * hh[4]))) + hh[5] * invT;
    const double* gg = sp[k].g[r];
    c.G[k] = gg[0] + gg[1] * lnT + T * (gg[2] + T * (gg[3] + T * (gg[4] + T * gg[5]))) + gg[6] * invT;
    pcp += yw * cp;
    if (JAC) {
      const double* dc = sp[k].dcp[r];
      pdcp += yw * (dc[0] + T * (dc[1] + T * (dc[2] + T * dc[3])));
      c.CPR[k] = cp;
    }
  }
  const double Msum = block_sum(pM, c.red);
  const double cpm = block_sum(pcp, c.red);
  const double dcpm = JAC ? block_sum(pdcp, c.red) : 0.0;
  const double lnPRT = kLnPstdOverRu - lnT;
  // per-reaction values: RS[r] = gf[3], gb[3], allc, q, dq/dT
  for (int r = tid; r < R; r += kLT) {
    const int4 mt = c.rmeta[r];
    const int type = mt.x & 3, nf = (mt.x >> 3) & 3, nb = (mt.x >> 5) & 3;
    const bool rev = (mt.x >> 2) & 1;
    int fi[kMaxSide], bi[kMaxSide], fo[kMaxSide], bo[kMaxSide];
#pragma unroll
    for (int q = 0; q < kMaxSide; ++q) {
      fi[q] = (mt.y >> (10 * q)) & 1023;
      bi[q] = (mt.z >> (10 * q)) & 1023;
      fo[q] = (mt.x >> (8 + 2 * q)) & 3;
      bo[q] = (mt.x >> (14 + 2 * q)) & 3;
    }
    const double lnk = c.rlnA[r] + c.rb[r] * lnT - c.rEaR[r] * invT;
    double M = 1.0;
    if (type != RX_ELEM) {
      const RxnPacked& x = m.rx[r];
      M = Msum;
      for (int e = x.eff_begin; e < x.eff_end; ++e) M += m.eff[e].alpha_minus_1 * c.C[m.eff[e].k];
    }
    const bool fo_r = (type == RX_LINDEMANN || type == RX_TROE);
    double kf, dlnkf = 0.0, dkf_dM = 0.0;
    if (fo_r) {
      kf = falloff<JAC>(m, RxView{m.rx[r]}, T, lnT, invT, M, exp_tab(lnk, m.exptab), dlnkf, dkf_dM);
    } else {
      kf = exp_tab(lnk, m.exptab);
      if (JAC) dlnkf = (c.rb[r] + c.rEaR[r] * invT) * invT;
    }
    double kr = 0.0, dlnKc = 0.0;
    if (rev) {
      const double dnu = c.rdnu[r];
      double lnKc = dnu * lnPRT, dh = 0.0;
#pragma unroll
      for (int q = 0; q < kMaxSide; ++q) {
        if (q < nf) {
          const double o = ord_d(fo[q]);
          lnKc += o * c.G[fi[q]];
          if (JAC) dh -= o * c.HRT[fi[q]];
        }
        if (q < nb) {
          const double o = ord_d(bo[q]);
          lnKc -= o * c.G[bi[q]];
          if (JAC) dh += o * c.HRT[bi[q]];
        }
      }
      kr = fo_r ? kf * exp_tab(-lnKc, m.exptab) : exp_tab(lnk - lnKc, m.exptab);
      if (JAC) dlnKc = (dh - dnu) * invT;
    }
    double cf[kMaxSide], cb[kMaxSide], pf[kMaxSide], pb[kMaxSide];
#pragma unroll
    for (int q = 0; q < kMaxSide; ++q) {
      cf[q] = (q < nf) ? c.C[fi[q]] : 1.0;
      cb[q] = (q < nb) ? c.C[bi[q]] : 1.0;
      pf[q] = (q < nf) ? ipow(cf[q], fo[q]) : 1.0;
      pb[q] = (q < nb) ? ipow(cb[q], bo[q]) : 1.0;
    }
    double Pf = pf[0], Pb = pb[0];
    if (nf > 1) Pf *= pf[1];
    if (nf > 2) Pf *= pf[2];
    if (nb > 1) Pb *= pb[1];
    if (nb > 2) Pb *= pb[2];
    const double q0 = kf * Pf - kr * Pb;
    const bool tb = (type == RX_THREEBODY);
    const double mf = tb ? M : 1.0;
    double* rs = c.RS + 9 * r;
    rs[7] = mf * q0;
    if (JAC) {
      rs[8] = mf * (kf * dlnkf * Pf - kr * (dlnkf - dlnKc) * Pb);
      const double mkf = mf * kf, mkr = mf * kr;
#pragma unroll
      for (int s = 0; s < kMaxSide; ++s) {
        const double df = (fo[s] == 1) ? 1.0 : (fo[s] == 2 ? 2.0 * cf[s] : 3.0 * cf[s] * cf[s]);
        const double db = (bo[s] == 1) ? 1.0 : (bo[s] == 2 ? 2.0 * cb[s] : 3.0 * cb[s] * cb[s]);
        double of = 1.0, ob = 1.0;
#pragma unroll
        for (int t = 0; t < kMaxSide; ++t) {
          if (t != s && t < nf) of *= pf[t];
          if (t != s && t < nb) ob *= pb[t];
        }
        rs[s] = (s < nf) ? mkf * df * of : 0.0;
        rs[3 + s] = (s < nb) ? -(mkr * db * ob) : 0.0;
      }
      double allc = 0.0;
      if (tb) allc = q0;
      else if (fo_r) allc = (kf != 0.0) ? dkf_dM * (q0 / kf) : 0.0;
      rs[6] = allc;
    }
  }
  __syncthreads();
  // net production (and its T derivative) per species, reactions in a fixed order;
  // with JAC also A_k, the all-species [M] term of row k of D (into BK)
  for (int k = tid; k < K; k += kLT) {
    double w = 0.0, wt = 0.0;
    for (int e = pl.spr_ptr[k]; e < pl.spr_ptr[k + 1]; ++e) {
      const double nu = pl.spr_nu[e];
      const double* rs = c.RS + 9 * pl.spr_r[e];
      w += nu * rs[7];
      if (JAC) wt += nu * rs[8];
    }
    c.WDOT[k] = w;
    if (JAC) {
      c.WT[k] = wt;
      double ak = 0.0;
      for (int e = pl.row_ptr[k]; e < pl.row_ptr[k + 1]; ++e) ak += pl.row_nu[e] * c.RS[9 * pl.row_r[e] + 6];
      c.BK[k] = ak;
    }
  }
  if (JAC) {
    __syncthreads();
    // D = d omega / d c (fixed T): A_k plus the entry's contributions in a fixed order
    for (int idx = tid; idx < K * K; idx += kLT) {
      const int k = idx / K;
      const int e = pl.ent_index[idx];
      double d = c.BK[k];
      if (e >= 0)
        for (int q = pl.ent_ptr[e]; q < pl.ent_ptr[e + 1]; ++q)
          d += pl.con_coef[q] * c.RS[9 * pl.con_r[q] + pl.con_slot[q]];
      c.MX[k * c.LD + idx % K] = d;
    }
  }
  __syncthreads();
  double phw = 0.0;
  for (int k = tid; k < K; k += kLT) {
    const double w = c.WDOT[k];
    c.VEC[k] = sp[k].W * w * invrho;
    phw += c.HRT[k] * w;
  }
  const double sum_hw = block_sum(phw, c.red);
  const double cpm_J = kRu * cpm;
  if (tid == 0) c.VEC[K] = -RT * sum_hw * invrho / cpm_J;
  __syncthreads();
  MixState ms;
  ms.rho = rho;
  ms.invrho = invrho;
  ms.cpm = cpm_J;
  ms.dcpm = kRu * dcpm;
  ms.sumYW = sumYW;
  return ms;
}

// I/(gamma h) - J into MX from D (MX), f (VEC) and the species arrays
__device__ void assemble_block(const MechView& m, const Cell& c, double T, const MixState& ms, double inv_gh) {
  const int K = c.K, N = c.N, LD = c.LD, tid = threadIdx.x;
  const double invT = 1.0 / T, RT = kRu * T, Wbar = 1.0 / ms.sumYW;
  const SpecPacked* sp = m.sp;
  // D c into BK, H^T D into ARG (the state copy is no longer needed)
  for (int k = tid; k < K; k += kLT) {
    double acc = 0.0;
    for (int j = 0; j < K; ++j) acc += c.MX[k * LD + j] * c.C[j];
    c.BK[k] = acc;
  }
  for (int i = tid; i < K; i += kLT) {
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc += c.HRT[k] * c.MX[k * LD + i];
    c.ARG[i] = acc;
  }
  __syncthreads();
  double pH = 0.0, pC = 0.0, pW = 0.0;
  for (int k = tid; k < K; k += kLT) {
    const double Dc = c.BK[k], h = c.HRT[k];
    pH += h * Dc;
    pC += c.CPR[k] * c.WDOT[k];
    pW += h * (c.WT[k] - Dc * invT);
  }
  const double HDc = block_sum(pH, c.red);
  const double Cw = block_sum(pC, c.red);
  const double HwT = block_sum(pW, c.red);
  const double fT = c.VEC[K];
  // J_kT column first (needs Dc in BK); then BK <- B_k
  for (int k = tid; k < K; k += kLT) {
    const double e = c.WDOT[k] - c.BK[k];
    c.MX[k * LD + K] = -(sp[k].W * ms.invrho * (c.WT[k] + e * invT));
    c.BK[k] = sp[k].W * Wbar * e * ms.invrho;
  }
  __syncthreads();
  for (int idx = tid; idx < K * K; idx += kLT) {
    const int k = idx / K, i = idx % K;
    const double J = sp[i].Winv * (sp[k].W * c.MX[k * LD + i] + c.BK[k]);
    c.MX[k * LD + i] = (i == k ? inv_gh : 0.0) - J;
  }
  const double inv_cp = 1.0 / ms.cpm, coef = -RT * inv_cp, wHDc = Wbar * ms.invrho * HDc, fcp = fT * inv_cp;
  for (int i = tid; i < K; i += kLT) {
    const double J = sp[i].Winv * (coef * (c.ARG[i] - wHDc) - fcp * (kRu * c.CPR[i] - ms.cpm * Wbar));
    c.MX[K * LD + i] = -J;
  }
  if (tid == 0) {
    const double JTT = -(kRu * Cw + RT * HwT) * ms.invrho * inv_cp + fT * invT - fT * ms.dcpm * inv_cp;
    c.MX[K * LD + K] = inv_gh - JTT;
  }
  (void)N;
  __syncthreads();
}

// LU with partial pivoting of MX (the first maximum wins a tie, as a serial scan finds
// it).  Per column, warp 0 finds the pivot, swaps the rows, stores 1/U_kk and scales
// the multipliers; after one barrier all warps update the trailing block, warp w
// taking rows k+1+w, k+5+w, ... and each lane fixed columns (no index division).
// The row interchanges are composed into perm.  Returns false on a zero pivot.
__device__ bool lu_block(const Cell& c) {
  const int N = c.N, LD = c.LD, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < N; i += kLT) c.perm[i] = i;
  __syncthreads();
  int ok = 1;
  for (int k = 0; k < N; ++k) {
    if (warp == 0) {
      // NaN entries never win; if none is a number the pivot stays on the diagonal
      double best = -1.0;
      int bi = N;
      for (int i = k + lane; i < N; i += 32) {
        const double v = fabs(c.MX[i * LD + k]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(kFullL, best, off);
        const int oi = __shfl_down_sync(kFullL, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      const int p = __shfl_sync(kFullL, bi < N ? bi : k, 0);
      ok &= __shfl_sync(kFullL, best == 0.0 ? 0 : 1, 0);
      if (p != k) {
        for (int j = lane; j < N; j += 32) {
          const double t = c.MX[k * LD + j];
          c.MX[k * LD + j] = c.MX[p * LD + j];
          c.MX[p * LD + j] = t;
        }
        if (lane == 0) {
          const int t = c.perm[k];
          c.perm[k] = c.perm[p];
          c.perm[p] = t;
        }
      }
      __syncwarp();
      const double inv = 1.0 / c.MX[k * LD + k];
      if (lane == 0) c.INVD[k] = inv;
      for (int i = k + 1 + lane; i < N; i += 32) c.MX[i * LD + k] *= inv;
    }
    __syncthreads();
    // trailing update; a lane's columns of row k stay in registers
    const int j0 = k + 1 + lane, j1 = j0 + 32;
    const double u0 = (j0 < N) ? c.MX[k * LD + j0] : 0.0;
    const double u1 = (j1 < N) ? c.MX[k * LD + j1] : 0.0;
    for (int i = k + 1 + warp; i < N; i += kLT / 32) {
      const double l = c.MX[i * LD + k];
      if (j0 < N) c.MX[i * LD + j0] -= l * u0;
      if (j1 < N) c.MX[i * LD + j1] -= l * u1;
    }
    __syncthreads();
  }
  return ok != 0;
}

// Triangular solves of (LU) x = P b, b in VEC; x back in VEC.  Warp 0 holds x in
// registers (lane l: rows l and l + 32) and broadcasts each solved component by
// shuffle; the column entries of the next step are loaded ahead.  N <= 64.
__device__ void solve_block(const Cell& c) {
  const int N = c.N, LD = c.LD, tid = threadIdx.x;
  if (tid < 32) {
    const int r0 = tid, r1 = tid + 32;
    double x0 = (r0 < N) ? c.VEC[c.perm[r0]] : 0.0;
    double x1 = (r1 < N) ? c.VEC[c.perm[r1]] : 0.0;
    // forward: unit lower triangle
    double l0 = (r0 < N && r0 > 0) ? c.MX[r0 * LD] : 0.0;
    double l1 = (r1 < N) ? c.MX[r1 * LD] : 0.0;
    for (int j = 0; j < N - 1; ++j) {
      const double xj = __shfl_sync(kFullL, j < 32 ? x0 : x1, j & 31);
      const int jn = j + 1;
      const double n0 = (r0 < N && r0 > jn) ? c.MX[r0 * LD + jn] : 0.0;
      const double n1 = (r1 < N && r1 > jn) ? c.MX[r1 * LD + jn] : 0.0;
      if (r0 > j) x0 -= l0 * xj;
      if (r1 > j && r1 < N) x1 -= l1 * xj;
      l0 = n0;
      l1 = n1;
    }
    // backward: upper triangle with 1/U_jj
    const int last = N - 1;
    double a0 = (r0 < last) ? c.MX[r0 * LD + last] : 0.0;
    double a1 = (r1 < last) ? c.MX[r1 * LD + last] : 0.0;
    for (int j = last; j >= 0; --j) {
      const double dinv = c.INVD[j];
      const int owner = j & 31;
      double xj;
      if (j < 32) {
        if (tid == owner) x0 *= dinv;
        xj = __shfl_sync(kFullL, x0, owner);
      } else {
        if (tid == owner) x1 *= dinv;
        xj = __shfl_sync(kFullL, x1, owner);
      }
      const int jp = j - 1;
      const double n0 = (jp >= 0 && r0 < jp) ? c.MX[r0 * LD + jp] : 0.0;
      const double n1 = (jp >= 0 && r1 < jp) ? c.MX[r1 * LD + jp] : 0.0;
      if (r0 < j) x0 -= a0 * xj;
      if (r1 < j) x1 -= a1 * xj;
      a0 = n0;
      a1 = n1;
    }
    __syncwarp();
    if (r0 < N) c.VEC[r0] = x0;
    if (r1 < N) c.VEC[r1] = x1;
  }
  __syncthreads();
}

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
      acc += a.blocks[b].n;
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
    }
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
      for (int k = tid; k < N; k += kLT) c.ARG[k] = c.Yv[k];
      __syncthreads();
      const MixState ms = rhs_block<true>(m, pl, c, invp);
      for (int k = tid; k < N; k += kLT) c.F0[k] = c.VEC[k];
      assemble_block(m, c, c.Yv[K], ms, 1.0 / (kGamma * h));
      if (!lu_block(c)) {
        status = RDE_CELL_LU_SINGULAR;
        break;
      }
      const double invh = 1.0 / h;
      for (int k = tid; k < N; k += kLT) c.VEC[k] = c.F0[k];
      __syncthreads();
      solve_block(c);
      for (int k = tid; k < N; k += kLT) {
        c.U1[k] = c.VEC[k];
        c.VEC[k] = c.F0[k] + (kC21 * invh) * c.VEC[k];
      }
      __syncthreads();
      solve_block(c);
      for (int k = tid; k < N; k += kLT) {
        c.U2[k] = c.VEC[k];
        c.ARG[k] = c.Yv[k] + 2.0 * c.U1[k];
      }
      __syncthreads();
      rhs_block<false>(m, pl, c, invp);
      for (int k = tid; k < N; k += kLT) c.VEC[k] += invh * (c.U1[k] - c.U2[k]);
      __syncthreads();
      solve_block(c);
      for (int k = tid; k < N; k += kLT) {
        c.U3[k] = c.VEC[k];
        c.ARG[k] = c.Yv[k] + 2.0 * c.U1[k] + c.U3[k];
      }
      __syncthreads();
      rhs_block<false>(m, pl, c, invp);
      for (int k = tid; k < N; k += kLT) c.VEC[k] += invh * (c.U1[k] - c.U2[k] + kC43 * c.U3[k]);
      __syncthreads();
      solve_block(c);
      double pe = 0.0;
      int fin = 1;
      for (int k = tid; k < N; k += kLT) {
        const double yn = c.ARG[k] + c.VEC[k];
        const double sc = o.atol + o.rtol * fmax(fabs(c.Yv[k]), fabs(yn));
        const double e = c.VEC[k] / sc;
        pe += e * e;
        fin &= isfinite(yn) ? 1 : 0;
        c.U4[k] = yn;
      }
      const double sum = block_sum(pe, c.red);
      fin = block_and(fin, c.ired);
      const double err = sqrt(sum / N);
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
