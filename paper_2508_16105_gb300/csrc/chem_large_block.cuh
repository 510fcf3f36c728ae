// Block-cooperative pieces of the CTA-per-cell chemistry step (sm_103a, FP64):
// one CTA of 128 threads works on one cell whose matrix, species arrays, stage
// vectors and per-reaction values live in shared memory.  f and the analytic
// Jacobian are written for a value type S: double in the step itself, Dual in
// the discrete adjoint, which needs the derivative of the Jacobian along a
// direction.  Used by the forward kernel (chem_large.cu) and the CTA-per-cell
// adjoint (chem_large_adjoint.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "chem_device.cuh"
#include "chem_launch.h"
#include "dual_math.cuh"
#include "large_plan.h"

namespace rde {
namespace {

constexpr int kLT = 128;          // threads of the CTA that shares one cell
constexpr int kLargeMaxN = 64;    // register solves hold N <= 64
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

// both parts of a dual number summed over the block
__device__ __forceinline__ Dual block_sum(Dual v, double* red) {
  const double a = block_sum(v.v, red);
  const double b = block_sum(v.d, red);
  return mk(a, b);
}

// a reaction order (1, 2 or 3) as a double, without an integer conversion
__device__ __forceinline__ double ord_d(int o) { return o == 1 ? 1.0 : (o == 2 ? 2.0 : 3.0); }

// shared-memory arrays of one cell; the arrays that f and the Jacobian write hold
// values of S (double, or Dual for a directional derivative of the Jacobian)
template <class S>
struct CellT {
  S* MX;   // N x LD
  S *C, *G, *HRT, *CPR, *WDOT, *WT, *BK;  // K each
  double* Yv;
  S *ARG, *VEC;  // N each
  double *F0, *U1, *U2, *U3, *U4, *INVD;  // N each
  S* RS;        // R x 9 per-reaction values
  double* red;  // 4 (+4) reduction slots
  int* perm;    // N: row i of P b is b[perm[i]] (the LU's row interchanges composed)
  int* ired;    // 4 + bookkeeping
  // reaction table staged from the plan (structure of arrays)
  const double *rlnA, *rb, *rEaR, *rdnu;
  const int4* rmeta;
  int N, LD, K, R;
};
using Cell = CellT<double>;

// mixture state of one f evaluation
template <class S>
struct MixT {
  S rho, invrho, cpm, dcpm, sumYW, Msum;
};

// falloff blend: the forward kernel's double version, or the dual one
template <bool JAC>
__device__ __forceinline__ double falloff_any(const MechView& m, const RxView& x, double T, double lnT, double invT,
                                              double M, double kinf, double& dlnkf, double& dkf_dM) {
  return falloff<JAC>(m, x, T, lnT, invT, M, kinf, dlnkf, dkf_dM);
}
template <bool JAC>
__device__ __forceinline__ Dual falloff_any(const MechView& m, const RxView& x, Dual T, Dual lnT, Dual invT, Dual M,
                                            Dual kinf, Dual& dlnkf, Dual& dkf_dM) {
  Dual phi;
  return falloff_s<Dual>(m, x, T, lnT, invT, M, kinf, dlnkf, dkf_dM, phi);
}

// f at ARG into VEC; with JAC also D (K x K block of MX), WT, CPR.  Returns mixture state.
template <class S, bool JAC>
__device__ MixT<S> rhs_block(const MechView& m, const PlanView& pl, const CellT<S>& c, double invp) {
  const int K = c.K, R = c.R, tid = threadIdx.x;
  const S T = c.ARG[K];
  const S invT = 1.0 / T;
  const S lnT = slog(m, T);
  const SpecPacked* sp = m.sp;
  S part = cst<S>(0.0);
  for (int k = tid; k < K; k += kLT) {
    const S yw = c.ARG[k] * sp[k].Winv;
    c.C[k] = yw;
    part += yw;
  }
  const S sumYW = block_sum(part, c.red);
  const S RT = kRu * T;
  const S invrho = RT * sumYW * invp;
  const S rho = 1.0 / invrho;
  S pM = cst<S>(0.0), pcp = cst<S>(0.0), pdcp = cst<S>(0.0);
  for (int k = tid; k < K; k += kLT) {
    const S yw = c.C[k];
    const S cc = yw * rho;
    c.C[k] = cc;
    pM += cc;
    const int r = (val(T) >= sp[k].Tmid) ? 1 : 0;
    const double* a = sp[k].cp[r];
    const S cp = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
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
  const S Msum = block_sum(pM, c.red);
  const S cpm = block_sum(pcp, c.red);
  const S dcpm = JAC ? block_sum(pdcp, c.red) : cst<S>(0.0);
  const S lnPRT = kLnPstdOverRu - lnT;
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
    const S lnk = c.rlnA[r] + c.rb[r] * lnT - c.rEaR[r] * invT;
    S M = cst<S>(1.0);
    if (type != RX_ELEM) {
      const RxnPacked& x = m.rx[r];
      M = Msum;
      for (int e = x.eff_begin; e < x.eff_end; ++e) M += m.eff[e].alpha_minus_1 * c.C[m.eff[e].k];
    }
    const bool fo_r = (type == RX_LINDEMANN || type == RX_TROE);
    S kf, dlnkf = cst<S>(0.0), dkf_dM = cst<S>(0.0);
    if (fo_r) {
      kf = falloff_any<JAC>(m, RxView{m.rx[r]}, T, lnT, invT, M, sexp(m, lnk), dlnkf, dkf_dM);
    } else {
      kf = sexp(m, lnk);
      if (JAC) dlnkf = (c.rb[r] + c.rEaR[r] * invT) * invT;
    }
    S kr = cst<S>(0.0), dlnKc = cst<S>(0.0);
    if (rev) {
      const double dnu = c.rdnu[r];
      S lnKc = dnu * lnPRT, dh = cst<S>(0.0);
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
      kr = fo_r ? kf * sexp(m, -lnKc) : sexp(m, lnk - lnKc);
      if (JAC) dlnKc = (dh - dnu) * invT;
    }
    S cf[kMaxSide], cb[kMaxSide], pf[kMaxSide], pb[kMaxSide];
#pragma unroll
    for (int q = 0; q < kMaxSide; ++q) {
      cf[q] = (q < nf) ? c.C[fi[q]] : cst<S>(1.0);
      cb[q] = (q < nb) ? c.C[bi[q]] : cst<S>(1.0);
      pf[q] = (q < nf) ? ipow_s(cf[q], fo[q]) : cst<S>(1.0);
      pb[q] = (q < nb) ? ipow_s(cb[q], bo[q]) : cst<S>(1.0);
    }
    S Pf = pf[0], Pb = pb[0];
    if (nf > 1) Pf *= pf[1];
    if (nf > 2) Pf *= pf[2];
    if (nb > 1) Pb *= pb[1];
    if (nb > 2) Pb *= pb[2];
    const S q0 = kf * Pf - kr * Pb;
    const bool tb = (type == RX_THREEBODY);
    const S mf = tb ? M : cst<S>(1.0);
    S* rs = c.RS + 9 * r;
    rs[7] = mf * q0;
    if (JAC) {
      rs[8] = mf * (kf * dlnkf * Pf - kr * (dlnkf - dlnKc) * Pb);
      const S mkf = mf * kf, mkr = mf * kr;
#pragma unroll
      for (int s = 0; s < kMaxSide; ++s) {
        const S df = (fo[s] == 1) ? cst<S>(1.0) : (fo[s] == 2 ? 2.0 * cf[s] : 3.0 * cf[s] * cf[s]);
        const S db = (bo[s] == 1) ? cst<S>(1.0) : (bo[s] == 2 ? 2.0 * cb[s] : 3.0 * cb[s] * cb[s]);
        S of = cst<S>(1.0), ob = cst<S>(1.0);
#pragma unroll
        for (int t = 0; t < kMaxSide; ++t) {
          if (t != s && t < nf) of *= pf[t];
          if (t != s && t < nb) ob *= pb[t];
        }
        rs[s] = (s < nf) ? mkf * df * of : cst<S>(0.0);
        rs[3 + s] = (s < nb) ? -(mkr * db * ob) : cst<S>(0.0);
      }
      S allc = cst<S>(0.0);
      if (tb) allc = q0;
      else if (fo_r) allc = (val(kf) != 0.0) ? dkf_dM * (q0 / kf) : cst<S>(0.0);
      rs[6] = allc;
    }
  }
  __syncthreads();
  // net production (and its T derivative) per species, reactions in a fixed order;
  // with JAC also A_k, the all-species [M] term of row k of D (into BK)
  for (int k = tid; k < K; k += kLT) {
    S w = cst<S>(0.0), wt = cst<S>(0.0);
    for (int e = pl.spr_ptr[k]; e < pl.spr_ptr[k + 1]; ++e) {
      const double nu = pl.spr_nu[e];
      const S* rs = c.RS + 9 * pl.spr_r[e];
      w += nu * rs[7];
      if (JAC) wt += nu * rs[8];
    }
    c.WDOT[k] = w;
    if (JAC) {
      c.WT[k] = wt;
      S ak = cst<S>(0.0);
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
      S d = c.BK[k];
      if (e >= 0)
        for (int q = pl.ent_ptr[e]; q < pl.ent_ptr[e + 1]; ++q)
          d += pl.con_coef[q] * c.RS[9 * pl.con_r[q] + pl.con_slot[q]];
      c.MX[k * c.LD + idx % K] = d;
    }
  }
  __syncthreads();
  S phw = cst<S>(0.0);
  for (int k = tid; k < K; k += kLT) {
    const S w = c.WDOT[k];
    c.VEC[k] = sp[k].W * w * invrho;
    phw += c.HRT[k] * w;
  }
  const S sum_hw = block_sum(phw, c.red);
  const S cpm_J = kRu * cpm;
  if (tid == 0) c.VEC[K] = -RT * sum_hw * invrho / cpm_J;
  __syncthreads();
  MixT<S> ms;
  ms.rho = rho;
  ms.invrho = invrho;
  ms.cpm = cpm_J;
  ms.dcpm = kRu * dcpm;
  ms.sumYW = sumYW;
  ms.Msum = Msum;
  return ms;
}

// I/(gamma h) - J into MX from D (MX), f (VEC) and the species arrays
template <class S>
__device__ void assemble_block(const MechView& m, const CellT<S>& c, S T, const MixT<S>& ms, S inv_gh) {
  const int K = c.K, N = c.N, LD = c.LD, tid = threadIdx.x;
  const S invT = 1.0 / T, RT = kRu * T, Wbar = 1.0 / ms.sumYW;
  const SpecPacked* sp = m.sp;
  // D c into BK, H^T D into ARG (the state copy is no longer needed)
  for (int k = tid; k < K; k += kLT) {
    S acc = cst<S>(0.0);
    for (int j = 0; j < K; ++j) acc += c.MX[k * LD + j] * c.C[j];
    c.BK[k] = acc;
  }
  for (int i = tid; i < K; i += kLT) {
    S acc = cst<S>(0.0);
    for (int k = 0; k < K; ++k) acc += c.HRT[k] * c.MX[k * LD + i];
    c.ARG[i] = acc;
  }
  __syncthreads();
  S pH = cst<S>(0.0), pC = cst<S>(0.0), pW = cst<S>(0.0);
  for (int k = tid; k < K; k += kLT) {
    const S Dc = c.BK[k], h = c.HRT[k];
    pH += h * Dc;
    pC += c.CPR[k] * c.WDOT[k];
    pW += h * (c.WT[k] - Dc * invT);
  }
  const S HDc = block_sum(pH, c.red);
  const S Cw = block_sum(pC, c.red);
  const S HwT = block_sum(pW, c.red);
  const S fT = c.VEC[K];
  // J_kT column first (needs Dc in BK); then BK <- B_k
  for (int k = tid; k < K; k += kLT) {
    const S e = c.WDOT[k] - c.BK[k];
    c.MX[k * LD + K] = -(sp[k].W * ms.invrho * (c.WT[k] + e * invT));
    c.BK[k] = sp[k].W * Wbar * e * ms.invrho;
  }
  __syncthreads();
  for (int idx = tid; idx < K * K; idx += kLT) {
    const int k = idx / K, i = idx % K;
    const S J = sp[i].Winv * (sp[k].W * c.MX[k * LD + i] + c.BK[k]);
    c.MX[k * LD + i] = (i == k ? inv_gh : cst<S>(0.0)) - J;
  }
  const S inv_cp = 1.0 / ms.cpm, coef = -RT * inv_cp, wHDc = Wbar * ms.invrho * HDc, fcp = fT * inv_cp;
  for (int i = tid; i < K; i += kLT) {
    const S J = sp[i].Winv * (coef * (c.ARG[i] - wHDc) - fcp * (kRu * c.CPR[i] - ms.cpm * Wbar));
    c.MX[K * LD + i] = -J;
  }
  if (tid == 0) {
    const S JTT = -(kRu * Cw + RT * HwT) * ms.invrho * inv_cp + fT * invT - fT * ms.dcpm * inv_cp;
    c.MX[K * LD + K] = inv_gh - JTT;
  }
  (void)N;
  __syncthreads();
}

// LU with partial pivoting of MX (the first maximum wins a tie, as a serial scan finds
// it).  Per column, warp 0 finds the pivot, swaps the rows, stores 1/U_kk and scales
// the multipliers; after one barrier all threads update the trailing block, taking
// its elements in a flat (row-major) index order.
// The row interchanges are composed into perm.  Returns false on a zero pivot (the
// same value in every thread: warp 0 finds it, a block reduction shares it).
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
    // trailing update over the w x w block as one flat index range, so that every lane
    // of every warp has an element while w^2 >= 128 (a row-per-warp split leaves most
    // lanes idle once w < 32)
    const int w = N - k - 1;
    const int tot = w * w;
    for (int idx = tid; idx < tot; idx += kLT) {
      const int ii = idx / w, jj = idx - ii * w;
      const int i = k + 1 + ii, j = k + 1 + jj;
      c.MX[i * LD + j] -= c.MX[i * LD + k] * c.MX[k * LD + j];
    }
    __syncthreads();
  }
  return block_and(ok, c.ired) != 0;
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

// One Rosenbrock attempt of the cell in Yv with step h: f and J at Yv, the LU of
// M = I/(gamma h) - J, the four stages (u_1..u_3 in U1..U3, u_4 in VEC), the
// candidate state y + 2 u_1 + u_3 + u_4 in U4 and the RMS error estimate.
// Returns false (in every thread) on a zero pivot; err and fin are then unset.
__device__ __forceinline__ bool large_attempt(const MechView& m, const PlanView& pl, const Cell& c, double invp,
                                              double h, const Opts& o, double& err, int& fin) {
  const int N = c.N, K = c.K, tid = threadIdx.x;
  for (int k = tid; k < N; k += kLT) c.ARG[k] = c.Yv[k];
  __syncthreads();
  const MixT<double> ms = rhs_block<double, true>(m, pl, c, invp);
  for (int k = tid; k < N; k += kLT) c.F0[k] = c.VEC[k];
  assemble_block(m, c, c.Yv[K], ms, 1.0 / (kGamma * h));
  if (!lu_block(c)) return false;
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
  rhs_block<double, false>(m, pl, c, invp);
  for (int k = tid; k < N; k += kLT) c.VEC[k] += invh * (c.U1[k] - c.U2[k]);
  __syncthreads();
  solve_block(c);
  for (int k = tid; k < N; k += kLT) {
    c.U3[k] = c.VEC[k];
    c.ARG[k] = c.Yv[k] + 2.0 * c.U1[k] + c.U3[k];
  }
  __syncthreads();
  rhs_block<double, false>(m, pl, c, invp);
  for (int k = tid; k < N; k += kLT) c.VEC[k] += invh * (c.U1[k] - c.U2[k] + kC43 * c.U3[k]);
  __syncthreads();
  solve_block(c);
  double pe = 0.0;
  int fn = 1;
  for (int k = tid; k < N; k += kLT) {
    const double yn = c.ARG[k] + c.VEC[k];
    const double sc = o.atol + o.rtol * fmax(fabs(c.Yv[k]), fabs(yn));
    const double e = c.VEC[k] / sc;
    pe += e * e;
    fn &= isfinite(yn) ? 1 : 0;
    c.U4[k] = yn;
  }
  const double sum = block_sum(pe, c.red);
  fin = block_and(fn, c.ired);
  err = sqrt(sum / N);
  return true;
}

// Transposed solve M^T x = b with the factors of lu_block (P M = L U, so
// M^T = U^T L^T P): U^T z = b forward, L^T v = z backward, x[perm[i]] = v[i].
// b in VEC; x back in VEC.  Warp 0 holds the vector in registers (lane l: rows l
// and l + 32) and broadcasts each solved component by shuffle.  N <= 64.
__device__ void solve_block_t(const Cell& c) {
  const int N = c.N, LD = c.LD, tid = threadIdx.x;
  if (tid < 32) {
    const int r0 = tid, r1 = tid + 32;
    double x0 = (r0 < N) ? c.VEC[r0] : 0.0;
    double x1 = (r1 < N) ? c.VEC[r1] : 0.0;
    // U^T z = b: z_j = x_j / U_jj, then x_i -= U_ji z_j for i > j (row j of U)
    for (int j = 0; j < N; ++j) {
      const double dinv = c.INVD[j];
      const int owner = j & 31;
      double zj;
      if (j < 32) {
        if (tid == owner) x0 *= dinv;
        zj = __shfl_sync(kFullL, x0, owner);
      } else {
        if (tid == owner) x1 *= dinv;
        zj = __shfl_sync(kFullL, x1, owner);
      }
      if (r0 > j && r0 < N) x0 -= c.MX[j * LD + r0] * zj;
      if (r1 > j && r1 < N) x1 -= c.MX[j * LD + r1] * zj;
    }
    // L^T v = z with the unit lower triangle: x_i -= L_ji v_j for i < j (row j of L)
    for (int j = N - 1; j > 0; --j) {
      const double vj = __shfl_sync(kFullL, j < 32 ? x0 : x1, j & 31);
      if (r0 < j) x0 -= c.MX[j * LD + r0] * vj;
      if (r1 < j) x1 -= c.MX[j * LD + r1] * vj;
    }
    __syncwarp();
    if (r0 < N) c.VEC[c.perm[r0]] = x0;
    if (r1 < N) c.VEC[c.perm[r1]] = x1;
  }
  __syncthreads();
}

}  // namespace
}  // namespace rde
