// Discrete adjoint of the CTA-per-cell chemistry step (large mechanisms, sm_103a,
// FP64): the derivative of (T0, Y0, ln A_r, E_r) -> (T, Y)(dt) along each cell's
// frozen sequence of accepted RODAS3 steps, as in chem_adjoint_body.cuh, for
// mechanisms whose N x N matrix does not fit the thread-per-cell lane slots.
//
// One persistent CTA of 128 threads per cell (work queue; the cells come in the
// cost order of order_kernel, most accepted steps first).  Per cell it
//  1. re-integrates the cell with the forward kernel's attempt (large_attempt),
//     writing the start state y_n and size h_n of every accepted step into the
//     pool at the cell's offset (an exclusive scan of the forward pass's counts);
//  2. walks the steps backwards: recomputes the step's Jacobian, LU factors and
//     stages (stage recompute; a 53-species step checkpoint would be 25 KB), then
//         w_i = M^-T ubar_i                       (solve_block_t)
//         ybar += J(Y_i)^T w_i,  ubar_j += a_ij J(Y_i)^T w_i + c_ij/h w_i
//         ybar += grad_y (w_i^T J(y) u_i)  and the ln A / E terms of both.
//     J(Y_i) is formed explicitly (rhs_block + assemble_block with 1/(gamma h) = 0
//     give -J) and contracted by a block matrix-vector product; the second-
//     derivative terms d/de [J(y + e u_i)^T w_i] are the derivative parts of the
//     same Jacobian formed with two-direction dual numbers, along (u_1, u_2) and
//     (u_3, u_4); the first one's value part, J(y), also serves the stage-1 term;
//  3. writes gY0, gT0 and the cell's parameter rows; the host reduces the rows.
#include <cuda_runtime.h>
#include <stdint.h>

#include "chem_adjoint_body.cuh"
#include "chem_large_block.cuh"

namespace rde {

// block sums and the falloff blend for values with several derivative directions
// (found by argument-dependent lookup from the block templates)
template <int ND>
__device__ __forceinline__ DualN<ND> block_sum(const DualN<ND>& v, double* red) {
  DualN<ND> r;
  r.v = block_sum(v.v, red);
#pragma unroll
  for (int i = 0; i < ND; ++i) r.d[i] = block_sum(v.d[i], red);
  return r;
}
template <bool JAC, int ND>
__device__ __forceinline__ DualN<ND> falloff_any(const MechView& m, const RxView& x, DualN<ND> T, DualN<ND> lnT,
                                                 DualN<ND> invT, DualN<ND> M, DualN<ND> kinf, DualN<ND>& dlnkf,
                                                 DualN<ND>& dkf_dM) {
  DualN<ND> phi;
  return falloff_s<DualN<ND>>(m, x, T, lnT, invT, M, kinf, dlnkf, dkf_dM, phi);
}

namespace {

using D2 = DualN<2>;   // value and the derivatives along two stage vectors

// The forward attempt compiled once for the self-checkpointing kernel, so that its
// re-integration and its segment replays run the very same instructions (bitwise equal
// steps); the recorded-mode kernel inlines the attempt as the forward kernel does.
__device__ __noinline__ bool large_attempt_once(const MechView m, const PlanView pl, const Cell c, double invp,
                                                double h, const Opts o, double* err, int* fin) {
  return large_attempt(m, pl, c, invp, h, o, *err, *fin);
}

template <bool SELF>
__device__ __forceinline__ bool adj_large_attempt(const MechView& m, const PlanView& pl, const Cell& c, double invp,
                                                  double h, const Opts& o, double& err, int& fin) {
  if constexpr (SELF) return large_attempt_once(m, pl, c, invp, h, o, &err, &fin);
  else return large_attempt(m, pl, c, invp, h, o, err, fin);
}

// shared-memory layout (doubles after the exp/log tables), in this order:
//   the forward cell (N LD + 7 K + 9 N + 9 R + 8), the two-direction dual cell
//   (3 (N LD + 7 K + 2 N + 9 R); its matrix's memory also holds the explicit Jacobian
//   at a stage argument, never live at the same time), the adjoint vectors (10 N),
//   the parameter cotangents TH (2 R); then N + 8 ints (permutation, flags)
__host__ __device__ inline size_t large_adj_doubles(int K, int R) {
  const size_t N = (size_t)K + 1, LD = N | 1;
  return N * LD + 7 * (size_t)K + 9 * N + 9 * (size_t)R + 8 + 3 * (N * LD + 7 * (size_t)K + 2 * N + 9 * (size_t)R) +
         10 * N + 2 * (size_t)R;
}

// g = -(MX)^T w over N columns (MX holds -J): thread j sums column j in a fixed order
__device__ __forceinline__ void neg_mt_w(const double* MX, int N, int LD, const double* w, double* g) {
  for (int j = threadIdx.x; j < N; j += kLT) {
    double acc = 0.0;
    for (int i = 0; i < N; ++i) acc += MX[i * LD + j] * w[i];
    g[j] = -acc;
  }
}

// w^T df/d(ln A_r) and w^T df/dE_r added to TH[r], TH[R + r]; reaction r by one
// thread.  The state of the f evaluation: the cell's species arrays and RS after
// rhs_block, its mixture state and temperature.
__device__ void param_terms(const MechView& m, const Cell& c, const MixT<double>& ms, double T, const double* w,
                            double* TH) {
  const int K = c.K, R = c.R;
  const double invT = 1.0 / T, lnT = slog(m, T), RT = kRu * T;
  const double facT = (w[K] * RT) / ms.cpm;
  for (int r = threadIdx.x; r < R; r += kLT) {
    const RxView x{m.rx[r]};
    double phi = 1.0;
    if (x.type() == RX_LINDEMANN || x.type() == RX_TROE) {
      double M = ms.Msum;
      for (int e = x.eff_begin(); e < x.eff_end(); ++e) M += x.eff_am1(m, e) * c.C[x.eff_k(m, e)];
      const double lnk = c.rlnA[r] + c.rb[r] * lnT - c.rEaR[r] * invT;
      double dlnkf, dkf_dM;
      falloff_s<double>(m, x, T, lnT, invT, M, sexp(m, lnk), dlnkf, dkf_dM, phi);
    }
    double s1 = 0.0, s2 = 0.0;
    for (int pp = 0; pp < x.np(); ++pp) {
      const int k = x.pi(pp);
      s1 += w[k] * m.sp[k].W * x.pnu(pp);
      s2 += x.pnu(pp) * c.HRT[k];
    }
    const double q = c.RS[9 * r + 7];
    const double sr = (s1 - facT * s2) * ms.invrho;
    const double tA = sr * phi * q;
    TH[r] += tA;
    TH[R + r] += -(tA / RT);
  }
}

// g = -(der_0(MX)^T wa + der_1(MX)^T wb) and, when wv is given, -(val(MX)^T wv): the
// two directions' second-derivative terms (and the value term) of a dual Jacobian
__device__ __forceinline__ void neg_mt_w2(const D2* MX, int N, int LD, const double* wa, const double* wb,
                                          const double* wv, double* g) {
  for (int j = threadIdx.x; j < N; j += kLT) {
    double acc = 0.0, accv = 0.0;
    for (int i = 0; i < N; ++i) {
      const D2& x = MX[i * LD + j];
      acc += x.d[0] * wa[i] + x.d[1] * wb[i];
      if (wv) accv += x.v * wv[i];
    }
    g[j] = -acc - accv;
  }
}

// param_terms for two directions: derivative part of direction 0 with weights wa, of
// direction 1 with wb, and (wv given) the value part with wv, added to TH
__device__ void param_terms2(const MechView& m, const CellT<D2>& c, const MixT<D2>& ms, D2 T, const double* wa,
                             const double* wb, double* TH, const double* wv) {
  const int K = c.K, R = c.R;
  const D2 invT = 1.0 / T, lnT = slog(m, T), RT = kRu * T;
  const double* ws[2] = {wa, wb};
  Dual facT[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) facT[i] = (ws[i][K] * view(RT, i)) / view(ms.cpm, i);
  const double facTv = wv ? (wv[K] * RT.v) / ms.cpm.v : 0.0;
  for (int r = threadIdx.x; r < R; r += kLT) {
    const RxView x{m.rx[r]};
    D2 phi = cst<D2>(1.0);
    if (x.type() == RX_LINDEMANN || x.type() == RX_TROE) {
      D2 M = ms.Msum;
      for (int e = x.eff_begin(); e < x.eff_end(); ++e) M += x.eff_am1(m, e) * c.C[x.eff_k(m, e)];
      const D2 lnk = c.rlnA[r] + c.rb[r] * lnT - c.rEaR[r] * invT;
      D2 dlnkf, dkf_dM;
      falloff_s<D2>(m, x, T, lnT, invT, M, sexp(m, lnk), dlnkf, dkf_dM, phi);
    }
    double s1[2] = {0.0, 0.0}, s1v = 0.0;
    D2 s2 = cst<D2>(0.0);
    for (int pp = 0; pp < x.np(); ++pp) {
      const int k = x.pi(pp);
      s1[0] += wa[k] * m.sp[k].W * x.pnu(pp);
      s1[1] += wb[k] * m.sp[k].W * x.pnu(pp);
      if (wv) s1v += wv[k] * m.sp[k].W * x.pnu(pp);
      s2 += x.pnu(pp) * c.HRT[k];
    }
    const D2 q = c.RS[9 * r + 7];
    double dA = 0.0, dE = 0.0;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const Dual sr = (s1[i] - facT[i] * view(s2, i)) * view(ms.invrho, i);
      const Dual tA = sr * view(phi, i) * view(q, i);
      const Dual tE = -(tA / view(RT, i));
      dA += tA.d;
      dE += tE.d;
    }
    if (wv) {
      const double vA = (s1v - facTv * s2.v) * ms.invrho.v * phi.v * q.v;
      dA += vA;
      dE += -(vA / RT.v);
    }
    TH[r] += dA;
    TH[R + r] += dE;
  }
}

template <bool SELF>
__global__ void __launch_bounds__(kLT, 1) chem_large_adjoint_kernel(const AdjArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const MechHeader* H = reinterpret_cast<const MechHeader*>(a.mech);
  const int K = a.K, N = K + 1, R = H->R, LD = N | 1, tid = threadIdx.x;
  const int tab_bytes = (int)(sizeof(double) * (kExpTabSize + 2 * kLogTabSize));
  {
    const int4* src = reinterpret_cast<const int4*>(a.mech + H->tab_offset);
    int4* dst = reinterpret_cast<int4*>(smem);
    for (int i = tid; i < tab_bytes / 16; i += blockDim.x) dst[i] = src[i];
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
  c.MX = d; d += N * LD;
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
  // the explicit Jacobian at a stage argument: the forward cell with its own matrix, in
  // the memory of the dual cell's matrix (the two are never live at the same time)
  Cell cj = c;
  cj.MX = d;
  // the two-direction dual cell (J and its derivatives along two stage vectors)
  CellT<D2> dc;
  D2* dd = reinterpret_cast<D2*>(d);
  dc.MX = dd; dd += N * LD;
  dc.C = dd; dd += K;
  dc.G = dd; dd += K;
  dc.HRT = dd; dd += K;
  dc.CPR = dd; dd += K;
  dc.WDOT = dd; dd += K;
  dc.WT = dd; dd += K;
  dc.BK = dd; dd += K;
  dc.ARG = dd; dd += N;
  dc.VEC = dd; dd += N;
  dc.RS = dd; dd += 9 * R;
  dc.Yv = nullptr;
  dc.F0 = dc.U1 = dc.U2 = dc.U3 = dc.U4 = dc.INVD = nullptr;
  dc.red = c.red;
  dc.rlnA = c.rlnA;
  dc.rb = c.rb;
  dc.rEaR = c.rEaR;
  dc.rdnu = c.rdnu;
  dc.rmeta = c.rmeta;
  dc.N = N;
  dc.LD = LD;
  dc.K = K;
  dc.R = R;
  d = reinterpret_cast<double*>(dd);
  double* LAM = d; d += N;
  double* YB = d; d += N;
  double* UB1 = d; d += N;
  double* UB2 = d; d += N;
  double* UB3 = d; d += N;
  double* W = d; d += 4 * N;   // w_1 .. w_4
  double* GV = d; d += N;
  double* TH = d; d += 2 * R;
  c.perm = reinterpret_cast<int*>(d);
  c.ired = c.perm + N;
  cj.perm = c.perm;
  cj.ired = c.ired;
  dc.perm = c.perm;
  dc.ired = c.ired;
  const Opts o{a.opt.rtol, a.opt.atol, a.opt.h_min, a.opt.facmax, a.opt.facmin, a.opt.safety, a.opt.max_substeps, 0};
  const double dt = a.dt;
  __syncthreads();

  // g = J(arg)^T w and the parameter terms at arg (arg in c.ARG): GV, TH
  auto jtw_primal = [&](const double* w, double invp) {
    const MixT<double> ms = rhs_block<double, true>(m, pl, cj, invp);
    const double T = cj.ARG[K];
    param_terms(m, cj, ms, T, w, TH);
    assemble_block<double>(m, cj, T, ms, 0.0);
    neg_mt_w(cj.MX, N, LD, w, GV);
    __syncthreads();
  };
  // g = d/de [J(y + e ua)^T wa] + d/de [J(y + e ub)^T wb] and the parameter terms'
  // derivatives: GV, TH; with wv also J(y)^T wv and its parameter terms from the value
  // part of the same evaluation
  auto jtw_dual2 = [&](const double* y, const double* ua, const double* ub, const double* wa, const double* wb,
                       double invp, const double* wv) {
    for (int k = tid; k < N; k += kLT) {
      D2 v;
      v.v = y[k];
      v.d[0] = ua[k];
      v.d[1] = ub[k];
      dc.ARG[k] = v;
    }
    __syncthreads();
    const MixT<D2> ms = rhs_block<D2, true>(m, pl, dc, invp);
    const D2 T = dc.ARG[K];
    param_terms2(m, dc, ms, T, wa, wb, TH, wv);
    assemble_block<D2>(m, dc, T, ms, cst<D2>(0.0));
    neg_mt_w2(dc.MX, N, LD, wa, wb, wv, GV);
    __syncthreads();
  };

  for (;;) {
    if (tid == 0) cellidx[0] = (long long)atomicAdd(a.queue + 1, 1ull);
    __syncthreads();
    const long long q = cellidx[0];
    __syncthreads();
    if (q >= a.n) break;
    // queue position q holds the q-th cell of the cost order (most accepted steps first)
    const long long g = a.order ? a.order[q] : q;
    if (g < 0 || g >= a.n) continue;   // an order entry outside [0, n): nothing to do
    // ---- 1. re-integrate, recording the accepted steps ----
    const double p = a.p[g];
    for (int k = tid; k < N; k += kLT) c.Yv[k] = (k < K) ? a.Y0[k * a.ldY + g] : a.T0[g];
    __syncthreads();
    int good = 1;
    for (int k = tid; k < N; k += kLT) good &= isfinite(c.Yv[k]) ? 1 : 0;
    good = block_and(good, c.ired) && isfinite(p) && p > 0.0 && c.Yv[K] > 0.0;
    const double invp = 1.0 / p;
    // self-checkpointing mode: this CTA's checkpoints (S entries of y_n, t_n, the proposed
    // step size and h_n, thinned to every other one whenever full) and segment buffer
    constexpr bool self = SELF;   // self-checkpointing (a.ckpt_S > 0) or the caller's step counts
    const int S = a.ckpt_S;
    double* ck = self ? a.ckpt + (long long)blockIdx.x * S * (N + 3) : nullptr;
    double* sg = self ? a.seg + (long long)blockIdx.x * a.seg_max * (N + 1) : nullptr;
    long long off = 0, cap = 0;
    int status = RDE_CELL_OK;
    if (!self) {
      off = a.offsets[g];
      cap = a.offsets[g + 1] - off;
      if (a.offsets[g + 1] > a.total_steps) status = RDE_CELL_ADJ_MISMATCH;   // no room in the pool
    }
    if (status == RDE_CELL_OK && !good) status = RDE_CELL_BAD_STATE;
    double t = 0.0, h = dt, hp0 = dt;
    long long nrec = 0;
    int attempts = 0, stride = 1;
    bool reject_prev = false;
    while (status == RDE_CELL_OK && dt - t > 1e-14 * dt) {
      if (attempts >= o.max_substeps) {
        status = RDE_CELL_MAX_SUBSTEPS;
        break;
      }
      ++attempts;
      h = fmin(h, dt - t);
      double err;
      int fin;
      if (!adj_large_attempt<SELF>(m, pl, c, invp, h, o, err, fin)) {
        status = RDE_CELL_LU_SINGULAR;
        break;
      }
      if (fin && err <= 1.0) {
        if (self) {
          if ((nrec & (stride - 1)) == 0) {
            long long e = nrec / stride;
            if (e == S) {
              // keep every other entry: round r moves entries [2^(r+1), 2^(r+2)) to
              // [2^r, 2^(r+1)), which no earlier round wrote and no later round reads
              for (int lo = 1; lo < S / 2; lo <<= 1) {
                for (int q = lo * (N + 3) + tid; q < 2 * lo * (N + 3); q += kLT) {
                  const int qe = q / (N + 3), f = q - qe * (N + 3);
                  ck[q] = ck[2 * qe * (N + 3) + f];
                }
                __syncthreads();
              }
              stride <<= 1;
              e = S / 2;
            }
            double* en = ck + e * (N + 3);
            for (int k = tid; k < N + 3; k += kLT)
              en[k] = (k < N) ? c.Yv[k] : (k == N) ? t : (k == N + 1) ? hp0 : h;
          }
        } else if (nrec < cap) {
          double* rec = a.pool + (off + nrec) * (N + 1);
          for (int k = tid; k <= N; k += kLT) rec[k] = (k < N) ? c.Yv[k] : h;
        }
        ++nrec;
        __syncthreads();
        for (int k = tid; k < N; k += kLT) c.Yv[k] = c.U4[k];
        __syncthreads();
        t += h;
        h *= fmin(reject_prev ? 1.0 : o.facmax, fmax(o.facmin, o.safety / cbrt(err)));
        hp0 = h;
        reject_prev = false;
      } else {
        h *= (fin && isfinite(err)) ? fmax(o.facmin, o.safety / cbrt(err)) : o.facmin;
        reject_prev = true;
        if (h < o.hmin) status = RDE_CELL_H_UNDERFLOW;
      }
    }
    if (status == RDE_CELL_OK && !self && nrec != cap) status = RDE_CELL_ADJ_MISMATCH;
    for (int j = tid; j < 2 * R; j += kLT) TH[j] = 0.0;
    for (int k = tid; k < N; k += kLT) LAM[k] = (status != RDE_CELL_OK) ? 0.0 : (k < K) ? a.gY[k * a.ldY + g] : a.gT[g];
    __syncthreads();
    // ---- 2. reverse sweep ----
    const int cs = self ? ckpt_stride((int)nrec, S) : 1;
    long long seg0 = nrec;   // first step the segment buffer holds
    for (long long s = (status == RDE_CELL_OK) ? nrec - 1 : -1; s >= 0; --s) {
      if (self && cs > 1 && s < seg0) {
        // replay segment j from its checkpoint with the record pass's attempt
        const long long j = s / cs;
        const double* en = ck + j * (N + 3);
        for (int k = tid; k < N; k += kLT) c.Yv[k] = en[k];
        double rt = en[N], rh = en[N + 1];
        bool rrej = false;
        const long long target = min((long long)cs, nrec - j * cs);
        long long cnt = 0;
        int tries = 0;
        __syncthreads();
        while (cnt < target && tries++ < o.max_substeps) {
          const double hatt = fmin(rh, dt - rt);
          double err;
          int fin;
          if (!adj_large_attempt<SELF>(m, pl, c, invp, hatt, o, err, fin)) break;
          if (fin && err <= 1.0) {
            double* sq = sg + cnt * (N + 1);
            for (int k = tid; k <= N; k += kLT) sq[k] = (k < N) ? c.Yv[k] : hatt;
            ++cnt;
            __syncthreads();
            for (int k = tid; k < N; k += kLT) c.Yv[k] = c.U4[k];
            __syncthreads();
            rt += hatt;
            rh = hatt * fmin(rrej ? 1.0 : o.facmax, fmax(o.facmin, o.safety / cbrt(err)));
            rrej = false;
          } else {
            rh = hatt * ((fin && isfinite(err)) ? fmax(o.facmin, o.safety / cbrt(err)) : o.facmin);
            rrej = true;
            if (rh < o.hmin) break;
          }
        }
        // the replay must take the segment's steps and end on the next checkpoint, bit for bit
        int same = cnt == target ? 1 : 0;
        if (same && j * cs + cnt < nrec) {
          const double* nx = ck + (j + 1) * (N + 3);
          int ok = 1;
          for (int k = tid; k < N; k += kLT) ok &= __double_as_longlong(nx[k]) == __double_as_longlong(c.Yv[k]);
          same = block_and(ok, c.ired) && nx[N] == rt;
        }
        if (!same) {
          status = RDE_CELL_ADJ_MISMATCH;
          for (int j2 = tid; j2 < 2 * R; j2 += kLT) TH[j2] = 0.0;
          for (int k = tid; k < N; k += kLT) LAM[k] = 0.0;
          __syncthreads();
          break;
        }
        seg0 = j * cs;
      }
      const double* rec = !self ? a.pool + (off + s) * (N + 1)
                                : (cs == 1 ? ck + s * (N + 3) : sg + (s - seg0) * (N + 1));
      for (int k = tid; k < N; k += kLT) c.Yv[k] = rec[k];
      const double hs = (self && cs == 1) ? rec[N + 2] : rec[N];
      const double invh = 1.0 / hs;
      __syncthreads();
      double err;
      int fin;
      large_attempt(m, pl, c, invp, hs, o, err, fin);   // the record pass factorised this matrix
      for (int k = tid; k < N; k += kLT) {
        c.U4[k] = c.VEC[k];   // u_4
        YB[k] = LAM[k];
        UB1[k] = 2.0 * LAM[k];
        UB2[k] = 0.0;
        UB3[k] = LAM[k];
        c.VEC[k] = LAM[k];
      }
      __syncthreads();
      // stage 4: r4 = f(y + 2 u1 + u3) + (u1 - u2 + c43 u3)/h
      solve_block_t(c);
      for (int k = tid; k < N; k += kLT) {
        W[3 * N + k] = c.VEC[k];
        c.ARG[k] = c.Yv[k] + 2.0 * c.U1[k] + c.U3[k];
      }
      __syncthreads();
      jtw_primal(W + 3 * N, invp);
      for (int k = tid; k < N; k += kLT) {
        const double w = W[3 * N + k], gk = GV[k];
        YB[k] += gk;
        UB1[k] += 2.0 * gk + invh * w;
        UB2[k] -= invh * w;
        UB3[k] += gk + (kC43 * invh) * w;
        c.VEC[k] = UB3[k];
      }
      __syncthreads();
      // stage 3: r3 = f(y + 2 u1) + (u1 - u2)/h
      solve_block_t(c);
      for (int k = tid; k < N; k += kLT) {
        W[2 * N + k] = c.VEC[k];
        c.ARG[k] = c.Yv[k] + 2.0 * c.U1[k];
      }
      __syncthreads();
      jtw_primal(W + 2 * N, invp);
      for (int k = tid; k < N; k += kLT) {
        const double w = W[2 * N + k], gk = GV[k];
        YB[k] += gk;
        UB1[k] += 2.0 * gk + invh * w;
        UB2[k] -= invh * w;
        c.VEC[k] = UB2[k];
      }
      __syncthreads();
      // stage 2: r2 = f(y) + (c21/h) u1
      solve_block_t(c);
      for (int k = tid; k < N; k += kLT) {
        const double w = c.VEC[k];
        W[N + k] = w;
        UB1[k] += (kC21 * invh) * w;
        c.VEC[k] = UB1[k];
      }
      __syncthreads();
      // stage 1: r1 = f(y); f(y) enters stages 1 and 2.  Its J(y)^T (w1 + w2) term is
      // the value part of the first dual Jacobian below (also at y)
      solve_block_t(c);
      for (int k = tid; k < N; k += kLT) {
        W[k] = c.VEC[k];
        UB2[k] = c.VEC[k] + W[N + k];
      }
      __syncthreads();
      // M = I/(gamma h) - J(y): terms grad (w_i^T J(y) u_i), two stages per dual Jacobian
      jtw_dual2(c.Yv, c.U1, c.U2, W, W + N, invp, UB2);
      for (int k = tid; k < N; k += kLT) YB[k] += GV[k];
      __syncthreads();
      jtw_dual2(c.Yv, c.U3, c.U4, W + 2 * N, W + 3 * N, invp, nullptr);
      for (int k = tid; k < N; k += kLT) YB[k] += GV[k];
      __syncthreads();
      for (int k = tid; k < N; k += kLT) LAM[k] = YB[k];
      __syncthreads();
    }
    // ---- 3. outputs ----
    for (int k = tid; k < N; k += kLT) {
      if (k < K) a.gY0[k * a.ldY + g] = LAM[k];
      else a.gT0[g] = LAM[k];
    }
    for (int j = tid; j < 2 * R; j += kLT) a.rows[(long long)j * a.n + g] = TH[j];
    if (tid == 0) {
      a.rec[g] = (status == RDE_CELL_OK) ? (int)nrec : -status;
      if (a.status) a.status[g] = status;
    }
    __syncthreads();
  }
}

}  // namespace

size_t large_adjoint_shared_bytes(int K, int R) {
  const int N = K + 1;
  return sizeof(double) * (kExpTabSize + 2 * kLogTabSize) + sizeof(double) * large_adj_doubles(K, R) +
         sizeof(int) * ((size_t)N + 8);
}

cudaError_t prepare_large_adjoint(int K, int R) {
  if (K < 1 || K + 1 > kLargeMaxN) return cudaErrorInvalidConfiguration;
  const size_t smem = large_adjoint_shared_bytes(K, R);
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (smem > (size_t)optin) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(chem_large_adjoint_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chem_large_adjoint_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e;
}

cudaError_t launch_large_adjoint_kernel(const AdjArgs& a, cudaStream_t stream) {
  const size_t smem = large_adjoint_shared_bytes(a.K, a.R);
  const long long grid = max(1LL, min(a.n, (long long)a.num_sms));
  if (a.ckpt_S > 0)
    chem_large_adjoint_kernel<true><<<(unsigned)grid, kLT, smem, stream>>>(a);
  else
    chem_large_adjoint_kernel<false><<<(unsigned)grid, kLT, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace rde
