// Discrete adjoint of the CTA-per-cell chemistry step (large mechanisms, sm_103a,
// FP64): the derivative of (T0, Y0, ln A_r, E_r) -> (T, Y)(dt) along each cell's
// frozen sequence of accepted RODAS3 steps, as in chem_adjoint_body.cuh, for
// mechanisms whose N x N matrix does not fit the thread-per-cell lane slots.
//
// One persistent CTA of 128 threads per cell (work queue).  Per cell it
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
//     derivative term d/de [J(y + e u_i)^T w_i] is the derivative part of the same
//     Jacobian formed with dual numbers along u_i (whose value part, J(y), also
//     serves the stage-1 term);
//  3. writes gY0, gT0 and the cell's parameter rows; the host reduces the rows.
#include <cuda_runtime.h>
#include <stdint.h>

#include "chem_adjoint_body.cuh"
#include "chem_large_block.cuh"

namespace rde {
namespace {

// shared-memory layout (doubles after the exp/log tables), in this order:
//   the forward cell (N LD + 7 K + 9 N + 9 R + 8), the explicit Jacobian MXV (N LD),
//   the dual cell (2 N LD + 14 K + 4 N + 18 R), the adjoint vectors (10 N),
//   the parameter cotangents TH (2 R); then N + 8 ints (permutation, flags)
__host__ __device__ inline size_t large_adj_doubles(int K, int R) {
  const size_t N = (size_t)K + 1, LD = N | 1;
  return N * LD + 7 * (size_t)K + 9 * N + 9 * (size_t)R + 8 + N * LD + 2 * N * LD + 14 * (size_t)K + 4 * N +
         18 * (size_t)R + 10 * N + 2 * (size_t)R;
}

// g = -(MX)^T w over N columns (MX holds -J): thread j sums column j in a fixed order.
// For S = Dual the derivative part is contracted with w and, when wv is given, the
// value part with wv, both into g.
template <class S>
__device__ __forceinline__ void neg_mt_w(const S* MX, int N, int LD, const double* w, double* g,
                                         const double* wv = nullptr) {
  for (int j = threadIdx.x; j < N; j += kLT) {
    double acc = 0.0, accv = 0.0;
    for (int i = 0; i < N; ++i) {
      if constexpr (sizeof(S) == sizeof(double)) {
        acc += val(MX[i * LD + j]) * w[i];
      } else {
        acc += der(MX[i * LD + j]) * w[i];
        if (wv) accv += val(MX[i * LD + j]) * wv[i];
      }
    }
    g[j] = -acc - accv;
  }
}

// w^T df/d(ln A_r) and w^T df/dE_r (value part for S = double, derivative part for
// Dual) added to TH[r], TH[R + r]; reaction r by one thread.  For S = Dual and a
// second weight vector wv, the value part's terms with wv are added as well.  The
// state of the f evaluation: the cell's species arrays and RS after rhs_block, its
// mixture state and temperature.
template <class S>
__device__ void param_terms(const MechView& m, const CellT<S>& c, const MixT<S>& ms, S T, const double* w,
                            double* TH, const double* wv = nullptr) {
  const int K = c.K, R = c.R;
  const S invT = 1.0 / T, lnT = slog(m, T), RT = kRu * T;
  const S facT = (w[K] * RT) / ms.cpm;
  const double facTv = wv ? (wv[K] * val(RT)) / val(ms.cpm) : 0.0;
  for (int r = threadIdx.x; r < R; r += kLT) {
    const RxView x{m.rx[r]};
    S phi = cst<S>(1.0);
    if (x.type() == RX_LINDEMANN || x.type() == RX_TROE) {
      S M = ms.Msum;
      for (int e = x.eff_begin(); e < x.eff_end(); ++e) M += x.eff_am1(m, e) * c.C[x.eff_k(m, e)];
      const S lnk = c.rlnA[r] + c.rb[r] * lnT - c.rEaR[r] * invT;
      S dlnkf, dkf_dM;
      falloff_s<S>(m, x, T, lnT, invT, M, sexp(m, lnk), dlnkf, dkf_dM, phi);
    }
    double s1 = 0.0, s1v = 0.0;
    S s2 = cst<S>(0.0);
    for (int pp = 0; pp < x.np(); ++pp) {
      const int k = x.pi(pp);
      s1 += w[k] * m.sp[k].W * x.pnu(pp);
      if (wv) s1v += wv[k] * m.sp[k].W * x.pnu(pp);
      s2 += x.pnu(pp) * c.HRT[k];
    }
    const S q = c.RS[9 * r + 7];
    const S sr = (s1 - facT * s2) * ms.invrho;
    const S tA = sr * phi * q;
    const S tE = -(tA / RT);
    if constexpr (sizeof(S) == sizeof(double)) {
      TH[r] += val(tA);
      TH[R + r] += val(tE);
    } else {
      double vA = 0.0, vE = 0.0;
      if (wv) {
        vA = (s1v - facTv * val(s2)) * val(ms.invrho) * val(phi) * val(q);
        vE = -(vA / val(RT));
      }
      TH[r] += der(tA) + vA;
      TH[R + r] += der(tE) + vE;
    }
  }
}

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
  // the explicit Jacobian at a stage argument: the forward cell with its own matrix
  Cell cj = c;
  cj.MX = d; d += N * LD;
  // the dual cell (J and its derivative along a stage vector)
  CellT<Dual> dc;
  Dual* dd = reinterpret_cast<Dual*>(d);
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
    param_terms<double>(m, cj, ms, T, w, TH);
    assemble_block<double>(m, cj, T, ms, 0.0);
    neg_mt_w<double>(cj.MX, N, LD, w, GV);
    __syncthreads();
  };
  // g = d/de [J(y + e u)^T w] and the parameter terms' derivative: GV, TH; with wv also
  // J(y)^T wv and its parameter terms from the value part of the same evaluation
  auto jtw_dual = [&](const double* y, const double* u, const double* w, double invp, const double* wv) {
    for (int k = tid; k < N; k += kLT) dc.ARG[k] = mk(y[k], u[k]);
    __syncthreads();
    const MixT<Dual> ms = rhs_block<Dual, true>(m, pl, dc, invp);
    const Dual T = dc.ARG[K];
    param_terms<Dual>(m, dc, ms, T, w, TH, wv);
    assemble_block<Dual>(m, dc, T, ms, mk(0.0, 0.0));
    neg_mt_w<Dual>(dc.MX, N, LD, w, GV, wv);
    __syncthreads();
  };

  for (;;) {
    if (tid == 0) cellidx[0] = (long long)atomicAdd(a.queue + 1, 1ull);
    __syncthreads();
    const long long g = cellidx[0];
    __syncthreads();
    if (g >= a.n) break;
    // ---- 1. re-integrate, recording the accepted steps ----
    const double p = a.p[g];
    for (int k = tid; k < N; k += kLT) c.Yv[k] = (k < K) ? a.Y0[k * a.ldY + g] : a.T0[g];
    __syncthreads();
    int good = 1;
    for (int k = tid; k < N; k += kLT) good &= isfinite(c.Yv[k]) ? 1 : 0;
    good = block_and(good, c.ired) && isfinite(p) && p > 0.0 && c.Yv[K] > 0.0;
    const double invp = 1.0 / p;
    const long long off = a.offsets[g];
    const long long cap = a.offsets[g + 1] - off;
    int status = RDE_CELL_OK;
    if (a.offsets[g + 1] > a.total_steps) status = RDE_CELL_ADJ_MISMATCH;   // no room in the pool
    else if (!good) status = RDE_CELL_BAD_STATE;
    double t = 0.0, h = dt;
    long long nrec = 0;
    int attempts = 0;
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
      if (!large_attempt(m, pl, c, invp, h, o, err, fin)) {
        status = RDE_CELL_LU_SINGULAR;
        break;
      }
      if (fin && err <= 1.0) {
        if (nrec < cap) {
          double* rec = a.pool + (off + nrec) * (N + 1);
          for (int k = tid; k <= N; k += kLT) rec[k] = (k < N) ? c.Yv[k] : h;
        }
        ++nrec;
        __syncthreads();
        for (int k = tid; k < N; k += kLT) c.Yv[k] = c.U4[k];
        __syncthreads();
        t += h;
        h *= fmin(reject_prev ? 1.0 : o.facmax, fmax(o.facmin, o.safety / cbrt(err)));
        reject_prev = false;
      } else {
        h *= (fin && isfinite(err)) ? fmax(o.facmin, o.safety / cbrt(err)) : o.facmin;
        reject_prev = true;
        if (h < o.hmin) status = RDE_CELL_H_UNDERFLOW;
      }
    }
    if (status == RDE_CELL_OK && nrec != cap) status = RDE_CELL_ADJ_MISMATCH;
    for (int j = tid; j < 2 * R; j += kLT) TH[j] = 0.0;
    for (int k = tid; k < N; k += kLT) LAM[k] = (status != RDE_CELL_OK) ? 0.0 : (k < K) ? a.gY[k * a.ldY + g] : a.gT[g];
    __syncthreads();
    // ---- 2. reverse sweep ----
    for (long long s = (status == RDE_CELL_OK) ? nrec - 1 : -1; s >= 0; --s) {
      const double* rec = a.pool + (off + s) * (N + 1);
      for (int k = tid; k < N; k += kLT) c.Yv[k] = rec[k];
      const double hs = rec[N];
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
      // M = I/(gamma h) - J(y): terms grad (w_i^T J(y) u_i), one dual Jacobian per stage
      const double* Us[4] = {c.U1, c.U2, c.U3, c.U4};
      for (int st = 0; st < 4; ++st) {
        jtw_dual(c.Yv, Us[st], W + st * N, invp, st == 0 ? UB2 : nullptr);
        for (int k = tid; k < N; k += kLT) YB[k] += GV[k];
        __syncthreads();
      }
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
  return cudaFuncSetAttribute(chem_large_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_large_adjoint_kernel(const AdjArgs& a, cudaStream_t stream) {
  const size_t smem = large_adjoint_shared_bytes(a.K, a.R);
  const long long grid = max(1LL, min(a.n, (long long)a.num_sms));
  chem_large_adjoint_kernel<<<(unsigned)grid, kLT, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace rde
