/*
 * Complex-step tangent of the oracle's frozen-step integration.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.c).  The discrete adjoint of the
 * chemistry step differentiates the map from (T0, Y0, ln A_r, E_r) to the final
 * state along a frozen sequence of accepted Rosenbrock steps (the step sizes do
 * not vary).  This file evaluates that same map in complex arithmetic: with
 * inputs x + i*eps*dx, the imaginary part of the output divided by eps is the
 * exact directional derivative (complex-step differentiation, Squire & Trapp
 * 1998): no subtraction, hence no cancellation error.  The reactor model, its
 * analytic Jacobian and the RODAS3 step are the oracle's formulas written out
 * again on `double complex`; because the analytic Jacobian is an analytic
 * function of the state, evaluating it at a complex state carries the
 * Jacobian's own dependence on the state (the second-derivative terms of the
 * discrete adjoint) into the imaginary part.  Comparisons (NASA range, pivot
 * search, Troe floor) use real parts.  Parameters per reaction: ln A (of k_inf
 * for falloff reactions) and E in J/mol.
 *
 * Pins: tests/test_oracle_tangent.py checks the tangent against central finite
 * differences of the real replay (orc_replay) and against the closed-form
 * derivative of first-order kinetics.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define RU 8.31446261815324
#define PSTD 101325.0

typedef double complex cx;

static const double GAMMA_ = 0.5;
static const double A_[4][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {2, 0, 0, 0}, {2, 0, 1, 0}};
static const double C_[4][4] = {{0, 0, 0, 0}, {4, 0, 0, 0}, {1, -1, 0, 0}, {1, -1, -8.0 / 3.0, 0}};
static const double M_[4] = {2, 0, 1, 1};

static const double *nasa_c(const orc_mech *m, int k, cx T)
{
    return (creal(T) < m->Tmid[k]) ? m->lo + 7 * k : m->hi + 7 * k;
}

static cx cp_c(const double *a, cx T) { return a[0] + a[1] * T + a[2] * T * T + a[3] * T * T * T + a[4] * T * T * T * T; }
static cx h_c(const double *a, cx T)
{
    return a[0] + a[1] * T / 2 + a[2] * T * T / 3 + a[3] * T * T * T / 4 + a[4] * T * T * T * T / 5 + a[5] / T;
}
static cx s_c(const double *a, cx T)
{
    return a[0] * clog(T) + a[1] * T + a[2] * T * T / 2 + a[3] * T * T * T / 3 + a[4] * T * T * T * T / 4 + a[6];
}
static cx dcp_c(const double *a, cx T) { return a[1] + 2 * a[2] * T + 3 * a[3] * T * T + 4 * a[4] * T * T * T; }

typedef struct {
    const orc_mech *m;
    const cx *A;     /* per reaction: (perturbed) pre-factor of k, k_inf for falloff */
    const cx *EaR;   /* per reaction: (perturbed) E / R_u */
} cmech;

typedef struct { cx kf, kr, dkf_dT, dkr_dT, dkf_dM; } crate_t;

static cx arrh_c(cx A, double b, cx EaR, cx T) { return A * cexp(b * clog(T)) * cexp(-EaR / T); }

static crate_t rates_c(const cmech *cm, int r, cx T, cx M)
{
    const orc_mech *m = cm->m;
    const int K = m->K;
    crate_t o;
    cx kinf = arrh_c(cm->A[r], m->b[r], cm->EaR[r], T);
    cx dlnkinf = m->b[r] / T + cm->EaR[r] / (T * T);
    cx kf = kinf, dlnkf = dlnkinf, dkf_dM = 0.0;
    if (m->type[r] == RX_LINDEMANN || m->type[r] == RX_TROE) {
        cx k0 = arrh_c(m->A0[r], m->b0[r], m->EaR0[r], T);
        cx dlnk0 = m->b0[r] / T + m->EaR0[r] / (T * T);
        cx Pr = k0 * M / kinf;
        cx dlnPr = dlnk0 - dlnkinf;
        cx F = 1.0, D = 0.0, dlnF_T = 0.0;
        if (m->type[r] == RX_TROE) {
            const double *tp = m->troe + 4 * r;
            double a = tp[0], T3 = tp[1], T1 = tp[2], T2 = tp[3];
            cx Fc = (1 - a) * cexp(-T / T3) + a * cexp(-T / T1);
            cx dFc = -(1 - a) / T3 * cexp(-T / T3) - a / T1 * cexp(-T / T1);
            if (m->ntroe[r] == 4) { Fc += cexp(-T2 / T); dFc += T2 / (T * T) * cexp(-T2 / T); }
            cx Lc = clog(Fc) / log(10.0), dLc = dFc / (Fc * log(10.0));
            cx c = -0.4 - 0.67 * Lc, n = 0.75 - 1.27 * Lc;
            double d = 0.14;
            cx L = clog(creal(Pr) > 1e-300 ? Pr : 1e-300) / log(10.0);
            cx u = L + c, den = n - d * u, X = u / den;
            cx logF = Lc / (1.0 + X * X);
            F = cexp(log(10.0) * logF);
            cx dX_du = n / (den * den);
            D = -Lc * 2.0 * X / ((1.0 + X * X) * (1.0 + X * X)) * dX_du;
            cx du_dT = -0.67 * dLc, dn_dT = -1.27 * dLc;
            cx dX_dT = (du_dT * den - u * (dn_dT - d * du_dT)) / (den * den);
            cx dlogF_dT = dLc / (1.0 + X * X) - Lc * 2.0 * X / ((1.0 + X * X) * (1.0 + X * X)) * dX_dT;
            dlnF_T = log(10.0) * dlogF_dT;
        }
        kf = kinf * Pr / (1.0 + Pr) * F;
        dlnkf = dlnkinf + dlnF_T + D * dlnPr + dlnPr / (1.0 + Pr);
        dkf_dM = k0 * F / (1.0 + Pr) * (D + 1.0 / (1.0 + Pr));
    }
    o.kf = kf;
    o.dkf_dT = kf * dlnkf;
    o.dkf_dM = dkf_dM;
    if (m->rev[r]) {
        cx sum_g = 0.0, sum_h = 0.0;
        int dnu = 0;
        for (int k = 0; k < K; ++k) {
            int nu = m->nur[r * K + k] - m->nuf[r * K + k];
            if (nu == 0) continue;
            const double *a = nasa_c(m, k, T);
            sum_g += nu * (s_c(a, T) - h_c(a, T));
            sum_h += nu * h_c(a, T);
            dnu += nu;
        }
        cx Kc = cexp(sum_g) * cpow(PSTD / (RU * T), dnu);
        cx dlnKc = (sum_h - dnu) / T;
        o.kr = kf / Kc;
        o.dkr_dT = o.kr * (dlnkf - dlnKc);
    } else {
        o.kr = 0.0;
        o.dkr_dT = 0.0;
    }
    return o;
}

static cx prod_c(int K, const int *nu, const cx *c)
{
    cx P = 1.0;
    for (int j = 0; j < K; ++j)
        for (int e = 0; e < nu[j]; ++e) P *= c[j];
    return P;
}

static cx dprod_c(int K, const int *nu, const cx *c, int j)
{
    if (nu[j] == 0) return 0.0;
    cx P = nu[j];
    for (int i = 0; i < K; ++i) {
        int e = (i == j) ? nu[i] - 1 : nu[i];
        for (int t = 0; t < e; ++t) P *= c[i];
    }
    return P;
}

/* f and (if J != NULL) the analytic Jacobian, in complex arithmetic */
static void rhs_jac_c(const cmech *cm, double p, const cx *y, cx *f, cx *J, cx *wk)
{
    const orc_mech *m = cm->m;
    const int K = m->K, R = m->R, N = K + 1;
    const cx T = y[K];
    cx *c = wk, *wdot = c + K, *Hm = wdot + K, *Cpm = Hm + K, *wT = Cpm + K, *Dc = wT + K, *dq = Dc + K;
    cx *D = dq + K;
    cx sumYW = 0.0, cp = 0.0, dcp = 0.0;
    for (int k = 0; k < K; ++k) sumYW += y[k] / m->W[k];
    cx rho = p / (RU * T * sumYW);
    cx Wbar = 1.0 / sumYW;
    for (int k = 0; k < K; ++k) {
        const double *a = nasa_c(m, k, T);
        c[k] = rho * y[k] / m->W[k];
        Hm[k] = RU * T * h_c(a, T);
        Cpm[k] = RU * cp_c(a, T);
        cp += y[k] * Cpm[k] / m->W[k];
        dcp += y[k] * RU * dcp_c(a, T) / m->W[k];
        wdot[k] = 0.0;
        wT[k] = 0.0;
    }
    if (J) for (int i = 0; i < K * K; ++i) D[i] = 0.0;
    for (int r = 0; r < R; ++r) {
        const int *nuf = m->nuf + r * K, *nur = m->nur + r * K;
        const double *eff = m->eff + r * K;
        cx M = 0.0;
        if (m->type[r] != RX_ELEM)
            for (int k = 0; k < K; ++k) M += eff[k] * c[k];
        crate_t rc = rates_c(cm, r, T, M);
        cx Pf = prod_c(K, nuf, c), Pb = prod_c(K, nur, c);
        cx q0 = rc.kf * Pf - rc.kr * Pb;
        cx q = (m->type[r] == RX_THREEBODY) ? M * q0 : q0;
        for (int k = 0; k < K; ++k) wdot[k] += (nur[k] - nuf[k]) * q;
        if (!J) continue;
        cx dqdT = rc.dkf_dT * Pf - rc.dkr_dT * Pb;
        for (int j = 0; j < K; ++j) dq[j] = rc.kf * dprod_c(K, nuf, c, j) - rc.kr * dprod_c(K, nur, c, j);
        if (m->type[r] == RX_THREEBODY) {
            for (int j = 0; j < K; ++j) dq[j] = M * dq[j] + eff[j] * q0;
            dqdT *= M;
        } else if (m->type[r] == RX_LINDEMANN || m->type[r] == RX_TROE) {
            cx ratio = (creal(rc.kf) != 0.0) ? q0 / rc.kf : 0.0;
            for (int j = 0; j < K; ++j) dq[j] += eff[j] * rc.dkf_dM * ratio;
        }
        for (int k = 0; k < K; ++k) {
            int nu = nur[k] - nuf[k];
            if (nu == 0) continue;
            wT[k] += nu * dqdT;
            for (int j = 0; j < K; ++j) D[k * K + j] += nu * dq[j];
        }
    }
    cx Q = 0.0;
    for (int k = 0; k < K; ++k) {
        f[k] = m->W[k] * wdot[k] / rho;
        Q += Hm[k] * wdot[k];
    }
    cx fT = -Q / (rho * cp);
    f[K] = fT;
    if (!J) return;
    for (int k = 0; k < K; ++k) {
        Dc[k] = 0.0;
        for (int j = 0; j < K; ++j) Dc[k] += D[k * K + j] * c[j];
    }
    cx HDc = 0.0, Cw = 0.0, HwT = 0.0;
    for (int k = 0; k < K; ++k) { HDc += Hm[k] * Dc[k]; Cw += Cpm[k] * wdot[k]; HwT += Hm[k] * (wT[k] - Dc[k] / T); }
    for (int k = 0; k < K; ++k) {
        for (int i = 0; i < K; ++i)
            J[k * N + i] = m->W[k] / m->W[i] * D[k * K + i] + m->W[k] * Wbar / (m->W[i] * rho) * (wdot[k] - Dc[k]);
        J[k * N + K] = m->W[k] / rho * (wT[k] + (wdot[k] - Dc[k]) / T);
    }
    for (int i = 0; i < K; ++i) {
        cx HD = 0.0;
        for (int k = 0; k < K; ++k) HD += Hm[k] * D[k * K + i];
        cx dQ = rho / m->W[i] * HD - Wbar / m->W[i] * HDc;
        J[K * N + i] = -dQ / (rho * cp) - fT / m->W[i] * (Cpm[i] - cp * Wbar) / cp;
    }
    J[K * N + K] = -(Cw + HwT) / (rho * cp) + fT / T - fT * dcp / cp;
}

static int lu_factor_c(int N, cx *a, int *piv)
{
    for (int k = 0; k < N; ++k) {
        int p = k;
        double amax = fabs(creal(a[k * N + k]));
        for (int i = k + 1; i < N; ++i)
            if (fabs(creal(a[i * N + k])) > amax) { amax = fabs(creal(a[i * N + k])); p = i; }
        piv[k] = p;
        if (amax == 0.0) return -1;
        if (p != k)
            for (int j = 0; j < N; ++j) { cx t = a[k * N + j]; a[k * N + j] = a[p * N + j]; a[p * N + j] = t; }
        for (int i = k + 1; i < N; ++i) {
            a[i * N + k] /= a[k * N + k];
            for (int j = k + 1; j < N; ++j) a[i * N + j] -= a[i * N + k] * a[k * N + j];
        }
    }
    return 0;
}

static void lu_solve_c(int N, const cx *a, const int *piv, cx *x)
{
    for (int k = 0; k < N; ++k)
        if (piv[k] != k) { cx t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < i; ++j) x[i] -= a[i * N + j] * x[j];
    for (int i = N - 1; i >= 0; --i) {
        for (int j = i + 1; j < N; ++j) x[i] -= a[i * N + j] * x[j];
        x[i] /= a[i * N + i];
    }
}

/* One RODAS3 step of size h in complex arithmetic; y advanced in place. */
static int step_c(const cmech *cm, double p, cx *y, double h, cx *wk)
{
    const int K = cm->m->K, N = K + 1;
    cx *f0 = wk, *J = f0 + N, *Mx = J + N * N, *u = Mx + N * N, *ys = u + 4 * N, *rw = ys + N;
    int *piv = malloc(sizeof(int) * N);
    rhs_jac_c(cm, p, y, f0, J, rw);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) Mx[i * N + j] = -J[i * N + j] + (i == j ? 1.0 / (GAMMA_ * h) : 0.0);
    if (lu_factor_c(N, Mx, piv)) { free(piv); return -1; }
    for (int s = 0; s < 4; ++s) {
        cx *us = u + s * N;
        int newf = 0;
        for (int j = 0; j < s; ++j) if (A_[s][j] != 0.0) newf = 1;
        if (!newf) {
            memcpy(us, f0, sizeof(cx) * N);
        } else {
            for (int i = 0; i < N; ++i) {
                ys[i] = y[i];
                for (int j = 0; j < s; ++j) ys[i] += A_[s][j] * u[j * N + i];
            }
            rhs_jac_c(cm, p, ys, us, NULL, rw);
        }
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < s; ++j) us[i] += C_[s][j] / h * u[j * N + i];
        lu_solve_c(N, Mx, piv, us);
    }
    for (int i = 0; i < N; ++i)
        for (int s = 0; s < 4; ++s) y[i] += M_[s] * u[s * N + i];
    free(piv);
    return 0;
}

/*
 * Directional derivative of the frozen-step map.
 *   y0 [N], dy0 [N]: state (Y_0..Y_{K-1}, T) and its perturbation direction
 *   dlnA [R], dE [R]: perturbation direction of ln A_r and E_r (J/mol); may be NULL
 *   h_list [nsteps]: the frozen accepted step sizes
 *   y_out [N]: the (real) end state;  dy_out [N]: its directional derivative
 */
int orc_tangent(const orc_mech *m, double p, const double *y0, const double *dy0, const double *dlnA,
                const double *dE, const double *h_list, int nsteps, double *y_out, double *dy_out)
{
    const int K = m->K, R = m->R, N = K + 1;
    const double eps = 1e-20;
    cx *A = malloc(sizeof(cx) * R), *EaR = malloc(sizeof(cx) * R);
    for (int r = 0; r < R; ++r) {
        A[r] = m->A[r] * cexp(I * eps * (dlnA ? dlnA[r] : 0.0));
        EaR[r] = m->EaR[r] + I * eps * (dE ? dE[r] : 0.0) / RU;
    }
    cmech cm = {m, A, EaR};
    cx *y = malloc(sizeof(cx) * N);
    for (int i = 0; i < N; ++i) y[i] = y0[i] + I * eps * (dy0 ? dy0[i] : 0.0);
    size_t wk_n = (size_t)N + 2 * (size_t)N * N + 4 * (size_t)N + N + 7 * (size_t)K + (size_t)K * K;
    cx *wk = malloc(sizeof(cx) * wk_n);
    int rc = 0;
    for (int s = 0; s < nsteps && rc == 0; ++s) rc = step_c(&cm, p, y, h_list[s], wk);
    for (int i = 0; i < N; ++i) {
        y_out[i] = creal(y[i]);
        dy_out[i] = cimag(y[i]) / eps;
    }
    free(wk); free(y); free(A); free(EaR);
    return rc;
}
