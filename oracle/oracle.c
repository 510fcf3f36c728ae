/*
 * CPU oracle for the per-cell chemistry step: serial, FP64, plain C.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of the benchmark load this file's library.  It shares no code, header,
 * table or helper with the CUDA library; it reads the mechanism through its
 * own parser (oracle/mech.py) and is written to be checked by eye against the
 * formulas below, not to be fast.
 *
 * What it computes.  The paper integrates the species and energy equations
 * (Appendix A, Eqs. 20-21) with an operator-split "detailed chemistry model"
 * (Section 2.1).  The chemical source terms omega_dot_i (Eq. 21) and the heat
 * release Q_dot (Eq. 20) are advanced per cell over one flow time step dt as a
 * closed, adiabatic, constant-pressure homogeneous reactor:
 *
 *   dY_k/dt = W_k omega_dot_k / rho
 *   dT/dt   = - sum_k H_k omega_dot_k / (rho c_p)
 *
 * with mass-action kinetics (Arrhenius forward rates, reverse rates from NASA-7
 * equilibrium constants, three-body and Lindemann/Troe falloff terms), an
 * analytic Jacobian, a dense LU with partial pivoting and an adaptive, L-stable
 * Rosenbrock method (RODAS3, Sandu et al. 1997, 4 stages, order 3 with an
 * embedded order-2 estimate) under per-cell error control.
 *
 * Readings where the paper is silent (it names no solver, prints no mechanism):
 *   - standard pressure 101325 Pa; R_u = 8.31446261815324 J/(mol K)
 *   - NASA-7 low range for T < Tmid, high range for T >= Tmid, no clamping
 *   - Troe blending in the Gilbert-Luther-Troe form, log10 of the reduced
 *     pressure taken at max(Pr, 1e-300)
 *   - RMS error norm over the K+1 unknowns, scale atol + rtol max(|y|, |y_new|)
 *   - step factor 0.9 err^(-1/3) bounded to [0.2, 5] (upper bound 1 right after
 *     a rejection); a non-finite error estimate is a rejection with factor 0.2
 *   - J and f(y_n) are evaluated once per accepted state and reused on rejection
 *   - no clipping of Y or of concentrations anywhere
 *
 * A third method (method 2) integrates the same reactor with a linearly implicit
 * Euler extrapolation of fixed order 3 (the SEULEX family), the comparison method
 * of a different family (extrapolation rather than Rosenbrock stages).
 *
 * Parity status: every function below is pinned by a test against closed forms,
 * invariants, finite differences, a brute-force Gibbs minimisation or a library
 * integrator; see tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define RU 8.31446261815324   /* J/(mol K) */
#define PSTD 101325.0         /* Pa */

#include "oracle.h"

/* ------------------------------------------------------------------------- */
/* Rosenbrock tableaus in the transformed Hairer-Wanner form:                 */
/*  (I/(h gamma) - J) u_i = f(y + sum_j a_ij u_j) + sum_j (c_ij / h) u_j      */
/*  y_new = y + sum_i m_i u_i ;  error estimate = sum_i e_i u_i               */
/* Method 0, RODAS3 (Sandu et al. 1997): 4 stages, order 3, embedded order 2. */
/* Method 1, ROS2: 2 stages, order 2, embedded order 1 (y + k_1), L-stable;   */
/*   classical parameters gamma = 1 - 1/sqrt(2), alpha21 = 1,                 */
/*   beta21 = 1 - 2 gamma, b = (1/2, 1/2); transformed: a21 = 1/gamma,       */
/*   c21 = (beta21 - alpha21)/gamma^2, m = b Gamma^-1, e = (b - (1,0)) Gamma^-1 */
/* ------------------------------------------------------------------------- */
typedef struct {
    int stages, qhat;          /* stage count, order of the embedded estimate */
    double gamma;
    double a[4][4], c[4][4], m[4], e[4];
} orc_method;

static const orc_method METHODS[2] = {
    {4, 2, 0.5,
     {{0, 0, 0, 0}, {0, 0, 0, 0}, {2, 0, 0, 0}, {2, 0, 1, 0}},
     {{0, 0, 0, 0}, {4, 0, 0, 0}, {1, -1, 0, 0}, {1, -1, -8.0 / 3.0, 0}},
     {2, 0, 1, 1},
     {0, 0, 0, 1}},
    {2, 1, 0.29289321881345248,
     {{0, 0, 0, 0}, {3.4142135623730949, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
     {{0, 0, 0, 0}, {-6.8284271247461898, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
     {5.1213203435596428, 1.7071067811865475, 0, 0},
     {1.7071067811865475, 1.7071067811865475, 0, 0}},
};

/* the tableau of method k; the extrapolation method (2) has no tableau, and its error
   estimate has order 2 like RODAS3's, so it shares RODAS3's controller exponent 1/3 */
static const orc_method *method_of(int k) { return &METHODS[(k == 1) ? 1 : 0]; }

/* the RODAS3 tableau (4 x 4 arrays) */
void orc_tableau(double *gamma, double *a, double *c, double *m, double *e)
{
    const orc_method *t = method_of(0);
    *gamma = t->gamma;
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) { a[4 * i + j] = t->a[i][j]; c[4 * i + j] = t->c[i][j]; }
        m[i] = t->m[i];
        e[i] = t->e[i];
    }
}

/* any method's tableau; returns its stage count and the order of its error estimate */
int orc_tableau_method(int method, double *gamma, double *a, double *c, double *m, double *e, int *qhat)
{
    const orc_method *t = method_of(method);
    *gamma = t->gamma;
    *qhat = t->qhat;
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) { a[4 * i + j] = t->a[i][j]; c[4 * i + j] = t->c[i][j]; }
        m[i] = t->m[i];
        e[i] = t->e[i];
    }
    return t->stages;
}

/* ------------------------------------------------------------------------- */
/* NASA-7 thermodynamics (dimensionless): Cp/R, H/(R T), S/R, d(Cp/R)/dT      */
/* ------------------------------------------------------------------------- */
static const double *nasa(const orc_mech *m, int k, double T)
{
    return (T < m->Tmid[k]) ? m->lo + 7 * k : m->hi + 7 * k;
}

static double cp_R(const double *a, double T)
{
    return a[0] + a[1] * T + a[2] * T * T + a[3] * T * T * T + a[4] * T * T * T * T;
}

static double h_RT(const double *a, double T)
{
    return a[0] + a[1] * T / 2 + a[2] * T * T / 3 + a[3] * T * T * T / 4 + a[4] * T * T * T * T / 5 + a[5] / T;
}

static double s_R(const double *a, double T)
{
    return a[0] * log(T) + a[1] * T + a[2] * T * T / 2 + a[3] * T * T * T / 3 + a[4] * T * T * T * T / 4 + a[6];
}

static double dcpR_dT(const double *a, double T)
{
    return a[1] + 2 * a[2] * T + 3 * a[3] * T * T + 4 * a[4] * T * T * T;
}

int orc_thermo(const orc_mech *m, int k, double T, double *cp, double *h, double *s)
{
    const double *a = nasa(m, k, T);
    *cp = cp_R(a, T);
    *h = h_RT(a, T);
    *s = s_R(a, T);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Rate constants of reaction r at temperature T and third-body conc. M.      */
/* Returns k_f, k_r and their T-derivatives (at fixed M), plus dk_f/dM.       */
/* ------------------------------------------------------------------------- */
typedef struct { double kf, kr, dkf_dT, dkr_dT, dkf_dM; } rate_t;

static double arrhenius(double A, double b, double EaR, double T) { return A * pow(T, b) * exp(-EaR / T); }

static rate_t rate_constants(const orc_mech *m, int r, double T, double M)
{
    rate_t o;
    const int K = m->K;
    double kinf = arrhenius(m->A[r], m->b[r], m->EaR[r], T);
    double dlnkinf = m->b[r] / T + m->EaR[r] / (T * T);
    double kf = kinf, dlnkf = dlnkinf, dkf_dM = 0.0;

    if (m->type[r] == RX_LINDEMANN || m->type[r] == RX_TROE) {
        double k0 = arrhenius(m->A0[r], m->b0[r], m->EaR0[r], T);
        double dlnk0 = m->b0[r] / T + m->EaR0[r] / (T * T);
        double Pr = k0 * M / kinf;                 /* reduced pressure */
        double dlnPr = dlnk0 - dlnkinf;            /* d ln Pr / dT at fixed M */
        double F = 1.0, D = 0.0, dlnF_T = 0.0;     /* D = d log10 F / d log10 Pr */
        if (m->type[r] == RX_TROE) {
            const double *tp = m->troe + 4 * r;
            double a = tp[0], T3 = tp[1], T1 = tp[2], T2 = tp[3];
            double Fc = (1 - a) * exp(-T / T3) + a * exp(-T / T1);
            double dFc = -(1 - a) / T3 * exp(-T / T3) - a / T1 * exp(-T / T1);
            if (m->ntroe[r] == 4) { Fc += exp(-T2 / T); dFc += T2 / (T * T) * exp(-T2 / T); }
            double Lc = log10(Fc), dLc = dFc / (Fc * log(10.0));
            double c = -0.4 - 0.67 * Lc, n = 0.75 - 1.27 * Lc, d = 0.14;
            double L = log10(fmax(Pr, 1e-300));
            double u = L + c, den = n - d * u, X = u / den;
            double logF = Lc / (1 + X * X);
            F = pow(10.0, logF);
            /* derivatives of log10 F */
            double dX_du = n / (den * den);
            D = -Lc * 2 * X / ((1 + X * X) * (1 + X * X)) * dX_du;
            double du_dT = -0.67 * dLc, dn_dT = -1.27 * dLc;
            double dX_dT = (du_dT * den - u * (dn_dT - d * du_dT)) / (den * den);  /* at fixed L */
            double dlogF_dT = dLc / (1 + X * X) - Lc * 2 * X / ((1 + X * X) * (1 + X * X)) * dX_dT;
            dlnF_T = log(10.0) * dlogF_dT;
        }
        kf = kinf * Pr / (1 + Pr) * F;
        /* ln kf = ln kinf + ln F + ln Pr - ln(1 + Pr); F depends on T directly and through Pr */
        double dlnF = dlnF_T + D * dlnPr;
        dlnkf = dlnkinf + dlnF + dlnPr / (1 + Pr);
        dkf_dM = k0 * F / (1 + Pr) * (D + 1 / (1 + Pr));
    }
    o.kf = kf;
    o.dkf_dT = kf * dlnkf;
    o.dkf_dM = dkf_dM;
    if (m->rev[r]) {
        /* K_c = exp(sum_k nu_k (S_k/R - H_k/RT)) (P_std / (R_u T))^(sum_k nu_k) */
        double sum_g = 0.0, sum_h = 0.0;
        int dnu = 0;
        for (int k = 0; k < K; ++k) {
            int nu = m->nur[r * K + k] - m->nuf[r * K + k];
            if (nu == 0) continue;
            const double *a = nasa(m, k, T);
            sum_g += nu * (s_R(a, T) - h_RT(a, T));
            sum_h += nu * h_RT(a, T);
            dnu += nu;
        }
        double Kc = exp(sum_g) * pow(PSTD / (RU * T), dnu);
        double dlnKc = (sum_h - dnu) / T;          /* van 't Hoff */
        o.kr = kf / Kc;
        o.dkr_dT = o.kr * (dlnkf - dlnKc);
    } else {
        o.kr = 0.0;
        o.dkr_dT = 0.0;
    }
    return o;
}

/* product of c_j^nu_j and its derivative with respect to c_j */
static double conc_product(int K, const int *nu, const double *c)
{
    double P = 1.0;
    for (int j = 0; j < K; ++j)
        for (int e = 0; e < nu[j]; ++e) P *= c[j];
    return P;
}

static double conc_product_deriv(int K, const int *nu, const double *c, int j)
{
    if (nu[j] == 0) return 0.0;
    double P = nu[j];
    for (int i = 0; i < K; ++i) {
        int e = (i == j) ? nu[i] - 1 : nu[i];
        for (int t = 0; t < e; ++t) P *= c[i];
    }
    return P;
}

/* ------------------------------------------------------------------------- */
/* Source terms and analytic Jacobian.  y = (Y_0 .. Y_{K-1}, T).              */
/* J (optional, row-major N x N) = d f / d y.                                 */
/* ------------------------------------------------------------------------- */
static int rhs_jac(const orc_mech *m, double p, const double *y, double *f, double *J, double *wk)
{
    const int K = m->K, R = m->R, N = K + 1;
    const double T = y[K];
    double *c = wk, *wdot = c + K, *Hm = wdot + K, *Cpm = Hm + K, *wT = Cpm + K, *Dc = wT + K, *dq = Dc + K;
    double *D = dq + K;  /* [K][K] d omega_dot / d c (fixed T) */

    /* mixture: sum_k Y_k / W_k, density, concentrations, c_p */
    double sumYW = 0.0, cp = 0.0, dcp = 0.0;
    for (int k = 0; k < K; ++k) sumYW += y[k] / m->W[k];
    double rho = p / (RU * T * sumYW);
    double Wbar = 1.0 / sumYW;
    for (int k = 0; k < K; ++k) {
        const double *a = nasa(m, k, T);
        c[k] = rho * y[k] / m->W[k];
        Hm[k] = RU * T * h_RT(a, T);               /* J/mol */
        Cpm[k] = RU * cp_R(a, T);                  /* J/(mol K) */
        cp += y[k] * Cpm[k] / m->W[k];
        dcp += y[k] * RU * dcpR_dT(a, T) / m->W[k];
        wdot[k] = 0.0;
        wT[k] = 0.0;
    }
    if (J) memset(D, 0, sizeof(double) * K * K);

    for (int r = 0; r < R; ++r) {
        const int *nuf = m->nuf + r * K, *nur = m->nur + r * K;
        const double *eff = m->eff + r * K;
        double M = 0.0;
        if (m->type[r] != RX_ELEM)
            for (int k = 0; k < K; ++k) M += eff[k] * c[k];
        rate_t rc = rate_constants(m, r, T, M);
        double Pf = conc_product(K, nuf, c), Pb = conc_product(K, nur, c);
        double q0 = rc.kf * Pf - rc.kr * Pb;
        double q = (m->type[r] == RX_THREEBODY) ? M * q0 : q0;
        for (int k = 0; k < K; ++k) wdot[k] += (nur[k] - nuf[k]) * q;
        if (!J) continue;

        /* d q / d c_j at fixed T, and d q / dT at fixed c */
        double dqdT = rc.dkf_dT * Pf - rc.dkr_dT * Pb;
        for (int j = 0; j < K; ++j)
            dq[j] = rc.kf * conc_product_deriv(K, nuf, c, j) - rc.kr * conc_product_deriv(K, nur, c, j);
        if (m->type[r] == RX_THREEBODY) {
            for (int j = 0; j < K; ++j) dq[j] = M * dq[j] + eff[j] * q0;
            dqdT *= M;
        } else if (m->type[r] == RX_LINDEMANN || m->type[r] == RX_TROE) {
            /* k_f and k_r = k_f / K_c both scale with d k_f / d M */
            double ratio = (rc.kf != 0.0) ? q0 / rc.kf : 0.0;   /* Pf - Pb / K_c */
            for (int j = 0; j < K; ++j) dq[j] += eff[j] * rc.dkf_dM * ratio;
        }
        for (int k = 0; k < K; ++k) {
            int nu = nur[k] - nuf[k];
            if (nu == 0) continue;
            wT[k] += nu * dqdT;
            for (int j = 0; j < K; ++j) D[k * K + j] += nu * dq[j];
        }
    }

    /* f */
    double Q = 0.0;
    for (int k = 0; k < K; ++k) {
        f[k] = m->W[k] * wdot[k] / rho;
        Q += Hm[k] * wdot[k];
    }
    double fT = -Q / (rho * cp);
    f[K] = fT;
    if (!J) return 0;

    /* chain rule from (c, T) to (Y, T):
       dc_j/dY_i = rho/W_j delta_ij - c_j Wbar / W_i ;  dc_j/dT = -c_j / T        */
    for (int k = 0; k < K; ++k) {
        Dc[k] = 0.0;
        for (int j = 0; j < K; ++j) Dc[k] += D[k * K + j] * c[j];
    }
    double HDc = 0.0, Cw = 0.0, HwT = 0.0;
    for (int k = 0; k < K; ++k) { HDc += Hm[k] * Dc[k]; Cw += Cpm[k] * wdot[k]; HwT += Hm[k] * (wT[k] - Dc[k] / T); }
    for (int k = 0; k < K; ++k) {
        for (int i = 0; i < K; ++i)
            J[k * N + i] = m->W[k] / m->W[i] * D[k * K + i]
                         + m->W[k] * Wbar / (m->W[i] * rho) * (wdot[k] - Dc[k]);
        J[k * N + K] = m->W[k] / rho * (wT[k] + (wdot[k] - Dc[k]) / T);
    }
    for (int i = 0; i < K; ++i) {
        double HD = 0.0;
        for (int k = 0; k < K; ++k) HD += Hm[k] * D[k * K + i];
        double dQ = rho / m->W[i] * HD - Wbar / m->W[i] * HDc;
        J[K * N + i] = -dQ / (rho * cp) - fT / m->W[i] * (Cpm[i] - cp * Wbar) / cp;
    }
    J[K * N + K] = -(Cw + HwT) / (rho * cp) + fT / T - fT * dcp / cp;
    (void)N;
    return 0;
}

static size_t rhs_work_doubles(int K) { return (size_t)7 * K + (size_t)K * K; }

int orc_rhs(const orc_mech *m, double p, const double *y, double *f)
{
    double *wk = malloc(sizeof(double) * rhs_work_doubles(m->K));
    rhs_jac(m, p, y, f, NULL, wk);
    free(wk);
    return 0;
}

int orc_jac(const orc_mech *m, double p, const double *y, double *f, double *J)
{
    double *wk = malloc(sizeof(double) * rhs_work_doubles(m->K));
    rhs_jac(m, p, y, f, J, wk);
    free(wk);
    return 0;
}

/* k_f, k_r and rates of progress q_r at state y (tests) */
int orc_rates(const orc_mech *m, double p, const double *y, double *kf, double *kr, double *q)
{
    const int K = m->K;
    const double T = y[K];
    double sumYW = 0.0;
    for (int k = 0; k < K; ++k) sumYW += y[k] / m->W[k];
    double rho = p / (RU * T * sumYW);
    double *c = malloc(sizeof(double) * K);
    for (int k = 0; k < K; ++k) c[k] = rho * y[k] / m->W[k];
    for (int r = 0; r < m->R; ++r) {
        double M = 0.0;
        if (m->type[r] != RX_ELEM)
            for (int k = 0; k < K; ++k) M += m->eff[r * K + k] * c[k];
        rate_t rc = rate_constants(m, r, T, M);
        kf[r] = rc.kf;
        kr[r] = rc.kr;
        double q0 = rc.kf * conc_product(K, m->nuf + r * K, c) - rc.kr * conc_product(K, m->nur + r * K, c);
        q[r] = (m->type[r] == RX_THREEBODY) ? M * q0 : q0;
    }
    free(c);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Dense LU with partial pivoting (row-major), and the triangular solves.     */
/* ------------------------------------------------------------------------- */
static int lu_factor(int N, double *a, int *piv)
{
    for (int k = 0; k < N; ++k) {
        int p = k;
        double amax = fabs(a[k * N + k]);
        for (int i = k + 1; i < N; ++i)
            if (fabs(a[i * N + k]) > amax) { amax = fabs(a[i * N + k]); p = i; }
        piv[k] = p;
        if (amax == 0.0) return -1;
        if (p != k)
            for (int j = 0; j < N; ++j) { double t = a[k * N + j]; a[k * N + j] = a[p * N + j]; a[p * N + j] = t; }
        for (int i = k + 1; i < N; ++i) {
            a[i * N + k] /= a[k * N + k];
            for (int j = k + 1; j < N; ++j) a[i * N + j] -= a[i * N + k] * a[k * N + j];
        }
    }
    return 0;
}

static void lu_solve(int N, const double *a, const int *piv, double *x)
{
    for (int k = 0; k < N; ++k)
        if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < i; ++j) x[i] -= a[i * N + j] * x[j];
    for (int i = N - 1; i >= 0; --i) {
        for (int j = i + 1; j < N; ++j) x[i] -= a[i * N + j] * x[j];
        x[i] /= a[i * N + i];
    }
}

int orc_lu_solve(int N, double *a, int *piv, double *x, int nrhs)
{
    if (lu_factor(N, a, piv)) return -1;
    for (int r = 0; r < nrhs; ++r) lu_solve(N, a, piv, x + r * N);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* One Rosenbrock step of size h from y with f0 = f(y) and J = J(y).          */
/* ------------------------------------------------------------------------- */
typedef struct {
    double *f0, *J, *M, *u, *ys, *fs, *ynew, *err, *wk;
    int *piv;
    double *tab;   /* extrapolation table T[j][k], 3 x 3 x N */
} orc_ws;

static orc_ws ws_alloc(int K)
{
    const int N = K + 1;
    orc_ws w;
    w.f0 = malloc(sizeof(double) * N);
    w.J = malloc(sizeof(double) * N * N);
    w.M = malloc(sizeof(double) * N * N);
    w.u = malloc(sizeof(double) * 4 * N);
    w.ys = malloc(sizeof(double) * N);
    w.fs = malloc(sizeof(double) * N);
    w.ynew = malloc(sizeof(double) * N);
    w.err = malloc(sizeof(double) * N);
    w.wk = malloc(sizeof(double) * rhs_work_doubles(K));
    w.piv = malloc(sizeof(int) * N);
    w.tab = malloc(sizeof(double) * 9 * N);
    return w;
}

static void ws_free(orc_ws *w)
{
    free(w->f0); free(w->J); free(w->M); free(w->u); free(w->ys); free(w->fs);
    free(w->ynew); free(w->err); free(w->wk); free(w->piv); free(w->tab);
}

static int ros_step(const orc_mech *m, double p, const double *y, double h, orc_ws *w, const orc_method *t)
{
    const int N = m->K + 1;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) w->M[i * N + j] = -w->J[i * N + j] + (i == j ? 1.0 / (t->gamma * h) : 0.0);
    if (lu_factor(N, w->M, w->piv)) return -1;
    for (int s = 0; s < t->stages; ++s) {
        double *us = w->u + s * N;
        /* stage argument y + sum_j a_sj u_j ; where all a_sj vanish (stages 1 and 2
           of RODAS3) the argument is y itself and f(y) is reused */
        int newf = 0;
        for (int j = 0; j < s; ++j) if (t->a[s][j] != 0.0) newf = 1;
        if (!newf) {
            memcpy(us, w->f0, sizeof(double) * N);
        } else {
            for (int i = 0; i < N; ++i) {
                w->ys[i] = y[i];
                for (int j = 0; j < s; ++j) w->ys[i] += t->a[s][j] * w->u[j * N + i];
            }
            rhs_jac(m, p, w->ys, w->fs, NULL, w->wk);
            memcpy(us, w->fs, sizeof(double) * N);
        }
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < s; ++j) us[i] += t->c[s][j] / h * w->u[j * N + i];
        lu_solve(N, w->M, w->piv, us);
    }
    for (int i = 0; i < N; ++i) {
        w->ynew[i] = y[i];
        w->err[i] = 0.0;
        for (int s = 0; s < t->stages; ++s) {
            w->ynew[i] += t->m[s] * w->u[s * N + i];
            w->err[i] += t->e[s] * w->u[s * N + i];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Method 2: linearly implicit Euler extrapolation of fixed order 3           */
/* (Deuflhard's extrapolated linearly implicit Euler, the base of SEULEX;     */
/* Hairer and Wanner, Solving ODEs II, Section IV.9).  One step of size H     */
/* from y with f0 = f(y) and J = J(y): for the substep counts n_j = 1, 2, 3,  */
/* h_j = H / n_j and                                                          */
/*   (I/h_j - J) (y_{i+1} - y_i) = f(y_i),  i = 0 .. n_j - 1,  T_{j,1} = y_{n_j} */
/* whose error expands in powers of h_j; Aitken-Neville extrapolation         */
/*   T_{j,k+1} = T_{j,k} + (T_{j,k} - T_{j-1,k}) / (n_j / n_{j-k} - 1)         */
/* gives y_new = T_{3,3} (order 3) and the error estimate T_{3,3} - T_{3,2}   */
/* (T_{3,2} has order 2).  Per step: one Jacobian, three LU factorisations,   */
/* six solves, three f evaluations besides f(y).                              */
/* ------------------------------------------------------------------------- */
static int extrap_step(const orc_mech *m, double p, const double *y, double H, orc_ws *w)
{
    const int N = m->K + 1;
    double *T = w->tab;                       /* T[(j * 3 + k) * N + i] */
    for (int j = 0; j < 3; ++j) {
        const int n = j + 1;
        const double h = H / n;
        for (int a = 0; a < N; ++a)
            for (int b = 0; b < N; ++b) w->M[a * N + b] = -w->J[a * N + b] + (a == b ? 1.0 / h : 0.0);
        if (lu_factor(N, w->M, w->piv)) return -1;
        double *yi = T + (j * 3 + 0) * N;
        memcpy(yi, y, sizeof(double) * N);
        for (int i = 0; i < n; ++i) {
            if (i == 0) memcpy(w->fs, w->f0, sizeof(double) * N);
            else rhs_jac(m, p, yi, w->fs, NULL, w->wk);
            lu_solve(N, w->M, w->piv, w->fs);
            for (int a = 0; a < N; ++a) yi[a] += w->fs[a];
        }
    }
    for (int k = 1; k < 3; ++k)
        for (int j = k; j < 3; ++j) {
            const double r = (double)(j + 1) / (double)(j + 1 - k) - 1.0;
            for (int a = 0; a < N; ++a) {
                const double tj = T[(j * 3 + k - 1) * N + a], tm = T[((j - 1) * 3 + k - 1) * N + a];
                T[(j * 3 + k) * N + a] = tj + (tj - tm) / r;
            }
        }
    for (int a = 0; a < N; ++a) {
        w->ynew[a] = T[(2 * 3 + 2) * N + a];
        w->err[a] = T[(2 * 3 + 2) * N + a] - T[(2 * 3 + 1) * N + a];
    }
    return 0;
}

/* one step of the selected method: 0 RODAS3, 1 ROS2, 2 extrapolation */
static int method_step(const orc_mech *m, double p, const double *y, double h, orc_ws *w, int method)
{
    if (method == 2) return extrap_step(m, p, y, h, w);
    return ros_step(m, p, y, h, w, method_of(method));
}

/* err^(1/(qhat + 1)) of the step-size controller */
static double err_root(double err, const orc_method *t) { return t->qhat == 2 ? cbrt(err) : sqrt(err); }

/* single fixed step (order-of-convergence tests): ynew and the error vector */
int orc_fixed_step_method(const orc_mech *m, int method, double p, const double *y, double h, double *ynew,
                          double *err)
{
    const int N = m->K + 1;
    orc_ws w = ws_alloc(m->K);
    rhs_jac(m, p, y, w.f0, w.J, w.wk);
    int rc = method_step(m, p, y, h, &w, method);
    memcpy(ynew, w.ynew, sizeof(double) * N);
    memcpy(err, w.err, sizeof(double) * N);
    ws_free(&w);
    return rc;
}

int orc_fixed_step(const orc_mech *m, double p, const double *y, double h, double *ynew, double *err)
{
    return orc_fixed_step_method(m, 0, p, y, h, ynew, err);
}

/* ------------------------------------------------------------------------- */
/* Adaptive integration of one cell over [0, dt].                             */
/* ------------------------------------------------------------------------- */
static int advance_cell(const orc_mech *m, const orc_opts *o, double p, double *y, double dt, double *hint,
                        int *nacc, int *nrej, orc_ws *w)
{
    const int N = m->K + 1;
    const orc_method *tab = method_of(o->method);
    *nacc = 0;
    *nrej = 0;
    for (int i = 0; i < N; ++i) if (!isfinite(y[i])) return ORC_BAD_STATE;
    if (!(y[N - 1] > 0.0) || !(p > 0.0) || !isfinite(p)) return ORC_BAD_STATE;

    double t = 0.0;
    double h = (hint && *hint > 0.0) ? fmin(dt, *hint) : dt;
    int attempts = 0, reject_prev = 0;
    while (dt - t > 1e-14 * dt) {
        h = fmin(h, dt - t);
        rhs_jac(m, p, y, w->f0, w->J, w->wk);
        for (;;) {
            if (attempts >= o->max_substeps) return ORC_MAX_SUBSTEPS;
            ++attempts;
            if (method_step(m, p, y, h, w, o->method)) return ORC_LU_SINGULAR;
            double sum = 0.0;
            int finite = 1;
            for (int i = 0; i < N; ++i) {
                double sc = o->atol + o->rtol * fmax(fabs(y[i]), fabs(w->ynew[i]));
                double e = w->err[i] / sc;
                sum += e * e;
                if (!isfinite(w->ynew[i])) finite = 0;
            }
            double err = sqrt(sum / N);
            if (finite && isfinite(err) && err <= 1.0) {
                memcpy(y, w->ynew, sizeof(double) * N);
                t += h;
                ++*nacc;
                double fac = fmin(reject_prev ? 1.0 : o->facmax, fmax(o->facmin, o->safety / err_root(err, tab)));
                h *= fac;
                reject_prev = 0;
                break;
            }
            ++*nrej;
            double fac = (finite && isfinite(err)) ? fmax(o->facmin, o->safety / err_root(err, tab)) : o->facmin;
            h *= fac;
            reject_prev = 1;
            if (h < o->hmin) return ORC_H_UNDERFLOW;
        }
    }
    if (hint) *hint = h;
    return ORC_OK;
}

/* n cells; T [n] and Y [K][ldY] (species-major) advanced in place over dt.
   hint, status, nacc, nrej may be NULL. */
int orc_advance(const orc_mech *m, const orc_opts *o, long n, const double *p, double *T, double *Y, long ldY,
                double dt, double *hint, int *status, int *nacc, int *nrej)
{
    const int K = m->K, N = K + 1;
    orc_ws w = ws_alloc(K);
    double *y = malloc(sizeof(double) * N);
    for (long i = 0; i < n; ++i) {
        for (int k = 0; k < K; ++k) y[k] = Y[k * ldY + i];
        y[K] = T[i];
        int na = 0, nr = 0;
        int st = advance_cell(m, o, p[i], y, dt, hint ? hint + i : NULL, &na, &nr, &w);
        if (st != ORC_BAD_STATE) {
            for (int k = 0; k < K; ++k) Y[k * ldY + i] = y[k];
            T[i] = y[K];
        }
        if (status) status[i] = st;
        if (nacc) nacc[i] = na;
        if (nrej) nrej[i] = nr;
    }
    free(y);
    ws_free(&w);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Frozen step sequences (for the discrete adjoint's checks).                 */
/* ------------------------------------------------------------------------- */

/* Adaptive integration of one cell that also records its accepted step sizes
   h_list[0..*nsteps) (at most cap; ORC_MAX_SUBSTEPS if more are needed).
   y [N] is advanced in place. */
int orc_advance_record(const orc_mech *m, const orc_opts *o, double p, double *y, double dt, double *h_list,
                       int cap, int *nsteps)
{
    const int N = m->K + 1;
    orc_ws w = ws_alloc(m->K);
    *nsteps = 0;
    int rc = ORC_OK;
    double t = 0.0, h = dt;
    int attempts = 0, reject_prev = 0;
    for (int i = 0; i < N; ++i) if (!isfinite(y[i])) { ws_free(&w); return ORC_BAD_STATE; }
    while (rc == ORC_OK && dt - t > 1e-14 * dt) {
        h = fmin(h, dt - t);
        rhs_jac(m, p, y, w.f0, w.J, w.wk);
        for (;;) {
            if (attempts >= o->max_substeps || *nsteps >= cap) { rc = ORC_MAX_SUBSTEPS; break; }
            ++attempts;
            if (ros_step(m, p, y, h, &w, method_of(0))) { rc = ORC_LU_SINGULAR; break; }
            double sum = 0.0;
            int finite = 1;
            for (int i = 0; i < N; ++i) {
                double sc = o->atol + o->rtol * fmax(fabs(y[i]), fabs(w.ynew[i]));
                double e = w.err[i] / sc;
                sum += e * e;
                if (!isfinite(w.ynew[i])) finite = 0;
            }
            double err = sqrt(sum / N);
            if (finite && isfinite(err) && err <= 1.0) {
                memcpy(y, w.ynew, sizeof(double) * N);
                h_list[(*nsteps)++] = h;
                t += h;
                double fac = fmin(reject_prev ? 1.0 : o->facmax, fmax(o->facmin, o->safety / cbrt(err)));
                h *= fac;
                reject_prev = 0;
                break;
            }
            double fac = (finite && isfinite(err)) ? fmax(o->facmin, o->safety / cbrt(err)) : o->facmin;
            h *= fac;
            reject_prev = 1;
            if (h < o->hmin) { rc = ORC_H_UNDERFLOW; break; }
        }
    }
    ws_free(&w);
    return rc;
}

/* Replay a recorded step sequence with fixed steps (no error control). */
int orc_replay(const orc_mech *m, double p, double *y, const double *h_list, int nsteps)
{
    const int N = m->K + 1;
    orc_ws w = ws_alloc(m->K);
    int rc = 0;
    for (int s = 0; s < nsteps && rc == 0; ++s) {
        rhs_jac(m, p, y, w.f0, w.J, w.wk);
        if (ros_step(m, p, y, h_list[s], &w, method_of(0))) rc = ORC_LU_SINGULAR;
        else memcpy(y, w.ynew, sizeof(double) * N);
    }
    ws_free(&w);
    return rc;
}

