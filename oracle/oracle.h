/* Shared declarations of the CPU oracle (oracle.c, oracle_cs.c).  TEST INFRASTRUCTURE. */
#ifndef ORC_ORACLE_H
#define ORC_ORACLE_H

enum { ORC_OK = 0, ORC_MAX_SUBSTEPS = 1, ORC_H_UNDERFLOW = 2, ORC_BAD_STATE = 3, ORC_LU_SINGULAR = 4 };
enum { RX_ELEM = 0, RX_THREEBODY = 1, RX_LINDEMANN = 2, RX_TROE = 3 };

typedef struct {
    int K, R;
    const double *W;              /* [K] kg/mol */
    const double *Tmid;           /* [K] K */
    const double *lo, *hi;        /* [K][7] NASA-7 coefficients, low / high range */
    const int *type;              /* [R] RX_* */
    const int *rev;               /* [R] 1 if reversible */
    const int *nuf, *nur;         /* [R][K] reactant / product stoichiometric coefficients */
    const double *A, *b, *EaR;    /* [R] SI pre-factor, T exponent, E/R_u (K); k_inf for falloff */
    const double *A0, *b0, *EaR0; /* [R] low-pressure limit k_0 (falloff only) */
    const double *troe;           /* [R][4] a, T***, T*, T** */
    const int *ntroe;             /* [R] number of Troe parameters given (3 or 4) */
    const double *eff;            /* [R][K] third-body efficiencies */
} orc_mech;

typedef struct {
    double rtol, atol, hmin, facmax, facmin, safety;
    int max_substeps;
    int method;                   /* 0: RODAS3, 1: ROS2 (see oracle.c) */
} orc_opts;


#endif
