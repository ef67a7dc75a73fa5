/*
 * Plain CPU oracle of the Pade-based dimension-split ETD2RK scheme (ETD2RK-DS).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the cpu_baseline
 * and reference legs of bench.py may load this library. The product (the CUDA
 * library under paper_2601_06849_gb300/) neither links nor calls it, and this
 * file shares no code, header, table or helper with it.
 *
 * What it computes, by the paper's own route:
 *   - Section 2.1: centred differences, h = 1/(n+1), n interior points per axis,
 *     A_x = (1/h^2) tridiag(-kappa, 2 kappa + (q/d) h^2, -kappa).
 *   - Section 3.1, eq. (13)-(16): the Pade P_{0,2} ETD2RK-DS step, the rational
 *     functions Q_1, Q_2, Q_3 applied through their partial fractions
 *     Q_l(x) = 2 Re(r_l / (x - s)), s = -1 + i, r = (-i, (1-i)/2, 1/2).
 *   - Section 5 (the P_{0,4} variant): R_1, R_2, R_3 over the quartic
 *     denominator x^4 + 4x^3 + 12x^2 + 24x + 24, applied as 2 Re of a sum over its
 *     two upper-half-plane poles. The paper does not print poles or residues; they
 *     are computed here from the polynomials (roots of the quartic, residues
 *     N_l(s)/D'(s)). The paper's R_2 numerator ends in "+ I"; the constant is 24
 *     (R_2 = (1 - R_1)/x forces it, and R_2(0) must equal 1).
 *   - Section 3.2: every shifted solve (tau A_nu - s I) v = r g splits into
 *     independent 1D systems along one axis (x lines contiguous, y lines with
 *     stride n, z lines with stride n^2).
 *   - Section 3.3.1: one LU (Thomas) factorisation of tau A - s I per
 *     (component, pole), reused for every line and every step. tau A - s I is
 *     strictly diagonally dominant for Re(-s) > 0, so no pivoting.
 *   - Algorithm 1 (2D) and Algorithm 2 (3D), with the Sylvester solves replaced
 *     by the LU solves (Remark 3 of Section 3.4). The last stage multiplies by
 *     tau as eq. (14)/(16) state (the algorithm listings drop that factor).
 *
 * The same step is built twice from etd_oracle_step.h: in double (the oracle)
 * and in float (the "FP32 shadow", used only to measure the error floor that
 * FP32 storage alone imposes).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORX_NONE 0
#define ORX_LINEAR 1
#define ORX_ALLEN_CAHN 2
#define ORX_FHN 3
#define ORX_AC_MANUFACTURED 4
#define ORX_SINGULAR 5

typedef struct {
    int d;           /* 2 or 3 */
    int n;           /* interior points per axis */
    int ncomp;       /* 1, or 2 for FitzHugh-Nagumo */
    int pade;        /* 2 -> P_{0,2}, 4 -> P_{0,4} */
    int reaction;    /* ORX_* */
    int pad_;
    double kappa[2]; /* diffusivity per component */
    double q;        /* potential q >= 0 (split q/d per axis) */
    double tau;      /* time step */
    double rp[8];    /* reaction parameters, see oracle.py */
} oracle_problem;

/* ---- Pade data, computed in FP64 once per call ---------------------------- */

typedef struct {
    int npoles;              /* 1 for P_{0,2}, 2 for P_{0,4} */
    double complex s[2];     /* poles with positive imaginary part */
    double complex r[3][2];  /* r[l-1][pole]: residue of E_l at that pole */
} pade_data;

static double complex poly_eval(const double* c, int deg, double complex x) {
    /* c[k] is the coefficient of x^k */
    double complex v = 0.0;
    for (int k = deg; k >= 0; --k) v = v * x + c[k];
    return v;
}

/* Roots of the monic quartic x^4 + 4x^3 + 12x^2 + 24x + 24 by Durand-Kerner
 * iteration, each then polished by Newton steps. */
static void quartic_roots(double complex out[4]) {
    const double c[5] = {24.0, 24.0, 12.0, 4.0, 1.0};
    const double dc[4] = {24.0, 24.0, 12.0, 4.0}; /* derivative 4x^3+12x^2+24x+24 */
    double complex z[4];
    const double complex seed = 0.4 + 0.9 * I;
    z[0] = seed;
    for (int j = 1; j < 4; ++j) z[j] = z[j - 1] * seed;
    for (int it = 0; it < 500; ++it) {
        for (int j = 0; j < 4; ++j) {
            double complex den = 1.0;
            for (int k = 0; k < 4; ++k)
                if (k != j) den *= (z[j] - z[k]);
            z[j] = z[j] - poly_eval(c, 4, z[j]) / den;
        }
    }
    for (int j = 0; j < 4; ++j)
        for (int it = 0; it < 5; ++it) z[j] -= poly_eval(c, 4, z[j]) / poly_eval(dc, 3, z[j]);
    for (int j = 0; j < 4; ++j) out[j] = z[j];
}

static void pade_setup(int order, pade_data* P) {
    memset(P, 0, sizeof(*P));
    if (order == 2) {
        /* Section 3.1: Q_l(x) = 2 Re(r_l (x - s)^{-1}) */
        P->npoles = 1;
        P->s[0] = -1.0 + 1.0 * I;
        P->r[0][0] = -1.0 * I;
        P->r[1][0] = 0.5 - 0.5 * I;
        P->r[2][0] = 0.5;
        return;
    }
    /* P_{0,4}: E_1 = 24/D, E_2 = (x^3+4x^2+12x+24)/D, E_3 = (x^3+3x^2+8x+12)/D */
    const double num[3][4] = {{24.0, 0.0, 0.0, 0.0}, {24.0, 12.0, 4.0, 1.0}, {12.0, 8.0, 3.0, 1.0}};
    const double dden[4] = {24.0, 24.0, 12.0, 4.0}; /* D'(x) = 4x^3+12x^2+24x+24 */
    double complex roots[4];
    quartic_roots(roots);
    int k = 0;
    for (int j = 0; j < 4 && k < 2; ++j)
        if (cimag(roots[j]) > 0.0) P->s[k++] = roots[j];
    P->npoles = 2;
    for (int l = 0; l < 3; ++l)
        for (int p = 0; p < 2; ++p) P->r[l][p] = poly_eval(num[l], 3, P->s[p]) / poly_eval(dden, 3, P->s[p]);
}

/* 2 Re sum_p r_l,p / (x - s_p): the rational function E_l at a real scalar x. */
double oracle_rational(int order, int ell, double x) {
    pade_data P;
    pade_setup(order, &P);
    double complex acc = 0.0;
    for (int p = 0; p < P.npoles; ++p) acc += P.r[ell - 1][p] / (x - P.s[p]);
    return 2.0 * creal(acc);
}

/* Poles (upper half plane) and residues, for inspection by tests. */
int oracle_pade_data(int order, double* s_re, double* s_im, double* r_re, double* r_im) {
    pade_data P;
    pade_setup(order, &P);
    for (int p = 0; p < P.npoles; ++p) {
        s_re[p] = creal(P.s[p]);
        s_im[p] = cimag(P.s[p]);
        for (int l = 0; l < 3; ++l) {
            r_re[l * 2 + p] = creal(P.r[l][p]);
            r_im[l * 2 + p] = cimag(P.r[l][p]);
        }
    }
    return P.npoles;
}

void oracle_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- the step, once per precision ------------------------------------------ */

#define REAL double
#define FN(name) name##_f64
#include "etd_oracle_step.h"
#undef REAL
#undef FN

#define REAL float
#define FN(name) name##_f32
#include "etd_oracle_step.h"
#undef REAL
#undef FN
