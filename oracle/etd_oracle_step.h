/*
 * Precision-generic body of the oracle step; included twice by etd_oracle.c with
 * REAL = double (the oracle) and REAL = float (the FP32 shadow). FN(name) appends
 * the precision suffix. Test infrastructure only (see etd_oracle.c).
 */

typedef REAL _Complex FN(cplx);

/* LU (Thomas) factors of the tridiagonal Toeplitz matrix M = tau A - s I,
 * diagonal a, off-diagonal b (Section 3.3.1): M = L U with unit lower L. */
typedef struct {
    int n;
    FN(cplx) b;     /* off-diagonal entry of M */
    FN(cplx) * l;   /* l[i] = b / d[i-1], i >= 1 (sub-diagonal of L) */
    FN(cplx) * dinv;/* 1 / d[i], d = diagonal of U */
} FN(tfactor);

static void FN(factor_init)(FN(tfactor) * F, int n, double complex a, double complex b) {
    F->n = n;
    F->b = (FN(cplx))b;
    F->l = (FN(cplx)*)calloc((size_t)n, sizeof(FN(cplx)));
    F->dinv = (FN(cplx)*)calloc((size_t)n, sizeof(FN(cplx)));
    double complex dprev = a;
    F->dinv[0] = (FN(cplx))(1.0 / a);
    for (int i = 1; i < n; ++i) {
        double complex li = b / dprev;
        double complex di = a - li * b;
        F->l[i] = (FN(cplx))li;
        F->dinv[i] = (FN(cplx))(1.0 / di);
        dprev = di;
    }
}

static void FN(factor_free)(FN(tfactor) * F) {
    free(F->l);
    free(F->dinv);
}

/* y = M^{-1} g by forward and backward substitution (g real, y complex). */
static void FN(thomas_solve)(const FN(tfactor) * F, const REAL* g, FN(cplx) * y) {
    const int n = F->n;
    y[0] = g[0];
    for (int i = 1; i < n; ++i) y[i] = g[i] - F->l[i] * y[i - 1];
    y[n - 1] = y[n - 1] * F->dinv[n - 1];
    for (int i = n - 2; i >= 0; --i) y[i] = (y[i] - F->b * y[i + 1]) * F->dinv[i];
}

/* First element of 1D line L along axis dir (Section 3.2 slicing): x lines are
 * contiguous rows, y lines run at stride n, z lines at stride n^2. */
static long FN(line_base)(int n, int dir, long L) {
    if (dir == 0) return L * (long)n;
    if (dir == 1) return (L % n) + (L / n) * (long)n * n;
    return L;
}

/* out = [out] + coef * E_ell(tau A_dir) g on every 1D line along axis dir.
 * E_ell(x) g = 2 Re sum_p r_{ell,p} (x - s_p)^{-1} g, each inverse one Thomas
 * solve with the factors of tau A - s_p I. */
static void FN(apply_axis)(int d, int n, int dir, const FN(tfactor) * fac, int npoles, const FN(cplx) * r,
                           REAL coef, const REAL* g, REAL* out, int accumulate) {
    long nlines = (d == 2) ? (long)n : (long)n * n;
    long stride = (dir == 0) ? 1 : (dir == 1 ? (long)n : (long)n * n);
#pragma omp parallel
    {
        REAL* gl = (REAL*)malloc(sizeof(REAL) * (size_t)n);
        REAL* acc = (REAL*)malloc(sizeof(REAL) * (size_t)n);
        FN(cplx)* y = (FN(cplx)*)malloc(sizeof(FN(cplx)) * (size_t)n);
#pragma omp for schedule(static)
        for (long L = 0; L < nlines; ++L) {
            long base = FN(line_base)(n, dir, L);
            for (int i = 0; i < n; ++i) gl[i] = g[base + i * stride];
            for (int i = 0; i < n; ++i) acc[i] = 0;
            for (int p = 0; p < npoles; ++p) {
                FN(thomas_solve)(&fac[p], gl, y);
                for (int i = 0; i < n; ++i) acc[i] += (REAL)2 * (REAL)creal(r[p] * y[i]);
            }
            for (int i = 0; i < n; ++i) {
                REAL prev = accumulate ? out[base + i * stride] : (REAL)0;
                out[base + i * stride] = prev + coef * acc[i];
            }
        }
        free(gl);
        free(acc);
        free(y);
    }
}

/* Reaction f(x, t, u) at every grid point, all components at once
 * (Example 5.1 Allen-Cahn with manufactured forcing, Example 5.2 singular
 * source, Example 5.3 FitzHugh-Nagumo with parametric coefficients). */
static void FN(react)(const oracle_problem* P, double t, const REAL* u, REAL* f) {
    const int n = P->n, d = P->d;
    const long N = (d == 2) ? (long)n * n : (long)n * n * n;
    const double h = 1.0 / (double)(n + 1);
    const double* rp = P->rp;
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < N; ++idx) {
        switch (P->reaction) {
            case ORX_NONE:
                for (int c = 0; c < P->ncomp; ++c) f[c * N + idx] = 0;
                break;
            case ORX_LINEAR:
                for (int c = 0; c < P->ncomp; ++c) f[c * N + idx] = (REAL)rp[0] * u[c * N + idx];
                break;
            case ORX_ALLEN_CAHN: {
                REAL v = u[idx];
                f[idx] = v - v * v * v;
                break;
            }
            case ORX_FHN: {
                /* f_u = u - c3 u^3 - v,  f_v = eps (u - a v - b) */
                REAL uu = u[idx], vv = u[N + idx];
                f[idx] = uu - (REAL)rp[0] * uu * uu * uu - vv;
                f[N + idx] = (REAL)rp[1] * (uu - (REAL)rp[2] * vv - (REAL)rp[3]);
                break;
            }
            case ORX_AC_MANUFACTURED: {
                /* f = u(1 - u^2) + psi, psi chosen so that u = e^{-lambda t} u0 with
                 * u0 = prod_axis sin(pi x_axis): -kappa Lap u0 = d pi^2 kappa u0. */
                const double lam = rp[0], kap = P->kappa[0];
                long i = idx % n, j = (idx / n) % n, k = idx / ((long)n * n);
                double u0 = sin(M_PI * (double)(i + 1) * h) * sin(M_PI * (double)(j + 1) * h);
                if (d == 3) u0 *= sin(M_PI * (double)(k + 1) * h);
                double e = exp(-lam * t);
                double ue = e * u0;
                double psi = (-lam + (double)d * M_PI * M_PI * kap) * ue - ue * (1.0 - ue * ue);
                REAL v = u[idx];
                f[idx] = v * ((REAL)1 - v * v) + (REAL)psi;
                break;
            }
            case ORX_SINGULAR: {
                REAL v = u[idx];
                f[idx] = (REAL)rp[0] * v / ((REAL)1 - v);
                break;
            }
            default:
                break;
        }
    }
}

/* Advance u (ncomp blocks of n^d values, x fastest, then y, then z) by nsteps
 * Pade ETD2RK-DS steps from time t0. Returns 0, or -1 for bad arguments.
 *
 * 2D (Algorithm 1 with LU solves):
 *   F = f(t_n, U)
 *   y lines:  a = E1(tau A_y) U,  b = E1(tau A_y) F
 *   x lines:  W = E1(tau A_x) a + tau E2(tau A_x) b                     eq. (13)
 *   U+ = W + tau E3(tau A_x) [f(t_{n+1}, W) - b]                        eq. (14)
 * 3D (Algorithm 2): a and b come from a z pass, then a y pass, eq. (15)-(16). */
int FN(oracle_run)(const oracle_problem* P, REAL* u, int nsteps, double t0) {
    if (!P || !u || (P->d != 2 && P->d != 3) || P->n < 1 || P->ncomp < 1 || P->ncomp > 2 ||
        (P->pade != 2 && P->pade != 4) || !(P->tau > 0.0) || nsteps < 0)
        return -1;
    if (P->reaction == ORX_FHN && P->ncomp != 2) return -1;
    const int n = P->n, d = P->d, nc = P->ncomp;
    const long N = (d == 2) ? (long)n * n : (long)n * n * n;
    const double h = 1.0 / (double)(n + 1);
    const double tau = P->tau;

    pade_data PD;
    pade_setup(P->pade, &PD);
    FN(cplx) r[3][2];
    for (int l = 0; l < 3; ++l)
        for (int p = 0; p < 2; ++p) r[l][p] = (FN(cplx))PD.r[l][p];

    /* tau A - s I, A = (1/h^2) tridiag(-kappa, 2 kappa + (q/d) h^2, -kappa) */
    FN(tfactor) fac[2][2];
    for (int c = 0; c < nc; ++c)
        for (int p = 0; p < PD.npoles; ++p) {
            double kap = P->kappa[c];
            double complex a = tau * (2.0 * kap / (h * h) + P->q / (double)d) - PD.s[p];
            double complex b = -tau * kap / (h * h);
            FN(factor_init)(&fac[c][p], n, a, b);
        }

    REAL* F = (REAL*)malloc(sizeof(REAL) * (size_t)(nc * N));
    REAL* W = (REAL*)malloc(sizeof(REAL) * (size_t)(nc * N));
    REAL* FW = (REAL*)malloc(sizeof(REAL) * (size_t)(nc * N));
    REAL* A = (REAL*)malloc(sizeof(REAL) * (size_t)(nc * N));
    REAL* B = (REAL*)malloc(sizeof(REAL) * (size_t)(nc * N));
    REAL* T1 = (REAL*)malloc(sizeof(REAL) * (size_t)N);
    REAL* T2 = (REAL*)malloc(sizeof(REAL) * (size_t)N);
    const REAL one = 1, rtau = (REAL)tau;

    for (int step = 0; step < nsteps; ++step) {
        double tn = t0 + step * tau;
        FN(react)(P, tn, u, F);
        for (int c = 0; c < nc; ++c) {
            REAL* Uc = u + c * N;
            REAL* Fc = F + c * N;
            REAL* Ac = A + c * N;
            REAL* Bc = B + c * N;
            if (d == 2) {
                FN(apply_axis)(d, n, 1, fac[c], PD.npoles, r[0], one, Uc, Ac, 0);
                FN(apply_axis)(d, n, 1, fac[c], PD.npoles, r[0], one, Fc, Bc, 0);
            } else {
                FN(apply_axis)(d, n, 2, fac[c], PD.npoles, r[0], one, Uc, T1, 0);
                FN(apply_axis)(d, n, 2, fac[c], PD.npoles, r[0], one, Fc, T2, 0);
                FN(apply_axis)(d, n, 1, fac[c], PD.npoles, r[0], one, T1, Ac, 0);
                FN(apply_axis)(d, n, 1, fac[c], PD.npoles, r[0], one, T2, Bc, 0);
            }
            REAL* Wc = W + c * N;
            FN(apply_axis)(d, n, 0, fac[c], PD.npoles, r[0], one, Ac, Wc, 0);
            FN(apply_axis)(d, n, 0, fac[c], PD.npoles, r[1], rtau, Bc, Wc, 1);
        }
        FN(react)(P, tn + tau, W, FW);
        for (int c = 0; c < nc; ++c) {
            REAL* Uc = u + c * N;
            REAL* Wc = W + c * N;
            REAL* Gc = FW + c * N;
            const REAL* Bc = B + c * N;
            for (long i = 0; i < N; ++i) Gc[i] -= Bc[i];
            for (long i = 0; i < N; ++i) Uc[i] = Wc[i];
            FN(apply_axis)(d, n, 0, fac[c], PD.npoles, r[2], rtau, Gc, Uc, 1);
        }
    }

    for (int c = 0; c < nc; ++c)
        for (int p = 0; p < PD.npoles; ++p) FN(factor_free)(&fac[c][p]);
    free(F);
    free(W);
    free(FW);
    free(A);
    free(B);
    free(T1);
    free(T2);
    return 0;
}
