/*
 * Plain, slow, scalar-loop FP64 reference kernels for the structure-preserving
 * spectral divide-and-conquer of definite pseudosymmetric matrices
 * (Benner, Nakatsukasa, Penke, arXiv 2203.08900).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle: it is called by the
 * tests, by __graft_entry__.smoke() and by bench.py's CPU-baseline leg, and by
 * nothing else.  It shares no code, header, table or constant with the CUDA
 * library.  Every loop is the textbook definition, with no blocking, fusion or
 * reordering, so that it can be checked against the paper by eye.
 *
 * Storage: dense row-major, element (i,j) of an n-by-m matrix at [i*m + j].
 * All routines return 0 on success and a positive code on breakdown.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Cholesky factorisation A = L L^T (lower L), column by column.            */
/* Used for M = Sigma*A in the definite case (Sec. 5, "definite" means       */
/* Sigma*A is positive definite) and for Algs. 4 and 6.                     */
/* Returns 0, or j+1 when the j-th pivot is not positive (not definite).    */
/* ------------------------------------------------------------------------ */
int or_cholesky(int n, const double *A, double *L)
{
    memset(L, 0, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) return j + 1;
        double d = sqrt(s);
        L[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / d;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Gaussian elimination with partial (row) pivoting: solve A X = B for       */
/* X (n-by-m).  A is overwritten by its LU factors, B by X.  This is the     */
/* plain "inverse" of Eq. (ZoloIt2): the paper forms                          */
/* (X^T Sigma X + c Sigma)^{-1}, a symmetric indefinite matrix, by pivoted    */
/* LDL^T (Eq. LDLZolo); any backward-stable pivoted elimination gives the    */
/* same result in exact arithmetic.  Returns k+1 for an exactly zero pivot.  */
/* ------------------------------------------------------------------------ */
int or_lu_solve(int n, double *A, int m, double *B)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = fabs(A[(size_t)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        if (best == 0.0) return k + 1;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[(size_t)k * n + j]; A[(size_t)k * n + j] = A[(size_t)p * n + j]; A[(size_t)p * n + j] = t;
            }
            for (int j = 0; j < m; ++j) {
                double t = B[(size_t)k * m + j]; B[(size_t)k * m + j] = B[(size_t)p * m + j]; B[(size_t)p * m + j] = t;
            }
        }
        double piv = A[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            double f = A[(size_t)i * n + k] / piv;
            A[(size_t)i * n + k] = f;
            if (f == 0.0) continue;
            for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
            for (int j = 0; j < m; ++j) B[(size_t)i * m + j] -= f * B[(size_t)k * m + j];
        }
    }
    /* back substitution with the upper factor */
    for (int k = n - 1; k >= 0; --k) {
        double piv = A[(size_t)k * n + k];
        for (int j = 0; j < m; ++j) {
            double t = B[(size_t)k * m + j];
            for (int i = k + 1; i < n; ++i) t -= A[(size_t)k * n + i] * B[(size_t)i * m + j];
            B[(size_t)k * m + j] = t / piv;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cyclic-by-row Jacobi eigensolver for a symmetric matrix.  This is the     */
/* "existing algorithm" for the symmetric definite subproblems that remain   */
/* after one split (Thm. DefDivConq and the remark following it), and the    */
/* definition-level eigensolver of the oracle.                               */
/* A (n-by-n, symmetric) is destroyed.  On exit w holds the eigenvalues      */
/* (unsorted) and V (n-by-n) the eigenvectors as columns.  Rotation formulas */
/* are the classical ones (Golub & Van Loan, Alg. 8.5.1, "sym.schur2").      */
/* Returns the number of sweeps used, or -1 if max_sweeps was exceeded.      */
/* ------------------------------------------------------------------------ */
int or_jacobi_eigh(int n, double *A, double *w, double *V, int max_sweeps)
{
    memset(V, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double v = A[(size_t)i * n + j];
                if (i == j) dia += v * v; else off += v * v;
            }
        if (off <= 1e-30 * dia || off == 0.0) {
            for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
            return sweep;
        }
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J with J the rotation in the (p,q) plane */
                for (int k = 0; k < n; ++k) {
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                A[(size_t)p * n + q] = 0.0;
                A[(size_t)q * n + p] = 0.0;
                for (int k = 0; k < n; ++k) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Low-rank Cholesky with diagonal pivoting of a symmetric positive          */
/* semidefinite matrix: A ~= W W^T with W n-by-rank.  At every step the      */
/* largest remaining diagonal entry is the pivot (ties: lowest index).       */
/* This is the pivoted, truncated LDL^T of Alg. 7: for a positive            */
/* semidefinite Sigma*P_+ every pivot is 1-by-1 and positive, so             */
/* L D^{1/2} = W, and the truncation keeps the first r_+ columns.            */
/* piv[k] (optional) receives the row chosen at step k.                      */
/* Returns 0, or k+1 if the k-th pivot is not positive before rank steps.    */
/* ------------------------------------------------------------------------ */
int or_pivoted_lowrank_chol(int n, const double *A, int rank, double *W, int *piv)
{
    double *R = (double *)malloc(sizeof(double) * (size_t)n * n);
    char *used = (char *)calloc((size_t)n, 1);
    if (!R || !used) { free(R); free(used); return -1; }
    memcpy(R, A, sizeof(double) * (size_t)n * n);
    memset(W, 0, sizeof(double) * (size_t)n * rank);
    int status = 0;
    for (int k = 0; k < rank; ++k) {
        int p = -1; double best = -INFINITY;
        for (int i = 0; i < n; ++i)
            if (!used[i] && R[(size_t)i * n + i] > best) { best = R[(size_t)i * n + i]; p = i; }
        if (p < 0 || !(best > 0.0)) { status = k + 1; break; }
        used[p] = 1;
        if (piv) piv[k] = p;
        double d = sqrt(best);
        for (int i = 0; i < n; ++i) W[(size_t)i * rank + k] = used[i] && i != p ? 0.0 : R[(size_t)i * n + p] / d;
        /* Schur complement: R <- R - w w^T on the unused rows and columns */
        for (int i = 0; i < n; ++i) {
            if (used[i]) continue;
            double wi = W[(size_t)i * rank + k];
            for (int j = 0; j < n; ++j) {
                if (used[j]) continue;
                R[(size_t)i * n + j] -= wi * W[(size_t)j * rank + k];
            }
        }
    }
    free(R); free(used);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Jacobi elliptic functions by the arithmetic-geometric mean and the        */
/* descending Landen transformation (Abramowitz & Stegun 16.4 and 17.6).    */
/* The modulus is k' with complementary modulus kc = sqrt(1-k'^2) passed     */
/* directly, so that the AGM is seeded with b0 = kc and no cancellation      */
/* 1 - k'^2 ever happens (the Zolotarev parameter l can be 1e-16).           */
/* ------------------------------------------------------------------------ */

/* complete elliptic integral of the first kind for the modulus whose       */
/* complementary modulus is kc: K = pi / (2 AGM(1, kc))                      */
double or_ellipk_from_comp(double kc)
{
    double a = 1.0, b = kc;
    for (int it = 0; it < 100; ++it) {
        double an = 0.5 * (a + b), bn = sqrt(a * b);
        a = an; b = bn;
        if (fabs(a - b) <= 1e-17 * a) break;
    }
    return M_PI / (2.0 * a);
}

/* sn(u), cn(u) for the modulus with complementary modulus kc */
void or_sncn(double u, double kc, double *sn, double *cn)
{
    double a[128], c[128];
    double b = kc;
    a[0] = 1.0; c[0] = 0.0;
    int N = 0;
    for (int it = 1; it < 127; ++it) {
        a[it] = 0.5 * (a[it - 1] + b);
        c[it] = 0.5 * (a[it - 1] - b);
        b = sqrt(a[it - 1] * b);
        N = it;
        if (fabs(c[it]) <= 1e-17 * a[it]) break;
    }
    double phi = ldexp(a[N] * u, N);           /* phi_N = 2^N a_N u */
    for (int m = N; m >= 1; --m)                /* sin(2 phi_{m-1} - phi_m) = (c_m/a_m) sin(phi_m) */
        phi = 0.5 * (phi + asin(c[m] / a[m] * sin(phi)));
    *sn = sin(phi);
    *cn = cos(phi);
}

/* ------------------------------------------------------------------------ */
/* sc(u) = sn(u)/cn(u) for the modulus k' = sqrt(1-kc^2), kc small, for     */
/* real u in [0, K(k')).  Near u = K(k') with kc ~ 1e-16, cn(u) is below     */
/* 1e-15, so sn/cn from the real-argument Landen recursion above has no      */
/* correct digit.  Instead use Jacobi's imaginary transformation              */
/*     sn(i u; kc) = i sc(u; k')                                             */
/* and evaluate sn at the imaginary argument for the SMALL modulus kc by     */
/* the descending Landen transformation (A&S 16.12):                         */
/*     mu = (1 - kc')/(1 + kc'),  v = w/(1 + mu),                            */
/*     sn(w; kc) = (1 + mu) sn(v; mu) / (1 + mu sn^2(v; mu)),                */
/* down to a modulus so small that sn(i y; 0) = i sinh(y) is exact to FP64.  */
/* With sn(i y_j; k_j) = i T_j the recursion reads                           */
/*     T_j = (1 + k_{j+1}) T_{j+1} / (1 - k_{j+1} T_{j+1}^2).                 */
/* ------------------------------------------------------------------------ */
double or_sc_comp(double u, double kc)
{
    double k[64], y[64];
    int N = 0;
    k[0] = kc; y[0] = u;
    while (N < 62) {
        double ch = cosh(y[N]);
        if (k[N] * k[N] * ch * ch < 1e-34) break;      /* sn(iy; k) = i sinh(y) to FP64 */
        double kcp = sqrt((1.0 - k[N]) * (1.0 + k[N]));   /* complementary modulus of k_N */
        double one_minus = k[N] * k[N] / (1.0 + kcp);      /* 1 - kc' without cancellation */
        k[N + 1] = one_minus / (1.0 + kcp);
        y[N + 1] = y[N] / (1.0 + k[N + 1]);
        ++N;
    }
    double T = sinh(y[N]);
    for (int j = N - 1; j >= 0; --j)
        T = (1.0 + k[j + 1]) * T / (1.0 - k[j + 1] * T * T);
    return T;
}

/* ------------------------------------------------------------------------ */
/* Coefficients of the scaled type (2r+1,2r) Zolotarev function on [l,1]:  */
/*   c_i = l^2 sn^2(i K'/(2r+1); l') / cn^2(i K'/(2r+1); l'),  i = 1..2r     */
/*   (Eq. Compcis, with the argument read as the integer index i times K'), */
/*   l' = sqrt(1-l^2), K' = K(l') (complete integral with modulus l').       */
/*   a_j = -prod_k (c_{2j-1} - c_{2k}) / prod_{k!=j} (c_{2j-1} - c_{2k-1})   */
/*   (Eq. ZPartialFrac2, the printed product read as a quotient),           */
/*   Chat = prod_j (1 + c_{2j-1}) / (1 + c_{2j})  (Eq. hatZ),                */
/*   l_next = Chat l prod_j (l^2 + c_{2j}) / (l^2 + c_{2j-1})  (Alg. 8).    */
/* c has 2r entries (c[0] = c_1), a has r entries.                           */
/* ------------------------------------------------------------------------ */
int or_zolo_coeffs(double ell, int r, double *c, double *a, double *chat, double *ell_next)
{
    if (!(ell > 0.0) || !(ell <= 1.0) || r < 1) return 1;
    double Kp = or_ellipk_from_comp(ell);      /* modulus l', complementary modulus l */
    for (int i = 1; i <= 2 * r; ++i) {
        double sc = or_sc_comp((double)i * Kp / (2.0 * r + 1.0), ell);   /* sn/cn, modulus l' */
        c[i - 1] = ell * ell * sc * sc;
    }
    for (int j = 1; j <= r; ++j) {
        double num = 1.0, den = 1.0;
        double codd = c[2 * j - 2];             /* c_{2j-1} */
        for (int k = 1; k <= r; ++k) {
            num *= codd - c[2 * k - 1];         /* c_{2j-1} - c_{2k}   */
            if (k != j) den *= codd - c[2 * k - 2];  /* c_{2j-1} - c_{2k-1} */
        }
        a[j - 1] = -num / den;
    }
    double C = 1.0, prod = 1.0;
    for (int j = 1; j <= r; ++j) {
        C *= (1.0 + c[2 * j - 2]) / (1.0 + c[2 * j - 1]);
        prod *= (ell * ell + c[2 * j - 1]) / (ell * ell + c[2 * j - 2]);
    }
    *chat = C;
    *ell_next = C * ell * prod;
    return 0;
}
