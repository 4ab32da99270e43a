/*
 * pssd -- structure-preserving spectral divide-and-conquer for definite
 * pseudosymmetric matrices on GB300 (sm_103a).
 *
 * Method: Benner, Nakatsukasa, Penke, "A Structure-Preserving
 * Divide-and-Conquer Method for Pseudosymmetric Matrices" (arXiv 2203.08900).
 *
 * C ABI.  No C++ types and no exceptions cross this boundary.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are dense, ROW-MAJOR, FP64, with a leading dimension (the
 *    distance in elements between the starts of consecutive rows), exactly as
 *    a contiguous torch tensor.  Row-major matters: H is not symmetric and
 *    sign(H^T) = sign(H)^T.
 *  - Every matrix pointer is a DEVICE pointer owned by the caller; the
 *    library never frees it.  Inputs are not modified.
 *  - `sigma` is a HOST array of n entries in {+1,-1}: the diagonal of the
 *    signature matrix Sigma (Def. pseudosym, Sec. 3).  NULL means
 *    Sigma = diag(I_{n/2}, -I_{n/2}) (the Casida / BSE form, Eq. Casida).
 *  - H must be pseudosymmetric (Sigma H symmetric, relative defect at most
 *    1e-12 in the Frobenius norm) and definite (Sigma H positive definite,
 *    Sec. 5).  Violations are reported, never trapped.
 *  - All GPU work is issued on the handle's stream.  Entry points that need a
 *    host scalar mid-way (bounds, stopping test, ranks) synchronise that
 *    stream; on return every output is complete.
 *  - Return value: PSSD_OK (0), a negative value -i if argument i (1-based)
 *    is invalid (LAPACK style), or one of the positive PSSD_ERR_* codes.  On
 *    error the outputs are unspecified; `info` (if not NULL) is filled as far
 *    as the run got.
 *  - Orders are limited to 1 <= n <= PSSD_MAX_N (some passes put one matrix
 *    row per grid row); larger n is rejected as an invalid argument.
 *  - Workspace is allocated by the handle on first use and grown as needed
 *    (cudaMalloc outside any stream capture); pssd_destroy frees it.  A
 *    caller can supply the workspace instead (pssd_set_workspace).
 */
#ifndef PSSD_H
#define PSSD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* largest supported order n (one grid row per matrix row in some passes) */
#define PSSD_MAX_N 65535

/* status codes */
#define PSSD_OK 0
#define PSSD_ERR_NOT_DEFINITE 1        /* Sigma H not positive definite (Cholesky pivot <= 0); info->fail_index */
#define PSSD_ERR_NO_CONVERGENCE 2      /* Alg. 8 stopping test still failing after max_restarts restarts */
#define PSSD_ERR_BASIS 3               /* split: basis rank or orthogonalisation breakdown */
#define PSSD_ERR_NONFINITE 4           /* NaN/Inf in the input or an iterate */
#define PSSD_ERR_TIMEOUT 5             /* a bounded device wait gave up (tensor-core pipeline) */
#define PSSD_ERR_CUDA 6                /* a CUDA call failed; see pssd_last_cuda_error */
#define PSSD_ERR_ALLOC 7               /* workspace allocation failed, or the caller's workspace is too small */
#define PSSD_ERR_NOT_PSEUDOSYMMETRIC 8 /* ||Sigma H - (Sigma H)^T||_F > 1e-12 ||Sigma H||_F */
#define PSSD_ERR_NOALLOC_TOO_LARGE 9   /* pssd_sign_noalloc: n exceeds PSSD_NOALLOC_MAX_N, or the temporaries exceed the scratch array */

/* precision modes */
#define PSSD_FP64 0          /* every step in native FP64 (DFMA) */
#define PSSD_MIXED 1         /* Zolotarev steps in FP32 on tensor cores (3xTF32); Newton-Schulz refinement,
                                basis and projections in FP64-accurate emulated arithmetic */
#define PSSD_FP64_EMULATED 2 /* the PSSD_FP64 algorithm with every contraction FP64-accurate but emulated:
                                by default exact integer slices of the operands multiplied on the BF16
                                tensor cores; with PSSD_FLAG_EMU_SIMT, float pairs on the FP32 pipe */
#define PSSD_FLAG_RESIDUALS 1 /* pssd_sign: also compute info->s2_resid = ||S^2 - I||_F;
                                 pssd_split / pssd_eig: info->split_backerr exactly (else estimated) */
#define PSSD_FLAG_NO_TENSOR_CORES 2 /* no tensor-core kernels: FP32 contractions on the FP32 SIMT kernel,
                                       emulated FP64 contractions with float pairs (for comparison) */
#define PSSD_FLAG_EMU_SIMT 4        /* emulated FP64 contractions with float pairs on the FP32 pipe instead of
                                       integer slices on the tensor cores (for comparison) */
#define PSSD_FLAG_RECOMPUTE 16      /* pssd_sign_vjp_rev: keep only the per-step iterates and recompute the
                                       shifted factorisations in the backward pass (less memory) */
#define PSSD_FLAG_NO_REFINE 8       /* pssd_eig, pssd_casida_eig: skip the final refinement step of the
                                       symmetric eigendecomposition (one Ogita-Aishima correction, about
                                       6 m^3 flops for an m x m symmetric problem) */

/* iteration for the sign function (pssd_opts.method; PSSD_FP64 and PSSD_FP64_EMULATED).
 * All three run on the same congruence form K = L^T Sigma L and the same kernels.
 *  PSSD_METHOD_ZOLO    hyperbolic Zolo-PD, Alg. 8: two steps of degree r, stopping test, restarts.
 *  PSSD_METHOD_DWH     the Sigma-DWH iteration the paper compares against in Sec. 6: the Zolotarev
 *                      step of degree r = 1 (the dynamically weighted Halley step, Sec. 5.3) repeated
 *                      with the l-update until ||X_{k+1} - X_k||_F / ||X_{k+1}||_F <= u^{1/3}
 *                      (cubic convergence), at most 30 steps.
 *  PSSD_METHOD_NEWTON  the scaled Newton iteration X <- (z X + (z X)^{-1})/2 of Eq. (NewtonSign) with
 *                      the suboptimal scaling of Byers and Xu that Sec. 6 compares against:
 *                      z_0 = 1/sqrt(ab), z_1 = sqrt(2 sqrt(ab)/(a+b)), z_{k+1} = 1/sqrt((z_k + 1/z_k)/2)
 *                      for spectral bounds a = 1, b = l of X_0; stops when the relative change is
 *                      at most u^{1/2} (quadratic convergence), at most 60 steps.  X_0^{-1} comes from
 *                      the Cholesky factor (K^{-1} = L^{-1} Sigma L^{-T}); later inverses as
 *                      (X^2)^{-1} X from the Cholesky factor of X^2, whose condition number is at most
 *                      kappa/4 after the first scaled step. */
#define PSSD_METHOD_ZOLO 0
#define PSSD_METHOD_DWH 1
#define PSSD_METHOD_NEWTON 2

typedef struct pssd_handle_s *pssd_handle;

typedef struct {
    int r;              /* Zolotarev rank per step; 0 = smallest r with 1-l_2 <= tau (reading of Sec. 5.3) */
    double alpha;       /* upper bound on max|lambda(H)|; 0 = estimate (power iteration on Sigma H) */
    double beta;        /* lower bound on min|lambda(H)|; 0 = estimate (power iteration on (Sigma H)^{-1}) */
    int precision;      /* PSSD_FP64, PSSD_MIXED or PSSD_FP64_EMULATED */
    int max_restarts;   /* restarts allowed after a failed stopping test (Alg. 8); < 0 = default (2) */
    int leaf;           /* pssd_eig: subproblems of at most this order are solved by Jacobi; 0 = 64 */
    int flags;          /* bitwise OR of PSSD_FLAG_* (0: none) */
    int method;         /* PSSD_METHOD_* (0: Zolo-PD); PSSD_MIXED accepts only PSSD_METHOD_ZOLO */
    long long wait_cycles; /* bound on each pipeline wait inside the tensor-core kernels, in polls of the
                              mbarrier (0 = default, 2^26); when a wait runs out the kernel stops, waits for
                              its own copies and products in flight, frees its tensor memory and the call
                              returns PSSD_ERR_TIMEOUT with the handle still usable */
} pssd_opts;

typedef struct {
    int r_used[4];       /* r of each pass of Alg. 8 (first pass, restarts) */
    int passes;          /* passes of Alg. 8 (1 + restarts) */
    int steps;           /* Zolotarev steps taken (2 per pass) */
    int restarts;
    int p;               /* number of positive eigenvalues = number of +1 in sigma */
    double alpha, beta;  /* bounds used in the first pass */
    double ell[6];       /* l, l_1, l_2 of the first pass, then of the first restart */
    double stop_crit[4]; /* ||X_2 - X_1||_F / ||X_2||_F of each pass */
    double s2_resid;     /* ||S^2 - I||_F (pssd_sign only; -1 if not computed) */
    double jsym_resid;   /* ||Sigma S - (Sigma S)^T||_F / ||S||_F (pssd_sign only) */
    double split_backerr;/* ||U_+^T K U_-||_F / ||K||_F: the backward error of the split (Sec. 6.1 metric)
                            of K = L^T Sigma L ~ H, U_+- the orthonormal invariant-subspace bases;
                            exact with PSSD_FLAG_RESIDUALS, else estimated from a 16-column Gaussian
                            probe (||E Omega||_F / 4, an unbiased estimate of ||E||_F^2 in square) */
    int fail_index;      /* failing Cholesky pivot (0-based) for PSSD_ERR_NOT_DEFINITE, else -1 */
    int levels;          /* pssd_eig: recursion depth reached */
    double seconds;      /* wall time of the call (host clock, stream synchronised) */
    int precision;       /* precision mode used */
    int fp32_steps;      /* PSSD_MIXED: FP32 Zolotarev steps taken (r of the first four in r_used, l in ell) */
    int ns_steps;        /* PSSD_MIXED: third-order Newton-Schulz steps applied */
    double ns_resid;     /* PSSD_MIXED: ||I - sign(K)^2||_F after refinement, K = L^T Sigma L (from a
                            64-column Gaussian probe when the step's prediction was within tolerance) */
    double comm_resid;   /* ||S H - H S||_F / ||H||_F of the returned result (pssd_sign: S; pssd_split:
                            S = Q Sigma_hat Q^T Sigma; pssd_eig: S = V V^T Sigma): exact with
                            PSSD_FLAG_RESIDUALS, else estimated from a 16-column Gaussian probe;
                            -1 if not computed.  S^2 = I alone does not certify the invariant
                            subspaces; this commutator does (Lemma SignProj) */
    int method;          /* iteration used (PSSD_METHOD_*) */
    int iterations;      /* sign iterations taken (Zolotarev steps of all passes, DWH or Newton steps) */
} pssd_info;

/* Fill `o` with the defaults (r = 0, alpha = beta = 0, FP64, 2 restarts, leaf 64, Zolo-PD,
 * default wait bound).  Every entry point rejects options outside their ranges with the
 * invalid-argument status of its opts argument: r outside [0, 64], alpha or beta negative or
 * not finite, beta > alpha when both are given, precision or method unknown, wait_cycles < 0. */
void pssd_opts_init(pssd_opts *o);

/* Create a handle bound to `stream` (a cudaStream_t; NULL = the legacy default
 * stream).  Allocates nothing on the device.  Returns PSSD_OK or PSSD_ERR_CUDA. */
int pssd_create(pssd_handle *h, void *stream);
int pssd_destroy(pssd_handle h);
int pssd_set_stream(pssd_handle h, void *stream);
/* Last CUDA error or failure message recorded by the handle (never NULL). */
const char *pssd_last_cuda_error(pssd_handle h);
const char *pssd_status_string(int status);

/* ---------------------------------------------------------------------------
 * Workspace.  By default a handle allocates device workspace on first use and
 * keeps it (grown as needed) until pssd_destroy.  A caller that manages its own
 * device memory can hand the handle one buffer instead; the handle then never
 * allocates, and a call that needs more returns PSSD_ERR_ALLOC (the handle
 * stays usable).  The worker handles of pssd_eig_batched keep library-managed
 * workspaces.
 * ------------------------------------------------------------------------- */
/* Upper bound on the workspace bytes of one pssd_sign / pssd_split / pssd_eig
 * call of order n with these options (r = 0 counts r = 8): (20 + 3 r) n^2
 * doubles + 256 MiB.  Returns -2 for n outside [1, PSSD_MAX_N]. */
int pssd_workspace_bytes(pssd_handle h, int n, const pssd_opts *opts, size_t *bytes);
/* Use [dptr, dptr + bytes) (device memory, at least 4096 bytes, owned by the
 * caller, kept alive until the handle is destroyed or the workspace replaced)
 * as the handle's only workspace; dptr = NULL returns to library-managed
 * workspace.  Synchronises the handle's stream and frees any workspace the
 * library had allocated; resets the peak. */
int pssd_set_workspace(pssd_handle h, void *dptr, size_t bytes);
/* Largest workspace (bytes) a call on this handle has needed since it was
 * created or since pssd_set_workspace: the exact size a caller-owned buffer
 * needs for the same calls. */
int pssd_workspace_peak(pssd_handle h, size_t *bytes);

/*
 * Zolotarev coefficients (host only, FP64; Sec. 5.3).
 *   c_i = l^2 sn^2(i K'/(2r+1); l') / cn^2(i K'/(2r+1); l'), i = 1..2r  (Eq. Compcis,
 *         read with the integer index i), l' = sqrt(1-l^2), K' = K(l');
 *   a_j = -prod_k (c_{2j-1} - c_{2k}) / prod_{k != j} (c_{2j-1} - c_{2k-1})  (Eq. ZPartialFrac2,
 *         the printed product read as a quotient);
 *   chat = prod_j (1 + c_{2j-1}) / (1 + c_{2j})   (Eq. hatZ);
 *   ell_next = chat l prod_j (l^2 + c_{2j}) / (l^2 + c_{2j-1})   (Alg. 8, l-update).
 * Arguments: ell in (0,1]; r in [1,64]; c: host array of 2r doubles (c[i-1] = c_i);
 * a: host array of r doubles; chat, ell_next: host scalars.  Returns -1 / -2 for
 * an invalid ell / r, -3..-6 for a NULL output.
 */
int pssd_zolo_coeffs(double ell, int r, double *c, double *a, double *chat, double *ell_next);

/* Smallest r in [1, r_max] such that two Zolotarev steps map [ell,1] into
 * [1-tau, 1] (reading of the choice of r in Sec. 5.3); r_max if none. */
int pssd_choose_r(double ell, double tau, int r_max);

/*
 * S = sign(H) (Eq. signDef) by the two-step Zolotarev iteration of Alg. 8
 * with its stopping test and restarts.
 *   n      order of H (n >= 1; with sigma == NULL n must be even)
 *   sigma  host signature (see above) or NULL
 *   H      device, n x n, leading dimension ldh >= n
 *   S      device, n x n output, leading dimension lds >= n; must not alias H
 *   opts   NULL = defaults
 *   info   NULL or filled (s2_resid and jsym_resid are computed)
 */
int pssd_sign(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh,
              double *S, int lds, const pssd_opts *opts, pssd_info *info);

/*
 * One structure-preserving spectral division of a definite H (Alg. 3 step
 * with Thm. DefDivConq): a (Sigma, Sigma_hat)-orthogonal basis Q = [Q_+ Q_-]
 * of the invariant subspaces of the p positive / n-p negative eigenvalues,
 * Q^T Sigma Q = diag(I_p, -I_{n-p}), and the projected blocks
 *   A11 = Q_+^T (Sigma H) Q_+   (p x p, symmetric positive definite),
 *   A22 = -Q_-^T (Sigma H) Q_-  ((n-p) x (n-p), symmetric negative definite),
 * so that Q^{-1} H Q = diag(A11, A22).  p = number of +1 in sigma (Thm. EVRealSigmaOrth).
 *   S      device, n x n, leading dimension lds >= n: a precomputed sign(H) (for example from
 *          pssd_sign) from which the projectors P_+- = (I +- S)/2 of Lemma SignProj are taken;
 *          NULL computes it (Alg. 8, as pssd_sign).  A given S is used as it is (its defect
 *          shows in info->split_backerr and info->comm_resid); it is not modified.
 *   Q      device, n x n output (columns 0..p-1 = Q_+), leading dimension ldq >= n
 *   A11    device, p x p output, lda11 >= p;  A22 device, (n-p) x (n-p), lda22 >= n-p
 *   p      host int output (may be NULL)
 * info->split_backerr = ||U_+^T K U_-||_F / ||K||_F (the metric of Sec. 6.1 for the symmetric K ~ H;
 * exact with PSSD_FLAG_RESIDUALS, otherwise a probe estimate).
 */
int pssd_split(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh,
               const double *S, int lds, double *Q, int ldq, double *A11, int lda11, double *A22,
               int lda22, int *p, const pssd_opts *opts, pssd_info *info);

/*
 * Full diagonalisation V^{-1} H V = D (Alg. 3; after one split the
 * subproblems are symmetric definite, Thm. DefDivConq, and are diagonalised
 * by the symmetric divide-and-conquer of Alg. 2 down to Jacobi leaves).
 *   V   device, n x n output, leading dimension ldv >= n; column j is the
 *       eigenvector of D[j]; V^T Sigma V = diag(I_p, -I_{n-p}) (Eq. VSigmaOrth)
 *   D   device, n output: the p positive eigenvalues ascending, then the
 *       negative ones by ascending magnitude
 * Each eigenvector's largest-magnitude entry is made positive.
 */
int pssd_eig(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh,
             double *V, int ldv, double *D, const pssd_opts *opts, pssd_info *info);

/*
 * Batched full diagonalisation of `count` independent definite pseudosymmetric
 * matrices of (possibly) different orders: for each i, what pssd_eig computes
 * for (n[i], sigma[i], H[i], ldh[i]) into (V[i], ldv[i], D[i]).
 * All arrays are HOST arrays of `count` entries; H[i], V[i], D[i] are device
 * pointers; sigma may be NULL (every instance Casida-signed) or hold per-
 * instance host signatures (NULL entries allowed); infos NULL or `count` entries.
 * Instances run concurrently on up to PSSD_BATCH_WORKERS internal streams (one
 * host thread and workspace each, kept by the handle); the environment variable
 * PSSD_BATCH_WORKERS (an integer in [1, 64], read at each call) overrides that
 * default.  The handle's stream is ordered before and after the whole batch.
 * Returns the first failing instance's status.
 */
#define PSSD_BATCH_WORKERS 16
int pssd_eig_batched(pssd_handle h, int count, const int *n, const signed char *const *sigma,
                     const double *const *H, const int *ldh, double *const *V, const int *ldv,
                     double *const *D, const pssd_opts *opts, pssd_info *infos);

/*
 * Adjoint (reverse mode) of S = sign(H) and of the eigenvalues of H.
 * For the scalar loss L = <Sbar, S> + sum_i lambar_i lambda_i (S = sign(H) of
 * Eq. signDef, lambda_i in the output order of pssd_eig) returns Hbar = dL/dH.
 * Uses H = V Lambda V^{-1} with V^{-1} = Sigma_hat V^T Sigma (Eq. VSigmaOrth)
 * and the Daleckii-Krein form of the Frechet derivative of the sign function:
 *   Hbar = V^{-T} (F o (V^T Sbar V^{-T}) + diag(lambar)) V^T,
 *   F_ij = (sign lambda_i - sign lambda_j) / (lambda_i - lambda_j).
 *   Sbar    device n x n (ld ldsb >= n), or NULL (no sign term)
 *   lambar  device vector of n, or NULL (no eigenvalue term); e.g. 1 for the p
 *           positive eigenvalues and 0 otherwise gives d(sum of positive eigenvalues)/dH
 *   Hbar    device n x n output, ld ldhb >= n
 * opts/info as for pssd_eig (the eigendecomposition is computed internally).
 */
int pssd_sign_vjp(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh,
                  const double *Sbar, int ldsb, const double *lambar, double *Hbar, int ldhb,
                  const pssd_opts *opts, pssd_info *info);

/*
 * Step-reversal adjoint of S = sign(H) (Alg. 8 run backwards) and of the sum of the positive
 * eigenvalues: Hbar = d<Sbar, S>/dH + pos_weight * d(sum_{lambda > 0} lambda)/dH, where the
 * second term is P_+^T, P_+ = (I + S)/2 (Lemma SignProj).  The forward computation (pssd_sign,
 * Zolotarev method, PSSD_FP64 or PSSD_FP64_EMULATED) records every step's input iterate and,
 * unless opts->flags has PSSD_FLAG_RECOMPUTE, the r shifted inverses (X_k^2 + c I)^{-1} of the
 * step; the backward pass reverses each step X_{k+1} = Chat (X_k + X_k sum_j a_j Z_j) through
 * them, then the congruence K = L^T Sigma L and the Cholesky factorisation M = L L^T.  The
 * coefficients and the bounds alpha, beta are held fixed: the result is the exact gradient of
 * the computed iteration.  H enters only through sym(Sigma H), so Hbar is the gradient with
 * respect to pseudosymmetric H (the unconstrained gradient projected by X -> Sigma sym(Sigma X)).
 *   Sbar     device n x n (ld ldsb) or NULL (zero cotangent of S)
 *   Hbar     device n x n (ld ldhb), written
 * Memory: about (2 (max_restarts + 1) (1 + r) + 16) n^2 doubles with stored inverses,
 * (2 (max_restarts + 1) + 16 + r) n^2 with PSSD_FLAG_RECOMPUTE (r: the first pass's degree).
 * Returns -7 (ldsb), -8 (pos_weight not finite), -9/-10 (Hbar, ldhb), -11 (options: mixed
 * precision or a method other than PSSD_METHOD_ZOLO), or a status of pssd_sign.
 */
int pssd_sign_vjp_rev(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh,
                      const double *Sbar, int ldsb, double pos_weight, double *Hbar, int ldhb,
                      const pssd_opts *opts, pssd_info *info);

/*
 * Structure-aware variants for the Casida form (Eq. Casida): they operate on the
 * blocks A and B directly (the direction named in Sec. 7) and return what
 * pssd_sign / pssd_split / pssd_eig return for H = [[A, B], [-B, -A]] with
 * sigma = NULL (n = 2k), in the same layouts and conventions.
 *
 * With T = [[I, I], [I, -I]]/sqrt 2, T H T = [[0, R], [P, 0]] (P = A + B,
 * R = A - B, both SPD exactly when H is definite).  With P = L_P L_P^T,
 * R = L_R L_R^T the congruence form of the definite case becomes
 * [[0, C], [C^T, 0]] with the k x k matrix C = L_P^T L_R, whose sign is built from
 * the orthogonal polar factor U of C: the two-step Zolotarev iteration of Alg. 8
 * (same coefficients, stopping test and restarts) acts on C alone, every shifted
 * matrix C_k^T C_k + c I is SPD, and every product is k x k -- about a sixth of
 * the n x n path's work.  The eigenvalues of H are +-sigma_i(C), and the full
 * diagonalisation needs one k x k symmetric divide-and-conquer (Alg. 2) of
 * H_C = U^T C instead of a split of H and two of them.
 *   k          order of the blocks (n = 2k <= PSSD_MAX_N)
 *   A, B       device, k x k, symmetric (relative defect at most 1e-12), leading
 *              dimensions lda, ldb >= k
 *   precision  PSSD_FP64 or PSSD_FP64_EMULATED; method PSSD_METHOD_ZOLO
 * Outputs (device): S or Q (2k x 2k, ld >= 2k), A11 and A22 (k x k, A22 = -A11),
 * V (2k x 2k) and D (2k) exactly as for the n x n entry points.
 * info->split_backerr is ||U_+^T K U_-||_F / ||K||_F of this congruence form,
 * ||U^T C - C^T U||_F / (2 sqrt 2 ||C||_F); info->comm_resid as for the n x n calls.
 */
int pssd_casida_sign(pssd_handle h, int k, const double *A, int lda, const double *B, int ldb, double *S,
                     int lds, const pssd_opts *opts, pssd_info *info);
int pssd_casida_split(pssd_handle h, int k, const double *A, int lda, const double *B, int ldb, double *Q,
                      int ldq, double *A11, int lda11, double *A22, int lda22, const pssd_opts *opts,
                      pssd_info *info);
int pssd_casida_eig(pssd_handle h, int k, const double *A, int lda, const double *B, int ldb, double *V,
                    int ldv, double *D, const pssd_opts *opts, pssd_info *info);

/*
 * Allocation-free pssd_sign for small problems (the paper has no counterpart;
 * this entry point exists for callers of the library).
 *
 * Some callers cannot let a library call cudaMalloc: applications whose device
 * memory is owned by their own pool or caching allocator (a stray allocation
 * outside it can fail once the pool has reserved the device, or fragments it),
 * and latency-critical loops for which the device-wide synchronisation that
 * cudaMalloc and cudaFree can cause is not acceptable.  pssd_sign_noalloc
 * computes what pssd_sign computes (same arguments, same results) but takes
 * every temporary from one fixed scratch array of PSSD_NOALLOC_SCRATCH_BYTES in
 * the library's device memory, which every GPU that loads the library holds
 * until the process exits.  It calls no cudaMalloc or cudaFree (nor any
 * allocating library routine), and the handle's own workspace is not touched.
 *   - n must be at most PSSD_NOALLOC_MAX_N; larger n returns
 *     PSSD_ERR_NOALLOC_TOO_LARGE without doing any work.  A call whose
 *     temporaries do not fit the scratch array (for example a large explicit
 *     opts->r) stops with PSSD_ERR_NOALLOC_TOO_LARGE as soon as a temporary
 *     would overflow it, also without allocating.
 *   - The first call on each device looks up the scratch array's device
 *     address (cudaGetSymbolAddress, with that device current); make that
 *     first call before any stream capture begins.
 *   - All calls on a device share the one array and it keeps the previous
 *     call's contents (every value the computation reads is written first in
 *     the same call).  Calls that can overlap on the GPU -- on different
 *     streams, or from several host threads -- race on the array: serialise
 *     them.
 *   - Like pssd_sign, the call synchronises the handle's stream where it needs
 *     a host scalar (bounds, stopping test, residuals).
 */
#define PSSD_NOALLOC_MAX_N 128
#define PSSD_NOALLOC_SCRATCH_BYTES (8u << 20)
int pssd_sign_noalloc(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh,
                      double *S, int lds, const pssd_opts *opts, pssd_info *info);

/*
 * Test hook (not part of the method): one FP32 contraction
 *   C = alpha op(A) diag(kscale) op(B) + beta Cin   (batched, strides in elements)
 * through the library's GEMM dispatch, on the tcgen05 tensor-core kernel
 * (use_tc = 1, 3xTF32) or the FP32 SIMT kernel (use_tc = 0).  ta/tb: 1 = transpose;
 * triA/triB: 0 none, 1 lower, 2 upper (structure of op(A), op(B)); lowerC: write
 * only C[i][j] with i >= j.  All pointers are device pointers.
 */
int pssd_test_gemm_f32(pssd_handle h, int use_tc, int m, int n, int k, int batch, int ta, int tb, int triA,
                       int triB, int lowerC, double alpha, double beta, const float *A, long long lda,
                       long long sA, const float *B, long long ldb, long long sB, const float *Cin,
                       long long ldcin, long long sCin, float *C, long long ldc, long long sC,
                       const float *kscale);
/* Test hook: the same for FP64 data with engine 0 (native DFMA), 1 (float pairs on the FP32
 * pipe) or 2 (exact integer slices on the BF16 tensor cores). */
int pssd_test_gemm_f64(pssd_handle h, int engine, int m, int n, int k, int batch, int ta, int tb, int triA,
                       int triB, int lowerC, double alpha, double beta, const double *A, long long lda,
                       long long sA, const double *B, long long ldb, long long sB, const double *Cin,
                       long long ldcin, long long sCin, double *C, long long ldc, long long sC,
                       const double *kscale);

/*
 * Complex pseudo-Hermitian matrices (the Bethe-Salpeter forms, Eqs. BSE1 and BSE2: H = Sigma M
 * with M Hermitian positive definite, e.g. [[A, B], [-conj(B), -conj(A)]] with A Hermitian and
 * B complex symmetric, or [[A, B], [-B, -A]] with A, B Hermitian).  H is an n x n complex matrix,
 * row-major, interleaved (re, im) doubles (the layout of cuDoubleComplex and torch.complex128),
 * leading dimension ldh counted in complex elements; sigma as for pssd_sign (NULL:
 * diag(I_{n/2}, -I_{n/2})).  The computation runs on the real embedding
 * R(H) = [[Re H, -Im H], [Im H, Re H]] (2n x 2n), which is real definite pseudosymmetric with
 * signature [sigma; sigma] and satisfies sign(R(H)) = R(sign(H)); 2n <= PSSD_MAX_N.
 *
 * pssd_zsign: S = sign(H) (complex n x n, ld lds in complex elements; S != H).
 *   Returns -2..-5 as pssd_sign's checks of n, sigma, H, ldh; -6 (S), -7 (lds), -8 (options).
 * pssd_zeig: V^{-1} H V = diag(D): D real (n, positive eigenvalues ascending, then negative ones
 *   by ascending magnitude), V complex n x n (ld ldv in complex elements) with
 *   V^H Sigma V = diag(sign(D)) (Eq. VSigmaOrth) and the largest-modulus entry of each column
 *   real and positive.  Each eigenvalue of H appears twice in R(H); a pair gives one eigenvector
 *   of H, and a group of 2q values within 1e-12 max|lambda| gives q eigenvectors: q random
 *   vectors of the group's real eigenspace, orthonormalised in the group's definite form
 *   s x^H Sigma y by the inverse square root of their (embedded) Gram matrix.
 *   Returns -6 (V), -7 (ldv), -8 (D), -9 (options), or PSSD_ERR_BASIS if the doubled spectrum
 *   cannot be paired.
 */
int pssd_zsign(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, double *S, int lds,
               const pssd_opts *opts, pssd_info *info);
int pssd_zeig(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, double *V, int ldv,
              double *D, const pssd_opts *opts, pssd_info *info);

/*
 * sign(H) of a GENERAL pseudosymmetric H: Sigma H symmetric but not necessarily
 * definite, so the spectrum may hold negative and positive real eigenvalues of
 * either sign characteristic and complex conjugate pairs (Def. pseudosym; the
 * setting of Alg. 3).  sign(H) = X sign(Re Lambda) X^{-1} needs no eigenvalue on
 * the imaginary axis.  Method: the Newton iteration of Eq. NewtonSign, X <- (mu X +
 * X^{-1}/mu)/2 with Frobenius-norm scaling mu = (||X^{-1}||_F/||X||_F)^{1/2} (dropped
 * once the relative step is below 1e-2), run on the symmetric W = Sigma X: W^{-1} =
 * (W^2)^{-1} W through the Cholesky factor of the positive definite W^2, so no
 * pivoted indefinite factorisation is needed; stopped when the relative step is
 * <= 2^-26.  The conditioning of W^2 is that of H squared: the method suits
 * moderately conditioned H.
 *   n, sigma, H, ldh, S, lds  as pssd_sign (S must not alias H)
 *   opts   NULL = defaults; precision PSSD_FP64 or PSSD_FP64_EMULATED (PSSD_MIXED
 *          returns -8); r, alpha, beta, method and max_restarts are not used
 *   info   NULL or filled: iterations, stop_crit (first four steps), p = the number of
 *          eigenvalues with positive real part (n + trace S)/2, s2_resid = ||S^2 - I||_F
 *          (exact), jsym_resid = 0 (Sigma S is symmetric by construction)
 * Status: PSSD_ERR_NOT_PSEUDOSYMMETRIC as pssd_sign; PSSD_ERR_NO_CONVERGENCE if an
 * iterate is numerically singular (an eigenvalue on or next to the imaginary axis;
 * info->fail_index = the failing Cholesky pivot of W^2) or 100 steps do not converge;
 * PSSD_ERR_NONFINITE for NaN/Inf.
 */
int pssd_gsign(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, double *S, int lds,
               const pssd_opts *opts, pssd_info *info);

/*
 * Spectral division of a GENERAL pseudosymmetric H (the division step of Alg. 3):
 * S = sign(H) as pssd_gsign; p = (n + trace S)/2 eigenvalues with positive real part;
 * a Gaussian sketch of each projector (I +- S)/2 made orthonormal (U_+, U_-); the
 * symmetric Sigma-Gram matrix U^T Sigma U of each basis diagonalised (= W Lambda W^T,
 * symmetric divide-and-conquer of Alg. 2), Q_+- = U_+- W |Lambda|^{-1/2} and
 * Sigma_hat_+- = sign(Lambda): the (Sigma, Sigma_hat)-orthogonal basis of Alg. 5 /
 * Thm. HRisLDL (Q^T Sigma Q = Sigma_hat), obtained without a pivoted LDL^T.  Then
 * Q^{-1} H Q = diag(A11, A22) with Q^{-1} = Sigma_hat Q^T Sigma, A11 = Sigma_hat_+
 * Q_+^T Sigma H Q_+ (pseudosymmetric with respect to Sigma_hat_+), A22 likewise.
 *   n, sigma, H, ldh   as pssd_sign
 *   Q          device, n x n, ldq >= n: [Q_+ Q_-]; must not alias H
 *   A11, A22   device, room for n x n each with leading dimension >= n (p is known
 *              only after the sign): the p x p and (n-p) x (n-p) blocks are written
 *              to their leading corners
 *   sigma_hat  host, n entries: Sigma_hat_+ then Sigma_hat_- (+1 / -1)
 *   p_out      host or NULL
 *   opts       as pssd_gsign (PSSD_MIXED returns -14)
 *   info       as pssd_gsign, plus split_backerr = ||Sigma_hat_+ Q_+^T Sigma H Q_-||_F /
 *              ||H||_F, the coupling block the division drops (exact)
 * Status: as pssd_gsign; PSSD_ERR_BASIS if a sketch loses rank or a Sigma-Gram
 * matrix has an eigenvalue below 1e-10 of its largest (a basis close to Sigma-neutral).
 */
int pssd_gsplit(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, double *Q, int ldq,
                double *A11, int lda11, double *A22, int lda22, signed char *sigma_hat, int *p_out,
                const pssd_opts *opts, pssd_info *info);

/* Test hook: the Krylov loops the library runs for the bounds of Alg. 8 (largest
 * eigenvalue of M and of L^{-T} L^{-1}), the shift search of Alg. 2 (Lanczos
 * quadrature nodes) and the screening of a shift (power iteration on R^{-T} R^{-1}).
 * op: PSSD_KRYLOV_SYM (y = A x, A symmetric, full storage) or PSSD_KRYLOV_TRI_PAIR
 * (y = A^T (A x) with A lower triangular; entries above the diagonal are not read).
 * A: device, m x m, row-major, ld lda.  power = 0: `steps` Lanczos steps from the
 * normalised seeded Gaussian vector, out[j] = alpha_j (j < steps), out[steps + 1 + j]
 * = beta_j (device, 2 steps + 2 doubles).  power > 0: that many normalised power
 * steps from the Gaussian vector of seed 0x5eed, then out[0] = v^T op(A) v.
 * fused = 0: one launch per vector operation; fused = 1: the whole loop in one
 * thread-block-cluster launch (m <= 1024).  v0 (device, m, or NULL) receives the
 * starting vector before normalisation.  Returns 0 or a negative argument index
 * (-6: power outside [0, 1000], or power = 0 with steps outside [1, m]). */
#define PSSD_KRYLOV_SYM 0
#define PSSD_KRYLOV_TRI_PAIR 1
int pssd_test_krylov(pssd_handle h, int op, int m, const double *A, int lda, int steps, int power,
                     unsigned long long seed, int fused, double *out, double *v0);

/* Test hook: the symmetric divide-and-conquer of Alg. 2 (Zolotarev sign of the
 * shifted subproblem, orthonormal split, recursion to Jacobi leaves of order <=
 * opts->leaf) on a symmetric m x m B (device, ld ldb), in the arithmetic of
 * opts->precision (PSSD_FP64 or PSSD_FP64_EMULATED), followed by one refinement
 * step unless opts->flags has PSSD_FLAG_NO_REFINE: W (device m x m, ld ldw)
 * receives orthonormal eigenvectors as columns and w (device, m) the eigenvalues,
 * in no particular order.  B is not modified. */
int pssd_test_sym_eig(pssd_handle h, int m, const double *B, int ldb, double *W, int ldw, double *w,
                      const pssd_opts *opts, pssd_info *info);

/* ---------------------------------------------------------------------------
 * Profiling hooks (no counterpart in the paper; for measurement only).
 * With profiling on, each library kernel region on the handle's stream is
 * bracketed by CUDA events and its time, launch count and algorithmic FLOPs
 * are added to one of the kinds below when the call returns.
 * ------------------------------------------------------------------------- */
#define PSSD_KIND_DGEMM 0       /* FP64 DFMA contraction */
#define PSSD_KIND_CHOL_LEAF 1   /* fused Cholesky + inverse of a diagonal block */
#define PSSD_KIND_HBM 2         /* elementwise / copy / reduction passes */
#define PSSD_KIND_GEMV 3        /* matrix-vector products (bound estimation) */
#define PSSD_KIND_JACOBI 4      /* Jacobi leaf eigensolver */
#define PSSD_KIND_SGEMM 5       /* FP32 FFMA contraction */
#define PSSD_KIND_DFGEMM 6      /* FP64 contraction in float pairs (its operand split counts under PSSD_KIND_HBM) */
#define PSSD_KIND_TCGEMM 7      /* FP32 contraction, 3xTF32 on tcgen05: the tensor-core kernel alone */
#define PSSD_KIND_OZGEMM 8      /* FP64 contraction, integer slices on tcgen05: the tensor-core kernel alone */
#define PSSD_KIND_OZPREP 9      /* exponent and slicing passes feeding PSSD_KIND_OZGEMM */
#define PSSD_KIND_TCPREP 10     /* tf32 split passes feeding PSSD_KIND_TCGEMM */
#define PSSD_NKIND 11
/* on != 0 enables event timing on the handle (adds two events per region). */
int pssd_profile_enable(pssd_handle h, int on);
/* Zero the per-kind totals of the handle. */
int pssd_profile_reset(pssd_handle h);
/* Totals of one kind since the last reset: milliseconds, timed regions,
 * algorithmic FLOPs (contractions: the exact structural multiply-add count x 2)
 * and algorithmic HBM bytes (memory-bound passes: the bytes each pass must read
 * and write; 0 where not counted).  Any pointer may be NULL; -2 if kind is out
 * of range. */
int pssd_profile_read(pssd_handle h, int kind, double *total_ms, long long *launches, double *flops,
                      double *bytes);
/* Number of kernels the library has launched in this process (all handles;
 * one count per launch).  -1 if h is NULL. */
long long pssd_launch_count(pssd_handle h);
/* The same count split by the phase of the solve that launched each kernel
 * (per host thread: the batched entry point's workers count in the phases of
 * their own instances).  Phases, in index order:
 *   PSSD_PHASE_OTHER    everything not listed below
 *   PSSD_PHASE_FRONT    structure check M = Sigma H, Cholesky of M, K (Sec. 4, Eq. SignCong)
 *   PSSD_PHASE_BOUNDS   the bounds alpha, beta of the top-level sign (Alg. 8, input)
 *   PSSD_PHASE_SIGN     the top-level sign iteration (Alg. 8; mixed: FP32 steps + refinement)
 *   PSSD_PHASE_SPLIT    the top-level split (Alg. 3 / Alg. 6: basis, projected blocks)
 *   PSSD_PHASE_SHIFT    recursion nodes: shift search and screening (Alg. 2, "find shift")
 *   PSSD_PHASE_NODE_SIGN  recursion nodes: sign of B - sigma I (Alg. 2 with Alg. 8)
 *   PSSD_PHASE_NODE_SPLIT recursion nodes: orthogonal split (Alg. 2 with Alg. 4)
 *   PSSD_PHASE_ASSEMBLE eigenvector products V <- V diag(V1, V2) and the final scaling
 *   PSSD_PHASE_LEAF     Jacobi leaves of the recursion
 *   PSSD_PHASE_REFINE   the refinement step of the symmetric eigendecomposition
 * Writes min(n, PSSD_PHASE_COUNT) counts to `counts` (host array; may be NULL
 * when n = 0) and returns PSSD_PHASE_COUNT. */
#define PSSD_PHASE_OTHER 0
#define PSSD_PHASE_FRONT 1
#define PSSD_PHASE_BOUNDS 2
#define PSSD_PHASE_SIGN 3
#define PSSD_PHASE_SPLIT 4
#define PSSD_PHASE_SHIFT 5
#define PSSD_PHASE_NODE_SIGN 6
#define PSSD_PHASE_NODE_SPLIT 7
#define PSSD_PHASE_ASSEMBLE 8
#define PSSD_PHASE_LEAF 9
#define PSSD_PHASE_REFINE 10
#define PSSD_PHASE_COUNT 11
int pssd_launch_count_phases(long long *counts, int n);
/* Number of device allocations (cudaMalloc calls) the library has made in this
 * process (all handles, workspace growth included). */
long long pssd_device_alloc_count(void);

#ifdef __cplusplus
}
#endif
#endif /* PSSD_H */
