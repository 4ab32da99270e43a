// Internal declarations shared by the CUDA translation units of libpssd.
// Not part of the public C ABI (include/pssd.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace pssd {

// Phases of a solve, for the launch counters below (the public indices are
// PSSD_PHASE_* in pssd.h, in the same order)
enum Phase {
    PH_OTHER = 0, PH_FRONT, PH_BOUNDS, PH_SIGN, PH_SPLIT, PH_SHIFT, PH_NODE_SIGN, PH_NODE_SPLIT, PH_ASSEMBLE,
    PH_LEAF, PH_REFINE, PH_COUNT
};

// process-wide count of kernels launched by the library (one increment per
// launch statement, after the launch), in total and by the phase the
// launching thread is in
extern std::atomic<long long> g_launches;
extern std::atomic<long long> g_phase_launches[PH_COUNT];
extern thread_local int g_phase;
inline void count_launch()
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    g_phase_launches[g_phase].fetch_add(1, std::memory_order_relaxed);
}

// sets the calling thread's phase for its lifetime, then restores the previous one
struct PhaseScope {
    int saved;
    explicit PhaseScope(int p) : saved(g_phase) { g_phase = p; }
    ~PhaseScope() { g_phase = saved; }
    PhaseScope(const PhaseScope &) = delete;
    PhaseScope &operator=(const PhaseScope &) = delete;
};

// Allow `func` (a __global__ function) `bytes` of dynamic shared memory on the
// current device: set once per (device, function), thread-safe.  False if the
// attribute call failed.
bool ensure_dynamic_smem(const void *func, int bytes);

enum Tri { TRI_NONE = 0, TRI_LOWER = 1, TRI_UPPER = 2 };
enum GemmMode { GM_F64 = 0, GM_F32 = 1, GM_DF = 2, GM_OZ = 3 };

// granularity of the recursive Cholesky's splits
constexpr int PB = 32;

// C[z] = alpha * op(A[z]) * diag(kscale) * op(B[z]) + beta * Cin[z]
//   op(A) is m x k, op(B) is k x n, all row-major with leading dimensions.
//   triA / triB describe the structure of op(A) / op(B): entries outside the
//   triangle are never read (treated as zero), and k-ranges that multiply
//   only zeros are skipped.  lowerC: only C[i][j] with i >= j is written.
//   Batch index z runs over `batch`, pointers advance by the strides (elements).
//   mode: GM_F64 (double data, DFMA), GM_F32 (float data, FFMA),
//         GM_DF (double data, FP64 emulated with float pairs on the FP32 pipe).
struct GemmArgs {
    int m = 0, n = 0, k = 0, batch = 1;
    const void *A = nullptr; long long lda = 0, sA = 0; int ta = 0, triA = TRI_NONE;
    const void *B = nullptr; long long ldb = 0, sB = 0; int tb = 0, triB = TRI_NONE;
    const void *Cin = nullptr; long long ldcin = 0, sCin = 0;
    void *C = nullptr; long long ldc = 0, sC = 0;
    const void *kscale = nullptr;   // same element type as A
    double alpha = 1.0, beta = 0.0;
    int lowerC = 0;
    int mode = -1;   // -1: double data in the caller's FP64 mode (resolved before launch)
    // GM_DF only: A, B point to the float high parts and Alo, Blo to the float low parts
    // of the operands, split once by split_pairs(); kscale must be exact in FP32 (e.g. +-1)
    const void *Alo = nullptr, *Blo = nullptr;
    // tensor-core engines: polls per pipeline wait before the kernel gives up (0 = default)
    long long wait_limit = 0;
};
// x -> (hi, lo) = (fl32(x), fl32(x - hi)) for a batch of rows x cols blocks, written compactly
void split_pairs(const double *x, long long ld, long long sb, int rows, int cols, int batch, float *hi, float *lo,
                 cudaStream_t s);
void gemm_launch(const GemmArgs &g, cudaStream_t s);
// FP32 GEMM on tcgen05 tensor cores (3xTF32), same conventions as GM_F32;
// ws: tc_gemm_workspace_bytes(g) bytes of device memory; err: device flag.
size_t tc_gemm_workspace_bytes(const GemmArgs &g);
int tc_gemm_launch(const GemmArgs &g, void *ws, int *err, cudaStream_t s);
int tc_gemm_prepare(const GemmArgs &g, void *ws, cudaStream_t s);           // operand split pass only
int tc_gemm_run(const GemmArgs &g, void *ws, int *err, cudaStream_t s);     // product on prepared operands
// FP64-accurate GEMM on tcgen05 BF16 tensor cores by exact integer slicing
// (double data, conventions of GM_F64); ws: oz_gemm_workspace_bytes(g) bytes.
size_t oz_gemm_workspace_bytes(const GemmArgs &g);
int oz_gemm_launch(const GemmArgs &g, void *ws, int *err, cudaStream_t s);
int oz_gemm_prepare(const GemmArgs &g, void *ws, cudaStream_t s);           // exponent and slicing passes only
int oz_gemm_run(const GemmArgs &g, void *ws, int *err, cudaStream_t s);     // product on prepared slices

// Cholesky and triangular inverse of the s x s diagonal block at (off, off)
// of each batch matrix, in one launch: L (lower) in place in A with zeros
// above the diagonal inside the block, L^{-1} (lower) in the same block of
// Rinv.  info[z] = (first failing global pivot + 1) if a pivot is not
// positive or finite (the factorisation then continues with pivot 1).
// s <= CholLeaf<T>::max_s; returns nonzero on a launch-configuration error.
template <class T> struct CholLeaf;
template <> struct CholLeaf<float> { static constexpr int max_s = 128; };
template <> struct CholLeaf<double> { static constexpr int max_s = 64; };
template <class T>
int chol_leaf(T *A, long long lda, long long sA, T *Rinv, long long ldr, long long sR, int off, int s, int batch,
              int *info, cudaStream_t st);

// Elementwise / HBM passes
void sym_prepare(const double *H, long long ldh, const double *sig, int n, double *M, long long ldm,
                 double *partials, cudaStream_t s);  // M = sym(diag(sig) H); partials: defect^2, norm^2 per block
int sym_prepare_blocks(int n);
void reduce_sum(const double *x, int count, double *out, cudaStream_t s);
// Casida blocks: P = sym(A + B), R = sym(A - B); partials per tile pair: symmetry defect^2, ||H||_F^2 share
void casida_prepare(const double *A, long long lda, const double *B, long long ldb, int k, double *P, double *R,
                    long long ldp, double *partials, cudaStream_t s);
// rows 0..k-1 of out = c (sx X + sy Y), rows k..2k-1 = c (sx X - sy Y) (k x m blocks)
void casida_combine(const double *X, long long ldx, const double *Y, long long ldy, int k, int m, double sx,
                    double sy, double c, double *out, long long ldo, cudaStream_t s);
void casida_build(const double *A, long long lda, const double *B, long long ldb, int k, double *H, long long ldh,
                  cudaStream_t s);  // H = [[A, B], [-B, -A]]
void j_resym(double *S, long long lds, const double *sig, int n, cudaStream_t s);  // S = (S + Sig S^T Sig)/2
template <class T>
void sym_average(T *S, long long lds, int n, cudaStream_t s);  // S = (S + S^T)/2 in place
void dk_combine(const double *W, long long ldw, const double *lam, const double *lambar, int n, double *X,
                long long ldx, cudaStream_t s);  // Daleckii-Krein weights of sign(), plus diag(lambar)
// F = refinement correction of A ~ Z diag(lam) Z^T from S = Z^T A Z and Gm = Z^T Z - I (full, symmetric)
void eig_refine_correction(const double *S, long long lds, const double *Gm, long long ldg, const double *lam, int n,
                           double omega, double *F, long long ldf, cudaStream_t s);
void tril_half_diag(double *X, long long ldx, int n, cudaStream_t s);   // lower part, diagonal halved, upper zeroed
// complex n x n (interleaved, ld in complex elements) <-> real embedding [[Re, -Im], [Im, Re]]
void complex_embed(const double *Z, long long ldz, int n, double *R, long long ldr, cudaStream_t s);
void complex_extract(const double *R, long long ldr, int n, int m, const int *perm, double *Z, long long ldz,
                     cudaStream_t s);   // Z[:, j] = R[:n, perm[j]] + i R[n:, perm[j]]
void complex_phase_fix(double *Z, long long ldz, int m, int n, cudaStream_t s);   // largest entry of each column real > 0
void scale_rows(double *X, long long ldx, int m, int n, const double *r, cudaStream_t s);  // out[0] = sum x (one block, fixed order)
template <class T>
void mirror_lower(T *A, long long lda, long long sA, int n, int batch, cudaStream_t s);
template <class T>  // Z[z] = G + shifts[z] I (lower)
void shift_copy_lower(const T *G, long long ldg, T *Z, long long ldz, long long sZ, int n,
                      const double *shifts, int batch, cudaStream_t s);
template <class T>  // T = sum_z a[z] Zinv[z] (lower)
void combine_lower(const T *Zinv, long long ldz, long long sZ, const double *a, int r, int n,
                   T *Tm, long long ldt, cudaStream_t s);
template <class TI, class TO>  // Y = alpha X (with conversion)
void scale_copy(const TI *X, long long ldx, TO *Y, long long ldy, int m, int n, double alpha,
                cudaStream_t s);
template <class T>  // Y[z] = X[z], z < batch (m x n blocks; strides sX, sY), one launch
void copy_batched(const T *X, long long ldx, long long sX, T *Y, long long ldy, long long sY, int m, int n, int batch,
                  cudaStream_t s);
// Z <- (B + Z)/2 in columns j < p, (B - Z)/2 in columns j >= p (m x n)
void half_sum_diff(const double *B, long long ldb, double *Z, long long ldz, int m, int n, int p, cudaStream_t s);
// Y = a diag(sig)^rx X + b diag(sig) T diag(sig) (n x n; T may be null; Y may alias X or T)
void sig_affine(const double *X, long long ldx, int rx, const double *T, long long ldt, const double *sig, int n,
                double a, double b, double *Y, long long ldy, cudaStream_t s);
template <class T>
void add_diag(T *X, long long ldx, int n, double v, cudaStream_t s);
template <class T>  // partials[2*b] = sum (X-Y)^2, [2*b+1] = sum Y^2 (X may be null)
void frob_diff(const T *X, long long ldx, const T *Y, long long ldy, int m, int n,
               double *partials, cudaStream_t s);
int frob_blocks(int m, int n);
void fill_gaussian(double *X, long long ldx, int m, int n, uint64_t seed, cudaStream_t s);
void trace_partial(const double *X, long long ldx, int n, double *out, cudaStream_t s);
void get_diag(const double *X, long long ldx, int n, double *d, cudaStream_t s);
void row_abs_sum_max(const double *X, long long ldx, int n, double *tmp, double *out, cudaStream_t s);  // tmp: n
void gemv(const double *A, long long lda, int ta, int tri, int n, const double *x, double *y,
          double *tmp, cudaStream_t s);  // y = op(A) x, square n; tmp: 32 n doubles (ta = 1)
void normalize_vec(double *y, double *x, int n, double *norm_out, cudaStream_t s);  // x = y/||y||
void dot_vec(const double *x, const double *y, int n, double *out, cudaStream_t s);
// w <- w - alpha[0] v - beta[0] vprev (device scalars; vprev and beta may be null)
void lanczos_update(double *w, const double *v, const double *vprev, const double *alpha, const double *beta, int n,
                    cudaStream_t s);

// Krylov loops in one launch for operators of order m <= KRY_MAX_M (one thread-block
// cluster; see kernels.cu).  Operators: KRY_SYM y = A x (A symmetric, full storage);
// KRY_TRI_PAIR y = L^T (L x) (L lower triangular, entries above the diagonal not read).
// The starting vector is the Gaussian vector fill_gaussian(v, m, 1, m, seed) makes.
//   power == 0: `steps` Lanczos steps; out[j] = alpha_j (j < steps) and
//               out[steps + 1 + j] = beta_j, the layout of the step-by-step loop.
//   power  > 0: `power` normalised power steps, then out[0] = v^T A v.
// Returns false (nothing launched) if m is outside [1, KRY_MAX_M].
constexpr int KRY_MAX_M = 1024;
enum KryOp { KRY_SYM = 0, KRY_TRI_PAIR = 1 };
bool krylov_cluster(const double *A, long long lda, int op, int m, int steps, int power, uint64_t seed, double *out,
                    cudaStream_t s);
void scale_columns(double *X, long long ldx, int m, int n, const double *d, int use_sqrt_abs,
                   cudaStream_t s);
void sign_fix_columns(double *X, long long ldx, int m, int n, cudaStream_t s);
void gather_columns(const double *X, long long ldx, double *Y, long long ldy, int m, int n,
                    const int *perm, cudaStream_t s);
void copy_matrix(const double *X, long long ldx, double *Y, long long ldy, int m, int n,
                 cudaStream_t s);
void jacobi_leaf(double *A, long long lda, int m, double *W, long long ldw, double *w,
                 int *sweeps_out, cudaStream_t s);  // m <= 64; W eigenvectors (columns), w values

// host-side Zolotarev coefficients (theta-function evaluation)
int zolo_coeffs_host(double ell, int r, double *c, double *a, double *chat, double *ell_next);
int choose_r_host(double ell, double tau, int r_max);

}  // namespace pssd
