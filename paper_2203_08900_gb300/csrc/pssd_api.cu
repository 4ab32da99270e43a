// Host drivers and the C ABI of libpssd.
//
// Layout of the computation (all device work on the handle's stream):
//
//   M = Sigma H (symmetrised; defect checked)          Def. pseudosym, Sec. 5 (definite)
//   M = L L^T, L^{-1}                                   blocked Cholesky + recursive triangular inverse
//   K = L^T Sigma L                                     symmetric, similar to H (L^T H L^{-T} = K)
//   alpha, beta from M and M^{-1} (power iteration)      Alg. 8, first step
//   Zolotarev steps on X_0 = K/alpha                    Alg. 8, Eqs. ZoloIt1 / ZPartialFrac
//     X_{k+1} = Chat (X_k + X_k sum_j a_j (X_k^2 + c_{2j-1} I)^{-1})
//     each shift: Cholesky R_j R_j^T, R_j^{-1}, R_j^{-T} R_j^{-1}  (r chains batched per launch)
//   stopping test, restarts                             Alg. 8
//   S = L^{-T} sign(K) L^T                              since H = L^{-T} K L^T
//   split: orthonormal bases U_+-, of range((I +- sign K)/2), B_+- = U_+-^T K U_+-,
//     Q_+- = L^{-T} U_+- C_+-  with  +-B_+- = C C^T        Alg. 3 step, Thm. DefDivConq
//   symmetric recursion on B_+-                         Alg. 2, Jacobi leaves
//
// Every iterate of the congruence form is symmetric and every shifted system
// is symmetric positive definite, so no pivoting is needed on the GPU; the
// paper's pivoted LDL^T / hyperbolic QR forms (Eqs. LDLZolo, HRZolo) compute
// the same iterates X_k = L^{-T} K_k L^T in exact arithmetic.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>
#include <type_traits>
#include <string>
#include <vector>
#include <cfloat>

#include "pssd.h"
#include "pssd_internal.h"

using namespace pssd;

namespace {

constexpr double U64 = 1.1102230246251565e-16;  // 2^-53

struct Chunk { char *base; size_t cap; size_t off; bool owned; };   // owned: allocated by the library

std::atomic<long long> g_device_allocs{0};   // device allocations (cudaMalloc) made by the library

struct ProfEvent { cudaEvent_t a, b; int kind; double flops, bytes; };

}  // namespace

struct pssd_handle_s {
    cudaStream_t stream = nullptr;
    std::vector<Chunk> chunks;
    std::string last_err = "no error";
    int prof = 0;
    std::vector<ProfEvent> events;
    std::vector<cudaEvent_t> free_events;
    double prof_ms[16] = {0}, prof_flops[16] = {0}, prof_bytes[16] = {0};
    long long prof_count[16] = {0};
    int dmode = GM_F64;   // arithmetic of FP64 contractions in the current call (GM_F64 or GM_DF)
    std::vector<pssd_handle_s *> workers;   // pssd_eig_batched: one handle (own stream, workspace) per worker
    int *derr = nullptr;    // device error flag of the current call (bounded waits in the tensor-core kernel)
    int use_tc = 1;         // FP32 contractions on tcgen05 tensor cores (0: FP32 SIMT kernel)
    int force_engine = 0;   // test hooks: no size-based engine selection
    bool user_ws = false;   // chunks[0] is caller-owned memory (pssd_set_workspace); never allocate
    size_t depth = 0;       // bytes of workspace live in the current call (stack discipline)
    size_t peak = 0;        // largest depth reached since creation or pssd_set_workspace
    long long wait_limit = 0;   // pipeline wait bound of the tensor-core kernels in this call (0 = default)
    cudaStream_t side = nullptr;               // the symmetric recursion's Jacobi leaves (created on first use)
    std::vector<cudaEvent_t> leaf_pending;     // leaves launched on `side` that the main stream has not joined
    std::vector<cudaEvent_t> sync_events;      // events without timing for the joins (pooled)
    size_t sync_used = 0;
};

namespace {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
struct Fail { int code; };

inline void cuda_check(pssd_handle h, cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        h->last_err = std::string(what) + ": " + cudaGetErrorString(e);
        throw Fail{PSSD_ERR_CUDA};
    }
}

// ---------------------------------------------------------------------------
// workspace: chunked bump allocator with stack marks; chunks are kept for reuse
// ---------------------------------------------------------------------------
struct Mark { size_t chunk; size_t off; size_t depth; };

Mark mark(pssd_handle h)
{
    if (h->chunks.empty()) return {0, 0, h->depth};
    // the active chunk is the last one with off > 0, or 0
    size_t c = 0;
    for (size_t i = 0; i < h->chunks.size(); ++i) if (h->chunks[i].off > 0) c = i;
    return {c, h->chunks[c].off, h->depth};
}

void release(pssd_handle h, Mark m)
{
    for (size_t i = 0; i < h->chunks.size(); ++i) {
        if (i > m.chunk) h->chunks[i].off = 0;
        else if (i == m.chunk) h->chunks[i].off = m.off;
    }
    h->depth = m.depth;
}

void *walloc(pssd_handle h, size_t bytes)
{
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    h->depth += bytes;
    h->peak = std::max(h->peak, h->depth);
    if (h->user_ws) {   // caller-owned workspace: one chunk, no allocation
        Chunk &c = h->chunks[0];
        if (c.off + bytes > c.cap) {
            h->depth -= bytes;
            h->last_err = "workspace set by pssd_set_workspace is too small (" + std::to_string(c.cap) +
                          " bytes; this call needs more than " + std::to_string(c.off + bytes) + ")";
            throw Fail{PSSD_ERR_ALLOC};
        }
        void *p = c.base + c.off;
        c.off += bytes;
        return p;
    }
    Mark m = mark(h);
    for (size_t i = m.chunk; i < h->chunks.size(); ++i) {
        Chunk &c = h->chunks[i];
        size_t off = (i == m.chunk) ? c.off : 0;
        if (off + bytes <= c.cap) { c.off = off + bytes; return c.base + off; }
    }
    size_t cap = std::max(bytes, size_t(1) << 30);
    void *p = nullptr;
    g_device_allocs.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaMalloc(&p, cap);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        h->last_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        throw Fail{PSSD_ERR_ALLOC};
    }
    h->chunks.push_back({(char *)p, cap, bytes, true});
    return p;
}

double *dalloc(pssd_handle h, size_t count) { return (double *)walloc(h, count * sizeof(double)); }
int *ialloc(pssd_handle h, size_t count) { return (int *)walloc(h, count * sizeof(int)); }

// ---------------------------------------------------------------------------
// launch accounting and optional per-launch CUDA-event timing
// ---------------------------------------------------------------------------
enum Kind { K_DGEMM = 0, K_CHOL_LEAF = 1, K_HBM = 2, K_GEMV = 3, K_JACOBI = 4, K_SGEMM = 5, K_DFGEMM = 6, K_TCGEMM = 7,
            K_OZGEMM = 8, K_OZPREP = 9, K_TCPREP = 10, K_NKIND = 11 };
static_assert(K_DGEMM == PSSD_KIND_DGEMM && K_CHOL_LEAF == PSSD_KIND_CHOL_LEAF && K_HBM == PSSD_KIND_HBM &&
                  K_GEMV == PSSD_KIND_GEMV && K_JACOBI == PSSD_KIND_JACOBI && K_SGEMM == PSSD_KIND_SGEMM &&
                  K_DFGEMM == PSSD_KIND_DFGEMM && K_TCGEMM == PSSD_KIND_TCGEMM && K_OZGEMM == PSSD_KIND_OZGEMM &&
                  K_OZPREP == PSSD_KIND_OZPREP && K_TCPREP == PSSD_KIND_TCPREP && K_NKIND == PSSD_NKIND,
              "profiling kinds match the public header");

cudaEvent_t get_event(pssd_handle h)
{
    if (!h->free_events.empty()) { cudaEvent_t e = h->free_events.back(); h->free_events.pop_back(); return e; }
    cudaEvent_t e;
    cuda_check(h, cudaEventCreate(&e), "cudaEventCreate");
    return e;
}

// one timed region: algorithmic FLOPs (contractions) or algorithmic HBM bytes
// (memory-bound passes: the bytes the pass must read and write at least), on the handle's
// stream or on another stream of the handle
struct Timed {
    pssd_handle h; int kind; double flops, bytes; cudaStream_t st; cudaEvent_t a = nullptr, b = nullptr;
    Timed(pssd_handle h_, int kind_, double flops_, double bytes_ = 0.0, cudaStream_t st_ = nullptr)
        : h(h_), kind(kind_), flops(flops_), bytes(bytes_), st(st_ ? st_ : h_->stream)
    {
        if (h->prof) { a = get_event(h); b = get_event(h); cudaEventRecord(a, st); }
    }
    ~Timed()
    {
        if (h->prof) { cudaEventRecord(b, st); h->events.push_back({a, b, kind, flops, bytes}); }
    }
};

// an event for ordering between the handle's streams (pooled for the handle's lifetime)
cudaEvent_t sync_event(pssd_handle h)
{
    if (h->sync_used == h->sync_events.size()) {
        cudaEvent_t e;
        cuda_check(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
        h->sync_events.push_back(e);
    }
    return h->sync_events[h->sync_used++];
}

// the handle's main stream waits for every leaf launched on the side stream so far
void join_leaves(pssd_handle h)
{
    for (cudaEvent_t e : h->leaf_pending) cuda_check(h, cudaStreamWaitEvent(h->stream, e, 0), "cudaStreamWaitEvent");
    h->leaf_pending.clear();
}

void prof_collect(pssd_handle h)
{
    if (!h->prof || h->events.empty()) return;
    cudaStreamSynchronize(h->stream);
    for (auto &e : h->events) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e.a, e.b);
        h->prof_ms[e.kind] += ms;
        h->prof_flops[e.kind] += e.flops;
        h->prof_bytes[e.kind] += e.bytes;
        h->prof_count[e.kind] += 1;
        h->free_events.push_back(e.a);
        h->free_events.push_back(e.b);
    }
    h->events.clear();
}

// exact count of multiply-adds of one GEMM launch (algorithmic work):
// output (i,j) needs the p with op(A)[i][p] and op(B)[p][j] structurally nonzero.
double gemm_macs(const GemmArgs &g)
{
    double total = 0.0;
    const double k = g.k;
    for (int i = 0; i < g.m; ++i) {
        double alo = 0, ahi = k;
        if (g.triA == TRI_LOWER) ahi = std::min(k, (double)i + 1);
        if (g.triA == TRI_UPPER) alo = i;
        int jmax = g.lowerC ? std::min(g.n, i + 1) : g.n;
        // len(j) = max(0, min(ahi, bhi(j)) - max(alo, blo(j)));
        // bhi(j) = j+1 (triB upper) or k; blo(j) = j (triB lower) or 0
        if (g.triB == TRI_NONE) {
            total += jmax * std::max(0.0, ahi - alo);
        } else if (g.triB == TRI_LOWER) {
            // len = max(0, ahi - max(alo, j)); j < alo: ahi-alo ; alo <= j < ahi: ahi - j
            double s = 0;
            double j1 = std::min((double)jmax, alo);
            if (j1 > 0) s += j1 * std::max(0.0, ahi - alo);
            double ja = std::max(0.0, alo), jb = std::min((double)jmax, ahi);
            if (jb > ja) s += (jb - ja) * ahi - (jb - 1 + ja) * (jb - ja) / 2.0;
            total += s;
        } else {  // TRI_UPPER: len = max(0, min(ahi, j+1) - alo)
            double s = 0;
            // j+1 <= ahi  <=> j <= ahi-1 : len = j + 1 - alo (if > 0)
            double ja = std::max(0.0, alo), jb = std::min((double)jmax, ahi);  // j in [alo, ahi)
            if (jb > ja) s += (jb - ja) * (1 - alo) + (jb - 1 + ja) * (jb - ja) / 2.0;
            double jc = std::max(ahi, 0.0);
            if (jmax > jc) s += (jmax - jc) * std::max(0.0, ahi - alo);
            total += s;
        }
    }
    return total * g.batch;
}

// mode < 0 in GemmArgs means "double data, the handle's FP64 contraction mode"
constexpr int GM_DOUBLE = -1;

template <class T> int gm_of() { return std::is_same<T, float>::value ? GM_F32 : GM_DOUBLE; }

void gemm(pssd_handle h, const GemmArgs &g0)
{
    if (g0.m <= 0 || g0.n <= 0 || g0.batch <= 0) return;
    GemmArgs g = g0;
    if (g.mode < 0) g.mode = h->dmode;
    g.wait_limit = h->wait_limit;
    double fl = h->prof ? 2.0 * gemm_macs(g) : 0.0;
    Mark mk = mark(h);
    if (g.mode == GM_OZ && !h->derr) g.mode = GM_DF;   // (no error flag outside a guarded call)
    // very thin or tiny products: the slicing passes would dominate; use float pairs
    // (the slices are FP64-accurate, the float pairs carry ~2^-47 per product)
    if (g.mode == GM_OZ && !h->force_engine && (g.k < 16 || (double)g.m * g.n * g.k * g.batch < 262144.0))
        g.mode = GM_DF;
    if (g.mode == GM_DF) {
        // split each FP64 operand into compact float pairs once (stream-ordered temporaries)
        const int ra = g.ta ? g.k : g.m, cla = g.ta ? g.m : g.k;
        const int rb = g.tb ? g.n : g.k, clb = g.tb ? g.k : g.n;
        const size_t na = (size_t)g.batch * ra * cla, nb = (size_t)g.batch * rb * clb;
        float *ah = (float *)walloc(h, sizeof(float) * na), *al = (float *)walloc(h, sizeof(float) * na);
        {
            Timed t(h, K_HBM, 0, 16.0 * na);
            split_pairs((const double *)g.A, g.lda, g.sA, ra, cla, g.batch, ah, al, h->stream);
        }
        float *bh = ah, *bl = al;
        const bool same = g.B == g.A && rb == ra && clb == cla && g.ldb == g.lda && g.sB == g.sA;
        if (!same) {
            bh = (float *)walloc(h, sizeof(float) * nb); bl = (float *)walloc(h, sizeof(float) * nb);
            Timed t(h, K_HBM, 0, 16.0 * nb);
            split_pairs((const double *)g.B, g.ldb, g.sB, rb, clb, g.batch, bh, bl, h->stream);
        }
        g.lda = cla; g.sA = (long long)ra * cla;
        g.ldb = clb; g.sB = (long long)rb * clb;
        g.A = ah; g.Alo = al; g.B = bh; g.Blo = bl;
    }
    // operand elements read by the preparation passes (for their HBM byte count)
    const double opA = (double)g.batch * g.m * g.k, opB = (double)g.batch * g.n * g.k;
    if (g.mode == GM_OZ) {
        void *ws = walloc(h, oz_gemm_workspace_bytes(g));
        {   // exponent pass (8 B read) + slicing pass (8 B read, 8 slices x 2 B written) per element
            Timed t(h, K_OZPREP, 0, 32.0 * (opA + opB));
            oz_gemm_prepare(g, ws, h->stream);
        }
        Timed t(h, K_OZGEMM, fl);
        int st = oz_gemm_run(g, ws, h->derr, h->stream);
        if (st) { h->last_err = "tensor-core FP64 GEMM setup failed"; throw Fail{PSSD_ERR_CUDA}; }
    } else if (g.mode == GM_F32 && h->use_tc && h->derr) {
        void *ws = walloc(h, tc_gemm_workspace_bytes(g));
        {   // split pass: 4 B read, hi + lo (8 B) written per element
            Timed t(h, K_TCPREP, 0, 12.0 * (opA + opB));
            tc_gemm_prepare(g, ws, h->stream);
        }
        Timed t(h, K_TCGEMM, fl);
        int st = tc_gemm_run(g, ws, h->derr, h->stream);
        if (st) { h->last_err = "tensor-core GEMM setup failed"; throw Fail{PSSD_ERR_CUDA}; }
    } else {
        Timed t(h, g.mode == GM_F32 ? K_SGEMM : (g.mode == GM_DF ? K_DFGEMM : K_DGEMM), fl);
        gemm_launch(g, h->stream);
    }
    release(h, mk);
}

// ---------------------------------------------------------------------------
// small host <-> device helpers
// ---------------------------------------------------------------------------
void h2d(pssd_handle h, void *d, const void *src, size_t bytes)
{
    cuda_check(h, cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, h->stream), "cudaMemcpyAsync H2D");
}

void d2h_sync(pssd_handle h, void *dst, const void *d, size_t bytes)
{
    cuda_check(h, cudaMemcpyAsync(dst, d, bytes, cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync D2H");
    cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
}

void frob_pair(pssd_handle h, const double *X, long long ldx, const double *Y, long long ldy, int m, int n,
               double *part, double *d2, double *y2)
{
    {
        Timed t(h, K_HBM, 0, (X ? 16.0 : 8.0) * m * (double)n);
        frob_diff(X, ldx, Y, ldy, m, n, part, h->stream);
    }
    int nb = frob_blocks(m, n);
    std::vector<double> hp(2 * (size_t)nb);
    d2h_sync(h, hp.data(), part, hp.size() * sizeof(double));
    double a = 0, b = 0;
    for (int i = 0; i < nb; ++i) { a += hp[2 * i]; b += hp[2 * i + 1]; }
    *d2 = a; *y2 = b;
}

// ---------------------------------------------------------------------------
// blocked Cholesky (lower, in place) of `batch` matrices; optional inverse
// ---------------------------------------------------------------------------
template <class T>
T *talloc(pssd_handle h, size_t count) { return (T *)walloc(h, count * sizeof(T)); }

int check_info(pssd_handle h, const int *dinfo, int batch, int *fail_index)
{
    std::vector<int> hi(batch);
    d2h_sync(h, hi.data(), dinfo, sizeof(int) * batch);
    for (int z = 0; z < batch; ++z)
        if (hi[z]) { if (fail_index) *fail_index = hi[z] - 1; return 1; }
    return 0;
}

// Recursive Cholesky with inverse, in place on the diagonal block (off, s):
//   L11 = chol(A11), L21 = A21 L11^{-T}, A22 <- A22 - L21 L21^T, L22 = chol(A22),
//   L^{-1}_21 = -L22^{-1} L21 L11^{-1};
// the work sits in GEMMs of order s/2, which the tensor-core engines take;
// diagonal blocks of at most CholLeaf<T>::max_s are factorised and inverted
// by one fused kernel (one CTA per batch matrix).
template <class T>
void chol_rec(pssd_handle h, T *A, int off, int s, long long lda, long long sA, int batch, T *Rinv, long long sR,
              int *dinfo, T *tmp, long long sT)
{
    if (s <= CholLeaf<T>::max_s) {
        Timed t(h, K_CHOL_LEAF, batch * (double)s * s * s);
        if (chol_leaf<T>(A, lda, sA, Rinv, lda, sR, off, s, batch, dinfo, h->stream)) {
            h->last_err = "Cholesky leaf launch configuration failed";
            throw Fail{PSSD_ERR_CUDA};
        }
        return;
    }
    const int nbk = (s + PB - 1) / PB;
    const int hh = ((nbk + 1) / 2) * PB, q = s - hh;
    chol_rec<T>(h, A, off, hh, lda, sA, batch, Rinv, sR, dinfo, tmp, sT);
    T *A21 = A + (long long)(off + hh) * lda + off;
    T *A22 = A + (long long)(off + hh) * lda + (off + hh);
    {   // L21 = A21 L11^{-T} into tmp (the product reads whole rows of A21), then back
        GemmArgs g; g.mode = gm_of<T>(); g.m = q; g.n = hh; g.k = hh; g.batch = batch;
        g.A = A21; g.lda = lda; g.sA = sA;
        g.B = Rinv + (long long)off * lda + off; g.ldb = lda; g.sB = sR; g.tb = 1; g.triB = TRI_UPPER;
        g.C = tmp; g.ldc = hh; g.sC = sT;
        gemm(h, g);
        Timed t(h, K_HBM, 0, 2.0 * sizeof(T) * q * (double)hh * batch);
        copy_batched<T>(tmp, hh, sT, A21, lda, sA, q, hh, batch, h->stream);
    }
    {   // A22 -= L21 L21^T (lower)
        GemmArgs g; g.mode = gm_of<T>(); g.m = q; g.n = q; g.k = hh; g.batch = batch;
        g.A = A21; g.lda = lda; g.sA = sA; g.B = A21; g.ldb = lda; g.sB = sA; g.tb = 1;
        g.Cin = A22; g.ldcin = lda; g.sCin = sA; g.C = A22; g.ldc = lda; g.sC = sA;
        g.alpha = -1.0; g.beta = 1.0; g.lowerC = 1;
        gemm(h, g);
    }
    chol_rec<T>(h, A, off + hh, q, lda, sA, batch, Rinv, sR, dinfo, tmp, sT);
    if (Rinv) {   // L^{-1}_21 = -L22^{-1} (L21 L11^{-1})
        GemmArgs a; a.mode = gm_of<T>(); a.m = q; a.n = hh; a.k = hh; a.batch = batch;
        a.A = A21; a.lda = lda; a.sA = sA;
        a.B = Rinv + (long long)off * lda + off; a.ldb = lda; a.sB = sR; a.triB = TRI_LOWER;
        a.C = tmp; a.ldc = hh; a.sC = sT;
        gemm(h, a);
        GemmArgs b; b.mode = gm_of<T>(); b.m = q; b.n = hh; b.k = q; b.batch = batch;
        b.A = Rinv + (long long)(off + hh) * lda + (off + hh); b.lda = lda; b.sA = sR; b.triA = TRI_LOWER;
        b.B = tmp; b.ldb = hh; b.sB = sT;
        b.C = Rinv + (long long)(off + hh) * lda + off; b.ldc = lda; b.sC = sR;
        b.alpha = -1.0;
        gemm(h, b);
    }
}

// Cholesky + inverse of `batch` SPD matrices; returns nonzero on breakdown
template <class T>
int chol_inv(pssd_handle h, T *A, int n, long long lda, long long sA, int batch, T *Rinv, long long sR,
             int *fail_index)
{
    Mark mk = mark(h);
    int *dinfo = ialloc(h, batch);
    cuda_check(h, cudaMemsetAsync(dinfo, 0, sizeof(int) * batch, h->stream), "memset");
    size_t tsz = (size_t)((n + 1) / 2 + PB) * ((n + 1) / 2 + PB);
    T *tmp = talloc<T>(h, tsz * batch);
    if (!Rinv) {   // the recursion needs L11^{-1}; keep it in a temporary
        Rinv = talloc<T>(h, (size_t)lda * n * batch);
        sR = lda * (long long)n;
    }
    chol_rec<T>(h, A, 0, n, lda, sA, batch, Rinv, sR, dinfo, tmp, (long long)tsz);
    int bad = check_info(h, dinfo, batch, fail_index);
    release(h, mk);
    return bad;
}

template <class T>
void mirror(pssd_handle h, T *A, long long lda, long long sA, int n, int batch)
{
    Timed t(h, K_HBM, 0, (double)sizeof(T) * n * (double)(n - 1) * batch);
    mirror_lower<T>(A, lda, sA, n, batch, h->stream);
}

// ---------------------------------------------------------------------------
// Tm = sum_j a_j (G + c_{2j-1} I)^{-1} for a symmetric positive (semi)definite m x m G
// (lower part read), full symmetric output: the partial-fraction sum of Eq. ZPartialFrac.
// The r shifted matrices are factorised by one batched Cholesky-with-inverse launch
// sequence, each inverse is R_j^{-T} R_j^{-1} (one batched product, lower) and the
// weighted sum is one HBM pass.
// ---------------------------------------------------------------------------
template <class T>
int shifted_inverse_sum(pssd_handle h, const T *G, int m, int r, const double *c, const double *a, T *Tm,
                        int *fail_index, T *zstore = nullptr)
{
    // zstore (r m^2, optional): receives the r inverses Z_j, full symmetric, for the adjoint
    Mark mk = mark(h);
    const long long ld = m, msz = (long long)m * m;
    T *Z = zstore ? zstore : talloc<T>(h, msz * r);
    T *Ri = talloc<T>(h, msz * r);
    double *dsh = dalloc(h, 2 * r + 2);
    std::vector<double> hs(2 * r);
    for (int j = 0; j < r; ++j) { hs[j] = c[2 * j]; hs[r + j] = a[j]; }
    h2d(h, dsh, hs.data(), sizeof(double) * 2 * r);
    {
        Timed t(h, K_HBM, 0, sizeof(T) * 0.5 * m * (double)m * (1 + r));
        shift_copy_lower<T>(G, ld, Z, ld, msz, m, dsh, r, h->stream);   // Z_j = G + c_{2j-1} I
    }
    int bad = chol_inv<T>(h, Z, m, ld, msz, r, Ri, msz, fail_index);   // R_j, R_j^{-1}
    if (bad) { release(h, mk); return PSSD_ERR_NOT_DEFINITE; }
    GemmArgs l;                                 // Z_j^{-1} = R_j^{-T} R_j^{-1} (lower)
    l.mode = gm_of<T>();
    l.m = l.n = l.k = m; l.batch = r;
    l.A = Ri; l.lda = ld; l.sA = msz; l.ta = 1; l.triA = TRI_UPPER;
    l.B = Ri; l.ldb = ld; l.sB = msz; l.triB = TRI_LOWER;
    l.C = Z; l.ldc = ld; l.sC = msz; l.lowerC = 1;
    gemm(h, l);
    if (zstore) mirror<T>(h, Z, ld, msz, m, r);
    {
        Timed t(h, K_HBM, 0, sizeof(T) * 0.5 * m * (double)m * (r + 1));
        combine_lower<T>(Z, ld, msz, dsh + r, r, m, Tm, ld, h->stream);   // T = sum a_j Z_j^{-1}
    }
    mirror<T>(h, Tm, ld, 0, m, 1);
    release(h, mk);
    return PSSD_OK;
}

// ---------------------------------------------------------------------------
// one Zolotarev step on a symmetric m x m X (full storage):
//   Xn = Chat (X + X T),  T = sum_j a_j (X^2 + c_{2j-1} I)^{-1}
// (Eq. ZPartialFrac applied to the symmetric congruence iterate)
// ---------------------------------------------------------------------------
template <class T>
int zolo_step(pssd_handle h, const T *X, T *Xn, int m, int r, const double *c, const double *a, double chat,
              int *fail_index, const T *G0 = nullptr, double ell = 1.0, T *zstore = nullptr)
{
    Mark mk = mark(h);
    const long long ld = m, msz = (long long)m * m;
    T *Tm = talloc<T>(h, msz);
    const T *G = G0;
    if (!G) {                                   // G = X X (lower), unless the caller has it
        T *Gw = talloc<T>(h, msz);
        GemmArgs g;
        g.mode = gm_of<T>();
        g.m = g.n = g.k = m; g.A = X; g.lda = ld; g.B = X; g.ldb = ld; g.C = Gw; g.ldc = ld; g.lowerC = 1;
        gemm(h, g);
        G = Gw;
    }
    int st = shifted_inverse_sum<T>(h, G, m, r, c, a, Tm, fail_index, zstore);
    if (st) { release(h, mk); return st; }
    // Xn = chat (X + X T).  X and T commute in exact arithmetic, but T is as large as
    // a_1 / (x^2 + c_1) where X has eigenvalues x near 0, and the computed X T carries a
    // commutator error of that size; its symmetric part (X T + T X)/2 cancels the error to
    // first order.  FP64 steps whose lower bound l is small form the full product and
    // average it; later steps (l near 1, T of moderate size) and the FP32 steps (whose
    // shifts are floored away from 0) take the lower triangle and mirror it.
    const bool full = std::is_same<T, double>::value && ell < 0.05;
    GemmArgs f;
    f.mode = gm_of<T>();
    f.m = f.n = f.k = m; f.A = X; f.lda = ld; f.B = Tm; f.ldb = ld; f.Cin = X; f.ldcin = ld;
    f.C = Xn; f.ldc = ld; f.alpha = chat; f.beta = chat; f.lowerC = full ? 0 : 1;
    gemm(h, f);
    if (full) {
        Timed t(h, K_HBM, 0, 2.0 * sizeof(T) * m * (double)m);
        sym_average<T>(Xn, ld, m, h->stream);
    } else {
        mirror<T>(h, Xn, ld, 0, m, 1);
    }
    release(h, mk);
    return PSSD_OK;
}

// one Zolotarev step for the polar factor of a square (non-symmetric) m x m C:
//   Cn = Chat (C + C T),  T = sum_j a_j (C^T C + c_{2j-1} I)^{-1}
// (the same rational function of the singular values as zolo_step applies to
// eigenvalues: Zolo-PD for the polar decomposition, Sec. 5.3)
template <class T>
int zolo_step_polar(pssd_handle h, const T *C, T *Cn, int m, int r, const double *c, const double *a, double chat,
                    int *fail_index)
{
    Mark mk = mark(h);
    const long long ld = m, msz = (long long)m * m;
    T *G = talloc<T>(h, msz);
    T *Tm = talloc<T>(h, msz);
    GemmArgs g;                                 // G = C^T C (lower)
    g.mode = gm_of<T>();
    g.m = g.n = g.k = m; g.A = C; g.lda = ld; g.ta = 1; g.B = C; g.ldb = ld; g.C = G; g.ldc = ld; g.lowerC = 1;
    gemm(h, g);
    int st = shifted_inverse_sum<T>(h, G, m, r, c, a, Tm, fail_index);
    if (st) { release(h, mk); return st; }
    GemmArgs f;                                 // Cn = chat (C + C T)
    f.mode = gm_of<T>();
    f.m = f.n = f.k = m; f.A = C; f.lda = ld; f.B = Tm; f.ldb = ld; f.Cin = C; f.ldcin = ld;
    f.C = Cn; f.ldc = ld; f.alpha = chat; f.beta = chat;
    gemm(h, f);
    release(h, mk);
    return PSSD_OK;
}

struct SignResult { double *Y; };

// Record of a Zolotarev sign computation for the step-reversal adjoint: for every step its
// input iterate X_k (a checkpoint), its coefficients and, unless they are to be recomputed
// from X_k, the shifted inverses Z_j = (X_k^2 + c_{2j-1} I)^{-1} (full, symmetric).  The
// slots are allocated before the iteration (xslot[s]: m^2, zslot[s]: r_s m^2 or null).
struct SignTape {
    struct Step { int r = 0; double c[128], a[64], chat = 0.0; double *X = nullptr, *Z = nullptr; };
    std::vector<Step> steps;
    std::vector<double *> xslot, zslot;
};

// Alg. 8 on the symmetric X0 (scaled so that |lambda| in [ell, 1]); result in Y
// (one of the two ping-pong buffers, returned).  Fills the pass statistics.
// polar: X0 is a square non-symmetric matrix with singular values in [ell, 1] and
// the iteration computes its orthogonal polar factor (the sign of [[0, X0], [X0^T, 0]]).
int zolo_sign(pssd_handle h, double *X0, int m, double ell, int r_opt, int max_restarts, double tau,
              double *bufA, double *bufB, double **Yout, pssd_info *info, int *fail_index, bool polar = false,
              const double *G0 = nullptr, SignTape *tape = nullptr, double accept_s2 = 0.0)
{
    // accept_s2 > 0 (symmetric case): when the stopping test fails, X_2 is still taken if
    // ||X_2^2 - I||_F <= accept_s2 (one product), instead of restarting
    // G0: X0^2 (lower) when the caller has formed it (symmetric case, first step only)
    // tape: record every step for the adjoint (symmetric case)
    double step_ell = 1.0;   // lower bound of the step being taken
    auto step = [&](const double *X, double *Xn, int r, const double *c, const double *a, double chat) {
        const double *G = (X == X0 && !polar) ? G0 : nullptr;
        double *zs = nullptr;
        if (tape && !polar) {
            const size_t s = tape->steps.size();
            if (s >= tape->xslot.size()) return PSSD_ERR_NO_CONVERGENCE;   // more steps than planned
            SignTape::Step rec;
            rec.r = r; rec.chat = chat; rec.X = tape->xslot[s]; rec.Z = tape->zslot[s];
            std::copy(c, c + 2 * r, rec.c);
            std::copy(a, a + r, rec.a);
            {
                Timed t(h, K_HBM, 0, 16.0 * m * (double)m);
                copy_matrix(X, m, rec.X, m, m, m, h->stream);
            }
            zs = rec.Z;
            tape->steps.push_back(rec);
        }
        // The slice engine rounds each product relative to its operands' row and column maxima;
        // a step with l < 1e-6 forms inverses whose entries span ~1/l^2, and their small parts
        // (the directions of the eigenvalues near l) fall below the 56 bits kept per row.  Such
        // steps run their products on the FP64 pipe (the later steps' l is far larger).
        const int saved_mode = h->dmode;
        if (saved_mode != GM_F64 && step_ell < 1e-6) h->dmode = GM_F64;
        const int st = polar ? zolo_step_polar<double>(h, X, Xn, m, r, c, a, chat, fail_index)
                             : zolo_step<double>(h, X, Xn, m, r, c, a, chat, fail_index, G, step_ell, zs);
        h->dmode = saved_mode;
        return st;
    };
    const long long ld = m;
    double *X = X0;
    Mark mk = mark(h);
    double *part = dalloc(h, 2 * (size_t)frob_blocks(m, m));
    int pass = 0;
    for (;; ++pass) {
        if (!(ell > 0.0)) { release(h, mk); return PSSD_ERR_NONFINITE; }
        ell = std::min(ell, 1.0);
        int r = (pass == 0 && r_opt > 0) ? r_opt : choose_r_host(ell, tau, 8);
        double c[128], a[64], chat, ell1, ell2;
        if (zolo_coeffs_host(ell, r, c, a, &chat, &ell1)) { release(h, mk); return PSSD_ERR_NONFINITE; }
        if (ell1 > 1.0) ell1 = 1.0;
        double *X1 = (X == bufA) ? bufB : bufA;
        step_ell = ell;
        int st = step(X, X1, r, c, a, chat);
        if (st) { release(h, mk); return st; }
        if (zolo_coeffs_host(ell1, r, c, a, &chat, &ell2)) { release(h, mk); return PSSD_ERR_NONFINITE; }
        if (ell2 > 1.0) ell2 = 1.0;
        double *X2 = (X1 == bufA) ? bufB : bufA;   // may be X itself on a restart (no longer needed)
        step_ell = ell1;
        st = step(X1, X2, r, c, a, chat);
        if (st) { release(h, mk); return st; }
        double d2, y2;
        frob_pair(h, X1, ld, X2, ld, m, m, part, &d2, &y2);
        double crit = std::sqrt(d2 / y2);
        if (info) {
            if (pass < 4) { info->r_used[pass] = r; info->stop_crit[pass] = crit; }
            if (pass < 2) { info->ell[3 * pass] = ell; info->ell[3 * pass + 1] = ell1; info->ell[3 * pass + 2] = ell2; }
            info->passes = pass + 1; info->steps = 2 * (pass + 1); info->restarts = pass;
            info->iterations = info->steps;
        }
        if (!std::isfinite(crit)) { release(h, mk); return PSSD_ERR_NONFINITE; }
        if (crit <= std::pow(U64, 1.0 / (2 * r + 1))) { *Yout = X2; release(h, mk); return PSSD_OK; }
        if (accept_s2 > 0.0 && !polar) {
            Mark ms = mark(h);
            double *Q2 = dalloc(h, (size_t)m * m);
            GemmArgs g; g.m = g.n = g.k = m; g.A = X2; g.lda = ld; g.B = X2; g.ldb = ld; g.C = Q2; g.ldc = ld;
            gemm(h, g);                                                   // X_2^2
            {
                Timed t(h, K_HBM, 0, 8.0 * m);
                add_diag<double>(Q2, ld, m, -1.0, h->stream);
            }
            double e2, q2;
            frob_pair(h, nullptr, ld, Q2, ld, m, m, part, &e2, &q2);
            release(h, ms);
            if (std::sqrt(q2) <= accept_s2) { *Yout = X2; release(h, mk); return PSSD_OK; }
        }
        if (pass >= max_restarts) { *Yout = X2; release(h, mk); return PSSD_ERR_NO_CONVERGENCE; }
        // restart (reading R6): A <- X_2, alpha = 1, beta = l_2
        ell = ell2;
        X = X2;
    }
}

// Sigma-DWH (the comparison method of Sec. 6): the Zolotarev step of degree 1
// -- the dynamically weighted Halley step, Sec. 5.3 -- repeated on the
// symmetric X0 (|lambda| in [ell, 1]) with the l-update after every step,
// until ||X_{k+1} - X_k||_F / ||X_{k+1}||_F <= u^{1/3}: the step converges
// cubically, so the next step's change would be at rounding level.
int dwh_sign(pssd_handle h, double *X0, int m, double ell, double *bufA, double *bufB, double **Yout,
             pssd_info *info, int *fail_index)
{
    const long long ld = m;
    Mark mk = mark(h);
    double *part = dalloc(h, 2 * (size_t)frob_blocks(m, m));
    double *X = X0;
    const double tol = std::cbrt(U64);
    for (int it = 0; it < 30; ++it) {
        if (!(ell > 0.0)) { release(h, mk); return PSSD_ERR_NONFINITE; }
        ell = std::min(ell, 1.0);
        double c[2], a[1], chat, ell1;
        if (zolo_coeffs_host(ell, 1, c, a, &chat, &ell1)) { release(h, mk); return PSSD_ERR_NONFINITE; }
        double *Xn = (X == bufA) ? bufB : bufA;
        const int saved_mode = h->dmode;   // as in zolo_sign: steps with l < 1e-6 on the FP64 pipe
        if (saved_mode != GM_F64 && ell < 1e-6) h->dmode = GM_F64;
        int st = zolo_step<double>(h, X, Xn, m, 1, c, a, chat, fail_index, nullptr, ell);
        h->dmode = saved_mode;
        if (st) { release(h, mk); return st; }
        double d2, y2;
        frob_pair(h, X, ld, Xn, ld, m, m, part, &d2, &y2);
        const double crit = std::sqrt(d2 / y2);
        if (info) {
            if (it < 6) info->ell[it] = ell;
            if (it < 4) { info->stop_crit[it] = crit; info->r_used[it] = 1; }
            info->iterations = info->steps = it + 1; info->passes = 1;
        }
        if (!std::isfinite(crit)) { release(h, mk); return PSSD_ERR_NONFINITE; }
        ell = std::min(ell1, 1.0);
        X = Xn;
        if (crit <= tol) { *Yout = X; release(h, mk); return PSSD_OK; }
    }
    *Yout = X;
    release(h, mk);
    return PSSD_ERR_NO_CONVERGENCE;
}

// Scaled Newton iteration (Eq. NewtonSign) with the suboptimal scaling of Byers
// and Xu that Sec. 6 compares against: for X0 with |lambda| in [b, a] (here
// a = 1, b = ell), X_{k+1} = (z_k X_k + (z_k X_k)^{-1})/2 with
//   z_0 = 1/sqrt(ab),  z_1 = sqrt(2 sqrt(ab)/(a + b)),  z_{k+1} = 1/sqrt((z_k + 1/z_k)/2);
// after the first step |lambda| lies in [1, (a + b)/(2 sqrt(ab))] and each z_k
// is the optimal scaling for the interval bound carried forward.  The first
// inverse comes from the Cholesky factor of M: X0 = K/alpha with K = L^T Sigma L,
// so X0^{-1} = alpha L^{-1} Sigma L^{-T}; later inverses are (X^2)^{-1} X with the
// Cholesky factor of the SPD X^2 (condition number at most kappa/4 after the
// first step).  Stops when the relative change is at most u^{1/2} (quadratic
// convergence).
int newton_sign(pssd_handle h, const double *Linv, const double *sig, double alpha, double *X0, int m, double ell,
                double *bufA, double *bufB, double **Yout, pssd_info *info, int *fail_index)
{
    const long long ld = m, msz = (long long)m * m;
    Mark mk = mark(h);
    double *part = dalloc(h, 2 * (size_t)frob_blocks(m, m));
    double *G = dalloc(h, msz), *Ri = dalloc(h, msz), *Gi = dalloc(h, msz);
    const double a = 1.0, b = std::min(std::max(ell, 1e-300), 1.0);
    double z = 1.0 / std::sqrt(a * b);
    double *X = X0;
    const double tol = std::sqrt(U64);
    for (int it = 0; it < 60; ++it) {
        double *Xn = (X == bufA) ? bufB : bufA;
        if (it == 0) {   // X1 = (z/2) X0 + (alpha / (2 z)) L^{-1} Sigma L^{-T}   (lower, then mirrored)
            GemmArgs g; g.m = g.n = g.k = m; g.A = Linv; g.lda = ld; g.triA = TRI_LOWER; g.kscale = sig;
            g.B = Linv; g.ldb = ld; g.tb = 1; g.triB = TRI_UPPER; g.Cin = X; g.ldcin = ld;
            g.C = Xn; g.ldc = ld; g.alpha = 0.5 * alpha / z; g.beta = 0.5 * z; g.lowerC = 1;
            gemm(h, g);
        } else {
            GemmArgs g; g.m = g.n = g.k = m; g.A = X; g.lda = ld; g.B = X; g.ldb = ld; g.C = G; g.ldc = ld;
            g.lowerC = 1;
            gemm(h, g);                                                   // G = X^2 (lower)
            if (chol_inv<double>(h, G, m, ld, 0, 1, Ri, 0, fail_index)) { release(h, mk); return PSSD_ERR_NOT_DEFINITE; }
            GemmArgs l; l.m = l.n = l.k = m; l.A = Ri; l.lda = ld; l.ta = 1; l.triA = TRI_UPPER;
            l.B = Ri; l.ldb = ld; l.triB = TRI_LOWER; l.C = Gi; l.ldc = ld; l.lowerC = 1;
            gemm(h, l);                                                   // (X^2)^{-1} = R^{-T} R^{-1}
            mirror<double>(h, Gi, ld, 0, m, 1);
            GemmArgs f; f.m = f.n = f.k = m; f.A = Gi; f.lda = ld; f.B = X; f.ldb = ld; f.Cin = X; f.ldcin = ld;
            f.C = Xn; f.ldc = ld; f.alpha = 0.5 / z; f.beta = 0.5 * z; f.lowerC = 1;
            gemm(h, f);                                                   // (z X + (X^2)^{-1} X / z) / 2
        }
        // lower part, mirrored: the first step is a symmetric sandwich; after it |lambda(X)| >= 1,
        // so (X^2)^{-1} is of moderate size and so is the commutator error of (X^2)^{-1} X
        mirror<double>(h, Xn, ld, 0, m, 1);
        double d2, y2;
        frob_pair(h, X, ld, Xn, ld, m, m, part, &d2, &y2);
        const double crit = std::sqrt(d2 / y2);
        if (info) {
            if (it < 4) info->stop_crit[it] = crit;
            info->iterations = info->steps = it + 1; info->passes = 1;
        }
        if (!std::isfinite(crit)) { release(h, mk); return PSSD_ERR_NONFINITE; }
        X = Xn;
        if (it > 0 && crit <= tol) { *Yout = X; release(h, mk); return PSSD_OK; }
        z = (it == 0) ? std::sqrt(2.0 * std::sqrt(a * b) / (a + b)) : 1.0 / std::sqrt(0.5 * (z + 1.0 / z));
    }
    *Yout = X;
    release(h, mk);
    return PSSD_ERR_NO_CONVERGENCE;
}

// scaled Zolotarev function (Eq. hatZ), product form, for tracking the image of l
double zolo_eval_host(double x, double ell, int r)
{
    double c[128], a[64], chat, l1;
    if (zolo_coeffs_host(ell, r, c, a, &chat, &l1)) return NAN;
    double y = chat * x;
    for (int j = 0; j < r; ++j) y *= (x * x + c[2 * j + 1]) / (x * x + c[2 * j]);
    return y;
}

// Zolotarev steps in FP32 on the symmetric X (|lambda| in [ell, 1]) until the
// image of ell reaches 1 - tau32.  The shifted FP32 Cholesky factorisations
// stay well conditioned because every step uses l_used = max(l, ell_floor):
// c_1(l_used) bounds X^2 + c_1 I below, and eigenvalues below l_used are still
// mapped monotonically upward (their image is tracked exactly on the host).
int zolo_sign_fp32(pssd_handle h, float *X0, int m, double ell, double tau32, double ell_floor, float *bufA,
                   float *bufB, float **Yout, pssd_info *info, int *fail_index)
{
    float *X = X0;
    for (int step = 0; step < 8; ++step) {
        double eu = std::max(ell, ell_floor);
        if (!(eu > 0.0) || !(eu <= 1.0)) return PSSD_ERR_NONFINITE;
        int r = choose_r_host(eu, tau32, 8);
        double c[128], a[64], chat, l1;
        if (zolo_coeffs_host(eu, r, c, a, &chat, &l1)) return PSSD_ERR_NONFINITE;
        float *Xn = (X == bufA) ? bufB : bufA;
        int st = zolo_step<float>(h, X, Xn, m, r, c, a, chat, fail_index);
        if (st) return st;
        double en = std::min(zolo_eval_host(ell, eu, r), 1.0);
        if (!(en > 0.0)) return PSSD_ERR_NONFINITE;
        if (info) {
            if (step < 4) info->r_used[step] = r;
            if (step < 6) info->ell[step] = ell;
            info->fp32_steps = step + 1; info->steps = step + 1; info->passes = 1; info->iterations = step + 1;
        }
        ell = en;
        X = Xn;
        if (1.0 - ell <= tau32) break;
    }
    *Yout = X;
    return PSSD_OK;
}

// Newton-Schulz refinement of a symmetric Y ~ sign(.):  Y <- Y + Y (I - Y^2) / 2
// (the FP64 half of the mixed path; contractions in the handle's FP64 mode).
// Stops when ||I - Y^2||_F <= tol or stops decreasing.
// ||I - Y^2||_F estimated from a Gaussian probe: for Omega (m x s) with
// independent N(0,1) entries E ||(I - Y^2) Omega||_F^2 = s ||I - Y^2||_F^2;
// with s = 64 the estimate is within 25 % of the norm except with
// probability about 1e-3 (chi-square with 64 degrees of freedom).
double ns_probe(pssd_handle h, const double *Y, long long ldy, int m, uint64_t seed)
{
    constexpr int s = 64;
    Mark mk = mark(h);
    double *Om = dalloc(h, (size_t)m * s), *T1 = dalloc(h, (size_t)m * s), *Z = dalloc(h, (size_t)m * s);
    double *part = dalloc(h, 2 * (size_t)frob_blocks(m, s));
    {
        Timed t(h, K_HBM, 0, 8.0 * m * s);
        fill_gaussian(Om, s, m, s, seed, h->stream);
    }
    GemmArgs a; a.m = m; a.n = s; a.k = m; a.A = Y; a.lda = ldy; a.B = Om; a.ldb = s; a.C = T1; a.ldc = s;
    gemm(h, a);                                                          // T1 = Y Omega
    GemmArgs b; b.m = m; b.n = s; b.k = m; b.A = Y; b.lda = ldy; b.B = T1; b.ldb = s;
    b.Cin = Om; b.ldcin = s; b.beta = -1.0; b.C = Z; b.ldc = s;
    gemm(h, b);                                                          // Z = Y^2 Omega - Omega
    double d2, z2;
    frob_pair(h, nullptr, s, Z, s, m, s, part, &d2, &z2);
    release(h, mk);
    return std::sqrt(z2 / s);
}

// Third-order Newton-Schulz refinement towards sign(Y): with E = I - Y^2,
//   Y <- Y (I + E/2 + 3 E^2/8)     (= Y (15 I - 10 Y^2 + 3 Y^4)/8),
// until ||I - Y^2||_F <= tol.  E commutes with Y, so one step maps E to
// (5/8) E^3 + (15/64) E^4 + (9/64) E^5 and ||E_new||_F <= (5/8) r^3 +
// (15/64) r^4 + (9/64) r^5 for r = ||E||_F (up to rounding): from an FP32
// iterate (r ~ 1e-5) one step reaches FP64 rounding, with three products
// (E, P = 3 E^2/8 + E/2, Y + Y P) where two second-order steps take four.
// When the prediction is at most tol, the residual after the step is taken
// from ns_probe instead of forming I - Y^2 (the full product is formed if the
// probe's estimate exceeds tol).
int ns_refine(pssd_handle h, double *Y, int m, double tol, int max_it, double *resid_out, int *its_out,
              bool symmetric = true, long long ldy = 0)
{
    Mark mk = mark(h);
    const long long ld = m, msz = (long long)m * m;
    if (ldy == 0) ldy = ld;
    double *G = dalloc(h, msz), *Yn = dalloc(h, msz), *Pm = dalloc(h, msz);
    double *part = dalloc(h, 2 * (size_t)frob_blocks(m, m));
    double prev = INFINITY, res = INFINITY, predicted = INFINITY;
    int it = 0;
    double *cur = Y;
    long long ldc = ldy;
    for (; it <= max_it; ++it) {
        if (it > 0 && predicted <= tol) {
            const double est = ns_probe(h, cur, ldc, m, 0x9e3779b97f4a7c15ull + (uint64_t)it);
            if (!std::isfinite(est)) { release(h, mk); return PSSD_ERR_NONFINITE; }
            if (est <= tol) { res = est; break; }
        }
        GemmArgs g; g.m = g.n = g.k = m; g.A = cur; g.lda = ldc; g.B = cur; g.ldb = ldc; g.C = G; g.ldc = ld;
        g.alpha = -1.0; g.lowerC = symmetric ? 1 : 0;                   // G = -Y^2
        gemm(h, g);
        if (symmetric) mirror<double>(h, G, ld, 0, m, 1);
        {
            Timed t(h, K_HBM, 0, 16.0 * m);
            add_diag<double>(G, ld, m, 1.0, h->stream);                // G = I - Y^2
        }
        double d2, y2;
        frob_pair(h, nullptr, ld, G, ld, m, m, part, &d2, &y2);
        res = std::sqrt(y2);
        if (!std::isfinite(res)) { release(h, mk); return PSSD_ERR_NONFINITE; }
        if (res <= tol || res > 0.5 * prev || it == max_it) break;
        prev = res;
        predicted = res * res * res * (0.625 + res * (0.234375 + res * 0.140625));
        GemmArgs pp; pp.m = pp.n = pp.k = m; pp.A = G; pp.lda = ld; pp.B = G; pp.ldb = ld; pp.Cin = G; pp.ldcin = ld;
        pp.C = Pm; pp.ldc = ld; pp.alpha = 0.375; pp.beta = 0.5; pp.lowerC = symmetric ? 1 : 0;   // P = 3E^2/8 + E/2
        gemm(h, pp);
        if (symmetric) mirror<double>(h, Pm, ld, 0, m, 1);
        GemmArgs u; u.m = u.n = u.k = m; u.A = cur; u.lda = ldc; u.B = Pm; u.ldb = ld; u.Cin = cur; u.ldcin = ldc;
        u.C = Yn; u.ldc = ld; u.alpha = 1.0; u.beta = 1.0; u.lowerC = symmetric ? 1 : 0;   // Y + Y P
        gemm(h, u);
        if (symmetric) mirror<double>(h, Yn, ld, 0, m, 1);
        if (cur == Y) { cur = Yn; Yn = dalloc(h, msz); } else std::swap(cur, Yn);
        ldc = ld;
    }
    if (cur != Y) {
        Timed t(h, K_HBM, 0, 16.0 * m * (double)m);
        copy_matrix(cur, ld, Y, ldy, m, m, h->stream);
    }
    if (resid_out) *resid_out = res;
    if (its_out) *its_out = it;
    release(h, mk);
    return PSSD_OK;
}

// The operator of a Krylov loop in the form the one-launch cluster kernel takes
// (krylov_cluster: y = A x, or y = L^T (L x) for lower triangular L); A = null: none,
// the loop then runs step by step through its `apply` callback.
struct KryFused {
    const double *A = nullptr;
    long long lda = 0;
    int op = KRY_SYM;
    bool usable(int m) const { return A && m >= 1 && m <= KRY_MAX_M; }
};

// power iteration estimate of lambda_max of an SPD operator given by `apply` (or by `kf`:
// the same iteration in one launch, the same starting vector)
template <class F>
void power_device(pssd_handle h, int n, F apply, double *v, double *w, double *dscal, int iters,
                  const KryFused *kf = nullptr)
{
    if (kf && kf->usable(n) && iters > 0) {
        Timed t(h, K_GEMV, (iters + 1) * 2.0 * n * (double)n, (iters + 1) * 8.0 * n * (double)n);
        krylov_cluster(kf->A, kf->lda, kf->op, n, 0, iters, 0x5eedull, dscal, h->stream);
    } else {
        {
            Timed t(h, K_HBM, 0, 24.0 * n);
            fill_gaussian(v, n, 1, n, 0x5eedull, h->stream);
            normalize_vec(v, v, n, nullptr, h->stream);
        }
        for (int it = 0; it < iters; ++it) {
            apply(v, w);
            Timed t(h, K_GEMV, 0, 16.0 * n);
            normalize_vec(w, v, n, nullptr, h->stream);
        }
        apply(v, w);
        Timed t(h, K_GEMV, 0, 16.0 * n);
        dot_vec(v, w, n, dscal, h->stream);
    }
}

template <class F>
double power_max(pssd_handle h, int n, F apply, double *v, double *w, double *dscal, int iters,
                 const KryFused *kf = nullptr)
{
    power_device(h, n, apply, v, w, dscal, iters, kf);
    double rq;
    d2h_sync(h, &rq, dscal, sizeof(double));
    return rq;
}

// ---------------------------------------------------------------------------
// orthonormal basis of the columns of Y (n x m, ld ldy) by Cholesky QR repeated
// `passes` times (CholeskyQR2 by default) -> U (ld ldu), for `batch` independent
// blocks Y + z sY -> U + z sU
// ---------------------------------------------------------------------------
int cholqr2(pssd_handle h, const double *Y, long long ldy, int n, int m, double *U, long long ldu, int batch = 1,
            long long sY = 0, long long sU = 0, int passes = 2)
{
    Mark mk = mark(h);
    const long long gsz = (long long)m * m, wsz = (long long)n * m;
    double *G = dalloc(h, (size_t)(gsz * batch));
    double *Gi = dalloc(h, (size_t)(gsz * batch));
    double *W = dalloc(h, (size_t)(wsz * batch));
    const double *src = Y; long long lds = ldy, ss = sY;
    for (int pass = 0; pass < passes; ++pass) {
        GemmArgs g;  // G = Y^T Y (lower)
        g.m = g.n = m; g.k = n; g.batch = batch; g.A = src; g.lda = lds; g.sA = ss; g.ta = 1; g.B = src; g.ldb = lds;
        g.sB = ss; g.C = G; g.ldc = m; g.sC = gsz; g.lowerC = 1;
        gemm(h, g);
        int fi;
        if (chol_inv(h, G, m, m, gsz, batch, Gi, gsz, &fi)) { release(h, mk); return PSSD_ERR_BASIS; }
        const bool last = pass == passes - 1;
        double *dst = last ? U : W;
        long long ldd = last ? ldu : m, sd = last ? sU : wsz;
        GemmArgs q;  // U = Y G^{-T}
        q.m = n; q.n = m; q.k = m; q.batch = batch; q.A = src; q.lda = lds; q.sA = ss; q.B = Gi; q.ldb = m;
        q.sB = gsz; q.tb = 1; q.triB = TRI_UPPER; q.C = dst; q.ldc = ldd; q.sC = sd;
        gemm(h, q);
        src = dst; lds = ldd; ss = sd;
    }
    release(h, mk);
    return PSSD_OK;
}

// Symmetric split of B (m x m, symmetric) given Y ~ sign(B - sigma I):
//   U = [U_+ U_-] (m x m, ld m), Bp = U_+^T B U_+ (p x p), Bm = U_-^T B U_- ;
//   E = U_+^T B U_- (p x (m-p)) if E != nullptr.
// The sketch (I +- Y)/2 Omega has the condition number of a Gaussian block, which
// multiplies the projector's error in the cross product U_+^T U_-.  refine: apply
// the projectors once more to the orthonormal bases, (I +- Y)/2 U_+-, and take one
// Cholesky QR pass of the result (condition number 1 + O(error)), which brings
// ||U^T U - I|| back to the projector's own error.
int sym_split(pssd_handle h, const double *B, const double *Y, int m, int p, double *U, double *Bp, double *Bm,
              double *E, uint64_t seed, bool refine = false)
{
    Mark mk = mark(h);
    const long long ld = m;
    double *Om = dalloc(h, (size_t)m * m);
    double *Yb = dalloc(h, (size_t)m * m);
    {
        Timed t(h, K_HBM, 0, 8.0 * m * (double)m);
        fill_gaussian(Om, ld, m, m, seed, h->stream);
    }
    // [Y_+ Y_-] = [(I + Y)/2 Omega_+, (I - Y)/2 Omega_-]: one product Y Omega, then one pass
    auto project = [&](const double *X) {
        GemmArgs g; g.m = m; g.n = m; g.k = m; g.A = Y; g.lda = ld; g.B = X; g.ldb = ld; g.C = Yb; g.ldc = ld;
        gemm(h, g);
        Timed t(h, K_HBM, 0, 24.0 * m * (double)m);
        half_sum_diff(X, ld, Yb, ld, m, m, p, h->stream);
    };
    project(Om);
    int st = PSSD_OK;
    if (p > 0 && p == m - p) {   // equal halves: both bases in one batched pass
        st = cholqr2(h, Yb, ld, m, p, U, ld, 2, p, p);
    } else {
        if (p > 0) st = cholqr2(h, Yb, ld, m, p, U, ld);
        if (!st && m - p > 0) st = cholqr2(h, Yb + p, ld, m, m - p, U + p, ld);
    }
    if (!st && refine) {
        project(U);   // [(I + Y)/2 U_+, (I - Y)/2 U_-]
        if (p > 0 && p == m - p) {
            st = cholqr2(h, Yb, ld, m, p, U, ld, 2, p, p, 1);
        } else {
            if (p > 0) st = cholqr2(h, Yb, ld, m, p, U, ld, 1, 0, 0, 1);
            if (!st && m - p > 0) st = cholqr2(h, Yb + p, ld, m, m - p, U + p, ld, 1, 0, 0, 1);
        }
    }
    if (st) { release(h, mk); return st; }
    double *W = Yb;   // reuse: W = B U  (m x m)
    {
        GemmArgs g; g.m = m; g.n = m; g.k = m; g.A = B; g.lda = ld; g.B = U; g.ldb = ld; g.C = W; g.ldc = ld;
        gemm(h, g);
    }
    if (p > 0) {
        GemmArgs g; g.m = p; g.n = p; g.k = m; g.A = U; g.lda = ld; g.ta = 1; g.B = W; g.ldb = ld;
        g.C = Bp; g.ldc = p; g.lowerC = 1;
        gemm(h, g);
        mirror(h, Bp, p, 0, p, 1);
    }
    if (m - p > 0) {
        GemmArgs g; g.m = m - p; g.n = m - p; g.k = m; g.A = U + p; g.lda = ld; g.ta = 1; g.B = W + p; g.ldb = ld;
        g.C = Bm; g.ldc = m - p; g.lowerC = 1;
        gemm(h, g);
        mirror(h, Bm, m - p, 0, m - p, 1);
    }
    if (E && p > 0 && m - p > 0) {   // E = U_+^T B U_- : the off-diagonal block left by the split
        GemmArgs g; g.m = p; g.n = m - p; g.k = m; g.A = U; g.lda = ld; g.ta = 1; g.B = W + p; g.ldb = ld;
        g.C = E; g.ldc = m - p;
        gemm(h, g);
    }
    release(h, mk);
    return PSSD_OK;
}

// backward error of the split of K by the basis U = [U_+ U_-]:
// ||U_+^T K U_-||_F / ||K||_F, exactly from E = U_+^T K U_- when E is given,
// else estimated with a Gaussian probe Omega ((n-p) x 16, N(0,1) entries):
// E ||E Omega||_F^2 = 16 ||E||_F^2, with E Omega = U_+^T (K (U_- Omega)).
double split_backward_error(pssd_handle h, const double *K, const double *U, int n, int p, const double *E)
{
    constexpr int s = 16;
    const int q = n - p;
    const long long ld = n;
    Mark mk = mark(h);
    double *part = dalloc(h, 2 * (size_t)frob_blocks(n, n));
    double d2, e2, k2;
    if (E) {
        frob_pair(h, nullptr, q, E, q, p, q, part, &d2, &e2);
    } else {
        double *Om = dalloc(h, (size_t)q * s), *T1 = dalloc(h, (size_t)n * s), *T2 = dalloc(h, (size_t)n * s);
        double *T3 = dalloc(h, (size_t)p * s);
        {
            Timed t(h, K_HBM, 0, 8.0 * q * s);
            fill_gaussian(Om, s, q, s, 0xbac3e77ull, h->stream);
        }
        GemmArgs a; a.m = n; a.n = s; a.k = q; a.A = U + p; a.lda = ld; a.B = Om; a.ldb = s; a.C = T1; a.ldc = s;
        gemm(h, a);                                                      // U_- Omega
        GemmArgs b; b.m = n; b.n = s; b.k = n; b.A = K; b.lda = ld; b.B = T1; b.ldb = s; b.C = T2; b.ldc = s;
        gemm(h, b);                                                      // K U_- Omega
        GemmArgs c; c.m = p; c.n = s; c.k = n; c.A = U; c.lda = ld; c.ta = 1; c.B = T2; c.ldb = s; c.C = T3;
        c.ldc = s;
        gemm(h, c);                                                      // U_+^T K U_- Omega
        frob_pair(h, nullptr, s, T3, s, p, s, part, &d2, &e2);
        e2 /= s;
    }
    frob_pair(h, nullptr, ld, K, ld, n, n, part, &d2, &k2);
    release(h, mk);
    return std::sqrt(e2 / k2);
}

// Relative commutator ||S H - H S||_F / ||H||_F (Lemma SignProj: the projectors
// (I +- S)/2 are spectral exactly when S commutes with H).  S is given either
// explicitly (S != nullptr, ld lds) or as S = A A^T Sigma with A = Q of a split
// or V of a diagonalisation (A^{-1} = Sigma_hat A^T Sigma and Sigma_hat^2 = I, so
// S = A Sigma_hat A^{-1} = A A^T Sigma).  exact: forms S H - H S (two n^3
// products); otherwise a 16-column Gaussian probe, E ||C Omega||_F^2 = 16 ||C||_F^2.
double comm_resid(pssd_handle h, int n, const double *H, long long ldh, double normH, const double *S,
                  long long lds, const double *A, long long lda, const double *sig, bool exact)
{
    Mark mk = mark(h);
    const long long nn = (long long)n * n;
    double d2 = 0, c2 = 0;
    if (exact) {
        double *Sm = const_cast<double *>(S);
        long long ldm = lds;
        if (!S) {
            Sm = dalloc(h, nn); ldm = n;
            GemmArgs g; g.m = g.n = g.k = n; g.A = A; g.lda = lda; g.B = A; g.ldb = lda; g.tb = 1;
            g.C = Sm; g.ldc = n;
            gemm(h, g);                                                        // A A^T
            Timed t(h, K_HBM, 0, 16.0 * nn);
            scale_columns(Sm, n, n, n, sig, 0, h->stream);                     // (A A^T) Sigma
        }
        double *C = dalloc(h, nn);
        GemmArgs a; a.m = a.n = a.k = n; a.A = Sm; a.lda = ldm; a.B = H; a.ldb = ldh; a.C = C; a.ldc = n;
        gemm(h, a);                                                            // S H
        GemmArgs b; b.m = b.n = b.k = n; b.A = H; b.lda = ldh; b.B = Sm; b.ldb = ldm; b.Cin = C; b.ldcin = n;
        b.C = C; b.ldc = n; b.alpha = -1.0; b.beta = 1.0;
        gemm(h, b);                                                            // S H - H S
        double *part = dalloc(h, 2 * (size_t)frob_blocks(n, n));
        frob_pair(h, nullptr, n, C, n, n, n, part, &d2, &c2);
    } else {
        constexpr int s = 16;
        double *Om = dalloc(h, (size_t)n * s), *HO = dalloc(h, (size_t)n * s), *T = dalloc(h, (size_t)n * s);
        double *SHO = dalloc(h, (size_t)n * s), *SO = dalloc(h, (size_t)n * s);
        {
            Timed t(h, K_HBM, 0, 8.0 * n * s);
            fill_gaussian(Om, s, n, s, 0xc033e7ull, h->stream);
        }
        auto applyS = [&](const double *x, double *y) {   // y = S x  (n x s blocks, ld s)
            if (S) {
                GemmArgs g; g.m = n; g.n = s; g.k = n; g.A = S; g.lda = lds; g.B = x; g.ldb = s; g.C = y; g.ldc = s;
                gemm(h, g);
            } else {
                GemmArgs g; g.m = n; g.n = s; g.k = n; g.A = A; g.lda = lda; g.ta = 1; g.B = x; g.ldb = s;
                g.kscale = sig; g.C = T; g.ldc = s;
                gemm(h, g);                                                    // A^T Sigma x
                GemmArgs f; f.m = n; f.n = s; f.k = n; f.A = A; f.lda = lda; f.B = T; f.ldb = s; f.C = y; f.ldc = s;
                gemm(h, f);                                                    // A (A^T Sigma x)
            }
        };
        GemmArgs g; g.m = n; g.n = s; g.k = n; g.A = H; g.lda = ldh; g.B = Om; g.ldb = s; g.C = HO; g.ldc = s;
        gemm(h, g);                                                            // H Omega
        applyS(HO, SHO);                                                       // S H Omega
        applyS(Om, SO);                                                        // S Omega
        GemmArgs c; c.m = n; c.n = s; c.k = n; c.A = H; c.lda = ldh; c.B = SO; c.ldb = s; c.Cin = SHO; c.ldcin = s;
        c.C = SHO; c.ldc = s; c.alpha = -1.0; c.beta = 1.0;
        gemm(h, c);                                                            // (S H - H S) Omega
        double *part = dalloc(h, 2 * (size_t)frob_blocks(n, s));
        frob_pair(h, nullptr, s, SHO, s, n, s, part, &d2, &c2);
        c2 /= s;
    }
    release(h, mk);
    return normH > 0 ? std::sqrt(c2) / normH : NAN;
}

// eigenvalues (ascending) and eigenvectors (columns of Z, row-major n x n) of a small
// symmetric matrix by cyclic Jacobi on the host
void small_sym_eig(std::vector<double> A, int n, std::vector<double> &w, std::vector<double> &Z)
{
    Z.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += A[(size_t)i * n + j] * A[(size_t)i * n + j];
                if (i != j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {   // A <- A J (columns p, q)
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {   // A <- J^T A (rows p, q)
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {   // Z <- Z J
                    const double zkp = Z[(size_t)k * n + p], zkq = Z[(size_t)k * n + q];
                    Z[(size_t)k * n + p] = c * zkp - sn * zkq;
                    Z[(size_t)k * n + q] = sn * zkp + c * zkq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return A[(size_t)x * n + x] < A[(size_t)y * n + y]; });
    std::vector<double> Zs((size_t)n * n);
    w.resize(n);
    for (int j = 0; j < n; ++j) {
        w[j] = A[(size_t)idx[j] * n + idx[j]];
        for (int i = 0; i < n; ++i) Zs[(size_t)i * n + j] = Z[(size_t)i * n + idx[j]];
    }
    Z.swap(Zs);
}

// Lanczos quadrature of the spectrum of a symmetric m x m B: s steps from a Gaussian
// start vector v give a tridiagonal T whose eigenvalues theta_j (ascending) and squared
// first eigenvector components tau_j are the nodes and weights of the Gauss rule for the
// spectral measure of v; with v random, sum_{theta_j <= x} tau_j approximates the
// fraction of the eigenvalues of B below x, and wide gaps between consecutive nodes mark
// sparse parts of the spectrum.  The recurrence runs on the device (alpha_j, beta_j stay
// in device memory); the host reads T once.  *resid = beta_s, the norm of the residual
// after the last step: [theta_1 - beta_s, theta_s + beta_s] encloses the spectrum of B in
// practice (the extreme Ritz values converge first, from inside).  Returns false if the
// recurrence produced a non-finite value.
// `steps` Lanczos steps from the seeded Gaussian vector: ab[j] = alpha_j, ab[steps + 1 + j] =
// beta_j (device), step by step through `apply`, or in one launch through `kf` when m fits it
template <class F>
void lanczos_device(pssd_handle h, int m, F apply, uint64_t seed, int steps, double *ab, const KryFused *kf)
{
    if (kf && kf->usable(m)) {
        Timed t(h, K_GEMV, steps * 2.0 * m * (double)m, steps * 8.0 * m * (double)m);
        krylov_cluster(kf->A, kf->lda, kf->op, m, steps, 0, seed, ab, h->stream);
        return;
    }
    Mark mk = mark(h);
    double *V = dalloc(h, 3 * (size_t)m);
    double *vp = V, *vc = V + m, *w = V + 2 * m;
    double *al = ab, *be = ab + steps + 1;
    {
        Timed t(h, K_GEMV, 0, 24.0 * m);
        fill_gaussian(vc, m, 1, m, seed, h->stream);
        normalize_vec(vc, vc, m, nullptr, h->stream);
    }
    for (int j = 0; j < steps; ++j) {
        apply(vc, w);                                                         // w = A v_j
        Timed t(h, K_GEMV, 0, 40.0 * m);
        dot_vec(vc, w, m, al + j, h->stream);                                 // alpha_j
        lanczos_update(w, vc, j ? vp : nullptr, al + j, j ? be + j - 1 : nullptr, m, h->stream);
        normalize_vec(w, vp, m, be + j, h->stream);                           // beta_j, v_{j+1}
        std::swap(vp, vc);
    }
    release(h, mk);
}

template <class F>
bool lanczos_run(pssd_handle h, int m, F apply, uint64_t seed, std::vector<double> &th, std::vector<double> &tau,
                 double *resid, double *rtop = nullptr, const KryFused *kf = nullptr)
{
    // apply(v, w): w = A v for the symmetric operator A (m-vectors on the device); kf: the
    // same operator for the one-launch loop (used when m fits it).
    // rtop (optional): beta_s |z_s| of the largest Ritz value, the norm of its Ritz residual
    const int steps = std::min(m, 24);
    Mark mk = mark(h);
    double *ab = dalloc(h, 2 * (size_t)steps + 2);
    lanczos_device(h, m, apply, seed, steps, ab, kf);
    std::vector<double> hab(2 * (size_t)steps + 2);
    d2h_sync(h, hab.data(), ab, hab.size() * sizeof(double));
    release(h, mk);
    int s = steps;
    for (int j = 0; j < steps - 1; ++j)
        if (!(hab[steps + 1 + j] > 1e-12 * std::fabs(hab[j]) + 1e-300)) { s = j + 1; break; }
    std::vector<double> T((size_t)s * s, 0.0), Z;
    for (int j = 0; j < s; ++j) {
        T[(size_t)j * s + j] = hab[j];
        if (j + 1 < s) T[(size_t)j * s + j + 1] = T[(size_t)(j + 1) * s + j] = hab[steps + 1 + j];
    }
    for (double x : T) if (!std::isfinite(x)) return false;
    *resid = std::fabs(hab[steps + 1 + s - 1]);
    if (!std::isfinite(*resid)) return false;
    small_sym_eig(T, s, th, Z);
    tau.resize(s);
    for (int j = 0; j < s; ++j) tau[j] = Z[j] * Z[j];   // first component of eigenvector j
    if (rtop) *rtop = *resid * std::fabs(Z[(size_t)(s - 1) * s + (s - 1)]);
    return true;
}

bool lanczos_nodes(pssd_handle h, const double *B, int m, uint64_t seed, std::vector<double> &th,
                   std::vector<double> &tau, double *resid)
{
    Mark mk = mark(h);
    double *tmp = dalloc(h, 32 * (size_t)m + 8);
    KryFused kf; kf.A = B; kf.lda = m; kf.op = KRY_SYM;
    const bool ok = lanczos_run(h, m, [&](const double *x, double *y) {
        Timed t(h, K_GEMV, 2.0 * m * (double)m, 8.0 * m * (double)m);
        gemv(B, m, 0, TRI_NONE, m, x, y, tmp, h->stream);
    }, seed, th, tau, resid, nullptr, &kf);
    release(h, mk);
    return ok;
}

// An estimate of lambda_max of a symmetric positive semidefinite operator (apply: y = A x)
// from below: the largest Ritz value of 24 Lanczos steps (the extreme Ritz value converges
// first and faster than the power method's Rayleigh quotient), or 60 power steps if the
// recurrence fails.  Callers add their safety factors (reading R5).
template <class F>
double lmax_estimate(pssd_handle h, int n, F apply, uint64_t seed, double *v, double *w, double *dscal,
                     const KryFused *kf = nullptr)
{
    std::vector<double> th, tau;
    double res;
    if (lanczos_run(h, n, apply, seed, th, tau, &res, nullptr, kf) && th.back() > 0.0) return th.back();
    return power_max(h, n, apply, v, w, dscal, 60, kf);
}

// symmetric eigendecomposition of B (m x m) by Alg. 2 with Zolotarev signs
// and Jacobi leaves: W (m x m, ld m) eigenvectors as columns, w eigenvalues
// (device).  B is preserved.
int sym_eig_node(pssd_handle h, const double *B, int m, double *W, double *w, int leaf, int depth, int *maxdepth,
                 uint64_t seed)
{
    if (depth > *maxdepth) *maxdepth = depth;
    PhaseScope phase(m <= leaf ? PH_LEAF : PH_SHIFT);
    if (m <= leaf) {
        // a Jacobi leaf is one CTA: it runs on the side stream, after the main stream has
        // produced B, while the recursion goes on with the sibling; the parent joins it before
        // forming its eigenvectors (B, W and w belong to the parent until then)
        if (!h->side) cuda_check(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking), "cudaStreamCreate");
        cudaEvent_t ready = sync_event(h), done = sync_event(h);
        cuda_check(h, cudaEventRecord(ready, h->stream), "cudaEventRecord");
        cuda_check(h, cudaStreamWaitEvent(h->side, ready, 0), "cudaStreamWaitEvent");
        {
            Timed t(h, K_JACOBI, 0, 0.0, h->side);
            jacobi_leaf(const_cast<double *>(B), m, m, W, m, w, nullptr, h->side);
        }
        cuda_check(h, cudaEventRecord(done, h->side), "cudaEventRecord");
        h->leaf_pending.push_back(done);
        return PSSD_OK;
    }
    const long long ld = m, msz = (long long)m * m;
    Mark outer = mark(h);
    std::vector<double> dg(m);
    double *dd = dalloc(h, m);
    {
        Timed t(h, K_HBM, 0, 16.0 * m);
        get_diag(B, ld, m, dd, h->stream);
    }
    d2h_sync(h, dg.data(), dd, sizeof(double) * m);
    std::vector<double> srt = dg;
    std::sort(srt.begin(), srt.end());
    double dmin = srt.front(), dmax = srt.back();
    double *U = dalloc(h, msz);
    int p = 0;
    // Candidate shifts (Alg. 2, "find shift"; reading R7).  The inverse-form Zolotarev step
    // loses accuracy like u / xmin, xmin = min |lambda(X0)| of X0 = (B - sigma I)/alpha, so the
    // shift should sit in a sparse part of the spectrum but still split it roughly in half:
    // the midpoints of the widest gaps between Lanczos quadrature nodes whose cumulative
    // weight lies in [0.35, 0.65], the median of the diagonal, the widest gaps with weight in
    // [0.25, 0.75], then points of the diagonal's range (fallbacks).
    std::vector<double> cands;
    double lan_lo = 0.0, lan_hi = -1.0;   // spectral enclosure from the Lanczos run (empty if it failed)
    bool deg = false;
    {
        std::vector<double> th, tau;
        std::vector<std::pair<double, double>> inner, outer_gaps;   // (width, midpoint)
        double bs;
        if (lanczos_nodes(h, B, m, seed ^ 0x1a2c05ull, th, tau, &bs)) {
            // a recurrence that broke down early (B v in a small Krylov space: a few distinct
            // eigenvalues) gives no reliable enclosure; keep the infinity norm then
            if (th.size() >= 8) { lan_lo = th.front() - bs; lan_hi = th.back() + bs; }
            // B = sigma I to rounding (a multiple eigenvalue): any orthonormal basis diagonalises it
            const double scale = std::max(std::fabs(th.front()), std::fabs(th.back()));
            if (th.back() - th.front() + 2.0 * bs <= 32.0 * DBL_EPSILON * scale) deg = true;
            double cum = 0.0;
            for (size_t j = 0; j + 1 < th.size(); ++j) {
                cum += tau[j];
                const std::pair<double, double> gp{th[j + 1] - th[j], 0.5 * (th[j] + th[j + 1])};
                if (cum >= 0.35 && cum <= 0.65) inner.push_back(gp);
                else if (cum >= 0.25 && cum <= 0.75) outer_gaps.push_back(gp);
            }
            std::sort(inner.rbegin(), inner.rend());
            std::sort(outer_gaps.rbegin(), outer_gaps.rend());
        }
        for (size_t i = 0; i < inner.size() && i < 3; ++i) cands.push_back(inner[i].second);
        cands.push_back(0.5 * (srt[(m - 1) / 2] + srt[m / 2]));
        for (size_t i = 0; i < outer_gaps.size() && i < 2; ++i) cands.push_back(outer_gaps[i].second);
        for (int a = 1; a <= 3; ++a) cands.push_back(dmin + (dmax - dmin) * (0.5 + 0.11 * a));
    }
    double *Xa = dalloc(h, msz), *Ga = dalloc(h, msz), *Xb = dalloc(h, msz), *Gb = dalloc(h, msz);
    double *tmp = dalloc(h, 32 * (size_t)m + 8);
    // X0 = (B - sigma I)/alpha and G = X0^2 (lower); false if B = sigma I.  alpha bounds
    // ||B - sigma I||_2: ||B - sigma I||_inf always does, but overestimates a dense matrix's
    // 2-norm by a factor growing like sqrt(m), which shrinks every |lambda(X0)| (and so the
    // accuracy and the convergence rate of the sign iteration) by the same factor; the
    // Lanczos enclosure is within a small factor of the 2-norm and is taken when smaller.
    auto prepare = [&](double sigma, double *X0, double *G, double &alpha) -> bool {
        {
            Timed t(h, K_HBM, 0, 24.0 * m * (double)m);
            copy_matrix(B, ld, X0, ld, m, m, h->stream);
            add_diag(X0, ld, m, -sigma, h->stream);
            row_abs_sum_max(X0, ld, m, tmp, tmp + m, h->stream);
        }
        d2h_sync(h, &alpha, tmp + m, sizeof(double));
        if (!(alpha > 0.0)) return false;
        if (lan_hi >= lan_lo) {
            const double a2 = std::max(lan_hi - sigma, sigma - lan_lo);
            if (a2 > 0.0 && a2 < alpha) alpha = a2;
        }
        {
            Timed t(h, K_HBM, 0, 16.0 * m * (double)m);
            scale_copy(X0, ld, X0, ld, m, m, 1.0 / alpha, h->stream);
        }
        GemmArgs g; g.m = g.n = g.k = m; g.A = X0; g.lda = ld; g.B = X0; g.ldb = ld; g.C = G; g.ldc = ld; g.lowerC = 1;
        gemm(h, g);
        return true;
    };
    // xmin^2 = lambda_min(G) by 20 steps of power iteration on G^{-1} = R^{-T} R^{-1}
    // (R = chol(G)); 0 if G is not numerically positive definite (sigma on an eigenvalue)
    auto screen = [&](const double *G) -> double {
        Mark ms = mark(h);
        double *Rc = dalloc(h, msz), *Ri = dalloc(h, msz), *v = dalloc(h, m), *vw = dalloc(h, m), *u = dalloc(h, m);
        {
            Timed t(h, K_HBM, 0, 16.0 * m * (double)m);
            copy_matrix(G, ld, Rc, ld, m, m, h->stream);
        }
        int fi;
        double xm = 0.0;
        if (!chol_inv<double>(h, Rc, m, ld, 0, 1, Ri, 0, &fi)) {
            KryFused kf; kf.A = Ri; kf.lda = ld; kf.op = KRY_TRI_PAIR;
            const double rq = power_max(h, m, [&](double *x, double *y) {
                Timed t(h, K_GEMV, 2.0 * m * (double)m, 8.0 * m * (double)m);
                gemv(Ri, ld, 0, TRI_LOWER, m, x, u, tmp, h->stream);      // R^{-1} x
                gemv(Ri, ld, 1, TRI_UPPER, m, u, y, tmp, h->stream);      // R^{-T} .
            }, v, vw, tmp + 32 * (size_t)m, 20, &kf);
            if (rq > 0.0 && std::isfinite(rq)) xm = 1.0 / std::sqrt(rq);
        }
        release(h, ms);
        return xm;
    };
    auto identity = [&]() {   // B = sigma I: any orthonormal basis diagonalises it
        std::vector<double> eye((size_t)m * m, 0.0);
        for (int i = 0; i < m; ++i) eye[(size_t)i * m + i] = 1.0;
        h2d(h, W, eye.data(), sizeof(double) * msz);
        h2d(h, w, dg.data(), sizeof(double) * m);
        cudaStreamSynchronize(h->stream);
        release(h, outer);
        return PSSD_OK;
    };
    if (deg) return identity();
    double best_x = -1.0;
    size_t ci = 0;
    for (int screened = 0; ci < cands.size() && screened < 3; ++ci, ++screened) {
        double alpha;
        if (!prepare(cands[ci], Xa, Ga, alpha)) return identity();
        const double xm = screen(Ga);
        if (xm > best_x) { best_x = xm; std::swap(Xa, Xb); std::swap(Ga, Gb); }
        if (best_x >= 1e-5) { ++ci; break; }
    }
    for (int attempt = 0;; ++attempt) {
        double *X0, *G0, ell;
        if (attempt == 0 && best_x > 0.0) {
            // the screened shift; l from the estimate (the power iteration approaches xmin from
            // above, hence the factor); a wrong l shows in the stopping test and falls back
            X0 = Xb; G0 = Gb; ell = std::max(1e-10, 0.3 * best_x);
        } else {
            if (ci >= cands.size()) { release(h, outer); return PSSD_ERR_BASIS; }
            g_phase = PH_SHIFT;
            double alpha;
            if (!prepare(cands[ci++], Xa, Ga, alpha)) return identity();
            X0 = Xa; G0 = Ga; ell = 1e-10;   // conservative lower bound on |lambda(X0)|
        }
        Mark mk = mark(h);
        double *bA = dalloc(h, msz), *bB = dalloc(h, msz);
        double *Y = nullptr;
        int fi;
        // Alg. 2's iteration: X_2 is accepted once it meets the involution bound 1e-12 m
        // (the stopping test of Alg. 8 compares X_2 with the unconverged X_1; reading R6)
        g_phase = PH_NODE_SIGN;
        int st = zolo_sign(h, X0, m, ell, 0, 2, 1e-15, bA, bB, &Y, nullptr, &fi, false, G0, nullptr, 1e-12 * m);
        if (st == PSSD_ERR_NOT_DEFINITE || st == PSSD_ERR_NO_CONVERGENCE || st == PSSD_ERR_NONFINITE) {
            release(h, mk);
            continue;
        }
        if (st) { release(h, outer); return st; }
        g_phase = PH_NODE_SPLIT;
        {
            Timed t(h, K_HBM, 0, 8.0 * m);
            trace_partial(Y, ld, m, tmp, h->stream);
        }
        double tr;
        d2h_sync(h, &tr, tmp, sizeof(double));
        p = (int)std::lround(0.5 * (m + tr));
        if (p <= 0 || p >= m) { release(h, mk); continue; }
        // bases and projected blocks; Bp, Bm persist below the Zolotarev temporaries
        double *Bp = dalloc(h, (size_t)p * p), *Bm = dalloc(h, (size_t)(m - p) * (m - p));
        st = sym_split(h, B, Y, m, p, U, Bp, Bm, nullptr, seed + 17 * depth + attempt, true);
        if (st) { release(h, mk); continue; }
        // recurse
        double *Wp = dalloc(h, (size_t)p * p), *Wm = dalloc(h, (size_t)(m - p) * (m - p));
        st = sym_eig_node(h, Bp, p, Wp, w, leaf, depth + 1, maxdepth, seed * 3 + 1);
        if (!st) st = sym_eig_node(h, Bm, m - p, Wm, w + p, leaf, depth + 1, maxdepth, seed * 3 + 2);
        if (st) { release(h, outer); return st; }
        g_phase = PH_ASSEMBLE;
        join_leaves(h);
        {   // W = [U_+ W_+, U_- W_-]
            GemmArgs g; g.m = m; g.n = p; g.k = p; g.A = U; g.lda = ld; g.B = Wp; g.ldb = p; g.C = W; g.ldc = ld;
            gemm(h, g);
            GemmArgs g2; g2.m = m; g2.n = m - p; g2.k = m - p; g2.A = U + p; g2.lda = ld; g2.B = Wm; g2.ldb = m - p;
            g2.C = W + p; g2.ldc = ld;
            gemm(h, g2);
        }
        release(h, mk);
        break;
    }
    release(h, outer);
    return PSSD_OK;
}

// Alg. 2 from the outside: the recursion, then the main stream joins its last leaves
int sym_eig(pssd_handle h, const double *B, int m, double *W, double *w, int leaf, int depth, int *maxdepth,
            uint64_t seed)
{
    const int st = sym_eig_node(h, B, m, W, w, leaf, depth, maxdepth, seed);
    join_leaves(h);
    return st;
}

// One step of iterative refinement of an approximate eigendecomposition A ~ Z diag(d) Z^T
// of a symmetric m x m A (Ogita and Aishima, "Iterative refinement for symmetric
// eigenvalue decomposition", 2018): from the first-order expansion of the exact
// eigenvectors Z (I + F), with S = Z^T A Z and R = I - Z^T Z,
//   d_i = S_ii / (1 - R_ii),  F_ii = R_ii / 2,
//   F_ij = (S_ij + d_j R_ij) / (d_j - d_i) for pairs farther apart than
//   omega = 2 (||offdiag S||_F + max|d| ||R||_F), else R_ij / 2,
// and Z <- Z + Z F.  The splits of the recursion leave a residual set by the sign
// iteration's accuracy; one step brings ||A Z - Z D|| / ||A|| and ||Z^T Z - I|| down to
// the rounding level of the products above.  Z (ld ldz) and d (device) in place.
int sym_refine(pssd_handle h, const double *A, long long lda, int m, double *Z, long long ldz, double *d)
{
    Mark mk = mark(h);
    const long long msz = (long long)m * m;
    double *W = dalloc(h, msz), *S = dalloc(h, msz), *Gm = dalloc(h, msz), *dg = dalloc(h, 2 * (size_t)m);
    double *part = dalloc(h, 2 * (size_t)frob_blocks(m, m));
    {
        GemmArgs g; g.m = g.n = g.k = m; g.A = A; g.lda = lda; g.B = Z; g.ldb = ldz; g.C = W; g.ldc = m;
        gemm(h, g);                                                          // A Z
        GemmArgs s2; s2.m = s2.n = m; s2.k = m; s2.A = Z; s2.lda = ldz; s2.ta = 1; s2.B = W; s2.ldb = m;
        s2.C = S; s2.ldc = m; s2.lowerC = 1;
        gemm(h, s2);                                                         // S = Z^T A Z (lower)
        GemmArgs gg; gg.m = gg.n = m; gg.k = m; gg.A = Z; gg.lda = ldz; gg.ta = 1; gg.B = Z; gg.ldb = ldz;
        gg.C = Gm; gg.ldc = m; gg.lowerC = 1;
        gemm(h, gg);                                                         // Z^T Z (lower)
    }
    mirror(h, S, m, 0, m, 1);
    mirror(h, Gm, m, 0, m, 1);
    {
        Timed t(h, K_HBM, 0, 16.0 * m * (double)m + 32.0 * m);
        add_diag<double>(Gm, m, m, -1.0, h->stream);                         // Gm = Z^T Z - I = -R
        get_diag(S, m, m, dg, h->stream);
        get_diag(Gm, m, m, dg + m, h->stream);
    }
    std::vector<double> hd(2 * (size_t)m);
    d2h_sync(h, hd.data(), dg, hd.size() * sizeof(double));
    double s2, r2, dd;
    frob_pair(h, nullptr, m, S, m, m, m, part, &dd, &s2);
    frob_pair(h, nullptr, m, Gm, m, m, m, part, &dd, &r2);
    double diag2 = 0.0, dmax = 0.0;
    std::vector<double> lam(m);
    for (int i = 0; i < m; ++i) {
        diag2 += hd[i] * hd[i];
        lam[i] = hd[i] / (1.0 + hd[m + i]);
        if (!std::isfinite(lam[i])) { release(h, mk); return PSSD_ERR_NONFINITE; }
        dmax = std::max(dmax, std::fabs(lam[i]));
    }
    const double omega = 2.0 * (std::sqrt(std::max(0.0, s2 - diag2)) + dmax * std::sqrt(r2));
    h2d(h, dg, lam.data(), sizeof(double) * m);
    {
        Timed t(h, K_HBM, 0, 24.0 * m * (double)m);
        eig_refine_correction(S, m, Gm, m, dg, m, omega, W, m, h->stream);  // F (in W)
    }
    {
        GemmArgs g; g.m = g.n = g.k = m; g.A = Z; g.lda = ldz; g.B = W; g.ldb = m; g.Cin = Z; g.ldcin = ldz;
        g.C = S; g.ldc = m; g.beta = 1.0;
        gemm(h, g);                                                          // Z + Z F
        Timed t(h, K_HBM, 0, 16.0 * m * (double)m + 16.0 * m);
        copy_matrix(S, m, Z, ldz, m, m, h->stream);
        copy_matrix(dg, m, d, m, 1, m, h->stream);
    }
    cuda_check(h, cudaStreamSynchronize(h->stream), "sync");   // lam goes out of scope
    release(h, mk);
    return PSSD_OK;
}

// ---------------------------------------------------------------------------
// shared front end: M, L, L^{-1}, K, bounds, Zolotarev sign of K
// ---------------------------------------------------------------------------
struct Front {
    int n = 0, p = 0;
    double *sig = nullptr;   // device signature
    double *M = nullptr, *L = nullptr, *Linv = nullptr, *K = nullptr;
    double *Y = nullptr;     // ~ sign(K)
    double normH = 0.0;
    double alpha = 0.0;      // X0 = K / alpha
};

int validate(int n, const signed char *sigma, const double *H, int ldh)
{
    if (n < 1 || n > PSSD_MAX_N) return -2;
    if (!sigma && (n % 2)) return -3;
    if (sigma)
        for (int i = 0; i < n; ++i) if (sigma[i] != 1 && sigma[i] != -1) return -3;
    if (!H) return -4;
    if (ldh < n) return -5;
    return 0;
}

int front(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, const pssd_opts &o,
          pssd_info *info, Front &F, const double *S_in = nullptr, long long lds_in = 0, SignTape *tape = nullptr,
          bool tape_store = true)
{
    // tape: record the Zolotarev steps for the adjoint (FP64 / FP64e Zolotarev only); tape_store:
    // keep the shifted inverses of every step, else only the per-step iterates
    PhaseScope phase(PH_FRONT);
    F.n = n;
    h->wait_limit = o.wait_cycles;
    if (info) info->method = o.method;
    h->use_tc = (o.flags & PSSD_FLAG_NO_TENSOR_CORES) ? 0 : 1;
    h->dmode = (o.precision == PSSD_FP64) ? GM_F64 : ((o.flags & PSSD_FLAG_EMU_SIMT) || !h->use_tc ? GM_DF : GM_OZ);
    if (info) info->precision = o.precision;
    const long long ld = n, nsz = (long long)n * n;
    std::vector<double> hs(n);
    int p = 0;
    for (int i = 0; i < n; ++i) { hs[i] = sigma ? (double)sigma[i] : (i < n / 2 ? 1.0 : -1.0); p += hs[i] > 0; }
    F.p = p;
    if (info) info->p = p;
    F.sig = dalloc(h, n);
    h2d(h, F.sig, hs.data(), sizeof(double) * n);
    F.M = dalloc(h, nsz);
    F.L = dalloc(h, nsz);
    F.Linv = dalloc(h, nsz);
    F.K = dalloc(h, nsz);
    // a1: M = Sigma H, symmetry defect
    {
        int nb = sym_prepare_blocks(n);
        Mark mk = mark(h);
        double *part = dalloc(h, 2 * (size_t)nb);
        {
            Timed t(h, K_HBM, 0, 16.0 * n * (double)n);
            sym_prepare(H, ldh, F.sig, n, F.M, ld, part, h->stream);
        }
        std::vector<double> hp(2 * (size_t)nb);
        d2h_sync(h, hp.data(), part, hp.size() * sizeof(double));
        release(h, mk);
        double d2 = 0, m2 = 0;
        for (int i = 0; i < nb; ++i) { d2 += hp[2 * i]; m2 += hp[2 * i + 1]; }
        if (!std::isfinite(d2) || !std::isfinite(m2)) return PSSD_ERR_NONFINITE;
        F.normH = std::sqrt(m2);
        if (!(m2 > 0.0)) return PSSD_ERR_NOT_DEFINITE;
        if (std::sqrt(d2) > 1e-12 * std::sqrt(m2)) return PSSD_ERR_NOT_PSEUDOSYMMETRIC;
    }
    // a2: L = chol(M), L^{-1}
    {
        Timed t(h, K_HBM, 0, 16.0 * n * (double)n);
        copy_matrix(F.M, ld, F.L, ld, n, n, h->stream);
    }
    int fi = -1;
    if (chol_inv(h, F.L, n, ld, 0, 1, F.Linv, 0, &fi)) {
        if (info) info->fail_index = fi;
        return PSSD_ERR_NOT_DEFINITE;
    }
    if (S_in) {   // a precomputed S = sign(H): K = L^T Sigma L and sign(K) = L^T S L^{-T} (H = L^{-T} K L^T)
        GemmArgs g; g.m = g.n = g.k = n; g.A = F.L; g.lda = ld; g.ta = 1; g.triA = TRI_UPPER; g.kscale = F.sig;
        g.B = F.L; g.ldb = ld; g.triB = TRI_LOWER; g.C = F.K; g.ldc = ld; g.lowerC = 1;
        gemm(h, g);
        mirror(h, F.K, ld, 0, n, 1);
        F.Y = dalloc(h, nsz);
        Mark mk = mark(h);
        double *T1 = dalloc(h, nsz);
        GemmArgs a; a.m = a.n = a.k = n; a.A = S_in; a.lda = lds_in; a.B = F.Linv; a.ldb = ld; a.tb = 1;
        a.triB = TRI_UPPER; a.C = T1; a.ldc = ld;
        gemm(h, a);                                                      // S L^{-T}
        GemmArgs b; b.m = b.n = b.k = n; b.A = F.L; b.lda = ld; b.ta = 1; b.triA = TRI_UPPER; b.B = T1; b.ldb = ld;
        b.C = F.Y; b.ldc = ld; b.lowerC = 1;
        gemm(h, b);                                                      // L^T S L^{-T} (symmetric; lower, mirrored)
        mirror(h, F.Y, ld, 0, n, 1);
        release(h, mk);
        return PSSD_OK;
    }
    // a3: bounds (reading R5: |lambda(H)| in [lambda_min(M), lambda_max(M)])
    double alpha = o.alpha, beta = o.beta;
    if (!(alpha > 0.0) || !(beta > 0.0)) {
        PhaseScope phase_b(PH_BOUNDS);
        Mark mk = mark(h);
        double *v = dalloc(h, n), *w = dalloc(h, n), *u = dalloc(h, n), *tmp = dalloc(h, 32 * (size_t)n + 8);
        double *M = F.M, *Li = F.Linv;
        cudaStream_t s = h->stream;
        KryFused kM, kL;
        kM.A = M; kM.lda = ld; kM.op = KRY_SYM;
        kL.A = Li; kL.lda = ld; kL.op = KRY_TRI_PAIR;
        if (!(alpha > 0.0))
            alpha = 1.05 * lmax_estimate(h, n, [&](const double *x, double *y) {
                Timed t(h, K_GEMV, 2.0 * n * (double)n, 8.0 * n * (double)n);
                gemv(M, ld, 0, TRI_NONE, n, x, y, tmp, s);
            }, 0xa1fa0001ull, v, w, tmp + 32 * (size_t)n, &kM);
        if (!(beta > 0.0))
            beta = 0.9 / lmax_estimate(h, n, [&](const double *x, double *y) {
                Timed t(h, K_GEMV, 2.0 * n * (double)n, 8.0 * n * (double)n);  // two triangular halves
                gemv(Li, ld, 0, TRI_LOWER, n, x, u, tmp, s);     // u = L^{-1} x
                gemv(Li, ld, 1, TRI_UPPER, n, u, y, tmp, s);     // y = L^{-T} u
            }, 0xbe7a0001ull, v, w, tmp + 32 * (size_t)n, &kL);
        release(h, mk);
    }
    if (!(alpha > 0.0) || !(beta > 0.0) || !std::isfinite(alpha) || !std::isfinite(beta)) return PSSD_ERR_NONFINITE;
    if (beta > alpha) beta = alpha;
    if (info) { info->alpha = alpha; info->beta = beta; }
    F.alpha = alpha;
    // a5: K = L^T Sigma L (lower, mirrored), X0 = K / alpha
    {
        GemmArgs g; g.m = g.n = g.k = n; g.A = F.L; g.lda = ld; g.ta = 1; g.triA = TRI_UPPER; g.kscale = F.sig;
        g.B = F.L; g.ldb = ld; g.triB = TRI_LOWER; g.C = F.K; g.ldc = ld; g.lowerC = 1;
        gemm(h, g);
        mirror(h, F.K, ld, 0, n, 1);
    }
    g_phase = PH_SIGN;   // restored by `phase` on return
    if (o.precision == PSSD_MIXED) {
        // FP32 Zolotarev steps, then FP64-accurate Newton-Schulz refinement
        F.Y = dalloc(h, nsz);
        Mark mk = mark(h);
        float *X32 = talloc<float>(h, nsz), *fA = talloc<float>(h, nsz), *fB = talloc<float>(h, nsz);
        {
            Timed t(h, K_HBM, 0, 12.0 * n * (double)n);
            scale_copy<double, float>(F.K, ld, X32, ld, n, n, 1.0 / alpha, h->stream);
        }
        float *Y32 = nullptr;
        int st = zolo_sign_fp32(h, X32, n, beta / alpha, 1e-6, 3e-3, fA, fB, &Y32, info, &fi);
        if (st) { if (info) info->fail_index = fi; release(h, mk); return st; }
        {
            Timed t(h, K_HBM, 0, 12.0 * n * (double)n);
            scale_copy<float, double>(Y32, ld, F.Y, ld, n, n, 1.0, h->stream);
        }
        release(h, mk);
        double res; int its;
        st = ns_refine(h, F.Y, n, 1e-14 * n, 4, &res, &its);
        if (info) { info->ns_steps = its; info->ns_resid = res; }
        return st;
    }
    double *X0 = dalloc(h, nsz), *bA = dalloc(h, nsz), *bB = dalloc(h, nsz);
    {
        Timed t(h, K_HBM, 0, 16.0 * n * (double)n);
        scale_copy<double, double>(F.K, ld, X0, ld, n, n, 1.0 / alpha, h->stream);
    }
    int maxr = o.max_restarts < 0 ? 2 : o.max_restarts;
    if (tape) {   // slots in the order zolo_sign takes the steps: two per pass, r from the same rule
        double l = beta / alpha;
        for (int pass = 0; pass <= maxr; ++pass) {
            l = std::min(l, 1.0);
            const int r = (pass == 0 && o.r > 0) ? o.r : choose_r_host(l, 1e-15, 8);
            double c[128], a[64], ch, l1, l2;
            if (r < 1 || zolo_coeffs_host(l, r, c, a, &ch, &l1)) return PSSD_ERR_NONFINITE;
            l1 = std::min(l1, 1.0);
            if (zolo_coeffs_host(l1, r, c, a, &ch, &l2)) return PSSD_ERR_NONFINITE;
            for (int t = 0; t < 2; ++t) {
                tape->xslot.push_back(dalloc(h, nsz));
                tape->zslot.push_back(tape_store ? dalloc(h, nsz * r) : nullptr);
            }
            l = std::min(l2, 1.0);
        }
    }
    int st;
    if (o.method == PSSD_METHOD_DWH)
        st = dwh_sign(h, X0, n, beta / alpha, bA, bB, &F.Y, info, &fi);
    else if (o.method == PSSD_METHOD_NEWTON)
        st = newton_sign(h, F.Linv, F.sig, alpha, X0, n, beta / alpha, bA, bB, &F.Y, info, &fi);
    else
        st = zolo_sign(h, X0, n, beta / alpha, o.r, maxr, 1e-15, bA, bB, &F.Y, info, &fi, false, nullptr, tape);
    if (st == PSSD_ERR_NOT_DEFINITE && info) info->fail_index = fi;
    return st;
}

pssd_opts defaults()
{
    pssd_opts o;
    pssd_opts_init(&o);
    return o;
}

void info_init(pssd_info *info)
{
    if (!info) return;
    std::memset(info, 0, sizeof(*info));
    info->fail_index = -1;
    info->s2_resid = -1.0;
    info->jsym_resid = -1.0;
    info->split_backerr = -1.0;
    info->comm_resid = -1.0;
}

// options outside their documented ranges (nonzero = invalid)
int opts_bad(const pssd_opts &o)
{
    if (o.r < 0 || o.r > 64) return 1;
    if (!(o.alpha >= 0.0) || !std::isfinite(o.alpha) || !(o.beta >= 0.0) || !std::isfinite(o.beta)) return 1;
    if (o.alpha > 0.0 && o.beta > 0.0 && o.beta > o.alpha) return 1;
    if (o.precision < 0 || o.precision > 2) return 1;
    if (o.method < 0 || o.method > 2) return 1;
    if (o.precision == PSSD_MIXED && o.method != PSSD_METHOD_ZOLO) return 1;
    if (o.wait_cycles < 0 || o.leaf < 0) return 1;
    return 0;
}

template <class F>
int guarded(pssd_handle h, pssd_info *info, F body)
{
    if (!h) return -1;
    auto t0 = std::chrono::steady_clock::now();
    Mark mk = mark(h);
    int st;
    h->wait_limit = 0;   // the default bound unless the call's options set one (front())
    int *outer_err = h->derr;
    try {
        if (!outer_err) {
            h->derr = ialloc(h, 1);
            cuda_check(h, cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream), "memset");
        }
        st = body();
        if (st == PSSD_OK) cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { h->last_err = cudaGetErrorString(e); st = PSSD_ERR_CUDA; }
        if (!outer_err) {
            int herr = 0;
            cudaMemcpyAsync(&herr, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
            cudaStreamSynchronize(h->stream);
            // a tensor-core kernel that gave up leaves garbage behind it, so the later
            // steps may fail too; the timeout is the cause that is reported
            if (herr && st != PSSD_ERR_CUDA) st = PSSD_ERR_TIMEOUT;
        }
    } catch (Fail &f) {
        st = f.code;
    }
    if (!outer_err) h->derr = nullptr;
    if (h->side) cudaStreamSynchronize(h->side);   // leaves still running on an error path
    h->leaf_pending.clear();
    h->sync_used = 0;
    cudaStreamSynchronize(h->stream);
    prof_collect(h);
    release(h, mk);
    if (info) info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void pssd_opts_init(pssd_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = PSSD_FP64;
    o->max_restarts = 2;
    o->leaf = 64;
}

int pssd_create(pssd_handle *h, void *stream)
{
    if (!h) return -1;
    *h = new pssd_handle_s();
    (*h)->stream = (cudaStream_t)stream;
    return PSSD_OK;
}

int pssd_destroy(pssd_handle h)
{
    if (!h) return -1;
    cudaStreamSynchronize(h->stream);
    auto drop_side = [](pssd_handle x) {
        if (x->side) { cudaStreamSynchronize(x->side); cudaStreamDestroy(x->side); }
        for (auto &e : x->sync_events) cudaEventDestroy(e);
    };
    for (auto *w : h->workers) {
        cudaStreamSynchronize(w->stream);
        drop_side(w);
        for (auto &c : w->chunks) if (c.owned) cudaFree(c.base);
        for (auto &e : w->free_events) cudaEventDestroy(e);
        cudaStreamDestroy(w->stream);
        delete w;
    }
    drop_side(h);
    for (auto &c : h->chunks) if (c.owned) cudaFree(c.base);
    for (auto &e : h->free_events) cudaEventDestroy(e);
    for (auto &e : h->events) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    delete h;
    return PSSD_OK;
}

int pssd_set_stream(pssd_handle h, void *stream)
{
    if (!h) return -1;
    h->stream = (cudaStream_t)stream;
    return PSSD_OK;
}

const char *pssd_last_cuda_error(pssd_handle h) { return h ? h->last_err.c_str() : "invalid handle"; }

const char *pssd_status_string(int status)
{
    switch (status) {
    case PSSD_OK: return "ok";
    case PSSD_ERR_NOT_DEFINITE: return "Sigma*H is not positive definite";
    case PSSD_ERR_NO_CONVERGENCE: return "Zolotarev stopping test failed after the allowed restarts";
    case PSSD_ERR_BASIS: return "invariant-subspace basis breakdown";
    case PSSD_ERR_NONFINITE: return "non-finite value in the input or an iterate";
    case PSSD_ERR_TIMEOUT: return "a bounded device wait timed out";
    case PSSD_ERR_CUDA: return "CUDA error";
    case PSSD_ERR_ALLOC: return "device allocation failed";
    case PSSD_ERR_NOT_PSEUDOSYMMETRIC: return "Sigma*H is not symmetric";
    case PSSD_ERR_NOALLOC_TOO_LARGE: return "n exceeds the allocation-free scratch limit (PSSD_NOALLOC_MAX_N)";
    default: return status < 0 ? "invalid argument" : "unknown status";
    }
}

int pssd_zolo_coeffs(double ell, int r, double *c, double *a, double *chat, double *ell_next)
{
    return zolo_coeffs_host(ell, r, c, a, chat, ell_next);
}

int pssd_choose_r(double ell, double tau, int r_max)
{
    if (!(ell > 0.0) || !(ell <= 1.0)) return -1;
    if (!(tau > 0.0)) return -2;
    if (r_max < 1) return -3;
    return choose_r_host(ell, tau, r_max);
}

}  // extern "C"

namespace {
// the body of pssd_sign (inside a guarded call): S = L^{-T} sign(K) L^T, mixed-precision
// re-symmetrisation and Newton-Schulz, residuals
int sign_core(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, double *S, int lds,
              const pssd_opts &o, pssd_info *info)
{
    Front F;
    int st = front(h, n, sigma, H, ldh, o, info, F);
    if (st) return st;
    const long long ld = n, nsz = (long long)n * n;
    double *T1 = dalloc(h, nsz);
    GemmArgs a;   // T1 = Y L^T
    a.m = a.n = a.k = n; a.A = F.Y; a.lda = ld; a.B = F.L; a.ldb = ld; a.tb = 1; a.triB = TRI_UPPER;
    a.C = T1; a.ldc = ld;
    gemm(h, a);
    GemmArgs b;   // S = L^{-T} T1
    b.m = b.n = b.k = n; b.A = F.Linv; b.lda = ld; b.ta = 1; b.triA = TRI_UPPER; b.B = T1; b.ldb = ld;
    b.C = S; b.ldc = lds;
    gemm(h, b);
    if (o.precision == PSSD_MIXED) {
        // mixed precision: J-re-symmetrisation, then Newton-Schulz on S itself (polynomials of a
        // Sigma-symmetric S stay Sigma-symmetric), in FP64-accurate arithmetic
        {
            Timed t(h, K_HBM, 0, 16.0 * n * (double)n);
            j_resym(S, lds, F.sig, n, h->stream);
        }
        double res; int its;
        int st2 = ns_refine(h, S, n, 1e-14 * n, 3, &res, &its, false, lds);
        if (st2) return st2;
        if (info) info->ns_steps += its;
    }
    if (info)
        info->comm_resid = comm_resid(h, n, H, ldh, F.normH, S, lds, nullptr, 0, F.sig,
                                      (o.flags & PSSD_FLAG_RESIDUALS) != 0);
    if (o.flags & 1) {   // residuals
        double *S2 = dalloc(h, nsz);
        GemmArgs c; c.m = c.n = c.k = n; c.A = S; c.lda = lds; c.B = S; c.ldb = lds; c.C = S2; c.ldc = ld;
        gemm(h, c);
        {
            Timed t(h, K_HBM, 0, 16.0 * n);
            add_diag(S2, ld, n, -1.0, h->stream);
        }
        double *part = dalloc(h, 2 * (size_t)frob_blocks(n, n));
        double d2, y2;
        frob_pair(h, nullptr, ld, S2, ld, n, n, part, &d2, &y2);
        if (info) info->s2_resid = std::sqrt(y2);
    }
    return PSSD_OK;
}
}  // namespace

extern "C" {

int pssd_sign(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, double *S, int lds,
              const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    int v = validate(n, sigma, H, ldh);
    if (v) return v;
    if (!S) return -6;
    if (lds < n) return -7;
    if (S == H) return -6;
    pssd_opts o = opts ? *opts : defaults();
    if (opts_bad(o)) return -8;
    info_init(info);
    return guarded(h, info, [&]() -> int { return sign_core(h, n, sigma, H, ldh, S, lds, o, info); });
}

int pssd_split(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, const double *S_in,
               int lds_in, double *Q, int ldq, double *A11, int lda11, double *A22, int lda22, int *p_out,
               const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    int v = validate(n, sigma, H, ldh);
    if (v) return v;
    if (S_in && lds_in < n) return -7;
    if (!Q) return -8;
    if (ldq < n) return -9;
    pssd_opts o = opts ? *opts : defaults();
    if (opts_bad(o)) return -15;
    int p0 = 0;
    for (int i = 0; i < n; ++i) p0 += sigma ? (sigma[i] > 0) : (i < n / 2);
    if (p0 > 0 && !A11) return -10;
    if (p0 > 0 && lda11 < p0) return -11;
    if (n - p0 > 0 && !A22) return -12;
    if (n - p0 > 0 && lda22 < n - p0) return -13;
    info_init(info);
    return guarded(h, info, [&]() -> int {
        Front F;
        int st = front(h, n, sigma, H, ldh, o, info, F, S_in, lds_in);
        if (st) return st;
        const int p = F.p, q = n - p;
        if (p_out) *p_out = p;
        const long long ld = n, nsz = (long long)n * n;
        double *U = dalloc(h, nsz);
        double *Bp = dalloc(h, (size_t)p * p + 1), *Bm = dalloc(h, (size_t)q * q + 1);
        const bool exact_be = (o.flags & PSSD_FLAG_RESIDUALS) != 0;
        double *E = exact_be ? dalloc(h, (size_t)p * q + 1) : nullptr;
        PhaseScope phase(PH_SPLIT);
        st = sym_split(h, F.K, F.Y, n, p, U, Bp, Bm, E, 0x51a7ull);
        if (st) return st;
        // C_+ = chol(B_+), C_- = chol(-B_-)
        double *Cpm = dalloc(h, (size_t)p * p + (size_t)q * q + 1);
        double *Cp = Cpm, *Cm = Cpm + (size_t)p * p;
        double *X = dalloc(h, nsz);
        int fi;
        if (p > 0) {
            Timed t(h, K_HBM, 0, 16.0 * p * (double)p);
            copy_matrix(Bp, p, Cp, p, p, p, h->stream);
        }
        if (q > 0) {
            Timed t(h, K_HBM, 0, 16.0 * q * (double)q);
            scale_copy(Bm, q, Cm, q, q, q, -1.0, h->stream);
        }
        if (p > 0 && p == q) {   // both factors in one batched call
            if (chol_inv<double>(h, Cp, p, p, (long long)p * p, 2, nullptr, 0, &fi)) return PSSD_ERR_BASIS;
        } else {
            if (p > 0 && chol_inv<double>(h, Cp, p, p, 0, 1, nullptr, 0, &fi)) return PSSD_ERR_BASIS;
            if (q > 0 && chol_inv<double>(h, Cm, q, q, 0, 1, nullptr, 0, &fi)) return PSSD_ERR_BASIS;
        }
        if (p > 0) {   // X_+ = U_+ C_+, Q_+ = L^{-T} X_+, A11 = C_+^T C_+
            GemmArgs g; g.m = n; g.n = p; g.k = p; g.A = U; g.lda = ld; g.B = Cp; g.ldb = p; g.triB = TRI_LOWER;
            g.C = X; g.ldc = ld;
            gemm(h, g);
            GemmArgs a; a.m = p; a.n = p; a.k = p; a.A = Cp; a.lda = p; a.ta = 1; a.triA = TRI_UPPER; a.B = Cp;
            a.ldb = p; a.triB = TRI_LOWER; a.C = A11; a.ldc = lda11; a.lowerC = 1;
            gemm(h, a);
            mirror(h, A11, lda11, 0, p, 1);
        }
        if (q > 0) {
            GemmArgs g; g.m = n; g.n = q; g.k = q; g.A = U + p; g.lda = ld; g.B = Cm; g.ldb = q; g.triB = TRI_LOWER;
            g.C = X + p; g.ldc = ld;
            gemm(h, g);
            GemmArgs a; a.m = q; a.n = q; a.k = q; a.A = Cm; a.lda = q; a.ta = 1; a.triA = TRI_UPPER; a.B = Cm;
            a.ldb = q; a.triB = TRI_LOWER; a.C = A22; a.ldc = lda22; a.lowerC = 1; a.alpha = -1.0;
            gemm(h, a);
            mirror(h, A22, lda22, 0, q, 1);
        }
        {
            GemmArgs g; g.m = g.n = g.k = n; g.A = F.Linv; g.lda = ld; g.ta = 1; g.triA = TRI_UPPER; g.B = X;
            g.ldb = ld; g.C = Q; g.ldc = ldq;
            gemm(h, g);
        }
        if (info && p > 0 && q > 0)     // ||U_+^T K U_-||_F / ||K||_F (backward error of the split of K ~ H)
            info->split_backerr = split_backward_error(h, F.K, U, n, p, E);
        if (info)
            info->comm_resid = comm_resid(h, n, H, ldh, F.normH, nullptr, 0, Q, ldq, F.sig, exact_be);
        return PSSD_OK;
    });
}

}  // extern "C"

namespace {
// full diagonalisation (the body of pssd_eig), inside a guarded call
int eig_core(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, double *V, int ldv,
             double *D, const pssd_opts &o, pssd_info *info, int leaf)
{
        Front F;
        int st = front(h, n, sigma, H, ldh, o, info, F);
        if (st) return st;
        const int p = F.p, q = n - p;
        const long long ld = n, nsz = (long long)n * n;
        double *U = dalloc(h, nsz);
        double *Bp = dalloc(h, (size_t)p * p + 1), *Bm = dalloc(h, (size_t)q * q + 1);
        const bool exact_be = (o.flags & PSSD_FLAG_RESIDUALS) != 0;
        double *E = exact_be ? dalloc(h, (size_t)p * q + 1) : nullptr;
        PhaseScope phase(PH_SPLIT);
        st = sym_split(h, F.K, F.Y, n, p, U, Bp, Bm, E, 0x51a7ull, true);
        if (st) return st;
        g_phase = PH_OTHER;
        double *Wp = dalloc(h, (size_t)p * p + 1), *Wm = dalloc(h, (size_t)q * q + 1);
        double *w = dalloc(h, n);
        int maxdepth = 0;
        if (p > 0) st = sym_eig(h, Bp, p, Wp, w, leaf, 1, &maxdepth, 0x1001ull);
        if (!st && q > 0) st = sym_eig(h, Bm, q, Wm, w + p, leaf, 1, &maxdepth, 0x2002ull);
        if (st) return st;
        if (info) info->levels = maxdepth;
        g_phase = PH_ASSEMBLE;
        double *Uf = dalloc(h, nsz);
        if (p > 0) {
            GemmArgs g; g.m = n; g.n = p; g.k = p; g.A = U; g.lda = ld; g.B = Wp; g.ldb = p; g.C = Uf; g.ldc = ld;
            gemm(h, g);
        }
        if (q > 0) {
            GemmArgs g; g.m = n; g.n = q; g.k = q; g.A = U + p; g.lda = ld; g.B = Wm; g.ldb = q; g.C = Uf + p;
            g.ldc = ld;
            gemm(h, g);
        }
        if (!(o.flags & PSSD_FLAG_NO_REFINE)) {   // K ~ Uf diag(w) Uf^T, refined once
            g_phase = PH_REFINE;
            st = sym_refine(h, F.K, ld, n, Uf, ld, w);
            if (st) return st;
            g_phase = PH_ASSEMBLE;
        }
        double *Vt = dalloc(h, nsz);
        {   // V = L^{-T} Uf |Lambda|^{1/2}
            GemmArgs g; g.m = g.n = g.k = n; g.A = F.Linv; g.lda = ld; g.ta = 1; g.triA = TRI_UPPER; g.B = Uf;
            g.ldb = ld; g.C = Vt; g.ldc = ld;
            gemm(h, g);
        }
        {
            Timed t(h, K_HBM, 0, 32.0 * n * (double)n);
            scale_columns(Vt, ld, n, n, w, 1, h->stream);
            sign_fix_columns(Vt, ld, n, n, h->stream);
        }
        // order: positive ascending, then negative by ascending magnitude
        std::vector<double> hw(n);
        d2h_sync(h, hw.data(), w, sizeof(double) * n);
        std::vector<int> pos, neg;
        for (int i = 0; i < n; ++i) (hw[i] > 0 ? pos : neg).push_back(i);
        std::stable_sort(pos.begin(), pos.end(), [&](int a, int b) { return hw[a] < hw[b]; });
        std::stable_sort(neg.begin(), neg.end(), [&](int a, int b) { return hw[a] > hw[b]; });
        std::vector<int> perm(pos);
        perm.insert(perm.end(), neg.begin(), neg.end());
        std::vector<double> hd(n);
        for (int i = 0; i < n; ++i) hd[i] = hw[perm[i]];
        int *dperm = ialloc(h, n);
        h2d(h, dperm, perm.data(), sizeof(int) * n);
        h2d(h, D, hd.data(), sizeof(double) * n);
        {
            Timed t(h, K_HBM, 0, 16.0 * n * (double)n);
            gather_columns(Vt, ld, V, ldv, n, n, dperm, h->stream);
        }
        cuda_check(h, cudaStreamSynchronize(h->stream), "sync");   // host vectors above go out of scope
        g_phase = PH_OTHER;
        if (info && p > 0 && q > 0)     // ||U_+^T K U_-||_F / ||K||_F
            info->split_backerr = split_backward_error(h, F.K, U, n, p, E);
        if (info)
            info->comm_resid = comm_resid(h, n, H, ldh, F.normH, nullptr, 0, V, ldv, F.sig, exact_be);
        return PSSD_OK;
}
}  // namespace

extern "C" {

int pssd_eig(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, double *V, int ldv,
             double *D, const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    int v = validate(n, sigma, H, ldh);
    if (v) return v;
    if (!V) return -6;
    if (ldv < n) return -7;
    if (!D) return -8;
    pssd_opts o = opts ? *opts : defaults();
    if (opts_bad(o)) return -9;
    int leaf = o.leaf > 0 ? std::min(o.leaf, 64) : 64;
    info_init(info);
    return guarded(h, info, [&]() -> int { return eig_core(h, n, sigma, H, ldh, V, ldv, D, o, info, leaf); });
}

// --------------------------------------------------------------------------
// measurement hooks (not part of the method): launch counting and per-kind
// CUDA-event timing of every kernel launch the library makes
// --------------------------------------------------------------------------
int pssd_profile_enable(pssd_handle h, int on)
{
    if (!h) return -1;
    h->prof = on ? 1 : 0;
    return PSSD_OK;
}

int pssd_profile_reset(pssd_handle h)
{
    if (!h) return -1;
    for (int i = 0; i < 16; ++i) { h->prof_ms[i] = 0; h->prof_flops[i] = 0; h->prof_bytes[i] = 0; h->prof_count[i] = 0; }
    return PSSD_OK;
}

int pssd_profile_read(pssd_handle h, int kind, double *total_ms, long long *launches, double *flops, double *bytes)
{
    if (!h) return -1;
    if (kind < 0 || kind >= K_NKIND) return -2;
    if (total_ms) *total_ms = h->prof_ms[kind];
    if (launches) *launches = h->prof_count[kind];
    if (flops) *flops = h->prof_flops[kind];
    if (bytes) *bytes = h->prof_bytes[kind];
    return PSSD_OK;
}

int pssd_set_workspace(pssd_handle h, void *dptr, size_t bytes)
{
    if (!h) return -1;
    if (dptr && bytes < 4096) return -3;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        h->last_err = "cudaStreamSynchronize before replacing the workspace failed";
        return PSSD_ERR_CUDA;
    }
    for (auto &c : h->chunks) if (c.owned) cudaFree(c.base);
    h->chunks.clear();
    h->user_ws = false;
    h->depth = 0;
    h->peak = 0;
    if (dptr) {   // align the start to 256 bytes inside the caller's buffer
        const uintptr_t a = ((uintptr_t)dptr + 255) & ~(uintptr_t)255;
        const size_t lost = (size_t)(a - (uintptr_t)dptr);
        h->chunks.push_back({(char *)a, bytes - lost, 0, false});
        h->user_ws = true;
    }
    return PSSD_OK;
}

int pssd_workspace_peak(pssd_handle h, size_t *bytes)
{
    if (!h) return -1;
    if (!bytes) return -2;
    *bytes = h->peak;
    return PSSD_OK;
}

int pssd_workspace_bytes(pssd_handle h, int n, const pssd_opts *opts, size_t *bytes)
{
    if (!h) return -1;
    if (n < 1 || n > PSSD_MAX_N) return -2;
    if (!bytes) return -4;
    pssd_opts o = opts ? *opts : defaults();
    const double rmax = o.r > 0 ? o.r : 8;
    const double nn = (double)n * (double)n * sizeof(double);
    *bytes = (size_t)((20.0 + 3.0 * rmax) * nn) + ((size_t)256 << 20);
    return PSSD_OK;
}

// process-wide number of kernels the library has launched (all handles)
long long pssd_launch_count(pssd_handle h) { return h ? g_launches.load() : -1; }

// process-wide number of device allocations (cudaMalloc calls) the library has made
long long pssd_device_alloc_count(void) { return g_device_allocs.load(); }

// the launch count by phase (PSSD_PHASE_* = PH_*)
int pssd_launch_count_phases(long long *counts, int n)
{
    static_assert(PSSD_PHASE_COUNT == PH_COUNT && PSSD_PHASE_SHIFT == PH_SHIFT && PSSD_PHASE_REFINE == PH_REFINE,
                  "phase indices");
    for (int i = 0; i < n && i < PH_COUNT && counts; ++i) counts[i] = g_phase_launches[i].load();
    return PH_COUNT;
}

}  // extern "C"

// ===========================================================================
// Allocation-free variant of pssd_sign for small problems.
//
// Some callers cannot call cudaMalloc at all: code that runs while a CUDA
// graph is being captured, applications whose device memory is owned by a
// pool or arena that the library must not bypass, and latency-critical
// loops where a first-call allocation (and the implicit synchronisation it
// can cause) is not acceptable.  For them, pssd_sign_noalloc carves every
// temporary of the sign computation out of one file-scope device array of
// PSSD_NOALLOC_SCRATCH_BYTES bytes (8 MiB), which every GPU that loads this
// library holds until the process exits.  The caller still supplies H and S.
// ===========================================================================
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(8) << 20;
constexpr int NOALLOC_MAX_N = 128;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// g_noalloc_scratch names a host-side shadow, not device memory, so the
// address must come from cudaGetSymbolAddress, once per device, with that
// device current.
int noalloc_scratch(void **ptr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return PSSD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return PSSD_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
    return PSSD_OK;
}

}  // namespace

extern "C" int pssd_sign_noalloc(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh,
                                 double *S, int lds, const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    if (n > NOALLOC_MAX_N) return PSSD_ERR_NOALLOC_TOO_LARGE;
    void *scratch = nullptr;
    if (noalloc_scratch(&scratch) != PSSD_OK) return PSSD_ERR_CUDA;
    // A private handle whose only workspace is the scratch array, marked as
    // caller-owned: every temporary of pssd_sign is carved from it, and a
    // temporary that would overflow it stops the call (PSSD_ERR_ALLOC inside,
    // reported as PSSD_ERR_NOALLOC_TOO_LARGE) instead of allocating.
    pssd_handle_s local;
    local.stream = h->stream;
    local.user_ws = true;
    local.chunks.push_back({(char *)scratch, NOALLOC_SCRATCH_BYTES, 0, false});
    int st = pssd_sign(&local, n, sigma, H, ldh, S, lds, opts, info);
    local.chunks.clear();   // the scratch array is not owned by the local handle
    if (st == PSSD_ERR_ALLOC) {
        st = PSSD_ERR_NOALLOC_TOO_LARGE;
        h->last_err = local.last_err;
    }
    if (st == PSSD_ERR_CUDA) h->last_err = local.last_err;
    return st;
}

// ===========================================================================
// Adjoint: cotangents of S = sign(H) and of the eigenvalues
// pulled back to H.  With H = V Lambda V^{-1} (V from pssd_eig, V^{-1} =
// Sigma_hat V^T Sigma by Eq. VSigmaOrth) the Frechet derivative of the sign
// function is the Daleckii-Krein form
//     dS = V (F o (V^{-1} dH V)) V^{-1},   F_ij = (s_i - s_j)/(lambda_i - lambda_j),
// and d lambda_i = (V^{-1} dH V)_ii, so for L = <Sbar, S> + sum_i lambar_i lambda_i
//     Hbar = V^{-T} (F o (V^T Sbar V^{-T}) + diag(lambar)) V^T,   V^{-T} = Sigma V Sigma_hat.
// F vanishes between eigenvalues of the same sign and is at most 1/min|lambda|
// elsewhere, so the pull-back is as well conditioned as the split itself.
// ===========================================================================
namespace {
// Step-reversal adjoint of S = L^{-T} Y L^T with Y = X_N, the last Zolotarev iterate, and of
// the sum of the positive eigenvalues (gradient P_+^T, P_+ = (I + S)/2): the gradient of the
// computed function, coefficients and bounds held fixed.  Backward of one step
// X' = chat (X + X T), T = sum_j a_j Z_j, Z_j = (X^2 + c_{2j-1} I)^{-1}:
//   Abar = chat X X'bar,  B = sum_j a_j Z_j Abar Z_j,
//   Xbar = chat (X'bar + X'bar T) - (X B + B X)
// (dZ_j = -Z_j (X dX + dX X) Z_j; X, T, Z_j symmetric and commuting).  Then K = alpha X_0,
// K = L^T Sigma L gives Lbar += Sigma L (Kbar + Kbar^T); S = L^{-T} Y L^T gives, with
// Ghat = L^{-1} G L, Ybar = sym(Ghat) and Lbar += L^{-T} (Ghat^T Y - Y Ghat^T); the
// Cholesky factorisation M = L L^T gives Mbar = sym(L^{-T} Phi(L^T Lbar) L^{-1}) (Phi: lower
// triangle, diagonal halved); M = sym(Sigma H) gives Hbar = Sigma Mbar.  Since the forward
// reads H only through sym(Sigma H), Hbar is the gradient with respect to pseudosymmetric H:
// the unconstrained gradient projected by X -> Sigma sym(Sigma X).
int sign_vjp_steps(pssd_handle h, const Front &F, const SignTape &tape, const double *Gb, long long ldg,
                   double pos_weight, double *Hbar, long long ldhb)
{
    const int n = F.n;
    const long long ld = n, nsz = (long long)n * n;
    const double *L = F.L, *Li = F.Linv, *Y = F.Y;
    Mark mk = mark(h);
    double *T1 = dalloc(h, nsz), *W = dalloc(h, nsz), *Lb = dalloc(h, nsz), *Xb = dalloc(h, nsz);
    double *Xn = dalloc(h, nsz);
    if (Gb) {
        double *Gh = Xn;
        GemmArgs a; a.m = a.n = a.k = n; a.A = Gb; a.lda = ldg; a.B = L; a.ldb = ld; a.triB = TRI_LOWER;
        a.C = T1; a.ldc = ld;
        gemm(h, a);                                                            // G L
        GemmArgs b; b.m = b.n = b.k = n; b.A = Li; b.lda = ld; b.triA = TRI_LOWER; b.B = T1; b.ldb = ld;
        b.C = Gh; b.ldc = ld;
        gemm(h, b);                                                            // Ghat = L^{-1} G L
        GemmArgs c; c.m = c.n = c.k = n; c.A = Gh; c.lda = ld; c.ta = 1; c.B = Y; c.ldb = ld; c.C = T1; c.ldc = ld;
        gemm(h, c);                                                            // Ghat^T Y
        GemmArgs d; d.m = d.n = d.k = n; d.A = Y; d.lda = ld; d.B = Gh; d.ldb = ld; d.tb = 1; d.Cin = T1;
        d.ldcin = ld; d.C = T1; d.ldc = ld; d.alpha = -1.0; d.beta = 1.0;
        gemm(h, d);                                                            // - Y Ghat^T
        Timed t(h, K_HBM, 0, 32.0 * n * (double)n);
        copy_matrix(Gh, ld, Xb, ld, n, n, h->stream);                          // Ybar = sym(Ghat) (below)
    }
    if (Gb) {
        for (int s = (int)tape.steps.size() - 1; s >= 0; --s) {
            const SignTape::Step &stp = tape.steps[s];
            const int r = stp.r;
            Mark ms = mark(h);
            double *Tm = dalloc(h, nsz), *Ab = dalloc(h, nsz), *Bs = dalloc(h, nsz), *W1 = dalloc(h, nsz);
            double *Z = stp.Z;
            {
                Timed t(h, K_HBM, 0, 16.0 * n * (double)n);
                sym_average<double>(Xb, ld, n, h->stream);
            }
            if (!Z) {   // recompute the shifted inverses from the checkpointed iterate
                Z = dalloc(h, nsz * r);
                double *G2 = W1;
                GemmArgs g; g.m = g.n = g.k = n; g.A = stp.X; g.lda = ld; g.B = stp.X; g.ldb = ld; g.C = G2;
                g.ldc = ld; g.lowerC = 1;
                gemm(h, g);                                                    // X^2 (lower)
                int fi;
                int st = shifted_inverse_sum<double>(h, G2, n, r, stp.c, stp.a, Tm, &fi, Z);
                if (st) { release(h, mk); return st; }
            } else {    // T = sum_j a_j Z_j from the stored inverses
                double *da = dalloc(h, r);
                h2d(h, da, stp.a, sizeof(double) * r);
                Timed t(h, K_HBM, 0, 8.0 * 0.5 * n * (double)n * (r + 1));
                combine_lower<double>(Z, ld, nsz, da, r, n, Tm, ld, h->stream);
            }
            if (stp.Z) mirror<double>(h, Tm, ld, 0, n, 1);
            GemmArgs ga; ga.m = ga.n = ga.k = n; ga.A = stp.X; ga.lda = ld; ga.B = Xb; ga.ldb = ld; ga.C = Ab;
            ga.ldc = ld; ga.alpha = stp.chat;
            gemm(h, ga);                                                       // Abar = chat X Xbar'
            for (int j = 0; j < r; ++j) {
                const double *Zj = Z + (long long)j * nsz;
                GemmArgs g1; g1.m = g1.n = g1.k = n; g1.A = Zj; g1.lda = ld; g1.B = Ab; g1.ldb = ld; g1.C = W1;
                g1.ldc = ld;
                gemm(h, g1);                                                   // Z_j Abar
                GemmArgs g2; g2.m = g2.n = g2.k = n; g2.A = W1; g2.lda = ld; g2.B = Zj; g2.ldb = ld; g2.C = Bs;
                g2.ldc = ld; g2.alpha = stp.a[j];
                if (j) { g2.Cin = Bs; g2.ldcin = ld; g2.beta = 1.0; }
                gemm(h, g2);                                                   // B += a_j Z_j Abar Z_j
            }
            GemmArgs gx; gx.m = gx.n = gx.k = n; gx.A = Xb; gx.lda = ld; gx.B = Tm; gx.ldb = ld; gx.Cin = Xb;
            gx.ldcin = ld; gx.C = Xn; gx.ldc = ld; gx.alpha = stp.chat; gx.beta = stp.chat;
            gemm(h, gx);                                                       // chat (Xbar' + Xbar' T)
            GemmArgs g3; g3.m = g3.n = g3.k = n; g3.A = stp.X; g3.lda = ld; g3.B = Bs; g3.ldb = ld; g3.Cin = Xn;
            g3.ldcin = ld; g3.C = Xn; g3.ldc = ld; g3.alpha = -1.0; g3.beta = 1.0;
            gemm(h, g3);                                                       // - X B
            GemmArgs g4; g4.m = g4.n = g4.k = n; g4.A = Bs; g4.lda = ld; g4.B = stp.X; g4.ldb = ld; g4.Cin = Xn;
            g4.ldcin = ld; g4.C = Xn; g4.ldc = ld; g4.alpha = -1.0; g4.beta = 1.0;
            gemm(h, g4);                                                       // - B X
            std::swap(Xb, Xn);
            release(h, ms);
        }
        {
            Timed t(h, K_HBM, 0, 16.0 * n * (double)n);
            sym_average<double>(Xb, ld, n, h->stream);                         // Xbar_0
        }
        GemmArgs gk; gk.m = gk.n = gk.k = n; gk.A = L; gk.lda = ld; gk.triA = TRI_LOWER; gk.B = Xb; gk.ldb = ld;
        gk.C = W; gk.ldc = ld; gk.alpha = 2.0 / F.alpha;
        gemm(h, gk);                                                           // (2/alpha) L Xbar_0
        {
            Timed t(h, K_HBM, 0, 16.0 * n * (double)n);
            scale_rows(W, ld, n, n, F.sig, h->stream);                         // Sigma L (Kbar + Kbar^T)
        }
        GemmArgs gl; gl.m = gl.n = gl.k = n; gl.A = Li; gl.lda = ld; gl.ta = 1; gl.triA = TRI_UPPER; gl.B = T1;
        gl.ldb = ld; gl.Cin = W; gl.ldcin = ld; gl.C = Lb; gl.ldc = ld; gl.beta = 1.0;
        gemm(h, gl);                                                           // Lbar
        GemmArgs gp; gp.m = gp.n = gp.k = n; gp.A = L; gp.lda = ld; gp.ta = 1; gp.triA = TRI_UPPER; gp.B = Lb;
        gp.ldb = ld; gp.C = T1; gp.ldc = ld;
        gemm(h, gp);                                                           // L^T Lbar
        {
            Timed t(h, K_HBM, 0, 16.0 * n * (double)n);
            tril_half_diag(T1, ld, n, h->stream);                              // Phi
        }
        GemmArgs gq; gq.m = gq.n = gq.k = n; gq.A = T1; gq.lda = ld; gq.triA = TRI_LOWER; gq.B = Li; gq.ldb = ld;
        gq.triB = TRI_LOWER; gq.C = W; gq.ldc = ld;
        gemm(h, gq);                                                           // Phi L^{-1}
        GemmArgs gm; gm.m = gm.n = gm.k = n; gm.A = Li; gm.lda = ld; gm.ta = 1; gm.triA = TRI_UPPER; gm.B = W;
        gm.ldb = ld; gm.C = T1; gm.ldc = ld;
        gemm(h, gm);                                                           // L^{-T} Phi L^{-1}
        Timed t(h, K_HBM, 0, 48.0 * n * (double)n);
        sym_average<double>(T1, ld, n, h->stream);                             // Mbar
        copy_matrix(T1, ld, Hbar, ldhb, n, n, h->stream);
        scale_rows(Hbar, ldhb, n, n, F.sig, h->stream);                        // Hbar = Sigma Mbar
    } else {
        cuda_check(h, cudaMemset2DAsync(Hbar, sizeof(double) * ldhb, 0, sizeof(double) * n, n, h->stream),
                   "memset");
    }
    if (pos_weight != 0.0) {   // + pos_weight P_+^T = (pos_weight / 2)(I + L Y L^{-1})
        GemmArgs g1; g1.m = g1.n = g1.k = n; g1.A = Y; g1.lda = ld; g1.B = Li; g1.ldb = ld; g1.triB = TRI_LOWER;
        g1.C = W; g1.ldc = ld;
        gemm(h, g1);                                                           // Y L^{-1}
        GemmArgs g2; g2.m = g2.n = g2.k = n; g2.A = L; g2.lda = ld; g2.triA = TRI_LOWER; g2.B = W; g2.ldb = ld;
        g2.Cin = Hbar; g2.ldcin = ldhb; g2.C = Hbar; g2.ldc = ldhb; g2.alpha = 0.5 * pos_weight; g2.beta = 1.0;
        gemm(h, g2);
        Timed t(h, K_HBM, 0, 16.0 * n);
        add_diag<double>(Hbar, ldhb, n, 0.5 * pos_weight, h->stream);
    }
    cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
    release(h, mk);
    return PSSD_OK;
}
}  // namespace

extern "C" int pssd_sign_vjp_rev(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh,
                                 const double *Sbar, int ldsb, double pos_weight, double *Hbar, int ldhb,
                                 const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    int v = validate(n, sigma, H, ldh);
    if (v) return v;
    if (Sbar && ldsb < n) return -7;
    if (!std::isfinite(pos_weight)) return -8;
    if (!Hbar) return -9;
    if (ldhb < n) return -10;
    pssd_opts o = opts ? *opts : defaults();
    if (opts_bad(o) || o.precision == PSSD_MIXED || o.method != PSSD_METHOD_ZOLO) return -11;
    info_init(info);
    return guarded(h, info, [&]() -> int {
        Front F;
        SignTape tape;
        int st = front(h, n, sigma, H, ldh, o, info, F, nullptr, 0, &tape, !(o.flags & PSSD_FLAG_RECOMPUTE));
        if (st) return st;
        return sign_vjp_steps(h, F, tape, Sbar, ldsb, pos_weight, Hbar, ldhb);
    });
}

extern "C" int pssd_sign_vjp(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh,
                             const double *Sbar, int ldsb, const double *lambar, double *Hbar, int ldhb,
                             const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    int v = validate(n, sigma, H, ldh);
    if (v) return v;
    if (Sbar && ldsb < n) return -7;
    if (!Hbar) return -9;
    if (ldhb < n) return -10;
    pssd_opts o = opts ? *opts : defaults();
    if (opts_bad(o)) return -11;
    int leaf = o.leaf > 0 ? std::min(o.leaf, 64) : 64;
    info_init(info);
    return guarded(h, info, [&]() -> int {
        const long long ld = n, nsz = (long long)n * n;
        double *V = dalloc(h, nsz), *D = dalloc(h, n);
        int st = eig_core(h, n, sigma, H, ldh, V, n, D, o, info, leaf);
        if (st) return st;
        std::vector<double> hs(n), hD(n), hsh(n);
        for (int i = 0; i < n; ++i) hs[i] = sigma ? (double)sigma[i] : (i < n / 2 ? 1.0 : -1.0);
        d2h_sync(h, hD.data(), D, sizeof(double) * n);
        for (int i = 0; i < n; ++i) hsh[i] = hD[i] > 0 ? 1.0 : -1.0;
        double *dsig = dalloc(h, n), *dsh = dalloc(h, n);
        h2d(h, dsig, hs.data(), sizeof(double) * n);
        h2d(h, dsh, hsh.data(), sizeof(double) * n);
        double *Vit = dalloc(h, nsz);   // V^{-T} = Sigma V Sigma_hat
        {
            Timed t(h, K_HBM, 0, 48.0 * n * (double)n);
            copy_matrix(V, ld, Vit, ld, n, n, h->stream);
            scale_rows(Vit, ld, n, n, dsig, h->stream);
            scale_columns(Vit, ld, n, n, dsh, 0, h->stream);
        }
        double *W = dalloc(h, nsz), *T = dalloc(h, nsz);
        if (Sbar) {
            GemmArgs a; a.m = a.n = a.k = n; a.A = Sbar; a.lda = ldsb; a.B = Vit; a.ldb = ld; a.C = T; a.ldc = ld;
            gemm(h, a);                                   // T = Sbar V^{-T}
            GemmArgs b; b.m = b.n = b.k = n; b.A = V; b.lda = ld; b.ta = 1; b.B = T; b.ldb = ld; b.C = W; b.ldc = ld;
            gemm(h, b);                                   // W = V^T Sbar V^{-T}
        } else {
            cuda_check(h, cudaMemsetAsync(W, 0, sizeof(double) * nsz, h->stream), "memset");
        }
        double *dlb = nullptr;
        if (lambar) {   // lambar is a device vector in the output order of pssd_eig
            dlb = dalloc(h, n);
            cuda_check(h, cudaMemcpyAsync(dlb, lambar, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream),
                       "memcpy");
        }
        {
            Timed t(h, K_HBM, 0, 16.0 * n * (double)n);
            dk_combine(W, ld, D, dlb, n, T, ld, h->stream);   // T = F o W + diag(lambar)
        }
        GemmArgs c; c.m = c.n = c.k = n; c.A = Vit; c.lda = ld; c.B = T; c.ldb = ld; c.C = W; c.ldc = ld;
        gemm(h, c);                                       // W = V^{-T} T
        GemmArgs d; d.m = d.n = d.k = n; d.A = W; d.lda = ld; d.B = V; d.ldb = ld; d.tb = 1; d.C = Hbar; d.ldc = ldhb;
        gemm(h, d);                                       // Hbar = W V^T
        return PSSD_OK;
    });
}


// ===========================================================================
// Structure-aware variant for the Casida form (Eq. Casida), operating on the
// blocks A and B directly (the direction named in Sec. 7):
//   H = [[A, B], [-B, -A]],  A, B symmetric,  Sigma = diag(I_k, -I_k).
// With the orthogonal T = [[I, I], [I, -I]]/sqrt 2 (T^2 = I):
//   T H T = [[0, R], [P, 0]],  T Sigma T = [[0, I], [I, 0]],  T (Sigma H) T = diag(P, R),
//   P = A + B,  R = A - B  (both SPD exactly when H is definite).
// With P = L_P L_P^T, R = L_R L_R^T the congruence form K = L^T Sigma L of the n x n path
// becomes, in this basis,
//   K_T = diag(L_P, L_R)^T [[0, I], [I, 0]] diag(L_P, L_R) = [[0, C], [C^T, 0]],  C = L_P^T L_R,
// and sign(K_T) = [[0, U], [U^T, 0]] with U the orthogonal polar factor of C = U H_C
// (H_C = U^T C SPD).  The Zolotarev iteration of Alg. 8 on K_T keeps this block form and
// acts on C alone: C_{k+1} = Chat (C_k + C_k sum_j a_j (C_k^T C_k + c_{2j-1} I)^{-1}), with the
// same coefficients, stopping quantity (||K_2 - K_1||_F / ||K_2||_F = ||C_2 - C_1||_F / ||C_2||_F)
// and restarts: every shifted matrix is an SPD k x k Gram matrix (Cholesky, no pivoting).
// The eigenvalues of H are +-sigma_i(C) (C^T C = L_R^T P L_R is similar to P R), so
//   S  = T [[0, L_P^{-T} U L_R^T], [L_R^{-T} U^T L_P^T, 0]] T,
//   Q_+ = T [L_P^{-T} U F; L_R^{-T} F] / sqrt 2,  Q_- = T [L_P^{-T} U F; -L_R^{-T} F] / sqrt 2,
//        F = chol(sym(U^T C)),  A11 = F^T F,  A22 = -F^T F,
//   V_+- = T [L_P^{-T} U W; +-L_R^{-T} W] diag(sqrt(omega)) / sqrt 2 from H_C = W diag(omega) W^T,
// all from k x k products: about a sixth of the n x n path's work per step.
// ===========================================================================
namespace {

struct CasFront {
    int k = 0;
    double *L = nullptr, *Li = nullptr;   // [L_P; L_R] and their inverses (two k x k, stride k^2)
    double *C = nullptr;                   // C = L_P^T L_R
    double *U = nullptr;                   // polar factor of C
    double *Hd = nullptr;                  // H = [[A, B], [-B, -A]] (for the commutator probe)
    double normH = 0.0;
};

int casida_validate(int k, const double *A, int lda, const double *B, int ldb)
{
    if (k < 1 || 2 * (long long)k > PSSD_MAX_N) return -2;
    if (!A) return -3;
    if (lda < k) return -4;
    if (!B) return -5;
    if (ldb < k) return -6;
    return 0;
}

int casida_front(pssd_handle h, int k, const double *A, int lda, const double *B, int ldb, const pssd_opts &o,
                 pssd_info *info, CasFront &F)
{
    F.k = k;
    h->wait_limit = o.wait_cycles;
    h->use_tc = (o.flags & PSSD_FLAG_NO_TENSOR_CORES) ? 0 : 1;
    h->dmode = (o.precision == PSSD_FP64) ? GM_F64 : ((o.flags & PSSD_FLAG_EMU_SIMT) || !h->use_tc ? GM_DF : GM_OZ);
    if (info) { info->precision = o.precision; info->method = o.method; info->p = k; }
    const long long ksz = (long long)k * k;
    F.L = dalloc(h, 2 * ksz);
    F.Li = dalloc(h, 2 * ksz);
    F.C = dalloc(h, ksz);
    {   // P = sym(A + B), R = sym(A - B); symmetry defects of A and B
        const int t = (k + 31) / 32, nb = t * t;
        Mark mk = mark(h);
        double *part = dalloc(h, 2 * (size_t)nb);
        {
            Timed tt(h, K_HBM, 0, 32.0 * ksz);
            casida_prepare(A, lda, B, ldb, k, F.L, F.L + ksz, k, part, h->stream);
        }
        std::vector<double> hp(2 * (size_t)nb);
        d2h_sync(h, hp.data(), part, hp.size() * sizeof(double));
        release(h, mk);
        double d2 = 0, m2 = 0;
        for (int i = 0; i < nb; ++i) { d2 += hp[2 * i]; m2 += hp[2 * i + 1]; }
        if (!std::isfinite(d2) || !std::isfinite(m2)) return PSSD_ERR_NONFINITE;
        F.normH = std::sqrt(m2);
        if (!(m2 > 0.0)) return PSSD_ERR_NOT_DEFINITE;
        if (std::sqrt(d2) > 1e-12 * std::sqrt(m2)) return PSSD_ERR_NOT_PSEUDOSYMMETRIC;
    }
    int fi = -1;   // L_P, L_R and their inverses in one batched factorisation
    if (chol_inv<double>(h, F.L, k, k, ksz, 2, F.Li, ksz, &fi)) {
        if (info) info->fail_index = fi;
        return PSSD_ERR_NOT_DEFINITE;
    }
    GemmArgs g;   // C = L_P^T L_R
    g.m = g.n = g.k = k; g.A = F.L; g.lda = k; g.ta = 1; g.triA = TRI_UPPER;
    g.B = F.L + ksz; g.ldb = k; g.triB = TRI_LOWER; g.C = F.C; g.ldc = k;
    gemm(h, g);
    return PSSD_OK;
}

// bounds alpha >= sigma_max(C) = max|lambda(H)|, beta <= sigma_min(C) = min|lambda(H)| by power
// iteration on C^T C and on (C^T C)^{-1} = L_R^{-1} L_P^{-T} L_P^{-1} L_R^{-T} (the reading of
// Alg. 8's first step used by the n x n path, with the same safety factors), then the polar
// factor U of C by Alg. 8 on C / alpha
int casida_polar(pssd_handle h, CasFront &F, const pssd_opts &o, pssd_info *info)
{
    const int k = F.k;
    const long long ksz = (long long)k * k;
    double alpha = o.alpha, beta = o.beta;
    if (!(alpha > 0.0) || !(beta > 0.0)) {
        Mark mk = mark(h);
        double *v = dalloc(h, k), *w = dalloc(h, 2 * (size_t)k), *u = dalloc(h, k), *tmp = dalloc(h, 32 * (size_t)k + 8);
        cudaStream_t s = h->stream;
        const double *C = F.C, *LPi = F.Li, *LRi = F.Li + ksz;
        if (!(alpha > 0.0))
            alpha = 1.05 * std::sqrt(lmax_estimate(h, k, [&](const double *x, double *y) {
                Timed t(h, K_GEMV, 4.0 * k * (double)k, 16.0 * k * (double)k);
                gemv(C, k, 0, TRI_NONE, k, x, u, tmp, s);           // u = C x
                gemv(C, k, 1, TRI_NONE, k, u, y, tmp, s);           // y = C^T u
            }, 0xa1fa0002ull, v, w, tmp + 32 * (size_t)k));
        if (!(beta > 0.0))
            beta = 0.9 / std::sqrt(lmax_estimate(h, k, [&](const double *x, double *y) {
                Timed t(h, K_GEMV, 4.0 * k * (double)k, 16.0 * k * (double)k);
                double *z = w + k;                                   // second scratch vector
                gemv(LRi, k, 1, TRI_UPPER, k, x, u, tmp, s);        // L_R^{-T} x
                gemv(LPi, k, 0, TRI_LOWER, k, u, z, tmp, s);        // L_P^{-1} .
                gemv(LPi, k, 1, TRI_UPPER, k, z, u, tmp, s);        // L_P^{-T} .
                gemv(LRi, k, 0, TRI_LOWER, k, u, y, tmp, s);        // L_R^{-1} .
            }, 0xbe7a0002ull, v, w, tmp + 32 * (size_t)k));
        release(h, mk);
    }
    if (!(alpha > 0.0) || !(beta > 0.0) || !std::isfinite(alpha) || !std::isfinite(beta)) return PSSD_ERR_NONFINITE;
    if (beta > alpha) beta = alpha;
    if (info) { info->alpha = alpha; info->beta = beta; }
    double *X0 = dalloc(h, ksz), *bA = dalloc(h, ksz), *bB = dalloc(h, ksz);
    {
        Timed t(h, K_HBM, 0, 16.0 * ksz);
        scale_copy<double, double>(F.C, k, X0, k, k, k, 1.0 / alpha, h->stream);
    }
    int fi = -1;
    const int maxr = o.max_restarts < 0 ? 2 : o.max_restarts;
    int st = zolo_sign(h, X0, k, beta / alpha, o.r, maxr, 1e-15, bA, bB, &F.U, info, &fi, /*polar=*/true);
    if (st == PSSD_ERR_NOT_DEFINITE && info) info->fail_index = fi;
    return st;
}

// the full H in the workspace (for the commutator probe of the outputs)
void casida_materialise(pssd_handle h, CasFront &F, const double *A, int lda, const double *B, int ldb)
{
    const int n = 2 * F.k;
    F.Hd = dalloc(h, (size_t)n * n);
    Timed t(h, K_HBM, 0, 48.0 * F.k * (double)F.k);
    casida_build(A, lda, B, ldb, F.k, F.Hd, n, h->stream);
}

int casida_check_opts(const pssd_opts &o)
{
    if (opts_bad(o)) return 1;
    if (o.precision == PSSD_MIXED || o.method != PSSD_METHOD_ZOLO) return 1;
    return 0;
}

}  // namespace

extern "C" int pssd_casida_sign(pssd_handle h, int k, const double *A, int lda, const double *B, int ldb, double *S,
                                int lds, const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    int v = casida_validate(k, A, lda, B, ldb);
    if (v) return v;
    if (!S) return -7;
    if (lds < 2 * k) return -8;
    pssd_opts o = opts ? *opts : defaults();
    if (casida_check_opts(o)) return -9;
    info_init(info);
    return guarded(h, info, [&]() -> int {
        CasFront F;
        int st = casida_front(h, k, A, lda, B, ldb, o, info, F);
        if (!st) st = casida_polar(h, F, o, info);
        if (st) return st;
        const long long ksz = (long long)k * k;
        const double *LP = F.L, *LR = F.L + ksz, *LPi = F.Li, *LRi = F.Li + ksz;
        double *T1 = dalloc(h, ksz), *X = dalloc(h, ksz), *Y = dalloc(h, ksz);
        GemmArgs a; a.m = a.n = a.k = k; a.A = LPi; a.lda = k; a.ta = 1; a.triA = TRI_UPPER; a.B = F.U; a.ldb = k;
        a.C = T1; a.ldc = k;
        gemm(h, a);                                   // L_P^{-T} U
        GemmArgs b; b.m = b.n = b.k = k; b.A = T1; b.lda = k; b.B = LR; b.ldb = k; b.tb = 1; b.triB = TRI_UPPER;
        b.C = X; b.ldc = k;
        gemm(h, b);                                   // X = L_P^{-T} U L_R^T
        GemmArgs c; c.m = c.n = c.k = k; c.A = LRi; c.lda = k; c.ta = 1; c.triA = TRI_UPPER; c.B = F.U; c.ldb = k;
        c.tb = 1; c.C = T1; c.ldc = k;
        gemm(h, c);                                   // L_R^{-T} U^T
        GemmArgs d; d.m = d.n = d.k = k; d.A = T1; d.lda = k; d.B = LP; d.ldb = k; d.tb = 1; d.triB = TRI_UPPER;
        d.C = Y; d.ldc = k;
        gemm(h, d);                                   // Y = L_R^{-T} U^T L_P^T
        {   // S = T [[0, X], [Y, 0]] T = (1/2) [[X + Y, Y - X], [X - Y, -X - Y]]
            Timed t(h, K_HBM, 0, 64.0 * ksz);
            casida_combine(X, k, Y, k, k, k, 1.0, 1.0, 0.5, S, lds, h->stream);
            casida_combine(X, k, Y, k, k, k, -1.0, 1.0, 0.5, S + k, lds, h->stream);
        }
        if (info) {
            casida_materialise(h, F, A, lda, B, ldb);
            const int n = 2 * k;
            std::vector<double> hs(n);
            for (int i = 0; i < n; ++i) hs[i] = i < k ? 1.0 : -1.0;
            double *sig = dalloc(h, n);
            h2d(h, sig, hs.data(), sizeof(double) * n);
            info->comm_resid = comm_resid(h, n, F.Hd, n, F.normH, S, lds, nullptr, 0, sig,
                                          (o.flags & PSSD_FLAG_RESIDUALS) != 0);
        }
        return PSSD_OK;
    });
}

extern "C" int pssd_casida_split(pssd_handle h, int k, const double *A, int lda, const double *B, int ldb, double *Q,
                                 int ldq, double *A11, int lda11, double *A22, int lda22, const pssd_opts *opts,
                                 pssd_info *info)
{
    if (!h) return -1;
    int v = casida_validate(k, A, lda, B, ldb);
    if (v) return v;
    if (!Q) return -7;
    if (ldq < 2 * k) return -8;
    if (!A11) return -9;
    if (lda11 < k) return -10;
    if (!A22) return -11;
    if (lda22 < k) return -12;
    pssd_opts o = opts ? *opts : defaults();
    if (casida_check_opts(o)) return -13;
    info_init(info);
    return guarded(h, info, [&]() -> int {
        CasFront F;
        int st = casida_front(h, k, A, lda, B, ldb, o, info, F);
        if (!st) st = casida_polar(h, F, o, info);
        if (st) return st;
        const long long ksz = (long long)k * k;
        const double *LPi = F.Li, *LRi = F.Li + ksz;
        double *Hc = dalloc(h, ksz), *Fi = dalloc(h, ksz), *T1 = dalloc(h, ksz), *X = dalloc(h, ksz);
        double *Y = dalloc(h, ksz);
        GemmArgs g; g.m = g.n = g.k = k; g.A = F.U; g.lda = k; g.ta = 1; g.B = F.C; g.ldb = k; g.C = Hc; g.ldc = k;
        gemm(h, g);                                   // U^T C
        {
            Timed t(h, K_HBM, 0, 16.0 * ksz);
            sym_average<double>(Hc, k, k, h->stream);  // H_C = sym(U^T C), the polar decomposition's SPD factor
        }
        int fi;
        if (chol_inv<double>(h, Hc, k, k, 0, 1, Fi, 0, &fi)) return PSSD_ERR_BASIS;   // F = chol(H_C)
        GemmArgs a; a.m = a.n = a.k = k; a.A = F.U; a.lda = k; a.B = Hc; a.ldb = k; a.triB = TRI_LOWER;
        a.C = T1; a.ldc = k;
        gemm(h, a);                                   // U F
        GemmArgs b; b.m = b.n = b.k = k; b.A = LPi; b.lda = k; b.ta = 1; b.triA = TRI_UPPER; b.B = T1; b.ldb = k;
        b.C = X; b.ldc = k;
        gemm(h, b);                                   // X = L_P^{-T} U F
        GemmArgs c; c.m = c.n = c.k = k; c.A = LRi; c.lda = k; c.ta = 1; c.triA = TRI_UPPER; c.B = Hc; c.ldb = k;
        c.triB = TRI_LOWER; c.C = Y; c.ldc = k;
        gemm(h, c);                                   // Y = L_R^{-T} F
        {   // Q_+ = T [X; Y]/sqrt 2 = [X + Y; X - Y]/2,  Q_- = T [X; -Y]/sqrt 2 = [X - Y; X + Y]/2
            Timed t(h, K_HBM, 0, 64.0 * ksz);
            casida_combine(X, k, Y, k, k, k, 1.0, 1.0, 0.5, Q, ldq, h->stream);
            casida_combine(X, k, Y, k, k, k, 1.0, -1.0, 0.5, Q + k, ldq, h->stream);
        }
        GemmArgs e; e.m = e.n = e.k = k; e.A = Hc; e.lda = k; e.ta = 1; e.triA = TRI_UPPER; e.B = Hc; e.ldb = k;
        e.triB = TRI_LOWER; e.C = A11; e.ldc = lda11; e.lowerC = 1;
        gemm(h, e);                                   // A11 = F^T F
        mirror(h, A11, lda11, 0, k, 1);
        {
            Timed t(h, K_HBM, 0, 16.0 * ksz);
            scale_copy<double, double>(A11, lda11, A22, lda22, k, k, -1.0, h->stream);   // A22 = -F^T F
        }
        if (info) {
            // backward error of the split of K_T: ||U_+^T K_T U_-||_F / ||K_T||_F with
            // U_+- = [U; +-I]/sqrt 2 is ||U^T C - C^T U||_F / (2 sqrt 2 ||C||_F)
            const bool exact = (o.flags & PSSD_FLAG_RESIDUALS) != 0;
            double d2, e2, c2;
            double *part = dalloc(h, 2 * (size_t)frob_blocks(k, k));
            if (exact) {
                GemmArgs p1; p1.m = p1.n = p1.k = k; p1.A = F.U; p1.lda = k; p1.ta = 1; p1.B = F.C; p1.ldb = k;
                p1.C = T1; p1.ldc = k;
                gemm(h, p1);                          // U^T C
                GemmArgs p2; p2.m = p2.n = p2.k = k; p2.A = F.C; p2.lda = k; p2.ta = 1; p2.B = F.U; p2.ldb = k;
                p2.C = X; p2.ldc = k;
                gemm(h, p2);                          // C^T U
                frob_pair(h, T1, k, X, k, k, k, part, &e2, &d2);
            } else {   // 16-column probe of E = U^T C - C^T U
                constexpr int sc = 16;
                double *Om = dalloc(h, (size_t)k * sc), *P1 = dalloc(h, (size_t)k * sc), *P2 = dalloc(h, (size_t)k * sc);
                {
                    Timed t(h, K_HBM, 0, 8.0 * k * sc);
                    fill_gaussian(Om, sc, k, sc, 0xca51dull, h->stream);
                }
                GemmArgs q1; q1.m = k; q1.n = sc; q1.k = k; q1.A = F.C; q1.lda = k; q1.B = Om; q1.ldb = sc; q1.C = P1; q1.ldc = sc;
                gemm(h, q1);                          // C Om
                GemmArgs q2; q2.m = k; q2.n = sc; q2.k = k; q2.A = F.U; q2.lda = k; q2.ta = 1; q2.B = P1; q2.ldb = sc;
                q2.C = P2; q2.ldc = sc;
                gemm(h, q2);                          // U^T C Om
                GemmArgs q3; q3.m = k; q3.n = sc; q3.k = k; q3.A = F.U; q3.lda = k; q3.B = Om; q3.ldb = sc; q3.C = P1; q3.ldc = sc;
                gemm(h, q3);                          // U Om
                GemmArgs q4; q4.m = k; q4.n = sc; q4.k = k; q4.A = F.C; q4.lda = k; q4.ta = 1; q4.B = P1; q4.ldb = sc;
                q4.Cin = P2; q4.ldcin = sc; q4.beta = -1.0; q4.C = Om; q4.ldc = sc;
                gemm(h, q4);                          // C^T U Om - U^T C Om
                frob_pair(h, nullptr, sc, Om, sc, k, sc, part, &d2, &e2);
                e2 /= sc;
            }
            frob_pair(h, nullptr, k, F.C, k, k, k, part, &d2, &c2);
            info->split_backerr = std::sqrt(e2 / c2) / (2.0 * std::sqrt(2.0));
            casida_materialise(h, F, A, lda, B, ldb);
            const int n = 2 * k;
            std::vector<double> hs(n);
            for (int i = 0; i < n; ++i) hs[i] = i < k ? 1.0 : -1.0;
            double *sig = dalloc(h, n);
            h2d(h, sig, hs.data(), sizeof(double) * n);
            info->comm_resid = comm_resid(h, n, F.Hd, n, F.normH, nullptr, 0, Q, ldq, sig, exact);
        }
        return PSSD_OK;
    });
}

extern "C" int pssd_casida_eig(pssd_handle h, int k, const double *A, int lda, const double *B, int ldb, double *V,
                               int ldv, double *D, const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    int v = casida_validate(k, A, lda, B, ldb);
    if (v) return v;
    if (!V) return -7;
    if (ldv < 2 * k) return -8;
    if (!D) return -9;
    pssd_opts o = opts ? *opts : defaults();
    if (casida_check_opts(o)) return -10;
    const int leaf = o.leaf > 0 ? std::min(o.leaf, 64) : 64;
    info_init(info);
    return guarded(h, info, [&]() -> int {
        CasFront F;
        int st = casida_front(h, k, A, lda, B, ldb, o, info, F);
        if (!st) st = casida_polar(h, F, o, info);
        if (st) return st;
        const long long ksz = (long long)k * k;
        const double *LR = F.L + ksz, *LRi = F.Li + ksz;
        double *Hc = dalloc(h, ksz), *W = dalloc(h, ksz), *w = dalloc(h, k);
        GemmArgs g; g.m = g.n = g.k = k; g.A = F.U; g.lda = k; g.ta = 1; g.B = F.C; g.ldb = k; g.C = Hc; g.ldc = k;
        gemm(h, g);                                   // U^T C
        {
            Timed t(h, K_HBM, 0, 16.0 * ksz);
            sym_average<double>(Hc, k, k, h->stream);  // H_C = sym(U^T C), eigenvalues sigma_i(C)
        }
        int maxdepth = 0;
        st = sym_eig(h, Hc, k, W, w, leaf, 1, &maxdepth, 0x3003ull);   // H_C = W diag(w) W^T (Alg. 2)
        if (st) return st;
        if (info) info->levels = maxdepth;
        // W also diagonalises C^T C = H_C^2, which does not involve U: one refinement step
        // against C^T C (eigenvalues omega^2) removes the error that U's inexactness left in H_C.
        const bool refine = !(o.flags & PSSD_FLAG_NO_REFINE);
        if (refine) {
            GemmArgs g2; g2.m = g2.n = g2.k = k; g2.A = F.C; g2.lda = k; g2.ta = 1; g2.B = F.C; g2.ldb = k;
            g2.C = Hc; g2.ldc = k; g2.lowerC = 1;
            gemm(h, g2);                              // C^T C (lower)
            mirror(h, Hc, k, 0, k, 1);
            st = sym_refine(h, Hc, k, k, W, k, w);
            if (st) return st;
        }
        std::vector<double> hw(k);
        d2h_sync(h, hw.data(), w, sizeof(double) * k);
        std::vector<double> hs(2 * (size_t)k);       // column scales of X and Y
        for (int i = 0; i < k; ++i) {
            if (refine) hw[i] = hw[i] > 0.0 ? std::sqrt(hw[i]) : -1.0;
            if (!(hw[i] > 0.0) || !std::isfinite(hw[i])) return PSSD_ERR_NOT_DEFINITE;
            hs[i] = 1.0 / std::sqrt(hw[i]);           // X: sqrt(omega) / omega
            hs[k + i] = std::sqrt(hw[i]);             // Y: sqrt(omega)
        }
        double *dsc = dalloc(h, 2 * (size_t)k);
        h2d(h, dsc, hs.data(), sizeof(double) * 2 * k);
        double *T1 = dalloc(h, ksz), *X = dalloc(h, ksz), *Y = dalloc(h, ksz);
        // R y = omega x with y = L_R^{-T} W gives x = L_R W / omega (the eigenvectors of
        // C^T C alone fix both halves; L_P^{-T} U W is the same vector in exact arithmetic)
        GemmArgs b; b.m = b.n = b.k = k; b.A = LR; b.lda = k; b.triA = TRI_LOWER; b.B = W; b.ldb = k;
        b.C = X; b.ldc = k;
        gemm(h, b);                                   // L_R W
        GemmArgs c; c.m = c.n = c.k = k; c.A = LRi; c.lda = k; c.ta = 1; c.triA = TRI_UPPER; c.B = W; c.ldb = k;
        c.C = Y; c.ldc = k;
        gemm(h, c);                                   // L_R^{-T} W
        // order: eigenvalues ascending (D: +omega ascending, then -omega in the same order)
        std::vector<int> perm(k);
        for (int i = 0; i < k; ++i) perm[i] = i;
        std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return hw[x] < hw[y]; });
        std::vector<double> hd(2 * (size_t)k);
        for (int i = 0; i < k; ++i) { hd[i] = hw[perm[i]]; hd[k + i] = -hw[perm[i]]; }
        int *dperm = ialloc(h, k);
        h2d(h, dperm, perm.data(), sizeof(int) * k);
        h2d(h, D, hd.data(), sizeof(double) * 2 * k);
        {   // columns scaled (v = sqrt|lambda| [x; y] up to T) and put in order
            Timed t(h, K_HBM, 0, 64.0 * ksz);
            scale_columns(X, k, k, k, dsc, 0, h->stream);
            scale_columns(Y, k, k, k, dsc + k, 0, h->stream);
            gather_columns(X, k, T1, k, k, k, dperm, h->stream);
            gather_columns(Y, k, X, k, k, k, dperm, h->stream);
        }
        {   // V_+ = T [X; Y]/sqrt 2 = [X + Y; X - Y]/2,  V_- = T [X; -Y]/sqrt 2 = [X - Y; X + Y]/2
            Timed t(h, K_HBM, 0, 96.0 * ksz);
            casida_combine(T1, k, X, k, k, k, 1.0, 1.0, 0.5, V, ldv, h->stream);
            casida_combine(T1, k, X, k, k, k, 1.0, -1.0, 0.5, V + k, ldv, h->stream);
            sign_fix_columns(V, ldv, 2 * k, 2 * k, h->stream);
        }
        cuda_check(h, cudaStreamSynchronize(h->stream), "sync");   // host vectors above go out of scope
        if (info) {
            casida_materialise(h, F, A, lda, B, ldb);
            const int n = 2 * k;
            std::vector<double> hs(n);
            for (int i = 0; i < n; ++i) hs[i] = i < k ? 1.0 : -1.0;
            double *sig = dalloc(h, n);
            h2d(h, sig, hs.data(), sizeof(double) * n);
            info->comm_resid = comm_resid(h, n, F.Hd, n, F.normH, nullptr, 0, V, ldv, sig,
                                          (o.flags & PSSD_FLAG_RESIDUALS) != 0);
            cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
        }
        return PSSD_OK;
    });
}


// ===========================================================================
// Batching: many independent Hamiltonians of uneven sizes.
// A host work queue hands instances, largest first, to a pool of workers;
// each worker owns a handle with its own non-blocking stream and workspace and
// runs the full pssd_eig pipeline of its instance there, so the kernels of up
// to PSSD_BATCH_WORKERS instances execute concurrently on the GPU.  The
// workers' streams wait on the caller's stream at entry and the caller's
// stream waits on them at exit.
// ===========================================================================
extern "C" int pssd_eig_batched(pssd_handle h, int count, const int *n, const signed char *const *sigma,
                                const double *const *H, const int *ldh, double *const *V, const int *ldv,
                                double *const *D, const pssd_opts *opts, pssd_info *infos)
{
    if (!h) return -1;
    if (count < 0) return -2;
    if (count == 0) return PSSD_OK;
    if (!n) return -3;
    if (!H || !ldh) return -5;
    if (!V || !ldv) return -7;
    if (!D) return -9;
    if (opts && opts_bad(*opts)) return -10;
    for (int i = 0; i < count; ++i) {
        int v = validate(n[i], sigma ? sigma[i] : nullptr, H[i], ldh[i]);
        if (v) return v;
        if (!V[i] || ldv[i] < n[i] || !D[i]) return -7;
    }
    int nw_max = PSSD_BATCH_WORKERS;
    if (const char *env = std::getenv("PSSD_BATCH_WORKERS")) {
        const long v = std::strtol(env, nullptr, 10);
        if (v >= 1 && v <= 64) nw_max = (int)v;
    }
    const int nw = std::min(count, nw_max);
    try {
        while ((int)h->workers.size() < nw) {
            auto *w = new pssd_handle_s();
            cudaError_t e = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) { delete w; h->last_err = cudaGetErrorString(e); return PSSD_ERR_CUDA; }
            h->workers.push_back(w);
        }
        cudaEvent_t start;
        cuda_check(h, cudaEventCreateWithFlags(&start, cudaEventDisableTiming), "cudaEventCreate");
        cuda_check(h, cudaEventRecord(start, h->stream), "cudaEventRecord");
        for (int w = 0; w < nw; ++w)
            cuda_check(h, cudaStreamWaitEvent(h->workers[w]->stream, start, 0), "cudaStreamWaitEvent");
        std::vector<int> order(count);
        for (int i = 0; i < count; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
        std::atomic<int> next(0);
        std::vector<int> status(count, PSSD_OK);
        auto run = [&](int w) {
            pssd_handle_s *wh = h->workers[w];
            for (;;) {
                int q = next.fetch_add(1);
                if (q >= count) break;
                int i = order[q];
                status[i] = pssd_eig(wh, n[i], sigma ? sigma[i] : nullptr, H[i], ldh[i], V[i], ldv[i], D[i], opts,
                                     infos ? &infos[i] : nullptr);
            }
        };
        std::vector<std::thread> pool;
        for (int w = 1; w < nw; ++w) pool.emplace_back(run, w);
        run(0);
        for (auto &t : pool) t.join();
        for (int w = 0; w < nw; ++w) {
            cudaEvent_t done;
            cuda_check(h, cudaEventCreateWithFlags(&done, cudaEventDisableTiming), "cudaEventCreate");
            cuda_check(h, cudaEventRecord(done, h->workers[w]->stream), "cudaEventRecord");
            cuda_check(h, cudaStreamWaitEvent(h->stream, done, 0), "cudaStreamWaitEvent");
            cudaEventDestroy(done);
        }
        cudaEventDestroy(start);
        for (int i = 0; i < count; ++i)
            if (status[i] != PSSD_OK) return status[i];
        return PSSD_OK;
    } catch (Fail &f) {
        return f.code;
    }
}


// ---------------------------------------------------------------------------
// test hook: the symmetric divide-and-conquer of Alg. 2 (Zolotarev signs of
// shifted subproblems, Jacobi leaves) on a symmetric m x m B, in the handle's
// arithmetic for the given precision mode (PSSD_FP64 or PSSD_FP64_EMULATED):
// W (m x m, columns eigenvectors, unordered) and w (m eigenvalues), device
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Complex pseudo-Hermitian H = Sigma M (M Hermitian positive definite; the BSE forms,
// Eqs. BSE1 and BSE2) through the real embedding R(Z) = [[Re Z, -Im Z], [Im Z, Re Z]]:
// R is an injective real algebra homomorphism with R(Z^H) = R(Z)^T, so R(H) = R(Sigma) R(M)
// is real definite pseudosymmetric with signature [sigma; sigma], sign(R(H)) = R(sign(H)),
// and every eigenvalue of H appears twice in R(H) with the real eigenvectors [Re v; Im v]
// and [-Im v; Re v] of an eigenvector v of H.
// ---------------------------------------------------------------------------
namespace {
int zvalidate(int n, const signed char *sigma, const double *H, int ldh)
{
    if (n < 1 || 2LL * n > PSSD_MAX_N) return -2;
    if (!sigma && (n % 2)) return -3;
    if (sigma)
        for (int i = 0; i < n; ++i) if (sigma[i] != 1 && sigma[i] != -1) return -3;
    if (!H) return -4;
    if (ldh < n) return -5;
    return 0;
}

std::vector<signed char> embedded_signature(int n, const signed char *sigma)
{
    std::vector<signed char> s2(2 * (size_t)n);
    for (int i = 0; i < n; ++i) s2[i] = s2[i + n] = sigma ? sigma[i] : (i < n / 2 ? 1 : -1);
    return s2;
}
}  // namespace

extern "C" int pssd_zsign(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, double *S,
                          int lds, const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    int v = zvalidate(n, sigma, H, ldh);
    if (v) return v;
    if (!S || S == H) return -6;
    if (lds < n) return -7;
    pssd_opts o = opts ? *opts : defaults();
    if (opts_bad(o)) return -8;
    info_init(info);
    return guarded(h, info, [&]() -> int {
        const int m = 2 * n;
        const long long msz = (long long)m * m;
        double *R = dalloc(h, msz), *SR = dalloc(h, msz);
        {
            Timed t(h, K_HBM, 0, 48.0 * n * (double)n);
            complex_embed(H, ldh, n, R, m, h->stream);
        }
        std::vector<signed char> s2 = embedded_signature(n, sigma);
        int st = sign_core(h, m, s2.data(), R, m, SR, m, o, info);
        if (st) return st;
        if (info) info->p /= 2;
        Timed t(h, K_HBM, 0, 32.0 * n * (double)n);
        complex_extract(SR, m, n, n, nullptr, S, lds, h->stream);
        return PSSD_OK;
    });
}

extern "C" int pssd_zeig(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, double *V,
                         int ldv, double *D, const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    int v = zvalidate(n, sigma, H, ldh);
    if (v) return v;
    if (!V) return -6;
    if (ldv < n) return -7;
    if (!D) return -8;
    pssd_opts o = opts ? *opts : defaults();
    if (opts_bad(o)) return -9;
    const int leaf = o.leaf > 0 ? std::min(o.leaf, 64) : 64;
    info_init(info);
    return guarded(h, info, [&]() -> int {
        const int m = 2 * n;
        const long long msz = (long long)m * m;
        double *R = dalloc(h, msz), *VR = dalloc(h, msz), *DR = dalloc(h, m);
        {
            Timed t(h, K_HBM, 0, 48.0 * n * (double)n);
            complex_embed(H, ldh, n, R, m, h->stream);
        }
        std::vector<signed char> s2 = embedded_signature(n, sigma);
        int st = eig_core(h, m, s2.data(), R, m, VR, m, DR, o, info, leaf);
        if (st) return st;
        if (info) info->p /= 2;
        std::vector<double> hd(m);
        d2h_sync(h, hd.data(), DR, sizeof(double) * m);
        // Each eigenvalue of H appears twice, adjacent in the library's order (positive ascending,
        // then negative by ascending magnitude).  Groups of values within 1e-12 max|lambda| of
        // their neighbour (extended to an even size) are one eigenspace of H: a pair gives one
        // eigenvector from either real vector; a larger group of 2q gives q eigenvectors (below).
        double scale = 0.0;
        for (double x : hd) scale = std::max(scale, std::fabs(x));
        const double tol = 1e-12 * scale;
        std::vector<int> perm(n, 0);
        std::vector<double> dout(n);
        struct Group { int first, size, out; };
        std::vector<Group> groups;                 // groups larger than a pair
        int outpos = 0;
        for (int i = 0; i < m;) {
            int j = i + 1;
            while (j < m && ((j - i) % 2 == 1 || std::fabs(hd[j] - hd[j - 1]) <= tol) &&
                   (hd[j] > 0) == (hd[i] > 0))
                ++j;
            const int sz = j - i;
            if (sz % 2) return PSSD_ERR_BASIS;
            double mean = 0.0;
            for (int t = i; t < j; ++t) mean += hd[t];
            mean /= sz;
            for (int q = 0; q < sz / 2; ++q) { perm[outpos + q] = i; dout[outpos + q] = mean; }
            if (sz > 2) groups.push_back({i, sz, outpos});
            outpos += sz / 2;
            i = j;
        }
        if (outpos != n) return PSSD_ERR_BASIS;
        int *dperm = ialloc(h, n);
        h2d(h, dperm, perm.data(), sizeof(int) * n);
        h2d(h, D, dout.data(), sizeof(double) * n);
        {
            Timed t(h, K_HBM, 0, 32.0 * n * (double)n);
            complex_extract(VR, m, n, n, dperm, V, ldv, h->stream);
        }
        if (!groups.empty()) {
            // q eigenvectors of a group of 2q real ones, on the device: Y = R_g Omega (q random
            // vectors of the group's real eigenspace; their complex versions are C-independent
            // with probability 1), Y_e = [Y, J Y] with J [a; b] = [-b; a] (multiplication by i),
            // G_e = s Y_e^T [Sigma; Sigma] Y_e = R(s Y_c^H Sigma Y_c) (the embedding of the complex
            // Gram matrix, positive definite in the group's definite form), and
            // Z_e = Y_e G_e^{-1/2} = R(Y_c G^{-1/2}): the inverse square root of an embedded matrix
            // is the embedding of the inverse square root, so Z_e's first block column is the
            // complex basis, with Z^H Sigma Z = s I.
            std::vector<double> hs2(m);
            for (int i = 0; i < n; ++i) hs2[i] = hs2[i + n] = sigma ? (double)sigma[i] : (i < n / 2 ? 1.0 : -1.0);
            double *sig2 = dalloc(h, m);
            h2d(h, sig2, hs2.data(), sizeof(double) * m);
            for (const Group &g : groups) {
                const int i = g.first, sz = g.size, q = sz / 2, q2 = sz, pos = g.out;
                const double sgn = hd[i] > 0 ? 1.0 : -1.0;
                Mark mg = mark(h);
                double *Om = dalloc(h, (size_t)sz * q), *Ye = dalloc(h, (size_t)m * q2), *Ze = dalloc(h, (size_t)m * q2);
                double *Ge = dalloc(h, (size_t)q2 * q2), *Qe = dalloc(h, (size_t)q2 * q2), *Te = dalloc(h, (size_t)q2 * q2);
                double *Fe = dalloc(h, (size_t)q2 * q2), *le = dalloc(h, q2);
                {
                    Timed t(h, K_HBM, 0, 8.0 * sz * q);
                    fill_gaussian(Om, q, sz, q, 0x2e16ull + (uint64_t)i, h->stream);
                }
                GemmArgs ga; ga.m = m; ga.n = q; ga.k = sz; ga.A = VR + i; ga.lda = m; ga.B = Om; ga.ldb = q;
                ga.C = Ye; ga.ldc = q2;
                gemm(h, ga);                                                   // Y = R_g Omega
                {
                    Timed t(h, K_HBM, 0, 32.0 * n * q);
                    scale_copy<double, double>(Ye + (size_t)n * q2, q2, Ye + q, q2, n, q, -1.0, h->stream);
                    scale_copy<double, double>(Ye, q2, Ye + (size_t)n * q2 + q, q2, n, q, 1.0, h->stream);
                }
                GemmArgs gg; gg.m = gg.n = q2; gg.k = m; gg.A = Ye; gg.lda = q2; gg.ta = 1; gg.B = Ye; gg.ldb = q2;
                gg.kscale = sig2; gg.alpha = sgn; gg.C = Ge; gg.ldc = q2;
                gemm(h, gg);                                                   // G_e
                {
                    Timed t(h, K_HBM, 0, 16.0 * q2 * q2);
                    sym_average<double>(Ge, q2, q2, h->stream);
                }
                if (q2 <= 64) {
                    Timed t(h, K_JACOBI, 0);
                    jacobi_leaf(Ge, q2, q2, Qe, q2, le, nullptr, h->stream);
                } else {
                    int md = 0;
                    int st2 = sym_eig(h, Ge, q2, Qe, le, 64, 1, &md, 0x2e17ull + (uint64_t)i);
                    if (st2) return st2;
                }
                std::vector<double> hl(q2);
                d2h_sync(h, hl.data(), le, sizeof(double) * q2);
                for (double &x : hl) {
                    if (!(x > 0.0) || !std::isfinite(x)) return PSSD_ERR_BASIS;
                    x = 1.0 / std::sqrt(x);
                }
                h2d(h, le, hl.data(), sizeof(double) * q2);
                {
                    Timed t(h, K_HBM, 0, 32.0 * q2 * q2);
                    copy_matrix(Qe, q2, Te, q2, q2, q2, h->stream);
                    scale_columns(Te, q2, q2, q2, le, 0, h->stream);           // Q diag(l^{-1/2})
                }
                GemmArgs gf; gf.m = gf.n = gf.k = q2; gf.A = Te; gf.lda = q2; gf.B = Qe; gf.ldb = q2; gf.tb = 1;
                gf.C = Fe; gf.ldc = q2;
                gemm(h, gf);                                                   // G_e^{-1/2}
                GemmArgs gz; gz.m = m; gz.n = q2; gz.k = q2; gz.A = Ye; gz.lda = q2; gz.B = Fe; gz.ldb = q2;
                gz.C = Ze; gz.ldc = q2;
                gemm(h, gz);                                                   // Z_e = Y_e G_e^{-1/2}
                {
                    Timed t(h, K_HBM, 0, 32.0 * n * q);
                    complex_extract(Ze, q2, n, q, nullptr, V + 2 * (size_t)pos, ldv, h->stream);
                }
                cuda_check(h, cudaStreamSynchronize(h->stream), "sync");      // hl goes out of scope
                release(h, mg);
            }
        }
        {
            Timed t(h, K_HBM, 0, 32.0 * n * (double)n);
            complex_phase_fix(V, ldv, n, n, h->stream);
        }
        cuda_check(h, cudaStreamSynchronize(h->stream), "sync");   // host vectors above go out of scope
        return PSSD_OK;
    });
}

extern "C" int pssd_test_sym_eig(pssd_handle h, int m, const double *B, int ldb, double *W, int ldw, double *w,
                                 const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    if (m < 1 || m > PSSD_MAX_N) return -2;
    if (!B) return -3;
    if (ldb < m) return -4;
    if (!W) return -5;
    if (ldw < m) return -6;
    if (!w) return -7;
    pssd_opts o = opts ? *opts : defaults();
    if (opts_bad(o) || o.precision == PSSD_MIXED) return -8;
    const int leaf = o.leaf > 0 ? std::min(o.leaf, 64) : 64;
    info_init(info);
    return guarded(h, info, [&]() -> int {
        h->wait_limit = o.wait_cycles;
        h->use_tc = (o.flags & PSSD_FLAG_NO_TENSOR_CORES) ? 0 : 1;
        h->dmode = (o.precision == PSSD_FP64) ? GM_F64 : ((o.flags & PSSD_FLAG_EMU_SIMT) || !h->use_tc ? GM_DF : GM_OZ);
        const long long msz = (long long)m * m;
        double *Bc = dalloc(h, msz), *Wc = dalloc(h, msz);
        {
            Timed t(h, K_HBM, 0, 16.0 * msz);
            copy_matrix(B, ldb, Bc, m, m, m, h->stream);
        }
        int maxdepth = 0;
        int st = sym_eig(h, Bc, m, Wc, w, leaf, 0, &maxdepth, 0x5e11ull);
        if (!st && !(o.flags & PSSD_FLAG_NO_REFINE)) st = sym_refine(h, Bc, m, m, Wc, m, w);
        if (st) return st;
        if (info) info->levels = maxdepth;
        Timed t(h, K_HBM, 0, 16.0 * msz);
        copy_matrix(Wc, m, W, ldw, m, m, h->stream);
        return PSSD_OK;
    });
}

// ---------------------------------------------------------------------------
// sign(H) of a general (not necessarily definite) pseudosymmetric H, Sigma H
// symmetric but indefinite (Def. pseudosym; the case of Alg. 3): the Newton
// iteration of Eq. NewtonSign with Frobenius-norm scaling, run on the symmetric
// W = Sigma X.  With X = Sigma W, X^{-1} = W^{-1} Sigma, so Sigma X_{k+1} =
// (mu W_k + Sigma W_k^{-1} Sigma / mu) / 2 stays symmetric; and W^{-1} =
// (W^2)^{-1} W with W^2 symmetric positive definite for every nonsingular W, so a
// step is one product W W, one Cholesky with inverse, two products and one pass --
// no pivoted indefinite factorisation.  S = Sigma W at convergence.
// ---------------------------------------------------------------------------
namespace {
// the general sign iteration on the device (see pssd_gsign): S = sign(H), sig the device
// signature; the handle's engines and modes are set by the caller
int gsign_core(pssd_handle h, int n, const double *sig, const double *H, int ldh, double *S, int lds,
               pssd_info *info)
{
    const long long ld = n, nsz = (long long)n * n;
    Mark outer = mark(h);
    const int st = [&]() -> int {
        double *W = dalloc(h, nsz), *Wn = dalloc(h, nsz), *G = dalloc(h, nsz), *Ri = dalloc(h, nsz);
        double *Gi = dalloc(h, nsz), *T = dalloc(h, nsz);
        {   // W_0 = sym(Sigma H), and the symmetry defect of Sigma H
            const int nb = sym_prepare_blocks(n);
            Mark mk = mark(h);
            double *pp = dalloc(h, 2 * (size_t)nb);
            {
                Timed t(h, K_HBM, 0, 16.0 * n * (double)n);
                sym_prepare(H, ldh, sig, n, W, ld, pp, h->stream);
            }
            std::vector<double> hp(2 * (size_t)nb);
            d2h_sync(h, hp.data(), pp, hp.size() * sizeof(double));
            release(h, mk);
            double d2 = 0, m2 = 0;
            for (int i = 0; i < nb; ++i) { d2 += hp[2 * i]; m2 += hp[2 * i + 1]; }
            if (!std::isfinite(d2) || !std::isfinite(m2)) return PSSD_ERR_NONFINITE;
            if (!(m2 > 0.0)) return PSSD_ERR_NO_CONVERGENCE;        // H = 0: sign(H) undefined
            if (std::sqrt(d2) > 1e-12 * std::sqrt(m2)) return PSSD_ERR_NOT_PSEUDOSYMMETRIC;
        }
        double *part = dalloc(h, 2 * (size_t)frob_blocks(n, n));
        const double tol = std::sqrt(U64);
        bool scaled = true, done = false;
        for (int it = 0; it < 100 && !done; ++it) {
            {   // W^2 (lower)
                GemmArgs g; g.m = g.n = g.k = n; g.A = W; g.lda = ld; g.B = W; g.ldb = ld; g.C = G; g.ldc = ld;
                g.lowerC = 1;
                gemm(h, g);
            }
            int fi = -1;
            if (chol_inv<double>(h, G, n, ld, 0, 1, Ri, 0, &fi)) {   // W_k numerically singular
                if (info) info->fail_index = fi;
                return PSSD_ERR_NO_CONVERGENCE;
            }
            {   // (W^2)^{-1} = R^{-T} R^{-1} (lower, mirrored)
                GemmArgs l; l.m = l.n = l.k = n; l.A = Ri; l.lda = ld; l.ta = 1; l.triA = TRI_UPPER;
                l.B = Ri; l.ldb = ld; l.triB = TRI_LOWER; l.C = Gi; l.ldc = ld; l.lowerC = 1;
                gemm(h, l);
                mirror<double>(h, Gi, ld, 0, n, 1);
            }
            {   // W^{-1} = (W^2)^{-1} W (symmetric: lower, mirrored)
                GemmArgs f; f.m = f.n = f.k = n; f.A = Gi; f.lda = ld; f.B = W; f.ldb = ld; f.C = T; f.ldc = ld;
                f.lowerC = 1;
                gemm(h, f);
                mirror<double>(h, T, ld, 0, n, 1);
            }
            double mu = 1.0;
            if (scaled) {   // mu = (||X^{-1}||_F / ||X||_F)^{1/2} = (||W^{-1}||_F / ||W||_F)^{1/2}
                double a2, w2, b2, t2;
                frob_pair(h, nullptr, ld, W, ld, n, n, part, &a2, &w2);
                frob_pair(h, nullptr, ld, T, ld, n, n, part, &b2, &t2);
                mu = std::sqrt(std::sqrt(t2 / w2));
                if (!std::isfinite(mu) || !(mu > 0.0)) return PSSD_ERR_NONFINITE;
            }
            {   // W_{k+1} = (mu W + Sigma W^{-1} Sigma / mu) / 2
                Timed t(h, K_HBM, 0, 24.0 * n * (double)n);
                sig_affine(W, ld, 0, T, ld, sig, n, 0.5 * mu, 0.5 / mu, Wn, ld, h->stream);
            }
            double d2, y2;
            frob_pair(h, W, ld, Wn, ld, n, n, part, &d2, &y2);
            if (!std::isfinite(d2) || !std::isfinite(y2)) return PSSD_ERR_NONFINITE;
            if (!(y2 > 0.0)) return PSSD_ERR_NO_CONVERGENCE;   // the iterate vanished: eigenvalues +-i t
            const double crit = std::sqrt(d2 / y2);
            if (info) {
                if (it < 4) info->stop_crit[it] = crit;
                info->iterations = info->steps = it + 1;
                info->passes = 1;
            }
            std::swap(W, Wn);
            if (crit < 1e-2) scaled = false;   // near the limit: unscaled steps keep the quadratic rate
            done = crit <= tol;
        }
        if (!done) return PSSD_ERR_NO_CONVERGENCE;
        {   // S = Sigma W
            Timed t(h, K_HBM, 0, 16.0 * n * (double)n);
            sig_affine(W, ld, 1, nullptr, 0, sig, n, 1.0, 0.0, S, lds, h->stream);
        }
        {   // p = (n + trace S) / 2: the eigenvalues with positive real part
            Timed t(h, K_HBM, 0, 8.0 * n);
            trace_partial(S, lds, n, part, h->stream);
        }
        double tr;
        d2h_sync(h, &tr, part, sizeof(double));
        if (info) {
            info->p = (int)std::lround(0.5 * (n + tr));
            info->jsym_resid = 0.0;                  // Sigma S = W is symmetric by construction
            GemmArgs g; g.m = g.n = g.k = n; g.A = S; g.lda = lds; g.B = S; g.ldb = lds; g.C = G; g.ldc = ld;
            gemm(h, g);                                                   // S^2
            {
                Timed t(h, K_HBM, 0, 8.0 * n);
                add_diag<double>(G, ld, n, -1.0, h->stream);
            }
            double d2, q2;
            frob_pair(h, nullptr, ld, G, ld, n, n, part, &d2, &q2);
            info->s2_resid = std::sqrt(q2);
        }
    return PSSD_OK;
    }();
    release(h, outer);
    return st;
}
}  // namespace

extern "C" int pssd_gsign(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, double *S,
                          int lds, const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    int v = validate(n, sigma, H, ldh);
    if (v) return v;
    if (!S || S == H) return -6;
    if (lds < n) return -7;
    pssd_opts o = opts ? *opts : defaults();
    if (opts_bad(o) || o.precision == PSSD_MIXED) return -8;
    info_init(info);
    return guarded(h, info, [&]() -> int {
        PhaseScope phase(PH_SIGN);
        h->wait_limit = o.wait_cycles;
        h->use_tc = (o.flags & PSSD_FLAG_NO_TENSOR_CORES) ? 0 : 1;
        h->dmode = (o.precision == PSSD_FP64) ? GM_F64 : ((o.flags & PSSD_FLAG_EMU_SIMT) || !h->use_tc ? GM_DF : GM_OZ);
        if (info) { info->method = PSSD_METHOD_NEWTON; info->precision = o.precision; }
        std::vector<double> hs(n);
        for (int i = 0; i < n; ++i) hs[i] = sigma ? (double)sigma[i] : (i < n / 2 ? 1.0 : -1.0);
        double *sig = dalloc(h, n);
        h2d(h, sig, hs.data(), sizeof(double) * n);
        return gsign_core(h, n, sig, H, ldh, S, lds, info);
    });
}

// ---------------------------------------------------------------------------
// Split of a general pseudosymmetric H (Alg. 3's division step): S from the general
// sign iteration; a Gaussian sketch of each projector (I +- S)/2 made orthonormal
// (CholeskyQR2, then the projector applied once more and one Cholesky QR pass);
// the symmetric Sigma-Gram matrix G = U^T Sigma U of each basis diagonalised by the
// symmetric recursion (G = W Lambda W^T), Q = U W |Lambda|^{-1/2}, Sigma_hat =
// sign(Lambda), so Q^T Sigma Q = Sigma_hat: the (Sigma, Sigma_hat)-orthogonal basis
// that Alg. 5 obtains from a pivoted LDL^T, reached without pivoting.  Then
// A11 = Sigma_hat_+ Q_+^T Sigma H Q_+, A22 likewise (pseudosymmetric with respect
// to Sigma_hat_+ and Sigma_hat_-).
// ---------------------------------------------------------------------------
extern "C" int pssd_gsplit(pssd_handle h, int n, const signed char *sigma, const double *H, int ldh, double *Q,
                           int ldq, double *A11, int lda11, double *A22, int lda22, signed char *sigma_hat,
                           int *p_out, const pssd_opts *opts, pssd_info *info)
{
    if (!h) return -1;
    int v = validate(n, sigma, H, ldh);
    if (v) return v;
    if (!Q || Q == H) return -6;
    if (ldq < n) return -7;
    if (!A11) return -8;
    if (lda11 < n) return -9;
    if (!A22) return -10;
    if (lda22 < n) return -11;
    if (!sigma_hat) return -12;
    pssd_opts o = opts ? *opts : defaults();
    if (opts_bad(o) || o.precision == PSSD_MIXED) return -14;
    info_init(info);
    return guarded(h, info, [&]() -> int {
        PhaseScope phase(PH_SIGN);
        h->wait_limit = o.wait_cycles;
        h->use_tc = (o.flags & PSSD_FLAG_NO_TENSOR_CORES) ? 0 : 1;
        h->dmode = (o.precision == PSSD_FP64) ? GM_F64 : ((o.flags & PSSD_FLAG_EMU_SIMT) || !h->use_tc ? GM_DF : GM_OZ);
        if (info) { info->method = PSSD_METHOD_NEWTON; info->precision = o.precision; }
        const long long ld = n, nsz = (long long)n * n;
        std::vector<double> hs(n);
        for (int i = 0; i < n; ++i) hs[i] = sigma ? (double)sigma[i] : (i < n / 2 ? 1.0 : -1.0);
        double *sig = dalloc(h, n);
        h2d(h, sig, hs.data(), sizeof(double) * n);
        double *S = dalloc(h, nsz);
        int st = gsign_core(h, n, sig, H, ldh, S, ld, info);
        if (st) return st;
        g_phase = PH_SPLIT;
        double *tmp = dalloc(h, 2 * (size_t)frob_blocks(n, n) + 8);
        {
            Timed t(h, K_HBM, 0, 8.0 * n);
            trace_partial(S, ld, n, tmp, h->stream);
        }
        double tr;
        d2h_sync(h, &tr, tmp, sizeof(double));
        const int p = (int)std::lround(0.5 * (n + tr)), q = n - p;
        if (p < 0 || q < 0) return PSSD_ERR_BASIS;
        if (p_out) *p_out = p;
        if (info) info->p = p;
        // sketches of the two projectors, orthonormal bases U = [U_+ U_-]
        double *Om = dalloc(h, nsz), *Yb = dalloc(h, nsz), *U = dalloc(h, nsz);
        {
            Timed t(h, K_HBM, 0, 8.0 * n * (double)n);
            fill_gaussian(Om, ld, n, n, 0x9e5b17ull, h->stream);
        }
        auto project = [&](const double *X) {   // Yb = [(I + S)/2 X_+, (I - S)/2 X_-]
            GemmArgs g; g.m = g.n = g.k = n; g.A = S; g.lda = ld; g.B = X; g.ldb = ld; g.C = Yb; g.ldc = ld;
            gemm(h, g);
            Timed t(h, K_HBM, 0, 24.0 * n * (double)n);
            half_sum_diff(X, ld, Yb, ld, n, n, p, h->stream);
        };
        auto bases = [&](int passes) -> int {
            int r = PSSD_OK;
            if (p > 0) r = cholqr2(h, Yb, ld, n, p, U, ld, 1, 0, 0, passes);
            if (!r && q > 0) r = cholqr2(h, Yb + p, ld, n, q, U + p, ld, 1, 0, 0, passes);
            return r;
        };
        project(Om);
        if (bases(2)) return PSSD_ERR_BASIS;
        project(U);
        if (bases(1)) return PSSD_ERR_BASIS;
        // Sigma-Gram matrices and their eigendecompositions: Q = U W |Lambda|^{-1/2}
        std::vector<double> shat(n);
        auto hyperbolic = [&](const double *Uh, int r, double *Qh, double *sh) -> int {
            Mark mk = mark(h);
            double *Gm = dalloc(h, (size_t)r * r), *Wg = dalloc(h, (size_t)r * r), *wg = dalloc(h, r);
            double *inv = dalloc(h, r);
            GemmArgs g; g.m = g.n = r; g.k = n; g.A = Uh; g.lda = ld; g.ta = 1; g.kscale = sig; g.B = Uh;
            g.ldb = ld; g.C = Gm; g.ldc = r; g.lowerC = 1;
            gemm(h, g);                                                   // U^T Sigma U (lower)
            mirror<double>(h, Gm, r, 0, r, 1);
            int maxdepth = 0;
            int e = sym_eig(h, Gm, r, Wg, wg, 64, 1, &maxdepth, 0x6e9a11ull + r);
            if (!e) e = sym_refine(h, Gm, r, r, Wg, r, wg);
            if (e) { release(h, mk); return e; }
            std::vector<double> hw(r);
            d2h_sync(h, hw.data(), wg, sizeof(double) * r);
            double wmax = 0.0;
            for (double x : hw) wmax = std::max(wmax, std::fabs(x));
            std::vector<double> hinv(r);
            for (int i = 0; i < r; ++i) {
                if (!(std::fabs(hw[i]) > 1e-10 * wmax)) { release(h, mk); return PSSD_ERR_BASIS; }
                sh[i] = hw[i] > 0.0 ? 1.0 : -1.0;
                hinv[i] = 1.0 / std::fabs(hw[i]);
            }
            h2d(h, inv, hinv.data(), sizeof(double) * r);
            GemmArgs b; b.m = n; b.n = r; b.k = r; b.A = Uh; b.lda = ld; b.B = Wg; b.ldb = r; b.C = Qh; b.ldc = ldq;
            gemm(h, b);                                                   // U W
            {
                Timed t(h, K_HBM, 0, 16.0 * n * (double)r);
                scale_columns(Qh, ldq, n, r, inv, 1, h->stream);          // . |Lambda|^{-1/2}
            }
            cuda_check(h, cudaStreamSynchronize(h->stream), "sync");      // hinv goes out of scope
            release(h, mk);
            return PSSD_OK;
        };
        if (p > 0 && (st = hyperbolic(U, p, Q, shat.data()))) return st;
        if (q > 0 && (st = hyperbolic(U + p, q, Q + p, shat.data() + p))) return st;
        for (int i = 0; i < n; ++i) sigma_hat[i] = (signed char)(shat[i] > 0.0 ? 1 : -1);
        // blocks: A = Sigma_hat Q^T Sigma (H Q), diagonal blocks and (info) the coupling block
        double *HQ = dalloc(h, nsz), *shd = dalloc(h, n);
        h2d(h, shd, shat.data(), sizeof(double) * n);
        {
            GemmArgs g; g.m = g.n = g.k = n; g.A = H; g.lda = ldh; g.B = Q; g.ldb = ldq; g.C = HQ; g.ldc = ld;
            gemm(h, g);
        }
        auto block = [&](int off, int r, double *Ab, int ldab) {
            GemmArgs g; g.m = g.n = r; g.k = n; g.A = Q + off; g.lda = ldq; g.ta = 1; g.kscale = sig;
            g.B = HQ + off; g.ldb = ld; g.C = Ab; g.ldc = ldab;
            gemm(h, g);
            Timed t(h, K_HBM, 0, 16.0 * r * (double)r);
            sig_affine(Ab, ldab, 1, nullptr, 0, shd + off, r, 1.0, 0.0, Ab, ldab, h->stream);
        };
        if (p > 0) block(0, p, A11, lda11);
        if (q > 0) block(p, q, A22, lda22);
        if (info && p > 0 && q > 0) {   // ||Q_+^dagger H Q_-||_F / ||H||_F
            double *E = dalloc(h, (size_t)p * q);
            GemmArgs g; g.m = p; g.n = q; g.k = n; g.A = Q; g.lda = ldq; g.ta = 1; g.kscale = sig;
            g.B = HQ + p; g.ldb = ld; g.C = E; g.ldc = q;
            gemm(h, g);
            double a2, e2, b2, h2;
            frob_pair(h, nullptr, q, E, q, p, q, tmp, &a2, &e2);
            frob_pair(h, nullptr, ldh, H, ldh, n, n, tmp, &b2, &h2);
            info->split_backerr = std::sqrt(e2 / h2);
        }
        cuda_check(h, cudaStreamSynchronize(h->stream), "sync");          // shat goes out of scope
        return PSSD_OK;
    });
}

// ---------------------------------------------------------------------------
// test hook: the Krylov loops behind the bounds, the shift search and the shift
// screening, step by step or in one cluster launch, on the operators they use
// ---------------------------------------------------------------------------
extern "C" int pssd_test_krylov(pssd_handle h, int op, int m, const double *A, int lda, int steps, int power,
                                unsigned long long seed, int fused, double *out, double *v0)
{
    if (!h) return -1;
    if (op != PSSD_KRYLOV_SYM && op != PSSD_KRYLOV_TRI_PAIR) return -2;
    if (m < 1 || m > PSSD_MAX_N || (fused && m > KRY_MAX_M)) return -3;
    if (!A) return -4;
    if (lda < m) return -5;
    if (power < 0 || power > 1000 || (power == 0 && (steps < 1 || steps > m))) return -6;
    if (!out) return -7;
    return guarded(h, nullptr, [&]() -> int {
        Mark mk = mark(h);
        double *v = dalloc(h, m), *w = dalloc(h, m), *u = dalloc(h, m), *tmp = dalloc(h, 32 * (size_t)m + 8);
        KryFused kf; kf.A = A; kf.lda = lda; kf.op = op == PSSD_KRYLOV_SYM ? KRY_SYM : KRY_TRI_PAIR;
        auto apply = [&](const double *x, double *y) {
            if (kf.op == KRY_SYM) {
                gemv(A, lda, 0, TRI_NONE, m, x, y, tmp, h->stream);
            } else {
                gemv(A, lda, 0, TRI_LOWER, m, x, u, tmp, h->stream);
                gemv(A, lda, 1, TRI_UPPER, m, u, y, tmp, h->stream);
            }
        };
        if (power > 0) power_device(h, m, apply, v, w, out, power, fused ? &kf : nullptr);
        else lanczos_device(h, m, apply, seed, steps, out, fused ? &kf : nullptr);
        if (v0) fill_gaussian(v0, m, 1, m, power > 0 ? 0x5eedull : seed, h->stream);
        cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
        release(h, mk);
        return PSSD_OK;
    });
}

// ---------------------------------------------------------------------------
// test hook: one FP32 contraction through the library's GEMM dispatch
// (tensor-core kernel or FP32 SIMT kernel), for parity tests of the kernels
// ---------------------------------------------------------------------------
extern "C" int pssd_test_gemm_f32(pssd_handle h, int use_tc, int m, int n, int k, int batch, int ta, int tb,
                                  int triA, int triB, int lowerC, double alpha, double beta, const float *A,
                                  long long lda, long long sA, const float *B, long long ldb, long long sB,
                                  const float *Cin, long long ldcin, long long sCin, float *C, long long ldc,
                                  long long sC, const float *kscale)
{
    if (!h) return -1;
    if (m < 0 || n < 0 || k < 0 || batch < 1) return -3;
    return guarded(h, nullptr, [&]() -> int {
        h->use_tc = use_tc ? 1 : 0;
        GemmArgs g; g.mode = GM_F32; g.m = m; g.n = n; g.k = k; g.batch = batch;
        g.A = A; g.lda = lda; g.sA = sA; g.ta = ta; g.triA = triA;
        g.B = B; g.ldb = ldb; g.sB = sB; g.tb = tb; g.triB = triB;
        g.Cin = Cin; g.ldcin = ldcin; g.sCin = sCin; g.C = C; g.ldc = ldc; g.sC = sC;
        g.kscale = kscale; g.alpha = alpha; g.beta = beta; g.lowerC = lowerC;
        gemm(h, g);
        h->use_tc = 1;
        return PSSD_OK;
    });
}


// test hook: one FP64 contraction with a chosen engine (0 DFMA, 1 float pairs on
// the FP32 pipe, 2 integer slices on the BF16 tensor cores)
extern "C" int pssd_test_gemm_f64(pssd_handle h, int engine, int m, int n, int k, int batch, int ta, int tb,
                                  int triA, int triB, int lowerC, double alpha, double beta, const double *A,
                                  long long lda, long long sA, const double *B, long long ldb, long long sB,
                                  const double *Cin, long long ldcin, long long sCin, double *C, long long ldc,
                                  long long sC, const double *kscale)
{
    if (!h) return -1;
    if (engine < 0 || engine > 2) return -2;
    if (m < 0 || n < 0 || k < 0 || batch < 1) return -3;
    return guarded(h, nullptr, [&]() -> int {
        h->force_engine = 1;
        GemmArgs g; g.mode = engine == 0 ? GM_F64 : (engine == 1 ? GM_DF : GM_OZ);
        g.m = m; g.n = n; g.k = k; g.batch = batch;
        g.A = A; g.lda = lda; g.sA = sA; g.ta = ta; g.triA = triA;
        g.B = B; g.ldb = ldb; g.sB = sB; g.tb = tb; g.triB = triB;
        g.Cin = Cin; g.ldcin = ldcin; g.sCin = sCin; g.C = C; g.ldc = ldc; g.sC = sC;
        g.kscale = kscale; g.alpha = alpha; g.beta = beta; g.lowerC = lowerC;
        gemm(h, g);
        h->force_engine = 0;
        return PSSD_OK;
    });
}
