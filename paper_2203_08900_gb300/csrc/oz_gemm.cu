// FP64-accurate GEMM on the BF16 tensor cores of sm_103a (tcgen05), by exact
// integer slicing (the error-free splitting scheme of Ozaki, Ogita, Oishi and
// Rump, 2012).
//
//   C = alpha * op(A) * diag(kscale) * op(B) + beta * Cin        (FP64 data)
//
// 1. Every row i of op(A) is scaled by 2^{-e_i} and every column j of op(B)
//    by 2^{-f_j} (exact) so that all entries lie in (-1, 1).
// 2. Each scaled entry x is rounded to F = round(x 2^56) (error <= 2^-57)
//    and F is cut into S = 8 integer digits of 7 bits, balanced base 128:
//      x ~ sum_t d_t 2^{-7t},  |d_1| <= 128,  |d_t| <= 64 (t > 1);
//    the d_t are exact in BF16.  (Integer work only: FP64 arithmetic is a
//    slow pipe on this part.)
// 3. For every level L = a + b (2 <= L <= S+1) the slice products
//    sum_{a+b=L} D^A_a D^B_b are integers; one term is at most
//    2^14 + max(0, L-3) 2^12 (two products with a slice d_1, the rest 2^12).
//    Over a 512-term stretch of k the levels L <= 7 stay at or below 2^24, so
//    the tensor cores' FP32 accumulation of them is exact.  Levels 8 and 9 can
//    pass 2^24 only when the (1, L-1) and (L-1, 1) products are near 2^13,
//    i.e. when the entries are near their row/column maxima; their rounding
//    (at most 512 units at weight 2^{-7L}) is then below 2^-55 of
//    sum_p |a_ip b_pj|.  Each level has its own accumulator in tensor memory
//    (8 levels x 64 columns = all 512).
// 4. Every 512 terms of k the eight level sums are scaled by 2^{-7L} (exact)
//    and added into a float-pair (TwoSum) accumulator per output; at the end
//    C = alpha 2^{e_i + f_j} (hi + lo) + beta Cin in FP64.
// Products with a + b > S + 1 (36 of 64 kept) are dropped.  Level L = a + b
// carries weight 2^{-7L} and its terms are at most 2^12 (2^14 with a d_1 slice),
// so the first dropped level (L = 10, seven products) contributes up to about
// 7 * 2^12 * 2^-70 ~ 2^-55 of the row/column maxima per term, and the levels
// beyond it less: the dropped part is ~2^-55 relative to sum_p |a_ip||b_pj| in
// the worst case (the measured error is 0.9-1.7e-15 of that sum).
//
// Kernel layout: one CTA of 18 warps per 128 x 64 output tile, warp-specialised:
// warp 16 streams the 8 A-slice tiles (128 x 16 BF16) and 8 B-slice tiles
// (64 x 16) of one k block, stored pre-tiled and pre-swizzled (32-byte swizzle)
// by the slicing pass, as two contiguous bulk copies into a 4-stage mbarrier ring; warp 17 issues 12
// tcgen05.mma kind::f16 (M=128, N=64..256, K=16) per stage, which cover the 36
// slice products, into 8 accumulators of 64 TMEM columns and frees each stage
// with tcgen05.commit; warps 0-15 flush the accumulators every 512 terms
// (warp w reads TMEM lanes 32 (w % 4) .. and 16 columns per level, so four
// warps per SM sub-partition hide the TwoSum latency) while the producer keeps
// prefetching, then signal the MMA warp that the accumulators are free.
// Every pipeline mbarrier wait is bounded by the caller's limit (error flag,
// then the kernel waits -- under a fixed, longer bound -- for its own bulk
// copies and MMAs in flight, frees TMEM and returns).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "pssd_internal.h"

namespace pssd {

namespace {

constexpr int OZ_S = 8;                    // slices
constexpr int OZ_LEVELS = OZ_S;            // levels L = 2 .. S+1
constexpr int OZ_BM = 128, OZ_BN = 64, OZ_BK = 16;   // BK in BF16 elements = 32 bytes = one MMA K
constexpr int OZ_STAGES = 4;
constexpr int OZ_CHUNK_STAGES = 32;        // flush every 32 x 16 = 512 terms of k
constexpr int OZ_A_TILE = OZ_BM * OZ_BK * 2;          // 4 KB
constexpr int OZ_B_TILE = OZ_BN * OZ_BK * 2;          // 2 KB
constexpr int OZ_STAGE_BYTES = OZ_S * (OZ_A_TILE + OZ_B_TILE);   // 48 KB
constexpr int OZ_SMEM_BYTES = OZ_STAGES * OZ_STAGE_BYTES + 1024 + 256;
constexpr unsigned long long OZ_WAIT_LIMIT = 1ull << 26;   // default pipeline bound and the drain bound
constexpr int OZ_TMEM_COLS = 512;
constexpr int OZ_FLUSH_WARPS = 16;         // warp w: TMEM lanes 32 (w % 4) .., columns 16 (w / 4) ..
constexpr int OZ_FCOLS = OZ_BN / (OZ_FLUSH_WARPS / 4);   // 16 output columns per flush thread
constexpr int OZ_PRODUCER_WARP = OZ_FLUSH_WARPS, OZ_MMA_WARP = OZ_FLUSH_WARPS + 1;
constexpr int OZ_THREADS = 32 * (OZ_FLUSH_WARPS + 2);
constexpr int OZ_GROUP_M = 8;              // row blocks per group of the tile order

struct OzArgs {
    // slices, tiled: block (z, row tile, k block) = 8 slices x tile rows x 16 k,
    // 32-byte-swizzled rows, contiguous (32 KB for A, 16 KB for B)
    const __nv_bfloat16 *sa, *sb;
    int kblocks;                           // k_pad / 16
    int m, n, k, batch, m_pad, n_pad;
    int triA, triB, lowerC;
    const int *ea, *eb;                    // exponents per row of op(A) (batch*m_pad), per column of op(B)
    double *C; long long ldc, sC;
    const double *Cin; long long ldcin, sCin;
    double alpha, beta;
    int alpha_e, alpha_e_valid, alpha_neg;   // alpha = (-1)^neg 2^alpha_e when valid
    int *err;
    unsigned long long wait_limit;         // polls per pipeline wait before giving up
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit)
{
    for (unsigned long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"((unsigned long long)src), "r"(bytes), "r"(bar)
        : "memory");
}

// K-major operand, 32-byte swizzle: rows of 32 bytes, 8-row groups 256 bytes apart
__device__ __forceinline__ unsigned long long smem_desc_sw32(uint32_t addr)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFF);
    d |= (unsigned long long)(16 >> 4) << 16;
    d |= (unsigned long long)(256 >> 4) << 32;
    d |= 1ull << 46;
    d |= 6ull << 61;                       // 32-byte swizzle
    return d;
}

// kind::f16, D = F32, A = B = BF16, both K-major, M = 128, N = 64 .. 256
__host__ __device__ constexpr uint32_t oz_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, unsigned long long a, unsigned long long b, uint32_t idesc,
                                         uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// float-pair accumulation (TwoSum, then renormalisation)
__device__ __forceinline__ void df_add(float &hi, float &lo, float x)
{
    float s = __fadd_rn(hi, x);
    float bp = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    float l = __fadd_rn(lo, e);
    float s2 = __fadd_rn(s, l);              // Fast2Sum renormalisation (|s| >= |l|)
    lo = __fsub_rn(l, __fsub_rn(s2, s));
    hi = s2;
}

// f 2^E as a double from the bit fields (exact); false when f is not a normal
// float or the result leaves the normal double range
__device__ __forceinline__ bool f2d_scaled(float f, int E, double &out)
{
    const uint32_t u = __float_as_uint(f);
    if ((u & 0x7FFFFFFFu) == 0) { out = 0.0; return true; }
    const int ef = (int)((u >> 23) & 0xFF);
    if (ef == 0 || ef == 255) return false;
    const int ed = ef - 127 + 1023 + E;
    if (ed < 1 || ed > 2046) return false;
    const unsigned long long b = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)ed << 52) |
                                 ((unsigned long long)(u & 0x7FFFFFu) << 29);
    out = __longlong_as_double((long long)b);
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(const __grid_constant__ OzArgs g)
{
    // grouped tile order: runs of OZ_GROUP_M row blocks sweep the column blocks
    // together, so the CTAs resident at one time share their A and B tiles in L2
    const int mt = (g.m + OZ_BM - 1) / OZ_BM, nt = (g.n + OZ_BN - 1) / OZ_BN;
    const int pid = blockIdx.x, per_group = OZ_GROUP_M * nt;
    const int first_m = (pid / per_group) * OZ_GROUP_M, gm = min(mt - first_m, OZ_GROUP_M);
    const int tm = first_m + (pid % per_group) % gm, tn = (pid % per_group) / gm;
    const int i0 = tm * OZ_BM, j0 = tn * OZ_BN, z = blockIdx.z;
    if (i0 >= g.m || j0 >= g.n) return;
    if (g.lowerC && j0 > i0 + OZ_BM - 1) return;

    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned long long *bars = (unsigned long long *)(smem + OZ_STAGES * OZ_STAGE_BYTES);
    // bars[0..ST): full, [ST..2ST): empty, [2ST]: chunk done (MMA -> flush), [2ST+1]: accumulators free
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * OZ_STAGES + 4);
    __shared__ int s_abort, s_issued;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    int kbeg = 0, kend = g.k;
    if (g.triA == TRI_LOWER) kend = min(kend, i0 + OZ_BM);
    if (g.triA == TRI_UPPER) kbeg = max(kbeg, i0);
    if (g.triB == TRI_LOWER) kbeg = max(kbeg, j0);
    if (g.triB == TRI_UPPER) kend = min(kend, j0 + OZ_BN);
    const int kb0 = kbeg / OZ_BK;
    const int nkb = (kend > kbeg) ? (kend + OZ_BK - 1) / OZ_BK - kb0 : 0;
    const int nchunks = (nkb + OZ_CHUNK_STAGES - 1) / OZ_CHUNK_STAGES;
    const uint32_t b_full = smem_u32(&bars[0]), b_empty = smem_u32(&bars[OZ_STAGES]);
    const uint32_t b_done = smem_u32(&bars[2 * OZ_STAGES]), b_free = smem_u32(&bars[2 * OZ_STAGES + 1]);
    const uint32_t b_drain = smem_u32(&bars[2 * OZ_STAGES + 2]);   // MMA drain after an abort

    if (tid == 0) {
        s_abort = 0;
        s_issued = 0;
        for (int s = 0; s < OZ_STAGES; ++s) {
            mbar_init(b_full + 8 * s, 1);
            mbar_init(b_empty + 8 * s, 1);
        }
        mbar_init(b_done, 1);
        mbar_init(b_free, 32 * OZ_FLUSH_WARPS);
        mbar_init(b_drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(OZ_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == OZ_PRODUCER_WARP) {
        // ---------------- bulk-copy producer ----------------
        if (lane == 0) {
            const __nv_bfloat16 *srca = g.sa + (((long long)z * (g.m_pad / OZ_BM) + tm) * g.kblocks + kb0) *
                                                   (OZ_S * OZ_BM * OZ_BK);
            const __nv_bfloat16 *srcb = g.sb + (((long long)z * (g.n_pad / OZ_BN) + tn) * g.kblocks + kb0) *
                                                   (OZ_S * OZ_BN * OZ_BK);
            for (int q = 0; q < nkb; ++q) {
                const int s = q % OZ_STAGES;
                if (q >= OZ_STAGES &&
                    !mbar_wait(b_empty + 8 * s, (uint32_t)(((q / OZ_STAGES) - 1) & 1), g.wait_limit)) {
                    s_abort = 1; atomicExch(g.err, 1); break;
                }
                if (s_abort) break;
                const uint32_t st = smem_u32(smem + s * OZ_STAGE_BYTES);
                mbar_expect_tx(b_full + 8 * s, OZ_STAGE_BYTES);
                bulk_load(st, srca + (long long)q * (OZ_S * OZ_BM * OZ_BK), OZ_S * OZ_A_TILE, b_full + 8 * s);
                bulk_load(st + OZ_S * OZ_A_TILE, srcb + (long long)q * (OZ_S * OZ_BN * OZ_BK), OZ_S * OZ_B_TILE,
                          b_full + 8 * s);
                s_issued = q + 1;
            }
        }
    } else if (warp == OZ_MMA_WARP) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            for (int c = 0; c < nchunks && !s_abort; ++c) {
                if (c > 0 && !mbar_wait(b_free, (uint32_t)((c - 1) & 1), g.wait_limit)) {
                    s_abort = 1; atomicExch(g.err, 2); break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int q0 = c * OZ_CHUNK_STAGES, q1 = min(nkb, q0 + OZ_CHUNK_STAGES);
                bool ok = true;
                for (int q = q0; q < q1; ++q) {
                    const int s = q % OZ_STAGES;
                    if (!mbar_wait(b_full + 8 * s, (uint32_t)((q / OZ_STAGES) & 1), g.wait_limit)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t st = smem_u32(smem + s * OZ_STAGE_BYTES);
                    // A slice a against B slices b = 1 .. S+1-a stacked along N: the product
                    // (a, b) belongs to level a+b-2, whose accumulator starts at column
                    // 64 (a+b-2), so slices b..b+3 form one N <= 256 MMA into consecutive levels.
#pragma unroll
                    for (int a = 1; a <= OZ_S; ++a) {
                        const unsigned long long ad = smem_desc_sw32(st + (a - 1) * OZ_A_TILE);
                        const uint32_t acc = (q == q0 && a == 1) ? 0u : 1u;   // a = 1 reaches every level first
#pragma unroll
                        for (int b0 = 1; b0 <= OZ_S + 1 - a; b0 += 4) {
                            const int nb = min(4, OZ_S + 2 - a - b0);
                            const unsigned long long bd = smem_desc_sw32(st + OZ_S * OZ_A_TILE + (b0 - 1) * OZ_B_TILE);
                            mma_bf16(tmem + (uint32_t)((a + b0 - 2) * OZ_BN), ad, bd, oz_idesc(nb * OZ_BN), acc);
                        }
                    }
                    mma_commit(b_empty + 8 * s);
                }
                if (!ok) { s_abort = 1; atomicExch(g.err, 3); break; }
                mma_commit(b_done);
            }
            // Every MMA issued has retired before TMEM and the stages go away, whatever
            // the other roles did (a flush warp that gave up no longer waits for them).
            mma_commit(b_drain);
            mbar_wait(b_drain, 0u, OZ_WAIT_LIMIT);
        }
    } else {
        // ---------------- flush warps: lanes 32 (w % 4) .., columns c0 .. c0 + 15 ----------------
        const int quad = warp & 3, c0 = (warp >> 2) * OZ_FCOLS;
        float hi[OZ_FCOLS], lo[OZ_FCOLS];
#pragma unroll
        for (int q = 0; q < OZ_FCOLS; ++q) { hi[q] = 0.f; lo[q] = 0.f; }
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            if (!mbar_wait(b_done, (uint32_t)(c & 1), g.wait_limit)) { ok = false; atomicExch(g.err, 4); break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int L = 0; L < OZ_LEVELS; ++L) {
                const float sc = __int_as_float((127 - 7 * (L + 2)) << 23);   // 2^{-7(L+2)}
                uint32_t r[OZ_FCOLS];
                tmem_ld16_nowait(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(L * OZ_BN + c0), r);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < OZ_FCOLS; ++q) df_add(hi[q], lo[q], __fmul_rn(__uint_as_float(r[q]), sc));
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(b_free);
        }
        const int i = i0 + quad * 32 + lane;
        if (ok && !s_abort && i < g.m) {
            double *C = g.C + (long long)z * g.sC;
            const double *Cin = g.Cin ? g.Cin + (long long)z * g.sCin : nullptr;
            // exponents of all-zero rows / columns are very negative; their pairs are 0
            const int ei = max(g.ea[z * g.m_pad + i], -4000) + g.alpha_e;
            const double *eCin = Cin ? Cin + (long long)i * g.ldcin : nullptr;
            double *eC = C + (long long)i * g.ldc;
#pragma unroll
            for (int q = 0; q < OZ_FCOLS; ++q) {
                const int j = j0 + c0 + q;
                if (j >= g.n || (g.lowerC && j > i)) continue;
                const int E = ei + max(g.eb[z * g.n_pad + j], -4000);
                double dh, dl, v;
                if (f2d_scaled(hi[q], E, dh) && f2d_scaled(lo[q], E, dl)) {
                    v = dh + dl;                  // a power-of-two alpha is folded into E and the sign
                    if (g.alpha_neg) v = -v;
                    if (!g.alpha_e_valid) v *= g.alpha;
                } else {
                    v = ldexp((double)hi[q] + (double)lo[q], E - g.alpha_e) * g.alpha;
                }
                if (g.beta != 0.0) v = fma(g.beta, eCin[j], v);
                eC[j] = v;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (s_abort && tid == 32 * OZ_PRODUCER_WARP) {   // producer lane: let the last copies issued land
        for (int q = max(0, s_issued - OZ_STAGES); q < s_issued; ++q)
            mbar_wait(b_full + 8 * (q % OZ_STAGES), (uint32_t)((q / OZ_STAGES) & 1), OZ_WAIT_LIMIT);
    }
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS));
}

// ---------------------------------------------------------------------------
// operand preparation
//   logical operand X(r, p), r < rows, p < k:  trans ? src[p][r] : src[r][p],
//   structural zeros (tri, in (r, p) terms) forced to 0, optional ks[p] scaling
// ---------------------------------------------------------------------------
__device__ __forceinline__ double oz_load(const double *X, long long ld, int trans, int rows, int k, int tri,
                                          const double *ks, int r, int p)
{
    if (r >= rows || p >= k) return 0.0;
    if (tri == TRI_LOWER && p > r) return 0.0;
    if (tri == TRI_UPPER && p < r) return 0.0;
    double v = trans ? X[(long long)p * ld + r] : X[(long long)r * ld + p];
    if (ks) v *= ks[p];
    return v;
}

// frexp exponent of v (v = f 2^e, 0.5 <= |f| < 1) from the IEEE-754 fields;
// a very small value for zero
__device__ __forceinline__ int oz_frexp_exp(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int bexp = (int)((b >> 52) & 0x7FF);
    const unsigned long long m = b & ((1ull << 52) - 1);
    if (bexp != 0) return bexp - 1022;
    if (m == 0) return INT_MIN / 2;
    return -1010 - __clzll((long long)m);      // subnormal: leading bit of m at 63 - clz
}

// round(v 2^{56-e}) as an integer, for |v| < 2^e: |result| <= 2^56, error <= 1/2
__device__ __forceinline__ long long oz_fixed56(double v, int e)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    int bexp = (int)((b >> 52) & 0x7FF);
    unsigned long long m = b & ((1ull << 52) - 1);
    if (bexp == 0) { if (m == 0 || e < -1100) return 0; bexp = 1; }
    else m |= 1ull << 52;
    const int sh = (bexp - 1075) - e + 56;    // v = m 2^{bexp-1075};  m 2^sh < 2^56
    unsigned long long f;
    if (sh >= 0) f = m << sh;
    else if (sh > -64) f = (m >> (-sh)) + ((m >> (-sh - 1)) & 1ull);
    else f = 0;
    return (b >> 63) ? -(long long)f : (long long)f;
}

// float bit pattern of a small integer d (|d| <= 256) through the float 2^23 + 128: the
// integer add lands d in the last mantissa bits and one float subtraction (exact, Sterbenz)
// leaves float(d); its upper 16 bits are the BF16 pattern of d, exactly, since d has at most
// 9 significant bits.  Full-rate integer and FP32 instructions instead of two conversions.
__device__ __forceinline__ uint32_t oz_small_int_bits(int d)
{
    return __float_as_uint(__int_as_float(0x4B000080 + d) - 8388736.0f);
}

// the eight balanced base-128 digits of F (|F| <= 2^56) as float bit patterns, most
// significant first: d_8 .. d_2 in [-64, 63], the rest d_1 (|d_1| <= 128).  F = hi 2^28 + lo
// with lo in [0, 2^28): the four low digits come from lo in 32-bit arithmetic (leaving a carry
// of 0 or 1, added to hi), the other four from hi -- the same digits as extracting from F.
__device__ __forceinline__ void oz_digits(long long F, uint32_t *bits)
{
    int lo = (int)(F & 0x0FFFFFFFLL);
    int hi = (int)(F >> 28);
#pragma unroll
    for (int t = OZ_S; t >= OZ_S - 3; --t) {
        const int c = ((lo + 64) & 127) - 64;
        lo = (lo - c) >> 7;
        bits[t - 1] = oz_small_int_bits(c);
    }
    hi += lo;
#pragma unroll
    for (int t = OZ_S - 4; t >= 2; --t) {
        const int c = ((hi + 64) & 127) - 64;
        hi = (hi - c) >> 7;
        bits[t - 1] = oz_small_int_bits(c);
    }
    bits[0] = oz_small_int_bits(hi);
}

// One operand of the preparation passes: op(X) is rows x k (trans: op(X)[r][p] = X[p][r]),
// with structural zeros (tri), an optional inner scaling ks[p], rows padded to rows_pad.
struct OzOperand {
    const double *X; long long ld, sb; int trans, rows, tri; const double *ks;
    int rows_pad, tile_rows; int *e; __nv_bfloat16 *out;
};

// exponents e(r) with max_p |op(X)[r][p]| < 2^e of both operands in one launch; blocks
// [0, nA) serve A, the rest B.  Rows contiguous in memory (trans = 0): a block holds 8 warps,
// each one row over a 1024-column chunk (8 loads in flight per lane), a shuffle max and an
// atomicMax.  Transposed (trans = 1): a block covers 32 rows of op(X) (32 memory columns)
// over a 256-term chunk of p, its 8 warps each reading 32 p rows of 32 consecutive doubles,
// then a shared-memory max and one atomicMax per row.
__global__ void __launch_bounds__(256) oz_exp_kernel(OzOperand a, OzOperand b, int k, int nA)
{
    const bool isA = (int)blockIdx.x < nA;
    const OzOperand &o = isA ? a : b;
    const int blk = isA ? (int)blockIdx.x : (int)blockIdx.x - nA;
    const int z = blockIdx.z, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const double *X = o.X + (long long)z * o.sb;
    if (!o.trans) {
        const int kc = (k + 1023) / 1024;                  // chunks per row
        const int r = (blk / kc) * 8 + warp, p0 = (blk % kc) * 1024;
        if (r >= o.rows) return;
        int mx = INT_MIN / 2;
        for (int pp = p0; pp < p0 + 1024 && pp < k; pp += 256) {
#pragma unroll
            for (int t = 0; t < 8; ++t)
                mx = max(mx, oz_frexp_exp(oz_load(X, o.ld, 0, o.rows, k, o.tri, o.ks, r, pp + t * 32 + lane)));
        }
#pragma unroll
        for (int q = 16; q > 0; q >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, q));
        if (lane == 0 && mx > INT_MIN / 2) atomicMax(&o.e[z * o.rows_pad + r], mx);
    } else {
        __shared__ int red[8][33];
        const int kc = (k + 255) / 256;
        const int r0 = (blk / kc) * 32, p0 = (blk % kc) * 256;
        const int r = r0 + lane;
        int mx = INT_MIN / 2;
#pragma unroll 4
        for (int t = 0; t < 32; ++t) {
            const int pp = p0 + warp + 8 * t;
            mx = max(mx, oz_frexp_exp(oz_load(X, o.ld, 1, o.rows, k, o.tri, o.ks, r, pp)));
        }
        red[warp][lane] = mx;
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int w = 1; w < 8; ++w) mx = max(mx, red[w][lane]);
            if (r < o.rows && mx > INT_MIN / 2) atomicMax(&o.e[z * o.rows_pad + r], mx);
        }
    }
}

// number of blocks oz_exp_kernel uses for one operand
int oz_exp_blocks(const OzOperand &o, int k)
{
    if (!o.trans) return ((o.rows + 7) / 8) * ((k + 1023) / 1024);
    return ((o.rows + 31) / 32) * ((k + 255) / 256);
}

// eight BF16 slices in the tiled layout the GEMM streams: for row r of tile
// rr = r % tile_rows and column p (k block p / 16, kk = p % 16) of slice t the
// element sits in block ((z * rows_pad / tile_rows + r / tile_rows) * kblocks + p / 16)
// of 8 * tile_rows * 16 elements, at t * tile_rows * 16 + rr * 16 + kk with the
// 16-byte half of the 32-byte row flipped when bit 2 of rr is set (the 32-byte
// shared-memory swizzle the MMA descriptors expect).
// F = round(x 2^{56-e}) is cut into balanced base-128 digits d_8 .. d_2 in
// [-64, 63]; the rest is d_1, |d_1| <= 128; x 2^{-e} = sum_t d_t 2^{-7t} + O(2^-57).
// One CTA per 32 rows x 64 columns of op(X): the tile is read coalesced (along memory
// rows, transposing through shared memory when trans = 1), then each thread takes 8
// consecutive columns of one row -- half of a 16-column k block -- and writes each of
// its 8 slices as one 16-byte store; the 32 lanes of a warp cover 16 rows x both halves
// of one k block, i.e. 512 contiguous bytes per slice.
__global__ void __launch_bounds__(256) oz_slice_kernel(OzOperand a, OzOperand b, int k, int k_pad, int nA)
{
    __shared__ double T[32][65];               // T[row][column] of the tile
    const bool isA = (int)blockIdx.x < nA;
    const OzOperand &o = isA ? a : b;
    const int blk = isA ? (int)blockIdx.x : (int)blockIdx.x - nA;
    const int pt = (k_pad + 63) / 64;           // 64-column tiles per row band
    const int z = blockIdx.z, r0 = (blk / pt) * 32, p0 = (blk % pt) * 64;
    const int tid = threadIdx.x;
    const double *X = o.X + (long long)z * o.sb;
    const int trans = o.trans, rows = o.rows, tri = o.tri, rows_pad = o.rows_pad, tile_rows = o.tile_rows;
    const long long ld = o.ld;
    const double *ks = o.ks;
    const int *e = o.e;
    __nv_bfloat16 *out = o.out;
    if (trans) {   // memory rows are p: a warp reads 32 consecutive r of one p
        for (int it = 0; it < 8; ++it) {
            const int pl = it * 8 + (tid >> 5), rl = tid & 31;
            T[rl][pl] = oz_load(X, ld, 1, rows, k, tri, ks, r0 + rl, p0 + pl);
        }
    } else {       // memory rows are r: a warp reads 32 consecutive p of one r
        for (int it = 0; it < 8; ++it) {
            const int rl = it * 4 + (tid >> 6), pl = tid & 63;
            T[rl][pl] = oz_load(X, ld, 0, rows, k, tri, ks, r0 + rl, p0 + pl);
        }
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    const int rl = (warp & 1) * 16 + (lane >> 1);          // row within the tile
    const int kb = warp >> 1;                              // k block within the tile (0..3)
    const int half = lane & 1;                             // columns 8 half .. 8 half + 7 of the k block
    const int r = r0 + rl, pb = p0 + kb * 16 + half * 8;
    if (r >= rows_pad || pb >= k_pad) return;
    const int ex = (r < rows) ? e[z * rows_pad + r] : -4000;
    long long f[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) f[q] = (ex > -2000) ? oz_fixed56(T[rl][kb * 16 + half * 8 + q], ex) : 0;
    const int kblocks = k_pad / 16, tiles = rows_pad / tile_rows;
    const int rr = r % tile_rows;
    const long long oblk = ((long long)z * tiles + r / tile_rows) * kblocks + (pb >> 4);
    __nv_bfloat16 *dst = out + oblk * (OZ_S * tile_rows * 16) + rr * 16 + ((half ^ (rr >> 2)) & 1) * 8;
    const int sstride = tile_rows * 16;
    uint32_t w[OZ_S][4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        uint32_t ba[OZ_S], bb[OZ_S];
        oz_digits(f[q], ba);
        oz_digits(f[q + 1], bb);
#pragma unroll
        for (int t = 0; t < OZ_S; ++t) w[t][q >> 1] = __byte_perm(ba[t], bb[t], 0x7632);   // two upper halves
    }
#pragma unroll
    for (int t = 0; t < OZ_S; ++t)
        *reinterpret_cast<uint4 *>(dst + t * sstride) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

__global__ void fill_int_kernel(int *x, long long n, int v)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = v;
}

}  // namespace

size_t oz_gemm_workspace_bytes(const GemmArgs &g)
{
    const long long kp = (g.k + 15) / 16 * 16;
    const long long mp = (g.m + OZ_BM - 1) / OZ_BM * OZ_BM, np = (g.n + OZ_BN - 1) / OZ_BN * OZ_BN;
    return (size_t)(OZ_S * (mp + np) * kp * g.batch) * 2 + (size_t)(mp + np) * g.batch * sizeof(int) + 2048;
}

namespace {
struct OzLayout {
    int kp, mp, np;
    __nv_bfloat16 *sa, *sb;
    int *ea, *eb;
};
OzLayout oz_layout(const GemmArgs &g, void *ws)
{
    OzLayout L;
    L.kp = (g.k + 15) / 16 * 16;
    L.mp = (g.m + OZ_BM - 1) / OZ_BM * OZ_BM; L.np = (g.n + OZ_BN - 1) / OZ_BN * OZ_BN;
    unsigned char *base = (unsigned char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    L.sa = (__nv_bfloat16 *)base;
    L.sb = L.sa + (size_t)OZ_S * L.mp * L.kp * g.batch;
    L.ea = (int *)(L.sb + (size_t)OZ_S * L.np * L.kp * g.batch);
    L.eb = L.ea + (size_t)L.mp * g.batch;
    return L;
}
}  // namespace

// operand preparation: exponents and pre-tiled slices of op(A) and op(B) into ws
int oz_gemm_prepare(const GemmArgs &g, void *ws, cudaStream_t s)
{
    if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return 0;
    const OzLayout L = oz_layout(g, ws);
    const int triB = g.triB == TRI_LOWER ? TRI_UPPER : (g.triB == TRI_UPPER ? TRI_LOWER : TRI_NONE);
    fill_int_kernel<<<64, 256, 0, s>>>(L.ea, (long long)(L.mp + L.np) * g.batch, INT_MIN / 2); count_launch();
    // op(A) rows are memory rows unless A is transposed; op(B) columns are memory rows when B is transposed
    OzOperand oa{(const double *)g.A, g.lda, g.sA, g.ta, g.m, g.triA, (const double *)g.kscale, L.mp, OZ_BM, L.ea, L.sa};
    OzOperand ob{(const double *)g.B, g.ldb, g.sB, g.tb ? 0 : 1, g.n, triB, nullptr, L.np, OZ_BN, L.eb, L.sb};
    {
        const int nA = oz_exp_blocks(oa, g.k), nB = oz_exp_blocks(ob, g.k);
        oz_exp_kernel<<<dim3(nA + nB, 1, g.batch), 256, 0, s>>>(oa, ob, g.k, nA); count_launch();
    }
    {
        const int pt = (L.kp + 63) / 64;
        const int nA = pt * (L.mp / 32), nB = pt * (L.np / 32);
        oz_slice_kernel<<<dim3(nA + nB, 1, g.batch), 256, 0, s>>>(oa, ob, g.k, L.kp, nA); count_launch();
    }
    return 0;
}

// the tensor-core product on operands prepared by oz_gemm_prepare(g, ws)
int oz_gemm_run(const GemmArgs &g, void *ws, int *err, cudaStream_t s)
{
    if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return 0;
    if (!ensure_dynamic_smem((const void *)oz_gemm_kernel, OZ_SMEM_BYTES)) return -2;
    const OzLayout L = oz_layout(g, ws);
    OzArgs a;
    a.sa = L.sa; a.sb = L.sb; a.kblocks = L.kp / 16;
    a.m = g.m; a.n = g.n; a.k = g.k; a.batch = g.batch; a.m_pad = L.mp; a.n_pad = L.np;
    a.triA = g.triA; a.triB = g.triB; a.lowerC = g.lowerC;
    a.ea = L.ea; a.eb = L.eb;
    a.C = (double *)g.C; a.ldc = g.ldc; a.sC = g.sC;
    a.Cin = (const double *)g.Cin; a.ldcin = g.ldcin; a.sCin = g.sCin;
    a.alpha = g.alpha; a.beta = g.beta; a.err = err;
    a.wait_limit = g.wait_limit > 0 ? (unsigned long long)g.wait_limit : OZ_WAIT_LIMIT;
    {
        int ex = 0;
        const double fr = std::frexp(std::fabs(g.alpha), &ex);
        a.alpha_e_valid = (fr == 0.5) ? 1 : 0;            // |alpha| = 2^(ex-1)
        a.alpha_e = a.alpha_e_valid ? ex - 1 : 0;
        a.alpha_neg = (a.alpha_e_valid && g.alpha < 0) ? 1 : 0;
    }
    dim3 grid(((g.n + OZ_BN - 1) / OZ_BN) * ((g.m + OZ_BM - 1) / OZ_BM), 1, g.batch);
    oz_gemm_kernel<<<grid, OZ_THREADS, OZ_SMEM_BYTES, s>>>(a); count_launch();
    return 0;
}

int oz_gemm_launch(const GemmArgs &g, void *ws, int *err, cudaStream_t s)
{
    int st = oz_gemm_prepare(g, ws, s);
    return st ? st : oz_gemm_run(g, ws, err, s);
}

}  // namespace pssd
