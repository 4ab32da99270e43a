// FP32-accurate GEMM on the 5th-generation tensor cores of sm_103a (tcgen05).
//
//   C = alpha * op(A) * diag(kscale) * op(B) + beta * Cin        (FP32 data)
//
// with the same operand conventions as gemm_kernel (triangular operands,
// lower-only output, batch).  Each FP32 operand x is split once, in an HBM
// pass that also applies the triangular masks, the inner scaling and the
// transposition to K-major order, into x = hi + lo with hi = tf32(x) and
// lo = x - hi; the product is accumulated in FP32 in tensor memory as
//     A_lo B_hi + A_hi B_lo + A_hi B_hi      (3xTF32, ~FP32 accuracy).
//
// Kernel layout (one CTA of 10 warps per 128 x 256 output tile):
//   * the split pass writes, for every (row tile, 16-term k block), the hi
//     and lo parts as one contiguous block already in the 64-byte-swizzled
//     order the MMA descriptors read (A: 2 x 128 rows x 64 bytes = 16 KB,
//     B: 2 x 256 rows x 64 bytes = 32 KB);
//   * warp 8 streams one k block per stage with two cp.async.bulk copies into
//     a 4-stage ring of 48 KB with full/empty mbarriers;
//   * warp 9 issues per stage 2 (K = 8) x 3 tcgen05.mma kind::tf32 (M = 128,
//     N = 256) into one FP32 accumulator of 256 TMEM columns and frees each
//     stage with tcgen05.commit;
//   * warps 0-7 wait for the final commit and write C (warp w: TMEM lanes
//     32 (w % 4) .., i.e. tile rows, and columns 128 (w / 4) ..).
// Every pipeline mbarrier wait is bounded by the caller's limit: on timeout the
// kernel sets *err, skips the remaining work, waits (under a fixed, longer
// bound) for its own bulk copies and MMAs in flight, frees its TMEM and returns.
#include <cuda_runtime.h>

#include "pssd_internal.h"

namespace pssd {

namespace {

constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 16;    // BK in FP32 elements = 64 bytes per row
constexpr int TC_STAGES = 4;
constexpr int TC_A_BYTES = 2 * TC_BM * TC_BK * 4;      // hi + lo, 16 KB
constexpr int TC_B_BYTES = 2 * TC_BN * TC_BK * 4;      // hi + lo, 32 KB
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr int TC_SMEM_BYTES = TC_STAGES * TC_STAGE_BYTES + 1024 /* alignment */ + 256 /* barriers */;
constexpr unsigned long long TC_WAIT_LIMIT = 1ull << 26;   // default pipeline bound and the drain bound
constexpr int TC_EPI_WARPS = 8;                        // warp w: lanes 32 (w % 4) .., columns 128 (w / 4) ..
constexpr int TC_ECOLS = TC_BN / (TC_EPI_WARPS / 4);
constexpr int TC_PRODUCER_WARP = TC_EPI_WARPS, TC_MMA_WARP = TC_EPI_WARPS + 1;
constexpr int TC_THREADS = 32 * (TC_EPI_WARPS + 2);
constexpr int TC_GROUP_M = 8;                          // row blocks per group of the tile order
constexpr int TC_TMEM_COLS = TC_BN;

struct TcArgs {
    const float *a, *b;                        // tiled split operands (see the split kernel)
    int kblocks;                               // k_pad / 16
    int m, n, k, batch;
    int m_pad, n_pad;
    int triA, triB, lowerC;
    float *C; long long ldc, sC;
    const float *Cin; long long ldcin, sCin;
    float alpha, beta;
    int *err;
    unsigned long long wait_limit;             // polls per pipeline wait before giving up
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bounded wait for the phase with the given parity; returns false on timeout
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

// shared-memory matrix descriptor: K-major operand, 64-byte swizzle, 8-row
// groups 512 bytes apart (SBO), version 1 (sm_100 family)
__device__ __forceinline__ unsigned long long smem_desc(uint32_t addr)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFF);          // start address
    d |= (unsigned long long)(16 >> 4) << 16;                  // leading byte offset (unused, swizzled K-major)
    d |= (unsigned long long)(512 >> 4) << 32;                 // stride byte offset
    d |= 1ull << 46;                                           // descriptor version
    d |= 4ull << 61;                                           // 64-byte swizzle
    return d;
}

// instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 256
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(TC_BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, unsigned long long a, unsigned long long b, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const __grid_constant__ TcArgs g)
{
    // grouped tile order: runs of TC_GROUP_M row blocks sweep the column blocks together
    const int mt = (g.m + TC_BM - 1) / TC_BM, nt = (g.n + TC_BN - 1) / TC_BN;
    const int pid = blockIdx.x, per_group = TC_GROUP_M * nt;
    const int first_m = (pid / per_group) * TC_GROUP_M, gm = min(mt - first_m, TC_GROUP_M);
    const int tm = first_m + (pid % per_group) % gm, tn = (pid % per_group) / gm;
    const int i0 = tm * TC_BM, j0 = tn * TC_BN, z = blockIdx.z;
    if (i0 >= g.m || j0 >= g.n) return;
    if (g.lowerC && j0 > i0 + TC_BM - 1) return;

    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned long long *bars = (unsigned long long *)(smem + TC_STAGES * TC_STAGE_BYTES);
    // bars[0..ST): full, [ST..2ST): empty, [2ST]: accumulator done
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * TC_STAGES + 2);
    __shared__ int s_abort, s_issued;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // k range that can contribute to this tile (structural zeros skipped)
    int kbeg = 0, kend = g.k;
    if (g.triA == TRI_LOWER) kend = min(kend, i0 + TC_BM);
    if (g.triA == TRI_UPPER) kbeg = max(kbeg, i0);
    if (g.triB == TRI_LOWER) kbeg = max(kbeg, j0);
    if (g.triB == TRI_UPPER) kend = min(kend, j0 + TC_BN);
    const int kb0 = kbeg / TC_BK;
    const int nkb = (kend > kbeg) ? (kend + TC_BK - 1) / TC_BK - kb0 : 0;
    const uint32_t b_full = smem_u32(&bars[0]), b_empty = smem_u32(&bars[TC_STAGES]);
    const uint32_t b_done = smem_u32(&bars[2 * TC_STAGES]);
    const uint32_t b_drain = smem_u32(&bars[2 * TC_STAGES + 1]);   // MMA drain after an abort

    if (tid == 0) {
        s_abort = 0;
        s_issued = 0;
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(b_full + 8 * s, 1);
            mbar_init(b_empty + 8 * s, 1);
        }
        mbar_init(b_done, 1);
        mbar_init(b_drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == TC_PRODUCER_WARP) {
        // ---------------- bulk-copy producer ----------------
        if (lane == 0) {
            const float *srca = g.a + (((long long)z * (g.m_pad / TC_BM) + tm) * g.kblocks + kb0) * (TC_A_BYTES / 4);
            const float *srcb = g.b + (((long long)z * (g.n_pad / TC_BN) + tn) * g.kblocks + kb0) * (TC_B_BYTES / 4);
            for (int q = 0; q < nkb; ++q) {
                const int s = q % TC_STAGES;
                if (q >= TC_STAGES && !mbar_wait(b_empty + 8 * s, (uint32_t)(((q / TC_STAGES) - 1) & 1), g.wait_limit)) {
                    s_abort = 1; atomicExch(g.err, 1); break;
                }
                if (s_abort) break;
                const uint32_t st = smem_u32(smem + s * TC_STAGE_BYTES);
                mbar_expect_tx(b_full + 8 * s, TC_STAGE_BYTES);
                bulk_load(st, srca + (long long)q * (TC_A_BYTES / 4), TC_A_BYTES, b_full + 8 * s);
                bulk_load(st + TC_A_BYTES, srcb + (long long)q * (TC_B_BYTES / 4), TC_B_BYTES, b_full + 8 * s);
                s_issued = q + 1;
            }
        }
    } else if (warp == TC_MMA_WARP) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            bool ok = true;
            for (int q = 0; q < nkb; ++q) {
                const int s = q % TC_STAGES;
                if (!mbar_wait(b_full + 8 * s, (uint32_t)((q / TC_STAGES) & 1), g.wait_limit)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t st = smem_u32(smem + s * TC_STAGE_BYTES);
                const uint32_t ah = st, al = st + TC_A_BYTES / 2;
                const uint32_t bh = st + TC_A_BYTES, bl = st + TC_A_BYTES + TC_B_BYTES / 2;
#pragma unroll
                for (int kk = 0; kk < TC_BK / 8; ++kk) {           // K = 8 TF32 = 32 bytes per instruction
                    const uint32_t off = kk * 32;
                    mma_tf32(tmem, smem_desc(al + off), smem_desc(bh + off), (q > 0 || kk > 0) ? 1u : 0u);
                    mma_tf32(tmem, smem_desc(ah + off), smem_desc(bl + off), 1u);
                    mma_tf32(tmem, smem_desc(ah + off), smem_desc(bh + off), 1u);
                }
                mma_commit(b_empty + 8 * s);                   // stage s is free when these MMAs retire
            }
            if (nkb > 0) {
                if (ok) mma_commit(b_done);
                else { s_abort = 1; atomicExch(g.err, 2); }
            }
            // Every MMA issued has retired before TMEM and the stages go away, whatever
            // the other roles did (an epilogue warp that gave up no longer waits for them).
            mma_commit(b_drain);
            mbar_wait(b_drain, 0u, TC_WAIT_LIMIT);
        }
    } else {
        // ---------------- epilogue warps ----------------
        const int quad = warp & 3, c0 = (warp >> 2) * TC_ECOLS;
        bool have = nkb > 0;
        if (have && !mbar_wait(b_done, 0u, g.wait_limit)) { have = false; atomicExch(g.err, 3); }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int i = i0 + quad * 32 + lane;
        float *C = g.C + (long long)z * g.sC + (long long)i * g.ldc;
        const float *Cin = g.Cin ? g.Cin + (long long)z * g.sCin + (long long)i * g.ldcin : nullptr;
        {   // nkb == 0: the product is zero and C = beta Cin; a failed wait writes nothing
#pragma unroll 1
            for (int cc = 0; cc < TC_ECOLS; cc += 16) {
                float v[16];
                if (have) {
                    uint32_t r[16];
                    const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c0 + cc);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                          "=r"(r[15])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = 0.f;
                }
                if (i < g.m && (have || nkb == 0)) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int j = j0 + c0 + cc + q;
                        if (j >= g.n || (g.lowerC && j > i)) continue;
                        float o = g.alpha * v[q];
                        if (g.beta != 0.f) o += g.beta * Cin[j];
                        C[j] = o;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (s_abort && tid == 32 * TC_PRODUCER_WARP) {   // producer lane: let the last copies issued land
        for (int q = max(0, s_issued - TC_STAGES); q < s_issued; ++q)
            mbar_wait(b_full + 8 * (q % TC_STAGES), (uint32_t)((q / TC_STAGES) & 1), TC_WAIT_LIMIT);
    }
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// ---------------------------------------------------------------------------
// operand preparation: masked, scaled, K-major, split into tf32 hi + lo
//   logical operand row r < rows, column p < k:
//   src = trans ? X[z][p][r] : X[z][r][p]; structural zeros (tri) forced to 0
// tri: relation of (r, p) that is structurally nonzero:
//   TRI_LOWER: p <= r,  TRI_UPPER: p >= r  (for A: op(A)[i][p]);
//   for B the caller passes the relation in terms of (j, p) of op(B)[p][j]:
//   op(B) lower (p >= j) -> TRI_UPPER here, op(B) upper (p <= j) -> TRI_LOWER
// Output, tiled for the GEMM's bulk copies: block
//   ((z * rows_pad / tile_rows + r / tile_rows) * (k_pad / 16) + p / 16)
// of 2 * tile_rows * 16 floats holds the hi part (rows rr = r % tile_rows,
// 16 floats each) then the lo part; inside a 64-byte row the 16-byte chunk
// (p % 16) / 4 is stored at chunk ((p % 16) / 4) ^ ((rr / 2) % 4) (the
// 64-byte shared-memory swizzle the MMA descriptors expect).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tf32_split_kernel(const float *X, long long ld, long long sb, int trans,
                                                         int rows, int k, int k_pad, int rows_pad, int tile_rows,
                                                         int tri, const float *ks, float *out)
{
    __shared__ float T[32][33];
    const int z = blockIdx.z;
    const int r0 = blockIdx.y * 32, p0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    X += (long long)z * sb;
    // load the 32 x 32 block in the orientation that is contiguous in memory
    for (int yy = ty; yy < 32; yy += 8) {
        float v = 0.f;
        if (trans) {   // memory rows are p, contiguous r
            int p = p0 + yy, r = r0 + tx;
            if (p < k && r < rows) v = X[(long long)p * ld + r];
            T[tx][yy] = v;   // T[r][p]
        } else {
            int r = r0 + yy, p = p0 + tx;
            if (r < rows && p < k) v = X[(long long)r * ld + p];
            T[yy][tx] = v;
        }
    }
    __syncthreads();
    // each thread: one row of the tile and four consecutive k -- one 16-byte chunk of the
    // swizzled layout -- written as one 16-byte store for the hi parts and one for the lo parts
    const int kblocks = k_pad / 16, tiles = rows_pad / tile_rows;
    const int yy = threadIdx.x >> 3, q4 = (threadIdx.x & 7) * 4;
    const int r = r0 + yy, pq = p0 + q4;
    if (r >= rows_pad || pq >= k_pad) return;      // k_pad is a multiple of 16: the four p all fit
    float hv[4], lv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int p = pq + t;
        float v = (r < rows && p < k) ? T[yy][q4 + t] : 0.f;
        if (tri == TRI_LOWER && p > r) v = 0.f;
        if (tri == TRI_UPPER && p < r) v = 0.f;
        if (ks && p < k) v *= ks[p];
        uint32_t u;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
        hv[t] = __uint_as_float(u);
        lv[t] = v - hv[t];
    }
    const int rr = r % tile_rows, kk = pq & 15;
    const long long blk = ((long long)z * tiles + r / tile_rows) * kblocks + (pq >> 4);
    float *o = out + blk * (2 * tile_rows * 16) + rr * 16 + ((((kk >> 2) ^ (rr >> 1)) & 3) << 2);
    *reinterpret_cast<float4 *>(o) = make_float4(hv[0], hv[1], hv[2], hv[3]);
    *reinterpret_cast<float4 *>(o + tile_rows * 16) = make_float4(lv[0], lv[1], lv[2], lv[3]);
}

}  // namespace

size_t tc_gemm_workspace_bytes(const GemmArgs &g)
{
    const long long kp = (g.k + 15) / 16 * 16;
    const long long mp = (g.m + TC_BM - 1) / TC_BM * TC_BM, np = (g.n + TC_BN - 1) / TC_BN * TC_BN;
    return (size_t)(2 * (mp + np) * kp * g.batch) * sizeof(float) + 1024;
}

namespace {
void tc_layout(const GemmArgs &g, void *ws, int &kp, int &mp, int &np, float *&ta, float *&tb)
{
    kp = (g.k + 15) / 16 * 16;
    mp = (g.m + TC_BM - 1) / TC_BM * TC_BM; np = (g.n + TC_BN - 1) / TC_BN * TC_BN;
    float *base = (float *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    ta = base; tb = ta + (size_t)2 * mp * kp * g.batch;
}
}  // namespace

// operand preparation: masked, scaled, K-major tf32 hi/lo tiles of op(A), op(B) into ws
int tc_gemm_prepare(const GemmArgs &g, void *ws, cudaStream_t s)
{
    if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return 0;
    int kp, mp, np; float *ta, *tb;
    tc_layout(g, ws, kp, mp, np, ta, tb);
    {   // A: rows i of op(A), K-major
        dim3 grid((kp + 31) / 32, (mp + 31) / 32, g.batch);
        tf32_split_kernel<<<grid, 256, 0, s>>>((const float *)g.A, g.lda, g.sA, g.ta, g.m, g.k, kp, mp, TC_BM,
                                               g.triA, (const float *)g.kscale, ta); count_launch();
    }
    {   // B: rows j of op(B)^T, K-major (op(B)[p][j] = B[p][j] or B[j][p])
        int triB = g.triB == TRI_LOWER ? TRI_UPPER : (g.triB == TRI_UPPER ? TRI_LOWER : TRI_NONE);
        dim3 grid((kp + 31) / 32, (np + 31) / 32, g.batch);
        tf32_split_kernel<<<grid, 256, 0, s>>>((const float *)g.B, g.ldb, g.sB, g.tb ? 0 : 1, g.n, g.k, kp, np, TC_BN,
                                               triB, nullptr, tb); count_launch();
    }
    return 0;
}

// the tensor-core product on operands prepared by tc_gemm_prepare(g, ws); err: device int (0 on entry)
int tc_gemm_run(const GemmArgs &g, void *ws, int *err, cudaStream_t s)
{
    if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return 0;
    if (!ensure_dynamic_smem((const void *)tc_gemm_kernel, TC_SMEM_BYTES)) return -2;
    int kp, mp, np; float *ta, *tb;
    tc_layout(g, ws, kp, mp, np, ta, tb);
    TcArgs a;
    a.a = ta; a.b = tb; a.kblocks = kp / 16;
    a.m = g.m; a.n = g.n; a.k = g.k; a.batch = g.batch; a.m_pad = mp; a.n_pad = np;
    a.triA = g.triA; a.triB = g.triB; a.lowerC = g.lowerC;
    a.C = (float *)g.C; a.ldc = g.ldc; a.sC = g.sC;
    a.Cin = (const float *)g.Cin; a.ldcin = g.ldcin; a.sCin = g.sCin;
    a.alpha = (float)g.alpha; a.beta = (float)g.beta;
    a.err = err;
    a.wait_limit = g.wait_limit > 0 ? (unsigned long long)g.wait_limit : TC_WAIT_LIMIT;
    dim3 grid(((g.n + TC_BN - 1) / TC_BN) * ((g.m + TC_BM - 1) / TC_BM), 1, g.batch);
    tc_gemm_kernel<<<grid, TC_THREADS, TC_SMEM_BYTES, s>>>(a); count_launch();
    return 0;
}

// ws: device workspace of tc_gemm_workspace_bytes(g) bytes; err: device int (0 on entry)
int tc_gemm_launch(const GemmArgs &g, void *ws, int *err, cudaStream_t s)
{
    int st = tc_gemm_prepare(g, ws, s);
    return st ? st : tc_gemm_run(g, ws, err, s);
}

}  // namespace pssd
