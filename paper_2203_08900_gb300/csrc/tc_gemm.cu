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
// Kernel layout (one CTA of 128 threads per 128 x 128 output tile):
//   * operand tiles of 128 rows x 32 K (128 bytes per row) are fetched by TMA
//     (cp.async.bulk.tensor, 128-byte swizzle) into a 3-stage ring of
//     4 x 16 KB buffers (A_hi, A_lo, B_hi, B_lo) with an mbarrier per stage;
//   * thread 0 issues the TMA loads and the tcgen05.mma instructions
//     (kind::tf32, M = N = 128, K = 8) and frees a stage with tcgen05.commit;
//   * the 128 x 128 FP32 accumulator lives in 128 TMEM columns; the epilogue
//     reads it with tcgen05.ld (each warp its 32 lanes = 32 rows).
// Every mbarrier wait is bounded: on timeout the kernel sets *err, skips the
// remaining work, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "pssd_internal.h"

namespace pssd {

namespace {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 32;    // BK in FP32 elements = 128 bytes
constexpr int TC_STAGES = 3;
constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 4;       // 16 KB per operand tile
constexpr int TC_STAGE_BYTES = 4 * TC_TILE_BYTES;      // A_hi, A_lo, B_hi, B_lo
constexpr int TC_SMEM_BYTES = TC_STAGES * TC_STAGE_BYTES + 1024 /* alignment */ + 256 /* barriers */;
constexpr unsigned long long TC_WAIT_LIMIT = 1ull << 26;

struct TcArgs {
    CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo;   // K-major operands, rows stacked over the batch
    int m, n, k, batch;
    int m_pad, n_pad;                          // rows per batch entry in the A / B tensors
    int triA, triB, lowerC;
    float *C; long long ldc, sC;
    const float *Cin; long long ldcin, sCin;
    float alpha, beta;
    int *err;
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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (unsigned long long it = 0; it < TC_WAIT_LIMIT; ++it) {
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

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (SBO), version 1 (sm_100 family)
__device__ __forceinline__ unsigned long long smem_desc(uint32_t addr)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFF);          // start address
    d |= (unsigned long long)(16 >> 4) << 16;                  // leading byte offset (unused for SW128 K-major)
    d |= (unsigned long long)(1024 >> 4) << 32;                // stride byte offset
    d |= 1ull << 46;                                           // descriptor version
    d |= 2ull << 61;                                           // 128-byte swizzle
    return d;
}

// instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, N = M = 128
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

__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ TcArgs g)
{
    const int i0 = blockIdx.y * TC_BM, j0 = blockIdx.x * TC_BN, z = blockIdx.z;
    if (i0 >= g.m || j0 >= g.n) return;
    if (g.lowerC && j0 > i0 + TC_BM - 1) return;

    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned long long *bars = (unsigned long long *)(smem + TC_STAGES * TC_STAGE_BYTES);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * TC_STAGES + 2);
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // k range that can contribute to this tile (structural zeros skipped)
    int kbeg = 0, kend = g.k;
    if (g.triA == TRI_LOWER) kend = min(kend, i0 + TC_BM);
    if (g.triA == TRI_UPPER) kbeg = max(kbeg, i0);
    if (g.triB == TRI_LOWER) kbeg = max(kbeg, j0);
    if (g.triB == TRI_UPPER) kend = min(kend, j0 + TC_BN);
    const int kb0 = kbeg / TC_BK;
    const int nkb = (kend > kbeg) ? (kend + TC_BK - 1) / TC_BK - kb0 : 0;

    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(smem_u32(&bars[s]), 1);                   // full[s]
            mbar_init(smem_u32(&bars[TC_STAGES + s]), 1);       // empty[s]
        }
        mbar_init(smem_u32(&bars[2 * TC_STAGES]), 1);           // done
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (tid == 0 && nkb > 0) {
        const int ya = z * g.m_pad + i0, yb = z * g.n_pad + j0;
        auto issue = [&](int q) {   // TMA for k-block q into stage q % STAGES
            const int s = q % TC_STAGES;
            const uint32_t st = smem_u32(smem + s * TC_STAGE_BYTES);
            const uint32_t full = smem_u32(&bars[s]);
            const int x = (kb0 + q) * TC_BK;
            mbar_expect_tx(full, TC_STAGE_BYTES);
            tma_load_2d(st + 0 * TC_TILE_BYTES, &g.ta_hi, x, ya, full);
            tma_load_2d(st + 1 * TC_TILE_BYTES, &g.ta_lo, x, ya, full);
            tma_load_2d(st + 2 * TC_TILE_BYTES, &g.tb_hi, x, yb, full);
            tma_load_2d(st + 3 * TC_TILE_BYTES, &g.tb_lo, x, yb, full);
        };
        int issued = 0;
        for (; issued < nkb && issued < TC_STAGES; ++issued) issue(issued);
        bool ok = true;
        for (int q = 0; q < nkb && ok; ++q) {
            const int s = q % TC_STAGES;
            if (!mbar_wait(smem_u32(&bars[s]), (uint32_t)((q / TC_STAGES) & 1))) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t st = smem_u32(smem + s * TC_STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < TC_BK / 8; ++kk) {           // K = 8 TF32 = 32 bytes per instruction
                const uint32_t off = kk * 32;
                const unsigned long long ah = smem_desc(st + 0 * TC_TILE_BYTES + off);
                const unsigned long long al = smem_desc(st + 1 * TC_TILE_BYTES + off);
                const unsigned long long bh = smem_desc(st + 2 * TC_TILE_BYTES + off);
                const unsigned long long bl = smem_desc(st + 3 * TC_TILE_BYTES + off);
                mma_tf32(tmem, al, bh, (q > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, ah, bl, 1u);
                mma_tf32(tmem, ah, bh, 1u);
            }
            mma_commit(smem_u32(&bars[TC_STAGES + s]));       // stage s is free when these MMAs retire
            // refill the stage of block q-1 (its MMAs were queued one iteration earlier)
            if (q >= 1 && issued < nkb) {
                const int sp = (q - 1) % TC_STAGES;
                if (!mbar_wait(smem_u32(&bars[TC_STAGES + sp]), (uint32_t)(((q - 1) / TC_STAGES) & 1))) {
                    ok = false;
                    break;
                }
                issue(issued++);
            }
        }
        if (ok) {
            mma_commit(smem_u32(&bars[2 * TC_STAGES]));
        } else {
            s_abort = 1;
            atomicExch(g.err, 1);
            // let the copies already in flight land (bounded) before the buffers go away
            for (int q = 0; q < issued; ++q) mbar_wait(smem_u32(&bars[q % TC_STAGES]), (uint32_t)((q / TC_STAGES) & 1));
        }
    }
    __syncthreads();
    bool have = nkb > 0 && !s_abort;
    if (have) {
        if (!mbar_wait(smem_u32(&bars[2 * TC_STAGES]), 0u)) {
            atomicExch(g.err, 2);
            have = false;
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;");

    // epilogue: warp w owns TMEM lanes 32w..32w+31 = tile rows
    const int i = i0 + warp * 32 + lane;
    float *C = g.C + (long long)z * g.sC;
    const float *Cin = g.Cin ? g.Cin + (long long)z * g.sCin : nullptr;
#pragma unroll 1
    for (int c0 = 0; c0 < TC_BN; c0 += 16) {
        float v[16];
        if (have) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
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
        if (i < g.m) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = j0 + c0 + q;
                if (j >= g.n || (g.lowerC && j > i)) continue;
                float o = g.alpha * v[q];
                if (g.beta != 0.f) o += g.beta * Cin[(long long)i * g.ldcin + j];
                C[(long long)i * g.ldc + j] = o;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// ---------------------------------------------------------------------------
// operand preparation: masked, scaled, K-major, split into tf32 hi + lo
//   out[z][r][p] = src(z, r, p) for r < rows, p < k, zero padded to k_pad
//   src = trans ? X[z][p][r] : X[z][r][p]; structural zeros (tri) forced to 0
// tri: relation of (r, p) that is structurally nonzero:
//   TRI_LOWER: p <= r,  TRI_UPPER: p >= r  (for A: op(A)[i][p]);
//   for B the caller passes the relation in terms of (j, p) of op(B)[p][j]:
//   op(B) lower (p >= j) -> TRI_UPPER here, op(B) upper (p <= j) -> TRI_LOWER
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tf32_split_kernel(const float *X, long long ld, long long sb, int trans,
                                                         int rows, int k, int k_pad, int rows_pad, int tri,
                                                         const float *ks, float *hi, float *lo)
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
    for (int yy = ty; yy < 32; yy += 8) {
        const int r = r0 + yy, p = p0 + tx;
        if (r >= rows_pad || p >= k_pad) continue;
        float v = (r < rows && p < k) ? T[yy][tx] : 0.f;
        if (tri == TRI_LOWER && p > r) v = 0.f;
        if (tri == TRI_UPPER && p < r) v = 0.f;
        if (ks && p < k) v *= ks[p];
        uint32_t u;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
        const float h = __uint_as_float(u);
        const long long o = ((long long)z * rows_pad + r) * k_pad + p;
        hi[o] = h;
        lo[o] = v - h;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool get_encoder()
{
    std::call_once(g_encode_once, []() {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode != nullptr;
}

bool make_map(CUtensorMap *m, const float *base, long long rows_total, int k_pad)
{
    cuuint64_t dims[2] = {(cuuint64_t)k_pad, (cuuint64_t)rows_total};
    cuuint64_t strides[1] = {(cuuint64_t)k_pad * sizeof(float)};
    cuuint32_t box[2] = {TC_BK, TC_BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

size_t tc_gemm_workspace_bytes(const GemmArgs &g)
{
    const long long kp = (g.k + 3) / 4 * 4;
    const long long mp = (g.m + TC_BM - 1) / TC_BM * TC_BM, np = (g.n + TC_BN - 1) / TC_BN * TC_BN;
    return (size_t)(2 * (mp + np) * kp * g.batch) * sizeof(float) + 1024;
}

// ws: device workspace of tc_gemm_workspace_bytes(g) bytes; err: device int (0 on entry)
int tc_gemm_launch(const GemmArgs &g, void *ws, int *err, cudaStream_t s)
{
    if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return 0;
    if (!get_encoder()) return -1;
    static bool attr_done = false;
    if (!attr_done) {
        if (cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BYTES) !=
            cudaSuccess)
            return -2;
        attr_done = true;
    }
    const int kp = (g.k + 3) / 4 * 4;
    const int mp = (g.m + TC_BM - 1) / TC_BM * TC_BM, np = (g.n + TC_BN - 1) / TC_BN * TC_BN;
    float *base = (float *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    float *ah = base, *al = ah + (size_t)mp * kp * g.batch;
    float *bh = al + (size_t)mp * kp * g.batch, *bl = bh + (size_t)np * kp * g.batch;
    {   // A: rows i of op(A), K-major
        dim3 grid((kp + 31) / 32, (mp + 31) / 32, g.batch);
        tf32_split_kernel<<<grid, 256, 0, s>>>((const float *)g.A, g.lda, g.sA, g.ta, g.m, g.k, kp, mp, g.triA,
                                               (const float *)g.kscale, ah, al); count_launch();
    }
    {   // B: rows j of op(B)^T, K-major (op(B)[p][j] = B[p][j] or B[j][p])
        int triB = g.triB == TRI_LOWER ? TRI_UPPER : (g.triB == TRI_UPPER ? TRI_LOWER : TRI_NONE);
        dim3 grid((kp + 31) / 32, (np + 31) / 32, g.batch);
        tf32_split_kernel<<<grid, 256, 0, s>>>((const float *)g.B, g.ldb, g.sB, g.tb ? 0 : 1, g.n, g.k, kp, np, triB,
                                               nullptr, bh, bl); count_launch();
    }
    TcArgs a;
    if (!make_map(&a.ta_hi, ah, (long long)mp * g.batch, kp) || !make_map(&a.ta_lo, al, (long long)mp * g.batch, kp) ||
        !make_map(&a.tb_hi, bh, (long long)np * g.batch, kp) || !make_map(&a.tb_lo, bl, (long long)np * g.batch, kp))
        return -3;
    a.m = g.m; a.n = g.n; a.k = g.k; a.batch = g.batch; a.m_pad = mp; a.n_pad = np;
    a.triA = g.triA; a.triB = g.triB; a.lowerC = g.lowerC;
    a.C = (float *)g.C; a.ldc = g.ldc; a.sC = g.sC;
    a.Cin = (const float *)g.Cin; a.ldcin = g.ldcin; a.sCin = g.sCin;
    a.alpha = (float)g.alpha; a.beta = (float)g.beta;
    a.err = err;
    dim3 grid((g.n + TC_BN - 1) / TC_BN, (g.m + TC_BM - 1) / TC_BM, g.batch);
    tc_gemm_kernel<<<grid, 128, TC_SMEM_BYTES, s>>>(a); count_launch();
    return 0;
}

}  // namespace pssd
