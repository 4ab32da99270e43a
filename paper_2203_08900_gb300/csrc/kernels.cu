// FP64 kernels of libpssd (sm_103a).
//
// On GB300 the FP64 pipe retires 2 DFMA per clock per SM (about 1.1 TFLOP/s
// for the chip), so every FP64 contraction here is bound by the DFMA issue
// rate, not by memory: the GEMM below stages 64x64x16 tiles of both operands
// in shared memory and keeps a 4x4 register tile per thread, which already
// makes shared-memory and HBM traffic a small fraction of the DFMA time.
// The HBM-bound passes (symmetrisation, mirror, shift, combine, norms) use
// 32x32 shared-memory transposes so that both the row and the column access
// are coalesced.
#include <algorithm>
#include <mutex>
#include <set>
#include <utility>

#include "pssd_internal.h"

#include <cooperative_groups.h>

#include <math.h>

#include <type_traits>

namespace pssd {

std::atomic<long long> g_launches{0};
std::atomic<long long> g_phase_launches[PH_COUNT];
thread_local int g_phase = PH_OTHER;

bool ensure_dynamic_smem(const void *func, int bytes)
{
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, func})) return true;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return false;
    done.insert({dev, func});
    return true;
}


// --------------------------------------------------------------------------
// GEMM with triangular operands, lower-only output and inner scaling, in
// three arithmetic modes:
//   GM_F64  FP64 storage, DFMA accumulation
//   GM_F32  FP32 storage, FFMA accumulation
//   GM_DF   FP64 storage, FP64 emulated on the FP32 pipe: each operand is
//           split into a pair of floats (hi = fl32(x), lo = fl32(x - hi)), the
//           product hi*hi is made error-free with an FMA, the cross terms are
//           added in FP32, the running sum is a float pair updated by TwoSum
//           (Knuth) and flushed into an FP64 accumulator every 128 k-steps.
//           The operands arrive already split (split_pairs, one HBM pass),
//           so the FP64 pipe -- 1/64 of the FP32 rate on GB300 -- only sees
//           the flushes.  Relative error per 128-term block ~2^-46.
// --------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 16;

template <class T>
__device__ __forceinline__ T load_op(const T *P, long long ld, int trans, int r, int c)
{
    return trans ? P[(long long)c * ld + r] : P[(long long)r * ld + c];
}

template <int MODE>
__global__ void __launch_bounds__(256) gemm_kernel(GemmArgs g)
{
    using T = typename std::conditional<MODE == GM_F32, float, double>::type;
    const int z = blockIdx.z;
    const int i0 = blockIdx.y * GBM, j0 = blockIdx.x * GBN;
    if (i0 >= g.m || j0 >= g.n) return;
    if (g.lowerC && j0 > i0 + GBM - 1) return;   // tile strictly above the diagonal

    const T *A = (const T *)g.A + (long long)z * g.sA;
    const T *B = (const T *)g.B + (long long)z * g.sB;
    const T *ks = (const T *)g.kscale;
    // GM_DF: float pairs split beforehand
    const float *Ah = (const float *)g.A + (long long)z * g.sA, *Al = (const float *)g.Alo + (long long)z * g.sA;
    const float *Bh = (const float *)g.B + (long long)z * g.sB, *Bl = (const float *)g.Blo + (long long)z * g.sB;
    int kbeg = 0, kend = g.k;
    if (g.triA == TRI_LOWER) kend = min(kend, i0 + GBM);   // op(A)[i][p] = 0 for p > i
    if (g.triA == TRI_UPPER) kbeg = max(kbeg, i0);         // op(A)[i][p] = 0 for p < i
    if (g.triB == TRI_LOWER) kbeg = max(kbeg, j0);         // op(B)[p][j] = 0 for p < j
    if (g.triB == TRI_UPPER) kend = min(kend, j0 + GBN);   // op(B)[p][j] = 0 for p > j

    using S = typename std::conditional<MODE == GM_F64, double, float>::type;
    __shared__ S As[GBK][GBM + 1], Bs[GBK][GBN + 1];
    __shared__ float Asl[MODE == GM_DF ? GBK : 1][GBM + 1], Bsl[MODE == GM_DF ? GBK : 1][GBN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
    float ah_[4][4], al_[4][4];   // DF running float pair (unused otherwise)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) { acc[a][b] = 0; ah_[a][b] = 0.f; al_[a][b] = 0.f; }

    int kt_count = 0;
    for (int kt = kbeg; kt < kend; kt += GBK) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int e = tid + 256 * u;
            int il, pl;
            if (g.ta == 0) { il = e >> 4; pl = e & 15; } else { pl = e >> 6; il = e & 63; }
            int i = i0 + il, p = kt + pl;
            bool ok = (i < g.m) && (p < kend);
            if (g.triA == TRI_LOWER) ok = ok && (p <= i);
            if (g.triA == TRI_UPPER) ok = ok && (p >= i);
            if (MODE == GM_DF) {
                float hi = 0.f, lo = 0.f;
                if (ok) {
                    hi = load_op(Ah, g.lda, g.ta, i, p); lo = load_op(Al, g.lda, g.ta, i, p);
                    if (ks) { float f = (float)ks[p]; hi *= f; lo *= f; }
                }
                As[pl][il] = hi;
                Asl[pl][il] = lo;
            } else {
                T v = 0;
                if (ok) {
                    v = load_op(A, g.lda, g.ta, i, p);
                    if (ks) v *= ks[p];
                }
                As[pl][il] = (S)v;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int e = tid + 256 * u;
            int jl, pl;
            if (g.tb == 0) { pl = e >> 6; jl = e & 63; } else { jl = e >> 4; pl = e & 15; }
            int j = j0 + jl, p = kt + pl;
            bool ok = (j < g.n) && (p < kend);
            if (g.triB == TRI_LOWER) ok = ok && (p >= j);
            if (g.triB == TRI_UPPER) ok = ok && (p <= j);
            if (MODE == GM_DF) {
                float hi = 0.f, lo = 0.f;
                if (ok) { hi = load_op(Bh, g.ldb, g.tb, p, j); lo = load_op(Bl, g.ldb, g.tb, p, j); }
                Bs[pl][jl] = hi;
                Bsl[pl][jl] = lo;
            } else {
                T v = 0;
                if (ok) v = load_op(B, g.ldb, g.tb, p, j);
                Bs[pl][jl] = (S)v;
            }
        }
        __syncthreads();
        if (MODE != GM_DF) {
#pragma unroll
            for (int p = 0; p < GBK; ++p) {
                S a[4], b[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) { a[q] = As[p][ty + 16 * q]; b[q] = Bs[p][tx + 16 * q]; }
#pragma unroll
                for (int qa = 0; qa < 4; ++qa)
#pragma unroll
                    for (int qb = 0; qb < 4; ++qb) acc[qa][qb] = fma((T)a[qa], (T)b[qb], acc[qa][qb]);
            }
        } else {
#pragma unroll 4
            for (int p = 0; p < GBK; ++p) {
                float ahv[4], alv[4], bhv[4], blv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ahv[q] = As[p][ty + 16 * q]; alv[q] = Asl[p][ty + 16 * q];
                    bhv[q] = Bs[p][tx + 16 * q]; blv[q] = Bsl[p][tx + 16 * q];
                }
#pragma unroll
                for (int qa = 0; qa < 4; ++qa)
#pragma unroll
                    for (int qb = 0; qb < 4; ++qb) {
                        // rounded intrinsics: never contracted, so the transformations stay error-free
                        float ph = __fmul_rn(ahv[qa], bhv[qb]);
                        float pe = __fmaf_rn(ahv[qa], bhv[qb], -ph);                 // hi*hi = ph + pe exactly
                        float cr = __fmaf_rn(ahv[qa], blv[qb], __fmul_rn(alv[qa], bhv[qb]));
                        float x = ah_[qa][qb];
                        float s = __fadd_rn(x, ph);                                  // TwoSum(x, ph)
                        float bp = __fsub_rn(s, x);
                        float er = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bp)), __fsub_rn(ph, bp));
                        ah_[qa][qb] = s;
                        al_[qa][qb] = __fadd_rn(al_[qa][qb], __fadd_rn(er, __fadd_rn(pe, cr)));
                    }
            }
            if (((++kt_count) & 7) == 0) {   // flush the float pairs into FP64 every 128 k
#pragma unroll
                for (int qa = 0; qa < 4; ++qa)
#pragma unroll
                    for (int qb = 0; qb < 4; ++qb) {
                        acc[qa][qb] += (double)ah_[qa][qb] + (double)al_[qa][qb];
                        ah_[qa][qb] = 0.f; al_[qa][qb] = 0.f;
                    }
            }
        }
        __syncthreads();
    }
    if (MODE == GM_DF) {
#pragma unroll
        for (int qa = 0; qa < 4; ++qa)
#pragma unroll
            for (int qb = 0; qb < 4; ++qb) acc[qa][qb] += (double)ah_[qa][qb] + (double)al_[qa][qb];
    }

    T *C = (T *)g.C + (long long)z * g.sC;
    const T *Cin = g.Cin ? (const T *)g.Cin + (long long)z * g.sCin : nullptr;
    const T alpha = (T)g.alpha, beta = (T)g.beta;
#pragma unroll
    for (int qa = 0; qa < 4; ++qa) {
        int i = i0 + ty + 16 * qa;
        if (i >= g.m) continue;
#pragma unroll
        for (int qb = 0; qb < 4; ++qb) {
            int j = j0 + tx + 16 * qb;
            if (j >= g.n) continue;
            if (g.lowerC && j > i) continue;
            T v = alpha * acc[qa][qb];
            if (g.beta != 0.0) v += beta * Cin[(long long)i * g.ldcin + j];
            C[(long long)i * g.ldc + j] = v;
        }
    }
}

void gemm_launch(const GemmArgs &g, cudaStream_t s)
{
    if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return;
    dim3 grid((g.n + GBN - 1) / GBN, (g.m + GBM - 1) / GBM, g.batch);
    switch (g.mode) {
    case GM_F32: gemm_kernel<GM_F32><<<grid, 256, 0, s>>>(g); count_launch(); break;
    case GM_DF: gemm_kernel<GM_DF><<<grid, 256, 0, s>>>(g); count_launch(); break;
    default: gemm_kernel<GM_F64><<<grid, 256, 0, s>>>(g); count_launch(); break;
    }
}

// --------------------------------------------------------------------------
// Cholesky of one diagonal block (<= 128 in FP32, <= 64 in FP64) and its
// triangular inverse, blocked by 32 columns
// --------------------------------------------------------------------------
template <class T> struct LeafPivot;
template <> struct LeafPivot<float> {
    static __device__ __forceinline__ void get(float d, float &piv, float &r) { piv = sqrtf(d); r = 1.0f / piv; }
};
template <> struct LeafPivot<double> {
    // the FP64 pipe is narrow: a float reciprocal square root refined by two Newton steps
    // y <- y (3 - d y^2) / 2 (each doubles the number of correct bits) replaces the square
    // root and the division; outside the float range the library functions are used
    static __device__ __forceinline__ void get(double d, double &piv, double &r)
    {
        if (d > 1e-30 && d < 1e30) {
            double y = (double)rsqrtf((float)d);
            y = y * (1.5 - 0.5 * d * y * y);
            y = y * (1.5 - 0.5 * d * y * y);
            piv = d * y;
            r = y;
        } else {
            piv = sqrt(d);
            r = 1.0 / piv;
        }
    }
};

__device__ __forceinline__ void leaf_bar128() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// pivot j of the block at Lb: L_jj = sqrt(D_jj) and rv[j] = 1 / L_jj; a pivot that is not
// positive and finite is recorded in info[z] (global index gpiv + j + 1, first one only)
// and taken as 1
template <class T>
__device__ __forceinline__ void leaf_pivot(T *Lb, int ls, int j, T *rv, int *info, int z, int gpiv, int *bad)
{
    T d = Lb[j * ls + j];
    if (!(d > (T)0) || !isfinite((double)d)) {
        if (!*bad) { *bad = 1; if (info[z] == 0) info[z] = gpiv + j + 1; }
        d = (T)1;
    }
    T piv, r;
    LeafPivot<T>::get(d, piv, r);
    Lb[j * ls + j] = piv;
    rv[j] = r;
}

// Warps 0-3 (thread t < 128, named barrier 1): the w x w (w <= 32) diagonal block D at Lb
// (row stride ls) is factorised in place, D = L_D L_D^T, column by column: the column below
// the pivot is scaled, then row i = j + 1 + t / 4 of the trailing triangle is updated by four
// threads (every fourth column), and the thread that updates (j+1, j+1) takes pivot j + 1 at
// once: two barriers per column.  Then X_D = L_D^{-1} into Xb: column c by four lanes of one
// warp (forward substitution, x_c = 1/L_cc, x_k = -(sum_{m=c}^{k-1} L_km x_m) / L_kk, the sum
// split over the four lanes and reduced with shuffles).  The four warps sit on the four SM
// sub-partitions, which matters for FP64, whose pipe is narrow.
template <class T>
__device__ __forceinline__ void leaf_diag_block(T *Lb, T *Xb, int ls, int w, T *rv, int t, int *info, int z,
                                                int gpiv, int *bad)
{
    if (t == 0) leaf_pivot<T>(Lb, ls, 0, rv, info, z, gpiv, bad);
    leaf_bar128();
    for (int j = 0; j < w; ++j) {
        if (t > j && t < w) Lb[t * ls + j] *= rv[j];
        leaf_bar128();
        const int i = j + 1 + (t >> 2);
        if (i < w) {
            T *row = Lb + i * ls;
            const T lij = row[j];
            for (int c = j + 1 + (t & 3); c <= i; c += 4) row[c] -= lij * Lb[c * ls + j];
            if (t == 0) leaf_pivot<T>(Lb, ls, j + 1, rv, info, z, gpiv, bad);   // (j+1, j+1) is final
        }
        leaf_bar128();
    }
    const int lane = t & 31, c = (t >> 5) * 8 + (lane >> 2), part = lane & 3;
    for (int k = 0; k < w; ++k) {
        T acc = (T)0;
        if (c < w && k > c)
            for (int m = c + part; m < k; m += 4) acc += Lb[k * ls + m] * Xb[m * ls + c];
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (c < w && part == 0 && k >= c) Xb[k * ls + c] = (k == c) ? rv[c] : -acc * rv[k];
        __syncwarp();
    }
}

// FP32 variant of leaf_diag_block for one warp: lane i holds row i of the block in
// registers; column j's scaled entries go through a shared-memory buffer (double-buffered by
// j), and each lane loads the ones it needs before its updates, so the loads pipeline.  (In
// FP64 one warp is limited to its sub-partition's share of the narrow FP64 pipe; the four-warp
// version above is faster there.)
__device__ __forceinline__ void leaf_diag_block_warp(float *Lb, float *Xb, int ls, int w, float *rv, int lane,
                                                     int *info, int z, int gpiv, int *bad, float *colbuf)
{
    float d[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) d[c] = (lane < w && c <= lane) ? Lb[lane * ls + c] : 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        if (j < w) {
            float pj = __shfl_sync(0xffffffffu, d[j], j);
            if (!(pj > 0.f) || !isfinite(pj)) {
                if (lane == 0 && !*bad) { *bad = 1; if (info[z] == 0) info[z] = gpiv + j + 1; }
                pj = 1.f;
            }
            float piv, r;
            LeafPivot<float>::get(pj, piv, r);
            const float lij = (lane == j) ? piv : ((lane > j) ? d[j] * r : d[j]);
            d[j] = lij;
            float *cb = colbuf + (j & 1) * 32;
            cb[lane] = lij;
            if (lane == 0) rv[j] = r;
            __syncwarp();
            float lc[32];
#pragma unroll
            for (int c = j + 1; c < 32; ++c) lc[c] = cb[c];
#pragma unroll
            for (int c = j + 1; c < 32; ++c)
                if (lane >= c) d[c] -= lij * lc[c];
        }
    }
#pragma unroll
    for (int c = 0; c < 32; ++c)
        if (lane < w && c <= lane) Lb[lane * ls + c] = d[c];
    __syncwarp();
    float x[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        float v = 0.f;
        if (k < w) {
            float acc = 0.f;
#pragma unroll
            for (int m = 0; m < k; ++m) acc += Lb[k * ls + m] * x[m];
            v = (k == lane) ? rv[k] : ((k > lane) ? -acc * rv[k] : 0.f);
        }
        x[k] = v;
    }
    if (lane < w) {
#pragma unroll
        for (int k = 0; k < 32; ++k)
            if (k < w && k >= lane) Xb[k * ls + lane] = x[k];
    }
}

// The s x s diagonal block at (off, off) of batch matrix blockIdx.x, in shared memory (row
// stride s + 1), factorised right-looking by blocks of 32 columns with 8 warps:
//   1. warps 0-3 (FP64) or warp 0 (FP32) factorise the diagonal block and invert it;
//   2. panel L_21 = A_21 X_D^T: a warp per row of A_21, lane c holding row c of X_D in
//      registers, the row of A_21 read as shared-memory broadcasts;
//   3. trailing update A_22 -= L_21 L_21^T: lane j holding rows j, j + 32, j + 64 of L_21 in
//      registers, a warp per row i, the lower triangle stored;
// three barriers per block of 32 columns.  Then the off-diagonal blocks of X = L^{-1}, block
// row i after block row i - 1: X_ik = -X_ii (sum_{m=k}^{i-1} L_im X_mk), all k < i at once,
// two rows per warp.
template <class T>
__global__ void __launch_bounds__(256) chol_leaf_kernel(T *A, long long lda, long long sA, T *Rinv, long long ldr,
                                                        long long sR, int off, int s, int *info)
{
    constexpr int NQ = (CholLeaf<T>::max_s - 1) / 32;   // 32-row groups of a panel (3 FP32, 1 FP64)
    extern __shared__ unsigned char leaf_smem[];
    const int ls = s + 1;
    T *L = (T *)leaf_smem;                    // the block, then L
    T *X = L + (size_t)s * ls;                // L^{-1}
    T *W = X + (size_t)s * ls;                // s x 33: the panel, then block products of the inverse
    T *rv = W + (size_t)s * 33;               // 1 / L_jj
    __shared__ int bad;
    __shared__ T colbuf[64];                  // the FP32 diagonal block's column buffer
    const int z = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    A += (long long)z * sA + (long long)off * lda + off;
    Rinv += (long long)z * sR + (long long)off * ldr + off;
    if (tid == 0) bad = 0;
    for (int r = warp; r < s; r += 8)
        for (int c = lane; c < s; c += 32) {
            L[r * ls + c] = (c <= r) ? A[(long long)r * lda + c] : (T)0;
            X[r * ls + c] = (T)0;
        }
    __syncthreads();
    const int nb = (s + 31) >> 5;
    for (int kb = 0; kb < nb; ++kb) {
        const int o = kb * 32, w = min(32, s - o), o2 = o + w, rows = s - o2;
        if constexpr (sizeof(T) == 4) {
            if (warp == 0)
                leaf_diag_block_warp((float *)(L + o * ls + o), (float *)(X + o * ls + o), ls, w, (float *)(rv + o), lane,
                                     info, z, off + o, &bad, (float *)colbuf);
        } else {
            if (warp < 4) leaf_diag_block<T>(L + o * ls + o, X + o * ls + o, ls, w, rv + o, tid, info, z, off + o, &bad);
        }
        __syncthreads();
        if (rows > 0) {
            {   // W[i][c] = sum_{m <= c} A[o2 + i][o + m] X_D[c][m]
                T xd[32];
#pragma unroll
                for (int m = 0; m < 32; ++m) xd[m] = (lane < w && m < w) ? X[(o + lane) * ls + o + m] : (T)0;
                for (int i = warp; i < rows; i += 8) {
                    const T *a = L + (o2 + i) * ls + o;
                    T acc = (T)0;
#pragma unroll
                    for (int m = 0; m < 32; ++m)
                        if (m < w) acc += a[m] * xd[m];
                    W[i * 33 + lane] = acc;
                }
            }
            __syncthreads();
            {
                T wr[NQ][32];
#pragma unroll
                for (int q = 0; q < NQ; ++q)
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        const int j = lane + 32 * q;
                        wr[q][c] = (j < rows && c < w) ? W[j * 33 + c] : (T)0;
                    }
                for (int i = warp; i < rows; i += 8) {
                    const T *wi = W + i * 33;
                    T acc[NQ];
#pragma unroll
                    for (int q = 0; q < NQ; ++q) acc[q] = (T)0;
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        const T v = wi[c];
#pragma unroll
                        for (int q = 0; q < NQ; ++q) acc[q] += v * wr[q][c];
                    }
                    T *lrow = L + (o2 + i) * ls;
                    if (lane < w) lrow[o + lane] = wi[lane];
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const int j = lane + 32 * q;
                        if (j <= i) lrow[o2 + j] -= acc[q];
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int ib = 1; ib < nb; ++ib) {
        const int o = ib * 32, w = min(32, s - o), hw = (w + 1) >> 1;
        for (int idx = warp; idx < ib * hw; idx += 8) {    // W[32 k + r][c] = sum_{q in [32 k, o)} L[o + r][q] X[q][32 k + c]
            const int k = idx / hw, r0 = 2 * (idx - k * hw), r1 = r0 + 1;
            const T *l0 = L + (o + r0) * ls, *l1 = L + (o + (r1 < w ? r1 : r0)) * ls;
            T a0 = (T)0, a1 = (T)0;
            for (int q = k * 32; q < o; ++q) {
                const T xv = X[q * ls + k * 32 + lane];
                a0 += l0[q] * xv;
                a1 += l1[q] * xv;
            }
            W[(k * 32 + r0) * 33 + lane] = a0;
            if (r1 < w) W[(k * 32 + r1) * 33 + lane] = a1;
        }
        __syncthreads();
        for (int idx = warp; idx < ib * hw; idx += 8) {    // X[o + r][32 k + c] = -sum_{q <= r} X_ii[r][q] W[32 k + q][c]
            const int k = idx / hw, r0 = 2 * (idx - k * hw), r1 = r0 + 1;
            const T *d0 = X + (o + r0) * ls + o, *d1 = X + (o + (r1 < w ? r1 : r0)) * ls + o;
            T a0 = (T)0, a1 = (T)0;
            for (int q = 0; q <= r0; ++q) {
                const T wv = W[(k * 32 + q) * 33 + lane];
                a0 += d0[q] * wv;
                a1 += d1[q] * wv;
            }
            if (r1 < w) a1 += d1[r1] * W[(k * 32 + r1) * 33 + lane];
            X[(o + r0) * ls + k * 32 + lane] = -a0;
            if (r1 < w) X[(o + r1) * ls + k * 32 + lane] = -a1;
        }
        __syncthreads();
    }
    for (int r = warp; r < s; r += 8)
        for (int c = lane; c < s; c += 32) {
            A[(long long)r * lda + c] = (c <= r) ? L[r * ls + c] : (T)0;
            Rinv[(long long)r * ldr + c] = (c <= r) ? X[r * ls + c] : (T)0;
        }
}

template <class T>
size_t chol_leaf_smem(int s)
{
    return (2 * (size_t)s * (s + 1) + 34 * (size_t)s) * sizeof(T);
}

template <class T>
int chol_leaf(T *A, long long lda, long long sA, T *Rinv, long long ldr, long long sR, int off, int s, int batch,
              int *info, cudaStream_t st)
{
    const size_t sm = chol_leaf_smem<T>(CholLeaf<T>::max_s);
    if (!ensure_dynamic_smem((const void *)chol_leaf_kernel<T>, (int)sm)) return -1;
    if (s <= 0 || s > CholLeaf<T>::max_s) return -2;
    chol_leaf_kernel<T><<<batch, 256, chol_leaf_smem<T>(s), st>>>(A, lda, sA, Rinv, ldr, sR, off, s, info); count_launch();
    return 0;
}

template int chol_leaf<double>(double *, long long, long long, double *, long long, long long, int, int, int, int *,
                               cudaStream_t);
template int chol_leaf<float>(float *, long long, long long, float *, long long, long long, int, int, int, int *,
                              cudaStream_t);

// --------------------------------------------------------------------------
// HBM passes with 32x32 shared-memory tiles
// --------------------------------------------------------------------------
constexpr int TT = 32;

// M = (Sig H + (Sig H)^T)/2 and the squared defect ||Sig H - (Sig H)^T||_F^2 and
// ||Sig H||_F^2, block partials, over tile pairs (bi >= bj).
__global__ void __launch_bounds__(256) sym_prepare_kernel(const double *H, long long ldh, const double *sig,
                                                          int n, double *M, long long ldm, double *partials)
{
    const int bi = blockIdx.y, bj = blockIdx.x;
    const int blin = blockIdx.y * gridDim.x + blockIdx.x;
    __shared__ double P[TT][TT + 1], Q[TT][TT + 1];
    __shared__ double red[2][256];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    double dsum = 0.0, nsum = 0.0;
    if (bi >= bj) {
        for (int yy = ty; yy < TT; yy += 8) {
            int i = bi * TT + yy, j = bj * TT + tx;
            P[yy][tx] = (i < n && j < n) ? sig[i] * H[(long long)i * ldh + j] : 0.0;
            int i2 = bj * TT + yy, j2 = bi * TT + tx;
            Q[yy][tx] = (i2 < n && j2 < n) ? sig[i2] * H[(long long)i2 * ldh + j2] : 0.0;
        }
        __syncthreads();
        for (int yy = ty; yy < TT; yy += 8) {
            int i = bi * TT + yy, j = bj * TT + tx;
            double a = P[yy][tx], b = Q[tx][yy];     // (Sig H)[i][j] and (Sig H)[j][i]
            if (i < n && j < n) {
                double m = 0.5 * (a + b);
                M[(long long)i * ldm + j] = m;
                double d = a - b;
                double w = (bi == bj) ? 1.0 : 2.0;     // off-diagonal tile pairs count twice
                if (bi == bj) { dsum += d * d; nsum += a * a; }
                else { dsum += w * d * d; nsum += a * a + b * b; }
            }
            int i2 = bj * TT + yy, j2 = bi * TT + tx;
            if (bi != bj && i2 < n && j2 < n) M[(long long)i2 * ldm + j2] = 0.5 * (Q[yy][tx] + P[tx][yy]);
        }
    }
    red[0][threadIdx.x] = dsum; red[1][threadIdx.x] = nsum;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            red[0][threadIdx.x] += red[0][threadIdx.x + st];
            red[1][threadIdx.x] += red[1][threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { partials[2 * blin] = red[0][0]; partials[2 * blin + 1] = red[1][0]; }
}

int sym_prepare_blocks(int n) { int t = (n + TT - 1) / TT; return t * t; }

void sym_prepare(const double *H, long long ldh, const double *sig, int n, double *M, long long ldm,
                 double *partials, cudaStream_t s)
{
    int t = (n + TT - 1) / TT;
    sym_prepare_kernel<<<dim3(t, t), 256, 0, s>>>(H, ldh, sig, n, M, ldm, partials); count_launch();
}

// Casida blocks (Eq. Casida): P = sym(A + B), R = sym(A - B) over 32x32 tile pairs;
// partials[2 b] = squared symmetry defects ||A - A^T||^2 + ||B - B^T||^2 of the tile pair,
// partials[2 b + 1] = its share of ||H||_F^2 = 2 (||A||_F^2 + ||B||_F^2).
__global__ void __launch_bounds__(256) casida_prepare_kernel(const double *A, long long lda, const double *B,
                                                             long long ldb, int k, double *P, double *R,
                                                             long long ldp, double *partials)
{
    const int bi = blockIdx.y, bj = blockIdx.x;
    const int blin = blockIdx.y * gridDim.x + blockIdx.x;
    __shared__ double Ta[TT][TT + 1], Tb[TT][TT + 1], Ua[TT][TT + 1], Ub[TT][TT + 1];
    __shared__ double red[2][256];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double dsum = 0.0, nsum = 0.0;
    if (bi >= bj) {
        for (int yy = ty; yy < TT; yy += 8) {
            int i = bi * TT + yy, j = bj * TT + tx;
            bool in = i < k && j < k;
            Ta[yy][tx] = in ? A[(long long)i * lda + j] : 0.0;
            Tb[yy][tx] = in ? B[(long long)i * ldb + j] : 0.0;
            int i2 = bj * TT + yy, j2 = bi * TT + tx;
            bool in2 = i2 < k && j2 < k;
            Ua[yy][tx] = in2 ? A[(long long)i2 * lda + j2] : 0.0;
            Ub[yy][tx] = in2 ? B[(long long)i2 * ldb + j2] : 0.0;
        }
        __syncthreads();
        for (int yy = ty; yy < TT; yy += 8) {
            int i = bi * TT + yy, j = bj * TT + tx;
            double a = Ta[yy][tx], at = Ua[tx][yy], b = Tb[yy][tx], bt = Ub[tx][yy];   // (i,j) and (j,i)
            if (i < k && j < k) {
                double sa = 0.5 * (a + at), sb = 0.5 * (b + bt);
                P[(long long)i * ldp + j] = sa + sb;
                R[(long long)i * ldp + j] = sa - sb;
                double da = a - at, db = b - bt;
                if (bi == bj) { dsum += da * da + db * db; nsum += 2.0 * (a * a + b * b); }
                else { dsum += 2.0 * (da * da + db * db); nsum += 2.0 * (a * a + at * at + b * b + bt * bt); }
            }
            int i2 = bj * TT + yy, j2 = bi * TT + tx;
            if (bi != bj && i2 < k && j2 < k) {
                double sa = 0.5 * (Ua[yy][tx] + Ta[tx][yy]), sb = 0.5 * (Ub[yy][tx] + Tb[tx][yy]);
                P[(long long)i2 * ldp + j2] = sa + sb;
                R[(long long)i2 * ldp + j2] = sa - sb;
            }
        }
    }
    red[0][threadIdx.x] = dsum; red[1][threadIdx.x] = nsum;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            red[0][threadIdx.x] += red[0][threadIdx.x + st];
            red[1][threadIdx.x] += red[1][threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { partials[2 * blin] = red[0][0]; partials[2 * blin + 1] = red[1][0]; }
}

void casida_prepare(const double *A, long long lda, const double *B, long long ldb, int k, double *P, double *R,
                    long long ldp, double *partials, cudaStream_t s)
{
    int t = (k + TT - 1) / TT;
    casida_prepare_kernel<<<dim3(t, t), 256, 0, s>>>(A, lda, B, ldb, k, P, R, ldp, partials); count_launch();
}

// The orthogonal change of basis T = [[I, I], [I, -I]] / sqrt 2 applied to a pair of k x m
// blocks: top = c (sx X + sy Y), bottom = c (sx X - sy Y), written to rows 0..k-1 and
// k..2k-1 of `out` (ld ldo).  Two doubles per thread, coalesced along rows.
__global__ void casida_combine_kernel(const double *X, long long ldx, const double *Y, long long ldy, int k, int m,
                                      double sx, double sy, double c, double *out, long long ldo)
{
    const long long total = (long long)k * m;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / m), j = (int)(e % m);
        const double x = sx * X[(long long)i * ldx + j], y = sy * Y[(long long)i * ldy + j];
        out[(long long)i * ldo + j] = c * (x + y);
        out[(long long)(i + k) * ldo + j] = c * (x - y);
    }
}

void casida_combine(const double *X, long long ldx, const double *Y, long long ldy, int k, int m, double sx,
                    double sy, double c, double *out, long long ldo, cudaStream_t s)
{
    const long long total = (long long)k * m;
    int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    if (blocks < 1) blocks = 1;
    casida_combine_kernel<<<blocks, 256, 0, s>>>(X, ldx, Y, ldy, k, m, sx, sy, c, out, ldo); count_launch();
}

// H = [[A, B], [-B, -A]] (Eq. Casida) assembled from its blocks
__global__ void casida_build_kernel(const double *A, long long lda, const double *B, long long ldb, int k, double *H,
                                    long long ldh)
{
    const long long total = (long long)k * k;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / k), j = (int)(e % k);
        const double a = A[(long long)i * lda + j], b = B[(long long)i * ldb + j];
        H[(long long)i * ldh + j] = a;
        H[(long long)i * ldh + j + k] = b;
        H[(long long)(i + k) * ldh + j] = -b;
        H[(long long)(i + k) * ldh + j + k] = -a;
    }
}

void casida_build(const double *A, long long lda, const double *B, long long ldb, int k, double *H, long long ldh,
                  cudaStream_t s)
{
    const long long total = (long long)k * k;
    int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    if (blocks < 1) blocks = 1;
    casida_build_kernel<<<blocks, 256, 0, s>>>(A, lda, B, ldb, k, H, ldh); count_launch();
}

// S <- (S + S^T) / 2 in place, over 32x32 tile pairs: the symmetric part of a product of
// two commuting symmetric matrices, whose computed value carries a first-order commutator
// error that averaging cancels (taking one triangle would keep it)
template <class T>
__global__ void __launch_bounds__(256) sym_average_kernel(T *S, long long lds, int n)
{
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bi < bj) return;
    __shared__ T P[TT][TT + 1], Q[TT][TT + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int yy = ty; yy < TT; yy += 8) {
        int i = bi * TT + yy, j = bj * TT + tx;
        P[yy][tx] = (i < n && j < n) ? S[(long long)i * lds + j] : (T)0;
        int i2 = bj * TT + yy, j2 = bi * TT + tx;
        Q[yy][tx] = (i2 < n && j2 < n) ? S[(long long)i2 * lds + j2] : (T)0;
    }
    __syncthreads();
    for (int yy = ty; yy < TT; yy += 8) {
        int i = bi * TT + yy, j = bj * TT + tx;
        if (i < n && j < n) S[(long long)i * lds + j] = (T)0.5 * (P[yy][tx] + Q[tx][yy]);
        int i2 = bj * TT + yy, j2 = bi * TT + tx;
        if (bi != bj && i2 < n && j2 < n) S[(long long)i2 * lds + j2] = (T)0.5 * (Q[yy][tx] + P[tx][yy]);
    }
}

template <class T>
void sym_average(T *S, long long lds, int n, cudaStream_t s)
{
    int t = (n + TT - 1) / TT;
    sym_average_kernel<T><<<dim3(t, t), 256, 0, s>>>(S, lds, n); count_launch();
}
template void sym_average<double>(double *, long long, int, cudaStream_t);
template void sym_average<float>(float *, long long, int, cudaStream_t);

// S <- (S + Sigma S^T Sigma) / 2: the nearest Sigma-symmetric matrix (Sigma S symmetric), in
// place, over 32x32 tile pairs
__global__ void __launch_bounds__(256) j_resym_kernel(double *S, long long lds, const double *sig, int n)
{
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bi < bj) return;
    __shared__ double P[TT][TT + 1], Q[TT][TT + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int yy = ty; yy < TT; yy += 8) {
        int i = bi * TT + yy, j = bj * TT + tx;
        P[yy][tx] = (i < n && j < n) ? S[(long long)i * lds + j] : 0.0;
        int i2 = bj * TT + yy, j2 = bi * TT + tx;
        Q[yy][tx] = (i2 < n && j2 < n) ? S[(long long)i2 * lds + j2] : 0.0;
    }
    __syncthreads();
    for (int yy = ty; yy < TT; yy += 8) {
        int i = bi * TT + yy, j = bj * TT + tx;
        if (i < n && j < n) S[(long long)i * lds + j] = 0.5 * (P[yy][tx] + sig[i] * sig[j] * Q[tx][yy]);
        int i2 = bj * TT + yy, j2 = bi * TT + tx;
        if (bi != bj && i2 < n && j2 < n)
            S[(long long)i2 * lds + j2] = 0.5 * (Q[yy][tx] + sig[i2] * sig[j2] * P[tx][yy]);
    }
}

void j_resym(double *S, long long lds, const double *sig, int n, cudaStream_t s)
{
    int t = (n + TT - 1) / TT;
    j_resym_kernel<<<dim3(t, t), 256, 0, s>>>(S, lds, sig, n); count_launch();
}

// Daleckii-Krein weights of the sign function:
//   X[i][j] = W[i][j] (s_i - s_j) / (lam_i - lam_j) + [i == j] lambar_i,  s = sign(lam)
// (divided differences of sign(x); zero between eigenvalues of the same sign)
__global__ void dk_combine_kernel(const double *W, long long ldw, const double *lam, const double *lambar, int n,
                                  double *X, long long ldx)
{
    const int i = blockIdx.y;
    const double li = lam[i];
    const double si = li > 0.0 ? 1.0 : -1.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double lj = lam[j];
        const double sj = lj > 0.0 ? 1.0 : -1.0;
        double v = (si != sj) ? W[(long long)i * ldw + j] * (si - sj) / (li - lj) : 0.0;
        if (i == j && lambar) v += lambar[i];
        X[(long long)i * ldx + j] = v;
    }
}

void dk_combine(const double *W, long long ldw, const double *lam, const double *lambar, int n, double *X,
                long long ldx, cudaStream_t s)
{
    int gx = (n + 255) / 256; if (gx > 16) gx = 16;
    dk_combine_kernel<<<dim3(gx, n), 256, 0, s>>>(W, ldw, lam, lambar, n, X, ldx); count_launch();
}

// Correction of one refinement step of an approximate symmetric eigendecomposition
// A ~ Z diag(lam) Z^T (Ogita and Aishima's iteration): with S = Z^T A Z and
// Gm = Z^T Z - I (both full, symmetric), R = -Gm and
//   F_ii = R_ii / 2,
//   F_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i)   if |lam_j - lam_i| > omega,
//   F_ij = R_ij / 2                                  otherwise (a cluster: keep orthogonality only).
__global__ void eig_refine_correction_kernel(const double *S, long long lds, const double *Gm, long long ldg,
                                             const double *lam, int n, double omega, double *F, long long ldf)
{
    const int i = blockIdx.y;
    const double li = lam[i];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double r = -Gm[(long long)i * ldg + j];
        const double d = lam[j] - li;
        double v = 0.5 * r;
        if (i != j && fabs(d) > omega) v = (S[(long long)i * lds + j] + lam[j] * r) / d;
        F[(long long)i * ldf + j] = v;
    }
}

void eig_refine_correction(const double *S, long long lds, const double *Gm, long long ldg, const double *lam, int n,
                           double omega, double *F, long long ldf, cudaStream_t s)
{
    int gx = (n + 255) / 256; if (gx > 16) gx = 16;
    eig_refine_correction_kernel<<<dim3(gx, n), 256, 0, s>>>(S, lds, Gm, ldg, lam, n, omega, F, ldf);
    count_launch();
}

// Phi(X): the lower triangle with its diagonal halved, the strict upper triangle zeroed
// (the operator of the Cholesky factorisation's adjoint)
__global__ void tril_half_diag_kernel(double *X, long long ldx, int n)
{
    const int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double *x = X + (long long)i * ldx + j;
        if (j > i) *x = 0.0;
        else if (j == i) *x *= 0.5;
    }
}

void tril_half_diag(double *X, long long ldx, int n, cudaStream_t s)
{
    int gx = (n + 255) / 256; if (gx > 16) gx = 16;
    tril_half_diag_kernel<<<dim3(gx, n), 256, 0, s>>>(X, ldx, n); count_launch();
}

// Real embedding of a complex n x n matrix Z (interleaved re/im doubles, row-major, ld in
// complex elements): R = [[Re Z, -Im Z], [Im Z, Re Z]] (2n x 2n, ld ldr).  Z -> R is an
// injective real algebra homomorphism with R(Z^H) = R(Z)^T.
__global__ void complex_embed_kernel(const double *Z, long long ldz, int n, double *R, long long ldr)
{
    const int i = blockIdx.y;
    const double2 *z = reinterpret_cast<const double2 *>(Z) + (long long)i * ldz;
    double *r0 = R + (long long)i * ldr, *r1 = R + (long long)(i + n) * ldr;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double2 v = z[j];
        r0[j] = v.x; r0[j + n] = -v.y;
        r1[j] = v.y; r1[j + n] = v.x;
    }
}

void complex_embed(const double *Z, long long ldz, int n, double *R, long long ldr, cudaStream_t s)
{
    int gx = (n + 255) / 256; if (gx > 16) gx = 16;
    complex_embed_kernel<<<dim3(gx, n), 256, 0, s>>>(Z, ldz, n, R, ldr); count_launch();
}

// The inverse on the first block column: Z[i][j] = R[i][j] + i R[i + n][j] for j < m
// (columns j of R taken in the order perm[0..m) when perm is given)
__global__ void complex_extract_kernel(const double *R, long long ldr, int n, int m, const int *perm, double *Z,
                                       long long ldz)
{
    const int i = blockIdx.y;
    double2 *z = reinterpret_cast<double2 *>(Z) + (long long)i * ldz;
    const double *r0 = R + (long long)i * ldr, *r1 = R + (long long)(i + n) * ldr;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const int c = perm ? perm[j] : j;
        z[j] = make_double2(r0[c], r1[c]);
    }
}

void complex_extract(const double *R, long long ldr, int n, int m, const int *perm, double *Z, long long ldz,
                     cudaStream_t s)
{
    int gx = (m + 255) / 256; if (gx > 16) gx = 16;
    complex_extract_kernel<<<dim3(gx, n), 256, 0, s>>>(R, ldr, n, m, perm, Z, ldz); count_launch();
}

// Column phase convention for complex eigenvectors: each column of Z (m x n, interleaved)
// is multiplied by conj(z_max)/|z_max|, z_max its entry of largest modulus (first one on
// ties), so that entry becomes real and positive.  One block per column.
__global__ void complex_phase_fix_kernel(double *Z, long long ldz, int m, int n)
{
    __shared__ double bm[256];
    __shared__ int bi[256];
    const int c = blockIdx.x, t = threadIdx.x;
    double2 *z = reinterpret_cast<double2 *>(Z);
    double best = -1.0; int bidx = 0;
    for (int i = t; i < m; i += blockDim.x) {
        const double2 v = z[(long long)i * ldz + c];
        const double a = v.x * v.x + v.y * v.y;
        if (a > best) { best = a; bidx = i; }
    }
    bm[t] = best; bi[t] = bidx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o && (bm[t + o] > bm[t] || (bm[t + o] == bm[t] && bi[t + o] < bi[t]))) {
            bm[t] = bm[t + o]; bi[t] = bi[t + o];
        }
        __syncthreads();
    }
    const double2 p = z[(long long)bi[0] * ldz + c];
    const double a = sqrt(p.x * p.x + p.y * p.y);
    if (!(a > 0.0)) return;
    const double cr = p.x / a, ci = -p.y / a;     // conj(p) / |p|
    for (int i = t; i < m; i += blockDim.x) {
        double2 &v = z[(long long)i * ldz + c];
        const double x = v.x * cr - v.y * ci, y = v.x * ci + v.y * cr;
        v = make_double2(x, y);
    }
}

void complex_phase_fix(double *Z, long long ldz, int m, int n, cudaStream_t s)
{
    complex_phase_fix_kernel<<<n, 256, 0, s>>>(Z, ldz, m, n); count_launch();
}

// X[i][j] *= r[i] (row scaling)
__global__ void scale_rows_kernel(double *X, long long ldx, int m, int n, const double *r)
{
    const int i = blockIdx.y;
    const double f = r[i];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        X[(long long)i * ldx + j] *= f;
}

void scale_rows(double *X, long long ldx, int m, int n, const double *r, cudaStream_t s)
{
    int gx = (n + 255) / 256; if (gx > 16) gx = 16;
    scale_rows_kernel<<<dim3(gx, m), 256, 0, s>>>(X, ldx, m, n, r); count_launch();
}

// (hi, lo) = (fl32(x), fl32(x - hi)) for a batch of rows x cols blocks (source
// leading dimension ld, batch stride sb), written compactly (ld = cols)
__global__ void split_pairs_kernel(const double *x, long long ld, long long sb, int rows, int cols, float *hi,
                                   float *lo)
{
    const int z = blockIdx.z, i = blockIdx.y;
    const double *xr = x + (long long)z * sb + (long long)i * ld;
    const long long o = ((long long)z * rows + i) * cols;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cols; j += gridDim.x * blockDim.x) {
        double v = xr[j];
        float h = __double2float_rn(v);
        hi[o + j] = h;
        lo[o + j] = __double2float_rn(v - (double)h);
    }
}

void split_pairs(const double *x, long long ld, long long sb, int rows, int cols, int batch, float *hi, float *lo,
                 cudaStream_t s)
{
    int gx = (cols + 255) / 256; if (gx > 16) gx = 16;
    split_pairs_kernel<<<dim3(gx, rows, batch), 256, 0, s>>>(x, ld, sb, rows, cols, hi, lo); count_launch();
}

// fixed-order single-block sum (deterministic)
__global__ void reduce_sum_kernel(const double *x, int count, int stride, double *out)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += 1024) s += x[(long long)i * stride];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 512; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

void reduce_sum(const double *x, int count, double *out, cudaStream_t s)
{
    reduce_sum_kernel<<<1, 1024, 0, s>>>(x, count, 1, out); count_launch();
}

// copy the strictly lower triangle onto the upper one
template <class T>
__global__ void __launch_bounds__(256) mirror_lower_kernel(T *A, long long lda, long long sA, int n)
{
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bi < bj) return;
    A += (long long)blockIdx.z * sA;
    __shared__ T P[TT][TT + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int yy = ty; yy < TT; yy += 8) {
        int i = bi * TT + yy, j = bj * TT + tx;
        P[yy][tx] = (i < n && j < n) ? A[(long long)i * lda + j] : (T)0;
    }
    __syncthreads();
    for (int yy = ty; yy < TT; yy += 8) {
        int i = bj * TT + yy, j = bi * TT + tx;   // target (i, j) in the upper tile
        if (i < n && j < n && j > i) A[(long long)i * lda + j] = P[tx][yy];
    }
}

template <class T>
void mirror_lower(T *A, long long lda, long long sA, int n, int batch, cudaStream_t s)
{
    int t = (n + TT - 1) / TT;
    mirror_lower_kernel<T><<<dim3(t, t, batch), 256, 0, s>>>(A, lda, sA, n); count_launch();
}
template void mirror_lower<double>(double *, long long, long long, int, int, cudaStream_t);
template void mirror_lower<float>(float *, long long, long long, int, int, cudaStream_t);

template <class T>
__global__ void shift_copy_lower_kernel(const T *G, long long ldg, T *Z, long long ldz, long long sZ, int n,
                                        const double *shifts)
{
    const int z = blockIdx.z;
    const int i = blockIdx.y;
    const T c = (T)shifts[z];
    T *Zr = Z + (long long)z * sZ + (long long)i * ldz;
    const T *Gr = G + (long long)i * ldg;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= i && j < n; j += gridDim.x * blockDim.x)
        Zr[j] = Gr[j] + (i == j ? c : (T)0);
}

template <class T>
void shift_copy_lower(const T *G, long long ldg, T *Z, long long ldz, long long sZ, int n, const double *shifts,
                      int batch, cudaStream_t s)
{
    int gx = (n + 255) / 256; if (gx > 8) gx = 8;
    shift_copy_lower_kernel<T><<<dim3(gx, n, batch), 256, 0, s>>>(G, ldg, Z, ldz, sZ, n, shifts); count_launch();
}
template void shift_copy_lower<double>(const double *, long long, double *, long long, long long, int,
                                       const double *, int, cudaStream_t);
template void shift_copy_lower<float>(const float *, long long, float *, long long, long long, int,
                                      const double *, int, cudaStream_t);

template <class T>
__global__ void combine_lower_kernel(const T *Zinv, long long ldz, long long sZ, const double *a, int r, int n,
                                     T *Tm, long long ldt)
{
    const int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= i && j < n; j += gridDim.x * blockDim.x) {
        T v = 0;
        for (int q = 0; q < r; ++q) v = fma((T)a[q], Zinv[(long long)q * sZ + (long long)i * ldz + j], v);
        Tm[(long long)i * ldt + j] = v;
    }
}

template <class T>
void combine_lower(const T *Zinv, long long ldz, long long sZ, const double *a, int r, int n, T *Tm, long long ldt,
                   cudaStream_t s)
{
    int gx = (n + 255) / 256; if (gx > 8) gx = 8;
    combine_lower_kernel<T><<<dim3(gx, n), 256, 0, s>>>(Zinv, ldz, sZ, a, r, n, Tm, ldt); count_launch();
}
template void combine_lower<double>(const double *, long long, long long, const double *, int, int, double *,
                                    long long, cudaStream_t);
template void combine_lower<float>(const float *, long long, long long, const double *, int, int, float *,
                                   long long, cudaStream_t);

template <class TI, class TO>
__global__ void scale_copy_kernel(const TI *X, long long ldx, TO *Y, long long ldy, int m, int n, double alpha)
{
    const int i = blockIdx.y;
    if (i >= m) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        Y[(long long)i * ldy + j] = (TO)(alpha * (double)X[(long long)i * ldx + j]);
}

template <class TI, class TO>
void scale_copy(const TI *X, long long ldx, TO *Y, long long ldy, int m, int n, double alpha, cudaStream_t s)
{
    if (m <= 0 || n <= 0) return;
    int gx = (n + 255) / 256; if (gx > 16) gx = 16;
    scale_copy_kernel<TI, TO><<<dim3(gx, m), 256, 0, s>>>(X, ldx, Y, ldy, m, n, alpha); count_launch();
}
template void scale_copy<double, double>(const double *, long long, double *, long long, int, int, double, cudaStream_t);
template void scale_copy<double, float>(const double *, long long, float *, long long, int, int, double, cudaStream_t);
template void scale_copy<float, double>(const float *, long long, double *, long long, int, int, double, cudaStream_t);
template void scale_copy<float, float>(const float *, long long, float *, long long, int, int, double, cudaStream_t);

void copy_matrix(const double *X, long long ldx, double *Y, long long ldy, int m, int n, cudaStream_t s)
{
    scale_copy<double, double>(X, ldx, Y, ldy, m, n, 1.0, s);
}

// Y[z] = X[z] for z < batch (m x n blocks, strides sX, sY): one launch for the batch
template <class T>
__global__ void copy_batched_kernel(const T *X, long long ldx, long long sX, T *Y, long long ldy, long long sY, int m,
                                    int n)
{
    const int i = blockIdx.y;
    const T *x = X + (long long)blockIdx.z * sX + (long long)i * ldx;
    T *y = Y + (long long)blockIdx.z * sY + (long long)i * ldy;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) y[j] = x[j];
}

template <class T>
void copy_batched(const T *X, long long ldx, long long sX, T *Y, long long ldy, long long sY, int m, int n, int batch,
                  cudaStream_t s)
{
    if (m <= 0 || n <= 0 || batch <= 0) return;
    int gx = (n + 255) / 256; if (gx > 16) gx = 16;
    copy_batched_kernel<T><<<dim3(gx, m, batch), 256, 0, s>>>(X, ldx, sX, Y, ldy, sY, m, n); count_launch();
}
template void copy_batched<double>(const double *, long long, long long, double *, long long, long long, int, int, int,
                                   cudaStream_t);
template void copy_batched<float>(const float *, long long, long long, float *, long long, long long, int, int, int,
                                  cudaStream_t);

// Z[i][j] <- (B[i][j] + Z[i][j]) / 2 for j < p, (B[i][j] - Z[i][j]) / 2 for j >= p (m x n):
// with Z = Y B on entry, the columns (I + Y)/2 B_+ and (I - Y)/2 B_- of the two projectors
__global__ void half_sum_diff_kernel(const double *B, long long ldb, double *Z, long long ldz, int m, int n, int p)
{
    const int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double b = B[(long long)i * ldb + j], z = Z[(long long)i * ldz + j];
        Z[(long long)i * ldz + j] = 0.5 * (j < p ? b + z : b - z);
    }
}

void half_sum_diff(const double *B, long long ldb, double *Z, long long ldz, int m, int n, int p, cudaStream_t s)
{
    if (m <= 0 || n <= 0) return;
    int gx = (n + 255) / 256; if (gx > 16) gx = 16;
    half_sum_diff_kernel<<<dim3(gx, m), 256, 0, s>>>(B, ldb, Z, ldz, m, n, p); count_launch();
}

// Y = a diag(sig)^rx X + b diag(sig) T diag(sig) (n x n; T may be null): the signature
// scalings of the general sign iteration, one pass (Y may alias X or T: entry by entry)
__global__ void sig_affine_kernel(const double *X, long long ldx, int rx, const double *T, long long ldt,
                                  const double *sig, int n, double a, double b, double *Y, long long ldy)
{
    const int i = blockIdx.y;
    const double si = sig[i], ai = rx ? a * si : a;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double v = ai * X[(long long)i * ldx + j];
        if (T) v += b * si * sig[j] * T[(long long)i * ldt + j];
        Y[(long long)i * ldy + j] = v;
    }
}

void sig_affine(const double *X, long long ldx, int rx, const double *T, long long ldt, const double *sig, int n,
                double a, double b, double *Y, long long ldy, cudaStream_t s)
{
    if (n <= 0) return;
    int gx = (n + 255) / 256; if (gx > 16) gx = 16;
    sig_affine_kernel<<<dim3(gx, n), 256, 0, s>>>(X, ldx, rx, T, ldt, sig, n, a, b, Y, ldy); count_launch();
}

template <class T>
__global__ void add_diag_kernel(T *X, long long ldx, int n, double v)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        X[(long long)i * ldx + i] += (T)v;
}

template <class T>
void add_diag(T *X, long long ldx, int n, double v, cudaStream_t s)
{
    add_diag_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(X, ldx, n, v); count_launch();
}
template void add_diag<double>(double *, long long, int, double, cudaStream_t);
template void add_diag<float>(float *, long long, int, double, cudaStream_t);

// per-block partials of ||X - Y||_F^2 and ||Y||_F^2 (grid-stride over rows)
constexpr int FROB_BLOCKS = 608;  // 4 x 152 SMs

template <class T>
__global__ void __launch_bounds__(256) frob_diff_kernel(const T *X, long long ldx, const T *Y, long long ldy, int m,
                                                        int n, double *partials)
{
    __shared__ double red[2][256];
    double d2 = 0.0, y2 = 0.0;
    for (int i = blockIdx.x; i < m; i += gridDim.x) {
        for (int j = threadIdx.x; j < n; j += 256) {
            double y = (double)Y[(long long)i * ldy + j];
            double d = (X ? (double)X[(long long)i * ldx + j] : 0.0) - y;
            d2 += d * d; y2 += y * y;
        }
    }
    red[0][threadIdx.x] = d2; red[1][threadIdx.x] = y2;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            red[0][threadIdx.x] += red[0][threadIdx.x + st];
            red[1][threadIdx.x] += red[1][threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { partials[2 * blockIdx.x] = red[0][0]; partials[2 * blockIdx.x + 1] = red[1][0]; }
}

int frob_blocks(int m, int n) { (void)n; return m < FROB_BLOCKS ? (m > 0 ? m : 1) : FROB_BLOCKS; }

template <class T>
void frob_diff(const T *X, long long ldx, const T *Y, long long ldy, int m, int n, double *partials, cudaStream_t s)
{
    frob_diff_kernel<T><<<frob_blocks(m, n), 256, 0, s>>>(X, ldx, Y, ldy, m, n, partials); count_launch();
}
template void frob_diff<double>(const double *, long long, const double *, long long, int, int, double *, cudaStream_t);
template void frob_diff<float>(const float *, long long, const float *, long long, int, int, double *, cudaStream_t);

// counter-based normal variates: splitmix64 hash of (seed, index) -> two
// uniforms -> Box-Muller
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// entry `idx` of the seeded Gaussian stream (Box-Muller on two splitmix64 draws)
__device__ __forceinline__ double gauss_at(uint64_t seed, uint64_t idx)
{
    uint64_t h1 = splitmix64(seed ^ (idx * 2 + 1)), h2 = splitmix64(seed + idx * 2 + 0x1234567ull);
    double u1 = ((h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

__global__ void fill_gaussian_kernel(double *X, long long ldx, int m, int n, uint64_t seed)
{
    for (int i = blockIdx.y; i < m; i += gridDim.y)
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
            X[(long long)i * ldx + j] = gauss_at(seed, (uint64_t)i * (uint64_t)n + (uint64_t)j);
}

void fill_gaussian(double *X, long long ldx, int m, int n, uint64_t seed, cudaStream_t s)
{
    int gx = (n + 255) / 256; if (gx > 16) gx = 16;
    const int gy = m < 65535 ? m : 65535;
    if (gy <= 0) return;
    fill_gaussian_kernel<<<dim3(gx, gy), 256, 0, s>>>(X, ldx, m, n, seed); count_launch();
}

__global__ void trace_kernel(const double *X, long long ldx, int n, double *out)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) s += X[(long long)i * ldx + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 512; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

void trace_partial(const double *X, long long ldx, int n, double *out, cudaStream_t s)
{
    trace_kernel<<<1, 1024, 0, s>>>(X, ldx, n, out); count_launch();
}

__global__ void get_diag_kernel(const double *X, long long ldx, int n, double *d)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        d[i] = X[(long long)i * ldx + i];
}

void get_diag(const double *X, long long ldx, int n, double *d, cudaStream_t s)
{
    get_diag_kernel<<<(n + 255) / 256, 256, 0, s>>>(X, ldx, n, d); count_launch();
}

// max over rows of sum_j |X[i][j]| (the infinity norm, an upper bound on
// ||X||_2 for symmetric X): one warp per row, then a fixed-order max.
__global__ void row_abs_sums_kernel(const double *X, long long ldx, int n, double *sums)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += fabs(X[(long long)warp * ldx + j]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sums[warp] = s;
}

__global__ void reduce_max_kernel(const double *x, int n, double *out)
{
    __shared__ double red[1024];
    double b = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) b = fmax(b, x[i]);
    red[threadIdx.x] = b;
    __syncthreads();
    for (int st = 512; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

void row_abs_sum_max(const double *X, long long ldx, int n, double *tmp, double *out, cudaStream_t s)
{
    row_abs_sums_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(X, ldx, n, tmp); count_launch();
    reduce_max_kernel<<<1, 1024, 0, s>>>(tmp, n, out); count_launch();
}

// y = op(A) x for square n, op(A) optionally triangular (masked)
__global__ void gemv_n_kernel(const double *A, long long lda, int tri, int n, const double *x, double *y)
{
    // one warp per row
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int i = warp;
    int jb = 0, je = n;
    if (tri == TRI_LOWER) je = i + 1;
    if (tri == TRI_UPPER) jb = i;
    double s = 0.0;
    for (int j = jb + lane; j < je; j += 32) s = fma(A[(long long)i * lda + j], x[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) y[i] = s;
}

// y[i] = sum_p A[p][i] x[p] (op(A) = A^T, `tri` describes op(A)); rows are
// split into GEMV_CHUNKS slices whose partial sums are added in a fixed order.
constexpr int GEMV_CHUNKS = 32;

__global__ void gemv_t_partial_kernel(const double *A, long long lda, int tri, int n, const double *x,
                                      double *part)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int ch = blockIdx.y;
    if (i >= n) return;
    const int len = (n + GEMV_CHUNKS - 1) / GEMV_CHUNKS;
    int pb = ch * len, pe = min(n, pb + len);
    if (tri == TRI_LOWER) pe = min(pe, i + 1);   // op(A)[i][p] = A[p][i] nonzero for p <= i
    if (tri == TRI_UPPER) pb = max(pb, i);
    double s = 0.0;
    for (int p = pb; p < pe; ++p) s = fma(A[(long long)p * lda + i], x[p], s);
    part[(long long)ch * n + i] = s;
}

__global__ void gemv_t_reduce_kernel(const double *part, int n, double *y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int c = 0; c < GEMV_CHUNKS; ++c) s += part[(long long)c * n + i];
    y[i] = s;
}

void gemv(const double *A, long long lda, int ta, int tri, int n, const double *x, double *y, double *tmp,
          cudaStream_t s)
{
    if (ta == 0) {
        gemv_n_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(A, lda, tri, n, x, y); count_launch();
    } else {
        gemv_t_partial_kernel<<<dim3((n + 127) / 128, GEMV_CHUNKS), 128, 0, s>>>(A, lda, tri, n, x, tmp); count_launch();
        gemv_t_reduce_kernel<<<(n + 255) / 256, 256, 0, s>>>(tmp, n, y); count_launch();
    }
}

__global__ void normalize_kernel(double *y, double *x, int n, double *norm_out)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) s += y[i] * y[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 512; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    double nrm = sqrt(red[0]);
    double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) x[i] = y[i] * inv;
    if (threadIdx.x == 0 && norm_out) norm_out[0] = nrm;
}

void normalize_vec(double *y, double *x, int n, double *norm_out, cudaStream_t s)
{
    normalize_kernel<<<1, 1024, 0, s>>>(y, x, n, norm_out); count_launch();
}

// Lanczos three-term update w <- w - alpha v - beta vprev with alpha, beta read
// from device memory (beta may be null): no host round trip per step
__global__ void lanczos_update_kernel(double *w, const double *v, const double *vprev, const double *alpha,
                                      const double *beta, int n)
{
    const double a = alpha[0], b = beta ? beta[0] : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        w[i] = w[i] - a * v[i] - (vprev ? b * vprev[i] : 0.0);
}

void lanczos_update(double *w, const double *v, const double *vprev, const double *alpha, const double *beta, int n,
                    cudaStream_t s)
{
    int blocks = (n + 255) / 256; if (blocks > 64) blocks = 64;
    lanczos_update_kernel<<<blocks, 256, 0, s>>>(w, v, vprev, alpha, beta, n); count_launch();
}

__global__ void dot_kernel(const double *x, const double *y, int n, double *out)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) s += x[i] * y[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 512; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

void dot_vec(const double *x, const double *y, int n, double *out, cudaStream_t s)
{
    dot_kernel<<<1, 1024, 0, s>>>(x, y, n, out); count_launch();
}

// ---------------------------------------------------------------------------
// Krylov loops in one launch.  Step by step, a Lanczos step takes four launches
// (product, alpha, three-term update, beta with the new vector) and a power
// step three or four; the recursion's nodes, the bounds of small inputs and
// the shift screening run such loops hundreds of times on operators whose
// matrix sits in L2.  Here one cluster of KRY_CLUSTER CTAs runs a whole loop.
// CTA c owns rows [c R, (c + 1) R) of the operator, R = ceil(m / KRY_CLUSTER);
// every CTA keeps the whole current and previous vectors in shared memory.  A
// dot product is summed per CTA (warps, then warps in order), then across the
// cluster through distributed shared memory in rank order, so every CTA holds
// the same scalar to the bit.  A new vector is all-gathered by each CTA storing
// its rows into every CTA's buffer.  Each exchange ends at a cluster barrier, a
// hardware barrier that every thread of every CTA reaches equally often (all
// loop bounds are uniform across the cluster): no thread waits on a flag.
// ---------------------------------------------------------------------------
constexpr int KRY_CLUSTER = 8, KRY_THREADS = 1024, KRY_WARPS = KRY_THREADS / 32;
constexpr int KRY_ROWS = KRY_MAX_M / KRY_CLUSTER;      // rows (and columns) owned by a CTA, at most
constexpr int KRY_GROUPS = KRY_THREADS / KRY_ROWS;     // row groups of the transposed product
constexpr int KRY_SMEM = (4 * KRY_MAX_M + KRY_ROWS + KRY_GROUPS * KRY_ROWS) * (int)sizeof(double);
static_assert(KRY_THREADS % KRY_ROWS == 0 && KRY_SMEM <= 48 * 1024, "Krylov kernel layout");

namespace cg = cooperative_groups;

// sum of x over the CTA, returned to every thread
__device__ double kry_block_sum(double x, double *red, double *bc)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < KRY_WARPS; ++w) s += red[w];
        *bc = s;
    }
    __syncthreads();
    return *bc;
}

// sum over the cluster of the CTAs' partial sums `part`, returned to every thread of
// every CTA.  Two slots alternate: a slot is rewritten only after another cluster
// barrier, by which time every CTA has read it.
__device__ double kry_cluster_sum(cg::cluster_group &cl, double part, double *slot, int &turn, double *bc)
{
    double *my = slot + turn;
    turn ^= 1;
    if (threadIdx.x == 0) *my = part;
    cl.sync();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int c = 0; c < KRY_CLUSTER; ++c) s += *cl.map_shared_rank(my, c);
        *bc = s;
    }
    __syncthreads();
    return *bc;
}

// rows r0 .. r0 + nr - 1 of A x (tri: of L x, L lower triangular) -> wl; one warp per row
__device__ void kry_rows(const double *__restrict__ A, long long lda, bool tri, const double *x, double *wl,
                         int r0, int nr, int m)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < nr; i += KRY_WARPS) {
        const double *row = A + (long long)(r0 + i) * lda;
        const int len = tri ? r0 + i + 1 : m;
        double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int k = lane;
        for (; k + 224 < len; k += 256) {   // eight independent loads in flight per lane
            double r[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) r[q] = __ldg(row + k + 32 * q);
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = fma(r[q], x[k + 32 * q], a[q]);
        }
        if (k + 96 < len) {
            double r[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) r[q] = __ldg(row + k + 32 * q);
#pragma unroll
            for (int q = 0; q < 4; ++q) a[q] = fma(r[q], x[k + 32 * q], a[q]);
            k += 128;
        }
        for (; k < len; k += 32) a[0] = fma(__ldg(row + k), x[k], a[0]);
        double s = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) wl[i] = s;
    }
    __syncthreads();
}

// entries r0 .. r0 + nr - 1 of L^T u (L lower triangular) -> wl: thread (g, c) sums
// L[p][r0 + c] u[p] over p = r0 + g, r0 + g + KRY_GROUPS, ... (a warp reads 32
// consecutive entries of a row), then the groups' sums are added in order
__device__ void kry_tri_t_cols(const double *__restrict__ A, long long lda, const double *u, double *wl,
                               double *colp, int r0, int nr, int m)
{
    const int c = threadIdx.x % KRY_ROWS, g = threadIdx.x / KRY_ROWS;
    double acc = 0.0;
    if (c < nr) {
        const int col = r0 + c;
        for (int p = max(r0 + g, col - (col - r0 - g) % KRY_GROUPS); p < m; p += KRY_GROUPS)
            if (p >= col) acc = fma(__ldg(A + (long long)p * lda + col), u[p], acc);
    }
    colp[g * KRY_ROWS + c] = acc;
    __syncthreads();
    for (int i = threadIdx.x; i < nr; i += KRY_THREADS) {
        double s = 0.0;
        for (int q = 0; q < KRY_GROUPS; ++q) s += colp[q * KRY_ROWS + i];
        wl[i] = s;
    }
    __syncthreads();
}

// scale * src[0 .. nr) -> dst[r0 .. r0 + nr) in every CTA of the cluster, then a cluster barrier
__device__ void kry_gather(cg::cluster_group &cl, const double *src, double scale, double *dst, int r0, int nr)
{
    for (int c = 0; c < KRY_CLUSTER; ++c) {
        double *rd = cl.map_shared_rank(dst, c);
        for (int i = threadIdx.x; i < nr; i += KRY_THREADS) rd[r0 + i] = src[i] * scale;
    }
    cl.sync();
}

template <int OP>
__global__ void __cluster_dims__(KRY_CLUSTER, 1, 1) __launch_bounds__(KRY_THREADS, 1)
krylov_cluster_kernel(const double *__restrict__ A, long long lda, int m, int steps, int power, uint64_t seed,
                      double *out)
{
    extern __shared__ __align__(16) double kry_sm[];
    __shared__ double red[KRY_WARPS], slot[2], bc;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int R = (m + KRY_CLUSTER - 1) / KRY_CLUSTER;
    const int r0 = min(m, rank * R), nr = min(m, r0 + R) - r0;
    double *cur = kry_sm, *prv = cur + KRY_MAX_M, *nxt = prv + KRY_MAX_M, *ub = nxt + KRY_MAX_M;
    double *wl = ub + KRY_MAX_M, *colp = wl + KRY_ROWS;
    int turn = 0;
    // the starting vector, whole in every CTA (same entries, same summation order)
    double sq = 0.0;
    for (int i = threadIdx.x; i < m; i += KRY_THREADS) {
        const double g = gauss_at(seed, (uint64_t)i);
        cur[i] = g;
        prv[i] = 0.0;
        sq += g * g;
    }
    sq = kry_block_sum(sq, red, &bc);
    const double inv0 = sq > 0.0 ? 1.0 / sqrt(sq) : 0.0;
    for (int i = threadIdx.x; i < m; i += KRY_THREADS) cur[i] *= inv0;
    cl.sync();   // every CTA has started (its shared memory exists) before the first remote access
    auto apply = [&](const double *x) {   // the CTA's rows of op(A) x -> wl
        if (OP == KRY_SYM) {
            kry_rows(A, lda, false, x, wl, r0, nr, m);
        } else {
            kry_rows(A, lda, true, x, wl, r0, nr, m);         // u = L x, own rows
            kry_gather(cl, wl, 1.0, ub, r0, nr);               // u whole in every CTA
            kry_tri_t_cols(A, lda, ub, wl, colp, r0, nr, m);   // L^T u, own entries
        }
    };
    if (power == 0) {
        double beta_prev = 0.0;
        for (int j = 0; j < steps; ++j) {
            apply(cur);
            double pa = 0.0;
            for (int i = threadIdx.x; i < nr; i += KRY_THREADS) pa += cur[r0 + i] * wl[i];
            const double alpha = kry_cluster_sum(cl, kry_block_sum(pa, red, &bc), slot, turn, &bc);
            double pb = 0.0;
            for (int i = threadIdx.x; i < nr; i += KRY_THREADS) {
                const double w = wl[i] - alpha * cur[r0 + i] - beta_prev * prv[r0 + i];
                wl[i] = w;
                pb += w * w;
            }
            const double beta = sqrt(kry_cluster_sum(cl, kry_block_sum(pb, red, &bc), slot, turn, &bc));
            if (rank == 0 && threadIdx.x == 0) { out[j] = alpha; out[steps + 1 + j] = beta; }
            kry_gather(cl, wl, beta > 0.0 ? 1.0 / beta : 0.0, nxt, r0, nr);
            double *t = prv; prv = cur; cur = nxt; nxt = t;
            beta_prev = beta;
        }
    } else {
        for (int it = 0; it < power; ++it) {
            apply(cur);
            double pb = 0.0;
            for (int i = threadIdx.x; i < nr; i += KRY_THREADS) pb += wl[i] * wl[i];
            const double nrm = sqrt(kry_cluster_sum(cl, kry_block_sum(pb, red, &bc), slot, turn, &bc));
            kry_gather(cl, wl, nrm > 0.0 ? 1.0 / nrm : 0.0, nxt, r0, nr);
            double *t = cur; cur = nxt; nxt = t;
        }
        apply(cur);
        double pa = 0.0;
        for (int i = threadIdx.x; i < nr; i += KRY_THREADS) pa += cur[r0 + i] * wl[i];
        const double rq = kry_cluster_sum(cl, kry_block_sum(pa, red, &bc), slot, turn, &bc);
        if (rank == 0 && threadIdx.x == 0) out[0] = rq;
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

bool krylov_cluster(const double *A, long long lda, int op, int m, int steps, int power, uint64_t seed, double *out,
                    cudaStream_t s)
{
    if (m < 1 || m > KRY_MAX_M || steps < 0 || power < 0) return false;
    if (op == KRY_SYM)
        krylov_cluster_kernel<KRY_SYM><<<KRY_CLUSTER, KRY_THREADS, KRY_SMEM, s>>>(A, lda, m, steps, power, seed, out);
    else
        krylov_cluster_kernel<KRY_TRI_PAIR><<<KRY_CLUSTER, KRY_THREADS, KRY_SMEM, s>>>(A, lda, m, steps, power, seed,
                                                                                      out);
    count_launch();
    return true;
}

__global__ void scale_columns_kernel(double *X, long long ldx, int m, int n, const double *d, int use_sqrt_abs)
{
    const int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double f = use_sqrt_abs ? sqrt(fabs(d[j])) : d[j];
        X[(long long)i * ldx + j] *= f;
    }
}

void scale_columns(double *X, long long ldx, int m, int n, const double *d, int use_sqrt_abs, cudaStream_t s)
{
    int gx = (n + 255) / 256; if (gx > 16) gx = 16;
    scale_columns_kernel<<<dim3(gx, m), 256, 0, s>>>(X, ldx, m, n, d, use_sqrt_abs); count_launch();
}

// make the largest-magnitude entry of each column positive (ties: lowest row)
__global__ void sign_fix_columns_kernel(double *X, long long ldx, int m, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double best = -1.0, val = 0.0;
    for (int i = 0; i < m; ++i) {
        double v = X[(long long)i * ldx + j];
        if (fabs(v) > best) { best = fabs(v); val = v; }
    }
    if (val < 0.0)
        for (int i = 0; i < m; ++i) X[(long long)i * ldx + j] = -X[(long long)i * ldx + j];
}

void sign_fix_columns(double *X, long long ldx, int m, int n, cudaStream_t s)
{
    sign_fix_columns_kernel<<<(n + 127) / 128, 128, 0, s>>>(X, ldx, m, n); count_launch();
}

__global__ void gather_columns_kernel(const double *X, long long ldx, double *Y, long long ldy, int m, int n,
                                      const int *perm)
{
    const int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        Y[(long long)i * ldy + j] = X[(long long)i * ldx + perm[j]];
}

void gather_columns(const double *X, long long ldx, double *Y, long long ldy, int m, int n, const int *perm,
                    cudaStream_t s)
{
    int gx = (n + 255) / 256; if (gx > 16) gx = 16;
    gather_columns_kernel<<<dim3(gx, m), 256, 0, s>>>(X, ldx, Y, ldy, m, n, perm); count_launch();
}

// --------------------------------------------------------------------------
// Jacobi eigensolver for one symmetric matrix of order m <= 64 (one CTA).
// Parallel cyclic order: in each of the m'-1 rounds (m' = m rounded up to
// even) the pairs of a round-robin tournament are disjoint, so all their
// rotations are applied together (rows, then columns, then eigenvectors).
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) jacobi_leaf_kernel(double *Ag, long long lda, int m, double *W,
                                                          long long ldw, double *w, int *sweeps_out)
{
    __shared__ double A[64][65];
    __shared__ double V[64][65];
    __shared__ double cs[32], sn[32];
    __shared__ int pp[32], qq[32];
    __shared__ int order[64];
    __shared__ double offn, dian;
    const int tid = threadIdx.x;
    const int me = (m + 1) & ~1;   // even
    for (int e = tid; e < 64 * 64; e += 256) {
        int i = e >> 6, j = e & 63;
        A[i][j] = (i < m && j < m) ? 0.5 * (Ag[(long long)i * lda + j] + Ag[(long long)j * lda + i]) : 0.0;
        V[i][j] = (i == j) ? 1.0 : 0.0;
    }
    if (tid < 64) order[tid] = tid;
    __syncthreads();
    int sweep = 0;
    for (; sweep < 40; ++sweep) {
        if (tid == 0) { offn = 0.0; dian = 0.0; }
        __syncthreads();
        {
            double o = 0.0, d = 0.0;
            for (int e = tid; e < m * m; e += 256) {
                int i = e / m, j = e % m;
                double v = A[i][j];
                if (i == j) d += v * v; else o += v * v;
            }
            atomicAdd(&offn, o);
            atomicAdd(&dian, d);
        }
        __syncthreads();
        if (offn <= 1e-30 * dian || offn == 0.0) break;
        for (int round = 0; round < me - 1; ++round) {
            // pairs of this round: (order[k], order[me-1-k])
            if (tid < me / 2) {
                int p = order[tid], q = order[me - 1 - tid];
                if (p > q) { int t = p; p = q; q = t; }
                pp[tid] = p; qq[tid] = q;
                double c = 1.0, s = 0.0;
                if (q < m) {
                    double apq = A[p][q];
                    if (apq != 0.0) {
                        double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
                        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t); s = t * c;
                    }
                }
                cs[tid] = c; sn[tid] = s;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = tid; e < (me / 2) * m; e += 256) {
                int k = e / m, col = e % m;
                int p = pp[k], q = qq[k];
                if (q >= m) continue;
                double c = cs[k], s = sn[k];
                double ap = A[p][col], aq = A[q][col];
                A[p][col] = c * ap - s * aq;
                A[q][col] = s * ap + c * aq;
            }
            __syncthreads();
            // columns: A <- A J, and V <- V J
            for (int e = tid; e < (me / 2) * m; e += 256) {
                int k = e / m, row = e % m;
                int p = pp[k], q = qq[k];
                if (q >= m) continue;
                double c = cs[k], s = sn[k];
                double ap = A[row][p], aq = A[row][q];
                A[row][p] = c * ap - s * aq;
                A[row][q] = s * ap + c * aq;
                double vp = V[row][p], vq = V[row][q];
                V[row][p] = c * vp - s * vq;
                V[row][q] = s * vp + c * vq;
            }
            __syncthreads();
            // rotate the tournament: keep order[0], shift the rest
            if (tid == 0) {
                int last = order[me - 1];
                for (int k = me - 1; k > 1; --k) order[k] = order[k - 1];
                order[1] = last;
            }
            __syncthreads();
        }
    }
    for (int e = tid; e < m * m; e += 256) {
        int i = e / m, j = e % m;
        W[(long long)i * ldw + j] = V[i][j];
    }
    if (tid < m) w[tid] = A[tid][tid];
    if (tid == 0 && sweeps_out) sweeps_out[0] = sweep;
}

void jacobi_leaf(double *A, long long lda, int m, double *W, long long ldw, double *w, int *sweeps_out,
                 cudaStream_t s)
{
    jacobi_leaf_kernel<<<1, 256, 0, s>>>(A, lda, m, W, ldw, w, sweeps_out); count_launch();
}

}  // namespace pssd
