// Binary32-accuracy GEMM on the 5th-generation tensor cores (tcgen05, sm_103a):
//   C (m x n, column-major, ldc) = alpha * op(A) op(B) + beta * C.
// Each operand x is split into two TF32 planes, x = hi + lo (hi = tf32(x), lo = tf32(x - hi)),
// and the product is accumulated in FP32 as A_hi B_hi + A_hi B_lo + A_lo B_hi (the A_lo B_lo
// term is below binary32 rounding). This is the binary32 GEMM of the reduction and the
// back-transformations of the binary32 route.
//
// Structure of one CTA (320 threads; persistent over 128 x 128 tiles of C):
//   warp 0, one lane : TMA producer. Loads the K-major hi and lo tiles of A and B (32 fp32 of
//                      K = 128 bytes per row, 128-byte swizzle) into a 3-stage ring, one
//                      mbarrier per stage with the transaction byte count;
//   warp 1, one lane : MMA issuer. tcgen05.mma kind::tf32, M = 128, N = 128, K = 8 per
//                      instruction, accumulator in tensor memory (128 lanes x 128 columns);
//                      tcgen05.commit frees a stage when its MMAs have read it;
//   warps 2-9        : epilogue: warp w owns rows 32 (w mod 4) .. + 31 and columns
//                      64 h .. 64 h + 63 (h = (w - 2) / 4) of the tile. It sums the K
//                      chunks of the two tensor-memory accumulators (tcgen05.ld) in
//                      registers, then loads its part of C (beta != 0; 32 columns in flight
//                      at once) and writes C = alpha acc + beta C with coalesced
//                      column-major stores; warp 2 allocates and frees the tensor memory.
// Every wait is bounded; on expiry the kernel records ELSI_ERR_TIMEOUT and finishes without
// further waits on the pipeline (after a bounded wait for its own TMA copies in flight).
#include <cuda.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace egb {
namespace tcg {

using namespace tc5;

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 3;
constexpr int CH = 2;  // k-tiles per tensor-memory accumulation chunk (K = 64)
constexpr int TILE_BYTES = BM * BK * 4;  // 16 KB (BN == BM)
constexpr int STAGE_BYTES = 4 * TILE_BYTES;  // A_hi, A_lo, B_hi, B_lo
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int TMEM_COLS = 4 * BN;  // two buffers x (hi*hi sum, cross-term sum)
constexpr int EPI_WARPS = 8, CW = BN / 2;  // epilogue warps; columns per epilogue warp
constexpr int THREADS = 32 * (2 + EPI_WARPS);

__device__ __forceinline__ void mma_tf32(unsigned tmem_d, unsigned long long a, unsigned long long b,
                                         unsigned idesc, unsigned accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

struct Maps {
    CUtensorMap a_hi, a_lo, b_hi, b_lo;
};


// Warps: 0 = TMA producer (one lane), 1 = MMA issuer (one lane), 2..9 = epilogue (warp w
// reads tensor-memory lanes 32 (w mod 4) .. + 31, i.e. those rows of the tile). K is
// accumulated in chunks of CH k-tiles in one of two tensor-memory buffers, each holding the
// hi*hi sum and the (2^-11 times smaller) cross-term sum separately; the epilogue warps add
// each chunk into binary32 registers (round to nearest) while the MMA issuer fills the other
// buffer. The tensor-memory accumulation is not rounded to nearest, so its error grows with
// the number of MMAs summed into one accumulator and with that accumulator's magnitude;
// short chunks and the separate small sum keep it at the binary32 level.
//
// Persistent: one CTA per SM walks the tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// (row tile fastest; with uplo the tiles strictly above the diagonal are skipped), all three
// roles in the same order, so that the k-tile ring and the two accumulator buffers keep
// their phases across tiles: while the epilogue warps read-modify-write C for one tile the
// MMA issuer already fills the accumulator buffers with the next tile's first chunks and the
// producer keeps the ring full.
__device__ __forceinline__ bool tile_of(int t, int tiles_m, int uplo, int *m0, int *n0)
{
    *m0 = (t % tiles_m) * BM;
    *n0 = (t / tiles_m) * BN;
    return !(uplo && *m0 + BM - 1 < *n0);  // false: strictly above the diagonal
}

__global__ void __launch_bounds__(THREADS, 1)
gemm_tf32x3_kernel(const __grid_constant__ Maps maps, int m, int n, int kp, float alpha,
                   float beta, float *__restrict__ C, int ldc, int uplo, int *status)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((size_t)smem_raw + 1023) & ~(size_t)1023);
    unsigned long long *bars = (unsigned long long *)(smem + STAGES * STAGE_BYTES);
    // bars: [0,S) full, [S,2S) empty, 2S+b accumulator b full, 2S+2+b accumulator b empty
    unsigned *tmem_slot = (unsigned *)(bars + 2 * STAGES + 4);
    __shared__ int aborted;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_m = (m + BM - 1) / BM, tiles_n = (n + BN - 1) / BN;
    const int ntiles = tiles_m * tiles_n;
    const int nk = kp / BK;
    const int nchunk = (nk + CH - 1) / CH;
    const unsigned full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[STAGES]);
    const unsigned accf0 = smem_u32(&bars[2 * STAGES]), acce0 = smem_u32(&bars[2 * STAGES + 2]);

    if (tid == 0) {
        for (int s = 0; s < 2 * STAGES + 2; ++s) mbar_init(smem_u32(&bars[s]), 1);
        mbar_init(acce0, EPI_WARPS);
        mbar_init(acce0 + 8, EPI_WARPS);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        aborted = 0;
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;

    int armed = 0;  // producer: k-tiles loaded (over all tiles of this CTA)
    if (warp == 0) {
        if (lane == 0) {
            int ktg = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
                int m0, n0;
                if (!tile_of(t, tiles_m, uplo, &m0, &n0)) continue;
                for (int kt = 0; kt < nk; ++kt, ++ktg) {
                    const int s = ktg % STAGES;
                    const unsigned ph = (ktg / STAGES) & 1;
                    if (ktg >= STAGES && !mbar_wait(empty0 + 8 * s, ph ^ 1)) {
                        report_error(status, ELSI_ERR_TIMEOUT, 1);
                        atomicExch(&aborted, 1);
                        stop = true;
                        break;
                    }
                    if (*(volatile int *)&aborted) { stop = true; break; }
                    unsigned char *st = smem + s * STAGE_BYTES;
                    const unsigned full = full0 + 8 * s;
                    mbar_expect_tx(full, STAGE_BYTES);
                    tma_load_2d(smem_u32(st), &maps.a_hi, full, kt * BK, m0);
                    tma_load_2d(smem_u32(st + TILE_BYTES), &maps.a_lo, full, kt * BK, m0);
                    tma_load_2d(smem_u32(st + 2 * TILE_BYTES), &maps.b_hi, full, kt * BK, n0);
                    tma_load_2d(smem_u32(st + 3 * TILE_BYTES), &maps.b_lo, full, kt * BK, n0);
                    armed = ktg + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const unsigned idesc = idesc_f32acc(2, BM, BN);
            int ktg = 0, gbase = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
                int m0, n0;
                if (!tile_of(t, tiles_m, uplo, &m0, &n0)) continue;
                for (int kt = 0; kt < nk; ++kt, ++ktg) {
                    const int s = ktg % STAGES, g = gbase + kt / CH, bsel = g & 1;
                    const unsigned ph = (ktg / STAGES) & 1;
                    const bool first = (kt % CH) == 0;
                    if (first && g >= 2 && !mbar_wait(acce0 + 8 * bsel, ((g >> 1) - 1) & 1)) {
                        report_error(status, ELSI_ERR_TIMEOUT, 4);
                        atomicExch(&aborted, 1);
                        stop = true;
                        break;
                    }
                    if (!mbar_wait(full0 + 8 * s, ph)) {
                        report_error(status, ELSI_ERR_TIMEOUT, 2);
                        atomicExch(&aborted, 1);
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const unsigned base = smem_u32(smem + s * STAGE_BYTES);
                    const unsigned d = tmem + bsel * 2 * BN;  // hi*hi sum; cross terms at + BN
#pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        const unsigned off = kk * 32;  // 8 tf32 = 32 bytes along K
                        const unsigned long long ah = sdesc(base + off), al = sdesc(base + TILE_BYTES + off);
                        const unsigned long long bh = sdesc(base + 2 * TILE_BYTES + off);
                        const unsigned long long bl = sdesc(base + 3 * TILE_BYTES + off);
                        const unsigned acc = (first && kk == 0) ? 0u : 1u;
                        mma_tf32(d + BN, al, bh, idesc, acc);
                        mma_tf32(d + BN, ah, bl, idesc, 1u);
                        mma_tf32(d, ah, bh, idesc, acc);
                    }
                    mma_commit(empty0 + 8 * s);
                    if ((kt % CH) == CH - 1 || kt == nk - 1) mma_commit(accf0 + 8 * bsel);
                }
                gbase += nchunk;
            }
        }
    } else {
        // tensor-memory loads are warp-collective: every lane runs them (rows past m only
        // skip their global-memory accesses) and the wait results are made uniform
        const int quarter = warp & 3, c0 = ((warp - 2) >> 2) * CW;
        bool ok = true;
        int gbase = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            int m0, n0;
            if (!tile_of(t, tiles_m, uplo, &m0, &n0)) continue;
            const int row = m0 + quarter * 32 + lane;
            const bool row_in = row < m;
            float *crow = C + (size_t)row;
            float acc[CW];
#pragma unroll
            for (int j = 0; j < CW; ++j) acc[j] = 0.0f;
            for (int c = 0; c < nchunk && ok; ++c) {
                const int g = gbase + c, bsel = g & 1;
                ok = __all_sync(0xffffffffu, mbar_wait(accf0 + 8 * bsel, (g >> 1) & 1));
                if (!ok) {
                    if (lane == 0) {
                        report_error(status, ELSI_ERR_TIMEOUT, 3);
                        atomicExch(&aborted, 1);
                    }
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int q = 0; q < CW / 32; ++q) {
                    float v[32];
                    const unsigned ta =
                        tmem + ((unsigned)(quarter * 32) << 16) + bsel * 2 * BN + c0 + q * 32;
                    tmem_ld32(ta + BN, v);  // cross terms
#pragma unroll
                    for (int j = 0; j < 32; ++j) acc[q * 32 + j] += v[j];
                    tmem_ld32(ta, v);  // hi * hi
#pragma unroll
                    for (int j = 0; j < 32; ++j) acc[q * 32 + j] += v[j];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce0 + 8 * bsel);
            }
            gbase += nchunk;
            if (ok && row_in) {
                // 32 loads of C at a time (one 128-byte line per column and warp, 32 KB in
                // flight per CTA), then their stores
#pragma unroll
                for (int h = 0; h < CW / 32; ++h) {
                    float cv[32];
                    float *cp = crow + (size_t)(n0 + c0 + h * 32) * ldc;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = n0 + c0 + h * 32 + j;
                        const bool in = col < n && (!uplo || row >= col);
                        cv[j] = (beta != 0.0f && in) ? cp[(size_t)j * ldc] : 0.0f;
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = n0 + c0 + h * 32 + j;
                        if (col < n && (!uplo || row >= col))
                            cp[(size_t)j * ldc] = alpha * acc[h * 32 + j] + beta * cv[j];
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (aborted && warp == 0 && lane == 0) {
        // bounded wait for this CTA's own TMA copies still in flight
        for (int kt = (armed > STAGES ? armed - STAGES : 0); kt < armed; ++kt)
            mbar_wait(full0 + 8 * (kt % STAGES), (kt / STAGES) & 1);
    }
    __syncthreads();
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
}

// Columns [q_off, q_off + kw) of the rows x kp plane (K-major) of hi / lo TF32 parts of the
// operand piece element (r, q) = src[r * sr + q * sq] (one of sr, sq is 1), q < k, zero for
// k <= q < kw. 32 x 32 tiles through shared memory so that reads and writes coalesce.
__global__ void split_planes_kernel(int rows, int k, int kw, int kp, int q_off,
                                    const float *__restrict__ src, long long sr, long long sq,
                                    float *__restrict__ hi, float *__restrict__ lo)
{
    __shared__ float t[32][33];
    const int r0 = blockIdx.y * 32, q0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    if (sq == 1) {
        for (int i = ty; i < 32; i += 8) {
            const int r = r0 + i, q = q0 + tx;
            t[i][tx] = (r < rows && q < k) ? src[r * sr + q] : 0.0f;
        }
    } else {
        for (int i = ty; i < 32; i += 8) {
            const int q = q0 + i, r = r0 + tx;
            t[tx][i] = (r < rows && q < k) ? src[r + q * sq] : 0.0f;
        }
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int r = r0 + i, q = q0 + tx;
        if (r < rows && q < kw) {
            const float x = t[i][tx];
            unsigned h;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
            h &= 0xFFFFE000u;
            const float xh = __uint_as_float(h);
            unsigned l;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - xh));
            l &= 0xFFFFE000u;
            hi[(size_t)r * kp + q_off + q] = xh;
            lo[(size_t)r * kp + q_off + q] = __uint_as_float(l);
        }
    }
}

// rows x kp fp32 plane, K-major, boxes of 32 (K) x 128 (rows), 128-byte swizzle.
static bool make_map(CUtensorMap *map, const float *plane, int rows, int kp)
{
    return make_map_2d(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, plane, rows, kp, kp, BK, BM);
}

}  // namespace tcg

static inline int kround(int k) { return ((k + tcg::BK - 1) / tcg::BK) * tcg::BK; }

size_t tc_gemm_work_elems(int m, int n, int k)
{
    return 2 * ((size_t)m + n) * (size_t)kround(k) + 64;
}

cudaError_t tc_gemm_f32_parts(cudaStream_t st, int m, int n, int nparts, const TcPart *a,
                              const TcPart *b, float alpha, float beta, float *C, int ldc, int uplo,
                              float *work, size_t work_elems, int *status)
{
    using namespace tcg;
    if (m <= 0 || n <= 0) return cudaSuccess;
    int kp = 0;
    for (int i = 0; i < nparts; ++i) {
        if (a[i].k != b[i].k || a[i].k <= 0) return cudaErrorNotSupported;
        kp += kround(a[i].k);
    }
    if (kp <= 0 || work_elems < 2 * ((size_t)m + n) * kp + 64 || ((size_t)work & 15))
        return cudaErrorNotSupported;
    float *ahi = work, *alo = ahi + (size_t)m * kp, *bhi = alo + (size_t)m * kp, *blo = bhi + (size_t)n * kp;
    dim3 tb32(32, 8);
    int off = 0;
    for (int i = 0; i < nparts; ++i) {
        const int kw = kround(a[i].k);
        // op(A) element (i, q): trans = 0 -> A[i + q ld]; trans = 1 -> A[q + i ld]
        EGB_COUNT_LAUNCH();
        split_planes_kernel<<<dim3(kw / 32, (m + 31) / 32), tb32, 0, st>>>(
            m, a[i].k, kw, kp, off, a[i].p, a[i].trans ? (long long)a[i].ld : 1,
            a[i].trans ? 1 : (long long)a[i].ld, ahi, alo);
        // op(B) element (q, j) is plane row j: trans = 0 -> B[q + j ld]; trans = 1 -> B[j + q ld]
        EGB_COUNT_LAUNCH();
        split_planes_kernel<<<dim3(kw / 32, (n + 31) / 32), tb32, 0, st>>>(
            n, b[i].k, kw, kp, off, b[i].p, b[i].trans ? 1 : (long long)b[i].ld,
            b[i].trans ? (long long)b[i].ld : 1, bhi, blo);
        off += kw;
    }
    Maps maps;
    if (!make_map(&maps.a_hi, ahi, m, kp) || !make_map(&maps.a_lo, alo, m, kp) ||
        !make_map(&maps.b_hi, bhi, n, kp) || !make_map(&maps.b_lo, blo, n, kp))
        return cudaErrorNotSupported;
    static PerDeviceOnce attr_once;
    cudaError_t attr_err = once_per_device(attr_once, [] {
        return cudaFuncSetAttribute(gemm_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    });
    if (attr_err != cudaSuccess) return attr_err;
    // persistent: one CTA per SM (the ring takes 192 KB of shared memory), at most one per tile
    static int sms[kMaxDevices] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int nsm = (dev >= 0 && dev < kMaxDevices) ? sms[dev] : 0;
    if (nsm <= 0) {
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
        if (dev >= 0 && dev < kMaxDevices) sms[dev] = nsm;
    }
    const long long ntiles = (long long)((m + BM - 1) / BM) * ((n + BN - 1) / BN);
    const int grid = (int)(ntiles < nsm ? ntiles : nsm);
    EGB_COUNT_LAUNCH();
    gemm_tf32x3_kernel<<<grid, THREADS, SMEM_BYTES, st>>>(maps, m, n, kp, alpha, beta, C, ldc, uplo, status);
    return cudaGetLastError();
}

cudaError_t tc_gemm_f32(cudaStream_t st, int ta, int tb, int m, int n, int k, float alpha,
                        const float *A, int lda, const float *B, int ldb, float beta, float *C,
                        int ldc, int uplo, float *work, size_t work_elems, int *status)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (k <= 0) return cudaErrorNotSupported;
    TcPart pa{A, lda, ta, k}, pb{B, ldb, tb, k};
    return tc_gemm_f32_parts(st, m, n, 1, &pa, &pb, alpha, beta, C, ldc, uplo, work, work_elems, status);
}

}  // namespace egb

extern "C" size_t elsi_gb_gemm_f32_work(int m, int n, int k)
{
    return egb::tc_gemm_work_elems(m, n, k);
}

extern "C" int elsi_gb_gemm_f32(int ta, int tb, int m, int n, int k, float alpha, const float *A,
                                int lda, const float *B, int ldb, float beta, float *C, int ldc,
                                int uplo, float *work, size_t work_elems, int *status, void *stream)
{
    if (m < 0 || n < 0 || k < 1 || !A || !B || !C || !work || !status) return ELSI_ERR_ARG;
    cudaError_t e = egb::tc_gemm_f32((cudaStream_t)stream, ta, tb, m, n, k, alpha, A, lda, B, ldb,
                                     beta, C, ldc, uplo, work, work_elems, status);
    if (e == cudaErrorNotSupported) return ELSI_ERR_ARG;
    return e == cudaSuccess ? ELSI_OK : ELSI_ERR_CUDA;
}
