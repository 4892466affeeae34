// X = A V for a symmetric m x m binary32 matrix A (full column-major storage) and an
// m x N panel V, N <= 64: the product A22 V of the two-sided update of the full-to-band
// reduction (Eq. 11, first line; sec. 3.1, step (1)), in binary32 accuracy on the tcgen05
// tensor cores as three TF32 products of hi/lo splits (A_hi V_hi + A_hi V_lo + A_lo V_hi).
//
// The product reads each element of A once and does 2N flops with it, so it is bound by
// the HBM stream of A. Unlike the general binary32 GEMM, A is not split into TF32 planes in
// global memory beforehand: its raw tiles come in by TMA and are split in shared memory.
// By symmetry, X_i. = sum_q A(q, i) V(q, .), so row i of the product needs column i of A,
// which is contiguous in memory: the K-major operand layout the MMA wants, loaded as a
// 32 (K) x 128 (rows of X) box of the column-major matrix.
//
// Work split (stream-K): the rows of X are cut into 128-row tiles and K into 32-wide
// k-tiles; the tiles_m * nk (tile, k-tile) steps, tile-major, are cut into G contiguous
// ranges, one per CTA (G = number of SMs), so that every SM streams the same share of A.
// A CTA writes one 128 x 64 partial sum per tile its range touches; a second kernel adds
// the partials of each tile in a fixed order (deterministic).
//
// One CTA, 320 threads:
//   warp 0, one lane: TMA producer: raw A tile (16 KB) and the V hi / lo tiles (8 KB each)
//                     of a k-tile into a STAGES ring;
//   warps 2..5:       split the raw A tile in place into its TF32 hi part and write the lo
//                     part next to it (elementwise, so the 128-byte swizzle is kept);
//   warp 1, one lane: MMA issuer, kind::tf32, M = 128, N = 64, K = 8, hi*hi and the two
//                     cross terms into two separate accumulators, chunks of CH k-tiles in
//                     one of two tensor-memory buffers;
//   warps 6..9:       epilogue: warp w reads tensor-memory lanes 32 (w mod 4) .. + 31, adds
//                     the chunks in binary32 registers (round to nearest) and writes the
//                     partial of each tile segment.
// Every wait is bounded; on expiry the kernel records ELSI_ERR_TIMEOUT and finishes.
#include <cuda.h>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace egb {
namespace symv {

using namespace tc5;

constexpr int BM = 128, BN = 64, BK = 32, STAGES = 4, CH = 2;
constexpr int A_BYTES = BM * BK * 4;                    // 16 KB
constexpr int B_BYTES = BN * BK * 4;                    // 8 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // A hi (raw), A lo, V hi, V lo
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int TMEM_COLS = 4 * BN;  // two buffers x (hi*hi, cross)
constexpr int SPLIT_WARPS = 4, EPI_WARPS = 4;
constexpr int THREADS = 32 * (2 + SPLIT_WARPS + EPI_WARPS);
constexpr int TILE_ELEMS = BM * BN;  // one partial: 128 rows x 64 columns, column-major

struct Maps {
    CUtensorMap a, v_hi, v_lo;
};

struct Args {
    int m, nk, G, slots;
    long long T;  // tiles_m * nk steps
    float *part;  // G * slots partial tiles
    int *status;
};

__device__ __forceinline__ long long range_begin(long long c, long long T, int G) { return c * T / G; }

__device__ __forceinline__ void mma_tf32(unsigned tmem_d, unsigned long long a, unsigned long long b,
                                         unsigned idesc, unsigned accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

// hi = TF32 rounding of x (to nearest, ties away), lo = TF32 rounding of x - hi.
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo)
{
    unsigned h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    h &= 0xFFFFE000u;
    hi = __uint_as_float(h);
    unsigned l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hi));
    lo = __uint_as_float(l & 0xFFFFE000u);
}

__global__ void __launch_bounds__(THREADS, 1)
symm_tall_kernel(const __grid_constant__ Maps maps, const Args a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((size_t)smem_raw + 1023) & ~(size_t)1023);
    unsigned long long *bars = (unsigned long long *)(smem + STAGES * STAGE_BYTES);
    // bars: [0,S) full (TMA), [S,2S) ready (split), [2S,3S) empty (MMA done),
    //       3S+b accumulator b full, 3S+2+b accumulator b empty
    unsigned *tmem_slot = (unsigned *)(bars + 3 * STAGES + 4);
    __shared__ int aborted;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long beg = range_begin(blockIdx.x, a.T, a.G), end = range_begin(blockIdx.x + 1, a.T, a.G);
    const unsigned full0 = smem_u32(&bars[0]), ready0 = smem_u32(&bars[STAGES]),
                   empty0 = smem_u32(&bars[2 * STAGES]);
    const unsigned accf0 = smem_u32(&bars[3 * STAGES]), acce0 = smem_u32(&bars[3 * STAGES + 2]);

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(ready0 + 8 * s, SPLIT_WARPS);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accf0, 1);
        mbar_init(accf0 + 8, 1);
        mbar_init(acce0, EPI_WARPS);
        mbar_init(acce0 + 8, EPI_WARPS);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        aborted = 0;
    }
    if (warp == 6) tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;

    long long armed = 0;  // producer: k-tiles loaded
    if (warp == 0) {
        if (lane == 0) {
            long long it = 0;
            for (long long g = beg; g < end; ++g, ++it) {
                const int s = (int)(it % STAGES);
                const unsigned ph = (unsigned)((it / STAGES) & 1);
                if (it >= STAGES && !mbar_wait(empty0 + 8 * s, ph ^ 1)) {
                    report_error(a.status, ELSI_ERR_TIMEOUT, 21);
                    atomicExch(&aborted, 1);
                    break;
                }
                if (*(volatile int *)&aborted) break;
                const int tile = (int)(g / a.nk), kt = (int)(g % a.nk);
                unsigned char *st = smem + s * STAGE_BYTES;
                const unsigned full = full0 + 8 * s;
                mbar_expect_tx(full, A_BYTES + 2 * B_BYTES);
                tma_load_2d(smem_u32(st), &maps.a, full, kt * BK, tile * BM);
                tma_load_2d(smem_u32(st + 2 * A_BYTES), &maps.v_hi, full, kt * BK, 0);
                tma_load_2d(smem_u32(st + 2 * A_BYTES + B_BYTES), &maps.v_lo, full, kt * BK, 0);
                armed = it + 1;
            }
        }
    } else if (warp >= 2 && warp < 2 + SPLIT_WARPS) {
        const int t = tid - 64;  // 0 .. 127
        long long it = 0;
        for (long long g = beg; g < end; ++g, ++it) {
            const int s = (int)(it % STAGES);
            const bool ok = __all_sync(0xffffffffu, mbar_wait(full0 + 8 * s, (unsigned)((it / STAGES) & 1)));
            if (!ok) {
                if (lane == 0) {
                    report_error(a.status, ELSI_ERR_TIMEOUT, 22);
                    atomicExch(&aborted, 1);
                }
                break;
            }
            float4 *hi = reinterpret_cast<float4 *>(smem + s * STAGE_BYTES);
            float4 *lo = reinterpret_cast<float4 *>(smem + s * STAGE_BYTES + A_BYTES);
#pragma unroll
            for (int e = t; e < A_BYTES / 16; e += 32 * SPLIT_WARPS) {
                const float4 x = hi[e];
                float4 h, l;
                split_tf32(x.x, h.x, l.x);
                split_tf32(x.y, h.y, l.y);
                split_tf32(x.z, h.z, l.z);
                split_tf32(x.w, h.w, l.w);
                hi[e] = h;
                lo[e] = l;
            }
            // the tensor cores read shared memory through the async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(ready0 + 8 * s);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const unsigned idesc = idesc_f32acc(2, BM, BN);
            long long it = 0, gch = 0;
            for (long long g = beg; g < end; ++g, ++it) {
                const int s = (int)(it % STAGES);
                const long long tile = g / a.nk, kt = g % a.nk;
                const long long seg0 = tile * a.nk > beg ? tile * a.nk : beg;
                const long long p = g - seg0;
                const bool first = (p % CH) == 0;
                const bool last = (p % CH) == CH - 1 || kt == a.nk - 1 || g == end - 1;
                const int bsel = (int)(gch & 1);
                if (first && gch >= 2 && !mbar_wait(acce0 + 8 * bsel, (unsigned)(((gch >> 1) - 1) & 1))) {
                    report_error(a.status, ELSI_ERR_TIMEOUT, 23);
                    atomicExch(&aborted, 1);
                    break;
                }
                if (!mbar_wait(ready0 + 8 * s, (unsigned)((it / STAGES) & 1))) {
                    report_error(a.status, ELSI_ERR_TIMEOUT, 24);
                    atomicExch(&aborted, 1);
                    break;
                }
                tc_fence_after();
                const unsigned base = smem_u32(smem + s * STAGE_BYTES);
                const unsigned d = tmem + bsel * 2 * BN;  // hi*hi; cross terms at + BN
#pragma unroll
                for (int kk = 0; kk < BK / 8; ++kk) {
                    const unsigned off = kk * 32;  // 8 tf32 along K
                    const unsigned long long ah = sdesc(base + off), al = sdesc(base + A_BYTES + off);
                    const unsigned long long vh = sdesc(base + 2 * A_BYTES + off);
                    const unsigned long long vl = sdesc(base + 2 * A_BYTES + B_BYTES + off);
                    const unsigned acc = (first && kk == 0) ? 0u : 1u;
                    mma_tf32(d + BN, al, vh, idesc, acc);
                    mma_tf32(d + BN, ah, vl, idesc, 1u);
                    mma_tf32(d, ah, vh, idesc, acc);
                }
                mma_commit(empty0 + 8 * s);
                if (last) {
                    mma_commit(accf0 + 8 * bsel);
                    ++gch;
                }
            }
        }
    } else if (warp >= 2 + SPLIT_WARPS) {
        const int quarter = warp & 3;
        const int rl = quarter * 32 + lane;  // row within the tile
        const unsigned tl = tmem + ((unsigned)(quarter * 32) << 16);
        const long long tile0 = beg / a.nk, tile1 = (end - 1) / a.nk;
        long long gch = 0;
        bool ok = true;
        for (long long tile = tile0; tile <= tile1 && ok; ++tile) {
            const long long s0 = tile * a.nk > beg ? tile * a.nk : beg;
            const long long s1 = (tile + 1) * a.nk < end ? (tile + 1) * a.nk : end;
            const long long nch = (s1 - s0 + CH - 1) / CH;
            float acc[BN];
#pragma unroll
            for (int j = 0; j < BN; ++j) acc[j] = 0.0f;
            for (long long c = 0; c < nch; ++c, ++gch) {
                const int bsel = (int)(gch & 1);
                ok = __all_sync(0xffffffffu, mbar_wait(accf0 + 8 * bsel, (unsigned)((gch >> 1) & 1)));
                if (!ok) {
                    if (lane == 0) {
                        report_error(a.status, ELSI_ERR_TIMEOUT, 25);
                        atomicExch(&aborted, 1);
                    }
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int q = 0; q < BN / 32; ++q) {
                    float v[32];
                    const unsigned ta = tl + bsel * 2 * BN + q * 32;
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
            if (!ok) break;
            float *pt = a.part + ((size_t)blockIdx.x * a.slots + (size_t)(tile - tile0)) * TILE_ELEMS + rl;
#pragma unroll
            for (int j = 0; j < BN; ++j) pt[(size_t)j * BM] = acc[j];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (aborted && warp == 0 && lane == 0) {
        // bounded wait for this CTA's own TMA copies still in flight
        for (long long it = (armed > STAGES ? armed - STAGES : 0); it < armed; ++it)
            mbar_wait(full0 + 8 * (int)(it % STAGES), (unsigned)((it / STAGES) & 1));
    }
    __syncthreads();
    if (warp == 6) tmem_free(tmem, TMEM_COLS);
}

// X(r, c) = sum of the partials of tile r / 128 over the CTAs whose ranges touch it, in
// CTA order; r < m, c < nv.
__global__ void symm_tall_reduce_kernel(int m, int nv, int nk, long long T, int G, int slots,
                                        const float *__restrict__ part, float *__restrict__ X, int ldx)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
    if (r >= m || c >= nv) return;
    const long long tile = r / BM;
    const long long g0 = tile * nk, g1 = ((tile + 1) * nk < T ? (tile + 1) * nk : T) - 1;
    // CTA of step g: the largest cta with range_begin(cta) <= g
    const long long c0 = ((g0 + 1) * G - 1) / T, c1 = ((g1 + 1) * G - 1) / T;
    float sum = 0.0f;
    for (long long cta = c0; cta <= c1; ++cta) {
        const long long j = tile - (cta * T / G) / nk;
        sum += part[((size_t)cta * slots + (size_t)j) * TILE_ELEMS + (size_t)c * BM + (r % BM)];
    }
    X[(size_t)r + (size_t)c * ldx] = sum;
}

__global__ void split_panel_kernel(int nv, int m, int kp, const float *__restrict__ V, int ldv,
                                   float *__restrict__ hi, float *__restrict__ lo)
{
    // plane row c (column c of V), K index q: contiguous in q on both sides
    const int c = blockIdx.y;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kp; q += gridDim.x * blockDim.x) {
        const float x = (q < m) ? V[(size_t)q + (size_t)c * ldv] : 0.0f;
        float h, l;
        split_tf32(x, h, l);
        hi[(size_t)c * kp + q] = h;
        lo[(size_t)c * kp + q] = l;
    }
}

}  // namespace symv

// G CTAs with ranges of at most ceil(T / G) steps write G * slots <= tiles_m + 3 G partial
// tiles; the scratch is sized for G = min(T, kMaxSms).
constexpr int kMaxSms = 256;

size_t symm_tall_work_elems(int m)
{
    using namespace symv;
    const int kp = ((m + BK - 1) / BK) * BK;
    const long long tiles_m = (m + BM - 1) / BM, T = tiles_m * (kp / BK);
    const long long G = kMaxSms < T ? kMaxSms : T;
    return 2 * (size_t)BN * kp + (size_t)(tiles_m + 3 * G) * TILE_ELEMS + 64;
}

cudaError_t symm_tall_f32(cudaStream_t st, int m, int nv, const float *A, int lda, const float *V,
                          int ldv, float *X, int ldx, float *work, size_t work_elems, int *status)
{
    using namespace symv;
    if (m <= 0 || nv <= 0) return cudaSuccess;
    if (nv > BN || ((size_t)A & 15) || (lda % 4) != 0 || ((size_t)work & 15) || lda < m || ldv < m || ldx < m)
        return cudaErrorNotSupported;
    static int sms[kMaxDevices] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int nsm = (dev >= 0 && dev < kMaxDevices) ? sms[dev] : 0;
    if (nsm <= 0) {
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
        if (nsm > kMaxSms) nsm = kMaxSms;
        if (dev >= 0 && dev < kMaxDevices) sms[dev] = nsm;
    }
    const int kp = ((m + BK - 1) / BK) * BK;
    Args a;
    a.m = m;
    a.nk = kp / BK;
    a.T = (long long)((m + BM - 1) / BM) * a.nk;
    a.G = (int)(nsm < a.T ? nsm : a.T);
    a.slots = (int)((a.T + a.G - 1) / a.G / a.nk + 2);
    a.status = status;
    if (work_elems < symm_tall_work_elems(m) ||
        (long long)a.G * a.slots > (a.T / a.nk) + 3ll * a.G)
        return cudaErrorNotSupported;
    float *vhi = work, *vlo = vhi + (size_t)BN * kp;
    a.part = vlo + (size_t)BN * kp;  // 2 BN kp floats: 16-byte aligned
    Maps maps;
    // A as a K-major operand: inner dimension = rows of A (K), outer = columns (rows of X)
    if (!make_map_2d(&maps.a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, A, m, m, lda, BK, BM) ||
        !make_map_2d(&maps.v_hi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, vhi, BN, kp, kp, BK, BN) ||
        !make_map_2d(&maps.v_lo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, vlo, BN, kp, kp, BK, BN))
        return cudaErrorNotSupported;
    static PerDeviceOnce attr_once;
    cudaError_t e = once_per_device(attr_once, [] {
        return cudaFuncSetAttribute(symm_tall_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    });
    if (e != cudaSuccess) return e;
    // V planes: rows nv .. BN - 1 zero
    if ((e = cudaMemsetAsync(vhi, 0, sizeof(float) * 2 * (size_t)BN * kp, st)) != cudaSuccess) return e;
    EGB_COUNT_LAUNCH();
    split_panel_kernel<<<dim3(ceil_div(kp, 256) < 64 ? ceil_div(kp, 256) : 64, nv), 256, 0, st>>>(
        nv, m, kp, V, ldv, vhi, vlo);
    EGB_COUNT_LAUNCH();
    symm_tall_kernel<<<a.G, THREADS, SMEM_BYTES, st>>>(maps, a);
    EGB_COUNT_LAUNCH();
    symm_tall_reduce_kernel<<<dim3(ceil_div(m, 256), nv), 256, 0, st>>>(m, nv, a.nk, a.T, a.G, a.slots,
                                                                        a.part, X, ldx);
    return cudaGetLastError();
}

}  // namespace egb

extern "C" size_t elsi_gb_symm_tall_f32_work(int m)
{
    if (m < 1) return 0;
    return egb::symm_tall_work_elems(m);
}

extern "C" int elsi_gb_symm_tall_f32(int m, int nv, const float *A, int lda, const float *V, int ldv,
                                     float *X, int ldx, float *work, size_t work_elems, int *status,
                                     void *stream)
{
    if (m < 1 || nv < 1 || nv > 64 || !A || !V || !X || !work || !status) return ELSI_ERR_ARG;
    cudaError_t e = egb::symm_tall_f32((cudaStream_t)stream, m, nv, A, lda, V, ldv, X, ldx, work,
                                       work_elems, status);
    if (e == cudaErrorNotSupported) return ELSI_ERR_ARG;
    return e == cudaSuccess ? ELSI_OK : ELSI_ERR_CUDA;
}
