// Binary64-accurate matrix products on the bf16 tensor cores (Ozaki et al.,
// "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59 (2012); the
// integer-digit form).
//
// Every row of A (and column of B) is scaled by a power of two 2^e so that its entries
// lie in (-1, 1), then cut into D signed 7-bit integer digits:
//     x = 2^e sum_{s=1..D} d_s 2^{-7s} (+ a remainder below 2^{-7D}),  |d_1| <= 128,
//     |d_s| <= 64 for s >= 2,
// each digit exactly representable in bf16. Then
//     (A B)_ij = 2^{e_i + f_j} sum_L 2^{-7L} sum_{s+t=L} (D_s^A D_t^B)_ij
// and every digit product is an exact integer. The tensor cores accumulate the products
// of one level L over chunks of 256 along K in binary32, which stays exact (the sum of
// absolute values stays below 2^24); chunk results are converted to int32 and summed
// (exact), and each level is finally scaled and added in binary64. Levels L = 2..D+1 are
// kept, which leaves a truncation error of about 2^{-7(D+1)} relative to
// max|A_i.| max|B_.j| per product term.
//
// One chunk of level L sums at most 256 (2 * 128 * 64 + (D - 2) * 64 * 64) < 9.5e6 in
// magnitude, so the int32 level sum is exact for up to 227 chunks (K = 58 112); longer
// products are cut along K into segments of kOzSegK and the segments added in binary64.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace egb {

constexpr int kOzD = 7;         // digits per operand
constexpr int kOzBits = 7;      // bits per digit
constexpr int kOzBM = 128, kOzBN = 128, kOzBK = 16;  // plane padding: rows, K
constexpr int kOzSegK = 32768;  // K per kernel launch (128 chunks of 256: int32-exact sums)

// ------------------------------------------------------------------ splitting
// The digits are those of the binary64 steps r = x 2^-e, then for s = 1..D: t = 128 r,
// d_s = rint(t), r = t - d_s (every step exact). They are formed here with integer
// operations on the bit pattern x = +-M 2^E (binary64 arithmetic is scarce on this chip):
// the running value A_s = sum_{i<=s} d_i 128^{s-i} equals rint(x 2^{7s-e}) (rounding half
// to even; 128 A_{s-1} is even, so the parity of the ties is the same), hence
// A_s = +-rne(M / 2^{e-E-7s}) and d_s = A_s - 128 A_{s-1}.

// M / 2^k rounded to nearest, ties to even (M < 2^53, k >= 0).
__device__ __forceinline__ unsigned long long rne_shift(unsigned long long M, int k)
{
    if (k == 0) return M;
    if (k > 63) return 0ull;  // M < 2^53 < 2^(k-1): below one half
    unsigned long long q = M >> k;
    const unsigned long long rem = M & ((1ull << k) - 1ull), half = 1ull << (k - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    return q;
}

// Vector v (0 <= v < V) has elements x(v, q) = src[v * sv + q * sq], q < K. Writes
// D digit planes out[s * plane + v * ldo + q] (bf16, q < Kpad, zero padded) and the
// exponent e_v (max_q |x(v, q)| = m 2^e_v, m in [0.5, 1)). Vectors V <= v < Vpad get zero
// digits. Optional per-element factor scale[q] (a diagonal matrix multiplied in before
// splitting).
__global__ void ozaki_split_kernel(int V, int Vpad, int K, int Kpad, const double *__restrict__ src,
                                   long long sv, long long sq, const double *__restrict__ scale,
                                   const double *__restrict__ scale2, __nv_bfloat16 *__restrict__ out,
                                   int ldo, size_t plane, int *__restrict__ exps)
{
    __shared__ unsigned long long red[32];
    const int v = blockIdx.x;
    if (v >= Vpad) return;
    __nv_bfloat16 *o = out + (size_t)v * ldo;
    if (v >= V) {
        for (int q = threadIdx.x; q < Kpad; q += blockDim.x)
            for (int s = 0; s < kOzD; ++s) o[(size_t)s * plane + q] = __float2bfloat16(0.0f);
        if (threadIdx.x == 0) exps[v] = 0;
        return;
    }
    const double *x = src + (size_t)v * sv;
    auto elem = [&](int q) {
        double val = x[(size_t)q * sq];
        if (scale) val *= scale[q];
        if (scale2) val *= scale2[q];
        return val;
    };
    // max |x| as the largest magnitude bit pattern (finite values order like their bits)
    unsigned long long mb = 0ull;
    for (int q = threadIdx.x; q < K; q += blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(elem(q)) & 0x7FFFFFFFFFFFFFFFull;
        mb = b > mb ? b : mb;
    }
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mb, o2);
        mb = t > mb ? t : mb;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mb;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long m = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0ull;
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o2);
            m = t > m ? t : m;
        }
        if (threadIdx.x == 0) red[0] = m;
    }
    __syncthreads();
    mb = red[0];
    // frexp exponent of the maximum: e = (bit length of M) + E
    int e = 0;
    if (mb != 0ull) {
        const int xf = (int)(mb >> 52);
        e = xf ? xf - 1022 : (64 - __clzll((long long)(mb & 0xFFFFFFFFFFFFFull))) - 1074;
    }
    if (threadIdx.x == 0) exps[v] = e;
    for (int q = threadIdx.x; q < Kpad; q += blockDim.x) {
        const unsigned long long u = (q < K) ? (unsigned long long)__double_as_longlong(elem(q)) : 0ull;
        const int xf = (int)((u >> 52) & 0x7FF);
        const unsigned long long M = xf ? ((u & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : (u & 0xFFFFFFFFFFFFFull);
        const int E = xf ? xf - 1075 : -1074;
        const bool neg = (u >> 63) != 0ull;
        long long aprev = 0;
#pragma unroll
        for (int s = 1; s <= kOzD; ++s) {
            const int k = e - E - kOzBits * s;
            long long a = 0;
            if (M != 0ull) a = (long long)(k <= 0 ? (M << (-k)) : rne_shift(M, k));
            if (neg) a = -a;
            const long long dgt = a - aprev * (1ll << kOzBits);
            aprev = a;
            o[(size_t)(s - 1) * plane + q] = __float2bfloat16(__int2float_rn((int)dgt));
        }
    }
}

// ------------------------------------------------------------------ GEMM (tcgen05)
// One CTA per 128 x 128 tile of C, 320 threads:
//   warp 0, one lane: TMA producer of the (A digit plane, B digit plane) k-tiles, 64 bf16 of
//                     K (128 bytes, 128-byte swizzle) x 128 rows each, into a STAGES ring;
//   warp 1, one lane: MMA issuer, tcgen05.mma kind::f16 (bf16 x bf16 -> fp32), M = N = 128,
//                     K = 16 per instruction;
//   warps 2..9:       epilogue, warp w owns tensor-memory lanes (rows) 32 (w mod 4) .. + 31
//                     and the tile columns 64 h .. 64 h + 63, h = (w - 2) / 4.
// Work order: levels L = D+1 down to 2 (smallest contributions first), chunks of 256 along
// K, pairs (s, L - s), k-tiles. Each chunk's sum over its pairs and k-tiles goes to one of
// two tensor-memory accumulators (columns 0..127 and 128..255): the products are integers
// and the sum stays below 2^24, so the accumulation is exact whatever its rounding. The
// epilogue converts each chunk to int32 and adds it in registers (exact); at the end of a
// level it adds alpha 2^(e_i + f_j - 7L) times the level sum to a binary64 running sum of
// the tile kept in tensor memory (columns 256..511, the two 32-bit halves of column j's
// value at 256 + 2j and 257 + 2j), and C is written once, after the last level. (Adding
// each level to C in global memory instead costs a 256 KB read-modify-write per tile and
// level, which stalls the MMA issuer once it has filled the second accumulator and
// dominates products with a short K.)
namespace oztc {
constexpr int BM = 128, BN = 128, BK = 64, STAGES = 7;
constexpr int CHUNK_TILES = 256 / BK;         // k-tiles per exact chunk
constexpr int TILE_BYTES = BM * BK * 2;       // 16 KB
constexpr int STAGE_BYTES = 2 * TILE_BYTES;   // A tile + B tile
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int TMEM_COLS = 4 * BN;  // two accumulators + the binary64 running sum
constexpr int EPI_WARPS = 8, CW = BN / 2;  // epilogue warps; columns per epilogue warp
constexpr int THREADS = 32 * (2 + EPI_WARPS);

struct Maps {
    CUtensorMap a, b;  // planes as (D * Mpad) x Kpad and (D * Npad) x Kpad bf16 matrices
};

struct Args {
    int m_real, n_real, kpad, mpad, npad, uplo, ldc;
    int kt0;     // first k-tile of this launch's K segment; kpad is the segment's end
    int digits;  // D <= kOzD: digit planes used per operand (levels 2 .. D + 1)
    const int *ea, *eb;
    double alpha, beta;
    double *C;
    int *status;
};
}  // namespace oztc

// x 2^e: a multiplication by a power of two built from its bit pattern where 2^e is a normal
// number (exact, like ldexp), ldexp elsewhere.
__device__ __forceinline__ double scale2(double x, int e)
{
    if (e >= -1022 && e <= 1023) return x * __longlong_as_double((long long)(e + 1023) << 52);
    return ldexp(x, e);
}

__global__ void __launch_bounds__(oztc::THREADS, 1)
ozaki_gemm_tc_kernel(const __grid_constant__ oztc::Maps maps, const oztc::Args a)
{
    using namespace oztc;
    using namespace tc5;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((size_t)smem_raw + 1023) & ~(size_t)1023);
    unsigned long long *bars = (unsigned long long *)(smem + STAGES * STAGE_BYTES);
    // bars: [0,S) full, [S,2S) empty, 2S+b accumulator b full, 2S+2+b accumulator b empty
    unsigned *tmem_slot = (unsigned *)(bars + 2 * STAGES + 4);
    __shared__ int aborted;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    if (m0 >= a.m_real || n0 >= a.n_real) return;
    if (a.uplo && m0 + BM - 1 < n0) return;  // tile strictly above the diagonal
    const int nkt = (a.kpad + BK - 1) / BK - a.kt0;  // k-tiles of this segment
    const int nch = (nkt + CHUNK_TILES - 1) / CHUNK_TILES;
    const unsigned full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[STAGES]);
    const unsigned accf0 = smem_u32(&bars[2 * STAGES]), acce0 = smem_u32(&bars[2 * STAGES + 2]);

    if (tid == 0) {
        for (int q = 0; q < 2 * STAGES + 2; ++q) mbar_init(smem_u32(&bars[q]), 1);
        mbar_init(acce0, EPI_WARPS);
        mbar_init(acce0 + 8, EPI_WARPS);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        aborted = 0;
    }
    if (warp == 2) tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;

    int armed = 0;
    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool stop = false;
            for (int L = a.digits + 1; L >= 2 && !stop; --L) {
                const int s_lo = max(1, L - a.digits), s_hi = min(a.digits, L - 1);
                for (int c = 0; c < nch && !stop; ++c) {
                    const int kt1 = min(nkt, (c + 1) * CHUNK_TILES);
                    for (int sa = s_lo; sa <= s_hi && !stop; ++sa)
                        for (int kt = c * CHUNK_TILES; kt < kt1; ++kt, ++it) {
                            const int st = it % STAGES;
                            if (it >= STAGES && !mbar_wait(empty0 + 8 * st, ((it / STAGES) & 1) ^ 1)) {
                                report_error(a.status, ELSI_ERR_TIMEOUT, 11);
                                atomicExch(&aborted, 1);
                                stop = true;
                                break;
                            }
                            if (*(volatile int *)&aborted) { stop = true; break; }
                            unsigned char *dst = smem + st * STAGE_BYTES;
                            const unsigned full = full0 + 8 * st;
                            mbar_expect_tx(full, STAGE_BYTES);
                            const int kx = (a.kt0 + kt) * BK;
                            tma_load_2d(smem_u32(dst), &maps.a, full, kx, (sa - 1) * a.mpad + m0);
                            tma_load_2d(smem_u32(dst + TILE_BYTES), &maps.b, full, kx,
                                        (L - sa - 1) * a.npad + n0);
                            armed = it + 1;
                        }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const unsigned idesc = idesc_f32acc(1, BM, BN);
            int it = 0, g = 0;
            bool stop = false;
            for (int L = a.digits + 1; L >= 2 && !stop; --L) {
                const int s_lo = max(1, L - a.digits), s_hi = min(a.digits, L - 1);
                for (int c = 0; c < nch && !stop; ++c, ++g) {
                    const int bsel = g & 1;
                    if (g >= 2 && !mbar_wait(acce0 + 8 * bsel, ((g >> 1) - 1) & 1)) {
                        report_error(a.status, ELSI_ERR_TIMEOUT, 12);
                        atomicExch(&aborted, 1);
                        stop = true;
                        break;
                    }
                    const unsigned d = tmem + bsel * BN;
                    const int kt1 = min(nkt, (c + 1) * CHUNK_TILES);
                    bool first = true;
                    for (int sa = s_lo; sa <= s_hi && !stop; ++sa)
                        for (int kt = c * CHUNK_TILES; kt < kt1; ++kt, ++it) {
                            const int st = it % STAGES;
                            if (!mbar_wait(full0 + 8 * st, (it / STAGES) & 1)) {
                                report_error(a.status, ELSI_ERR_TIMEOUT, 13);
                                atomicExch(&aborted, 1);
                                stop = true;
                                break;
                            }
                            tc_fence_after();
                            const unsigned base = smem_u32(smem + st * STAGE_BYTES);
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk) {
                                const unsigned off = kk * 32;  // 16 bf16 along K
                                mma_bf16(d, sdesc(base + off), sdesc(base + TILE_BYTES + off), idesc,
                                         first ? 0u : 1u);
                                first = false;
                            }
                            mma_commit(empty0 + 8 * st);
                        }
                    if (!stop) mma_commit(accf0 + 8 * bsel);
                }
            }
        }
    } else {
        // tensor-memory loads and stores are warp-collective: every lane runs them (rows past
        // m only skip their global-memory accesses) and the wait results are made uniform
        const int quarter = warp & 3, c0 = ((warp - 2) >> 2) * CW;  // rows, first column
        const int row = m0 + quarter * 32 + lane;
        const bool row_in = row < a.m_real;
        const int er = row_in ? a.ea[row] : 0;
        const unsigned tlane = tmem + ((unsigned)(quarter * 32) << 16);
        const unsigned tsum = tlane + 2 * BN + 2 * c0;
        int iacc[CW];
        bool ok = true;
        int g = 0;
        for (int L = a.digits + 1; L >= 2 && ok; --L) {
#pragma unroll
            for (int j = 0; j < CW; ++j) iacc[j] = 0;
            for (int c = 0; c < nch; ++c, ++g) {
                const int bsel = g & 1;
                ok = __all_sync(0xffffffffu, mbar_wait(accf0 + 8 * bsel, (g >> 1) & 1));
                if (!ok) {
                    if (lane == 0) {
                        report_error(a.status, ELSI_ERR_TIMEOUT, 14);
                        atomicExch(&aborted, 1);
                    }
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int q = 0; q < CW / 32; ++q) {
                    float v[32];
                    tmem_ld32(tlane + bsel * BN + c0 + q * 32, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) iacc[q * 32 + j] += __float2int_rn(v[j]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce0 + 8 * bsel);
            }
            if (!ok) break;
            // running sum += alpha 2^(e_i + f_j - 7L) level sum, 16 columns at a time
            const bool firstL = (L == a.digits + 1);
#pragma unroll
            for (int q = 0; q < CW / 16; ++q) {
                unsigned w[32];
                if (!firstL) tmem_ld32_u(tsum + q * 32, w);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + q * 16 + j;
                    const int ec = col < a.n_real ? a.eb[col] : 0;
                    const double val = a.alpha * scale2((double)iacc[q * 16 + j], er + ec - kOzBits * L);
                    const double sum = firstL ? val : __hiloint2double((int)w[2 * j + 1], (int)w[2 * j]) + val;
                    w[2 * j] = (unsigned)__double2loint(sum);
                    w[2 * j + 1] = (unsigned)__double2hiint(sum);
                }
                tmem_st32_u(tsum + q * 32, w);
            }
        }
        if (ok) {
            // C = beta C + running sum, 16 columns at a time (the loads of C first)
            double *crow = a.C + (size_t)row;
#pragma unroll 1
            for (int q = 0; q < CW / 16; ++q) {
                unsigned w[32];
                tmem_ld32_u(tsum + q * 32, w);
                double cv[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + q * 16 + j;
                    const bool in = row_in && col < a.n_real && (!a.uplo || row >= col);
                    cv[j] = (in && a.beta != 0.0) ? crow[(size_t)col * a.ldc] : 0.0;
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + q * 16 + j;
                    if (row_in && col < a.n_real && (!a.uplo || row >= col)) {
                        const double sum = __hiloint2double((int)w[2 * j + 1], (int)w[2 * j]);
                        crow[(size_t)col * a.ldc] = a.beta != 0.0 ? fma(a.beta, cv[j], sum) : sum;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (aborted && warp == 0 && lane == 0) {
        for (int it = (armed > STAGES ? armed - STAGES : 0); it < armed; ++it)
            mbar_wait(full0 + 8 * (it % STAGES), (it / STAGES) & 1);
    }
    __syncthreads();
    if (warp == 2) tmem_free(tmem, TMEM_COLS);
}

size_t ozaki_plane_elems(int V, int K)
{
    return (size_t)ceil_div(V, kOzBM) * kOzBM * (size_t)(ceil_div(K, kOzBK) * kOzBK);
}

size_t ozaki_split_elems(int V, int K) { return ozaki_plane_elems(V, K) * kOzD; }

cudaError_t ozaki_split(cudaStream_t st, int V, int K, const double *src, long long sv,
                        long long sq, const double *scale, const double *scale2,
                        __nv_bfloat16 *planes, int *exps)
{
    const int Vpad = ceil_div(V, kOzBM) * kOzBM;
    const int Kpad = ceil_div(K, kOzBK) * kOzBK;
    EGB_COUNT_LAUNCH();
    ozaki_split_kernel<<<Vpad, 256, 0, st>>>(V, Vpad, K, Kpad, src, sv, sq, scale, scale2, planes,
                                             Kpad, ozaki_plane_elems(V, K), exps);
    return cudaGetLastError();
}

cudaError_t ozaki_gemm(cudaStream_t st, int m, int n, int k, double alpha,
                       const __nv_bfloat16 *Ad, const int *ea, const __nv_bfloat16 *Bd,
                       const int *eb, double beta, double *C, int ldc, int uplo, int digits)
{
    if (digits < 1 || digits > kOzD) return cudaErrorInvalidValue;
    using namespace oztc;
    if (m <= 0 || n <= 0) return cudaSuccess;
    const int mpad = ceil_div(m, kOzBM) * kOzBM, npad = ceil_div(n, kOzBN) * kOzBN;
    const int kpad = ceil_div(k, kOzBK) * kOzBK;
    Maps maps;
    if (!tc5::make_map_2d(&maps.a, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Ad, (long long)kOzD * mpad, kpad,
                          kpad, BK, BM) ||
        !tc5::make_map_2d(&maps.b, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Bd, (long long)kOzD * npad, kpad,
                          kpad, BK, BN))
        return cudaErrorNotSupported;
    Args a;
    a.m_real = m; a.n_real = n; a.kpad = kpad; a.mpad = mpad; a.npad = npad; a.uplo = uplo;
    a.ldc = ldc; a.ea = ea; a.eb = eb; a.alpha = alpha; a.beta = beta; a.C = C;
    a.digits = digits;
    float *tw;
    size_t te;
    int *ts = nullptr;
    tc_scratch(&tw, &te, &ts);
    // a status word for calls outside a solve (one per device, kept until exit)
    static int *dummy_status[kMaxDevices] = {};
    static PerDeviceOnce once;
    cudaError_t attr_err = once_per_device(once, [] {
        int dev = 0;
        cudaError_t r = cudaGetDevice(&dev);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(ozaki_gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (r == cudaSuccess && dev >= 0 && dev < kMaxDevices && !dummy_status[dev]) {
            int *p = nullptr;
            r = cudaMalloc((void **)&p, 8 * sizeof(int));
            if (r == cudaSuccess) r = cudaMemset(p, 0, 8 * sizeof(int));
            if (r == cudaSuccess) dummy_status[dev] = p;
        }
        return r;
    });
    if (attr_err != cudaSuccess) return attr_err;
    int dev_now = 0;
    cudaGetDevice(&dev_now);
    a.status = ts ? ts : (dev_now >= 0 && dev_now < kMaxDevices ? dummy_status[dev_now] : nullptr);
    if (!a.status) return cudaErrorInvalidDevice;
    dim3 grid(mpad / BM, npad / BN);
    // K segments of kOzSegK (a multiple of BK): the first applies beta, the rest add
    for (int k0 = 0; k0 < kpad; k0 += kOzSegK) {
        a.kt0 = k0 / BK;
        a.kpad = min(kpad, k0 + kOzSegK);
        a.beta = k0 == 0 ? beta : 1.0;
        EGB_COUNT_LAUNCH();
        ozaki_gemm_tc_kernel<<<grid, THREADS, SMEM_BYTES, st>>>(maps, a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace egb
