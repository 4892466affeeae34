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
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace egb {

constexpr int kOzD = 7;         // digits per operand
constexpr int kOzBits = 7;      // bits per digit
constexpr int kOzBM = 128, kOzBN = 128, kOzBK = 16;
constexpr int kOzStages = 3;
constexpr int kOzChunkSteps = 16;  // k16 steps per exact binary32 chunk (256 along K)

// ------------------------------------------------------------------ splitting
// Vector v (0 <= v < V) has elements x(v, q) = src[v * sv + q * sq], q < K. Writes
// D digit planes out[s * plane + v * ldo + q] (bf16, q < Kpad, zero padded) and the
// exponent e_v. Vectors V <= v < Vpad get zero digits. Optional per-element factor
// scale[q] (a diagonal matrix multiplied in before splitting).
__global__ void ozaki_split_kernel(int V, int Vpad, int K, int Kpad, const double *__restrict__ src,
                                   long long sv, long long sq, const double *__restrict__ scale,
                                   const double *__restrict__ scale2, __nv_bfloat16 *__restrict__ out,
                                   int ldo, size_t plane, int *__restrict__ exps)
{
    __shared__ double red[32];
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
    double mx = 0.0;
    for (int q = threadIdx.x; q < K; q += blockDim.x) mx = fmax(mx, fabs(elem(q)));
    for (int o2 = 16; o2 > 0; o2 >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o2));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        double m = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o2 = 16; o2 > 0; o2 >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o2));
        if (threadIdx.x == 0) red[0] = m;
    }
    __syncthreads();
    mx = red[0];
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx = m 2^e, m in [0.5, 1): |x| 2^-e < 1
    if (threadIdx.x == 0) exps[v] = e;
    for (int q = threadIdx.x; q < Kpad; q += blockDim.x) {
        double r = (q < K) ? ldexp(elem(q), -e) : 0.0;
#pragma unroll
        for (int s = 0; s < kOzD; ++s) {
            double t = r * (double)(1 << kOzBits);
            double dgt = rint(t);
            r = t - dgt;
            o[(size_t)s * plane + q] = __float2bfloat16((float)dgt);
        }
    }
}

// ------------------------------------------------------------------ GEMM
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(unsigned dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2,
                                            unsigned &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float *c, const unsigned *a, unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared tile: 128 rows x 16 bf16 (32 bytes = two 16-byte chunks per row). Chunk c of row
// r is stored at chunk c ^ ((r >> 2) & 1): the 8 row addresses of every ldmatrix 8x8
// matrix then hit distinct banks.
__device__ __forceinline__ int tile_off(int r, int c) { return r * 32 + ((c ^ ((r >> 2) & 1)) << 4); }

struct OzArgs {
    int M, N, Kpad;                 // padded sizes: M, N multiples of 128, Kpad of 16
    const __nv_bfloat16 *A;         // planes [D][M][Kpad]
    size_t a_plane;
    const int *ea;                  // M
    const __nv_bfloat16 *B;         // planes [D][N][Kpad]
    size_t b_plane;
    const int *eb;                  // N
    double alpha, beta;
    double *C;                      // m_real x n_real, ldc
    int ldc, m_real, n_real, uplo;
};

// C = alpha * A B + beta * C for the 128 x 128 tile of this CTA; 8 warps (2 x 4), warp tile
// 64 x 32; one pass over K per level L.
__global__ void __launch_bounds__(256) ozaki_gemm_kernel(OzArgs a)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const int m0 = blockIdx.x * kOzBM, n0 = blockIdx.y * kOzBN;
    if (m0 >= a.m_real || n0 >= a.n_real) return;
    if (a.uplo == 1 && m0 + kOzBM - 1 < n0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;
    const int tile_bytes = kOzBM * kOzBK * 2;  // 4096
    const int nks = a.Kpad / kOzBK;

    for (int L = kOzD + 1; L >= 2; --L) {
        const int s_lo = max(1, L - kOzD), s_hi = min(kOzD, L - 1);
        const int np = s_hi - s_lo + 1;                 // pairs (s, L - s)
        const int stage_bytes = 2 * np * tile_bytes;    // A planes s_lo..s_hi, B planes L-s_hi..L-s_lo
        float acc[4][4][4];
        int iacc[4][4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) { acc[i][j][q] = 0.f; iacc[i][j][q] = 0; }

        auto load_stage = [&](int ks, int stage) {
            unsigned base = smem_u32(sm) + stage * stage_bytes;
            const int kq = ks * kOzBK;
            // 2*np tiles x 128 rows x 2 chunks
            const int chunks = 2 * np * kOzBM * 2;
            for (int c = tid; c < chunks; c += 256) {
                int tile = c / (kOzBM * 2);
                int rem = c % (kOzBM * 2);
                int r = rem >> 1, ch = rem & 1;
                const __nv_bfloat16 *src;
                if (tile < np) {
                    int s = s_lo + tile;
                    src = a.A + (size_t)(s - 1) * a.a_plane + (size_t)(m0 + r) * a.Kpad + kq + ch * 8;
                } else {
                    int s = s_lo + (tile - np);
                    int t = L - s;
                    src = a.B + (size_t)(t - 1) * a.b_plane + (size_t)(n0 + r) * a.Kpad + kq + ch * 8;
                }
                cp_async16(base + tile * tile_bytes + tile_off(r, ch), src);
            }
        };

#pragma unroll
        for (int st = 0; st < kOzStages - 1; ++st) {
            if (st < nks) load_stage(st, st);
            cp_async_commit();
        }
        for (int ks = 0; ks < nks; ++ks) {
            cp_async_wait<kOzStages - 2>();
            __syncthreads();
            {
                int nxt = ks + kOzStages - 1;
                if (nxt < nks) load_stage(nxt, nxt % kOzStages);
                cp_async_commit();
            }
            const unsigned base = smem_u32(sm) + (ks % kOzStages) * stage_bytes;
            for (int p = 0; p < np; ++p) {
                const unsigned at = base + p * tile_bytes;          // A plane s_lo + p
                const unsigned bt = base + (np + p) * tile_bytes;   // B plane L - (s_lo + p)
                unsigned af[4][4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    int r = wm + i * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                    int ch = lane >> 4;
                    ldmatrix_x4(at + tile_off(r, ch), af[i][0], af[i][1], af[i][2], af[i][3]);
                }
                unsigned bf[4][2];
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) {
                    int r = wn + jj * 16 + (lane & 7) + (lane >> 4) * 8;
                    int ch = (lane >> 3) & 1;
                    unsigned r0, r1, r2, r3;
                    ldmatrix_x4(bt + tile_off(r, ch), r0, r1, r2, r3);
                    bf[jj * 2][0] = r0; bf[jj * 2][1] = r1;
                    bf[jj * 2 + 1][0] = r2; bf[jj * 2 + 1][1] = r3;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j][0], bf[j][1]);
            }
            if ((ks + 1) % kOzChunkSteps == 0 || ks == nks - 1) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            iacc[i][j][q] += __float2int_rn(acc[i][j][q]);
                            acc[i][j][q] = 0.f;
                        }
            }
        }
        cp_async_wait<0>();
        __syncthreads();
        // level epilogue: C (+)= alpha 2^(e_i + f_j - 7L) iacc
        const bool first = (L == kOzD + 1);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int r = m0 + wm + i * 16 + (lane >> 2) + (q >> 1) * 8;
                    int c = n0 + wn + j * 8 + (lane & 3) * 2 + (q & 1);
                    if (r >= a.m_real || c >= a.n_real) continue;
                    if (a.uplo == 1 && r < c) continue;
                    double val = a.alpha * ldexp((double)iacc[i][j][q], a.ea[r] + a.eb[c] - kOzBits * L);
                    double *cp = a.C + (size_t)r + (size_t)c * a.ldc;
                    if (first) *cp = (a.beta == 0.0) ? val : fma(a.beta, *cp, val);
                    else *cp += val;
                }
    }
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
                       const int *eb, double beta, double *C, int ldc, int uplo)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    OzArgs a;
    a.M = ceil_div(m, kOzBM) * kOzBM;
    a.N = ceil_div(n, kOzBN) * kOzBN;
    a.Kpad = ceil_div(k, kOzBK) * kOzBK;
    a.A = Ad; a.a_plane = ozaki_plane_elems(m, k); a.ea = ea;
    a.B = Bd; a.b_plane = ozaki_plane_elems(n, k); a.eb = eb;
    a.alpha = alpha; a.beta = beta; a.C = C; a.ldc = ldc; a.m_real = m; a.n_real = n; a.uplo = uplo;
    const size_t smem = (size_t)kOzStages * 2 * kOzD * kOzBM * kOzBK * 2;  // 172032
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(ozaki_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid(a.M / kOzBM, a.N / kOzBN);
    EGB_COUNT_LAUNCH();
    ozaki_gemm_kernel<<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace egb
