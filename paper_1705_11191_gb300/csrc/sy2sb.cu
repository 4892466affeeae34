// Full -> band reduction B = Q1^T H~ Q1 (arXiv:1705.11191 Eq. 11, first line; step (1)
// of the two-stage tridiagonalisation in sec. 3.1).
//
// Panel p (columns [p*b, p*b+b), rows [p*b+b, n)) is factorised by blocked Householder
// QR (compact-WY form Q_p = I - V T V^T); then the trailing symmetric matrix gets the
// two-sided update A22 <- Q_p^T A22 Q_p = A22 - V W^T - W V^T with
// X = A22 V T and W = X - (1/2) V (T^T (V^T X)).
//
// The panel QR is one cooperative launch: the m x b panel is split by rows over G CTAs,
// each holding its rows in shared memory; one grid barrier per column exchanges the
// partial norm and the partial products of the column with the remaining columns. The
// trailing update is GEMM work.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace egb {

struct PanelArgs {
    int m, bw, rows_per_cta;
    int lda, ldv;
    unsigned *count;         // grid barrier counter (zeroed before the launch)
    double *part;            // 2 x gstride partial norms (by column parity)
    double *alpha;           // 2 x 64: row j of the panel (by column parity)
    double *wpart;           // 2 x gstride x 64 partial dot products (by column parity)
    int gstride;             // >= G
    double *gram;            // scratch of the W kernels (not used by the panel kernel)
    int *status;
    long long spin_limit;    // polls of a grid-barrier wait before ELSI_ERR_TIMEOUT
};

template <typename T>
__global__ void __launch_bounds__(256) panel_qr_kernel(T *P, T *V, T *Tm, int ldt, PanelArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    const int bw = a.bw, bwp = bw + 1;
    const int R = a.rows_per_cta;
    T *Ploc = reinterpret_cast<T *>(smem_raw);          // R x bwp, row-major
    __shared__ double red[32];
    __shared__ double tau_s[64];
    __shared__ double wsum[64];
    __shared__ double colpart[4][64];
    __shared__ double prow_s[64];  // row j of the panel (published by the CTA holding it)
    __shared__ double refl[3];  // beta, tau, 1 / (alpha - beta) of the current column
    const int g = blockIdx.x, G = gridDim.x;
    const int tid = threadIdx.x;
    const int row0 = g * R;
    const int nrow = max(0, min(a.m - row0, R));
    const int tc = tid & 63, tr = tid >> 6;  // 64 column lanes x 4 row lanes
    // T of the compact-WY form, column by column (CTA 0), after the panel rows
    double *tloc = reinterpret_cast<double *>(smem_raw + (((size_t)R * bwp * sizeof(T) + 15) & ~(size_t)15));

    // the panel rows of this CTA, 16 loads of a thread in flight at a time
    for (int e0 = 0; e0 < R * bw; e0 += 16 * 256) {
        T v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int e = e0 + u * 256 + tid, i = e % R, c = e / R;
            v[u] = (e < R * bw && i < nrow) ? P[(size_t)(row0 + i) + (size_t)c * a.lda] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int e = e0 + u * 256 + tid, i = e % R, c = e / R;
            if (e < R * bw) Ploc[i * bwp + c] = v[u];
        }
    }
    if (g == 0)
        for (int e = tid; e < 64 * 64; e += blockDim.x) tloc[e] = 0.0;
    __syncthreads();
    // sum over the rows gi >= first (gi = row0 + i, i = tr, tr + 4, ...) of x_i Ploc[i][c],
    // x_i = Ploc[i][col] (1 at gi == col when unit): four independent partial sums
    auto col_dot = [&](int c, int col, int first, bool unit) -> T {
        auto xv = [&](int i) -> T {
            const int gi = row0 + i;
            return gi < first ? T(0) : ((unit && gi == col) ? T(1) : Ploc[i * bwp + col]);
        };
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        int i = tr;
        for (; i + 12 < nrow; i += 16) {
            s0 = fma(xv(i), Ploc[i * bwp + c], s0);
            s1 = fma(xv(i + 4), Ploc[(i + 4) * bwp + c], s1);
            s2 = fma(xv(i + 8), Ploc[(i + 8) * bwp + c], s2);
            s3 = fma(xv(i + 12), Ploc[(i + 12) * bwp + c], s3);
        }
        for (; i < nrow; i += 4) s0 = fma(xv(i), Ploc[i * bwp + c], s0);
        return (s0 + s1) + (s2 + s3);
    };

    const int nref = min(bw, a.m);
    // One grid barrier per column. Before it, every CTA publishes (for column j, already
    // updated by reflectors 0..j-1) the partial sum of squares below the diagonal and the
    // unscaled partial dot products d_c = sum_{i>j} x_i P[i][c] (c > j); the CTA holding
    // row j publishes that row. After it, every CTA forms the same reflector
    // v = [1; x scl] and w_c = v . P_c = P[j][c] + scl d_c, and updates its rows. The
    // published values alternate between two buffers by column parity: a CTA can be at
    // most one column ahead of another. The free slots c < j - 1 of the same exchange
    // carry the partial Gram column G[c][j-1] = v_c . v_(j-1) of the finished reflectors,
    // from which CTA 0 forms column j - 1 of T (forward recurrence) while the others
    // update their rows.
    for (int j = 0; j < nref; ++j) {
        const int par = j & 1;
        double *part = a.part + (size_t)par * a.gstride;              // [G]
        double *dpart = a.wpart + (size_t)par * a.gstride * 64;       // [G][64]
        double *prow = a.alpha + par * 64;                            // [64]
        {
            T ss = T(0), s = T(0);
            const int c = tc;
            for (int i = tid; i < nrow; i += blockDim.x)
                if (row0 + i > j) { T x = Ploc[i * bwp + j]; ss = fma(x, x, ss); }
            if (c > j && c < bw) s = col_dot(c, j, j + 1, false);
            // v_c . v_(j-1) over the rows >= j - 1 (v_c is zero above c)
            if (c < j - 1) s = col_dot(c, j - 1, j - 1, true);
            colpart[tr][tc] = (double)s;
            double sst = block_sum((double)ss, red);  // also orders colpart
            if (tid < bw)
                dpart[(size_t)g * 64 + tid] = colpart[0][tid] + colpart[1][tid] + colpart[2][tid] + colpart[3][tid];
            if (tid == 0) part[g] = sst;
            if (j >= row0 && j < row0 + nrow && tid >= j && tid < bw)
                prow[tid] = (double)Ploc[(j - row0) * bwp + tid];
        }
        if (!grid_barrier(a.count, (unsigned)G * (unsigned)(j + 1), a.status, a.spin_limit)) return;
        // ---- reflector of column j (every CTA computes the same numbers)
        {
            // sigma2 by warp 0; d_c by 64 column lanes x 4 row groups of CTAs
            if (tid < 32) {
                double v = 0.0;
                for (int q = tid; q < G; q += 32) v += __ldcg(part + q);
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (tid == 0) red[0] = v;
            }
            // L2-coherent loads (written by other CTAs before the barrier), all issued
            // before they are summed
            // (up to 64 CTAs: all 16 loads of a thread in flight at once)
            // row j entries c >= j, loaded with the partials (one round trip for both)
            const double pv = (tid >= j && tid < bw) ? __ldcg(prow + tid) : 0.0;
            double dv = 0.0;
            if ((tc > j && tc < bw) || tc < j - 1) {
                double acc[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int q = tr + 4 * u;
                    acc[u] = (q < G) ? __ldcg(dpart + (size_t)q * 64 + tc) : 0.0;
                }
                for (int q = tr + 64; q < G; q += 4) acc[0] += __ldcg(dpart + (size_t)q * 64 + tc);
#pragma unroll
                for (int h = 8; h > 0; h >>= 1)
#pragma unroll
                    for (int u = 0; u < h; ++u) acc[u] += acc[u + h];
                dv = acc[0];
            }
            colpart[tr][tc] = dv;
            if (tid < bw) prow_s[tid] = pv;
            __syncthreads();
            if (tid < bw) wsum[tid] = colpart[0][tid] + colpart[1][tid] + colpart[2][tid] + colpart[3][tid];
            // the reflector's scalars, once, in the panel's precision (one thread's
            // binary64 square root and two divisions per column cost microseconds on this
            // chip, whose binary64 units are few)
            if (tid == 0) {
                const T sigma2 = (T)red[0];
                const T alpha = (T)prow_s[j];
                if (sigma2 == T(0)) { refl[0] = (double)alpha; refl[1] = 0.0; refl[2] = 0.0; }
                else {
                    const T nrm = dsqrt<T>(fma(alpha, alpha, sigma2));
                    const T bt = (alpha >= T(0)) ? -nrm : nrm;
                    refl[0] = (double)bt;
                    refl[1] = (double)((bt - alpha) / bt);
                    refl[2] = (double)(T(1) / (alpha - bt));
                }
            }
            __syncthreads();
        }
        const double beta = refl[0], tau = refl[1], scl = refl[2];
        // column j - 1 of T: T[c][j-1] = -tau_(j-1) sum_(c <= q < j-1) T[c][q] G[q][j-1]
        if (g == 0 && j >= 1) {
            if (tid < j - 1) {
                double acc = 0.0;
                for (int q = tid; q < j - 1; ++q) acc += tloc[tid + q * 64] * wsum[q];
                tloc[tid + (j - 1) * 64] = -tau_s[j - 1] * acc;
            }
            if (tid == 0) tloc[(j - 1) + (j - 1) * 64] = tau_s[j - 1];
            __syncthreads();
        }
        // w_c = P[j][c] + scl d_c; stored pre-multiplied by tau
        if (tid > j && tid < bw) wsum[tid] = tau * (prow_s[tid] + scl * wsum[tid]);
        __syncthreads();
        const T sclT = (T)scl;
        for (int i = tid; i < nrow; i += blockDim.x)
            if (row0 + i > j) Ploc[i * bwp + j] = Ploc[i * bwp + j] * sclT;
        __syncthreads();
        {
            const int c = tc;
            if (c > j && c < bw) {
                const T wt = (T)wsum[c];
#pragma unroll 4
                for (int i = tr; i < nrow; i += 4) {
                    const int gi = row0 + i;
                    if (gi >= j) {
                        const T v = (gi == j) ? T(1) : Ploc[i * bwp + j];
                        Ploc[i * bwp + c] = fma(-v, wt, Ploc[i * bwp + c]);
                    }
                }
            }
        }
        if (tid == 0) tau_s[j] = tau;
        __syncthreads();
        if (tid == 0 && j >= row0 && j < row0 + nrow) Ploc[(j - row0) * bwp + j] = (T)beta;
        __syncthreads();
    }
    if (tid == 0)
        for (int j = nref; j < bw; ++j) tau_s[j] = 0.0;
    __syncthreads();

    // ---- write back the panel (R on/above the diagonal, reflector tails below) and the
    //      explicit V (unit diagonal, zeros above) for the GEMM updates
    for (int e = tid; e < nrow * bw; e += blockDim.x) {
        int i = e % nrow, c = e / nrow;
        int gi = row0 + i;
        T pv = Ploc[i * bwp + c];
        P[(size_t)gi + (size_t)c * a.lda] = pv;
        T vv = (c >= nref) ? T(0) : ((gi > c) ? pv : ((gi == c) ? T(1) : T(0)));
        V[(size_t)gi + (size_t)c * a.ldv] = vv;
    }
    // ---- the last column of T: partial Gram column G[c][nref-1] (c < nref - 1) through the
    //      buffer of the next parity, one more barrier, then CTA 0 sums and finishes T
    const int jl = nref - 1;
    {
        double *dpart = a.wpart + (size_t)(nref & 1) * a.gstride * 64;
        const T s = (tc < jl) ? col_dot(tc, jl, jl, true) : T(0);
        colpart[tr][tc] = (double)s;
        __syncthreads();
        if (tid < bw) dpart[(size_t)g * 64 + tid] = colpart[0][tid] + colpart[1][tid] + colpart[2][tid] + colpart[3][tid];
    }
    if (!grid_barrier(a.count, (unsigned)G * (unsigned)(nref + 1), a.status, a.spin_limit)) return;
    if (g != 0) return;
    {
        const double *dpart = a.wpart + (size_t)(nref & 1) * a.gstride * 64;
        double dv = 0.0;
        if (tc < jl) {
            double acc[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int q = tr + 4 * u;
                acc[u] = (q < G) ? __ldcg(dpart + (size_t)q * 64 + tc) : 0.0;
            }
            for (int q = tr + 64; q < G; q += 4) acc[0] += __ldcg(dpart + (size_t)q * 64 + tc);
#pragma unroll
            for (int h = 8; h > 0; h >>= 1)
#pragma unroll
                for (int u = 0; u < h; ++u) acc[u] += acc[u + h];
            dv = acc[0];
        }
        colpart[tr][tc] = dv;
        __syncthreads();
        if (tid < bw) wsum[tid] = colpart[0][tid] + colpart[1][tid] + colpart[2][tid] + colpart[3][tid];
        __syncthreads();
        if (tid < jl) {
            double acc = 0.0;
            for (int q = tid; q < jl; ++q) acc += tloc[tid + q * 64] * wsum[q];
            tloc[tid + jl * 64] = -tau_s[jl] * acc;
        }
        if (tid == 0) tloc[jl + jl * 64] = tau_s[jl];
        __syncthreads();
    }
    for (int e = tid; e < bw * bw; e += blockDim.x) {
        int r = e % bw, c = e / bw;
        Tm[(size_t)r + (size_t)c * ldt] = (T)tloc[r + c * 64];
    }
}

// ---- W of the two-sided update, fused (three small launches instead of five GEMMs):
//   X = (A22 V) T,  Y = V^T X,  Z = T^T Y,  W = X - (1/2) V Z.
// Row blocks of kWRows rows; tiles of 64 x 64 (bw <= 64, zero padded) in shared memory,
// each of the 256 threads computing a 4 x 4 block of a tile product.
constexpr int kWRows = 64;
constexpr int kWLd = 65;

// c[4][4] = sum_k A[r0 + i][k] B[k][c0 + j] for tiles A (64 x kWLd), B (64 x kWLd)
template <typename T>
__device__ __forceinline__ void tile_mm(const T *A, const T *B, int kmax, T (&c)[4][4])
{
    const int tr = (threadIdx.x >> 4) * 4, tc = (threadIdx.x & 15) * 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) c[i][j] = T(0);
    for (int k = 0; k < kmax; ++k) {
        T a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = A[(tr + i) * kWLd + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = B[k * kWLd + tc + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) c[i][j] = fma(a[i], b[j], c[i][j]);
    }
}

// A 64 x 64 tile from global memory, element (i, c) = ld(i, c) stored by st(i, c, value):
// 16 elements per thread (256 threads), all loads in flight before the first store.
template <typename T, typename Ld, typename St>
__device__ __forceinline__ void tile_in(Ld ld, St st)
{
    T v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int e = threadIdx.x + 256 * u;
        v[u] = ld(e & 63, e >> 6);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int e = threadIdx.x + 256 * u;
        st(e & 63, e >> 6, v[u]);
    }
}

// tile[i][c] = src[(r0 + i) + c * ld] for i < rows, c < bw; zero elsewhere
template <typename T>
__device__ __forceinline__ void load_rows(T *tile, const T *src, int ld, int r0, int rows, int bw)
{
    tile_in<T>([&](int i, int c) { return (i < rows && c < bw) ? src[(size_t)(r0 + i) + (size_t)c * ld] : T(0); },
               [&](int i, int c, T x) { tile[i * kWLd + c] = x; });
}

// X rows = Xa rows T; partial Y (64 x 64 per block, column-major) = V rows^T X rows
template <typename T>
__global__ void __launch_bounds__(256) w_stage1_kernel(int m, int bw, const T *xa, const T *V, int ldv,
                                                       const T *Tm, int ldt, T *X, T *ypart)
{
    extern __shared__ unsigned char wsm_raw[];
    T *sT = reinterpret_cast<T *>(wsm_raw), *sA = sT + 64 * kWLd, *sX = sA + 64 * kWLd;
    const int r0 = blockIdx.x * kWRows, rows = min(kWRows, m - r0);
    load_rows(sT, Tm, ldt, 0, bw, bw);
    load_rows(sA, xa, m, r0, rows, bw);
    __syncthreads();
    T c[4][4];
    tile_mm(sA, sT, bw, c);
    const int tr = (threadIdx.x >> 4) * 4, tc = (threadIdx.x & 15) * 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            sX[(tr + i) * kWLd + tc + j] = c[i][j];
            if (tr + i < rows && tc + j < bw) X[(size_t)(r0 + tr + i) + (size_t)(tc + j) * m] = c[i][j];
        }
    __syncthreads();
    // V rows transposed into sA: sA[a][i] = V[r0 + i][a]
    tile_in<T>([&](int i, int a) { return (i < rows && a < bw) ? V[(size_t)(r0 + i) + (size_t)a * ldv] : T(0); },
               [&](int i, int a, T x) { sA[a * kWLd + i] = x; });
    __syncthreads();
    tile_mm(sA, sX, kWRows, c);
    T *yp = ypart + (size_t)blockIdx.x * 64 * 64;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) yp[(tr + i) + (tc + j) * 64] = c[i][j];
}

// Y[e] = sum over blocks g of ypart[g][e] (e < 64 * 64, ascending g)
template <typename T>
__global__ void w_stage2_kernel(int nblk, const T *ypart, T *Y)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 64 * 64) return;
    T s = T(0);
    int g = 0;
    for (; g + 8 <= nblk; g += 8) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = ypart[(size_t)(g + u) * 64 * 64 + e];
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; g < nblk; ++g) s += ypart[(size_t)g * 64 * 64 + e];
    Y[e] = s;
}

// Z = T^T Y (every block, in shared memory); W rows = X rows - (1/2) V rows Z
template <typename T>
__global__ void __launch_bounds__(256) w_stage3_kernel(int m, int bw, const T *X, const T *V, int ldv,
                                                       const T *Tm, int ldt, const T *Y, T *W)
{
    extern __shared__ unsigned char wsm_raw[];
    T *sA = reinterpret_cast<T *>(wsm_raw), *sB = sA + 64 * kWLd, *sZ = sB + 64 * kWLd;
    const int r0 = blockIdx.x * kWRows, rows = min(kWRows, m - r0);
    // sA = T^T (sA[a][k] = T[k][a]), sB = Y
    tile_in<T>([&](int i, int c) { return (i < bw && c < bw) ? Tm[(size_t)i + (size_t)c * ldt] : T(0); },
               [&](int i, int c, T x) { sA[c * kWLd + i] = x; });
    tile_in<T>([&](int i, int c) { return Y[i + c * 64]; }, [&](int i, int c, T x) { sB[i * kWLd + c] = x; });
    __syncthreads();
    T c[4][4];
    tile_mm(sA, sB, bw, c);
    const int tr = (threadIdx.x >> 4) * 4, tc = (threadIdx.x & 15) * 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sZ[(tr + i) * kWLd + tc + j] = c[i][j];
    __syncthreads();
    load_rows(sA, V, ldv, r0, rows, bw);
    __syncthreads();
    tile_mm(sA, sZ, bw, c);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (tr + i < rows && tc + j < bw) {
                const size_t q = (size_t)(r0 + tr + i) + (size_t)(tc + j) * m;
                W[q] = X[q] - T(0.5) * c[i][j];
            }
}

template <typename T>
static cudaError_t form_w(cudaStream_t st, int m, int bw, const T *xa, const T *V, int ldv,
                          const T *Tm, int ldt, T *X, T *Y, T *W, T *ypart)
{
    const int nblk = ceil_div(m, kWRows);
    const size_t smem = (size_t)3 * 64 * kWLd * sizeof(T);
    static PerDeviceOnce attr;  // per instantiation
    cudaError_t e = once_per_device(attr, [&] {
        cudaError_t r = cudaFuncSetAttribute(w_stage1_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(w_stage3_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return r;
    });
    if (e != cudaSuccess) return e;
    EGB_COUNT_LAUNCH();
    w_stage1_kernel<T><<<nblk, 256, smem, st>>>(m, bw, xa, V, ldv, Tm, ldt, X, ypart);
    EGB_COUNT_LAUNCH();
    w_stage2_kernel<T><<<16, 256, 0, st>>>(nblk, ypart, Y);
    EGB_COUNT_LAUNCH();
    w_stage3_kernel<T><<<nblk, 256, smem, st>>>(m, bw, X, V, ldv, Tm, ldt, Y, W);
    return cudaGetLastError();
}

size_t sy2sb_work_elems(int n, int b)
{
    // X (n x b), W (n x b), Y (b x b), Z (b x b)
    return (size_t)4 * n * b + 4 * (size_t)b * b;
}

template <typename T>
cudaError_t sy2sb(cudaStream_t st, int n, int b, T *a, int lda, T *v1, T *t1, T *work,
                  size_t work_elems, unsigned *sync, int *status, int num_sms)
{
    cudaError_t e;
    if (b > 64 || b < 1) return cudaErrorInvalidValue;
    // sync layout: [0..1] barrier words, then doubles
    double *dsync = reinterpret_cast<double *>(sync + 64);
    const int max_g = 512;
    double *part = dsync;                           // 2 x max_g
    double *alpha = part + 2 * max_g;               // 2 x 64
    double *wpart = alpha + 128;                    // 2 x max_g x 64
    double *gram = wpart + 2 * (size_t)max_g * 64;  // max_g x 64 x 64

    int dev = 0;
    cudaGetDevice(&dev);
    // V1 explicit and zero outside each panel's reflectors (the back-transformation merges
    // consecutive panels into one block)
    if ((e = cudaMemsetAsync(v1, 0, sizeof(T) * (size_t)n * n, st)) != cudaSuccess) return e;
    for (int c0 = 0; c0 + b <= n - 2; c0 += b) {
        const int r0 = c0 + b;
        const int m = n - r0;
        const int bw = b;
        T *P = a + r0 + (size_t)c0 * lda;
        T *V = v1 + r0 + (size_t)c0 * n;
        T *Tm = t1 + (size_t)c0 * b;
        int ldt = b;
        // rows per CTA: 256 (fewer CTAs make the per-column barrier and the reductions of
        // the partials cheaper; the per-column work of a CTA stays small), more if needed
        // for co-residency
        int rows = 256;
        int G = ceil_div(m, rows);
        // panel rows, then T (64 x 64 binary64) at the next 16-byte boundary
        auto panel_smem = [&](int r) {
            return (((size_t)r * (bw + 1) * sizeof(T) + 15) & ~(size_t)15) + 64 * 64 * sizeof(double);
        };
        size_t smem = panel_smem(rows);
        static PerDeviceOnce attr_set;  // per instantiation
        e = once_per_device(attr_set, [] {
            return cudaFuncSetAttribute(panel_qr_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        });
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_qr_kernel<T>, 256, smem);
        int max_coresident = per_sm * num_sms;
        while (G > max_coresident || G > max_g) {
            rows *= 2;
            G = ceil_div(m, rows);
            smem = panel_smem(rows);
            if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_qr_kernel<T>, 256, smem);
            max_coresident = per_sm * num_sms;
        }
        if ((e = cudaMemsetAsync(sync, 0, 2 * sizeof(unsigned), st)) != cudaSuccess) return e;
        PanelArgs pa;
        pa.m = m; pa.bw = bw; pa.rows_per_cta = rows; pa.lda = lda; pa.ldv = n;
        pa.count = sync;
        pa.part = part; pa.alpha = alpha; pa.wpart = wpart; pa.gram = gram; pa.status = status;
        pa.gstride = max_g;
        pa.spin_limit = spin_limit();
        void *args[] = {&P, &V, &Tm, &ldt, &pa};
        EGB_COUNT_LAUNCH();
        if ((e = cudaLaunchCooperativeKernel((void *)panel_qr_kernel<T>, dim3(G), dim3(256), args,
                                             smem, st)) != cudaSuccess) return e;

        // ---- two-sided update of A22 = a[r0:, r0:] (full symmetric storage)
        T *A22 = a + r0 + (size_t)r0 * lda;
        T *X = work;                      // m x b
        T *W = work + (size_t)n * b;      // m x b
        T *Y = work + (size_t)2 * n * b;  // b x b
        T *Z = Y + (size_t)b * b;         // b x b
        // X = A22 V (binary32: the symmetric panel product that streams A22 once)
        bool xdone = false;
        if constexpr (sizeof(T) == 4) {
            float *tw;
            size_t te;
            int *ts;
            if (tc_scratch(&tw, &te, &ts)) {
                e = symm_tall_f32(st, m, bw, (const float *)A22, lda, (const float *)V, n, (float *)W, m,
                                  tw, te, ts);
                if (e != cudaErrorNotSupported) {
                    if (e != cudaSuccess) return e;
                    xdone = true;
                }
            }
        }
        if (!xdone && (e = gemm<T>(st, 0, 0, m, bw, m, T(1), A22, lda, V, n, T(0), W, m)) != cudaSuccess)
            return e;
        if (ceil_div(m, kWRows) + 1 <= max_g) {
            // X = (A22 V) T, W = X - 1/2 V (T^T (V^T X)); the per-block partials of V^T X
            // and their sum use the (now idle) Gram scratch of the panel factorisation
            T *yp = reinterpret_cast<T *>(gram);
            T *ysum = yp + (size_t)ceil_div(m, kWRows) * 64 * 64;
            if ((e = form_w<T>(st, m, bw, W, V, n, Tm, ldt, X, ysum, W, yp)) != cudaSuccess) return e;
        } else {
            // X = (A22 V) T
            if ((e = gemm<T>(st, 0, 0, m, bw, bw, T(1), W, m, Tm, ldt, T(0), X, m)) != cudaSuccess) return e;
            // Y = V^T X
            if ((e = gemm_splitk<T>(st, 1, 0, bw, bw, m, T(1), V, n, X, m, Y, bw, W,
                                    (size_t)n * b)) != cudaSuccess) return e;
            // Z = T^T Y
            if ((e = gemm<T>(st, 1, 0, bw, bw, bw, T(1), Tm, ldt, Y, bw, T(0), Z, bw)) != cudaSuccess) return e;
            // W = X - 1/2 V Z
            if ((e = cudaMemcpyAsync(W, X, sizeof(T) * (size_t)m * bw, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
            if ((e = gemm<T>(st, 0, 0, m, bw, bw, T(-0.5), V, n, Z, bw, T(1), W, m)) != cudaSuccess) return e;
        }
        // A22 -= V W^T + W V^T   (lower triangle), then mirror. On the tensor-core path the
        // two products are one GEMM over K = 2 bw: [V W] [W V]^T.
        bool done = false;
        if constexpr (sizeof(T) == 4) {
            float *tw;
            size_t te;
            int *ts;
            if (tc_scratch(&tw, &te, &ts)) {
                TcPart pa[2] = {{(const float *)V, n, 0, bw}, {(const float *)W, m, 0, bw}};
                TcPart pb[2] = {{(const float *)W, m, 1, bw}, {(const float *)V, n, 1, bw}};
                e = tc_gemm_f32_parts(st, m, m, 2, pa, pb, -1.0f, 1.0f, (float *)A22, lda, 1, tw, te, ts);
                if (e != cudaErrorNotSupported) {
                    if (e != cudaSuccess) return e;
                    done = true;
                }
            }
        }
        if (!done) {
            if ((e = gemm<T>(st, 0, 1, m, m, bw, T(-1), V, n, W, m, T(1), A22, lda, 1)) != cudaSuccess) return e;
            if ((e = gemm<T>(st, 0, 1, m, m, bw, T(-1), W, m, V, n, T(1), A22, lda, 1)) != cudaSuccess) return e;
        }
        if ((e = mirror_lower<T>(st, m, A22, lda)) != cudaSuccess) return e;
    }
    (void)work_elems;
    return cudaSuccess;
}

template cudaError_t sy2sb<double>(cudaStream_t, int, int, double *, int, double *, double *,
                                   double *, size_t, unsigned *, int *, int);
template cudaError_t sy2sb<float>(cudaStream_t, int, int, float *, int, float *, float *,
                                  float *, size_t, unsigned *, int *, int);

}  // namespace egb
