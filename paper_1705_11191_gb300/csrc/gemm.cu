// Register-tiled SIMT GEMM and small matrix utilities.
//
// The binary64 path of this solver is bound by the FP64 FMA rate of the chip, which
// any register-tiled kernel saturates, so the GEMM here is a plain shared-memory tiled
// kernel: each CTA computes a BM x BN tile of C, staging BK-deep slices of op(A) and
// op(B) in shared memory, each thread accumulating a TM x TN block in registers.
#include "common.cuh"
#include "kernels.h"

namespace egb {

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_kernel(int m, int n, int k, T alpha, const T *__restrict__ A, int lda, int ta,
            const T *__restrict__ B, int ldb, int tb, T beta, T *__restrict__ C, int ldc,
            int uplo, int kchunk, size_t cstride)
{
    // split-K: CTA z covers k in [z*kchunk, min(k, (z+1)*kchunk)) and writes C + z*cstride
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(k, kbeg + kchunk);
    C += (size_t)blockIdx.z * cstride;
    constexpr int NT = (BM / TM) * (BN / TN);
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];

    const int m0 = blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    if (uplo == 1 && m0 + BM - 1 < n0) return;  // tile entirely above the diagonal

    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN);  // column group
    const int ty = tid / (BN / TN);  // row group

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        // ---- stage op(A)[m0:m0+BM, k0:k0+BK] as As[kk][i]
#pragma unroll
        for (int r = 0; r < (BM * BK + NT - 1) / NT; ++r) {
            int e = tid + r * NT;
            if (e < BM * BK) {
                int i, kk;
                if (ta == 0) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
                int gi = m0 + i, gk = k0 + kk;
                T v = T(0);
                if (gi < m && gk < kend)
                    v = (ta == 0) ? A[(size_t)gi + (size_t)gk * lda] : A[(size_t)gk + (size_t)gi * lda];
                As[kk][i] = v;
            }
        }
        // ---- stage op(B)[k0:k0+BK, n0:n0+BN] as Bs[kk][j]
#pragma unroll
        for (int r = 0; r < (BN * BK + NT - 1) / NT; ++r) {
            int e = tid + r * NT;
            if (e < BN * BK) {
                int j, kk;
                if (tb == 0) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
                int gj = n0 + j, gk = k0 + kk;
                T v = T(0);
                if (gj < n && gk < kend)
                    v = (tb == 0) ? B[(size_t)gk + (size_t)gj * ldb] : B[(size_t)gj + (size_t)gk * ldb];
                Bs[kk][j] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], bb[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
            for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + j * (BN / TN)];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int gi = m0 + ty + i * (BM / TM);
        if (gi >= m) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int gj = n0 + tx + j * (BN / TN);
            if (gj >= n) continue;
            if (uplo == 1 && gi < gj) continue;
            T *c = C + (size_t)gi + (size_t)gj * ldc;
            T v = alpha * acc[i][j];
            if (beta != T(0)) v = fma(beta, *c, v);
            *c = v;
        }
    }
}

template <typename T> struct GemmCfg;
template <> struct GemmCfg<double> { static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4; };
template <> struct GemmCfg<float> { static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8; };

// Scratch for the tensor-core binary32 GEMM of the calling thread's current solve (set by
// the solver around a binary32-route solve; absent elsewhere).
static thread_local float *t_tc_work = nullptr;
static thread_local size_t t_tc_elems = 0;
static thread_local int *t_tc_status = nullptr;

void set_tc_scratch(float *work, size_t elems, int *status)
{
    t_tc_work = work;
    t_tc_elems = elems;
    t_tc_status = status;
}

bool tc_scratch(float **work, size_t *elems, int **status)
{
    *work = t_tc_work;
    *elems = t_tc_elems;
    *status = t_tc_status;
    return t_tc_work != nullptr;
}

// Scratch of the calling thread for binary64-accurate products on the tensor cores (the
// Ozaki digit planes and row exponents; set around the binary64 Cholesky of the binary32
// route, absent elsewhere).
static thread_local __nv_bfloat16 *t_oz_planes = nullptr;
static thread_local size_t t_oz_elems = 0;
static thread_local int *t_oz_exps = nullptr;
static thread_local size_t t_oz_exp_elems = 0;

void set_f64_tc_scratch(__nv_bfloat16 *planes, size_t elems, int *exps, size_t exp_elems)
{
    t_oz_planes = planes;
    t_oz_elems = elems;
    t_oz_exps = exps;
    t_oz_exp_elems = exp_elems;
}

// C = alpha op(A) op(B) + beta C with binary64-accurate digit products: op(A) split by
// rows, op(B) by columns (once for A A^T). cudaErrorNotSupported if the scratch is short.
static cudaError_t gemm_f64_digits(cudaStream_t st, int ta, int tb, int m, int n, int k, double alpha,
                                   const double *A, int lda, const double *B, int ldb, double beta,
                                   double *C, int ldc, int uplo, int digits = kOzDigits)
{
    const bool same = A == B && lda == ldb && ta != tb && m == n;
    const size_t ea = ozaki_split_elems(m, k), eb = same ? 0 : ozaki_split_elems(n, k);
    const size_t xa = (size_t)ceil_div(m, 128) * 128, xb = same ? 0 : (size_t)ceil_div(n, 128) * 128;
    if (ea + eb > t_oz_elems || xa + xb > t_oz_exp_elems) return cudaErrorNotSupported;
    __nv_bfloat16 *ad = t_oz_planes, *bd = same ? t_oz_planes : t_oz_planes + ea;
    int *xe = t_oz_exps, *ye = same ? t_oz_exps : t_oz_exps + xa;
    cudaError_t e;
    // row i of op(A): ta = 0 -> A[i + q lda], ta = 1 -> A[q + i lda]
    if ((e = ozaki_split(st, m, k, A, ta ? lda : 1, ta ? 1 : lda, nullptr, nullptr, ad, xe)) != cudaSuccess)
        return e;
    // column j of op(B): tb = 0 -> B[q + j ldb], tb = 1 -> B[j + q ldb]
    if (!same &&
        (e = ozaki_split(st, n, k, B, tb ? 1 : ldb, tb ? ldb : 1, nullptr, nullptr, bd, ye)) != cudaSuccess)
        return e;
    return ozaki_gemm(st, m, n, k, alpha, ad, xe, bd, ye, beta, C, ldc, uplo, digits);
}

template <typename T>
cudaError_t gemm(cudaStream_t st, int ta, int tb, int m, int n, int k, T alpha, const T *A,
                 int lda, const T *B, int ldb, T beta, T *C, int ldc, int uplo)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        // binary32 products large enough for the tensor-core path
        if (t_tc_work && k >= 16 && (double)m * n * k >= 4.0e6) {
            cudaError_t e = tc_gemm_f32(st, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                                        uplo, t_tc_work, t_tc_elems, t_tc_status);
            if (e != cudaErrorNotSupported) return e;
        }
    } else {
        // binary64 products large enough for the digit products on the tensor cores
        if (t_oz_planes && k >= 32 && (double)m * n * k >= 1.6e7) {
            cudaError_t e = gemm_f64_digits(st, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, uplo);
            if (e != cudaErrorNotSupported) return e;
        }
    }
    using G = GemmCfg<T>;
    dim3 grid(ceil_div(m, G::BM), ceil_div(n, G::BN));
    dim3 block((G::BM / G::TM) * (G::BN / G::TN));
    EGB_COUNT_LAUNCH();
    gemm_kernel<T, G::BM, G::BN, G::BK, G::TM, G::TN><<<grid, block, 0, st>>>(
        m, n, k, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, uplo, k > 0 ? k : 1, 0);
    return cudaGetLastError();
}

template <typename T>
__global__ void splitk_reduce_kernel(int m, int n, int splits, const T *part, T alpha, T *C, int ldc)
{
    size_t total = (size_t)m * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        T s = T(0);
        for (int z = 0; z < splits; ++z) s += part[(size_t)z * total + e];
        int i = (int)(e % m), j = (int)(e / m);
        C[(size_t)i + (size_t)j * ldc] = alpha * s;
    }
}

template <typename T>
cudaError_t gemm_splitk(cudaStream_t st, int ta, int tb, int m, int n, int k, T alpha,
                        const T *A, int lda, const T *B, int ldb, T *C, int ldc, T *part,
                        size_t part_elems)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        if (t_tc_work && k >= 16 && (double)m * n * k >= 4.0e6) {
            cudaError_t e = tc_gemm_f32(st, ta, tb, m, n, k, alpha, A, lda, B, ldb, 0.0f, C, ldc, 0,
                                        t_tc_work, t_tc_elems, t_tc_status);
            if (e != cudaErrorNotSupported) return e;
        }
    }
    using G = GemmCfg<T>;
    const int tiles = ceil_div(m, G::BM) * ceil_div(n, G::BN);
    int splits = ceil_div(2 * 152, tiles);
    int maxs = k / 256;
    if (splits > maxs) splits = maxs;
    if ((size_t)splits * m * n > part_elems) splits = (int)(part_elems / ((size_t)m * n));
    if (splits <= 1) return gemm<T>(st, ta, tb, m, n, k, alpha, A, lda, B, ldb, T(0), C, ldc, 0);
    int kchunk = ceil_div(k, splits);
    kchunk = ceil_div(kchunk, G::BK) * G::BK;
    splits = ceil_div(k, kchunk);
    dim3 grid(ceil_div(m, G::BM), ceil_div(n, G::BN), splits);
    dim3 block((G::BM / G::TM) * (G::BN / G::TN));
    EGB_COUNT_LAUNCH();
    gemm_kernel<T, G::BM, G::BN, G::BK, G::TM, G::TN><<<grid, block, 0, st>>>(
        m, n, k, T(1), A, lda, ta, B, ldb, tb, T(0), part, m, 0, kchunk, (size_t)m * n);
    size_t total = (size_t)m * n;
    int rg = (int)((total + 255) / 256);
    if (rg > 152 * 8) rg = 152 * 8;
    EGB_COUNT_LAUNCH();
    splitk_reduce_kernel<T><<<rg, 256, 0, st>>>(m, n, splits, part, alpha, C, ldc);
    return cudaGetLastError();
}
template cudaError_t gemm_splitk<double>(cudaStream_t, int, int, int, int, int, double, const double *,
                                         int, const double *, int, double *, int, double *, size_t);
template cudaError_t gemm_splitk<float>(cudaStream_t, int, int, int, int, int, float, const float *,
                                        int, const float *, int, float *, int, float *, size_t);

template cudaError_t gemm<double>(cudaStream_t, int, int, int, int, int, double, const double *,
                                  int, const double *, int, double, double *, int, int);
template cudaError_t gemm<float>(cudaStream_t, int, int, int, int, int, float, const float *,
                                 int, const float *, int, float, float *, int, int);

// ------------------------------------------------------------------ utilities
template <typename Td, typename Ts>
__global__ void copy_matrix_kernel(int m, int n, const Ts *__restrict__ src, int lds,
                                   Td *__restrict__ dst, int ldd)
{
    size_t total = (size_t)m * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % m), j = (int)(e / m);
        dst[(size_t)i + (size_t)j * ldd] = (Td)src[(size_t)i + (size_t)j * lds];
    }
}

template <typename Td, typename Ts>
cudaError_t copy_matrix(cudaStream_t st, int m, int n, const Ts *src, int lds, Td *dst, int ldd)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    size_t total = (size_t)m * n;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 32) grid = 152 * 32;
    EGB_COUNT_LAUNCH();
    copy_matrix_kernel<Td, Ts><<<grid, 256, 0, st>>>(m, n, src, lds, dst, ldd);
    return cudaGetLastError();
}
template cudaError_t copy_matrix<double, double>(cudaStream_t, int, int, const double *, int, double *, int);
template cudaError_t copy_matrix<float, double>(cudaStream_t, int, int, const double *, int, float *, int);
template cudaError_t copy_matrix<double, float>(cudaStream_t, int, int, const float *, int, double *, int);
template cudaError_t copy_matrix<float, float>(cudaStream_t, int, int, const float *, int, float *, int);

// 32x32 tiles; mode 0: dst = src^T (general), mode 1: upper := lower^T, mode 2: (a+a^T)/2
template <typename T>
__global__ void tile_transpose_kernel(int m, int n, const T *src, int lds, T *dst, int ldd,
                                      int mode)
{
    __shared__ T tile[32][33];
    int bi = blockIdx.x * 32, bj = blockIdx.y * 32;  // tile of src rows bi.., cols bj..
    if (mode != 0 && bi < bj) return;                  // symmetric modes: lower tiles only
    int tx = threadIdx.x, ty = threadIdx.y;            // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        int i = bi + tx, j = bj + r;
        if (i < m && j < n) tile[r][tx] = src[(size_t)i + (size_t)j * lds];
    }
    __syncthreads();
    if (mode == 2) {
        // average tile (bi,bj) with tile (bj,bi) and write both
        __shared__ T tile2[32][33];
        for (int r = ty; r < 32; r += 8) {
            int i = bj + tx, j = bi + r;
            if (i < n && j < m) tile2[r][tx] = src[(size_t)i + (size_t)j * lds];
        }
        __syncthreads();
        // tile[r][c] = a(bi+c, bj+r); tile2[r][c] = a(bj+c, bi+r)
        for (int r = ty; r < 32; r += 8) {
            int i = bi + tx, j = bj + r;
            if (i < m && j < n) {
                T v = T(0.5) * (tile[r][tx] + tile2[tx][r]);
                dst[(size_t)i + (size_t)j * ldd] = v;
            }
        }
        for (int r = ty; r < 32; r += 8) {
            int i = bj + tx, j = bi + r;
            if (i < n && j < m) {
                T v = T(0.5) * (tile2[r][tx] + tile[tx][r]);
                dst[(size_t)i + (size_t)j * ldd] = v;
            }
        }
        return;
    }
    // write transposed: dst(j, i) = src(i, j)
    for (int r = ty; r < 32; r += 8) {
        int j = bj + tx, i = bi + r;  // dst row j = src col, dst col i = src row
        if (i < m && j < n) {
            if (mode == 1 && i <= j) continue;  // only strictly-lower sources to upper
            dst[(size_t)j + (size_t)i * ldd] = tile[tx][r];
        }
    }
}

template <typename T>
cudaError_t transpose(cudaStream_t st, int m, int n, const T *src, int lds, T *dst, int ldd)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    dim3 grid(ceil_div(m, 32), ceil_div(n, 32)), block(32, 8);
    EGB_COUNT_LAUNCH();
    tile_transpose_kernel<T><<<grid, block, 0, st>>>(m, n, src, lds, dst, ldd, 0);
    return cudaGetLastError();
}

// upper := lower^T in place, 64 x 64 tiles (tile (bi, bj) of the lower triangle is read
// and its transpose written to tile (bj, bi)); 256 threads, each with its 16 loads in
// flight together (the copy is bound by HBM traffic, which needs many bytes in flight).
template <typename T>
__global__ void __launch_bounds__(256) mirror64_kernel(int n, T *a, int lda)
{
    __shared__ T tile[64][65];
    const int bi = blockIdx.x * 64, bj = blockIdx.y * 64;
    if (bi < bj) return;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 x 4
    T v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int i = bi + tx, j = bj + ty + 4 * u;
        v[u] = (i < n && j < n) ? a[(size_t)i + (size_t)j * lda] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) tile[ty + 4 * u][tx] = v[u];
    __syncthreads();
    // a(j, i) = a(i, j) for i > j: destination row j = bj + tx, column i = bi + r
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int r = ty + 4 * u, j = bj + tx, i = bi + r;
        if (i < n && j < n && i > j) a[(size_t)j + (size_t)i * lda] = tile[tx][r];
    }
}

template <typename T>
cudaError_t mirror_lower(cudaStream_t st, int n, T *a, int lda)
{
    if (n <= 0) return cudaSuccess;
    dim3 grid(ceil_div(n, 64), ceil_div(n, 64));
    EGB_COUNT_LAUNCH();
    mirror64_kernel<T><<<grid, 256, 0, st>>>(n, a, lda);
    return cudaGetLastError();
}

template <typename T>
cudaError_t symmetrize(cudaStream_t st, int n, T *a, int lda)
{
    if (n <= 0) return cudaSuccess;
    dim3 grid(ceil_div(n, 32), ceil_div(n, 32)), block(32, 8);
    EGB_COUNT_LAUNCH();
    tile_transpose_kernel<T><<<grid, block, 0, st>>>(n, n, a, lda, a, lda, 2);
    return cudaGetLastError();
}

template cudaError_t transpose<double>(cudaStream_t, int, int, const double *, int, double *, int);
template cudaError_t transpose<float>(cudaStream_t, int, int, const float *, int, float *, int);
template cudaError_t mirror_lower<double>(cudaStream_t, int, double *, int);
template cudaError_t mirror_lower<float>(cudaStream_t, int, float *, int);
template cudaError_t symmetrize<double>(cudaStream_t, int, double *, int);
template cudaError_t symmetrize<float>(cudaStream_t, int, float *, int);

template <typename T>
__global__ void check_finite_kernel(int m, int n, const T *a, int lda, int *status)
{
    size_t total = (size_t)m * n;
    bool bad = false;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % m), j = (int)(e / m);
        T v = a[(size_t)i + (size_t)j * lda];
        if (!isfinite(v)) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
        report_error(status, ELSI_ERR_NONFINITE, 0);
}

template <typename T>
cudaError_t check_finite(cudaStream_t st, int m, int n, const T *a, int lda, int *status)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    size_t total = (size_t)m * n;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    EGB_COUNT_LAUNCH();
    check_finite_kernel<T><<<grid, 256, 0, st>>>(m, n, a, lda, status);
    return cudaGetLastError();
}
template cudaError_t check_finite<double>(cudaStream_t, int, int, const double *, int, int *);
template cudaError_t check_finite<float>(cudaStream_t, int, int, const float *, int, int *);

}  // namespace egb

extern "C" size_t elsi_gb_gemm_f64_digits_planes(int m, int n, int k)
{
    if (m < 1 || n < 1 || k < 1) return 0;
    return egb::ozaki_split_elems(m, k) + egb::ozaki_split_elems(n, k);
}

extern "C" size_t elsi_gb_gemm_f64_digits_exps(int m, int n)
{
    if (m < 1 || n < 1) return 0;
    return (size_t)egb::ceil_div(m, 128) * 128 + (size_t)egb::ceil_div(n, 128) * 128;
}

extern "C" int elsi_gb_gemm_f64_digits(int ta, int tb, int m, int n, int k, double alpha,
                                       const double *A, int lda, const double *B, int ldb,
                                       double beta, double *C, int ldc, int uplo, int digits,
                                       void *planes, size_t plane_elems, int *exps, size_t exp_elems,
                                       int *status, void *stream)
{
    if (m < 1 || n < 1 || k < 1 || digits < 1 || digits > egb::kOzDigits || !A || !B || !C || !planes ||
        !exps || !status)
        return ELSI_ERR_ARG;
    if (ldc < m || lda < (ta ? k : m) || ldb < (tb ? n : k)) return ELSI_ERR_ARG;
    if ((size_t)planes % 16 != 0 || plane_elems < elsi_gb_gemm_f64_digits_planes(m, n, k) ||
        exp_elems < elsi_gb_gemm_f64_digits_exps(m, n))
        return ELSI_ERR_ARG;
    // the pipeline's status word comes from the binary32 scratch slot of this thread
    float *tw;
    size_t te;
    int *ts;
    egb::tc_scratch(&tw, &te, &ts);
    egb::set_tc_scratch(tw, te, status);
    egb::set_f64_tc_scratch(reinterpret_cast<__nv_bfloat16 *>(planes), plane_elems, exps, exp_elems);
    cudaError_t e = egb::gemm_f64_digits((cudaStream_t)stream, ta, tb, m, n, k, alpha, A, lda, B, ldb,
                                         beta, C, ldc, uplo, digits);
    egb::set_f64_tc_scratch(nullptr, 0, nullptr, 0);
    egb::set_tc_scratch(tw, te, ts);
    if (e == cudaErrorNotSupported) return ELSI_ERR_ARG;
    return e == cudaSuccess ? ELSI_OK : ELSI_ERR_CUDA;
}
