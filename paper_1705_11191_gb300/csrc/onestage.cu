// One-stage tridiagonalisation T = Q^T H~ Q (arXiv:1705.11191 Eq. 11, the ELPA 1-stage
// route) and its back-transformation Z <- Q Z.
//
// Blocked Householder reduction in panels of nb columns (the blocking of Dongarra,
// Hammarling and Sorensen): for column j of a panel, with the panel's earlier reflectors
// V and the vectors W not yet applied to the trailing matrix,
//   a_j  -= V W[j,:]^T + W V[j,:]^T                    (column j brought up to date)
//   v, tau, beta from a_j[j+1:]                          (Householder)
//   y     = A22 v - V (W^T v) - W (V^T v)                (A22 = A[j+1:, j+1:] as stored)
//   w     = tau y - (tau^2 / 2) (y^T v) v
// and after the panel A22 -= V W^T + W V^T for the rows and columns beyond the panel
// (tensor-core GEMM in the binary32 route). The symmetric matrix-vector product reads
// the trailing matrix once per column, which is what makes this route memory-bound
// (BLAS-2) and the reason for the two-stage reduction (sec. 3.1).
//
// Per column: K1 (one CTA) updates column j and forms the reflector; K2 (rows x column
// chunks) forms partial products A22 v and the partial dot products needed for
// V^T v, W^T v and v^T A22 v; K3 (rows) sums the partials and writes w.
#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace egb {

constexpr int kOsNb = kOneStageNb;  // panel width
constexpr int kOsRows = 256;     // rows per CTA in K2 / K3
constexpr int kOsChunk = 512;    // columns per CTA in K2

// V, W: n x nb panel arrays (ld n), column jj holds the panel's reflector / w vector with
// zeros above its start. tau: n. d, e: binary64 tridiagonal.
template <typename T>
__global__ void __launch_bounds__(1024) os_column_kernel(int n, int j, int jj, T *A, int lda,
                                                         const T *V, const T *W, T *vcol,
                                                         T *tau, double *d, double *e)
{
    __shared__ double red[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int m = n - j - 1;
    T *a = A + (size_t)j * lda;  // column j
    // bring rows j .. n-1 of column j up to date with the panel's earlier columns
    for (int i = j + tid; i < n; i += nt) {
        T s = a[i];
        for (int q = 0; q < jj; ++q)
            s -= V[i + (size_t)q * n] * W[j + (size_t)q * n] + W[i + (size_t)q * n] * V[j + (size_t)q * n];
        a[i] = s;
    }
    __syncthreads();
    double ss = 0.0;
    for (int i = j + 2 + tid; i < n; i += nt) ss += (double)a[i] * (double)a[i];
    ss = block_sum(ss, red);
    const double alpha = (m >= 1) ? (double)a[j + 1] : 0.0;
    double beta = alpha, t = 0.0, scl = 0.0;
    if (ss != 0.0) {
        const double nrm = sqrt(alpha * alpha + ss);
        beta = (alpha >= 0.0) ? -nrm : nrm;
        t = (beta - alpha) / beta;
        scl = 1.0 / (alpha - beta);
    }
    // reflector v (unit first entry at row j+1) into the panel's V column and vcol
    for (int i = tid; i < n; i += nt) {
        T v = T(0);
        if (i == j + 1) v = T(1);
        else if (i > j + 1) v = (T)((double)a[i] * scl);
        vcol[i] = v;
    }
    if (tid == 0) {
        tau[j] = (T)t;
        d[j] = (double)a[j];
        if (m >= 1) e[j] = beta;
    }
}

// partials of y = A22 v (chunk of columns c0 .. c0 + kOsChunk), of v^T (A22 v) and, in the
// first column chunk, of V^T v and W^T v over this CTA's rows
template <typename T>
__global__ void __launch_bounds__(kOsRows) os_symv_kernel(int n, int j, int jj, const T *A, int lda,
                                                          const T *vcol, const T *V, const T *W,
                                                          T *ypart, double *spart, double *upart)
{
    __shared__ T vs[kOsChunk];
    __shared__ double red[32];
    const int m = n - j - 1, off = j + 1;
    const int r = blockIdx.x * kOsRows + threadIdx.x;  // row within A22
    const int c0 = blockIdx.y * kOsChunk;
    const int cn = min(kOsChunk, m - c0);
    for (int c = threadIdx.x; c < cn; c += kOsRows) vs[c] = vcol[off + c0 + c];
    __syncthreads();
    T y = T(0);
    if (r < m) {
        const T *col = A + (size_t)(off + r) + (size_t)(off + c0) * lda;
        for (int c = 0; c < cn; ++c) y = fma(col[(size_t)c * lda], vs[c], y);
        ypart[(size_t)blockIdx.y * m + r] = y;
    }
    const double vy = (r < m) ? (double)vcol[off + r] * (double)y : 0.0;
    const double s = block_sum(vy, red);
    if (threadIdx.x == 0) spart[blockIdx.y * gridDim.x + blockIdx.x] = s;
    if (blockIdx.y == 0) {
        const double vr = (r < m) ? (double)vcol[off + r] : 0.0;
        for (int q = 0; q < jj; ++q) {
            const double a1 = (r < m) ? (double)W[off + r + (size_t)q * n] * vr : 0.0;
            const double a2 = (r < m) ? (double)V[off + r + (size_t)q * n] * vr : 0.0;
            const double s1 = block_sum(a1, red), s2 = block_sum(a2, red);
            if (threadIdx.x == 0) {
                upart[((size_t)blockIdx.x * kOsNb + q) * 2] = s1;      // (W^T v)_q
                upart[((size_t)blockIdx.x * kOsNb + q) * 2 + 1] = s2;  // (V^T v)_q
            }
        }
    }
}

// w = tau y - (tau^2/2)(y^T v) v with y = sum of partials - V u1 - W u2 (u1 = W^T v,
// u2 = V^T v), y^T v = v^T A22 v - 2 u1 . u2; also writes v and w into the panel arrays
template <typename T>
__global__ void __launch_bounds__(kOsRows) os_w_kernel(int n, int j, int jj, int nrb, int nch,
                                                       const T *ypart, const double *spart,
                                                       const double *upart, const T *vcol,
                                                       const T *tau, T *V, T *W)
{
    __shared__ double u1[kOsNb], u2[kOsNb];
    __shared__ double red[32];
    __shared__ double coef;
    const int m = n - j - 1, off = j + 1;
    const int tid = threadIdx.x;
    if (tid < 2 * kOsNb) {
        const int q = tid >> 1, which = tid & 1;
        double s = 0.0;
        if (q < jj)
            for (int b = 0; b < nrb; ++b) s += upart[((size_t)b * kOsNb + q) * 2 + which];
        if (which == 0) u1[q] = s; else u2[q] = s;
    }
    double sp = 0.0;
    for (int i = tid; i < nrb * nch; i += blockDim.x) sp += spart[i];
    sp = block_sum(sp, red);
    __syncthreads();
    if (tid == 0) {
        double uu = 0.0;
        for (int q = 0; q < jj; ++q) uu += u1[q] * u2[q];
        const double t = (double)tau[j];
        coef = 0.5 * t * t * (sp - 2.0 * uu);
    }
    __syncthreads();
    const double t = (double)tau[j];
    const int r = blockIdx.x * kOsRows + tid;
    if (r < m) {
        double y = 0.0;
        for (int ch = 0; ch < nch; ++ch) y += (double)ypart[(size_t)ch * m + r];
        for (int q = 0; q < jj; ++q)
            y -= (double)V[off + r + (size_t)q * n] * u1[q] + (double)W[off + r + (size_t)q * n] * u2[q];
        const double v = (double)vcol[off + r];
        W[off + r + (size_t)jj * n] = (T)(t * y - coef * v);
        V[off + r + (size_t)jj * n] = (T)v;
    }
    if (blockIdx.x == 0)  // rows 0 .. j of the panel columns are zero
        for (int i = tid; i <= j; i += blockDim.x) {
            W[i + (size_t)jj * n] = T(0);
            V[i + (size_t)jj * n] = T(0);
        }
}

// T (w x w, ld ldt) of the panel's compact WY form I - V T V^T from G = V^T V and tau:
// T_jj = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] G[0:j, j] (forward recurrence). One CTA.
template <typename T>
__global__ void os_tfactor_kernel(int w, const T *G, int ldg, const T *tau, T *Tm, int ldt)
{
    __shared__ double tl[kOsNb * kOsNb];
    const int tid = threadIdx.x;
    for (int e = tid; e < kOsNb * kOsNb; e += blockDim.x) tl[e] = 0.0;
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        if (tid < j) {
            double s = 0.0;
            for (int p = tid; p < j; ++p) s += tl[tid + p * kOsNb] * (double)G[p + (size_t)j * ldg];
            tl[tid + j * kOsNb] = -(double)tau[j] * s;
        }
        if (tid == 0) tl[j + j * kOsNb] = (double)tau[j];
        __syncthreads();
    }
    for (int e = tid; e < w * w; e += blockDim.x) {
        const int r = e % w, c = e / w;
        Tm[r + (size_t)c * ldt] = (T)tl[r + c * kOsNb];
    }
}

template <typename T>
__global__ void os_last_kernel(int n, const T *A, int lda, double *d)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) d[n - 1] = (double)A[(size_t)(n - 1) * (lda + 1)];
}

static inline int os_nrb(int m) { return (m + kOsRows - 1) / kOsRows; }
static inline int os_nch(int m) { return (m + kOsChunk - 1) / kOsChunk; }

size_t onestage_work_elems(int n)
{
    // W (n x nb), vcol (n), tau (n), ypart (nch x m), spart (nrb x nch), upart
    // (nrb x nb x 2), G (nb x nb); in doubles (also enough for binary32)
    const size_t nrb = os_nrb(n), nch = os_nch(n);
    return (size_t)n * kOsNb + 2 * (size_t)n + nch * n + nrb * nch + nrb * kOsNb * 2 +
           kOsNb * kOsNb + 256;
}

template <typename T>
cudaError_t onestage_tridiag(cudaStream_t st, int n, T *A, int lda, double *d, double *e, T *v1,
                             T *t1, double *work)
{
    cudaError_t err;
    if (n <= 0) return cudaSuccess;
    // scratch layout (binary64 slots; binary32 arrays use the start of their slot)
    T *W = reinterpret_cast<T *>(work);
    T *vcol = reinterpret_cast<T *>(work + (size_t)n * kOsNb);
    T *tau = reinterpret_cast<T *>(work + (size_t)n * kOsNb + n);
    T *ypart = reinterpret_cast<T *>(work + (size_t)n * kOsNb + 2 * (size_t)n);
    double *spart = work + (size_t)n * kOsNb + 2 * (size_t)n + (size_t)os_nch(n) * n;
    double *upart = spart + (size_t)os_nrb(n) * os_nch(n);
    T *G = reinterpret_cast<T *>(upart + (size_t)os_nrb(n) * kOsNb * 2);
    if ((err = cudaMemsetAsync(tau, 0, sizeof(T) * n, st)) != cudaSuccess) return err;
    for (int p0 = 0; p0 < n - 1; p0 += kOsNb) {
        const int w = min(kOsNb, n - 1 - p0);
        T *V = v1 + (size_t)p0 * n;
        for (int jj = 0; jj < w; ++jj) {
            const int j = p0 + jj, m = n - j - 1;
            EGB_COUNT_LAUNCH();
            os_column_kernel<T><<<1, 1024, 0, st>>>(n, j, jj, A, lda, V, W, vcol, tau, d, e);
            const int nrb = os_nrb(m), nch = os_nch(m);
            EGB_COUNT_LAUNCH();
            os_symv_kernel<T><<<dim3(nrb, nch), kOsRows, 0, st>>>(n, j, jj, A, lda, vcol, V, W, ypart,
                                                                   spart, upart);
            EGB_COUNT_LAUNCH();
            os_w_kernel<T><<<nrb, kOsRows, 0, st>>>(n, j, jj, nrb, nch, ypart, spart, upart, vcol, tau, V, W);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
        }
        // trailing update A22 -= V W^T + W V^T beyond the panel (lower), then mirror
        const int r1 = p0 + w, m2 = n - r1;
        if (m2 > 0) {
            T *A22 = A + r1 + (size_t)r1 * lda;
            bool done = false;
            if constexpr (sizeof(T) == 4) {
                float *tw;
                size_t te;
                int *ts;
                if (tc_scratch(&tw, &te, &ts)) {
                    TcPart pa[2] = {{(const float *)V + r1, n, 0, w}, {(const float *)W + r1, n, 0, w}};
                    TcPart pb[2] = {{(const float *)W + r1, n, 1, w}, {(const float *)V + r1, n, 1, w}};
                    err = tc_gemm_f32_parts(st, m2, m2, 2, pa, pb, -1.0f, 1.0f, (float *)A22, lda, 1, tw, te, ts);
                    if (err != cudaErrorNotSupported) {
                        if (err != cudaSuccess) return err;
                        done = true;
                    }
                }
            }
            if (!done) {
                if ((err = gemm<T>(st, 0, 1, m2, m2, w, T(-1), V + r1, n, W + r1, n, T(1), A22, lda, 1)) != cudaSuccess) return err;
                if ((err = gemm<T>(st, 0, 1, m2, m2, w, T(-1), W + r1, n, V + r1, n, T(1), A22, lda, 1)) != cudaSuccess) return err;
            }
            if ((err = mirror_lower<T>(st, m2, A22, lda)) != cudaSuccess) return err;
        }
        // compact-WY factor of the panel for the back-transformation
        const int r0 = p0 + 1, mv = n - r0;
        if ((err = gemm<T>(st, 1, 0, w, w, mv, T(1), V + r0, n, V + r0, n, T(0), G, kOsNb)) != cudaSuccess) return err;
        EGB_COUNT_LAUNCH();
        os_tfactor_kernel<T><<<1, 256, 0, st>>>(w, G, kOsNb, tau + p0, t1 + (size_t)p0 * kOsNb, kOsNb);
    }
    EGB_COUNT_LAUNCH();
    os_last_kernel<T><<<1, 32, 0, st>>>(n, A, lda, d);
    return cudaGetLastError();
}

// Z (n x k) <- Q Z with Q = Q_0 Q_1 ... (panels of the one-stage reduction, last first)
template <typename T>
cudaError_t apply_q_onestage(cudaStream_t st, int n, int k, const T *v1, const T *t1, T *z, int ldz,
                             T *work)
{
    cudaError_t err;
    if (n <= 2 || k <= 0) return cudaSuccess;
    const int npan = (n - 1 + kOsNb - 1) / kOsNb;
    for (int p = npan - 1; p >= 0; --p) {
        const int p0 = p * kOsNb, w = min(kOsNb, n - 1 - p0);
        const int r0 = p0 + 1, m = n - r0;
        const T *V = v1 + r0 + (size_t)p0 * n;
        const T *Tm = t1 + (size_t)p0 * kOsNb;
        T *Y = work;                         // w x k
        T *Y2 = work + (size_t)kOsNb * k;    // w x k
        T *Zr = z + r0;
        if ((err = gemm_splitk<T>(st, 1, 0, w, k, m, T(1), V, n, Zr, ldz, Y, w, Y2 + (size_t)kOsNb * k,
                                  (size_t)16 * kOsNb * k)) != cudaSuccess) return err;
        if ((err = gemm<T>(st, 0, 0, w, k, w, T(1), Tm, kOsNb, Y, w, T(0), Y2, w)) != cudaSuccess) return err;
        if ((err = gemm<T>(st, 0, 0, m, k, w, T(-1), V, n, Y2, w, T(1), Zr, ldz)) != cudaSuccess) return err;
    }
    return cudaSuccess;
}

template cudaError_t onestage_tridiag<double>(cudaStream_t, int, double *, int, double *, double *,
                                              double *, double *, double *);
template cudaError_t onestage_tridiag<float>(cudaStream_t, int, float *, int, double *, double *,
                                             float *, float *, double *);
template cudaError_t apply_q_onestage<double>(cudaStream_t, int, int, const double *, const double *,
                                              double *, int, double *);
template cudaError_t apply_q_onestage<float>(cudaStream_t, int, int, const float *, const float *,
                                             float *, int, float *);

}  // namespace egb
