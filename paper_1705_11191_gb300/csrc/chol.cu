// Blocked Cholesky factorisation S = L L^T (arXiv:1705.11191 Eq. 8) and the blocked
// triangular solves with L used for the standard form H~ = L^{-1} H L^{-T} and the
// back-substitution c = L^{-T} c~ (Eq. 9).
//
// Right-looking blocked algorithm with block nb = kTriBlock: the nb x nb diagonal block is
// factorised and inverted by one CTA in shared memory; the panel below it is multiplied
// by the inverse (a GEMM) and the trailing matrix gets a lower-triangular rank-nb update
// (a GEMM restricted to the lower triangle). The triangular solves reuse the inverted
// diagonal blocks so that every O(n^3) flop is in a GEMM.
#include "common.cuh"
#include "kernels.h"

namespace egb {

// One CTA: factor the jb x jb diagonal block at a (lower triangle read), write L back
// (upper part of the block zeroed) and its inverse to inv (ld ldi).
template <typename T>
__global__ void potrf_diag_kernel(int jb, T *a, int lda, T *inv, int ldi, int *status,
                                  int pivot_base)
{
    extern __shared__ unsigned char smem_raw[];
    T *L = reinterpret_cast<T *>(smem_raw);  // jb x jb, ld = jb
    T *X = L + jb * jb;                      // inverse
    __shared__ int bad;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < jb * jb; e += nt) {
        int i = e % jb, j = e / jb;
        L[e] = (i >= j) ? a[(size_t)i + (size_t)j * lda] : T(0);
        X[e] = T(0);
    }
    if (tid == 0) bad = -1;
    __syncthreads();
    for (int k = 0; k < jb; ++k) {
        if (tid == 0) {
            T d = L[k + k * jb];
            if (!(d > T(0)) || !isfinite(d)) {
                if (bad < 0) bad = k;
                d = T(1);  // keep going with a harmless pivot; the status reports the failure
            }
            L[k + k * jb] = dsqrt(d);
        }
        __syncthreads();
        T piv = L[k + k * jb];
        for (int i = k + 1 + tid; i < jb; i += nt) L[i + k * jb] /= piv;
        __syncthreads();
        // trailing lower update: L[i][j] -= L[i][k] * L[j][k], k < j <= i
        int rem = jb - k - 1;
        for (int e = tid; e < rem * rem; e += nt) {
            int i = k + 1 + e % rem, j = k + 1 + e / rem;
            if (i >= j) L[i + j * jb] -= L[i + k * jb] * L[j + k * jb];
        }
        __syncthreads();
    }
    if (tid == 0 && bad >= 0) report_error(status, ELSI_ERR_NOT_PD, pivot_base + bad);
    // inverse of the lower-triangular block, one column per thread
    for (int c = tid; c < jb; c += nt) {
        X[c + c * jb] = T(1) / L[c + c * jb];
        for (int i = c + 1; i < jb; ++i) {
            T s = T(0);
            for (int p = c; p < i; ++p) s += L[i + p * jb] * X[p + c * jb];
            X[i + c * jb] = -s / L[i + i * jb];
        }
    }
    __syncthreads();
    for (int e = tid; e < jb * jb; e += nt) {
        int i = e % jb, j = e / jb;
        a[(size_t)i + (size_t)j * lda] = L[e];  // upper part zero
        inv[(size_t)i + (size_t)j * ldi] = X[e];
    }
}

template <typename T>
__global__ void zero_upper_kernel(int n, T *a, int lda)
{
    size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), j = (int)(e / n);
        if (i < j) a[(size_t)i + (size_t)j * lda] = T(0);
    }
}

template <typename T>
static cudaError_t launch_potrf_diag(cudaStream_t st, int jb, T *a, int lda, T *inv, int ldi,
                                     int *status, int base)
{
    size_t smem = 2 * sizeof(T) * jb * jb;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(potrf_diag_kernel<T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(2 * sizeof(T) * kTriBlock * kTriBlock));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    EGB_COUNT_LAUNCH();
    potrf_diag_kernel<T><<<1, 256, smem, st>>>(jb, a, lda, inv, ldi, status, base);
    return cudaGetLastError();
}

template <typename T>
cudaError_t potrf(cudaStream_t st, int n, T *a, int lda, T *inv_diag, T *work, int *status)
{
    const int nb = kTriBlock;
    cudaError_t e;
    for (int j0 = 0; j0 < n; j0 += nb) {
        int jb = (n - j0 < nb) ? n - j0 : nb;
        T *a11 = a + j0 + (size_t)j0 * lda;
        T *inv11 = inv_diag + j0;  // ld = n
        if ((e = launch_potrf_diag<T>(st, jb, a11, lda, inv11, n, status, j0)) != cudaSuccess) return e;
        int m2 = n - j0 - jb;
        if (m2 > 0) {
            T *a21 = a + (j0 + jb) + (size_t)j0 * lda;
            T *a22 = a + (j0 + jb) + (size_t)(j0 + jb) * lda;
            // L21 = A21 * inv(L11)^T
            if ((e = gemm<T>(st, 0, 1, m2, jb, jb, T(1), a21, lda, inv11, n, T(0), work, m2)) != cudaSuccess) return e;
            if ((e = cudaMemcpy2DAsync(a21, sizeof(T) * lda, work, sizeof(T) * m2, sizeof(T) * m2, jb,
                                       cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
            // A22 -= L21 L21^T (lower triangle)
            if ((e = gemm<T>(st, 0, 1, m2, m2, jb, T(-1), a21, lda, a21, lda, T(1), a22, lda, 1)) != cudaSuccess) return e;
        }
    }
    size_t total = (size_t)n * n;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    EGB_COUNT_LAUNCH();
    zero_upper_kernel<T><<<grid, 256, 0, st>>>(n, a, lda);
    return cudaGetLastError();
}

template <typename T>
cudaError_t trsm_left_lower(cudaStream_t st, int trans, int n, int ncol, const T *L, int ldl,
                            const T *inv_diag, T *B, int ldb, T *work)
{
    const int nb = kTriBlock;
    cudaError_t e;
    if (n <= 0 || ncol <= 0) return cudaSuccess;
    const int nblk = ceil_div(n, nb);
    for (int bi = 0; bi < nblk; ++bi) {
        int blk = trans ? (nblk - 1 - bi) : bi;
        int j0 = blk * nb;
        int jb = (n - j0 < nb) ? n - j0 : nb;
        const T *inv11 = inv_diag + j0;  // ld n
        T *bj = B + j0;
        // B_j := inv(L_jj) B_j   or   inv(L_jj)^T B_j
        if ((e = gemm<T>(st, trans, 0, jb, ncol, jb, T(1), inv11, n, bj, ldb, T(0), work, jb)) != cudaSuccess) return e;
        if ((e = cudaMemcpy2DAsync(bj, sizeof(T) * ldb, work, sizeof(T) * jb, sizeof(T) * jb, ncol,
                                   cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
        if (!trans) {
            int m2 = n - j0 - jb;
            if (m2 > 0) {
                const T *l21 = L + (j0 + jb) + (size_t)j0 * ldl;
                if ((e = gemm<T>(st, 0, 0, m2, ncol, jb, T(-1), l21, ldl, bj, ldb, T(1), B + j0 + jb, ldb)) != cudaSuccess) return e;
            }
        } else if (j0 > 0) {
            // B_{<j} -= (L_{j,<j})^T B_j ; L_{j,<j} is jb x j0 at rows j0
            const T *lj = L + j0;
            if ((e = gemm<T>(st, 1, 0, j0, ncol, jb, T(-1), lj, ldl, bj, ldb, T(1), B, ldb)) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

template cudaError_t potrf<double>(cudaStream_t, int, double *, int, double *, double *, int *);
template cudaError_t potrf<float>(cudaStream_t, int, float *, int, float *, float *, int *);
template cudaError_t trsm_left_lower<double>(cudaStream_t, int, int, int, const double *, int,
                                             const double *, double *, int, double *);
template cudaError_t trsm_left_lower<float>(cudaStream_t, int, int, int, const float *, int,
                                            const float *, float *, int, float *);

}  // namespace egb
