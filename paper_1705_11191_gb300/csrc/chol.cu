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
    static PerDeviceOnce attr_set;  // per instantiation
    cudaError_t e = once_per_device(attr_set, [] {
        return cudaFuncSetAttribute(potrf_diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(2 * sizeof(T) * kTriBlock * kTriBlock));
    });
    if (e != cudaSuccess) return e;
    EGB_COUNT_LAUNCH();
    potrf_diag_kernel<T><<<1, 256, smem, st>>>(jb, a, lda, inv, ldi, status, base);
    return cudaGetLastError();
}

// Left-looking over panels of kTriPanel columns: the panel's diagonal block is factored by
// kTriBlock blocks (updates inside the block), the rows below it are solved against the
// panel's L (right triangular solve by blocks), and the trailing matrix gets one rank-
// kTriPanel update per panel.
template <typename T>
cudaError_t potrf(cudaStream_t st, int n, T *a, int lda, T *inv_diag, T *work, int *status)
{
    const int nb = kTriBlock, np = kTriPanel;
    cudaError_t e;
    for (int p0 = 0; p0 < n; p0 += np) {
        const int p1 = (n - p0 < np) ? n : p0 + np;
        // (1) diagonal block [p0, p1)
        for (int j0 = p0; j0 < p1; j0 += nb) {
            const int jb = (p1 - j0 < nb) ? p1 - j0 : nb;
            T *a11 = a + j0 + (size_t)j0 * lda;
            T *inv11 = inv_diag + j0;  // ld = n
            if ((e = launch_potrf_diag<T>(st, jb, a11, lda, inv11, n, status, j0)) != cudaSuccess) return e;
            const int m2 = p1 - j0 - jb;
            if (m2 > 0) {
                T *a21 = a + (j0 + jb) + (size_t)j0 * lda;
                T *a22 = a + (j0 + jb) + (size_t)(j0 + jb) * lda;
                if ((e = gemm<T>(st, 0, 1, m2, jb, jb, T(1), a21, lda, inv11, n, T(0), work, m2)) != cudaSuccess) return e;
                if ((e = cudaMemcpy2DAsync(a21, sizeof(T) * lda, work, sizeof(T) * m2, sizeof(T) * m2, jb,
                                           cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
                if ((e = gemm<T>(st, 0, 1, m2, m2, jb, T(-1), a21, lda, a21, lda, T(1), a22, lda, 1)) != cudaSuccess) return e;
            }
        }
        const int m2 = n - p1;
        if (m2 <= 0) continue;
        // (2) rows below: X L_pp^T = A21, block column by block column
        T *a21 = a + p1 + (size_t)p0 * lda;
        for (int j0 = p0; j0 < p1; j0 += nb) {
            const int jb = (p1 - j0 < nb) ? p1 - j0 : nb;
            T *xj = a + p1 + (size_t)j0 * lda;
            if (j0 > p0) {
                // A21_j -= X_{p0..j0} L_{j, p0..j0}^T
                if ((e = gemm<T>(st, 0, 1, m2, jb, j0 - p0, T(-1), a21, lda, a + j0 + (size_t)p0 * lda, lda,
                                 T(1), xj, lda)) != cudaSuccess) return e;
            }
            if ((e = gemm<T>(st, 0, 1, m2, jb, jb, T(1), xj, lda, inv_diag + j0, n, T(0), work, m2)) != cudaSuccess) return e;
            if ((e = cudaMemcpy2DAsync(xj, sizeof(T) * lda, work, sizeof(T) * m2, sizeof(T) * m2, jb,
                                       cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
        }
        // (3) A22 -= L21 L21^T (lower triangle), K = panel width
        T *a22 = a + p1 + (size_t)p1 * lda;
        if ((e = gemm<T>(st, 0, 1, m2, m2, p1 - p0, T(-1), a21, lda, a21, lda, T(1), a22, lda, 1)) != cudaSuccess) return e;
    }
    size_t total = (size_t)n * n;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    EGB_COUNT_LAUNCH();
    zero_upper_kernel<T><<<grid, 256, 0, st>>>(n, a, lda);
    return cudaGetLastError();
}

// Triangular solve restricted to the row range [r0, r1): the blocks of kTriBlock rows in the
// range are solved one after another and each updates only the rows of the range.
template <typename T>
static cudaError_t trsm_range(cudaStream_t st, int trans, int r0, int r1, int ncol, const T *L,
                              int ldl, const T *inv_diag, int ldi, T *B, int ldb, T *work)
{
    const int nb = kTriBlock;
    cudaError_t e;
    const int nblk = ceil_div(r1 - r0, nb);
    for (int bi = 0; bi < nblk; ++bi) {
        const int blk = trans ? (nblk - 1 - bi) : bi;
        const int j0 = r0 + blk * nb;
        const int jb = (r1 - j0 < nb) ? r1 - j0 : nb;
        const T *inv11 = inv_diag + j0;
        T *bj = B + j0;
        // B_j := inv(L_jj) B_j   or   inv(L_jj)^T B_j
        if ((e = gemm<T>(st, trans, 0, jb, ncol, jb, T(1), inv11, ldi, bj, ldb, T(0), work, jb)) != cudaSuccess) return e;
        if ((e = cudaMemcpy2DAsync(bj, sizeof(T) * ldb, work, sizeof(T) * jb, sizeof(T) * jb, ncol,
                                   cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
        if (!trans) {
            const int m2 = r1 - j0 - jb;
            if (m2 > 0) {
                const T *l21 = L + (j0 + jb) + (size_t)j0 * ldl;
                if ((e = gemm<T>(st, 0, 0, m2, ncol, jb, T(-1), l21, ldl, bj, ldb, T(1), B + j0 + jb, ldb)) != cudaSuccess) return e;
            }
        } else if (j0 > r0) {
            // B_{r0..j0} -= (L_{j, r0..j0})^T B_j
            const T *lj = L + j0 + (size_t)r0 * ldl;
            if ((e = gemm<T>(st, 1, 0, j0 - r0, ncol, jb, T(-1), lj, ldl, bj, ldb, T(1), B + r0, ldb)) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// Two block levels: panels of kTriPanel rows are solved by trsm_range (kTriBlock blocks with
// updates inside the panel); the rest of B is updated once per panel with K = kTriPanel,
// which keeps the read-modify-write traffic on B at n / kTriPanel passes.
template <typename T>
cudaError_t trsm_left_lower(cudaStream_t st, int trans, int n, int ncol, const T *L, int ldl,
                            const T *inv_diag, T *B, int ldb, T *work)
{
    constexpr int np = kTriPanel;
    cudaError_t e;
    if (n <= 0 || ncol <= 0) return cudaSuccess;
    const int npan = ceil_div(n, np);
    for (int pi = 0; pi < npan; ++pi) {
        const int pan = trans ? (npan - 1 - pi) : pi;
        const int r0 = pan * np, r1 = (n - r0 < np) ? n : r0 + np;
        if ((e = trsm_range<T>(st, trans, r0, r1, ncol, L, ldl, inv_diag, n, B, ldb, work)) != cudaSuccess) return e;
        if (!trans) {
            if (r1 < n) {
                // B_{r1..n} -= L_{r1..n, r0..r1} B_{r0..r1}
                if ((e = gemm<T>(st, 0, 0, n - r1, ncol, r1 - r0, T(-1), L + r1 + (size_t)r0 * ldl, ldl,
                                 B + r0, ldb, T(1), B + r1, ldb)) != cudaSuccess) return e;
            }
        } else if (r0 > 0) {
            // B_{0..r0} -= (L_{r0..r1, 0..r0})^T B_{r0..r1}
            if ((e = gemm<T>(st, 1, 0, r0, ncol, r1 - r0, T(-1), L + r0, ldl, B + r0, ldb, T(1), B, ldb)) != cudaSuccess) return e;
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
