/*
 * Internal kernels of libelsi_gb exposed for their own tests (not part of the solver
 * interface of arXiv:1705.11191; no counterpart in the paper).
 *
 * elsi_gb_gemm_f32: the binary32 GEMM of the reduction and back-transformations,
 *   C (m x n, column-major, ldc) = alpha * op(A) op(B) + beta * C,
 *   op(A) m x k (ta = 0: A column-major m x k, lda; ta = 1: A is k x m), op(B) k x n
 *   (tb likewise), on the tcgen05 tensor cores as three TF32 products of hi/lo splits.
 *   uplo = 1 writes only the lower triangle (row >= column) of C. All pointers are
 *   device pointers; work: device scratch of elsi_gb_gemm_f32_work(m, n, k) floats
 *   (16-byte aligned); status: device int[8], zeroed by the caller, receives
 *   ELSI_ERR_TIMEOUT if a pipeline wait expired. Enqueued on stream (cudaStream_t, may
 *   be NULL); returns 0, ELSI_ERR_ARG for bad sizes or scratch, ELSI_ERR_CUDA.
 */
#ifndef ELSI_GB_TESTING_H
#define ELSI_GB_TESTING_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * elsi_gb_set_spin_limit: iteration limit of the library's SIMT spin waits (the grid
 *   barrier of the cooperative panel factorisation and the per-sweep progress flags of the
 *   bulge chase; the mbarrier waits of the tensor-core pipelines keep their own limit).
 *   A wait that has polled more than `polls` times records ELSI_ERR_TIMEOUT in the
 *   solve's status word and its kernel returns, so the solve returns ELSI_ERR_TIMEOUT and
 *   the CUDA context stays usable. Process-wide; read at each launch. Default 2^26
 *   (seconds); 0 makes every wait that has to wait at all expire. Returns ELSI_ERR_ARG
 *   for polls < 0. elsi_gb_get_spin_limit returns the limit in force.
 */
int elsi_gb_set_spin_limit(long long polls);
long long elsi_gb_get_spin_limit(void);

/*
 * elsi_gb_q2_apply_f32: the binary32 back-transformation through Q2 of the band-to-
 *   tridiagonal reduction (step (4) of the two-stage method, sec. 3.1), Z <- Q2 Z, on the
 *   tcgen05 tensor cores. v2: device float[(n-2) * S * b], S = (n-2)/b + 1, the Householder
 *   vector of bulge-chase step t of sweep j at v2[(j*S + t)*b ...] (v[0] = 1, acting on rows
 *   j+1+t*b .. j+t*b+b, entries beyond row n-1 zero); tau2: device float[(n-2) * S];
 *   Z: device n x k column-major, ld ldz >= n; b a multiple of 8 in 8..64. work: device
 *   scratch of elsi_gb_q2_work(n, b) floats (16-byte aligned); status: device int[8], zeroed
 *   by the caller (ELSI_ERR_TIMEOUT if a bounded wait expired). Enqueued on stream (may be
 *   NULL). Returns 0, ELSI_ERR_ARG, ELSI_ERR_CUDA.
 */
size_t elsi_gb_q2_work(int n, int b);
int elsi_gb_q2_apply_f32(int n, int b, const float *v2, const float *tau2, int k, float *z, int ldz,
                         float *work, size_t work_elems, int *status, void *stream);

/*
 * elsi_gb_symm_tall_f32: X (m x nv, column-major, ldx) = A V for a symmetric m x m binary32
 *   matrix A (full column-major storage, lda a multiple of 4, A 16-byte aligned) and an
 *   m x nv panel V (ldv), 1 <= nv <= 64: the product A22 V of the two-sided update of the
 *   full-to-band reduction (Eq. 11, sec. 3.1), binary32 accuracy on the tcgen05 tensor
 *   cores, A read once (split into TF32 hi/lo parts in shared memory). Only the symmetry of
 *   A is used: column i of A stands for row i. work: device scratch of
 *   elsi_gb_symm_tall_f32_work(m) floats (16-byte aligned); status: device int[8], zeroed
 *   by the caller (ELSI_ERR_TIMEOUT if a pipeline wait expired). Enqueued on stream (may
 *   be NULL). Returns 0, ELSI_ERR_ARG for bad sizes, alignment or scratch, ELSI_ERR_CUDA.
 */
size_t elsi_gb_symm_tall_f32_work(int m);
int elsi_gb_symm_tall_f32(int m, int nv, const float *A, int lda, const float *V, int ldv, float *X,
                          int ldx, float *work, size_t work_elems, int *status, void *stream);

size_t elsi_gb_gemm_f32_work(int m, int n, int k);
int elsi_gb_gemm_f32(int ta, int tb, int m, int n, int k, float alpha, const float *A, int lda,
                     const float *B, int ldb, float beta, float *C, int ldc, int uplo,
                     float *work, size_t work_elems, int *status, void *stream);

/*
 * elsi_gb_gemm_f64_digits: the binary64-accurate product of the refinement and of P, W
 *   (Ozaki et al., Numer. Algorithms 59 (2012), integer-digit form):
 *   C (m x n, column-major, ldc) = alpha * op(A) op(B) + beta * C, op() as for
 *   elsi_gb_gemm_f32, every row of op(A) and column of op(B) cut into `digits` (1..7)
 *   signed 7-bit digits after scaling by a power of two, the digit products summed
 *   exactly on the bf16 tensor cores, levels 2..digits+1 kept (truncation about
 *   2^(-7 digits) relative to max|op(A)_i.| max|op(B)_.j| per term). uplo = 1 writes
 *   only the lower triangle of C. planes: device scratch of
 *   elsi_gb_gemm_f64_digits_planes(m, n, k) bf16 values (2 bytes each; 16-byte aligned);
 *   exps: device int[elsi_gb_gemm_f64_digits_exps(m, n)]; status: device int[8], zeroed
 *   by the caller (ELSI_ERR_TIMEOUT if a pipeline wait expired). Any k >= 1 (products
 *   longer than 32768 run as several K segments added in binary64). Enqueued on stream
 *   (may be NULL). Returns 0, ELSI_ERR_ARG for bad sizes, digits or scratch,
 *   ELSI_ERR_CUDA.
 */
size_t elsi_gb_gemm_f64_digits_planes(int m, int n, int k);
size_t elsi_gb_gemm_f64_digits_exps(int m, int n);
int elsi_gb_gemm_f64_digits(int ta, int tb, int m, int n, int k, double alpha, const double *A,
                            int lda, const double *B, int ldb, double beta, double *C, int ldc,
                            int uplo, int digits, void *planes, size_t plane_elems, int *exps,
                            size_t exp_elems, int *status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ELSI_GB_TESTING_H */
