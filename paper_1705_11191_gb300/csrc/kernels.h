// Internal launchers of the solver kernels (not part of the C ABI).
// All matrices are column-major; every launcher enqueues on `st` and returns the launch
// status (cudaSuccess or the error of the launch).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace egb {

// C = alpha * op(A) * op(B) + beta * C, op(A) m x k, op(B) k x n. ta/tb: 0 = N, 1 = T.
// uplo = 1: only the lower triangle (row >= col) of C is computed and written.
// beta == 0 means C is not read.
template <typename T>
cudaError_t gemm(cudaStream_t st, int ta, int tb, int m, int n, int k, T alpha,
                 const T *A, int lda, const T *B, int ldb, T beta, T *C, int ldc,
                 int uplo = 0);

// Binary32-accuracy GEMM on the tcgen05 tensor cores (three TF32 products of hi/lo splits;
// tc_gemm.cu). work: tc_gemm_work_elems(m, n, k) floats, 16-byte aligned. Returns
// cudaErrorNotSupported when it cannot run (scratch too small, no tensor-map encoder).
size_t tc_gemm_work_elems(int m, int n, int k);

// X (m x nv, ldx) = A V for a symmetric m x m binary32 A (full storage, lda a multiple of 4,
// 16-byte aligned) and an m x nv panel V (nv <= 64), binary32 accuracy on the tensor cores
// (symm_tall.cu). work: symm_tall_work_elems(m) floats, 16-byte aligned. Returns
// cudaErrorNotSupported when the operands do not fit its constraints.
size_t symm_tall_work_elems(int m);
cudaError_t symm_tall_f32(cudaStream_t st, int m, int nv, const float *A, int lda, const float *V,
                          int ldv, float *X, int ldx, float *work, size_t work_elems, int *status);
// Sum of products over K pieces: C = alpha * sum_i op(A_i) op(B_i) + beta * C, piece i of
// width k (the same for A_i and B_i), op(A_i) m x k (trans = 0: p[r + q ld], 1: p[q + r ld]),
// op(B_i) k x n (trans = 0: p[q + c ld], 1: p[c + q ld]).
struct TcPart {
    const float *p;
    int ld, trans, k;
};
cudaError_t tc_gemm_f32_parts(cudaStream_t st, int m, int n, int nparts, const TcPart *a,
                              const TcPart *b, float alpha, float beta, float *C, int ldc, int uplo,
                              float *work, size_t work_elems, int *status);
// Scratch of this thread's current solve for the tensor-core path (nullptr if none).
bool tc_scratch(float **work, size_t *elems, int **status);
// Routes this thread's binary32 gemm() calls with large enough shapes to tc_gemm_f32 with
// the given scratch (work = nullptr: SIMT kernel only).
void set_tc_scratch(float *work, size_t elems, int *status);
// Routes this thread's binary64 gemm() calls with large enough shapes to binary64-accurate
// digit products on the tensor cores (ozaki_split + ozaki_gemm) with the given digit-plane
// and exponent scratch (planes = nullptr: SIMT binary64 kernel only). Uses the status word
// of set_tc_scratch for timeouts.
void set_f64_tc_scratch(__nv_bfloat16 *planes, size_t elems, int *exps, size_t exp_elems);
cudaError_t tc_gemm_f32(cudaStream_t st, int ta, int tb, int m, int n, int k, float alpha,
                        const float *A, int lda, const float *B, int ldb, float beta, float *C,
                        int ldc, int uplo, float *work, size_t work_elems, int *status);

// C = alpha * op(A) * op(B) with K split over several CTAs (for small outputs with a long
// K); part: scratch of part_elems elements for the partial products.
template <typename T>
cudaError_t gemm_splitk(cudaStream_t st, int ta, int tb, int m, int n, int k, T alpha,
                        const T *A, int lda, const T *B, int ldb, T *C, int ldc, T *part,
                        size_t part_elems);

// dst(m x n, ldd) = src(m x n, lds), with type conversion.
template <typename Td, typename Ts>
cudaError_t copy_matrix(cudaStream_t st, int m, int n, const Ts *src, int lds, Td *dst, int ldd);

// a(n x n): upper triangle := transpose of the lower triangle.
template <typename T>
cudaError_t mirror_lower(cudaStream_t st, int n, T *a, int lda);

// dst(n x m) = src(m x n)^T
template <typename T>
cudaError_t transpose(cudaStream_t st, int m, int n, const T *src, int lds, T *dst, int ldd);

// a := (a + a^T) / 2 for an n x n matrix.
template <typename T>
cudaError_t symmetrize(cudaStream_t st, int n, T *a, int lda);

// Sets status ELSI_ERR_NONFINITE if any entry of the m x n matrix is NaN/Inf.
template <typename T>
cudaError_t check_finite(cudaStream_t st, int m, int n, const T *a, int lda, int *status);

// ---- Cholesky and triangular solves (Eqs. 8-9) ----
// Lower Cholesky of the n x n matrix a in place (upper triangle zeroed). inv_diag
// receives the inverses of the nb x nb diagonal blocks of L (n x nb, block j at rows
// j*nb). work: n x nb scratch. Status ELSI_ERR_NOT_PD with the pivot on failure.
template <typename T>
cudaError_t potrf(cudaStream_t st, int n, T *a, int lda, T *inv_diag, T *work, int *status);
constexpr int kTriBlock = 64;   // nb of potrf / trsm
constexpr int kTriPanel = 256;  // outer panel of trsm (rank-256 updates of the rest of B)

// B (n x ncol) := L^{-1} B (trans = 0) or L^{-T} B (trans = 1), L lower from potrf,
// inv_diag its diagonal-block inverses. work: kTriBlock x ncol scratch.
template <typename T>
cudaError_t trsm_left_lower(cudaStream_t st, int trans, int n, int ncol, const T *L, int ldl,
                            const T *inv_diag, T *B, int ldb, T *work);

// ---- full -> band (Eq. 11, first line) ----
template <typename T>
cudaError_t sy2sb(cudaStream_t st, int n, int b, T *a, int lda, T *v1, T *t1, T *work,
                  size_t work_elems, unsigned *sync, int *status, int num_sms);
size_t sy2sb_work_elems(int n, int b);

// ---- band -> tridiagonal (Eq. 11, second line) ----
// band: lower band storage with ldb >= 2b+1 (element (r,c), r>=c, at band[(r-c) + c*ldb]).
// Outputs d (n), e (n-1) as double, reflectors v2 (b per slot) and tau2.
int sb2st_steps(int n, int b);
template <typename T>
cudaError_t sb2st(cudaStream_t st, int n, int b, T *band, int ldb, double *d, double *e,
                  T *v2, T *tau2, int *status, unsigned *sync, int num_sms);
template <typename T>
cudaError_t extract_band(cudaStream_t st, int n, int b, const T *a, int lda, T *band, int ldb);

// ---- tridiagonal eigensolver (sec. 3.1, step 3) ----
// Eigenvalues 0..count-1 (ascending) of the symmetric tridiagonal (d, e) by Sturm
// bisection (w needs count + 8 entries: the Gershgorin bounds follow the values), then
// eigenvectors of the first kvec of them into z (n x kvec, ldz) as type T.
// scratch: 3*n*kvec + kvec + 16 doubles.
// tol_rel: stop when the bracket is narrower than tol_rel * ||T|| (0: full binary64).
// Off-diagonals of e below 2 eps ||T|| are set to zero first (T splits into blocks).
cudaError_t stebz(cudaStream_t st, int n, const double *d, double *e, int count,
                  double *w, int *status, double tol_rel = 0.0);
template <typename T>
cudaError_t stein(cudaStream_t st, int n, const double *d, const double *e, int kvec,
                  const double *w, T *z, int ldz, double *scratch, int *status);

// ---- back-transformations (steps 4 and 5) ----
template <typename T>
cudaError_t apply_q2(cudaStream_t st, int n, int b, const T *v2, const T *tau2, int k,
                     T *z, int ldz, int *status);
// binary32 Z <- Q2 Z with compact-WY groups of 64 reflectors on the tcgen05 tensor cores
// (q2tc.cu); fac: scratch of q2_factor_elems(n, b) floats (16-byte aligned) for the
// per-group operand blocks; b a multiple of 8 in 8..64. Timeouts of its bounded waits go
// to status (ELSI_ERR_TIMEOUT).
size_t q2_factor_elems(int n, int b);
cudaError_t apply_q2_tc(cudaStream_t st, int n, int b, const float *v2, const float *tau2, int k,
                        float *z, int ldz, float *fac, int *status);
// Z <- Q1 Z in groups of kQ1Group panels; work: q1_work_elems(b, k) elements.
constexpr int kQ1Group = 4;
inline size_t q1_work_elems(int b, int k)
{
    const size_t g = (size_t)kQ1Group * b;
    return g * g + 2 * g * b + 4 * g * (size_t)k + 64;
}
template <typename T>
cudaError_t apply_q1(cudaStream_t st, int n, int b, int k, const T *v1, const T *t1, T *z,
                     int ldz, T *work);

// ---- one-stage tridiagonalisation (Eq. 11 line 1; onestage.cu) ----
constexpr int kOneStageNb = 32;  // panel width (T factors: kOneStageNb x n in t1)
size_t onestage_work_elems(int n);  // binary64 scratch elements
template <typename T>
cudaError_t onestage_tridiag(cudaStream_t st, int n, T *A, int lda, double *d, double *e, T *v1,
                             T *t1, double *work);
// Z <- Q Z; work: 18 kOneStageNb k elements
template <typename T>
cudaError_t apply_q_onestage(cudaStream_t st, int n, int k, const T *v1, const T *t1, T *z, int ldz,
                             T *work);

// ---- occupation, density matrices ----
// stride 2: consecutive pairs of states are one complex state (see density.cu).
cudaError_t occupation(cudaStream_t st, int k, const double *eps, double n_el, int scheme,
                       double kt, double occ_accuracy, int mu_max_steps, double *f,
                       double *out /* [0]=mu [1]=energy */, int *status, int stride = 1);
// One chemical potential over m weighted entries of several problems (see density.cu).
cudaError_t occupation_weighted(cudaStream_t st, int m, const double *eps, const double *wt,
                                double n_el, int scheme, double kt, double occ_accuracy,
                                int mu_max_steps, double *f, double *out /* [0]=mu [1]=energy */,
                                int *status);
// out[i] = sum_{off[i] <= j < off[i+1]} f[j] eps[j] (off: device, nseg + 1 ints).
cudaError_t segment_energy(cudaStream_t st, int nseg, const int *off, const double *f,
                           const double *eps, double *out);
// P = C diag(f) C^T and W = C diag(f eps) C^T (lower + mirror); cw: n x k scratch.
template <typename T>
cudaError_t density_pw(cudaStream_t st, int n, int k, const T *c, int ldc, const double *f,
                       const double *eps, T *p, T *w, T *cw);

// ---- complex Hermitian problems through the real form (complex.cu) ----
// dst (2n x 2n) = [[Re A, -Im A], [Im A, Re A]] of A (n x n, interleaved complex).
cudaError_t embed_hermitian(cudaStream_t st, int n, const double *src, double *dst);
// dst (n x n complex) = emb[0:n, 0:n] + i emb[n:2n, 0:n].
cudaError_t fold_hermitian(cudaStream_t st, int n, const double *emb, double *dst);
// w[i] = (w2[2i] + w2[2i+1]) / 2: one eigenvalue per pair of the real form.
cudaError_t pair_evals(cudaStream_t st, int n, const double *w2, double *w);
// f2[2i] = f2[2i+1] = f[i].
cudaError_t dup_pairs(cudaStream_t st, int n, const double *f, double *f2);

// ---- binary64-accurate products on the bf16 tensor cores (ozaki.cu) ----
// Splits V vectors of length K (element (v, q) at src[v * sv + q * sq], optionally times
// scale[q] * scale2[q]) into the digit planes consumed by ozaki_gemm.
size_t ozaki_split_elems(int V, int K);  // bf16 elements of the planes of V vectors
cudaError_t ozaki_split(cudaStream_t st, int V, int K, const double *src, long long sv,
                        long long sq, const double *scale, const double *scale2,
                        __nv_bfloat16 *planes, int *exps);
// C (m x n, ldc) = alpha * A B + beta * C with A given by the split of its m rows and B
// by the split of its n columns (both of length k). uplo = 1: lower triangle only.
// digits (1..7, default 7): leading digit planes used, i.e. D(D+1)/2 digit products and a
// truncation error of about 2^(-7(D+1)) relative to max|A_i.| max|B_.j| per product term.
constexpr int kOzDigits = 7;
cudaError_t ozaki_gemm(cudaStream_t st, int m, int n, int k, double alpha,
                       const __nv_bfloat16 *Ad, const int *ea, const __nv_bfloat16 *Bd,
                       const int *eb, double beta, double *C, int ldc, int uplo,
                       int digits = kOzDigits);

}  // namespace egb
