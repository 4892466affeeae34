// Derivatives of the solve for reverse-mode differentiation (no counterpart in the paper,
// which has no derivatives; these are the first-order perturbation results of the
// generalized symmetric eigenproblem H C = S C diag(eps), C^T S C = I).
//
// Free energy F = E_band - kT S_ent (the entropy term that makes F stationary in the
// occupations at fixed electron count): dF/dH = P and dF/dS = -W.
//
// Eigenpairs: with M = C^T dH C and N = C^T dS C,
//   d eps_j = M_jj - eps_j N_jj,   dC = C Omega,
//   Omega_ij = (M_ij - eps_j N_ij) / (eps_j - eps_i) (i != j),  Omega_jj = -N_jj / 2,
// so a loss with dL/d eps = eb and dL/dC[:, :k] = G has, with A = C^T G and
// F_ij = 1 / (eps_j - eps_i) (zero for i = j and for |eps_i - eps_j| < guard),
//   X_H = diag(eb) + [F o A | 0],
//   X_S = -diag(eb eps) - [(F o A) diag(eps_1..k) | 0] - diag(A_jj / 2, j < k),
//   dL/dH = C sym(X_H) C^T,  dL/dS = C sym(X_S) C^T,  sym(X) = (X + X^T) / 2.
#include "common.cuh"
#include "kernels.h"
#include "solver.h"

namespace egb {

__global__ void dm_adjoint_kernel(size_t total, double fb, const double *__restrict__ p,
                                  const double *__restrict__ w, double *__restrict__ hb,
                                  double *__restrict__ sb)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        hb[e] = fb * p[e];
        if (sb) sb[e] = -fb * w[e];
    }
}

// XH, XS (n x kk, column-major): the matrices X_H, X_S above restricted to their first kk
// columns (kk = n with an eigenvalue upstream, else k).
__global__ void adjoint_x_kernel(int n, int k, int kk, const double *__restrict__ eps,
                                 const double *__restrict__ eb, const double *__restrict__ a,
                                 double guard, double *__restrict__ xh, double *__restrict__ xs)
{
    const size_t total = (size_t)n * kk;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        double vh = 0.0, vs = 0.0;
        if (a && j < k) {
            const double aij = a[(size_t)i + (size_t)j * n];
            const double d = eps[j] - eps[i];
            if (i != j && fabs(d) >= guard) {
                const double fa = aij / d;
                vh += fa;
                vs -= fa * eps[j];
            }
            if (i == j) vs -= 0.5 * aij;
        }
        if (eb && i == j) {
            vh += eb[j];
            vs -= eb[j] * eps[j];
        }
        xh[e] = vh;
        xs[e] = vs;
    }
}

static int grid_for(size_t total)
{
    size_t g = (total + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g ? g : 1);
}

int dm_adjoint(elsi_gb_handle_s *h, int n, double fb, const double *p, const double *w,
               double *hb, double *sb)
{
    const size_t total = (size_t)n * n;
    EGB_COUNT_LAUNCH();
    dm_adjoint_kernel<<<grid_for(total), 256, 0, h->stream>>>(total, fb, p, w, hb, sb);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return set_error(h, ELSI_ERR_CUDA, "free-energy adjoint: %s", cudaGetErrorString(e));
    return ELSI_OK;
}

int ev_adjoint(elsi_gb_handle_s *h, int n, int k, const double *eps, const double *c,
               const double *eb, const double *g, double *hb, double *sb)
{
    const int kk = eb ? n : k;
    if (kk == 0) {  // no upstream at all: zero gradients
        cudaError_t e = cudaMemsetAsync(hb, 0, sizeof(double) * n * (size_t)n, h->stream);
        if (e == cudaSuccess && sb) e = cudaMemsetAsync(sb, 0, sizeof(double) * n * (size_t)n, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        return e == cudaSuccess ? ELSI_OK : set_error(h, ELSI_ERR_CUDA, "adjoint: %s", cudaGetErrorString(e));
    }
    const size_t nk = (size_t)n * (g ? k : 0), nkk = (size_t)n * kk;
    Workspace &w = h->wk;
    if (!ensure_buf((void **)&w.adj, &w.adj_cap, sizeof(double) * (nk + 3 * nkk + 16)))
        return set_error(h, ELSI_ERR_NOMEM, "adjoint scratch");
    double *A = w.adj, *XH = A + nk, *XS = XH + nkk, *Y = XS + nkk;
    cudaStream_t st = h->stream;
    cudaError_t e = cudaSuccess;
#define ACK(x)                                                                             \
    if ((e = (x)) != cudaSuccess)                                                          \
        return set_error(h, ELSI_ERR_CUDA, "eigenpair adjoint: %s", cudaGetErrorString(e));
    if (g) ACK(gemm<double>(st, 1, 0, n, k, n, 1.0, c, n, g, n, 0.0, A, n));
    EGB_COUNT_LAUNCH();
    adjoint_x_kernel<<<grid_for(nkk), 256, 0, st>>>(n, k, kk, eps, eb, g ? A : nullptr, 1e-10, XH, XS);
    ACK(cudaGetLastError());
    // dL/dH = sym(C [X_H | 0] C^T): Y = C X_H (n x kk), then Y C[:, :kk]^T, then sym.
    ACK(gemm<double>(st, 0, 0, n, kk, n, 1.0, c, n, XH, n, 0.0, Y, n));
    ACK(gemm<double>(st, 0, 1, n, n, kk, 1.0, Y, n, c, n, 0.0, hb, n));
    ACK(symmetrize<double>(st, n, hb, n));
    if (sb) {
        ACK(gemm<double>(st, 0, 0, n, kk, n, 1.0, c, n, XS, n, 0.0, Y, n));
        ACK(gemm<double>(st, 0, 1, n, n, kk, 1.0, Y, n, c, n, 0.0, sb, n));
        ACK(symmetrize<double>(st, n, sb, n));
    }
    ACK(cudaStreamSynchronize(st));
#undef ACK
    return ELSI_OK;
}

}  // namespace egb
