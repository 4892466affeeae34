// Complex Hermitian problems (elsi_ev_complex, elsi_dm_complex, elsi_get_edm_complex;
// arXiv:1705.11191 sec. 4.4, "same as elsi_ev_real, except that the matrices are
// complex-valued").
//
// H = A + iB (A symmetric, B antisymmetric) acts on c = x + iy exactly as the real
// symmetric matrix [[A, -B], [B, A]] acts on [x; y]; the same holds for S. The 2n x 2n real
// pencil therefore has every eigenvalue of (H, S) twice, with eigenvectors [x; y] and
// [-y; x]. The solve runs the real route on that pencil (in an internal handle of size
// 2n, with 2 n_state states and 2 n_electron electrons, so that each complex state
// contributes two real states of equal occupation); then
//   eigenvalue l = real eigenvalue 2l, eigenvector l = x + iy from real eigenvector 2l,
//   P = P_emb[0:n, 0:n] + i P_emb[n:2n, 0:n]  (P_emb = [[Re P, -Im P], [Im P, Re P]]),
//   E_band = E_emb / 2.
// Complex arrays are interleaved (re, im) binary64 pairs, column-major.
#include <new>

#include "common.cuh"
#include "kernels.h"
#include "solver.h"

namespace egb {

__global__ void embed_hermitian_kernel(int n, const double *__restrict__ src, double *__restrict__ dst)
{
    const size_t N = 2 * (size_t)n;
    const size_t total = N * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % N), c = (int)(e / N);
        const int i = r % n, j = c % n;
        const double re = src[2 * ((size_t)i + (size_t)j * n)];
        const double im = src[2 * ((size_t)i + (size_t)j * n) + 1];
        double v;
        if ((r < n) == (c < n)) v = re;
        else v = (r < n) ? -im : im;
        dst[e] = v;
    }
}

__global__ void fold_hermitian_kernel(int n, const double *__restrict__ emb, double *__restrict__ dst)
{
    const size_t N = 2 * (size_t)n;
    const size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        dst[2 * e] = emb[(size_t)i + (size_t)j * N];
        dst[2 * e + 1] = emb[(size_t)(i + n) + (size_t)j * N];
    }
}

__global__ void complex_evec_kernel(int n, int k, const double *__restrict__ v, double *__restrict__ dst)
{
    const size_t N = 2 * (size_t)n;
    const size_t total = (size_t)n * k;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), l = (int)(e / n);
        const double *col = v + (size_t)(2 * l) * N;
        dst[2 * e] = col[i];
        dst[2 * e + 1] = col[i + n];
    }
}

__global__ void pair_eval_kernel(int n, const double *__restrict__ w2, double *__restrict__ w)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        w[i] = 0.5 * (w2[2 * i] + w2[2 * i + 1]);
}

static int grid_of(size_t total)
{
    size_t g = (total + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g ? g : 1);
}

__global__ void dup_pairs_kernel(int n, const double *__restrict__ f, double *__restrict__ f2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        f2[2 * i] = f2[2 * i + 1] = f[i];
}

cudaError_t embed_hermitian(cudaStream_t st, int n, const double *src, double *dst)
{
    EGB_COUNT_LAUNCH();
    embed_hermitian_kernel<<<grid_of(4 * (size_t)n * n), 256, 0, st>>>(n, src, dst);
    return cudaGetLastError();
}

cudaError_t fold_hermitian(cudaStream_t st, int n, const double *emb, double *dst)
{
    EGB_COUNT_LAUNCH();
    fold_hermitian_kernel<<<grid_of((size_t)n * n), 256, 0, st>>>(n, emb, dst);
    return cudaGetLastError();
}

cudaError_t pair_evals(cudaStream_t st, int n, const double *w2, double *w)
{
    EGB_COUNT_LAUNCH();
    pair_eval_kernel<<<grid_of(n), 256, 0, st>>>(n, w2, w);
    return cudaGetLastError();
}

cudaError_t dup_pairs(cudaStream_t st, int n, const double *f, double *f2)
{
    EGB_COUNT_LAUNCH();
    dup_pairs_kernel<<<grid_of(n), 256, 0, st>>>(n, f, f2);
    return cudaGetLastError();
}

// Internal handle of size 2n with the parent's settings.
elsi_gb_handle_s *complex_handle(elsi_gb_handle_s *h)
{
    if (!h->cplx) {
        h->cplx = new (std::nothrow) elsi_gb_handle_s();
        if (!h->cplx) return nullptr;
        h->cplx->magic = kHandleMagic;
        h->cplx->occ_stride = 2;
    }
    elsi_gb_handle_s *c = h->cplx;
    if (c->n != 2 * h->n) c->have_l = false;
    c->n = 2 * h->n;
    c->n_state = 2 * h->n_state;
    c->n_electron = 2.0 * h->n_electron;
    c->overlap_is_unit = h->overlap_is_unit;
    c->scheme = h->scheme;
    c->kt = h->kt;
    c->occ_accuracy = 2.0 * h->occ_accuracy;
    c->mu_max_steps = h->mu_max_steps;
    c->precision = h->precision;
    c->band_width = h->band_width;
    c->elpa_solver = h->elpa_solver;
    c->refine_max_iter = h->refine_max_iter;
    c->stream = h->stream;
    c->reuse_l = h->reuse_l;
    return c;
}

int solve_complex(elsi_gb_handle_s *h, const double *ham, const double *ovlp, double *eval,
                  double *evec, double *den_mat, double *energy)
{
    elsi_gb_handle_s *c = complex_handle(h);
    if (!c) return set_error(h, ELSI_ERR_NOMEM, "complex sub-handle");
    const size_t N = 2 * (size_t)h->n;
    Workspace &cw = c->wk;
    if (!ensure_buf((void **)&cw.host_h, &cw.host_h_cap, sizeof(double) * N * N) ||
        (ovlp && !ensure_buf((void **)&cw.host_s, &cw.host_s_cap, sizeof(double) * N * N)) ||
        !ensure_buf((void **)&cw.host_p, &cw.host_p_cap, sizeof(double) * N * N))
        return set_error(h, ELSI_ERR_NOMEM, "complex embedding buffers");
    cudaStream_t st = h->stream;
    EGB_COUNT_LAUNCH();
    embed_hermitian_kernel<<<grid_of(N * N), 256, 0, st>>>(h->n, ham, cw.host_h);
    if (ovlp) {
        EGB_COUNT_LAUNCH();
        embed_hermitian_kernel<<<grid_of(N * N), 256, 0, st>>>(h->n, ovlp, cw.host_s);
    }
    SolveRequest rq;
    rq.ham = cw.host_h;
    rq.ovlp = ovlp ? cw.host_s : nullptr;
    if (evec) {
        // real eigenpairs into the staging buffer: eval (2n) then vectors (2n x 2k)
        if (!ensure_buf((void **)&cw.rfc, &cw.rfc_cap, sizeof(double) * (N + N * 2 * h->n_state + 16)))
            return set_error(h, ELSI_ERR_NOMEM, "complex eigenvector staging");
        rq.eval = cw.rfc;
        rq.evec = cw.rfc + N;
    } else {
        rq.dm = cw.host_p;
        rq.want_edm = true;
    }
    int rc = run_solve(c, rq);
    if (rc) return set_error(h, rc, "%s", c->last_error.c_str());
    if (evec) {
        EGB_COUNT_LAUNCH();
        pair_eval_kernel<<<grid_of(h->n), 256, 0, st>>>(h->n, rq.eval, eval);
        EGB_COUNT_LAUNCH();
        complex_evec_kernel<<<grid_of((size_t)h->n * h->n_state), 256, 0, st>>>(h->n, h->n_state, rq.evec, evec);
    } else {
        EGB_COUNT_LAUNCH();
        fold_hermitian_kernel<<<grid_of((size_t)h->n * h->n), 256, 0, st>>>(h->n, cw.host_p, den_mat);
        if (energy) *energy = 0.5 * c->energy;
        h->mu = c->mu;
        h->energy = 0.5 * c->energy;
        h->entropy = 0.5 * c->entropy;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return set_error(h, ELSI_ERR_CUDA, "complex fold");
    h->refine_iters = c->refine_iters;
    h->orth_err = c->orth_err;
    for (int i = 0; i < kNumStages; ++i) h->stage_ms[i] = c->stage_ms[i];
    h->have_edm = false;
    h->have_occ = false;
    h->have_cedm = !evec;
    return ELSI_OK;
}

int get_edm_complex(elsi_gb_handle_s *h, double *edm)
{
    if (!h->have_cedm || !h->cplx) return set_error(h, ELSI_ERR_STATE, "no complex density-matrix solve yet");
    cudaStream_t st = h->stream;
    EGB_COUNT_LAUNCH();
    fold_hermitian_kernel<<<grid_of((size_t)h->n * h->n), 256, 0, st>>>(h->n, h->cplx->wk.edm, edm);
    if (cudaStreamSynchronize(st) != cudaSuccess) return set_error(h, ELSI_ERR_CUDA, "complex W fold");
    return ELSI_OK;
}

void free_complex(elsi_gb_handle_s *h)
{
    if (h->cplx) {
        if (h->cplx->wk.rfc) cudaFree(h->cplx->wk.rfc);
        h->cplx->wk.rfc = nullptr;
        free_workspace(h->cplx);
        delete h->cplx;
        h->cplx = nullptr;
    }
}

}  // namespace egb
