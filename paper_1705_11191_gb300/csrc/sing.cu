// Singularity check of the overlap matrix and the eigendecomposition transformation
// (arXiv:1705.11191 sec. 4.4, Eq. 10).
//
// All eigenvalues of S are computed and compared with the tolerance tau. If one or more
// are below tau (or the handle asks for the transformation always), the Cholesky
// factorisation is replaced by S = X X^T with X = x sqrt(lambda), the eigenvectors with
// lambda < tau dropped. With U = x_k lambda_k^{-1/2} (n x N_nonsing):
//     H~ = U^T H U  (N_nonsing x N_nonsing, standard form),   c = U c~,
// and C^T S C = I holds because U^T S U = I. The eigenpairs of S come from the solver
// itself: an internal handle solves the standard problem -S (its lowest eigenpairs are the
// largest of S); a second internal handle solves the reduced standard problem H~ in the
// precision of the parent handle. The transformation is kept for the next calls when the
// overlap factor is reused (elsi_set_reuse_ovlp_factor), like the Cholesky factor.
#include <cfloat>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "solver.h"

namespace egb {

struct SingState {
    elsi_gb_handle_s *sh = nullptr;  // eigendecomposition of -S (size n)
    elsi_gb_handle_s *rh = nullptr;  // reduced standard problem (size N_nonsing)
#define EGB_BUF(type, name) type *name = nullptr; size_t name##_cap = 0;
    EGB_BUF(double, negs)  // -S (n x n)
    EGB_BUF(double, vecs)  // eigenvectors of -S (n x n)
    EGB_BUF(double, evs)   // eigenvalues of -S (n)
    EGB_BUF(double, u)     // U (n x N_nonsing)
    EGB_BUF(double, w1)    // H U (n x N_nonsing)
    EGB_BUF(double, ht)    // H~ (N_nonsing x N_nonsing)
    EGB_BUF(double, evr)   // eigenvalues of H~ (N_nonsing)
    EGB_BUF(double, z)     // eigenvectors of H~ (N_nonsing x n_state)
    EGB_BUF(double, c)     // C = U Z (n x n_state), density-matrix calls
#undef EGB_BUF
    bool ready = false;  // a transformation decision for the current S exists
    int nn = 0;          // N_nonsing of that decision
};

#define SCK(...)                                                                           \
    do {                                                                                   \
        cudaError_t _e = (__VA_ARGS__);                                                    \
        if (_e != cudaSuccess)                                                             \
            return set_error(h, ELSI_ERR_CUDA, "%s failed: %s", #__VA_ARGS__,              \
                             cudaGetErrorString(_e));                                      \
    } while (0)

#define SENSURE(name, count)                                                               \
    if (!ensure_buf((void **)&g.name, &g.name##_cap, sizeof(double) * (size_t)(count)))   \
        return set_error(h, ELSI_ERR_NOMEM, "cannot allocate singularity-check %s", #name);

static int grid_of(size_t total)
{
    size_t g = (total + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g ? g : 1);
}

__global__ void negate_kernel(size_t total, const double *__restrict__ src, double *__restrict__ dst)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x)
        dst[e] = -src[e];
}

// U[:, j] = x[:, j] / sqrt(lambda_j) with lambda_j = -evs[j] (the j-th largest eigenvalue of S)
__global__ void canonical_columns_kernel(int n, int nn, const double *__restrict__ vecs,
                                         const double *__restrict__ evs, double *__restrict__ u)
{
    const size_t total = (size_t)n * nn;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / n);
        u[e] = vecs[e] / sqrt(-evs[j]);
    }
}

// eigenvalues of the reduced problem, then DBL_MAX in the slots of the dropped directions
__global__ void fill_eval_kernel(int n, int nn, const double *__restrict__ evr, double *__restrict__ w)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        w[i] = (i < nn) ? evr[i] : DBL_MAX;
}

static elsi_gb_handle_s *new_sub()
{
    elsi_gb_handle_s *s = new (std::nothrow) elsi_gb_handle_s();
    if (s) s->magic = kHandleMagic;
    return s;
}

static SingState *sing_state(elsi_gb_handle_s *h)
{
    if (!h->sing) h->sing = new (std::nothrow) SingState();
    if (!h->sing) return nullptr;
    if (!h->sing->sh) h->sing->sh = new_sub();
    if (!h->sing->rh) h->sing->rh = new_sub();
    if (!h->sing->sh || !h->sing->rh) return nullptr;
    return h->sing;
}

int sing_prepare(elsi_gb_handle_s *h, const double *ovlp, bool *active)
{
    SingState *gp = sing_state(h);
    if (!gp) return set_error(h, ELSI_ERR_NOMEM, "singularity-check state");
    SingState &g = *gp;
    const int n = h->n;
    if (h->reuse_l && g.ready) {
        *active = g.nn < n || h->sing_mode == 2;
        h->n_nonsing = g.nn;
        return ELSI_OK;
    }
    g.ready = false;
    cudaStream_t st = h->stream;
    SENSURE(negs, (size_t)n * n);
    SENSURE(vecs, (size_t)n * n);
    SENSURE(evs, (size_t)n + 8);
    EGB_COUNT_LAUNCH();
    negate_kernel<<<grid_of((size_t)n * n), 256, 0, st>>>((size_t)n * n, ovlp, g.negs);
    SCK(cudaGetLastError());
    elsi_gb_handle_s *s = g.sh;
    s->n = n;
    s->n_state = n;
    s->n_electron = 0.0;
    s->overlap_is_unit = true;
    s->precision = ELSI_PREC_FP64;
    s->band_width = h->band_width;
    s->stream = st;
    SolveRequest q;
    q.ham = g.negs;
    q.eval = g.evs;
    q.evec = g.vecs;
    int rc = run_solve(s, q);
    if (rc) return set_error(h, rc, "eigendecomposition of the overlap: %s", s->last_error.c_str());
    std::vector<double> ev(n);
    SCK(cudaMemcpyAsync(ev.data(), g.evs, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    int nn = 0;  // eigenvalues of S = -ev, descending: count those >= tau
    while (nn < n && -ev[nn] >= h->sing_tol) ++nn;
    h->have_l = false;
    if (nn == n && h->sing_mode != 2) {
        g.ready = true;
        g.nn = n;
        h->n_nonsing = n;
        *active = false;
        return ELSI_OK;
    }
    if (nn == 0)
        return set_error(h, ELSI_ERR_NOT_PD, "every eigenvalue of the overlap is below the singularity tolerance %g",
                         h->sing_tol);
    SENSURE(u, (size_t)n * nn);
    EGB_COUNT_LAUNCH();
    canonical_columns_kernel<<<grid_of((size_t)n * nn), 256, 0, st>>>(n, nn, g.vecs, g.evs, g.u);
    SCK(cudaGetLastError());
    g.ready = true;
    g.nn = nn;
    h->n_nonsing = nn;
    *active = true;
    return ELSI_OK;
}

int solve_singular(elsi_gb_handle_s *h, const SolveRequest &rq)
{
    SingState &g = *h->sing;
    const int n = h->n, k = h->n_state, nn = g.nn;
    const bool ev_mode = rq.evec != nullptr;
    if (k > nn)
        return set_error(h, ELSI_ERR_ARG, "n_state %d exceeds the %d non-singular basis directions", k, nn);
    int rc = ensure_workspace(h, k);
    if (rc) return rc;
    Workspace &w = h->wk;
    // scratch of the density-matrix products below: n x k binary64 values
    if (!ensure_buf((void **)&w.v1, &w.v1_cap, sizeof(double) * (size_t)n * k))
        return set_error(h, ELSI_ERR_NOMEM, "cannot allocate the density scratch");
    cudaStream_t st = h->stream;
    SCK(cudaMemsetAsync(w.status, 0, sizeof(int) * ST_WORDS, st));
    SENSURE(w1, (size_t)n * nn);
    SENSURE(ht, (size_t)nn * nn);
    SENSURE(evr, (size_t)nn + 8);
    SENSURE(z, (size_t)nn * k);
    if (!ev_mode) SENSURE(c, (size_t)n * k);
    // ---- H~ = U^T H U
    SCK(check_finite<double>(st, n, n, rq.ham, n, w.status));
    SCK(gemm<double>(st, 0, 0, n, nn, n, 1.0, rq.ham, n, g.u, n, 0.0, g.w1, n));
    SCK(gemm<double>(st, 1, 0, nn, nn, n, 1.0, g.u, n, g.w1, n, 0.0, g.ht, nn));
    SCK(symmetrize<double>(st, nn, g.ht, nn));
    // ---- reduced standard problem (the parent's route and settings)
    elsi_gb_handle_s *r = g.rh;
    r->n = nn;
    r->n_state = k;
    r->n_electron = h->n_electron;
    r->overlap_is_unit = true;
    r->precision = h->precision;
    r->band_width = h->band_width;
    r->elpa_solver = h->elpa_solver;
    r->refine_max_iter = h->refine_max_iter;
    r->stream = st;
    SolveRequest q;
    q.ham = g.ht;
    q.eval = g.evr;
    q.evec = g.z;
    rc = run_solve(r, q);
    if (rc) return set_error(h, rc, "reduced problem: %s", r->last_error.c_str());
    // ---- c = U c~, eigenvalues (dropped directions at DBL_MAX)
    double *C = ev_mode ? rq.evec : g.c;
    SCK(gemm<double>(st, 0, 0, n, k, nn, 1.0, g.u, n, g.z, nn, 0.0, C, n));
    EGB_COUNT_LAUNCH();
    fill_eval_kernel<<<grid_of(n), 256, 0, st>>>(n, nn, g.evr, w.w);
    SCK(cudaGetLastError());
    if (ev_mode) {
        SCK(cudaMemcpyAsync(rq.eval, w.w, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    } else {
        SCK(occupation(st, k, w.w, h->n_electron, h->scheme, h->kt, h->occ_accuracy, h->mu_max_steps,
                       w.f, w.scal, w.status, h->occ_stride));
        int kocc = k;
        if (h->scheme == ELSI_OCC_INTEGER) {
            kocc = (int)((h->n_electron / h->occ_stride + 1.999999999) / 2.0) * h->occ_stride;
            if (kocc > k) kocc = k;
            if (kocc < 1) kocc = 1;
        }
        SCK(density_pw<double>(st, n, kocc, C, n, w.f, w.w, rq.dm, rq.want_edm ? w.edm : nullptr, w.v1));
    }
    SCK(cudaMemcpyAsync(w.status_host, w.status, sizeof(int) * ST_WORDS, cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(w.scal_host, w.scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    for (int i = 0; i < kNumStages; ++i) h->stage_ms[i] = r->stage_ms[i];
    h->refine_iters = r->refine_iters;
    h->orth_err = r->orth_err;
    if (w.status_host[ST_CODE] != 0) {
        h->have_edm = h->have_occ = false;
        if (w.status_host[ST_CODE] == ELSI_ERR_NONFINITE)
            return set_error(h, ELSI_ERR_NONFINITE, "non-finite value in the input");
        return set_error(h, w.status_host[ST_CODE], "device error %d", w.status_host[ST_CODE]);
    }
    if (!ev_mode) {
        h->mu = w.scal_host[0];
        h->energy = w.scal_host[1];
        h->entropy = w.scal_host[2];
        h->have_occ = true;
        h->have_edm = rq.want_edm;
    } else {
        h->have_edm = false;
    }
    return ELSI_OK;
}

void sing_invalidate(elsi_gb_handle_s *h)
{
    if (h->sing) h->sing->ready = false;
}

void free_sing(elsi_gb_handle_s *h)
{
    if (!h->sing) return;
    SingState &g = *h->sing;
    void *bufs[] = {g.negs, g.vecs, g.evs, g.u, g.w1, g.ht, g.evr, g.z, g.c};
    for (void *p : bufs)
        if (p) cudaFree(p);
    for (elsi_gb_handle_s *s : {g.sh, g.rh})
        if (s) {
            free_workspace(s);
            delete s;
        }
    delete h->sing;
    h->sing = nullptr;
}

}  // namespace egb
