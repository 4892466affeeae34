// C ABI of the solver (declared in include/elsi_gb.h): handle management, customisation,
// workspace, and the stage sequence of one solve (arXiv:1705.11191 sec. 3.1 steps and
// sec. 4.3-4.6 interface).
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>

#include "common.cuh"
#include "kernels.h"
#include "solver.h"

using namespace egb;

namespace egb {

std::atomic<long long> g_launches{0};
static std::atomic<long long> g_spin_limit{kSpinLimit};

long long spin_limit() { return g_spin_limit.load(std::memory_order_relaxed); }

const char *const kStageNames[kNumStages] = {
    "cholesky",  "standard_form", "full_to_band", "band_to_tri", "tridiag_solve",
    "back_q2",   "back_q1",       "back_subst",   "refine",      "occupation",
    "density",
};

int set_error(elsi_gb_handle_s *h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    h->last_error = buf;
    return code;
}

bool ensure_buf(void **p, size_t *cap, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (*p && *cap >= bytes) return true;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, bytes) != cudaSuccess) { *p = nullptr; return false; }
    *cap = bytes;
    return true;
}

}  // namespace egb

static int check_handle(elsi_handle h)
{
    if (!h || h->magic != kHandleMagic) return ELSI_ERR_STATE;
    return ELSI_OK;
}

extern "C" {

const char *elsi_gb_version(void) { return "elsi-gb300 0.1"; }

long long elsi_gb_launch_count(void) { return egb::g_launches.load(); }

int elsi_gb_set_spin_limit(long long polls)
{
    if (polls < 0) return ELSI_ERR_ARG;
    egb::g_spin_limit.store(polls, std::memory_order_relaxed);
    return ELSI_OK;
}

long long elsi_gb_get_spin_limit(void) { return egb::spin_limit(); }

int elsi_init(elsi_handle *out, int solver, int fmt, int mode, int n_basis, int n_state,
              double n_electron)
{
    if (!out) return ELSI_ERR_ARG;
    *out = nullptr;
    if (solver != ELSI_SOLVER_ELPA) return ELSI_ERR_UNSUPPORTED;
    if (fmt != ELSI_FORMAT_DENSE && fmt != ELSI_FORMAT_CSC) return ELSI_ERR_UNSUPPORTED;
    if (mode != ELSI_MODE_MULTI_PROC && mode != ELSI_MODE_SINGLE_PROC) return ELSI_ERR_ARG;
    if (n_basis < 1 || n_state < 1 || n_state > n_basis) return ELSI_ERR_ARG;
    if (!(n_electron >= 0.0) || n_electron > 2.0 * n_state) return ELSI_ERR_ARG;
    elsi_gb_handle_s *h = new (std::nothrow) elsi_gb_handle_s();
    if (!h) return ELSI_ERR_NOMEM;
    h->magic = kHandleMagic;
    h->n = n_basis;
    h->n_state = n_state;
    h->n_electron = n_electron;
    *out = h;
    return ELSI_OK;
}

int elsi_finalize(elsi_handle *hp)
{
    if (!hp || check_handle(*hp)) return ELSI_ERR_STATE;
    elsi_gb_handle_s *h = *hp;
    free_complex(h);
    free_batch(h);
    free_sing(h);
    free_workspace(h);
    h->magic = 0;
    delete h;
    *hp = nullptr;
    return ELSI_OK;
}

int elsi_set_overlap_is_unit(elsi_handle h, int v)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    h->overlap_is_unit = v != 0;
    h->have_l = false;
    return ELSI_OK;
}

int elsi_set_broadening_scheme(elsi_handle h, int s)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (s < 0 || s > 4) return set_error(h, ELSI_ERR_ARG, "broadening scheme %d", s);
    h->scheme = s;
    return ELSI_OK;
}

int elsi_set_broadening_width(elsi_handle h, double w)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!(w > 0.0)) return set_error(h, ELSI_ERR_ARG, "broadening width must be > 0");
    h->kt = w;
    return ELSI_OK;
}

int elsi_set_occ_accuracy(elsi_handle h, double a)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!(a > 0.0)) return set_error(h, ELSI_ERR_ARG, "occ_accuracy must be > 0");
    h->occ_accuracy = a;
    return ELSI_OK;
}

int elsi_set_mu_max_steps(elsi_handle h, int s)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (s < 0) return set_error(h, ELSI_ERR_ARG, "mu_max_steps must be >= 0");
    h->mu_max_steps = s;
    return ELSI_OK;
}

int elsi_set_precision(elsi_handle h, int p)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (p != ELSI_PREC_FP64 && p != ELSI_PREC_FP32_REFINE)
        return set_error(h, ELSI_ERR_ARG, "precision %d", p);
    h->precision = p;
    return ELSI_OK;
}

int elsi_set_band_width(elsi_handle h, int b)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (b < 8 || b > 64 || (b % 8)) return set_error(h, ELSI_ERR_ARG, "band width %d", b);
    h->band_width = b;
    h->band_set = true;
    return ELSI_OK;
}

int elsi_set_refine_max_iter(elsi_handle h, int it)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (it < 0 || it > 8) return set_error(h, ELSI_ERR_ARG, "refine iterations %d", it);
    h->refine_max_iter = it;
    return ELSI_OK;
}

int elsi_set_stream(elsi_handle h, void *s)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    h->stream = (cudaStream_t)s;
    return ELSI_OK;
}

int elsi_set_reuse_ovlp_factor(elsi_handle h, int r)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    h->reuse_l = r != 0;
    return ELSI_OK;
}

int elsi_ev_real(elsi_handle h, double *ham, const double *ovlp, double *eval, double *evec)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!ham || !eval || !evec || (!ovlp && !h->overlap_is_unit))
        return set_error(h, ELSI_ERR_ARG, "null pointer argument");
    SolveRequest rq;
    rq.ham = ham; rq.ovlp = ovlp; rq.eval = eval; rq.evec = evec;
    return run_solve(h, rq);
}

int elsi_dm_real(elsi_handle h, double *ham, const double *ovlp, double *den_mat, double *energy)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!ham || !den_mat || (!ovlp && !h->overlap_is_unit))
        return set_error(h, ELSI_ERR_ARG, "null pointer argument");
    SolveRequest rq;
    rq.ham = ham; rq.ovlp = ovlp; rq.dm = den_mat; rq.want_edm = true;
    int rc = run_solve(h, rq);
    if (rc == ELSI_OK && energy) *energy = h->energy;
    return rc;
}

int elsi_ev_complex(elsi_handle h, const double *ham, const double *ovlp, double *eval, double *evec)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!ham || !eval || !evec || (!ovlp && !h->overlap_is_unit))
        return set_error(h, ELSI_ERR_ARG, "null pointer argument");
    return solve_complex(h, ham, h->overlap_is_unit ? nullptr : ovlp, eval, evec, nullptr, nullptr);
}

int elsi_dm_complex(elsi_handle h, const double *ham, const double *ovlp, double *den_mat,
                    double *energy)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!ham || !den_mat || (!ovlp && !h->overlap_is_unit))
        return set_error(h, ELSI_ERR_ARG, "null pointer argument");
    return solve_complex(h, ham, h->overlap_is_unit ? nullptr : ovlp, nullptr, nullptr, den_mat, energy);
}

int elsi_get_edm_complex(elsi_handle h, double *edm)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!edm) return set_error(h, ELSI_ERR_ARG, "null pointer argument");
    return get_edm_complex(h, edm);
}

int elsi_set_csc(elsi_handle h, int nnz, const int *row_idx, const int *col_ptr, int index_base)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    return csc_set(h, nnz, row_idx, col_ptr, index_base);
}

int elsi_ev_real_sparse(elsi_handle h, const double *ham, const double *ovlp, double *eval,
                        double *evec)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!ham || !eval || !evec || (!ovlp && !h->overlap_is_unit))
        return set_error(h, ELSI_ERR_ARG, "null pointer argument");
    return csc_solve(h, ham, ovlp, eval, evec, nullptr, nullptr);
}

int elsi_dm_real_sparse(elsi_handle h, const double *ham, const double *ovlp, double *den_mat,
                        double *energy)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!ham || !den_mat || (!ovlp && !h->overlap_is_unit))
        return set_error(h, ELSI_ERR_ARG, "null pointer argument");
    return csc_solve(h, ham, ovlp, nullptr, nullptr, den_mat, energy);
}

int elsi_get_edm_real_sparse(elsi_handle h, double *edm)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!edm) return set_error(h, ELSI_ERR_ARG, "null pointer argument");
    return csc_get_edm(h, edm);
}

int elsi_set_batch_streams(elsi_handle h, int streams)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (streams < 0 || streams > 16) return set_error(h, ELSI_ERR_ARG, "batch streams %d (0..16)", streams);
    h->batch_workers = streams;
    return ELSI_OK;
}

int elsi_set_batch_autotune(elsi_handle h, int on)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (on != 0 && on != 1) return set_error(h, ELSI_ERR_ARG, "batch autotune %d (0 or 1)", on);
    h->batch_autotune = on;
    return ELSI_OK;
}

int elsi_get_batch_tuning(elsi_handle h, int n, int cplx, int *band_width, int *elpa_solver,
                          int *streams)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (n < 1 || !band_width || !elpa_solver || !streams) return ELSI_ERR_ARG;
    if (!egb::batch_tuning_lookup(h, n, cplx != 0, band_width, elpa_solver, streams))
        return set_error(h, ELSI_ERR_STATE, "no tuning for n = %d yet", n);
    return ELSI_OK;
}

int elsi_set_elpa_solver(elsi_handle h, int solver)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (solver != 1 && solver != 2) return set_error(h, ELSI_ERR_ARG, "elpa_solver %d (1 or 2)", solver);
    h->elpa_solver = solver;
    h->solver_set = true;
    return ELSI_OK;
}

int elsi_set_sing_check(elsi_handle h, int mode)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (mode < 0 || mode > 2) return set_error(h, ELSI_ERR_ARG, "singularity-check mode %d", mode);
    h->sing_mode = mode;
    h->have_l = false;
    sing_invalidate(h);
    return ELSI_OK;
}

int elsi_set_sing_tol(elsi_handle h, double tau)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!(tau > 0.0)) return set_error(h, ELSI_ERR_ARG, "singularity tolerance %g", tau);
    h->sing_tol = tau;
    sing_invalidate(h);
    return ELSI_OK;
}

int elsi_get_n_nonsing(elsi_handle h, int *n_nonsing)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!n_nonsing) return set_error(h, ELSI_ERR_ARG, "null pointer argument");
    *n_nonsing = h->n_nonsing > 0 ? h->n_nonsing : h->n;
    return ELSI_OK;
}

int elsi_get_entropy(elsi_handle h, double *ts)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!ts) return set_error(h, ELSI_ERR_ARG, "null pointer argument");
    if (!h->have_occ && !h->have_cedm) return set_error(h, ELSI_ERR_STATE, "no density-matrix solve yet");
    *ts = h->entropy;
    return ELSI_OK;
}

int elsi_dm_adjoint_real(elsi_handle h, int n, double f_bar, const double *den_mat,
                         const double *edm, double *ham_bar, double *ovlp_bar)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (n < 1 || !den_mat || !ham_bar || (ovlp_bar && !edm))
        return set_error(h, ELSI_ERR_ARG, "n < 1 or null pointer argument");
    return dm_adjoint(h, n, f_bar, den_mat, edm, ham_bar, ovlp_bar);
}

int elsi_ev_adjoint_real(elsi_handle h, int n, int k, const double *eval, const double *evec,
                         const double *eval_bar, const double *evec_bar, double *ham_bar,
                         double *ovlp_bar)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (n < 1 || k < 0 || k > n || !eval || !evec || !ham_bar || (k > 0 && !evec_bar))
        return set_error(h, ELSI_ERR_ARG, "bad size or null pointer argument");
    return ev_adjoint(h, n, evec_bar ? k : 0, eval, evec, eval_bar, evec_bar, ham_bar, ovlp_bar);
}

int elsi_dm_batched_real(elsi_handle h, int nprob, const int *n_basis, const int *n_state,
                         const double *const *ham, const double *const *ovlp,
                         const double *weight, const double *n_electron, int shared_mu,
                         double *const *den_mat, double *const *edm, double *energy, double *mu)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    return dm_batched(h, nprob, n_basis, n_state, ham, ovlp, weight, n_electron, shared_mu,
                      den_mat, edm, energy, mu, false);
}

int elsi_dm_batched_complex(elsi_handle h, int nprob, const int *n_basis, const int *n_state,
                            const double *const *ham, const double *const *ovlp,
                            const double *weight, const double *n_electron, int shared_mu,
                            double *const *den_mat, double *const *edm, double *energy,
                            double *mu)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    return dm_batched(h, nprob, n_basis, n_state, ham, ovlp, weight, n_electron, shared_mu,
                      den_mat, edm, energy, mu, true);
}

int elsi_batch_ev_real(elsi_handle h, int nprob, const int *n_basis, const int *n_state,
                       const double *const *ham, const double *const *ovlp, double *eval)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    return batch_ev(h, nprob, n_basis, n_state, ham, ovlp, false, eval);
}

int elsi_batch_ev_complex(elsi_handle h, int nprob, const int *n_basis, const int *n_state,
                          const double *const *ham, const double *const *ovlp, double *eval)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    return batch_ev(h, nprob, n_basis, n_state, ham, ovlp, true, eval);
}

int elsi_occupation_weighted(elsi_handle h, int m, const double *eps, const double *weight,
                             double n_electron, double *occ, double *mu)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (m < 1 || !eps || !weight || !occ) return set_error(h, ELSI_ERR_ARG, "null pointer or m < 1");
    return batch_occupation(h, m, eps, weight, n_electron, occ, mu);
}

int elsi_batch_dm(elsi_handle h, const double *occ, double *const *den_mat, double *const *edm,
                  double *energy)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!occ) return set_error(h, ELSI_ERR_ARG, "null occupation array");
    return batch_dm(h, occ, den_mat, edm, energy);
}

int elsi_get_edm_real(elsi_handle h, double *edm)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!edm) return set_error(h, ELSI_ERR_ARG, "null pointer argument");
    if (!h->have_edm) return set_error(h, ELSI_ERR_STATE, "no density-matrix solve yet");
    size_t bytes = sizeof(double) * (size_t)h->n * h->n;
    if (cudaMemcpyAsync(edm, h->wk.edm, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return set_error(h, ELSI_ERR_CUDA, "copy of W failed");
    return ELSI_OK;
}

int elsi_get_mu(elsi_handle h, double *mu)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!mu) return ELSI_ERR_ARG;
    if (!h->have_occ) return set_error(h, ELSI_ERR_STATE, "no density-matrix solve yet");
    *mu = h->mu;
    return ELSI_OK;
}

int elsi_get_occ(elsi_handle h, double *occ)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!occ) return ELSI_ERR_ARG;
    if (!h->have_occ) return set_error(h, ELSI_ERR_STATE, "no density-matrix solve yet");
    if (cudaMemcpyAsync(occ, h->wk.f, sizeof(double) * h->n_state, cudaMemcpyDeviceToDevice,
                        h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return set_error(h, ELSI_ERR_CUDA, "copy of occupations failed");
    return ELSI_OK;
}

int elsi_get_eval(elsi_handle h, double *eval)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!eval) return ELSI_ERR_ARG;
    if (!h->have_occ) return set_error(h, ELSI_ERR_STATE, "no density-matrix solve yet");
    if (cudaMemcpyAsync(eval, h->wk.w, sizeof(double) * h->n_state, cudaMemcpyDeviceToDevice,
                        h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return set_error(h, ELSI_ERR_CUDA, "copy of eigenvalues failed");
    return ELSI_OK;
}

int elsi_dm_real_host(elsi_handle h, const double *ham_host, const double *ovlp_host,
                      double *den_host, double *edm_host, double *energy)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (!ham_host || !den_host || (!ovlp_host && !h->overlap_is_unit))
        return set_error(h, ELSI_ERR_ARG, "null pointer argument");
    const size_t bytes = sizeof(double) * (size_t)h->n * h->n;
    if (!ensure_buf((void **)&h->wk.host_h, &h->wk.host_h_cap, bytes) ||
        !ensure_buf((void **)&h->wk.host_s, &h->wk.host_s_cap, bytes) ||
        !ensure_buf((void **)&h->wk.host_p, &h->wk.host_p_cap, bytes))
        return set_error(h, ELSI_ERR_NOMEM, "staging buffers");
    cudaStream_t st = h->stream;
    if (cudaMemcpyAsync(h->wk.host_h, ham_host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return set_error(h, ELSI_ERR_CUDA, "H2D copy of ham");
    if (ovlp_host && !(h->reuse_l && h->have_l) &&
        cudaMemcpyAsync(h->wk.host_s, ovlp_host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return set_error(h, ELSI_ERR_CUDA, "H2D copy of ovlp");
    SolveRequest rq;
    rq.ham = h->wk.host_h; rq.ovlp = ovlp_host ? h->wk.host_s : nullptr;
    rq.dm = h->wk.host_p; rq.want_edm = true;
    int rc = run_solve(h, rq);
    if (rc != ELSI_OK) return rc;
    if (cudaMemcpyAsync(den_host, h->wk.host_p, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return set_error(h, ELSI_ERR_CUDA, "D2H copy of P");
    if (edm_host && cudaMemcpyAsync(edm_host, h->wk.edm, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return set_error(h, ELSI_ERR_CUDA, "D2H copy of W");
    if (cudaStreamSynchronize(st) != cudaSuccess) return set_error(h, ELSI_ERR_CUDA, "sync");
    if (energy) *energy = h->energy;
    return ELSI_OK;
}

int elsi_get_stage_times(elsi_handle h, float *ms, int n)
{
    if (check_handle(h)) return -1;
    if (!ms) return 0;
    int m = n < kNumStages ? n : kNumStages;
    for (int i = 0; i < m; ++i) ms[i] = h->stage_ms[i];
    return m;
}

const char *elsi_stage_name(int i)
{
    if (i < 0 || i >= kNumStages) return "";
    return kStageNames[i];
}

int elsi_get_refine_info(elsi_handle h, int *iters, double *orth_err)
{
    if (check_handle(h)) return ELSI_ERR_STATE;
    if (iters) *iters = h->refine_iters;
    if (orth_err) *orth_err = h->orth_err;
    return ELSI_OK;
}

const char *elsi_get_last_error(elsi_handle h)
{
    if (check_handle(h)) return "invalid handle";
    return h->last_error.c_str();
}

}  // extern "C"
