// Stage sequence of one solve (arXiv:1705.11191 sec. 3.1, Eqs. 8-11 and steps (1)-(5);
// sec. 4.4 for the occupation and density matrix).
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "solver.h"

namespace egb {

void free_workspace(elsi_gb_handle_s *h)
{
    Workspace &w = h->wk;
    void *bufs[] = {w.a, w.l, w.v1, w.edm, w.v2, w.tau2, w.band, w.t1, w.invd, w.work, w.z,
                    w.d, w.e, w.w, w.f, w.scal, w.stein, w.rf, w.oz, w.ozexp, w.q2f, w.sync, w.status,
                    w.host_h, w.host_s, w.host_p, w.adj, w.tcw, w.csc_row, w.csc_col, w.csc_status};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (w.status_host) cudaFreeHost(w.status_host);
    if (w.scal_host) cudaFreeHost(w.scal_host);
    if (w.events_ready)
        for (auto &e : w.ev) cudaEventDestroy(e);
    h->wk = Workspace();
}

#define ENSURE(name, type, count)                                                          \
    if (!ensure_buf((void **)&w.name, &w.name##_cap, sizeof(type) * (size_t)(count)))     \
        return set_error(h, ELSI_ERR_NOMEM, "cannot allocate %s (%zu bytes)", #name,       \
                         sizeof(type) * (size_t)(count));

// Buffers of one solve. In the binary32 route the reduction buffers (a, l, v1, v2, tau2,
// z) hold binary32 values and are sized for them; the tridiagonal eigenvector scratch and
// the binary64 Cholesky factor live in the digit-plane buffer oz, which is free at those
// stages (its planes are formed after the back-transformations). A binary64 fallback of a
// binary32 solve grows the buffers to binary64 sizes first.
int ensure_workspace(elsi_gb_handle_s *h, int kz)
{
    Workspace &w = h->wk;
    const size_t n = h->n;
    const int b = h->band_width;
    const int S = sb2st_steps(h->n, b);
    const size_t nsweep = n >= 3 ? n - 2 : 1;
    const bool fp32 = h->precision == ELSI_PREC_FP32_REFINE;
    const size_t eb = fp32 ? sizeof(float) : sizeof(double);  // reduction element size
    ENSURE(a, char, n * n * eb);
    ENSURE(l, char, n * n * eb);
    ENSURE(v1, char, n * n * eb);
    ENSURE(edm, double, n * n);
    ENSURE(v2, char, nsweep * S * b * eb);
    ENSURE(tau2, char, nsweep * S * eb);
    ENSURE(band, double, (2 * b + 1) * n);
    ENSURE(t1, double, (size_t)(b > kOneStageNb ? b : kOneStageNb) * n);
    ENSURE(invd, double, n * kTriBlock);
    size_t work = n * kTriBlock;
    size_t wsy = sy2sb_work_elems(h->n, b);
    if (wsy > work) work = wsy;
    if ((size_t)18 * b * kz > work) work = (size_t)18 * b * kz;
    if ((size_t)18 * kOneStageNb * kz > work) work = (size_t)18 * kOneStageNb * kz;
    if (q1_work_elems(b, kz) > work) work = q1_work_elems(b, kz);
    if (h->elpa_solver == 1 && onestage_work_elems(h->n) > work) work = onestage_work_elems(h->n);
    ENSURE(work, double, work + 64);
    ENSURE(z, char, n * kz * eb);
    ENSURE(d, double, n + 8);
    ENSURE(e, double, n + 8);
    ENSURE(w, double, n + 8);
    ENSURE(f, double, n + 8);
    ENSURE(scal, double, 64);
    if (fp32) {
        ENSURE(stein, double, n * kTriBlock + 64);  // binary64 diagonal-block inverses
    } else {
        ENSURE(stein, double, 3 * n * kz + kz + 64);
    }
    ENSURE(sync, unsigned, 64 + 2 * (1024 + 64 + 1024 * 64 + 1024 * 64 * 64));
    ENSURE(status, int, ST_WORDS);
    if (h->precision == ELSI_PREC_FP32_REFINE) {
        const size_t k = h->n_state;
        ENSURE(rf, double, 5 * n * k + 2 * k * k + 1040 * k + 64);
        // digits of H, S (n x n), of X_o, Y_H, Y_S (k columns of length n) and of the
        // rows of X_o for P and W (three splits of n rows of length k)
        ENSURE(oz, __nv_bfloat16, 2 * ozaki_split_elems((int)n, (int)n) +
                                      3 * ozaki_split_elems((int)k, (int)n) +
                                      3 * ozaki_split_elems((int)n, (int)k));
        ENSURE(ozexp, int, 8 * (n + k + 256));
        ENSURE(q2f, float, q2_factor_elems((int)n, b));
        // the largest binary32 tensor-core products: X E of the refinement (n x k x n) and
        // A22 V of the full-to-band reduction (n x b x n); the others have K <= 256
        ENSURE(tcw, float, tc_gemm_work_elems((int)n, (int)(k > 256 ? k : 256), (int)n));
    }
    if (!w.status_host && cudaMallocHost((void **)&w.status_host, sizeof(int) * ST_WORDS) != cudaSuccess)
        return set_error(h, ELSI_ERR_NOMEM, "pinned status");
    if (!w.scal_host && cudaMallocHost((void **)&w.scal_host, sizeof(double) * 64) != cudaSuccess)
        return set_error(h, ELSI_ERR_NOMEM, "pinned scalars");
    if (!w.events_ready) {
        for (auto &e : w.ev)
            if (cudaEventCreate(&e) != cudaSuccess) return set_error(h, ELSI_ERR_CUDA, "event create");
        w.events_ready = true;
    }
    return ELSI_OK;
}

#define CK(...)                                                                            \
    do {                                                                                   \
        cudaError_t _e = (__VA_ARGS__);                                                    \
        if (_e != cudaSuccess)                                                             \
            return set_error(h, ELSI_ERR_CUDA, "%s failed: %s", #__VA_ARGS__,              \
                             cudaGetErrorString(_e));                                      \
    } while (0)

static int num_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

int solve_fp32_refine(elsi_gb_handle_s *h, const SolveRequest &rq);

// FP64 route: every stage in binary64.
static int solve_fp64(elsi_gb_handle_s *h, const SolveRequest &rq)
{
    Workspace &w = h->wk;
    cudaStream_t st = h->stream;
    const int n = h->n, k = h->n_state, b = h->band_width;
    const bool unit = h->overlap_is_unit;
    const int sms = num_sms();
    const bool ev_mode = rq.evec != nullptr;

    CK(cudaEventRecord(w.ev[STAGE_CHOL], st));
    // ---- Eq. 8: S = L L^T (skipped when the factor of the previous call is reused)
    if (!unit && !(h->reuse_l && h->have_l && h->have_l_prec == ELSI_PREC_FP64)) {
        CK(check_finite<double>(st, n, n, rq.ovlp, n, w.status));
        CK(copy_matrix<double, double>(st, n, n, rq.ovlp, n, w.l, n));
        CK(potrf<double>(st, n, w.l, n, w.invd, w.work, w.status));
        h->have_l_prec = ELSI_PREC_FP64;
    }
    CK(cudaEventRecord(w.ev[STAGE_STDFORM], st));
    // ---- Eq. 9: H~ = L^{-1} H L^{-T}
    CK(check_finite<double>(st, n, n, rq.ham, n, w.status));
    double *A = w.a;
    if (!unit) {
        CK(copy_matrix<double, double>(st, n, n, rq.ham, n, w.edm, n));
        CK(trsm_left_lower<double>(st, 0, n, n, w.l, n, w.invd, w.edm, n, w.work));  // Y = L^{-1} H
        CK(transpose<double>(st, n, n, w.edm, n, A, n));                             // Y^T
        CK(trsm_left_lower<double>(st, 0, n, n, w.l, n, w.invd, A, n, w.work));      // L^{-1} Y^T
        CK(symmetrize<double>(st, n, A, n));
    } else {
        CK(copy_matrix<double, double>(st, n, n, rq.ham, n, A, n));
        CK(symmetrize<double>(st, n, A, n));
    }
    const bool one_stage = h->elpa_solver == 1;
    CK(cudaEventRecord(w.ev[STAGE_SY2SB], st));
    if (one_stage) {
        // ---- Eq. 11, first form: T = Q^T H~ Q directly (ELPA 1-stage)
        CK(onestage_tridiag<double>(st, n, A, n, w.d, w.e, w.v1, w.t1, w.work));
        CK(cudaEventRecord(w.ev[STAGE_SB2ST], st));
    } else {
        // ---- Eq. 11 (1): full -> band
        CK(sy2sb<double>(st, n, b, A, n, w.v1, w.t1, w.work, w.work_cap / sizeof(double), w.sync,
                         w.status, sms));
        CK(cudaEventRecord(w.ev[STAGE_SB2ST], st));
        // ---- Eq. 11 (2): band -> tridiagonal
        const int ldb = 2 * b + 1;
        CK(extract_band<double>(st, n, b, A, n, w.band, ldb));
        CK(sb2st<double>(st, n, b, w.band, ldb, w.d, w.e, w.v2, w.tau2, w.status, w.sync, sms));
    }
    CK(cudaEventRecord(w.ev[STAGE_TRIDIAG], st));
    // ---- step (3): eigenvalues (all n for ev, the n_state lowest for dm), k vectors
    const int nval = ev_mode ? n : k;
    CK(stebz(st, n, w.d, w.e, nval, w.w, w.status));
    CK(stein<double>(st, n, w.d, w.e, k, w.w, w.z, n, w.stein, w.status));
    CK(cudaEventRecord(w.ev[STAGE_Q2], st));
    // ---- step (4): Z <- Q2 Z
    if (!one_stage) CK(apply_q2<double>(st, n, b, w.v2, w.tau2, k, w.z, n, w.status));
    CK(cudaEventRecord(w.ev[STAGE_Q1], st));
    // ---- step (5): Z <- Q1 Z (one-stage: Z <- Q Z)
    if (one_stage) CK(apply_q_onestage<double>(st, n, k, w.v1, w.t1, w.z, n, w.work));
    else CK(apply_q1<double>(st, n, b, k, w.v1, w.t1, w.z, n, w.work));
    CK(cudaEventRecord(w.ev[STAGE_BACKSUB], st));
    // ---- Eq. 9: c = L^{-T} c~
    if (!unit) CK(trsm_left_lower<double>(st, 1, n, k, w.l, n, w.invd, w.z, n, w.work));
    CK(cudaEventRecord(w.ev[STAGE_REFINE], st));
    CK(cudaEventRecord(w.ev[STAGE_OCC], st));
    if (ev_mode) {
        CK(cudaMemcpyAsync(rq.eval, w.w, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(rq.evec, w.z, sizeof(double) * (size_t)n * k, cudaMemcpyDeviceToDevice, st));
        CK(cudaEventRecord(w.ev[STAGE_DENSITY], st));
    } else {
        // ---- sec. 4.4: mu, occupations, band energy
        CK(occupation(st, k, w.w, h->n_electron, h->scheme, h->kt, h->occ_accuracy, h->mu_max_steps,
                      w.f, w.scal, w.status, h->occ_stride));
        CK(cudaEventRecord(w.ev[STAGE_DENSITY], st));
        // ---- Eq. 7: P and W (only columns with possibly nonzero f)
        int kocc = k;
        if (h->scheme == ELSI_OCC_INTEGER) {
            kocc = (int)((h->n_electron / h->occ_stride + 1.999999999) / 2.0) * h->occ_stride;
            if (kocc > k) kocc = k;
            if (kocc < 1) kocc = 1;
        }
        CK(density_pw<double>(st, n, kocc, w.z, n, w.f, w.w, rq.dm, rq.want_edm ? w.edm : nullptr, w.v1));
    }
    CK(cudaEventRecord(w.ev[kNumStages], st));
    return ELSI_OK;
}

int run_solve(elsi_gb_handle_s *h, const SolveRequest &rq)
{
    h->last_error.clear();
    h->n_nonsing = h->n;
    if (h->sing_mode != 0 && !h->overlap_is_unit && rq.ovlp) {
        // singularity check of S (sec. 4.4): a singular S is handled by the eigendecomposition
        // transformation of Eq. 10 instead of the Cholesky factorisation
        bool active = false;
        int rc = sing_prepare(h, rq.ovlp, &active);
        if (rc) return rc;
        if (active) return solve_singular(h, rq);
    }
    const bool ev_mode = rq.evec != nullptr;
    int kz = h->n_state;
    if (h->precision == ELSI_PREC_FP32_REFINE) kz = h->n;
    int rc = ensure_workspace(h, kz);
    if (rc) return rc;
    Workspace &w = h->wk;
    cudaStream_t st = h->stream;
    CK(cudaMemsetAsync(w.status, 0, sizeof(int) * ST_WORDS, st));
    if (h->precision == ELSI_PREC_FP64) {
        rc = solve_fp64(h, rq);
    } else {
        set_tc_scratch(w.tcw, w.tcw_cap / sizeof(float), w.status);
        rc = solve_fp32_refine(h, rq);
        set_tc_scratch(nullptr, 0, nullptr);
        if (rc == ELSI_ERR_NO_CONVERGENCE) {
            // The binary32 start was too far from the solution for the refinement (e.g. a
            // badly conditioned S): solve the same problem along the binary64 route.
            cudaStreamSynchronize(st);
            const char *nf = getenv("ELSI_GB_NO_FALLBACK");
            if (nf && nf[0] == '1') return rc;
            CK(cudaMemsetAsync(w.status, 0, sizeof(int) * ST_WORDS, st));
            h->have_l = false;
            h->precision = ELSI_PREC_FP64;  // binary64 sizes of the reduction buffers
            rc = ensure_workspace(h, h->n_state);
            h->precision = ELSI_PREC_FP32_REFINE;
            if (rc) return rc;
            rc = solve_fp64(h, rq);
            h->refine_iters = -1;
        }
    }
    if (rc) {
        cudaStreamSynchronize(st);
        return rc;
    }
    CK(cudaMemcpyAsync(w.status_host, w.status, sizeof(int) * ST_WORDS, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(w.scal_host, w.scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < kNumStages; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, w.ev[i], w.ev[i + 1]) != cudaSuccess) {
            // a stage the solve did not reach (an early error exit): its events were not
            // recorded; clear the error so that the next launch check does not see it
            (void)cudaGetLastError();
            ms = 0.f;
        }
        h->stage_ms[i] = ms;
    }
    const int code = w.status_host[ST_CODE];
    if (code != 0) {
        h->have_edm = false;
        h->have_occ = false;
        if (code == ELSI_ERR_NOT_PD) {
            h->have_l = false;
            return set_error(h, code, "overlap matrix not positive definite (pivot %d)",
                             w.status_host[ST_AUX]);
        }
        if (code == ELSI_ERR_NONFINITE) return set_error(h, code, "non-finite value in the input");
        if (code == ELSI_ERR_TIMEOUT) return set_error(h, code, "device wait limit reached");
        if (code == ELSI_ERR_NO_CONVERGENCE)
            return set_error(h, code, "no convergence (index %d)", w.status_host[ST_AUX]);
        return set_error(h, code, "device error %d", code);
    }
    if (!h->overlap_is_unit) h->have_l = true;
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

}  // namespace egb
