// Handle and workspace of one solver instance (the elsi_handle of arXiv:1705.11191
// sec. 4.1: all runtime parameters live in the handle, no globals).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <string>

#include "elsi_gb.h"

namespace egb {

constexpr unsigned kHandleMagic = 0xE151C0DEu;
enum {
    STAGE_CHOL = 0, STAGE_STDFORM, STAGE_SY2SB, STAGE_SB2ST, STAGE_TRIDIAG, STAGE_Q2,
    STAGE_Q1, STAGE_BACKSUB, STAGE_REFINE, STAGE_OCC, STAGE_DENSITY, kNumStages
};
extern const char *const kStageNames[kNumStages];

// Device buffers, grown on demand and kept across calls.
struct Workspace {
#define EGB_BUF(type, name) type *name = nullptr; size_t name##_cap = 0;
    EGB_BUF(double, a)       // n x n: H~, then the full -> band reduction in place
    EGB_BUF(double, l)       // n x n: Cholesky factor (kept for reuse)
    EGB_BUF(double, v1)      // n x n: explicit panel reflectors of stage 1
    EGB_BUF(double, edm)     // n x n: W of the last dm call / scratch during a solve
    EGB_BUF(double, v2)      // stage-2 reflectors
    EGB_BUF(double, tau2)
    EGB_BUF(double, band)    // (2b+1) x n
    EGB_BUF(double, t1)      // b x n
    EGB_BUF(double, invd)    // n x nb inverses of the diagonal blocks of L
    EGB_BUF(double, work)
    EGB_BUF(double, z)       // n x k eigenvectors
    EGB_BUF(double, d)
    EGB_BUF(double, e)
    EGB_BUF(double, w)       // eigenvalues (+ bounds)
    EGB_BUF(double, f)       // occupations
    EGB_BUF(double, scal)    // device scalars: mu, energy, refinement diagnostics
    EGB_BUF(double, stein)   // tridiagonal-eigenvector scratch
    EGB_BUF(double, rf)      // refinement buffers
    EGB_BUF(__nv_bfloat16, oz)  // digit planes of the binary64-accurate products
    EGB_BUF(int, ozexp)      // their exponents
    EGB_BUF(float, q2f)      // compact-WY factors of Q2 (binary32 route)
    EGB_BUF(float, tcw)      // TF32 hi/lo operand planes of the tensor-core GEMM
    EGB_BUF(unsigned, sync)  // grid-barrier words + partial sums
    EGB_BUF(int, status)
    EGB_BUF(double, host_h)  // staging for the _host entry points
    EGB_BUF(double, host_s)
    EGB_BUF(double, host_p)
    EGB_BUF(double, rfc)     // complex route: real eigenpair staging
    EGB_BUF(double, adj)     // eigenpair adjoint scratch
    EGB_BUF(int, csc_row)    // CSC pattern (base 0): row indices
    EGB_BUF(int, csc_col)    // CSC pattern: column pointers (n + 1)
    EGB_BUF(int, csc_status)
#undef EGB_BUF
    int *status_host = nullptr;  // pinned
    double *scal_host = nullptr; // pinned
    cudaEvent_t ev[kNumStages + 1] = {};
    bool events_ready = false;
};

struct BatchState;
struct SingState;

}  // namespace egb

struct elsi_gb_handle_s {
    unsigned magic = 0;
    int n = 0, n_state = 0;
    double n_electron = 0.0;
    // customisation (sec. 4.5) and additions
    bool overlap_is_unit = false;
    int scheme = ELSI_OCC_INTEGER;
    double kt = 0.01;
    double occ_accuracy = 1e-12;
    int mu_max_steps = 200;
    int precision = ELSI_PREC_FP64;
    int band_width = 64;
    int elpa_solver = 2;  // 1: one-stage tridiagonalisation, 2: two-stage (sec. 4.5 elpa_solver)
    int refine_max_iter = 4;
    bool reuse_l = false;
    cudaStream_t stream = nullptr;
    int occ_stride = 1;  // 2 in the real form of a complex problem (pairs of states)
    // state
    bool have_l = false;
    int have_l_prec = -1;
    bool have_edm = false, have_occ = false;
    double mu = 0.0, energy = 0.0;
    double entropy = 0.0;  // -kT S_ent of the last dm call
    int refine_iters = 0;
    double orth_err = 0.0;
    float stage_ms[egb::kNumStages] = {};
    std::string last_error;
    egb::Workspace wk;
    // complex Hermitian problems are solved as real ones of size 2n in this sub-handle
    elsi_gb_handle_s *cplx = nullptr;
    bool have_cedm = false;
    // several independent problems (k-points / spin channels): batch.cu
    egb::BatchState *batch = nullptr;
    int batch_workers = 0;  // concurrent solves of a batch (0: chosen by the autotuner)
    int batch_autotune = 1; // tune band width, tridiagonalisation and concurrency per size
    bool band_set = false, solver_set = false;  // set explicitly: the autotuner keeps them
    // singularity check of the overlap (sec. 4.4): sing.cu. sing_mode 0 = off, 1 = check,
    // 2 = always transform by the eigendecomposition of S
    int sing_mode = 0;
    double sing_tol = 1e-5;
    int n_nonsing = 0;
    int csc_nnz = -1;  // non-zeros of the CSC pattern set by elsi_set_csc (-1: none)
    egb::SingState *sing = nullptr;
};

namespace egb {

struct SolveRequest {
    const double *ham = nullptr;   // device, n x n
    const double *ovlp = nullptr;  // device, n x n (may be null if overlap_is_unit)
    double *eval = nullptr;        // ev: n eigenvalues
    double *evec = nullptr;        // ev: n x n_state
    double *dm = nullptr;          // dm: P
    bool want_edm = false;         // dm: keep W in the handle
};

int set_error(elsi_gb_handle_s *h, int code, const char *fmt, ...);
bool ensure_buf(void **p, size_t *cap, size_t bytes);
int run_solve(elsi_gb_handle_s *h, const SolveRequest &rq);
int ensure_workspace(elsi_gb_handle_s *h, int kz);
int sing_prepare(elsi_gb_handle_s *h, const double *ovlp, bool *active);
int solve_singular(elsi_gb_handle_s *h, const SolveRequest &rq);
void free_sing(elsi_gb_handle_s *h);
int csc_set(elsi_gb_handle_s *h, int nnz, const int *row_idx, const int *col_ptr, int base);
int csc_solve(elsi_gb_handle_s *h, const double *hval, const double *sval, double *eval,
              double *evec, double *dm_val, double *energy);
int csc_get_edm(elsi_gb_handle_s *h, double *edm_val);
void sing_invalidate(elsi_gb_handle_s *h);  // forget the transformation decision
void free_workspace(elsi_gb_handle_s *h);
int solve_complex(elsi_gb_handle_s *h, const double *ham, const double *ovlp, double *eval,
                  double *evec, double *den_mat, double *energy);
int get_edm_complex(elsi_gb_handle_s *h, double *edm);
void free_complex(elsi_gb_handle_s *h);
void free_batch(elsi_gb_handle_s *h);
bool batch_tuning_lookup(elsi_gb_handle_s *h, int n, bool cplx, int *band, int *solver, int *workers);
int dm_adjoint(elsi_gb_handle_s *h, int n, double fb, const double *p, const double *w,
               double *hb, double *sb);
int ev_adjoint(elsi_gb_handle_s *h, int n, int k, const double *eps, const double *c,
               const double *eb, const double *g, double *hb, double *sb);
int batch_ev(elsi_gb_handle_s *h, int nprob, const int *n_basis, const int *n_state,
             const double *const *ham, const double *const *ovlp, bool cplx, double *eval);
int batch_occupation(elsi_gb_handle_s *h, int m, const double *eps, const double *wt, double n_el,
                     double *occ, double *mu);
int batch_dm(elsi_gb_handle_s *h, const double *occ, double *const *dm, double *const *edm,
             double *energy);
int dm_batched(elsi_gb_handle_s *h, int nprob, const int *n_basis, const int *n_state,
               const double *const *ham, const double *const *ovlp, const double *weight,
               const double *n_electron, int shared_mu, double *const *dm, double *const *edm,
               double *energy, double *mu, bool cplx);

}  // namespace egb
