/*
 * elsi_gb.h - C ABI of the single-GPU (GB300, sm_103a) dense Kohn-Sham solver.
 *
 * The library solves the generalized Kohn-Sham eigenproblem H c = eps S c
 * (arXiv:1705.11191, Eqs. 5-6, sec. 2) along the route ELSI drives through ELPA
 * (sec. 3.1, Eqs. 8-11): Cholesky S = L L^T, standard form H~ = L^{-1} H L^{-T},
 * two-stage reduction full -> band -> tridiagonal, tridiagonal eigensolver,
 * back-transformation of the eigenvectors through both stages and L^{-T}; then the
 * chemical potential and occupations (sec. 4.4, Eqs. 14-15, 17-18), the density
 * matrix P = sum_l f_l c_l c_l^T (Eq. 7), the energy-weighted density matrix
 * W = sum_l f_l eps_l c_l c_l^T and the band energy E = sum_l f_l eps_l.
 *
 * Conventions for every entry point:
 *  - Matrices are real symmetric, n_basis x n_basis, binary64, COLUMN-MAJOR with leading
 *    dimension n_basis, and BOTH triangles must be filled (the BLACS_DENSE reading of
 *    sec. 4.2 on one GPU). Eigenvector l is the contiguous column evec[l*n_basis ...].
 *  - Unless a name ends in _host, every array argument is a DEVICE pointer on the
 *    current CUDA device; scalars written back (energy, mu) are HOST pointers.
 *    The caller owns all buffers; the handle owns its workspace and the cached
 *    Cholesky factor.
 *  - Work is enqueued on the handle's stream (elsi_set_stream; default: the legacy
 *    default stream). Each solve synchronises that stream once at the end to read the
 *    device status word, so results are valid when the call returns.
 *  - Return value: ELSI_OK (0) or one of the ELSI_ERR_* codes below; a message is
 *    available from elsi_get_last_error(h).
 */
#ifndef ELSI_GB_H
#define ELSI_GB_H

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define ELSI_OK 0
#define ELSI_ERR_ARG 1          /* invalid argument (null pointer, bad size, bad enum) */
#define ELSI_ERR_UNSUPPORTED 2  /* option of the paper not provided on one GPU */
#define ELSI_ERR_NOT_PD 3       /* S not positive definite (failing pivot in aux) */
#define ELSI_ERR_NONFINITE 4    /* NaN or Inf met in the input or an intermediate */
#define ELSI_ERR_NO_CONVERGENCE 5 /* mu bisection or refinement did not converge */
#define ELSI_ERR_TIMEOUT 6      /* a bounded device-side wait expired */
#define ELSI_ERR_CUDA 7         /* a CUDA runtime call failed */
#define ELSI_ERR_STATE 8        /* call order violated (e.g. get_edm before dm) */
#define ELSI_ERR_NOMEM 9        /* workspace allocation failed */
#define ELSI_ERR_TOO_LARGE 10   /* request exceeds the fixed scratch of elsi_density_noalloc */

/* Enumerations of elsi_init (sec. 4.3). Only solver 1 (ELPA route) is accepted; format 1
 * (dense) or 2 (CSC: the pattern is set by elsi_set_csc, the dense entry points stay
 * available); either parallel mode (both mean "one GPU, whole matrix"). */
#define ELSI_SOLVER_ELPA 1
#define ELSI_FORMAT_DENSE 1
#define ELSI_FORMAT_CSC 2    /* PEXSI_CSC: use elsi_set_csc and the _sparse entry points */
#define ELSI_MODE_MULTI_PROC 1
#define ELSI_MODE_SINGLE_PROC 2

/* Broadening schemes (elsi_customize_mu, sec. 4.5). 0 is this library's addition:
 * integer (aufbau) occupation without broadening. 3 and 4 are the Methfessel-Paxton
 * schemes of order 0 and 1 that the paper names; their formulas (occupation
 * 0.5 erfc(x) + sum_n A_n H_{2n-1}(x) exp(-x^2), entropy term (1/2) A_N H_{2N}(x)
 * exp(-x^2)) are those of the original publication. Order-1 occupations may fall
 * slightly outside [0, 2]. */
#define ELSI_OCC_INTEGER 0
#define ELSI_OCC_GAUSSIAN 1
#define ELSI_OCC_FERMI 2
#define ELSI_OCC_MP0 3   /* Methfessel-Paxton order 0 (the Gaussian scheme) */
#define ELSI_OCC_MP1 4   /* Methfessel-Paxton order 1 (Phys. Rev. B 40, 3616 (1989)) */

/* Arithmetic of the reduction and back-transformations. */
#define ELSI_PREC_FP64 0        /* every stage in binary64 */
#define ELSI_PREC_FP32_REFINE 1 /* binary32 reduction, then refinement to FP64 accuracy */

typedef struct elsi_gb_handle_s *elsi_handle;

/* elsi_init (sec. 4.3): create a handle for problems of size n_basis with n_state
 * eigenstates and n_electron electrons. solver/format/parallel_mode as above.
 * Requires 1 <= n_state <= n_basis and 0 <= n_electron <= 2*n_state. Allocates
 * nothing on the GPU yet (workspace is sized at the first solve). */
int elsi_init(elsi_handle *h, int solver, int matrix_storage_format, int parallel_mode,
              int n_basis, int n_state, double n_electron);

/* elsi_finalize (sec. 4.6): free the handle and its workspace; *h is set to NULL. */
int elsi_finalize(elsi_handle *h);

/* Customisation (sec. 4.5, elsi_customize / elsi_customize_mu / _elpa), per handle. */
int elsi_set_overlap_is_unit(elsi_handle h, int overlap_is_unit);
int elsi_set_broadening_scheme(elsi_handle h, int scheme);
int elsi_set_broadening_width(elsi_handle h, double width); /* k_B T in Ha, > 0 */
int elsi_set_occ_accuracy(elsi_handle h, double occ_accuracy);
int elsi_set_mu_max_steps(elsi_handle h, int mu_max_steps);
/* Additions of this library (no counterpart in the paper's keyword list): */
int elsi_set_precision(elsi_handle h, int precision);      /* ELSI_PREC_* */
int elsi_set_band_width(elsi_handle h, int band_width);    /* 8..64, multiple of 8 (default 64) */
/* elsi_customize_elpa, keyword elpa_solver (sec. 4.5): 1 = one-stage tridiagonalisation
 * T = Q^T H~ Q (Eq. 11, first form; blocked Householder with a matrix-vector product per
 * column, memory-bound), 2 = two-stage full -> band -> tridiagonal (default). Applies to
 * both precision routes and to the complex, batched and singularity-check solves. */
int elsi_set_elpa_solver(elsi_handle h, int solver);
int elsi_set_refine_max_iter(elsi_handle h, int iters);    /* 0..8 */
int elsi_set_stream(elsi_handle h, void *cuda_stream);     /* cudaStream_t */
/* Reuse the Cholesky factor of the previous call instead of factorising ovlp again
 * (the reuse of L across an SCF cycle described in sec. 4.4). */
int elsi_set_reuse_ovlp_factor(elsi_handle h, int reuse);

/* elsi_ev_real (sec. 4.4): all n_basis eigenvalues (ascending) into eval[n_basis]
 * and the n_state lowest eigenvectors (S-orthonormal columns) into
 * evec[n_basis*n_state]. ham is used as workspace and destroyed on exit, as in the
 * paper; ovlp is left unchanged (the handle keeps L instead of overwriting ovlp). */
int elsi_ev_real(elsi_handle h, double *ham, const double *ovlp, double *eval, double *evec);

/* elsi_dm_real (sec. 4.4): density matrix P (Eq. 7) into den_mat[n_basis^2] and the
 * band energy sum_l f_l eps_l into *energy (host). The energy-weighted density matrix
 * of the same call is kept in the handle for elsi_get_edm_real. ham is destroyed. */
int elsi_dm_real(elsi_handle h, double *ham, const double *ovlp, double *den_mat,
                 double *energy);

/* elsi_ev_complex / elsi_dm_complex (sec. 4.4: "same as elsi_ev_real, except that the
 * Hamiltonian matrix, overlap matrix and eigenvectors are complex-valued"). ham, ovlp,
 * evec, den_mat are complex Hermitian arrays stored as interleaved (re, im) binary64 pairs,
 * column-major (2 * n_basis * n_basis doubles; evec 2 * n_basis * n_state doubles);
 * eval has n_basis real entries, ascending. The problem is solved as the real symmetric
 * pencil [[Re H, -Im H], [Im H, Re H]] of size 2 n_basis, which has each eigenvalue twice;
 * P = sum_l f_l c_l c_l^H, E = sum_l f_l eps_l. Inputs are not modified. */
int elsi_ev_complex(elsi_handle h, const double *ham, const double *ovlp, double *eval,
                    double *evec);
int elsi_dm_complex(elsi_handle h, const double *ham, const double *ovlp, double *den_mat,
                    double *energy);
/* W = sum_l f_l eps_l c_l c_l^H of the last elsi_dm_complex call (interleaved). */
int elsi_get_edm_complex(elsi_handle h, double *edm);

/* Energy-weighted density matrix W = sum_l f_l eps_l c_l c_l^T of the last
 * elsi_dm_real call (the paper names it only as a PEXSI output, sec. 4.4). */
int elsi_get_edm_real(elsi_handle h, double *edm);

/* Chemical potential (host scalar) and the n_state occupation numbers (device array)
 * of the last elsi_dm_real call. */
int elsi_get_mu(elsi_handle h, double *mu);
int elsi_get_occ(elsi_handle h, double *occ);
/* The n_state lowest eigenvalues (ascending, device array) that the last elsi_dm_real
 * call occupied (sec. 4.4 computes them on the way to P; the paper's dm call does not
 * return them; this accessor is an addition). ELSI_ERR_STATE before a dm solve. */
int elsi_get_eval(elsi_handle h, double *eval);

/* Same as elsi_dm_real + elsi_get_edm_real but with HOST (pageable or pinned)
 * buffers: copies ham/ovlp in, solves, copies P and W out, on the handle's stream.
 * ham_host is not modified. edm_host may be NULL. */
int elsi_dm_real_host(elsi_handle h, const double *ham_host, const double *ovlp_host,
                      double *den_mat_host, double *edm_host, double *energy);

/* Per-stage device times (ms) of the last solve, in the order of
 * elsi_stage_name(i), i < n; returns the number of stages written. */
int elsi_get_stage_times(elsi_handle h, float *ms, int n);
const char *elsi_stage_name(int i);

/* Diagnostics of the last FP32_REFINE solve: refinement iterations used and the
 * final max |(C^T S C - I)_ij| over the occupied block. */
int elsi_get_refine_info(elsi_handle h, int *iters, double *orth_err);

/* Allocation-free density matrices from caller-supplied orbitals (this entry point has
 * no counterpart in the paper). For callers that cannot allocate GPU memory when they
 * need the result: hosts whose GPU memory is owned by another framework's pre-sized pool
 * (an allocation outside it can fail or fragment it), and loops that forbid allocation
 * after start-up (cudaMalloc may synchronise the device and take unbounded time). Computes den_mat = evec diag(occ) evec^T and, if edm is not NULL,
 * edm = evec diag(occ * eval) evec^T (n_basis x n_basis, column-major, symmetric).
 * evec: n_basis x n_state column-major device array; occ, eval: n_state device arrays
 * (eval may be NULL when edm is NULL). All pointers are device pointers; work is
 * enqueued on `stream` (cudaStream_t, NULL = legacy default stream) and the call returns
 * without synchronising. Scratch: a fixed 16 MiB array inside the library
 * (n_basis * n_state <= 2^21); larger requests return ELSI_ERR_TOO_LARGE. No memory is
 * allocated. The first call on each device looks up the array's device address (and
 * keeps it for later calls), so make that first call before any stream capture; a call
 * whose launch fails forgets the address, so that a call after a reset of the device
 * looks it up again. Calls whose GPU work overlaps in time share the scratch and race. Returns ELSI_OK, ELSI_ERR_ARG, ELSI_ERR_TOO_LARGE or
 * ELSI_ERR_CUDA. */
int elsi_density_noalloc(int n_basis, int n_state, const double *evec, const double *occ,
                         const double *eval, double *den_mat, double *edm, void *stream);

/* ---- Sparse input: the PEXSI_CSC format (sec. 3.2, Fig. 2; elsi_set_csc and the
 * _sparse entry points of sec. 4.3-4.4) -----------------------------------------------
 * On one GPU the whole n_basis x n_basis matrix is one compressed-sparse-column block:
 * nnz values, row_idx (nnz row indices) and col_ptr (n_basis + 1 column starts, the last
 * equal to nnz), with indices counted from index_base (0, or 1 as in the paper's Fortran
 * examples). The pattern holds both triangles of the symmetric H and S (one pattern for
 * both). row_idx and col_ptr may be host or device pointers; they are copied into the
 * handle and checked (ELSI_ERR_ARG on an index out of range or a decreasing col_ptr).
 * elsi_ev_real_sparse: ham, ovlp = device arrays of the nnz values; eval (n_basis) and
 *   evec (n_basis x n_state, dense, column-major) as for elsi_ev_real (the eigenvectors
 *   are not sparse).
 * elsi_dm_real_sparse: den_mat = device array of nnz values, the density matrix P at the
 *   pattern's positions; energy as for elsi_dm_real.
 * elsi_get_edm_real_sparse: W of the last sparse density-matrix call at the pattern.
 * The solve itself is the dense path (the matrices are scattered into dense storage on
 * the device). ELSI_ERR_STATE without a pattern. */
int elsi_set_csc(elsi_handle h, int nnz, const int *row_idx, const int *col_ptr, int index_base);
int elsi_ev_real_sparse(elsi_handle h, const double *ham, const double *ovlp, double *eval,
                        double *evec);
int elsi_dm_real_sparse(elsi_handle h, const double *ham, const double *ovlp, double *den_mat,
                        double *energy);
int elsi_get_edm_real_sparse(elsi_handle h, double *edm);

/* Singularity check of the overlap matrix (sec. 4.4, Eq. 10; the customisation keywords
 * no_singularity_check and singularity_tolerance of sec. 4.5). mode 0 (default): no
 * check, S is factorised by Cholesky. mode 1: all eigenvalues of S are computed; if one
 * or more are below tau, S = X X^T with X = x sqrt(lambda), the eigenvectors of the
 * eigenvalues below tau are dropped and the problem is solved in the N_nonsing remaining
 * directions (H~ = U^T H U with U = x_k lambda_k^{-1/2}, c = U c~); otherwise the
 * Cholesky route is used. mode 2: the eigendecomposition transformation always (the
 * check still drops eigenvalues below tau). The check costs one binary64 eigensolve of
 * S; it is repeated on every call unless elsi_set_reuse_ovlp_factor is set. Real
 * problems only (the complex and batched entry points ignore the setting). With a
 * reduced basis, eval[l] = DBL_MAX for l >= N_nonsing and n_state must not exceed
 * N_nonsing (ELSI_ERR_ARG); a solve where every eigenvalue is below tau returns
 * ELSI_ERR_NOT_PD. tau > 0 (default 1e-5), else ELSI_ERR_ARG. */
int elsi_set_sing_check(elsi_handle h, int mode);
int elsi_set_sing_tol(elsi_handle h, double tau);
/* N_nonsing of the last real solve (n_basis when no direction was dropped). */
int elsi_get_n_nonsing(elsi_handle h, int *n_nonsing);

/* -kT S_ent of the last elsi_dm_real / elsi_dm_complex call (host scalar, <= 0): the
 * entropy term of the free energy F = E_band - kT S_ent that is stationary in the
 * occupations at fixed electron count, S_ent = -g sum_l [phi ln phi + (1-phi) ln(1-phi)]
 * (phi = f_l / g) for Fermi-Dirac, g sum_l exp(-x_l^2) / (2 sqrt(pi)) (x_l =
 * (eps_l - mu) / kT) for Gaussian broadening, 0 for integer occupation. The paper names
 * the schemes (sec. 4.4) but no entropy; this is the term for which dF/dH = P. */
int elsi_get_entropy(elsi_handle h, double *ts);

/* ---- Reverse-mode derivatives (no counterpart in the paper) ------------------------
 * elsi_dm_adjoint_real: for a loss L with dL/dF = f_bar, F = E_band - kT S_ent of a
 * density-matrix solve: ham_bar = f_bar P, ovlp_bar = -f_bar W (dF/dH = P, dF/dS = -W;
 * Hellmann-Feynman and Pulay terms). den_mat, edm: device n x n (P and W of that solve);
 * ham_bar, ovlp_bar: device n x n outputs (ovlp_bar may be NULL). */
int elsi_dm_adjoint_real(elsi_handle h, int n, double f_bar, const double *den_mat,
                         const double *edm, double *ham_bar, double *ovlp_bar);

/* elsi_ev_adjoint_real: reverse-mode derivative of H C = S C diag(eval), C^T S C = I.
 * eval: device, all n eigenvalues ascending; evec: device n x n, ALL n S-orthonormal
 * eigenvectors (column-major; the coupling to every other eigenvector enters the
 * eigenvector derivative). eval_bar: device, n values dL/d eval (may be NULL);
 * evec_bar: device n x k, dL/d evec[:, 0:k] (may be NULL), 0 <= k <= n.
 * Outputs (device n x n, symmetric: the gradient with respect to a symmetric matrix):
 * ham_bar = dL/dH = C sym(X_H) C^T, ovlp_bar = dL/dS = C sym(X_S) C^T (may be NULL) with,
 * for A = C^T evec_bar and F_ij = 1/(eval_j - eval_i) (set to 0 where
 * |eval_i - eval_j| < 1e-10, the degeneracy guard),
 *   X_H = diag(eval_bar) + [F o A | 0],
 *   X_S = -diag(eval_bar eval) - [(F o A) diag(eval_0..k-1) | 0] - diag(A_jj / 2).
 * Errors: ELSI_ERR_ARG, ELSI_ERR_NOMEM, ELSI_ERR_CUDA. */
int elsi_ev_adjoint_real(elsi_handle h, int n, int k, const double *eval, const double *evec,
                         const double *eval_bar, const double *evec_bar, double *ham_bar,
                         double *ovlp_bar);

/* ---- Several problems: k-points and spin channels ----------------------------------
 * Sec. 2 (SINGLE_PROC mode): one process solves a group of k-points one after another;
 * sec. 4.4: the chemical potential's electron count is summed over k-points, spin
 * channels and states. Problem i has n_basis[i] basis functions and n_state[i] states
 * (host int arrays); ham[i] and ovlp[i] are DEVICE pointers to its n_basis[i]^2 matrices
 * (column-major; interleaved complex for the _complex calls), passed in HOST arrays of
 * nprob pointers. ovlp (or any ovlp[i]) may be NULL only with overlap_is_unit set.
 * The handle's settings (broadening, width, accuracy, precision, band width, stream)
 * apply to every problem; its own n_basis, n_state, n_electron are not used. The
 * eigenpairs stay in the handle until the next batched call or elsi_finalize.
 *
 * elsi_dm_batched_real / _complex: all three phases below in one call.
 *   shared_mu = 1: one chemical potential with
 *       sum_i weight[i] sum_l f_il = n_electron[0]      (weight: host, nprob values >= 0,
 *       e.g. k-point weights; f_il in [0, 2] is the occupation of state l of problem i);
 *     integer occupation then fills the levels of all problems in ascending order, a
 *     level (entries with exactly equal eigenvalues) sharing the remaining electrons in
 *     proportion to the weights; smeared occupation bisects on the weighted count.
 *   shared_mu = 0: problem i is occupied on its own with n_electron[i] electrons
 *     (<= 2 n_state[i]) and its own chemical potential; weight may be NULL.
 *   Outputs: den_mat[i] (device, n_basis[i]^2) = P_i = sum_l f_il c_il c_il^H, edm[i]
 *   (device, may be NULL or the array NULL) = W_i = sum_l f_il eps_il c_il c_il^H, both
 *   unweighted (the k-summed density is sum_i weight[i] P_i); energy (host, nprob, may
 *   be NULL) = sum_l f_il eps_il per problem; mu (host, may be NULL): 1 value when
 *   shared_mu, else nprob.
 *   Errors: ELSI_ERR_ARG (sizes, null pointers, negative weight, electron count outside
 *   [0, 2 sum of weights x states]), the single-problem codes of any problem (message
 *   names the problem), ELSI_ERR_NOMEM, ELSI_ERR_CUDA. */
int elsi_dm_batched_real(elsi_handle h, int nprob, const int *n_basis, const int *n_state,
                         const double *const *ham, const double *const *ovlp,
                         const double *weight, const double *n_electron, int shared_mu,
                         double *const *den_mat, double *const *edm, double *energy, double *mu);
int elsi_dm_batched_complex(elsi_handle h, int nprob, const int *n_basis, const int *n_state,
                            const double *const *ham, const double *const *ovlp,
                            const double *weight, const double *n_electron, int shared_mu,
                            double *const *den_mat, double *const *edm, double *energy,
                            double *mu);

/* Number of problems of a batched call solved at the same time, each by its own solver
 * instance on its own stream and host thread (0, the default: 4 for problems up to
 * n = 4096 in the real form, 2 up to 8192, else 1; at most 16). Each instance keeps its
 * own workspace for the largest problem it solves. */
int elsi_set_batch_streams(elsi_handle h, int streams);

/* Autotuner of the batched calls (no counterpart in the paper; on by default). The first
 * time a batched call meets a problem size bucket (real-form size N rounded up to a power
 * of two) on a device, in a precision route, it times the solve of the bucket's first
 * problem with each candidate reduction (two-stage with band width 32 and 64, one-stage
 * tridiagonalisation), keeps the fastest, then times 1, 2, 4, 8, 16 concurrent solver
 * instances of that problem (as many as the free device memory allows) and keeps the
 * count with the highest throughput. The choice is cached for the process. Settings made
 * explicitly on the handle (elsi_set_band_width, elsi_set_elpa_solver,
 * elsi_set_batch_streams) are kept and not tuned. A batch then runs its problems largest
 * first, each taken by the next free solver instance.
 * elsi_get_batch_tuning: the choice for problems of n basis functions (cplx: complex), or
 * ELSI_ERR_STATE if that bucket has not been tuned. */
int elsi_set_batch_autotune(elsi_handle h, int on);
int elsi_get_batch_tuning(elsi_handle h, int n, int cplx, int *band_width, int *elpa_solver,
                          int *streams);

/* Phase 1: eigenpairs of every problem, kept in the handle. eval (device, may be NULL)
 * receives the n_state[i] lowest eigenvalues of each problem, concatenated in problem
 * order (sum_i n_state[i] doubles). */
int elsi_batch_ev_real(elsi_handle h, int nprob, const int *n_basis, const int *n_state,
                       const double *const *ham, const double *const *ovlp, double *eval);
int elsi_batch_ev_complex(elsi_handle h, int nprob, const int *n_basis, const int *n_state,
                          const double *const *ham, const double *const *ovlp, double *eval);

/* Phase 2: occupations with one chemical potential over m weighted entries (device
 * arrays eps, weight, occ of length m, any order; the eigenvalues of several problems,
 * possibly gathered from several processes). sum_j weight[j] occ[j] = n_electron with
 * occ[j] in [0, 2]; rules as for shared_mu above. mu: host, may be NULL. */
int elsi_occupation_weighted(elsi_handle h, int m, const double *eps, const double *weight,
                             double n_electron, double *occ, double *mu);

/* Phase 3: P_i and W_i of the problems of the last elsi_batch_ev_* call from the
 * occupations occ (device, laid out like that call's eval). Outputs as for
 * elsi_dm_batched_*: real matrices after _real, interleaved complex after _complex.
 * ELSI_ERR_STATE without a preceding batched eigensolve. */
int elsi_batch_dm(elsi_handle h, const double *occ, double *const *den_mat,
                  double *const *edm, double *energy);

/* Message describing the last error on this handle ("" if none). */
const char *elsi_get_last_error(elsi_handle h);

/* Library version string. */
const char *elsi_gb_version(void);

/* Number of CUDA kernels this library has launched in this process (all handles);
 * a benchmarking aid, no counterpart in the paper. */
long long elsi_gb_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* ELSI_GB_H */
