// Sparse input and output in compressed sparse column form (the PEXSI_CSC format of
// arXiv:1705.11191 sec. 3.2 and Fig. 2: values of the non-zero elements, their row
// indices, and the starting point of every column), for the entry points
// elsi_ev_real_sparse, elsi_dm_real_sparse and elsi_get_edm_real_sparse (sec. 4.4).
// On one GPU the whole matrix is one CSC block. The dense solver works on the matrices
// scattered from the pattern; the density matrices are returned at the pattern's
// positions (the eigenvectors stay dense, as the paper specifies).
#include "common.cuh"
#include "kernels.h"
#include "solver.h"

namespace egb {

static int grid_of(size_t total)
{
    size_t g = (total + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g ? g : 1);
}

// Checks (one thread per column): col_ptr non-decreasing from base to nnz + base, row
// indices in [base, n + base). Converts both arrays to base 0 in place.
__global__ void csc_check_kernel(int n, int nnz, int base, int *row, int *colp, int *status)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= n; c += gridDim.x * blockDim.x) {
        const int p = colp[c] - base;
        bool ok = p >= 0 && p <= nnz;
        if (c == 0) ok = ok && p == 0;
        if (c == n) ok = ok && p == nnz;
        if (c < n) {
            const int q = colp[c + 1] - base;
            ok = ok && q >= p && q <= nnz;
            if (ok)
                for (int e = p; e < q; ++e) {
                    const int r = row[e] - base;
                    if (r < 0 || r >= n) { ok = false; break; }
                }
        }
        if (!ok) report_error(status, ELSI_ERR_ARG, c);
    }
}

__global__ void rebase_kernel(int count, int base, int *a)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) a[i] -= base;
}

// dense (n x n, zeroed) <- values at the pattern; one warp per column
__global__ void csc_scatter_kernel(int n, const int *row, const int *colp, const double *val, double *dense)
{
    const int lane = threadIdx.x & 31;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n; c += (gridDim.x * blockDim.x) >> 5)
        for (int e = colp[c] + lane; e < colp[c + 1]; e += 32) dense[(size_t)row[e] + (size_t)c * n] = val[e];
}

// values at the pattern <- dense (n x n); one warp per column
__global__ void csc_gather_kernel(int n, const int *row, const int *colp, const double *dense, double *val)
{
    const int lane = threadIdx.x & 31;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n; c += (gridDim.x * blockDim.x) >> 5)
        for (int e = colp[c] + lane; e < colp[c + 1]; e += 32) val[e] = dense[(size_t)row[e] + (size_t)c * n];
}

#define CCK(...)                                                                           \
    do {                                                                                   \
        cudaError_t _e = (__VA_ARGS__);                                                    \
        if (_e != cudaSuccess)                                                             \
            return set_error(h, ELSI_ERR_CUDA, "%s failed: %s", #__VA_ARGS__,              \
                             cudaGetErrorString(_e));                                      \
    } while (0)

int csc_set(elsi_gb_handle_s *h, int nnz, const int *row_idx, const int *col_ptr, int base)
{
    if (nnz < 0 || !row_idx || !col_ptr || (base != 0 && base != 1))
        return set_error(h, ELSI_ERR_ARG, "csc: nnz < 0, null array or index base not 0 / 1");
    const int n = h->n;
    Workspace &w = h->wk;
    cudaStream_t st = h->stream;
    if (!ensure_buf((void **)&w.csc_row, &w.csc_row_cap, sizeof(int) * ((size_t)nnz + 1)) ||
        !ensure_buf((void **)&w.csc_col, &w.csc_col_cap, sizeof(int) * ((size_t)n + 1)) ||
        !ensure_buf((void **)&w.csc_status, &w.csc_status_cap, sizeof(int) * ST_WORDS))
        return set_error(h, ELSI_ERR_NOMEM, "csc pattern buffers");
    CCK(cudaMemcpyAsync(w.csc_row, row_idx, sizeof(int) * (size_t)nnz, cudaMemcpyDefault, st));
    CCK(cudaMemcpyAsync(w.csc_col, col_ptr, sizeof(int) * ((size_t)n + 1), cudaMemcpyDefault, st));
    CCK(cudaMemsetAsync(w.csc_status, 0, sizeof(int) * ST_WORDS, st));
    EGB_COUNT_LAUNCH();
    csc_check_kernel<<<grid_of((size_t)n + 1), 256, 0, st>>>(n, nnz, base, w.csc_row, w.csc_col, w.csc_status);
    CCK(cudaGetLastError());
    int stat[ST_WORDS];
    CCK(cudaMemcpyAsync(stat, w.csc_status, sizeof(stat), cudaMemcpyDeviceToHost, st));
    CCK(cudaStreamSynchronize(st));
    h->csc_nnz = -1;
    if (stat[ST_CODE] != 0)
        return set_error(h, ELSI_ERR_ARG, "csc: invalid column pointer or row index (column %d)", stat[ST_AUX]);
    if (base) {
        EGB_COUNT_LAUNCH();
        rebase_kernel<<<grid_of(nnz), 256, 0, st>>>(nnz, base, w.csc_row);
        EGB_COUNT_LAUNCH();
        rebase_kernel<<<grid_of((size_t)n + 1), 256, 0, st>>>(n + 1, base, w.csc_col);
        CCK(cudaGetLastError());
    }
    h->csc_nnz = nnz;
    return ELSI_OK;
}

// dense copies of the pattern's H and S in the handle's staging buffers
static int csc_to_dense(elsi_gb_handle_s *h, const double *hval, const double *sval)
{
    const int n = h->n;
    Workspace &w = h->wk;
    cudaStream_t st = h->stream;
    const size_t nn = (size_t)n * n;
    if (!ensure_buf((void **)&w.host_h, &w.host_h_cap, sizeof(double) * nn) ||
        (sval && !ensure_buf((void **)&w.host_s, &w.host_s_cap, sizeof(double) * nn)))
        return set_error(h, ELSI_ERR_NOMEM, "csc dense staging");
    const int grid = grid_of((size_t)n * 32);
    CCK(cudaMemsetAsync(w.host_h, 0, sizeof(double) * nn, st));
    EGB_COUNT_LAUNCH();
    csc_scatter_kernel<<<grid, 256, 0, st>>>(n, w.csc_row, w.csc_col, hval, w.host_h);
    if (sval) {
        CCK(cudaMemsetAsync(w.host_s, 0, sizeof(double) * nn, st));
        EGB_COUNT_LAUNCH();
        csc_scatter_kernel<<<grid, 256, 0, st>>>(n, w.csc_row, w.csc_col, sval, w.host_s);
    }
    CCK(cudaGetLastError());
    return ELSI_OK;
}

int csc_solve(elsi_gb_handle_s *h, const double *hval, const double *sval, double *eval,
              double *evec, double *dm_val, double *energy)
{
    if (h->csc_nnz < 0) return set_error(h, ELSI_ERR_STATE, "no CSC pattern set (elsi_set_csc)");
    const bool unit = h->overlap_is_unit;
    int rc = csc_to_dense(h, hval, unit ? nullptr : sval);
    if (rc) return rc;
    Workspace &w = h->wk;
    SolveRequest rq;
    rq.ham = w.host_h;
    rq.ovlp = unit ? nullptr : w.host_s;
    if (evec) {
        rq.eval = eval;
        rq.evec = evec;
        return run_solve(h, rq);
    }
    const size_t nn = (size_t)h->n * h->n;
    if (!ensure_buf((void **)&w.host_p, &w.host_p_cap, sizeof(double) * nn))
        return set_error(h, ELSI_ERR_NOMEM, "csc density staging");
    rq.dm = w.host_p;
    rq.want_edm = true;
    rc = run_solve(h, rq);
    if (rc) return rc;
    cudaStream_t st = h->stream;
    EGB_COUNT_LAUNCH();
    csc_gather_kernel<<<grid_of((size_t)h->n * 32), 256, 0, st>>>(h->n, w.csc_row, w.csc_col, w.host_p, dm_val);
    CCK(cudaGetLastError());
    CCK(cudaStreamSynchronize(st));
    if (energy) *energy = h->energy;
    return ELSI_OK;
}

int csc_get_edm(elsi_gb_handle_s *h, double *edm_val)
{
    if (h->csc_nnz < 0) return set_error(h, ELSI_ERR_STATE, "no CSC pattern set (elsi_set_csc)");
    if (!h->have_edm) return set_error(h, ELSI_ERR_STATE, "no density-matrix solve yet");
    cudaStream_t st = h->stream;
    EGB_COUNT_LAUNCH();
    csc_gather_kernel<<<grid_of((size_t)h->n * 32), 256, 0, st>>>(h->n, h->wk.csc_row, h->wk.csc_col, h->wk.edm, edm_val);
    CCK(cudaGetLastError());
    CCK(cudaStreamSynchronize(st));
    return ELSI_OK;
}

}  // namespace egb
