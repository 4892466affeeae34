// FP32 reduction + refinement route (ELSI_PREC_FP32_REFINE).
//
// The generalized eigenproblem is solved once in binary32 along the same two-stage route
// as the binary64 path (Cholesky, standard form, full -> band, band -> tridiagonal,
// binary64 tridiagonal solve, back-transformations), for ALL n eigenpairs. The n_state
// wanted eigenvectors are then refined to binary64 accuracy by the iterative refinement
// of Ogita & Aishima (Japan J. Indust. Appl. Math. 35 (2018) 1007-1035) written for the
// pencil (H, S): with X the current S-orthonormal approximation,
//     R = I - X^T S X,  G = X^T H X,  lambda_i = G_ii / (1 - R_ii),
//     E_ij = (G_ij + lambda_j R_ij) / (lambda_j - lambda_i)  if |lambda_j - lambda_i| > delta
//          = R_ij / 2                                          otherwise,
//     X <- X + X E.
// Only the columns of the wanted states are updated (E restricted to those columns), so
// for i outside the wanted set the numerator x_i^T (H - lambda_j S) x_j is formed from
// the binary64 residual block R_o = H X_o - S X_o diag(lambda) and needs only binary32
// relative accuracy; the products H X_o, S X_o, X_o^T H X_o, X_o^T S X_o are binary64.
// Eigenvalues closer than delta form clusters; at the start of every iteration each
// cluster is rotated by the eigenvectors of its small pencil (G_CC, S_CC) (a Rayleigh-Ritz
// step, the treatment of clustered eigenvalues in Ogita & Aishima's follow-up work), after
// which pairs inside a cluster only receive the R_ij / 2 re-orthonormalisation.
#include <float.h>
#include <stdio.h>
#include <stdlib.h>

#include "common.cuh"
#include "kernels.h"
#include "solver.h"

namespace egb {

#define CKR(...)                                                                           \
    do {                                                                                   \
        cudaError_t _e = (__VA_ARGS__);                                                    \
        if (_e != cudaSuccess)                                                             \
            return set_error(h, ELSI_ERR_CUDA, "%s failed: %s", #__VA_ARGS__,              \
                             cudaGetErrorString(_e));                                      \
    } while (0)

// out1[j] = x_j . y1_j, out2[j] = x_j . y2_j (binary64), one CTA per column.
__global__ void col_dots_kernel(int n, const double *x, const double *y1, const double *y2,
                                double *out1, double *out2)
{
    __shared__ double red[32];
    const int j = blockIdx.x;
    const double *xc = x + (size_t)j * n, *a = y1 + (size_t)j * n, *b = y2 + (size_t)j * n;
    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        s1 = fma(xc[i], a[i], s1);
        s2 = fma(xc[i], b[i], s2);
    }
    s1 = block_sum(s1, red);
    s2 = block_sum(s2, red);
    if (threadIdx.x == 0) { out1[j] = s1; out2[j] = s2; }
}

// lam_j = g_j / s_j ; R_o = YH - YS diag(lam) (in place in yh), and a binary32 copy.
__global__ void residual_kernel(int n, int k, const double *g, const double *s, double *lam,
                                double *yh, const double *ys, float *r32)
{
    size_t total = (size_t)n * k;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int j = (int)(e / n);
        double lj = g[j] / s[j];
        if (e % n == 0) lam[j] = lj;
        double r = fma(-lj, ys[e], yh[e]);
        yh[e] = r;
        r32[e] = (float)r;
    }
}

// Correction matrix E (n x k, binary32) of the refinement step.
//  rows i < k : from Goo = Xo^T H Xo and Soo = Xo^T S Xo (binary64, k x k); pairs in the
//               same cluster (cid[i] == cid[j]) only get R_ij / 2
//  rows i >= k: E_ij = M_ij / (lam_j - w_i), M = Xu^T R_o (binary32, (n-k) x k, ld n-k)
// Also accumulates max |E| and max |R_oo| into stats[0], stats[1] (as ordered ints).
__global__ void build_e_kernel(int n, int k, const double *goo, const double *soo,
                               const float *m, const double *lam, const double *w,
                               const int *cid, float *e32, unsigned long long *stats)
{
    size_t total = (size_t)n * k;
    double emax = 0.0, rmax = 0.0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total;
         q += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(q % n), j = (int)(q / n);
        double e;
        if (i < k) {
            double rij = (i == j ? 1.0 : 0.0) - soo[(size_t)i + (size_t)j * k];
            rmax = fmax(rmax, fabs(rij));
            if (i == j || cid[i] == cid[j]) {
                e = 0.5 * rij;
            } else {
                double dl = lam[j] - lam[i];
                e = (goo[(size_t)i + (size_t)j * k] + lam[j] * rij) / dl;
            }
        } else {
            double dl = lam[j] - w[i];
            double mij = (double)m[(size_t)(i - k) + (size_t)j * (n - k)];
            e = (fabs(dl) > 1e-13) ? mij / dl : 0.0;
        }
        emax = fmax(emax, fabs(e));
        e32[q] = (float)e;
    }
    // non-negative doubles order like their bit patterns
    for (int o = 16; o > 0; o >>= 1) {
        emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(stats + 0, (unsigned long long)__double_as_longlong(emax));
        atomicMax(stats + 1, (unsigned long long)__double_as_longlong(rmax));
    }
}

constexpr int kMaxCluster = 32;

// Clusters: maximal runs of consecutive indices whose Rayleigh quotients
// lam = G_jj / S_jj differ by less than delta, cut after kMaxCluster entries. One thread
// scans the k values: cid[i] = first index of i's cluster, csize[first] = its size.
__global__ void cluster_scan_kernel(int k, const double *goo, const double *soo, double delta,
                                    int *cid, int *csize)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int start = 0;
    double prev = goo[0] / soo[0];
    for (int i = 1; i <= k; ++i) {
        double cur = (i < k) ? goo[(size_t)i * k + i] / soo[(size_t)i * k + i] : 0.0;
        bool cut = (i == k) || !(fabs(cur - prev) < delta) || (i - start >= kMaxCluster);
        if (cut) {
            for (int q = start; q < i; ++q) cid[q] = start;
            csize[start] = i - start;
            start = i;
        }
        prev = cur;
    }
}

// The small Rayleigh-Ritz problem of every cluster C of size c >= 2 (one CTA per index,
// cluster starts only): S_CC = L L^T (Cholesky), A = L^{-1} G_CC L^{-T},
// A = V diag(mu) V^T by cyclic Jacobi, Q_C = L^{-T} V, so that Q^T S_CC Q = I and
// Q^T G_CC Q = diag(mu). Q_C goes to qbuf + i0 * kMaxCluster^2 (ld kMaxCluster).
__global__ void cluster_rr_kernel(int k, const double *goo, const double *soo, const int *cid,
                                  const int *csize, double *qbuf)
{
    const int start = blockIdx.x;
    __shared__ double G[kMaxCluster * kMaxCluster], Sm[kMaxCluster * kMaxCluster];
    __shared__ double V[kMaxCluster * kMaxCluster];
    if (cid[start] != start) return;
    const int c = csize[start];
    if (c < 2) return;
    double *q = qbuf + (size_t)start * kMaxCluster * kMaxCluster;
    for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
        int a = e % c, b = e / c;
        G[a + b * kMaxCluster] = goo[(size_t)(start + a) + (size_t)(start + b) * k];
        Sm[a + b * kMaxCluster] = soo[(size_t)(start + a) + (size_t)(start + b) * k];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int ld = kMaxCluster;
    // symmetrise, Cholesky of S_CC in place (lower)
    for (int b = 0; b < c; ++b)
        for (int a = b + 1; a < c; ++a) {
            double g = 0.5 * (G[a + b * ld] + G[b + a * ld]);
            G[a + b * ld] = G[b + a * ld] = g;
            double sv = 0.5 * (Sm[a + b * ld] + Sm[b + a * ld]);
            Sm[a + b * ld] = Sm[b + a * ld] = sv;
        }
    for (int j = 0; j < c; ++j) {
        double d = Sm[j + j * ld];
        for (int p = 0; p < j; ++p) d -= Sm[j + p * ld] * Sm[j + p * ld];
        d = sqrt(fmax(d, 1e-300));
        Sm[j + j * ld] = d;
        for (int i = j + 1; i < c; ++i) {
            double v = Sm[i + j * ld];
            for (int p = 0; p < j; ++p) v -= Sm[i + p * ld] * Sm[j + p * ld];
            Sm[i + j * ld] = v / d;
        }
    }
    // A = L^{-1} G L^{-T}: forward substitution on columns, then on rows
    for (int b = 0; b < c; ++b)
        for (int i = 0; i < c; ++i) {
            double v = G[i + b * ld];
            for (int p = 0; p < i; ++p) v -= Sm[i + p * ld] * G[p + b * ld];
            G[i + b * ld] = v / Sm[i + i * ld];
        }
    for (int a = 0; a < c; ++a)
        for (int i = 0; i < c; ++i) {
            double v = G[a + i * ld];
            for (int p = 0; p < i; ++p) v -= Sm[i + p * ld] * G[a + p * ld];
            G[a + i * ld] = v / Sm[i + i * ld];
        }
    for (int b = 0; b < c; ++b)
        for (int a = 0; a < c; ++a) V[a + b * ld] = (a == b) ? 1.0 : 0.0;
    // cyclic Jacobi on A (symmetric c x c)
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int b = 0; b < c; ++b)
            for (int a = 0; a < c; ++a) {
                if (a == b) dia += G[a + b * ld] * G[a + b * ld];
                else off += G[a + b * ld] * G[a + b * ld];
            }
        if (off <= 1e-32 * dia || off == 0.0) break;
        for (int p = 0; p < c - 1; ++p)
            for (int r = p + 1; r < c; ++r) {
                double apr = G[p + r * ld];
                if (apr == 0.0) continue;
                double th = (G[r + r * ld] - G[p + p * ld]) / (2.0 * apr);
                double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
                for (int i = 0; i < c; ++i) {  // columns p, r
                    double x = G[i + p * ld], y = G[i + r * ld];
                    G[i + p * ld] = cs * x - sn * y;
                    G[i + r * ld] = sn * x + cs * y;
                    double xv = V[i + p * ld], yv = V[i + r * ld];
                    V[i + p * ld] = cs * xv - sn * yv;
                    V[i + r * ld] = sn * xv + cs * yv;
                }
                for (int i = 0; i < c; ++i) {  // rows p, r
                    double x = G[p + i * ld], y = G[r + i * ld];
                    G[p + i * ld] = cs * x - sn * y;
                    G[r + i * ld] = sn * x + cs * y;
                }
            }
    }
    // ascending order of the Ritz values (selection sort of the columns of V)
    for (int a = 0; a < c; ++a) {
        int best = a;
        for (int b = a + 1; b < c; ++b)
            if (G[b + b * ld] < G[best + best * ld]) best = b;
        if (best != a) {
            double t = G[a + a * ld]; G[a + a * ld] = G[best + best * ld]; G[best + best * ld] = t;
            for (int i = 0; i < c; ++i) {
                double u = V[i + a * ld]; V[i + a * ld] = V[i + best * ld]; V[i + best * ld] = u;
            }
        }
    }
    // Q = L^{-T} V (back substitution with L^T)
    for (int b = 0; b < c; ++b)
        for (int i = c - 1; i >= 0; --i) {
            double v = V[i + b * ld];
            for (int p = i + 1; p < c; ++p) v -= Sm[p + i * ld] * q[p + b * ld];
            q[i + b * ld] = v / Sm[i + i * ld];
        }
}

// Rotate the cluster columns of an n x k binary64 block: Y[:, C] <- Y[:, C] Q_C.
// grid: (k, ceil(n / 256)); only cluster starts with size >= 2 work.
__global__ void rotate_cols_kernel(int n, int k, const int *cid, const int *csize,
                                   const double *qbuf, double *y0, double *y1, double *y2)
{
    const int i0 = blockIdx.x;
    if (cid[i0] != i0) return;
    const int c = csize[i0];
    if (c < 2) return;
    const double *q = qbuf + (size_t)i0 * kMaxCluster * kMaxCluster;
    const int r = blockIdx.y * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double *ys[3] = {y0, y1, y2};
    for (int which = 0; which < 3; ++which) {
        double *y = ys[which];
        if (!y) continue;
        double old[kMaxCluster];
        for (int a = 0; a < c; ++a) old[a] = y[(size_t)r + (size_t)(i0 + a) * n];
        for (int b = 0; b < c; ++b) {
            double s = 0.0;
            for (int a = 0; a < c; ++a) s = fma(old[a], q[a + b * kMaxCluster], s);
            y[(size_t)r + (size_t)(i0 + b) * n] = s;
        }
    }
}

// Rows (mode 0) or columns (mode 1) of the k x k matrices G and S for every cluster:
// rows: M[C, :] <- Q_C^T M[C, :]; cols: M[:, C] <- M[:, C] Q_C.
__global__ void rotate_gram_kernel(int k, const int *cid, const int *csize, const double *qbuf,
                                   double *g, double *sm, int mode)
{
    const int i0 = blockIdx.x;
    if (cid[i0] != i0) return;
    const int c = csize[i0];
    if (c < 2) return;
    const double *q = qbuf + (size_t)i0 * kMaxCluster * kMaxCluster;
    for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < k; t += gridDim.y * blockDim.x) {
        for (int which = 0; which < 2; ++which) {
            double *mtx = which ? sm : g;
            double old[kMaxCluster];
            if (mode == 0) {
                for (int a = 0; a < c; ++a) old[a] = mtx[(size_t)(i0 + a) + (size_t)t * k];
                for (int b = 0; b < c; ++b) {
                    double s = 0.0;
                    for (int a = 0; a < c; ++a) s = fma(q[a + b * kMaxCluster], old[a], s);
                    mtx[(size_t)(i0 + b) + (size_t)t * k] = s;
                }
            } else {
                for (int a = 0; a < c; ++a) old[a] = mtx[(size_t)t + (size_t)(i0 + a) * k];
                for (int b = 0; b < c; ++b) {
                    double s = 0.0;
                    for (int a = 0; a < c; ++a) s = fma(old[a], q[a + b * kMaxCluster], s);
                    mtx[(size_t)t + (size_t)(i0 + b) * k] = s;
                }
            }
        }
    }
}

__global__ void orth_defect_kernel(int k, const double *sm, unsigned long long *stats)
{
    double r = 0.0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (size_t)k * k;
         q += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(q % k), j = (int)(q / k);
        r = fmax(r, fabs((i == j ? 1.0 : 0.0) - sm[q]));
    }
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0) atomicMax(stats, (unsigned long long)__double_as_longlong(r));
}

// out[0] = max_j lam_j - w_k, the largest refined eigenvalue of the wanted block against
// the binary32-route estimate of the first unwanted one (-inf when k = n); out[1] =
// max(|w_0|, |w_(n-1)|, max_j |lam_j|), the scale of the spectrum. One CTA.
__global__ void wanted_order_kernel(int n, int k, const double *lam, const double *w, double *out)
{
    __shared__ double smax[32], sabs[32];
    double m = -INFINITY, a = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        m = fmax(m, lam[j]);
        a = fmax(a, fabs(lam[j]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    }
    if ((threadIdx.x & 31) == 0) {
        smax[threadIdx.x >> 5] = m;
        sabs[threadIdx.x >> 5] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            m = fmax(m, smax[q]);
            a = fmax(a, sabs[q]);
        }
        out[0] = k < n ? m - w[k] : -INFINITY;
        out[1] = fmax(a, fmax(fabs(w[0]), fabs(w[n - 1])));
    }
}

__global__ void gram_diag_kernel(int k, const double *g, const double *sm, double *gd, double *sd)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x) {
        gd[j] = g[(size_t)j * k + j];
        sd[j] = sm[(size_t)j * k + j];
    }
}

__global__ void add_f32_to_f64_kernel(size_t total, const float *src, double *dst)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x)
        dst[e] += (double)src[e];
}

__global__ void copy_eval_kernel(int n, int k, const double *lam, const double *w, double *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (i < k) ? lam[i] : w[i];
}

static int grid_for(size_t total)
{
    size_t g = (total + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g ? g : 1);
}

int solve_fp32_refine(elsi_gb_handle_s *h, const SolveRequest &rq)
{
    Workspace &w = h->wk;
    cudaStream_t st = h->stream;
    const int n = h->n, k = h->n_state, b = h->band_width;
    const bool unit = h->overlap_is_unit;
    const bool ev_mode = rq.evec != nullptr;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    // binary32 views of the workspace
    float *A = reinterpret_cast<float *>(w.a);
    float *L = reinterpret_cast<float *>(w.l);
    float *Y = reinterpret_cast<float *>(w.edm);
    float *V1 = reinterpret_cast<float *>(w.v1);
    float *V2 = reinterpret_cast<float *>(w.v2);
    float *TAU2 = reinterpret_cast<float *>(w.tau2);
    float *BAND = reinterpret_cast<float *>(w.band);
    float *T1 = reinterpret_cast<float *>(w.t1);
    float *INVD = reinterpret_cast<float *>(w.invd);
    float *WORK = reinterpret_cast<float *>(w.work);
    float *X32 = reinterpret_cast<float *>(w.z);  // n x n

    CKR(cudaEventRecord(w.ev[STAGE_CHOL], st));
    if (!unit && !(h->reuse_l && h->have_l && h->have_l_prec == ELSI_PREC_FP32_REFINE)) {
        // Eq. 8 in binary32: the factor only feeds the binary32 standard form and
        // back-substitution, where a binary64 factor rounded to binary32 has the same
        // backward error (about eps_32 ||S||); the refinement works with S itself.
        CKR(check_finite<double>(st, n, n, rq.ovlp, n, w.status));
        CKR(check_finite<double>(st, n, n, rq.ham, n, w.status));
        CKR(copy_matrix<float, double>(st, n, n, rq.ovlp, n, L, n));
        CKR(potrf<float>(st, n, L, n, INVD, WORK, w.status));
        CKR(cudaMemcpyAsync(w.status_host, w.status, sizeof(int) * ST_WORDS, cudaMemcpyDeviceToHost, st));
        CKR(cudaStreamSynchronize(st));
        if (w.status_host[ST_CODE] == ELSI_ERR_NOT_PD) {
            // S is positive definite in binary64 but not in binary32 (lambda_min(S) near or
            // below eps_32 ||S||): factor in binary64, with the trailing and panel updates as
            // binary64-accurate digit products on the tensor cores (binary64 FMAs are scarce
            // on this chip), and round the factor and its diagonal-block inverses.
            CKR(cudaMemsetAsync(w.status, 0, sizeof(int) * ST_WORDS, st));
            double *L64 = reinterpret_cast<double *>(w.oz);            // n x n, oz unused yet
            double *INV64 = reinterpret_cast<double *>(w.stein);       // n x kTriBlock
            __nv_bfloat16 *cdig = w.oz + (size_t)4 * n * n;             // after L64
            CKR(copy_matrix<double, double>(st, n, n, rq.ovlp, n, L64, n));
            set_f64_tc_scratch(cdig, w.oz_cap / sizeof(__nv_bfloat16) - (size_t)4 * n * n, w.ozexp,
                               w.ozexp_cap / sizeof(int));
            cudaError_t pe = potrf<double>(st, n, L64, n, INV64, w.edm, w.status);
            set_f64_tc_scratch(nullptr, 0, nullptr, 0);
            CKR(pe);
            CKR(copy_matrix<float, double>(st, n, n, L64, n, L, n));
            CKR(copy_matrix<float, double>(st, n, kTriBlock, INV64, n, INVD, n));
            CKR(cudaMemcpyAsync(w.status_host, w.status, sizeof(int) * ST_WORDS, cudaMemcpyDeviceToHost, st));
            CKR(cudaStreamSynchronize(st));
        }
        // not positive definite in binary64 either, or a non-finite input: stop here; the
        // caller reports the code (and the pivot) from the status words
        if (w.status_host[ST_CODE] != 0) return ELSI_OK;
        h->have_l_prec = ELSI_PREC_FP32_REFINE;
    } else {
        CKR(check_finite<double>(st, n, n, rq.ham, n, w.status));
    }
    CKR(cudaEventRecord(w.ev[STAGE_STDFORM], st));
    if (!unit) {
        CKR(copy_matrix<float, double>(st, n, n, rq.ham, n, Y, n));
        CKR(trsm_left_lower<float>(st, 0, n, n, L, n, INVD, Y, n, WORK));
        CKR(transpose<float>(st, n, n, Y, n, A, n));
        CKR(trsm_left_lower<float>(st, 0, n, n, L, n, INVD, A, n, WORK));
        CKR(symmetrize<float>(st, n, A, n));
    } else {
        CKR(copy_matrix<float, double>(st, n, n, rq.ham, n, A, n));
        CKR(symmetrize<float>(st, n, A, n));
    }
    const bool one_stage = h->elpa_solver == 1;
    CKR(cudaEventRecord(w.ev[STAGE_SY2SB], st));
    if (one_stage) {
        // Eq. 11 first form: T = Q^T H~ Q directly
        CKR(onestage_tridiag<float>(st, n, A, n, w.d, w.e, V1, T1, w.work));
        CKR(cudaEventRecord(w.ev[STAGE_SB2ST], st));
    } else {
        CKR(sy2sb<float>(st, n, b, A, n, V1, T1, WORK, w.work_cap / sizeof(float), w.sync, w.status, sms));
        CKR(cudaEventRecord(w.ev[STAGE_SB2ST], st));
        const int ldb = 2 * b + 1;
        CKR(extract_band<float>(st, n, b, A, n, BAND, ldb));
        CKR(sb2st<float>(st, n, b, BAND, ldb, w.d, w.e, V2, TAU2, w.status, w.sync, sms));
    }
    CKR(cudaEventRecord(w.ev[STAGE_TRIDIAG], st));
    // binary32-route eigenvalues: the wanted ones are recomputed by the refinement and the
    // rest are reported at the accuracy of this route. T itself carries the binary32
    // rounding of the reduction (about 6e-8 ||T||), so bisection to 1e-8 ||T|| changes
    // neither the eigenvalues nor, through the twisted factorisations, the eigenvectors
    // beyond that level. (At 1e-7 ||T|| the refinement of the 3D-cluster problem at
    // n = 16384 no longer converges and the solve falls back to the binary64 route.)
    CKR(stebz(st, n, w.d, w.e, n, w.w, w.status, 1e-8));
    // eigenvector scratch (3 n^2 + n binary64 values) in the digit-plane buffer, free here
    CKR(stein<float>(st, n, w.d, w.e, n, w.w, X32, n, reinterpret_cast<double *>(w.oz), w.status));
    CKR(cudaEventRecord(w.ev[STAGE_Q2], st));
    if (!one_stage) CKR(apply_q2_tc(st, n, b, V2, TAU2, n, X32, n, w.q2f, w.status));
    CKR(cudaEventRecord(w.ev[STAGE_Q1], st));
    if (one_stage) CKR(apply_q_onestage<float>(st, n, n, V1, T1, X32, n, WORK));
    else CKR(apply_q1<float>(st, n, b, n, V1, T1, X32, n, WORK));
    CKR(cudaEventRecord(w.ev[STAGE_BACKSUB], st));
    if (!unit) CKR(trsm_left_lower<float>(st, 1, n, n, L, n, INVD, X32, n, WORK));
    CKR(cudaEventRecord(w.ev[STAGE_REFINE], st));

    // ---------------- refinement of the k wanted eigenpairs
    const size_t nk = (size_t)n * k;
    double *XO = w.rf;                 // n x k binary64
    double *YH = XO + nk;              // n x k
    double *YS = YH + nk;              // n x k
    double *GOO = YS + nk;             // k x k
    double *SOO = GOO + (size_t)k * k; // k x k
    double *LAM = SOO + (size_t)k * k; // k
    double *GD = LAM + k;              // k
    double *SD = GD + k;               // k
    unsigned long long *STATS = reinterpret_cast<unsigned long long *>(SD + k);  // 4
    int *CID = reinterpret_cast<int *>(STATS + 4);        // k
    int *CSZ = CID + k;                                   // k
    double *QBUF = reinterpret_cast<double *>(CSZ + k);  // k x 32 x 32 (2k ints: 8-byte aligned)
    float *R32 = reinterpret_cast<float *>(QBUF + (size_t)k * kMaxCluster * kMaxCluster);  // n x k
    float *E32 = R32 + nk;                                // n x k
    float *M32 = E32 + nk;                                // (n-k) x k
    const double *S64 = unit ? nullptr : rq.ovlp;
    const double delta = 1e-4;  // Ha: eigenvalues closer than this are refined as a cluster

    // digit planes for the binary64-accurate products on the tensor cores
    const size_t pNN = ozaki_split_elems(n, n), pKN = ozaki_split_elems(k, n),
                 pNK = ozaki_split_elems(n, k);
    __nv_bfloat16 *HDG = w.oz, *SDG = HDG + pNN, *XDG = SDG + pNN, *YHDG = XDG + pKN,
                  *YSDG = YHDG + pKN, *PADG = YSDG + pKN, *PBDG = PADG + pNK, *WADG = PBDG + pNK;
    const size_t es = (size_t)n + k + 256;
    int *eH = w.ozexp, *eS = eH + es, *eX = eS + es, *eYH = eX + es, *eYS = eYH + es,
        *ePA = eYS + es, *ePB = ePA + es, *eWA = ePB + es;
    // H and S are symmetric: the split of their rows reads contiguous columns
    CKR(ozaki_split(st, n, n, rq.ham, n, 1, nullptr, nullptr, HDG, eH));
    if (S64) CKR(ozaki_split(st, n, n, S64, n, 1, nullptr, nullptr, SDG, eS));

    // products, cluster Rayleigh-Ritz rotation and the Rayleigh quotients of the
    // current X_o (steps shared by every iteration and the final polish). digits: digit
    // planes of the binary64-accurate products (D digits: D (D + 1) / 2 digit products,
    // truncation about 2^(-7 D) relative); the first iterations, which correct errors of
    // about 1e-3, need fewer than the later ones and the final polish (see the loop).
    auto products_and_rr = [&](int digits) -> int {
        CKR(ozaki_split(st, k, n, XO, n, 1, nullptr, nullptr, XDG, eX));
        CKR(ozaki_gemm(st, n, k, n, 1.0, HDG, eH, XDG, eX, 0.0, YH, n, 0, digits));
        if (S64) CKR(ozaki_gemm(st, n, k, n, 1.0, SDG, eS, XDG, eX, 0.0, YS, n, 0, digits));
        else CKR(cudaMemcpyAsync(YS, XO, sizeof(double) * nk, cudaMemcpyDeviceToDevice, st));
        CKR(ozaki_split(st, k, n, YH, n, 1, nullptr, nullptr, YHDG, eYH));
        CKR(ozaki_split(st, k, n, YS, n, 1, nullptr, nullptr, YSDG, eYS));
        // X^T H X and X^T S X are symmetric; the rounding of a full product is not, and an
        // antisymmetric error would enter E_ij + E_ji (the re-orthonormalisation) divided
        // by lambda_j - lambda_i. Form the lower triangles (half the work) and mirror them.
        CKR(ozaki_gemm(st, k, k, n, 1.0, XDG, eX, YHDG, eYH, 0.0, GOO, k, 1, digits));
        CKR(ozaki_gemm(st, k, k, n, 1.0, XDG, eX, YSDG, eYS, 0.0, SOO, k, 1, digits));
        CKR(mirror_lower<double>(st, k, GOO, k));
        CKR(mirror_lower<double>(st, k, SOO, k));
        cluster_scan_kernel<<<1, 1, 0, st>>>(k, GOO, SOO, delta, CID, CSZ);
        cluster_rr_kernel<<<k, 32, 0, st>>>(k, GOO, SOO, CID, CSZ, QBUF);
        rotate_cols_kernel<<<dim3(k, ceil_div(n, 256)), 256, 0, st>>>(n, k, CID, CSZ, QBUF, XO, YH, YS);
        rotate_gram_kernel<<<dim3(k, 1), 256, 0, st>>>(k, CID, CSZ, QBUF, GOO, SOO, 0);
        rotate_gram_kernel<<<dim3(k, 1), 256, 0, st>>>(k, CID, CSZ, QBUF, GOO, SOO, 1);
        gram_diag_kernel<<<grid_for(k), 256, 0, st>>>(k, GOO, SOO, GD, SD);
        residual_kernel<<<grid_for(nk), 256, 0, st>>>(n, k, GD, SD, LAM, YH, YS, R32);
        return cudaGetLastError() == cudaSuccess ? ELSI_OK
                                                 : set_error(h, ELSI_ERR_CUDA, "refinement launch");
    };

    CKR(copy_matrix<double, float>(st, n, k, X32, n, XO, n));
    const char *venv = getenv("ELSI_GB_VERBOSE");
    const bool verbose = venv && venv[0] == '1';
    int iters = 0;
    double emax = 1.0;
    for (int it = 0; it < h->refine_max_iter; ++it) {
        // digit planes of this iteration's products: 4 and 5 in the first two iterations
        // (binary32 start, errors of about 1e-3), 7 from the third on. The corrections of
        // the states next to the wanted/unwanted boundary are divided by their gap, which
        // can be far below the cluster threshold: with 5 digits in the third iteration
        // max|E| stalls near 6e-4 on the 3D-cluster problem at n = 16384 (the binary64
        // fallback follows), with 7 it reaches 9e-6 and then 1.4e-9.
        const int digits = it == 0 ? 4 : (it == 1 ? 5 : kOzDigits);
        int rc = products_and_rr(digits);
        if (rc) return rc;
        // M = Xu^T R_o in binary32
        if (n > k)
            CKR(gemm<float>(st, 1, 0, n - k, k, n, 1.0f, X32 + (size_t)k * n, n, R32, n, 0.0f, M32, n - k));
        CKR(cudaMemsetAsync(STATS, 0, 4 * sizeof(unsigned long long), st));
        EGB_COUNT_LAUNCH();
        build_e_kernel<<<grid_for(nk), 256, 0, st>>>(n, k, GOO, SOO, M32, LAM, w.w, CID, E32, STATS);
        // X_o += [X_o | X_u] E  (binary32 product of small corrections; the X_o block of
        // the binary32 matrix is refreshed from the current binary64 X_o first)
        CKR(copy_matrix<float, double>(st, n, k, XO, n, X32, n));
        CKR(gemm<float>(st, 0, 0, n, k, n, 1.0f, X32, n, E32, n, 0.0f, R32, n));
        EGB_COUNT_LAUNCH();
        add_f32_to_f64_kernel<<<grid_for(nk), 256, 0, st>>>(nk, R32, XO);
        CKR(cudaMemcpyAsync(w.scal_host + 8, STATS, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CKR(cudaStreamSynchronize(st));
        emax = w.scal_host[8];
        ++iters;
        if (verbose)
            fprintf(stderr, "[elsi-gb] refine iteration %d (%d digits): max|E| %.3e, max|R_oo| %.3e\n", iters,
                    digits, emax, w.scal_host[9]);
        if (emax < 1e-12) break;
    }
    // final polish: Rayleigh-Ritz inside clusters, Rayleigh quotients, orthonormality
    {
        int rc = products_and_rr(kOzDigits);
        if (rc) return rc;
        CKR(cudaMemsetAsync(STATS, 0, 4 * sizeof(unsigned long long), st));
        EGB_COUNT_LAUNCH();
        orth_defect_kernel<<<grid_for((size_t)k * k), 256, 0, st>>>(k, SOO, STATS);
        EGB_COUNT_LAUNCH();
        wanted_order_kernel<<<1, 256, 0, st>>>(n, k, LAM, w.w, reinterpret_cast<double *>(STATS + 2));
        CKR(cudaMemcpyAsync(w.scal_host + 8, STATS, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CKR(cudaStreamSynchronize(st));
    }
    h->refine_iters = iters;
    h->orth_err = w.scal_host[8];
    if (verbose) fprintf(stderr, "[elsi-gb] refine final orthonormality defect %.3e\n", h->orth_err);
    if (!(emax < 1e-8) || !(h->orth_err < 1e-10))
        return set_error(h, ELSI_ERR_NO_CONVERGENCE,
                         "refinement did not converge (max|E| %.3g, orthonormality %.3g)", emax,
                         h->orth_err);
    // The refinement converges to the eigenpairs nearest its binary32 start. A start whose
    // error exceeds the gaps (a standard form spoilt by a nearly singular S) can converge to
    // a pair above the k-th: a refined wanted eigenvalue above the binary32 estimate of the
    // first unwanted one, by more than that estimate's error, shows it.
    if (!(w.scal_host[10] <= 1e-4 * fmax(1.0, w.scal_host[11])))
        return set_error(h, ELSI_ERR_NO_CONVERGENCE,
                         "refined states are not the lowest %d (max refined eigenvalue %.6g above "
                         "the next binary32 one)", k, w.scal_host[10]);
    // eigenvalues: refined for the wanted states, binary32-route values for the rest
    EGB_COUNT_LAUNCH();
    copy_eval_kernel<<<grid_for(n), 256, 0, st>>>(n, k, LAM, w.w, w.w);
    CKR(cudaEventRecord(w.ev[STAGE_OCC], st));
    if (ev_mode) {
        CKR(cudaMemcpyAsync(rq.eval, w.w, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        CKR(cudaMemcpyAsync(rq.evec, XO, sizeof(double) * nk, cudaMemcpyDeviceToDevice, st));
        CKR(cudaEventRecord(w.ev[STAGE_DENSITY], st));
    } else {
        CKR(occupation(st, k, w.w, h->n_electron, h->scheme, h->kt, h->occ_accuracy,
                       h->mu_max_steps, w.f, w.scal, w.status, h->occ_stride));
        CKR(cudaEventRecord(w.ev[STAGE_DENSITY], st));
        int kocc = k;
        if (h->scheme == ELSI_OCC_INTEGER) {
            kocc = (int)((h->n_electron / h->occ_stride + 1.999999999) / 2.0) * h->occ_stride;
            if (kocc > k) kocc = k;
            if (kocc < 1) kocc = 1;
        }
        // P = X_o diag(f) X_o^T and W = X_o diag(f eps) X_o^T, binary64-accurate products
        // of the rows of X_o on the tensor cores (lower triangle, then mirrored)
        CKR(ozaki_split(st, n, kocc, XO, 1, n, nullptr, nullptr, PBDG, ePB));
        CKR(ozaki_split(st, n, kocc, XO, 1, n, w.f, nullptr, PADG, ePA));
        CKR(ozaki_gemm(st, n, n, kocc, 1.0, PADG, ePA, PBDG, ePB, 0.0, rq.dm, n, 1));
        CKR(mirror_lower<double>(st, n, rq.dm, n));
        if (rq.want_edm) {
            CKR(ozaki_split(st, n, kocc, XO, 1, n, w.f, w.w, WADG, eWA));
            CKR(ozaki_gemm(st, n, n, kocc, 1.0, WADG, eWA, PBDG, ePB, 0.0, w.edm, n, 1));
            CKR(mirror_lower<double>(st, n, w.edm, n));
        }
    }
    CKR(cudaEventRecord(w.ev[kNumStages], st));
    return ELSI_OK;
}

}  // namespace egb
