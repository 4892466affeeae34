// Panel factorisation of the full -> band reduction (Eq. 11, first line; step (1) of the
// two-stage method, sec. 3.1) without a grid-wide barrier per column: tall-skinny QR
// (TSQR: Demmel, Grigori, Hoemmen & Langou 2012) followed by Householder reconstruction
// (Ballard, Demmel, Grigori, Jacquelin, Nguyen & Solomonik 2014).
//
//  1. Every block of 256 panel rows is factored on its own, X_g = Q_g R_g (Householder QR
//     in shared memory, one CTA per block); the R_g are stacked and the stack is factored
//     the same way, level after level (4 R factors per block), until one block is left;
//     its R is the panel's R up to the signs of its rows.
//  2. The explicit first b columns of the orthogonal factor are formed top-down: the top
//     block's reflectors applied to [I; 0], then every block's reflectors applied to its
//     64-row slice of the level above, padded with zeros, down to the panel rows.
//  3. With Q (m x b) known, the compact-WY factors of the Householder QR of the panel are
//     recovered from the LU factorisation without pivoting of Q - [S; 0], S = diag(s_j),
//     s_j = -sign of the j-th pivot (so that no pivot is smaller than 1 in magnitude):
//     V = L (unit lower trapezoidal), T = -U S L_1^{-T}, R_H = S R. Then
//     (I - V T V^T)[:, 0:b] R_H is the panel, I - V T V^T is orthogonal.
// Every step is local to one CTA; a panel costs a handful of launches instead of one
// grid-wide barrier per column. Binary32 panels of more than 256 rows (the binary64
// route and short panels keep the cooperative one-barrier-per-column factorisation).
#include "common.cuh"
#include "kernels.h"

namespace egb {

constexpr int kTsRows = 256;  // rows per block
constexpr int kTsB = 64;      // panel width (band width b <= 64)
constexpr int kTsLd = kTsB + 1;

// Householder QR of the rows x bw block held row-major in shared memory (ld kTsLd, rows
// beyond the valid ones zero): on return the strict lower part holds the reflector tails
// v (v_j = 1 implied), the upper part R, tau[j] the reflector scalars. 256 threads.
template <typename T>
__device__ void block_house_qr(T *blk, int bw, T *tau, double *red, double *part, double *wcol)
{
    const int tid = threadIdx.x;
    const int tc = tid & 63, tr = tid >> 6;  // 64 column lanes x 4 row groups of 64 rows
    for (int j = 0; j < bw; ++j) {
        // sigma = sum_{i > j} x_i^2 (binary64 partials)
        double s = 0.0;
        for (int i = j + 1 + tid; i < kTsRows; i += blockDim.x) {
            const double x = (double)blk[i * kTsLd + j];
            s = fma(x, x, s);
        }
        s = block_sum(s, red);
        if (tid == 0) {
            const double alpha = (double)blk[j * kTsLd + j];
            if (s == 0.0) {
                red[1] = 0.0;  // tau
                red[2] = 0.0;  // scale of the tail
            } else {
                const double nrm = sqrt(alpha * alpha + s);
                const double beta = alpha >= 0.0 ? -nrm : nrm;
                red[1] = (beta - alpha) / beta;
                red[2] = 1.0 / (alpha - beta);
                blk[j * kTsLd + j] = (T)beta;
            }
            tau[j] = (T)red[1];
        }
        __syncthreads();
        const double tj = red[1];
        const T scl = (T)red[2];
        for (int i = j + 1 + tid; i < kTsRows; i += blockDim.x) blk[i * kTsLd + j] *= scl;
        __syncthreads();
        if (tj != 0.0) {
            // w_c = x_jc + sum_{i>j} v_i x_ic, then x_ic -= tau v_i w_c (i >= j)
            const int c = tc;
            double d = 0.0;
            if (c > j && c < bw)
                for (int i = max(j + 1, tr * 64); i < tr * 64 + 64; ++i)
                    d = fma((double)blk[i * kTsLd + j], (double)blk[i * kTsLd + c], d);
            part[tr * 64 + c] = d;
            __syncthreads();
            if (tr == 0 && c > j && c < bw)
                wcol[c] = tj * ((double)blk[j * kTsLd + c] + part[c] + part[64 + c] + part[128 + c] +
                                part[192 + c]);
            __syncthreads();
            if (c > j && c < bw) {
                const T w = (T)wcol[c];
                if (tr == (j >> 6)) blk[j * kTsLd + c] -= w;  // v_j = 1
                for (int i = max(j + 1, tr * 64); i < tr * 64 + 64; ++i)
                    blk[i * kTsLd + c] = fma(-blk[i * kTsLd + j], w, blk[i * kTsLd + c]);
            }
            __syncthreads();
        }
    }
}

// One level of the tree: X (rows x bw, column-major, ld ldx) in blocks of kTsRows rows,
// one CTA per block. The reflector tails go back into X (in place), tau to tau[g * 64 + j],
// R_g (bw x bw upper triangle, zeros below) to rows g * bw .. of Rn (column-major, ld ldr).
template <typename T>
__global__ void __launch_bounds__(256) tsqr_qr_kernel(int rows, int bw, T *X, int ldx, T *tau, T *Rn,
                                                      int ldr)
{
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    T *blk = reinterpret_cast<T *>(tsm_raw);
    __shared__ double red[32], part[256], wcol[64];
    __shared__ T tloc[64];
    const int g = blockIdx.x, r0 = g * kTsRows;
    const int nr = min(kTsRows, rows - r0);
    for (int e = threadIdx.x; e < kTsRows * bw; e += blockDim.x) {
        const int i = e % kTsRows, c = e / kTsRows;
        blk[i * kTsLd + c] = (i < nr) ? X[(size_t)(r0 + i) + (size_t)c * ldx] : T(0);
    }
    __syncthreads();
    block_house_qr<T>(blk, bw, tloc, red, part, wcol);
    for (int e = threadIdx.x; e < nr * bw; e += blockDim.x) {
        const int i = e % nr, c = e / nr;
        X[(size_t)(r0 + i) + (size_t)c * ldx] = blk[i * kTsLd + c];
    }
    for (int e = threadIdx.x; e < bw * bw; e += blockDim.x) {
        const int i = e % bw, c = e / bw;
        Rn[(size_t)(g * bw + i) + (size_t)c * ldr] = (i <= c) ? blk[i * kTsLd + c] : T(0);
    }
    if (threadIdx.x < bw) tau[g * 64 + threadIdx.x] = tloc[threadIdx.x];
}

// Explicit Q of one level, block g: the block's reflectors (tails in Y, ld ldy; tau)
// applied to E = [Qp[g * bw .. g * bw + bw - 1, :]; 0] (Qp = nullptr: E = [I; 0]), in the
// order H_0 H_1 ... H_{bw-1} E; rows of the block to Qo (ld ldo).
template <typename T>
__global__ void __launch_bounds__(256) tsqr_q_kernel(int rows, int bw, const T *Y, int ldy, const T *tau,
                                                     const T *Qp, int ldp, T *Qo, int ldo)
{
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    T *yb = reinterpret_cast<T *>(tsm_raw);      // reflector tails (kTsRows x bw)
    T *eb = yb + kTsRows * kTsLd;                // E (kTsRows x bw)
    __shared__ double part[256], wcol[64];
    const int g = blockIdx.x, r0 = g * kTsRows;
    const int nr = min(kTsRows, rows - r0);
    const int tid = threadIdx.x, tc = tid & 63, tr = tid >> 6;
    for (int e = tid; e < kTsRows * bw; e += blockDim.x) {
        const int i = e % kTsRows, c = e / kTsRows;
        yb[i * kTsLd + c] = (i < nr && i > c) ? Y[(size_t)(r0 + i) + (size_t)c * ldy] : T(0);
        T ev = T(0);
        if (i < bw) ev = Qp ? Qp[(size_t)(g * bw + i) + (size_t)c * ldp] : (i == c ? T(1) : T(0));
        eb[i * kTsLd + c] = ev;
    }
    __syncthreads();
    for (int j = bw - 1; j >= 0; --j) {
        const double tj = (double)tau[g * 64 + j];
        if (tj == 0.0) continue;
        // w_c = e_jc + sum_{i>j} v_i e_ic ; e_ic -= tau v_i w_c
        const int c = tc;
        double d = 0.0;
        if (c < bw)
            for (int i = max(j + 1, tr * 64); i < tr * 64 + 64; ++i)
                d = fma((double)yb[i * kTsLd + j], (double)eb[i * kTsLd + c], d);
        part[tr * 64 + c] = d;
        __syncthreads();
        if (tr == 0 && c < bw)
            wcol[c] = tj * ((double)eb[j * kTsLd + c] + part[c] + part[64 + c] + part[128 + c] + part[192 + c]);
        __syncthreads();
        if (c < bw) {
            const T w = (T)wcol[c];
            if (tr == (j >> 6)) eb[j * kTsLd + c] -= w;
            for (int i = max(j + 1, tr * 64); i < tr * 64 + 64; ++i)
                eb[i * kTsLd + c] = fma(-yb[i * kTsLd + j], w, eb[i * kTsLd + c]);
        }
        __syncthreads();
    }
    for (int e = tid; e < nr * bw; e += blockDim.x) {
        const int i = e % nr, c = e / nr;
        Qo[(size_t)(r0 + i) + (size_t)c * ldo] = eb[i * kTsLd + c];
    }
}

// Householder reconstruction, top block (one CTA): LU of Q_1 - S without pivoting
// (s_j = -sign of the current pivot), V_1 = L_1 (unit lower, written over Q_1 in V),
// T = -U S L_1^{-T}, the panel's R_H = S R (upper triangle of P's first bw rows, zeros
// below), U to Ub (bw x bw, ld bw) for the rows below.
template <typename T>
__global__ void __launch_bounds__(256) tsqr_recon_top_kernel(int bw, T *V, int ldv, const T *R, int ldr,
                                                             T *P, int ldp, T *Tm, int ldt, T *Ub)
{
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    double(*A)[65] = reinterpret_cast<double(*)[65]>(tsm_raw);              // Q_1, then L \ U
    double(*Li)[65] = reinterpret_cast<double(*)[65]>(tsm_raw + 64 * 65 * sizeof(double));
    __shared__ double sgn[64];
    const int tid = threadIdx.x;
    for (int e = tid; e < bw * bw; e += blockDim.x) {
        const int i = e % bw, c = e / bw;
        A[i][c] = (double)V[(size_t)i + (size_t)c * ldv];
    }
    __syncthreads();
    // right-looking LU: row j of U, column j of L
    for (int j = 0; j < bw; ++j) {
        if (tid == 0) {
            const double s = A[j][j] >= 0.0 ? -1.0 : 1.0;
            sgn[j] = s;
            A[j][j] -= s;
        }
        __syncthreads();
        const double piv = A[j][j];
        for (int i = j + 1 + tid; i < bw; i += blockDim.x) A[i][j] /= piv;
        __syncthreads();
        for (int e = tid; e < (bw - j - 1) * (bw - j - 1); e += blockDim.x) {
            const int i = j + 1 + e % (bw - j - 1), c = j + 1 + e / (bw - j - 1);
            A[i][c] = fma(-A[i][j], A[j][c], A[i][c]);
        }
        __syncthreads();
    }
    // L_1^{-1} (unit lower) by columns: Li[:, c] solves L x = e_c
    for (int c = tid; c < bw; c += blockDim.x) {
        for (int i = 0; i < bw; ++i) {
            double x = (i == c) ? 1.0 : 0.0;
            for (int p = c; p < i; ++p) x -= A[i][p] * Li[p][c];
            Li[i][c] = (i >= c) ? x : 0.0;
        }
    }
    __syncthreads();
    // T = -U S L_1^{-T}: T[i][c] = -sum_{p >= i} U[i][p] s_p Li[c][p]  (upper: p <= c)
    for (int e = tid; e < bw * bw; e += blockDim.x) {
        const int i = e % bw, c = e / bw;
        double t = 0.0;
        if (i <= c)
            for (int p = i; p <= c; ++p) t += A[i][p] * sgn[p] * Li[c][p];
        Tm[(size_t)i + (size_t)c * ldt] = (T)(-t);
    }
    for (int e = tid; e < bw * bw; e += blockDim.x) {
        const int i = e % bw, c = e / bw;
        V[(size_t)i + (size_t)c * ldv] = (T)(i > c ? A[i][c] : (i == c ? 1.0 : 0.0));
        Ub[i + c * bw] = (T)(i <= c ? A[i][c] : 0.0);
        P[(size_t)i + (size_t)c * ldp] = (T)(i <= c ? sgn[i] * (double)R[(size_t)i + (size_t)c * ldr] : 0.0);
    }
}

// Rows below the top block: V_2 = Q_2 U^{-1} (x U = q by forward substitution over the
// columns), one thread per row; the panel rows below its R are cleared.
template <typename T>
__global__ void __launch_bounds__(128) tsqr_recon_rows_kernel(int m, int bw, T *V, int ldv, const T *Ub,
                                                              T *P, int ldp)
{
    __shared__ T u[64 * 64];
    for (int e = threadIdx.x; e < bw * bw; e += blockDim.x) u[e] = Ub[e];
    __syncthreads();
    const int i = bw + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    T x[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) {
        if (c < bw) {
            T q = V[(size_t)i + (size_t)c * ldv];
            for (int p = 0; p < c; ++p) q = fma(-x[p], u[p + c * bw], q);
            x[c] = q / u[c + c * bw];
            V[(size_t)i + (size_t)c * ldv] = x[c];
            P[(size_t)i + (size_t)c * ldp] = T(0);
        }
    }
}

size_t tsqr_scratch_elems(int m, int bw)
{
    // stacked R factors of every level, their reflector scalars, two explicit-Q buffers,
    // the top R and U
    size_t total = 0;
    int rows = m, G = ceil_div(m, kTsRows);
    size_t qmax = 0;
    while (true) {
        total += (size_t)G * 64;  // tau
        const size_t next = (size_t)G * bw;
        total += next * bw;       // R stack (or the top R)
        if (G == 1) break;
        qmax = next > qmax ? next : qmax;
        rows = (int)next;
        G = ceil_div(rows, kTsRows);
    }
    return total + 2 * qmax * bw + (size_t)bw * bw + 64;
}

template <typename T>
cudaError_t tsqr_panel(cudaStream_t st, int m, int bw, T *P, int ldp, T *V, int ldv, T *Tm, int ldt,
                       T *scratch, size_t scratch_elems)
{
    if (bw > kTsB || m <= kTsRows || scratch_elems < tsqr_scratch_elems(m, bw)) return cudaErrorInvalidValue;
    const size_t qsm = (size_t)kTsRows * kTsLd * sizeof(T);
    const size_t rsm = (size_t)2 * 64 * 65 * sizeof(double);
    static PerDeviceOnce attr;  // per instantiation
    cudaError_t e = once_per_device(attr, [&] {
        cudaError_t r = cudaFuncSetAttribute(tsqr_qr_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsm);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(tsqr_q_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * qsm));
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(tsqr_recon_top_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)rsm);
        return r;
    });
    if (e != cudaSuccess) return e;
    // levels: X_0 = P; X_{l+1} = stack of the R factors of level l
    struct Level { T *X; int rows, ld, G; T *tau; };
    Level lv[16];
    int nl = 0;
    T *sp = scratch;
    T *X = P;
    int rows = m, ld = ldp;
    T *Rtop = nullptr;
    while (true) {
        const int G = ceil_div(rows, kTsRows);
        if (nl >= 16) return cudaErrorInvalidValue;
        T *tau = sp;
        sp += (size_t)G * 64;
        T *Rn = sp;
        const int nrows = G * bw;
        sp += (size_t)nrows * bw;
        lv[nl++] = Level{X, rows, ld, G, tau};
        EGB_COUNT_LAUNCH();
        tsqr_qr_kernel<T><<<G, 256, qsm, st>>>(rows, bw, X, ld, tau, Rn, nrows);
        if (G == 1) { Rtop = Rn; break; }
        X = Rn;
        rows = nrows;
        ld = nrows;
    }
    // explicit Q, top-down; level 0 writes into V
    size_t qmax = 0;
    for (int l = 1; l < nl; ++l) qmax = (size_t)lv[l].rows > qmax ? (size_t)lv[l].rows : qmax;
    T *qbuf[2] = {sp, sp + qmax * bw};
    sp += 2 * qmax * bw;
    T *Ub = sp;
    const T *Qp = nullptr;
    int ldq = 0;
    for (int l = nl - 1; l >= 0; --l) {
        T *Qo = (l == 0) ? V : qbuf[l & 1];
        const int ldo = (l == 0) ? ldv : lv[l].rows;
        EGB_COUNT_LAUNCH();
        tsqr_q_kernel<T><<<lv[l].G, 256, 2 * qsm, st>>>(lv[l].rows, bw, lv[l].X, lv[l].ld, lv[l].tau, Qp, ldq,
                                                        Qo, ldo);
        Qp = Qo;
        ldq = ldo;
    }
    EGB_COUNT_LAUNCH();
    tsqr_recon_top_kernel<T><<<1, 256, rsm, st>>>(bw, V, ldv, Rtop, bw, P, ldp, Tm, ldt, Ub);
    EGB_COUNT_LAUNCH();
    tsqr_recon_rows_kernel<T><<<ceil_div(m - bw, 128), 128, 0, st>>>(m, bw, V, ldv, Ub, P, ldp);
    return cudaGetLastError();
}

template cudaError_t tsqr_panel<float>(cudaStream_t, int, int, float *, int, float *, int, float *, int,
                                       float *, size_t);

}  // namespace egb

extern "C" size_t elsi_gb_tsqr_work(int m, int bw) { return egb::tsqr_scratch_elems(m, bw) + 64; }

extern "C" int elsi_gb_tsqr_panel_f32(int m, int bw, float *P, int ldp, float *V, int ldv, float *Tm,
                                      int ldt, float *work, size_t work_elems, void *stream)
{
    if (m <= 256 || bw < 1 || bw > 64 || ldp < m || ldv < m || ldt < bw || !P || !V || !Tm || !work)
        return ELSI_ERR_ARG;
    cudaError_t e = egb::tsqr_panel<float>((cudaStream_t)stream, m, bw, P, ldp, V, ldv, Tm, ldt, work,
                                           work_elems);
    if (e == cudaErrorInvalidValue) return ELSI_ERR_ARG;
    return e == cudaSuccess ? ELSI_OK : ELSI_ERR_CUDA;
}
