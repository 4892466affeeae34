// Band -> tridiagonal reduction T = Q2^T B Q2 by bulge chasing (arXiv:1705.11191 Eq. 11,
// second line; step (2) of the two-stage tridiagonalisation, sec. 3.1, after Bischof,
// Lang & Sun's successive band reduction), and the back-transformation of eigenvectors
// through Q2 (step (4)).
//
// Sweep j (0 <= j <= n-3) annihilates column j below the subdiagonal and chases the
// resulting bulge down the band in steps t = 0, 1, ...; step t owns the index window
// [j+1+(t-1)b, j+(t+1)b]. Among the tasks of sweep j-1 only step t+1 overlaps the window
// of step t of sweep j, so the sweeps run concurrently in a persistent cooperative kernel:
// CTA g takes sweeps g, g + G, ..., each (sweep, step) task out of shared memory, and
// before step t of sweep j it waits (bounded spin) on the progress flag of sweep j-1
// until that sweep has finished step t+1. No grid-wide barrier is involved.
//
// Each step stores its Householder reflector (b entries, v[0] = 1) and tau in slot
// j * S + t (S = steps of sweep 0); the back-transformation applies them in the
// reverse of a valid application order.
#include "common.cuh"
#include "kernels.h"

namespace egb {

int sb2st_steps(int n, int b) { return (n >= 3) ? (n - 2) / b + 1 : 1; }

template <typename T>
__global__ void extract_band_kernel(int n, int b, const T *a, int lda, T *band, int ldb)
{
    size_t total = (size_t)ldb * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int dd = (int)(e % ldb), c = (int)(e / ldb);
        int r = c + dd;
        T v = T(0);
        if (dd <= b && r < n) v = a[(size_t)r + (size_t)c * lda];
        band[e] = v;
    }
}

template <typename T>
cudaError_t extract_band(cudaStream_t st, int n, int b, const T *a, int lda, T *band, int ldb)
{
    size_t total = (size_t)ldb * n;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    EGB_COUNT_LAUNCH();
    extract_band_kernel<T><<<grid, 256, 0, st>>>(n, b, a, lda, band, ldb);
    return cudaGetLastError();
}
template cudaError_t extract_band<double>(cudaStream_t, int, int, const double *, int, double *, int);
template cudaError_t extract_band<float>(cudaStream_t, int, int, const float *, int, float *, int);

struct ChaseArgs {
    int n, b, ldb, S;
    long long tmax;
    unsigned *count, *gen;
    int *status;
    long long spin_limit;  // polls of a progress-flag wait before ELSI_ERR_TIMEOUT
};

// Householder vector for x (length L) in shared memory: on return x holds v (v[0]=1),
// and the function returns tau; *beta_out receives the new leading entry.
template <typename T>
__device__ T house_smem(int L, T *x, T *red, T *beta_out)
{
    T ss = T(0);
    for (int i = 1 + threadIdx.x; i < L; i += blockDim.x) ss = fma(x[i], x[i], ss);
    ss = block_sum(ss, red);
    T alpha = x[0];
    T tau = T(0), beta = alpha;
    if (ss != T(0)) {
        T nrm = dsqrt<T>(alpha * alpha + ss);
        beta = (alpha >= T(0)) ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        T scl = T(1) / (alpha - beta);
        for (int i = 1 + threadIdx.x; i < L; i += blockDim.x) x[i] = x[i] * scl;
    } else {
        for (int i = 1 + threadIdx.x; i < L; i += blockDim.x) x[i] = T(0);
    }
    __syncthreads();
    if (threadIdx.x == 0) x[0] = T(1);
    __syncthreads();
    *beta_out = beta;
    return tau;
}

// out[i] = scale * sum_{c < nc} M[i + c * ldm] v[c] for i < L (L <= 64), four lanes per
// row (columns c = part + 4j), blockDim.x == 256. Ends with __syncthreads().
template <typename T>
__device__ __forceinline__ void rows_dot(int L, int nc, const T *M, int ldm, const T *v, T scale,
                                         T *out)
{
    const int row = threadIdx.x >> 2, part = threadIdx.x & 3;
    T s = T(0);
    if (row < L)
        for (int c = part; c < nc; c += 4) s = fma(M[row + c * ldm], v[c], s);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (part == 0 && row < L) out[row] = scale * s;
    __syncthreads();
}

// out[c] = scale * sum_{i < L} v[i] M[i + c * ldm] for c0 <= c < nc (nc <= 64), four lanes per
// column (rows i = part + 4j). Ends with __syncthreads().
template <typename T>
__device__ __forceinline__ void cols_dot(int L, int c0, int nc, const T *M, int ldm, const T *v,
                                         T scale, T *out)
{
    const int c = threadIdx.x >> 2, part = threadIdx.x & 3;
    T s = T(0);
    if (c >= c0 && c < nc)
        for (int i = part; i < L; i += 4) s = fma(v[i], M[i + c * ldm], s);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (part == 0 && c >= c0 && c < nc) out[c] = scale * s;
    __syncthreads();
}

// D (L x L, symmetric, ld ldd) <- H D H, H = I - tau v v^T. p: scratch of length L.
template <typename T>
__device__ void two_sided(int L, T *D, int ldd, const T *v, T tau, T *p, T *red)
{
    if (tau == T(0)) return;
    rows_dot<T>(L, L, D, ldd, v, tau, p);  // p = tau D v
    T part = T(0);
    for (int i = threadIdx.x; i < L; i += blockDim.x) part = fma(p[i], v[i], part);
    T K = T(0.5) * tau * block_sum(part, red);
    for (int i = threadIdx.x; i < L; i += blockDim.x) p[i] -= K * v[i];  // q
    __syncthreads();
    const int i = threadIdx.x & 63;
    if (i < L)
        for (int c = threadIdx.x >> 6; c < L; c += 4) D[i + c * ldd] = D[i + c * ldd] - v[i] * p[c] - p[i] * v[c];
    __syncthreads();
}

// Loads of data that other CTAs of the same launch write (band, reflectors) bypass L1.
template <typename T>
__device__ __forceinline__ T ldg_l2(const T *p) { return __ldcg(p); }


// Columns of a b x b tile per thread in the element loops (row ti = tid mod 64, columns
// tc, tc + 4, ..., tc = tid / 64; 256 threads, b <= 64).
constexpr int kChaseCols = 16;

// One (sweep j, step t) task; all threads of the CTA take part. The b x b tiles use the
// leading dimension b + 8, which makes the four-lanes-per-row dot products
// conflict-free in shared memory.
template <typename T>
__device__ void chase_task(const ChaseArgs &a, T *band, T *v2, T *tau2, int j, int t, T *smem,
                           T *red)
{
    const int n = a.n, b = a.b, ldb = a.ldb;
    const int ld = b + 8;
    T *X = smem;                 // b x b (ld)
    T *D = X + b * ld;           // b x b (ld)
    T *vnew = D + b * ld;        // b
    T *vprev = vnew + b;         // b
    T *p = vprev + b;            // b
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ti = tid & 63, tc = tid >> 6;  // element loops: row ti, columns tc, tc + 4, ...
    size_t slot = (size_t)j * a.S + t;

    if (t == 0) {
        const int L = min(b, n - 1 - j);
        const int r0 = j + 1;
        for (int i = tid; i < b; i += nt) vnew[i] = (i < L) ? ldg_l2(band + (size_t)(1 + i) + (size_t)j * ldb) : T(0);
        // D = A[j+1 .. j+L]^2: lower triangle from the band, upper by symmetry (all loads of
        // a thread in flight together)
        {
            T dr[kChaseCols];
#pragma unroll
            for (int q = 0; q < kChaseCols; ++q) {
                const int c = tc + 4 * q;
                dr[q] = (ti < L && c <= ti) ? ldg_l2(band + (size_t)(ti - c) + (size_t)(r0 + c) * ldb) : T(0);
            }
#pragma unroll
            for (int q = 0; q < kChaseCols; ++q) {
                const int c = tc + 4 * q;
                if (ti < L && c <= ti) D[ti + c * ld] = dr[q];
            }
        }
        __syncthreads();
        if (ti < L)
            for (int c = ti + 1 + tc; c < L; c += 4) D[ti + c * ld] = D[c + ti * ld];
        __syncthreads();
        T beta;
        T tau = house_smem<T>(L, vnew, red, &beta);
        for (int i = tid; i < L; i += nt)
            band[(size_t)(1 + i) + (size_t)j * ldb] = (i == 0) ? beta : T(0);
        two_sided<T>(L, D, ld, vnew, tau, p, red);
        if (ti < L)
            for (int c = tc; c <= ti; c += 4) band[(size_t)(ti - c) + (size_t)(r0 + c) * ldb] = D[ti + c * ld];
        for (int i = tid; i < b; i += nt) v2[slot * b + i] = (i < L) ? vnew[i] : T(0);
        if (tid == 0) tau2[slot] = tau;
        __syncthreads();
        return;
    }
    const int r = j + 1 + t * b;
    const int L = min(b, n - r);
    const int cb = r - b;  // first column of X
    size_t pslot = slot - 1;
    // the previous step's reflector, loaded in the same batch as X and D below
    const T vp = (tid < b) ? ldg_l2(v2 + pslot * b + tid) : T(0);
    const T taup = ldg_l2(tau2 + pslot);
    // X = A[r .. r+L-1, cb .. cb+b-1]  (all strictly below the diagonal, distance 1..2b-1)
    // and D = A[r .. r+L-1]^2 (read now: the task's window is not touched by anyone else;
    // lower triangle from the band, upper by symmetry). Every load of a thread is issued
    // before the first store to shared memory, so that the (up to 32) L2 round trips of a
    // thread overlap instead of following one another.
    {
        T xr[kChaseCols], dr[kChaseCols];
#pragma unroll
        for (int q = 0; q < kChaseCols; ++q) {
            const int c = tc + 4 * q;
            xr[q] = (ti < L && c < b) ? ldg_l2(band + (size_t)(r + ti - (cb + c)) + (size_t)(cb + c) * ldb) : T(0);
            dr[q] = (ti < L && c <= ti) ? ldg_l2(band + (size_t)(ti - c) + (size_t)(r + c) * ldb) : T(0);
        }
#pragma unroll
        for (int q = 0; q < kChaseCols; ++q) {
            const int c = tc + 4 * q;
            if (ti < L && c < b) X[ti + c * ld] = xr[q];
            if (ti < L && c <= ti) D[ti + c * ld] = dr[q];
        }
        if (tid < b) vprev[tid] = vp;
    }
    __syncthreads();
    if (ti < L)
        for (int c = ti + 1 + tc; c < L; c += 4) D[ti + c * ld] = D[c + ti * ld];
    __syncthreads();
    // X <- X H_prev : y = X v, X -= tau y v^T
    if (taup != T(0)) {
        rows_dot<T>(L, b, X, ld, vprev, taup, p);
        if (ti < L)
            for (int c = tc; c < b; c += 4) X[ti + c * ld] = fma(-p[ti], vprev[c], X[ti + c * ld]);
        __syncthreads();
    }
    // new reflector from X[:, 0]
    for (int i = tid; i < b; i += nt) vnew[i] = (i < L) ? X[i] : T(0);
    __syncthreads();
    T beta;
    T tau = house_smem<T>(L, vnew, red, &beta);
    // left-apply to X[:, 1:]
    if (tau != T(0)) {
        cols_dot<T>(L, 1, b, X, ld, vnew, tau, p);
        if (ti < L)
            for (int c = 1 + tc; c < b; c += 4) X[ti + c * ld] = fma(-vnew[ti], p[c], X[ti + c * ld]);
        __syncthreads();
    }
    if (tid == 0) X[0] = beta;
    for (int i = 1 + tid; i < L; i += nt) X[i] = T(0);
    __syncthreads();
    if (ti < L)
        for (int c = tc; c < b; c += 4) band[(size_t)(r + ti - (cb + c)) + (size_t)(cb + c) * ldb] = X[ti + c * ld];
    two_sided<T>(L, D, ld, vnew, tau, p, red);
    if (ti < L)
        for (int c = tc; c <= ti; c += 4) band[(size_t)(ti - c) + (size_t)(r + c) * ldb] = D[ti + c * ld];
    for (int i = tid; i < b; i += nt) v2[slot * b + i] = (i < L) ? vnew[i] : T(0);
    if (tid == 0) tau2[slot] = tau;
    __syncthreads();
}

// Persistent bulge chase with point-to-point ordering: CTA g runs sweeps g, g + G, ... in
// order; step t of sweep j waits until sweep j-1 has finished step t+1 (or all its steps).
// Step t of sweep j touches rows and columns j+1+(t-1)b .. j+(t+1)b; among the tasks of
// sweep j-1 only step t+1 (rows from j+(t+1)b) overlaps that window, and step t+2 starts
// at row j+(t+2)b. With the same rule for j-1 this orders every pair of overlapping tasks
// as the sequential algorithm does. progress[j] = number of finished steps of sweep j.
template <typename T>
__global__ void __launch_bounds__(256) chase_kernel(T *band, T *v2, T *tau2, ChaseArgs a, int *progress)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    __shared__ T red[32];
    __shared__ int abort_flag;
    const int n = a.n, b = a.b;
    const int nsweep = n - 2;  // sweeps j = 0 .. n-3
    if (threadIdx.x == 0) abort_flag = 0;
    for (int j = blockIdx.x; j < nsweep; j += gridDim.x) {
        const int Sj = (n - 2 - j) / b + 1;
        const int Sprev = (j > 0) ? (n - 2 - (j - 1)) / b + 1 : 0;
        for (int t = 0; t < Sj; ++t) {
            if (j > 0) {
                const int need = min(t + 2, Sprev);
                if (threadIdx.x == 0) {
                    volatile int *pv = progress + (j - 1);
                    volatile int *vst = a.status;
                    long long it = 0;
                    while (*pv < need) {
                        if (vst[ST_CODE] != 0) { abort_flag = 1; break; }
                        if (++it > a.spin_limit) {
                            report_error(a.status, ELSI_ERR_TIMEOUT, j);
                            abort_flag = 1;
                            break;
                        }
                        __nanosleep(32);
                    }
                    __threadfence();
                }
                __syncthreads();
                if (abort_flag) return;
            }
            chase_task<T>(a, band, v2, tau2, j, t, smem, red);
            if (threadIdx.x == 0) {
                __threadfence();
                atomicExch(progress + j, t + 1);
            }
        }
    }
}

template <typename T>
__global__ void extract_tridiag_kernel(int n, const T *band, int ldb, double *d, double *e)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        d[i] = (double)band[(size_t)i * ldb];
        if (i + 1 < n) e[i] = (double)band[1 + (size_t)i * ldb];
    }
}

template <typename T>
cudaError_t sb2st(cudaStream_t st, int n, int b, T *band, int ldb, double *d, double *e,
                  T *v2, T *tau2, int *status, unsigned *sync, int num_sms)
{
    cudaError_t err;
    if (n >= 3) {
        const int S = sb2st_steps(n, b);
        ChaseArgs a;
        a.n = n; a.b = b; a.ldb = ldb; a.S = S;
        a.tmax = 3ll * (n - 3) + (S - 1);
        a.count = sync; a.gen = sync + 1; a.status = status;
        a.spin_limit = spin_limit();
        size_t smem = (2 * (size_t)b * (b + 8) + 3 * b) * sizeof(T);
        static PerDeviceOnce attr_set;  // per instantiation
        // opt in once per device for the largest band width (64)
        err = once_per_device(attr_set, [] {
            const size_t smax = (2 * 64 * 72 + 3 * 64) * sizeof(T);
            return cudaFuncSetAttribute(chase_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
        });
        if (err != cudaSuccess) return err;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chase_kernel<T>, 256, smem);
        int maxpar = (n - 2 + 1) / 2 + 1;  // upper bound of concurrently active sweeps
        int conc = S / 2 + 2;
        if (conc < maxpar) maxpar = conc;
        int G = per_sm * num_sms;
        if (G > maxpar) G = maxpar;
        if (G < 1) G = 1;
        int *progress = reinterpret_cast<int *>(sync + 64);
        if ((err = cudaMemsetAsync(progress, 0, sizeof(int) * (size_t)(n - 2), st)) != cudaSuccess) return err;
        void *args[] = {&band, &v2, &tau2, &a, &progress};
        EGB_COUNT_LAUNCH();
        if ((err = cudaLaunchCooperativeKernel((void *)chase_kernel<T>, dim3(G), dim3(256), args, smem,
                                               st)) != cudaSuccess)
            return err;
    }
    EGB_COUNT_LAUNCH();
    extract_tridiag_kernel<T><<<ceil_div(n, 256), 256, 0, st>>>(n, band, ldb, d, e);
    return cudaGetLastError();
}

template cudaError_t sb2st<double>(cudaStream_t, int, int, double *, int, double *, double *,
                                   double *, double *, int *, unsigned *, int);
template cudaError_t sb2st<float>(cudaStream_t, int, int, float *, int, double *, double *,
                                  float *, float *, int *, unsigned *, int);

// ------------------------------------------------------------------ Q2 back-transform
// Z <- Q2 Z. Q2 = prod over sweep blocks J (ascending) of prod over steps t (descending)
// of W(J,t) = H(J,t) H(J+1,t) ... H(J+m-1,t); so Z is updated for J descending, t
// ascending and, inside W(J,t), sweeps descending. Every lane owns one column of Z and
// keeps the rows of the current window in a shared-memory ring (row-major across the
// CTA's columns, so a warp's accesses are conflict-free); the dot product v^T z of each
// reflector is lane-local. The reflectors of one (J, t) are staged once per CTA.
constexpr int kQ2Sweeps = 64;   // m: sweeps per block
constexpr int kQ2Ring = 256;    // ring rows (>= m + 2b - 1 for b <= 64), power of two
constexpr int kQ2Lanes = 8;     // lanes per column
constexpr int kQ2RingLd = kQ2Ring + 8;  // column stride of the ring: the 4 columns of a warp
                                        // start 8 banks apart
// columns per CTA: binary32 32 (256 threads); binary64 8 (64 threads), so that the
// n_state columns of the binary64 route still spread over all SMs
template <typename T> struct Q2Cols;
template <> struct Q2Cols<float> { static constexpr int v = 32; };
template <> struct Q2Cols<double> { static constexpr int v = 8; };

__device__ __forceinline__ void cp_async_bytes(void *dst, const void *src, int bytes)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (bytes == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void q2_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void q2_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

template <typename T>
__global__ void __launch_bounds__(256)
apply_q2_kernel(int n, int b, int S, const T *__restrict__ v2, const T *__restrict__ tau2, int k,
                T *z, int ldz)
{
    constexpr int kQ2Cols = Q2Cols<T>::v;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *ring = reinterpret_cast<T *>(smem_raw);          // kQ2Cols x kQ2RingLd, [col][slot]
    T *vsb = ring + kQ2Cols * kQ2RingLd;                // 2 x (m x b) staged reflectors
    T *tsb = vsb + 2 * kQ2Sweeps * b;                   // 2 x m taus
    const int tid = threadIdx.x;
    const int lc = tid / kQ2Lanes;                      // local column
    const int sub = tid % kQ2Lanes;                     // row lane
    const int c0 = blockIdx.x * kQ2Cols;
    const int ncol = min(kQ2Cols, k - c0);
    const bool col_ok = lc < ncol;
    const int nsweep = n - 2;
    const int nblk = (nsweep + kQ2Sweeps - 1) / kQ2Sweeps;
    const unsigned gmask = 0xffu << ((tid & 31) & ~7);
    T *myring = ring + lc * kQ2RingLd;

    // asynchronous copy of rows [r0, r1) of the CTA's columns into the ring
    auto fetch_rows = [&](int r0, int r1) {
        const int nr = r1 - r0;
        for (int e = tid; e < nr * ncol; e += blockDim.x) {
            int r = r0 + e % nr, c = e / nr;
            cp_async_bytes(ring + c * kQ2RingLd + (r & (kQ2Ring - 1)), z + (size_t)r + (size_t)(c0 + c) * ldz,
                           (int)sizeof(T));
        }
    };
    auto store_rows = [&](int r0, int r1) {
        const int nr = r1 - r0;
        for (int e = tid; e < nr * ncol; e += blockDim.x) {
            int r = r0 + e % nr, c = e / nr;
            z[(size_t)r + (size_t)(c0 + c) * ldz] = ring[c * kQ2RingLd + (r & (kQ2Ring - 1))];
        }
    };
    // asynchronous staging of the reflectors of step t of sweeps [J, Jend) (zeros / tau 0
    // for sweeps that have no step t)
    auto fetch_refl = [&](int J, int Jend, int t, int buf) {
        T *vs = vsb + buf * kQ2Sweeps * b;
        T *ts = tsb + buf * kQ2Sweeps;
        for (int e = tid; e < (Jend - J) * b; e += blockDim.x) {
            int jj = e / b, i = e % b;
            int j = J + jj;
            int Sj = (n - 2 - j) / b + 1;
            if (t < Sj) cp_async_bytes(vs + jj * b + i, v2 + ((size_t)j * S + t) * b + i, (int)sizeof(T));
            else vs[jj * b + i] = T(0);
        }
        for (int jj = tid; jj < Jend - J; jj += blockDim.x) {
            int j = J + jj;
            int Sj = (n - 2 - j) / b + 1;
            if (t < Sj) cp_async_bytes(ts + jj, tau2 + (size_t)j * S + t, (int)sizeof(T));
            else ts[jj] = T(0);
        }
    };

    for (int jb = nblk - 1; jb >= 0; --jb) {
        const int J = jb * kQ2Sweeps;
        const int Jend = min(nsweep, J + kQ2Sweeps);  // sweeps J .. Jend-1
        const int SJ = (n - 2 - J) / b + 1;
        int lo = J + 1;                                // window [lo, hi)
        int hi = min(n, Jend + b);
        __syncthreads();
        fetch_rows(lo, hi);
        fetch_refl(J, Jend, 0, 0);
        q2_commit();
        for (int t = 0; t < SJ; ++t) {
            const int buf = t & 1;
            q2_wait_all();
            __syncthreads();
            // prefetch what step t+1 needs: its reflectors and the b rows entering the window
            const int nlo = min(lo + b, n), nhi = min(hi + b, n);
            if (t + 1 < SJ) {
                fetch_refl(J, Jend, t + 1, buf ^ 1);
                fetch_rows(hi, nhi);
            }
            q2_commit();
            const T *vs = vsb + buf * kQ2Sweeps * b;
            const T *ts = tsb + buf * kQ2Sweeps;
            for (int j = Jend - 1; j >= J; --j) {
                const int jj = j - J;
                const T tau = ts[jj];
                if (tau == T(0)) continue;
                const int r0 = j + 1 + t * b;
                const int L = min(b, n - r0);
                if (L <= 0) continue;
                const T *v = vs + jj * b;
                T sdot = T(0);
#pragma unroll 8
                for (int i = sub; i < L; i += kQ2Lanes)
                    sdot = fma(v[i], myring[(r0 + i) & (kQ2Ring - 1)], sdot);
                sdot += __shfl_xor_sync(gmask, sdot, 4);
                sdot += __shfl_xor_sync(gmask, sdot, 2);
                sdot += __shfl_xor_sync(gmask, sdot, 1);
                const T sc = tau * sdot;
#pragma unroll 8
                for (int i = sub; i < L; i += kQ2Lanes) {
                    T &zr = myring[(r0 + i) & (kQ2Ring - 1)];
                    zr = fma(-sc, v[i], zr);
                }
                __syncwarp(gmask);
            }
            __syncthreads();
            // rows [lo, nlo) are final for this block of sweeps
            if (t + 1 < SJ) {
                store_rows(lo, nlo);
                lo = nlo;
                hi = nhi;
            } else {
                store_rows(lo, hi);
            }
            (void)col_ok;
        }
    }
    q2_wait_all();
}

template <typename T>
cudaError_t apply_q2(cudaStream_t st, int n, int b, const T *v2, const T *tau2, int k, T *z,
                     int ldz, int *status)
{
    (void)status;
    if (n < 3 || k <= 0) return cudaSuccess;
    if (b > 64 || kQ2Sweeps + 2 * b - 1 > kQ2Ring) return cudaErrorInvalidValue;
    const int S = sb2st_steps(n, b);
    constexpr int kQ2Cols = Q2Cols<T>::v;
    size_t smem = ((size_t)kQ2Cols * kQ2RingLd + 2 * (size_t)kQ2Sweeps * b + 2 * kQ2Sweeps) * sizeof(T);
    static PerDeviceOnce attr_set;  // per instantiation
    cudaError_t e = once_per_device(attr_set, [] {
        const size_t smax =
            ((size_t)kQ2Cols * kQ2RingLd + 2 * (size_t)kQ2Sweeps * 64 + 2 * kQ2Sweeps) * sizeof(T);
        return cudaFuncSetAttribute(apply_q2_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    });
    if (e != cudaSuccess) return e;
    EGB_COUNT_LAUNCH();
    apply_q2_kernel<T><<<ceil_div(k, kQ2Cols), kQ2Cols * kQ2Lanes, smem, st>>>(n, b, S, v2, tau2, k, z, ldz);
    return cudaGetLastError();
}
template cudaError_t apply_q2<double>(cudaStream_t, int, int, const double *, const double *, int,
                                      double *, int, int *);
template cudaError_t apply_q2<float>(cudaStream_t, int, int, const float *, const float *, int,
                                     float *, int, int *);

// ------------------------------------------------------------------ Q1 back-transform
// Z <- Q1 Z, Q1 = Q_0 Q_1 ... Q_{P-1}, Q_p = I - V_p T_p V_p^T: panels descending.
// Z <- Q1 Z, Q1 = Q_0 Q_1 ... Q_{P-1} (panels of the full-to-band reduction, each
// Q_p = I - V_p T_p V_p^T). Groups of up to kQ1Group consecutive panels are applied as one
// compact-WY block Q_g = I - V T V^T, V = [V_p ... V_q] (explicit, zero above each panel's
// first row), T merged pairwise as [[T_a, -T_a (V_a^T V_b) T_b], [0, T_b]]: the passes
// over Z fall by the group size and the products have K = group width.
template <typename T>
cudaError_t apply_q1(cudaStream_t st, int n, int b, int k, const T *v1, const T *t1, T *z,
                     int ldz, T *work)
{
    cudaError_t e;
    int npan = 0;
    for (int c0 = 0; c0 + b <= n - 2; c0 += b) ++npan;
    // groups of kQ1Group panels on the tensor-core binary32 path; one panel at a time with
    // the SIMT binary64 GEMM (its split-K products lose parallelism with wide blocks)
    const int group = sizeof(T) == 4 ? kQ1Group : 1;
    const int gw_max = group * b;
    T *Tg = work;                                  // gw_max x gw_max (ld gw_max)
    T *M1 = Tg + (size_t)gw_max * gw_max;          // gw_max x b
    T *M2 = M1 + (size_t)gw_max * b;               // gw_max x b
    T *Y = M2 + (size_t)gw_max * b;                // gw_max x k
    T *Y2 = Y + (size_t)gw_max * k;                // gw_max x k
    T *part = Y2 + (size_t)gw_max * k;             // split-K partials (what is left)
    const size_t part_elems = (size_t)2 * gw_max * k;
    for (int phi = npan - 1; phi >= 0; phi -= group) {
        const int plo = phi - group + 1 < 0 ? 0 : phi - group + 1;
        const int c0 = plo * b, r0 = c0 + b, m = n - r0;
        const int gw = (phi - plo + 1) * b;
        const T *V = v1 + r0 + (size_t)c0 * n;  // m x gw
        // T of the group: start from the first panel's T, merge the others in order
        if ((e = copy_matrix<T, T>(st, b, b, t1 + (size_t)c0 * b, b, Tg, gw_max)) != cudaSuccess) return e;
        for (int p = plo + 1; p <= phi; ++p) {
            const int wa = (p - plo) * b;             // width merged so far
            const T *Vb = v1 + r0 + (size_t)(p * b) * n;
            const T *Tb = t1 + (size_t)(p * b) * b;
            // M1 = V_a^T V_b (wa x b), M2 = M1 T_b, T12 = -T_a M2
            if ((e = gemm<T>(st, 1, 0, wa, b, m, T(1), V, n, Vb, n, T(0), M1, gw_max)) != cudaSuccess) return e;
            if ((e = gemm<T>(st, 0, 0, wa, b, b, T(1), M1, gw_max, Tb, b, T(0), M2, gw_max)) != cudaSuccess) return e;
            if ((e = gemm<T>(st, 0, 0, wa, b, wa, T(-1), Tg, gw_max, M2, gw_max, T(0), Tg + (size_t)wa * gw_max,
                             gw_max)) != cudaSuccess) return e;
            // T22 = T_b, T21 = 0
            if ((e = copy_matrix<T, T>(st, b, b, Tb, b, Tg + wa + (size_t)wa * gw_max, gw_max)) != cudaSuccess) return e;
            if ((e = cudaMemset2DAsync(Tg + wa, sizeof(T) * gw_max, 0, sizeof(T) * b, wa, st)) != cudaSuccess) return e;
        }
        T *Zr = z + r0;
        if ((e = gemm_splitk<T>(st, 1, 0, gw, k, m, T(1), V, n, Zr, ldz, Y, gw, part, part_elems)) != cudaSuccess) return e;
        if ((e = gemm<T>(st, 0, 0, gw, k, gw, T(1), Tg, gw_max, Y, gw, T(0), Y2, gw)) != cudaSuccess) return e;
        if ((e = gemm<T>(st, 0, 0, m, k, gw, T(-1), V, n, Y2, gw, T(1), Zr, ldz)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t apply_q1<double>(cudaStream_t, int, int, int, const double *, const double *,
                                      double *, int, double *);
template cudaError_t apply_q1<float>(cudaStream_t, int, int, int, const float *, const float *,
                                     float *, int, float *);

}  // namespace egb
