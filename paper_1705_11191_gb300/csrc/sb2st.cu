// Band -> tridiagonal reduction T = Q2^T B Q2 by bulge chasing (arXiv:1705.11191 Eq. 11,
// second line; step (2) of the two-stage tridiagonalisation, sec. 3.1, after Bischof,
// Lang & Sun's successive band reduction), and the back-transformation of eigenvectors
// through Q2 (step (4)).
//
// Sweep j (0 <= j <= n-3) annihilates column j below the subdiagonal and chases the
// resulting bulge down the band in steps t = 0, 1, ...; step t owns the index window
// [j+1+(t-1)b, j+(t+1)b]. Step (j, t) of sweep j and step (j+1, t-3) of sweep j+1 touch
// disjoint windows, and every step of sweep j+1 only needs steps of sweep j that end at
// least one window earlier, so all steps with the same "time" 3j+t are independent:
// a persistent cooperative kernel walks the time axis with one grid barrier per time
// step, each CTA running one (sweep, step) task out of shared memory.
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

// D (L x L, symmetric, ld ldd) <- H D H, H = I - tau v v^T. p: scratch of length L.
template <typename T>
__device__ void two_sided(int L, T *D, int ldd, const T *v, T tau, T *p, T *red)
{
    if (tau == T(0)) return;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        T s = T(0);
        for (int c = 0; c < L; ++c) s = fma(D[i + c * ldd], v[c], s);
        p[i] = tau * s;
    }
    __syncthreads();
    T part = T(0);
    for (int i = threadIdx.x; i < L; i += blockDim.x) part = fma(p[i], v[i], part);
    T K = T(0.5) * tau * block_sum(part, red);
    for (int i = threadIdx.x; i < L; i += blockDim.x) p[i] -= K * v[i];  // q
    __syncthreads();
    for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
        int i = e % L, c = e / L;
        D[i + c * ldd] = D[i + c * ldd] - v[i] * p[c] - p[i] * v[c];
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T band_get(const T *band, int ldb, int r, int c)
{
    return (r >= c) ? band[(size_t)(r - c) + (size_t)c * ldb] : band[(size_t)(c - r) + (size_t)r * ldb];
}

// One (sweep j, step t) task; all threads of the CTA take part.
template <typename T>
__device__ void chase_task(const ChaseArgs &a, T *band, T *v2, T *tau2, int j, int t, T *smem,
                           T *red)
{
    const int n = a.n, b = a.b, ldb = a.ldb;
    T *X = smem;                 // b x b (ld b)
    T *D = X + b * b;            // b x b (ld b)
    T *vnew = D + b * b;         // b
    T *vprev = vnew + b;         // b
    T *p = vprev + b;            // b
    const int tid = threadIdx.x, nt = blockDim.x;
    size_t slot = (size_t)j * a.S + t;

    if (t == 0) {
        const int L = min(b, n - 1 - j);
        for (int i = tid; i < b; i += nt) vnew[i] = (i < L) ? band[(size_t)(1 + i) + (size_t)j * ldb] : T(0);
        __syncthreads();
        T beta;
        T tau = house_smem<T>(L, vnew, red, &beta);
        for (int i = tid; i < L; i += nt)
            band[(size_t)(1 + i) + (size_t)j * ldb] = (i == 0) ? beta : T(0);
        // D = A[j+1 .. j+L]^2
        const int r0 = j + 1;
        for (int e = tid; e < L * L; e += nt) {
            int i = e % L, c = e / L;
            D[i + c * b] = band_get(band, ldb, r0 + i, r0 + c);
        }
        __syncthreads();
        two_sided<T>(L, D, b, vnew, tau, p, red);
        for (int e = tid; e < L * L; e += nt) {
            int i = e % L, c = e / L;
            if (i >= c) band[(size_t)(i - c) + (size_t)(r0 + c) * ldb] = D[i + c * b];
        }
        for (int i = tid; i < b; i += nt) v2[slot * b + i] = (i < L) ? vnew[i] : T(0);
        if (tid == 0) tau2[slot] = tau;
        __syncthreads();
        return;
    }
    const int r = j + 1 + t * b;
    const int L = min(b, n - r);
    const int cb = r - b;  // first column of X
    size_t pslot = slot - 1;
    for (int i = tid; i < b; i += nt) vprev[i] = v2[pslot * b + i];
    const T taup = tau2[pslot];
    // X = A[r .. r+L-1, cb .. cb+b-1]  (all strictly below the diagonal, distance 1..2b-1)
    for (int e = tid; e < L * b; e += nt) {
        int i = e % L, c = e / L;
        X[i + c * b] = band[(size_t)(r + i - (cb + c)) + (size_t)(cb + c) * ldb];
    }
    __syncthreads();
    // X <- X H_prev : y = X v, X -= tau y v^T
    if (taup != T(0)) {
        for (int i = tid; i < L; i += nt) {
            T s = T(0);
            for (int c = 0; c < b; ++c) s = fma(X[i + c * b], vprev[c], s);
            p[i] = taup * s;
        }
        __syncthreads();
        for (int e = tid; e < L * b; e += nt) {
            int i = e % L, c = e / L;
            X[i + c * b] = fma(-p[i], vprev[c], X[i + c * b]);
        }
        __syncthreads();
    }
    // new reflector from X[:, 0]
    for (int i = tid; i < b; i += nt) vnew[i] = (i < L) ? X[i] : T(0);
    __syncthreads();
    T beta;
    T tau = house_smem<T>(L, vnew, red, &beta);
    // left-apply to X[:, 1:]
    if (tau != T(0)) {
        for (int c = 1 + tid; c < b; c += nt) {
            T s = T(0);
            for (int i = 0; i < L; ++i) s = fma(vnew[i], X[i + c * b], s);
            p[c] = tau * s;
        }
        __syncthreads();
        for (int e = tid; e < L * (b - 1); e += nt) {
            int i = e % L, c = 1 + e / L;
            X[i + c * b] = fma(-vnew[i], p[c], X[i + c * b]);
        }
        __syncthreads();
    }
    if (tid == 0) X[0] = beta;
    for (int i = 1 + tid; i < L; i += nt) X[i] = T(0);
    __syncthreads();
    for (int e = tid; e < L * b; e += nt) {
        int i = e % L, c = e / L;
        band[(size_t)(r + i - (cb + c)) + (size_t)(cb + c) * ldb] = X[i + c * b];
    }
    // diagonal block
    for (int e = tid; e < L * L; e += nt) {
        int i = e % L, c = e / L;
        D[i + c * b] = band_get(band, ldb, r + i, r + c);
    }
    __syncthreads();
    two_sided<T>(L, D, b, vnew, tau, p, red);
    for (int e = tid; e < L * L; e += nt) {
        int i = e % L, c = e / L;
        if (i >= c) band[(size_t)(i - c) + (size_t)(r + c) * ldb] = D[i + c * b];
    }
    for (int i = tid; i < b; i += nt) v2[slot * b + i] = (i < L) ? vnew[i] : T(0);
    if (tid == 0) tau2[slot] = tau;
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) chase_kernel(T *band, T *v2, T *tau2, ChaseArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    __shared__ T red[32];
    const int n = a.n, b = a.b;
    const int nsweep = n - 2;  // sweeps j = 0 .. n-3
    for (long long time = 0; time <= a.tmax; ++time) {
        int jhi = (int)min((long long)(nsweep - 1), time / 3);
        long long lo = (time - (a.S - 1) + 2) / 3;  // ceil((time - (S-1)) / 3)
        int jlo = (int)max(0ll, lo);
        for (int j = jlo + blockIdx.x; j <= jhi; j += gridDim.x) {
            int t = (int)(time - 3ll * j);
            int Sj = (n - 2 - j) / b + 1;
            if (t < 0 || t >= Sj) continue;
            chase_task<T>(a, band, v2, tau2, j, t, smem, red);
        }
        if (!grid_barrier(a.count, a.gen, gridDim.x, a.status)) return;
    }
    // volatile reads of the band happen in the next kernel (d, e extraction)
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
        size_t smem = (2 * (size_t)b * b + 3 * b) * sizeof(T);
        static bool attr_set[2] = {false, false};
        int ai = sizeof(T) == 8 ? 0 : 1;
        if (!attr_set[ai]) {
            // opt in once for the largest band width (64)
            const size_t smax = (2 * 64 * 64 + 3 * 64) * sizeof(T);
            if ((err = cudaFuncSetAttribute(chase_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smax)) != cudaSuccess)
                return err;
            attr_set[ai] = true;
        }
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chase_kernel<T>, 256, smem);
        int maxpar = (n - 2 + 2) / 3 + 1;  // upper bound of concurrently active sweeps
        int conc = S / 3 + 2;
        if (conc < maxpar) maxpar = conc;
        int G = per_sm * num_sms;
        if (G > maxpar) G = maxpar;
        if (G < 1) G = 1;
        if ((err = cudaMemsetAsync(sync, 0, 2 * sizeof(unsigned), st)) != cudaSuccess) return err;
        void *args[] = {&band, &v2, &tau2, &a};
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
// ascending and, inside W(J,t), sweeps descending. Each warp owns a pair of columns of
// Z and keeps the rows of the current window in a shared-memory ring; the reflectors of
// one (J, t) are staged once per CTA.
constexpr int kQ2Cols = 16;     // columns per CTA (2 per warp, 8 warps)
constexpr int kQ2Sweeps = 64;   // m: sweeps per block
constexpr int kQ2Ring = 256;    // ring rows (>= m + 2b - 1 for b <= 64)
constexpr int kQ2RingLd = kQ2Ring + 16;  // per-column stride: the two columns of a warp use
                                         // disjoint shared-memory banks

template <typename T>
__global__ void __launch_bounds__(256) apply_q2_kernel(int n, int b, int S, const T *__restrict__ v2,
                                                        const T *__restrict__ tau2, int k, T *z,
                                                        int ldz)
{
    extern __shared__ unsigned char smem_raw[];
    T *ring = reinterpret_cast<T *>(smem_raw);          // kQ2Cols x kQ2RingLd, [col][slot]
    T *vs = ring + kQ2RingLd * kQ2Cols;                 // m x b staged reflectors
    T *ts = vs + kQ2Sweeps * b;                         // m taus
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col0 = blockIdx.x * kQ2Cols;
    const int lc = warp * 2 + (lane >> 4);              // local column of this lane
    const int gc = col0 + lc;
    const int sub = lane & 15;                          // row lane within the column
    const bool col_ok = gc < k;
    const int nsweep = n - 2;
    const int nblk = (nsweep + kQ2Sweeps - 1) / kQ2Sweeps;

    for (int jb = nblk - 1; jb >= 0; --jb) {
        const int J = jb * kQ2Sweeps;
        const int Jend = min(nsweep, J + kQ2Sweeps);  // sweeps J .. Jend-1
        const int SJ = (n - 2 - J) / b + 1;
        int lo = J + 1;                                // window [lo, hi)
        int hi = min(n, Jend + b);                     // rows of step 0: up to (Jend-1)+1+b-1
        // initial load
        for (int r = lo + sub; r < hi; r += 16)
            ring[lc * kQ2RingLd + (r % kQ2Ring)] = col_ok ? z[(size_t)r + (size_t)gc * ldz] : T(0);
        for (int t = 0; t < SJ; ++t) {
            // stage reflectors (j, t) for j in [J, Jend)
            __syncthreads();
            for (int e = threadIdx.x; e < (Jend - J) * b; e += blockDim.x) {
                int jj = e / b, i = e % b;
                int j = J + jj;
                int Sj = (n - 2 - j) / b + 1;
                vs[jj * b + i] = (t < Sj) ? v2[((size_t)j * S + t) * b + i] : T(0);
            }
            for (int jj = threadIdx.x; jj < Jend - J; jj += blockDim.x) {
                int j = J + jj;
                int Sj = (n - 2 - j) / b + 1;
                ts[jj] = (t < Sj) ? tau2[(size_t)j * S + t] : T(0);
            }
            __syncthreads();
            for (int j = Jend - 1; j >= J; --j) {
                const int jj = j - J;
                const T tau = ts[jj];
                if (tau == T(0)) continue;
                const int r0 = j + 1 + t * b;
                const int L = min(b, n - r0);
                if (L <= 0) continue;
                T s = T(0);
                for (int i = sub; i < L; i += 16)
                    s = fma(vs[jj * b + i], ring[lc * kQ2RingLd + ((r0 + i) % kQ2Ring)], s);
                for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                s *= tau;
                for (int i = sub; i < L; i += 16) {
                    T &zr = ring[lc * kQ2RingLd + ((r0 + i) % kQ2Ring)];
                    zr = fma(-s, vs[jj * b + i], zr);
                }
                __syncwarp();
            }
            // slide the window by b rows: store [lo, lo+b), load [hi, hi+b)
            int nlo = min(lo + b, n), nhi = min(hi + b, n);
            __syncwarp();
            for (int r = lo + sub; r < nlo; r += 16)
                if (col_ok) z[(size_t)r + (size_t)gc * ldz] = ring[lc * kQ2RingLd + (r % kQ2Ring)];
            __syncwarp();
            for (int r = hi + sub; r < nhi; r += 16)
                ring[lc * kQ2RingLd + (r % kQ2Ring)] = col_ok ? z[(size_t)r + (size_t)gc * ldz] : T(0);
            __syncwarp();
            lo = nlo;
            hi = nhi;
        }
        for (int r = lo + sub; r < hi; r += 16)
            if (col_ok) z[(size_t)r + (size_t)gc * ldz] = ring[lc * kQ2RingLd + (r % kQ2Ring)];
        __syncwarp();
    }
}

template <typename T>
cudaError_t apply_q2(cudaStream_t st, int n, int b, const T *v2, const T *tau2, int k, T *z,
                     int ldz, int *status)
{
    (void)status;
    if (n < 3 || k <= 0) return cudaSuccess;
    if (b > 64 || kQ2Sweeps + 2 * b - 1 > kQ2Ring) return cudaErrorInvalidValue;
    const int S = sb2st_steps(n, b);
    size_t smem = ((size_t)kQ2RingLd * kQ2Cols + (size_t)kQ2Sweeps * b + kQ2Sweeps) * sizeof(T);
    static bool attr_set[2] = {false, false};
    int ai = sizeof(T) == 8 ? 0 : 1;
    if (!attr_set[ai]) {
        const size_t smax = ((size_t)kQ2RingLd * kQ2Cols + (size_t)kQ2Sweeps * 64 + kQ2Sweeps) * sizeof(T);
        cudaError_t e = cudaFuncSetAttribute(apply_q2_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smax);
        if (e != cudaSuccess) return e;
        attr_set[ai] = true;
    }
    EGB_COUNT_LAUNCH();
    apply_q2_kernel<T><<<ceil_div(k, kQ2Cols), 256, smem, st>>>(n, b, S, v2, tau2, k, z, ldz);
    return cudaGetLastError();
}
template cudaError_t apply_q2<double>(cudaStream_t, int, int, const double *, const double *, int,
                                      double *, int, int *);
template cudaError_t apply_q2<float>(cudaStream_t, int, int, const float *, const float *, int,
                                     float *, int, int *);

// ------------------------------------------------------------------ Q1 back-transform
// Z <- Q1 Z, Q1 = Q_0 Q_1 ... Q_{P-1}, Q_p = I - V_p T_p V_p^T: panels descending.
template <typename T>
cudaError_t apply_q1(cudaStream_t st, int n, int b, int k, const T *v1, const T *t1, T *z,
                     int ldz, T *work)
{
    cudaError_t e;
    int npan = 0;
    for (int c0 = 0; c0 + b <= n - 2; c0 += b) ++npan;
    for (int p = npan - 1; p >= 0; --p) {
        const int c0 = p * b, r0 = c0 + b, m = n - r0;
        const T *V = v1 + r0 + (size_t)c0 * n;
        const T *Tm = t1 + (size_t)c0 * b;
        T *Y = work;                    // b x k
        T *Y2 = work + (size_t)b * k;   // b x k
        T *Zr = z + r0;
        if ((e = gemm_splitk<T>(st, 1, 0, b, k, m, T(1), V, n, Zr, ldz, Y, b, Y2 + (size_t)b * k,
                                (size_t)16 * b * k)) != cudaSuccess) return e;
        if ((e = gemm<T>(st, 0, 0, b, k, b, T(1), Tm, b, Y, b, T(0), Y2, b)) != cudaSuccess) return e;
        if ((e = gemm<T>(st, 0, 0, m, k, b, T(-1), V, n, Y2, b, T(1), Zr, ldz)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}
template cudaError_t apply_q1<double>(cudaStream_t, int, int, int, const double *, const double *,
                                      double *, int, double *);
template cudaError_t apply_q1<float>(cudaStream_t, int, int, int, const float *, const float *,
                                     float *, int, float *);

}  // namespace egb
