// Occupation numbers, chemical potential, band energy (arXiv:1705.11191 sec. 4.4,
// elsi_dm_real; Eqs. 14-15 and 17-18) and the density matrices P = C diag(f) C^T
// (Eq. 7) and W = C diag(f eps) C^T.
#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace egb {

// Occupation fraction for x = (eps - mu) / kT: Gaussian and Methfessel-Paxton order 0,
// 0.5 erfc(x); Methfessel-Paxton order 1 (Phys. Rev. B 40, 3616 (1989)),
// 0.5 erfc(x) + A_1 H_1(x) exp(-x^2) = 0.5 erfc(x) - x exp(-x^2) / (2 sqrt(pi));
// Fermi-Dirac (Eq. 14) otherwise.
__device__ __forceinline__ double occ_phi(int scheme, double x)
{
    if (scheme == ELSI_OCC_GAUSSIAN || scheme == ELSI_OCC_MP0) return 0.5 * erfc(x);
    if (scheme == ELSI_OCC_MP1) return 0.5 * erfc(x) - x * exp(-x * x) * 0.28209479177387814347;
    if (x > 0.0) { double e = exp(-x); return e / (1.0 + e); }
    return 1.0 / (1.0 + exp(x));
}

// Per-state entropy summand s with -kT S_ent = kT g sum s, the term that makes the free
// energy E_band - kT S_ent stationary in the occupations at fixed electron count:
// Fermi-Dirac s = phi ln phi + (1 - phi) ln(1 - phi) (phi = f / g);
// Gaussian s = -exp(-x^2) / (2 sqrt(pi)) (x = (eps - mu) / kT); Methfessel-Paxton order 1
// s = -(1/2) A_1 H_2(x) exp(-x^2).
__device__ __forceinline__ double occ_entropy(int scheme, double phi, double x)
{
    // 0.28209... = 1 / (2 sqrt(pi))
    if (scheme == ELSI_OCC_GAUSSIAN || scheme == ELSI_OCC_MP0) return -exp(-x * x) * 0.28209479177387814347;
    // Methfessel-Paxton order 1: -(1/2) A_1 H_2(x) exp(-x^2) = (2 x^2 - 1) exp(-x^2) / (4 sqrt(pi))
    if (scheme == ELSI_OCC_MP1) return (2.0 * x * x - 1.0) * exp(-x * x) * 0.14104739588693907174;
    if (!(phi > 0.0 && phi < 1.0)) return 0.0;
    return phi * log(phi) + (1.0 - phi) * log1p(-phi);
}

// One CTA. Spin factor g = 2. scheme 0: aufbau filling; 1/2: bisection on mu with the
// exact-charge correction of sec. 4.4 when occ_accuracy is not reached.
// stride 2 ("pairs"): states 2i and 2i+1 are the two real forms of one complex state;
// occupations are computed on eps[2i] with n_el / 2 electrons and given to both, and the
// reported energy is the sum over all real states (twice the complex band energy).
__global__ void occupation_kernel(int k, const double *eps_all, double n_el_all, int scheme,
                                  double kt, double occ_accuracy, int mu_max_steps, double *f,
                                  double *out, int *status, int stride)
{
    __shared__ double red[32];
    const double g = 2.0;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int kk = k / stride;
    const double n_el = n_el_all / stride;
    auto eps = [&](int l) { return eps_all[(size_t)l * stride]; };
    if (scheme == ELSI_OCC_INTEGER) {
        double es = 0.0;
        for (int l = tid; l < kk; l += nt) {
            double fl = fmin(g, fmax(0.0, n_el - g * l));
            f[(size_t)l * stride] = fl;
            es += fl * eps(l);
        }
        es = block_sum(es, red);
        if (tid == 0) {
            int top = (int)ceil(n_el / g) - 1;
            if (top < 0) top = 0;
            if (top > kk - 1) top = kk - 1;
            out[0] = eps(top);
            out[1] = stride * es;
            out[2] = 0.0;
        }
    } else {
        auto count = [&](double mu) {
            double s2 = 0.0;
            for (int l = tid; l < kk; l += nt) s2 += g * occ_phi(scheme, (eps(l) - mu) / kt);
            return block_sum(s2, red);
        };
        double lo = eps(0), hi = eps(kk - 1);
        for (int it = 0; it < 1000 && count(lo) > n_el; ++it) lo -= 1.0;
        for (int it = 0; it < 1000 && count(hi) < n_el; ++it) hi += 1.0;
        double mu = hi;
        int converged = 0;
        for (int step = 0; step < mu_max_steps; ++step) {
            double mid = 0.5 * (lo + hi);
            double nm = count(mid);
            if (fabs(nm - n_el) <= occ_accuracy / stride) { mu = mid; converged = 1; break; }
            if (nm < n_el) lo = mid; else hi = mid;
        }
        if (!converged) mu = hi;
        for (int l = tid; l < kk; l += nt) f[(size_t)l * stride] = g * occ_phi(scheme, (eps(l) - mu) / kt);
        __syncthreads();
        if (!converged && tid == 0) {
            double surplus = -n_el;
            for (int l = 0; l < kk; ++l) surplus += f[(size_t)l * stride];
            for (int l = kk - 1; l >= 0 && surplus > 0.0; --l) {
                double fl = f[(size_t)l * stride];
                double take = fl < surplus ? fl : surplus;
                f[(size_t)l * stride] = fl - take;
                surplus -= take;
            }
        }
        __syncthreads();
        double es = 0.0, ts = 0.0;
        for (int l = tid; l < kk; l += nt) {
            es += f[(size_t)l * stride] * eps(l);
            ts += occ_entropy(scheme, f[(size_t)l * stride] / g, (eps(l) - mu) / kt);
        }
        es = block_sum(es, red);
        ts = block_sum(ts, red);
        if (tid == 0) { out[0] = mu; out[1] = stride * es; out[2] = stride * kt * g * ts; }
    }
    __syncthreads();
    if (stride > 1)
        for (int l = tid; l < kk; l += nt)
            for (int q = 1; q < stride; ++q) f[(size_t)l * stride + q] = f[(size_t)l * stride];
    (void)status;
}

cudaError_t occupation(cudaStream_t st, int k, const double *eps, double n_el, int scheme,
                       double kt, double occ_accuracy, int mu_max_steps, double *f, double *out,
                       int *status, int stride)
{
    EGB_COUNT_LAUNCH();
    occupation_kernel<<<1, 1024, 0, st>>>(k, eps, n_el, scheme, kt, occ_accuracy, mu_max_steps, f,
                                          out, status, stride);
    return cudaGetLastError();
}

__device__ __forceinline__ double block_max(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    double s = (lane < nw) ? red[lane] : -DBL_MAX;
    if (warp == 0) {
        for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
        if (lane == 0) red[0] = s;
    }
    __syncthreads();
    double r = red[0];
    __syncthreads();
    return r;
}

// One chemical potential for m weighted entries of several problems (k-points, spin
// channels; sec. 4.4 sums the electron count of the bisection over them). Entry j has
// eigenvalue eps[j] and weight wt[j]; the count is sum_j wt[j] f_j, f_j in [0, 2]. The
// entries need not be sorted: where an order is needed (aufbau filling, surplus
// removal) the level that the rule stops at is isolated by bisection on the eigenvalue
// axis until the interval holds a single distinct eigenvalue. Entries with exactly equal
// eigenvalues form one level and are treated alike. One CTA.
// out[0] = mu, out[1] = sum_j wt[j] f_j eps[j].
__global__ void occupation_weighted_kernel(int m, const double *eps, const double *wt, double n_el,
                                           int scheme, double kt, double occ_accuracy,
                                           int mu_max_steps, double *f, double *out, int *status)
{
    __shared__ double red[32];
    const double g = 2.0;
    const int tid = threadIdx.x, nt = blockDim.x;
    double mn = DBL_MAX, mx = -DBL_MAX, ws = 0.0;
    for (int j = tid; j < m; j += nt) {
        mn = fmin(mn, eps[j]);
        mx = fmax(mx, eps[j]);
        ws += wt[j];
    }
    mn = -block_max(-mn, red);
    mx = block_max(mx, red);
    ws = block_sum(ws, red);
    if (!(n_el >= 0.0) || n_el > g * ws * (1.0 + 1e-14)) {
        if (tid == 0) report_error(status, ELSI_ERR_ARG, 0);
        return;
    }
    // distinct eigenvalues in (lo, hi] (lower_open) or [lo, hi): min and max of them
    auto range_in = [&](double lo, double hi, bool lower_open, double &a, double &b) {
        double x = DBL_MAX, y = -DBL_MAX;
        for (int j = tid; j < m; j += nt) {
            const double v = eps[j];
            const bool in = lower_open ? (v > lo && v <= hi) : (v >= lo && v < hi);
            if (in) { x = fmin(x, v); y = fmax(y, v); }
        }
        a = -block_max(-x, red);
        b = block_max(y, red);
    };
    double mu;
    if (scheme == ELSI_OCC_INTEGER) {
        if (n_el <= 0.0) {
            for (int j = tid; j < m; j += nt) f[j] = 0.0;
            mu = mn;
        } else {
            // smallest level e* with N(<= e*) >= n_el; invariant N(<= lo) < n_el <= N(<= hi)
            auto n_le = [&](double x) {
                double s = 0.0;
                for (int j = tid; j < m; j += nt) s += (eps[j] <= x) ? g * wt[j] : 0.0;
                return block_sum(s, red);
            };
            double lo = mn - 1.0, hi = mx, estar = mx;
            bool found = false;
            for (int it = 0; it < 4096; ++it) {
                double a, b;
                range_in(lo, hi, true, a, b);
                if (a == b) { estar = a; found = true; break; }
                const double mid = 0.5 * (lo + hi);
                if (n_le(mid) >= n_el) hi = mid; else lo = mid;
            }
            if (!found && tid == 0) report_error(status, ELSI_ERR_NO_CONVERGENCE, 0);
            double below = 0.0, wl = 0.0;
            for (int j = tid; j < m; j += nt) {
                if (eps[j] < estar) below += g * wt[j];
                else if (eps[j] == estar) wl += wt[j];
            }
            below = block_sum(below, red);
            wl = block_sum(wl, red);
            const double fl = (wl > 0.0) ? fmin(g, fmax(0.0, (n_el - below) / wl)) : 0.0;
            for (int j = tid; j < m; j += nt)
                f[j] = (eps[j] < estar) ? g : ((eps[j] == estar) ? fl : 0.0);
            mu = estar;
        }
    } else {
        auto count = [&](double x) {
            double s = 0.0;
            for (int j = tid; j < m; j += nt) s += wt[j] * g * occ_phi(scheme, (eps[j] - x) / kt);
            return block_sum(s, red);
        };
        double lo = mn, hi = mx;
        for (int it = 0; it < 1000 && count(lo) > n_el; ++it) lo -= 1.0;
        for (int it = 0; it < 1000 && count(hi) < n_el; ++it) hi += 1.0;
        mu = hi;
        bool converged = false;
        for (int step = 0; step < mu_max_steps; ++step) {
            const double mid = 0.5 * (lo + hi);
            const double nm = count(mid);
            if (fabs(nm - n_el) <= occ_accuracy) { mu = mid; converged = true; break; }
            if (nm < n_el) lo = mid; else hi = mid;
        }
        if (!converged) mu = hi;
        for (int j = tid; j < m; j += nt) f[j] = g * occ_phi(scheme, (eps[j] - mu) / kt);
        __syncthreads();
        if (!converged) {
            double sur = 0.0;
            for (int j = tid; j < m; j += nt) sur += wt[j] * f[j];
            const double surplus = block_sum(sur, red) - n_el;
            if (surplus > 0.0) {
                // highest level x* with S(>= x*) >= surplus, S(>= x) = sum_{eps >= x} wt f
                auto s_ge = [&](double x) {
                    double s = 0.0;
                    for (int j = tid; j < m; j += nt) s += (eps[j] >= x) ? wt[j] * f[j] : 0.0;
                    return block_sum(s, red);
                };
                double lo2 = mn, hi2 = fmax(mx + 1.0, mx * (1.0 + 1e-15) + 1.0), xs = mn;
                bool found = false;
                for (int it = 0; it < 4096; ++it) {
                    double a, b;
                    range_in(lo2, hi2, false, a, b);
                    if (a == b) { xs = a; found = true; break; }
                    const double mid = 0.5 * (lo2 + hi2);
                    if (s_ge(mid) >= surplus) lo2 = mid; else hi2 = mid;
                }
                if (!found && tid == 0) report_error(status, ELSI_ERR_NO_CONVERGENCE, 1);
                double gt = 0.0, gl = 0.0;
                for (int j = tid; j < m; j += nt) {
                    if (eps[j] > xs) gt += wt[j] * f[j];
                    else if (eps[j] == xs) gl += wt[j] * f[j];
                }
                gt = block_sum(gt, red);
                gl = block_sum(gl, red);
                const double keep = (gl > 0.0) ? 1.0 - (surplus - gt) / gl : 0.0;
                for (int j = tid; j < m; j += nt) {
                    if (eps[j] > xs) f[j] = 0.0;
                    else if (eps[j] == xs) f[j] *= keep;
                }
            }
        }
    }
    __syncthreads();
    double es = 0.0, ts = 0.0;
    for (int j = tid; j < m; j += nt) {
        es += wt[j] * f[j] * eps[j];
        if (scheme != ELSI_OCC_INTEGER) ts += wt[j] * occ_entropy(scheme, f[j] / g, (eps[j] - mu) / kt);
    }
    es = block_sum(es, red);
    ts = block_sum(ts, red);
    if (tid == 0) { out[0] = mu; out[1] = es; out[2] = kt * g * ts; }
}

cudaError_t occupation_weighted(cudaStream_t st, int m, const double *eps, const double *wt,
                                double n_el, int scheme, double kt, double occ_accuracy,
                                int mu_max_steps, double *f, double *out, int *status)
{
    EGB_COUNT_LAUNCH();
    occupation_weighted_kernel<<<1, 1024, 0, st>>>(m, eps, wt, n_el, scheme, kt, occ_accuracy,
                                                   mu_max_steps, f, out, status);
    return cudaGetLastError();
}

// Band energy of each problem of a batch: out[i] = sum over its entries of f * eps
// (entries off[i] .. off[i+1]-1). One CTA per problem.
__global__ void segment_energy_kernel(const int *off, const double *f, const double *eps, double *out)
{
    __shared__ double red[32];
    const int i = blockIdx.x;
    double s = 0.0;
    for (int j = off[i] + threadIdx.x; j < off[i + 1]; j += blockDim.x) s += f[j] * eps[j];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[i] = s;
}

cudaError_t segment_energy(cudaStream_t st, int nseg, const int *off, const double *f,
                           const double *eps, double *out)
{
    EGB_COUNT_LAUNCH();
    segment_energy_kernel<<<nseg, 256, 0, st>>>(off, f, eps, out);
    return cudaGetLastError();
}

template <typename T>
__global__ void scale_columns_kernel(int n, int k, const T *c, int ldc, const double *f,
                                     const double *eps, T *out)
{
    size_t total = (size_t)n * k;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), l = (int)(e / n);
        double s = f[l] * (eps ? eps[l] : 1.0);
        out[e] = (T)(s * (double)c[(size_t)i + (size_t)l * ldc]);
    }
}

template <typename T>
cudaError_t density_pw(cudaStream_t st, int n, int k, const T *c, int ldc, const double *f,
                       const double *eps, T *p, T *w, T *cw)
{
    cudaError_t e;
    size_t total = (size_t)n * k;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    if (p) {
        EGB_COUNT_LAUNCH();
        scale_columns_kernel<T><<<grid, 256, 0, st>>>(n, k, c, ldc, f, nullptr, cw);
        if ((e = gemm<T>(st, 0, 1, n, n, k, T(1), cw, n, c, ldc, T(0), p, n, 1)) != cudaSuccess) return e;
        if ((e = mirror_lower<T>(st, n, p, n)) != cudaSuccess) return e;
    }
    if (w) {
        EGB_COUNT_LAUNCH();
        scale_columns_kernel<T><<<grid, 256, 0, st>>>(n, k, c, ldc, f, eps, cw);
        if ((e = gemm<T>(st, 0, 1, n, n, k, T(1), cw, n, c, ldc, T(0), w, n, 1)) != cudaSuccess) return e;
        if ((e = mirror_lower<T>(st, n, w, n)) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}
template cudaError_t density_pw<double>(cudaStream_t, int, int, const double *, int, const double *,
                                        const double *, double *, double *, double *);
template cudaError_t density_pw<float>(cudaStream_t, int, int, const float *, int, const double *,
                                       const double *, float *, float *, float *);

}  // namespace egb
