// Occupation numbers, chemical potential, band energy (arXiv:1705.11191 sec. 4.4,
// elsi_dm_real; Eqs. 14-15 and 17-18) and the density matrices P = C diag(f) C^T
// (Eq. 7) and W = C diag(f eps) C^T.
#include "common.cuh"
#include "kernels.h"

namespace egb {

__device__ __forceinline__ double occ_phi(int scheme, double x)
{
    if (scheme == ELSI_OCC_GAUSSIAN) return 0.5 * (1.0 - erf(x));
    if (x > 0.0) { double e = exp(-x); return e / (1.0 + e); }
    return 1.0 / (1.0 + exp(x));
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
        double es = 0.0;
        for (int l = tid; l < kk; l += nt) es += f[(size_t)l * stride] * eps(l);
        es = block_sum(es, red);
        if (tid == 0) { out[0] = mu; out[1] = stride * es; }
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
