// Symmetric tridiagonal eigensolver (step (3) of the two-stage method, arXiv:1705.11191
// sec. 3.1), restricted to the wanted eigenpairs as the paper describes for KS-DFT.
//
//  * eigenvalues: Sturm-sequence bisection (Givens 1954; Barth, Martin & Wilkinson
//    1967), a few threads per wanted eigenvalue index (multisection);
//  * eigenvectors: one twisted factorisation T - lambda I = N_r D_r N_r^T per
//    eigenvalue (Parlett & Dhillon 1997/2000), which gives the vector with residual
//    O(eps ||T||) in O(n) work; one thread per vector;
//  * vectors of eigenvalues closer than 1e-5 ||T|| are re-orthogonalised (two passes of
//    Gram-Schmidt within the cluster, as in inverse-iteration codes), which bounds the
//    loss of orthogonality between close vectors by about eps*1e5. A cluster is worked
//    on in pieces of 64 consecutive vectors and then in the 64-vector seams across piece
//    boundaries, so that a long chain of close eigenvalues (an ill-conditioned overlap
//    puts one huge eigenvalue into ||T|| and with it every gap of the rest of the
//    spectrum below the threshold) costs O(64 n) per vector instead of O(cluster n):
//    vectors more than 32 places apart are left as the twisted factorisation gives them,
//    orthogonal to about eps ||T|| / (32 times the eigenvalue spacing).
// All of this runs in binary64 regardless of the precision of the reduction.
#include <float.h>

#include "common.cuh"
#include "kernels.h"

namespace egb {

__device__ __forceinline__ double guard_pivot(double q, double pivmin)
{
    return (fabs(q) < pivmin) ? -pivmin : q;
}

// number of eigenvalues < sigma: the sign changes of the leading principal minors
// p_i = det(T[0:i, 0:i] - sigma I), p_0 = 1, p_{i+1} = (d_i - sigma) p_i - e_{i-1}^2 p_{i-1}
// (Sturm; Givens 1954). The ratio q_i = p_{i+1} / p_i is the pivot of the LDL^T
// factorisation of T - sigma I, and a pivot smaller than pivmin in magnitude is replaced
// by -pivmin as in the pivot form. This form needs no division (binary64 division is a long
// sequence of the few binary64 FMA units of this chip); the pair (p_i, p_{i-1}) is rescaled
// by an exact power of two whenever |p_i| leaves [2^-600, 2^600] (checked every 8 steps;
// one step changes |p| by at most a factor of about 2 ||T|| / pivmin, far below 2^50).
__device__ int sturm_count(int n, const double *__restrict__ d, const double *__restrict__ e,
                           double sigma, double pivmin)
{
    double pm = 1.0;                                // p_{i-1}
    double p = guard_pivot(d[0] - sigma, pivmin);   // p_1 = q_0
    int cnt = p < 0.0;
    int i = 1;
    while (i < n) {
        const int iend = min(n, i + 8);
        for (; i < iend; ++i) {
            const double ei = e[i - 1];
            double pn = fma(d[i] - sigma, p, -(ei * ei) * pm);
            // pivot q = pn / p below pivmin in magnitude: q = -pivmin
            if (fabs(pn) < pivmin * fabs(p)) pn = -pivmin * p;
            cnt += (pn < 0.0) != (p < 0.0);
            pm = p;
            p = pn;
        }
        const double ap = fabs(p);
        if (ap > 0x1p600) { p *= 0x1p-600; pm *= 0x1p-600; }
        else if (ap < 0x1p-600) { p *= 0x1p600; pm *= 0x1p600; }
    }
    return cnt;
}

// [0]=gl, [1]=gu, [2]=pivmin, [3]=||T|| bound, [4]=1 if T splits into blocks, else 0
__global__ void gershgorin_kernel(int n, const double *d, const double *e, double *out)
{
    __shared__ double red[32];
    double lo = DBL_MAX, hi = -DBL_MAX, e2max = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double r = 0.0;
        if (i > 0) r += fabs(e[i - 1]);
        if (i + 1 < n) { r += fabs(e[i]); e2max = fmax(e2max, e[i] * e[i]); }
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        e2max = fmax(e2max, __shfl_xor_sync(0xffffffffu, e2max, o));
    }
    __shared__ double slo[32], shi[32], se[32];
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { slo[w] = lo; shi[w] = hi; se[w] = e2max; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            lo = fmin(lo, slo[q]); hi = fmax(hi, shi[q]); e2max = fmax(e2max, se[q]);
        }
        double tn = fmax(fabs(lo), fabs(hi));
        double pad = 2.0 * DBL_EPSILON * tn * n + DBL_MIN;
        out[0] = lo - pad;
        out[1] = hi + pad;
        out[2] = DBL_MIN * fmax(1.0, e2max);
        out[3] = tn;
        red[0] = tn;
    }
    __syncthreads();
    // [4] = 1 if T splits (an off-diagonal at or below the threshold of split_kernel)
    const double thr = 2.0 * DBL_EPSILON * red[0];
    int split = 0;
    for (int i = threadIdx.x; i < n - 1; i += blockDim.x) split |= (fabs(e[i]) <= thr) ? 1 : 0;
    split = __syncthreads_or(split);
    if (threadIdx.x == 0) out[4] = split ? 1.0 : 0.0;
}

// number of eigenvalues < sigma, binary32 (used only to bracket)
__device__ int sturm_count32(int n, const double *__restrict__ d, const double *__restrict__ e,
                             float sigma, float pivmin)
{
    float q = (float)d[0] - sigma;
    if (fabsf(q) < pivmin) q = -pivmin;
    int cnt = q < 0.0f;
    for (int i = 1; i < n; ++i) {
        float ei = (float)e[i - 1];
        q = (float)d[i] - sigma - __fdividef(ei * ei, q);
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += q < 0.0f;
    }
    return cnt;
}

// Bisection for eigenvalue index idx = blockIdx.x * (blockDim.x / LANES) + group, with
// LANES threads per eigenvalue evaluating LANES interior points of the current interval
// (multisection: the interval shrinks by LANES + 1 per step).
// Phase 1 (bracket32 != 0): binary32 counts down to a width of 1e-6 ||T|| (a binary32
// Sturm count is exact for a matrix within a few binary32 roundings of T, so its
// eigenvalues move by far less), then the bracket is widened by 2e-6 ||T|| and checked
// with binary64 counts (falling back to the Gershgorin interval if the check fails). Phase 2: binary64 counts down to
// max(tol_rel * ||T||, 2 eps max|lo|,|hi|).
template <int LANES>
__global__ void bisect_kernel(int n, const double *d, const double *e, int count,
                              const double *bounds, double *w, double tol_rel, int bracket32)
{
    const int group = threadIdx.x / LANES, lane = threadIdx.x % LANES;
    const int idx = blockIdx.x * (blockDim.x / LANES) + group;
    const unsigned gmask = (LANES == 32) ? 0xffffffffu
                                         : (((1u << LANES) - 1u) << ((threadIdx.x & 31) / LANES * LANES));
    const bool active = idx < count;
    const double gl = bounds[0], gu = bounds[1], pivmin = bounds[2], tn = bounds[3];
    double lo = gl, hi = gu;
    if (bracket32 && active) {
        float flo = (float)gl, fhi = (float)gu;
        const float fpiv = fmaxf(1e-30f, (float)pivmin);
        for (int it = 0; it < 64 && (double)(fhi - flo) > 1e-6 * tn; ++it) {
            float sig = flo + (fhi - flo) * (float)(lane + 1) / (float)(LANES + 1);
            int c = sturm_count32(n, d, e, sig, fpiv);
            unsigned ok = __ballot_sync(gmask, c <= idx) & gmask;
            int pcount = __popc(ok);
            float nlo = __shfl_sync(gmask, sig, (threadIdx.x & 31) / LANES * LANES + max(pcount - 1, 0));
            float nhi = __shfl_sync(gmask, sig, (threadIdx.x & 31) / LANES * LANES + min(pcount, LANES - 1));
            if (pcount > 0) flo = nlo;
            if (pcount < LANES) fhi = nhi;
        }
        lo = (double)flo - 2e-6 * tn;
        hi = (double)fhi + 2e-6 * tn;
        if (lo < gl) lo = gl;
        if (hi > gu) hi = gu;
        // verify the bracket in binary64: count(lo) <= idx < count(hi)
        int c = sturm_count(n, d, e, lane == 0 ? lo : hi, pivmin);
        int clo = __shfl_sync(gmask, c, (threadIdx.x & 31) / LANES * LANES);
        int chi = (LANES > 1) ? __shfl_sync(gmask, c, (threadIdx.x & 31) / LANES * LANES + 1)
                              : sturm_count(n, d, e, hi, pivmin);
        if (!(clo <= idx && idx < chi)) { lo = gl; hi = gu; }
    }
    if (active) {
        for (int it = 0; it < 128; ++it) {
            // tol_rel relative to ||T||, but not looser than 10 tol_rel |lambda| (a single
            // huge eigenvalue of an ill-conditioned overlap must not loosen all others)
            const double scale = fmin(tn, 10.0 * fmax(1.0, fmax(fabs(lo), fabs(hi))));
            double tol = fmax(tol_rel * scale, 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi))) + 4.0 * pivmin;
            if (hi - lo <= tol) break;
            double sig = lo + (hi - lo) * (double)(lane + 1) / (double)(LANES + 1);
            int c = sturm_count(n, d, e, sig, pivmin);
            unsigned ok = __ballot_sync(gmask, c <= idx) & gmask;
            int pcount = __popc(ok);
            double nlo = __shfl_sync(gmask, sig, (threadIdx.x & 31) / LANES * LANES + max(pcount - 1, 0));
            double nhi = __shfl_sync(gmask, sig, (threadIdx.x & 31) / LANES * LANES + min(pcount, LANES - 1));
            if (pcount > 0) lo = nlo;
            if (pcount < LANES) hi = nhi;
        }
        if (lane == 0) w[idx] = 0.5 * (lo + hi);
    }
}

// Off-diagonals below 2 eps ||T|| are set to zero: T splits into unreduced blocks, which
// changes no eigenvalue by more than 2 eps ||T|| and lets exactly degenerate eigenvalues
// (e.g. those of a complex Hermitian matrix written as a real one) be found in
// different blocks.
__global__ void split_kernel(int n, double *e, const double *bounds)
{
    const double tn = bounds[3];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n - 1; i += gridDim.x * blockDim.x)
        if (fabs(e[i]) <= 2.0 * DBL_EPSILON * tn) e[i] = 0.0;
}

cudaError_t stebz(cudaStream_t st, int n, const double *d, double *e, int count,
                  double *w, int *status, double tol_rel)
{
    (void)status;
    if (n <= 0 || count <= 0) return cudaSuccess;
    // the Gershgorin bounds live right after the count eigenvalues (w has count + 8)
    double *bounds = w + count;
    EGB_COUNT_LAUNCH();
    gershgorin_kernel<<<1, 1024, 0, st>>>(n, d, e, bounds);
    EGB_COUNT_LAUNCH();
    split_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, e, bounds);
    // enough threads to cover the latency: multisection when there are few eigenvalues
    if (count <= 4096) {
        EGB_COUNT_LAUNCH();
        bisect_kernel<8><<<ceil_div(count, 16), 128, 0, st>>>(n, d, e, count, bounds, w, tol_rel, n > 512);
    } else {
        EGB_COUNT_LAUNCH();
        bisect_kernel<2><<<ceil_div(count, 64), 128, 0, st>>>(n, d, e, count, bounds, w, tol_rel, 1);
    }
    return cudaGetLastError();
}

// Block of each eigenvalue: with [lo, hi] a small interval around w[l], the eigenvalues of
// T in it are numbered by block order; w[l] is the (l - count(lo))-th of them. blk[2l],
// blk[2l+1] = [start, end) of its block.
__global__ void block_assign_kernel(int n, const double *d, const double *e, int kvec,
                                    const double *w, const double *bounds, int *blk)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= kvec) return;
    if (bounds[4] == 0.0) {  // T is one block
        blk[2 * l] = 0;
        blk[2 * l + 1] = n;
        return;
    }
    const double tn = bounds[3], pivmin = bounds[2];
    const double delta = 8.0 * DBL_EPSILON * fmax(fabs(w[l]), tn) + 4.0 * pivmin;
    const double lo = w[l] - delta, hi = w[l] + delta;
    const int clo = sturm_count(n, d, e, lo, pivmin);
    int r = l - clo;  // rank among the eigenvalues in [lo, hi]
    if (r < 0) r = 0;
    double qlo = 1.0, qhi = 1.0;
    int cl = 0, ch = 0, start = 0;
    int bs = 0, be = n;
    for (int i = 0; i < n; ++i) {
        const double ei2 = (i > 0) ? e[i - 1] * e[i - 1] : 0.0;
        if (i == 0 || e[i - 1] == 0.0) {
            qlo = d[i] - lo;
            qhi = d[i] - hi;
        } else {
            qlo = d[i] - lo - ei2 / qlo;
            qhi = d[i] - hi - ei2 / qhi;
        }
        if (fabs(qlo) < pivmin) qlo = -pivmin;
        if (fabs(qhi) < pivmin) qhi = -pivmin;
        cl += qlo < 0.0;
        ch += qhi < 0.0;
        const bool block_end = (i == n - 1) || (e[i] == 0.0);
        if (block_end) {
            if (ch - cl > r) { bs = start; be = i + 1; break; }
            start = i + 1;
        }
    }
    blk[2 * l] = bs;
    blk[2 * l + 1] = be;
}

// One twisted factorisation of T_b - lam I on the block [bs, be): the pivots D+ (dplus)
// and ratios L+ = e / D+ (lplus) of the forward factorisation, the ratios U- (uminus) of
// the backward one, the twist index r = argmin |gamma_i| with gamma_r (signed), and
// ||z||^2 of the vector z with z_r = 1 that solves (T_b - lam I) z = gamma_r e_r.
// Arrays are indexed [i * kvec + l].
struct Twist {
    int r;
    double gamma, nrm2;
};

__device__ Twist twisted_factor(const double *__restrict__ d, const double *__restrict__ e,
                                int bs, int be, double lam, double pivmin, int kvec, int l,
                                double *dplus, double *lplus, double *uminus)
{
    double dp = guard_pivot(d[bs] - lam, pivmin);
    dplus[(size_t)bs * kvec + l] = dp;
    for (int i = bs; i < be - 1; ++i) {
        const double lp = e[i] / dp;
        lplus[(size_t)i * kvec + l] = lp;
        dp = guard_pivot(d[i + 1] - lam - lp * e[i], pivmin);
        dplus[(size_t)(i + 1) * kvec + l] = dp;
    }
    double dm = guard_pivot(d[be - 1] - lam, pivmin);
    Twist t;
    t.gamma = dplus[(size_t)(be - 1) * kvec + l] + dm - (d[be - 1] - lam);
    t.r = be - 1;
    double best = fabs(t.gamma);
    for (int i = be - 2; i >= bs; --i) {
        const double um = e[i] / dm;
        uminus[(size_t)i * kvec + l] = um;
        dm = guard_pivot(d[i] - lam - um * e[i], pivmin);
        const double g = dplus[(size_t)i * kvec + l] + dm - (d[i] - lam);
        if (fabs(g) < best) { best = fabs(g); t.gamma = g; t.r = i; }
    }
    double nrm2 = 1.0, zi = 1.0;
    for (int i = t.r - 1; i >= bs; --i) {
        zi = -lplus[(size_t)i * kvec + l] * zi;
        nrm2 += zi * zi;
    }
    zi = 1.0;
    for (int i = t.r; i < be - 1; ++i) {
        zi = -uminus[(size_t)i * kvec + l] * zi;
        nrm2 += zi * zi;
    }
    t.nrm2 = nrm2;
    return t;
}

// Twisted factorisation eigenvector for each of the first kvec eigenvalues (w[l] is the
// eigenvalue of index l, zero outside its block).
template <typename T>
__global__ void twisted_kernel(int n, const double *__restrict__ d, const double *__restrict__ e,
                               int kvec, const double *__restrict__ w, const double *bounds,
                               const int *__restrict__ blk, T *z, int ldz, double *dplus,
                               double *uminus, double *lplus, int *status)
{
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= kvec) return;
    const double pivmin = bounds[2];
    const int bs = blk[2 * l], be = blk[2 * l + 1];  // the eigenvalue's block [bs, be)
    const Twist t = twisted_factor(d, e, bs, be, w[l], pivmin, kvec, l, dplus, lplus, uminus);
    const double nrm2 = t.nrm2;
    const int r = t.r;
    if (!(nrm2 < DBL_MAX)) { report_error(status, ELSI_ERR_NO_CONVERGENCE, l); }
    const double s = (nrm2 < DBL_MAX) ? 1.0 / sqrt(nrm2) : 1.0;
    // write z / ||z|| (zero outside the block)
    T *zc = z + (size_t)l * ldz;
    for (int i = 0; i < bs; ++i) zc[i] = T(0);
    for (int i = be; i < n; ++i) zc[i] = T(0);
    zc[r] = (T)s;
    double zi = 1.0;
    for (int i = r - 1; i >= bs; --i) {
        zi = -lplus[(size_t)i * kvec + l] * zi;
        zc[i] = (T)(zi * s);
    }
    zi = 1.0;
    for (int i = r; i < be - 1; ++i) {
        zi = -uminus[(size_t)i * kvec + l] * zi;
        zc[i + 1] = (T)(zi * s);
    }
}

// Gram-Schmidt of vector zv against the cluster vectors i0 .. v-1 (two passes); returns
// the squared norm left.
template <typename T>
__device__ double cluster_project(int n, int i0, int v, T *z, int ldz, double *red)
{
    T *zv = z + (size_t)v * ldz;
    for (int pass = 0; pass < 2; ++pass) {
        for (int u = i0; u < v; ++u) {
            const T *zu = z + (size_t)u * ldz;
            double s = 0.0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)zu[i] * (double)zv[i];
            s = block_sum(s, red);
            for (int i = threadIdx.x; i < n; i += blockDim.x) zv[i] = (T)((double)zv[i] - s * (double)zu[i]);
            __syncthreads();
        }
    }
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)zv[i] * (double)zv[i];
    return block_sum(s, red);
}

__device__ __forceinline__ double hash_unit(unsigned a, unsigned b)
{
    unsigned h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
    return (double)h * (2.0 / 4294967296.0) - 1.0;
}

constexpr int kOrthPiece = 64;  // vectors orthogonalised together (pieces and seams)

// cstart[i] = first index of the cluster of i (chains of eigenvalues closer than
// tol_rel * ||T||). One CTA: each thread scans a contiguous segment, then the segment
// results are combined in order.
__global__ void cluster_start_kernel(int kvec, const double *w, const double *bounds, double tol_rel,
                                     int *cstart)
{
    __shared__ int last[1024];
    const double tol = tol_rel * fmax(bounds[3], DBL_MIN);
    const int nt = blockDim.x, t = threadIdx.x;
    const int seg = (kvec + nt - 1) / nt;
    const int a = t * seg, b = min(kvec, a + seg);
    int cur = -1;  // start of the current cluster inside the segment (-1: continues from left)
    for (int i = a; i < b; ++i) {
        if (i == 0 || !(w[i] - w[i - 1] < tol)) cur = i;
        cstart[i] = cur;
    }
    last[t] = cur;
    __syncthreads();
    if (t == 0)
        for (int q = 1; q < nt; ++q)
            if (last[q] < 0) last[q] = last[q - 1];
    __syncthreads();
    if (a < b && t > 0) {
        const int carry = last[t - 1];
        for (int i = a; i < b && cstart[i] < 0; ++i) cstart[i] = carry;
    }
}

// Gram-Schmidt (two passes) within clusters of eigenvalues closer than tol_rel * ||T||,
// on ranges of at most kOrthPiece vectors: phase 0 takes the pieces [s + 64p, s + 64p + 64)
// of a cluster starting at s, phase 1 the seams [s + 64p + 32, s + 64p + 96) that cross a
// piece boundary; one CTA per range start. A vector that the projection nearly annihilates (its
// eigenvalue coincides with an earlier one to working accuracy, as for the pairs of the
// real form of a complex Hermitian matrix) is replaced by one step of inverse iteration
// on its block, x = (T_b - lambda I)^{-1} b for a pseudo-random b orthogonal to the
// cluster's vectors, using the L+ D+ L+^T factors that the twisted factorisation left in
// dplus (the vector's spent U- column holds the intermediate values), and is then
// projected and normalised again. When lambda sits much closer to an accepted vector's
// eigenvalue than to its own, that vector dominates x; what is left after the projection
// is still accurate as long as it is far above the rounding level.
template <typename T>
__global__ void cluster_orth_kernel(int n, int kvec, const int *cstart, int phase, const double *e,
                                    const int *blk, const double *dplus, double *work, T *z, int ldz,
                                    int *status)
{
    __shared__ double red[32];
    const int i0 = blockIdx.x;
    const int s = cstart[i0];
    const int off = phase == 0 ? 0 : kOrthPiece / 2;
    if ((i0 - s) % kOrthPiece != off) return;  // not a range start
    int cend = i0 + 1;  // end of the cluster, looked for up to the end of the range
    while (cend < kvec && cend < i0 + kOrthPiece && cstart[cend] == s) ++cend;
    if (phase == 1 && cend <= i0 + kOrthPiece / 2) return;  // no piece boundary inside
    const int i1 = cend;
    if (i1 - i0 < 2) return;
    for (int v = i0 + 1; v < i1; ++v) {
        T *zv = z + (size_t)v * ldz;
        double s = cluster_project(n, i0, v, z, ldz, red);
        // a regenerated vector is accepted when its part orthogonal to the cluster is far
        // above the rounding level of T (its direction error is then eps / sqrt(s))
        const double accept = sizeof(T) == 8 ? 1e-16 : 1e-8;
        bool regen = false;
        for (int attempt = 0; attempt < 3 && s < (regen ? accept : 1e-4); ++attempt) {
            regen = true;
            const int bs = blk[2 * v], be = blk[2 * v + 1];
            // start b: pseudo-random on the block, orthogonal to the cluster's vectors
            for (int i = threadIdx.x; i < n; i += blockDim.x)
                zv[i] = (i >= bs && i < be) ? (T)hash_unit((unsigned)(v * 7919 + attempt), (unsigned)i) : T(0);
            __syncthreads();
            cluster_project(n, i0, v, z, ldz, red);
            if (threadIdx.x == 0) {
                double *x = work + v;  // x[i * kvec]
                // forward: L+ y = b; backward: L+^T x = D+^{-1} y. Entries are rescaled
                // (all at once) whenever one exceeds 2^500.
                const double big = 0x1p500, shrink = 0x1p-500;
                double y = 0.0;
                for (int i = bs; i < be; ++i) {
                    const double bi = (double)zv[i];
                    y = (i == bs) ? bi : bi - (e[i - 1] / dplus[(size_t)(i - 1) * kvec + v]) * y;
                    if (fabs(y) > big) {
                        for (int j = bs; j < i; ++j) x[(size_t)j * kvec] *= shrink;
                        y *= shrink;
                    }
                    x[(size_t)i * kvec] = y;
                }
                double xi = 0.0;
                for (int i = be - 1; i >= bs; --i) {
                    const double yi = x[(size_t)i * kvec] / dplus[(size_t)i * kvec + v];
                    xi = (i == be - 1) ? yi : yi - (e[i] / dplus[(size_t)i * kvec + v]) * xi;
                    if (fabs(xi) > big) {
                        for (int j = i + 1; j < be; ++j) x[(size_t)j * kvec] *= shrink;
                        for (int j = bs; j < i; ++j) x[(size_t)j * kvec] *= shrink;
                        xi *= shrink;
                    }
                    x[(size_t)i * kvec] = xi;
                }
                double mx = 0.0;
                for (int i = bs; i < be; ++i) mx = fmax(mx, fabs(x[(size_t)i * kvec]));
                const double sc = (mx > 0.0 && mx <= DBL_MAX) ? 1.0 / mx : 0.0;
                for (int i = 0; i < n; ++i)
                    zv[i] = (i >= bs && i < be) ? (T)(x[(size_t)i * kvec] * sc) : T(0);
            }
            __syncthreads();
            double nr = 0.0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) nr += (double)zv[i] * (double)zv[i];
            nr = block_sum(nr, red);
            const double inv = (nr > 0.0) ? 1.0 / sqrt(nr) : 0.0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) zv[i] = (T)((double)zv[i] * inv);
            __syncthreads();
            s = cluster_project(n, i0, v, z, ldz, red);
        }
        if (s < (regen ? accept : 1e-4)) {
            if (threadIdx.x == 0) report_error(status, ELSI_ERR_NO_CONVERGENCE, v);
            return;
        }
        const double inv = 1.0 / sqrt(s);
        for (int i = threadIdx.x; i < n; i += blockDim.x) zv[i] = (T)((double)zv[i] * inv);
        __syncthreads();
    }
}

template <typename T>
cudaError_t stein(cudaStream_t st, int n, const double *d, const double *e, int kvec,
                  const double *w, T *z, int ldz, double *scratch, int *status)
{
    if (n <= 0 || kvec <= 0) return cudaSuccess;
    // scratch: D+ (n x kvec), U- (n x kvec), bounds (8), blk (2 kvec ints), L+ (n x kvec)
    double *dplus = scratch, *uminus = scratch + (size_t)n * kvec;
    double *bounds = scratch + (size_t)2 * n * kvec;
    int *blk = reinterpret_cast<int *>(bounds + 8);
    double *lplus = bounds + 16 + kvec;
    EGB_COUNT_LAUNCH();
    gershgorin_kernel<<<1, 1024, 0, st>>>(n, d, e, bounds);
    EGB_COUNT_LAUNCH();
    block_assign_kernel<<<ceil_div(kvec, 64), 64, 0, st>>>(n, d, e, kvec, w, bounds, blk);
    EGB_COUNT_LAUNCH();
    twisted_kernel<T><<<ceil_div(kvec, 64), 64, 0, st>>>(n, d, e, kvec, w, bounds, blk, z, ldz, dplus,
                                                        uminus, lplus, status);
    // cluster starts (in the L+ scratch, no longer needed), then pieces and seams
    int *cstart = reinterpret_cast<int *>(lplus);
    EGB_COUNT_LAUNCH();
    cluster_start_kernel<<<1, 1024, 0, st>>>(kvec, w, bounds, 1e-5, cstart);
    for (int phase = 0; phase < 2; ++phase) {
        EGB_COUNT_LAUNCH();
        cluster_orth_kernel<T><<<kvec, 256, 0, st>>>(n, kvec, cstart, phase, e, blk, dplus, uminus, z,
                                                     ldz, status);
    }
    return cudaGetLastError();
}

template cudaError_t stein<double>(cudaStream_t, int, const double *, const double *, int,
                                   const double *, double *, int, double *, int *);
template cudaError_t stein<float>(cudaStream_t, int, const double *, const double *, int,
                                  const double *, float *, int, double *, int *);

}  // namespace egb
