// Back-transformation through Q2 (step (4) of the two-stage method, arXiv:1705.11191
// sec. 3.1) for the binary32 route, blocked into compact-WY form and run on the tensor
// cores.
//
// The reflectors of sweeps J .. J+m-1 at bulge-chase step t (the group (J, t), m = 64) act
// on a window of m + b - 1 rows. In the order they are applied to the eigenvectors
// (sweep J+m-1 first), their product is I - V T^T V^T, where V holds the reflectors as
// columns (column a = sweep J+m-1-a, shifted down by J+m-1-a-J rows) and T is the upper
// triangular factor of the forward accumulation (Schreiber & Van Loan's compact WY).
// T is computed once per group (q2_tfactor_kernel); the application kernel keeps the
// current window of its 128 columns of Z in a shared-memory ring and performs, per group,
//     Y = V^T Z_w,  Y = T^T Y,  Z_w -= V Y
// with mma.sync m16n8k8 TF32 products in three-pass split precision
// (x = x_hi + x_lo, x_hi = x truncated to tf32; A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi),
// about binary32 accuracy.
#include "common.cuh"
#include "kernels.h"

namespace egb {

constexpr int kWyM = 64;          // reflectors per group (sweeps per block)
constexpr int kWyRows = 128;      // window rows covered (m + b - 1 <= 127)
constexpr int kWyCols = 128;      // columns of Z per CTA (8 warps x 16)
constexpr int kWyRing = 256;      // ring rows (power of two)
constexpr int kWyRingLd = kWyRing + 4;
constexpr int kWyVtLd = kWyRows + 8;   // V^T rows (a) stride
constexpr int kWyTLd = kWyM + 4;
constexpr int kWyYLd = kWyM + 4;

constexpr int kWyGroupWords = kWyM * kWyRows + kWyM * kWyM;

__device__ __forceinline__ int wy_steps(int n, int b, int j) { return (n - 2 - j) / b + 1; }


// x = hi + lo with hi = x truncated to TF32 (one bit mask) and lo = x - hi (exact); the
// tensor core reads lo truncated to TF32 as well, which leaves an error below
// 2^-20 |x|, ample for the binary32 route that the refinement corrects.
__device__ __forceinline__ void split_tf32(float x, unsigned &hi, unsigned &lo)
{
    hi = __float_as_uint(x) & 0xFFFFE000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}

// ---------------------------------------------------------------- T factors
// One CTA (128 threads) per group g = jb * S + t. Writes, for the application kernel,
// the group's V^T (64 x 128, [a][window row]) and T^T (64 x 64, [a][c] = T[c][a]) in
// binary32; layout per group: [Vt | Tt] = kWyGroupWords words. Reflectors with tau = 0 (none or
// trivial) are treated as zero columns of V, which does not change I - V T V^T.
// T is built by blocks: the 8 diagonal 8 x 8 blocks by the forward recurrence, then
// pairs of blocks are merged, T = [[T1, -T1 (V1^T V2) T2], [0, T2]], for block sizes
// 8 -> 16 -> 32 -> 64.
__global__ void __launch_bounds__(128) q2_tfactor_kernel(int n, int b, int S, int nblk,
                                                         const float *__restrict__ v2,
                                                         const float *__restrict__ tau2,
                                                         float *__restrict__ tfac)
{
    const int g = blockIdx.x;
    const int jb = g / S, t = g % S;
    const int J = jb * kWyM;
    const int Jend = min(n - 2, J + kWyM);
    unsigned *gw = reinterpret_cast<unsigned *>(tfac) + (size_t)g * kWyGroupWords;
    const int tid = threadIdx.x;
    if (t >= wy_steps(n, b, J)) {  // no sweep of this block reaches step t
        for (int e = tid; e < kWyGroupWords; e += blockDim.x) gw[e] = 0u;
        return;
    }
    extern __shared__ __align__(16) float tsm[];
    float(*Vc)[65] = reinterpret_cast<float(*)[65]>(tsm);                       // compact v_a[i]
    float(*Gm)[kWyM + 1] = reinterpret_cast<float(*)[kWyM + 1]>(tsm + kWyM * 65);  // v_a . v_c
    float(*Tm)[kWyM + 1] = reinterpret_cast<float(*)[kWyM + 1]>(tsm + kWyM * 65 + kWyM * (kWyM + 1));
    float(*Wk)[kWyM + 1] = reinterpret_cast<float(*)[kWyM + 1]>(tsm + kWyM * 65 + 2 * kWyM * (kWyM + 1));
    float *tau = tsm + kWyM * 65 + 3 * kWyM * (kWyM + 1);
    for (int a = tid; a < kWyM; a += blockDim.x) {
        int j = Jend - 1 - a;
        tau[a] = (j >= J && t < wy_steps(n, b, j)) ? tau2[(size_t)j * S + t] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < kWyM * 64; e += blockDim.x) {
        int a = e / 64, i = e % 64;
        int j = Jend - 1 - a;
        Vc[a][i] = (i < b && tau[a] != 0.f) ? v2[((size_t)j * S + t) * b + i] : 0.f;
    }
    __syncthreads();
    // G[a][c] (a < c): reflector a starts (c - a) rows below reflector c in the window
    for (int e = tid; e < kWyM * kWyM; e += blockDim.x) {
        int a = e / kWyM, c = e % kWyM;
        float s = 0.f;
        if (a < c) {
            const int d = c - a;  // off_a = off_c + d
            for (int i = 0; i + d < b; ++i) s = fmaf(Vc[a][i], Vc[c][i + d], s);
        }
        Gm[a][c] = s;
        Tm[a][c] = 0.f;
    }
    __syncthreads();
    // diagonal 8 x 8 blocks: warp w handles blocks 2w, 2w+1; lane = row within block pair
    {
        const int warp = tid >> 5, lane = tid & 31;
        const int blk = 2 * warp + (lane >> 4), r = lane & 15;  // r < 8 used
        const int base = blk * 8;
        for (int a = 0; a < 8; ++a) {
            if (r < a) {
                float s2 = 0.f;
                for (int p = r; p < a; ++p) s2 = fmaf(Tm[base + r][base + p], Gm[base + p][base + a], s2);
                Tm[base + r][base + a] = -tau[base + a] * s2;
            }
            if (r == a) Tm[base + a][base + a] = tau[base + a];
            __syncwarp();
        }
    }
    __syncthreads();
    // merges: blocks of size h -> 2h
    for (int h = 8; h < kWyM; h *= 2) {
        const int npair = kWyM / (2 * h);
        // Wk = G12 T2 for every pair (h x h each)
        for (int e = tid; e < npair * h * h; e += blockDim.x) {
            int pr = e / (h * h), rem = e % (h * h), i = rem / h, c = rem % h;
            int o1 = pr * 2 * h, o2 = o1 + h;
            float s2 = 0.f;
            for (int p = 0; p <= c; ++p) s2 = fmaf(Gm[o1 + i][o2 + p], Tm[o2 + p][o2 + c], s2);
            Wk[o1 + i][o2 + c] = s2;
        }
        __syncthreads();
        // T12 = -T1 Wk
        for (int e = tid; e < npair * h * h; e += blockDim.x) {
            int pr = e / (h * h), rem = e % (h * h), i = rem / h, c = rem % h;
            int o1 = pr * 2 * h, o2 = o1 + h;
            float s2 = 0.f;
            for (int p = i; p < h; ++p) s2 = fmaf(Tm[o1 + i][o1 + p], Wk[o1 + p][o2 + c], s2);
            Tm[o1 + i][o2 + c] = -s2;
        }
        __syncthreads();
    }
    // dense V^T rows: reflector a (application order) starts at window row off_a = Jend-1-a-J
    for (int e = tid; e < kWyM * kWyRows; e += blockDim.x) {
        int a = e / kWyRows, r = e % kWyRows;
        int i = r - (Jend - 1 - a - J);
        gw[e] = __float_as_uint((i >= 0 && i < 64) ? Vc[a][i] : 0.f);
    }
    for (int e = tid; e < kWyM * kWyM; e += blockDim.x) {
        int a = e / kWyM, c = e % kWyM;
        gw[kWyM * kWyRows + e] = __float_as_uint(Tm[c][a]);  // T^T row-major
    }
}

// ---------------------------------------------------------------- application
__device__ __forceinline__ void wy_cp_async4(float *dst, const float *src)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
}

__device__ __forceinline__ void mma_tf32_raw(float *c, unsigned a0, unsigned a1, unsigned a2,
                                             unsigned a3, unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void wy_cp_async16(void *dst, const void *src)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}

constexpr int kWyVLd = kWyRows + 8;   // 136 words
constexpr int kWyTLd2 = kWyM + 4;     // 68 words
constexpr int kWyWcols = 16;          // columns per warp
constexpr int kWyWarps = kWyCols / kWyWcols;

__device__ __forceinline__ void split4(const float *v, unsigned *h, unsigned *l)
{
#pragma unroll
    for (int q = 0; q < 4; ++q) split_tf32(v[q], h[q], l[q]);
}

// CTA: 256 threads (8 warps), 128 columns of Z; warp w owns columns [16w, 16w+16) in all
// three products, so only the staging of V and T needs a block-wide barrier. V^T and T^T are
// staged in binary32 and split into TF32 hi / lo parts as the fragments are read. The
// reflectors of a group form a band in the window (reflector a covers window rows
// off_a .. off_a + b - 1, off_a = m - 1 - a for the group's m reflectors), so the products
// with V skip the blocks of 16 x 8 that are zero.
__global__ void __launch_bounds__(256) q2_apply_tc_kernel(int n, int b, int S, const float *__restrict__ tfac,
                                                          int k, float *z, int ldz)
{
    extern __shared__ __align__(16) unsigned wsm[];
    float *ring = reinterpret_cast<float *>(wsm);                  // [col][slot]
    float *Vs = ring + kWyCols * kWyRingLd;                        // V^T [a][row]
    float *Ts = Vs + kWyM * kWyVLd;                                // T^T [a][c]
    float *Yall = Ts + kWyM * kWyTLd2;                             // per warp: [col][a]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gq = lane >> 2, tq = lane & 3;
    const int c0 = blockIdx.x * kWyCols;
    const int wc0 = warp * kWyWcols;                               // first local column of the warp
    const int ncol = min(kWyCols, k - c0);
    const int wncol = max(0, min(kWyWcols, ncol - wc0));
    float *Y = Yall + warp * kWyWcols * kWyTLd2;
    const int nsweep = n - 2;
    const int nblk = (nsweep + kWyM - 1) / kWyM;

    auto rs = [&](int col, int r) -> float & { return ring[col * kWyRingLd + (r & (kWyRing - 1))]; };
    // each warp moves the rows of its own columns
    auto fetch_rows = [&](int r0, int r1) {
        const int nr = r1 - r0;
        for (int e = lane; e < nr * wncol; e += 32) {
            int r = r0 + e % nr, c = wc0 + e / nr;
            wy_cp_async4(&rs(c, r), z + (size_t)r + (size_t)(c0 + c) * ldz);
        }
    };
    auto store_rows = [&](int r0, int r1) {
        const int nr = r1 - r0;
        for (int e = lane; e < nr * wncol; e += 32) {
            int r = r0 + e % nr, c = wc0 + e / nr;
            z[(size_t)r + (size_t)(c0 + c) * ldz] = rs(c, r);
        }
    };

    for (int jb = nblk - 1; jb >= 0; --jb) {
        const int J = jb * kWyM;
        const int Jend = min(nsweep, J + kWyM);
        const int mA = Jend - J;  // reflectors of this block (columns a >= mA of V are zero)
        const int SJ = wy_steps(n, b, J);
        int lo = J + 1;
        int hi = min(n, Jend + b);
        // columns the warp does not own stay zero
        for (int e = lane; e < kWyWcols * kWyRing; e += 32)
            if (e / kWyRing >= wncol) ring[(wc0 + e / kWyRing) * kWyRingLd + e % kWyRing] = 0.f;
        fetch_rows(lo, hi);
        asm volatile("cp.async.commit_group;\n" ::);
        for (int t = 0; t < SJ; ++t) {
            // ---- stage V^T and T^T of group (jb, t) (everyone finished step t-1)
            __syncthreads();
            {
                const float *gsrc = tfac + ((size_t)jb * S + t) * kWyGroupWords;
                for (int e = tid; e < kWyM * 32; e += 256) {  // 64 rows x 32 chunks of 4
                    int a = e >> 5, ch = e & 31;
                    wy_cp_async16(Vs + a * kWyVLd + ch * 4, gsrc + a * kWyRows + ch * 4);
                }
                for (int e = tid; e < kWyM * 16; e += 256) {  // 64 rows x 16 chunks
                    int a = e >> 4, ch = e & 15;
                    wy_cp_async16(Ts + a * kWyTLd2 + ch * 4, gsrc + kWyM * kWyRows + a * kWyM + ch * 4);
                }
                asm volatile("cp.async.commit_group;\n" ::);
            }
            const int nlo = min(lo + b, n), nhi = min(hi + b, n);
            asm volatile("cp.async.wait_group 0;\n" ::);
            __syncthreads();
            // prefetch the window rows of step t+1 (own columns)
            if (t + 1 < SJ) fetch_rows(hi, nhi);
            asm volatile("cp.async.commit_group;\n" ::);
            const int wrows = hi - lo;

            // ---- Y (64 x 16) = V^T Z_w[:, own columns]
#pragma unroll 1
            for (int im = 0; im < 4; ++im) {
                const int am = im * 16;
                float acc[2][4];
#pragma unroll
                for (int jn = 0; jn < 2; ++jn)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[jn][q] = 0.f;
                if (am < mA) {
                    // window rows covered by reflectors am .. am + 15
                    const int alast = min(am + 15, mA - 1);
                    const int klo = ((mA - 1 - alast) / 8) * 8;
                    const int khi = min(wrows, mA - 1 - am + b);
                    for (int k0 = klo; k0 < khi; k0 += 8) {
                        unsigned bh[2][2], bl[2][2];
#pragma unroll
                        for (int jn = 0; jn < 2; ++jn) {
                            const int col = wc0 + jn * 8 + gq;
                            float x0 = (k0 + tq < wrows) ? rs(col, lo + k0 + tq) : 0.f;
                            float x1 = (k0 + tq + 4 < wrows) ? rs(col, lo + k0 + tq + 4) : 0.f;
                            split_tf32(x0, bh[jn][0], bl[jn][0]);
                            split_tf32(x1, bh[jn][1], bl[jn][1]);
                        }
                        const int i0 = (am + gq) * kWyVLd + k0 + tq, i1 = (am + gq + 8) * kWyVLd + k0 + tq;
                        const float av[4] = {Vs[i0], Vs[i1], Vs[i0 + 4], Vs[i1 + 4]};
                        unsigned ah[4], al[4];
                        split4(av, ah, al);
#pragma unroll
                        for (int jn = 0; jn < 2; ++jn) {
                            mma_tf32_raw(acc[jn], al[0], al[1], al[2], al[3], bh[jn][0], bh[jn][1]);
                            mma_tf32_raw(acc[jn], ah[0], ah[1], ah[2], ah[3], bl[jn][0], bl[jn][1]);
                            mma_tf32_raw(acc[jn], ah[0], ah[1], ah[2], ah[3], bh[jn][0], bh[jn][1]);
                        }
                    }
                }
                // Y -> warp scratch as the B operand of the next product: [col][a]
#pragma unroll
                for (int jn = 0; jn < 2; ++jn)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int a = am + gq + (q >> 1) * 8, col = jn * 8 + 2 * tq + (q & 1);
                        Y[col * kWyTLd2 + a] = acc[jn][q];
                    }
            }
            __syncwarp();
            // ---- Y2 = T^T Y (64 x 16), stored negated
            {
                float acc[4][2][4];
#pragma unroll
                for (int im = 0; im < 4; ++im)
#pragma unroll
                    for (int jn = 0; jn < 2; ++jn)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[im][jn][q] = 0.f;
#pragma unroll 2
                for (int k0 = 0; k0 < kWyM; k0 += 8) {
                    unsigned bh[2][2], bl[2][2];
#pragma unroll
                    for (int jn = 0; jn < 2; ++jn) {
                        const int col = jn * 8 + gq;
                        split_tf32(Y[col * kWyTLd2 + k0 + tq], bh[jn][0], bl[jn][0]);
                        split_tf32(Y[col * kWyTLd2 + k0 + tq + 4], bh[jn][1], bl[jn][1]);
                    }
#pragma unroll
                    for (int im = 0; im < 4; ++im) {
                        const int am = im * 16;
                        // T^T is lower triangular: rows am .. am + 15 have no entry in
                        // columns >= am + 16
                        if (k0 >= am + 16) continue;
                        const int i0 = (am + gq) * kWyTLd2 + k0 + tq, i1 = (am + gq + 8) * kWyTLd2 + k0 + tq;
                        const float av[4] = {Ts[i0], Ts[i1], Ts[i0 + 4], Ts[i1 + 4]};
                        unsigned ah[4], al[4];
                        split4(av, ah, al);
#pragma unroll
                        for (int jn = 0; jn < 2; ++jn) {
                            mma_tf32_raw(acc[im][jn], al[0], al[1], al[2], al[3], bh[jn][0], bh[jn][1]);
                            mma_tf32_raw(acc[im][jn], ah[0], ah[1], ah[2], ah[3], bl[jn][0], bl[jn][1]);
                            mma_tf32_raw(acc[im][jn], ah[0], ah[1], ah[2], ah[3], bh[jn][0], bh[jn][1]);
                        }
                    }
                }
                __syncwarp();
#pragma unroll
                for (int im = 0; im < 4; ++im)
#pragma unroll
                    for (int jn = 0; jn < 2; ++jn)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int a = im * 16 + gq + (q >> 1) * 8, col = jn * 8 + 2 * tq + (q & 1);
                            Y[col * kWyTLd2 + a] = -acc[im][jn][q];
                        }
            }
            __syncwarp();
            // ---- Z_w[:, own columns] += V (-Y2): rows in 8 m-tiles of 16
            for (int mt = 0; mt < kWyRows / 16; ++mt) {
                const int r = mt * 16;
                if (r >= wrows) break;
                // reflectors with a nonzero entry in rows r .. r + 15
                const int alo = max(0, mA - 1 - min(r + 15, wrows - 1));
                const int ahi = min(mA - 1, mA + b - 2 - r);
                if (alo > ahi) continue;
                const int k0lo = (alo / 8) * 8, k0hi = ahi + 1;
                float acc[2][4];
#pragma unroll
                for (int jn = 0; jn < 2; ++jn) {
                    const int col = wc0 + jn * 8 + 2 * tq;
                    const int ra = r + gq, rb = r + gq + 8;
                    acc[jn][0] = (ra < wrows) ? rs(col, lo + ra) : 0.f;
                    acc[jn][1] = (ra < wrows) ? rs(col + 1, lo + ra) : 0.f;
                    acc[jn][2] = (rb < wrows) ? rs(col, lo + rb) : 0.f;
                    acc[jn][3] = (rb < wrows) ? rs(col + 1, lo + rb) : 0.f;
                }
                for (int k0 = k0lo; k0 < k0hi; k0 += 8) {
                    // A[row][a] = V[row][a] = Vt[a][row]
                    const int i0 = (k0 + tq) * kWyVLd + r + gq, i2 = (k0 + tq + 4) * kWyVLd + r + gq;
                    const float av[4] = {Vs[i0], Vs[i0 + 8], Vs[i2], Vs[i2 + 8]};
                    unsigned ah[4], al[4];
                    split4(av, ah, al);
#pragma unroll
                    for (int jn = 0; jn < 2; ++jn) {
                        const int col = jn * 8 + gq;
                        unsigned bh0, bl0, bh1, bl1;
                        split_tf32(Y[col * kWyTLd2 + k0 + tq], bh0, bl0);
                        split_tf32(Y[col * kWyTLd2 + k0 + tq + 4], bh1, bl1);
                        mma_tf32_raw(acc[jn], al[0], al[1], al[2], al[3], bh0, bh1);
                        mma_tf32_raw(acc[jn], ah[0], ah[1], ah[2], ah[3], bl0, bl1);
                        mma_tf32_raw(acc[jn], ah[0], ah[1], ah[2], ah[3], bh0, bh1);
                    }
                }
#pragma unroll
                for (int jn = 0; jn < 2; ++jn) {
                    const int col = wc0 + jn * 8 + 2 * tq;
                    const int ra = r + gq, rb = r + gq + 8;
                    if (ra < wrows) { rs(col, lo + ra) = acc[jn][0]; rs(col + 1, lo + ra) = acc[jn][1]; }
                    if (rb < wrows) { rs(col, lo + rb) = acc[jn][2]; rs(col + 1, lo + rb) = acc[jn][3]; }
                }
            }
            __syncwarp();
            // rows [lo, nlo) are final for this block of sweeps (own columns)
            if (t + 1 < SJ) {
                store_rows(lo, nlo);
                lo = nlo;
                hi = nhi;
            } else {
                store_rows(lo, hi);
            }
            __syncwarp();
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
}

size_t q2_tfactor_elems_legacy(int n, int b)
{
    if (n < 3) return 1;
    const int S = sb2st_steps(n, b);
    const int nblk = (n - 2 + kWyM - 1) / kWyM;
    return (size_t)nblk * S * kWyGroupWords;
}

cudaError_t apply_q2_tc_legacy(cudaStream_t st, int n, int b, const float *v2, const float *tau2, int k,
                        float *z, int ldz, float *tfac)
{
    if (n < 3 || k <= 0) return cudaSuccess;
    if (b > 64 || kWyM + b - 1 > kWyRows) return cudaErrorInvalidValue;
    const int S = sb2st_steps(n, b);
    const int nblk = (n - 2 + kWyM - 1) / kWyM;
    const size_t tsmem = (size_t)(kWyM * 65 + 3 * kWyM * (kWyM + 1) + kWyM) * sizeof(float);
    static PerDeviceOnce tattr;
    cudaError_t e = once_per_device(tattr, [&] {
        return cudaFuncSetAttribute(q2_tfactor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem);
    });
    if (e != cudaSuccess) return e;
    EGB_COUNT_LAUNCH();
    q2_tfactor_kernel<<<nblk * S, 128, tsmem, st>>>(n, b, S, nblk, v2, tau2, tfac);
    const size_t smem = (size_t)(kWyCols * kWyRingLd + kWyM * kWyVLd + kWyM * kWyTLd2 +
                                 kWyWarps * kWyWcols * kWyTLd2) * sizeof(float);
    static PerDeviceOnce attr;
    e = once_per_device(attr, [&] {
        return cudaFuncSetAttribute(q2_apply_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e != cudaSuccess) return e;
    (void)tau2;
    EGB_COUNT_LAUNCH();
    q2_apply_tc_kernel<<<ceil_div(k, kWyCols), 256, smem, st>>>(n, b, S, tfac, k, z, ldz);
    return cudaGetLastError();
}

}  // namespace egb
