// Back-transformation through Q2 (step (4) of the two-stage method, arXiv:1705.11191
// sec. 3.1) for the binary32 route, on the 5th-generation tensor cores (tcgen05).
//
// Grouping. The bulge chase leaves one Householder reflector per (sweep j, step t), acting
// on rows j+1+tb .. j+tb+b. The reflectors of the sweeps J .. J+63 of one block at step t
// form the group (J, t); in the order they are applied to the eigenvectors (sweep J+63
// first) their product is I - V T^T V^T (Schreiber & Van Loan's compact WY), with V the
// reflectors as columns, column a = sweep J+63-a, and T upper triangular. The groups are
// applied block by block (J descending), and inside a block in ascending t; within a block
// only group t-1 overlaps group t, and every pair of overlapping reflectors keeps the
// order of the sequential back-transformation (the later sweep first).
//
// Window. Group (J, t) touches rows J+1+tb .. J+tb+b+62; the kernel works on the 8-aligned
// window of 128 rows starting at w0 = J + tb (one row above the first reflector, so the
// window start is a multiple of 8 for every band width that is). After the group, the rows
// w0 .. w0+b-1 are final for this block and are replaced by the rows w0+128 .. w0+b+127.
// A window row r is kept in slot r mod 128, so a row stays in the same place while it is
// in the window; the logical position of slot s is p = (s - w0) mod 128.
//
// Per group, with W = -V T^T (window rows x 64, precomputed):
//     Y^T  = Z_w^T V         (MMA 1: M = 128 columns of Z, N = 64, K = 128 window rows)
//     dZ^T = Y^T W^T         (MMA 2: M = 128 columns of Z, N = 128 window rows, K = 64)
//     Z_w += dZ
// Both products are TF32 in three passes of hi/lo splits (x = hi + lo, hi = x with the low
// 13 mantissa bits cleared, lo = x - hi exactly; A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi),
// the hi*hi sum and the (2^-11 times smaller) cross-term sum in separate tensor-memory
// accumulators, added in binary32 registers. Z stays in binary32 registers between groups;
// each group's products start from fresh accumulators, so tensor-memory accumulation never
// sums more than 3 x K/8 partial products into one value.
//
// CTA (512 threads, 16 warps, one CTA per SM): 128 columns of Z; warp w owns the columns
// 32 (w mod 4) .. +31 (one per lane, the tensor-memory lane quarter of the warp) and the
// window slots 32 (w / 4) .. +31 of them, in registers. The A operands (Z_w^T, then Y^T,
// hi and lo) are written to tensor memory with tcgen05.st; V and W (hi and lo) come from a
// per-group block that the factor kernel writes already in the shared-memory layout of the
// B operand (K-major, 128-byte swizzle), fetched with bulk asynchronous copies: V of the
// next group as soon as MMA 1 has read the current one, W as soon as MMA 2 has. Thread 0
// issues the copies and the MMAs. Every wait is bounded; on expiry the CTA records
// ELSI_ERR_TIMEOUT, waits (bounded) for its own operations in flight, frees its tensor
// memory and returns.
#include <cuda.h>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace egb {
namespace q2tc {

using namespace tc5;

constexpr int kM = 64;       // reflectors per group (sweeps per block)
constexpr int kWin = 128;    // window rows
constexpr int kCols = 128;   // columns of Z per CTA
constexpr int kThreads = 512;                    // 16 warps
constexpr int kParts = kThreads / 128;           // warps per tensor-memory lane quarter
constexpr int kSlots = kWin / kParts;            // window slots per thread (32)
constexpr int kChunks = kSlots / 8;              // chunks of 8 slots per thread
constexpr int kVPlane = kWin * kM * 4;  // bytes of one plane of V: 4 K-chunks of [64 a][32 rows]
constexpr int kWPlane = kWin * kM * 4;  // bytes of one plane of W: 2 K-chunks of [128 rows][32 a]
constexpr int kGroupBytes = 2 * kVPlane + 2 * kWPlane;  // VH | VL | WH | WL = 128 KB
constexpr int kGroupFloats = kGroupBytes / 4;
constexpr int kSmemBytes = kGroupBytes + 1024 + 128;
constexpr unsigned kTmemCols = 512;
// tensor-memory columns
constexpr unsigned kZH = 0, kZL = 128;      // Z_w^T (A of MMA 1), later Y^T (A of MMA 2)
constexpr unsigned kAccH = 256, kAccX = 384;  // MMA 2: hi*hi and cross sums (128 columns each)
constexpr unsigned kYAccH = 256, kYAccX = 320;  // MMA 1: hi*hi and cross sums (64 columns each)

__host__ __device__ inline int block_steps(int n, int b, int J) { return (n - 2 - J) / b + 1; }

// Index of group (jb, 0) in the packed list of the groups that exist (t < steps of block jb).
__host__ __device__ inline long long group_base(int n, int b, int jb)
{
    long long s = 0;
    for (int i = 0; i < jb; ++i) s += block_steps(n, b, i * kM);
    return s;
}

__device__ __forceinline__ unsigned tf32_hi(float x) { return __float_as_uint(x) & 0xFFFFE000u; }

// Byte offset of element (row, kk) of a K-major operand tile with 128-byte swizzle: rows of
// 32 binary32 values, 16-byte chunk c of row r stored at chunk position c ^ (r mod 8).
__device__ __forceinline__ int swz(int row, int kk)
{
    return row * 128 + ((((kk >> 2) ^ (row & 7))) << 4) + ((kk & 3) << 2);
}

// ---------------------------------------------------------------- factors
// One CTA (256 threads) per group (jb, t) that exists. Builds V (application order, rows of
// the aligned window, zero outside the reflector and beyond row n-1), T by the forward
// recurrence on 8 x 8 diagonal blocks merged pairwise (8 -> 16 -> 32 -> 64), and
// W = -V T^T; writes the hi and lo TF32 planes of V ([a][window row], K = window row) and
// of W ([window row][a], K = a) in the swizzled operand layout.
__global__ void __launch_bounds__(256) q2_factor_kernel(int n, int b, int S, int jb_lo,
                                                        const float *__restrict__ v2,
                                                        const float *__restrict__ tau2,
                                                        float *__restrict__ fac)
{
    const int t = blockIdx.x, jb = jb_lo + blockIdx.y;
    const int J = jb * kM;
    if (t >= block_steps(n, b, J)) return;
    const int Jend = min(n - 2, J + kM);
    const int w0 = J + t * b;
    // groups of blocks jb_lo .. are packed from the start of fac
    unsigned char *out = reinterpret_cast<unsigned char *>(
        fac + (size_t)(group_base(n, b, jb) - group_base(n, b, jb_lo) + t) * kGroupFloats);
    extern __shared__ __align__(16) float fsm[];
    float(*Vc)[kM + 1] = reinterpret_cast<float(*)[kM + 1]>(fsm);                 // v_a[i]
    float(*Gm)[kM + 1] = reinterpret_cast<float(*)[kM + 1]>(fsm + kM * (kM + 1));  // v_a . v_c
    float(*Tm)[kM + 1] = reinterpret_cast<float(*)[kM + 1]>(fsm + 2 * kM * (kM + 1));
    float(*Wk)[kM + 1] = reinterpret_cast<float(*)[kM + 1]>(fsm + 3 * kM * (kM + 1));
    float *tau = fsm + 4 * kM * (kM + 1);
    int *off = reinterpret_cast<int *>(tau + kM);  // window row of v_a[0]
    const int tid = threadIdx.x;
    for (int a = tid; a < kM; a += blockDim.x) {
        const int j = Jend - 1 - a;  // sweep of column a
        const bool has = j >= J && t < block_steps(n, b, j);
        tau[a] = has ? tau2[(size_t)j * S + t] : 0.f;
        off[a] = j + 1 + t * b - w0;
    }
    __syncthreads();
    for (int e = tid; e < kM * kM; e += blockDim.x) {
        const int a = e / kM, i = e % kM;
        const int j = Jend - 1 - a;
        const bool in = i < b && tau[a] != 0.f && w0 + off[a] + i < n;
        Vc[a][i] = in ? v2[((size_t)j * S + t) * b + i] : 0.f;
    }
    __syncthreads();
    // G[a][c] = v_a . v_c for a < c: reflector a starts c - a rows below reflector c
    for (int e = tid; e < kM * kM; e += blockDim.x) {
        const int a = e / kM, c = e % kM;
        float s = 0.f;
        if (a < c) {
            const int d = c - a;
            for (int i = 0; i + d < b; ++i) s = fmaf(Vc[a][i], Vc[c][i + d], s);
        }
        Gm[a][c] = s;
        Tm[a][c] = 0.f;
    }
    __syncthreads();
    // diagonal 8 x 8 blocks of T: warp w builds block w, lane r < 8 holds row r
    {
        const int warp = tid >> 5, r = tid & 31;
        const int base = warp * 8;
        if (warp < kM / 8)
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
    // merge pairs of blocks: T12 = -T1 (V1^T V2) T2
    for (int h = 8; h < kM; h *= 2) {
        const int npair = kM / (2 * h);
        for (int e = tid; e < npair * h * h; e += blockDim.x) {
            const int pr = e / (h * h), rem = e % (h * h), i = rem / h, c = rem % h;
            const int o1 = pr * 2 * h, o2 = o1 + h;
            float s2 = 0.f;
            for (int p = 0; p <= c; ++p) s2 = fmaf(Gm[o1 + i][o2 + p], Tm[o2 + p][o2 + c], s2);
            Wk[o1 + i][o2 + c] = s2;
        }
        __syncthreads();
        for (int e = tid; e < npair * h * h; e += blockDim.x) {
            const int pr = e / (h * h), rem = e % (h * h), i = rem / h, c = rem % h;
            const int o1 = pr * 2 * h, o2 = o1 + h;
            float s2 = 0.f;
            for (int p = i; p < h; ++p) s2 = fmaf(Tm[o1 + i][o1 + p], Wk[o1 + p][o2 + c], s2);
            Tm[o1 + i][o2 + c] = -s2;
        }
        __syncthreads();
    }
    // V planes: element (a, window row r), K = r
    for (int e = tid; e < kM * kWin; e += blockDim.x) {
        const int a = e / kWin, r = e % kWin;
        const int i = r - off[a];
        const float x = (i >= 0 && i < b) ? Vc[a][i] : 0.f;
        const unsigned hi = tf32_hi(x);
        const int o = (r >> 5) * (kM * 128) + swz(a, r & 31);
        *reinterpret_cast<unsigned *>(out + o) = hi;
        *reinterpret_cast<float *>(out + kVPlane + o) = x - __uint_as_float(hi);
    }
    // W planes: W[r][c] = -sum_{a >= c} V[r][a] T[c][a]; element (window row r, c), K = c
    for (int e = tid; e < kWin * kM; e += blockDim.x) {
        const int r = e / kM, c = e % kM;
        float s = 0.f;
        for (int a = c; a < kM; ++a) {
            const int i = r - off[a];
            if (i >= 0 && i < b) s = fmaf(Vc[a][i], Tm[c][a], s);
        }
        const float x = -s;
        const unsigned hi = tf32_hi(x);
        const int o = (c >> 5) * (kWin * 128) + swz(r, c & 31);
        *reinterpret_cast<unsigned *>(out + 2 * kVPlane + o) = hi;
        *reinterpret_cast<float *>(out + 2 * kVPlane + kWPlane + o) = x - __uint_as_float(hi);
    }
}

// ---------------------------------------------------------------- application
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// D (tensor memory) [+]= A (tensor memory) x B (shared-memory descriptor), kind::tf32.
__device__ __forceinline__ void mma_tf32_ts(unsigned d, unsigned a, unsigned long long b, unsigned idesc,
                                            unsigned accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void tmem_st8(unsigned taddr, const unsigned *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8(unsigned taddr, float *v)
{
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// Eight consecutive rows r0 .. r0+7 of a column (rows >= n read as 0 / not stored); two
// 16-byte accesses when the column start allows it (vec: ld a multiple of 4) and the eight
// rows exist, since r0 is a multiple of 8.
__device__ __forceinline__ void load8(const float *zc, int r0, int n, bool ok, bool vec, float *v)
{
    if (ok && vec && r0 + 8 <= n) {
        const float4 a = *reinterpret_cast<const float4 *>(zc + r0);
        const float4 c = *reinterpret_cast<const float4 *>(zc + r0 + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = c.x; v[5] = c.y; v[6] = c.z; v[7] = c.w;
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (ok && r0 + i < n) ? zc[r0 + i] : 0.f;
    }
}

__device__ __forceinline__ void store8(float *zc, int r0, int n, bool ok, bool vec, const float *v)
{
    if (!ok) return;
    if (vec && r0 + 8 <= n) {
        *reinterpret_cast<float4 *>(zc + r0) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(zc + r0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (r0 + i < n) zc[r0 + i] = v[i];
    }
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct ApplyArgs {
    int n, b, jb_lo, jb_hi, k;  // blocks jb_lo <= jb < jb_hi, their groups packed in fac
    long long ldz;
    const float *fac;
    float *z;
    int *status;
};

__global__ void __launch_bounds__(kThreads, 1) q2_apply_tc5_kernel(const ApplyArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((size_t)smem_raw + 1023) & ~(size_t)1023);
    unsigned long long *bars = (unsigned long long *)(smem + kGroupBytes);
    unsigned *tmem_slot = (unsigned *)(bars + 4);
    __shared__ int abort_flag;
    const unsigned bar_v = smem_u32(&bars[0]), bar_w = smem_u32(&bars[1]);
    const unsigned bar_m1 = smem_u32(&bars[2]), bar_m2 = smem_u32(&bars[3]);
    const unsigned sV = smem_u32(smem), sW = sV + 2 * kVPlane;
    const int n = a.n, b = a.b;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, part = warp >> 2;
    const int gc = blockIdx.x * kCols + quarter * 32 + lane;  // column of Z
    const bool colok = gc < a.k;
    float *zc = a.z + (size_t)(colok ? gc : 0) * (size_t)a.ldz;
    const bool vec = (a.ldz & 3) == 0 && (((size_t)a.z) & 15) == 0;

    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(smem_u32(&bars[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;
    const unsigned tq = tmem + ((unsigned)(quarter * 32) << 16);  // this warp's lane quarter

    // outstanding asynchronous operations of thread 0 (for the exit path)
    bool v_out = false, w_out = false, m1_out = false, m2_out = false;
    unsigned gidx = 0;  // groups processed by this CTA (parity of every barrier)

    // packed index of group (jb, 0), kept up to date as jb decreases
    long long gbase = a.jb_hi > a.jb_lo ? group_base(n, b, a.jb_hi - 1) - group_base(n, b, a.jb_lo) : 0;
    auto fac_of = [&](long long g) -> const unsigned char * {
        return reinterpret_cast<const unsigned char *>(a.fac) + (size_t)g * kGroupBytes;
    };
    auto load_v = [&](const unsigned char *g) {
        mbar_expect_tx(bar_v, 2 * kVPlane);
#pragma unroll
        for (int p = 0; p < 4; ++p) bulk_g2s(sV + p * (kVPlane / 2), g + p * (kVPlane / 2), kVPlane / 2, bar_v);
    };
    auto load_w = [&](const unsigned char *g) {
        mbar_expect_tx(bar_w, 2 * kWPlane);
#pragma unroll
        for (int p = 0; p < 4; ++p)
            bulk_g2s(sW + p * (kWPlane / 2), g + 2 * kVPlane + p * (kWPlane / 2), kWPlane / 2, bar_w);
    };
    if (tid == 0 && a.jb_hi > a.jb_lo) {
        const unsigned char *g0 = fac_of(gbase);
        load_v(g0);
        load_w(g0);
        v_out = w_out = true;
    }

    float zr[kSlots];   // slots kSlots * part + i of this thread's column
    float pre[kSlots];  // rows entering the window after the current group
    const unsigned idesc1 = idesc_f32acc(2, 128, 64);
    const unsigned idesc2 = idesc_f32acc(2, 128, 128);
    bool ok = true;

    for (int jb = a.jb_hi - 1; jb >= a.jb_lo && ok; --jb) {
        const int J = jb * kM;
        const int SJ = block_steps(n, b, J);
        // packed index of the group after (jb, t): (jb, t + 1), or (jb - 1, 0) after the last
        const long long gnext_block = jb > a.jb_lo ? gbase - block_steps(n, b, J - kM) : -1;
        // initial window of the block: rows J .. J+127
#pragma unroll
        for (int c = 0; c < kChunks; ++c) {
            const int p = (part * kSlots + c * 8 - J) & (kWin - 1);
            load8(zc, J + p, n, colok, vec, zr + c * 8);
        }
        for (int t = 0; t < SJ; ++t) {
            const int w0 = J + t * b;
            const bool last = t + 1 == SJ;
            // prefetch the rows that replace the ones leaving after this group
            if (!last) {
#pragma unroll
                for (int c = 0; c < kChunks; ++c) {
                    const int p = (part * kSlots + c * 8 - w0) & (kWin - 1);
                    if (p < b) load8(zc, w0 + p + kWin, n, colok, vec, pre + c * 8);
                }
            }
            // ---- A of MMA 1: Z_w^T (hi, lo) at logical window positions
#pragma unroll
            for (int c = 0; c < kChunks; ++c) {
                const unsigned p = (unsigned)((part * kSlots + c * 8 - w0) & (kWin - 1));
                unsigned hi[8], lo[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    hi[i] = tf32_hi(zr[c * 8 + i]);
                    lo[i] = __float_as_uint(zr[c * 8 + i] - __uint_as_float(hi[i]));
                }
                tmem_st8(tq + kZH + p, hi);
                tmem_st8(tq + kZL + p, lo);
            }
            tmem_wait_st();
            tc_fence_before();
            __syncthreads();
            // ---- MMA 1: Y^T = Z_w^T V
            if (tid == 0) {
                if (!mbar_wait(bar_v, gidx & 1)) {
                    report_error(a.status, ELSI_ERR_TIMEOUT, 11);
                    abort_flag = 1;
                } else {
                    v_out = false;
                    tc_fence_after();
                    const unsigned long long dv_h = sdesc(sV), dv_l = sdesc(sV + kVPlane);
#pragma unroll
                    for (int kk = 0; kk < kWin / 8; ++kk) {
                        // the descriptor's start address is in 16-byte units
                        const unsigned boff = ((kk >> 2) * (kM * 128) + (kk & 3) * 32) >> 4;
                        const unsigned long long bh = dv_h + boff, bl = dv_l + boff;
                        const unsigned ah = tmem + kZH + kk * 8, al = tmem + kZL + kk * 8;
                        const unsigned acc = kk > 0 ? 1u : 0u;
                        mma_tf32_ts(tmem + kYAccX, al, bh, idesc1, acc);
                        mma_tf32_ts(tmem + kYAccX, ah, bl, idesc1, 1u);
                        mma_tf32_ts(tmem + kYAccH, ah, bh, idesc1, acc);
                    }
                    mma_commit(bar_m1);
                    m1_out = true;
                }
            }
            __syncthreads();
            if (abort_flag) { ok = false; break; }
            if (!mbar_wait(bar_m1, gidx & 1)) {
                report_error(a.status, ELSI_ERR_TIMEOUT, 12);
                abort_flag = 1;
            }
            tc_fence_after();
            // next group's V (MMA 1 has read the buffer)
            const long long gnext = last ? gnext_block : gbase + t + 1;
            if (tid == 0 && !abort_flag) {
                m1_out = false;
                if (gnext >= 0) { load_v(fac_of(gnext)); v_out = true; }
            }
            // ---- A of MMA 2: Y^T (hi, lo); warp part q takes a = 16 q .. 16 q + 15
            {
                constexpr int kA = kM / kParts;
                float yh[kA], yx[kA];
#pragma unroll
                for (int g = 0; g < kA / 8; ++g) {
                    tmem_ld8(tq + kYAccH + kA * part + 8 * g, yh + 8 * g);
                    tmem_ld8(tq + kYAccX + kA * part + 8 * g, yx + 8 * g);
                }
                tmem_wait_ld();
#pragma unroll
                for (int g = 0; g < kA / 8; ++g) {
                    unsigned hi[8], lo[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float y = yh[g * 8 + i] + yx[g * 8 + i];
                        hi[i] = tf32_hi(y);
                        lo[i] = __float_as_uint(y - __uint_as_float(hi[i]));
                    }
                    tmem_st8(tq + kZH + kA * part + 8 * g, hi);
                    tmem_st8(tq + kZL + kA * part + 8 * g, lo);
                }
            }
            tmem_wait_st();
            tc_fence_before();
            __syncthreads();
            if (abort_flag) { ok = false; break; }
            // ---- MMA 2: dZ^T = Y^T W^T
            if (tid == 0) {
                if (!mbar_wait(bar_w, gidx & 1)) {
                    report_error(a.status, ELSI_ERR_TIMEOUT, 13);
                    abort_flag = 1;
                } else {
                    w_out = false;
                    tc_fence_after();
                    const unsigned long long dw_h = sdesc(sW), dw_l = sdesc(sW + kWPlane);
#pragma unroll
                    for (int kk = 0; kk < kM / 8; ++kk) {
                        const unsigned boff = ((kk >> 2) * (kWin * 128) + (kk & 3) * 32) >> 4;
                        const unsigned long long bh = dw_h + boff, bl = dw_l + boff;
                        const unsigned ah = tmem + kZH + kk * 8, al = tmem + kZL + kk * 8;
                        const unsigned acc = kk > 0 ? 1u : 0u;
                        mma_tf32_ts(tmem + kAccX, al, bh, idesc2, acc);
                        mma_tf32_ts(tmem + kAccX, ah, bl, idesc2, 1u);
                        mma_tf32_ts(tmem + kAccH, ah, bh, idesc2, acc);
                    }
                    mma_commit(bar_m2);
                    m2_out = true;
                }
            }
            __syncthreads();
            if (abort_flag) { ok = false; break; }
            if (!mbar_wait(bar_m2, gidx & 1)) {
                report_error(a.status, ELSI_ERR_TIMEOUT, 14);
                abort_flag = 1;
            }
            tc_fence_after();
            if (tid == 0 && !abort_flag) {
                m2_out = false;
                if (gnext >= 0) { load_w(fac_of(gnext)); w_out = true; }
            }
            // ---- Z_w += dZ (all loads of the thread in flight together)
            {
                float dh[kSlots], dx[kSlots];
#pragma unroll
                for (int c = 0; c < kChunks; ++c) {
                    const unsigned p = (unsigned)((part * kSlots + c * 8 - w0) & (kWin - 1));
                    tmem_ld8(tq + kAccH + p, dh + 8 * c);
                    tmem_ld8(tq + kAccX + p, dx + 8 * c);
                }
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < kSlots; ++i) zr[i] += dh[i] + dx[i];
            }
            tc_fence_before();
            ++gidx;
            // ---- rows leaving the window: store, and take the prefetched rows in their slots
#pragma unroll
            for (int c = 0; c < kChunks; ++c) {
                const int p = (part * kSlots + c * 8 - w0) & (kWin - 1);
                if (last || p < b) {
                    store8(zc, w0 + p, n, colok, vec, zr + c * 8);
                    if (!last) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) zr[c * 8 + i] = pre[c * 8 + i];
                    }
                }
            }
            __syncthreads();
            if (abort_flag) { ok = false; break; }
        }
        gbase = gnext_block;
    }
    // exit: nothing of this CTA may still be in flight when its shared and tensor memory go
    __syncthreads();
    if (tid == 0) {
        const unsigned ph = gidx & 1;
        if (m1_out) mbar_wait(bar_m1, ph);
        if (m2_out) mbar_wait(bar_m2, ph);
        if (v_out) mbar_wait(bar_v, ph);
        if (w_out) mbar_wait(bar_w, ph);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free(tmem, kTmemCols);
}

}  // namespace q2tc

// The operand blocks of all groups take about n^2 / (2 * 64 * b) * 128 KB (4.3 GB at
// n = 16384, b = 64; 26 GB at n = 40000): larger problems are back-transformed a range of
// blocks at a time (one factor and one apply launch per range), with the blocks of a range
// holding at most kFacCapBytes.
constexpr size_t kFacCapBytes = (size_t)6 << 30;

// blocks per range: every range holds at most kFacCapBytes of operand blocks (the largest
// blocks are the first ones, jb = 0)
static int q2_blocks_per_range(int n, int b)
{
    using namespace q2tc;
    const int nblk = (n - 2 + kM - 1) / kM;
    const size_t per_block = (size_t)block_steps(n, b, 0) * kGroupBytes;
    size_t r = kFacCapBytes / (per_block ? per_block : 1);
    if (r < 1) r = 1;
    return (int)(r < (size_t)nblk ? r : (size_t)nblk);
}

size_t q2_factor_elems(int n, int b)
{
    using namespace q2tc;
    if (n < 3) return 1;
    const int nblk = (n - 2 + kM - 1) / kM;
    const int r = q2_blocks_per_range(n, b);
    // the largest range is the one that starts at block 0
    const int hi = r < nblk ? r : nblk;
    return (size_t)group_base(n, b, hi) * kGroupFloats;
}

cudaError_t apply_q2_tc(cudaStream_t st, int n, int b, const float *v2, const float *tau2, int k,
                        float *z, int ldz, float *fac, int *status)
{
    using namespace q2tc;
    if (n < 3 || k <= 0) return cudaSuccess;
    if (b < 8 || b > kM || (b & 7) || ((size_t)fac & 15)) return cudaErrorInvalidValue;
    const int S = sb2st_steps(n, b);
    const int nblk = (n - 2 + kM - 1) / kM;
    const size_t fsmem = (size_t)(4 * kM * (kM + 1) + 2 * kM) * sizeof(float);
    static PerDeviceOnce fattr, aattr;
    cudaError_t e = once_per_device(fattr, [&] {
        return cudaFuncSetAttribute(q2_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
    });
    if (e != cudaSuccess) return e;
    e = once_per_device(aattr, [] {
        return cudaFuncSetAttribute(q2_apply_tc5_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kSmemBytes);
    });
    if (e != cudaSuccess) return e;
    // ranges of blocks from the last (applied first) to the first
    const int per = q2_blocks_per_range(n, b);
    for (int hi = nblk; hi > 0; hi -= per) {
        const int lo = hi - per > 0 ? hi - per : 0;
        EGB_COUNT_LAUNCH();
        q2_factor_kernel<<<dim3(S, hi - lo), 256, fsmem, st>>>(n, b, S, lo, v2, tau2, fac);
        ApplyArgs a;
        a.n = n; a.b = b; a.jb_lo = lo; a.jb_hi = hi; a.k = k; a.ldz = ldz; a.fac = fac; a.z = z;
        a.status = status;
        EGB_COUNT_LAUNCH();
        q2_apply_tc5_kernel<<<ceil_div(k, kCols), kThreads, kSmemBytes, st>>>(a);
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) return le;
    }
    return cudaSuccess;
}

}  // namespace egb

extern "C" size_t elsi_gb_q2_work(int n, int b) { return egb::q2_factor_elems(n, b) + 64; }

extern "C" int elsi_gb_q2_apply_f32(int n, int b, const float *v2, const float *tau2, int k, float *z,
                                    int ldz, float *work, size_t work_elems, int *status, void *stream)
{
    if (n < 1 || k < 0 || ldz < n || !v2 || !tau2 || !z || !work || !status) return ELSI_ERR_ARG;
    if (b < 8 || b > 64 || (b & 7) || work_elems < elsi_gb_q2_work(n, b) - 64) return ELSI_ERR_ARG;
    cudaError_t e = egb::apply_q2_tc((cudaStream_t)stream, n, b, v2, tau2, k, z, ldz, work, status);
    if (e == cudaErrorInvalidValue) return ELSI_ERR_ARG;
    return e == cudaSuccess ? ELSI_OK : ELSI_ERR_CUDA;
}
