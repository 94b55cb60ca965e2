// Dense complex linear algebra for the truncation step (sm_103a, FP32 SIMT).
//
//  * k_gemm: strided complex GEMM, C = alpha * op(A) op(B), 64x64 tiles staged
//    through shared memory.  OUT_ATOMIC64 splits K across blockIdx.z and adds
//    the FP32 chunk results into an FP64 matrix: Gram matrices are accumulated
//    in FP64 while every product stays FP32.
//  * k_eig_jacobi: one-sided (Hestenes) Jacobi on the columns of a Hermitian
//    positive semidefinite r x r matrix G held in shared memory (r <= 160).
//    Columns converge to G V = U diag(lambda); normalised columns are the
//    eigenvectors and their norms the eigenvalues.  Block-cyclic ordering: pairs
//    inside 8-column blocks, then across the blocks of each round-robin block
//    pair, one warp per block (pair) with shuffle reductions and warp-level
//    synchronisation; pairs whose columns have not moved since their last
//    comparison are skipped.
//  * k_select: the truncation rule on the sorted spectrum (FP64 bookkeeping).
#include <math.h>
#include <stdlib.h>

#include <atomic>
#include <climits>

#include "qtn_internal.cuh"

namespace qtn {

// ------------------------------------------------------------------ GEMM
// Tiles of TM x TN outputs, 256 threads each holding RM x RN accumulators, K staged 16 at a time through shared
// memory.  Two shapes: 64 x 64 (the default) and 32 x 32 (four times the CTAs on the small contractions of
// chi <= 32 items, where a 64-wide tile leaves most of its threads idle); the batch tuner picks per workload.
constexpr int GB_K = 16, G_THREADS = 256;

__device__ __forceinline__ float2 mat_get(const Mat& m, int i, int j, long long rs, long long cs, int jdiv,
                                          long long cs_hi) {
    long long off = (long long)i * rs;
    if (jdiv > 0) off += (long long)(j / jdiv) * cs_hi + (long long)(j % jdiv) * cs;
    else off += (long long)j * cs;
    float2 v = m.p[off];
    return m.conj ? cconj(v) : v;
}

template <int TM, int TN, int RM, int RN>
__global__ void __launch_bounds__(G_THREADS) k_gemm_t(GemmDesc d, const int* __restrict__ R) {
    static_assert((TM / RM) * (TN / RN) == G_THREADS, "one accumulator block per thread");
    if (d.guard_reg >= 0 && R[d.guard_reg] != d.guard_val) return;
    const int M = d.M.eval(R), N = d.N.eval(R), K = d.K.eval(R);
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    if (m0 >= M || n0 >= N) return;
    int k_begin = 0, k_end = K;
    if (d.mode == OUT_ATOMIC64) {
        k_begin = blockIdx.z * d.kchunk;
        k_end = min(K, k_begin + d.kchunk);
        if (k_begin >= k_end) return;
    }
    const long long ars = d.A.rs.eval(R), acs = d.A.cs.eval(R);
    const long long brs = d.B.rs.eval(R), bcs = d.B.cs.eval(R);
    const int ajd = d.A.jdiv.eval(R), bjd = d.B.jdiv.eval(R);
    const long long ach = d.A.cs_hi.eval(R), bch = d.B.cs_hi.eval(R);
    const bool a_kfast = (acs == 1);   // K contiguous in A: let consecutive threads walk K
    const bool b_nfast = (bcs == 1);

    __shared__ float2 As[GB_K][TM + 1];
    __shared__ float2 Bs[GB_K][TN + 1];
    const int tid = threadIdx.x;
    const int ty = tid / (TN / RN), tx = tid % (TN / RN);
    float2 acc[RM][RN];
#pragma unroll
    for (int a = 0; a < RM; ++a)
#pragma unroll
        for (int b = 0; b < RN; ++b) acc[a][b] = make_float2(0.f, 0.f);

    for (int k0 = k_begin; k0 < k_end; k0 += GB_K) {
#pragma unroll
        for (int e = tid; e < GB_K * TM; e += G_THREADS) {
            int ii, kk;
            if (a_kfast) { ii = e / GB_K; kk = e % GB_K; } else { ii = e % TM; kk = e / TM; }
            const int gi = m0 + ii, gk = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (gi < M && gk < k_end) v = mat_get(d.A, gi, gk, ars, acs, ajd, ach);
            As[kk][ii] = v;
        }
#pragma unroll
        for (int e = tid; e < GB_K * TN; e += G_THREADS) {
            int jj, kk;
            if (b_nfast) { jj = e % TN; kk = e / TN; } else { jj = e / GB_K; kk = e % GB_K; }
            const int gj = n0 + jj, gk = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (gj < N && gk < k_end) {
                if (d.omega_seed >= 0) v = gauss2(d.omega_seed, gk, gj);
                else v = mat_get(d.B, gk, gj, brs, bcs, bjd, bch);
            }
            Bs[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            float2 av[RM], bv[RN];
#pragma unroll
            for (int a = 0; a < RM; ++a) av[a] = As[kk][ty * RM + a];
#pragma unroll
            for (int b = 0; b < RN; ++b) bv[b] = Bs[kk][tx * RN + b];
#pragma unroll
            for (int a = 0; a < RM; ++a)
#pragma unroll
                for (int b = 0; b < RN; ++b) cfma(acc[a][b], av[a], bv[b]);
        }
        __syncthreads();
    }
    if (d.flops != nullptr && threadIdx.x == 0)
        atomicAdd(d.flops, 8.0 * (double)min(TM, M - m0) * (double)min(TN, N - n0) * (double)(k_end - k_begin));
    const long long crs = d.crs.eval(R), ccs = d.ccs.eval(R);
    const float2 alpha = make_float2(d.alpha_re, d.alpha_im);
#pragma unroll
    for (int a = 0; a < RM; ++a) {
        const int gi = m0 + ty * RM + a;
        if (gi >= M) continue;
#pragma unroll
        for (int b = 0; b < RN; ++b) {
            const int gj = n0 + tx * RN + b;
            if (gj >= N) continue;
            const float2 v = cmul(alpha, acc[a][b]);
            const long long off = (long long)gi * crs + (long long)gj * ccs;
            if (d.mode == OUT_STORE) {
                ((float2*)d.C)[off] = v;
            } else if (d.mode == OUT_ACCUM) {
                float2* c = (float2*)d.C + off;
                *c = cadd(*c, v);
            } else {
                double2* c = (double2*)d.C + off;
                atomicAdd(&c->x, (double)v.x);
                atomicAdd(&c->y, (double)v.y);
            }
        }
    }
}

// GEMM tile of the launches made by the calling host thread (set per context by the entry points).
static thread_local int t_gemm_tile = 64;
static thread_local int t_gemm_sms = 0;       // SMs of the calling context's device (0: never shrink the tile)
void set_gemm_tile(int tile) { t_gemm_tile = (tile == 32) ? 32 : 64; }
void set_gemm_sms(int sms) { t_gemm_sms = sms > 0 ? sms : 0; }
int gemm_tile() { return t_gemm_tile; }

cudaError_t launch_gemm(const GemmDesc& d, int max_m, int max_n, int max_k, const int* R, cudaStream_t s) {
    if (max_m <= 0 || max_n <= 0) return cudaSuccess;
    int T = t_gemm_tile;
    // a 64-wide tiling that leaves most SMs idle (the skinny products of the range finder and the projections)
    // takes the 32-wide tile: four times the CTAs
    if (T == 64 && d.mode != OUT_ATOMIC64 && max_k >= 64 &&
        (long long)((max_n + 63) / 64) * ((max_m + 63) / 64) * 2 < (long long)t_gemm_sms)
        T = 32;
    dim3 grid((max_n + T - 1) / T, (max_m + T - 1) / T, 1);
    if (d.mode == OUT_ATOMIC64) {
        int kc = d.kchunk > 0 ? d.kchunk : 1;
        grid.z = (unsigned)((max(max_k, 1) + kc - 1) / kc);
    }
    GemmDesc dd = d;
    if (g_prof_ledger) dd.flops = g_prof_ledger + L_PROF_GEMM;
    count_launch(PROF_GEMM, s, true);
    if (T == 32) k_gemm_t<32, 32, 2, 2><<<grid, G_THREADS, 0, s>>>(dd, R);
    else k_gemm_t<64, 64, 4, 4><<<grid, G_THREADS, 0, s>>>(dd, R);
    count_launch(PROF_GEMM, s, false);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ one-sided Jacobi eigensolver
constexpr int EIG_THREADS = 1024;
constexpr int EIG_RS = EIG_MAX + 1;             // odd column stride: strided column reads hit distinct banks
constexpr int EIG_CB = 16;                      // columns per block of the re-orthonormalisation
constexpr int EIG_QC = EIG_THREADS / 32;        // finished columns per projection chunk (one per warp)
constexpr float EIG_DEP0 = 1e-3f;               // residual below which a column is dependent (first run)
constexpr float EIG_NOISE = 1.0e-13f;           // |w_i| |w_j| floor (matrix scaled to unit largest diagonal)
// The scaled Gram is stored in FP32, so eigenvalues below ~1e-7 of the largest are rounding.  A sweep that still
// rotates only pairs of columns whose norms (eigenvalues) are not both above EIG_SIG is chasing that rounding
// and does not count as unconverged.
constexpr float EIG_SIG = 1.0e-6f;

__device__ __forceinline__ void circle_pair(int t, int k, int rr, int& i, int& j) {
    // round-robin tournament (circle method) on rr players, round t in [0, rr-2]
    const int m = rr - 1;
    if (k == 0) { i = t; j = m; }
    else { i = (t + k) % m; j = (t - k + m) % m; }
}

// Block-cyclic ordering of a sweep.  Jacobi columns are grouped in blocks of EIG_BS.  A sweep first
// compares the pairs inside every block (one warp per block: EIG_BS - 1 rounds of EIG_BS / 2 pairs, 8 lanes
// per pair) and then, for each round of a round-robin over blocks, the EIG_BS^2 pairs across the two
// blocks of every block pair (one warp per block pair: EIG_BS rounds of the pairs (A_q, B_(q+s) mod EIG_BS),
// 4 lanes per pair).  Every column pair is compared once per sweep at a fixed slot, the rounds inside a
// warp synchronise with __syncwarp, and the block barrier runs once per round of blocks: ~20 barriers per
// sweep at r = 160 instead of r - 1.
constexpr int EIG_BS = 8;

// Shared-memory slot of Jacobi column c.  Inside every complete group of 16 columns the slots are permuted
// so that the 8 columns of a block start 8 banks apart (odd column stride: 2 banks per slot), which keeps
// the 4-lane groups of a warp free of bank conflicts; a trailing partial group keeps its order.  The
// ordering only decides which slots meet when: the eigenvectors are the normalised slots either way.
__device__ __forceinline__ int jacobi_slot(int c, int r16) {
    if (c >= r16) return c;
    const int b = (c >> 3) & 1, q = c & 7;
    return (c & ~15) + 2 * b + 4 * (q & 3) + (q >> 2);
}

// One pair (ci, cj) handled by LPP lanes (lane li of the pair, mask gmask): the inner product from LPP rows
// in flight four times over, a shuffle reduction, and, when the pair is not orthogonal to tol, the rotation
// with the squared norms carried.  Slot g of the sweep's SL slots: when neither column has rotated since
// this pair's comparison one sweep ago (tmod = slot of a column's last rotation), that comparison found the
// pair orthogonal and would return the same inner product (only the norms are refreshed each sweep), so it
// is skipped.  Every early return is uniform over the pair's lanes.
template <int LPP>
__device__ __forceinline__ void jacobi_pair(float2* __restrict__ W, float* __restrict__ cn2, int* __restrict__ tmod,
                                            int r, int r16, int col_i, int col_j, int li, unsigned gmask, int g, int SL,
                                            bool first_sweep, float tol, int* rotated, int* sig_rotated,
                                            unsigned long long& my_pairs, unsigned long long& my_rot) {
    if (col_i >= r || col_j >= r) return;
    const int si = jacobi_slot(col_i, r16), sj = jacobi_slot(col_j, r16);
    if (!first_sweep && max(tmod[si], tmod[sj]) < g - SL) return;
    float2* wi = W + si * EIG_RS;
    float2* wj = W + sj * EIG_RS;
    float cr0 = 0.f, ci0 = 0.f, cr1 = 0.f, ci1 = 0.f;   // four chains, eight loads in flight
    float cr2 = 0.f, ci2 = 0.f, cr3 = 0.f, ci3 = 0.f;
    int row = li;
    for (; row + 3 * LPP < r; row += 4 * LPP) {
        const float2 x0 = wi[row], y0 = wj[row], x1 = wi[row + LPP], y1 = wj[row + LPP];
        const float2 x2 = wi[row + 2 * LPP], y2 = wj[row + 2 * LPP];
        const float2 x3 = wi[row + 3 * LPP], y3 = wj[row + 3 * LPP];
        cr0 = fmaf(x0.x, y0.x, fmaf(x0.y, y0.y, cr0));    // conj(x) * y
        ci0 = fmaf(x0.x, y0.y, fmaf(-x0.y, y0.x, ci0));
        cr1 = fmaf(x1.x, y1.x, fmaf(x1.y, y1.y, cr1));
        ci1 = fmaf(x1.x, y1.y, fmaf(-x1.y, y1.x, ci1));
        cr2 = fmaf(x2.x, y2.x, fmaf(x2.y, y2.y, cr2));
        ci2 = fmaf(x2.x, y2.y, fmaf(-x2.y, y2.x, ci2));
        cr3 = fmaf(x3.x, y3.x, fmaf(x3.y, y3.y, cr3));
        ci3 = fmaf(x3.x, y3.y, fmaf(-x3.y, y3.x, ci3));
    }
    for (; row < r; row += LPP) {
        const float2 x0 = wi[row], y0 = wj[row];
        cr0 = fmaf(x0.x, y0.x, fmaf(x0.y, y0.y, cr0));
        ci0 = fmaf(x0.x, y0.y, fmaf(-x0.y, y0.x, ci0));
    }
    float cr = (cr0 + cr1) + (cr2 + cr3), ci = (ci0 + ci1) + (ci2 + ci3);
#pragma unroll
    for (int off = LPP / 2; off > 0; off >>= 1) {
        cr += __shfl_xor_sync(gmask, cr, off);
        ci += __shfl_xor_sync(gmask, ci, off);
    }
    if (li == 0) ++my_pairs;
    const float a = cn2[si], b = cn2[sj];
    const float c2 = fmaf(cr, cr, ci * ci);
    const float ab2 = a * b;
    // Columns of the scaled matrix whose norms are both below the FP32 resolution of G are round-off:
    // rotating them never converges and they are orthonormalised afterwards.
    if (!(c2 > tol * tol * ab2) || !(c2 > 0.f) || !(ab2 > EIG_NOISE * EIG_NOISE)) return;
    const float ic = rsqrtf(c2), cabs = c2 * ic;
    const float zeta = 0.5f * (b - a) * ic;
    const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
    const float cs = rsqrtf(fmaf(tt, tt, 1.f));
    const float tc = tt * cs * ic;
    const float pr = tc * cr, pi = tc * ci;                             // p = sin(theta) e
    // x' = cs x - conj(p) y ;  y' = p x + cs y
    int rw = li;
    for (; rw + 3 * LPP < r; rw += 4 * LPP) {
        float2 x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { x[u] = wi[rw + u * LPP]; y[u] = wj[rw + u * LPP]; }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            wi[rw + u * LPP] = make_float2(fmaf(cs, x[u].x, -fmaf(pr, y[u].x, pi * y[u].y)),
                                           fmaf(cs, x[u].y, -fmaf(pr, y[u].y, -pi * y[u].x)));
            wj[rw + u * LPP] = make_float2(fmaf(cs, y[u].x, fmaf(pr, x[u].x, -pi * x[u].y)),
                                           fmaf(cs, y[u].y, fmaf(pr, x[u].y, pi * x[u].x)));
        }
    }
    for (; rw < r; rw += LPP) {
        const float2 x = wi[rw], y = wj[rw];
        wi[rw] = make_float2(fmaf(cs, x.x, -fmaf(pr, y.x, pi * y.y)), fmaf(cs, x.y, -fmaf(pr, y.y, -pi * y.x)));
        wj[rw] = make_float2(fmaf(cs, y.x, fmaf(pr, x.x, -pi * x.y)), fmaf(cs, y.y, fmaf(pr, x.y, pi * x.x)));
    }
    if (li == 0) {
        cn2[si] = fmaxf(a - tt * cabs, 0.f);
        cn2[sj] = b + tt * cabs;
        tmod[si] = g;
        tmod[sj] = g;
        *rotated = 1;
        if (ab2 > EIG_SIG * EIG_SIG) *sig_rotated = 1;
        ++my_rot;
    }
}

// The cross-block pair (ci, cj) split over the three warps of a block pair: warp `sub` owns the rows
// [r0, r1) and its 4-lane group (lane li, mask gmask) the rows r0 + li, r0 + li + 4, ...  Each warp adds its
// partial inner product into part[sub][q], the three warps meet at named barrier bar_id (96 threads), every
// warp forms the same total (fixed summation order) and the same rotation and rotates its own rows; warp 0
// keeps the carried norms, slots and flags, and a second barrier ends the step.  The skip test of
// jacobi_pair reads slots written before the previous step's second barrier, so the three warps always take
// the same branch.
__device__ __forceinline__ void bar_named(int id, int count) {
    __syncwarp();
    asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void jacobi_pair3(float2* __restrict__ W, float* __restrict__ cn2, int* __restrict__ tmod,
                                             float2* __restrict__ part, int r, int r16, int col_i, int col_j, int q,
                                             int li, unsigned gmask, int sub, int r0, int r1, int bar_id, int g,
                                             int SL, bool first_sweep, float tol, int* rotated, int* sig_rotated,
                                             unsigned long long& my_pairs, unsigned long long& my_rot) {
    bool skip = !(col_i < r && col_j < r);
    int si = 0, sj = 0;
    if (!skip) {
        si = jacobi_slot(col_i, r16);
        sj = jacobi_slot(col_j, r16);
        if (!first_sweep && max(tmod[si], tmod[sj]) < g - SL) skip = true;
    }
    float2* wi = W + si * EIG_RS;
    float2* wj = W + sj * EIG_RS;
    float cr = 0.f, ci = 0.f;
    if (!skip) {
        float cr1 = 0.f, ci1 = 0.f;
        int row = r0 + li;
        for (; row + 4 < r1; row += 8) {
            const float2 x0 = wi[row], y0 = wj[row], x1 = wi[row + 4], y1 = wj[row + 4];
            cr = fmaf(x0.x, y0.x, fmaf(x0.y, y0.y, cr));      // conj(x) * y
            ci = fmaf(x0.x, y0.y, fmaf(-x0.y, y0.x, ci));
            cr1 = fmaf(x1.x, y1.x, fmaf(x1.y, y1.y, cr1));
            ci1 = fmaf(x1.x, y1.y, fmaf(-x1.y, y1.x, ci1));
        }
        if (row < r1) {
            const float2 x0 = wi[row], y0 = wj[row];
            cr = fmaf(x0.x, y0.x, fmaf(x0.y, y0.y, cr));
            ci = fmaf(x0.x, y0.y, fmaf(-x0.y, y0.x, ci));
        }
        cr += cr1;
        ci += ci1;
        cr += __shfl_xor_sync(gmask, cr, 2);
        ci += __shfl_xor_sync(gmask, ci, 2);
        cr += __shfl_xor_sync(gmask, cr, 1);
        ci += __shfl_xor_sync(gmask, ci, 1);
    }
    if (li == 0) part[sub * EIG_BS + q] = make_float2(cr, ci);
    bar_named(bar_id, 96);
    if (!skip) {
        const float2 p0 = part[q], p1 = part[EIG_BS + q], p2 = part[2 * EIG_BS + q];
        cr = (p0.x + p1.x) + p2.x;
        ci = (p0.y + p1.y) + p2.y;
        const bool lead = (sub == 0 && li == 0);
        if (lead) ++my_pairs;
        const float a = cn2[si], b = cn2[sj];
        const float c2 = fmaf(cr, cr, ci * ci);
        const float ab2 = a * b;
        if (c2 > tol * tol * ab2 && c2 > 0.f && ab2 > EIG_NOISE * EIG_NOISE) {
            const float ic = rsqrtf(c2), cabs = c2 * ic;
            const float zeta = 0.5f * (b - a) * ic;
            const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
            const float cs = rsqrtf(fmaf(tt, tt, 1.f));
            const float tc = tt * cs * ic;
            const float pr = tc * cr, pi = tc * ci;
            for (int rw = r0 + li; rw < r1; rw += 4) {
                const float2 x = wi[rw], y = wj[rw];
                wi[rw] = make_float2(fmaf(cs, x.x, -fmaf(pr, y.x, pi * y.y)), fmaf(cs, x.y, -fmaf(pr, y.y, -pi * y.x)));
                wj[rw] = make_float2(fmaf(cs, y.x, fmaf(pr, x.x, -pi * x.y)), fmaf(cs, y.y, fmaf(pr, x.y, pi * x.x)));
            }
            if (lead) {
                cn2[si] = fmaxf(a - tt * cabs, 0.f);
                cn2[sj] = b + tt * cabs;
                tmod[si] = g;
                tmod[sj] = g;
                *rotated = 1;
                if (ab2 > EIG_SIG * EIG_SIG) *sig_rotated = 1;
                ++my_rot;
            }
        }
    }
    bar_named(bar_id, 96);
}

// After the sweeps: eigenvalues from the column norms (FP64 accumulation), the columns re-orthonormalised
// in descending-eigenvalue order and completed, U and lam written (all r x r of W in this CTA's shared memory,
// column j at W + j * EIG_RS, in the units of the scaled Gram).
__device__ void eig_finish(float2* __restrict__ W, int r, double gscale, float2* __restrict__ U, long long ldu,
                           double* __restrict__ lam, float dead_rel) {
    __shared__ double nrm[EIG_MAX];
    __shared__ int rank_of[EIG_MAX];
    __shared__ double nmax_s;
    const int tid = threadIdx.x;
    // eigenvalues = column norms (FP64 accumulation), eigenvectors = normalised columns
    for (int j = tid / 32; j < r; j += EIG_THREADS / 32) {
        double s = 0.0;
        for (int row = tid % 32; row < r; row += 32) {
            float2 x = W[j * EIG_RS + row];
            s += (double)x.x * x.x + (double)x.y * x.y;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (tid % 32 == 0) nrm[j] = sqrt(s) * gscale;
    }
    __syncthreads();
    for (int j = tid; j < r; j += EIG_THREADS) {
        double v = nrm[j];
        int rk = 0;
        for (int i = 0; i < r; ++i) {
            double u = nrm[i];
            rk += (u > v) || (u == v && i < j);
        }
        rank_of[j] = rk;
        lam[rk] = v;
        if (rk == 0) nmax_s = v;
    }
    __syncthreads();
    // Re-orthonormalise the columns in descending-eigenvalue order: Jacobi leaves the directions below the
    // FP32 resolution of G non-orthogonal, and the new site must be an isometry.  Blocks of EIG_CB unit
    // columns are projected on the finished columns and orthonormalised internally by Cholesky QR; a second
    // run restores what cancellation took from the first, when some column lost more than 30 % of itself.
    // A column whose eigenvalue is below dead_rel of the largest carries no direction (its column of G V is
    // round-off) and is not processed; a column whose residual falls below EIG_DEP0 in the first run, or
    // loses half of itself in the second, is numerically dependent.  Both are set aside and replaced at the
    // end by completion vectors orthonormalised the same way, so the basis stays complete and no weight of
    // the factorised matrix is lost.
    __shared__ int col_of_rank[EIG_MAX];
    __shared__ unsigned char dead[EIG_MAX];          // by rank
    __shared__ float invn[EIG_MAX];
    __shared__ __align__(16) float2 Cs[EIG_QC * EIG_CB];   // projection coefficients (finished chunk x block)
    __shared__ float2 Rb[EIG_CB * EIG_CB];           // Gram of the block, overwritten by its Cholesky factor
    __shared__ unsigned char bdead[EIG_CB];
    __shared__ int nlive_s, npre_s;
    __shared__ int again_s;                           // the block needs its second run
    __shared__ float lev[EIG_MAX];                    // leverage of each row over the live columns
    const int warp = tid / 32, wl = tid % 32;
    for (int j = tid; j < r; j += EIG_THREADS) {
        col_of_rank[rank_of[j]] = j;
        const double nj = nrm[j] / gscale;           // column norm in the units of W
        invn[j] = nj > 0.0 ? (float)(1.0 / nj) : 0.f;
        dead[rank_of[j]] = !(nj > 0.0) || nrm[j] < (double)dead_rel * nmax_s;
    }
    __syncthreads();
    // dead ranks form a suffix (ranks descend with the eigenvalue): the first of them ends the main pass
    if (tid == 0) npre_s = r;
    __syncthreads();
    for (int t = tid; t < r; t += EIG_THREADS)
        if (dead[t] && (t == 0 || !dead[t - 1])) npre_s = t;
    __syncthreads();
    const int npre = npre_s;
    for (int e = tid; e < r * r; e += EIG_THREADS) {
        const int j = e / r, row = e % r;
        W[j * EIG_RS + row] = cscale(W[j * EIG_RS + row], invn[j]);
    }
    __syncthreads();
    auto ortho_block = [&](int t0, int nb) {
        for (int pass = 0; pass < 2; ++pass) {
            // projection on the finished columns (ranks < t0), EIG_QC of them at a time
            for (int qc = 0; qc < t0; qc += EIG_QC) {
                const int nq = min(EIG_QC, t0 - qc);
                // coefficients Cs[q][c] = <finished q, block column c>: warp w takes the finished columns 2w and
                // 2w + 1 (read once per row for both), lane (c, h) the block column c and every other row
                if (warp < (nq + 1) / 2) {
                    const int q0 = 2 * warp, q1 = q0 + 1;
                    const bool two = q1 < nq;
                    const float2* f0 = W + col_of_rank[qc + q0] * EIG_RS;
                    const float2* f1 = W + col_of_rank[qc + (two ? q1 : q0)] * EIG_RS;
                    const int c = wl & 15, h = wl >> 4;
                    float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;   // two chains per column
                    if (c < nb) {
                        const float2* wc = W + col_of_rank[t0 + c] * EIG_RS;
                        int row = h;
                        for (; row + 2 < r; row += 4) {
                            const float2 y0 = wc[row], y1 = wc[row + 2];
                            const float2 x0 = f0[row], x1 = f0[row + 2], z0 = f1[row], z1 = f1[row + 2];
                            a0.x = fmaf(x0.x, y0.x, fmaf(x0.y, y0.y, a0.x));   // conj(x) * y
                            a0.y = fmaf(x0.x, y0.y, fmaf(-x0.y, y0.x, a0.y));
                            a1.x = fmaf(x1.x, y1.x, fmaf(x1.y, y1.y, a1.x));
                            a1.y = fmaf(x1.x, y1.y, fmaf(-x1.y, y1.x, a1.y));
                            b0.x = fmaf(z0.x, y0.x, fmaf(z0.y, y0.y, b0.x));
                            b0.y = fmaf(z0.x, y0.y, fmaf(-z0.y, y0.x, b0.y));
                            b1.x = fmaf(z1.x, y1.x, fmaf(z1.y, y1.y, b1.x));
                            b1.y = fmaf(z1.x, y1.y, fmaf(-z1.y, y1.x, b1.y));
                        }
                        for (; row < r; row += 2) {
                            const float2 y0 = wc[row], x0 = f0[row], z0 = f1[row];
                            a0.x = fmaf(x0.x, y0.x, fmaf(x0.y, y0.y, a0.x));
                            a0.y = fmaf(x0.x, y0.y, fmaf(-x0.y, y0.x, a0.y));
                            b0.x = fmaf(z0.x, y0.x, fmaf(z0.y, y0.y, b0.x));
                            b0.y = fmaf(z0.x, y0.y, fmaf(-z0.y, y0.x, b0.y));
                        }
                        a0.x += a1.x; a0.y += a1.y;
                        b0.x += b1.x; b0.y += b1.y;
                    }
                    a0.x += __shfl_xor_sync(0xffffffffu, a0.x, 16);
                    a0.y += __shfl_xor_sync(0xffffffffu, a0.y, 16);
                    b0.x += __shfl_xor_sync(0xffffffffu, b0.x, 16);
                    b0.y += __shfl_xor_sync(0xffffffffu, b0.y, 16);
                    if (h == 0 && c < nb) {
                        Cs[q0 * EIG_CB + c] = a0;
                        if (two) Cs[q1 * EIG_CB + c] = b0;
                    }
                }
                __syncthreads();
                // block -= finished Cs: thread (g, row) updates block columns 4g .. 4g + 3 of one row, reading each
                // finished entry once
                for (int e = tid; e < r * (EIG_CB / 4); e += EIG_THREADS) {
                    const int g = e / r, row = e - g * r;
                    const int c0 = 4 * g;
                    if (c0 >= nb) continue;
                    float2 acc[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        acc[u] = (c0 + u < nb) ? W[col_of_rank[t0 + c0 + u] * EIG_RS + row] : make_float2(0.f, 0.f);
                    for (int q = 0; q < nq; ++q) {
                        const float2 f = W[col_of_rank[qc + q] * EIG_RS + row];
                        const float4 k01 = *reinterpret_cast<const float4*>(&Cs[q * EIG_CB + c0]);
                        const float4 k23 = *reinterpret_cast<const float4*>(&Cs[q * EIG_CB + c0 + 2]);
                        acc[0].x -= f.x * k01.x - f.y * k01.y;
                        acc[0].y -= f.x * k01.y + f.y * k01.x;
                        acc[1].x -= f.x * k01.z - f.y * k01.w;
                        acc[1].y -= f.x * k01.w + f.y * k01.z;
                        acc[2].x -= f.x * k23.x - f.y * k23.y;
                        acc[2].y -= f.x * k23.y + f.y * k23.x;
                        acc[3].x -= f.x * k23.z - f.y * k23.w;
                        acc[3].y -= f.x * k23.w + f.y * k23.z;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (c0 + u < nb) W[col_of_rank[t0 + c0 + u] * EIG_RS + row] = acc[u];
                }
                __syncthreads();
            }
            // Gram of the block (upper triangle), one warp per entry
            for (int p = warp; p < nb * nb; p += EIG_THREADS / 32) {
                const int c1 = p / nb, c2 = p % nb;
                if (c2 < c1) continue;
                const float2* x = W + col_of_rank[t0 + c1] * EIG_RS;
                const float2* y = W + col_of_rank[t0 + c2] * EIG_RS;
                float sr = 0.f, si = 0.f;
                for (int row = wl; row < r; row += 32) {
                    const float2 u = x[row], v = y[row];
                    sr = fmaf(u.x, v.x, fmaf(u.y, v.y, sr));
                    si = fmaf(u.x, v.y, fmaf(-u.y, v.x, si));
                }
                for (int off = 16; off > 0; off >>= 1) {
                    sr += __shfl_xor_sync(0xffffffffu, sr, off);
                    si += __shfl_xor_sync(0xffffffffu, si, off);
                }
                if (wl == 0) Rb[c1 * EIG_CB + c2] = make_float2(sr, si);
            }
            __syncthreads();
            // Cholesky factor (upper, row c of Rb), right-looking, one warp: the pivot is the diagonal of the
            // updated trailing Gram and the trailing update is spread over the lanes.  A pivot below the
            // threshold marks the column dependent (first run: relative residual EIG_DEP0 of a unit column;
            // second run: half of it).
            if (warp == 0) {
                const float thr2 = pass == 0 ? EIG_DEP0 * EIG_DEP0 : 0.25f;
                bool heavy = false;
                for (int c = 0; c < nb; ++c) {
                    const float d = Rb[c * EIG_CB + c].x;
                    const bool dc = bdead[c] || !(d > thr2);
                    heavy = heavy || (!dc && d < 0.5f);   // a live column lost more than 30 % of its norm
                    __syncwarp();
                    if (dc) {
                        if (wl >= c && wl < nb) Rb[c * EIG_CB + wl] = make_float2(0.f, 0.f);
                        if (wl == 0) bdead[c] = 1;
                        __syncwarp();
                        continue;
                    }
                    const float rcc = sqrtf(d), inv = 1.f / rcc;
                    if (wl > c && wl < nb) Rb[c * EIG_CB + wl] = cscale(Rb[c * EIG_CB + wl], inv);
                    if (wl == c) Rb[c * EIG_CB + c] = make_float2(rcc, 0.f);
                    __syncwarp();
                    // trailing block, upper triangle: lane wl owns entries wl + 32 u of the EIG_CB x EIG_CB array
#pragma unroll
                    for (int u8 = 0; u8 < EIG_CB * EIG_CB / 32; ++u8) {
                        const int e = wl + 32 * u8, i2 = e / EIG_CB, i3 = e % EIG_CB;
                        if (i2 > c && i3 >= i2 && i3 < nb) {
                            const float2 u = Rb[c * EIG_CB + i2], v = Rb[c * EIG_CB + i3];   // conj(u) * v
                            float2 g = Rb[e];
                            g.x -= u.x * v.x + u.y * v.y;
                            g.y -= u.x * v.y - u.y * v.x;
                            Rb[e] = g;
                        }
                    }
                    __syncwarp();
                }
                if (wl == 0) again_s = heavy ? 1 : 0;
            }
            __syncthreads();
            // block <- block R^{-1} by forward substitution in place, one row per thread (dependent columns
            // become zero)
            for (int row = tid; row < r; row += EIG_THREADS) {
                for (int c = 0; c < nb; ++c) {
                    float2* wc = W + col_of_rank[t0 + c] * EIG_RS + row;
                    float2 v = *wc, v1 = make_float2(0.f, 0.f);
                    int k = 0;
                    for (; k + 1 < c; k += 2) {
                        const float2 x0 = W[col_of_rank[t0 + k] * EIG_RS + row], r0 = Rb[k * EIG_CB + c];
                        const float2 x1 = W[col_of_rank[t0 + k + 1] * EIG_RS + row], r1 = Rb[(k + 1) * EIG_CB + c];
                        v.x -= x0.x * r0.x - x0.y * r0.y;
                        v.y -= x0.x * r0.y + x0.y * r0.x;
                        v1.x -= x1.x * r1.x - x1.y * r1.y;
                        v1.y -= x1.x * r1.y + x1.y * r1.x;
                    }
                    if (k < c) {
                        const float2 xk = W[col_of_rank[t0 + k] * EIG_RS + row], rk = Rb[k * EIG_CB + c];
                        v.x -= xk.x * rk.x - xk.y * rk.y;
                        v.y -= xk.x * rk.y + xk.y * rk.x;
                    }
                    v = make_float2(v.x + v1.x, v.y + v1.y);
                    *wc = bdead[c] ? make_float2(0.f, 0.f) : cscale(v, 1.f / Rb[c * EIG_CB + c].x);
                }
            }
            __syncthreads();
            // without cancellation in the first run the block is orthonormal to working precision already
            // (Cholesky QR of a well-conditioned block); the second run is for blocks that lost digits
            if (pass == 0 && !again_s) break;
        }
    };
    for (int t0 = 0; t0 < npre; t0 += EIG_CB) {
        const int nb = min(EIG_CB, r - t0);
        if (tid < EIG_CB) bdead[tid] = (tid < nb) ? dead[t0 + tid] : 1;
        __syncthreads();
        ortho_block(t0, nb);
        if (tid < nb) dead[t0 + tid] = bdead[tid];
        __syncthreads();
    }
    // Completion: dependent ranks move to the end (stable) and are replaced by unit vectors e_k of the rows
    // least covered by the live columns (smallest leverage sum_t |w_t(k)|^2), which are nearly orthogonal to
    // them, so one Cholesky-QR run usually suffices; any completion vector that turns out dependent is
    // replaced by a pseudo-random vector in a second attempt.
    int neig = r;                                     // live eigen-columns (ranks below carry eigenvalues)
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (tid == 0) {                               // rank_of serves as scratch; it is rewritten below
            int nl = 0;
            for (int t = 0; t < r; ++t)
                if (!dead[t]) rank_of[nl++] = col_of_rank[t];
            int nd = nl;
            for (int t = 0; t < r; ++t)
                if (dead[t]) rank_of[nd++] = col_of_rank[t];
            for (int t = 0; t < r; ++t) {
                col_of_rank[t] = rank_of[t];
                dead[t] = (t >= nl);
            }
            nlive_s = nl;
        }
        __syncthreads();
        const int nlive = nlive_s;
        if (attempt == 0) neig = nlive;
        if (nlive == r) break;
        if (attempt == 0) {
            for (int row = tid; row < r; row += EIG_THREADS) {
                float l = 0.f;
                for (int t = 0; t < nlive; ++t) {
                    const float2 v = W[col_of_rank[t] * EIG_RS + row];
                    l = fmaf(v.x, v.x, fmaf(v.y, v.y, l));
                }
                lev[row] = l;
            }
            for (int e = tid; e < (r - nlive) * r; e += EIG_THREADS)
                W[col_of_rank[nlive + e / r] * EIG_RS + e % r] = make_float2(0.f, 0.f);
            __syncthreads();
            for (int row = tid; row < r; row += EIG_THREADS) {
                const float l = lev[row];
                int rk = 0;
                for (int i = 0; i < r; ++i) {
                    const float u = lev[i];
                    rk += (u < l) || (u == l && i < row);
                }
                if (rk < r - nlive) W[col_of_rank[nlive + rk] * EIG_RS + row] = make_float2(1.f, 0.f);
            }
        } else {
            for (int t = nlive + warp; t < r; t += EIG_THREADS / 32) {
                float2* w = W + col_of_rank[t] * EIG_RS;
                float ss = 0.f;
                for (int row = wl; row < r; row += 32) {
                    const float2 v = gauss2(977 + t, row, t);
                    w[row] = v;
                    ss = fmaf(v.x, v.x, fmaf(v.y, v.y, ss));
                }
                for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
                const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
                for (int row = wl; row < r; row += 32) w[row] = cscale(w[row], inv);
            }
        }
        __syncthreads();
        for (int t0 = nlive; t0 < r; t0 += EIG_CB) {
            const int nb = min(EIG_CB, r - t0);
            if (tid < EIG_CB) bdead[tid] = (tid < nb) ? 0 : 1;
            __syncthreads();
            ortho_block(t0, nb);
            if (tid < nb) dead[t0 + tid] = bdead[tid];
            __syncthreads();
        }
    }
    for (int t = tid; t < r; t += EIG_THREADS) {
        const int j = col_of_rank[t];
        rank_of[j] = t;
        lam[t] = (t < neig) ? nrm[j] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < r * r; e += EIG_THREADS) {
        int j = e / r, row = e % r;
        U[(long long)rank_of[j] * ldu + row] = W[j * EIG_RS + row];
    }
}

__global__ void __launch_bounds__(EIG_THREADS, 1)
k_eig_jacobi(const double2* __restrict__ G, Dim ldd, Dim rdim, float2* __restrict__ U, Dim ldud,
             double* __restrict__ lam, const int* Rc, int* Rw, int max_sweeps,   // Rc, Rw: one register array
             double* __restrict__ ledger, int guard_reg, int guard_val, double* __restrict__ prof, float tol,
             float dead_rel, int report_nonconv, int r_limit) {
    if (guard_reg >= 0 && Rc[guard_reg] != guard_val) return;
    extern __shared__ float2 W[];                // column-major, W[j*EIG_RS + i]
    __shared__ int rotated, sig_rotated;
    const int r = rdim.eval(Rc);
    const long long ld = ldd.eval(Rc), ldu = ldud.eval(Rc);
    if (r <= 0 || r >= r_limit) return;   // r >= r_limit: solved by the cluster kernel
    __shared__ double gscale;
    __shared__ unsigned long long n_pairs, n_rot;
    const int tid = threadIdx.x;
    if (tid == 0) { n_pairs = 0ull; n_rot = 0ull; }
    // Scale by the largest diagonal entry so that squared column norms stay inside the FP32 range
    // (one-sided Jacobi on a Gram matrix works with fourth powers of the singular values).
    if (tid < 32) {
        double mx = 0.0;
        for (int i = tid; i < r; i += 32) mx = fmax(mx, fabs(G[(long long)i * ld + i].x));
        for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        if (tid == 0) gscale = (mx > 0.0 && isfinite(mx)) ? mx : 1.0;
    }
    __syncthreads();
    const double inv_scale = 1.0 / gscale;
    for (int e = tid; e < r * r; e += EIG_THREADS) {
        int i = e / r, j = e % r;                // G row-major; W column j holds G[:, j] / scale
        double2 g = G[(long long)i * ld + j];
        W[j * EIG_RS + i] = make_float2((float)(g.x * inv_scale), (float)(g.y * inv_scale));
    }
    __syncthreads();

    // squared column norms, exact at the start of every sweep and carried through each rotation by
    // |x'|^2 = |x|^2 - t |c|, |y'|^2 = |y|^2 + t |c|, so a pair needs only its inner product
    __shared__ float cn2[EIG_MAX];
    unsigned long long my_pairs = 0ull, my_rot = 0ull;
    __shared__ int tmod[EIG_MAX];                // slot of the last rotation of each column (by shared slot)
    __shared__ float2 part[(EIG_MAX / EIG_BS / 2) * 3 * EIG_BS];   // partial inner products per block pair
    for (int j = tid; j < r; j += EIG_THREADS) tmod[j] = -1;
    const int nblk = (r + EIG_BS - 1) / EIG_BS, nbr = nblk + (nblk & 1);
    const int SL = (EIG_BS - 1) + (nbr - 1) * EIG_BS;   // comparison slots per sweep
    const int r16 = r & ~15;
    const int warp_j = tid / 32, lane_j = tid % 32;
    int sweep = 0;
    bool converged = (r < 2);
    for (; sweep < max_sweeps && !converged; ++sweep) {
        if (tid == 0) { rotated = 0; sig_rotated = 0; }
        for (int j = tid / 32; j < r; j += EIG_THREADS / 32) {
            float s2 = 0.f;
            for (int row = tid % 32; row < r; row += 32) {
                const float2 x = W[j * EIG_RS + row];
                s2 = fmaf(x.x, x.x, fmaf(x.y, x.y, s2));
            }
            for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
            if (tid % 32 == 0) cn2[j] = s2;
        }
        __syncthreads();
        const int g0 = sweep * SL;
        if (warp_j < nblk) {                     // pairs inside block warp_j
            const int k = lane_j >> 3, li = lane_j & 7;
            const unsigned gmask = 0xFFu << (8 * k);
            for (int u = 0; u < EIG_BS - 1; ++u) {
                int a, b;
                circle_pair(u, k, EIG_BS, a, b);
                jacobi_pair<8>(W, cn2, tmod, r, r16, warp_j * EIG_BS + a, warp_j * EIG_BS + b, li, gmask, g0 + u, SL,
                               sweep == 0, tol, &rotated, &sig_rotated, my_pairs, my_rot);
                __syncwarp();
            }
        }
        __syncthreads();
        for (int t = 0; t < nbr - 1; ++t) {      // pairs across the blocks of every block pair of round t
            const int bp = warp_j / 3, sub = warp_j % 3;   // three warps per block pair, a third of the rows each
            if (bp < nbr / 2) {
                int A, B;
                circle_pair(t, bp, nbr, A, B);
                const int q = lane_j >> 2, li = lane_j & 3;
                const unsigned gmask = 0xFu << (4 * q);
                const int rt = (r + 2) / 3, r0 = min(r, sub * rt), r1 = min(r, r0 + rt);
                for (int s2 = 0; s2 < EIG_BS; ++s2)
                    jacobi_pair3(W, cn2, tmod, part + bp * 3 * EIG_BS, r, r16, A * EIG_BS + q,
                                 B * EIG_BS + ((q + s2) & (EIG_BS - 1)), q, li, gmask, sub, r0, r1, 1 + bp,
                                 g0 + (EIG_BS - 1) + t * EIG_BS + s2, SL, sweep == 0, tol, &rotated, &sig_rotated,
                                 my_pairs, my_rot);
            }
            __syncthreads();
        }
        converged = (rotated == 0);
        __syncthreads();
    }
    if (prof != nullptr && (my_pairs | my_rot)) {
        atomicAdd(&n_pairs, my_pairs);
        atomicAdd(&n_rot, my_rot);
    }
    eig_finish(W, r, gscale, U, ldu, lam, dead_rel);
    if (tid == 0) {
        atomicMax(&Rw[R_SWEEPS], sweep);
        // unconverged only when the last sweep still rotated a pair above the rounding level of the scaled Gram
        if (!converged && report_nonconv && sig_rotated) raise_flag(Rw, F_NOCONV);
        // algorithmic FLOPs: 8 per row for the inner product of a pair, 24 per row for a rotation,
        // 8 r^3 for the re-orthonormalisation (projections and Cholesky QR, complex)
        if (prof != nullptr)
            atomicAdd(prof, 8.0 * r * (double)n_pairs + 24.0 * r * (double)n_rot + 8.0 * (double)r * r * r);
    }
}

// Eigenvectors of the rotated columns of W left in U by the cluster sweeps (column j at U + j ldu, in the units of
// G / s, s the largest diagonal entry of G): the same finishing step as k_eig_jacobi, on one CTA.
__global__ void __launch_bounds__(EIG_THREADS, 1)
k_eig_finish(const double2* __restrict__ G, Dim ldd, Dim rdim, float2* U, Dim ldud, double* __restrict__ lam,
             const int* __restrict__ Rc, int guard_reg, int guard_val, float dead_rel, int r_min,
             double* __restrict__ prof) {
    if (guard_reg >= 0 && Rc[guard_reg] != guard_val) return;
    const int r = rdim.eval(Rc);
    if (r < r_min || r < 2 || r > EIG_MAX) return;
    extern __shared__ float2 W[];
    __shared__ double gscale;
    const long long ld = ldd.eval(Rc), ldu = ldud.eval(Rc);
    const int tid = threadIdx.x;
    if (tid < 32) {
        double mx = 0.0;
        for (int i = tid; i < r; i += 32) mx = fmax(mx, fabs(G[(long long)i * ld + i].x));
        for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        if (tid == 0) gscale = (mx > 0.0 && isfinite(mx)) ? mx : 1.0;
    }
    for (int e = tid; e < r * r; e += EIG_THREADS) {
        const int j = e / r, i = e - j * r;
        W[j * EIG_RS + i] = U[(long long)j * ldu + i];
    }
    __syncthreads();
    eig_finish(W, r, gscale, U, ldu, lam, dead_rel);
    if (prof != nullptr && tid == 0) atomicAdd(prof, 8.0 * (double)r * r * r);
}

cudaError_t launch_eig_finish(const double2* G, Dim ld, Dim r, float2* U, Dim ldu, double* lam, const int* R,
                              cudaStream_t s, int guard_reg, int guard_val, float dead_rel, int r_min) {
    const size_t smem = (size_t)EIG_MAX * EIG_RS * sizeof(float2);
    double* prof = g_prof_ledger ? g_prof_ledger + L_PROF_EIG : nullptr;
    k_eig_finish<<<1, EIG_THREADS, smem, s>>>(G, ld, r, U, ldu, lam, R, guard_reg, guard_val, dead_rel, r_min, prof);
    return cudaGetLastError();
}

cudaError_t launch_eig(const double2* G, Dim ld, Dim r, float2* U, Dim ldu, double* lam, const int* R,
                       int r_cap, int max_sweeps, double* ledger, cudaStream_t s, int guard_reg, int guard_val,
                       float tol, float dead_rel, bool report_nonconv,
                       bool rough_basis) {
    const size_t smem = (size_t)EIG_MAX * EIG_RS * sizeof(float2);
    double* prof = g_prof_ledger ? g_prof_ledger + L_PROF_EIG : nullptr;
    // r at or above the cluster threshold: the sweeps run on the cluster kernel (k_eig_cluster.cu).  A rough first
    // solve whose basis a refinement corrects (rough_basis) takes its eigenvectors from rotations accumulated into
    // an orthonormal basis; otherwise the eigenvectors are the normalised columns of G V (the product with G filters
    // the rounding-level mixing of directions whose eigenvalues are near the FP32 resolution of G), orthonormalised
    // in descending order by k_eig_finish on one CTA.  Below the threshold everything runs in one CTA
    // (k_eig_jacobi).  When the capacity allows either, both paths are launched and the one whose range does not
    // hold the live r returns at once.
    const int r_min = eig_cluster_min();
    const bool cl = (r_cap >= r_min);
    count_launch(PROF_EIG, s, true);
    k_eig_jacobi<<<1, EIG_THREADS, smem, s>>>(G, ld, r, U, ldu, lam, R, (int*)R, max_sweeps, ledger, guard_reg,
                                               guard_val, prof, tol, dead_rel, report_nonconv ? 1 : 0,
                                               cl ? r_min : INT_MAX);
    count_launch(PROF_EIG, s, false);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !cl) return e;
    count_launch(PROF_EIG, s, true);
    e = launch_eig_cluster(G, ld, r, U, ldu, lam, R, max_sweeps, s, guard_reg, guard_val, prof, tol, report_nonconv,
                           r_min, rough_basis);
    count_launch(PROF_EIG, s, false);
    if (e != cudaSuccess || rough_basis) return e;
    count_launch(PROF_EIG, s, true);
    e = launch_eig_finish(G, ld, r, U, ldu, lam, R, s, guard_reg, guard_val, dead_rel, r_min);
    count_launch(PROF_EIG, s, false);
    return e;
}

// Smallest live r solved by the cluster kernel (process-wide).
static std::atomic<int> g_eig_cluster_min{32};
int eig_cluster_min() { return g_eig_cluster_min.load(std::memory_order_relaxed); }
void set_eig_cluster_min(int r) { g_eig_cluster_min.store(r < 2 ? 2 : r, std::memory_order_relaxed); }

// ------------------------------------------------------------------ launch accounting / profiling
double* g_prof_ledger = nullptr;
static std::atomic<long long> g_launches{0};   // host threads may drive several contexts at once
static bool g_prof_on = false;
struct ProfPool {
    cudaEvent_t* ev = nullptr;   // pairs (start, stop)
    int cap = 0, used = 0;
    long long launches = 0;
    double ms = 0.0;             // durations of the pairs already drained
};
static ProfPool g_pool[PROF_NCLASS];

// Adds the durations of the recorded pairs to p.ms and frees the pool (waits for the last stop event).
static void prof_drain(ProfPool& p) {
    if (p.used >= 2) cudaEventSynchronize(p.ev[p.used - 1]);
    for (int i = 0; i + 1 < p.used; i += 2) {
        float e = 0.f;
        if (cudaEventElapsedTime(&e, p.ev[i], p.ev[i + 1]) == cudaSuccess) p.ms += e;
    }
    p.used = 0;
}

void count_launch(int cls, cudaStream_t s, bool before) {
    if (!before) g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_prof_on || cls == PROF_OTHER) return;
    // launches recorded into a graph are not timed here (an event node cannot sit in a conditional body)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    ProfPool& p = g_pool[cls];
    if (before) {
        if (p.used + 2 > p.cap) prof_drain(p);   // every launch is timed: a full pool is drained, not skipped
        cudaEventRecord(p.ev[p.used], s);
    } else {
        cudaEventRecord(p.ev[p.used + 1], s);
        p.used += 2;
        ++p.launches;
    }
}

long long launch_total() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void prof_begin(bool on, double* ledger) {
    g_prof_on = on;
    g_prof_ledger = on ? ledger : nullptr;
    for (int c = 0; c < PROF_NCLASS; ++c) {
        ProfPool& p = g_pool[c];
        if (on && p.ev == nullptr && c != PROF_OTHER) {
            p.cap = 1 << 16;
            p.ev = new cudaEvent_t[p.cap];
            for (int i = 0; i < p.cap; ++i) cudaEventCreate(&p.ev[i]);
        }
        p.used = 0;
        p.launches = 0;
        p.ms = 0.0;
    }
}

// Total device time (ms) and launch count of one kernel class since prof_begin.
void prof_read(int cls, double* ms, long long* launches) {
    ProfPool& p = g_pool[cls];
    prof_drain(p);
    *ms = p.ms;
    *launches = p.launches;
}

// ------------------------------------------------------------------ per-device kernel attributes
cudaError_t configure_eig_kernel() {
    cudaError_t e = cudaFuncSetAttribute(k_eig_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((size_t)EIG_MAX * EIG_RS * sizeof(float2)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_eig_finish, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)EIG_MAX * EIG_RS * sizeof(float2)));
    if (e == cudaSuccess) e = configure_eig_cluster_kernel();
    return e;
}

}  // namespace qtn
