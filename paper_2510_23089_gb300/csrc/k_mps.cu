// Site-level kernels of the zip-up sweep, encoder, MPO builders and contractions.
//
// Sweep orientation: a right-to-left pass is a left-to-right pass over the
// mirrored chain (sites reversed, left/right bonds swapped).  Kernels take a
// `mirror` flag and read/write the physical padded layout accordingly, so no
// site is ever copied to change orientation.
#include <math.h>

#include "qtn_internal.cuh"

namespace qtn {

// ------------------------------------------------------------------ planning

// Dimensions of zip-up site p (sweep order) -> dimension registers.
__global__ void k_plan_site(const int* __restrict__ bond, const int* __restrict__ mbond, int N, int d, int mirror,
                           int moff, int mn, int p, int* __restrict__ R) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int q = mirror ? N - 1 - p : p;
    const int chiL = (p == 0) ? 1 : R[R_CHIR];
    const int chiLn = (p == 0) ? 1 : R[R_K];
    const int wl = (p == 0) ? 1 : R[R_WR];
    const int chiR = mirror ? bond[q] : bond[q + 1];
    const int qm = q - moff;
    int wr = 1;
    if (mbond != nullptr && qm >= 0 && qm < mn) wr = mirror ? mbond[qm] : mbond[qm + 1];
    R[R_CHILN] = chiLn;
    R[R_CHIL] = chiL;
    R[R_CHIR] = chiR;
    R[R_WL] = wl;
    R[R_WR] = wr;
    R[R_M] = chiLn * d;
    R[R_N] = wr * chiR;
    R[R_MID] = chiLn * wl;
    R[R_DN] = d * chiR;
    R[R_LAST] = (p == N - 1);
    R[R_P] = min(chiLn * d, EIG_MAX);
}

// Encoder bond p: rows = previous rank * d, columns fixed by the host.
__global__ void k_plan_encode(int p, int d, int* __restrict__ R) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int r = (p == 0) ? 1 : R[R_K];
    R[R_CHILN] = r;
    R[R_M] = r * d;
    R[R_P] = min(r * d, EIG_MAX);
}

__global__ void k_reset_stats(int* __restrict__ R, double* __restrict__ ledger) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        R[R_SWEEPS] = 0;
        R[R_FLAGS] = 0;
        R[R_MAXBOND] = 0;
        R[R_K] = 1;
        R[R_CHIR] = 1;
        R[R_WR] = 1;
        // the profiling counters (L_PROF_GEMM onwards) accumulate across calls until qtn_profile resets them
        for (int i = 0; i < L_PROF_GEMM; ++i) ledger[i] = 0.0;
    }
}

// ------------------------------------------------------------------ contraction, second stage
// T[(x, t'), (b, k)] = sum_{a, t} P[(x, a), (t, k)] W[a, t', t, b] with the MPO acting on one bit of the
// physical index (d = 4: bit `axis` selects x = high or y = low; the other bit passes through).
__global__ void k_stage2(const float2* __restrict__ P, float2* __restrict__ T, const float2* __restrict__ Wc,
                         int wcap, int mirror, int d, int axis, const int* __restrict__ R) {
    const int chiLn = R[R_CHILN], wl = R[R_WL], wr = R[R_WR], chiR = R[R_CHIR];
    const int m = chiLn * d, n = wr * chiR;
    const long long total = (long long)m * n;
    const int dn = d * chiR;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(e / n), col = (int)(e % n);
        const int x = row / d, sp = row % d;
        const int b = col / chiR, k = col % chiR;
        if (Wc == nullptr) {
            T[e] = P[(long long)x * dn + sp * chiR + k];
            continue;
        }
        if (axis >= 2) {   // elementwise product with an MPS (the "MPO" is diagonal in the whole site index)
            float2 acc = make_float2(0.f, 0.f);
            for (int a = 0; a < wl; ++a) {
                float2 w = mirror ? Wc[((long long)b * d + sp) * wcap + a] : Wc[((long long)a * d + sp) * wcap + b];
                if (axis == 3) w.y = -w.y;
                cfma(acc, P[(long long)(x * wl + a) * dn + sp * chiR + k], w);
            }
            T[e] = acc;
            continue;
        }
        int t, so;
        if (d == 2) { t = sp; so = 0; }
        else if (axis == 0) { t = sp >> 1; so = sp & 1; }
        else { t = sp & 1; so = sp >> 1; }
        float2 acc = make_float2(0.f, 0.f);
        for (int a = 0; a < wl; ++a) {
            const float2* prow = P + (long long)(x * wl + a) * dn;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int sf = (d == 2) ? s : (axis == 0 ? ((s << 1) | so) : ((so << 1) | s));
                const float2 w = mirror ? Wc[((b * 2 + t) * 2 + s) * wcap + a] : Wc[((a * 2 + t) * 2 + s) * wcap + b];
                cfma(acc, prow[sf * chiR + k], w);
            }
        }
        T[e] = acc;
    }
}

// ------------------------------------------------------------------ truncation bookkeeping

// Trace of an FP64 Gram matrix (total weight of the factorised matrix) -> ledger[L_TRACE].
__global__ void k_trace(const double2* __restrict__ G, int ld, Dim rdim, int* __restrict__ R,
                        double* __restrict__ ledger) {
    if (R[R_RAND] != 0) return;
    const int r = rdim.eval(R);
    double s = 0.0;
    for (int i = threadIdx.x; i < r; i += blockDim.x) s += G[(long long)i * ld + i].x;
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
        ledger[L_TRACE] = t;
    }
}

// Path of the factorisation of an m-row matrix: the shared-memory eigensolver when m <= EIG_MAX, else the
// range finder on an EIG_MAX-column sketch.
__global__ void k_path(Dim mdim, int* __restrict__ R, double* __restrict__ ledger) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int m = mdim.eval(R);
    ledger[L_TRACE] = 0.0;
    R[R_RAND] = (m > EIG_MAX) ? 1 : 0;
    R[R_P] = min(m, EIG_MAX);
    R[R_ROWS] = min(m, EIG_MAX);
    R[R_DEP] = 0;
    R[R_PI] = 0;
}

// The power iteration of the range finder runs only for a full-rank sketch: when the sketch already has
// dependent columns, the rank of T is below the subspace size and the sketch spans the range of T.
__global__ void k_set_pi(int* __restrict__ R) {
    if (threadIdx.x == 0 && blockIdx.x == 0) R[R_PI] = (R[R_RAND] == 1 && R[R_DEP] == 0) ? 1 : 0;
}

// |T|_F^2 in FP64 accumulated into ledger[L_TRACE] (range-finder path: the total weight of the factorised
// matrix; L_TRACE is zeroed by k_path).
__global__ void k_total_weight(const float2* __restrict__ T, Dim ldt, Dim mdim, Dim ndim, const int* __restrict__ R,
                               double* __restrict__ ledger) {
    if (R[R_RAND] != 1) return;
    const int m = mdim.eval(R), n = ndim.eval(R);
    const long long ld = ldt.eval(R);
    double s = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)m * n;
         e += (long long)gridDim.x * blockDim.x) {
        const float2 v = T[(e / n) * ld + (e % n)];
        s += (double)v.x * v.x + (double)v.y * v.y;
    }
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
        atomicAdd(&ledger[L_TRACE], t);
    }
}

// Orthonormalise columns [c0, c0 + CGS_B) of the row-major m x ld matrix Q among themselves with classical
// Gram-Schmidt applied twice, in shared memory (m <= CGS_MAXM).  A column that is numerically dependent
// (residual below 1e-5 of its norm) is set to zero.  The columns are assumed already orthogonal to the
// columns before c0 (projected out by the caller).

// Column norms of a row-major m x ld matrix (columns [0, ncols)) -> out (FP32 norms).
__global__ void k_col_norms(const float2* __restrict__ Q, int ld, Dim mdim, Dim ncols, float* __restrict__ out,
                            const int* __restrict__ R, int greg) {
    if (R[greg] != 1) return;
    const int m = mdim.eval(R), nc = ncols.eval(R);
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < nc; c += nwarps) {
        float s = 0.f;
        for (int row = lane; row < m; row += 32) {
            const float2 v = Q[(long long)row * ld + c];
            s = fmaf(v.x, v.x, fmaf(v.y, v.y, s));
        }
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) out[c] = sqrtf(s);
    }
}

// Orthonormalisation of one block of NB columns against each other (classical Gram-Schmidt, two passes),
// after the block has been projected against the finished blocks.  The range finder runs it twice per
// block (block CGS2): the first run (decide = 1) finds dependent columns, the second (decide = 0), after a
// second projection against the finished blocks, restores orthogonality lost to the cancellation in the
// first.  pre[c]: norm of column c before any projection; in the first run a column whose residual falls
// below CGS_DEP of it is numerically dependent on the columns already orthonormalised, is set to zero and
// raises R[R_DEP].  The block runs only when R[greg] == 1.
constexpr float CGS_DEP = 1e-5f;

template <int NB, int MAXM>
__device__ __forceinline__ void cgs_block_body(float2* __restrict__ Q, int ld, Dim mdim, int c0, int ncols,
                                               const float* __restrict__ pre, int* __restrict__ R, int greg,
                                               int decide) {
    if (R[greg] != 1 || c0 >= ncols) return;
    const int nb = min(NB, ncols - c0);        // columns of this block inside the first ncols
    extern __shared__ float2 S[];              // column-major, S[c * MAXM + row]
    __shared__ float cr_s[NB], ci_s[NB], red[32];
    __shared__ float nrm;
    const int m = mdim.eval(R);
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    for (int e = tid; e < m * nb; e += blockDim.x) {
        const int row = e / nb, c = e % nb;
        S[c * MAXM + row] = Q[(long long)row * ld + c0 + c];
    }
    __syncthreads();
    auto norm_of = [&](const float2* w) {
        float ss = 0.f;
        for (int row = tid; row < m; row += blockDim.x) ss += w[row].x * w[row].x + w[row].y * w[row].y;
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
        if (lane == 0) red[warp] = ss;
        __syncthreads();
        if (tid == 0) {
            float t = 0.f;
            for (int q = 0; q < (int)blockDim.x / 32; ++q) t += red[q];
            nrm = sqrtf(t);
        }
        __syncthreads();
        return nrm;
    };
    bool dep = false;
    for (int c = 0; c < nb; ++c) {
        float2* w = S + c * MAXM;
        const float nraw = norm_of(w);
        // first run: dependent on the finished blocks when the projection left less than CGS_DEP of the
        // column; second run: the column was a unit vector, so a re-projection that removes half of it means
        // the first result was rounding, not a direction (Kahan-Parlett "twice is enough")
        const float n0 = decide ? ((nraw > CGS_DEP * pre[c0 + c]) ? nraw : 0.f) : ((nraw > 0.5f) ? nraw : 0.f);
        const float inv0 = n0 > 0.f ? 1.f / n0 : 0.f;
        for (int row = tid; row < m; row += blockDim.x) w[row] = cscale(w[row], inv0);
        __syncthreads();
        float a1 = 1.f, na = 0.f;
        for (int pass = 0; pass < 2 && n0 > 0.f; ++pass) {
            for (int q = warp; q < c; q += blockDim.x / 32) {
                const float2* u = S + q * MAXM;
                float ar = 0.f, ai = 0.f;
                for (int row = lane; row < m; row += 32) {
                    const float2 a = u[row], b = w[row];
                    ar = fmaf(a.x, b.x, fmaf(a.y, b.y, ar));
                    ai = fmaf(a.x, b.y, fmaf(-a.y, b.x, ai));
                }
                for (int off = 16; off > 0; off >>= 1) {
                    ar += __shfl_xor_sync(0xffffffffu, ar, off);
                    ai += __shfl_xor_sync(0xffffffffu, ai, off);
                }
                if (lane == 0) { cr_s[q] = ar; ci_s[q] = ai; }
            }
            __syncthreads();
            for (int row = tid; row < m; row += blockDim.x) {
                float2 acc = w[row];
                for (int q = 0; q < c; ++q) {
                    const float2 u = S[q * MAXM + row];
                    acc.x -= cr_s[q] * u.x - ci_s[q] * u.y;
                    acc.y -= cr_s[q] * u.y + ci_s[q] * u.x;
                }
                w[row] = acc;
            }
            __syncthreads();
            if (pass == 0) a1 = norm_of(w);
            else na = norm_of(w);
        }
        // the second in-block pass must not cancel either: otherwise the residual is rounding
        const float sc = (n0 > 0.f && na > CGS_DEP && na > 0.5f * a1) ? 1.f / na : 0.f;
        if (!(sc > 0.f) && (decide ? pre[c0 + c] > 0.f : nraw > 0.f)) dep = true;
        for (int row = tid; row < m; row += blockDim.x) w[row] = cscale(w[row], sc);
        __syncthreads();
    }
    if (tid == 0 && dep) R[R_DEP] = 1;
    for (int e = tid; e < m * nb; e += blockDim.x) {
        const int row = e / nb, c = e % nb;
        Q[(long long)row * ld + c0 + c] = S[c * MAXM + row];
    }
}

__global__ void __launch_bounds__(1024) k_cgs_block_32(float2* Q, int ld, Dim mdim, int c0, int ncols, const float* pre,
                                                      int* R, int greg, int decide) {
    cgs_block_body<32, 512>(Q, ld, mdim, c0, ncols, pre, R, greg, decide);
}
__global__ void __launch_bounds__(1024) k_cgs_block_16(float2* Q, int ld, Dim mdim, int c0, int ncols, const float* pre,
                                                      int* R, int greg, int decide) {
    cgs_block_body<16, 1024>(Q, ld, mdim, c0, ncols, pre, R, greg, decide);
}
__global__ void __launch_bounds__(1024) k_cgs_block_8(float2* Q, int ld, Dim mdim, int c0, int ncols, const float* pre,
                                                      int* R, int greg, int decide) {
    cgs_block_body<8, 2048>(Q, ld, mdim, c0, ncols, pre, R, greg, decide);
}

// Range finder with a rank-deficient sketch (R_DEP = 1): the block Gram-Schmidt left the dependent columns of
// the m x ld basis exactly zero.  k_sketch_live finds the live columns (one CTA), keeps their order, and makes
// their count the subspace size of everything that follows (R_P, and R_ROWS for the refinement); k_sketch_gather
// moves them to the front (reading a copy), so the Rayleigh-Ritz problem shrinks from EIG_MAX to the rank.
__global__ void k_sketch_live(const float2* __restrict__ Y, int ld, Dim mdim, int pc, int* __restrict__ perm,
                              int* __restrict__ R) {
    if (!(R[R_RAND] == 1 && R[R_DEP] == 1)) return;
    const int m = mdim.eval(R);
    __shared__ int live[1024];
    for (int c = threadIdx.x; c < pc; c += blockDim.x) {
        int nz = 0;
        for (int row = 0; row < m && !nz; ++row) {
            const float2 v = Y[(long long)row * ld + c];
            nz = (v.x != 0.f || v.y != 0.f);
        }
        live[c] = nz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int k = 0;
        for (int c = 0; c < pc; ++c)
            if (live[c]) perm[k++] = c;
        const int nl = max(k, 1);
        for (int c = 0; c < pc; ++c)
            if (!live[c] && k < pc) perm[k++] = c;
        R[R_P] = nl;
        R[R_ROWS] = nl;
    }
}

__global__ void k_sketch_gather(const float2* __restrict__ src, float2* __restrict__ Y, int ld, Dim mdim, int pc,
                                const int* __restrict__ perm, const int* __restrict__ R) {
    if (!(R[R_RAND] == 1 && R[R_DEP] == 1)) return;
    const int m = mdim.eval(R);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)m * pc;
         e += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(e / pc), j = (int)(e % pc);
        Y[(long long)row * ld + j] = src[(long long)row * ld + perm[j]];
    }
}

// Newton-Schulz coefficient matrix E = (3 I - S) / 2 of an FP64 Gram S = U^dagger U (r x r, row-major),
// rounded to FP32 (entries near 1 on the diagonal, near 0 off it).
__global__ void k_ns_coeff(const double2* __restrict__ S, int lds, float2* __restrict__ E, int lde, Dim rdim,
                           const int* __restrict__ R) {
    const int r = rdim.eval(R);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)r * r;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / r), j = (int)(e % r);
        const double2 v = S[(long long)i * lds + j];
        E[(long long)i * lde + j] = make_float2((float)((i == j ? 1.5 : 0.0) - 0.5 * v.x), (float)(-0.5 * v.y));
    }
}

// Guarded copy of n elements (runs when R[greg] == gval).
__global__ void k_copy_guarded(const float2* __restrict__ src, float2* __restrict__ dst, long long n,
                               const int* __restrict__ R, int greg, int gval) {
    if (R[greg] != gval) return;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dst[e] = src[e];
}

// Squared norms of the rows of X (FP64 accumulation): w[i] = sum_c |X[i, c]|^2.
__global__ void k_row_weights(const float2* __restrict__ X, Dim ldx, Dim rows, Dim cols, double* __restrict__ w,
                              const int* __restrict__ R) {
    const int r = rows.eval(R), n = cols.eval(R);
    const long long ld = ldx.eval(R);
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < r; i += nwarps) {
        double s = 0.0;
        const float2* row = X + (long long)i * ld;
        for (int c = lane; c < n; c += 32) {
            float2 v = row[c];
            s += (double)v.x * v.x + (double)v.y * v.y;
        }
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) w[i] = s;
    }
}

// Truncation rule on projected weights (FP64): sort descending, keep the smallest k >= 1 whose discarded
// weight is <= cutoff * total, cap by chi_max and the capacity.  The discarded weight is the sum of the
// weights left out, accumulated directly from the smallest upwards (suffix sums), never the difference
// total - kept: that difference carries the FP32 rounding of every projected weight (~1e-7 of the total),
// which would swamp cutoffs near 1e-10.  On the range-finder path with a full-rank sketch the weight of T
// outside the sketch, |T|^2 - sum of captured weights (L_TRACE holds |T|^2), is part of every tail; when the
// sketch has dependent columns it spans the range of T and that difference is rounding only.
// Writes perm[0..k), R[R_K], ledger[L_DISCARDED] += discarded.
__global__ void k_select(const double* __restrict__ w, Dim rdim, int chi_max, double cutoff, int chi_cap,
                         int unused, int* __restrict__ perm, int* __restrict__ R, double* __restrict__ ledger) {
    (void)unused;
    __shared__ double sorted_w[1024];
    __shared__ double tail[1025];
    const int r = rdim.eval(R);
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        const double v = w[j];
        int rk = 0;
        for (int i = 0; i < r; ++i) {
            const double u = w[i];
            rk += (u > v) || (u == v && i < j);
        }
        sorted_w[rk] = v;
        perm[rk] = j;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tail[r] = 0.0;
        for (int i = r - 1; i >= 0; --i) tail[i] = tail[i + 1] + fmax(sorted_w[i], 0.0);
        const double wsum = tail[0];
        const bool full_sketch = (R[R_RAND] == 1 && R[R_DEP] == 0);
        const double outside = full_sketch ? fmax(ledger[L_TRACE] - wsum, 0.0) : 0.0;
        const double total = wsum + outside;
        // directions whose captured weight is below NULL_FLOOR * total are numerically null for FP32 data
        // (singular value below ~3e-7 of the norm, a few FP32 ulps): they are never kept, whatever the cutoff
        const double NULL_FLOOR = 1e-13;
        int k = 1;
        while (k < r && tail[k] + outside > cutoff * total && sorted_w[k] > NULL_FLOOR * total) ++k;
        // a rank can never exceed the smaller dimension of the factorised matrix
        const int rank_bound = min(R[R_M], R[R_N]);
        int kk = min(min(k, chi_max), max(rank_bound, 1));
        // the rule asks for more directions than the bond can hold: clamp and report, never silently
        if (kk > chi_cap) { kk = chi_cap; raise_flag(R, F_CAPACITY); }
        ledger[L_DISCARDED] += tail[kk] + outside;
        if (!isfinite(total) || !isfinite(ledger[L_TRACE])) raise_flag(R, F_NONFINITE);
        R[R_K] = kk;
        R[R_MAXBOND] = max(R[R_MAXBOND], kk);
    }
}

// New site from kept left singular vectors: site[(x, t), j] = U[perm[j]][(x, t)] (U column-major), written
// in the physical layout of the sweep orientation; also stores the new bond.
__global__ void k_write_site(const float2* __restrict__ U, int ldu, const int* __restrict__ perm,
                             float2* __restrict__ site, int cap, int d, int mirror, int* __restrict__ bond,
                             int bond_index, const int* __restrict__ R) {
    const int chiLn = R[R_CHILN], k = R[R_K];
    const int total = chiLn * d * k;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int x = e / (d * k), t = (e / k) % d, j = e % k;
        const float2 v = U[(long long)perm[j] * ldu + x * d + t];
        if (mirror) site[((long long)j * d + t) * cap + x] = v;
        else site[((long long)x * d + t) * cap + j] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) bond[bond_index] = k;
}

// Carry rows in kept order: C[j, :] = X[perm[j], :].
__global__ void k_gather_rows(const float2* __restrict__ X, Dim ldx, const int* __restrict__ perm,
                              float2* __restrict__ C, Dim ldc, Dim cols, const int* __restrict__ R) {
    const int k = R[R_K], n = cols.eval(R);
    const long long lx = ldx.eval(R), lc = ldc.eval(R);
    const long long total = (long long)k * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / n), c = (int)(e % n);
        C[(long long)j * lc + c] = X[(long long)perm[j] * lx + c];
    }
}

// Last site of a sweep: the whole (x, t) column of T (n = 1) becomes the site.
__global__ void k_write_last(const float2* __restrict__ T, float2* __restrict__ site, int cap, int d, int mirror,
                             const int* __restrict__ R) {
    const int chiLn = R[R_CHILN];
    for (int e = threadIdx.x; e < chiLn * d; e += blockDim.x) {
        const int x = e / d, t = e % d;
        if (mirror) site[(long long)t * cap + x] = T[e];
        else site[((long long)x * d + t) * cap] = T[e];
    }
}

// Squared Frobenius norm of a padded site (l < bl, r < br) -> ledger[slot] (FP64).
__global__ void k_site_norm2(const float2* __restrict__ site, int cap, int d, const int* __restrict__ bond, int q,
                             double* __restrict__ ledger, int slot) {
    const int bl = bond[q], br = bond[q + 1];
    const int total = bl * d * br;
    double s = 0.0;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int l = e / (d * br), t = (e / br) % d, r = e % br;
        const float2 v = site[((long long)l * d + t) * cap + r];
        s += (double)v.x * v.x + (double)v.y * v.y;
    }
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
        ledger[slot] = t;
    }
}

// Convert an FP64 matrix to FP32 (r x r, same leading dimension).
__global__ void k_to_f32(const double2* __restrict__ G, float2* __restrict__ G32, int ld, Dim rdim,
                         const int* __restrict__ R) {
    if (R[R_RAND] != 1) return;
    const int r = rdim.eval(R);
    const long long total = (long long)r * r;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / r), j = (int)(e % r);
        const double2 g = G[(long long)i * ld + j];
        G32[(long long)i * ld + j] = make_float2((float)g.x, (float)g.y);
    }
}

// Whitening of an eigenbasis: Z[:, j] /= sqrt(lam_j), zeroed below floor * lam_0 (lam sorted descending).
__global__ void k_whiten(float2* __restrict__ Z, int ldz, const double* __restrict__ lam, Dim rdim, double floor_rel,
                         const int* __restrict__ R) {
    if (R[R_RAND] != 1) return;
    const int r = rdim.eval(R);
    const double l0 = lam[0];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x) {
        const int j = e / r, i = e % r;
        const double l = lam[j];
        const float s = (l > floor_rel * l0 && l > 0.0) ? (float)(1.0 / sqrt(l)) : 0.f;
        float2* z = Z + (long long)j * ldz + i;
        *z = cscale(*z, s);
    }
}

// ------------------------------------------------------------------ quantics permutations

__device__ __forceinline__ unsigned compact_bits(unsigned long long v, int n) {
    // gather bits 0, 2, 4, ... of v (n of them) into an integer
    unsigned out = 0;
    for (int i = 0; i < n; ++i) out |= (unsigned)((v >> (2 * i)) & 1ull) << i;
    return out;
}

// dense (row-major L x L, or 2^n vector for 1D) -> quantics-ordered vector; a NaN or Inf entry raises the
// non-finite flag in R
__global__ void k_dense_to_quantics(const float2* __restrict__ dense, float2* __restrict__ out, int n, int layout,
                                    int* __restrict__ R) {
    const long long total = (layout == QTN_LAYOUT_1D) ? (1ll << n) : (1ll << (2 * n));
    bool bad = false;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        float2 v;
        if (layout == QTN_LAYOUT_INTERLEAVED) {
            const unsigned a = compact_bits((unsigned long long)idx >> 1, n);
            const unsigned b = compact_bits((unsigned long long)idx, n);
            v = dense[((long long)a << n) | b];
        } else {
            v = dense[idx];
        }
        bad = bad || !isfinite(v.x) || !isfinite(v.y);
        out[idx] = v;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0 && R != nullptr) raise_flag(R, F_NONFINITE);
}

__global__ void k_quantics_to_dense(const float2* __restrict__ q, float2* __restrict__ dense, int n, int layout) {
    const long long total = (layout == QTN_LAYOUT_1D) ? (1ll << n) : (1ll << (2 * n));
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        if (layout == QTN_LAYOUT_INTERLEAVED) {
            const unsigned a = compact_bits((unsigned long long)idx >> 1, n);
            const unsigned b = compact_bits((unsigned long long)idx, n);
            dense[((long long)a << n) | b] = q[idx];
        } else {
            dense[idx] = q[idx];
        }
    }
}

// ------------------------------------------------------------------ MPO construction

// Hermitian conjugate of MPO cores: out[a, t, s, b] = conj(in[a, s, t, b]).
__global__ void k_mpo_dagger(const float2* __restrict__ in, const int* __restrict__ ibond, int icap,
                             float2* __restrict__ out, int* __restrict__ obond, int ocap, int n) {
    const int p = blockIdx.x;
    if (p >= n) return;
    const int bl = ibond[p], br = ibond[p + 1];
    const float2* a = in + (long long)p * icap * 4 * icap;
    float2* w = out + (long long)p * ocap * 4 * ocap;
    for (int e = threadIdx.x; e < bl * 4 * br; e += blockDim.x) {
        const int l = e / (4 * br), ts = (e / br) % 4, r = e % br;
        const int t = ts >> 1, s = ts & 1;
        w[((long long)l * 4 + ts) * ocap + r] = cconj(a[((long long)l * 4 + s * 2 + t) * icap + r]);
    }
    if (threadIdx.x == 0) {
        obond[p] = bl;
        if (p == n - 1) obond[n] = br;
    }
}

// ------------------------------------------------------------------ amplitudes and overlaps

// psi[digits] for `count` digit strings: one warp per string, row vector times site matrices.
__global__ void k_amplitudes(const float2* __restrict__ sites, const int* __restrict__ bond, int N, int d, int cap,
                             const int* __restrict__ digits, int count, float2* __restrict__ out,
                             float2* __restrict__ scratch) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= count) return;
    float2* v = scratch + (long long)warp * 2 * cap;
    float2* vn = v + cap;
    if (lane == 0) v[0] = make_float2(1.f, 0.f);
    __syncwarp();
    for (int p = 0; p < N; ++p) {
        const int bl = bond[p], br = bond[p + 1];
        const int s = digits[(long long)warp * N + p];
        const float2* A = sites + (long long)p * cap * d * cap;
        for (int r = lane; r < br; r += 32) {
            float2 acc = make_float2(0.f, 0.f);
            for (int l = 0; l < bl; ++l) cfma(acc, v[l], A[((long long)l * d + s) * cap + r]);
            vn[r] = acc;
        }
        __syncwarp();
        for (int r = lane; r < br; r += 32) v[r] = vn[r];
        __syncwarp();
    }
    if (lane == 0) out[warp] = v[0];
}

// Left transfer-matrix step of <a|b>: E'[k, l] = sum_{i, j, s} conj(A[i, s, k]) E[i, j] B[j, s, l], FP64 E.
// One block per output row k; threads over l.
__global__ void k_transfer_step(const double2* __restrict__ E, int lde, const float2* __restrict__ A, int acap,
                                int abl, int abr, const float2* __restrict__ B, int bcap, int bbl, int bbr, int d,
                                double2* __restrict__ En) {
    const int k = blockIdx.x;
    if (k >= abr) return;
    for (int l = threadIdx.x; l < bbr; l += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int s = 0; s < d; ++s) {
            for (int j = 0; j < bbl; ++j) {
                // t_j = sum_i conj(A[i, s, k]) E[i, j]
                double tr = 0.0, ti = 0.0;
                for (int i = 0; i < abl; ++i) {
                    const float2 a = A[((long long)i * d + s) * acap + k];
                    const double2 e = E[(long long)i * lde + j];
                    tr += (double)a.x * e.x + (double)a.y * e.y;
                    ti += (double)a.x * e.y - (double)a.y * e.x;
                }
                const float2 b = B[((long long)j * d + s) * bcap + l];
                re += tr * b.x - ti * b.y;
                im += tr * b.y + ti * b.x;
            }
        }
        En[(long long)k * lde + l] = make_double2(re, im);
    }
}

// Right transfer-matrix step of <a|b>: E'[k, l] = sum_{i, j, s} conj(A[k, s, i]) B[l, s, j] E[i, j], FP64 E.
// One block per output row k (bra bond); threads over l (ket bond).
__global__ void k_transfer_right(const double2* __restrict__ E, int lde, const float2* __restrict__ A, int acap,
                                 int abl, int abr, const float2* __restrict__ B, int bcap, int bbl, int bbr, int d,
                                 double2* __restrict__ En, int ldn) {
    const int k = blockIdx.x;
    if (k >= abl) return;
    for (int l = threadIdx.x; l < bbl; l += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int s = 0; s < d; ++s) {
            for (int i = 0; i < abr; ++i) {
                // t_i = sum_j B[l, s, j] E[i, j]
                double tr = 0.0, ti = 0.0;
                for (int j = 0; j < bbr; ++j) {
                    const float2 b = B[((long long)l * d + s) * bcap + j];
                    const double2 e = E[(long long)i * lde + j];
                    tr += (double)b.x * e.x - (double)b.y * e.y;
                    ti += (double)b.x * e.y + (double)b.y * e.x;
                }
                const float2 a = A[((long long)k * d + s) * acap + i];   // conj(a) * t
                re += (double)a.x * tr + (double)a.y * ti;
                im += (double)a.x * ti - (double)a.y * tr;
            }
        }
        En[(long long)k * ldn + l] = make_double2(re, im);
    }
}

// Derivative of <a|b> with respect to conj(a_p): H[k, s, m] = sum_{i, j} EL[k, i] B_p[i, s, j] ER[m, j]
// (EL: left environment of site p, bra index first; ER: right environment).  One block per k.
__global__ void k_env_grad(const double2* __restrict__ EL, int ldl, const double2* __restrict__ ER, int ldr,
                           const float2* __restrict__ B, int bcap, int bbl, int bbr, int abl, int abr, int d,
                           float2* __restrict__ H, int hcap) {
    const int k = blockIdx.x;
    if (k >= abl) return;
    for (int e = threadIdx.x; e < d * abr; e += blockDim.x) {
        const int s = e / abr, m = e % abr;
        double re = 0.0, im = 0.0;
        for (int i = 0; i < bbl; ++i) {
            const double2 el = EL[(long long)k * ldl + i];
            double tr = 0.0, ti = 0.0;   // sum_j B[i, s, j] ER[m, j]
            for (int j = 0; j < bbr; ++j) {
                const float2 b = B[((long long)i * d + s) * bcap + j];
                const double2 er = ER[(long long)m * ldr + j];
                tr += (double)b.x * er.x - (double)b.y * er.y;
                ti += (double)b.x * er.y + (double)b.y * er.x;
            }
            re += el.x * tr - el.y * ti;
            im += el.x * ti + el.y * tr;
        }
        H[((long long)k * d + s) * hcap + m] = make_float2((float)re, (float)im);
    }
}

// ------------------------------------------------------------------ state construction

// Interleaved d = 4 MPS of f(x) g(y) from 1-D MPS of f and g (Sec. III: site p holds mu_p = 2 x_p + y_p):
// out[(a*by + b), 2s + t, (a'*by' + b')] = X[a, s, a'] Y[b, t, b'].
__global__ void k_kron_interleave(const float2* __restrict__ X, const int* __restrict__ xb, int xcap,
                                  const float2* __restrict__ Y, const int* __restrict__ yb, int ycap,
                                  float2* __restrict__ O, int* __restrict__ ob, int ocap, int n) {
    const int p = blockIdx.x;
    if (p >= n) return;
    const int axl = xb[p], axr = xb[p + 1], byl = yb[p], byr = yb[p + 1];
    const int ol = axl * byl, orr = axr * byr;
    const float2* x = X + (long long)p * xcap * 2 * xcap;
    const float2* y = Y + (long long)p * ycap * 2 * ycap;
    float2* o = O + (long long)p * ocap * 4 * ocap;
    for (int e = threadIdx.x; e < ol * 4 * orr; e += blockDim.x) {
        const int l = e / (4 * orr), mu = (e / orr) % 4, r = e % orr;
        const int a = l / byl, b = l % byl, a2 = r / byr, b2 = r % byr;
        const int s = mu >> 1, t = mu & 1;
        o[((long long)l * 4 + mu) * ocap + r] =
            cmul(x[((long long)a * 2 + s) * xcap + a2], y[((long long)b * 2 + t) * ycap + b2]);
    }
    if (threadIdx.x == 0) {
        ob[p] = ol;
        if (p == n - 1) ob[n] = orr;
    }
}

// Elementwise (Hadamard) product of two MPS in the same site basis: O_p[(a, b), s, (a', b')] =
// A_p[a, s, a'] B_p[b, s, b'] (B conjugated when conj_b), bonds multiply.  One block per site.
__global__ void k_hadamard(const float2* __restrict__ A, const int* __restrict__ ab, int acap,
                           const float2* __restrict__ B, const int* __restrict__ bb, int bcap, int conj_b,
                           float2* __restrict__ O, int* __restrict__ ob, int ocap, int N, int d) {
    const int p = blockIdx.x;
    if (p >= N) return;
    const int al = ab[p], ar = ab[p + 1], bl = bb[p], br = bb[p + 1];
    const int ol = al * bl, orr = ar * br;
    const float2* a = A + (long long)p * acap * d * acap;
    const float2* b = B + (long long)p * bcap * d * bcap;
    float2* o = O + (long long)p * ocap * d * ocap;
    for (int e = threadIdx.x; e < ol * d * orr; e += blockDim.x) {
        const int l = e / (d * orr), s = (e / orr) % d, r = e % orr;
        const int l1 = l / bl, l2 = l % bl, r1 = r / br, r2 = r % br;
        float2 y = b[((long long)l2 * d + s) * bcap + r2];
        if (conj_b) y.y = -y.y;
        o[((long long)l * d + s) * ocap + r] = cmul(a[((long long)l1 * d + s) * acap + r1], y);
    }
    if (threadIdx.x == 0) {
        ob[p] = ol;
        if (p == N - 1) ob[N] = orr;
    }
}

// psi <- (re + i im) psi, applied to the site that holds the norm (site 0 unless the state is
// left-canonical, then site N-1).
__global__ void k_scale_site(float2* __restrict__ site, int cap, int d, const int* __restrict__ bond, int q, float re,
                             float im) {
    const int l = bond[q], r = bond[q + 1];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * d * r; e += gridDim.x * blockDim.x) {
        const int i = e / (d * r), s = (e / r) % d, j = e % r;
        float2* v = site + ((long long)i * d + s) * cap + j;
        *v = cmul(*v, make_float2(re, im));
    }
}

// MPS of |A> + |B>: block-diagonal bonds, boundaries concatenated.  O must not alias A or B.
__global__ void k_direct_sum(const float2* __restrict__ A, const int* __restrict__ ab, int acap,
                             const float2* __restrict__ B, const int* __restrict__ bb, int bcap,
                             float2* __restrict__ O, int* __restrict__ ob, int ocap, int N, int d) {
    const int p = blockIdx.x;
    if (p >= N) return;
    const int al = ab[p], ar = ab[p + 1], bl = bb[p], br = bb[p + 1];
    const int ol = (p == 0) ? 1 : al + bl, orr = (p == N - 1) ? 1 : ar + br;
    const float2* a = A + (long long)p * acap * d * acap;
    const float2* b = B + (long long)p * bcap * d * bcap;
    float2* o = O + (long long)p * ocap * d * ocap;
    for (int e = threadIdx.x; e < ol * d * orr; e += blockDim.x) {
        const int l = e / (d * orr), s = (e / orr) % d, r = e % orr;
        float2 v = make_float2(0.f, 0.f);
        if (N == 1) {
            v = cadd(a[s * acap], b[s * bcap]);
        } else if (p == 0) {
            if (r < ar) v = a[(long long)s * acap + r];
            else v = b[(long long)s * bcap + (r - ar)];
        } else if (p == N - 1) {
            if (l < al) v = a[((long long)l * d + s) * acap];
            else v = b[((long long)(l - al) * d + s) * bcap];
        } else {
            if (l < al && r < ar) v = a[((long long)l * d + s) * acap + r];
            else if (l >= al && r >= ar) v = b[((long long)(l - al) * d + s) * bcap + (r - ar)];
        }
        o[((long long)l * d + s) * ocap + r] = v;
    }
    if (threadIdx.x == 0) {
        ob[p] = ol;
        if (p == N - 1) ob[N] = orr;
    }
}

}  // namespace qtn
