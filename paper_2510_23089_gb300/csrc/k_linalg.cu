// Dense complex linear algebra for the truncation step (sm_103a, FP32 SIMT).
//
//  * k_gemm: strided complex GEMM, C = alpha * op(A) op(B), 64x64 tiles staged
//    through shared memory.  OUT_ATOMIC64 splits K across blockIdx.z and adds
//    the FP32 chunk results into an FP64 matrix: Gram matrices are accumulated
//    in FP64 while every product stays FP32.
//  * k_eig_jacobi: one-sided (Hestenes) Jacobi on the columns of a Hermitian
//    positive semidefinite r x r matrix G held in shared memory (r <= 160).
//    Columns converge to G V = U diag(lambda); normalised columns are the
//    eigenvectors and their norms the eigenvalues.  Disjoint column pairs of a
//    round-robin round are processed by 8-lane groups with shuffle reductions.
//  * k_select: the truncation rule on the sorted spectrum (FP64 bookkeeping).
#include <math.h>
#include <stdlib.h>

#include "qtn_internal.cuh"

namespace qtn {

// ------------------------------------------------------------------ GEMM
constexpr int GB_M = 64, GB_N = 64, GB_K = 16, G_THREADS = 256;

__device__ __forceinline__ float2 mat_get(const Mat& m, int i, int j, long long rs, long long cs, int jdiv,
                                          long long cs_hi) {
    long long off = (long long)i * rs;
    if (jdiv > 0) off += (long long)(j / jdiv) * cs_hi + (long long)(j % jdiv) * cs;
    else off += (long long)j * cs;
    float2 v = m.p[off];
    return m.conj ? cconj(v) : v;
}

__global__ void __launch_bounds__(G_THREADS) k_gemm(GemmDesc d, const int* __restrict__ R) {
    if (d.guard_reg >= 0 && R[d.guard_reg] != d.guard_val) return;
    const int M = d.M.eval(R), N = d.N.eval(R), K = d.K.eval(R);
    const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
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

    __shared__ float2 As[GB_K][GB_M + 1];
    __shared__ float2 Bs[GB_K][GB_N + 1];
    const int tid = threadIdx.x;
    const int ty = tid / 16, tx = tid % 16;
    float2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);

    for (int k0 = k_begin; k0 < k_end; k0 += GB_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int e = tid + q * G_THREADS;
            int ii, kk;
            if (a_kfast) { ii = e / GB_K; kk = e % GB_K; } else { ii = e % GB_M; kk = e / GB_M; }
            int gi = m0 + ii, gk = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (gi < M && gk < k_end) v = mat_get(d.A, gi, gk, ars, acs, ajd, ach);
            As[kk][ii] = v;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int e = tid + q * G_THREADS;
            int jj, kk;
            if (b_nfast) { jj = e % GB_N; kk = e / GB_N; } else { jj = e / GB_K; kk = e % GB_K; }
            int gj = n0 + jj, gk = k0 + kk;
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
            float2 av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) cfma(acc[a][b], av[a], bv[b]);
        }
        __syncthreads();
    }
    if (d.flops != nullptr && threadIdx.x == 0)
        atomicAdd(d.flops, 8.0 * (double)min(GB_M, M - m0) * (double)min(GB_N, N - n0) * (double)(k_end - k_begin));
    const long long crs = d.crs.eval(R), ccs = d.ccs.eval(R);
    const float2 alpha = make_float2(d.alpha_re, d.alpha_im);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int gi = m0 + ty * 4 + a;
        if (gi >= M) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int gj = n0 + tx * 4 + b;
            if (gj >= N) continue;
            float2 v = cmul(alpha, acc[a][b]);
            long long off = (long long)gi * crs + (long long)gj * ccs;
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

cudaError_t launch_gemm(const GemmDesc& d, int max_m, int max_n, int max_k, const int* R, cudaStream_t s) {
    if (max_m <= 0 || max_n <= 0) return cudaSuccess;
    dim3 grid((max_n + GB_N - 1) / GB_N, (max_m + GB_M - 1) / GB_M, 1);
    if (d.mode == OUT_ATOMIC64) {
        int kc = d.kchunk > 0 ? d.kchunk : 1;
        grid.z = (unsigned)((max(max_k, 1) + kc - 1) / kc);
    }
    GemmDesc dd = d;
    if (g_prof_ledger) dd.flops = g_prof_ledger + L_PROF_GEMM;
    count_launch(PROF_GEMM, s, true);
    k_gemm<<<grid, G_THREADS, 0, s>>>(dd, R);
    count_launch(PROF_GEMM, s, false);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ one-sided Jacobi eigensolver
constexpr int EIG_THREADS = 1024;
constexpr int EIG_GL = 8;                       // lanes per column pair
constexpr int EIG_GROUPS = EIG_THREADS / EIG_GL;
constexpr int EIG_RS = EIG_MAX + 4;             // padded column stride in shared memory
constexpr float EIG_TOL = 1.0e-6f;
constexpr float EIG_NOISE = 1.0e-13f;           // |w_i| |w_j| floor (matrix scaled to unit largest diagonal)

__device__ __forceinline__ void circle_pair(int t, int k, int rr, int& i, int& j) {
    // round-robin tournament (circle method) on rr players, round t in [0, rr-2]
    const int m = rr - 1;
    if (k == 0) { i = t; j = m; }
    else { i = (t + k) % m; j = (t - k + m) % m; }
}

__global__ void __launch_bounds__(EIG_THREADS, 1)
k_eig_jacobi(const double2* __restrict__ G, Dim ldd, Dim rdim, float2* __restrict__ U, Dim ldud,
             double* __restrict__ lam, const int* __restrict__ Rc, int* __restrict__ Rw, int max_sweeps,
             double* __restrict__ ledger, int guard_reg, int guard_val, double* __restrict__ prof, float tol) {
    if (guard_reg >= 0 && Rc[guard_reg] != guard_val) return;
    extern __shared__ float2 W[];                // column-major, W[j*EIG_RS + i]
    __shared__ double nrm[EIG_MAX];
    __shared__ int rank_of[EIG_MAX];
    __shared__ int rotated;
    const int r = rdim.eval(Rc);
    const long long ld = ldd.eval(Rc), ldu = ldud.eval(Rc);
    if (r <= 0) return;
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

    const int rr = r + (r & 1);
    const int grp = tid / EIG_GL, lane = tid % EIG_GL;
    const unsigned gmask = 0xFFu << ((tid % 32) / EIG_GL * EIG_GL);
    int sweep = 0;
    bool converged = (r < 2);
    for (; sweep < max_sweeps && !converged; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int t = 0; t < rr - 1; ++t) {
            for (int k = grp; k < rr / 2; k += EIG_GROUPS) {
                int i, j;
                circle_pair(t, k, rr, i, j);
                if (i >= r || j >= r) continue;
                float2* wi = W + i * EIG_RS;
                float2* wj = W + j * EIG_RS;
                float a = 0.f, b = 0.f, cr = 0.f, ci = 0.f;
                for (int row = lane; row < r; row += EIG_GL) {
                    float2 x = wi[row], y = wj[row];
                    a = fmaf(x.x, x.x, fmaf(x.y, x.y, a));
                    b = fmaf(y.x, y.x, fmaf(y.y, y.y, b));
                    cr = fmaf(x.x, y.x, fmaf(x.y, y.y, cr));    // conj(x) * y
                    ci = fmaf(x.x, y.y, fmaf(-x.y, y.x, ci));
                }
#pragma unroll
                for (int off = EIG_GL / 2; off > 0; off >>= 1) {
                    a += __shfl_xor_sync(gmask, a, off);
                    b += __shfl_xor_sync(gmask, b, off);
                    cr += __shfl_xor_sync(gmask, cr, off);
                    ci += __shfl_xor_sync(gmask, ci, off);
                }
                if (lane == 0 && prof != nullptr) atomicAdd(&n_pairs, 1ull);
                const float cabs = sqrtf(cr * cr + ci * ci);
                // Columns of the scaled matrix whose norms are both below the FP32 resolution of G are
                // round-off: rotating them never converges and they are orthonormalised afterwards.
                const float ab = sqrtf(a) * sqrtf(b);
                if (!(cabs > tol * ab) || !(cabs > 1e-30f) || !(ab > EIG_NOISE)) continue;
                const float zeta = (b - a) / (2.f * cabs);
                const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
                const float cs = rsqrtf(fmaf(tt, tt, 1.f));
                const float sn = tt * cs;
                const float er = cr / cabs, ei = ci / cabs;
                for (int row = lane; row < r; row += EIG_GL) {
                    float2 x = wi[row], y = wj[row];
                    // x' = cs x - sn conj(e) y ;  y' = sn e x + cs y
                    float2 cey = make_float2(er * y.x + ei * y.y, er * y.y - ei * y.x);
                    float2 ex = make_float2(er * x.x - ei * x.y, er * x.y + ei * x.x);
                    wi[row] = make_float2(cs * x.x - sn * cey.x, cs * x.y - sn * cey.y);
                    wj[row] = make_float2(sn * ex.x + cs * y.x, sn * ex.y + cs * y.y);
                }
                if (lane == 0) {
                    rotated = 1;
                    if (prof != nullptr) atomicAdd(&n_rot, 1ull);
                }
            }
            __syncthreads();
        }
        converged = (rotated == 0);
        __syncthreads();
    }
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
    }
    __syncthreads();
    // Re-orthonormalise the columns in descending-eigenvalue order (classical Gram-Schmidt, two passes):
    // directions below the FP32 resolution of G are not orthogonal to working precision after Jacobi, and
    // the new site must be an isometry.  A column that turns out numerically dependent on the previous
    // ones is replaced by a pseudo-random vector orthogonalised the same way, so the basis stays complete
    // and no weight of the factorised matrix is lost.
    __shared__ int col_of_rank[EIG_MAX];
    __shared__ float coef_r[EIG_MAX], coef_i[EIG_MAX];
    __shared__ float red_s[32];
    __shared__ float nrm_cur;
    for (int j = tid; j < r; j += EIG_THREADS) col_of_rank[rank_of[j]] = j;
    __syncthreads();
    const int warp = tid / 32, wl = tid % 32;
    auto block_norm = [&](float2* w) {
        float ss = 0.f;
        for (int row = tid; row < r; row += EIG_THREADS) ss += w[row].x * w[row].x + w[row].y * w[row].y;
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
        if (wl == 0) red_s[warp] = ss;
        __syncthreads();
        if (tid == 0) {
            float tot = 0.f;
            for (int q = 0; q < EIG_THREADS / 32; ++q) tot += red_s[q];
            nrm_cur = sqrtf(tot);
        }
        __syncthreads();
        return nrm_cur;
    };
    // w -= sum_{q<t} (u_q^dagger w) u_q: coefficients by warps (one dot per warp), then every warp updates a
    // slice of rows with its lanes splitting the q-sum (all 1024 threads busy).
    auto project_out = [&](float2* w, int t) {
        for (int q = warp; q < t; q += EIG_THREADS / 32) {
            const float2* u = W + col_of_rank[q] * EIG_RS;
            float cr = 0.f, ci = 0.f;
            for (int row = wl; row < r; row += 32) {
                float2 a = u[row], b = w[row];
                cr = fmaf(a.x, b.x, fmaf(a.y, b.y, cr));
                ci = fmaf(a.x, b.y, fmaf(-a.y, b.x, ci));
            }
            for (int off = 16; off > 0; off >>= 1) {
                cr += __shfl_xor_sync(0xffffffffu, cr, off);
                ci += __shfl_xor_sync(0xffffffffu, ci, off);
            }
            if (wl == 0) { coef_r[q] = cr; coef_i[q] = ci; }
        }
        __syncthreads();
        for (int row = warp; row < r; row += EIG_THREADS / 32) {
            float ar = 0.f, ai = 0.f;
            for (int q = wl; q < t; q += 32) {
                const float2 u = W[col_of_rank[q] * EIG_RS + row];
                ar += coef_r[q] * u.x - coef_i[q] * u.y;
                ai += coef_r[q] * u.y + coef_i[q] * u.x;
            }
            for (int off = 16; off > 0; off >>= 1) {
                ar += __shfl_xor_sync(0xffffffffu, ar, off);
                ai += __shfl_xor_sync(0xffffffffu, ai, off);
            }
            if (wl == 0) w[row] = make_float2(w[row].x - ar, w[row].y - ai);
        }
        __syncthreads();
    };
    auto scale_col = [&](float2* w, float sc) {
        for (int row = tid; row < r; row += EIG_THREADS) w[row] = cscale(w[row], sc);
        __syncthreads();
    };
    // The Jacobi columns are orthogonal to the solve's tolerance, so one classical pass restores working
    // precision; a second pass runs when the projection cancelled most of the column ("twice is enough").
    // A column found dependent gets a pseudo-random replacement.
    for (int t = 0; t < r; ++t) {
        float2* w = W + col_of_rank[t] * EIG_RS;
        for (int attempt = 0; attempt < 2; ++attempt) {
            if (attempt == 1) {
                for (int row = tid; row < r; row += EIG_THREADS) w[row] = gauss2(977 + t, row, t);
                __syncthreads();
            }
            const float n0 = block_norm(w);
            if (!(n0 > 0.f)) continue;
            scale_col(w, 1.f / n0);
            project_out(w, t);
            float na = block_norm(w);
            if (na < 0.7f) {   // heavy cancellation: a second classical pass restores orthogonality
                project_out(w, t);
                na = block_norm(w);
            }
            if (na > 1e-4f) { scale_col(w, 1.f / na); break; }
            if (attempt == 1) scale_col(w, 0.f);
        }
    }
    for (int e = tid; e < r * r; e += EIG_THREADS) {
        int j = e / r, row = e % r;
        U[(long long)rank_of[j] * ldu + row] = W[j * EIG_RS + row];
    }
    if (tid == 0) {
        atomicMax(&Rw[R_SWEEPS], sweep);
        if (!converged) atomicOr(&Rw[R_FLAGS], 1);
        // algorithmic FLOPs: 16 per row for the three inner products of a pair, 24 per row for a rotation,
        // 8 r^3 for the classical Gram-Schmidt pass (coefficients and updates, complex)
        if (prof != nullptr)
            atomicAdd(prof, 16.0 * r * (double)n_pairs + 24.0 * r * (double)n_rot + 8.0 * (double)r * r * r);
    }
}

cudaError_t launch_eig(const double2* G, Dim ld, Dim r, float2* U, Dim ldu, double* lam, const int* R,
                       int r_cap, int max_sweeps, double* ledger, cudaStream_t s, int guard_reg, int guard_val,
                       float tol, int method) {
    (void)r_cap;
    size_t smem = (size_t)EIG_MAX * EIG_RS * sizeof(float2);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_eig_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    // method: 0 = from-scratch solve, 1 = refinement of a nearly diagonal matrix.  Both use one-sided Jacobi
    // (relative accuracy) unless QTN_EIG=trd selects the Householder-tridiagonal solver for from-scratch
    // solves (absolute accuracy only; faster on large r).
    static int use_trd = -1;
    if (use_trd < 0) {
        const char* e = getenv("QTN_EIG");
        use_trd = (e != nullptr && e[0] == 't') ? 1 : 0;
    }
    if (method == 0 && use_trd) return launch_eig_trd(G, ld, r, U, ldu, lam, R, s, guard_reg, guard_val);
    count_launch(PROF_EIG, s, true);
    k_eig_jacobi<<<1, EIG_THREADS, smem, s>>>(G, ld, r, U, ldu, lam, R, (int*)R, max_sweeps, ledger, guard_reg,
                                               guard_val, g_prof_ledger ? g_prof_ledger + L_PROF_EIG : nullptr, tol);
    count_launch(PROF_EIG, s, false);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ launch accounting / profiling
double* g_prof_ledger = nullptr;
static long long g_launches = 0;
static bool g_prof_on = false;
struct ProfPool {
    cudaEvent_t* ev = nullptr;   // pairs (start, stop)
    int cap = 0, used = 0;
    long long launches = 0;
};
static ProfPool g_pool[PROF_NCLASS];

void count_launch(int cls, cudaStream_t s, bool before) {
    if (!before) ++g_launches;
    if (!g_prof_on || cls == PROF_OTHER) return;
    ProfPool& p = g_pool[cls];
    if (before) {
        if (p.used + 2 > p.cap) return;
        cudaEventRecord(p.ev[p.used], s);
    } else {
        if (p.used + 2 > p.cap) { ++p.launches; return; }
        cudaEventRecord(p.ev[p.used + 1], s);
        p.used += 2;
        ++p.launches;
    }
}

long long launch_total() { return g_launches; }

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
    }
}

// Total device time (ms) and launch count of one kernel class since prof_begin.
void prof_read(int cls, double* ms, long long* launches) {
    ProfPool& p = g_pool[cls];
    double t = 0.0;
    for (int i = 0; i + 1 < p.used; i += 2) {
        float e = 0.f;
        cudaEventSynchronize(p.ev[i + 1]);
        if (cudaEventElapsedTime(&e, p.ev[i], p.ev[i + 1]) == cudaSuccess) t += e;
    }
    *ms = t;
    *launches = p.launches;
}

}  // namespace qtn
