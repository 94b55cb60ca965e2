// Hermitian eigensolver for r <= 160 in one CTA: Householder tridiagonalisation, bisection, inverse iteration.
//
//   1. The matrix (scaled to a unit largest diagonal) is reduced to Hermitian tridiagonal form by r - 2
//      Householder reflectors, H_k = I - tau_k v_k v_k^dagger acting on rows/columns k+1..r-1.  Each step is
//      a Hermitian matrix-vector product and a rank-2 update of the trailing block, spread over all 1024
//      threads (about five block barriers per step).  The reflectors are parked in the output buffer.
//   2. A diagonal phase transform makes the tridiagonal real symmetric (|e_k| off the diagonal).
//   3. Every eigenvalue by bisection on Sturm counts (one thread per eigenvalue).
//   4. Every eigenvector of the real tridiagonal by inverse iteration (one thread per eigenvalue, three
//      solves of the shifted system by elimination; pivots below eps |T| are lifted to eps |T|).
//   5. Back-transformation: phases, then the reflectors in reverse order, in shared memory.
//   6. Classical Gram-Schmidt in descending eigenvalue order (a second pass on heavy cancellation;
//      dependent columns replaced by orthogonalised pseudo-random vectors): the result is orthonormal to
//      working precision even inside clusters of close eigenvalues, which inverse iteration alone is not.
// Output as the Jacobi kernel: eigenvectors as columns of U (leading dimension ldu) in descending order of
// eigenvalue, eigenvalues (FP64) in lam.
#include <math.h>

#include "qtn_internal.cuh"

namespace qtn {

constexpr int TR_THREADS = 1024;
constexpr int TR_RS = EIG_MAX + 4;

__device__ __forceinline__ float block_sum(float v, float* red, int tid) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    float t = 0.f;
#pragma unroll 8
    for (int q = 0; q < TR_THREADS / 32; ++q) t += red[q];
    return t;
}

__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int r, float x, float pivmin) {
    // number of eigenvalues of the real symmetric tridiagonal (d, e) smaller than x
    int cnt = 0;
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += (q < 0.f);
    for (int i = 1; i < r; ++i) {
        q = (d[i] - x) - e2[i - 1] / q;
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += (q < 0.f);
    }
    return cnt;
}

__global__ void __launch_bounds__(TR_THREADS, 1)
k_heev_trd(const double2* __restrict__ G, Dim ldd, Dim rdim, float2* __restrict__ U, Dim ldud,
           double* __restrict__ lam, const int* __restrict__ Rc, int guard_reg, int guard_val,
           double* __restrict__ prof) {
    if (guard_reg >= 0 && Rc[guard_reg] != guard_val) return;
    extern __shared__ float2 A[];                    // column-major, A[j * TR_RS + i]
    __shared__ float dd[EIG_MAX], e2[EIG_MAX], ee[EIG_MAX], taus[EIG_MAX], ev[EIG_MAX];
    __shared__ float2 ec[EIG_MAX], phs[EIG_MAX], pv[EIG_MAX], wv[EIG_MAX];
    __shared__ float red[32];
    __shared__ float bounds[2];
    __shared__ double gscale;
    __shared__ int order[EIG_MAX];
    __shared__ float coef_r[EIG_MAX], coef_i[EIG_MAX];
    const int r = rdim.eval(Rc);
    const long long ld = ldd.eval(Rc), ldu = ldud.eval(Rc);
    if (r <= 0) return;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    constexpr int NW = TR_THREADS / 32;

    if (tid < 32) {
        double mx = 0.0;
        for (int i = tid; i < r; i += 32) mx = fmax(mx, fabs(G[(long long)i * ld + i].x));
        for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        if (tid == 0) gscale = (mx > 0.0 && isfinite(mx)) ? mx : 1.0;
    }
    __syncthreads();
    const double inv_scale = 1.0 / gscale;
    for (int e = tid; e < r * r; e += TR_THREADS) {
        const int i = e % r, j = e / r;
        const double2 g = G[(long long)i * ld + j];
        A[j * TR_RS + i] = make_float2((float)(g.x * inv_scale), (float)(g.y * inv_scale));
    }
    __syncthreads();

    // ---------------------------------------------------------------- 1. tridiagonalisation
    for (int k = 0; k + 2 < r; ++k) {
        const int L = r - k - 1;
        float2* x = A + k * TR_RS + (k + 1);         // column k below the diagonal (contiguous)
        float s = 0.f;
        for (int i = tid; i < L; i += TR_THREADS) s += x[i].x * x[i].x + x[i].y * x[i].y;
        const float xn2 = block_sum(s, red, tid);
        const float xn = sqrtf(xn2);
        const float2 x0 = x[0];
        const float ax0 = sqrtf(x0.x * x0.x + x0.y * x0.y);
        const float2 ph = ax0 > 0.f ? make_float2(x0.x / ax0, x0.y / ax0) : make_float2(1.f, 0.f);
        const float vtv = 2.f * xn * (xn + ax0);
        const float tau = (xn > 0.f && vtv > 0.f) ? 2.f / vtv : 0.f;
        __syncthreads();
        if (tid == 0) {
            ec[k] = make_float2(-ph.x * xn, -ph.y * xn);          // the new subdiagonal alpha
            taus[k] = tau;
            if (tau > 0.f) x[0] = make_float2(ph.x * (ax0 + xn), ph.y * (ax0 + xn));
            else ec[k] = x0;
        }
        __syncthreads();
        if (tau == 0.f) continue;
        // p = tau A22 v, with A22[i][j] = conj(A22[j][i]) read down column i (contiguous)
        for (int i = warp; i < L; i += NW) {
            const float2* col = A + (k + 1 + i) * TR_RS + (k + 1);
            float ar = 0.f, ai = 0.f;
            for (int j = lane; j < L; j += 32) {
                const float2 a = col[j], v = x[j];                 // conj(a) * v
                ar = fmaf(a.x, v.x, fmaf(a.y, v.y, ar));
                ai = fmaf(a.x, v.y, fmaf(-a.y, v.x, ai));
            }
            for (int off = 16; off > 0; off >>= 1) {
                ar += __shfl_xor_sync(0xffffffffu, ar, off);
                ai += __shfl_xor_sync(0xffffffffu, ai, off);
            }
            if (lane == 0) pv[i] = make_float2(tau * ar, tau * ai);
        }
        __syncthreads();
        // K = (tau / 2) v^dagger p  (real for Hermitian A22)
        float kr = 0.f;
        for (int i = tid; i < L; i += TR_THREADS) kr += x[i].x * pv[i].x + x[i].y * pv[i].y;
        const float K = 0.5f * tau * block_sum(kr, red, tid);
        for (int i = tid; i < L; i += TR_THREADS) wv[i] = make_float2(pv[i].x - K * x[i].x, pv[i].y - K * x[i].y);
        __syncthreads();
        // A22 -= v w^dagger + w v^dagger
        for (int e = tid; e < L * L; e += TR_THREADS) {
            const int i = e % L, j = e / L;
            const float2 vi = x[i], vj = x[j], wi = wv[i], wj = wv[j];
            float2* a = A + (k + 1 + j) * TR_RS + (k + 1 + i);
            // v_i conj(w_j) + w_i conj(v_j)
            const float re = vi.x * wj.x + vi.y * wj.y + wi.x * vj.x + wi.y * vj.y;
            const float im = vi.y * wj.x - vi.x * wj.y + wi.y * vj.x - wi.x * vj.y;
            a->x -= re;
            a->y -= im;
        }
        __syncthreads();
    }
    for (int k = tid; k < r; k += TR_THREADS) dd[k] = A[k * TR_RS + k].x;
    if (tid == 0 && r >= 2) ec[r - 2] = A[(r - 2) * TR_RS + (r - 1)];
    // park the reflectors v_k (rows k+1..r-1) in column k of U
    for (int e = tid; e < r * r; e += TR_THREADS) {
        const int i = e % r, k = e / r;
        if (k + 2 < r && i > k) U[(long long)k * ldu + i] = A[k * TR_RS + i];
    }
    __syncthreads();
    if (tid == 0) {
        phs[0] = make_float2(1.f, 0.f);
        for (int k = 0; k + 1 < r; ++k) {
            const float a = sqrtf(ec[k].x * ec[k].x + ec[k].y * ec[k].y);
            ee[k] = a;
            e2[k] = a * a;
            const float2 u = a > 0.f ? make_float2(ec[k].x / a, ec[k].y / a) : make_float2(1.f, 0.f);
            phs[k + 1] = cmul(phs[k], u);
        }
        float lo = 1e30f, hi = -1e30f;
        for (int i = 0; i < r; ++i) {
            const float rad = (i > 0 ? ee[i - 1] : 0.f) + (i + 1 < r ? ee[i] : 0.f);
            lo = fminf(lo, dd[i] - rad);
            hi = fmaxf(hi, dd[i] + rad);
        }
        bounds[0] = lo;
        bounds[1] = hi;
    }
    __syncthreads();

    // ---------------------------------------------------------------- 2. eigenvalues (bisection)
    const float tnorm = fmaxf(fabsf(bounds[0]), fabsf(bounds[1]));
    const float pivmin = fmaxf(1e-30f, 1e-7f * tnorm * 1e-6f);
    for (int j = tid; j < r; j += TR_THREADS) {
        const int target = r - 1 - j;                // eigenvalue index in ascending order
        float lo = bounds[0] - 1e-6f * tnorm - 1e-30f, hi = bounds[1] + 1e-6f * tnorm + 1e-30f;
        for (int it = 0; it < 64; ++it) {
            const float mid = 0.5f * (lo + hi);
            if (!(hi - lo > 2.5e-7f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-30f) || mid == lo || mid == hi) break;
            if (sturm_count(dd, e2, r, mid, pivmin) <= target) lo = mid;
            else hi = mid;
        }
        ev[j] = 0.5f * (lo + hi);
    }
    __syncthreads();

    // ---------------------------------------------------------------- 3. eigenvectors (inverse iteration)
    // column j of A holds the real eigenvector z (.x) with the elimination pivots (.y) alongside
    const float eps_t = 1.2e-7f * fmaxf(tnorm, 1e-30f);
    for (int j = tid; j < r; j += TR_THREADS) {
        float2* z = A + j * TR_RS;
        const float lam_j = ev[j];
        // pivots u_i of T - lam I (no pivoting; tiny pivots lifted)
        float u = dd[0] - lam_j;
        if (fabsf(u) < eps_t) u = copysignf(eps_t, u == 0.f ? 1.f : u);
        z[0].y = u;
        for (int i = 1; i < r; ++i) {
            u = (dd[i] - lam_j) - e2[i - 1] / u;
            if (fabsf(u) < eps_t) u = copysignf(eps_t, u == 0.f ? 1.f : u);
            z[i].y = u;
        }
        for (int i = 0; i < r; ++i) z[i].x = gauss2(31 + j, i, 7).x;
        for (int it = 0; it < 3; ++it) {
            // forward: y_i = b_i - (e_{i-1} / u_{i-1}) y_{i-1}
            for (int i = 1; i < r; ++i) z[i].x -= (ee[i - 1] / z[i - 1].y) * z[i - 1].x;
            // backward: x_i = (y_i - e_i x_{i+1}) / u_i, rescaling the tail when it grows (several lifted
            // pivots inside a cluster of eigenvalues would otherwise overflow FP32)
            z[r - 1].x /= z[r - 1].y;
            for (int i = r - 2; i >= 0; --i) {
                z[i].x = (z[i].x - ee[i] * z[i + 1].x) / z[i].y;
                if (fabsf(z[i].x) > 1e15f) {
                    for (int q = i; q < r; ++q) z[q].x *= 1e-15f;
                }
            }
            float nn = 0.f;
            for (int i = 0; i < r; ++i) nn += z[i].x * z[i].x;
            const float inv = nn > 0.f ? rsqrtf(nn) : 0.f;
            for (int i = 0; i < r; ++i) z[i].x *= inv;
        }
    }
    __syncthreads();
    // complex vectors: y = D z (phases)
    for (int e = tid; e < r * r; e += TR_THREADS) {
        const int i = e % r, j = e / r;
        const float zz = A[j * TR_RS + i].x;
        A[j * TR_RS + i] = make_float2(phs[i].x * zz, phs[i].y * zz);
    }
    __syncthreads();

    // ---------------------------------------------------------------- 4. back-transformation
    for (int k = r - 3; k >= 0; --k) {
        const float tau = taus[k];
        if (tau == 0.f) continue;
        const int L = r - k - 1;
        const float2* v = U + (long long)k * ldu + (k + 1);
        // s_c = v^dagger Y[k+1:, c], Y[k+1:, c] -= tau s_c v ; one warp per column
        for (int c = warp; c < r; c += NW) {
            float2* y = A + c * TR_RS + (k + 1);
            float sr = 0.f, si = 0.f;
            for (int i = lane; i < L; i += 32) {
                const float2 a = v[i], b = y[i];
                sr = fmaf(a.x, b.x, fmaf(a.y, b.y, sr));
                si = fmaf(a.x, b.y, fmaf(-a.y, b.x, si));
            }
            for (int off = 16; off > 0; off >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, off);
                si += __shfl_xor_sync(0xffffffffu, si, off);
            }
            sr *= tau;
            si *= tau;
            for (int i = lane; i < L; i += 32) {
                const float2 a = v[i];
                y[i].x -= sr * a.x - si * a.y;
                y[i].y -= sr * a.y + si * a.x;
            }
        }
        __syncthreads();
    }

    // ---------------------------------------------------------------- 5. orthonormalisation, output
    // eigenvalues come out of bisection in descending order already
    for (int j = tid; j < r; j += TR_THREADS) order[j] = j;
    __syncthreads();
    auto bnorm = [&](const float2* w) {
        float ss = 0.f;
        for (int i = tid; i < r; i += TR_THREADS) ss += w[i].x * w[i].x + w[i].y * w[i].y;
        return sqrtf(block_sum(ss, red, tid));
    };
    auto project_out = [&](float2* w, int t) {
        for (int q = warp; q < t; q += NW) {
            const float2* u = A + q * TR_RS;
            float cr = 0.f, ci = 0.f;
            for (int i = lane; i < r; i += 32) {
                const float2 a = u[i], b = w[i];
                cr = fmaf(a.x, b.x, fmaf(a.y, b.y, cr));
                ci = fmaf(a.x, b.y, fmaf(-a.y, b.x, ci));
            }
            for (int off = 16; off > 0; off >>= 1) {
                cr += __shfl_xor_sync(0xffffffffu, cr, off);
                ci += __shfl_xor_sync(0xffffffffu, ci, off);
            }
            if (lane == 0) { coef_r[q] = cr; coef_i[q] = ci; }
        }
        __syncthreads();
        for (int i = warp; i < r; i += NW) {
            float ar = 0.f, ai = 0.f;
            for (int q = lane; q < t; q += 32) {
                const float2 u = A[q * TR_RS + i];
                ar += coef_r[q] * u.x - coef_i[q] * u.y;
                ai += coef_r[q] * u.y + coef_i[q] * u.x;
            }
            for (int off = 16; off > 0; off >>= 1) {
                ar += __shfl_xor_sync(0xffffffffu, ar, off);
                ai += __shfl_xor_sync(0xffffffffu, ai, off);
            }
            if (lane == 0) w[i] = make_float2(w[i].x - ar, w[i].y - ai);
        }
        __syncthreads();
    };
    for (int t = 0; t < r; ++t) {
        float2* w = A + t * TR_RS;
        for (int attempt = 0; attempt < 2; ++attempt) {
            if (attempt == 1) {
                for (int i = tid; i < r; i += TR_THREADS) w[i] = gauss2(977 + t, i, t);
                __syncthreads();
            }
            const float n0 = bnorm(w);
            if (!(n0 > 0.f)) continue;
            for (int i = tid; i < r; i += TR_THREADS) w[i] = cscale(w[i], 1.f / n0);
            __syncthreads();
            project_out(w, t);
            float na = bnorm(w);
            if (na < 0.7f) {
                project_out(w, t);
                na = bnorm(w);
            }
            const float sc = (na > 1e-4f) ? 1.f / na : 0.f;
            for (int i = tid; i < r; i += TR_THREADS) w[i] = cscale(w[i], sc);
            __syncthreads();
            if (na > 1e-4f) break;
        }
    }
    for (int e = tid; e < r * r; e += TR_THREADS) {
        const int i = e % r, j = e / r;
        U[(long long)j * ldu + i] = A[j * TR_RS + i];
    }
    for (int j = tid; j < r; j += TR_THREADS) lam[j] = (double)ev[j] * gscale;
    if (tid == 0 && prof != nullptr) {
        // algorithmic FLOPs: tridiagonalisation 16 r^3 / 3 (Hermitian matvec and rank-2 update, complex),
        // back-transformation 8 r^3, Gram-Schmidt 8 r^3
        atomicAdd(prof, (16.0 / 3.0 + 16.0) * (double)r * r * r);
    }
}

// ------------------------------------------------------------------ first-order basis refinement
// Given the Gram matrix G2 = X X^dagger of rows X = U^dagger T that are nearly orthogonal (U an approximate
// eigenbasis of T T^dagger), the rotation that diagonalises G2 is, to first order,
//     V = I + E,   E_ij = G2_ij / (d_j - d_i)   (i != j, d = diag G2),
// which cancels every off-diagonal entry of V^dagger G2 V to second order and keeps the relative accuracy of
// small directions (each E_ij is scaled by its own gap).  Pairs whose coupling is not small against their
// gap (|G2_ij| >= gap / 2, near-degenerate directions) are left unrotated.  V's columns are then
// orthonormalised (classical Gram-Schmidt in descending order of d, second pass on cancellation) so that
// U V stays an isometry.  Output: V column-major (ld ldv).
__global__ void __launch_bounds__(TR_THREADS, 1)
k_refine_basis(const double2* __restrict__ G, Dim ldd, Dim rdim, float2* __restrict__ V, int ldv,
               const int* __restrict__ Rc) {
    extern __shared__ float2 A[];                    // column-major, A[j * TR_RS + i]
    __shared__ double dg[EIG_MAX];
    __shared__ int order[EIG_MAX];
    __shared__ float coef_r[EIG_MAX], coef_i[EIG_MAX];
    __shared__ float red[32];
    const int r = rdim.eval(Rc);
    const long long ld = ldd.eval(Rc);
    if (r <= 0) return;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    constexpr int NW = TR_THREADS / 32;
    for (int i = tid; i < r; i += TR_THREADS) dg[i] = G[(long long)i * ld + i].x;
    __syncthreads();
    for (int i = tid; i < r; i += TR_THREADS) {      // descending order of the diagonal
        int rk = 0;
        for (int q = 0; q < r; ++q) rk += (dg[q] > dg[i]) || (dg[q] == dg[i] && q < i);
        order[rk] = i;
    }
    __syncthreads();
    // column t of A = column order[t] of V
    for (int e = tid; e < r * r; e += TR_THREADS) {
        const int i = e % r, t = e / r, j = order[t];
        float2 v = make_float2(i == j ? 1.f : 0.f, 0.f);
        if (i != j && j >= 0 && j < r) {
            const double2 g = G[(long long)i * ld + j];
            const double gap = dg[j] - dg[i];
            const double ag = sqrt(g.x * g.x + g.y * g.y);
            if (ag < 0.5 * fabs(gap)) v = make_float2((float)(g.x / gap), (float)(g.y / gap));
        }
        A[t * TR_RS + i] = v;
    }
    __syncthreads();
    auto bnorm = [&](const float2* w) {
        float ss = 0.f;
        for (int i = tid; i < r; i += TR_THREADS) ss += w[i].x * w[i].x + w[i].y * w[i].y;
        return sqrtf(block_sum(ss, red, tid));
    };
    auto project_out = [&](float2* w, int t) {
        for (int q = warp; q < t; q += NW) {
            const float2* u = A + q * TR_RS;
            float cr = 0.f, ci = 0.f;
            for (int i = lane; i < r; i += 32) {
                const float2 a = u[i], b = w[i];
                cr = fmaf(a.x, b.x, fmaf(a.y, b.y, cr));
                ci = fmaf(a.x, b.y, fmaf(-a.y, b.x, ci));
            }
            for (int off = 16; off > 0; off >>= 1) {
                cr += __shfl_xor_sync(0xffffffffu, cr, off);
                ci += __shfl_xor_sync(0xffffffffu, ci, off);
            }
            if (lane == 0) { coef_r[q] = cr; coef_i[q] = ci; }
        }
        __syncthreads();
        for (int i = warp; i < r; i += NW) {
            float ar = 0.f, ai = 0.f;
            for (int q = lane; q < t; q += 32) {
                const float2 u = A[q * TR_RS + i];
                ar += coef_r[q] * u.x - coef_i[q] * u.y;
                ai += coef_r[q] * u.y + coef_i[q] * u.x;
            }
            for (int off = 16; off > 0; off >>= 1) {
                ar += __shfl_xor_sync(0xffffffffu, ar, off);
                ai += __shfl_xor_sync(0xffffffffu, ai, off);
            }
            if (lane == 0) w[i] = make_float2(w[i].x - ar, w[i].y - ai);
        }
        __syncthreads();
    };
    for (int t = 0; t < r; ++t) {
        float2* w = A + t * TR_RS;
        for (int attempt = 0; attempt < 2; ++attempt) {
            if (attempt == 1) {
                for (int i = tid; i < r; i += TR_THREADS) w[i] = gauss2(977 + t, i, t);
                __syncthreads();
            }
            const float n0 = bnorm(w);
            if (!(n0 > 0.f)) continue;
            for (int i = tid; i < r; i += TR_THREADS) w[i] = cscale(w[i], 1.f / n0);
            __syncthreads();
            project_out(w, t);
            float na = bnorm(w);
            if (na < 0.7f) {
                project_out(w, t);
                na = bnorm(w);
            }
            const float sc = (na > 1e-4f) ? 1.f / na : 0.f;
            for (int i = tid; i < r; i += TR_THREADS) w[i] = cscale(w[i], sc);
            __syncthreads();
            if (na > 1e-4f) break;
        }
    }
    for (int e = tid; e < r * r; e += TR_THREADS) {
        const int i = e % r, t = e / r;
        V[(long long)order[t] * ldv + i] = A[t * TR_RS + i];
    }
}

cudaError_t launch_refine_basis(const double2* G, Dim ld, Dim r, float2* V, int ldv, const int* R, cudaStream_t s) {
    const size_t smem = (size_t)EIG_MAX * TR_RS * sizeof(float2);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_refine_basis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    count_launch(PROF_EIG, s, true);
    k_refine_basis<<<1, TR_THREADS, smem, s>>>(G, ld, r, V, ldv, R);
    count_launch(PROF_EIG, s, false);
    return cudaGetLastError();
}

cudaError_t launch_eig_trd(const double2* G, Dim ld, Dim r, float2* U, Dim ldu, double* lam, const int* R,
                           cudaStream_t s, int guard_reg, int guard_val) {
    const size_t smem = (size_t)EIG_MAX * TR_RS * sizeof(float2);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_heev_trd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    count_launch(PROF_EIG, s, true);
    k_heev_trd<<<1, TR_THREADS, smem, s>>>(G, ld, r, U, ldu, lam, R, guard_reg, guard_val,
                                          g_prof_ledger ? g_prof_ledger + L_PROF_EIG : nullptr);
    count_launch(PROF_EIG, s, false);
    return cudaGetLastError();
}

}  // namespace qtn
