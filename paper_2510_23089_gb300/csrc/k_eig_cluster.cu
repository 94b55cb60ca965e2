// One-sided Jacobi eigen-solve of a Hermitian positive semi-definite r x r matrix (the FP64-accumulated Gram
// of a truncation, Sec. IV and App. A: the SVD behind every truncation), spread over a thread-block cluster.
//
// The columns of W = G / s (s the largest diagonal entry) are split into 2 C blocks of BS columns; each of the
// C CTAs of the cluster holds two blocks in its shared memory together with the matching columns of V, which
// starts as the identity and receives every rotation applied to W.  A sweep is a round-robin tournament of
// the blocks (circle method, 2 C - 1 rounds): in a round every CTA orthogonalises all column pairs across its
// two blocks (BS slots of BS disjoint pairs, one warp per pair), in the first round of a sweep also the pairs
// inside each block; then the blocks move to their next CTA through distributed shared memory and the cluster
// meets at one barrier.  At convergence W = G V has orthogonal columns, so V diagonalises G: its columns are
// the eigenvectors, orthonormal to the FP32 rounding of the rotations whatever the eigenvalue (no
// re-orthonormalisation, no completion), and the column norms of W are the eigenvalues.
//
// Every CTA evaluates the same guards and the same convergence decision (the per-CTA rotation flags are
// exchanged through distributed shared memory before each sweep's last barrier), so all CTAs meet the same
// sequence of cluster barriers.
#include <cooperative_groups.h>

#include "qtn_internal.cuh"

namespace cg = cooperative_groups;

namespace qtn {

constexpr int ECL_C = 8;                          // CTAs per cluster
constexpr int ECL_BS = EIG_MAX / (2 * ECL_C);     // columns per block at most
constexpr int ECL_THREADS = 32 * ECL_BS;          // one warp per column pair of a slot
constexpr int ECL_LD = EIG_MAX;                   // rows of a stored column
constexpr float ECL_NOISE = 1.0e-13f;             // |w_i| |w_j| floor of the scaled matrix (rounding level)
constexpr float ECL_SIG = 1.0e-6f;                // pairs below this are rounding when judging convergence

// A block of columns: W and V columns of BS Jacobi columns and their global indices (-1: no column).
struct alignas(16) EclBlock {
    float2 W[ECL_BS][ECL_LD];
    float2 V[ECL_BS][ECL_LD];
    int id[16];
};
constexpr size_t ECL_SMEM = 4 * sizeof(EclBlock);   // two active blocks and two incoming

// Round-robin pairing of n (even) players, round u in [0, n-2], pair k in [0, n/2).
__device__ __forceinline__ void ecl_circle(int u, int k, int n, int& i, int& j) {
    const int m = n - 1;
    if (k == 0) { i = u; j = m; }
    else { i = (u + k) % m; j = (u - k + m) % m; }
}

constexpr int ECL_RPL = ECL_LD / 32;             // rows of a column held by one lane (rows lane + 32 k)

// Rows of one column, in registers (rows beyond the live order are zero in shared memory).
__device__ __forceinline__ void ecl_load(const float2* __restrict__ col, float2 (&x)[ECL_RPL], int lane) {
#pragma unroll
    for (int k = 0; k < ECL_RPL; ++k) x[k] = col[lane + 32 * k];
}
__device__ __forceinline__ void ecl_store(float2* __restrict__ col, const float2 (&x)[ECL_RPL], int lane) {
#pragma unroll
    for (int k = 0; k < ECL_RPL; ++k) col[lane + 32 * k] = x[k];
}

// The plane rotation that orthogonalises columns x and y (one warp, rows in registers) when their inner product
// exceeds tol of their norms: returns false when the pair is left alone.  The sums are butterfly reductions,
// so every lane holds the same bits and takes the same branch.
__device__ __forceinline__ bool ecl_rotation(const float2 (&x)[ECL_RPL], const float2 (&y)[ECL_RPL], float tol,
                                             float& cs, float& pr, float& pi, bool& sig) {
    float a = 0.f, b = 0.f, cr = 0.f, ci = 0.f;
#pragma unroll
    for (int k = 0; k < ECL_RPL; ++k) {
        a = fmaf(x[k].x, x[k].x, fmaf(x[k].y, x[k].y, a));
        b = fmaf(y[k].x, y[k].x, fmaf(y[k].y, y[k].y, b));
        cr = fmaf(x[k].x, y[k].x, fmaf(x[k].y, y[k].y, cr));      // conj(x) * y
        ci = fmaf(x[k].x, y[k].y, fmaf(-x[k].y, y[k].x, ci));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
        cr += __shfl_xor_sync(0xffffffffu, cr, off);
        ci += __shfl_xor_sync(0xffffffffu, ci, off);
    }
    const float c2 = fmaf(cr, cr, ci * ci);
    const float ab2 = a * b;
    if (!(c2 > tol * tol * ab2) || !(c2 > 0.f) || !(ab2 > ECL_NOISE * ECL_NOISE)) return false;
    // Hermitian 2 x 2 problem [[a, c], [conj c, b]]: tan(theta) from zeta = (b - a) / (2 |c|), smaller root
    const float ic = rsqrtf(c2);
    const float zeta = 0.5f * (b - a) * ic;
    const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
    cs = rsqrtf(fmaf(tt, tt, 1.f));
    const float tc = tt * cs * ic;
    pr = tc * cr;                                   // p = sin(theta) c / |c|
    pi = tc * ci;
    sig = ab2 > ECL_SIG * ECL_SIG;
    return true;
}

// x' = cs x - conj(p) y ;  y' = p x + cs y
__device__ __forceinline__ void ecl_apply(float2 (&x)[ECL_RPL], float2 (&y)[ECL_RPL], float cs, float pr, float pi) {
#pragma unroll
    for (int k = 0; k < ECL_RPL; ++k) {
        const float2 u = x[k], v = y[k];
        x[k] = make_float2(fmaf(cs, u.x, -fmaf(pr, v.x, pi * v.y)), fmaf(cs, u.y, -fmaf(pr, v.y, -pi * v.x)));
        y[k] = make_float2(fmaf(cs, v.x, fmaf(pr, u.x, -pi * u.y)), fmaf(cs, v.y, fmaf(pr, u.y, pi * u.x)));
    }
}

// One pair of columns held in shared memory (W, and V when ACCV), handled by one warp.
template <bool ACCV>
__device__ __forceinline__ void ecl_pair(float2* __restrict__ wx, float2* __restrict__ wy, float2* __restrict__ vx,
                                         float2* __restrict__ vy, int lane, float tol, int& rotated, int& sig_rotated,
                                         unsigned long long& n_pairs, unsigned long long& n_rot) {
    float2 x[ECL_RPL], y[ECL_RPL];
    ecl_load(wx, x, lane);
    ecl_load(wy, y, lane);
    ++n_pairs;
    float cs, pr, pi;
    bool sig;
    if (!ecl_rotation(x, y, tol, cs, pr, pi, sig)) return;
    ecl_apply(x, y, cs, pr, pi);
    ecl_store(wx, x, lane);
    ecl_store(wy, y, lane);
    if (ACCV) {
        ecl_load(vx, x, lane);
        ecl_load(vy, y, lane);
        ecl_apply(x, y, cs, pr, pi);
        ecl_store(vx, x, lane);
        ecl_store(vy, y, lane);
    }
    ++n_rot;
    rotated = 1;
    if (sig) sig_rotated = 1;
}

// Copies the BS live columns (W, and V when ACCV) and the column indices of `src` into buffer `dst_buf` of CTA
// `dst_cta` (its own shared memory when dst_cta is this CTA).
template <bool ACCV>
__device__ __forceinline__ void ecl_send(cg::cluster_group& cluster, const EclBlock& src, EclBlock* buf, int dst_buf,
                                         int dst_cta, int BS, int tid) {
    EclBlock* dst = cluster.map_shared_rank(buf + dst_buf, dst_cta);
    const float4* s4 = reinterpret_cast<const float4*>(&src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    constexpr int per_col = ECL_LD / 2;                        // float4 per column
    constexpr int per_mtx = ECL_BS * per_col;                  // float4 offset of V
    for (int e = tid; e < (ACCV ? 2 : 1) * BS * per_col; e += ECL_THREADS) {
        const int mtx = e / (BS * per_col), rem = e - mtx * (BS * per_col);
        d4[mtx * per_mtx + rem] = s4[mtx * per_mtx + rem];
    }
    if (tid < 16) dst->id[tid] = src.id[tid];
}

// ACCV: rotations accumulated into V and the sorted eigenvectors written to U (columns by descending
// eigenvalue) with the eigenvalues in lam.  !ACCV: the rotated columns of W = G V / s written unsorted to U
// (column j at U + j ldu, in the units of G / s) for k_eig_finish, which takes the eigenvectors as their
// normalised columns.
template <bool ACCV>
__global__ void __cluster_dims__(ECL_C, 1, 1) __launch_bounds__(ECL_THREADS, 1)
k_eig_cluster(const double2* __restrict__ G, Dim ldd, Dim rdim, float2* __restrict__ U, Dim ldud,
              double* __restrict__ lam, const int* Rc, int* Rw, int max_sweeps, int guard_reg, int guard_val,
              double* __restrict__ prof, float tol, int report_nonconv, int r_min) {
    // the guards read the same registers in every CTA: the whole cluster returns or none of it
    if (guard_reg >= 0 && Rc[guard_reg] != guard_val) return;
    const int r = rdim.eval(Rc);
    if (r < r_min || r < 2 || r > EIG_MAX) return;
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    extern __shared__ __align__(16) unsigned char ecl_smem[];
    EclBlock* buf = reinterpret_cast<EclBlock*>(ecl_smem);
    __shared__ int flag_all[2][ECL_C], sig_all[2][ECL_C];
    __shared__ int rot_s, sig_s;
    __shared__ double gscale_s;
    __shared__ double lam_all[EIG_MAX];
    const long long ld = ldd.eval(Rc), ldu = ldud.eval(Rc);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int BS = (r + 2 * ECL_C - 1) / (2 * ECL_C);
    // Scale by the largest diagonal entry: the squared column norms of W stay inside the FP32 range.
    if (warp == 0) {
        double mx = 0.0;
        for (int i = lane; i < r; i += 32) mx = fmax(mx, fabs(G[(long long)i * ld + i].x));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        if (lane == 0) gscale_s = (mx > 0.0 && isfinite(mx)) ? mx : 1.0;
    }
    if (tid == 0) { rot_s = 0; sig_s = 0; }
    __syncthreads();
    const double inv_scale = 1.0 / gscale_s;
    // Blocks q and C + q start in buffers 0 and 1.  Column j of W is column j of G (read as the conjugate of
    // row j: G is Hermitian and its rows are contiguous), column j of V is e_j.
    for (int h = 0; h < 2; ++h) {
        EclBlock& B = buf[h];
        const int b = (h == 0) ? q : ECL_C + q;
        if (tid < 16) B.id[tid] = (tid < BS && b * BS + tid < r) ? b * BS + tid : -1;
        for (int e = tid; e < BS * ECL_LD; e += ECL_THREADS) {
            const int k = e / ECL_LD, row = e - k * ECL_LD;
            const int j = b * BS + k;
            float2 wv = make_float2(0.f, 0.f), vv = wv;
            if (j < r && row < r) {
                const double2 g = G[(long long)j * ld + row];
                wv = make_float2((float)(g.x * inv_scale), (float)(-g.y * inv_scale));
                if (row == j) vv = make_float2(1.f, 0.f);
            }
            B.W[k][row] = wv;
            if (ACCV) B.V[k][row] = vv;
        }
    }
    __syncthreads();
    cluster.sync();   // every CTA of the cluster runs before the first store into another CTA's memory

    const int nrounds = 2 * ECL_C - 1;
    int my_rot = 0, my_sig = 0, last_sig = 0;
    unsigned long long n_pairs = 0ull, n_rot = 0ull;
    int par = 0;                                     // active buffers 2 par, 2 par + 1
    int sweep = 0;
    bool converged = false;
    for (; sweep < max_sweeps && !converged; ++sweep) {
        for (int t = 0; t < nrounds; ++t) {
            EclBlock& X = buf[2 * par];
            EclBlock& Y = buf[2 * par + 1];
            if (t == 0) {   // pairs inside each block: warps [0, BSe/2) on X, [BSe/2, BSe) on Y
                const int BSe = BS + (BS & 1), half = BSe / 2;
                for (int u = 0; u < BSe - 1; ++u) {
                    if (warp < BSe) {
                        EclBlock& Z = (warp < half) ? X : Y;
                        int i, j;
                        ecl_circle(u, warp % half, BSe, i, j);
                        if (i < BS && j < BS && Z.id[i] >= 0 && Z.id[j] >= 0)
                            ecl_pair<ACCV>(Z.W[i], Z.W[j], Z.V[i], Z.V[j], lane, tol, my_rot, my_sig, n_pairs, n_rot);
                    }
                    __syncthreads();
                }
            }
            {   // pairs across the two blocks: warp i keeps X_i in registers, slot s pairs it with Y_(i+s) mod BS
                const bool act = (warp < BS) && X.id[warp] >= 0;
                float2 xw[ECL_RPL], xv[ECL_RPL];
                if (act) {
                    ecl_load(X.W[warp], xw, lane);
                    if (ACCV) ecl_load(X.V[warp], xv, lane);
                }
                for (int s = 0; s < BS; ++s) {
                    const int j = (warp + s) % BS;
                    if (act && Y.id[j] >= 0) {
                        float2 yw[ECL_RPL];
                        ecl_load(Y.W[j], yw, lane);
                        ++n_pairs;
                        float cs, pr, pi;
                        bool sig;
                        if (ecl_rotation(xw, yw, tol, cs, pr, pi, sig)) {
                            ecl_apply(xw, yw, cs, pr, pi);
                            ecl_store(Y.W[j], yw, lane);
                            if (ACCV) {
                                float2 yv[ECL_RPL];
                                ecl_load(Y.V[j], yv, lane);
                                ecl_apply(xv, yv, cs, pr, pi);
                                ecl_store(Y.V[j], yv, lane);
                            }
                            ++n_rot;
                            my_rot = 1;
                            if (sig) my_sig = 1;
                        }
                    }
                    __syncthreads();
                }
                if (act) {
                    ecl_store(X.W[warp], xw, lane);
                    if (ACCV) ecl_store(X.V[warp], xv, lane);
                }
                __syncthreads();
            }
            if (t == nrounds - 1) {          // end of the sweep: this CTA's flags to every CTA of the cluster
                if (lane == 0 && (my_rot | my_sig)) {
                    atomicOr(&rot_s, my_rot);
                    atomicOr(&sig_s, my_sig);
                }
                __syncthreads();
                if (tid < ECL_C) {
                    int* rf = cluster.map_shared_rank(&flag_all[sweep & 1][0], tid);
                    int* sf = cluster.map_shared_rank(&sig_all[sweep & 1][0], tid);
                    rf[q] = rot_s;
                    sf[q] = sig_s;
                }
            }
            // Circle method: the top block of CTA 0 stays; top blocks move to the next CTA (the last CTA's top
            // becomes its bottom), bottom blocks to the previous CTA (CTA 0's bottom becomes CTA 1's top).
            const int nb = 1 - par;
            if (q == 0) {
                ecl_send<ACCV>(cluster, X, buf, 2 * nb, 0, BS, tid);
                ecl_send<ACCV>(cluster, Y, buf, 2 * nb, 1, BS, tid);
            } else {
                if (q < ECL_C - 1) ecl_send<ACCV>(cluster, X, buf, 2 * nb, q + 1, BS, tid);
                else ecl_send<ACCV>(cluster, X, buf, 2 * nb + 1, q, BS, tid);
                ecl_send<ACCV>(cluster, Y, buf, 2 * nb + 1, q - 1, BS, tid);
            }
            cluster.sync();
            par = nb;
        }
        // the same decision in every CTA
        int any = 0, anys = 0;
        for (int p = 0; p < ECL_C; ++p) {
            any |= flag_all[sweep & 1][p];
            anys |= sig_all[sweep & 1][p];
        }
        // The refinement (W out) stops once a sweep rotates no pair above the rounding level of the scaled Gram
        // (eigenvalue products below 1e-6 of the largest squared): pairs of directions that small are left to
        // the finishing step, which orthonormalises them after the larger ones; the rough first solve stops on
        // no rotation at all (or at its sweep cap).
        converged = ACCV ? (any == 0) : (anys == 0);
        last_sig = anys;
        if (tid == 0) { rot_s = 0; sig_s = 0; }
        my_rot = my_sig = 0;
    }
    if (!ACCV) {   // the rotated columns of W, unsorted, for the finishing kernel
        for (int h = 0; h < 2; ++h) {
            const EclBlock& B = buf[2 * par + h];
            for (int e = tid; e < BS * r; e += ECL_THREADS) {
                const int k = e / r, row = e - k * r;
                const int j = B.id[k];
                if (j >= 0) U[(long long)j * ldu + row] = B.W[k][row];
            }
        }
    } else {
        // eigenvalues: column norms of W (FP64 sums) in the units of G, published to every CTA
        for (int h = 0; h < 2; ++h) {
            EclBlock& B = buf[2 * par + h];
            for (int k = warp; k < BS; k += ECL_THREADS / 32) {
                const int j = B.id[k];
                if (j < 0) continue;
                double s2 = 0.0;
                for (int row = lane; row < r; row += 32) {
                    const float2 x = B.W[k][row];
                    s2 += (double)x.x * x.x + (double)x.y * x.y;
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
                if (lane < ECL_C) {
                    double* la = cluster.map_shared_rank(&lam_all[0], lane);
                    la[j] = sqrt(s2) * gscale_s;
                }
            }
        }
        cluster.sync();
        // descending-eigenvalue rank of every column (ties by index); U column rank = V column, lam[rank]
        for (int h = 0; h < 2; ++h) {
            EclBlock& B = buf[2 * par + h];
            for (int k = warp; k < BS; k += ECL_THREADS / 32) {
                const int j = B.id[k];
                if (j < 0) continue;
                const double v = lam_all[j];
                int rk = 0;
                for (int i = lane; i < r; i += 32) {
                    const double u = lam_all[i];
                    rk += (u > v) || (u == v && i < j);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) rk += __shfl_xor_sync(0xffffffffu, rk, off);
                for (int row = lane; row < r; row += 32) U[(long long)rk * ldu + row] = B.V[k][row];
                if (lane == 0) lam[rk] = v;
            }
        }
    }
    if (prof != nullptr && lane == 0 && (n_pairs | n_rot))
        atomicAdd(prof, 8.0 * r * (double)n_pairs + (ACCV ? 48.0 : 24.0) * r * (double)n_rot);
    if (q == 0 && tid == 0) {
        atomicMax(&Rw[R_SWEEPS], sweep);
        // unconverged only when the last sweep still rotated a pair above the rounding level of the scaled Gram
        if (!converged && report_nonconv && last_sig) raise_flag(Rw, F_NOCONV);
    }
}

cudaError_t launch_eig_cluster(const double2* G, Dim ld, Dim r, float2* U, Dim ldu, double* lam, const int* R,
                               int max_sweeps, cudaStream_t s, int guard_reg, int guard_val, double* prof, float tol,
                               bool report_nonconv, int r_min, bool accumulate) {
    if (accumulate)
        k_eig_cluster<true><<<ECL_C, ECL_THREADS, ECL_SMEM, s>>>(G, ld, r, U, ldu, lam, R, (int*)R, max_sweeps,
                                                                guard_reg, guard_val, prof, tol, report_nonconv ? 1 : 0,
                                                                r_min);
    else
        k_eig_cluster<false><<<ECL_C, ECL_THREADS, ECL_SMEM, s>>>(G, ld, r, U, ldu, lam, R, (int*)R, max_sweeps,
                                                                 guard_reg, guard_val, prof, tol,
                                                                 report_nonconv ? 1 : 0, r_min);
    return cudaGetLastError();
}

cudaError_t configure_eig_cluster_kernel() {
    cudaError_t e = cudaFuncSetAttribute(k_eig_cluster<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ECL_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_eig_cluster<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ECL_SMEM);
    return e;
}

}  // namespace qtn
