// FP64 construction of the per-axis diagonal and Fourier operators (one CTA per build).
//
// An operator on n qubits is held as a d = 4 matrix product state whose physical index is the pair
// (out, in) = (t, s), ph = 2 t + s (Sec. VI.A, Fig. MPO_construction: an MPO is an MPS with paired legs).
// Circuit layers (the QFT's Hadamard-plus-controlled-phase layers, the controlled-phase layers of the
// quadratic Fresnel phase, the Pauli-Z string gates of Sec. VI.B.3) are absorbed one at a time by a zip-up
// pass in FP64: the carry, the site and the layer core are contracted to T[(x, t, s), (b, k)], T is
// factorised through the eigen-decomposition of the FP64 Gram of its short side (cyclic two-sided Jacobi
// in shared memory), the rank follows the relative cutoff, and the pass direction alternates so every pass
// starts from the canonical form it needs.  The result is rounded once to complex64.
//
// The builds run once per operator; they are sequential small-matrix work in one CTA, so the FP64 rate of
// the chip does not matter and the operators are exact to FP64 rounding plus the requested cutoff.
#include <math.h>

#include "qtn_internal.cuh"

namespace qtn {

constexpr int B64_CAP = BUILD64_BOND_CAP;   // bond capacity of an operator under construction
constexpr int B64_EIG = 64;        // largest Gram (short side of a site unfolding: 2 * B64_CAP columns)
constexpr int B64_LD = B64_EIG + 1;
constexpr int B64_MAXN = 64;
constexpr int B64_THREADS = 256;
constexpr size_t B64_SMEM = 2 * (size_t)B64_EIG * B64_LD * sizeof(double2);

constexpr int BK_QFT = BUILD64_QFT, BK_QPHASE = BUILD64_QPHASE, BK_PAULIZ = BUILD64_PAULIZ,
              BK_BESSEL = BUILD64_BESSEL;
constexpr int BK_IDENT = 99;   // identity layer: a pass of it only moves the canonical centre

// Scratch of a build, in global memory (sizes for n <= B64_MAXN are in build64_scratch_bytes).
struct Scr64 {
    double2* site;    // [n][CAP][4][CAP], stored orientation
    double2* T;       // (4 CAP) x (2 CAP)
    double2* carry;   // CAP x (2 CAP)
    double2* U;       // (4 CAP) x CAP
    double* wh;       // 2^n reals (Walsh-Hadamard coefficients of the Pauli-Z builder)
};

size_t build64_scratch_bytes(int n) {
    const size_t site = (size_t)n * B64_CAP * 4 * B64_CAP * sizeof(double2);
    const size_t t = (size_t)4 * B64_CAP * 2 * B64_CAP * sizeof(double2);
    const size_t carry = (size_t)B64_CAP * 2 * B64_CAP * sizeof(double2);
    const size_t u = (size_t)4 * B64_CAP * B64_CAP * sizeof(double2);
    return site + t + carry + u + 4096;
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 zexpi_pi(double x) {   // exp(i pi x), argument reduced modulo 2 first
    double s, c;
    sincospi(fmod(x, 2.0), &s, &c);
    return make_double2(c, s);
}

// One layer (bond <= 2 MPO) in the stored site order.
struct Layer {
    int kind;          // BK_QFT, BK_QPHASE, BK_PAULIZ
    int n, j;          // qubits; QFT layer / control qubit of a phase layer
    double c;          // quadratic phase: lambda z / (L dx^2)
    double omega;      // Pauli-Z gate angle (c_S t)
    unsigned long long mask;   // Pauli-Z gate: sites of the string
    int first, last;   // Pauli-Z gate: first and last site of the string
};

__device__ void layer_bonds(const Layer& L, int q, int& wl, int& wr) {
    const int n = L.n;
    if (L.kind == BK_IDENT) {
        wl = wr = 1;
        return;
    }
    if (L.kind == BK_PAULIZ) {
        wl = (q > L.first && q <= L.last) ? 2 : 1;
        wr = (q >= L.first && q < L.last) ? 2 : 1;
        return;
    }
    // QFT and phase layers: bond 2 from the control qubit j to the chain end
    wl = (q > L.j) ? 2 : 1;
    wr = (q >= L.j && q < n - 1) ? 2 : 1;
}

// Two's-complement weight a_q of frequency bit q in k_f (bit-reversed order: site q holds bit q of k):
// k_f = sum_q a_q k_q with a_q = 2^q (q < n-1), a_{n-1} = -2^(n-1).  Returns (sign, exponent).
__device__ __forceinline__ void fbit_weight(int q, int n, double& sgn, int& e) {
    e = q;
    sgn = (q == n - 1) ? -1.0 : 1.0;
}

// Core value W_q[a, t, u, b] (a, b: layer bonds in stored orientation; t: out, u: in).
__device__ double2 layer_core(const Layer& L, int q, int a, int t, int u, int b) {
    const int n = L.n;
    const double2 zero = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0);
    int wl, wr;
    layer_bonds(L, q, wl, wr);
    if (a >= wl || b >= wr) return zero;
    if (L.kind == BK_IDENT) return (t == u) ? one : zero;
    if (L.kind == BK_QFT) {
        const int j = L.j;
        if (q < j) return (t == u) ? one : zero;
        if (q == j) {   // Hadamard, the output bit carried on the bond
            if (wr == 2 && b != t) return zero;
            const double h = 0.70710678118654752440;
            return make_double2((t == 1 && u == 1) ? -h : h, 0.0);
        }
        // controlled phase exp(i pi b s / 2^(q - j)) on target q
        if (t != u) return zero;
        if (wr == 2 && b != a) return zero;
        return zexpi_pi((double)(a * t) / (double)(1ll << (q - j)));
    }
    if (L.kind == BK_QPHASE) {
        // exp(-i pi c k_f^2 / L) = prod_q exp(-i pi c a_q^2 k_q / L) prod_{i<q} exp(-2 i pi c a_i a_q k_i k_q / L)
        if (t != u) return zero;
        const int i = L.j;
        if (q < i) return one;
        double si, sq;
        int ei, eq;
        fbit_weight(i, n, si, ei);
        if (q == i) {
            if (wr == 2 && b != t) return zero;
            // phase / pi = -c a_i^2 k_i / L = -c 2^(2 ei - n) k_i
            return t ? zexpi_pi(-L.c * ldexp(1.0, 2 * ei - n)) : one;
        }
        if (wr == 2 && b != a) return zero;
        fbit_weight(q, n, sq, eq);
        // phase / pi = -2 c a_i a_q k_i k_q / L = -c si sq 2^(ei + eq + 1 - n)
        return (a && t) ? zexpi_pi(-L.c * si * sq * ldexp(1.0, ei + eq + 1 - n)) : one;
    }
    // Pauli-Z string gate exp(-i omega P_S) = cos(omega) I - i sin(omega) P_S (Sec. VI.B.3, Eq. U-product_1)
    if (t != u) return zero;
    const bool in_s = (L.mask >> q) & 1ull;
    const double z = (t == 0) ? 1.0 : -1.0;
    if (q < L.first || q > L.last) return one;
    if (L.first == L.last) {
        double s, c;
        sincos(L.omega, &s, &c);
        return make_double2(c, -s * z);
    }
    if (q == L.first) {
        double s, c;
        sincos(L.omega, &s, &c);
        return (b == 0) ? make_double2(c, 0.0) : make_double2(0.0, -s * z);
    }
    if (q < L.last) {
        if (a != b) return zero;
        return make_double2((a == 1 && in_s) ? z : 1.0, 0.0);
    }
    return make_double2((a == 1) ? z : 1.0, 0.0);   // last site of the string closes the bond
}

// Cyclic two-sided Jacobi eigen-decomposition of a Hermitian r x r matrix A (shared memory, row stride
// B64_LD), eigenvectors in the columns of V; on return lam[i] = A_ii and perm sorts them descending.
// Parallel rounds of the round-robin ordering: the rotation parameters of all r/2 disjoint pairs come from
// the matrix at the start of the round, then every pair's columns, then every pair's rows are rotated (the
// pairs touch disjoint rows and columns, so this equals applying them one after another).
__device__ void eig_herm64(double2* A, double2* V, int r, double* lam, int* perm, double* cs_s, double* sn_s,
                           double2* ph_s, int* flag) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < r * r; e += nt) V[(e / r) * B64_LD + e % r] = make_double2((e / r) == (e % r), 0.0);
    const int rr = r + (r & 1);
    if (tid == 0) {
        double dmax = 0.0;
        for (int i = 0; i < r; ++i) dmax = fmax(dmax, fabs(A[i * B64_LD + i].x));
        lam[0] = dmax;
    }
    __syncthreads();
    const double floor_abs = 1e-18 * lam[0];   // off-diagonal entries below this are rounding of the scale
    __syncthreads();
    for (int sweep = 0; sweep < 60 && r > 1; ++sweep) {
        if (tid == 0) *flag = 0;
        __syncthreads();
        for (int round = 0; round < rr - 1; ++round) {
            // pair k of this round: (round + k) % (rr - 1) with (round - k) % (rr - 1), and k = 0 pairs with rr - 1
            for (int k = tid; k < rr / 2; k += nt) {
                int p, q;
                if (k == 0) { p = round; q = rr - 1; }
                else { p = (round + k) % (rr - 1); q = (round - k + rr - 1) % (rr - 1); }
                if (p > q) { const int tmp = p; p = q; q = tmp; }
                cs_s[k] = 1.0; sn_s[k] = 0.0; ph_s[k] = make_double2(1.0, 0.0);
                if (q >= r) continue;
                const double a = A[p * B64_LD + p].x, b = A[q * B64_LD + q].x;
                const double2 c = A[p * B64_LD + q];
                const double ca = hypot(c.x, c.y);
                if (!(ca > 1e-15 * sqrt(fabs(a * b))) || !(ca > floor_abs) || !(ca > 1e-300)) continue;
                // D = diag(1, e^{-i phi}) makes the pair real: [[a, |c|], [|c|, b]]; then a real rotation
                const double tau = (b - a) / (2.0 * ca);
                const double tt = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
                cs_s[k] = 1.0 / sqrt(1.0 + tt * tt);
                sn_s[k] = tt * cs_s[k];
                ph_s[k] = make_double2(c.x / ca, c.y / ca);   // e^{i phi}
                *flag = 1;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J with J = [[cs, sn], [-sn e^{-i phi}, cs e^{-i phi}]]
            for (int e = tid; e < (rr / 2) * r; e += nt) {
                const int k = e / r, i = e % r;
                int p, q;
                if (k == 0) { p = round; q = rr - 1; }
                else { p = (round + k) % (rr - 1); q = (round - k + rr - 1) % (rr - 1); }
                if (p > q) { const int tmp = p; p = q; q = tmp; }
                if (q >= r || sn_s[k] == 0.0) continue;
                const double cs = cs_s[k], sn = sn_s[k];
                const double2 em = zconj(ph_s[k]);
                double2* Ap = A + i * B64_LD + p;
                double2* Aq = A + i * B64_LD + q;
                const double2 xp = *Ap, xq = zmul(*Aq, em);
                *Ap = make_double2(cs * xp.x - sn * xq.x, cs * xp.y - sn * xq.y);
                *Aq = make_double2(sn * xp.x + cs * xq.x, sn * xp.y + cs * xq.y);
                double2* Vp = V + i * B64_LD + p;
                double2* Vq = V + i * B64_LD + q;
                const double2 vp = *Vp, vq = zmul(*Vq, em);
                *Vp = make_double2(cs * vp.x - sn * vq.x, cs * vp.y - sn * vq.y);
                *Vq = make_double2(sn * vp.x + cs * vq.x, sn * vp.y + cs * vq.y);
            }
            __syncthreads();
            // rows: A <- J^dagger A; row_p' = cs row_p - sn e^{i phi} row_q, row_q' = sn row_p + cs e^{i phi} row_q
            for (int e = tid; e < (rr / 2) * r; e += nt) {
                const int k = e / r, j = e % r;
                int p, q;
                if (k == 0) { p = round; q = rr - 1; }
                else { p = (round + k) % (rr - 1); q = (round - k + rr - 1) % (rr - 1); }
                if (p > q) { const int tmp = p; p = q; q = tmp; }
                if (q >= r || sn_s[k] == 0.0) continue;
                const double cs = cs_s[k], sn = sn_s[k];
                double2* Ap = A + p * B64_LD + j;
                double2* Aq = A + q * B64_LD + j;
                const double2 xp = *Ap, xq = zmul(*Aq, ph_s[k]);
                *Ap = make_double2(cs * xp.x - sn * xq.x, cs * xp.y - sn * xq.y);
                *Aq = make_double2(sn * xp.x + cs * xq.x, sn * xp.y + cs * xq.y);
            }
            __syncthreads();
        }
        const int any = *flag;
        __syncthreads();
        if (!any) break;
    }
    for (int i = tid; i < r; i += nt) lam[i] = A[i * B64_LD + i].x;
    __syncthreads();
    for (int i = tid; i < r; i += nt) {
        int rk = 0;
        for (int j = 0; j < r; ++j) rk += (lam[j] > lam[i]) || (lam[j] == lam[i] && j < i);
        perm[rk] = i;
    }
    __syncthreads();
}

// Stored offset of element (l, ph, r) of site q seen in sweep orientation (mirror swaps l and r).
__device__ __forceinline__ size_t s64_off(int q, int l, int ph, int r, int mirror) {
    const size_t base = (size_t)q * B64_CAP * 4 * B64_CAP;
    return mirror ? base + ((size_t)r * 4 + ph) * B64_CAP + l : base + ((size_t)l * 4 + ph) * B64_CAP + r;
}

// One zip-up pass of a layer over the operator-state (sweep orientation `mirror`: 0 left to right on a
// right-canonical state, 1 right to left on a left-canonical one).  bond[] in shared memory.
__device__ void zip64(const Layer& Ly, Scr64& S, int* bond, int n, int mirror, double cutoff, int* status,
                      double2* A, double2* V, double* lam, int* perm, double* cs_s, double* sn_s, double2* ph_s,
                      int* flag, int* dims) {
    const int tid = threadIdx.x, nt = blockDim.x;
    // carry C[x][a][j]: dims kx x wa x jj, row-major
    if (tid == 0) { S.carry[0] = make_double2(1.0, 0.0); dims[0] = 1; dims[1] = 1; dims[2] = 1; }
    __syncthreads();
    for (int p = 0; p < n; ++p) {
        const int q = mirror ? n - 1 - p : p;
        // left bond of the input site = the carry's last dimension (bond[] already holds the new bonds to the
        // left); right bond of the input site, not yet overwritten
        const int chl = dims[2], chr = mirror ? bond[q] : bond[q + 1];
        int wl, wr;
        layer_bonds(Ly, q, wl, wr);
        if (mirror) { const int tmp = wl; wl = wr; wr = tmp; }
        const int kx = dims[0];
        const int m = kx * 4, ncol = wr * chr;
        // T[(x, t, s), (b, k)] = sum_{a, u, j} C[x, a, j] A[j, (u, s), k] W[a, t, u, b]
        for (int e = tid; e < m * ncol; e += nt) {
            const int x = e / (4 * ncol), t = (e / (2 * ncol)) % 2, s = (e / ncol) % 2;
            const int b = (e % ncol) / chr, k = (e % ncol) % chr;
            double2 acc = make_double2(0.0, 0.0);
            for (int a = 0; a < wl; ++a)
                for (int u = 0; u < 2; ++u) {
                    const double2 w = mirror ? layer_core(Ly, q, b, t, u, a) : layer_core(Ly, q, a, t, u, b);
                    if (w.x == 0.0 && w.y == 0.0) continue;
                    double2 inner = make_double2(0.0, 0.0);
                    for (int j = 0; j < chl; ++j)
                        inner = zadd(inner, zmul(S.carry[(x * wl + a) * chl + j], S.site[s64_off(q, j, u * 2 + s, k, mirror)]));
                    acc = zadd(acc, zmul(inner, w));
                }
            S.T[e] = acc;
        }
        __syncthreads();
        if (p == n - 1) {   // ncol = 1: T is the last site
            for (int e = tid; e < B64_CAP * 4 * B64_CAP; e += nt) S.site[(size_t)q * B64_CAP * 4 * B64_CAP + e] =
                make_double2(0.0, 0.0);
            __syncthreads();
            for (int e = tid; e < m; e += nt) S.site[s64_off(q, e / 4, e % 4, 0, mirror)] = S.T[e];
            if (tid == 0) {
                if (mirror) { bond[q + 1] = kx; bond[q] = 1; }
                else { bond[q] = kx; bond[q + 1] = 1; }
            }
            __syncthreads();
            break;
        }
        // Gram of the short side of T in shared memory
        const bool rows = (m <= ncol);
        const int r = rows ? m : ncol;
        for (int e = tid; e < r * r; e += nt) {
            const int i = e / r, j = e % r;
            double2 g = make_double2(0.0, 0.0);
            if (rows) {   // G = T T^dagger
                for (int c = 0; c < ncol; ++c) g = zadd(g, zmul(S.T[i * ncol + c], zconj(S.T[j * ncol + c])));
            } else {      // G = T^dagger T
                for (int c = 0; c < m; ++c) g = zadd(g, zmul(zconj(S.T[c * ncol + i]), S.T[c * ncol + j]));
            }
            A[i * B64_LD + j] = g;
        }
        __syncthreads();
        eig_herm64(A, V, r, lam, perm, cs_s, sn_s, ph_s, flag);
        // rank by the relative cutoff on the eigenvalues (squared singular values)
        if (tid == 0) {
            double total = 0.0;
            for (int i = 0; i < r; ++i) total += fmax(lam[perm[i]], 0.0);
            int k = 1;
            double tail = total - fmax(lam[perm[0]], 0.0);
            while (k < r && tail > cutoff * total) { tail -= fmax(lam[perm[k]], 0.0); ++k; }
            if (!(total > 0.0) || !isfinite(total)) {
                k = 1;
                if (!isfinite(total)) *status = QTN_ERR_NONFINITE;
            }
            if (k > B64_CAP) { k = B64_CAP; *status = QTN_ERR_CAPACITY; }
            dims[3] = k;
        }
        __syncthreads();
        const int k = dims[3];
        // U (m x k) and the new carry (k x ncol)
        if (rows) {
            for (int e = tid; e < m * k; e += nt) S.U[e] = V[(e / k) * B64_LD + perm[e % k]];
            __syncthreads();
            for (int e = tid; e < k * ncol; e += nt) {
                const int i = e / ncol, c = e % ncol;
                double2 g = make_double2(0.0, 0.0);
                for (int row = 0; row < m; ++row) g = zadd(g, zmul(zconj(S.U[row * k + i]), S.T[row * ncol + c]));
                S.carry[e] = g;
            }
        } else {
            for (int e = tid; e < m * k; e += nt) {
                const int row = e / k, i = e % k;
                const double l = lam[perm[i]];
                double2 g = make_double2(0.0, 0.0);
                for (int c = 0; c < ncol; ++c) g = zadd(g, zmul(S.T[row * ncol + c], V[c * B64_LD + perm[i]]));
                S.U[e] = (l > 0.0) ? zscale(g, 1.0 / sqrt(l)) : make_double2(row == i ? 1.0 : 0.0, 0.0);
            }
            for (int e = tid; e < k * ncol; e += nt) {
                const int i = e / ncol, c = e % ncol;
                const double l = fmax(lam[perm[i]], 0.0);
                S.carry[e] = zscale(zconj(V[c * B64_LD + perm[i]]), sqrt(l));
            }
        }
        __syncthreads();
        // the new site: rows (x, t, s) of U
        for (int e = tid; e < B64_CAP * 4 * B64_CAP; e += nt) S.site[(size_t)q * B64_CAP * 4 * B64_CAP + e] =
            make_double2(0.0, 0.0);
        __syncthreads();
        for (int e = tid; e < m * k; e += nt) {
            const int row = e / k, i = e % k;
            S.site[s64_off(q, row / 4, row % 4, i, mirror)] = S.U[e];
        }
        if (tid == 0) {
            if (mirror) { bond[q + 1] = kx; bond[q] = k; }
            else { bond[q] = kx; bond[q + 1] = k; }
            dims[0] = k; dims[1] = wr; dims[2] = chr;
        }
        __syncthreads();
    }
}

// In-place fast Walsh-Hadamard transform of 2^n reals (one CTA), scaled by 2^-n:
// c_S = 2^-n sum_s eps(s) (-1)^(popcount(s & S)) (Sec. VI.B.3, Eq. coeff_trace).
__device__ void fwht64(double* v, int n) {
    const long long N = 1ll << n;
    for (int h = 0; h < n; ++h) {
        const long long stride = 1ll << h;
        for (long long e = threadIdx.x; e < N / 2; e += blockDim.x) {
            const long long blk = e / stride, off = e % stride;
            const long long i = blk * 2 * stride + off, j = i + stride;
            const double a = v[i], b = v[j];
            v[i] = a + b;
            v[j] = a - b;
        }
        __syncthreads();
    }
    const double sc = ldexp(1.0, -n);
    for (long long e = threadIdx.x; e < N; e += blockDim.x) v[e] *= sc;
    __syncthreads();
}

// The build.  kind: BK_QFT (param unused), BK_QPHASE (param = c), BK_PAULIZ (param = t, gate_cut = gate
// amplitude threshold), BK_BESSEL (param = t, pmax).  flags bit 0: Hermitian conjugate of the result
// (QFT inverse); bit 1: natural (not bit-reversed) site order for the diagonal operators.
// out: complex64 MPO cores [n][ocap][2][2][ocap], obond[n+1]; status: QTN_OK or an error code.
__global__ void __launch_bounds__(B64_THREADS, 1)
k_build64(int kind, int n, double param, double cutoff, double gate_cut, int pmax, int flags, Scr64 S,
          float2* __restrict__ out, int ocap, int* __restrict__ obond, int* __restrict__ status) {
    extern __shared__ double2 sm64[];
    double2* A = sm64;
    double2* V = sm64 + B64_EIG * B64_LD;
    __shared__ double lam[B64_EIG], cs_s[B64_EIG / 2 + 1], sn_s[B64_EIG / 2 + 1];
    __shared__ double2 ph_s[B64_EIG / 2 + 1];
    __shared__ int perm[B64_EIG], flag, dims[4], bond[B64_MAXN + 1], st;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) st = QTN_OK;
    const size_t site_elems = (size_t)B64_CAP * 4 * B64_CAP;
    for (size_t e = tid; e < (size_t)n * site_elems; e += nt) S.site[e] = make_double2(0.0, 0.0);
    __syncthreads();
    const bool natural = (flags & 2) != 0;
    if (kind == BK_BESSEL) {
        // exp(-i t cos(2 pi x)) = sum_{|p| <= pmax} (-i)^p J_p(t) prod_q exp(i p theta_q s_q) (Jacobi-Anger,
        // Sec. VI.B.4): a diagonal MPO of bond 2 pmax + 1 in closed form.  theta_q = 2 pi / 2^(q+1) in
        // natural order (site 0 the most significant bit), 2 pi 2^q / 2^n bit-reversed.
        const int chi = 2 * pmax + 1;
        for (int e = tid; e < n * chi * 2; e += nt) {
            const int q = e / (chi * 2), pi = (e / 2) % chi, s = e % 2;
            const int p = pi - pmax;
            const double th_over_pi = natural ? ldexp(2.0, -(q + 1)) : ldexp(2.0, q - n);
            double2 w = zexpi_pi((double)(p * s) * th_over_pi);
            const int bl = (q == 0) ? 0 : pi, br = (q == n - 1) ? 0 : pi;
            if (q == 0) {   // left boundary vector v^L_p = (-i)^p J_p(t), J_{-p} = (-1)^p J_p
                const int ap = abs(p);
                double jp = jn(ap, param);
                if (p < 0 && (ap & 1)) jp = -jp;
                const int m4 = ((p % 4) + 4) % 4;   // (-i)^p
                const double2 ip = m4 == 0 ? make_double2(1, 0) : m4 == 1 ? make_double2(0, -1)
                                 : m4 == 2 ? make_double2(-1, 0) : make_double2(0, 1);
                w = zmul(w, zscale(ip, jp));
            }
            if (n == 1) {   // both boundaries on one site: sum over p
                atomicAdd(&S.site[((size_t)0 * 4 + (s * 2 + s)) * B64_CAP].x, w.x);
                atomicAdd(&S.site[((size_t)0 * 4 + (s * 2 + s)) * B64_CAP].y, w.y);
            } else {
                S.site[(size_t)q * site_elems + ((size_t)bl * 4 + (s * 2 + s)) * B64_CAP + br] = w;
            }
        }
        for (int q = tid; q <= n; q += nt) bond[q] = (q == 0 || q == n) ? 1 : chi;
        __syncthreads();
    } else {
        // identity operator, left canonical: (1, 0, 0, 1)/sqrt(2) on sites 0..n-2, the norm on the last
        for (int q = tid; q < n; q += nt) {
            const double v = (q < n - 1) ? 0.70710678118654752440 : pow(2.0, 0.5 * (n - 1));
            S.site[(size_t)q * site_elems + 0 * B64_CAP] = make_double2(v, 0.0);
            S.site[(size_t)q * site_elems + 3 * B64_CAP] = make_double2(v, 0.0);
        }
        for (int q = tid; q <= n; q += nt) bond[q] = 1;
        __syncthreads();
        int canon_left = 1;
        auto pass = [&](const Layer& Ly) {
            zip64(Ly, S, bond, n, canon_left, cutoff, &st, A, V, lam, perm, cs_s, sn_s, ph_s, &flag, dims);
            canon_left = !canon_left;
        };
        if (kind == BK_QFT) {
            for (int j = 0; j < n; ++j) {
                Layer Ly{BK_QFT, n, j, 0.0, 0.0, 0ull, 0, 0};
                pass(Ly);
            }
        } else if (kind == BK_QPHASE) {
            for (int j = 0; j < n; ++j) {
                Layer Ly{BK_QPHASE, n, j, param, 0.0, 0ull, 0, 0};
                pass(Ly);
            }
        } else if (kind == BK_PAULIZ) {
            // c_S of eps(k) = cos(2 pi k / L) by the fast Walsh-Hadamard transform; bit b of S is frequency
            // bit b of k, carried by site b (bit-reversed order) or site n-1-b (natural order)
            const long long N = 1ll << n;
            for (long long e = tid; e < N; e += nt) S.wh[e] = cospi(2.0 * (double)e / (double)N);
            __syncthreads();
            fwht64(S.wh, n);
            // the empty string is a global phase exp(-i t c_0), put on site 0 below
            for (long long Sm = 1; Sm < N; ++Sm) {
                const double cS = S.wh[Sm];
                if (!(fabs(cS) >= gate_cut)) continue;
                unsigned long long mask = 0ull;
                for (int b = 0; b < n; ++b)
                    if ((Sm >> b) & 1ll) mask |= 1ull << (natural ? n - 1 - b : b);
                const int first = __ffsll((long long)mask) - 1;
                const int last = 63 - __clzll((long long)mask);
                Layer Ly{BK_PAULIZ, n, 0, 0.0, cS * param, mask, first, last};
                pass(Ly);
            }
            const double2 g0 = zexpi_pi(-S.wh[0] * param / 3.14159265358979323846);
            __syncthreads();
            // global phase on every entry of the norm-carrying site
            const int qn = canon_left ? n - 1 : 0;
            for (int e = tid; e < (int)site_elems; e += nt)
                S.site[(size_t)qn * site_elems + e] = zmul(S.site[(size_t)qn * site_elems + e], g0);
            __syncthreads();
        }
        // Deliver the operator right-canonical (as an MPS of (out, in) pairs): the zip-up truncation of Sec. V
        // depends on the gauge of the operator it applies, and two right-canonical forms differ only by unitary
        // bond transformations, to which it is blind.  A natural-order phase operator is reversed on output,
        // which swaps the forms, so it is left-canonical here.
        const int want_left = (natural && kind == BK_QPHASE) ? 1 : 0;
        if (canon_left != want_left) {
            Layer Ly{BK_IDENT, n, 0, 0.0, 0.0, 0ull, 0, 0};
            pass(Ly);
        }
    }
    // round to complex64 in the MPO core layout ((a, t, s, b)); optional conjugate transpose; optional reversal
    int wmax = 1;
    for (int q = 0; q <= n; ++q) wmax = max(wmax, bond[q]);
    if (wmax > ocap) {
        if (tid == 0) *status = QTN_ERR_CAPACITY;
        return;
    }
    const bool dag = (flags & 1) != 0;
    const bool rev = natural && (kind == BK_QPHASE);   // the phase layers are built bit-reversed
    for (size_t e = tid; e < (size_t)n * ocap * 4 * ocap; e += nt) out[e] = make_float2(0.f, 0.f);
    __syncthreads();
    for (size_t e = tid; e < (size_t)n * site_elems; e += nt) {
        const int q = (int)(e / site_elems);
        const int rem = (int)(e % site_elems);
        const int l = rem / (4 * B64_CAP), ph = (rem / B64_CAP) % 4, r = rem % B64_CAP;
        if (l >= bond[q] || r >= bond[q + 1]) continue;
        double2 v = S.site[e];
        int t = ph >> 1, s = ph & 1;
        if (dag) { const int tmp = t; t = s; s = tmp; v = zconj(v); }
        const int qo = rev ? n - 1 - q : q;
        const int lo = rev ? r : l, ro = rev ? l : r;
        out[(size_t)qo * ocap * 4 * ocap + (((size_t)lo * 2 + t) * 2 + s) * ocap + ro] =
            make_float2((float)v.x, (float)v.y);
    }
    for (int q = tid; q <= n; q += nt) obond[rev ? n - q : q] = bond[q];
    if (tid == 0) *status = st;
}

cudaError_t configure_build64_kernel() {
    return cudaFuncSetAttribute(k_build64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B64_SMEM);
}

cudaError_t launch_build64(int kind, int n, double param, double cutoff, double gate_cut, int pmax, int flags,
                           void* scratch, size_t scratch_bytes, double* wh, float2* out, int ocap, int* obond,
                           int* status, cudaStream_t s) {
    if (n < 1 || n > B64_MAXN || scratch_bytes < build64_scratch_bytes(n)) return cudaErrorInvalidValue;
    char* b = (char*)scratch;
    Scr64 S;
    S.site = (double2*)b;
    b += (size_t)n * B64_CAP * 4 * B64_CAP * sizeof(double2);
    S.T = (double2*)b;
    b += (size_t)4 * B64_CAP * 2 * B64_CAP * sizeof(double2);
    S.carry = (double2*)b;
    b += (size_t)B64_CAP * 2 * B64_CAP * sizeof(double2);
    S.U = (double2*)b;
    S.wh = wh;
    k_build64<<<1, B64_THREADS, B64_SMEM, s>>>(kind, n, param, cutoff, gate_cut, pmax, flags, S, out, ocap, obond,
                                               status);
    count_launch(PROF_OTHER, s, false);
    return cudaGetLastError();
}

}  // namespace qtn
