// Fixed-rank adjoint of a zip-up pass.
//
// A zip-up pass (Sec. V, Fig. fig_mpo) that applies the operator K to psi writes N - 1 isometric sites and
// one site that carries the rest (the centre): its output is V c with V the isometry of the isometric sites
// ("frame") and c = V^dagger K psi, because every carry the pass forms is the partial contraction of K psi
// with the adjoints of the sites already written.  With the frame held fixed (the truncation ranks and
// subspaces of the forward pass frozen), the pass is the linear map psi -> V V^dagger K psi, and its adjoint
// is g -> K^dagger V V^dagger g.  Chaining the passes of a forward computation backwards therefore needs one
// operation: given a state h (any MPS), an operator W (or the identity) and a frame V recorded by the
// forward pass, form V V^dagger W h as an MPS, i.e. keep the frame's isometric sites and replace its centre
// by V^dagger W h.  The centre is a chain of three-layer transfer contractions
//     E'[k, b, l] = sum_{i, a, j, s', s} conj(A[i, s', k]) E[i, a, j] W[a, s', s, b] B[j, s, l]
// from the frame's far end to its centre (A: frame sites, B: sites of h, W: the embedded operator), finished
// at the centre site without the conjugated frame site.  Each step is three contractions (E B, then W, then
// conj(A)), FP32 values with FP64 accumulation.  Nothing is truncated and nothing is factorised.
#include <math.h>

#include <algorithm>
#include <vector>

#include "qtn_internal.cuh"

namespace qtn {

// Site element (l, s, r) of a padded site in sweep orientation (mirror: l and r exchanged).
__device__ __forceinline__ float2 site_at(const float2* site, int cap, int d, int l, int s, int r, int mirror) {
    return mirror ? site[((long long)r * d + s) * cap + l] : site[((long long)l * d + s) * cap + r];
}

// Embedded operator element Wf[a, s', s, b] of a per-axis MPO core on a d = 4 site (axis 0: the x bit, the
// high bit of mu = 2x + y; axis 1: the y bit), a d = 2 site (the core itself), or the identity (Wc null).
__device__ __forceinline__ float2 op_at(const float2* Wc, int wcap, int d, int axis, int a, int sp, int s, int b,
                                        int mirror) {
    if (Wc == nullptr) return make_float2(sp == s ? 1.f : 0.f, 0.f);
    int t, u, pass_ok;
    if (d == 2) { t = sp; u = s; pass_ok = 1; }
    else if (axis == 0) { t = sp >> 1; u = s >> 1; pass_ok = ((sp & 1) == (s & 1)); }
    else { t = sp & 1; u = s & 1; pass_ok = ((sp >> 1) == (s >> 1)); }
    if (!pass_ok) return make_float2(0.f, 0.f);
    const int aa = mirror ? b : a, bb = mirror ? a : b;
    return Wc[(((long long)aa * 2 + t) * 2 + u) * wcap + bb];
}

// X[(i, a), (s, l)] = sum_j E[(i, a), j] B[j, s, l]
__global__ void k_env3_x(const float2* __restrict__ E, const float2* __restrict__ B, int bcap, int d, int mirror,
                         int ca, int wa, int bl, int br, float2* __restrict__ X) {
    const long long total = (long long)ca * wa * d * br;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int ia = (int)(e / (d * br)), s = (int)((e / br) % d), l = (int)(e % br);
        double re = 0.0, im = 0.0;
        for (int j = 0; j < bl; ++j) {
            const float2 x = E[(long long)ia * bl + j], y = site_at(B, bcap, d, j, s, l, mirror);
            re += (double)x.x * y.x - (double)x.y * y.y;
            im += (double)x.x * y.y + (double)x.y * y.x;
        }
        X[e] = make_float2((float)re, (float)im);
    }
}

// Y[(i, b), (s', l)] = sum_{a, s} X[(i, a), (s, l)] Wf[a, s', s, b]
__global__ void k_env3_y(const float2* __restrict__ X, const float2* __restrict__ Wc, int wcap, int d, int axis,
                         int mirror, int ca, int wa, int wb, int br, float2* __restrict__ Y) {
    const long long total = (long long)ca * wb * d * br;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ((long long)wb * d * br)), b = (int)((e / ((long long)d * br)) % wb);
        const int sp = (int)((e / br) % d), l = (int)(e % br);
        double re = 0.0, im = 0.0;
        for (int a = 0; a < wa; ++a)
            for (int s = 0; s < d; ++s) {
                const float2 w = op_at(Wc, wcap, d, axis, a, sp, s, b, mirror);
                if (w.x == 0.f && w.y == 0.f) continue;
                const float2 x = X[(((long long)i * wa + a) * d + s) * br + l];
                re += (double)x.x * w.x - (double)x.y * w.y;
                im += (double)x.x * w.y + (double)x.y * w.x;
            }
        Y[e] = make_float2((float)re, (float)im);
    }
}

// E'[(k, b), l] = sum_{i, s'} conj(A[i, s', k]) Y[(i, b), (s', l)]
__global__ void k_env3_e(const float2* __restrict__ A, int acap, int d, int mirror, int ca, int ck, int wb, int br,
                         const float2* __restrict__ Y, float2* __restrict__ En) {
    const long long total = (long long)ck * wb * br;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / ((long long)wb * br)), b = (int)((e / br) % wb), l = (int)(e % br);
        double re = 0.0, im = 0.0;
        for (int i = 0; i < ca; ++i)
            for (int sp = 0; sp < d; ++sp) {
                const float2 a = site_at(A, acap, d, i, sp, k, mirror);
                const float2 y = Y[(((long long)i * wb + b) * d + sp) * br + l];
                re += (double)a.x * y.x + (double)a.y * y.y;   // conj(a) * y
                im += (double)a.x * y.y - (double)a.y * y.x;
            }
        En[e] = make_float2((float)re, (float)im);
    }
}

// The frame's centre site <- Y[(i, 0), (s', 0)] (the last sweep site has trailing bonds 1), written in the
// frame's stored orientation; the rest of the padded site is cleared.
__global__ void k_env3_centre(const float2* __restrict__ Y, int ca, int d, float2* __restrict__ site, int cap,
                              int mirror) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cap * d * cap; e += gridDim.x * blockDim.x)
        site[e] = make_float2(0.f, 0.f);
    __syncthreads();
    if (blockIdx.x != 0) return;
    for (int e = threadIdx.x; e < ca * d; e += blockDim.x) {
        const int i = e / d, sp = e % d;
        const float2 v = Y[(long long)i * d + sp];
        if (mirror) site[(long long)sp * cap + i] = v;
        else site[((long long)i * d + sp) * cap] = v;
    }
}

}  // namespace qtn

using namespace qtn;

extern "C" qtn_status qtn_project_apply(void* ctx, const qtn_mpo* W, int axis, const qtn_mps* ket, qtn_mps* frame,
                                        void* ws, size_t ws_bytes) {
    if (!ctx || !ket || !frame || ket->n_sites != frame->n_sites || ket->d != frame->d) return QTN_ERR_ARG;
    if (frame->canon != QTN_CANON_LEFT && frame->canon != QTN_CANON_RIGHT) return QTN_ERR_ARG;
    if (ket->sites == frame->sites) return QTN_ERR_ARG;
    const int N = frame->n_sites, d = frame->d;
    if (W) {
        if (W->n_sites != N || (d == 4 && axis != 0 && axis != 1)) return QTN_ERR_SHAPE;
        if (d != 4 && d != 2) return QTN_ERR_SHAPE;
    }
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    cudaStream_t s = x->c.stream;
    std::vector<int> fb(N + 1), kb(N + 1), wbh(N + 1, 1);
    CK(cudaMemcpyAsync(fb.data(), frame->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(kb.data(), ket->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (W) CK(cudaMemcpyAsync(wbh.data(), W->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // the centre is the last site of the sweep: a LEFT frame (norm in site N-1) is swept left to right, a
    // RIGHT frame right to left (mirrored)
    const int mirror = (frame->canon == QTN_CANON_RIGHT) ? 1 : 0;
    auto lb = [&](const std::vector<int>& b, int q) { return mirror ? b[q + 1] : b[q]; };
    auto rb = [&](const std::vector<int>& b, int q) { return mirror ? b[q] : b[q + 1]; };
    // buffers: E and E' (carry, Z), X (T), Y (P); capacities checked per site
    float2* E = w.carry;
    float2* En = w.Z;
    const size_t cap_e = (size_t)w.L.chi * std::max(w.L.w, 1) * w.L.chi;
    const size_t cap_xy = (size_t)w.L.m_cap * w.L.n_cap;
    const size_t cap_p = (size_t)w.L.chi * std::max(w.L.w, 1) * w.L.d * w.L.chi;
    const float2 one = make_float2(1.f, 0.f);
    CK(cudaMemcpyAsync(E, &one, sizeof(float2), cudaMemcpyHostToDevice, s));
    int ca = 1, wa = 1, cbl = 1;   // current environment dims: frame bond x operator bond x ket bond
    for (int p = 0; p < N; ++p) {
        const int q = mirror ? N - 1 - p : p;
        const int ar = rb(fb, q), br = rb(kb, q);
        if (lb(fb, q) != ca || lb(kb, q) != cbl) return QTN_ERR_SHAPE;
        int wb = 1;
        const float2* Wc = nullptr;
        if (W) {
            Wc = (const float2*)W->sites + (size_t)q * W->w_cap * 4 * W->w_cap;
            wb = rb(wbh, q);
            if (lb(wbh, q) != wa) return QTN_ERR_SHAPE;
        }
        const size_t nx = (size_t)ca * wa * d * br, ny = (size_t)ca * wb * d * br, ne = (size_t)ar * wb * br;
        if (nx > cap_xy || ny > cap_p || ne > cap_e || (size_t)ca * wa * cbl > cap_e) return QTN_ERR_WORKSPACE;
        const float2* Aq = (const float2*)frame->sites + (size_t)q * frame->chi_cap * d * frame->chi_cap;
        const float2* Bq = (const float2*)ket->sites + (size_t)q * ket->chi_cap * d * ket->chi_cap;
        k_env3_x<<<grid_for((long long)nx, 256, x->c.sm_count), 256, 0, s>>>(E, Bq, ket->chi_cap, d, mirror, ca, wa,
                                                                          cbl, br, w.T);
        CKL();
        k_env3_y<<<grid_for((long long)ny, 256, x->c.sm_count), 256, 0, s>>>(w.T, Wc, W ? W->w_cap : 1, d, axis,
                                                                          mirror, ca, wa, wb, br, w.P);
        CKL();
        if (p == N - 1) {
            if (wb != 1 || br != 1 || ar != 1) return QTN_ERR_SHAPE;
            k_env3_centre<<<1, 256, 0, s>>>(w.P, ca, d, (float2*)Aq, frame->chi_cap, mirror);
            CKL();
            break;
        }
        k_env3_e<<<grid_for((long long)ne, 256, x->c.sm_count), 256, 0, s>>>(Aq, frame->chi_cap, d, mirror, ca, ar, wb,
                                                                          br, w.P, En);
        CKL();
        std::swap(E, En);
        ca = ar;
        wa = wb;
        cbl = br;
    }
    return QTN_OK;
}
