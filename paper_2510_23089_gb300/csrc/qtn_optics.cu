// Imaging and free-space propagation on quantics MPS, built from the zip-up passes of the Fresnel path:
//
//  * the point spread function of Sec. V (Eq. psf_eq): |phi> = U_qft |E_0>, normalised, and
//    ||PSF>> = |phi> (.) |phi>^* (local product of physical legs), so that ||PSF||_L1 = <phi|phi> = 1;
//  * image formation by convolution (Eq. convolution_eq): U_iqft(U_qft ||PSF>> (.) U_qft |S>);
//  * the non-paraxial angular-spectrum step of Sec. VI.A (Eq. eq_astf): a transfer function that does not
//    factor over the axes, so it is applied in Fourier space as an interleaved d = 4 MPS acting diagonally
//    (the "fused" 2-D operator of Fig. fig_mpo_fresnel);
//  * site reversal.  The swap-free QFT leaves the frequency bits of each axis in reversed order; reversing
//    the order of the sites of an interleaved MPS reverses the bits of both axes at once and costs a
//    transposition of every site tensor, no factorisation.  Flipping the two bits of the most significant
//    site is the centring shift of the frequency plane (k -> k + L/2 on both axes).
#include <math.h>

#include <algorithm>
#include <vector>

#include "qtn_internal.cuh"

namespace qtn {

__global__ void k_site_norm2(const float2*, int, int, const int*, int, double*, int);

// Site p <-> site N-1-p with left and right bonds exchanged (whole padded blocks, so no bond is needed).
__global__ void k_reverse_sites(float2* __restrict__ sites, int N, int d, int cap) {
    const long long per = (long long)cap * d * cap;
    const int pairs = (N + 1) / 2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < pairs * per;
         e += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(e / per), q = N - 1 - p;
        const long long rem = e % per;
        const int l = (int)(rem / (d * cap)), s = (int)((rem / cap) % d), r = (int)(rem % cap);
        if (p == q && l >= r) continue;   // middle site: transpose, each off-diagonal pair once
        float2* a = sites + p * per + ((long long)l * d + s) * cap + r;
        float2* b = sites + q * per + ((long long)r * d + s) * cap + l;
        const float2 t = *a;
        *a = *b;
        *b = t;
    }
}

__global__ void k_reverse_bonds(int* __restrict__ bond, int N) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i < (N + 1) / 2; ++i) {
        const int t = bond[i];
        bond[i] = bond[N - i];
        bond[N - i] = t;
    }
}

// Physical index s -> d-1-s on one site (the most significant bit of every axis flipped).
__global__ void k_flip_digits(float2* __restrict__ site, int d, int cap) {
    const int half = d / 2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cap * half * cap; e += gridDim.x * blockDim.x) {
        const int l = e / (half * cap), s = (e / cap) % half, r = e % cap;
        float2* a = site + ((long long)l * d + s) * cap + r;
        float2* b = site + ((long long)l * d + (d - 1 - s)) * cap + r;
        const float2 t = *a;
        *a = *b;
        *b = t;
    }
}

// psi <- psi / sqrt(ledger[slot]) on the site that carries the norm (device-side: no host round trip).
__global__ void k_scale_by_norm(float2* __restrict__ site, int cap, int d, const double* __restrict__ ledger, int slot,
                                int* __restrict__ R) {
    const double n2 = ledger[slot];
    const float s = (n2 > 0.0 && isfinite(n2)) ? (float)(1.0 / sqrt(n2)) : 0.f;
    if (!(n2 > 0.0) || !isfinite(n2)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) raise_flag(R, F_NONFINITE);
        return;
    }
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)cap * d * cap;
         e += (long long)gridDim.x * blockDim.x)
        site[e] = make_float2(site[e].x * s, site[e].y * s);
}

// Padded copy of a state into one of another capacity (bonds copied too).
__global__ void k_copy_state(const float2* __restrict__ a, int acap, const int* __restrict__ ab, float2* __restrict__ o,
                             int ocap, int* __restrict__ ob, int N, int d) {
    const long long per = (long long)ocap * d * ocap;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * per;
         e += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(e / per);
        const long long rem = e % per;
        const int l = (int)(rem / (d * ocap)), s = (int)((rem / ocap) % d), r = (int)(rem % ocap);
        float2 v = make_float2(0.f, 0.f);
        if (l < acap && r < acap && l < ab[p] && r < ab[p + 1]) v = a[(long long)p * acap * d * acap + ((long long)l * d + s) * acap + r];
        o[e] = v;
    }
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i <= N; i += blockDim.x) ob[i] = ab[i];
}

// Angular-spectrum transfer function on the L x L frequency grid (row = k_x, column = k_y, bit reversed when
// asked): exp(2 pi i (z/lambda) (sqrt(1 - u) - 1)), u = (lambda f_x)^2 + (lambda f_y)^2, lambda f = (lambda/dx) k_f / L;
// evanescent (u > 1): exp(-2 pi (z/lambda) sqrt(u - 1)) exp(-2 pi i z/lambda).  The constant exp(2 pi i z / lambda)
// is divided out (as exp(i k z) is in the Fresnel step).
__global__ void k_astf_field(float2* __restrict__ out, int n, double z_over_lambda, double lambda_over_dx,
                             int bit_reversed) {
    const long long L = 1ll << n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L * L;
         e += (long long)gridDim.x * blockDim.x) {
        long long a = e / L, b = e % L;
        if (bit_reversed) {
            a = (long long)(__brevll((unsigned long long)a) >> (64 - n));
            b = (long long)(__brevll((unsigned long long)b) >> (64 - n));
        }
        const double fx = lambda_over_dx * (double)((a < L / 2) ? a : a - L) / (double)L;
        const double fy = lambda_over_dx * (double)((b < L / 2) ? b : b - L) / (double)L;
        const double u = fx * fx + fy * fy;
        double re, im;
        if (u <= 1.0) {
            // sqrt(1 - u) - 1 = -u / (1 + sqrt(1 - u)), without cancellation for small u
            const double ph = z_over_lambda * (-u / (1.0 + sqrt(1.0 - u)));   // phase / (2 pi)
            double s, c;
            sincospi(2.0 * fmod(ph, 1.0), &s, &c);
            re = c;
            im = s;
        } else {
            const double mag = exp(-2.0 * 3.14159265358979323846 * z_over_lambda * sqrt(u - 1.0));
            double s, c;
            sincospi(-2.0 * fmod(z_over_lambda, 1.0), &s, &c);
            re = mag * c;
            im = mag * s;
        }
        out[e] = make_float2((float)re, (float)im);
    }
}

}  // namespace qtn

using namespace qtn;

// Largest bond of a state (host copy; synchronises).
static qtn_status host_max_bond(cudaStream_t s, const qtn_mps* psi, int* out) {
    std::vector<int> hb(psi->n_sites + 1);
    CK(cudaMemcpyAsync(hb.data(), psi->bond, hb.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = std::max(1, *std::max_element(hb.begin(), hb.end()));
    return QTN_OK;
}

static qtn_status reverse_inplace(qtn_context* x, qtn_mps* psi) {
    cudaStream_t s = x->c.stream;
    const long long per = (long long)psi->chi_cap * psi->d * psi->chi_cap;
    k_reverse_sites<<<grid_for((psi->n_sites + 1) / 2 * per, 256, x->c.sm_count), 256, 0, s>>>(
        (float2*)psi->sites, psi->n_sites, psi->d, psi->chi_cap);
    CKL();
    k_reverse_bonds<<<1, 1, 0, s>>>(psi->bond, psi->n_sites);
    CKL();
    if (psi->canon == QTN_CANON_LEFT) psi->canon = QTN_CANON_RIGHT;
    else if (psi->canon == QTN_CANON_RIGHT) psi->canon = QTN_CANON_LEFT;
    return QTN_OK;
}

// Normalise a canonical state on the device: the norm sits in one site.
static qtn_status normalise(qtn_context* x, Ws& w, qtn_mps* psi) {
    cudaStream_t s = x->c.stream;
    const int N = psi->n_sites, d = psi->d, cap = psi->chi_cap;
    const int q = (psi->canon == QTN_CANON_LEFT) ? N - 1 : 0;
    float2* site = (float2*)psi->sites + (size_t)q * cap * d * cap;
    k_site_norm2<<<1, 512, 0, s>>>(site, cap, d, psi->bond, q, w.ledger, L_TRACE);
    CKL();
    k_scale_by_norm<<<grid_for((long long)cap * d * cap, 256, x->c.sm_count), 256, 0, s>>>(site, cap, d, w.ledger,
                                                                                         L_TRACE, w.R);
    CKL();
    return QTN_OK;
}

static qtn_status qft_both_axes(qtn_context* x, Ws& w, const qtn_mpo* W, qtn_mps* psi, const qtn_trunc& tr) {
    qtn_status st = apply_inner(x, w, W, 0, psi, tr, false);
    if (st) return st;
    return apply_inner(x, w, W, 1, psi, tr, false);
}

// b <- b (.) a (conj(a) when conj_a): a seen as an operator diagonal in the site index, by zip-up.
static qtn_status hadamard_into(qtn_context* x, Ws& w, const qtn_mps* a, int conj_a, qtn_mps* b, const qtn_trunc& tr) {
    int wmax = 1;
    qtn_status st = host_max_bond(x->c.stream, a, &wmax);
    if (st) return st;
    if (wmax > std::max(w.L.w, 1) || wmax * b->chi_cap > w.L.n_cap) return QTN_ERR_WORKSPACE;
    qtn_mpo view{a->n_sites, a->chi_cap, wmax, a->bond, a->sites};
    return apply_inner(x, w, &view, conj_a ? 3 : 2, b, tr, true);
}

extern "C" {

qtn_status qtn_reverse_sites(void* ctx, qtn_mps* psi) {
    if (!ctx || !psi || psi->n_sites < 1) return QTN_ERR_ARG;
    return reverse_inplace((qtn_context*)ctx, psi);
}

qtn_status qtn_psf(void* ctx, qtn_mps* phi, const qtn_mpo* qft, int centre, qtn_trunc trunc, qtn_mps* psf,
                   qtn_stats* stats, void* ws, size_t ws_bytes) {
    if (!ctx || !phi || !qft || !psf || !trunc_ok(trunc)) return QTN_ERR_ARG;
    if (phi->d != 4 || psf->d != 4 || psf->n_sites != phi->n_sites || qft->n_sites != phi->n_sites)
        return QTN_ERR_SHAPE;
    if (psf->sites == phi->sites) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    cudaStream_t s = x->c.stream;
    k_reset_stats<<<1, 1, 0, s>>>(w.R, w.ledger);
    CKL();
    // focal field |phi> = U_qft^(x) U_qft^(y) |E_0>, normalised (Eq. psf_eq)
    if ((st = qft_both_axes(x, w, qft, phi, trunc))) return st;
    if ((st = normalise(x, w, phi))) return st;
    // natural frequency order (the swap-free QFT reversed the bits of both axes), optionally centred
    if ((st = reverse_inplace(x, phi))) return st;
    if (centre) {
        k_flip_digits<<<grid_for((long long)phi->chi_cap * 2 * phi->chi_cap, 256, x->c.sm_count), 256, 0, s>>>(
            (float2*)phi->sites, 4, phi->chi_cap);
        CKL();
    }
    // ||PSF>> = |phi> (.) |phi>^*, truncated by `trunc`; the product starts from a copy of |phi>
    int bmax = 1;
    if ((st = host_max_bond(s, phi, &bmax))) return st;
    if (bmax > psf->chi_cap) return QTN_ERR_CAPACITY;
    k_copy_state<<<grid_for((long long)phi->n_sites * psf->chi_cap * 4 * psf->chi_cap, 256, x->c.sm_count), 256, 0,
                   s>>>((const float2*)phi->sites, phi->chi_cap, phi->bond, (float2*)psf->sites, psf->chi_cap,
                        psf->bond, phi->n_sites, 4);
    CKL();
    psf->canon = phi->canon;
    if ((st = hadamard_into(x, w, phi, 1, psf, trunc))) return st;
    return fill_stats(&x->c, w, stats);
}

qtn_status qtn_convolve(void* ctx, qtn_mps* a, qtn_mps* b, const qtn_mpo* qft, const qtn_mpo* qft_dagger,
                        qtn_trunc trunc, qtn_stats* stats, void* ws, size_t ws_bytes) {
    if (!ctx || !a || !b || !qft || !qft_dagger || !trunc_ok(trunc)) return QTN_ERR_ARG;
    if (a->d != 4 || b->d != 4 || a->n_sites != b->n_sites || qft->n_sites != a->n_sites) return QTN_ERR_SHAPE;
    if (a->sites == b->sites) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    cudaStream_t s = x->c.stream;
    k_reset_stats<<<1, 1, 0, s>>>(w.R, w.ledger);
    CKL();
    // U_iqft(U_qft a (.) U_qft b), both transforms in the same (bit-reversed) frequency order
    if ((st = qft_both_axes(x, w, qft, a, trunc))) return st;
    if ((st = qft_both_axes(x, w, qft, b, trunc))) return st;
    if ((st = hadamard_into(x, w, a, 0, b, trunc))) return st;
    if ((st = qft_both_axes(x, w, qft_dagger, b, trunc))) return st;
    // the unitary DFT turns a circular convolution into sqrt(L) times a product per axis: scale by L = 2^n
    const double Lsc = ldexp(1.0, a->n_sites);
    if ((st = qtn_scale(ctx, b, Lsc, 0.0))) return st;
    return fill_stats(&x->c, w, stats);
}

qtn_status qtn_astf_field(void* ctx, int n, double z_over_lambda, double lambda_over_dx, int bit_reversed,
                          void* dense, long long cap_elems) {
    if (!ctx || !dense || n < 1 || n > 15 || !isfinite(z_over_lambda) || !(lambda_over_dx > 0.0)) return QTN_ERR_ARG;
    if ((1ll << (2 * n)) > cap_elems) return QTN_ERR_CAPACITY;
    qtn_context* x = (qtn_context*)ctx;
    k_astf_field<<<grid_for(1ll << (2 * n), 256, x->c.sm_count), 256, 0, x->c.stream>>>(
        (float2*)dense, n, z_over_lambda, lambda_over_dx, bit_reversed ? 1 : 0);
    CKL();
    return QTN_OK;
}

qtn_status qtn_transfer_step(void* ctx, qtn_mps* psi, const qtn_mpo* qft, const qtn_mpo* qft_dagger,
                             const qtn_mps* transfer, qtn_trunc trunc, qtn_stats* stats, void* ws, size_t ws_bytes) {
    if (!ctx || !psi || !qft || !qft_dagger || !transfer || !trunc_ok(trunc)) return QTN_ERR_ARG;
    if (psi->d != 4 || transfer->d != 4 || transfer->n_sites != psi->n_sites || qft->n_sites != psi->n_sites)
        return QTN_ERR_SHAPE;
    if (transfer->sites == psi->sites) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    k_reset_stats<<<1, 1, 0, x->c.stream>>>(w.R, w.ledger);
    CKL();
    if ((st = qft_both_axes(x, w, qft, psi, trunc))) return st;
    if ((st = hadamard_into(x, w, transfer, 0, psi, trunc))) return st;
    if ((st = qft_both_axes(x, w, qft_dagger, psi, trunc))) return st;
    return fill_stats(&x->c, w, stats);
}

}  // extern "C"
