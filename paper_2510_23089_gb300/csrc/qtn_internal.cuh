// Internal declarations of the quantics tensor-network library (sm_103a).
//
// Data-dependent sizes (bond dimensions chosen by truncation) never travel to
// the host in the hot path: they live in a small array of device "dimension
// registers" in the workspace.  Every kernel receives Dim descriptors that are
// evaluated on the device (value = R[reg] * mul + add, or a constant), and is
// launched with a grid sized by capacities, retiring the blocks that fall
// outside the live extent.  A whole zip-up pass is therefore a fixed sequence
// of launches that can be captured in a CUDA graph.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/qtn.h"

namespace qtn {

// ------------------------------------------------------------------ complex helpers
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// acc += a * b
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// ------------------------------------------------------------------ pseudo-random Gaussian entries
// (deterministic counter-based hash; used for sketch matrices and basis completion, never for results)
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}
__device__ __forceinline__ float2 gauss2(int seed, int i, int j) {
    uint32_t h1 = mix32((uint32_t)i * 0x9E3779B1U ^ mix32((uint32_t)j + 0x85EBCA77U * (uint32_t)(seed + 1)));
    uint32_t h2 = mix32(h1 ^ 0xC2B2AE3DU);
    float u1 = ((h1 >> 8) + 1.0f) * (1.0f / 16777217.0f);
    float u2 = (h2 >> 8) * (1.0f / 16777216.0f);
    float rad = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return make_float2(rad * c, rad * s);
}

// ------------------------------------------------------------------ dimension registers
enum Reg : int {
    R_CHILN = 0,   // left bond of the site being produced (= rows of the carry)
    R_CHIL,        // left bond of the input site
    R_CHIR,        // right bond of the input site
    R_WL,          // MPO left bond at this site (1 for identity sites)
    R_WR,          // MPO right bond
    R_M,           // rows of the unfolded matrix T (chiLn * d)
    R_N,           // columns of T (wR * chiR)
    R_K,           // rank kept by the truncation
    R_P,           // subspace size of the randomised range finder
    R_LAST,        // 1 at the last site of a sweep
    R_MID,         // helper: chiLn * wL
    R_DN,          // helper: d * chiR
    R_ENC_ROWS,    // encode: rows of the current unfolding
    R_ENC_COLS,    // encode: columns of the current unfolding
    R_TMP0, R_TMP1, R_TMP2, R_TMP3,
    R_SWEEPS = 20, // statistics: largest Jacobi sweep count
    R_FLAGS = 21,  // statistics: bit 0 no convergence, bit 1 capacity clamp, bit 2 non-finite
    R_MAXBOND = 22,
    R_RAND = 23,   // 1 when the current factorisation takes the range-finder path (m > EIG_MAX)
    R_ROWS = 24,   // rows of the projected matrix U^dagger T (m, or the subspace size)
    R_DEP = 25,    // range finder: 1 when the sketch has dependent columns (rank below the subspace size)
    R_PI = 26,     // range finder: 1 when the power iteration runs (full-rank sketch)
    R_STICKY = 27, // status flags (as R_FLAGS) OR-ed over every call since the last qtn_check; never reset per call
    R_COUNT = 32
};

struct Dim {
    int c, reg, mul, add;
    __host__ __device__ __forceinline__ int eval(const int* R) const { return reg >= 0 ? R[reg] * mul + add : c; }
};
inline Dim dc(int v) { return Dim{v, -1, 0, 0}; }
inline Dim dr(int reg, int mul = 1, int add = 0) { return Dim{0, reg, mul, add}; }

// A strided complex matrix view: element (i, j) at
//   p[i*rs + j*cs]                                   (jdiv unset), or
//   p[i*rs + (j / jdiv)*cs_hi + (j % jdiv)*cs]       (jdiv set: a column index made of two digits,
//                                                     e.g. (physical index, bond index) of a padded site)
// optionally conjugated.
struct Mat {
    const float2* p;
    Dim rs, cs;
    int conj;
    Dim jdiv, cs_hi;
};
inline Mat mat(const void* p, Dim rs, Dim cs, int conj = 0) {
    return Mat{(const float2*)p, rs, cs, conj, Dim{0, -1, 0, 0}, Dim{0, -1, 0, 0}};
}
inline Mat mat2(const void* p, Dim rs, Dim jdiv, Dim cs_hi, Dim cs, int conj = 0) {
    return Mat{(const float2*)p, rs, cs, conj, jdiv, cs_hi};
}

// Output modes of the generic GEMM.
enum OutMode : int { OUT_STORE = 0, OUT_ACCUM = 1, OUT_ATOMIC64 = 2 };

struct GemmDesc {
    Mat A, B;          // C(MxN) = alpha * A(MxK) * B(KxN)
    void* C;           // float2* (STORE/ACCUM) or double2* (ATOMIC64)
    Dim crs, ccs;      // C strides
    Dim M, N, K;
    int mode = OUT_STORE;
    int kchunk = 0;        // ATOMIC64: K split into chunks of this size across blockIdx.z
    float alpha_re = 1.f, alpha_im = 0.f;
    int omega_seed = -1;   // >= 0: B is a generated pseudo-random Gaussian matrix (B.p ignored)
    int guard_reg = -1;    // >= 0: the launch does nothing unless R[guard_reg] == guard_val
    int guard_val = 0;
    double* flops = nullptr;   // profiling: add 8 M N K (this launch's share) here
};

// ------------------------------------------------------------------ ledger (device doubles in the workspace)
// Flag bits of R_FLAGS / R_STICKY.
enum Flag : int { F_NOCONV = 1, F_CAPACITY = 2, F_NONFINITE = 4, F_TIMEOUT = 8 };
__device__ __forceinline__ void raise_flag(int* R, int bit) {
    atomicOr(&R[R_FLAGS], bit);
    atomicOr(&R[R_STICKY], bit);
}

enum Ledger : int {
    L_DISCARDED = 0,  // accumulated discarded weight of the current call
    L_NORM2,          // squared norm of the result
    L_TRACE,          // scratch: total weight of the current factorisation
    L_FLAGS,          // bit flags (as double, written with atomicOr on an int view)
    L_SWEEPS,         // max sweeps used
    L_MAXBOND,
    L_PROF_GEMM = 8,  // profiling: algorithmic FLOPs of GEMM launches (8 M N K per complex GEMM)
    L_PROF_EIG = 9,   // profiling: algorithmic FLOPs of the shared-memory eigensolver
    L_PROF_TC = 10,   // profiling: algorithmic FLOPs of the tensor-core site contraction (8 M N K)
    L_COUNT = 16
};

// ------------------------------------------------------------------ launch accounting and profiling
enum ProfClass : int { PROF_GEMM = 0, PROF_EIG = 1, PROF_OTHER = 2, PROF_TC = 3, PROF_NCLASS = 4 };
void count_launch(int cls, cudaStream_t s, bool before);   // brackets a launch with events when profiling
extern double* g_prof_ledger;                              // ledger receiving device FLOP counts (or null)

// ------------------------------------------------------------------ workspace layout
struct WsLayout {
    size_t ledger, regs, T, P, carry, G64, G32, U, lam, Y, Q, S64, Z, X0, X1, omega, b64, tc, tc_bytes, total;
    int m_cap, n_cap, p_cap, chi, d, w, n_sites;
    long long dense;
};
WsLayout ws_layout(int n_sites, int d, int chi_max, int w_max, long long dense_elems);

// ------------------------------------------------------------------ context
struct Ctx {
    cudaStream_t stream;
    int sm_count;
    int device;
    int gemm_tile;   // 64 or 32: GEMM tile of this context's launches (batch tuner)
    cudaStream_t helper[2];   // capture the bodies of conditional graph nodes (null: guards only)
};

// Pointers into the caller's workspace.
struct Ws {
    double* ledger;
    int* R;
    float2 *T, *P, *carry, *G32, *U, *Y, *Q, *Z, *X0, *X1;
    double2 *G64, *S64;
    double* lam;
    void* tc;   // packed split-BF16 operands of the tensor-core site contraction
    WsLayout L;
};

// Devices a process may drive (per-device one-time set-up tables).
constexpr int QTN_MAX_DEVICES = 64;

// Largest eigen/SVD problem solved inside one CTA's shared memory.
constexpr int EIG_MAX = 160;
// Subspace size of the range finder (m > EIG_MAX rows) is EIG_MAX whatever chi_max is: a subspace of
// chi_max + 32 or + 64 left chi-limited truncations of slowly decaying spectra 1e-5 to 1e-3 above the
// Eckart-Young optimum after one power iteration, EIG_MAX keeps them within 1e-6.

// One-time per-device set-up of the kernels that need more than the default 48 KB of dynamic shared
// memory (cudaFuncSetAttribute acts on the current device only); thread-safe, once per device.
cudaError_t configure_device_kernels(int device);

// FP64 operator builders (k_build64.cu): kinds, scratch size, launch.
enum Build64Op : int { BUILD64_QFT = 0, BUILD64_QPHASE = 1, BUILD64_PAULIZ = 2, BUILD64_BESSEL = 3 };
constexpr int BUILD64_BOND_CAP = 32;   // largest bond of an operator built in FP64
size_t build64_scratch_bytes(int n);
cudaError_t launch_build64(int kind, int n, double param, double cutoff, double gate_cut, int pmax, int flags,
                           void* scratch, size_t scratch_bytes, double* wh, float2* out, int ocap, int* obond,
                           int* status, cudaStream_t s);

// ------------------------------------------------------------------ launches (defined in the .cu files)
cudaError_t launch_gemm(const GemmDesc& d, int max_m, int max_n, int max_k, const int* R, cudaStream_t s);
// Tile (64 or 32) of the generic GEMM launches made by the calling host thread.
void set_gemm_tile(int tile);
void set_gemm_sms(int sms);   // SM count of the calling context's device (automatic tile choice)
int gemm_tile();
// Split-BF16 tensor-core complex GEMM (STORE/ACCUM only), FP32 accumulation in TMEM (k_tc.cu): operands packed
// into `pack` (tc_pack_bytes of the capacities), then streamed by bulk copies into the tensor cores.
size_t tc_pack_bytes(int max_m, int max_n, int max_k);
cudaError_t launch_gemm_tc(const GemmDesc& d, int max_m, int max_n, int max_k, const int* R, void* pack,
                           size_t pack_bytes, int sm_count, cudaStream_t s);
cudaError_t launch_refine_basis(const double2* G, Dim ld, Dim r, float2* V, int ldv, const int* R, cudaStream_t s);
// One-sided Jacobi over a cluster of 8 CTAs with accumulated rotations (k_eig_cluster.cu); runs when
// r_min <= r (live) <= EIG_MAX and R[guard_reg] == guard_val.
cudaError_t launch_eig_cluster(const double2* G, Dim ld, Dim r, float2* U, Dim ldu, double* lam, const int* R,
                               int max_sweeps, cudaStream_t s, int guard_reg, int guard_val, double* prof, float tol,
                               bool report_nonconv, int r_min, bool accumulate);
// Eigenvectors from the rotated columns of W that k_eig_cluster<false> left in U (normalised, orthonormalised in
// descending-eigenvalue order, completed), one CTA; runs when r_min <= r <= EIG_MAX and R[guard_reg] == guard_val.
cudaError_t launch_eig_finish(const double2* G, Dim ld, Dim r, float2* U, Dim ldu, double* lam, const int* R,
                              cudaStream_t s, int guard_reg, int guard_val, float dead_rel, int r_min);
cudaError_t configure_eig_cluster_kernel();
int eig_cluster_min();
void set_eig_cluster_min(int r);
cudaError_t launch_eig(const double2* G, Dim ld, Dim r, float2* U, Dim ldu, double* lam, const int* R,
                       int r_cap, int max_sweeps, double* ledger, cudaStream_t s, int guard_reg = -1, int guard_val = 0,
                       float tol = 1e-6f, float dead_rel = 0.f, bool report_nonconv = true, bool rough_basis = false);

}  // namespace qtn

// ------------------------------------------------------------------ host-side helpers shared by the entry points
#define CK(expr)                                                                                          \
    do {                                                                                                  \
        cudaError_t _e = (expr);                                                                          \
        if (_e != cudaSuccess) {                                                                          \
            fprintf(stderr, "qtn: CUDA error %s at %s:%d\n", cudaGetErrorString(_e), __FILE__, __LINE__); \
            return QTN_ERR_CUDA;                                                                          \
        }                                                                                                 \
    } while (0)
#define CKL()                                         \
    do {                                              \
        qtn::count_launch(qtn::PROF_OTHER, 0, false); \
        CK(cudaGetLastError());                       \
    } while (0)

namespace qtn {
bool trunc_ok(const qtn_trunc& t);
int grid_for(long long n, int threads, int sm);
qtn_status fill_stats(Ctx* c, Ws& w, qtn_stats* st);
qtn_status zip_pass(Ctx* c, Ws& w, qtn_mps* psi, const qtn_mpo* W, int axis, int moff, int mn, int mirror,
                    const qtn_trunc& tr);
__global__ void k_reset_stats(int* R, double* ledger);
}  // namespace qtn

// Library context bound to a stream, with the layout of the workspace the caller sized.
struct qtn_context {
    qtn::Ctx c;
    qtn::WsLayout L;
    int have_layout;
};
qtn_status bind_ws(qtn_context* x, void* ws, size_t bytes, qtn::Ws& w);
// One zip-up application of W on `axis` (diag: W is an MPS seen as a diagonal operator, axis 2/3), bringing
// psi to a canonical form first when it has none.
qtn_status apply_inner(qtn_context* x, qtn::Ws& w, const qtn_mpo* W, int axis, qtn_mps* psi, const qtn_trunc& tr,
                       bool diag);
