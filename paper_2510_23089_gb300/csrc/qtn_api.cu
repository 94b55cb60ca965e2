// C ABI of the quantics tensor-network Fresnel library: host-side orchestration.
//
// Every entry point only enqueues kernels on the context's stream.  Sizes that
// depend on truncation are carried in device dimension registers (see
// qtn_internal.cuh), so the host never waits for a bond dimension.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <functional>
#include <mutex>
#include <vector>

#include "qtn_internal.cuh"

namespace qtn {

// kernels from k_mps.cu
__global__ void k_plan_site(const int*, const int*, int, int, int, int, int, int, int*);
__global__ void k_plan_encode(int, int, int*);
__global__ void k_reset_stats(int*, double*);
__global__ void k_stage2(const float2*, float2*, const float2*, int, int, int, int, const int*);
__global__ void k_trace(const double2*, int, Dim, int*, double*);
__global__ void k_path(Dim, int*, double*);
__global__ void k_total_weight(const float2*, Dim, Dim, Dim, const int*, double*);
__global__ void k_cgs_block_32(float2*, int, Dim, int, int, const float*, int*, int, int);
__global__ void k_ns_coeff(const double2*, int, float2*, int, Dim, const int*);
__global__ void k_cgs_block_16(float2*, int, Dim, int, int, const float*, int*, int, int);
__global__ void k_cgs_block_8(float2*, int, Dim, int, int, const float*, int*, int, int);
__global__ void k_col_norms(const float2*, int, Dim, Dim, float*, const int*, int);
__global__ void k_set_pi(int*);
__global__ void k_copy_guarded(const float2*, float2*, long long, const int*, int, int);
__global__ void k_sketch_live(const float2*, int, Dim, int, int*, int*);
__global__ void k_sketch_gather(const float2*, float2*, int, Dim, int, const int*, const int*);
__global__ void k_kron_interleave(const float2*, const int*, int, const float2*, const int*, int, float2*, int*, int,
                                  int);
__global__ void k_direct_sum(const float2*, const int*, int, const float2*, const int*, int, float2*, int*, int, int,
                             int);
__global__ void k_hadamard(const float2*, const int*, int, const float2*, const int*, int, int, float2*, int*, int, int,
                           int);
__global__ void k_scale_site(float2*, int, int, const int*, int, float, float);
constexpr int CGS_MAXM_ALL = 1024;
constexpr int RF_POWER_ITERS = 3;   // power iterations of the range finder (full-rank sketches only)
constexpr size_t CGS_SMEM = (size_t)32 * 512 * sizeof(float2);   // = 16 x 1024 = 8 x 2048 as well
__global__ void k_row_weights(const float2*, Dim, Dim, Dim, double*, const int*);
__global__ void k_select(const double*, Dim, int, double, int, int, int*, int*, double*);
__global__ void k_write_site(const float2*, int, const int*, float2*, int, int, int, int*, int, const int*);
__global__ void k_gather_rows(const float2*, Dim, const int*, float2*, Dim, Dim, const int*);
__global__ void k_write_last(const float2*, float2*, int, int, int, const int*);
__global__ void k_site_norm2(const float2*, int, int, const int*, int, double*, int);
__global__ void k_to_f32(const double2*, float2*, int, Dim, const int*);
__global__ void k_whiten(float2*, int, const double*, Dim, double, const int*);
__global__ void k_dense_to_quantics(const float2*, float2*, int, int, int*);
__global__ void k_quantics_to_dense(const float2*, float2*, int, int);
__global__ void k_mpo_dagger(const float2*, const int*, int, float2*, int*, int, int);
__global__ void k_amplitudes(const float2*, const int*, int, int, int, const int*, int, float2*, float2*);
__global__ void k_transfer_right(const double2*, int, const float2*, int, int, int, const float2*, int, int, int, int,
                                 double2*, int);
__global__ void k_env_grad(const double2*, int, const double2*, int, const float2*, int, int, int, int, int, int,
                           float2*, int);
__global__ void k_transfer_step(const double2*, int, const float2*, int, int, int, const float2*, int, int, int, int,
                                double2*);

// small helper kernels local to this file
__global__ void k_set_one(float2* p) {
    if (threadIdx.x == 0 && blockIdx.x == 0) p[0] = make_float2(1.f, 0.f);
}
__global__ void k_set_boundary(int* bond, int N) {
    if (threadIdx.x == 0 && blockIdx.x == 0) { bond[0] = 1; bond[N] = 1; }
}
__global__ void k_set_reg(int* R, int reg, int v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) R[reg] = v;
}
__global__ void k_plan_dense(const int* bond, int p, int d, int* R) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        R[R_TMP0] = bond[p];
        R[R_TMP1] = bond[p + 1];
        R[R_TMP2] = d * bond[p + 1];
    }
}
__global__ void k_copy_ledger_out(const double* ledger, const int* R, double* out_d, int* out_i) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        for (int i = 0; i < L_COUNT; ++i) out_d[i] = ledger[i];
        out_i[0] = R[R_SWEEPS];
        out_i[1] = R[R_FLAGS];
        out_i[2] = R[R_MAXBOND];
    }
}

// ------------------------------------------------------------------ workspace layout
// Offset of a region a layout does not provide: bound to a null pointer, so a use cannot alias another region.
constexpr size_t WS_UNUSED = ~(size_t)0;

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

WsLayout ws_layout(int N, int d, int chi, int w, long long dense) {
    WsLayout L{};
    L.n_sites = N;
    L.chi = chi;
    L.d = d;
    L.w = w;
    L.m_cap = d * chi;
    L.n_cap = std::max(w, 1) * chi;
    L.p_cap = EIG_MAX;
    L.dense = dense;
    const size_t c8 = sizeof(float2), c16 = sizeof(double2);
    const size_t mc = (size_t)L.m_cap, nc = (size_t)L.n_cap, pc = (size_t)L.p_cap;
    const size_t gdim = std::max(mc, pc);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    L.ledger = take(L_COUNT * sizeof(double) + 64 * sizeof(int));
    L.regs = take(R_COUNT * sizeof(int) + (2 * gdim + 1024) * sizeof(int));   // registers, perm, tmp bonds
    L.T = take(mc * nc * c8);
    L.P = take((size_t)chi * std::max(w, 1) * d * chi * c8);
    L.carry = take((size_t)chi * nc * c8 + c8);
    L.G64 = take(gdim * gdim * c16);
    L.G32 = take(std::max(gdim * gdim, pc * nc) * c8);   // B = Q^dagger T of the range finder
    L.U = take(gdim * gdim * c8);
    L.lam = take(4 * gdim * sizeof(double));
    L.Y = take(gdim * pc * c8);
    L.Q = take(std::max(gdim * pc, pc * pc) * c8);
    L.S64 = take(gdim * gdim * c16);
    L.Z = take(std::max(gdim * nc, pc * pc) * c8);   // projected rows X = U^dagger T (zip-up)
    L.omega = WS_UNUSED;
    const size_t dn = (size_t)std::max<long long>(dense, 1);
    L.X0 = take(dn * c8);
    L.X1 = take(dn * c8);
    L.b64 = take(build64_scratch_bytes(std::max(N, 1)));   // FP64 operator builds
    // packed operands of the tensor-core site contraction: (chi w) x (d chi) x chi at the capacities
    L.tc_bytes = tc_pack_bytes(chi * std::max(w, 1), d * chi, chi);
    L.tc = take(L.tc_bytes);
    L.total = off;
    return L;
}

static Ws ws_bind(void* base, const WsLayout& L) {
    char* b = (char*)base;
    auto at = [b](size_t off) -> char* { return off == WS_UNUSED ? nullptr : b + off; };
    Ws w;
    w.L = L;
    w.ledger = (double*)at(L.ledger);
    w.R = (int*)at(L.regs);
    w.T = (float2*)at(L.T);
    w.P = (float2*)at(L.P);
    w.carry = (float2*)at(L.carry);
    w.G64 = (double2*)at(L.G64);
    w.G32 = (float2*)at(L.G32);
    w.U = (float2*)at(L.U);
    w.lam = (double*)at(L.lam);
    w.Y = (float2*)at(L.Y);
    w.Q = (float2*)at(L.Q);
    w.S64 = (double2*)at(L.S64);
    w.Z = (float2*)at(L.Z);
    w.X0 = (float2*)at(L.X0);
    w.X1 = (float2*)at(L.X1);
    w.tc = at(L.tc);
    return w;
}

// extra int scratch after the registers: perm[gdim], tmp bonds[...]
static int* ws_perm(Ws& w) { return w.R + R_COUNT; }
static double* ws_weights(Ws& w) { return w.lam + std::max(w.L.m_cap, w.L.p_cap); }
static double* ws_lam2(Ws& w) { return w.lam + 2 * std::max(w.L.m_cap, w.L.p_cap); }


long long launch_total();
void add_launches(long long n);
void prof_begin(bool on, double* ledger);
void prof_read(int cls, double* ms, long long* launches);

// Truncation rules: FP32 plain or mixed (tensor-core site contractions), a finite non-negative cutoff.
bool trunc_ok(const qtn_trunc& t) {
    return (t.prec == QTN_PLAIN_FP32 || t.prec == QTN_MIXED) && t.cutoff >= 0.0 && isfinite(t.cutoff) &&
           t.max_sweeps >= 0;
}

// Relative weight below which a direction of an untruncated (gauge-only) sweep is FP32 round-off.
constexpr double EXACT_CUTOFF = 1e-13;

cudaError_t configure_eig_kernel();
cudaError_t configure_build64_kernel();
cudaError_t configure_tc_kernel();

// Kernels with more than 48 KB of dynamic shared memory need the opt-in on every device they run on.
static std::once_flag g_dev_once[QTN_MAX_DEVICES];
static cudaError_t g_dev_err[QTN_MAX_DEVICES];

cudaError_t configure_device_kernels(int device) {
    if (device < 0 || device >= QTN_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::call_once(g_dev_once[device], [device]() {
        int prev = -1;
        cudaError_t e = cudaGetDevice(&prev);
        if (e == cudaSuccess && prev != device) e = cudaSetDevice(device);
        if (e == cudaSuccess) e = configure_eig_kernel();
        if (e == cudaSuccess) e = configure_build64_kernel();
        if (e == cudaSuccess) e = configure_tc_kernel();
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_cgs_block_32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CGS_SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_cgs_block_16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CGS_SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_cgs_block_8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CGS_SMEM);
        if (prev >= 0 && prev != device) cudaSetDevice(prev);
        g_dev_err[device] = e;
    });
    return g_dev_err[device];
}

int grid_for(long long n, int threads, int sm) {
    long long g = (n + threads - 1) / threads;
    long long cap = (long long)sm * 8;
    return (int)std::max(1LL, std::min(g, cap));
}

// ------------------------------------------------------------------ truncated SVD of T (m x n, row stride n)
//
// 1. G = T T^dagger, FP32 products accumulated in FP64 (split-K atomics).
// 2. Eigenbasis U of G: one-sided Jacobi in shared memory when m <= EIG_MAX; otherwise a randomised
//    range finder with power iterations and a Rayleigh-Ritz step on an EIG_MAX-dimensional subspace.
// 3. X = U^dagger T; row weights |x_i|^2 (FP64) are the captured weights of every direction; the
//    truncation rule runs on them with total = trace(G).  The kept columns of U become the new
//    site and the kept rows of X the carry.
struct TsvdIO {
    const float2* T;     // input, row stride R_N
    Dim m, n;            // live dims
    int m_cap;           // capacity of m (host)
    long long n_cap;     // capacity of n (host)
    float2* X;           // output rows U^dagger T, row stride R_N, capacity m_cap x n_cap (or p x n)
};

// Kernels launched inside the bodies of conditional graph nodes that ran (added by the condition kernel, so
// that the launch count reports what executed, not what was recorded).
__device__ unsigned long long g_cond_launches = 0;
static std::atomic<bool> g_cond_used{false};

// Condition of a graph conditional node from a dimension register: R[reg] == val selects the first body.
__global__ void k_set_cond(cudaGraphConditionalHandle h, const int* __restrict__ R, int reg, int val,
                           unsigned long long n_first, unsigned long long n_second) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const bool first = (R[reg] == val);
        cudaGraphSetConditional(h, first ? 1u : 0u);
        atomicAdd(&g_cond_launches, first ? n_first : n_second);
    }
}

// Under stream capture on `s`: records a conditional node whose first body (then_fn) runs when R[reg] == val
// and whose second body (else_fn, when given) runs otherwise.  The bodies are captured into the node's child
// graphs on the context's helper stream of nesting level `depth` (the enqueueing code reads its stream from
// `s`, which is switched for the duration); the condition kernel follows on `s` and the node depends on it;
// capture of the outer graph continues after the node.
static qtn_status capture_if(Ctx* c, cudaStream_t& s, int* R, int reg, int val, int depth,
                             const std::function<qtn_status()>& then_fn, const std::function<qtn_status()>& else_fn) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = else_fn ? 2 : 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p));
    const cudaStream_t outer = s;
    const cudaStream_t helper = c->helper[depth];
    long long n_body[2] = {0, 0};
    for (unsigned b = 0; b < p.conditional.size; ++b) {
        CK(cudaStreamBeginCaptureToGraph(helper, p.conditional.phGraph_out[b], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed));
        const long long l0 = launch_total();
        s = helper;
        const qtn_status st = (b == 0) ? then_fn() : else_fn();
        s = outer;
        n_body[b] = launch_total() - l0;
        cudaGraph_t body = nullptr;
        const cudaError_t e = cudaStreamEndCapture(helper, &body);
        if (st) return st;
        CK(e);
    }
    add_launches(-(n_body[0] + n_body[1]));   // counted on the device by the condition kernel instead
    g_cond_used = true;
    k_set_cond<<<1, 1, 0, s>>>(h, R, reg, val, (unsigned long long)n_body[0], (unsigned long long)n_body[1]);
    CKL();
    count_launch(PROF_OTHER, s, false);
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    std::vector<cudaGraphNode_t> to(nd, node);
    CK(cudaGraphAddDependencies(g, deps, to.data(), nullptr, nd));
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return QTN_OK;
}

static qtn_status tsvd(Ctx* c, Ws& w, const TsvdIO& io, const qtn_trunc& tr, int chi_cap_out, Dim& rows_out) {
    cudaStream_t s = c->stream;
    const int mc = io.m_cap;
    const int gld = std::max(w.L.m_cap, w.L.p_cap);
    const int pc = w.L.p_cap;
    const int max_sweeps = tr.max_sweeps > 0 ? tr.max_sweeps : 30;
    const int ncap = (int)std::min<long long>(io.n_cap, 1 << 30);
    // The FP32 refinement pass below corrects the first eigen-solve, which only has to give a rough basis.
    constexpr float tol1 = 1e-4f;
    // Eigenvalues below dead_rel of the largest are FP32 round-off of the Gram: the rough first solve hands
    // those directions to the refinement as completion vectors; the refinement itself only drops what it
    // cannot rotate (products of eigenvalues below the noise floor of the Jacobi sweeps).  At 1e-8 the
    // refinement converges in as many sweeps as from the full first basis and the norm of a Fresnel step
    // stays as close to the FP64 result as without the cut (1e-6 doubled both).
    constexpr float dead1 = 1e-8f;
    constexpr float DEAD_REFINE = 1e-13f;
    // The rough first solve stops after four sweeps (its non-convergence is not reported: the refinement
    // finishes the job); the refinement's tolerance sits five times above the FP32 rounding of a
    // 160-term inner product (~6e-7 of |x||y|), below which rotations only chase rounding.
    const int sweeps1 = std::min(max_sweeps, 4);
    constexpr float TOL_REFINE = 3e-6f;
    k_path<<<1, 1, 0, s>>>(io.m, w.R, w.ledger);
    CKL();
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cap_status));
    const bool capturing = (cap_status == cudaStreamCaptureStatusActive) && c->helper[1] != nullptr;
    // Gram G = A A^dagger of an m x n matrix with row stride ld (FP32 products, FP64 split-K accumulation)
    auto gram = [&](const float2* A, Dim m, Dim ld, Dim n, int m_cap, int guard, bool zero,
                    long long n_cap) -> qtn_status {
        if (zero) CK(cudaMemsetAsync(w.G64, 0, (size_t)m_cap * gld * sizeof(double2), s));
        GemmDesc g{};
        g.A = mat(A, ld, dc(1));
        g.B = mat(A, dc(1), ld, 1);
        g.C = w.G64; g.crs = dc(gld); g.ccs = dc(1);
        g.M = m; g.N = m; g.K = n;
        g.mode = OUT_ATOMIC64;
        const int tiles = ((m_cap + 63) / 64) * ((m_cap + 63) / 64);
        const long long want = std::max(1, (c->sm_count * 4) / std::max(tiles, 1));
        long long kc = std::max<long long>(256, (n_cap + want - 1) / want);
        g.kchunk = (int)std::min<long long>((kc + 15) / 16 * 16, 1 << 30);
        if (guard >= 0) { g.guard_reg = R_RAND; g.guard_val = guard; }
        CK(launch_gemm(g, m_cap, m_cap, (int)std::min<long long>(n_cap, 1 << 30), w.R, s));
        return QTN_OK;
    };
    qtn_status st;
    // ---- shared-memory path (m <= EIG_MAX): eigenbasis U of G = T T^dagger, X = U^dagger T
    auto shared_path = [&]() -> qtn_status {
    if ((st = gram(io.T, io.m, io.n, io.n, std::min(mc, EIG_MAX), 0, true, io.n_cap))) return st;
    k_trace<<<1, 256, 0, s>>>(w.G64, gld, io.m, w.R, w.ledger);
    CKL();
    CK(launch_eig(w.G64, dc(gld), io.m, w.U, dc(gld), w.lam, w.R, std::min(mc, EIG_MAX), sweeps1, w.ledger, s,
                  R_RAND, 0, tol1, dead1, false, true));
    {
        GemmDesc g{};
        g.A = mat(w.U, dc(gld), dc(1), 1);
        g.B = mat(io.T, io.n, dc(1));
        g.C = io.X; g.crs = io.n; g.ccs = dc(1);
        g.M = io.m; g.N = io.n; g.K = io.m;
        g.guard_reg = R_RAND; g.guard_val = 0;
        CK(launch_gemm(g, std::min(mc, EIG_MAX), ncap, std::min(mc, EIG_MAX), w.R, s));
    }
    return QTN_OK;
    };
    // ---- range-finder path (m > EIG_MAX): Q = orth(T Omega) by block CGS2, exact path on B = Q^dagger T,
    //      U = Q U_B.  No product with G is ever formed, so the FP32 dynamic range is that of T itself.
    auto range_path = [&]() -> qtn_status {
        if (mc > CGS_MAXM_ALL) return QTN_ERR_WORKSPACE;
        const int Ph = EIG_MAX;                             // = R[R_P] on this path
        const Dim P = dc(Ph);
        k_total_weight<<<grid_for((long long)mc * ncap, 256, c->sm_count), 256, 0, s>>>(io.T, io.n, io.m, io.n,
                                                                                            w.R, w.ledger);
        CKL();
        float* pre = (float*)ws_lam2(w);                       // pre-projection column norms
        const long long bcap = (long long)std::max<size_t>((size_t)gld * gld, (size_t)pc * w.L.n_cap);
        const long long cw = std::max<long long>(1, bcap / pc);  // column chunk of T that fits the B buffer
        const bool one_chunk = (io.n_cap <= cw);
        {   // Y = T Omega
            GemmDesc g{};
            g.A = mat(io.T, io.n, dc(1));
            g.C = w.Y; g.crs = dc(pc); g.ccs = dc(1);
            g.M = io.m; g.N = P; g.K = io.n;
            g.omega_seed = 7919;
            g.guard_reg = R_RAND; g.guard_val = 1;
            CK(launch_gemm(g, mc, pc, ncap, w.R, s));
        }
        const size_t cgs_smem = CGS_SMEM;
        // orthonormalise the p columns of Yb (rows live `rows`, at most rows_cap) in place by block classical
        // Gram-Schmidt with reorthogonalisation: each block is projected against the finished blocks and
        // orthonormalised internally, twice; runs when R[greg] == 1
        auto block_orth = [&](float2* Yb, Dim rows, int rows_cap, int greg) -> qtn_status {
            const int CGS_B = (rows_cap <= 512) ? 32 : (rows_cap <= 1024 ? 16 : 8);
            k_col_norms<<<grid_for((long long)pc * 32, 256, c->sm_count), 256, 0, s>>>(Yb, pc, rows, P, pre, w.R,
                                                                                      greg);
            CKL();
            for (int b0 = 0; b0 < Ph; b0 += CGS_B) {
                for (int pass = 0; pass < (b0 > 0 ? 2 : 1); ++pass) {
                    if (b0 > 0) {
                        GemmDesc g{};                               // Cb = Q[:, :b0]^dagger Y[:, b0:b0+B]
                        g.A = mat(Yb, dc(1), dc(pc), 1);
                        g.B = mat(Yb + b0, dc(pc), dc(1));
                        g.C = w.Z; g.crs = dc(CGS_B); g.ccs = dc(1);
                        g.M = dc(b0); g.N = dc(CGS_B); g.K = rows;
                        g.guard_reg = greg; g.guard_val = 1;
                        CK(launch_gemm(g, b0, CGS_B, rows_cap, w.R, s));
                        GemmDesc h{};                               // Y[:, b0:b0+B] -= Q[:, :b0] Cb
                        h.A = mat(Yb, dc(pc), dc(1));
                        h.B = mat(w.Z, dc(CGS_B), dc(1));
                        h.C = Yb + b0; h.crs = dc(pc); h.ccs = dc(1);
                        h.M = rows; h.N = dc(CGS_B); h.K = dc(b0);
                        h.mode = OUT_ACCUM; h.alpha_re = -1.f;
                        h.guard_reg = greg; h.guard_val = 1;
                        CK(launch_gemm(h, rows_cap, CGS_B, b0, w.R, s));
                    }
                    const int decide = (pass == 0);
                    if (CGS_B == 32)
                        k_cgs_block_32<<<1, 1024, cgs_smem, s>>>(Yb, pc, rows, b0, Ph, pre, w.R, greg, decide);
                    else if (CGS_B == 16)
                        k_cgs_block_16<<<1, 1024, cgs_smem, s>>>(Yb, pc, rows, b0, Ph, pre, w.R, greg, decide);
                    else k_cgs_block_8<<<1, 1024, cgs_smem, s>>>(Yb, pc, rows, b0, Ph, pre, w.R, greg, decide);
                    CKL();
                }
            }
            return QTN_OK;
        };
        if ((st = block_orth(w.Y, io.m, mc, R_RAND))) return st;
        // Power iteration, only for a full-rank sketch (otherwise the sketch already spans the range of T).
        // Each product with T or T^dagger is orthonormalised before the next, so a direction is never
        // represented at the square of its relative singular value.
        k_set_pi<<<1, 1, 0, s>>>(w.R);
        CKL();
        // Three power iterations: for a chi-limited truncation of a slowly decaying spectrum every iteration
        // shrinks the weight the sketch misses near the kept rank by about (s_(p+1) / s_k)^4 (one was measured
        // 2.6e-5 of |T|^2 above the Eckart-Young optimum at 512 x 768, chi 128, s_k / s_1 = 0.08).
        auto power_iters = [&]() -> qtn_status {
        for (int it = 0; it < RF_POWER_ITERS; ++it) {
            if (one_chunk && ncap <= 2048) {   // Z fits the B buffer whole and the block orthonormaliser
                {   // Z = T^dagger Q (n x p) in the B buffer
                    GemmDesc g{};
                    g.A = mat(io.T, dc(1), io.n, 1);
                    g.B = mat(w.Y, dc(pc), dc(1));
                    g.C = w.G32; g.crs = dc(pc); g.ccs = dc(1);
                    g.M = io.n; g.N = P; g.K = io.m;
                    g.guard_reg = R_PI; g.guard_val = 1;
                    CK(launch_gemm(g, ncap, pc, mc, w.R, s));
                }
                if ((st = block_orth(w.G32, io.n, ncap, R_PI))) return st;
                {   // Y = T Z
                    GemmDesc g{};
                    g.A = mat(io.T, io.n, dc(1));
                    g.B = mat(w.G32, dc(pc), dc(1));
                    g.C = w.Y; g.crs = dc(pc); g.ccs = dc(1);
                    g.M = io.m; g.N = P; g.K = io.n;
                    g.guard_reg = R_PI; g.guard_val = 1;
                    CK(launch_gemm(g, mc, pc, ncap, w.R, s));
                }
                if ((st = block_orth(w.Y, io.m, mc, R_PI))) return st;
            } else {
                // T too wide for the intermediate: Y' = T (T^dagger Q) accumulated over column chunks of T
                CK(cudaMemsetAsync(w.Q, 0, (size_t)mc * pc * sizeof(float2), s));
                for (long long c0 = 0; c0 < io.n_cap; c0 += cw) {
                    const int cwid = (int)std::min<long long>(cw, io.n_cap - c0);
                    const Dim ncol = one_chunk ? io.n : dc(cwid);
                    GemmDesc g{};                                       // Z1 = T_c^dagger Q  (cw x p) in the B buffer
                    g.A = mat(io.T + c0, dc(1), io.n, 1);
                    g.B = mat(w.Y, dc(pc), dc(1));
                    g.C = w.G32; g.crs = dc(pc); g.ccs = dc(1);
                    g.M = ncol; g.N = P; g.K = io.m;
                    g.guard_reg = R_PI; g.guard_val = 1;
                    CK(launch_gemm(g, cwid, pc, mc, w.R, s));
                    GemmDesc h{};                                       // Y' += T_c Z1
                    h.A = mat(io.T + c0, io.n, dc(1));
                    h.B = mat(w.G32, dc(pc), dc(1));
                    h.C = w.Q; h.crs = dc(pc); h.ccs = dc(1);
                    h.M = io.m; h.N = P; h.K = ncol;
                    h.mode = OUT_ACCUM;
                    h.guard_reg = R_PI; h.guard_val = 1;
                    CK(launch_gemm(h, mc, pc, cwid, w.R, s));
                }
                if ((st = block_orth(w.Q, io.m, mc, R_PI))) return st;
                k_copy_guarded<<<grid_for((long long)mc * pc, 256, c->sm_count), 256, 0, s>>>(w.Q, w.Y,
                                                                                           (long long)mc * pc, w.R,
                                                                                           R_PI, 1);
                CKL();
            }
        }
        return QTN_OK;
        };
        // under graph capture the iterations sit in the body of a conditional node (skipped, not replayed as
        // no-ops, when the sketch is rank-deficient); eagerly they are launched and retire on the device guard
        if (capturing) {
            if ((st = capture_if(c, s, w.R, R_PI, 1, 1, power_iters, nullptr))) return st;
        } else if ((st = power_iters())) {
            return st;
        }
        // a rank-deficient sketch: its live columns first, their count the subspace size from here on
        {
            int* sperm = (int*)ws_lam2(w);
            k_sketch_live<<<1, 256, 0, s>>>(w.Y, pc, io.m, pc, sperm, w.R);
            CKL();
            k_copy_guarded<<<grid_for((long long)mc * pc, 256, c->sm_count), 256, 0, s>>>(w.Y, w.Q, (long long)mc * pc,
                                                                                       w.R, R_DEP, 1);
            CKL();
            k_sketch_gather<<<grid_for((long long)mc * pc, 256, c->sm_count), 256, 0, s>>>(w.Q, w.Y, pc, io.m, pc,
                                                                                        sperm, w.R);
            CKL();
        }
        const Dim Pl = dr(R_P);    // live subspace size (EIG_MAX for a full-rank sketch)
        float2* Qb = w.Y;          // orthonormal basis of the sketch
        float2* UB = w.Q;          // eigenvectors of the Gram of B (p x p, column-major)
        // Gram of B = Q^dagger T accumulated over column chunks of T that fit the B buffer (B is never
        // needed whole: X is formed from T and U directly)
        CK(cudaMemsetAsync(w.G64, 0, (size_t)pc * gld * sizeof(double2), s));
        for (long long c0 = 0; c0 < io.n_cap; c0 += cw) {
            const int cwid = (int)std::min<long long>(cw, io.n_cap - c0);
            const Dim ncol = one_chunk ? io.n : dc(cwid);
            GemmDesc g{};
            g.A = mat(Qb, dc(1), dc(pc), 1);
            g.B = mat(io.T + c0, io.n, dc(1));
            g.C = w.G32; g.crs = ncol; g.ccs = dc(1);
            g.M = Pl; g.N = ncol; g.K = io.m;
            g.guard_reg = R_RAND; g.guard_val = 1;
            CK(launch_gemm(g, pc, cwid, mc, w.R, s));
            if ((st = gram(w.G32, Pl, ncol, ncol, pc, 1, false, cwid))) return st;
        }
        CK(launch_eig(w.G64, dc(gld), Pl, UB, dc(pc), w.lam, w.R, pc, sweeps1, w.ledger, s, R_RAND, 1, tol1, dead1,
                      false, true));
        {   // U = Q U_B  (m x p, column-major with leading dimension gld)
            GemmDesc g{};
            g.A = mat(Qb, dc(pc), dc(1));
            g.B = mat(UB, dc(1), dc(pc));
            g.C = w.U; g.crs = dc(1); g.ccs = dc(gld);
            g.M = io.m; g.N = Pl; g.K = Pl;
            g.guard_reg = R_RAND; g.guard_val = 1;
            CK(launch_gemm(g, mc, pc, pc, w.R, s));
        }
        {   // X = U^dagger T  (p x n)
            GemmDesc g{};
            g.A = mat(w.U, dc(gld), dc(1), 1);
            g.B = mat(io.T, io.n, dc(1));
            g.C = io.X; g.crs = io.n; g.ccs = dc(1);
            g.M = Pl; g.N = io.n; g.K = io.m;
            g.guard_reg = R_RAND; g.guard_val = 1;
            CK(launch_gemm(g, pc, ncap, mc, w.R, s));
        }
        return QTN_OK;
    };
    // The two paths: under graph capture the bodies of one IF/ELSE conditional node on R_RAND (only the path
    // taken runs); eagerly both are launched and the one not taken retires on its device guard.
    if (mc <= EIG_MAX) {
        if ((st = shared_path())) return st;
    } else if (capturing) {
        if ((st = capture_if(c, s, w.R, R_RAND, 1, 0, range_path, shared_path))) return st;
    } else {
        if ((st = shared_path())) return st;
        if ((st = range_path())) return st;
    }
    const Dim rows = dr(R_ROWS);
    const int rcap = std::min(mc, EIG_MAX);
    {
        // Refinement: the Gram of the projected rows X = U^dagger T is diagonal up to the FP32 error of the
        // first eigenbasis; Jacobi on it converges in a couple of sweeps and, unlike a tridiagonal solver,
        // keeps every direction accurate relative to its own scale.  U <- U V2 and X is formed again from T.
        // This removes the weight that first-pass eigenvectors leak into numerically null directions.
        if ((st = gram(io.X, rows, io.n, io.n, rcap, -1, true, io.n_cap))) return st;
        CK(launch_eig(w.G64, dc(gld), rows, w.Y, dc(pc), w.lam, w.R, rcap, max_sweeps, w.ledger, s, -1, 0, TOL_REFINE,
                      DEAD_REFINE));
        GemmDesc g{};                                   // U2 = U V2 (column-major, ld gld) in the Q buffer
        g.A = mat(w.U, dc(1), dc(gld));
        g.B = mat(w.Y, dc(1), dc(pc));
        g.C = w.Q; g.crs = dc(1); g.ccs = dc(gld);
        g.M = io.m; g.N = rows; g.K = rows;
        CK(launch_gemm(g, mc, rcap, rcap, w.R, s));
        // One Newton-Schulz step U = U2 (3 I - S) / 2 with S = U2^dagger U2 (FP64-accumulated): the eigenbases
        // are products of FP32 plane rotations, unitary to ~1e-6; the step takes the isometry error to its
        // square (below the FP32 rounding of the product) without touching the subspace at first order.
        CK(cudaMemsetAsync(w.G64, 0, (size_t)rcap * gld * sizeof(double2), s));
        GemmDesc sg{};                                  // S = U2^dagger U2  (rows x rows, FP64)
        sg.A = mat(w.Q, dc(gld), dc(1), 1);
        sg.B = mat(w.Q, dc(1), dc(gld));
        sg.C = w.G64; sg.crs = dc(gld); sg.ccs = dc(1);
        sg.M = rows; sg.N = rows; sg.K = io.m;
        sg.mode = OUT_ATOMIC64;
        {
            const int tiles = ((rcap + 63) / 64) * ((rcap + 63) / 64);
            const int want = std::max(1, (c->sm_count * 4) / std::max(tiles, 1));
            const int kc = std::max(256, (mc + want - 1) / want);
            sg.kchunk = (kc + 15) / 16 * 16;
        }
        CK(launch_gemm(sg, rcap, rcap, mc, w.R, s));
        k_ns_coeff<<<grid_for((long long)rcap * rcap, 256, c->sm_count), 256, 0, s>>>(w.G64, gld, w.G32, gld, rows,
                                                                                     w.R);
        CKL();
        GemmDesc ng{};                                  // U = U2 (3 I - S) / 2  (column-major, ld gld)
        ng.A = mat(w.Q, dc(1), dc(gld));
        ng.B = mat(w.G32, dc(gld), dc(1));
        ng.C = w.U; ng.crs = dc(1); ng.ccs = dc(gld);
        ng.M = io.m; ng.N = rows; ng.K = rows;
        CK(launch_gemm(ng, mc, rcap, rcap, w.R, s));
        GemmDesc h{};                                   // X = U^dagger T
        h.A = mat(w.U, dc(gld), dc(1), 1);
        h.B = mat(io.T, io.n, dc(1));
        h.C = io.X; h.crs = io.n; h.ccs = dc(1);
        h.M = rows; h.N = io.n; h.K = io.m;
        CK(launch_gemm(h, rcap, ncap, mc, w.R, s));
    }
    k_row_weights<<<grid_for((long long)gld * 32, 256, c->sm_count), 256, 0, s>>>(io.X, io.n, rows, io.n,
                                                                                    ws_weights(w), w.R);
    CKL();
    k_select<<<1, 256, 0, s>>>(ws_weights(w), rows, tr.chi_max, tr.cutoff, chi_cap_out, -1, ws_perm(w), w.R,
                               w.ledger);
    CKL();
    rows_out = rows;
    return QTN_OK;
}

// ------------------------------------------------------------------ one zip-up sweep
qtn_status zip_pass(Ctx* c, Ws& w, qtn_mps* psi, const qtn_mpo* W, int axis, int moff, int mn, int mirror,
                           const qtn_trunc& tr) {
    cudaStream_t s = c->stream;
    const int N = psi->n_sites, d = psi->d, cap = psi->chi_cap;
    const int wcap = W ? W->w_cap : 1, wmax = W ? std::max(W->w_max, 1) : 1;
    if (d * cap > w.L.m_cap || wmax * cap > w.L.n_cap || wmax > std::max(w.L.w, 1)) return QTN_ERR_WORKSPACE;
    float2* sites = (float2*)psi->sites;
    const size_t sstride = (size_t)cap * d * cap;
    k_set_one<<<1, 1, 0, s>>>(w.carry);
    CKL();
    qtn_trunc t2 = tr;
    if (t2.chi_max <= 0) t2.chi_max = INT_MAX;   // no cap: the bond capacity limits (and reports)
    for (int p = 0; p < N; ++p) {
        const int q = mirror ? N - 1 - p : p;
        float2* site_q = sites + (size_t)q * sstride;
        k_plan_site<<<1, 1, 0, s>>>(psi->bond, W ? W->bond : nullptr, N, d, mirror, moff, mn, p, w.R);
        CKL();
        {   // P[(x a), (t k)] = sum_j carry[(x a), j] A_q[j, t, k]
            GemmDesc g{};
            g.A = mat(w.carry, dr(R_CHIL), dc(1));
            g.B = mirror ? mat2(site_q, dc(1), dr(R_CHIR), dc(cap), dc(d * cap))
                         : mat2(site_q, dc(d * cap), dr(R_CHIR), dc(cap), dc(1));
            g.C = w.P; g.crs = dr(R_DN); g.ccs = dc(1);
            g.M = dr(R_MID); g.N = dr(R_DN); g.K = dr(R_CHIL);
            g.mode = OUT_STORE; g.alpha_re = 1.f; g.omega_seed = -1;
            // the site contraction: split-BF16 tensor cores with FP32 accumulation in mixed precision
            if (tr.prec == QTN_MIXED)
                CK(launch_gemm_tc(g, cap * wmax, d * cap, cap, w.R, w.tc, w.L.tc_bytes, c->sm_count, s));
            else CK(launch_gemm(g, cap * wmax, d * cap, cap, w.R, s));
        }
        const float2* Wc = nullptr;
        const int qm = q - moff;
        if (W && qm >= 0 && qm < mn) Wc = (const float2*)W->sites + (size_t)qm * wcap * 4 * wcap;
        k_stage2<<<grid_for((long long)d * cap * wmax * cap, 256, c->sm_count), 256, 0, s>>>(w.P, w.T, Wc, wcap,
                                                                                             mirror, d, axis, w.R);
        CKL();
        if (p == N - 1) {
            k_write_last<<<1, 256, 0, s>>>(w.T, site_q, cap, d, mirror, w.R);
            CKL();
            break;
        }
        TsvdIO io{w.T, dr(R_M), dr(R_N), d * cap, (long long)wmax * cap, w.Z};
        Dim rows;
        qtn_status st = tsvd(c, w, io, t2, cap, rows);
        if (st) return st;
        const int gld = std::max(w.L.m_cap, w.L.p_cap);
        k_write_site<<<grid_for((long long)cap * d * cap, 256, c->sm_count), 256, 0, s>>>(
            w.U, gld, ws_perm(w), site_q, cap, d, mirror, psi->bond, mirror ? q : q + 1, w.R);
        CKL();
        k_gather_rows<<<grid_for((long long)cap * wmax * cap, 256, c->sm_count), 256, 0, s>>>(
            w.Z, dr(R_N), ws_perm(w), w.carry, dr(R_N), dr(R_N), w.R);
        CKL();
    }
    const int qlast = mirror ? 0 : N - 1;
    k_site_norm2<<<1, 512, 0, s>>>(sites + (size_t)qlast * sstride, cap, d, psi->bond, qlast, w.ledger, L_NORM2);
    CKL();
    psi->canon = mirror ? QTN_CANON_RIGHT : QTN_CANON_LEFT;
    return QTN_OK;
}

// Status of a set of flag bits, most severe first.
static qtn_status flags_status(int f) {
    if (f & F_TIMEOUT) return QTN_ERR_TIMEOUT;
    if (f & F_NONFINITE) return QTN_ERR_NONFINITE;
    if (f & F_CAPACITY) return QTN_ERR_CAPACITY;
    if (f & F_NOCONV) return QTN_ERR_NOCONV;
    return QTN_OK;
}

// With a statistics struct the call waits for its work, copies the statistics and returns the status of the
// flags its kernels raised (the flags stay in the sticky status word too, until qtn_check reads them).
// Without one the call returns at once; its flags are read by the next qtn_check.
qtn_status fill_stats(Ctx* c, Ws& w, qtn_stats* st) {
    if (!st) return QTN_OK;
    double hd[L_COUNT];
    int hi[4];
    CK(cudaMemcpyAsync(hd, w.ledger, sizeof(hd), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(hi, w.R + R_SWEEPS, 3 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    st->discarded = hd[L_DISCARDED];
    st->norm2 = hd[L_NORM2];
    st->sweeps_used = hi[0];
    st->flags = hi[1];
    st->max_bond = hi[2];
    return flags_status(hi[1]);
}

// Reads and clears the sticky status word of a workspace (synchronises the stream).
static qtn_status check_sticky(cudaStream_t s, Ws& w) {
    int f = 0;
    CK(cudaMemcpyAsync(&f, w.R + R_STICKY, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemsetAsync(w.R + R_STICKY, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    return flags_status(f);
}

static qtn_status check_ws(const WsLayout& need, void* ws, size_t bytes) {
    if (!ws) return QTN_ERR_WORKSPACE;
    if (bytes < need.total) return QTN_ERR_WORKSPACE;
    return QTN_OK;
}

static int mps_layout_n(const qtn_mps* psi, qtn_layout layout) {
    if (layout == QTN_LAYOUT_INTERLEAVED) return psi->n_sites;
    if (layout == QTN_LAYOUT_SERIAL) return psi->n_sites / 2;
    return psi->n_sites;
}

}  // namespace qtn

using namespace qtn;

// ============================================================================ C ABI

qtn_status bind_ws(qtn_context* x, void* ws, size_t bytes, Ws& w) {
    set_gemm_tile(x->c.gemm_tile);
    set_gemm_sms(x->c.sm_count);
    if (!x->have_layout) return QTN_ERR_WORKSPACE;
    qtn_status st = check_ws(x->L, ws, bytes);
    if (st) return st;
    w = ws_bind(ws, x->L);
    return QTN_OK;
}

extern "C" {

int qtn_version(void) { return 1; }

long long qtn_launch_count(void) {
    unsigned long long cond = 0;
    if (g_cond_used && cudaMemcpyFromSymbol(&cond, g_cond_launches, sizeof(cond)) != cudaSuccess) cond = 0;
    return launch_total() + (long long)cond;
}

qtn_status qtn_profile(void* ctx, int enable, void* ws, size_t ws_bytes) {
    if (!ctx) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    double* ledger = nullptr;
    if (enable) {
        Ws w;
        qtn_status st = bind_ws(x, ws, ws_bytes, w);
        if (st) return st;
        ledger = w.ledger;
        CK(cudaMemsetAsync(ledger + L_PROF_GEMM, 0, 3 * sizeof(double), x->c.stream));
    }
    prof_begin(enable != 0, ledger);
    return QTN_OK;
}

qtn_status qtn_profile_read(void* ctx, int kernel_class, double* ms, long long* launches, double* flops, void* ws,
                            size_t ws_bytes) {
    if (!ctx || !ms || !launches || !flops || kernel_class < 0 || kernel_class > 2) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    CK(cudaStreamSynchronize(x->c.stream));
    const int cls = kernel_class == 0 ? PROF_GEMM : (kernel_class == 1 ? PROF_EIG : PROF_TC);
    const int slot = kernel_class == 0 ? L_PROF_GEMM : (kernel_class == 1 ? L_PROF_EIG : L_PROF_TC);
    prof_read(cls, ms, launches);
    CK(cudaMemcpy(flops, w.ledger + slot, sizeof(double), cudaMemcpyDeviceToHost));
    return QTN_OK;
}

const char* qtn_status_string(qtn_status s) {
    switch (s) {
        case QTN_OK: return "ok";
        case QTN_ERR_ARG: return "invalid argument";
        case QTN_ERR_SHAPE: return "inconsistent shapes";
        case QTN_ERR_CAPACITY: return "capacity exceeded";
        case QTN_ERR_NOCONV: return "eigen-solve did not converge";
        case QTN_ERR_NONFINITE: return "non-finite value";
        case QTN_ERR_TIMEOUT: return "bounded device wait gave up";
        case QTN_ERR_CUDA: return "CUDA runtime error";
        case QTN_ERR_BOUNDS: return "index out of bounds";
        case QTN_ERR_WORKSPACE: return "workspace missing or too small";
    }
    return "unknown status";
}

qtn_status qtn_create(void** ctx, void* stream) {
    if (!ctx) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)calloc(1, sizeof(qtn_context));
    if (!x) return QTN_ERR_ARG;
    x->c.stream = (cudaStream_t)stream;
    if (cudaGetDevice(&x->c.device) != cudaSuccess) { free(x); return QTN_ERR_CUDA; }
    if (cudaDeviceGetAttribute(&x->c.sm_count, cudaDevAttrMultiProcessorCount, x->c.device) != cudaSuccess) {
        free(x);
        return QTN_ERR_CUDA;
    }
    if (configure_device_kernels(x->c.device) != cudaSuccess) {
        free(x);
        return QTN_ERR_CUDA;
    }
    x->c.gemm_tile = 64;
    // helper streams that capture the bodies of conditional graph nodes (two nesting levels)
    for (int i = 0; i < 2; ++i)
        if (cudaStreamCreateWithFlags(&x->c.helper[i], cudaStreamNonBlocking) != cudaSuccess) x->c.helper[i] = nullptr;
    *ctx = x;
    return QTN_OK;
}

qtn_status qtn_destroy(void* ctx) {
    if (!ctx) return QTN_OK;
    qtn_context* x = (qtn_context*)ctx;
    for (int i = 0; i < 2; ++i)
        if (x->c.helper[i]) cudaStreamDestroy(x->c.helper[i]);
    free(ctx);
    return QTN_OK;
}

qtn_status qtn_set_stream(void* ctx, void* stream) {
    if (!ctx) return QTN_ERR_ARG;
    ((qtn_context*)ctx)->c.stream = (cudaStream_t)stream;
    return QTN_OK;
}

qtn_status qtn_workspace_init(void* ctx, void* ws, size_t ws_bytes) {
    if (!ctx) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    // ledger and registers (with the sticky status word) are the only state a workspace carries across calls
    CK(cudaMemsetAsync(ws, 0, x->L.T, x->c.stream));
    return QTN_OK;
}

qtn_status qtn_check(void* ctx, void* ws, size_t ws_bytes) {
    if (!ctx) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    return check_sticky(x->c.stream, w);
}

qtn_status qtn_workspace_size(void* ctx, int n_sites, int d, int chi_max, int w_max, long long dense_elems,
                              size_t* bytes) {
    if (!ctx || !bytes || n_sites < 1 || (d != 2 && d != 4) || chi_max < 1 || w_max < 1 || dense_elems < 0)
        return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    x->L = ws_layout(n_sites, d, chi_max, w_max, dense_elems);
    x->have_layout = 1;
    *bytes = x->L.total;
    return QTN_OK;
}

qtn_status qtn_encode(void* ctx, const void* dense, int n, qtn_layout layout, qtn_trunc trunc, qtn_mps* out,
                      qtn_stats* stats, void* ws, size_t ws_bytes) {
    if (!ctx || !dense || !out || n < 1 || n > 30 || !trunc_ok(trunc)) return QTN_ERR_ARG;
    if (layout < QTN_LAYOUT_SERIAL || layout > QTN_LAYOUT_1D) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    const int N = layout == QTN_LAYOUT_INTERLEAVED ? n : (layout == QTN_LAYOUT_SERIAL ? 2 * n : n);
    const int d = layout == QTN_LAYOUT_INTERLEAVED ? 4 : 2;
    if (out->n_sites != N || out->d != d) return QTN_ERR_SHAPE;
    const long long total = layout == QTN_LAYOUT_1D ? (1ll << n) : (1ll << (2 * n));
    if (total > w.L.dense || d * out->chi_cap > w.L.m_cap) return QTN_ERR_WORKSPACE;
    Ctx* c = &x->c;
    cudaStream_t s = c->stream;
    k_reset_stats<<<1, 1, 0, s>>>(w.R, w.ledger);
    CKL();
    k_set_boundary<<<1, 1, 0, s>>>(out->bond, N);
    CKL();
    k_dense_to_quantics<<<grid_for(total, 256, c->sm_count), 256, 0, s>>>((const float2*)dense, w.X0, n, layout,
                                                                         w.R);
    CKL();
    qtn_trunc t2 = trunc;
    if (t2.chi_max <= 0) t2.chi_max = INT_MAX;
    const int cap = out->chi_cap;
    const size_t sstride = (size_t)cap * d * cap;
    float2* cur = w.X0;
    float2* nxt = w.X1;
    long long ncols = total / d;
    for (int p = 0; p < N - 1; ++p) {
        k_plan_encode<<<1, 1, 0, s>>>(p, d, w.R);
        CKL();
        k_set_reg<<<1, 1, 0, s>>>(w.R, R_N, (int)ncols);
        CKL();
        TsvdIO io{cur, dr(R_M), dr(R_N), d * cap, ncols, nxt};
        Dim rows;
        st = tsvd(c, w, io, t2, cap, rows);
        if (st) return st;
        const int gld = std::max(w.L.m_cap, w.L.p_cap);
        k_write_site<<<grid_for((long long)cap * d * cap, 256, c->sm_count), 256, 0, s>>>(
            w.U, gld, ws_perm(w), (float2*)out->sites + (size_t)p * sstride, cap, d, 0, out->bond, p + 1, w.R);
        CKL();
        k_gather_rows<<<grid_for((long long)cap * ncols, 256, c->sm_count), 256, 0, s>>>(nxt, dr(R_N), ws_perm(w),
                                                                                          cur, dr(R_N), dr(R_N), w.R);
        CKL();
        ncols /= d;
    }
    k_plan_encode<<<1, 1, 0, s>>>(N - 1, d, w.R);
    CKL();
    k_write_last<<<1, 256, 0, s>>>(cur, (float2*)out->sites + (size_t)(N - 1) * sstride, cap, d, 0, w.R);
    CKL();
    k_site_norm2<<<1, 512, 0, s>>>((float2*)out->sites + (size_t)(N - 1) * sstride, cap, d, out->bond, N - 1, w.ledger,
                                   L_NORM2);
    CKL();
    out->canon = QTN_CANON_LEFT;
    return fill_stats(c, w, stats);
}

}  // extern "C"

// Internal: zip-up application without resetting the statistics.
qtn_status apply_inner(qtn_context* x, Ws& w, const qtn_mpo* W, int axis, qtn_mps* psi, const qtn_trunc& tr,
                       bool diag) {
    const int d = psi->d, N = psi->n_sites;
    int moff = 0, mn = N;
    if (W) {
        mn = W->n_sites;
        if (d == 4) {
            if (N != mn) return QTN_ERR_SHAPE;
            // axis 2/3: W is an MPS viewed as a diagonal operator (elementwise product, conjugated for 3)
            if (diag ? (axis != 2 && axis != 3) : (axis != 0 && axis != 1)) return QTN_ERR_ARG;
        } else if (N == mn) {
            axis = 0;
        } else if (N == 2 * mn) {
            if (axis != 0 && axis != 1) return QTN_ERR_ARG;
            moff = axis * mn;
        } else {
            return QTN_ERR_SHAPE;
        }
    }
    qtn_status st;
    if (psi->canon == QTN_CANON_NONE) {
        qtn_trunc exact = tr;
        exact.chi_max = psi->chi_cap;
        exact.cutoff = EXACT_CUTOFF;
        st = zip_pass(&x->c, w, psi, nullptr, 0, 0, N, 0, exact);
        if (st) return st;
    }
    const int mirror = (psi->canon == QTN_CANON_LEFT) ? 1 : 0;
    return zip_pass(&x->c, w, psi, W, axis, moff, mn, mirror, tr);
}

extern "C" {

qtn_status qtn_apply_mpo(void* ctx, const qtn_mpo* W, int axis, qtn_mps* psi, qtn_trunc trunc, qtn_stats* stats,
                         void* ws, size_t ws_bytes) {
    if (!ctx || !W || !psi || !trunc_ok(trunc)) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    k_reset_stats<<<1, 1, 0, x->c.stream>>>(w.R, w.ledger);
    CKL();
    st = apply_inner(x, w, W, axis, psi, trunc, false);
    if (st) return st;
    return fill_stats(&x->c, w, stats);
}

qtn_status qtn_truncate(void* ctx, qtn_mps* psi, qtn_trunc trunc, qtn_stats* stats, void* ws, size_t ws_bytes) {
    if (!ctx || !psi || !trunc_ok(trunc)) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    k_reset_stats<<<1, 1, 0, x->c.stream>>>(w.R, w.ledger);
    CKL();
    if (psi->canon != QTN_CANON_LEFT) {
        qtn_trunc exact = trunc;
        exact.chi_max = psi->chi_cap;
        exact.cutoff = EXACT_CUTOFF;
        st = zip_pass(&x->c, w, psi, nullptr, 0, 0, psi->n_sites, 0, exact);
        if (st) return st;
        // the exact sweep discards nothing of substance; keep its FP32 round-off out of the report
        CK(cudaMemsetAsync(w.ledger + L_DISCARDED, 0, sizeof(double), x->c.stream));
    }
    st = zip_pass(&x->c, w, psi, nullptr, 0, 0, psi->n_sites, 1, trunc);
    if (st) return st;
    return fill_stats(&x->c, w, stats);
}

qtn_status qtn_fresnel_step(void* ctx, qtn_mps* psi, qtn_layout layout, const qtn_mpo* qft, const qtn_mpo* qft_dagger,
                            const qtn_mpo* phase, int n_steps, qtn_trunc trunc, qtn_stats* stats, void* ws,
                            size_t ws_bytes) {
    if (!ctx || !psi || !qft || !qft_dagger || !phase || n_steps < 0 || !trunc_ok(trunc)) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    k_reset_stats<<<1, 1, 0, x->c.stream>>>(w.R, w.ledger);
    CKL();
    const int naxes = (layout == QTN_LAYOUT_1D) ? 1 : 2;
    const qtn_mpo* ops[3] = {qft, phase, qft_dagger};
    for (int step = 0; step < n_steps; ++step)
        for (int o = 0; o < 3; ++o)
            for (int ax = 0; ax < naxes; ++ax) {
                st = apply_inner(x, w, ops[o], ax, psi, trunc, false);
                if (st) return st;
            }
    return fill_stats(&x->c, w, stats);
}

// Runs one FP64 build into `out` and returns its status; synchronises (the host needs w_max).
static qtn_status run_build64(qtn_context* x, Ws& w, void* ws, int kind, int n, double param, double cutoff,
                              double gate_cut, int pmax, int flags, qtn_mpo* out) {
    cudaStream_t s = x->c.stream;
    if (n > w.L.n_sites) return QTN_ERR_WORKSPACE;
    char* scratch = (char*)ws + w.L.b64;
    int* status = w.R + R_TMP3;
    CK(cudaMemsetAsync(status, 0, sizeof(int), s));
    CK(launch_build64(kind, n, param, cutoff, gate_cut, pmax, flags, scratch, build64_scratch_bytes(n),
                      (double*)w.X0, (float2*)out->sites, out->w_cap, out->bond, status, s));
    std::vector<int> hb(n + 2);
    CK(cudaMemcpyAsync(hb.data(), out->bond, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hb.data() + n + 1, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hb[n + 1] != QTN_OK) return (qtn_status)hb[n + 1];
    out->w_max = *std::max_element(hb.begin(), hb.begin() + n + 1);
    return QTN_OK;
}

qtn_status qtn_build_qft_mpo(void* ctx, int n, int inverse, double cutoff, qtn_mpo* out, void* ws, size_t ws_bytes) {
    if (!ctx || !out || n < 1 || n > 62 || out->n_sites != n || out->w_cap < 2 || !(cutoff >= 0.0))
        return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    return run_build64(x, w, ws, BUILD64_QFT, n, 0.0, cutoff, 0.0, 0, inverse ? 1 : 0, out);
}

qtn_status qtn_build_phase_mpo(void* ctx, int n, double c, int bit_reversed, double cutoff, qtn_mpo* out, void* ws,
                               size_t ws_bytes) {
    if (!ctx || !out || n < 1 || n > 62 || out->n_sites != n || out->w_cap < 1 || !isfinite(c) || !(cutoff >= 0.0))
        return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    return run_build64(x, w, ws, BUILD64_QPHASE, n, c, cutoff, 0.0, 0, bit_reversed ? 0 : 2, out);
}

qtn_status qtn_build_bessel_mpo(void* ctx, int n, double t, int p_max, int bit_reversed, qtn_mpo* out, void* ws,
                                size_t ws_bytes) {
    if (!ctx || !out || n < 1 || n > 62 || out->n_sites != n || p_max < 0 || !isfinite(t)) return QTN_ERR_ARG;
    if (2 * p_max + 1 > BUILD64_BOND_CAP || 2 * p_max + 1 > out->w_cap) return QTN_ERR_CAPACITY;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    return run_build64(x, w, ws, BUILD64_BESSEL, n, t, 0.0, 0.0, p_max, bit_reversed ? 0 : 2, out);
}

qtn_status qtn_build_pauliz_mpo(void* ctx, int n, double t, double gate_cutoff, int bit_reversed, double cutoff,
                                qtn_mpo* out, void* ws, size_t ws_bytes) {
    if (!ctx || !out || n < 1 || n > 24 || out->n_sites != n || out->w_cap < 1 || !isfinite(t) ||
        !(gate_cutoff >= 0.0) || !(cutoff >= 0.0))
        return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    if ((1ll << n) > w.L.dense) return QTN_ERR_WORKSPACE;   // the 2^n Walsh-Hadamard coefficients
    return run_build64(x, w, ws, BUILD64_PAULIZ, n, t, cutoff, gate_cutoff, 0, bit_reversed ? 0 : 2, out);
}

__global__ void k_copy_cols(const float2* __restrict__ U, int ldu, const int* __restrict__ perm, float2* __restrict__ out,
                            int k_cap, int m, const int* __restrict__ R) {
    const int k = R[R_K];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * k; e += gridDim.x * blockDim.x) {
        const int i = e / k, j = e % k;
        out[(long long)i * k_cap + j] = U[(long long)perm[j] * ldu + i];
    }
}

qtn_status qtn_tsvd(void* ctx, const void* T, int m, int n, qtn_trunc trunc, void* U, void* C, int k_cap, int* k_out,
                    qtn_stats* stats, void* ws, size_t ws_bytes) {
    if (!ctx || !T || !U || !C || !k_out || m < 1 || n < 1 || k_cap < 1 || !trunc_ok(trunc)) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    if (m > w.L.m_cap || (long long)m * n > (long long)w.L.m_cap * w.L.n_cap) return QTN_ERR_WORKSPACE;
    cudaStream_t s = x->c.stream;
    k_reset_stats<<<1, 1, 0, s>>>(w.R, w.ledger);
    CKL();
    k_set_reg<<<1, 1, 0, s>>>(w.R, R_M, m);
    CKL();
    k_set_reg<<<1, 1, 0, s>>>(w.R, R_N, n);
    CKL();
    k_set_reg<<<1, 1, 0, s>>>(w.R, R_P, std::min(m, EIG_MAX));
    CKL();
    qtn_trunc t2 = trunc;
    if (t2.chi_max <= 0) t2.chi_max = INT_MAX;
    // the factorised matrix is copied to T-space so that the projection buffer has its capacity layout
    TsvdIO io{(const float2*)T, dr(R_M), dr(R_N), m, (long long)n, w.Z};
    Dim rows;
    st = tsvd(&x->c, w, io, t2, k_cap, rows);
    if (st) return st;
    const int gld = std::max(w.L.m_cap, w.L.p_cap);
    k_copy_cols<<<grid_for((long long)m * k_cap, 256, x->c.sm_count), 256, 0, s>>>(w.U, gld, ws_perm(w), (float2*)U,
                                                                                   k_cap, m, w.R);
    CKL();
    k_gather_rows<<<grid_for((long long)k_cap * n, 256, x->c.sm_count), 256, 0, s>>>(w.Z, dr(R_N), ws_perm(w),
                                                                                      (float2*)C, dr(R_N), dr(R_N), w.R);
    CKL();
    int hk[2] = {0, 0};
    CK(cudaMemcpyAsync(hk, w.R + R_K, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hk + 1, w.R + R_FLAGS, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *k_out = hk[0];
    if (!stats) return flags_status(hk[1]);
    return fill_stats(&x->c, w, stats);
}

qtn_status qtn_kron_interleave(void* ctx, const qtn_mps* x, const qtn_mps* y, qtn_mps* out) {
    if (!ctx || !x || !y || !out) return QTN_ERR_ARG;
    const int n = x->n_sites;
    if (y->n_sites != n || out->n_sites != n || x->d != 2 || y->d != 2 || out->d != 4) return QTN_ERR_SHAPE;
    if (out->sites == x->sites || out->sites == y->sites) return QTN_ERR_ARG;
    qtn_context* c = (qtn_context*)ctx;
    std::vector<int> hx(n + 1), hy(n + 1);
    CK(cudaMemcpyAsync(hx.data(), x->bond, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, c->c.stream));
    CK(cudaMemcpyAsync(hy.data(), y->bond, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, c->c.stream));
    CK(cudaStreamSynchronize(c->c.stream));
    for (int p = 0; p <= n; ++p)
        if (hx[p] * hy[p] > out->chi_cap) return QTN_ERR_CAPACITY;
    k_kron_interleave<<<n, 256, 0, c->c.stream>>>((const float2*)x->sites, x->bond, x->chi_cap, (const float2*)y->sites,
                                                  y->bond, y->chi_cap, (float2*)out->sites, out->bond, out->chi_cap, n);
    CKL();
    out->canon = QTN_CANON_NONE;
    return QTN_OK;
}

qtn_status qtn_add(void* ctx, const qtn_mps* a, const qtn_mps* b, qtn_mps* out) {
    if (!ctx || !a || !b || !out) return QTN_ERR_ARG;
    const int N = a->n_sites, d = a->d;
    if (b->n_sites != N || out->n_sites != N || b->d != d || out->d != d) return QTN_ERR_SHAPE;
    if (out->sites == a->sites || out->sites == b->sites) return QTN_ERR_ARG;
    qtn_context* c = (qtn_context*)ctx;
    std::vector<int> ha(N + 1), hb(N + 1);
    CK(cudaMemcpyAsync(ha.data(), a->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, c->c.stream));
    CK(cudaMemcpyAsync(hb.data(), b->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, c->c.stream));
    CK(cudaStreamSynchronize(c->c.stream));
    for (int p = 1; p < N; ++p)
        if (ha[p] + hb[p] > out->chi_cap) return QTN_ERR_CAPACITY;
    k_direct_sum<<<N, 256, 0, c->c.stream>>>((const float2*)a->sites, a->bond, a->chi_cap, (const float2*)b->sites,
                                             b->bond, b->chi_cap, (float2*)out->sites, out->bond, out->chi_cap, N, d);
    CKL();
    out->canon = QTN_CANON_NONE;
    return QTN_OK;
}

qtn_status qtn_hadamard(void* ctx, const qtn_mps* a, const qtn_mps* b, int conj_b, qtn_mps* out) {
    if (!ctx || !a || !b || !out) return QTN_ERR_ARG;
    const int N = a->n_sites, d = a->d;
    if (b->n_sites != N || out->n_sites != N || b->d != d || out->d != d) return QTN_ERR_SHAPE;
    if (out->sites == a->sites || out->sites == b->sites) return QTN_ERR_ARG;
    qtn_context* c = (qtn_context*)ctx;
    std::vector<int> ha(N + 1), hb(N + 1);
    CK(cudaMemcpyAsync(ha.data(), a->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, c->c.stream));
    CK(cudaMemcpyAsync(hb.data(), b->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, c->c.stream));
    CK(cudaStreamSynchronize(c->c.stream));
    for (int p = 0; p <= N; ++p)
        if ((long long)ha[p] * hb[p] > out->chi_cap) return QTN_ERR_CAPACITY;
    k_hadamard<<<N, 256, 0, c->c.stream>>>((const float2*)a->sites, a->bond, a->chi_cap, (const float2*)b->sites,
                                           b->bond, b->chi_cap, conj_b ? 1 : 0, (float2*)out->sites, out->bond,
                                           out->chi_cap, N, d);
    CKL();
    out->canon = QTN_CANON_NONE;
    return QTN_OK;
}

qtn_status qtn_hadamard_zipup(void* ctx, const qtn_mps* b, int conj_b, qtn_mps* psi, qtn_trunc trunc,
                              qtn_stats* stats, void* ws, size_t ws_bytes) {
    if (!ctx || !b || !psi || !trunc_ok(trunc)) return QTN_ERR_ARG;
    if (b->d != 4 || psi->d != 4 || b->n_sites != psi->n_sites) return QTN_ERR_SHAPE;
    if (b->sites == psi->sites) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    const int N = b->n_sites;
    std::vector<int> hb(N + 1);
    CK(cudaMemcpyAsync(hb.data(), b->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, x->c.stream));
    CK(cudaStreamSynchronize(x->c.stream));
    int wmax = 1;
    for (int p = 0; p <= N; ++p) wmax = std::max(wmax, hb[p]);
    // the MPS b seen as a diagonal operator: its sites have the stride of an MPO core when d = 4
    qtn_mpo view{N, b->chi_cap, wmax, b->bond, b->sites};
    k_reset_stats<<<1, 1, 0, x->c.stream>>>(w.R, w.ledger);
    CKL();
    st = apply_inner(x, w, &view, conj_b ? 3 : 2, psi, trunc, true);
    if (st) return st;
    return fill_stats(&x->c, w, stats);
}

qtn_status qtn_overlap_grad(void* ctx, const qtn_mps* a, const qtn_mps* b, void* grad, void* ws, size_t ws_bytes) {
    if (!ctx || !a || !b || !grad || a->n_sites != b->n_sites || a->d != b->d) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    cudaStream_t s = x->c.stream;
    const int N = a->n_sites, d = a->d;
    const int gld = std::max(w.L.m_cap, w.L.p_cap);
    // environments, bra index first: EL[p] (sites < p) in G64, ER[p] (sites > p) in S64, stride ea x eb
    const int ea = a->chi_cap, eb = b->chi_cap;
    const size_t env = (size_t)ea * eb;
    if (env * N > (size_t)gld * gld) return QTN_ERR_WORKSPACE;
    std::vector<int> ba(N + 1), bb(N + 1);
    CK(cudaMemcpyAsync(ba.data(), a->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(bb.data(), b->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double2* EL = w.G64;
    double2* ER = w.S64;
    const double2 one = make_double2(1.0, 0.0);
    CK(cudaMemcpyAsync(EL, &one, sizeof(double2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ER + (size_t)(N - 1) * env, &one, sizeof(double2), cudaMemcpyHostToDevice, s));
    const size_t sa = (size_t)ea * d * ea, sb = (size_t)eb * d * eb;
    for (int p = 0; p + 1 < N; ++p) {
        const float2* A = (const float2*)a->sites + p * sa;
        const float2* B = (const float2*)b->sites + p * sb;
        k_transfer_step<<<ba[p + 1], 128, 0, s>>>(EL + p * env, eb, A, ea, ba[p], ba[p + 1], B, eb, bb[p], bb[p + 1],
                                                  d, EL + (p + 1) * env);
        CKL();
    }
    for (int p = N - 1; p > 0; --p) {
        const float2* A = (const float2*)a->sites + p * sa;
        const float2* B = (const float2*)b->sites + p * sb;
        k_transfer_right<<<ba[p], 128, 0, s>>>(ER + p * env, eb, A, ea, ba[p], ba[p + 1], B, eb, bb[p], bb[p + 1], d,
                                               ER + (p - 1) * env, eb);
        CKL();
    }
    CK(cudaMemsetAsync(grad, 0, (size_t)N * sa * sizeof(float2), s));
    for (int p = 0; p < N; ++p) {
        const float2* B = (const float2*)b->sites + p * sb;
        k_env_grad<<<ba[p], 256, 0, s>>>(EL + p * env, eb, ER + p * env, eb, B, eb, bb[p], bb[p + 1], ba[p], ba[p + 1],
                                         d, (float2*)grad + p * sa, ea);
        CKL();
    }
    return QTN_OK;
}

qtn_status qtn_scale(void* ctx, qtn_mps* psi, double re, double im) {
    if (!ctx || !psi || psi->n_sites < 1) return QTN_ERR_ARG;
    qtn_context* c = (qtn_context*)ctx;
    const int N = psi->n_sites, cap = psi->chi_cap, d = psi->d;
    const int q = (psi->canon == QTN_CANON_LEFT) ? N - 1 : 0;
    float2* site = (float2*)psi->sites + (size_t)q * cap * d * cap;
    k_scale_site<<<grid_for((long long)cap * d * cap, 256, c->c.sm_count), 256, 0, c->c.stream>>>(
        site, cap, d, psi->bond, q, (float)re, (float)im);
    CKL();
    return QTN_OK;
}

qtn_status qtn_mpo_dagger(void* ctx, const qtn_mpo* in, qtn_mpo* out) {
    if (!ctx || !in || !out || in->n_sites != out->n_sites || out->w_cap < in->w_max) return QTN_ERR_ARG;
    if (in->sites == out->sites) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    k_mpo_dagger<<<in->n_sites, 128, 0, x->c.stream>>>((const float2*)in->sites, in->bond, in->w_cap,
                                                        (float2*)out->sites, out->bond, out->w_cap, in->n_sites);
    CKL();
    out->w_max = in->w_max;
    return QTN_OK;
}

qtn_status qtn_to_dense(void* ctx, const qtn_mps* psi, qtn_layout layout, void* dense, long long cap_elems, void* ws,
                        size_t ws_bytes) {
    if (!ctx || !psi || !dense) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    const int N = psi->n_sites, d = psi->d, cap = psi->chi_cap;
    const int n = mps_layout_n(psi, layout);
    const long long total = (long long)llround(pow((double)d, (double)N));
    if (total > cap_elems) return QTN_ERR_CAPACITY;
    if (total > w.L.dense) return QTN_ERR_WORKSPACE;
    cudaStream_t s = x->c.stream;
    {   // every intermediate d^p x bond[p] must fit the workspace buffers
        std::vector<int> hb(N + 1);
        CK(cudaMemcpyAsync(hb.data(), psi->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        long long rows_p = 1;
        for (int p = 0; p <= N; ++p) {
            if (hb[p] < 1 || hb[p] > cap) return QTN_ERR_SHAPE;
            if (rows_p * hb[p] > w.L.dense) return QTN_ERR_CAPACITY;
            rows_p *= d;
        }
        if (hb[0] != 1 || hb[N] != 1) return QTN_ERR_SHAPE;
    }
    float2* cur = w.X0;
    float2* nxt = w.X1;
    k_set_one<<<1, 1, 0, s>>>(cur);
    CKL();
    long long rows = 1;
    for (int p = 0; p < N; ++p) {
        k_plan_dense<<<1, 1, 0, s>>>(psi->bond, p, d, w.R);
        CKL();
        GemmDesc g{};
        g.A = mat(cur, dr(R_TMP0), dc(1));
        g.B = mat2((const float2*)psi->sites + (size_t)p * cap * d * cap, dc(d * cap), dr(R_TMP1), dc(cap), dc(1));
        g.C = nxt; g.crs = dr(R_TMP2); g.ccs = dc(1);
        g.M = dc((int)rows); g.N = dr(R_TMP2); g.K = dr(R_TMP0);
        g.mode = OUT_STORE; g.alpha_re = 1.f; g.omega_seed = -1;
        CK(launch_gemm(g, (int)rows, d * cap, cap, w.R, s));
        std::swap(cur, nxt);
        rows *= d;
    }
    k_quantics_to_dense<<<grid_for(total, 256, x->c.sm_count), 256, 0, s>>>(cur, (float2*)dense, n, layout);
    CKL();
    return QTN_OK;
}

qtn_status qtn_norm2(void* ctx, const qtn_mps* psi, double* norm2, void* ws, size_t ws_bytes) {
    if (!ctx || !psi || !norm2) return QTN_ERR_ARG;
    double re_im[2];
    qtn_status st = qtn_overlap(ctx, psi, psi, re_im, ws, ws_bytes);
    *norm2 = re_im[0];
    return st;
}

qtn_status qtn_overlap(void* ctx, const qtn_mps* a, const qtn_mps* b, double* result, void* ws, size_t ws_bytes) {
    if (!ctx || !a || !b || !result || a->n_sites != b->n_sites || a->d != b->d) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    cudaStream_t s = x->c.stream;
    const int N = a->n_sites, d = a->d;
    const int gld = std::max(w.L.m_cap, w.L.p_cap);
    if (a->chi_cap > gld || b->chi_cap > gld) return QTN_ERR_WORKSPACE;
    std::vector<int> ba(N + 1), bb(N + 1);
    CK(cudaMemcpyAsync(ba.data(), a->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(bb.data(), b->bond, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double2 one = make_double2(1.0, 0.0);
    double2* E = w.G64;
    double2* En = w.S64;
    CK(cudaMemcpyAsync(E, &one, sizeof(double2), cudaMemcpyHostToDevice, s));
    for (int p = 0; p < N; ++p) {
        const float2* A = (const float2*)a->sites + (size_t)p * a->chi_cap * d * a->chi_cap;
        const float2* B = (const float2*)b->sites + (size_t)p * b->chi_cap * d * b->chi_cap;
        k_transfer_step<<<ba[p + 1], 128, 0, s>>>(E, gld, A, a->chi_cap, ba[p], ba[p + 1], B, b->chi_cap, bb[p],
                                                  bb[p + 1], d, En);
        CKL();
        std::swap(E, En);
    }
    double2 h;
    CK(cudaMemcpyAsync(&h, E, sizeof(double2), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    result[0] = h.x;
    result[1] = h.y;
    return QTN_OK;
}

qtn_status qtn_amplitudes(void* ctx, const qtn_mps* psi, const int* digits, int count, void* out, void* ws,
                          size_t ws_bytes) {
    if (!ctx || !psi || count < 0) return QTN_ERR_ARG;
    if (count == 0) return QTN_OK;   // nothing to read (the pointers of an empty request may be NULL)
    if (!digits || !out) return QTN_ERR_ARG;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    const int cap = psi->chi_cap;
    const long long per = 2ll * cap;
    const long long room = w.L.dense > 0 ? w.L.dense : 0;
    const int batch = (int)std::max(1LL, std::min<long long>(count, room / per));
    if (room < per) return QTN_ERR_WORKSPACE;
    for (int s0 = 0; s0 < count; s0 += batch) {
        const int cnt = std::min(batch, count - s0);
        const int threads = 256;
        const int blocks = (cnt * 32 + threads - 1) / threads;
        k_amplitudes<<<blocks, threads, 0, x->c.stream>>>((const float2*)psi->sites, psi->bond, psi->n_sites, psi->d,
                                                         cap, digits + (size_t)s0 * psi->n_sites, cnt,
                                                         (float2*)out + s0, w.X0);
        CKL();
    }
    return QTN_OK;
}

// ---------------------------------------------------------------------------- batched steps in CUDA graphs

}  // extern "C"

struct qtn_batch {
    cudaGraphExec_t exec = nullptr;
    cudaStream_t master = nullptr;
    std::vector<cudaStream_t> stream;   // every item's stream (its status word is read on it)
    std::vector<int*> sticky;           // each item's sticky status word (in its workspace)
    std::vector<cudaStream_t> own;      // the streams of branches 1.. (created and destroyed by the batch)
    int branches = 1;
    long long kernels_per_launch = 0;
};

extern "C" {

qtn_status qtn_batch_create(int count, void* const* ctxs, qtn_mps* items, const qtn_mpo* qft, const qtn_mpo* qft_dagger,
                            const qtn_mpo* phase, int n_steps, qtn_trunc trunc, void* const* ws,
                            const size_t* ws_bytes, int branches, void** batch) {
    if (count < 1 || !ctxs || !items || !qft || !qft_dagger || !phase || !ws || !ws_bytes || !batch || n_steps < 1 ||
        !trunc_ok(trunc))
        return QTN_ERR_ARG;
    if (branches <= 0) branches = count;
    branches = std::max(1, std::min(branches, count));
    std::vector<Ws> wss(count);
    for (int i = 0; i < count; ++i) {
        qtn_context* x = (qtn_context*)ctxs[i];
        if (!x || x->c.stream == nullptr) return QTN_ERR_ARG;   // the legacy stream cannot be captured
        qtn_status st = bind_ws(x, ws[i], ws_bytes[i], wss[i]);
        if (st) return st;
        // a graph replays the same passes every launch: the item must enter in the canonical form it leaves in
        // after a whole number of steps (an item with none would replay its canonicalisation sweep each time)
        if (items[i].canon == QTN_CANON_NONE) return QTN_ERR_ARG;
    }
    // branch 0 runs on the first context's stream (the launch stream); the others on streams the batch owns
    std::vector<cudaStream_t> bs(branches, nullptr);
    bs[0] = ((qtn_context*)ctxs[0])->c.stream;
    // longest-processing-time assignment of items to branches by the cost of a step ~ n chi^3 (zip-up of chi-wide
    // bonds over n sites)
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    auto cost = [&](int i) { return (double)items[i].n_sites * std::pow((double)items[i].chi_cap, 3.0); };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<double> load(branches, 0.0);
    std::vector<std::vector<int>> plan(branches);
    for (int i : order) {
        const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        plan[g].push_back(i);
        load[g] += cost(i);
    }
    qtn_batch* b = new qtn_batch;
    b->master = bs[0];
    b->branches = branches;
    for (int g = 1; g < branches; ++g) {
        if (cudaStreamCreateWithFlags(&bs[g], cudaStreamNonBlocking) != cudaSuccess) {
            bs[g] = nullptr;
            qtn_batch_destroy(b);
            return QTN_ERR_CUDA;
        }
        b->own.push_back(bs[g]);
    }
    const long long launches0 = launch_total();
    qtn_status result = QTN_OK;
    std::vector<cudaEvent_t> ev(branches + 1, nullptr);
    for (auto& e : ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) result = QTN_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    if (result == QTN_OK && cudaStreamBeginCapture(b->master, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        result = QTN_ERR_CUDA;
    if (result == QTN_OK) {
        // fork: every branch stream joins the capture after an event of the master stream
        cudaEventRecord(ev[branches], b->master);
        for (int g = 1; g < branches; ++g) cudaStreamWaitEvent(bs[g], ev[branches], 0);
        for (int g = 0; g < branches && result == QTN_OK; ++g) {
            for (int i : plan[g]) {
                qtn_context* x = (qtn_context*)ctxs[i];
                const cudaStream_t own = x->c.stream;
                x->c.stream = bs[g];
                set_gemm_tile(x->c.gemm_tile);
                set_gemm_sms(x->c.sm_count);
                Ws& w = wss[i];
                qtn_mps* psi = items + i;
                const int canon0 = psi->canon;
                const qtn_mpo* ops[3] = {qft + i, phase + i, qft_dagger + i};
                // every item truncates to its own bond capacity (or chi_max, when smaller)
                qtn_trunc ti = trunc;
                ti.chi_max = (trunc.chi_max <= 0) ? psi->chi_cap : std::min(trunc.chi_max, psi->chi_cap);
                k_reset_stats<<<1, 1, 0, bs[g]>>>(w.R, w.ledger);
                count_launch(PROF_OTHER, 0, false);
                qtn_status st = QTN_OK;
                for (int step = 0; step < n_steps && st == QTN_OK; ++step)
                    for (int o = 0; o < 3 && st == QTN_OK; ++o)
                        for (int ax = 0; ax < 2 && st == QTN_OK; ++ax)
                            st = apply_inner(x, w, ops[o], ax, psi, ti, false);
                psi->canon = canon0;   // capturing executed nothing
                x->c.stream = own;
                if (st) { result = st; break; }
            }
        }
        // join
        for (int g = 1; g < branches; ++g) {
            cudaEventRecord(ev[g], bs[g]);
            cudaStreamWaitEvent(b->master, ev[g], 0);
        }
        const cudaError_t ec = cudaStreamEndCapture(b->master, &graph);
        if (result == QTN_OK && (ec != cudaSuccess || !graph)) result = QTN_ERR_CUDA;
    }
    if (result == QTN_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) result = QTN_ERR_CUDA;
    if (graph) cudaGraphDestroy(graph);
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
    if (result != QTN_OK) {
        qtn_batch_destroy(b);
        return result;
    }
    for (int i = 0; i < count; ++i) {
        b->stream.push_back(((qtn_context*)ctxs[i])->c.stream);
        b->sticky.push_back(wss[i].R + R_STICKY);
    }
    b->kernels_per_launch = launch_total() - launches0;
    *batch = b;
    return QTN_OK;
}

qtn_status qtn_batch_launch(void* batch, int repeats) {
    if (!batch || repeats < 0) return QTN_ERR_ARG;
    qtn_batch* b = (qtn_batch*)batch;
    for (int rep = 0; rep < repeats; ++rep) CK(cudaGraphLaunch(b->exec, b->master));
    add_launches(b->kernels_per_launch * repeats);
    return QTN_OK;
}

qtn_status qtn_batch_stream(void* batch, void** stream) {
    if (!batch || !stream) return QTN_ERR_ARG;
    *stream = (void*)((qtn_batch*)batch)->master;
    return QTN_OK;
}

qtn_status qtn_batch_sync(void* batch) {
    if (!batch) return QTN_ERR_ARG;
    qtn_batch* b = (qtn_batch*)batch;
    CK(cudaStreamSynchronize(b->master));
    int worst = 0;
    for (size_t i = 0; i < b->sticky.size(); ++i) {
        int f = 0;
        CK(cudaMemcpyAsync(&f, b->sticky[i], sizeof(int), cudaMemcpyDeviceToHost, b->master));
        CK(cudaMemsetAsync(b->sticky[i], 0, sizeof(int), b->master));
        CK(cudaStreamSynchronize(b->master));
        worst |= f;
    }
    return flags_status(worst);
}

qtn_status qtn_batch_destroy(void* batch) {
    if (!batch) return QTN_OK;
    qtn_batch* b = (qtn_batch*)batch;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaStream_t t : b->own) cudaStreamDestroy(t);
    delete b;
    return QTN_OK;
}

qtn_status qtn_batch_tune_branches(int count, void* const* ctxs, qtn_mps* items, const qtn_mpo* qft,
                                   const qtn_mpo* qft_dagger, const qtn_mpo* phase, qtn_trunc trunc, void* const* ws,
                                   const size_t* ws_bytes, const int* candidates, int n_candidates,
                                   const char* cache_path, int* best_out, double* ms_out) {
    if (count < 1 || !candidates || n_candidates < 1 || !best_out || !ctxs || !items) return QTN_ERR_ARG;
    // workload key: device, item count and the (n, chi) multiset of the items
    qtn_context* x0 = (qtn_context*)ctxs[0];
    if (!x0) return QTN_ERR_ARG;
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, x0->c.device));
    unsigned long long h = 1469598103934665603ull;
    for (int i = 0; i < count; ++i) {
        h = (h ^ (unsigned long long)items[i].n_sites) * 1099511628211ull;
        h = (h ^ (unsigned long long)items[i].chi_cap) * 1099511628211ull;
    }
    char key[512];
    snprintf(key, sizeof(key), "batch_branches|%s|count=%d|items=%016llx|prec=%d", prop.name, count, h, trunc.prec);
    for (char* c = key; *c; ++c)
        if (*c == ' ') *c = '_';
    const char* path = cache_path ? cache_path : getenv("QTN_TUNE_CACHE");
    if (path) {
        if (FILE* f = fopen(path, "r")) {
            char k[512];
            int t = 0;
            double ms = 0.0;
            int found = 0;
            while (fscanf(f, "%511s %d %lf", k, &t, &ms) == 3)
                if (strcmp(k, key) == 0 && t >= 1) { found = 1; *best_out = t; if (ms_out) *ms_out = ms; }
            fclose(f);
            if (found) return QTN_OK;
        }
    }
    // one step per candidate after one step of warm-up (the items are advanced by the trials)
    double best_ms = 1e300;
    int best = candidates[0];
    for (int ci = 0; ci < n_candidates; ++ci) {
        const int br = std::max(1, std::min(candidates[ci], count));
        void* b = nullptr;
        qtn_status st = qtn_batch_create(count, ctxs, items, qft, qft_dagger, phase, 1, trunc, ws, ws_bytes, br, &b);
        if (st) return st;
        qtn_batch* bb = (qtn_batch*)b;
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        float ms = 0.f;
        if ((st = qtn_batch_launch(b, 1)) == QTN_OK) {
            cudaEventRecord(e0, bb->master);
            st = qtn_batch_launch(b, 1);
            cudaEventRecord(e1, bb->master);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        qtn_batch_destroy(b);
        if (st) return st;
        if (ms < best_ms) { best_ms = ms; best = br; }
    }
    *best_out = best;
    if (ms_out) *ms_out = best_ms;
    if (path)
        if (FILE* f = fopen(path, "a")) {
            fprintf(f, "%s %d %.6f\n", key, best, best_ms);
            fclose(f);
        }
    return QTN_OK;
}

qtn_status qtn_set_eig_cluster_min(int r_min) {
    set_eig_cluster_min(r_min);
    return QTN_OK;
}

qtn_status qtn_set_gemm_tile(void* ctx, int tile) {
    if (!ctx || (tile != 64 && tile != 32)) return QTN_ERR_ARG;
    ((qtn_context*)ctx)->c.gemm_tile = tile;
    return QTN_OK;
}

qtn_status qtn_tune_gemm_tile(void* ctx, qtn_mps* item, const qtn_mpo* qft, const qtn_mpo* qft_dagger,
                              const qtn_mpo* phase, qtn_trunc trunc, void* ws, size_t ws_bytes, const char* cache_path,
                              int* tile_out, double* ms_out) {
    if (!ctx || !item || !qft || !qft_dagger || !phase || !tile_out || !trunc_ok(trunc)) return QTN_ERR_ARG;
    if (item->d != 4) return QTN_ERR_SHAPE;
    qtn_context* x = (qtn_context*)ctx;
    Ws w;
    qtn_status st = bind_ws(x, ws, ws_bytes, w);
    if (st) return st;
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, x->c.device));
    char key[512];
    snprintf(key, sizeof(key), "gemm_tile|%s|n=%d|d=%d|chi=%d|w=%d|chi_max=%d|prec=%d", prop.name, item->n_sites,
             item->d, item->chi_cap, std::max(qft->w_max, phase->w_max), trunc.chi_max, trunc.prec);
    for (char* c = key; *c; ++c)
        if (*c == ' ') *c = '_';
    const char* path = cache_path ? cache_path : getenv("QTN_TUNE_CACHE");
    if (path) {   // a cached decision: "<key> <tile> <ms of the chosen tile>"
        if (FILE* f = fopen(path, "r")) {
            char k[512];
            int t = 0;
            double ms = 0.0;
            int found = 0;
            while (fscanf(f, "%511s %d %lf", k, &t, &ms) == 3)
                if (strcmp(k, key) == 0 && (t == 64 || t == 32)) { found = 1; *tile_out = t; if (ms_out) *ms_out = ms; }
            fclose(f);
            if (found) { x->c.gemm_tile = *tile_out; return QTN_OK; }
        }
    }
    // time one Fresnel step of the item per tile (one step of warm-up first); the item is advanced by the trials
    const qtn_mpo* ops[3] = {qft, phase, qft_dagger};
    double best_ms = 1e300;
    int best = 64;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int tile : {64, 32}) {
        x->c.gemm_tile = tile;
        set_gemm_tile(tile);
        float ms = 0.f;
        for (int rep = 0; rep < 3 && st == QTN_OK; ++rep) {
            if (rep == 1) cudaEventRecord(e0, x->c.stream);
            for (int o = 0; o < 3 && st == QTN_OK; ++o)
                for (int ax = 0; ax < 2 && st == QTN_OK; ++ax) st = apply_inner(x, w, ops[o], ax, item, trunc, false);
        }
        cudaEventRecord(e1, x->c.stream);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (st) break;
        if (ms / 2.0 < best_ms) { best_ms = ms / 2.0; best = tile; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    x->c.gemm_tile = best;
    *tile_out = best;
    if (ms_out) *ms_out = best_ms;
    if (path)
        if (FILE* f = fopen(path, "a")) {
            fprintf(f, "%s %d %.6f\n", key, best, best_ms);
            fclose(f);
        }
    return QTN_OK;
}

}  // extern "C"

// ============================================================================ truncated SVD without allocation
//
// qtn_tsvd_noalloc runs the truncated SVD of qtn_tsvd with its scratch in the fixed device array below
// instead of a caller workspace.  Every device that loads the library holds the array until the process
// exits.  The array's name is a host-side stand-in: its device address is looked up once per device, with
// that device current, by cudaGetSymbolAddress and handed to the kernels.
#include <atomic>
#include <mutex>

static __device__ __align__(256) unsigned char g_noalloc_scratch[QTN_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
struct NoallocDevice {
    void* base;
    int sm_count;
};
NoallocDevice g_noalloc_dev[NOALLOC_MAX_DEVICES];
std::atomic<bool> g_noalloc_ready[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mu;

// Only the regions the truncated SVD touches: ledger, registers (+ permutation), the FP64 Gram, the B
// buffer, the eigenbasis, eigenvalues/weights, the sketch Y and its basis Q, and the projected rows X.
// Sized for m <= QTN_NOALLOC_MAX_M, n <= QTN_NOALLOC_MAX_N exactly as the general layout sizes them.
// Computed at compile time: the static_assert below fails the build if the regions outgrow the array.
constexpr size_t ca256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr WsLayout noalloc_layout() {
    WsLayout L{};
    L.n_sites = 1;
    L.d = 1;
    L.chi = QTN_NOALLOC_MAX_M;
    L.w = 1;
    L.m_cap = QTN_NOALLOC_MAX_M;
    L.n_cap = QTN_NOALLOC_MAX_N;
    L.p_cap = EIG_MAX;
    L.dense = 0;
    const size_t c8 = sizeof(float2), c16 = sizeof(double2);
    const size_t mc = (size_t)L.m_cap, nc = (size_t)L.n_cap, pc = (size_t)L.p_cap;
    const size_t gdim = std::max(mc, pc);
    size_t off = 0;
    auto take = [&off](size_t bytes) { size_t o = off; off = ca256(off + bytes); return o; };
    L.ledger = take(L_COUNT * sizeof(double) + 64 * sizeof(int));
    L.regs = take(R_COUNT * sizeof(int) + (2 * gdim + 1024) * sizeof(int));
    L.G64 = take(gdim * gdim * c16);
    L.G32 = take(std::max(gdim * gdim, pc * nc) * c8);
    L.U = take(gdim * gdim * c8);
    L.lam = take(4 * gdim * sizeof(double));
    L.Y = take(gdim * pc * c8);
    L.Q = take(std::max(gdim * pc, pc * pc) * c8);
    L.Z = take(std::max(gdim * nc, pc * pc) * c8);
    L.total = off;
    // regions of the zip-up and of the dense transforms: not used by the truncated SVD (bound to null)
    L.T = L.P = L.carry = L.S64 = L.omega = L.X0 = L.X1 = L.b64 = L.tc = WS_UNUSED;
    L.tc_bytes = 0;
    return L;
}
constexpr WsLayout kNoallocLayout = noalloc_layout();
static_assert(kNoallocLayout.total <= (size_t)QTN_NOALLOC_SCRATCH_BYTES,
              "the truncated-SVD regions do not fit the fixed scratch array");

// One-time set-up of the calling thread's current device: the array's device address and the SM count.
qtn_status noalloc_device(int dev, NoallocDevice* out) {
    if (!g_noalloc_ready[dev].load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ready[dev].load(std::memory_order_relaxed)) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) {
                fprintf(stderr, "qtn_tsvd_noalloc: cudaGetSymbolAddress failed on device %d: %s\n", dev,
                        cudaGetErrorString(e));
                return QTN_ERR_CUDA;
            }
            int sm = 0;
            e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) {
                fprintf(stderr, "qtn_tsvd_noalloc: cudaDeviceGetAttribute failed on device %d: %s\n", dev,
                        cudaGetErrorString(e));
                return QTN_ERR_CUDA;
            }
            e = configure_device_kernels(dev);
            if (e != cudaSuccess) {
                fprintf(stderr, "qtn_tsvd_noalloc: kernel set-up failed on device %d: %s\n", dev,
                        cudaGetErrorString(e));
                return QTN_ERR_CUDA;
            }
            g_noalloc_dev[dev] = NoallocDevice{ptr, sm};
            g_noalloc_ready[dev].store(true, std::memory_order_release);
        }
    }
    *out = g_noalloc_dev[dev];
    return QTN_OK;
}

}  // namespace

extern "C" qtn_status qtn_tsvd_noalloc(const void* T, int m, int n, qtn_trunc trunc, void* U, void* C, int k_cap,
                                       int* k_out, qtn_stats* stats, void* stream) {
    if (!T || !U || !C || !k_out || m < 1 || n < 1 || k_cap < 1 || !trunc_ok(trunc)) return QTN_ERR_ARG;
    if (m > QTN_NOALLOC_MAX_M || n > QTN_NOALLOC_MAX_N) {
        fprintf(stderr, "qtn_tsvd_noalloc: a %d x %d matrix exceeds the fixed scratch (m <= %d, n <= %d)\n", m, n,
                QTN_NOALLOC_MAX_M, QTN_NOALLOC_MAX_N);
        return QTN_ERR_CAPACITY;
    }
    const WsLayout& L = kNoallocLayout;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return QTN_ERR_ARG;
    NoallocDevice nd;
    qtn_status st = noalloc_device(dev, &nd);
    if (st) return st;
    Ctx c{(cudaStream_t)stream, nd.sm_count, dev, 64, {nullptr, nullptr}};
    set_gemm_tile(64);
    set_gemm_sms(nd.sm_count);
    Ws w = ws_bind(nd.base, L);
    cudaStream_t s = c.stream;
    // The array keeps the previous call's contents.  The ledger and the registers are cleared; every other
    // region is written before it is read (the Gram and the power-iteration sum are zeroed inside tsvd).
    CK(cudaMemsetAsync(w.ledger, 0, L.G64 - L.ledger, s));
    k_reset_stats<<<1, 1, 0, s>>>(w.R, w.ledger);
    CKL();
    k_set_reg<<<1, 1, 0, s>>>(w.R, R_M, m);
    CKL();
    k_set_reg<<<1, 1, 0, s>>>(w.R, R_N, n);
    CKL();
    k_set_reg<<<1, 1, 0, s>>>(w.R, R_P, std::min(m, EIG_MAX));
    CKL();
    qtn_trunc t2 = trunc;
    if (t2.chi_max <= 0) t2.chi_max = INT_MAX;
    TsvdIO io{(const float2*)T, dr(R_M), dr(R_N), m, (long long)n, w.Z};
    Dim rows;
    st = tsvd(&c, w, io, t2, k_cap, rows);
    if (st) return st;
    const int gld = std::max(L.m_cap, L.p_cap);
    k_copy_cols<<<grid_for((long long)m * k_cap, 256, c.sm_count), 256, 0, s>>>(w.U, gld, ws_perm(w), (float2*)U,
                                                                               k_cap, m, w.R);
    CKL();
    k_gather_rows<<<grid_for((long long)k_cap * n, 256, c.sm_count), 256, 0, s>>>(w.Z, dr(R_N), ws_perm(w),
                                                                                  (float2*)C, dr(R_N), dr(R_N), w.R);
    CKL();
    int hk[2] = {0, 0};
    CK(cudaMemcpyAsync(hk, w.R + R_K, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hk + 1, w.R + R_FLAGS, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *k_out = hk[0];
    if (!stats) return flags_status(hk[1]);
    return fill_stats(&c, w, stats);
}
