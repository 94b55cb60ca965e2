// Mixed-precision complex GEMM on the 5th-generation tensor cores (tcgen05, sm_103a): the site contraction of
// the zip-up (carry x site, Sec. V, Fig. fig_mpo; cost O(2 n chi_1^2 chi_2^2)) in BF16 with FP32 accumulation.
//
// Complex to real: C = A B with A = Ar + i Ai, B = Br + i Bi is the real product of the (2M x 2K) matrix whose
// rows 2i and 2i+1 are [Ar_i, -Ai_i] and [Ai_i, Ar_i] with the (2K x N) matrix [Br; Bi]: rows 2i and 2i+1 of
// the result are Re C_i and Im C_i.
//
// Split BF16: x = hi(x) + lo(x), hi = bf16(x), lo = bf16(x - hi); the product keeps hi*hi + hi*lo + lo*hi
// (the lo*lo term is below FP32 rounding), so the K dimension of the real GEMM is 3 x 2K: A segments
// [hi, hi, lo] against B segments [hi, lo, hi].  A plain BF16 product (one segment) misses the 3e-3 budget of
// a Fresnel step; the split keeps the step within FP32 rounding of the plain path.
//
// One CTA computes a 128 x 128 tile of the real result (64 complex rows x 128 columns) in TMEM.  Its four
// warps convert their share of each 64-wide K chunk of A and B from the strided complex operands straight into
// shared memory in the canonical no-swizzle K-major layout (8 x 16-byte core matrices; 128 bytes between core
// matrices along K, 1024 bytes between 8-row groups), fence the writes to the async proxy, and one thread
// issues four tcgen05.mma (M = 128, N = 128, K = 16) per chunk and commits them to an mbarrier.  Two stages:
// the warps convert chunk c + 1 while the tensor cores run chunk c.  Every mbarrier wait is bounded; a wait
// that gives up raises the timeout flag, drains what is in flight (bounded again), frees TMEM and returns.
#include <cuda_bf16.h>
#include <math.h>

#include "qtn_internal.cuh"

namespace qtn {

constexpr int TC_M = 128, TC_N = 128, TC_KC = 64, TC_THREADS = 128;
constexpr int TC_TILE_ELEMS = TC_M * TC_KC;                              // bf16 per operand tile per stage
constexpr size_t TC_SMEM = 2 * 2 * (size_t)TC_TILE_ELEMS * sizeof(__nv_bfloat16) + 1024;   // + alignment slack
constexpr uint32_t TC_WAIT_LIMIT = 1u << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Offset (elements) of (row r < 128, k < 64) in the canonical no-swizzle K-major tile.
__device__ __forceinline__ int tc_off(int r, int k) { return (((r >> 3) * 8 + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           (1ull << 46);
}

// kind::f16 instruction descriptor: D F32, A and B BF16, both K-major, N = 128, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
    for (uint32_t i = 0; i < TC_WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ float2 tc_get(const Mat& m, int i, int j, long long rs, long long cs, int jdiv,
                                         long long cs_hi) {
    long long off = (long long)i * rs;
    if (jdiv > 0) off += (long long)(j / jdiv) * cs_hi + (long long)(j % jdiv) * cs;
    else off += (long long)j * cs;
    float2 v = m.p[off];
    return m.conj ? make_float2(v.x, -v.y) : v;
}

__device__ __forceinline__ __nv_bfloat16 split_part(float v, int lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    return lo ? __float2bfloat16_rn(v - __bfloat162float(h)) : h;
}

__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(GemmDesc d, int* R) {
    if (d.guard_reg >= 0 && R[d.guard_reg] != d.guard_val) return;
    const int M = d.M.eval(R), N = d.N.eval(R), K = d.K.eval(R);
    const int m0 = blockIdx.y * (TC_M / 2), n0 = blockIdx.x * TC_N;   // complex rows / columns of this tile
    if (m0 >= M || n0 >= N) return;
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __nv_bfloat16* smem = (__nv_bfloat16*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    __nv_bfloat16* sA[2] = {smem, smem + TC_TILE_ELEMS};
    __nv_bfloat16* sB[2] = {smem + 2 * TC_TILE_ELEMS, smem + 3 * TC_TILE_ELEMS};
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_s, issued_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long ars = d.A.rs.eval(R), acs = d.A.cs.eval(R), brs = d.B.rs.eval(R), bcs = d.B.cs.eval(R);
    const int ajd = d.A.jdiv.eval(R), bjd = d.B.jdiv.eval(R);
    const long long ach = d.A.cs_hi.eval(R), bch = d.B.cs_hi.eval(R);
    const bool a_kfast = (acs == 1), b_nfast = (bcs == 1);
    const int Kp = ((K + TC_KC - 1) / TC_KC) * TC_KC;   // K padded per half-segment: a chunk never straddles one
    const int cps = Kp / TC_KC;                          // chunks per half-segment
    const int nch = 6 * cps;                             // 3 segments x 2 halves

    if (tid == 0) {
        mbar_init(smem_u32(&bar[0]), 1);
        mbar_init(smem_u32(&bar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
        issued_s = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    for (int c = 0; c < nch; ++c) {
        const int s = c & 1;
        if (c >= 2) {   // stage s still feeds the MMAs of chunk c - 2
            if (tid == 0 && !mbar_wait(smem_u32(&bar[s]), ((c - 2) >> 1) & 1)) abort_s = 1;
            __syncthreads();
            if (abort_s) break;
        }
        const int seg = c / (2 * cps), half = (c / cps) & 1, kb = (c % cps) * TC_KC;
        const int lo_a = (seg == 2), lo_b = (seg == 1);
        // A'' rows 2i, 2i+1 of the 64 complex rows of this tile, k in [kb, kb + 64); consecutive threads walk the
        // contiguous index of A
        for (int e = tid; e < (TC_M / 2) * TC_KC; e += TC_THREADS) {
            const int ir = a_kfast ? e / TC_KC : e % (TC_M / 2), kk = a_kfast ? e % TC_KC : e / (TC_M / 2);
            const int i = m0 + ir, k = kb + kk;
            float2 a = make_float2(0.f, 0.f);
            if (i < M && k < K) a = tc_get(d.A, i, k, ars, acs, ajd, ach);
            // half 0: [Ar | Ai] on (re, im) rows; half 1: [-Ai | Ar]
            const float vr = half ? -a.y : a.x, vi = half ? a.x : a.y;
            sA[s][tc_off(2 * ir, kk)] = split_part(vr, lo_a);
            sA[s][tc_off(2 * ir + 1, kk)] = split_part(vi, lo_a);
        }
        // B'' (stored as N rows x K): half 0 Re B, half 1 Im B
        for (int e = tid; e < TC_N * TC_KC; e += TC_THREADS) {
            const int jr = b_nfast ? e % TC_N : e / TC_KC, kk = b_nfast ? e / TC_N : e % TC_KC;
            const int j = n0 + jr, k = kb + kk;
            float v = 0.f;
            if (j < N && k < K) {
                const float2 b = tc_get(d.B, k, j, brs, bcs, bjd, bch);
                v = half ? b.y : b.x;
            }
            sB[s][tc_off(jr, kk)] = split_part(v, lo_b);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA[s]), b0 = smem_u32(sB[s]);
#pragma unroll
            for (int kk = 0; kk < TC_KC / 16; ++kk) {
                const uint64_t ad = tc_desc(a0 + 256 * kk), bd = tc_desc(b0 + 256 * kk);
                const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar[s]))
                         : "memory");
            issued_s = c + 1;   // read by the other threads only after the next barrier
        }
    }
    // wait for the last commit (it covers every MMA issued before it); after a timeout, wait (bounded) for what
    // was issued so the tensor memory is no longer written when it is freed
    if (tid == 0 && issued_s > 0) {
        const int cl = issued_s - 1;
        if (!mbar_wait(smem_u32(&bar[cl & 1]), (cl >> 1) & 1)) abort_s = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok = !abort_s && issued_s == nch && nch > 0;
    if (!ok && tid == 0) raise_flag(R, F_TIMEOUT);
    if (ok) {
        // epilogue: warp w holds real rows 32w .. 32w + 31 (TMEM lanes); even lanes real, odd lanes imaginary
        const long long crs = d.crs.eval(R), ccs = d.ccs.eval(R);
        const float2 alpha = make_float2(d.alpha_re, d.alpha_im);
        const int i = m0 + (warp * 32 + lane) / 2;
        for (int c0 = 0; c0 < TC_N; c0 += 32) {
            uint32_t v[32];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const float mine = __uint_as_float(v[q]);
                const float other = __shfl_xor_sync(0xffffffffu, mine, 1);
                const int j = n0 + c0 + q;
                if ((lane & 1) == 0 && i < M && j < N) {
                    const float2 z = cmul(alpha, make_float2(mine, other));
                    float2* cp = (float2*)d.C + (long long)i * crs + (long long)j * ccs;
                    if (d.mode == OUT_ACCUM) *cp = cadd(*cp, z);
                    else *cp = z;
                }
            }
        }
        if (d.flops != nullptr && tid == 0) atomicAdd(d.flops, 8.0 * (double)min(TC_M / 2, M - m0) *
                                                                   (double)min(TC_N, N - n0) * (double)K);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N) : "memory");
}

cudaError_t configure_tc_kernel() {
    return cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
}

// Complex GEMM (STORE or ACCUM output, FP32) on the tensor cores; same descriptor as launch_gemm.
cudaError_t launch_gemm_tc(const GemmDesc& d, int max_m, int max_n, int max_k, const int* R, cudaStream_t s) {
    (void)max_k;
    if (max_m <= 0 || max_n <= 0) return cudaSuccess;
    if (d.mode == OUT_ATOMIC64 || d.omega_seed >= 0) return cudaErrorInvalidValue;
    dim3 grid((max_n + TC_N - 1) / TC_N, (max_m + TC_M / 2 - 1) / (TC_M / 2), 1);
    GemmDesc dd = d;
    if (g_prof_ledger) dd.flops = g_prof_ledger + L_PROF_TC;
    count_launch(PROF_TC, s, true);
    k_gemm_tc<<<grid, TC_THREADS, TC_SMEM, s>>>(dd, (int*)R);
    count_launch(PROF_TC, s, false);
    return cudaGetLastError();
}

}  // namespace qtn
