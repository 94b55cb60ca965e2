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
// The operands are packed once per GEMM (k_pack_a, k_pack_b: every complex element read once, its six BF16
// entries written straight into 128 x 64 tiles in the canonical no-swizzle K-major layout of the tensor
// cores: 8 x 16-byte core matrices, 128 bytes apart along K and 1024 bytes apart between 8-row groups).  One
// CTA of k_gemm_tc computes a 128 x 128 tile of the real result (64 complex rows x 128 columns) in tensor
// memory: one thread streams the A and B tiles of each 64-wide K chunk into shared memory with cp.async.bulk
// (16 KB each, completion on an mbarrier), four stages deep, and issues four tcgen05.mma (M = 128, N = 128,
// K = 16) per chunk, committed to the stage's mbarrier so the stage is refilled as soon as its MMAs have read
// it.  The four warps then read the accumulator with tcgen05.ld and write complex FP32 results.  Every
// mbarrier wait is bounded; a wait that gives up raises the timeout flag, drains what is in flight (bounded
// again), frees the tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <math.h>

#include "qtn_internal.cuh"

namespace qtn {

constexpr int TC_M = 128, TC_N = 128, TC_KC = 64, TC_THREADS = 128, TC_STAGES = 4;
constexpr int TC_TILE_ELEMS = TC_M * TC_KC;                               // bf16 per operand tile
constexpr uint32_t TC_TILE_BYTES = TC_TILE_ELEMS * 2;                     // 16 KB
constexpr size_t TC_SMEM = 2 * TC_STAGES * (size_t)TC_TILE_BYTES + 1024;   // A and B stages + alignment slack
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
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ float2 tc_get(const Mat& m, int i, int j, long long rs, long long cs, int jdiv,
                                         long long cs_hi) {
    long long off = (long long)i * rs;
    if (jdiv > 0) off += (long long)(j / jdiv) * cs_hi + (long long)(j % jdiv) * cs;
    else off += (long long)j * cs;
    float2 v = m.p[off];
    return m.conj ? make_float2(v.x, -v.y) : v;
}

__device__ __forceinline__ void split2(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// K padded per half-segment to whole 64-wide chunks (a chunk never straddles a half-segment).
__device__ __forceinline__ int tc_kp(int K) { return ((K + TC_KC - 1) / TC_KC) * TC_KC; }

// A'' tiles: rows 2i, 2i+1 of complex row i; chunk c = seg * 2 cps + half * cps + k / 64 with segments
// [hi, hi, lo] and halves [Ar | -Ai] (row 2i), [Ai | Ar] (row 2i+1).  Tile (mt, c) at (mt * nkc + c) tiles.
__global__ void k_pack_a(GemmDesc d, const int* __restrict__ R, __nv_bfloat16* __restrict__ out, int nkc) {
    if (d.guard_reg >= 0 && R[d.guard_reg] != d.guard_val) return;
    const int M = d.M.eval(R), K = d.K.eval(R);
    const int Kp = tc_kp(K), cps = Kp / TC_KC;
    const long long ars = d.A.rs.eval(R), acs = d.A.cs.eval(R), ach = d.A.cs_hi.eval(R);
    const int ajd = d.A.jdiv.eval(R);
    const bool kfast = (acs == 1);
    const long long total = (long long)M * Kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = kfast ? (int)(e / Kp) : (int)(e % M), k = kfast ? (int)(e % Kp) : (int)(e / M);
        float2 a = make_float2(0.f, 0.f);
        if (k < K) a = tc_get(d.A, i, k, ars, acs, ajd, ach);
        const int mt = (2 * i) / TC_M, r = (2 * i) % TC_M, kk = k % TC_KC, kb = k / TC_KC;
        __nv_bfloat16 rh, rl, ih, il, nh, nl;
        split2(a.x, rh, rl);
        split2(a.y, ih, il);
        split2(-a.y, nh, nl);
        for (int seg = 0; seg < 3; ++seg)
            for (int half = 0; half < 2; ++half) {
                const int c = seg * 2 * cps + half * cps + kb;
                __nv_bfloat16* t = out + ((long long)mt * nkc + c) * TC_TILE_ELEMS;
                const bool lo = (seg == 2);
                // half 0: row 2i Re, row 2i+1 Im;  half 1: row 2i -Im, row 2i+1 Re
                t[tc_off(r, kk)] = half ? (lo ? nl : nh) : (lo ? rl : rh);
                t[tc_off(r + 1, kk)] = half ? (lo ? rl : rh) : (lo ? il : ih);
            }
    }
}

// B'' tiles (stored as N rows x K): segments [hi, lo, hi], halves [Re B | Im B].  Tile (nt, c) at (nt * nkc + c).
__global__ void k_pack_b(GemmDesc d, const int* __restrict__ R, __nv_bfloat16* __restrict__ out, int nkc) {
    if (d.guard_reg >= 0 && R[d.guard_reg] != d.guard_val) return;
    const int N = d.N.eval(R), K = d.K.eval(R);
    const int Kp = tc_kp(K), cps = Kp / TC_KC;
    const long long brs = d.B.rs.eval(R), bcs = d.B.cs.eval(R), bch = d.B.cs_hi.eval(R);
    const int bjd = d.B.jdiv.eval(R);
    const bool nfast = (bcs == 1);
    const long long total = (long long)N * Kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = nfast ? (int)(e % N) : (int)(e / Kp), k = nfast ? (int)(e / N) : (int)(e % Kp);
        float2 b = make_float2(0.f, 0.f);
        if (k < K) b = tc_get(d.B, k, j, brs, bcs, bjd, bch);
        const int nt = j / TC_N, r = j % TC_N, kk = k % TC_KC, kb = k / TC_KC;
        __nv_bfloat16 rh, rl, ih, il;
        split2(b.x, rh, rl);
        split2(b.y, ih, il);
        for (int seg = 0; seg < 3; ++seg)
            for (int half = 0; half < 2; ++half) {
                const int c = seg * 2 * cps + half * cps + kb;
                const bool lo = (seg == 1);
                out[((long long)nt * nkc + c) * TC_TILE_ELEMS + tc_off(r, kk)] = half ? (lo ? il : ih) : (lo ? rl : rh);
            }
    }
}

__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(GemmDesc d, int* R, const __nv_bfloat16* __restrict__ Apk,
                                                        const __nv_bfloat16* __restrict__ Bpk, int nkc) {
    if (d.guard_reg >= 0 && R[d.guard_reg] != d.guard_val) return;
    const int M = d.M.eval(R), N = d.N.eval(R), K = d.K.eval(R);
    const int m0 = blockIdx.y * (TC_M / 2), n0 = blockIdx.x * TC_N;   // complex rows / columns of this tile
    if (m0 >= M || n0 >= N) return;
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_s, issued_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = 6 * (tc_kp(K) / TC_KC);   // 3 segments x 2 halves x chunks per half
    const __nv_bfloat16* Ab = Apk + (long long)blockIdx.y * nkc * TC_TILE_ELEMS;
    const __nv_bfloat16* Bb = Bpk + (long long)blockIdx.x * nkc * TC_TILE_ELEMS;
    auto sA = [&](int st) { return smem + (size_t)st * TC_TILE_BYTES; };
    auto sB = [&](int st) { return smem + (size_t)(TC_STAGES + st) * TC_TILE_BYTES; };

    if (tid == 0) {
        for (int st = 0; st < TC_STAGES; ++st) {
            mbar_init(smem_u32(&full[st]), 1);
            mbar_init(smem_u32(&empty[st]), 1);
        }
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

    if (tid == 0) {
        // prologue: fill the stages
        for (int c = 0; c < nch && c < TC_STAGES; ++c) {
            const uint32_t fb = smem_u32(&full[c]);
            mbar_expect_tx(fb, 2 * TC_TILE_BYTES);
            bulk_g2s(smem_u32(sA(c)), Ab + (long long)c * TC_TILE_ELEMS, TC_TILE_BYTES, fb);
            bulk_g2s(smem_u32(sB(c)), Bb + (long long)c * TC_TILE_ELEMS, TC_TILE_BYTES, fb);
        }
        int issued = 0;
        for (int c = 0; c < nch; ++c) {
            const int st = c % TC_STAGES, use = c / TC_STAGES;
            if (!mbar_wait(smem_u32(&full[st]), use & 1)) { abort_s = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA(st)), b0 = smem_u32(sB(st));
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
                             smem_u32(&empty[st]))
                         : "memory");
            issued = c + 1;
            const int cn = c + TC_STAGES;   // refill this stage once its MMAs have read it
            if (cn < nch) {
                if (!mbar_wait(smem_u32(&empty[st]), use & 1)) { abort_s = 1; break; }
                const uint32_t fb = smem_u32(&full[st]);
                mbar_expect_tx(fb, 2 * TC_TILE_BYTES);
                bulk_g2s(smem_u32(sA(st)), Ab + (long long)cn * TC_TILE_ELEMS, TC_TILE_BYTES, fb);
                bulk_g2s(smem_u32(sB(st)), Bb + (long long)cn * TC_TILE_ELEMS, TC_TILE_BYTES, fb);
            }
        }
        // the last commit covers every MMA issued before it
        if (issued > 0) {
            const int cl = issued - 1;
            if (!mbar_wait(smem_u32(&empty[cl % TC_STAGES]), (cl / TC_STAGES) & 1)) abort_s = 1;
        }
        // after a timeout, let the bulk copies already issued land (bounded) before the CTA leaves
        if (abort_s)
            for (int c = issued; c < nch && c < issued + TC_STAGES; ++c)
                mbar_wait(smem_u32(&full[c % TC_STAGES]), (c / TC_STAGES) & 1);
        issued_s = issued;
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

// Bytes of packed operands for a GEMM of capacity max_m x max_n x max_k.
size_t tc_pack_bytes(int max_m, int max_n, int max_k) {
    const size_t nkc = 6 * (size_t)((max_k + TC_KC - 1) / TC_KC);
    const size_t mt = (size_t)(2 * max_m + TC_M - 1) / TC_M, nt = (size_t)(max_n + TC_N - 1) / TC_N;
    return (mt + nt) * nkc * TC_TILE_BYTES;
}

// Complex GEMM (STORE or ACCUM output, FP32) on the tensor cores; same descriptor as launch_gemm.  `pack` holds
// the packed operands (tc_pack_bytes of the capacities, 16-byte aligned).
cudaError_t launch_gemm_tc(const GemmDesc& d, int max_m, int max_n, int max_k, const int* R, void* pack,
                           size_t pack_bytes, int sm_count, cudaStream_t s) {
    if (max_m <= 0 || max_n <= 0 || max_k <= 0) return cudaSuccess;
    if (d.mode == OUT_ATOMIC64 || d.omega_seed >= 0) return cudaErrorInvalidValue;
    if (!pack || pack_bytes < tc_pack_bytes(max_m, max_n, max_k) || ((uintptr_t)pack & 15)) return cudaErrorInvalidValue;
    const int nkc = 6 * ((max_k + TC_KC - 1) / TC_KC);
    const int mt = (2 * max_m + TC_M - 1) / TC_M, nt = (max_n + TC_N - 1) / TC_N;
    __nv_bfloat16* Apk = (__nv_bfloat16*)pack;
    __nv_bfloat16* Bpk = Apk + (size_t)mt * nkc * TC_TILE_ELEMS;
    const int kp = ((max_k + TC_KC - 1) / TC_KC) * TC_KC;
    const long long na = (long long)max_m * kp, nb = (long long)max_n * kp;
    auto blocks = [&](long long n) { return (int)std::max(1LL, std::min((n + 255) / 256, (long long)sm_count * 8)); };
    k_pack_a<<<blocks(na), 256, 0, s>>>(d, R, Apk, nkc);
    count_launch(PROF_OTHER, s, false);
    k_pack_b<<<blocks(nb), 256, 0, s>>>(d, R, Bpk, nkc);
    count_launch(PROF_OTHER, s, false);
    dim3 grid(nt, mt, 1);
    GemmDesc dd = d;
    if (g_prof_ledger) dd.flops = g_prof_ledger + L_PROF_TC;
    count_launch(PROF_TC, s, true);
    k_gemm_tc<<<grid, TC_THREADS, TC_SMEM, s>>>(dd, (int*)R, Apk, Bpk, nkc);
    count_launch(PROF_TC, s, false);
    return cudaGetLastError();
}

}  // namespace qtn
