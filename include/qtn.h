/*
 * qtn.h -- C ABI of the quantics tensor-network Fresnel library (CUDA, sm_103a).
 *
 * The library implements the hot path of arXiv:2510.23089 ("Tensor network
 * methods for quantum-inspired image processing and classical optics"):
 * a 2^n x 2^n field is encoded as a quantics MPS by sequential truncated SVD
 * (Sec. III, Sec. IV, App. A) and propagated by the Fresnel transfer function
 * in that compressed form as U_QFT^dagger U(z) U_QFT (Sec. VI.A, Fig.
 * fig_mpo_mpo), each operator applied per axis as an MPO by zip-up
 * contraction with SVD truncation (Sec. V, Fig. fig_mpo).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Plain C types only; every pointer documented "device" must be CUDA device
 *    memory owned by the caller.  The library never allocates or frees device
 *    memory: scratch space is the caller's workspace (see qtn_workspace_size).
 *  - All work is enqueued on the stream given to qtn_create and is
 *    stream-ordered.  No entry point synchronises the stream except when a
 *    non-NULL qtn_stats* is passed, in which case the call waits for its own
 *    work and copies the statistics to that host struct.
 *  - Complex numbers are interleaved single precision (re, im) pairs
 *    ("complex64", 8 bytes), C99 float _Complex / CUDA float2 layout.
 *  - Bond dimensions chosen by truncation live in device int arrays so that a
 *    whole sequence of calls can be captured in a CUDA graph; kernels are sized
 *    by capacities.
 *  - Errors are returned as qtn_status; nothing is truncated silently: a bond
 *    that the truncation rule would make larger than the state's chi_cap is
 *    clamped to chi_cap and reported as QTN_ERR_CAPACITY.  Failures found on
 *    the device (QTN_ERR_NONFINITE, QTN_ERR_CAPACITY, QTN_ERR_NOCONV, in this
 *    order of precedence) are returned by the call itself when it synchronises
 *    (a non-NULL qtn_stats*, or a call documented as synchronising); every
 *    call also ORs them into a sticky status word of its workspace, which
 *    qtn_check (or qtn_batch_sync for graph-replayed batches) reads and clears.
 *  - A new workspace is prepared once by qtn_workspace_init (or zero-filled by
 *    the caller) before its first use.
 */
#ifndef QTN_H
#define QTN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QTN_OK = 0,
    QTN_ERR_ARG = 1,        /* invalid argument (NULL pointer, bad enum, bad size) */
    QTN_ERR_SHAPE = 2,      /* inconsistent shapes between arguments */
    QTN_ERR_CAPACITY = 3,   /* a result does not fit the caller's capacity */
    QTN_ERR_NOCONV = 4,     /* an iterative eigen/SVD solve hit max_sweeps unconverged */
    QTN_ERR_NONFINITE = 5,  /* NaN or Inf met in the input or produced */
    QTN_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up */
    QTN_ERR_CUDA = 7,       /* a CUDA runtime call failed */
    QTN_ERR_BOUNDS = 8,     /* an index was out of range (checked builds) */
    QTN_ERR_WORKSPACE = 9   /* the workspace is NULL or smaller than required */
} qtn_status;

/* Quantics index layouts (Sec. III).  Bits are most-significant first:
 * a = sum_p x_p 2^(n-p).
 *   SERIAL      2n sites of d = 2, (x_1..x_n, y_1..y_n): row-major flattening.
 *   INTERLEAVED n sites of d = 4, site p holds mu_p = (x_p y_p)_2 = 2 x_p + y_p.
 *   ONE_D       n sites of d = 2 for a single axis (a vector of 2^n samples). */
typedef enum { QTN_LAYOUT_SERIAL = 0, QTN_LAYOUT_INTERLEAVED = 1, QTN_LAYOUT_1D = 2 } qtn_layout;

/* Arithmetic of the site contractions.  PLAIN_FP32: FP32 SIMT FMA, FP64-accumulated Grams.
 * MIXED: the site contraction of every zip-up step (carry x site, Sec. V) runs on the tcgen05 tensor cores
 * with BF16 operands split as x = hi + lo (three products per term) and FP32 accumulation in tensor memory;
 * the truncation SVD (FP64-accumulated Gram, FP32 rotations, FP32 re-orthonormalisation) and the FP64
 * bookkeeping are those of the plain path.  A tensor-core wait that gives up returns QTN_ERR_TIMEOUT. */
typedef enum { QTN_PLAIN_FP32 = 0, QTN_MIXED = 1 } qtn_precision;

/* Canonical form of an MPS, tracked on the host by the library. */
typedef enum { QTN_CANON_NONE = 0, QTN_CANON_LEFT = 1, QTN_CANON_RIGHT = 2 } qtn_canon;

/* Matrix product state (Sec. IV, MPS factorisation):
 *   psi[s_1..s_N] = A_1[:, s_1, :] ... A_N[:, s_N, :].
 * Site p (0-based) is stored padded at
 *   sites + p * chi_cap*d*chi_cap, element (l, s, r) at (l*d + s)*chi_cap + r,
 * with l < bond[p], r < bond[p+1]; bond[0] = bond[N] = 1.
 * LEFT canonical: sites 0..N-2 are left isometries, the norm sits in site N-1.
 * RIGHT canonical: sites 1..N-1 are right isometries, the norm sits in site 0. */
typedef struct {
    int n_sites;     /* N >= 1 */
    int d;           /* physical dimension, 2 or 4 */
    int chi_cap;     /* capacity of every bond */
    int canon;       /* qtn_canon; updated by the library */
    int* bond;       /* device int[N+1] */
    void* sites;     /* device complex64 [N][chi_cap][d][chi_cap] */
} qtn_mps;

/* Per-axis matrix product operator on n sites of d = 2 (Sec. V, Fig. fig_mpo):
 *   O[s'_1..s'_n, s_1..s_n] = W_1[:, s'_1, s_1, :] ... W_n[:, s'_n, s_n, :].
 * Core p stored padded at sites + p * w_cap*4*w_cap, element (a, s', s, b) at
 * ((a*2 + s')*2 + s)*w_cap + b.  w_max is the largest bond (host copy). */
typedef struct {
    int n_sites;
    int w_cap;
    int w_max;       /* host-side max over bond[]; set by the builders */
    int* bond;       /* device int[n+1] */
    void* sites;     /* device complex64 [n][w_cap][2][2][w_cap] */
} qtn_mpo;

/* Truncation rule: keep the smallest k >= 1 whose discarded weight
 * sum_{i>=k} s_i^2 is at most cutoff * sum_i s_i^2, capped by chi_max
 * (the paper's relative cutoff, Sec. VI.B.3, read as a relative weight). */
typedef struct {
    int chi_max;      /* <= 0: no cap (the state's chi_cap still bounds every bond, see QTN_ERR_CAPACITY) */
    double cutoff;
    int prec;         /* qtn_precision */
    int max_sweeps;   /* Jacobi sweep limit per eigen-solve (0 = default 30); the rough first solve of
                         each truncation, which the refinement solve corrects, stops after at most 4 */
} qtn_trunc;

/* Statistics of one call (filled only when a non-NULL pointer is passed). */
typedef struct {
    double discarded;   /* sum of discarded squared singular values (FP64) */
    double norm2;       /* squared norm of the result (FP64) */
    int max_bond;       /* largest bond of the result */
    int sweeps_used;    /* largest Jacobi sweep count of any solve */
    int flags;          /* bit 0: some solve did not converge; bit 1: a bond was clamped to capacity;
                           bit 2: non-finite value met */
} qtn_stats;

/* Library context bound to one CUDA stream (cudaStream_t passed as void*;
 * NULL = legacy default stream).  Owns no device memory. */
qtn_status qtn_create(void** ctx, void* cuda_stream);
qtn_status qtn_destroy(void* ctx);
qtn_status qtn_set_stream(void* ctx, void* cuda_stream);
const char* qtn_status_string(qtn_status s);
int qtn_version(void);

/* Clears the state a workspace carries between calls (ledger, dimension
 * registers and the sticky status word); enqueued on the context's stream.
 * Call once on a newly allocated workspace (zero-filling it has the same
 * effect).  ws: device memory of at least qtn_workspace_size bytes. */
qtn_status qtn_workspace_init(void* ctx, void* ws, size_t ws_bytes);

/* Waits for the context's stream and returns the most severe device-side
 * failure (QTN_ERR_NONFINITE > QTN_ERR_CAPACITY > QTN_ERR_NOCONV) that any
 * call on this workspace raised since the previous qtn_check, then clears it.
 * This is how callers that pass no qtn_stats* (asynchronous calls) learn of
 * a clamped bond, a non-finite value or a solve that hit max_sweeps. */
qtn_status qtn_check(void* ctx, void* ws, size_t ws_bytes);

/* Number of kernels the library has launched in this process (all contexts). */
long long qtn_launch_count(void);

/* Opt-in kernel profiling (not needed for computation).  While enabled, the
 * launches of two kernel classes are bracketed by CUDA events on their stream
 * and their algorithmic FLOPs are accumulated on the device in the workspace:
 *   class 0: the complex GEMM kernel (8 M N K FLOPs per product);
 *   class 1: the shared-memory Jacobi eigensolver (8 r FLOPs per evaluated
 *            column pair, 24 r per rotation, 8 r^3 for the re-orthonormalisation).
 * qtn_profile_read synchronises and returns the total device time (ms), the
 * launch count and the FLOP total of one class since qtn_profile(.., 1, ..). */
qtn_status qtn_profile(void* ctx, int enable, void* ws, size_t ws_bytes);
qtn_status qtn_profile_read(void* ctx, int kernel_class, double* ms, long long* launches, double* flops,
                            void* ws, size_t ws_bytes);

/* Bytes of device workspace needed by any call on states of n_sites sites of
 * dimension d with bonds up to chi_max, MPOs with bonds up to w_max, and
 * (for qtn_encode) dense inputs of dense_elems complex entries. */
qtn_status qtn_workspace_size(void* ctx, int n_sites, int d, int chi_max, int w_max,
                              long long dense_elems, size_t* bytes);

/* TT-SVD encoding (Sec. IV, Fig. MPS; App. A): sequential truncated SVD of the
 * quantics tensor of a dense field, left to right.
 *   dense      device complex64; layout SERIAL/INTERLEAVED: L x L row-major
 *              (row = x, column = y), L = 2^n; layout 1D: 2^n entries.
 *   out        caller-allocated MPS with n_sites/d matching the layout and
 *              chi_cap >= trunc.chi_max; overwritten; result LEFT canonical.
 *   stats      optional; discarded = sum of per-bond discarded weights. */
qtn_status qtn_encode(void* ctx, const void* dense, int n, qtn_layout layout, qtn_trunc trunc,
                      qtn_mps* out, qtn_stats* stats, void* ws, size_t ws_bytes);

/* Operator builders.  Each runs once per operator in one CTA in FP64: the
 * operator is held as a d = 4 MPS of (out, in) index pairs, circuit layers are
 * absorbed one at a time by FP64 zip-up passes with SVD compression at the
 * relative cutoff `cutoff` (eigen-decomposition of the FP64 Gram, cyclic
 * Jacobi), and the result is rounded once to complex64.  Bonds of an operator
 * under construction are at most 32 (QTN_ERR_CAPACITY beyond, or beyond
 * out->w_cap).  The workspace must have been sized for at least n sites.
 * Every builder synchronises the stream (it sets out->w_max on the host). */

/* Swap-free quantum Fourier transform MPO (Sec. V: the QFT as a finite-rank MPO):
 * unitary kernel exp(+2 pi i j k / L)/sqrt(L), output site p carries frequency
 * bit k_{n+1-p} (bit-reversed order).  The product of the n circuit layers (H,
 * then controlled phases carried on a bond of 2).  inverse != 0 gives the
 * Hermitian conjugate.  At cutoff 1e-12 the bonds stay below 8. */
qtn_status qtn_build_qft_mpo(void* ctx, int n, int inverse, double cutoff, qtn_mpo* out,
                             void* ws, size_t ws_bytes);

/* Quadratic-phase (Fresnel transfer function) diagonal MPO (Sec. VI.A:
 * T_z(f) = exp(-i pi lambda z f^2)): diagonal entry of frequency k is
 * exp(-i pi c k_f^2 / L) with k_f the signed fftfreq integer and
 * c = lambda z / (L dx^2); indexed in bit-reversed order when bit_reversed != 0
 * (matching the swap-free QFT output).  With k_f = sum_q a_q k_q over the bits
 * of k (two's complement weights), the phase is a product of one- and two-bit
 * diagonal gates; it is built as n controlled-phase layers. */
qtn_status qtn_build_phase_mpo(void* ctx, int n, double c, int bit_reversed, double cutoff,
                               qtn_mpo* out, void* ws, size_t ws_bytes);

/* Lattice-dispersion propagator U(t) = diag(exp(-i t cos(2 pi k / L))) in the
 * closed form of Sec. VI.B.4 (Jacobi-Anger expansion): the sum over
 * |p| <= p_max of (-i)^p J_p(t) exp(2 pi i p k / L), each term a product over
 * the bits of k, so the MPO is diagonal in the bond index p with bond
 * 2 p_max + 1 (<= 31) and boundary vectors (-i)^p J_p(t) and 1.  No
 * compression.  bit_reversed: site q carries bit q of k (as the QFT output);
 * else site q carries bit n-1-q.  The truncation error is at most
 * sum_{|p| > p_max} |J_p(t)| (below 1e-10 for p_max = 14, t = 1). */
qtn_status qtn_build_bessel_mpo(void* ctx, int n, double t, int p_max, int bit_reversed, qtn_mpo* out,
                                void* ws, size_t ws_bytes);

/* The same U(t) as a circuit of commuting Pauli-Z string gates (Sec. VI.B.3,
 * Eq. U-product_1): c_S = 2^-n sum_k cos(2 pi k / L) (-1)^{|S & k|} by a fast
 * Walsh-Hadamard transform on the device, every string with
 * |c_S| >= gate_cutoff becomes the gate exp(-i t c_S P_S) =
 * cos(t c_S) I - i sin(t c_S) P_S (a bond-2 MPO from the first to the last
 * qubit of S), c_0 a global phase; the gates are absorbed into the identity
 * MPO with SVD compression at `cutoff`.  The operator error is at most
 * t * sum_{|c_S| < gate_cutoff} |c_S|.  Needs n <= 24 and a workspace sized
 * with dense_elems >= 2^n (the coefficients live there). */
qtn_status qtn_build_pauliz_mpo(void* ctx, int n, double t, double gate_cutoff, int bit_reversed, double cutoff,
                                qtn_mpo* out, void* ws, size_t ws_bytes);

/* Hermitian conjugate of an MPO: out[a, s', s, b] = conj(in[a, s, s', b]). */
qtn_status qtn_mpo_dagger(void* ctx, const qtn_mpo* in, qtn_mpo* out);

/* Truncated SVD of one matrix, the factorisation every truncation of the
 * method performs (Sec. IV, App. A: a Schmidt decomposition per bond).
 *   T       device complex64, m x n row-major (row stride n); not modified.
 *   U       device complex64 output, m x k_cap row-major (row stride k_cap):
 *           the kept left singular vectors, orthonormal columns.
 *   C       device complex64 output, k_cap x n row-major: C = U^dagger T
 *           (= diag(s) V^dagger), rows in the same order as U's columns.
 *   k_out   host int: the rank kept by the rule of qtn_trunc (k <= k_cap).
 *   stats   optional; discarded = |T|^2 - |C|^2 (FP64).
 * Sizes: m <= d*chi_max and n <= w_max*chi_max of the workspace sizing call.
 * A rank above k_cap asked for by the rule is clamped to k_cap and returns
 * QTN_ERR_CAPACITY (the outputs hold the k_cap leading directions).
 * The call synchronises the stream (it returns k on the host) and returns the
 * device-side status of its own work. */
qtn_status qtn_tsvd(void* ctx, const void* T, int m, int n, qtn_trunc trunc, void* U, void* C, int k_cap,
                    int* k_out, qtn_stats* stats, void* ws, size_t ws_bytes);

/* qtn_tsvd for callers that cannot allocate device memory.  The paper has no
 * counterpart to this call.  Such callers are handed only their input and
 * output buffers: a custom-operator hook inside a host framework that owns
 * the device memory and offers no workspace, or a deployment that budgets
 * device memory once at start-up and forbids cudaMalloc/cudaFree afterwards
 * (cudaFree also synchronises the whole device).
 *   T, U, C, k_out, stats, trunc, m, n, k_cap: as for qtn_tsvd.
 *   stream: the cudaStream_t to run on (NULL = legacy default stream) of the
 *           current device.  No context and no workspace.
 * Scratch: a fixed device array of QTN_NOALLOC_SCRATCH_BYTES inside the
 * library; every GPU that loads the library holds it until the process
 * exits.  The call makes no cudaMalloc, cudaFree or other allocating call.
 * Limits: m <= QTN_NOALLOC_MAX_M and n <= QTN_NOALLOC_MAX_N; larger sizes
 * return QTN_ERR_CAPACITY (and a message on stderr) before any device work.
 * The first call on each device does a one-time set-up with that device
 * current (it looks up the array's device address); make that first call
 * before any stream capture.  All calls share the one array, which keeps the
 * last call's contents: calls whose GPU work overlaps (several streams or
 * host threads at once) race and must be serialised by the caller.
 * The call synchronises the stream (it returns k on the host). */
#define QTN_NOALLOC_MAX_M 256
#define QTN_NOALLOC_MAX_N 2048
#define QTN_NOALLOC_SCRATCH_BYTES (10 << 20)
qtn_status qtn_tsvd_noalloc(const void* T, int m, int n, qtn_trunc trunc, void* U, void* C, int k_cap,
                            int* k_out, qtn_stats* stats, void* stream);

/* Interleaved d = 4 MPS of the separable field f(x) g(y) from the 1-D MPS
 * (d = 2, n sites each) of f and g (Sec. III: site p holds mu_p = 2 x_p + y_p,
 * so each site tensor is the Kronecker product of the two 1-D site tensors and
 * the bonds multiply).  out: n sites, d = 4, chi_cap >= every product bond
 * (QTN_ERR_CAPACITY otherwise); must not alias x or y.  Result canon NONE.
 * The call synchronises (it checks the product bonds on the host). */
qtn_status qtn_kron_interleave(void* ctx, const qtn_mps* x, const qtn_mps* y, qtn_mps* out);

/* MPS of the sum |a> + |b> (block-diagonal bonds; the boundary sites are
 * concatenated).  out: same n_sites and d, chi_cap >= bond_a + bond_b at
 * every inner bond (QTN_ERR_CAPACITY otherwise); must not alias a or b.
 * Result canon NONE; compress with qtn_truncate.  The FP32 compression is
 * accurate when a and b are in the same canonical form (right-canonical, as
 * qtn_truncate leaves them); a left-canonical part turns the unswept
 * environment into a non-isometry that amplifies rounding.  The call
 * synchronises. */
qtn_status qtn_add(void* ctx, const qtn_mps* a, const qtn_mps* b, qtn_mps* out);

/* Batched Fresnel steps over many independent interleaved wavefronts (the
 * data-parallel execution of Sec. VI.A over a batch; the paper treats one field
 * at a time).  Item i has its own context ctxs[i] (its own created stream, not
 * the legacy default stream), workspace ws[i] and operators qft[i],
 * qft_dagger[i], phase[i] (arrays of count; items may differ in n and chi).
 * qtn_batch_create records n_steps steps of every item into ONE CUDA graph
 * without running them: the items are split into `branches` parallel branches
 * (<= 0: one per item), assigned longest-first by the cost n chi^3 of a step
 * to the least loaded branch, each branch running its items one after the
 * other; branch 0 runs on the first context's stream, the others on streams
 * the batch creates (and destroys with it), forked from and joined into the
 * first context's stream (contexts may share a stream).  qtn_batch_launch(batch, k) launches that graph k times on that
 * stream (qtn_batch_stream returns it), so all items advance concurrently in
 * one launch.  Each item truncates to min(trunc.chi_max, its chi_cap) (its
 * chi_cap when chi_max <= 0) and uses its context's GEMM tile
 * (qtn_set_gemm_tile, qtn_tune_gemm_tile).  Items must be in a canonical form (LEFT or RIGHT, as
 * qtn_encode and qtn_truncate leave them): QTN_CANON_NONE returns QTN_ERR_ARG.
 * The items, operators, workspaces and streams must stay allocated and unmoved
 * while the batch exists; profiling must be off; statistics are not collected
 * (use qtn_norm2 / qtn_overlap afterwards, and qtn_batch_sync for the status). */
qtn_status qtn_batch_create(int count, void* const* ctxs, qtn_mps* items, const qtn_mpo* qft,
                            const qtn_mpo* qft_dagger, const qtn_mpo* phase, int n_steps, qtn_trunc trunc,
                            void* const* ws, const size_t* ws_bytes, int branches, void** batch);
qtn_status qtn_batch_launch(void* batch, int repeats);
/* The stream the batch's graph is launched on (cudaStream_t as void*). */
qtn_status qtn_batch_stream(void* batch, void** stream);
/* Waits for the batch and returns the most severe failure any item's replays
 * raised since the last qtn_batch_sync (as qtn_check). */
qtn_status qtn_batch_sync(void* batch);
qtn_status qtn_batch_destroy(void* batch);

/* Autotuner of the batch's launch shape: for each of the n_candidates branch
 * counts, records a one-step batch (qtn_batch_create), launches it once as
 * warm-up and once timed, and returns the fastest count (best_out, and its ms
 * per step in ms_out when non-NULL).  Cached like qtn_tune_gemm_tile, keyed by
 * the device, the item count and the (n, chi) multiset of the items.  The items
 * are advanced by the trial steps (tune on copies).  Synchronises. */
qtn_status qtn_batch_tune_branches(int count, void* const* ctxs, qtn_mps* items, const qtn_mpo* qft,
                                   const qtn_mpo* qft_dagger, const qtn_mpo* phase, qtn_trunc trunc,
                                   void* const* ws, const size_t* ws_bytes, const int* candidates,
                                   int n_candidates, const char* cache_path, int* best_out, double* ms_out);

/* Tile of the generic complex GEMM for the launches of a context: 64 (64 x 64
 * outputs per CTA, the default) or 32 (32 x 32: four times the CTAs on the
 * small contractions of low-chi items).  QTN_ERR_ARG for any other value. */
qtn_status qtn_set_gemm_tile(void* ctx, int tile);

/* Eigen-solver of the truncation SVD (Sec. IV, App. A: the SVD of every truncation is taken through the
 * eigenvectors of the Gram matrix).  For a live order r >= r_min (at most 160) the Jacobi sweeps run over a
 * cluster of 8 CTAs: the rough first solve of a truncation accumulates its rotations into an orthonormal
 * basis, the refinement solve hands its rotated columns to a one-CTA kernel that normalises and
 * orthonormalises them; a smaller problem runs entirely in a single CTA.  Process-wide (all contexts and devices); default 32; values below 2 are taken as 2 and
 * values above 160 send every problem to the single CTA.  Takes effect for launches recorded after the
 * call (graphs already recorded keep their choice). */
qtn_status qtn_set_eig_cluster_min(int r_min);

/* Autotuner of the GEMM tile: times one Fresnel step of `item` (after one step
 * of warm-up) with each tile, keeps the faster for the context and returns it
 * (tile_out, and its ms per step in ms_out when non-NULL).  The decision is
 * cached in a text file, one line "<key> <tile> <ms>" per workload class (device
 * name, n, d, chi capacity, operator bond, chi_max, precision), at cache_path,
 * or at $QTN_TUNE_CACHE when cache_path is NULL (no caching when both are
 * absent); a cached class is not timed again.  The item is advanced by the
 * trial steps (tune on a copy).  Synchronises. */
qtn_status qtn_tune_gemm_tile(void* ctx, qtn_mps* item, const qtn_mpo* qft, const qtn_mpo* qft_dagger,
                              const qtn_mpo* phase, qtn_trunc trunc, void* ws, size_t ws_bytes,
                              const char* cache_path, int* tile_out, double* ms_out);

/* Elementwise (Hadamard) product of two MPS in the same site basis (Sec. V,
 * Eq. psf_eq: the local product of physical legs, O(d chi^3) per site):
 * out[s] = a[s] * b[s] (conj(b[s]) when conj_b != 0); bonds multiply.
 * out: same n_sites and d, chi_cap >= bond_a * bond_b at every bond
 * (QTN_ERR_CAPACITY otherwise); must not alias a or b.  Result canon NONE;
 * compress with qtn_truncate.  The call synchronises (it checks the bonds). */
qtn_status qtn_hadamard(void* ctx, const qtn_mps* a, const qtn_mps* b, int conj_b, qtn_mps* out);

/* psi <- truncate(psi (.) b): the elementwise product with the MPS b (conj(b)
 * when conj_b != 0) applied by zip-up, i.e. b acts as an operator that is
 * diagonal in the site index, with SVD truncation by `trunc` (the product of
 * Sec. V, Eq. psf_eq, without forming the chi_psi * chi_b intermediate).  Both
 * states interleaved (d = 4) with the same n_sites; b must not alias psi; the
 * workspace must allow MPO bonds up to b's largest bond.  psi is brought to a
 * canonical form first when it has none.  The call reads b's bonds on the host. */
qtn_status qtn_hadamard_zipup(void* ctx, const qtn_mps* b, int conj_b, qtn_mps* psi, qtn_trunc trunc,
                              qtn_stats* stats, void* ws, size_t ws_bytes);

/* Derivative of the overlap <a|b> = sum_s conj(a[s]) b[s] with respect to the
 * conjugate of every site tensor of a (left and right transfer-matrix
 * environments, FP64 accumulation): grad[p][k, s, m] = sum over all other
 * site indices of b[s] conj(L_p[k]) conj(R_p[m]), L_p/R_p the products of a's
 * sites left/right of p.  This is the chain rule from a field gradient to the
 * site tensors that parametrise it.  grad: device complex64 with a's site
 * layout [N][chi_cap_a][d][chi_cap_a].  The environments must fit the
 * workspace (N chi_cap_a chi_cap_b <= its Gram capacity). */
qtn_status qtn_overlap_grad(void* ctx, const qtn_mps* a, const qtn_mps* b, void* grad, void* ws, size_t ws_bytes);

/* Reverses the site order in place: site p <-> site N-1-p, left and right
 * bonds exchanged (LEFT and RIGHT canonical forms swap).  For an interleaved
 * state this reverses the bit order of both axes, i.e. it turns the
 * bit-reversed frequency order left by the swap-free QFT into natural order
 * without any factorisation.  Enqueued; no synchronisation. */
qtn_status qtn_reverse_sites(void* ctx, qtn_mps* psi);

/* Point spread function (Sec. V, Eq. psf_eq; Fig. fig_psf_mps):
 *   phi: in: the pupil field E_0 as an interleaved MPS (any canonical form);
 *        out: the normalised focal field |phi> = U_qft^(x) U_qft^(y) |E_0> /
 *        norm, in natural frequency order (sites reversed after the
 *        swap-free QFT) and, when centre != 0, with the zero frequency moved
 *        to the centre (k -> k + L/2 on both axes: the two bits of the most
 *        significant site flipped).
 *   psf: out: ||PSF>> = |phi> (.) |phi>^* (the local product of physical legs),
 *        truncated by trunc; entries |phi|^2 summing to <phi|phi> = 1
 *        (||PSF||_L1 = 1, minus the discarded weight).  psf->chi_cap must hold
 *        phi's bonds (QTN_ERR_CAPACITY otherwise); must not alias phi.
 *   qft: the per-axis QFT MPO (qtn_build_qft_mpo, not inverted).
 * Workspace: MPO bonds up to phi's largest bond.  Synchronises (it reads the
 * bonds of |phi> on the host). */
qtn_status qtn_psf(void* ctx, qtn_mps* phi, const qtn_mpo* qft, int centre, qtn_trunc trunc, qtn_mps* psf,
                   qtn_stats* stats, void* ws, size_t ws_bytes);

/* Image formation by convolution (Sec. V, Eq. convolution_eq):
 *   b <- L * U_iqft(U_qft a (.) U_qft b), the circular convolution a * b of two
 *   interleaved L x L images (L = 2^n; the factor L undoes the normalisation
 *   of the unitary DFT: F(a * b) = sqrt(L) F(a) F(b) per axis).
 *   a is overwritten by U_qft a (both axes, bit-reversed frequency order).
 *   Every pass truncates by trunc.  Synchronises (reads a's bonds). */
qtn_status qtn_convolve(void* ctx, qtn_mps* a, qtn_mps* b, const qtn_mpo* qft, const qtn_mpo* qft_dagger,
                        qtn_trunc trunc, qtn_stats* stats, void* ws, size_t ws_bytes);

/* Angular-spectrum transfer function (Sec. VI.A, Eq. eq_astf) on the L x L
 * frequency grid, written to dense (device complex64, L x L row-major, row =
 * k_x, column = k_y; entries indexed bit-reversed per axis when bit_reversed
 * != 0, matching the swap-free QFT output):
 *   exp(2 pi i (z/lambda) (sqrt(1 - u) - 1)),  u = (lambda f_x)^2 + (lambda f_y)^2,
 *   lambda f = (lambda / dx) k_f / L with k_f the signed fftfreq integer;
 *   evanescent components (u > 1) decay as exp(-2 pi (z/lambda) sqrt(u - 1)).
 * The constant exp(2 pi i z / lambda) is divided out (as exp(i k z) is in the
 * Fresnel step).  It does not factor over the axes: encode it with qtn_encode
 * (INTERLEAVED) into the fused 2-D operator applied by qtn_transfer_step.
 * QTN_ERR_CAPACITY if L^2 > cap_elems.  Enqueued; no synchronisation. */
qtn_status qtn_astf_field(void* ctx, int n, double z_over_lambda, double lambda_over_dx, int bit_reversed,
                          void* dense, long long cap_elems);

/* One propagation step with a 2-D transfer function that need not factor over
 * the axes: psi <- U_qft^dagger (T (.) U_qft psi) with T an interleaved MPS in
 * the bit-reversed frequency order of the swap-free QFT (e.g. the encoded
 * qtn_astf_field), applied as an operator diagonal in the site index by
 * zip-up.  Per pass truncation by trunc.  Synchronises (reads T's bonds). */
qtn_status qtn_transfer_step(void* ctx, qtn_mps* psi, const qtn_mpo* qft, const qtn_mpo* qft_dagger,
                             const qtn_mps* transfer, qtn_trunc trunc, qtn_stats* stats, void* ws, size_t ws_bytes);

/* psi <- (re + i im) psi, applied to the site that carries the norm (the last
 * site of a left-canonical state, the first otherwise); canon unchanged. */
qtn_status qtn_scale(void* ctx, qtn_mps* psi, double re, double im);

/* Building block of the fixed-rank adjoint of zip-up passes (the adjoint is
 * not in the paper; the passes are those of Sec. V, Fig. fig_mpo).  A zip-up
 * pass that applies K to psi writes N-1 isometric sites (the frame V) and a
 * centre c = V^dagger K psi, so with V held fixed it is psi -> V V^dagger K psi
 * and its adjoint is g -> K^dagger V V^dagger g.  This call forms
 *     frame <- V V^dagger W ket
 * as an MPS: the frame's isometric sites are kept and its centre site (site
 * N-1 of a LEFT frame, site 0 of a RIGHT one) is replaced by V^dagger W ket,
 * contracted by three-layer transfer matrices (FP64 accumulation; nothing is
 * truncated or factorised).
 *   W:     per-axis MPO acting on `axis` (0 = x, 1 = y bit of interleaved
 *          sites; d = 2 states: the whole site), or NULL for the identity.
 *          For the backward chain pass W = K^dagger of the forward pass that
 *          follows the frame.
 *   ket:   any MPS with frame's n_sites and d (not aliasing frame).
 *   frame: in: a state left by a zip-up pass (canon LEFT or RIGHT, else
 *          QTN_ERR_ARG); out: its centre replaced.
 * Workspace: environments of frame bond x W bond x ket bond.  Synchronises
 * (it reads the bonds on the host). */
qtn_status qtn_project_apply(void* ctx, const qtn_mpo* W, int axis, const qtn_mps* ket, qtn_mps* frame,
                             void* ws, size_t ws_bytes);

/* Zip-up MPO x MPS application with SVD truncation (Sec. V, Fig. fig_mpo).
 * The per-axis MPO W acts on axis `axis` (0 = x, 1 = y) of psi:
 *   INTERLEAVED: on the x (high) or y (low) bit of every d = 4 site;
 *   SERIAL: on sites [axis*n, axis*n + n); 1D: on all sites (axis ignored).
 * Direction follows psi->canon: LEFT -> right-to-left sweep (result RIGHT
 * canonical), RIGHT -> left-to-right (result LEFT); NONE is first brought to
 * LEFT canonical form without truncation.  psi is updated in place. */
qtn_status qtn_apply_mpo(void* ctx, const qtn_mpo* W, int axis, qtn_mps* psi, qtn_trunc trunc,
                         qtn_stats* stats, void* ws, size_t ws_bytes);

/* Canonical SVD compression (Sec. IV; every truncation acts on a Schmidt
 * decomposition, App. A): left sweep without truncation, then right-to-left
 * truncating sweep.  Result RIGHT canonical; stats.discarded is the exact
 * squared error (Eckart-Young per bond). */
qtn_status qtn_truncate(void* ctx, qtn_mps* psi, qtn_trunc trunc, qtn_stats* stats,
                        void* ws, size_t ws_bytes);

/* n_steps Fresnel steps (Fig. fig_mpo_mpo): per step Q_x, Q_y, D_x, D_y,
 * Qd_x, Qd_y applied in this order by qtn_apply_mpo (alternating sweep
 * directions).  Q = qft, Qd = its dagger, D = phase (all per-axis MPOs on the
 * state's n = bits per axis).  For layout 1D only the x passes run. */
qtn_status qtn_fresnel_step(void* ctx, qtn_mps* psi, qtn_layout layout, const qtn_mpo* qft,
                            const qtn_mpo* qft_dagger, const qtn_mpo* phase, int n_steps,
                            qtn_trunc trunc, qtn_stats* stats, void* ws, size_t ws_bytes);

/* Contract an MPS to its dense field (inverse quantics map of the layout).
 * dense: device complex64 with room for cap_elems entries; the field has
 * d^N entries, written L x L row-major for SERIAL/INTERLEAVED.
 * The contraction runs left to right through intermediates of d^p * bond[p]
 * entries, which must fit the workspace's dense_elems (bonds produced by
 * zip-up may exceed the exact Schmidt rank near the chain ends).
 * QTN_ERR_CAPACITY if d^N > cap_elems or an intermediate does not fit. */
qtn_status qtn_to_dense(void* ctx, const qtn_mps* psi, qtn_layout layout, void* dense,
                        long long cap_elems, void* ws, size_t ws_bytes);

/* Squared norm <psi|psi> in FP64 (transfer matrices; never densifies).
 * norm2: host double, written after the call's stream work completes. */
qtn_status qtn_norm2(void* ctx, const qtn_mps* psi, double* norm2, void* ws, size_t ws_bytes);

/* Overlap <a|b> (complex, FP64 accumulation) by transfer matrices.
 * result: host double[2] (re, im); the call synchronises. */
qtn_status qtn_overlap(void* ctx, const qtn_mps* a, const qtn_mps* b, double* result,
                       void* ws, size_t ws_bytes);

/* Amplitudes psi[s] for `count` site-digit strings (O(N chi^2) each).
 * digits: device int[count][N]; out: device complex64[count]. */
qtn_status qtn_amplitudes(void* ctx, const qtn_mps* psi, const int* digits, int count, void* out,
                          void* ws, size_t ws_bytes);

#ifdef __cplusplus
}
#endif
#endif /* QTN_H */
