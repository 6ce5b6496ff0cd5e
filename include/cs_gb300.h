/*
 * cs_gb300.h -- C ABI of the GB300 (sm_103a) greedy compressive-sensing decoders.
 *
 * The library recovers a K-sparse s from y = A s (+ noise) with the greedy decoders OMP, SP
 * (Subspace Pursuit) and OMPR (OMP with Replacement), each using the paper's CG-based weighted
 * least-squares step (Hsieh, Lu & Pei, "Fast Greedy Approaches for Compressive Sensing of
 * Large-Scale Signals", arXiv:1509.03979).
 *
 * Operator (Sec. III-A, Eq. 7):  A = P_Omega . C_N . diag(d)  in R^{M x N}
 *   d      Rademacher signs (the randomiser), regenerated from the seed (SplitMix64 hash)
 *   C_N    orthonormal DCT-II, C_N[k,n] = w_k cos(pi (2n+1) k / (2N)), w_0 = sqrt(1/N),
 *          w_k = sqrt(2/N); no sqrt(N/M) rescaling, so A A^T = I_M
 *   Omega  M distinct rows, partial Fisher-Yates from a SplitMix64 stream, sorted ascending
 * Random-draw definitions (both must match exactly for the oracle cross-check):
 *   gamma = 0x9E3779B97F4A7C15, mix = SplitMix64 finaliser, h(x) = mix(x + gamma)
 *   d_n = -1 iff the top bit of h((seed ^ 0xD1B54A32D192ED03) + n) is set
 *   Omega: for i = 0..M-1: j = i + (mix((seed ^ gamma) + (i+1) gamma) mod (N-i)); swap
 *
 * Conventions for every entry point below:
 *   - Array arguments are caller-owned DEVICE pointers (e.g. torch tensor data_ptr()),
 *     FP32 values and int32 indices, contiguous, unless a comment says "host".
 *   - Calls are asynchronous on the operator's stream (cs_op_set_stream); they return after
 *     the launch.  Argument errors are returned synchronously and nothing is launched.
 *   - N must be a power of two with 16 <= N <= 2^24, or any N with 16 <= N <= 4096 (else
 *     CS_ERR_UNSUPPORTED_N);
 *     1 <= M <= N; 0 <= K <= M; for SP also 2K <= M, for CoSaMP 3K <= M (else
 *     CS_ERR_INVALID_ARG).
 *     An N that is not a power of two runs on the any-N path: one CTA per signal holds it in
 *     natural order and computes the DCT-II / DCT-III as chirp-z transforms (Bluestein) over
 *     power-of-two FFTs of at least 2N - 1 points; the sign randomiser only.
 *     A power of two N <= 2^18 runs on one thread-block cluster per signal; 2^18 < N <= 2^24 runs on a
 *     cooperative grid of up to 128 CTAs per signal that streams the transform through L2
 *     (such signals are processed one after another, also inside the batched calls).
 *     A grid-wide wait that does not finish within its iteration limit ends the launch early:
 *     recoveries report CS_ERR_TIMEOUT in cs_stats.status, every call through cs_op_sync.
 *   - cg_tol is RELATIVE by default: CG stops when ||r_j|| <= cg_tol * ||W A^T y|| (or after
 *     cg_maxit steps; reaching cg_maxit is not an error, it is counted in
 *     cs_stats.cg_maxit_hits).  cs_op_set_cg_tol_mode(op, CS_CG_TOL_ABSOLUTE) makes it the
 *     paper's absolute xi on ||r_j|| (Algorithm 1), floored at the FP32 limit: an absolute
 *     solve also stops once ||r_j|| <= 1e-6 ||W A^T y||, so xi = 0 (the paper's exact
 *     precision, Sec. IV-C) or xi = 1e-10 yields the LS solution to FP32 precision.
 *     cg_maxit = 0 means at most |S| steps, the bound of Theorem 5.  A step whose H d
 *     vanishes in FP32 ends the solve (the residual is at rounding level).
 *   - Per-call scratch is stream-ordered (cudaMallocAsync / cudaFreeAsync on the call's
 *     stream).  The first operator creation or selection call on a device raises the release
 *     threshold of that device's default memory pool to its maximum, so freed scratch stays
 *     pooled for the next call instead of returning to the CUDA driver at every synchronisation
 *     (a setting of this process; it also applies to the host program's own cudaMallocAsync).
 *   - cs_last_error() returns a thread-local message describing the last failure.
 *   - Operators are not thread-safe: one host thread at a time per cs_op_t.
 *   - CUDA graphs: cs_op_apply(_t)(_batched), cs_recover, cs_recover_batched (stats_host
 *     NULL), cs_ls_* and cs_recover_noalloc may be captured into a graph on the op's stream
 *     once the same call has run uncaptured (first calls set kernel attributes and look up
 *     device addresses); every launch carries its tables in its own parameters, so a replay
 *     needs no host memory of the capturing call.  The concurrent launches of
 *     cs_recover_batched (one per cluster size) run on streams that ops[0] keeps for the
 *     purpose, so under capture they become parallel branches of the graph.  The autotuners,
 *     cs_get_stats, cs_op_sync and a non-NULL stats_host wait on the host and cannot be
 *     captured.
 */
#ifndef CS_GB300_H
#define CS_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cs_op* cs_op_t;

typedef enum { CS_OMP = 0, CS_SP = 1, CS_OMPR = 2, CS_COSAMP = 3 } cs_algo;

typedef enum {
  CS_OK = 0,
  CS_ERR_INVALID_ARG = 1,
  CS_ERR_UNSUPPORTED_N = 2,
  CS_ERR_OOM = 3,
  CS_ERR_CUDA = 4,
  CS_ERR_TIMEOUT = 5
} cs_status;

/* Per-recovery statistics (written on the device, read back by cs_get_stats). */
typedef struct {
  int32_t outer_iters;     /* greedy iterations (OMP: K; SP/OMPR: rounds run) */
  int32_t cg_iters_total;  /* CG steps over all LS solves (each = one H d product) */
  int32_t cg_maxit_hits;   /* LS solves that stopped on cg_maxit */
  int32_t near_ties;       /* recoveries: selections and stop tests whose margin is <= 1e-3
                              (see cs_op_set_trace for the margins); LS calls: 0 */
  float final_resid;       /* ||y - A s_hat||_2 of the returned solution */
  float min_margin;        /* recoveries: the smallest margin (1 if none); LS calls: -1 */
  int32_t status;          /* cs_status of the device-side run */
  int32_t transforms;      /* N-point DCT-II / DCT-III applications executed */
} cs_stats;

/* Create the operator A = P_Omega C_N diag(d) for (N, M, seed) (Sec. III-A, Eq. 7).
 * Builds Omega on the host, uploads its bitmask/rank tables and the twiddle tables.
 * Returns NULL on failure (see cs_last_error()).  Owns all its device memory. */
cs_op_t cs_op_create(int64_t N, int64_t M, uint64_t seed);

/* The operator with a chosen randomiser R of the SRM (Sec. III-A): CS_RANDOMIZER_SIGNS is
 * diag(d) as in cs_op_create; CS_RANDOMIZER_PERMUTATION is the paper's uniform random
 * permutation, A = P_Omega C_N Pi with (Pi x)_n = x_{perm[n]} and no sign flips, perm drawn by a
 * full Fisher-Yates shuffle: for i = 0 .. N-2, j = i + (mix((seed ^ 0xA0761D6478BD642F) +
 * (i+1) gamma) mod (N-i)), swap.  Every entry point works with both; the streamed batched
 * operator is not used for permutation operators (their x gather is not contiguous).
 * Returns NULL on failure. */
enum { CS_RANDOMIZER_SIGNS = 0, CS_RANDOMIZER_PERMUTATION = 1 };
cs_op_t cs_op_create_ex(int64_t N, int64_t M, uint64_t seed, int32_t randomizer);

/* The operator with a sparsifying basis Psi (Sec. III-A: y = Phi Psi s, the signal sparse in
 * the basis; the image experiment of Sec. IV-A takes a DCT basis): A = P_Omega C_N diag(d) Psi,
 * the unknown s holds the basis coefficients of x = Psi s, and every entry point recovers,
 * solves and differentiates in s.  CS_BASIS_IDENTITY is cs_op_create's operator;
 * CS_BASIS_DCT is Psi = C_N^T (s = the orthonormal DCT-II coefficients of x); CS_BASIS_DCT2D is
 * the separable 2-D basis Psi_2 (x) Psi_1 of an n1 x n2 image stored row-major (x = C_{n1}^T S
 * C_{n2} for the n1 x n2 coefficient array S; n1 >= 2 divides N, n2 = N / n1 >= 2; n1 is
 * ignored for the other bases).  A basis needs 16 <= N <= 4096 (else CS_ERR_UNSUPPORTED_N) and
 * takes the sign randomiser d.  Psi is orthonormal, so A A^T = I_M still holds.  Such operators
 * run on the any-N path (one CTA, chirp-z DCTs), whatever N is.  Returns NULL on failure. */
enum { CS_BASIS_IDENTITY = 0, CS_BASIS_DCT = 1, CS_BASIS_DCT2D = 2 };
cs_op_t cs_op_create_basis(int64_t N, int64_t M, uint64_t seed, int32_t basis, int32_t n1);

/* Host-only draw of the permutation randomiser for (N, seed) into perm_N_host [N] HOST. */
cs_status cs_operator_perm(int64_t N, uint64_t seed, int32_t* perm_N_host);

/* Copy a permutation operator's perm to perm_N_host [N] HOST (CS_ERR_INVALID_ARG otherwise). */
cs_status cs_op_export_perm(cs_op_t op, int32_t* perm_N_host);

/* Free the operator and every buffer it owns.  Waits for its stream first. */
void cs_op_destroy(cs_op_t op);

/* Launch all further work of `op` on `cuda_stream` (a cudaStream_t; NULL = legacy default). */
cs_status cs_op_set_stream(cs_op_t op, void* cuda_stream);

/* y_M = A x_N: randomiser (sign flip or permutation), orthonormal DCT-II, keep rows Omega
 * (Sec. III-D operator list).
 * x_N: [N] device, y_M: [M] device (written).  Buffers must not overlap. */
cs_status cs_op_apply(cs_op_t op, const float* x_N, float* y_M);

/* x_N = A^T y_M: scatter onto Omega, orthonormal DCT-III, randomiser transposed (the
 * correlation A^T r of Eq. 6).  y_M: [M] device; x_N: [N] device (written).  Buffers must not overlap. */
cs_status cs_op_apply_t(cs_op_t op, const float* y_M, float* x_N);

/* Batched A / A^T: B independent vectors through the same operator, one persistent launch.
 * X [B][N] and Y [B][M] device, row-major contiguous; U [B][M] -> X [B][N] for the transpose.
 * Two implementations compute the same operator (results agree to rounding, not bitwise):
 *   CS_BATCHED_CLUSTER   one thread-block cluster per vector, the transform resident in the
 *                        cluster's shared memory (the engine the decoders use);
 *   CS_BATCHED_STREAMED  a small cluster of CTAs per vector for 2^15 <= N <= 2^18: a
 *                        decimation-in-frequency split into 8192-point rows, a column pass
 *                        and a row pass through a per-cluster buffer in L2, x read and written
 *                        in coalesced 16-byte groups.  Uses 1.1 MiB (N = 2^18) of stream-
 *                        ordered temporary device memory per resident cluster, allocated and
 *                        freed on the op's stream per call.
 * CS_BATCHED_AUTO (the default) takes the choice of cs_op_tune_batched when it has run, else
 * the streamed kernel (4 CTAs per vector, at most N/2^15) whenever N allows it and B >= 2. */
cs_status cs_op_apply_batched(cs_op_t op, int32_t B, const float* X, float* Y);
cs_status cs_op_apply_t_batched(cs_op_t op, int32_t B, const float* U, float* X);

/* Cluster size P (CTAs per signal) of this op's cluster engine, N <= 2^18 (no counterpart in
 * the paper).  Default 0 = the smallest that holds the transform on chip (P = max(1, N/2^14)),
 * which fits the most signals on the GPU at once; a larger P (power of two <= 16, N >= 4 P^2)
 * spreads one signal over more SMs and lowers its latency.  Waits for the op's stream and
 * reallocates the op's scratch.  CS_ERR_UNSUPPORTED_N for N > 2^18 (one geometry). */
cs_status cs_op_set_cluster_size(cs_op_t op, int32_t P);
int32_t cs_op_cluster_size(cs_op_t op);   /* current P (0 for a NULL op) */

/* Autotuner of the single-signal recovery: times cs_recover(K, algo, cg_tol, cg_maxit) of an
 * internal K-sparse test signal for every cluster size P in {1, 2, 4, 8, 16} that is valid
 * for this op, keeps the fastest (cs_op_set_cluster_size), and writes the milliseconds per
 * recovery to ms_out (HOST [5] or NULL; -1 where P does not apply).  Allocates and frees
 * 2N + M + K words of device memory, synchronises the op's stream.  No-op for N > 2^18. */
cs_status cs_op_tune_recover(cs_op_t op, int32_t K, int32_t algo, float cg_tol, int32_t cg_maxit,
                             float* ms_out);

/* OMPR replacements per round l for this op's later CS_OMPR recoveries (default 1: one swap
 * z_j <-> z_i per round, |z_j| > |z_i|).  l > 1 is OMPR(l) (Jain, Tewari & Dhillon 2011, the
 * generalisation of the OMPR the paper cites): J = the l largest |z| outside S, S' = the K
 * largest |z| over S u J (ties to the lowest index), stop when S' = S; the swap cap of
 * cs_recover counts rounds.  l is clamped to N - K. */
cs_status cs_op_set_ompr_replacements(cs_op_t op, int32_t l);

/* Cap on the outer iterations of this op's later recoveries (no counterpart in the paper, which
 * leaves SP's and OMPR's iteration limits open): SP and CoSaMP rounds, OMPR swaps (single-swap)
 * or rounds (OMPR(l)).  0 (the default) means 50 SP / CoSaMP rounds and 100 OMPR swaps or
 * rounds.  A recovery that reaches the cap returns its current state; cs_stats.outer_iters
 * equals the cap then. */
cs_status cs_op_set_outer_cap(cs_op_t op, int32_t cap);

enum { CS_CG_TOL_RELATIVE = 0, CS_CG_TOL_ABSOLUTE = 1 };
/* Stopping rule of every CG solve of this op's later recover / LS calls (see the conventions
 * above): CS_CG_TOL_RELATIVE (default) or CS_CG_TOL_ABSOLUTE (Algorithm 1's ||r_j|| <= xi). */
cs_status cs_op_set_cg_tol_mode(cs_op_t op, int32_t mode);

enum { CS_BATCHED_AUTO = 0, CS_BATCHED_CLUSTER = 1, CS_BATCHED_STREAMED = 2 };
/* Choose the implementation of cs_op_apply_batched / cs_op_apply_t_batched for this op.
 * CS_ERR_UNSUPPORTED_N if CS_BATCHED_STREAMED is asked for outside 2^15 <= N <= 2^18. */
cs_status cs_op_set_batched_impl(cs_op_t op, int32_t impl);

/* Autotuner of the batched operator (no counterpart in the paper): times every candidate that
 * can run this op -- the cluster engine, and the streamed kernel with 1, 2, 4 or 8 CTAs per
 * vector (at most P/2 = N/2^15) -- on B internally generated vectors, for A and A^T
 * separately, and keeps the fastest for later batched calls under CS_BATCHED_AUTO (under
 * CS_BATCHED_STREAMED the tuned CTAs per vector are kept when the winner is streamed).
 * ms_out: HOST [2][5] or NULL, milliseconds per call in the order {cluster engine, 1, 2, 4, 8}
 * for A then A^T, -1 where a candidate does not apply.  Allocates and frees B (N + M) floats
 * of device memory, runs on the op's stream and returns after synchronising it. */
cs_status cs_op_tune_batched(cs_op_t op, int32_t B, float* ms_out);

/* Number of signals of this operator's size that the device runs at the same time (one per
 * resident thread-block cluster); a batch of this many fills the GPU.  >= 1. */
int32_t cs_op_concurrency(cs_op_t op);

/* Copy the operator's random draws to HOST memory for cross-checking: omega_M_host [M]
 * (sorted row indices) and d_N_host [N] (+1/-1; all +1 for a permutation operator).  Either
 * pointer may be NULL. */
cs_status cs_op_export(cs_op_t op, int32_t* omega_M_host, int8_t* d_N_host);

/* Host-only: the same random draws cs_op_create(N, M, seed) uses, without touching a GPU.
 * omega_M_host [M] HOST (sorted), d_N_host [N] HOST (+1/-1); either may be NULL.
 * Returns CS_ERR_UNSUPPORTED_N / CS_ERR_INVALID_ARG under the same rules as cs_op_create. */
cs_status cs_operator_draws(int64_t N, int64_t M, uint64_t seed, int32_t* omega_M_host, int8_t* d_N_host);

/* Greedy recovery (Sec. II steps 1-4; Algorithm 1 for OMP; SP and OMPR as cited in
 * Sec. IV) with the CG weighted LS step (Eq. 8-10, the CG function of Algorithm 1).
 *   y           [M] device measurements
 *   K           sparsity (number of support entries returned)
 *   algo        CS_OMP, CS_SP, CS_OMPR, or CS_COSAMP (CoSaMP, Needell & Tropp 2009, which the paper
 *               does not treat: T = S u {2K largest |A^T r|}, LS on T, keep the K largest of
 *               that solution without a second solve, SP's stopping rule, <= 50 rounds)
 *   cg_tol      CG tolerance, relative or absolute (see conventions); cg_maxit >= 0 (0: at most
 *               |S| steps, Theorem 5)
 *   s_out       [N] device, dense estimate, zeros off the support
 *   support_out [K] device, selected indices sorted ascending
 * One kernel launch on the op's stream; the whole greedy + CG loop runs on the device
 * without host synchronisation.  K = 0 writes zeros. */
cs_status cs_recover(cs_op_t op, const float* y, int32_t K, cs_algo algo, float cg_tol,
                     int32_t cg_maxit, float* s_out, int32_t* support_out);

/* Selection trace of this op's later recoveries (cs_recover, cs_recover_batched,
 * cs_recover_noalloc; no counterpart in the paper).  The decoders are heuristics whose discrete
 * choices can legitimately differ from an FP64 run where two candidates are nearly tied; the
 * trace records every choice and its margin, so a reference implementation can compare the
 * choices one by one and follow this run's choice at a near-tie (replay).
 *   trace_dev  [words] device int32, caller-owned; NULL disables the trace.  Every traced
 *              recovery first zeroes it on the op's stream, then writes it.
 *   words      capacity, 4 <= words < 2^31.
 * Layout (32-bit words): header {words used, records, overflow (1 if a record did not fit: the
 * records before it are complete, nothing after it is written), W = ceil(N / 32)}, then records
 * {kind, payload words, margin (float bits), aux} + payload, in decoder order:
 *   kind 1 argmax  (OMP selection; OMPR j = argmax outside S of |z|): aux = index
 *   kind 2 argmin  (OMPR i = argmin inside S of |z|): aux = index
 *   kind 3 top-K   (SP, CoSaMP, OMPR initial support and OMPR(l)): aux = K requested, payload =
 *                  W words, the bitmask of the selected indices (bit n & 31 of word n >> 5)
 *   kind 4 stop    (the SP / CoSaMP / OMPR(l) stopping test of a round): aux = 1 if it stopped
 *   kind 5 swap    (the OMPR swap test |z_j| > |z_i|): aux = 1 if it swapped
 * Margins (FP32, from the values the GPU selected on): argmax (a1 - a2) / a1 with a2 the
 * runner-up; argmin (a2 - a1) / a2; top-K (a_K - a_{K+1}) / a_K with a_{K+1} the largest
 * candidate not taken; a comparison x' >= x: |x - x'| / max(x, x'); a test decided by set
 * equality: 1.  The same margins feed cs_stats.near_ties and min_margin, which every
 * recovery that reports statistics computes (cs_recover; cs_recover_batched with stats_host). */
cs_status cs_op_set_trace(cs_op_t op, int32_t* trace_dev, int64_t words);

/* Same recovery as cs_recover, for callers that cannot allocate device memory when they
 * recover (a host framework that owns every device allocation, a loop that forbids allocation
 * after start-up, or a caller for whom cudaMalloc/cudaFree would synchronise the device).
 * The paper has no counterpart: this is a deployment variant of the same computation.
 * It calls no cudaMalloc, cudaFree or allocating library routine: the engine's per-call
 * scratch lives in one file-scope device array of 2.25 MiB + 8 KiB that every GPU loading the
 * library holds until the process exits.  Limit: N <= 65536 (larger N returns
 * CS_ERR_INVALID_ARG); all other argument rules are those of cs_recover.
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current and caches it: make that first call before any stream capture.
 * Every call shares the one array and the engine rewrites every scratch word it reads, so
 * nothing is cleared between calls; calls whose work overlaps on the GPU (other streams, or
 * other host threads) race on the array and must be serialised by the caller.
 * cs_get_stats does not report these calls. */
cs_status cs_recover_noalloc(cs_op_t op, const float* y, int32_t K, cs_algo algo, float cg_tol,
                             int32_t cg_maxit, float* s_out, int32_t* support_out);

/* Batched recovery of B independent signals in one persistent launch per cluster size; the
 * launches of different sizes run concurrently on streams forked from (and joined back into)
 * ops[0]'s stream, and the clusters of each launch claim signals largest-work first.  Signals
 * with N > 2^18 run one cooperative launch each, after the rest.
 * ops[b], y[b], K[b], algo[b], s_out[b], support_out[b] describe signal b (HOST arrays of
 * handles/device pointers).  All ops must share one stream (taken from ops[0]).
 * stats_host [B] HOST (may be NULL): filled after the work completes -- a non-NULL
 * stats_host makes the call wait for the stream. */
cs_status cs_recover_batched(int32_t B, const cs_op_t* ops, const float* const* y,
                             const int32_t* K, const int32_t* algo, float cg_tol,
                             int32_t cg_maxit, float* const* s_out,
                             int32_t* const* support_out, cs_stats* stats_host);

/* LS on a FIXED support (Sec. II step 3 solved as Algorithm 1's CG on
 * H = W A^T A W, b = W A^T y; Theorems 1-2 make the on-support entries equal).
 *   support [k] device, sorted ascending, distinct; y [M] device; s_S_out [k] device,
 *   s_S_out[i] is the coefficient of column support[i]. */
cs_status cs_ls_solve(cs_op_t op, const int32_t* support, int32_t k, const float* y,
                      float cg_tol, int32_t cg_maxit, float* s_S_out);

/* Adjoint of cs_ls_solve on a fixed support: dy = A_S (A_S^T A_S)^{-1} g, i.e. a CG solve
 * with the normal-equation matrix of Eq. 10 followed by one application of A_S.
 *   support [k] device sorted; g [k] device (dL/ds_S); dy_out [M] device. */
cs_status cs_ls_backward(cs_op_t op, const int32_t* support, int32_t k, const float* g,
                         float cg_tol, int32_t cg_maxit, float* dy_out);

/* Batched fixed-support LS solve / adjoint: B right-hand sides sharing one operator and one
 * support length k.  support, y/g, out are device arrays laid out [B][k], [B][M] or
 * [B][k], [B][k] -> [B][M] respectively (row-major, contiguous). */
cs_status cs_ls_solve_batched(cs_op_t op, int32_t B, const int32_t* support, int32_t k,
                              const float* y, float cg_tol, int32_t cg_maxit, float* s_S_out);
cs_status cs_ls_backward_batched(cs_op_t op, int32_t B, const int32_t* support, int32_t k,
                                 const float* g, float cg_tol, int32_t cg_maxit, float* dy_out);

/* Batched top-K support selection over |c| (Sec. II step 2: the K largest correlations, as in
 * SP's merge and the SP / OMPR initial support), independent of any operator.
 *   c        [B][N] device, row-major; c[b * N + n].
 *   exclude  [B][ceil(N/32)] device or NULL: bit n % 32 of word n / 32 of row b set means entry
 *            n of row b is not eligible (e.g. the current support, for top-K over j not in S).
 *   idx_out  [B][K] device: for every row the K eligible indices with the largest |c[b][n]|,
 *            ties broken towards the lowest index, sorted ascending; a row with fewer than K
 *            eligible entries gets all of them followed by -1.
 *   stream   the CUDA stream (a cudaStream_t; NULL: the legacy default stream).
 * 1 <= N <= 2^30, 0 <= K <= N, B >= 0 (B = 0 or K = 0: nothing to do).  NaN entries order
 * above +inf.  Asynchronous; allocates its workspace stream-ordered (cudaMallocAsync), so it
 * can be captured into a CUDA graph.  The result is exact for every input; one pass over c in
 * HBM suffices unless the row's values defeat the kernel's strided sample, in which case that
 * row is re-read (slower, still exact). */
cs_status cs_select_topk_batched(int32_t B, int64_t N, int32_t K, const float* c,
                                 const uint32_t* exclude, int32_t* idx_out, void* stream);

/* Statistics of the last single-signal call on this op (synchronises the op's stream). */
cs_status cs_get_stats(cs_op_t op, cs_stats* out);

/* Wait for the op's stream and report how its last launch ended: CS_ERR_CUDA if the stream
 * holds a CUDA error, CS_ERR_TIMEOUT if a bounded device wait gave up (a grid-wide barrier of
 * the streamed path, N > 2^18, or a bulk-copy completion of the last streamed batched A / A^T;
 * the outputs are then undefined), else CS_OK.
 * Apply and LS calls have no cs_stats; this is how their callers see a timeout. */
cs_status cs_op_sync(cs_op_t op);

/* Failure-path self test (no counterpart in the paper): runs, in a one-CTA kernel, the bounded
 * poll that the streamed path's grid barrier uses, on a device flag that is already set
 * (set_flag != 0: returns CS_OK at once) or that nothing sets (set_flag = 0: gives up after
 * `polls` polls, about 100 ns apart, and returns the CS_ERR_TIMEOUT the kernel reports).
 * 1 <= polls <= 2^24.  Synchronises the device. */
cs_status cs_probe_bounded_wait(uint64_t polls, int32_t set_flag);

/* Kernel launches this library has issued in this process, over all devices and operators:
 * every engine, grid, streamed-operator, task-table-upload and probe launch that was accepted
 * by the runtime (launches captured into a graph count once, at capture; replays do not).
 * The difference of two readings counts the launches of the calls made between them. */
int64_t cs_launch_count(void);

/* Thread-local description of the last error (never NULL). */
const char* cs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CS_GB300_H */
