// Internal declarations shared by the device engine (cs_engine.cu) and the C ABI (cs_api.cu).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/cs_gb300.h"

namespace csg {

constexpr int NT = 512;             // threads per CTA
constexpr int F_MAX = 8192;         // complex FFT points held by one CTA (64 KiB per buffer)
constexpr int P_MAX = 16;           // CTAs per cluster (non-portable size 16 on sm_103a)
constexpr int N_MIN = 16;
constexpr int N_MAX = 2 * F_MAX * P_MAX;   // 2^18: the largest N one cluster holds on chip
constexpr int SCRATCH_ARRAYS = 8;   // per-CTA global arrays of 2F words (see Scratch below)
// Streamed ("grid") geometry for N > N_MAX: the L = N/2 point FFT is split into S2 rows of
// S1 = GRID_S1 points; G = min(GRID_G_MAX, S2) CTAs of one cooperative launch own R = S2/G
// rows each, and a second pass runs S2-point column FFTs over blocks of W columns.
constexpr int GRID_S1 = 4096;
constexpr int GRID_LOG_S1 = 12;
static_assert((1 << GRID_LOG_S1) == GRID_S1, "GRID_LOG_S1 = log2 GRID_S1");
constexpr int GRID_G_MAX = 128;
constexpr int GRID_BLOCK = 4096;    // complex points per column block (W = GRID_BLOCK / S2)
constexpr int N_MAX_GRID = 1 << 24;   // 2^24: with the quarter-period twiddle table and global Omega task bits
constexpr int N_TW_QUARTER = 1 << 24;  // from this N on the twiddle table covers a quarter period

// Shared-memory sizing of one launch.
struct SmemPlan {
  int fft_n;        // complex points of each FFT buffer (A, B)
  int tw_lo_n;      // entries of the low twiddle table
  int tw_hi_n;      // entries of the high twiddle table
  int slot_words;   // 32-bit words of each per-slot bitmask (2F slots)
  int fb_bytes;     // Omega bits of the CTA's frequency tasks
  int cg_cap;       // support entries per CTA whose list and CG vectors live in shared memory
  int slot_n;       // any-N path: complex entries of the slot buffer S (0 otherwise)
  int tw2_lo_n;     // any-N path: entries of the FFT twiddle tables (0 otherwise)
  int tw2_hi_n;
  int tperm_n;      // cluster path: entries of the frequency-task order (0 otherwise)
};

enum Mode : int {
  MODE_APPLY = 0,        // out[M] = A in[N]
  MODE_APPLY_T = 1,      // out[N] = A^T in[M]
  MODE_RECOVER = 2,      // greedy decoder (algo), in = y
  MODE_LS_SOLVE = 3,     // fixed support LS, in = y, out = s_S[k]
  MODE_LS_BACKWARD = 4   // fixed support adjoint, in = g[k], out = dy[M]
};

// Operator constants as the device sees them.
struct OpDev {
  int N, M;
  int P, F;                  // cluster size and complex points per CTA (P * F = N / 2)
  int lo_bits, hi_bits;      // twiddle table split: 4N = 2^(lo_bits + hi_bits), or N with tw_quarter
  int tw_quarter;            // 1: the table covers omega_{4N}^j for j < N only (N >= N_TW_QUARTER)
  uint64_t sign_key;         // seed ^ 0xD1B54A32D192ED03
  const uint32_t* omask;     // [N/32] bitmask of Omega
  const int32_t* orank;      // [N/32] number of Omega members below word w
  const float2* tw;          // [2^lo_bits] then [2^hi_bits]: omega_{4N}^j = lo[j & m] * hi[j >> lo]
  const int32_t* perm;       // permutation randomiser: DCT input n holds x[perm[n]] (null: signs d)
  const int32_t* iperm;      // its inverse
  // streamed geometry (grid != 0 only)
  int grid;
  int S1, S2, G, R, W, NB, bpc;  // row length, rows, CTAs, rows per CTA, block width, blocks, blocks per CTA
  float2* gY;                // [S2][S1] row-major intermediate between the two passes
  float2* gsig;              // [G][R][apad(S1)] signal-domain rows owned by each CTA
  unsigned* gbar;            // [2] grid barrier: arrival count (zeroed before every launch), spare
  int* gerr;                 // device-side status of the last grid launch (0 = ok)
  float* gred;               // [4][G][4] reduction partials
  unsigned long long* gred64;   // [4][G][2]
  uint32_t* ghist;           // [2][G][256] radix histograms
  uint8_t* gfb;              // [G][gfb_stride] Omega bits of the frequency tasks (N = 2^24), or null
  int gfb_stride;
  // any-N path (N not a power of two, N <= N_MAX_ANY): one CTA, natural order, chirp-z DCTs
  int generic;               // 1 for this path
  int czt_n;                 // power-of-two FFT length of the chirp-z convolution, >= 2N - 1
  const float2* czt_hat;     // [czt_n] FFT of the chirp kernel, scaled by 1 / czt_n
  const float2* tw2;         // [2^tw2_lo_bits] then [2^tw2_hi_bits]: omega_{4 czt_n}^j, two levels
  int tw2_lo_bits, tw2_hi_bits;
  int psi;                   // sparsifying basis (any-N path): 0 identity, 1 Psi = C_N^T, 2 the separable
                             // 2-D basis C_{n1}^T (.) C_{n2} of an n1 x n2 array (Sec. III-A, IV-A)
  int n1, n2;                // 2-D basis: array shape, row-major (n1 n2 = N)
  const float* c1;           // 2-D basis: the orthonormal DCT-II matrices C_{n1} [n1][n1] and
  const float* c2;           //   C_{n2} [n2][n2], row k = frequency k
};
constexpr int N_MAX_ANY = 4096;   // largest N (not a power of two) of the any-N path: czt_n <= F_MAX

// One unit of work for a cluster.
struct Task {
  OpDev op;
  int mode, algo;
  int K;                     // sparsity (recover)
  int k_in;                  // support length (LS modes)
  float cg_tol;
  int cg_maxit;              // 0: at most |S| steps (Theorem 5)
  int cg_abs;                // 1: cg_tol bounds ||r_j|| absolutely, 0: relative to ||b||
  int outer_max;             // SP rounds / OMPR swaps cap
  int ompr_l;                // OMPR replacements per round (1: one swap)
  const float* in;
  const int32_t* supp_in;    // [k_in] (LS modes)
  float* out;
  int32_t* supp_out;         // [K] (recover)
  cs_stats* stats;           // device, may be null
  float* grid_scratch;       // streamed geometry: the op's own scratch and output bitmask
  uint32_t* grid_bits;
  uint32_t* trace;           // selection trace (recover), zeroed by the host, or null
  int trace_cap;             // its capacity in 32-bit words
};

// Selection trace written by a recovery (cs_op_set_trace): a header of TRACE_HEADER words
// {words used, records, overflow flag, N/32 rounded up}, then records of TRACE_HEADER words
// {kind, payload words, margin (float bits), aux} followed by the payload.  Kinds follow the
// decoders' selections and stop tests; a top-K record's payload is the N-bit mask of the
// selected signal indices, the other kinds carry the index or the decision in aux.
enum TraceKind : int { TR_ARGMAX = 1, TR_ARGMIN = 2, TR_TOPK = 3, TR_STOP = 4, TR_SWAP = 5 };
constexpr int TRACE_HEADER = 4;

// Kernel launch parameters (passed by value).
struct Launch {
  const Task* tasks;         // device array, or null when ntasks == 1 (then `single` is used)
  Task single;
  int ntasks;
  int F_alloc;               // scratch strides (max F over the tasks)
  SmemPlan plan;             // shared-memory sizing
  float* scratch;            // per cluster: P_MAX-strided per-CTA arrays, see scratch_floats()
  size_t scratch_per_cluster;   // floats
  uint32_t* bits;            // per cluster: N_MAX/32 words for the sorted support output
  size_t bits_per_cluster;   // words
  int* claim;                // task counter for dynamic claiming (zeroed), or null: static round robin
};

// Per-CTA global scratch: SCRATCH_ARRAYS arrays of 2*F_alloc 32-bit words, then the rank
// table (4 ints per frequency task; a CTA runs at most F/2 + P_MAX + 1 tasks).
__host__ __device__ constexpr size_t rank_ints_per_cta(int F_alloc) { return 4 * ((size_t)F_alloc / 2 + P_MAX + 16); }
__host__ __device__ constexpr size_t scratch_floats_per_cta(int F_alloc) {
  return (size_t)SCRATCH_ARRAYS * 2 * F_alloc + rank_ints_per_cta(F_alloc);
}

// Streamed batched operator (A x or A^T u for a batch of vectors, one CTA per vector): rows of
// STREAM_F points, P = N / (2 STREAM_F) rows, for STREAM_N_MIN <= N <= N_MAX.
constexpr int STREAM_F = F_MAX;
constexpr int STREAM_N_MIN = 4 * STREAM_F;   // P >= 2
struct StreamArgs {
  OpDev op;                  // N, M, P, twiddles and Omega tables
  const uint32_t* dbits;     // [N/32] sign bits of d (bit set: d_n = -1)
  const int4* prank;         // [N/4 + 1] per DCT pair of the row pass: ranks in Omega of its outputs
  int mode;                  // MODE_APPLY or MODE_APPLY_T
  int B;                     // vectors
  const float* in;           // [B][N] (A) or [B][M] (A^T), contiguous
  float* out;                // [B][M] (A) or [B][N] (A^T)
  float2* T;                 // per cluster: [P][apad(STREAM_F)] intermediate rows
  int* err;                  // status word: CS_ERR_TIMEOUT if a bulk-copy wait ran out
};
size_t stream_row_floats();    // floats of one padded intermediate row
int stream_clusters(int nc);   // clusters of nc CTAs resident at once (0: cannot launch)
cudaError_t launch_stream(const StreamArgs& a, int nc, int clusters, cudaStream_t stream);

cudaError_t launch_wait_probe(unsigned* flag, unsigned long long limit, int* status, cudaStream_t stream);

// Batched top-K selection (cs_select.cu): one CTA per row at a time, workspace per CTA.
struct SelectArgs {
  const float* c;            // [B][N] rows
  const uint32_t* excl;      // [B][W] exclusion bits (bit n of row b set: entry n is not eligible), or null
  int32_t* out;              // [B][K] selected indices, ascending (-1 past the eligible count)
  uint2* cand;               // per CTA and warp: [capw] (key, index) candidates of the warp's range
  long long N;
  int B, K, W;               // rows, selected per row, 32-bit words per row of excl
  int capw;                  // candidate capacity per warp
  int S, r;                  // sample keys (a multiple of 4) and the sample rank of the threshold
  int vec;                   // 1: N % 4 == 0 and c 16-byte aligned (16-byte loads)
};
constexpr int SELECT_SAMPLE_MAX = 4096;   // sample keys of cs_select.cu
constexpr int SELECT_WARPS = 16;          // warps per CTA of cs_select.cu
int select_ctas_per_sm();
cudaError_t launch_select(const SelectArgs& a, int grid, cudaStream_t stream);

SmemPlan cluster_plan(int F_alloc);
SmemPlan generic_plan(int czt_n, int F_alloc, int tw_hi_n, int tw2_lo_n, int tw2_hi_n);
SmemPlan op_plan(const OpDev& op);              // the plan a single task of this operator runs with
int max_active_plan(int P, const SmemPlan& plan);   // clusters of P CTAs resident with this plan
SmemPlan grid_plan(const OpDev& op);
size_t smem_bytes(const SmemPlan& plan);
cudaError_t launch_engine(const Launch& L, int P, int num_clusters, cudaStream_t stream);
cudaError_t launch_grid(const Launch& L, int G, cudaStream_t stream);
int max_active_clusters(int P, int F_alloc);   // 0 if the configuration cannot be scheduled
int grid_fits(const OpDev& op);                // 1 if a cooperative launch of G CTAs fits

}  // namespace csg
