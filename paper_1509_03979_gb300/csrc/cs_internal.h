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
  int lo_bits, hi_bits;      // twiddle table split: 4N = 2^(lo_bits + hi_bits)
  uint64_t sign_key;         // seed ^ 0xD1B54A32D192ED03
  const uint32_t* omask;     // [N/32] bitmask of Omega
  const int32_t* orank;      // [N/32] number of Omega members below word w
  const float2* tw;          // [2^lo_bits] then [2^hi_bits]: omega_{4N}^j = lo[j & m] * hi[j >> lo]
};

// One unit of work for a cluster.
struct Task {
  OpDev op;
  int mode, algo;
  int K;                     // sparsity (recover)
  int k_in;                  // support length (LS modes)
  float cg_tol;
  int cg_maxit;
  int outer_max;             // SP rounds / OMPR swaps cap
  const float* in;
  const int32_t* supp_in;    // [k_in] (LS modes)
  float* out;
  int32_t* supp_out;         // [K] (recover)
  cs_stats* stats;           // device, may be null
};

// Kernel launch parameters (passed by value).
struct Launch {
  const Task* tasks;         // device array, or null when ntasks == 1 (then `single` is used)
  Task single;
  int ntasks;
  int F_alloc;               // shared-memory sizing (max F over the tasks)
  float* scratch;            // per cluster: P_MAX-strided per-CTA arrays, see scratch_floats()
  size_t scratch_per_cluster;   // floats
  uint32_t* bits;            // per cluster: N_MAX/32 words for the sorted support output
  size_t bits_per_cluster;   // words
};

// Per-CTA global scratch: SCRATCH_ARRAYS arrays of 2*F_alloc 32-bit words.
__host__ __device__ inline size_t scratch_floats_per_cta(int F_alloc) { return (size_t)SCRATCH_ARRAYS * 2 * F_alloc; }

size_t smem_bytes(int F_alloc);
cudaError_t launch_engine(const Launch& L, int P, int num_clusters, cudaStream_t stream);
int max_active_clusters(int P, int F_alloc);   // 0 if the configuration cannot be scheduled

}  // namespace csg
