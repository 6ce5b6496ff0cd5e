// cs_api.cu -- host side of the C ABI declared in include/cs_gb300.h.
//
// Builds the operator's random draws and tables (Sec. III-A, Eq. 7), validates arguments,
// packs tasks and launches the cluster engine of cs_engine.cu.  No compute happens here; the
// one kernel defined in this file copies task tables from its launch parameters to the device.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "cs_internal.h"

using namespace csg;

namespace {

thread_local std::string g_err = "no error";

cs_status fail(cs_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
cs_status cuda_fail(cudaError_t e, const char* what) {
  return fail(CS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Kernel launches issued by this library in this process (cs_launch_count).
std::atomic<int64_t> g_launches{0};
cudaError_t counted(cudaError_t e) {
  if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ull;
constexpr uint64_t SIGN_SALT = 0xD1B54A32D192ED03ull;

uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Omega: partial Fisher-Yates driven by the SplitMix64 stream seeded with seed ^ gamma,
// j = i + (u_{i+1} mod (N - i)); the first M entries, sorted.
std::vector<int32_t> draw_omega(int64_t N, int64_t M, uint64_t seed) {
  std::vector<int32_t> perm((size_t)N);
  std::iota(perm.begin(), perm.end(), 0);
  uint64_t st = seed ^ GAMMA;
  for (int64_t i = 0; i < M; ++i) {
    st += GAMMA;
    const uint64_t u = mix64(st);
    const int64_t j = i + (int64_t)(u % (uint64_t)(N - i));
    std::swap(perm[(size_t)i], perm[(size_t)j]);
  }
  std::vector<int32_t> om(perm.begin(), perm.begin() + M);
  std::sort(om.begin(), om.end());
  return om;
}

// Permutation randomiser R: a full Fisher-Yates shuffle of [0, N) driven by the SplitMix64
// stream seeded with seed ^ PERM_SALT, j = i + (u_{i+1} mod (N - i)) for i < N - 1; the DCT
// input n holds x[perm[n]].
constexpr uint64_t PERM_SALT = 0xA0761D6478BD642Full;
std::vector<int32_t> draw_perm(int64_t N, uint64_t seed) {
  std::vector<int32_t> perm((size_t)N);
  std::iota(perm.begin(), perm.end(), 0);
  uint64_t st = seed ^ PERM_SALT;
  for (int64_t i = 0; i + 1 < N; ++i) {
    st += GAMMA;
    const uint64_t u = mix64(st);
    const int64_t j = i + (int64_t)(u % (uint64_t)(N - i));
    std::swap(perm[(size_t)i], perm[(size_t)j]);
  }
  return perm;
}

// d_n = -1 iff the top bit of mix((seed ^ salt) + n + gamma) is set.
int8_t draw_sign(uint64_t sign_key, int64_t n) {
  return (mix64(sign_key + (uint64_t)n + GAMMA) >> 63) ? (int8_t)-1 : (int8_t)1;
}

// The library's stream-ordered scratch comes from the device's default memory pool.  Its
// release threshold is raised once per device (a setting of this process only, not of the
// GPU), so memory freed at the end of one call is reused by the next instead of going back to
// the CUDA driver at every synchronisation and being mapped again.
void retain_pool() {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  const uint64_t bit = 1ull << dev;
  if (done.load() & bit) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  done.fetch_or(bit);
}

cs_status check_nm(int64_t N, int64_t M) {
  if (N < N_MIN || N > N_MAX_GRID || (!is_pow2(N) && N > N_MAX_ANY))
    return fail(CS_ERR_UNSUPPORTED_N, "N must be in [16, 4096] or a power of two in [16, 2^24], got " +
                                          std::to_string(N));
  if (M < 1 || M > N) return fail(CS_ERR_INVALID_ARG, "M must satisfy 1 <= M <= N");
  return CS_OK;
}
int log2i(int64_t v) { int r = 0; while ((int64_t(1) << r) < v) ++r; return r; }

// In-place radix-2 FFT in FP64 (exp(-2 pi i j k / n)), n a power of two: the host builds the
// any-N path's chirp-kernel table with it.
void fft_host(std::vector<std::complex<double>>& a) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const double ang = -2.0 * M_PI / (double)len;
    for (size_t i = 0; i < n; i += len)
      for (size_t k = 0; k < len / 2; ++k) {
        const std::complex<double> w(std::cos(ang * (double)k), std::sin(ang * (double)k));
        const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
  }
}

// Two-level table of omega_T^j = exp(-2 pi i j / T) for j < 2^(lo_bits + hi_bits):
// [2^lo_bits] entries omega^i, then [2^hi_bits] entries omega^(j << lo_bits).
std::vector<float2> twiddle_table(double T, int lo_bits, int hi_bits) {
  const int nlo = 1 << lo_bits, nhi = 1 << hi_bits;
  std::vector<float2> tw((size_t)(nlo + nhi));
  for (int i = 0; i < nlo; ++i) {
    const double a = 2.0 * M_PI * (double)i / T;
    tw[(size_t)i] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  for (int j = 0; j < nhi; ++j) {
    const double a = 2.0 * M_PI * (double)((int64_t)j << lo_bits) / T;
    tw[(size_t)(nlo + j)] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  return tw;
}

}  // namespace

struct cs_op {
  int64_t N = 0, M = 0;
  uint64_t seed = 0;
  OpDev dev{};
  int32_t* d_omega = nullptr;
  uint32_t* d_omask = nullptr;
  int32_t* d_orank = nullptr;
  float2* d_tw = nullptr;
  std::vector<int32_t> h_omega;
  cudaStream_t stream = nullptr;
  float* d_scratch = nullptr;   // one cluster's scratch (or the whole grid's)
  uint32_t* d_bits = nullptr;
  cs_stats* d_stats = nullptr;
  void* d_grid = nullptr;       // streamed geometry: rows, signal rows, barrier and reduction state
  uint32_t* d_dbits = nullptr;  // [N/32] sign bits of d, for the streamed batched operator
  int32_t* d_prank = nullptr;   // [N/4 + 1][4] Omega ranks of the streamed row pass's pair outputs
  int32_t* d_perm = nullptr;    // permutation randomiser: [N] perm then [N] its inverse
  int randomizer = CS_RANDOMIZER_SIGNS;
  int* d_stream_err = nullptr;  // status word of the last streamed batched launch
  int batched_impl = CS_BATCHED_AUTO;
  int cg_abs = 0;               // CG stopping rule: 0 relative, 1 absolute (cs_op_set_cg_tol_mode)
  int ompr_l = 1;               // OMPR replacements per round (cs_op_set_ompr_replacements)
  int outer_cap = 0;            // cap on SP / CoSaMP rounds and OMPR swaps (0: 50 and 100)
  int tuned_nc[2] = {0, 0};     // per mode (A, A^T): 0 untuned, -1 cluster engine, else CTAs per vector
  std::vector<cudaStream_t> fork_streams;   // created on first use, kept until cs_op_destroy
  float2* d_czt = nullptr;      // any-N path: chirp-kernel FFT [czt_n], then the FFT twiddle table
  uint32_t* trace = nullptr;    // selection trace of later recoveries (cs_op_set_trace), caller-owned
  int64_t trace_words = 0;
};

namespace {

void free_op(cs_op* op) {
  if (!op) return;
  cudaFree(op->d_omega);
  cudaFree(op->d_omask);
  cudaFree(op->d_orank);
  cudaFree(op->d_tw);
  cudaFree(op->d_scratch);
  cudaFree(op->d_bits);
  cudaFree(op->d_stats);
  cudaFree(op->d_grid);
  cudaFree(op->d_dbits);
  cudaFree(op->d_prank);
  cudaFree(op->d_perm);
  cudaFree(op->d_stream_err);
  cudaFree(op->d_czt);
  for (cudaStream_t s : op->fork_streams) cudaStreamDestroy(s);
  delete op;
}

Task base_task(const cs_op* op, int mode) {
  Task t{};
  t.op = op->dev;
  t.mode = mode;
  t.algo = 0;
  t.K = 0;
  t.k_in = 0;
  t.cg_tol = 1e-6f;
  t.cg_maxit = 100;
  t.cg_abs = op->cg_abs;
  t.ompr_l = op->ompr_l;
  t.outer_max = 0;
  t.stats = op->d_stats;
  t.grid_scratch = op->d_scratch;
  t.grid_bits = op->d_bits;
  t.trace = op->trace;
  t.trace_cap = (int)op->trace_words;
  return t;
}

// A recovery with a trace starts from a zeroed trace buffer (its top-K records are OR-ed in).
cudaError_t clear_trace(const cs_op* op, cudaStream_t s) {
  if (!op->trace) return cudaSuccess;
  return cudaMemsetAsync(op->trace, 0, sizeof(uint32_t) * (size_t)op->trace_words, s);
}

Launch single_launch(const cs_op* op, const Task& t) {
  Launch L{};
  L.tasks = nullptr;
  L.single = t;
  L.ntasks = 1;
  L.F_alloc = op->dev.F;
  L.plan = op_plan(op->dev);
  L.scratch = op->d_scratch;
  L.scratch_per_cluster = (size_t)op->dev.P * scratch_floats_per_cta(op->dev.F);
  L.bits = op->d_bits;
  L.bits_per_cluster = (size_t)(op->N + 31) / 32;
  return L;
}

cs_status run_single(cs_op* op, const Task& t) {
  const Launch L = single_launch(op, t);
  cudaError_t e;
  if (op->dev.grid) {
    if ((e = cudaMemsetAsync(op->dev.gerr, 0, sizeof(int), op->stream)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(op->dev.gbar, 0, 2 * sizeof(unsigned), op->stream)) != cudaSuccess) return cuda_fail(e, "memset");
    e = counted(launch_grid(L, op->dev.G, op->stream));
    if (e != cudaSuccess) return cuda_fail(e, "grid launch");
    return CS_OK;
  }
  e = counted(launch_engine(L, op->dev.P, 1, op->stream));
  if (e != cudaSuccess) return cuda_fail(e, "engine launch");
  return CS_OK;
}

cs_status check_cg(float cg_tol, int32_t cg_maxit) {
  if (!(cg_tol >= 0.f) || cg_maxit < 0) return fail(CS_ERR_INVALID_ARG, "cg_tol must be >= 0 and cg_maxit >= 0");
  return CS_OK;
}

constexpr int SP_ROUNDS = 50;     // SP / CoSaMP outer-iteration cap
constexpr int STREAM_CLUSTER = 4;  // default CTAs per vector of the streamed batched operator (fastest untuned at 256 vectors)
constexpr int OMPR_SWAPS = 100;   // OMPR replacement cap

int outer_cap_of(const cs_op* op, int algo) {
  if (op->outer_cap > 0) return op->outer_cap;
  return (algo == CS_SP || algo == CS_COSAMP) ? SP_ROUNDS : OMPR_SWAPS;
}

}  // namespace

extern "C" {

const char* cs_last_error(void) { return g_err.c_str(); }

int64_t cs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

cs_status cs_operator_draws(int64_t N, int64_t M, uint64_t seed, int32_t* omega_M_host, int8_t* d_N_host) {
  const cs_status st = check_nm(N, M);
  if (st != CS_OK) return st;
  if (omega_M_host) {
    const std::vector<int32_t> om = draw_omega(N, M, seed);
    std::memcpy(omega_M_host, om.data(), sizeof(int32_t) * (size_t)M);
  }
  if (d_N_host)
    for (int64_t n = 0; n < N; ++n) d_N_host[n] = draw_sign(seed ^ SIGN_SALT, n);
  return CS_OK;
}

cs_status cs_operator_perm(int64_t N, uint64_t seed, int32_t* perm_N_host) {
  const cs_status st = check_nm(N, 1);
  if (st != CS_OK) return st;
  if (!perm_N_host) return fail(CS_ERR_INVALID_ARG, "null argument");
  const std::vector<int32_t> p = draw_perm(N, seed);
  std::memcpy(perm_N_host, p.data(), sizeof(int32_t) * (size_t)N);
  return CS_OK;
}

cs_op_t cs_op_create(int64_t N, int64_t M, uint64_t seed) { return cs_op_create_ex(N, M, seed, CS_RANDOMIZER_SIGNS); }

static cs_op_t create_op(int64_t N, int64_t M, uint64_t seed, int32_t randomizer, int32_t basis, int32_t n1);

cs_op_t cs_op_create_ex(int64_t N, int64_t M, uint64_t seed, int32_t randomizer) {
  return create_op(N, M, seed, randomizer, CS_BASIS_IDENTITY, 0);
}

cs_op_t cs_op_create_basis(int64_t N, int64_t M, uint64_t seed, int32_t basis, int32_t n1) {
  if (basis != CS_BASIS_IDENTITY && basis != CS_BASIS_DCT && basis != CS_BASIS_DCT2D) {
    fail(CS_ERR_INVALID_ARG, "unknown sparsifying basis");
    return nullptr;
  }
  if (basis != CS_BASIS_IDENTITY && N > N_MAX_ANY) {
    fail(CS_ERR_UNSUPPORTED_N, "a sparsifying basis needs N <= 4096");
    return nullptr;
  }
  if (basis == CS_BASIS_DCT2D && (n1 < 2 || N % n1 != 0 || N / n1 < 2)) {
    fail(CS_ERR_INVALID_ARG, "the 2-D basis needs n1 >= 2 dividing N with N / n1 >= 2");
    return nullptr;
  }
  return create_op(N, M, seed, CS_RANDOMIZER_SIGNS, basis, basis == CS_BASIS_DCT2D ? n1 : 0);
}

// Orthonormal DCT-II matrix C_n [n][n] (row k = frequency k) in FP64, stored as FP32.
static std::vector<float> dct_matrix_host(int n) {
  std::vector<float> c((size_t)n * n);
  for (int k = 0; k < n; ++k) {
    const double w = k == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
    for (int j = 0; j < n; ++j) c[(size_t)k * n + j] = (float)(w * std::cos(M_PI * (2.0 * j + 1.0) * k / (2.0 * n)));
  }
  return c;
}

static cs_op_t create_op(int64_t N, int64_t M, uint64_t seed, int32_t randomizer, int32_t basis, int32_t n1) {
  if (check_nm(N, M) != CS_OK) return nullptr;
  if (randomizer != CS_RANDOMIZER_SIGNS && randomizer != CS_RANDOMIZER_PERMUTATION) {
    fail(CS_ERR_INVALID_ARG, "unknown randomiser");
    return nullptr;
  }
  retain_pool();
  cs_op* op = new cs_op();
  op->N = N;
  op->M = M;
  op->seed = seed;
  op->randomizer = randomizer;
  op->h_omega = draw_omega(N, M, seed);
  const int64_t W = (N + 31) / 32;
  std::vector<uint32_t> omask((size_t)W, 0u);
  std::vector<int32_t> orank((size_t)W, 0);
  for (int32_t v : op->h_omega) omask[(size_t)(v >> 5)] |= 1u << (v & 31);
  for (int64_t w = 1; w < W; ++w) orank[(size_t)w] = orank[(size_t)w - 1] + __builtin_popcount(omask[(size_t)w - 1]);
  // twiddles omega_{4N}^j = exp(-2 pi i j / 4N), two-level split over j < 4N, or for
  // N >= N_TW_QUARTER over one quarter period j < N (the device folds j = q N + r); for an N
  // that is not a power of two (the any-N path) 128 low entries and enough high ones for j < 4N
  const bool generic = !is_pow2(N) || basis != CS_BASIS_IDENTITY;
  if (generic && randomizer != CS_RANDOMIZER_SIGNS) {
    fail(CS_ERR_UNSUPPORTED_N, "N that is not a power of two supports the sign randomiser only");
    delete op;
    return nullptr;
  }
  const bool quarter = N >= N_TW_QUARTER;
  int lo_bits, hi_bits;
  if (generic) {
    lo_bits = 7;
    hi_bits = log2i((4 * N + 127) / 128);
  } else {
    const int T = log2i(quarter ? N : 4 * N);
    lo_bits = (T + 1) / 2;
    hi_bits = T - lo_bits;
  }
  const std::vector<float2> tw = twiddle_table(4.0 * (double)N, lo_bits, hi_bits);
  const int64_t L = N / 2;
  OpDev& d = op->dev;
  d.N = (int)N;
  d.M = (int)M;
  d.lo_bits = lo_bits;
  d.hi_bits = hi_bits;
  d.tw_quarter = quarter ? 1 : 0;
  d.sign_key = seed ^ SIGN_SALT;
  d.grid = N > N_MAX ? 1 : 0;
  int P = 1, F = (int)L;
  d.generic = generic ? 1 : 0;
  d.psi = basis == CS_BASIS_DCT ? 1 : (basis == CS_BASIS_DCT2D ? 2 : 0);
  if (generic) {
    F = (int)((N + 1) / 2);   // 2F >= N real slots on one CTA
  } else if (d.grid) {
    // streamed geometry: rows of S1 points, G CTAs owning R rows each, column blocks of W
    d.S1 = GRID_S1;
    d.S2 = (int)(L / GRID_S1);
    d.G = std::min(GRID_G_MAX, d.S2);
    d.R = d.S2 / d.G;
    d.W = GRID_BLOCK / d.S2;
    d.NB = d.S1 / d.W;
    d.bpc = d.NB / d.G;
    P = d.G;
    F = d.R * d.S1;
  } else if (L > F_MAX) {
    P = (int)(L / F_MAX);
    F = F_MAX;
  }
  d.P = P;
  d.F = F;
  cudaError_t e;
  const size_t scratch = (size_t)P * scratch_floats_per_cta(F) * sizeof(float);
#define CSG_TRY(call)                                   \
  if ((e = (call)) != cudaSuccess) {                    \
    cuda_fail(e, #call);                                \
    free_op(op);                                        \
    return nullptr;                                     \
  }
  CSG_TRY(cudaMalloc(&op->d_omega, sizeof(int32_t) * (size_t)M));
  CSG_TRY(cudaMalloc(&op->d_omask, sizeof(uint32_t) * (size_t)W));
  CSG_TRY(cudaMalloc(&op->d_orank, sizeof(int32_t) * (size_t)W));
  CSG_TRY(cudaMalloc(&op->d_tw, sizeof(float2) * tw.size()));
  CSG_TRY(cudaMalloc(&op->d_scratch, scratch));
  CSG_TRY(cudaMalloc(&op->d_bits, sizeof(uint32_t) * (size_t)W));
  CSG_TRY(cudaMalloc(&op->d_stats, sizeof(cs_stats)));
  CSG_TRY(cudaMemcpy(op->d_omega, op->h_omega.data(), sizeof(int32_t) * (size_t)M, cudaMemcpyHostToDevice));
  CSG_TRY(cudaMemcpy(op->d_omask, omask.data(), sizeof(uint32_t) * (size_t)W, cudaMemcpyHostToDevice));
  CSG_TRY(cudaMemcpy(op->d_orank, orank.data(), sizeof(int32_t) * (size_t)W, cudaMemcpyHostToDevice));
  CSG_TRY(cudaMemcpy(op->d_tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice));
  CSG_TRY(cudaMemset(op->d_scratch, 0, scratch));
  CSG_TRY(cudaMemset(op->d_stats, 0, sizeof(cs_stats)));
  if (randomizer == CS_RANDOMIZER_PERMUTATION) {
    const std::vector<int32_t> perm = draw_perm(N, seed);
    std::vector<int32_t> both((size_t)(2 * N));
    for (int64_t n = 0; n < N; ++n) {
      both[(size_t)n] = perm[(size_t)n];
      both[(size_t)(N + perm[(size_t)n])] = (int32_t)n;
    }
    CSG_TRY(cudaMalloc(&op->d_perm, sizeof(int32_t) * both.size()));
    CSG_TRY(cudaMemcpy(op->d_perm, both.data(), sizeof(int32_t) * both.size(), cudaMemcpyHostToDevice));
    d.perm = op->d_perm;
    d.iperm = op->d_perm + N;
  }
  if (generic) {
    // chirp-z tables: the FFT over czt_n >= 2N - 1 points of the kernel b_m = c_{|m|} (indices
    // mod czt_n, zero for |m| >= N), c_m = exp(i pi m^2 / 2N), scaled by 1 / czt_n; then the
    // two-level omega_{4 czt_n} table of that FFT
    const int cn = 1 << log2i(2 * N - 1);
    std::vector<std::complex<double>> b((size_t)cn, 0.0);
    for (int64_t m = 0; m < N; ++m) {
      const double ph = M_PI * (double)((m * m) % (4 * N)) / (2.0 * (double)N);
      const std::complex<double> c(std::cos(ph), std::sin(ph));
      b[(size_t)m] = c;
      if (m > 0) b[(size_t)(cn - m)] = c;
    }
    fft_host(b);
    const int T2 = log2i(4 * (int64_t)cn);
    const int lo2 = (T2 + 1) / 2, hi2 = T2 - lo2;
    const std::vector<float2> tw2 = twiddle_table(4.0 * (double)cn, lo2, hi2);
    std::vector<float2> tab((size_t)cn + tw2.size());
    for (int k = 0; k < cn; ++k)
      tab[(size_t)k] = make_float2((float)(b[(size_t)k].real() / cn), (float)(b[(size_t)k].imag() / cn));
    std::copy(tw2.begin(), tw2.end(), tab.begin() + cn);
    if (basis == CS_BASIS_DCT2D) {   // the two small DCT-II matrices follow, as floats
      const std::vector<float> m1 = dct_matrix_host(n1), m2 = dct_matrix_host((int)(N / n1));
      const size_t base = tab.size();
      tab.resize(base + (m1.size() + m2.size() + 1) / 2);
      float* f = reinterpret_cast<float*>(tab.data() + base);
      std::copy(m1.begin(), m1.end(), f);
      std::copy(m2.begin(), m2.end(), f + m1.size());
      d.n1 = n1;
      d.n2 = (int)(N / n1);
    }
    CSG_TRY(cudaMalloc(&op->d_czt, sizeof(float2) * tab.size()));
    CSG_TRY(cudaMemcpy(op->d_czt, tab.data(), sizeof(float2) * tab.size(), cudaMemcpyHostToDevice));
    if (basis == CS_BASIS_DCT2D) {
      const float* f = reinterpret_cast<const float*>(op->d_czt + cn + tw2.size());
      d.c1 = f;
      d.c2 = f + (size_t)n1 * n1;
    }
    d.czt_n = cn;
    d.czt_hat = op->d_czt;
    d.tw2 = op->d_czt + cn;
    d.tw2_lo_bits = lo2;
    d.tw2_hi_bits = hi2;
  }
  if (!d.grid && N >= STREAM_N_MIN && randomizer == CS_RANDOMIZER_SIGNS && !generic) {
    std::vector<uint32_t> dbits((size_t)W, 0u);
    for (int64_t n = 0; n < N; ++n)
      if (draw_sign(d.sign_key, n) < 0) dbits[(size_t)(n >> 5)] |= 1u << (n & 31);
    CSG_TRY(cudaMalloc(&op->d_dbits, sizeof(uint32_t) * (size_t)W));
    CSG_TRY(cudaMemcpy(op->d_dbits, dbits.data(), sizeof(uint32_t) * (size_t)W, cudaMemcpyHostToDevice));
    // the row pass visits the pairs (Z_k, Z_{L-k}) unit by unit (ra = 0 .. P/2), k = ra + P k1;
    // store the rank in Omega of each pair output (-1: not in Omega) in that order
    const int SF = STREAM_F, SP = (int)(L / STREAM_F);
    auto rank_of = [&](int64_t f) -> int32_t {
      const uint32_t w = omask[(size_t)(f >> 5)];
      if (!((w >> (f & 31)) & 1u)) return -1;
      return orank[(size_t)(f >> 5)] + (int32_t)__builtin_popcount(w & ((1u << (f & 31)) - 1u));
    };
    std::vector<int32_t> prank((size_t)(L / 2 + 1) * 4, -1);
    size_t idx = 0;
    for (int ra = 0; ra <= SP / 2; ++ra) {
      const int np = ra == 0 ? SF / 2 + 1 : (2 * ra == SP ? SF / 2 : SF);
      for (int k1 = 0; k1 < np; ++k1, ++idx) {
        const int64_t k = ra + (int64_t)SP * k1;
        const bool self = ra == 0 && (k1 == 0 || 2 * k1 == SF);
        int64_t f[4];
        int nf = 4;
        if (k == 0) { f[0] = 0; f[1] = L; nf = 2; }
        else if (self) { f[0] = k; f[1] = N - k; nf = 2; }
        else { f[0] = k; f[1] = N - k; f[2] = L + k; f[3] = L - k; }
        for (int i = 0; i < nf; ++i) prank[idx * 4 + (size_t)i] = rank_of(f[i]);
      }
    }
    if (idx != (size_t)(L / 2 + 1)) {
      fail(CS_ERR_INVALID_ARG, "internal: streamed pair table size");
      free_op(op);
      return nullptr;
    }
    CSG_TRY(cudaMalloc(&op->d_stream_err, sizeof(int)));
    CSG_TRY(cudaMemset(op->d_stream_err, 0, sizeof(int)));
    CSG_TRY(cudaMalloc(&op->d_prank, sizeof(int32_t) * prank.size()));
    CSG_TRY(cudaMemcpy(op->d_prank, prank.data(), sizeof(int32_t) * prank.size(), cudaMemcpyHostToDevice));
  }
#undef CSG_TRY
  d.omask = op->d_omask;
  d.orank = op->d_orank;
  d.tw = op->d_tw;
  if (d.grid) {
    // one allocation: rows [S2][S1], signal rows [G][R][apad(S1)], barrier (2) + status (1),
    // reduction partials [4][G][4] floats and [4][G][2] u64, histograms [2][G][256]
    const size_t nY = (size_t)L, nsig = (size_t)d.G * d.R * (d.S1 + d.S1 / 16);
    const size_t off_sig = nY * sizeof(float2);
    const size_t off_bar = off_sig + nsig * sizeof(float2);
    const size_t off_red = off_bar + 64;
    const size_t off_red64 = off_red + (size_t)4 * d.G * 4 * sizeof(float);
    const size_t off_hist = off_red64 + (size_t)4 * d.G * 2 * sizeof(unsigned long long);
    const size_t off_fb = off_hist + (size_t)2 * d.G * 256 * sizeof(uint32_t);
    // N = 2^24: the Omega bits of each CTA's frequency tasks live here, not in shared memory
    const int fb_stride = N >= N_TW_QUARTER ? (d.bpc * ((d.W / 2) * d.S2 + d.S2 + 1) + 15) / 16 * 16 : 0;
    const size_t total = off_fb + (size_t)d.G * fb_stride;
    if ((e = cudaMalloc(&op->d_grid, total)) != cudaSuccess) {
      cuda_fail(e, "cudaMalloc(grid state)");
      free_op(op);
      return nullptr;
    }
    if ((e = cudaMemset(op->d_grid, 0, total)) != cudaSuccess) {
      cuda_fail(e, "cudaMemset(grid state)");
      free_op(op);
      return nullptr;
    }
    unsigned char* b = static_cast<unsigned char*>(op->d_grid);
    d.gY = reinterpret_cast<float2*>(b);
    d.gsig = reinterpret_cast<float2*>(b + off_sig);
    d.gbar = reinterpret_cast<unsigned*>(b + off_bar);
    d.gerr = reinterpret_cast<int*>(b + off_bar + 8);
    d.gred = reinterpret_cast<float*>(b + off_red);
    d.gred64 = reinterpret_cast<unsigned long long*>(b + off_red64);
    d.ghist = reinterpret_cast<uint32_t*>(b + off_hist);
    d.gfb = fb_stride ? reinterpret_cast<uint8_t*>(b + off_fb) : nullptr;
    d.gfb_stride = fb_stride;
    if (!grid_fits(d)) {
      fail(CS_ERR_UNSUPPORTED_N, "the streamed geometry's cooperative launch does not fit this device");
      free_op(op);
      return nullptr;
    }
    return op;
  }
  if (max_active_plan(P, op_plan(d)) < 1) {
    fail(CS_ERR_UNSUPPORTED_N, "a cluster of " + std::to_string(P) + " CTAs cannot be scheduled on this device");
    free_op(op);
    return nullptr;
  }
  return op;
}

void cs_op_destroy(cs_op_t op) {
  if (!op) return;
  if (op->stream) cudaStreamSynchronize(op->stream);
  else cudaDeviceSynchronize();
  free_op(op);
}

cs_status cs_op_set_stream(cs_op_t op, void* cuda_stream) {
  if (!op) return fail(CS_ERR_INVALID_ARG, "null operator");
  op->stream = (cudaStream_t)cuda_stream;
  return CS_OK;
}

cs_status cs_op_apply(cs_op_t op, const float* x_N, float* y_M) {
  if (!op || !x_N || !y_M) return fail(CS_ERR_INVALID_ARG, "null argument");
  Task t = base_task(op, MODE_APPLY);
  t.in = x_N;
  t.out = y_M;
  return run_single(op, t);
}

cs_status cs_op_apply_t(cs_op_t op, const float* y_M, float* x_N) {
  if (!op || !y_M || !x_N) return fail(CS_ERR_INVALID_ARG, "null argument");
  Task t = base_task(op, MODE_APPLY_T);
  t.in = y_M;
  t.out = x_N;
  return run_single(op, t);
}

static cs_status launch_tasks(std::vector<Task>& tasks, cudaStream_t stream, cs_op* owner);

// Streamed batched operator: one cluster of nc CTAs per vector, a per-cluster intermediate
// freed after the launch.
static int stream_default_nc(int P) { return std::min(STREAM_CLUSTER, P / 2); }

static cs_status stream_apply(cs_op_t op, int mode, int32_t B, const float* in, float* out, int nc) {
  const int clusters = std::min<int>(B, stream_clusters(nc));
  if (clusters < 1) return fail(CS_ERR_CUDA, "the streamed operator kernel cannot be launched on this device");
  StreamArgs a{};
  a.op = op->dev;
  a.dbits = op->d_dbits;
  a.prank = reinterpret_cast<const int4*>(op->d_prank);
  a.mode = mode;
  a.B = B;
  a.in = in;
  a.out = out;
  a.err = op->d_stream_err;
  cudaError_t e;
  if ((e = cudaMemsetAsync(op->d_stream_err, 0, sizeof(int), op->stream)) != cudaSuccess) return cuda_fail(e, "memset");
  const size_t bytes = sizeof(float) * stream_row_floats() * (size_t)op->dev.P * (size_t)clusters;
  if ((e = cudaMallocAsync(&a.T, bytes, op->stream)) != cudaSuccess) return cuda_fail(e, "alloc stream rows");
  e = counted(launch_stream(a, nc, clusters, op->stream));
  cudaFreeAsync(a.T, op->stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream launch");
  return CS_OK;
}

// The batched path for one call: 0 = cluster engine, else the streamed kernel with that many
// CTAs per vector (the tuned choice when there is one).
static int batched_choice(const cs_op* op, int mode, int32_t B) {
  if (!op->d_dbits || op->batched_impl == CS_BATCHED_CLUSTER) return 0;
  const int tuned = op->tuned_nc[mode == MODE_APPLY ? 0 : 1];
  if (op->batched_impl == CS_BATCHED_STREAMED) return tuned > 0 ? tuned : stream_default_nc(op->dev.P);
  if (tuned != 0) return tuned < 0 ? 0 : tuned;
  return B >= 2 ? stream_default_nc(op->dev.P) : 0;
}

static cs_status apply_with(cs_op_t op, int mode, int32_t B, const float* in, float* out, int nc) {
  if (nc > 0) return stream_apply(op, mode, B, in, out, nc);
  const size_t nin = mode == MODE_APPLY ? (size_t)op->N : (size_t)op->M;
  const size_t nout = mode == MODE_APPLY ? (size_t)op->M : (size_t)op->N;
  std::vector<Task> tasks;
  tasks.reserve((size_t)B);
  for (int b = 0; b < B; ++b) {
    Task t = base_task(op, mode);
    t.in = in + (size_t)b * nin;
    t.out = out + (size_t)b * nout;
    t.stats = nullptr;
    tasks.push_back(t);
  }
  if (B == 1) return run_single(op, tasks[0]);
  return launch_tasks(tasks, op->stream, op);
}

static cs_status apply_batched(cs_op_t op, int mode, int32_t B, const float* in, float* out) {
  if (!op || B < 0 || (B > 0 && (!in || !out))) return fail(CS_ERR_INVALID_ARG, "null argument or B < 0");
  if (B == 0) return CS_OK;
  return apply_with(op, mode, B, in, out, batched_choice(op, mode, B));
}

cs_status cs_op_apply_batched(cs_op_t op, int32_t B, const float* X, float* Y) {
  return apply_batched(op, MODE_APPLY, B, X, Y);
}

cs_status cs_op_apply_t_batched(cs_op_t op, int32_t B, const float* U, float* X) {
  return apply_batched(op, MODE_APPLY_T, B, U, X);
}

cs_status cs_op_set_cluster_size(cs_op_t op, int32_t P) {
  if (!op) return fail(CS_ERR_INVALID_ARG, "null operator");
  if (op->dev.grid) return fail(CS_ERR_UNSUPPORTED_N, "the cluster size applies to N <= 2^18");
  if (op->dev.generic) return fail(CS_ERR_UNSUPPORTED_N, "an N that is not a power of two runs on one CTA");
  const int64_t L = op->N / 2;
  const int Pmin = L > F_MAX ? (int)(L / F_MAX) : 1;
  if (P == 0) P = Pmin;
  if (P < Pmin || P > P_MAX || (P & (P - 1)) != 0 || L < 2 * (int64_t)P * P)
    return fail(CS_ERR_INVALID_ARG, "cluster size must be a power of two with N/(2 F_max) <= P <= 16 and N >= 4 P^2");
  const int F = (int)(L / P);
  if (max_active_clusters(P, F) < 1) return fail(CS_ERR_UNSUPPORTED_N, "this cluster size cannot be scheduled on this device");
  if (P == op->dev.P) return CS_OK;
  cudaError_t e = cudaStreamSynchronize(op->stream);   // queued work still uses the old scratch
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  const size_t bytes = (size_t)P * scratch_floats_per_cta(F) * sizeof(float);
  float* scratch = nullptr;
  if ((e = cudaMalloc(&scratch, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(scratch)");
  if ((e = cudaMemset(scratch, 0, bytes)) != cudaSuccess) {
    cudaFree(scratch);
    return cuda_fail(e, "cudaMemset(scratch)");
  }
  cudaFree(op->d_scratch);
  op->d_scratch = scratch;
  op->dev.P = P;
  op->dev.F = F;
  return CS_OK;
}

int32_t cs_op_cluster_size(cs_op_t op) { return op ? op->dev.P : 0; }

cs_status cs_op_tune_recover(cs_op_t op, int32_t K, int32_t algo, float cg_tol, int32_t cg_maxit, float* ms_out) {
  if (!op) return fail(CS_ERR_INVALID_ARG, "null operator");
  constexpr int NCAND = 5;
  if (ms_out)
    for (int i = 0; i < NCAND; ++i) ms_out[i] = -1.f;
  if (op->dev.grid || op->dev.generic) return CS_OK;   // one geometry only
  cs_status st = check_cg(cg_tol, cg_maxit);
  if (st != CS_OK) return st;
  if (K < 1 || K > op->M || algo < CS_OMP || algo > CS_COSAMP || (algo == CS_SP && 2 * (int64_t)K > op->M) ||
      (algo == CS_COSAMP && 3 * (int64_t)K > op->M))
    return fail(CS_ERR_INVALID_ARG, "K or algo out of range");
  // a K-sparse test signal: evenly spread positions, values alternating in sign and size
  std::vector<float> hs((size_t)op->N, 0.f);
  for (int64_t i = 0; i < K; ++i) hs[(size_t)(i * op->N / K)] = (i & 1) ? -0.5f - 0.25f * (float)(i % 5) : 1.f;
  float *s = nullptr, *y = nullptr, *so = nullptr;
  int32_t* supp = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&s, sizeof(float) * (size_t)op->N);
  if (e == cudaSuccess) e = cudaMalloc(&y, sizeof(float) * (size_t)op->M);
  if (e == cudaSuccess) e = cudaMalloc(&so, sizeof(float) * (size_t)op->N);
  if (e == cudaSuccess) e = cudaMalloc(&supp, sizeof(int32_t) * (size_t)K);
  if (e == cudaSuccess) e = cudaMemcpy(s, hs.data(), sizeof(float) * hs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) st = cuda_fail(e, "tuning buffers");
  if (st == CS_OK) st = cs_op_apply(op, s, y);
  const int start_P = op->dev.P;
  int best_P = start_P;
  float best = -1.f;
  for (int ci = 0; ci < NCAND && st == CS_OK; ++ci) {
    const int P = 1 << ci;
    if (cs_op_set_cluster_size(op, P) != CS_OK) continue;   // not a valid shape for this N
    float ms = -1.f;
    for (int rep = 0; rep < 3 && st == CS_OK; ++rep) {     // one warm-up, then the faster of two
      if ((e = cudaEventRecord(e0, op->stream)) != cudaSuccess) { st = cuda_fail(e, "event"); break; }
      st = cs_recover(op, y, K, (cs_algo)algo, cg_tol, cg_maxit, so, supp);
      if (st != CS_OK) break;
      if ((e = cudaEventRecord(e1, op->stream)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
        st = cuda_fail(e, "event");
        break;
      }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0 && (ms < 0.f || t < ms)) ms = t;
    }
    if (st != CS_OK) break;
    if (ms_out) ms_out[ci] = ms;
    if (best < 0.f || ms < best) { best = ms; best_P = P; }
  }
  const cs_status st2 = cs_op_set_cluster_size(op, st == CS_OK ? best_P : start_P);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(op->stream);
  cudaFree(s);
  cudaFree(y);
  cudaFree(so);
  cudaFree(supp);
  return st != CS_OK ? st : st2;
}

cs_status cs_op_set_outer_cap(cs_op_t op, int32_t cap) {
  if (!op) return fail(CS_ERR_INVALID_ARG, "null operator");
  if (cap < 0) return fail(CS_ERR_INVALID_ARG, "the outer-iteration cap must be >= 0");
  op->outer_cap = cap;
  return CS_OK;
}

cs_status cs_op_set_ompr_replacements(cs_op_t op, int32_t l) {
  if (!op) return fail(CS_ERR_INVALID_ARG, "null operator");
  if (l < 1) return fail(CS_ERR_INVALID_ARG, "OMPR replacements per round must be >= 1");
  op->ompr_l = l;
  return CS_OK;
}

cs_status cs_op_set_cg_tol_mode(cs_op_t op, int32_t mode) {
  if (!op) return fail(CS_ERR_INVALID_ARG, "null operator");
  if (mode != CS_CG_TOL_RELATIVE && mode != CS_CG_TOL_ABSOLUTE) return fail(CS_ERR_INVALID_ARG, "unknown CG tolerance mode");
  op->cg_abs = mode == CS_CG_TOL_ABSOLUTE ? 1 : 0;
  return CS_OK;
}

cs_status cs_op_set_batched_impl(cs_op_t op, int32_t impl) {
  if (!op) return fail(CS_ERR_INVALID_ARG, "null operator");
  if (impl != CS_BATCHED_AUTO && impl != CS_BATCHED_CLUSTER && impl != CS_BATCHED_STREAMED)
    return fail(CS_ERR_INVALID_ARG, "unknown batched implementation");
  if (impl == CS_BATCHED_STREAMED && !op->d_dbits)
    return fail(CS_ERR_UNSUPPORTED_N, "the streamed batched operator needs 2^15 <= N <= 2^18");
  op->batched_impl = impl;
  return CS_OK;
}

cs_status cs_op_tune_batched(cs_op_t op, int32_t B, float* ms_out) {
  if (!op || B < 1) return fail(CS_ERR_INVALID_ARG, "null operator or B < 1");
  constexpr int NCAND = 5;
  const int cand[NCAND] = {0, 1, 2, 4, 8};   // cluster engine, then CTAs per vector
  if (ms_out)
    for (int i = 0; i < 2 * NCAND; ++i) ms_out[i] = -1.f;
  const size_t nx = (size_t)B * (size_t)op->N, ny = (size_t)B * (size_t)op->M;
  float* X = nullptr;
  float* Y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&X, sizeof(float) * nx);
  if (e == cudaSuccess) e = cudaMalloc(&Y, sizeof(float) * ny);
  if (e == cudaSuccess) e = cudaMemsetAsync(X, 0x3c, sizeof(float) * nx, op->stream);   // 0.0115 in every entry
  if (e == cudaSuccess) e = cudaMemsetAsync(Y, 0x3c, sizeof(float) * ny, op->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  cs_status st = e == cudaSuccess ? CS_OK : cuda_fail(e, "tuning buffers");
  for (int mi = 0; mi < 2 && st == CS_OK; ++mi) {
    const int mode = mi == 0 ? MODE_APPLY : MODE_APPLY_T;
    const float* in = mi == 0 ? X : Y;
    float* out = mi == 0 ? Y : X;
    float best = 0.f;
    int best_nc = -1;
    for (int ci = 0; ci < NCAND && st == CS_OK; ++ci) {
      const int nc = cand[ci];
      if (nc > 0 && (!op->d_dbits || nc > op->dev.P / 2 || stream_clusters(nc) < 1)) continue;
      float ms = -1.f;
      for (int rep = 0; rep < 3 && st == CS_OK; ++rep) {   // one warm-up, then the faster of two
        if ((e = cudaEventRecord(e0, op->stream)) != cudaSuccess) { st = cuda_fail(e, "event"); break; }
        st = apply_with(op, mode, B, in, out, nc);
        if (st != CS_OK) break;
        if ((e = cudaEventRecord(e1, op->stream)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
          st = cuda_fail(e, "event");
          break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0 && (ms < 0.f || t < ms)) ms = t;
      }
      if (st != CS_OK) break;
      if (ms_out) ms_out[mi * NCAND + ci] = ms;
      if (best_nc < 0 || ms < best) { best = ms; best_nc = nc; }
    }
    if (st == CS_OK) op->tuned_nc[mi] = best_nc > 0 ? best_nc : -1;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(op->stream);
  cudaFree(X);
  cudaFree(Y);
  return st;
}

cs_status cs_select_topk_batched(int32_t B, int64_t N, int32_t K, const float* c, const uint32_t* exclude,
                                 int32_t* idx_out, void* stream) {
  if (B < 0) return fail(CS_ERR_INVALID_ARG, "B must be >= 0");
  if (N < 1 || N > (int64_t(1) << 30)) return fail(CS_ERR_INVALID_ARG, "N must be in [1, 2^30]");
  if (K < 0 || K > N) return fail(CS_ERR_INVALID_ARG, "K must satisfy 0 <= K <= N");
  if (B == 0 || K == 0) return CS_OK;
  if (!c || !idx_out) return fail(CS_ERR_INVALID_ARG, "null argument");
  retain_pool();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SelectArgs a = {};
  a.c = c;
  a.excl = exclude;
  a.out = idx_out;
  a.N = N;
  a.B = B;
  a.K = K;
  a.W = (int)((N + 31) / 32);
  const int64_t groups = (N + 3) / 4;
  a.S = 4 * (int)std::min<int64_t>(groups, SELECT_SAMPLE_MAX / 4);
  // sample rank of the threshold: the K-th largest of the row sits near rank mu = K S / N of
  // the sample (standard deviation about sqrt(mu)); r = 1.15 mu + 4 sqrt(mu) + 8 keeps at least
  // K entries at or above the threshold except with negligible probability, and about
  // N r / S of them (+- N sqrt(r) / S) are candidates
  const double mu = (double)K * a.S / (double)N;
  a.r = (int)std::min<double>(a.S, std::ceil(1.15 * mu + 4.0 * std::sqrt(mu) + 8.0));
  // each warp keeps the candidates of its sixteenth of the row: the expected count plus six
  // standard deviations of the threshold's and of the warp's own fluctuation, at most the range
  const double ew = (double)N * (a.r + 6.0 * std::sqrt((double)a.r) + 6.0) / a.S / SELECT_WARPS;
  const int64_t range = 4 * ((groups + SELECT_WARPS - 1) / SELECT_WARPS);
  a.capw = (int)std::min<double>((double)range, std::ceil(ew + 6.0 * std::sqrt(ew) + 64.0));
  a.vec = (N % 4 == 0 && (reinterpret_cast<uintptr_t>(c) & 15u) == 0) ? 1 : 0;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device query");
  const int per_sm = select_ctas_per_sm();
  if (per_sm < 1) return fail(CS_ERR_CUDA, "the selection kernel cannot be launched on this device");
  const int grid = (int)std::min<int64_t>(B, (int64_t)per_sm * sms);
  const size_t cand_bytes = sizeof(uint2) * (size_t)a.capw * SELECT_WARPS;
  void* ws = nullptr;
  if ((e = cudaMallocAsync(&ws, (size_t)grid * cand_bytes, s)) != cudaSuccess)
    return cuda_fail(e, "alloc selection workspace");
  a.cand = static_cast<uint2*>(ws);
  e = counted(launch_select(a, grid, s));
  cudaFreeAsync(ws, s);
  if (e != cudaSuccess) return cuda_fail(e, "selection launch");
  return CS_OK;
}

cs_status cs_probe_bounded_wait(uint64_t polls, int32_t set_flag) {
  if (polls < 1 || polls > (1ull << 24)) return fail(CS_ERR_INVALID_ARG, "polls must be in [1, 2^24]");
  unsigned* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 2 * sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(probe)");
  const unsigned init[2] = {set_flag ? 1u : 0u, 0xffffffffu};
  int status = -1;
  e = cudaMemcpy(buf, init, sizeof(init), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = counted(launch_wait_probe(buf, polls, reinterpret_cast<int*>(buf + 1), nullptr));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&status, buf + 1, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "probe");
  if (status == CS_ERR_TIMEOUT) return fail(CS_ERR_TIMEOUT, "the bounded wait ran out (as the probe intends when the flag is never set)");
  return (cs_status)status;
}

int32_t cs_op_concurrency(cs_op_t op) {
  if (!op) return 1;
  if (op->dev.grid) return 1;
  return std::max(1, max_active_plan(op->dev.P, op_plan(op->dev)));
}

cs_status cs_op_export(cs_op_t op, int32_t* omega_M_host, int8_t* d_N_host) {
  if (!op) return fail(CS_ERR_INVALID_ARG, "null operator");
  if (omega_M_host) std::memcpy(omega_M_host, op->h_omega.data(), sizeof(int32_t) * (size_t)op->M);
  if (d_N_host)
    for (int64_t n = 0; n < op->N; ++n)
      d_N_host[n] = op->randomizer == CS_RANDOMIZER_SIGNS ? draw_sign(op->dev.sign_key, n) : (int8_t)1;
  return CS_OK;
}

cs_status cs_op_export_perm(cs_op_t op, int32_t* perm_N_host) {
  if (!op || !perm_N_host) return fail(CS_ERR_INVALID_ARG, "null argument");
  if (op->randomizer != CS_RANDOMIZER_PERMUTATION) return fail(CS_ERR_INVALID_ARG, "the operator has no permutation");
  cudaError_t e = cudaMemcpy(perm_N_host, op->d_perm, sizeof(int32_t) * (size_t)op->N, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "perm copy");
  return CS_OK;
}

static cs_status check_recover(const cs_op* op, const float* y, int32_t K, int algo, float* s_out,
                               int32_t* support_out) {
  if (!op || !y || !s_out || (K > 0 && !support_out)) return fail(CS_ERR_INVALID_ARG, "null argument");
  if (algo < CS_OMP || algo > CS_COSAMP) return fail(CS_ERR_INVALID_ARG, "unknown algo");
  if (K < 0 || K > op->M) return fail(CS_ERR_INVALID_ARG, "K must satisfy 0 <= K <= M");
  if (algo == CS_SP && 2 * (int64_t)K > op->M) return fail(CS_ERR_INVALID_ARG, "SP needs 2K <= M");
  if (algo == CS_COSAMP && 3 * (int64_t)K > op->M) return fail(CS_ERR_INVALID_ARG, "CoSaMP needs 3K <= M");
  return CS_OK;
}

cs_status cs_recover(cs_op_t op, const float* y, int32_t K, cs_algo algo, float cg_tol, int32_t cg_maxit,
                     float* s_out, int32_t* support_out) {
  cs_status st = check_recover(op, y, K, (int)algo, s_out, support_out);
  if (st != CS_OK) return st;
  if ((st = check_cg(cg_tol, cg_maxit)) != CS_OK) return st;
  if (K == 0) {
    cudaError_t e = cudaMemsetAsync(s_out, 0, sizeof(float) * (size_t)op->N, op->stream);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    return CS_OK;
  }
  Task t = base_task(op, MODE_RECOVER);
  t.algo = (int)algo;
  t.K = K;
  t.cg_tol = cg_tol;
  t.cg_maxit = cg_maxit;
  t.outer_max = outer_cap_of(op, (int)algo);
  t.in = y;
  t.out = s_out;
  t.supp_out = support_out;
  cudaError_t e = clear_trace(op, op->stream);
  if (e != cudaSuccess) return cuda_fail(e, "trace memset");
  return run_single(op, t);
}

cs_status cs_op_set_trace(cs_op_t op, int32_t* trace_dev, int64_t words) {
  if (!op) return fail(CS_ERR_INVALID_ARG, "null operator");
  if (trace_dev && (words < TRACE_HEADER || words > INT32_MAX))
    return fail(CS_ERR_INVALID_ARG, "trace capacity must be in [4, 2^31 - 1] words");
  op->trace = reinterpret_cast<uint32_t*>(trace_dev);
  op->trace_words = trace_dev ? words : 0;
  return CS_OK;
}

// Task tables reach the device inside kernel launch parameters, TASK_CHUNK tasks per launch of
// task_upload_kernel, instead of a copy from host memory: parameter values are copied when the
// launch is issued, so the call can return (and its host vector die) at once, and a launch
// captured into a CUDA graph carries its own tables rather than a pointer into freed host
// memory.  The first chunk also zeroes the dynamic-claim counter that follows the table.
constexpr int TASK_CHUNK = (int)(31000 / sizeof(Task));   // as many tasks as fit the parameter space
struct TaskChunk {
  Task t[TASK_CHUNK];
  int n;                     // tasks in this chunk
  int first;                 // index of t[0] in the device table
};
static_assert(sizeof(TaskChunk) <= 32000, "task chunk must fit the 32 KB kernel-parameter limit");
static_assert(sizeof(Task) % 4 == 0, "tasks are copied as 32-bit words");

__global__ void task_upload_kernel(const __grid_constant__ TaskChunk c, Task* dst, int* claim) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(c.t);
  uint32_t* out = reinterpret_cast<uint32_t*>(dst + c.first);
  const int words = c.n * (int)(sizeof(Task) / 4);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x) out[i] = src[i];
  if (c.first == 0 && claim && blockIdx.x == 0 && threadIdx.x == 0) *claim = 0;
}

static cudaError_t upload_tasks(const std::vector<Task>& g, Task* dst, int* claim, cudaStream_t s) {
  auto chunk = std::make_unique<TaskChunk>();   // staging only: each launch copies it
  TaskChunk& c = *chunk;
  for (size_t first = 0; first < g.size(); first += TASK_CHUNK) {
    c.n = (int)std::min<size_t>(TASK_CHUNK, g.size() - first);
    c.first = (int)first;
    std::memcpy(c.t, g.data() + first, sizeof(Task) * (size_t)c.n);
    const int words = c.n * (int)(sizeof(Task) / 4);
    task_upload_kernel<<<(words + 255) / 256, 256, 0, s>>>(c, dst, claim);
    const cudaError_t e = counted(cudaGetLastError());
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Launch a list of tasks grouped by cluster size; scratch and task arrays come from the
// stream-ordered allocator and are released on the same stream.
static cs_status launch_tasks(std::vector<Task>& tasks, cudaStream_t stream, cs_op* owner) {
  // groups: cluster size P (power-of-two N), or 1000 + czt_n for the any-N path (own plan)
  std::map<int, std::vector<Task>> groups;
  std::vector<Task> grid_tasks;
  for (const Task& t : tasks) {
    if (t.op.grid) grid_tasks.push_back(t);
    else groups[t.op.generic ? 1000 + t.op.czt_n : t.op.P].push_back(t);
  }
  // One persistent launch per cluster size.  With several sizes the launches run concurrently on
  // streams forked from `stream` (event record + wait) and joined back into it, so a long signal
  // of one size does not hold the others back; clusters claim tasks dynamically, largest work
  // first.  The forked streams belong to the owning operator and outlive the call, so the same
  // fork and join also work while `stream` is being captured into a CUDA graph (they become
  // parallel branches of the graph).
  const bool fork = groups.size() > 1;
  std::vector<cudaStream_t> aux;
  cudaError_t e;
  cudaEvent_t start = nullptr;
  if (fork) {
    if ((e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "event");
    if ((e = cudaEventRecord(start, stream)) != cudaSuccess) return cuda_fail(e, "event record");
  }
  // Launch the group holding the largest single task first: the makespan is set by the
  // longest recoveries, and a group launched later finds the SMs taken by the earlier ones.
  auto work = [](const Task& t) { return (int64_t)t.op.N * std::max(t.K, t.k_in); };
  std::vector<std::pair<int, std::vector<Task>*>> order;
  for (auto& kv : groups) order.emplace_back(kv.first, &kv.second);
  std::stable_sort(order.begin(), order.end(), [&](const auto& a, const auto& b) {
    int64_t wa = 0, wb = 0;
    for (const Task& t : *a.second) wa = std::max(wa, work(t));
    for (const Task& t : *b.second) wb = std::max(wb, work(t));
    return wa > wb;
  });
  cs_status st = CS_OK;
  for (auto& og : order) {
    std::vector<Task>& g = *og.second;
    const int P = g[0].op.P;
    const bool generic = g[0].op.generic != 0;
    cudaStream_t s = stream;
    if (fork) {
      const size_t i = aux.size();
      if (i >= owner->fork_streams.size()) {
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) { st = cuda_fail(e, "stream"); break; }
        owner->fork_streams.push_back(s);
      }
      s = owner->fork_streams[i];
      aux.push_back(s);
      if ((e = cudaStreamWaitEvent(s, start, 0)) != cudaSuccess) { st = cuda_fail(e, "stream wait"); break; }
    }
    std::stable_sort(g.begin(), g.end(), [](const Task& a, const Task& b) {
      return (int64_t)a.op.N * std::max(a.K, a.k_in) > (int64_t)b.op.N * std::max(b.K, b.k_in);
    });
    int F_alloc = 0, Nmax = 0, hi_max = 0, t2l = 0, t2h = 0;
    for (const Task& t : g) {
      F_alloc = std::max(F_alloc, t.op.F);
      Nmax = std::max(Nmax, t.op.N);
      hi_max = std::max(hi_max, 1 << t.op.hi_bits);
      if (generic) { t2l = std::max(t2l, 1 << t.op.tw2_lo_bits); t2h = std::max(t2h, 1 << t.op.tw2_hi_bits); }
    }
    const SmemPlan plan = generic ? generic_plan(g[0].op.czt_n, F_alloc, hi_max, t2l, t2h) : cluster_plan(F_alloc);
    const int maxc = max_active_plan(P, plan);
    if (maxc < 1) { st = fail(CS_ERR_UNSUPPORTED_N, "cluster configuration cannot be scheduled"); break; }
    const int G = std::min<int>((int)g.size(), maxc);
    Launch L{};
    L.ntasks = (int)g.size();
    L.F_alloc = F_alloc;
    L.plan = plan;
    L.scratch_per_cluster = (size_t)P * scratch_floats_per_cta(F_alloc);
    L.bits_per_cluster = (size_t)(Nmax + 31) / 32;
    Task* d_tasks = nullptr;
    if ((e = cudaMallocAsync(&L.scratch, sizeof(float) * L.scratch_per_cluster * G, s)) != cudaSuccess) {
      st = cuda_fail(e, "alloc scratch");
      break;
    }
    if ((e = cudaMallocAsync(&L.bits, sizeof(uint32_t) * L.bits_per_cluster * G, s)) != cudaSuccess) {
      cudaFreeAsync(L.scratch, s);
      st = cuda_fail(e, "alloc bits");
      break;
    }
    if (g.size() == 1) {
      L.single = g[0];   // one task travels in the engine's own launch parameters
      e = cudaSuccess;
    } else {
      if ((e = cudaMallocAsync(&d_tasks, sizeof(Task) * g.size() + 16, s)) == cudaSuccess) {
        L.claim = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(d_tasks) + sizeof(Task) * g.size());
        e = upload_tasks(g, d_tasks, L.claim, s);
      }
      L.tasks = d_tasks;
    }
    if (e == cudaSuccess && (e = counted(launch_engine(L, P, G, s))) != cudaSuccess) st = cuda_fail(e, "engine launch");
    else if (e != cudaSuccess) st = cuda_fail(e, "upload tasks");
    if (d_tasks) cudaFreeAsync(d_tasks, s);
    cudaFreeAsync(L.scratch, s);
    cudaFreeAsync(L.bits, s);
    if (st != CS_OK) break;
  }
  // join every forked stream back into `stream` (also after an error, so that the caller's
  // stream never runs ahead of work already queued); events are released once their work
  // completes, the streams stay with the operator
  for (cudaStream_t s : aux) {
    cudaEvent_t ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) == cudaSuccess && (e = cudaEventRecord(ev, s)) == cudaSuccess)
      e = cudaStreamWaitEvent(stream, ev, 0);
    if (e != cudaSuccess) {
      if (st == CS_OK) st = cuda_fail(e, "stream join");
      cudaStreamSynchronize(s);   // the join failed: wait for the work instead
    }
    if (ev) cudaEventDestroy(ev);
  }
  if (start) cudaEventDestroy(start);
  if (st != CS_OK) return st;
  // streamed geometry: the whole GPU per signal, one cooperative launch each, after the rest
  for (const Task& t : grid_tasks) {
    Launch L{};
    L.tasks = nullptr;
    L.single = t;
    L.ntasks = 1;
    L.F_alloc = t.op.F;
    L.plan = grid_plan(t.op);
    L.scratch = t.grid_scratch;
    L.scratch_per_cluster = 0;
    L.bits = t.grid_bits;
    L.bits_per_cluster = 0;
    if ((e = cudaMemsetAsync(t.op.gerr, 0, sizeof(int), stream)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(t.op.gbar, 0, 2 * sizeof(unsigned), stream)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = counted(launch_grid(L, t.op.G, stream))) != cudaSuccess) return cuda_fail(e, "grid launch");
  }
  return CS_OK;
}

cs_status cs_recover_batched(int32_t B, const cs_op_t* ops, const float* const* y, const int32_t* K,
                             const int32_t* algo, float cg_tol, int32_t cg_maxit, float* const* s_out,
                             int32_t* const* support_out, cs_stats* stats_host) {
  if (B < 0 || (B > 0 && (!ops || !y || !K || !algo || !s_out || !support_out)))
    return fail(CS_ERR_INVALID_ARG, "null argument");
  if (B == 0) return CS_OK;
  cs_status st = check_cg(cg_tol, cg_maxit);
  if (st != CS_OK) return st;
  cudaStream_t stream = ops[0] ? ops[0]->stream : nullptr;
  cs_stats* d_stats = nullptr;
  cudaError_t e;
  if (stats_host) {   // the statistics are read back synchronously: not inside a graph capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(stream, &cap)) != cudaSuccess) return cuda_fail(e, "stream capture query");
    if (cap != cudaStreamCaptureStatusNone)
      return fail(CS_ERR_INVALID_ARG, "stats_host must be null while the stream is captured into a graph");
  }
  if ((e = cudaMallocAsync(&d_stats, sizeof(cs_stats) * (size_t)B, stream)) != cudaSuccess) return cuda_fail(e, "alloc stats");
  if ((e = cudaMemsetAsync(d_stats, 0, sizeof(cs_stats) * (size_t)B, stream)) != cudaSuccess) return cuda_fail(e, "memset");
  std::vector<Task> tasks;
  tasks.reserve((size_t)B);
  for (int b = 0; b < B; ++b) {
    if ((st = check_recover(ops[b], y[b], K[b], algo[b], s_out[b], support_out[b])) != CS_OK) {
      cudaFreeAsync(d_stats, stream);
      return fail(st, "signal " + std::to_string(b) + ": " + g_err);
    }
    if (K[b] == 0) {
      cudaMemsetAsync(s_out[b], 0, sizeof(float) * (size_t)ops[b]->N, stream);
      continue;
    }
    if ((e = clear_trace(ops[b], stream)) != cudaSuccess) {
      cudaFreeAsync(d_stats, stream);
      return cuda_fail(e, "trace memset");
    }
    Task t = base_task(ops[b], MODE_RECOVER);
    t.algo = algo[b];
    t.K = K[b];
    t.cg_tol = cg_tol;
    t.cg_maxit = cg_maxit;
    t.outer_max = outer_cap_of(ops[b], algo[b]);
    t.in = y[b];
    t.out = s_out[b];
    t.supp_out = support_out[b];
    t.stats = d_stats + b;
    tasks.push_back(t);
  }
  st = launch_tasks(tasks, stream, ops[0]);
  if (st == CS_OK && stats_host) {
    if ((e = cudaMemcpyAsync(stats_host, d_stats, sizeof(cs_stats) * (size_t)B, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
      st = cuda_fail(e, "stats copy");
    else if ((e = cudaStreamSynchronize(stream)) != cudaSuccess)
      st = cuda_fail(e, "stats sync");
  }
  cudaFreeAsync(d_stats, stream);
  return st;
}

static cs_status ls_batched(cs_op_t op, int mode, int32_t B, const int32_t* support, int32_t k, const float* in,
                            float cg_tol, int32_t cg_maxit, float* out) {
  if (!op || (B > 0 && (!support || !in || !out))) return fail(CS_ERR_INVALID_ARG, "null argument");
  if (B < 0 || k < 0 || k > op->M) return fail(CS_ERR_INVALID_ARG, "need B >= 0 and 0 <= k <= M");
  cs_status st = check_cg(cg_tol, cg_maxit);
  if (st != CS_OK) return st;
  if (B == 0) return CS_OK;
  if (k == 0) {
    const size_t n = mode == MODE_LS_BACKWARD ? (size_t)op->M * B : 0;
    if (n) cudaMemsetAsync(out, 0, sizeof(float) * n, op->stream);
    return CS_OK;
  }
  std::vector<Task> tasks;
  for (int b = 0; b < B; ++b) {
    Task t = base_task(op, mode);
    t.k_in = k;
    t.cg_tol = cg_tol;
    t.cg_maxit = cg_maxit;
    t.supp_in = support + (size_t)b * k;
    if (mode == MODE_LS_SOLVE) {
      t.in = in + (size_t)b * op->M;
      t.out = out + (size_t)b * k;
    } else {
      t.in = in + (size_t)b * k;
      t.out = out + (size_t)b * op->M;
    }
    tasks.push_back(t);
  }
  if (B == 1) return run_single(op, tasks[0]);
  for (Task& t : tasks) t.stats = nullptr;
  return launch_tasks(tasks, op->stream, op);
}

cs_status cs_ls_solve(cs_op_t op, const int32_t* support, int32_t k, const float* y, float cg_tol, int32_t cg_maxit,
                      float* s_S_out) {
  return ls_batched(op, MODE_LS_SOLVE, 1, support, k, y, cg_tol, cg_maxit, s_S_out);
}

cs_status cs_ls_backward(cs_op_t op, const int32_t* support, int32_t k, const float* g, float cg_tol,
                         int32_t cg_maxit, float* dy_out) {
  return ls_batched(op, MODE_LS_BACKWARD, 1, support, k, g, cg_tol, cg_maxit, dy_out);
}

cs_status cs_ls_solve_batched(cs_op_t op, int32_t B, const int32_t* support, int32_t k, const float* y,
                              float cg_tol, int32_t cg_maxit, float* s_S_out) {
  return ls_batched(op, MODE_LS_SOLVE, B, support, k, y, cg_tol, cg_maxit, s_S_out);
}

cs_status cs_ls_backward_batched(cs_op_t op, int32_t B, const int32_t* support, int32_t k, const float* g,
                                 float cg_tol, int32_t cg_maxit, float* dy_out) {
  return ls_batched(op, MODE_LS_BACKWARD, B, support, k, g, cg_tol, cg_maxit, dy_out);
}

cs_status cs_get_stats(cs_op_t op, cs_stats* out) {
  if (!op || !out) return fail(CS_ERR_INVALID_ARG, "null argument");
  cudaError_t e = cudaStreamSynchronize(op->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  e = cudaMemcpy(out, op->d_stats, sizeof(cs_stats), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "stats copy");
  return CS_OK;
}

cs_status cs_op_sync(cs_op_t op) {
  if (!op) return fail(CS_ERR_INVALID_ARG, "null operator");
  cudaError_t e = cudaStreamSynchronize(op->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  int err = 0;
  if (op->d_stream_err) {
    if ((e = cudaMemcpy(&err, op->d_stream_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "status copy");
    if (err != 0) return fail(CS_ERR_TIMEOUT, "a bulk-copy wait of the last streamed batched launch gave up");
  }
  if (!op->dev.grid) return CS_OK;
  e = cudaMemcpy(&err, op->dev.gerr, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "status copy");
  if (err != 0) return fail(CS_ERR_TIMEOUT, "a grid-wide wait of the last streamed launch gave up");
  return CS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Greedy recovery that allocates nothing (cs_recover_noalloc).
//
// Some callers cannot allocate device memory when they recover a signal: code running under a
// host framework that owns every device allocation (a plugin may not call cudaMalloc), loops
// that forbid allocation after start-up, or callers for whom a cudaMalloc/cudaFree would
// synchronise the device at the wrong moment.  For them the per-call scratch of the cluster
// engine (solution copies, A^T y by slot, support list, CG vectors, output bitmask) lives in one
// file-scope device array of fixed size, created when the library is loaded and held by every
// GPU that loads it until the process exits.
namespace {

constexpr int64_t NOALLOC_N_MAX = 1 << 16;                        // largest supported N
// P CTAs of F = N / 2P points need P (18 F + 128) floats, the most at P = P_MAX
constexpr size_t NOALLOC_SCRATCH = (size_t)P_MAX * scratch_floats_per_cta(NOALLOC_N_MAX / 2 / P_MAX);
constexpr size_t NOALLOC_BITS = (size_t)NOALLOC_N_MAX / 32;
// 2.25 MiB of scratch floats followed by the N-bit support bitmask (8 KiB)
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_SCRATCH + NOALLOC_BITS];

std::mutex g_noalloc_mu;
float* g_noalloc_ptr[64] = {};                                    // per device ordinal

// The array's host-side name is only a stand-in: its device address is looked up once per
// device, with that device current, and cached.
cs_status noalloc_scratch(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(CS_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    float* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return CS_OK;
}

}  // namespace

extern "C" cs_status cs_recover_noalloc(cs_op_t op, const float* y, int32_t K, cs_algo algo, float cg_tol,
                                        int32_t cg_maxit, float* s_out, int32_t* support_out) {
  cs_status st = check_recover(op, y, K, (int)algo, s_out, support_out);
  if (st != CS_OK) return st;
  if ((st = check_cg(cg_tol, cg_maxit)) != CS_OK) return st;
  if (op->N > NOALLOC_N_MAX)
    return fail(CS_ERR_INVALID_ARG, "cs_recover_noalloc supports N <= 65536 (fixed scratch size)");
  if ((size_t)op->dev.P * scratch_floats_per_cta(op->dev.F) > NOALLOC_SCRATCH)
    return fail(CS_ERR_INVALID_ARG, "cs_recover_noalloc: this cluster size needs more than the fixed scratch");
  if (K == 0) {
    cudaError_t e = cudaMemsetAsync(s_out, 0, sizeof(float) * (size_t)op->N, op->stream);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    return CS_OK;
  }
  float* base = nullptr;
  if ((st = noalloc_scratch(&base)) != CS_OK) return st;
  Task t = base_task(op, MODE_RECOVER);
  t.algo = (int)algo;
  t.K = K;
  t.cg_tol = cg_tol;
  t.cg_maxit = cg_maxit;
  t.outer_max = outer_cap_of(op, (int)algo);
  t.in = y;
  t.out = s_out;
  t.supp_out = support_out;
  t.stats = nullptr;   // the op's statistics buffer is left untouched
  if (op->trace) {
    const cudaError_t e = cudaMemsetAsync(op->trace, 0, sizeof(uint32_t) * (size_t)op->trace_words, op->stream);
    if (e != cudaSuccess) return cuda_fail(e, "trace memset");
  }
  Launch L{};
  L.tasks = nullptr;
  L.single = t;
  L.ntasks = 1;
  L.F_alloc = op->dev.F;
  L.plan = op_plan(op->dev);
  L.scratch = base;
  L.scratch_per_cluster = (size_t)op->dev.P * scratch_floats_per_cta(op->dev.F);
  L.bits = reinterpret_cast<uint32_t*>(base + NOALLOC_SCRATCH);
  L.bits_per_cluster = (size_t)(op->N + 31) / 32;
  // every scratch word the engine reads is written earlier in the same launch, so nothing
  // needs clearing between calls
  const cudaError_t e = counted(launch_engine(L, op->dev.P, 1, op->stream));
  if (e != cudaSuccess) return cuda_fail(e, "engine launch");
  return CS_OK;
}
