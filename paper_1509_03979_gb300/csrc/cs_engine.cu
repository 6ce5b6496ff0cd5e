// cs_engine.cu -- cluster-resident device engine for the greedy CS decoders (sm_103a).
//
// One thread-block cluster of P CTAs (P = 1..16) owns one signal.  The N-point orthonormal
// DCT-II / DCT-III behind A = P_Omega C_N diag(d) (Sec. III-A, Eq. 7) is computed through an
// L = N/2 point complex FFT (Makhoul's reordering, J. Makhoul, IEEE TASSP 1980) that lives
// entirely in the cluster's shared memory:
//
//   * CTA p holds z[q P + p] (q < Q = L/P, "stride-P" layout) and runs a Q-point Stockham FFT
//     in shared memory (radix 16/8/4/2 butterflies in registers);
//   * a twiddle omega_L^{p k_q}, an all-to-all pull over distributed shared memory, and
//     P-point DFTs across CTAs finish the four-step FFT; CTA c then holds the frequency slots
//     k_q in [c h, c h + h) and their mirrors Q - k_q (h = Q / 2P), so each DCT output pair
//     (k, L - k) is CTA-local;
//   * the DCT post-processing, the Omega mask / residual / output step, and the DCT-III
//     pre-processing all happen in that frequency layout, and the inverse path mirrors the
//     forward one.
//
// Signal-domain values stay in the FFT buffer in "slot" order: real slot sigma = 2 q + b of
// CTA p is signal index n(p, sigma) (see n_of_slot).  The support W_S of Eq. 8 is a per-CTA
// bitmask over slots; CG vectors are compressed to the support entries a CTA owns, so the
// scatter W x and the gather W^T of Algorithm 1 are CTA-local.
//
// Every barrier is a hardware barrier (__syncthreads or barrier.cluster); every branch around
// a barrier depends only on task parameters or on cluster-reduced values that all CTAs compute
// in the same order, so control flow is uniform across the cluster and no wait can spin.
#include <cooperative_groups.h>

#include "cs_internal.h"

namespace cg = cooperative_groups;

namespace csg {

// ------------------------------------------------------------------------------- helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }   // a * i

// cos(2 pi j / 16): exact mathematical constants.
__device__ __forceinline__ float cos16(int j) {
  switch (j & 15) {
    case 0: return 1.0f;
    case 1: case 15: return 0.92387953251128674f;
    case 2: case 14: return 0.70710678118654752f;
    case 3: case 13: return 0.38268343236508977f;
    case 4: case 12: return 0.0f;
    case 5: case 11: return -0.38268343236508977f;
    case 6: case 10: return -0.70710678118654752f;
    case 7: case 9: return -0.92387953251128674f;
    default: return -1.0f;
  }
}
__device__ __forceinline__ float sin16(int j) { return cos16(j - 4); }

// b * omega_16^t with omega = exp(DIR * 2 pi i / 16); t is a compile-time constant after unrolling.
template <int DIR>
__device__ __forceinline__ float2 mul_w16(float2 b, int t) {
  t &= 15;
  if (t == 0) return b;
  if (t == 8) return make_float2(-b.x, -b.y);
  if (t == 4) return DIR > 0 ? cmuli(b) : make_float2(b.y, -b.x);
  if (t == 12) return DIR > 0 ? make_float2(b.y, -b.x) : cmuli(b);
  return cmul(b, make_float2(cos16(t), DIR * sin16(t)));
}

__host__ __device__ constexpr int brev_bits(int x, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1) << (bits - 1 - b);
  return r;
}
template <int R> struct Lg { static constexpr int v = R <= 1 ? 0 : 1 + Lg<R / 2>::v; };
template <> struct Lg<1> { static constexpr int v = 0; };

// In-register R-point DFT, natural order in and out (iterative radix-2 decimation in time).
template <int R, int DIR>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R > 1) {
    constexpr int LG = Lg<R>::v;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int j = brev_bits(i, LG);
      if (j > i) { float2 t = v[i]; v[i] = v[j]; v[j] = t; }
    }
#pragma unroll
    for (int len = 2; len <= R; len <<= 1) {
      const int half = len >> 1;
#pragma unroll
      for (int i = 0; i < R; i += len) {
#pragma unroll
        for (int j = 0; j < half; ++j) {
          const float2 a = v[i + j];
          const float2 b = mul_w16<DIR>(v[i + j + half], j * (16 / len));
          v[i + j] = cadd(a, b);
          v[i + j + half] = csub(a, b);
        }
      }
    }
  }
}

extern __shared__ __align__(16) unsigned char smem_raw[];

// Re-derive a pointer from the shared-memory base so the compiler knows its address space
// (pointers travelling through non-inlined calls are generic).
template <class T>
__device__ __forceinline__ T* shp(T* p) {
  const ptrdiff_t off = reinterpret_cast<const unsigned char*>(p) - smem_raw;
  return reinterpret_cast<T*>(smem_raw + off);
}

// Padded index into the local FFT buffer (one spare element every 16 keeps the strided
// Stockham stores of the early passes free of shared-memory bank conflicts).
__device__ __forceinline__ int aidx(int q) { return q + (q >> 4); }
__host__ __device__ constexpr int apad(int F) { return F + F / 16; }

// Two-level twiddle table: omega_{4N}^j = exp(-2 pi i j / 4N) = lo[j & m] * hi[j >> lo_bits];
// lo is stored with the same one-in-16 padding as the FFT buffer, which keeps the strided
// lookups of the FFT passes and the DCT twiddles (strides 1, 4, 8) free of bank conflicts.
struct Tw {
  const float2* lo;
  const float2* hi;
  int lo_bits;
  int lo_mask;
  int mask4n;   // 4N - 1
  template <int DIR>
  __device__ __forceinline__ float2 get(int j) const {
    j &= mask4n;
    const float2 w = cmul(lo[aidx(j & lo_mask)], hi[j >> lo_bits]);
    return DIR > 0 ? cconj(w) : w;
  }
};
// The streamed path's table.  For N = 2^24 the two levels would not fit next to the streamed
// plan, so the table covers one quarter period instead: j = q N + r with r < N,
// omega_{4N}^j = (-i)^q omega_{4N}^r (qbits = log2 N, qmask = N - 1); otherwise qbits = 31 and
// q is always 0.  Only the streamed path's functions are instantiated with it, so the fold
// costs the on-chip paths nothing.
struct TwQ : Tw {
  int qbits;
  int qmask;
  template <int DIR>
  __device__ __forceinline__ float2 get(int j) const {
    j &= mask4n;
    const int q = j >> qbits;
    j &= qmask;
    float2 w = cmul(lo[aidx(j & lo_mask)], hi[j >> lo_bits]);
    if (q != 0) {   // times (-i)^q, exact
      if (q & 1) w = make_float2(w.y, -w.x);
      if (q & 2) w = make_float2(-w.x, -w.y);
    }
    return DIR > 0 ? cconj(w) : w;
  }
};

// v[r] *= w^r with w = omega_{4N}^t (DIR < 0) or its conjugate; powers built from w, w^2,
// w^4, w^8 read from the table, so every factor carries at most three rounded products.
template <int R, int DIR, class TW>
__device__ __forceinline__ void twiddle_powers(float2* v, const TW& tw, int t) {
  const float2 w1 = tw.get<DIR>(t);
  v[1] = cmul(v[1], w1);
  if constexpr (R >= 4) {
    const float2 w2 = tw.get<DIR>(2 * t);
    const float2 w3 = cmul(w1, w2);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    if constexpr (R >= 8) {
      const float2 w4 = tw.get<DIR>(4 * t);
      v[4] = cmul(v[4], w4);
      v[5] = cmul(v[5], cmul(w1, w4));
      v[6] = cmul(v[6], cmul(w2, w4));
      v[7] = cmul(v[7], cmul(w3, w4));
      if constexpr (R >= 16) {
        const float2 w8 = tw.get<DIR>(8 * t);
        v[8] = cmul(v[8], w8);
        v[9] = cmul(v[9], cmul(w1, w8));
        v[10] = cmul(v[10], cmul(w2, w8));
        v[11] = cmul(v[11], cmul(w3, w8));
        v[12] = cmul(v[12], cmul(w4, w8));
        v[13] = cmul(v[13], cmul(cmul(w1, w4), w8));
        v[14] = cmul(v[14], cmul(cmul(w2, w4), w8));
        v[15] = cmul(v[15], cmul(cmul(w3, w4), w8));
      }
    }
  }
}

// One out-of-place Stockham pass of radix R from X to Y (padded indexing): butterfly j reads
// X[j + r F/R], applies omega_{Ns R}^{r k} (k = j mod Ns), and writes Y[(j - k) R + k + r Ns].
// One barrier per pass; a thread keeps one butterfly live at a time.
template <int R, int DIR, class TW>
__device__ __forceinline__ void fft_pass(const float2* X, float2* Y, int F, int Ns, const TW& tw, int four_n) {
  const int nb = F / R;
  for (int j = threadIdx.x; j < nb; j += NT) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = X[aidx(j + r * nb)];
    const int k = j & (Ns - 1);
    if (Ns > 1) twiddle_powers<R, DIR>(v, tw, k * (four_n / (Ns * R)));
    dft<R, DIR>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) Y[aidx(base + r * Ns)] = v[r];
  }
  __syncthreads();
}

// Q-point FFT of X (natural order in and out) using Y as the ping-pong buffer.  The plan is
// fixed at compile time for each F = 2^LOGF (a runtime pass loop measured worse register
// allocation): a radix-2/4/8 pass first when log2 F is not a multiple of 4, then radix 16,
// and when the pass count is odd the first pass runs in place through registers so that the
// result always lands back in X.
template <int R, int DIR, class TW>
__device__ __forceinline__ void fft_pass_inplace(float2* X, int F, const TW& tw, int four_n) {
  constexpr int BPT = (F_MAX / NT) / R;
  const int nb = F / R;
  float2 v[BPT][R];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int j = threadIdx.x + b * NT;
    if (j < nb) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = X[aidx(j + r * nb)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int j = threadIdx.x + b * NT;
    if (j < nb) {
      dft<R, DIR>(v[b]);   // first pass: Ns = 1, no twiddles, output index j R + r
#pragma unroll
      for (int r = 0; r < R; ++r) X[aidx(j * R + r)] = v[b][r];
    }
  }
  __syncthreads();
}

template <int LOGF, int DIR, int LOGNS, bool TO_Y, class TW>
__device__ __forceinline__ void fft_rest(float2* X, float2* Y, const TW& tw, int four_n) {
  // remaining passes are all radix 16; TO_Y: the next pass writes Y
  if constexpr (LOGNS < LOGF) {
    if constexpr (TO_Y) fft_pass<16, DIR>(X, Y, 1 << LOGF, 1 << LOGNS, tw, four_n);
    else fft_pass<16, DIR>(Y, X, 1 << LOGF, 1 << LOGNS, tw, four_n);
    fft_rest<LOGF, DIR, LOGNS + 4, !TO_Y>(X, Y, tw, four_n);
  }
}

template <int LOGF, int DIR, class TW>
__device__ __forceinline__ void fft_plan(float2* X, float2* Y, const TW& tw, int four_n) {
  constexpr int HEAD = LOGF % 4;                       // bits of the leading small-radix pass
  constexpr int NPASS = LOGF / 4 + (HEAD ? 1 : 0);
  constexpr int R0 = HEAD == 0 ? 16 : (1 << HEAD);
  if constexpr (NPASS % 2 == 1) {
    // odd pass count: first pass in place (registers), then an even number of ping-pongs
    fft_pass_inplace<R0, DIR>(X, 1 << LOGF, tw, four_n);
    fft_rest<LOGF, DIR, (HEAD ? HEAD : 4), true>(X, Y, tw, four_n);
  } else {
    fft_pass<R0, DIR>(X, Y, 1 << LOGF, 1, tw, four_n);
    fft_rest<LOGF, DIR, (HEAD ? HEAD : 4), false>(X, Y, tw, four_n);
  }
}

// One function per plan, so that each plan's register allocation is its own.
template <int LOGF, int DIR, class TW>
__device__ __noinline__ void fft_plan_call(float2* X, float2* Y, TW tw, int four_n) {
  X = shp(X);
  Y = shp(Y);
  tw.lo = shp(tw.lo);
  tw.hi = shp(tw.hi);
  fft_plan<LOGF, DIR>(X, Y, tw, four_n);
}

template <int DIR, class TW>
__device__ __noinline__ void local_fft(float2* X, float2* Y, int F, TW tw, int four_n) {
  switch (__ffs(F) - 1) {
    case 1: fft_plan_call<1, DIR>(X, Y, tw, four_n); break;
    case 2: fft_plan_call<2, DIR>(X, Y, tw, four_n); break;
    case 3: fft_plan_call<3, DIR>(X, Y, tw, four_n); break;
    case 4: fft_plan_call<4, DIR>(X, Y, tw, four_n); break;
    case 5: fft_plan_call<5, DIR>(X, Y, tw, four_n); break;
    case 6: fft_plan_call<6, DIR>(X, Y, tw, four_n); break;
    case 7: fft_plan_call<7, DIR>(X, Y, tw, four_n); break;
    case 8: fft_plan_call<8, DIR>(X, Y, tw, four_n); break;
    case 9: fft_plan_call<9, DIR>(X, Y, tw, four_n); break;
    case 10: fft_plan_call<10, DIR>(X, Y, tw, four_n); break;
    case 11: fft_plan_call<11, DIR>(X, Y, tw, four_n); break;
    case 12: fft_plan_call<12, DIR>(X, Y, tw, four_n); break;
    default: fft_plan_call<13, DIR>(X, Y, tw, four_n); break;
  }
}

// The F_MAX = 2^13 plan after its leading radix-2 pass, for input already in that pass's
// output layout in Y: three radix-16 passes, Y -> X -> Y -> X.
static_assert(F_MAX == 8192, "fft_after_radix2 follows the 2^13 plan");
template <int DIR>
__device__ __noinline__ void fft_after_radix2(float2* X, float2* Y, Tw tw, int four_n) {
  X = shp(X);
  Y = shp(Y);
  tw.lo = shp(tw.lo);
  tw.hi = shp(tw.hi);
  fft_rest<13, DIR, 1, false>(X, Y, tw, four_n);
}

// P-point DFT across CTAs, one frequency slot column per thread; B is laid out [p][s].
template <int R, int DIR>
__device__ __forceinline__ void pcol(float2* B, int s, int S2) {
  float2 v[R];
#pragma unroll
  for (int p = 0; p < R; ++p) v[p] = B[p * S2 + s];
  dft<R, DIR>(v);
#pragma unroll
  for (int p = 0; p < R; ++p) B[p * S2 + s] = v[p];
}
template <int DIR>
__device__ __forceinline__ void pstep(float2* B, int P, int S2) {
  if (P > 1) {
    for (int s = threadIdx.x; s < S2; s += NT) {
      switch (P) {
        case 2: pcol<2, DIR>(B, s, S2); break;
        case 4: pcol<4, DIR>(B, s, S2); break;
        case 8: pcol<8, DIR>(B, s, S2); break;
        default: pcol<16, DIR>(B, s, S2); break;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------ reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_max64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// ------------------------------------------------------------------------- shared layout

// Support entries per CTA whose list and CG vectors live in shared memory: up to 4096 when the
// transform is at most 4096 points per CTA (the rest of the plan is small); 1024 (20 KB) for
// the 8192-point CTAs, where a larger share costs more in L1 than it saves (SP at N = 2^18:
// 1024 measured 5 % faster than none, 2048 4 %; its merged support puts ~820 entries per CTA).
__host__ __device__ inline int cluster_cg_cap(int F_alloc) { return F_alloc <= 4096 ? (2 * F_alloc < 4096 ? 2 * F_alloc : 4096) : 1024; }

struct Smem {
  float2* A;          // local FFT buffer (padded), signal-domain slots between transforms
  float2* B;          // exchange / frequency buffer [P][2h]; FFT ping-pong buffer (padded)
  float2* twlo;
  float2* twhi;
  uint32_t* signw;    // d_n bits per local slot (1 = -1)
  uint32_t* mask[2];  // support bitmasks over local slots
  uint8_t* fbits;     // Omega membership of the (up to 4) DCT outputs of each frequency task
  uint32_t* hist;     // [2][256]
  uint32_t* htot;     // [256]
  float* ring;        // [4][4] cluster-reduction partials
  unsigned long long* ring64;   // [4][2]
  float* wsum;        // [4][16] warp partials
  unsigned long long* wmax;     // [2][16]
  int* iscr;          // [64] integer scratch / broadcast
  float* fscr;        // [8]
  int* cgl;           // [cap] support list when it fits
  float* cgv;         // [4][cap] CG x, r, p, q when they fit
  float2* S;          // any-N path: signal-domain values by slot (natural order)
  float2* tw2lo;      // any-N path: twiddles of the chirp-z FFT
  float2* tw2hi;
  uint16_t* tperm;    // cluster path: this CTA's frequency tasks, those with a kept output first
};

// Bump allocator over the dynamic shared-memory window (16-byte granules).
struct Bump {
  unsigned char* base;
  size_t off;
  __host__ __device__ unsigned char* operator()(size_t bytes) {
    unsigned char* p = base ? base + off : nullptr;
    off += (bytes + 15) & ~size_t(15);
    return p;
  }
};

__host__ __device__ inline void layout(const SmemPlan& pl, Bump& take, Smem* s) {
  const int nw = pl.slot_words;
  const int cap = pl.cg_cap;
  unsigned char* A = take(sizeof(float2) * apad(pl.fft_n));
  unsigned char* B = take(sizeof(float2) * apad(pl.fft_n));   // also the FFT ping-pong buffer (padded)
  unsigned char* tl = take(sizeof(float2) * apad(pl.tw_lo_n));
  unsigned char* th = take(sizeof(float2) * pl.tw_hi_n);
  unsigned char* sw = take(4 * nw);
  unsigned char* m0 = take(4 * nw);
  unsigned char* m1 = take(4 * nw);
  unsigned char* fb = take(pl.fb_bytes);
  unsigned char* hi = take(4 * 512);
  unsigned char* ht = take(4 * 256);
  unsigned char* rg = take(4 * 16);
  unsigned char* r64 = take(8 * 8);
  unsigned char* ws = take(4 * 64);
  unsigned char* wm = take(8 * 32);
  unsigned char* is = take(4 * 64);
  unsigned char* fs = take(4 * 8);
  unsigned char* cl = take(4 * (size_t)cap);
  unsigned char* cv = take(16 * (size_t)cap);
  unsigned char* sv = take(sizeof(float2) * (size_t)pl.slot_n);
  unsigned char* t2l = take(sizeof(float2) * (size_t)(pl.tw2_lo_n ? apad(pl.tw2_lo_n) : 0));
  unsigned char* t2h = take(sizeof(float2) * (size_t)pl.tw2_hi_n);
  unsigned char* tp = take(sizeof(uint16_t) * (size_t)pl.tperm_n);
  if (s) {
    s->S = (float2*)sv; s->tw2lo = (float2*)t2l; s->tw2hi = (float2*)t2h; s->tperm = (uint16_t*)tp;
    s->A = (float2*)A; s->B = (float2*)B; s->twlo = (float2*)tl; s->twhi = (float2*)th;
    s->signw = (uint32_t*)sw; s->mask[0] = (uint32_t*)m0; s->mask[1] = (uint32_t*)m1;
    s->fbits = (uint8_t*)fb; s->hist = (uint32_t*)hi; s->htot = (uint32_t*)ht; s->ring = (float*)rg;
    s->ring64 = (unsigned long long*)r64; s->wsum = (float*)ws; s->wmax = (unsigned long long*)wm;
    s->iscr = (int*)is; s->fscr = (float*)fs; s->cgl = (int*)cl; s->cgv = (float*)cv;
  }
}

__device__ Smem carve(const SmemPlan& pl) {
  Smem s;
  Bump b{smem_raw, 0};
  layout(pl, b, &s);
  return s;
}

// Cluster launches: FFT buffers of F points, twiddle levels of <= 1024 entries (4N <= 2^20),
// 2F slots, and CTA 0's F/2 + P + 1 frequency tasks.
SmemPlan cluster_plan(int F_alloc) {
  SmemPlan p;
  p.fft_n = F_alloc;
  p.tw_lo_n = 1024;
  p.tw_hi_n = 1024;
  p.slot_words = (2 * F_alloc + 31) / 32;
  p.fb_bytes = F_alloc / 2 + P_MAX + 16;
  p.cg_cap = cluster_cg_cap(F_alloc);
  p.slot_n = 0;
  p.tw2_lo_n = 0;
  p.tw2_hi_n = 0;
  p.tperm_n = F_alloc / 2 + P_MAX + 16;   // >= ntasks of every CTA
  return p;
}

// Any-N launches: FFT buffers of czt_n points, the DCT twiddle table (128 low entries), the
// slot buffer of F_alloc complex entries (2 F_alloc >= N real slots) and the FFT's twiddles.
SmemPlan generic_plan(int czt_n, int F_alloc, int tw_hi_n, int tw2_lo_n, int tw2_hi_n) {
  SmemPlan p;
  p.fft_n = czt_n;
  p.tw_lo_n = 128;
  p.tw_hi_n = tw_hi_n;
  p.slot_words = (2 * F_alloc + 31) / 32;
  p.fb_bytes = 16;
  // next to two 8192-point FFT buffers only 1024 support entries fit on chip (20 KB)
  p.cg_cap = czt_n >= F_MAX ? 1024 : cluster_cg_cap(F_alloc);
  p.slot_n = apad(F_alloc);
  p.tw2_lo_n = tw2_lo_n;
  p.tw2_hi_n = tw2_hi_n;
  p.tperm_n = 0;
  return p;
}

// Grid launches: FFT buffers of S1 points (rows and column blocks), the op's twiddle levels,
// 2 R S1 slots, and the frequency tasks of the CTA's column blocks (each h S2 + S2 + 1).
SmemPlan grid_plan(const OpDev& op) {
  SmemPlan p;
  p.fft_n = op.S1;
  p.tw_lo_n = 1 << op.lo_bits;
  p.tw_hi_n = 1 << op.hi_bits;
  p.slot_words = (2 * op.R * op.S1 + 31) / 32;
  p.fb_bytes = op.gfb ? 16 : op.bpc * ((op.W / 2) * op.S2 + op.S2 + 1) + 16;
  p.cg_cap = 0;
  p.slot_n = 0;
  p.tw2_lo_n = 0;
  p.tw2_hi_n = 0;
  p.tperm_n = 0;
  return p;
}

SmemPlan op_plan(const OpDev& op) {
  if (op.grid) return grid_plan(op);
  if (op.generic) return generic_plan(op.czt_n, op.F, 1 << op.hi_bits, 1 << op.tw2_lo_bits, 1 << op.tw2_hi_bits);
  return cluster_plan(op.F);
}

size_t smem_bytes(const SmemPlan& pl) {
  Bump b{nullptr, 0};
  layout(pl, b, nullptr);
  return b.off;
}

// ---------------------------------------------------------------------- per-signal context
enum MidKind : int { MID_MASK = 0, MID_RESID = 1, MID_OUT = 2, MID_IN = 3 };
enum SrcKind : int { SRC_NONE = 0, SRC_CG = 1, SRC_DENSE_SLOTS = 2, SRC_GLOBAL_N = 3 };

// Geometry of one signal as seen by one CTA (all sizes powers of two); kept in registers.
struct Geo {
  int N, L, P, F, h, lh, S2, c, four_n;
  int nat;   // 1: slot sigma is signal index sigma (the any-N path), 0: the stride-P Makhoul layout
};

// Per-CTA context of the signal being processed.  It lives in shared memory (one copy per CTA)
// so every function reads it with plain shared loads: a per-thread copy on the stack measured
// as the largest source of local-memory traffic.  Fields are written by thread 0 before a
// barrier that every later reader passes.
struct Ctx {
  Smem sm;
  TwQ tw;
  Geo g;
  int M, nwords, cap;
  const uint32_t* omask;
  const int32_t* orank;
  // global per-CTA scratch
  float* xd[2];
  float* cy;
  int* glist;          // global list (fallback when the support share exceeds cap)
  float* gcg;          // global CG vectors (fallback), 4 arrays of 2F
  // current support list and CG vectors (shared memory when they fit)
  int* list;
  float* cgx;
  float* cgr;
  float* cgp;
  float* cgq;
  uint32_t* bits;     // per-cluster N-bit output bitmask
  int4* rank4;        // cluster launches: per frequency task, the rank in Omega of each of its
                      // (up to 4) DCT outputs, -1 where the output is not kept (global scratch)
  const void* setup_key;   // operator whose twiddles, sign bits and Omega tables are loaded
  // signal-domain values by slot: the FFT buffer A (cluster launches) or the CTA's rows in
  // global memory (grid launches); slot q lives at (q & rmask) * rowstride + aidx(q >> rshift)
  float2* sig;
  int rmask, rshift, rowstride;
  int grid;           // 0: cluster launch, 1: cooperative grid launch
  OpDev op;           // the operator (grid launches read its streamed geometry and buffers)
  int ring_slot;      // next cluster-reduction slot (all CTAs advance it identically)
  int hist_slot;      // next radix-histogram buffer
  int cg_abs;         // CG stopping rule of the current task: 1 absolute, 0 relative
  int cg_total;       // statistics (thread 0 only)
  int cg_hits;
  int ntrans;         // N-point DCT applications (forward or inverse)
  int next_task;      // cluster rank 0: the task index it claimed for the cluster
  // selection margins and the selection trace (recoveries that report statistics or a trace)
  int want_margins;   // 1: compute the margin of every selection and stop test
  int near_ties;      // selections and stop tests with margin <= NEAR_TIE (thread 0)
  float min_margin;   // smallest margin seen (thread 0)
  uint32_t* trace;    // selection trace, or null
  int trace_cap;      // its capacity in words
  int trace_off;      // word offset of the next record (advanced identically in every CTA)
  int trace_recs;     // records written
  int trace_over;     // 1 once a record did not fit: nothing more is written
  // the any-N path
  int gen;            // 1: this task runs the any-N transform
  int nslots;         // valid slots of this CTA (2F, or N on the any-N path)
  int czt_n;
  const float2* czt_hat;
  Tw tw2;             // twiddles of the chirp-z FFT (omega_{4 czt_n})
  SmemPlan plan;      // the launch's shared-memory plan
  float cg_beta;      // CG: beta of the last step, applied by the next scatter of p (cluster path)
  int cg_fuse;        // 1 while cg_solve runs with the direction update in the scatter
  int tnz;            // cluster path: frequency tasks of this CTA with a kept output (tperm's first)
};
__shared__ Ctx C;

// The twiddle tables of the current task, addressed in shared memory: the plain table of the
// on-chip paths (ctx_tw: generic pointers, for the FFT entry points) and the streamed path's.
__device__ __forceinline__ Tw ctx_tw() { return static_cast<const Tw&>(C.tw); }
__device__ __forceinline__ void smem_tw_into(Tw& t) {
  t = static_cast<const Tw&>(C.tw);
  t.lo = shp(C.sm.twlo);
  t.hi = shp(C.sm.twhi);
}
__device__ __forceinline__ void smem_tw_into(TwQ& t) {
  t = C.tw;
  t.lo = shp(C.sm.twlo);
  t.hi = shp(C.sm.twhi);
}
__device__ __forceinline__ Tw smem_tw() {
  Tw t;
  smem_tw_into(t);
  return t;
}
__device__ __forceinline__ TwQ smem_twq() {
  TwQ t;
  smem_tw_into(t);
  return t;
}

__device__ __forceinline__ void cl_sync() { cg::this_cluster().sync(); }
template <class T>
__device__ __forceinline__ T* cl_map(T* p, int rank) { return cg::this_cluster().map_shared_rank(p, rank); }

// Bounded software barrier over the CTAs of a cooperative (grid) launch.  The launch guarantees
// co-residency; a wait that still exceeds GRID_SPIN_LIMIT polls sets CS_ERR_TIMEOUT in the
// op's status word and continues, and later barriers stop waiting once the status is set, so
// the launch always ends.  One monotonic arrival count (zeroed before every launch): the b-th
// barrier's arrivals are numbers (b-1) G + 1 .. b G, because no CTA passes barrier b before all
// G have arrived at it, so a CTA waits until the count reaches the next multiple of G.  The last
// arrival does no extra write (no reset, no generation word).
constexpr unsigned long long GRID_SPIN_LIMIT = 1ull << 26;

// Poll *word until it differs from `from`, at most `limit` times about 100 ns apart; false when
// the limit ran out.
__device__ __forceinline__ bool spin_until_changed(volatile unsigned* word, unsigned from, unsigned long long limit) {
  unsigned long long spins = 0;
  while (*word == from) {
    if (++spins > limit) return false;
    __nanosleep(100);
  }
  return true;
}

__device__ __noinline__ void grid_sync() {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* count = C.op.gbar;
    volatile int* err = C.op.gerr;
    __threadfence();
    const unsigned G = (unsigned)C.op.G;
    const unsigned arrived = atomicAdd(count, 1u) + 1u;
    const unsigned target = arrived + (G - arrived % G) % G;   // this barrier's last arrival
    if (arrived != target && *err == 0) {
      volatile unsigned* vc = count;
      unsigned long long spins = 0;
      while ((int)(*vc - target) < 0) {
        if (++spins > GRID_SPIN_LIMIT) { atomicExch(const_cast<int*>(err), (int)CS_ERR_TIMEOUT); break; }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Barrier over the CTAs that share one signal: the cluster, or the whole cooperative grid.
__device__ __forceinline__ void group_sync() {
  if (C.grid) grid_sync();
  else cl_sync();
}

// Signal-domain values by slot (A buffer for clusters, the CTA's global rows for the grid).
struct SigView {
  float* base;
  int rmask, rshift, rowstride;
  __device__ __forceinline__ float& at(int sg) const {
    const int q = sg >> 1;
    return base[2 * ((q & rmask) * rowstride + aidx(q >> rshift)) + (sg & 1)];
  }
};
__device__ __forceinline__ SigView sigview() {
  SigView v;
  if (C.grid) { v.base = reinterpret_cast<float*>(C.sig); v.rmask = C.rmask; v.rshift = C.rshift; v.rowstride = C.rowstride; }
  else { v.base = reinterpret_cast<float*>(C.gen ? shp(C.sm.S) : shp(C.sm.A)); v.rmask = 0; v.rshift = 0; v.rowstride = 0; }
  return v;
}

__device__ __forceinline__ float& slot_ref(float2* A, int sigma) {
  return reinterpret_cast<float*>(A)[2 * aidx(sigma >> 1) + (sigma & 1)];
}
// Signal index of local real slot sigma of CTA c: complex point m = q P + c of z, real index
// v = 2 m + b of Makhoul's reordered sequence, v < N/2 -> n = 2 v, else n = 2 (N - 1 - v) + 1.
__device__ __forceinline__ int n_of_slot_pow2(const Geo& g, int sigma) {
  const int m = (sigma >> 1) * g.P + g.c;
  const int v = 2 * m + (sigma & 1);
  return v < (g.N >> 1) ? 2 * v : 2 * (g.N - 1 - v) + 1;
}
__device__ __forceinline__ int n_of_slot(const Geo& g, int sigma) { return g.nat ? sigma : n_of_slot_pow2(g, sigma); }
__device__ __forceinline__ void slot_of_n(const Geo& g, int n, int& owner, int& sigma) {
  if (g.nat) {
    owner = 0;
    sigma = n;
    return;
  }
  const int v = (n & 1) ? g.N - 1 - (n >> 1) : (n >> 1);
  const int m = v >> 1;
  owner = m & (g.P - 1);
  sigma = 2 * (m / g.P) + (v & 1);
}
__device__ __forceinline__ float sgn_bits(const uint32_t* signw, int sigma) {
  return (signw[sigma >> 5] >> (sigma & 31)) & 1u ? -1.0f : 1.0f;
}
// Index of x (the signal) held by slot sigma: the DCT input index itself under the sign
// randomiser, perm[n] under the permutation randomiser R (Sec. III-A), whose DCT input n is
// x[perm[n]].  slot_of_sig inverts it.
__device__ __forceinline__ int sig_of_slot(const Geo& g, int sigma) {
  const int n = n_of_slot(g, sigma);
  const int32_t* perm = C.op.perm;
  return perm ? __ldg(perm + n) : n;
}
__device__ __forceinline__ void slot_of_sig(const Geo& g, int j, int& owner, int& sigma) {
  const int32_t* iperm = C.op.iperm;
  slot_of_n(g, iperm ? __ldg(iperm + j) : j, owner, sigma);
}
__device__ __forceinline__ bool mask_bit(const uint32_t* m, int sigma) { return (m[sigma >> 5] >> (sigma & 31)) & 1u; }

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

// Frequency slot k_q held by slot s of CTA c (mirror-paired assignment).
__device__ __forceinline__ int kq_of(const Geo& g, int s) {
  if (s < g.h) return g.c * g.h + s;
  const int j = g.c * g.h + s - g.h;
  return j == 0 ? (g.F >> 1) : g.F - j;
}
__device__ __forceinline__ void owner_of_kq(const Geo& g, int k, int& c, int& s) {
  const int Q = g.F;
  if (k < (Q >> 1)) { c = k >> g.lh; s = k - (c << g.lh); }
  else if (k == (Q >> 1)) { c = 0; s = g.h; }
  else { const int j = Q - k; c = j >> g.lh; s = g.h + (j - (c << g.lh)); }
}

// Frequency task t of this CTA -> the slot pair holding (Z_k, Z_{L-k}).  Tasks [0, h P) walk
// the (slot, k_p) grid of the lower half; CTA 0 skips its slot 0 there and instead runs P + 1
// tasks for its two self-mirrored columns (k_q = 0 and k_q = Q/2).  Returns false for a skip.
__device__ __forceinline__ int ntasks(const Geo& g) { return g.h * g.P + (g.c == 0 ? g.P + 1 : 0); }
__device__ __forceinline__ bool task_pair(const Geo& g, int t, int& sa, int& kpa, int& sb, int& kpb) {
  const int P = g.P, h = g.h;
  const int reg = h * P;
  if (t < reg) {
    sa = t & (h - 1);
    kpa = t >> g.lh;
    if (g.c == 0 && sa == 0) return false;
    sb = sa + h;
    kpb = P - 1 - kpa;
    return true;
  }
  const int u = t - reg;
  const int ncol0 = P > 1 ? P / 2 + 1 : 1;
  if (u < ncol0) { sa = 0; kpa = u; sb = 0; kpb = (P - u) & (P - 1); }
  else { const int v = u - ncol0; sa = h; kpa = v; sb = h; kpb = P - 1 - v; }
  return true;
}
// The DCT output indices produced by the pair whose first FFT bin is k.
__device__ __forceinline__ int pair_outputs(const Geo& g, int k, bool self, int* f) {
  if (k == 0) { f[0] = 0; f[1] = g.L; return 2; }
  if (self) { f[0] = k; f[1] = g.N - k; return 2; }
  f[0] = k; f[1] = g.N - k; f[2] = g.L + k; f[3] = g.L - k;
  return 4;
}

// Geometry of column block b in the frequency-stage conventions: P = S2 column-FFT outputs,
// F = S1 (Q), 2h = W slots, block index in the role of the CTA rank.
__device__ __forceinline__ Geo block_geo(const OpDev& op, int b) {
  Geo gb;
  gb.N = op.N; gb.L = op.N >> 1; gb.P = op.S2; gb.F = op.S1;
  gb.h = op.W >> 1; gb.lh = __ffs(gb.h) - 1; gb.S2 = op.W; gb.c = b; gb.four_n = 4 * op.N;
  return gb;
}

// ---------------------------------------------------------------- cluster-wide reductions
// Sum n (<= 4) per-thread values over the whole cluster; every thread gets the totals, and
// every CTA adds the partials in rank order, so all CTAs hold bit-identical results.
__device__ __noinline__ void cluster_sum(float* v, int n) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* wsum = shp(C.sm.wsum);
  for (int i = 0; i < n; ++i) {
    const float s = warp_sum(v[i]);
    if (lane == 0) wsum[i * 16 + warp] = s;
  }
  const int slot = C.ring_slot;                    // read by every thread before the barrier
  __syncthreads();
  float* ring = shp(C.sm.ring) + 4 * slot;
  const bool grid = C.grid;
  const int G = C.g.P;
  float* gred = grid ? C.op.gred + (size_t)slot * G * 4 : nullptr;
  if (threadIdx.x < n) {
    float t = 0.f;
    for (int w = 0; w < NT / 32; ++w) t += wsum[threadIdx.x * 16 + w];
    if (grid) gred[C.g.c * 4 + threadIdx.x] = t;
    else ring[threadIdx.x] = t;
  }
  if (threadIdx.x == 0) C.ring_slot = (slot + 1) & 3;   // next reader is past the barriers below
  group_sync();
  float* fscr = shp(C.sm.fscr);
  if (warp == 0) {
    for (int i = 0; i < n; ++i) {
      float t = 0.f;
      if (grid) {
        for (int r = lane; r < G; r += 32) t += __ldcg(gred + r * 4 + i);
      } else if (lane < G) {
        t = *cl_map(ring + i, lane);
      }
      // fixed lane assignment and fixed-shape tree: identical order in every CTA
      t = warp_sum(t);
      if (lane == 0) fscr[i] = t;
    }
  }
  __syncthreads();
  for (int i = 0; i < n; ++i) v[i] = fscr[i];
}

// A cluster-wide sum split around a barrier that the caller already has: reduce_publish
// stores this CTA's partial of v (fixed-order warp tree, then the warps in order) in the next
// ring slot (grid launches: the partials array) and returns the slot; after a cluster (grid)
// barrier that every CTA passes after publishing, reduce_collect adds the partials in rank order,
// so every CTA holds the bit-identical total.  Saves the barrier of a separate cluster_sum.
__device__ __noinline__ int reduce_publish(float v) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* wsum = shp(C.sm.wsum);
  const float s = warp_sum(v);
  if (lane == 0) wsum[warp] = s;
  const int slot = C.ring_slot;                    // read by every thread before the barrier
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < NT / 32; ++w) t += wsum[w];
    if (C.grid) C.op.gred[(size_t)slot * C.g.P * 4 + C.g.c * 4] = t;
    else shp(C.sm.ring)[4 * slot] = t;
    C.ring_slot = (slot + 1) & 3;                  // next reader is past the caller's barrier
  }
  return slot;
}
__device__ __noinline__ float reduce_collect(int slot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* fscr = shp(C.sm.fscr);
  const int G = C.g.P;
  if (warp == 0) {
    float t = 0.f;
    if (C.grid) {
      const float* gred = C.op.gred + (size_t)slot * G * 4;
      for (int r = lane; r < G; r += 32) t += __ldcg(gred + r * 4);
    } else if (lane < G) {
      t = *cl_map(shp(C.sm.ring) + 4 * slot, lane);
    }
    t = warp_sum(t);
    if (lane == 0) fscr[4] = t;
  }
  __syncthreads();
  const float r = fscr[4];
  __syncthreads();
  return r;
}

// Max of up to two 64-bit keys over the cluster.
__device__ __noinline__ void cluster_max64(unsigned long long* v, int n) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long* wmax = shp(C.sm.wmax);
  for (int i = 0; i < n; ++i) {
    const unsigned long long s = warp_max64(v[i]);
    if (lane == 0) wmax[i * 16 + warp] = s;
  }
  const int slot = C.ring_slot;
  __syncthreads();
  unsigned long long* ring = shp(C.sm.ring64) + 2 * slot;
  const bool grid = C.grid;
  const int G = C.g.P;
  unsigned long long* gred = grid ? C.op.gred64 + (size_t)slot * G * 2 : nullptr;
  if (threadIdx.x < n) {
    unsigned long long t = 0;
    for (int w = 0; w < NT / 32; ++w) t = max(t, wmax[threadIdx.x * 16 + w]);
    if (grid) gred[C.g.c * 2 + threadIdx.x] = t;
    else ring[threadIdx.x] = t;
  }
  if (threadIdx.x == 0) C.ring_slot = (slot + 1) & 3;
  group_sync();
  int* iscr = shp(C.sm.iscr);
  if (warp == 0) {
    for (int i = 0; i < n; ++i) {
      unsigned long long t = 0;
      if (grid) {
        for (int r = lane; r < G; r += 32) t = max(t, __ldcg(gred + r * 2 + i));
      } else if (lane < G) {
        t = *cl_map(ring + i, lane);
      }
      t = warp_max64(t);
      if (lane == 0) iscr[2 * i] = (int)(t & 0xffffffffu), iscr[2 * i + 1] = (int)(t >> 32);
    }
  }
  __syncthreads();
  for (int i = 0; i < n; ++i)
    v[i] = ((unsigned long long)(uint32_t)iscr[2 * i + 1] << 32) | (uint32_t)iscr[2 * i];
  __syncthreads();
}

// Exclusive block scan of one int per thread; returns the exclusive prefix, total via *tot.
__device__ __noinline__ int block_scan(int v, int* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* iscr = shp(C.sm.iscr);
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) iscr[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int w = lane < NT / 32 ? iscr[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < NT / 32) iscr[32 + lane] = wi - w;
    if (lane == 31) iscr[63] = wi;
  }
  __syncthreads();
  const int ex = iscr[32 + warp] + inc - v;
  *tot = iscr[63];
  __syncthreads();
  return ex;
}

// Rebuild this CTA's sorted support list (local slots) from a bitmask; returns its length.
// The list and the CG vectors go to shared memory when this CTA's share fits, else to the
// global fallback arrays (a per-CTA choice; no barrier depends on it).
__device__ __noinline__ int build_list(const uint32_t* m) {
  // total first (to choose the destination), then a chunked ordered compaction
  int total = 0;
  for (int w0 = 0; w0 < C.nwords; w0 += NT) {
    const int w = w0 + threadIdx.x;
    int t;
    block_scan(w < C.nwords ? __popc(m[w]) : 0, &t);
    total += t;
  }
  const bool on_chip = total <= C.cap;
  int* list = on_chip ? shp(C.sm.cgl) : C.glist;
  float* cg = on_chip ? shp(C.sm.cgv) : C.gcg;
  const int stride = on_chip ? C.cap : 2 * C.g.F;
  if (threadIdx.x == 0) {   // read by the callers after this function's final barrier
    C.list = list;
    C.cgx = cg;
    C.cgr = cg + stride;
    C.cgp = cg + 2 * stride;
    C.cgq = cg + 3 * stride;
  }
  int base = 0;
  for (int w0 = 0; w0 < C.nwords; w0 += NT) {
    const int w = w0 + threadIdx.x;
    const uint32_t word = w < C.nwords ? m[w] : 0u;
    int t;
    int off = base + block_scan(__popc(word), &t);
    uint32_t bitsleft = word;
    while (bitsleft) {
      const int b = __ffs(bitsleft) - 1;
      bitsleft &= bitsleft - 1;
      list[off++] = w * 32 + b;
    }
    base += t;
  }
  __syncthreads();
  return total;
}

// Omega bits of this CTA's frequency tasks on the streamed path: shared memory, or for
// N = 2^24 (whose plan has no room left) the CTA's slice of a global table.
__device__ __forceinline__ uint8_t* grid_fbits() {
  return C.op.gfb ? C.op.gfb + (size_t)C.g.c * C.op.gfb_stride : shp(C.sm.fbits);
}

// Omega membership bits of every frequency task of this CTA (bit i <-> output f[i]).
__device__ __noinline__ void build_fbits() {
  if (C.grid) {
    // one table per column block of this CTA, each of h S2 + S2 + 1 entries
    const OpDev& op = C.op;
    const int fbstride = (op.W / 2) * op.S2 + op.S2 + 1;
    uint8_t* fb0 = grid_fbits();
    for (int j = 0; j < op.bpc; ++j) {
      const Geo gb = block_geo(op, C.g.c + j * op.G);
      uint8_t* fb = fb0 + j * fbstride;
      const int nt = ntasks(gb);
      for (int t = threadIdx.x; t < nt; t += NT) {
        int sa, kpa, sb, kpb;
        uint8_t bits = 0;
        if (task_pair(gb, t, sa, kpa, sb, kpb)) {
          const int k = kq_of(gb, sa) + gb.F * kpa;
          int f[4];
          const int nf = pair_outputs(gb, k, sa == sb && kpa == kpb, f);
          for (int i = 0; i < nf; ++i) bits |= (uint8_t)(((C.omask[f[i] >> 5] >> (f[i] & 31)) & 1u) << i);
        }
        fb[t] = bits;
      }
    }
    __syncthreads();
    return;
  }
  // cluster launches also store the rank in Omega of every kept output (the position of its
  // value in y), so the frequency stage reads or writes y without touching omask / orank
  const Geo g = C.g;
  uint8_t* fb = shp(C.sm.fbits);
  int4* rank4 = C.rank4;
  const uint32_t* omask = C.omask;
  const int32_t* orank = C.orank;
  const int nt = ntasks(g);
  for (int t = threadIdx.x; t < nt; t += NT) {
    int sa, kpa, sb, kpb;
    uint8_t bits = 0;
    int rk[4] = {-1, -1, -1, -1};
    if (task_pair(g, t, sa, kpa, sb, kpb)) {
      const int k = kq_of(g, sa) + g.F * kpa;
      int f[4];
      const int nf = pair_outputs(g, k, sa == sb && kpa == kpb, f);
      for (int i = 0; i < nf; ++i) {
        const uint32_t w = omask[f[i] >> 5];
        if ((w >> (f[i] & 31)) & 1u) {
          bits |= (uint8_t)(1u << i);
          rk[i] = orank[f[i] >> 5] + __popc(w & ((1u << (f[i] & 31)) - 1u));
        }
      }
    }
    fb[t] = bits;
    rank4[t] = make_int4(rk[0], rk[1], rk[2], rk[3]);
  }
  __syncthreads();
  // the task order of the frequency stage: a stable partition, tasks with a kept output first
  // (every thread takes a contiguous chunk; deterministic, so every run gets the same order)
  uint16_t* perm = shp(C.sm.tperm);
  const int per = (nt + NT - 1) / NT;
  const int t0 = min(nt, (int)threadIdx.x * per), t1 = min(nt, t0 + per);
  int cnt = 0;
  for (int t = t0; t < t1; ++t) cnt += fb[t] != 0;
  int total;
  int pnz = block_scan(cnt, &total);
  int pz = total + (t0 - pnz);
  for (int t = t0; t < t1; ++t) {
    if (fb[t] != 0) perm[pnz++] = (uint16_t)t;
    else perm[pz++] = (uint16_t)t;
  }
  if (threadIdx.x == 0) C.tnz = total;
  __syncthreads();
}

// ------------------------------------------------------------------- the transform pair
// Forward half: scatter (W x, sign flip d and Makhoul's reordering are all in the slot map),
// local Q-point FFT, cluster barrier, then the all-to-all pull fused with the P-point DFT:
// the thread that owns frequency slot s loads A_p[k_q(s)] from every CTA p, multiplies by
// omega_L^{p k_q} = (omega_L^{k_q})^p and transforms over p in registers.
template <int PT>
__device__ __forceinline__ void pull_fwd(const Geo& g, const Tw& tw, float2* A, float2* B) {
  for (int s = threadIdx.x; s < g.S2; s += NT) {
    const int k = kq_of(g, s);
    float2 v[PT];
#pragma unroll
    for (int p = 0; p < PT; ++p) v[p] = cl_map(A, p)[aidx(k)];
    if constexpr (PT > 1) {
      twiddle_powers<PT, -1>(v, tw, 8 * k);
      dft<PT, -1>(v);
    }
#pragma unroll
    for (int p = 0; p < PT; ++p) B[p * g.S2 + s] = v[p];
  }
}

__device__ __noinline__ void scatter_fwd(int src, int nloc, const float* dense, const float* gin, bool pre2) {
  const Geo g = C.g;
  float2* A = shp(C.sm.A);
  const uint32_t* signw = shp(C.sm.signw);
  const int F = g.F;
  if (src == SRC_GLOBAL_N) {
    // the slots of one CTA are 2P floats apart in x: keep 8 loads in flight per thread
    constexpr int U = 8;
    for (int s0 = threadIdx.x; s0 < 2 * F; s0 += U * NT) {
      float v[U];
#pragma unroll
      for (int e = 0; e < U; ++e) {
        const int sg = s0 + e * NT;
        v[e] = sg < 2 * F ? __ldg(gin + sig_of_slot(g, sg)) : 0.f;
      }
#pragma unroll
      for (int e = 0; e < U; ++e) {
        const int sg = s0 + e * NT;
        if (sg < 2 * F) slot_ref(A, sg) = v[e] * sgn_bits(signw, sg);
      }
    }
  } else {
    // sparse sources: zero the buffer, then place the support values.  With pre2 the values go
    // straight into B in the layout after the FFT's leading radix-2 pass (F = 2^13 plans start
    // with one), Y[2j] = X[j] + X[j + F/2] and Y[2j+1] = X[j] - X[j + F/2], accumulated by
    // shared-memory atomics: an output has two terms at most, so the order cannot change it.
    float2* D = pre2 ? shp(C.sm.B) : A;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4* D4 = reinterpret_cast<float4*>(D);
    for (int q = threadIdx.x; q < apad(F) / 2; q += NT) D4[q] = z4;
    __syncthreads();
    const int* list = C.list;
    float* vals = C.cgp;
    const float* rv = C.cgr;
    const bool upd = src == SRC_CG && C.cg_fuse;
    const float beta = C.cg_beta;
    float* Df = reinterpret_cast<float*>(D);
    const int half = F >> 1;
    for (int i = threadIdx.x; i < nloc; i += NT) {
      const int sg = list[i];
      float pv = src == SRC_CG ? vals[i] : dense[sg];
      if (upd) {   // the CG direction p = r + beta p, stored back for the step's updates
        pv = fmaf(beta, pv, rv[i]);
        vals[i] = pv;
      }
      const float v = pv * sgn_bits(signw, sg);
      if (pre2) {
        const int q = sg >> 1, b = sg & 1, j = q & (half - 1);
        atomicAdd(Df + 2 * aidx(2 * j) + b, v);
        atomicAdd(Df + 2 * aidx(2 * j + 1) + b, q < half ? v : -v);
      } else {
        slot_ref(A, sg) = v;
      }
    }
  }
  __syncthreads();
}

// Cluster barrier (every CTA's A is final), then the fused pull + P-point DFT into B.
__device__ __noinline__ void exchange_fwd() {
  const Geo g = C.g;
  const Tw tw = smem_tw();
  float2* A = shp(C.sm.A);
  float2* B = shp(C.sm.B);
  cl_sync();
  switch (g.P) {
    case 1: pull_fwd<1>(g, tw, A, B); break;
    case 2: pull_fwd<2>(g, tw, A, B); break;
    case 4: pull_fwd<4>(g, tw, A, B); break;
    case 8: pull_fwd<8>(g, tw, A, B); break;
    default: pull_fwd<16>(g, tw, A, B); break;
  }
  __syncthreads();
}

// Makhoul's pair step between the L-point FFT Z of the reordered, paired sequence and the
// orthonormal DCT-II X (both directions share these twiddles): for the pair (Z_k, Z_{L-k}),
// E and O are the spectra of the even and odd reordered samples, and
//   X_k = w_k Re(omega_{4N}^k (E + omega_N^k O)),  X_{N-k} = -w_k Im(...),
//   X_{L-k} and X_{L+k} likewise from omega_{4N}^{k+L} (E - omega_N^k O).
struct PairTw {
  float2 wk1;   // omega_{4N}^k
  float2 wkL;   // omega_{4N}^{k+L} = omega_{4N}^k e^{-i pi/4}
  float2 w4k;   // omega_{4N}^{4k} = omega_N^k
};
template <class TW>
__device__ __forceinline__ PairTw pair_tw(const TW& tw, int k) {
  PairTw p;
  p.wk1 = tw.get<-1>(k);
  p.wkL = cmul(p.wk1, make_float2(0.70710678118654752f, -0.70710678118654752f));
  const float2 wk2 = cmul(p.wk1, p.wk1);
  p.w4k = cmul(wk2, wk2);
  return p;
}
// DCT-II outputs of the pair: X = {X_k, X_{N-k}, X_{L+k}, X_{L-k}} (k = 0: {X_0, X_L}).
__device__ __forceinline__ void dct2_pair(float2 Za, float2 Zb, int k, const PairTw& p, float wk, float w0,
                                          float* X) {
  const float2 E = cscale(cadd(Za, cconj(Zb)), 0.5f);
  const float2 O = cscale(make_float2(Za.y + Zb.y, Zb.x - Za.x), 0.5f);   // (Za - conj Zb) / 2i
  const float2 tO = cmul(p.w4k, O);
  const float2 u1 = cmul(p.wk1, cadd(E, tO));
  const float2 u2 = cmul(p.wkL, csub(E, tO));
  if (k == 0) { X[0] = w0 * u1.x; X[1] = wk * u2.x; }
  else { X[0] = wk * u1.x; X[1] = -wk * u1.y; X[2] = wk * u2.x; X[3] = -wk * u2.y; }
}
// Inverse (DCT-III pre-processing) with the 1/w_k and 1/L factors folded in: from the pair's
// X values (same order as dct2_pair), the values to store at Z_k (Va) and Z_{L-k} (Vb).
__device__ __forceinline__ void dct3_pair(const float* X, int k, bool self, const PairTw& p, float wk, float w0,
                                          float2& Va, float2& Vb) {
  float X4[4];
  if (k == 0) { X4[0] = X[0]; X4[1] = 0.f; X4[2] = X[1]; X4[3] = X[1]; }
  else if (self) { X4[0] = X[0]; X4[1] = X[1]; X4[2] = X[1]; X4[3] = X[0]; }
  else { X4[0] = X[0]; X4[1] = X[1]; X4[2] = X[2]; X4[3] = X[3]; }
  // (1/w_k)/L = w_k (k >= 1), 2 w_0 (k = 0)
  const float2 u1 = make_float2(X4[0] * (k == 0 ? 2.f * w0 : wk), -X4[1] * wk);
  const float2 u2 = make_float2(X4[2] * wk, -X4[3] * wk);
  const float2 V1 = cmul(cconj(p.wk1), u1);
  const float2 V2 = cmul(cconj(p.wkL), u2);
  const float2 E = cscale(cadd(V1, V2), 0.5f);
  const float2 O = cmul(cscale(csub(V1, V2), 0.5f), cconj(p.w4k));
  Va = cadd(E, cmuli(O));
  Vb = cadd(cconj(E), cmuli(cconj(O)));
}

// Frequency stage: DCT-II post-processing of (Z_k, Z_{L-k}), the Omega step, and DCT-III
// pre-processing back into the pair.  Returns this thread's sum of squares of the MID_RESID
// residual y - A x on Omega, or for MID_MASK of the kept outputs A d on Omega.
// MASK: the kind is MID_MASK (the H d step), compiled without the y-side state.
// PERM: tasks run in the order perm[] (the cluster path's partition); the tasks from position
// nnz on have no output in Omega, so their only effect is zero in the pair's slots (inv).
template <bool MASK, class TW, bool PERM>
__device__ __forceinline__ float freq_core(const Geo& g, float2* B, const uint8_t* fb, const int4* rank4, int kind,
                                           bool fwd_done, bool inv, const float* vin, float* vout,
                                           const uint16_t* perm, int nnz) {
  TW tw;
  smem_tw_into(tw);
  const uint32_t* omask = C.omask;
  const int32_t* orank = C.orank;
  const int F = g.F, S2 = g.S2;
  const float wk = sqrtf(2.0f / (float)g.N), w0 = sqrtf(1.0f / (float)g.N);
  const int nt = ntasks(g);
  float acc = 0.f;
  // Two tasks per iteration: the y-side ranks and loads of both are issued before either
  // task's arithmetic, so their global latencies overlap.
  for (int t0 = threadIdx.x; t0 < nt; t0 += 2 * NT) {
    int rk[2][4];
    float xin[2][4];
    int tt[2];      // task of slot u, -1 past the end
    bool live[2];   // the task has an output in Omega
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = t0 + u * NT;
      tt[u] = i < nt ? (PERM ? (int)perm[i] : i) : -1;
      live[u] = !PERM || i < nnz;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int t = tt[u];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        rk[u][i] = -1;
        xin[u][i] = 0.f;
      }
      if (MASK || t < 0 || !live[u]) continue;
      if (rank4) {
        const int4 r = rank4[t];
        rk[u][0] = r.x; rk[u][1] = r.y; rk[u][2] = r.z; rk[u][3] = r.w;
      } else {
        int sa, kpa, sb, kpb;
        if (task_pair(g, t, sa, kpa, sb, kpb)) {
          const int k = kq_of(g, sa) + F * kpa;
          int f[4];
          const int nf = pair_outputs(g, k, sa == sb && kpa == kpb, f);
          const uint32_t bits = fb[t];
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (i < nf && ((bits >> i) & 1u))
              rk[u][i] = orank[f[i] >> 5] + __popc(omask[f[i] >> 5] & ((1u << (f[i] & 31)) - 1u));
        }
      }
    }
    if (!MASK && (kind == MID_RESID || kind == MID_IN)) {
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (rk[u][i] >= 0) xin[u][i] = __ldg(vin + rk[u][i]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int t = tt[u];
      if (t < 0) continue;
      int sa, kpa, sb, kpb;
      if (!task_pair(g, t, sa, kpa, sb, kpb)) continue;
      const bool self = (sa == sb) && (kpa == kpb);
      if (!live[u]) {   // no output in Omega: the pre-processing of zeros
        if (inv) {
          B[kpa * S2 + sa] = make_float2(0.f, 0.f);
          if (!self) B[kpb * S2 + sb] = make_float2(0.f, 0.f);
        }
        continue;
      }
      const int k = kq_of(g, sa) + F * kpa;
      const PairTw pt = pair_tw(tw, k);
      float X[4] = {0.f, 0.f, 0.f, 0.f};
      if (fwd_done) dct2_pair(B[kpa * S2 + sa], B[kpb * S2 + sb], k, pt, wk, w0, X);
      if (MASK) {
        const uint32_t bits = fb[t];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (!((bits >> i) & 1u)) X[i] = 0.f;
          acc = fmaf(X[i], X[i], acc);             // ||P_Omega A W d||^2 = d^T H d (Parseval)
        }
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const bool in = rk[u][i] >= 0;
          if (kind == MID_RESID) {
            X[i] = in ? xin[u][i] - X[i] : 0.f;
            acc = fmaf(X[i], X[i], acc);
          } else if (kind == MID_OUT) {
            if (in) vout[rk[u][i]] = X[i];
          } else {   // MID_IN
            X[i] = in ? xin[u][i] : 0.f;
          }
        }
      }
      if (inv) {
        float2 Va, Vb;
        dct3_pair(X, k, self, pt, wk, w0, Va, Vb);
        B[kpa * S2 + sa] = Va;
        if (!self) B[kpb * S2 + sb] = Vb;
      }
    }
  }
  __syncthreads();
  return acc;
}

template <bool MASK>
__device__ __noinline__ float freq_half_k(int kind, bool fwd_done, bool inv, const float* vin, float* vout) {
  const Geo g = C.g;
  return freq_core<MASK, Tw, true>(g, shp(C.sm.B), shp(C.sm.fbits), C.rank4, kind, fwd_done, inv, vin, vout,
                                   shp(C.sm.tperm), C.tnz);
}
__device__ __forceinline__ float freq_half(int kind, bool fwd_done, bool inv, const float* vin, float* vout) {
  return kind == MID_MASK ? freq_half_k<true>(kind, fwd_done, inv, vin, vout)
                          : freq_half_k<false>(kind, fwd_done, inv, vin, vout);
}

// Inverse exchange: P-point inverse DFT per column, then an all-to-all PUSH back into the
// stride-P layout: row p of this CTA's columns goes to CTA p's A at k = k_q(s), times
// conj(omega_L^{p k}).  Remote stores do not stall the issuing warp the way remote loads do,
// and no barrier is needed before them: CTA p's A is the source of the forward pull, and the
// only slots written here (this CTA's own k_q) are the ones this CTA already pulled.  The
// caller's cluster barrier after this function makes every push visible before the inverse
// FFT reads A.
__device__ __noinline__ void exchange_inv() {
  const Geo g = C.g;
  const Tw tw = smem_tw();
  float2* A = shp(C.sm.A);
  float2* B = shp(C.sm.B);
  const int F = g.F, S2 = g.S2;
  pstep<1>(B, g.P, S2);
  {
    constexpr int EPT = F_MAX / NT;
    const int ls2 = g.lh + 1;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int idx = threadIdx.x + e * NT;
      if (idx < F) {
        const int p = idx >> ls2;
        const int s = idx & (S2 - 1);
        const int k = kq_of(g, s);
        float2 v = B[idx];
        if (p != 0) v = cmul(v, tw.get<1>(8 * p * k));
        cl_map(A, p)[aidx(k)] = v;
      }
    }
  }
}

// ------------------------------------------------------ streamed transform (grid launches)
// L = S1 S2 with rows of S1 points: z[m] with m = S2 n1 + n2 is element (n2, n1).  Pass 1 runs
// the S1-point FFT of each row and multiplies by omega_L^{n2 k1}; pass 2 runs the S2-point
// FFT of each column k1, so Z[k1 + S1 k2] = column k1, entry k2.  Columns are processed in
// blocks of W that pair k1 with its mirror S1 - k1 (the same assignment as the cluster
// layout, with the block index in the role of the CTA rank), so the DCT post-/pre-processing
// of every pair (k, L - k) stays inside one block.  Intermediate rows live in global memory
// (L2-resident), signal-domain rows in each CTA's own global rows.

// One out-of-place Stockham pass over the first index of a [Lc][W] array (W contiguous).
template <int R, int DIR>
__device__ __forceinline__ void col_pass(const float2* X, float2* Y, int Lc, int lw, int Ns, const TwQ& tw, int four_n) {
  const int W = 1 << lw;
  const int nb = Lc / R;
  const int total = nb << lw;
  for (int t = threadIdx.x; t < total; t += NT) {
    const int sidx = t & (W - 1), j = t >> lw;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = X[((j + r * nb) << lw) + sidx];
    const int k = j & (Ns - 1);
    if (Ns > 1) twiddle_powers<R, DIR>(v, tw, k * (four_n / (Ns * R)));
    dft<R, DIR>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) Y[((base + r * Ns) << lw) + sidx] = v[r];
  }
  __syncthreads();
}

template <int LOGL, int DIR, int LOGNS, bool TO_Y>
__device__ __forceinline__ void col_rest(float2* X, float2* Y, int lw, const TwQ& tw, int four_n) {
  if constexpr (LOGNS < LOGL) {
    if constexpr (TO_Y) col_pass<16, DIR>(X, Y, 1 << LOGL, lw, 1 << LOGNS, tw, four_n);
    else col_pass<16, DIR>(Y, X, 1 << LOGL, lw, 1 << LOGNS, tw, four_n);
    col_rest<LOGL, DIR, LOGNS + 4, !TO_Y>(X, Y, lw, tw, four_n);
  } else if constexpr (!TO_Y) {
    // odd number of passes: the result is in Y, copy it back to X
    const int n = (1 << LOGL) << lw;
    for (int i = threadIdx.x; i < n; i += NT) X[i] = Y[i];
    __syncthreads();
  }
}

// Batched FFT of length Lc = 2^LOGL along the first index of X [Lc][W]; Y is scratch.
template <int LOGL, int DIR>
__device__ __forceinline__ void col_plan(float2* X, float2* Y, int lw, const TwQ& tw, int four_n) {
  constexpr int HEAD = LOGL % 4;
  constexpr int R0 = HEAD == 0 ? 16 : (1 << HEAD);
  col_pass<R0, DIR>(X, Y, 1 << LOGL, lw, 1, tw, four_n);
  col_rest<LOGL, DIR, (HEAD ? HEAD : 4), false>(X, Y, lw, tw, four_n);
}

template <int DIR>
__device__ __noinline__ void col_fft(float2* X, float2* Y, int Lc, int lw, TwQ tw, int four_n) {
  X = shp(X);
  Y = shp(Y);
  tw.lo = shp(tw.lo);
  tw.hi = shp(tw.hi);
  switch (__ffs(Lc) - 1) {
    case 5: col_plan<5, DIR>(X, Y, lw, tw, four_n); break;
    case 6: col_plan<6, DIR>(X, Y, lw, tw, four_n); break;
    case 7: col_plan<7, DIR>(X, Y, lw, tw, four_n); break;
    case 8: col_plan<8, DIR>(X, Y, lw, tw, four_n); break;
    case 9: col_plan<9, DIR>(X, Y, lw, tw, four_n); break;
    case 10: col_plan<10, DIR>(X, Y, lw, tw, four_n); break;
    default: col_plan<11, DIR>(X, Y, lw, tw, four_n); break;
  }
}

// Pass 1, forward, row lr of this CTA (n2 = c + lr G): build the row from the source, FFT,
// multiply by omega_L^{n2 k1} and store it.  Element k1 = k0 + e NT uses
// omega_L^{n2 k0} (omega_L^{n2 NT})^e: one strided lookup per thread plus broadcast powers.
__device__ __noinline__ void grid_row_forward(int lr, int src, int nloc, const float* dense, const float* gin) {
  const Geo g = C.g;
  const int S1 = C.op.S1, R = C.op.R, n2 = g.c + lr * C.op.G;
  const int rmask = C.rmask, rshift = C.rshift;
  float2* X = shp(C.sm.A);
  const uint32_t* signw = shp(C.sm.signw);
  if (src == SRC_GLOBAL_N) {
    for (int n1 = threadIdx.x; n1 < S1; n1 += NT) {
      const int q = n1 * R + lr;
      X[aidx(n1)] = make_float2(gin[sig_of_slot(g, 2 * q)] * sgn_bits(signw, 2 * q),
                                gin[sig_of_slot(g, 2 * q + 1)] * sgn_bits(signw, 2 * q + 1));
    }
  } else {
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4* X4 = reinterpret_cast<float4*>(X);
    for (int q = threadIdx.x; q < apad(S1) / 2; q += NT) X4[q] = z4;
    __syncthreads();
    const int* list = C.list;
    const float* vals = src == SRC_CG ? C.cgp : dense;
    for (int i = threadIdx.x; i < nloc; i += NT) {
      const int sg = list[i];
      const int q = sg >> 1;
      if ((q & rmask) != lr) continue;
      const float v = (src == SRC_CG ? vals[i] : vals[sg]) * sgn_bits(signw, sg);
      reinterpret_cast<float*>(X)[2 * aidx(q >> rshift) + (sg & 1)] = v;
    }
  }
  __syncthreads();
  fft_plan_call<GRID_LOG_S1, -1>(C.sm.A, C.sm.B, C.tw, g.four_n);   // S1 = GRID_S1
  {
    const TwQ tw = smem_twq();
    float2* row = C.op.gY + (size_t)n2 * S1;
    float2 w = tw.get<-1>(8 * n2 * (int)threadIdx.x);
    const float2 step = tw.get<-1>(8 * n2 * NT);
    for (int k1 = threadIdx.x; k1 < S1; k1 += NT) {
      row[k1] = cmul(X[aidx(k1)], w);
      w = cmul(w, step);
    }
  }
  __syncthreads();
}

// Pass 2 for column block j of this CTA: load, column FFT, frequency stage, inverse column FFT,
// store.  Returns this thread's MID_RESID partial.
__device__ __noinline__ float grid_col_block(int j, int kind, bool fwd_done, bool inv, const float* vin, float* vout) {
  const OpDev& op = C.op;
  const Geo gb = block_geo(op, C.g.c + j * op.G);
  const int S1 = op.S1, S2 = op.S2, W = op.W, lw = __ffs(W) - 1;
  float2* X = shp(C.sm.A);
  if (fwd_done) {
    // S2 W = GRID_BLOCK entries, all loads of a thread in flight before any store
    constexpr int EPT = GRID_BLOCK / NT;
    float2 v[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int idx = threadIdx.x + e * NT;
      const int n2 = idx >> lw, sidx = idx & (W - 1);
      v[e] = __ldcg(op.gY + (size_t)n2 * S1 + kq_of(gb, sidx));
    }
#pragma unroll
    for (int e = 0; e < EPT; ++e) X[threadIdx.x + e * NT] = v[e];
    __syncthreads();
    col_fft<-1>(C.sm.A, C.sm.B, S2, lw, C.tw, gb.four_n);
  }
  const int fbstride = (W / 2) * S2 + S2 + 1;
  const uint8_t* fbj = grid_fbits() + j * fbstride;
  const float acc = kind == MID_MASK
                        ? freq_core<true, TwQ, false>(gb, X, fbj, nullptr, kind, fwd_done, inv, vin, vout, nullptr, 0)
                        : freq_core<false, TwQ, false>(gb, X, fbj, nullptr, kind, fwd_done, inv, vin, vout, nullptr, 0);
  __syncthreads();
  if (inv) {
    col_fft<1>(C.sm.A, C.sm.B, S2, lw, C.tw, gb.four_n);
    for (int idx = threadIdx.x; idx < (S2 << lw); idx += NT) {
      const int n2 = idx >> lw, sidx = idx & (W - 1);
      op.gY[(size_t)n2 * S1 + kq_of(gb, sidx)] = X[idx];
    }
  }
  __syncthreads();
  return acc;
}

// Pass 1, inverse, row lr: load with conj(omega_L^{n2 k1}), inverse FFT, store the row of
// signal-domain values into this CTA's rows (slot q = n1 R + lr).
__device__ __noinline__ void grid_row_inverse(int lr) {
  const Geo g = C.g;
  const int S1 = C.op.S1, n2 = g.c + lr * C.op.G;
  float2* X = shp(C.sm.A);
  {
    const TwQ tw = smem_twq();
    const float2* row = C.op.gY + (size_t)n2 * S1;
    float2 w = tw.get<1>(8 * n2 * (int)threadIdx.x);
    const float2 step = tw.get<1>(8 * n2 * NT);
    constexpr int EPT = GRID_S1 / NT;   // S1 = GRID_S1; all loads in flight before any use
    float2 v[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) v[e] = __ldcg(row + threadIdx.x + e * NT);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      X[aidx(threadIdx.x + e * NT)] = cmul(v[e], w);
      w = cmul(w, step);
    }
  }
  __syncthreads();
  fft_plan_call<GRID_LOG_S1, 1>(C.sm.A, C.sm.B, C.tw, g.four_n);
  float2* sig = C.sig + (size_t)lr * C.rowstride;
  for (int n1 = threadIdx.x; n1 < S1; n1 += NT) sig[aidx(n1)] = X[aidx(n1)];
  __syncthreads();
}

__device__ __noinline__ float transform_grid(int src, int nloc, const float* dense, const float* gin, int kind, bool inv,
                                             const float* vin, float* vout, bool fuse) {
  if (threadIdx.x == 0) C.ntrans += (src != SRC_NONE ? 1 : 0) + (inv ? 1 : 0);
  if (src != SRC_NONE)
    for (int lr = 0; lr < C.op.R; ++lr) grid_row_forward(lr, src, nloc, dense, gin);
  grid_sync();                                      // every row of pass 1 is stored
  float acc = 0.f;
  for (int j = 0; j < C.op.bpc; ++j) acc += grid_col_block(j, kind, src != SRC_NONE, inv, vin, vout);
  const int slot = fuse ? reduce_publish(acc) : 0;
  grid_sync();                                      // every column block is stored (and every partial)
  if (fuse) acc = reduce_collect(slot);
  if (inv)
    for (int lr = 0; lr < C.op.R; ++lr) grid_row_inverse(lr);
  return acc;
}

// ------------------------------------------------ any-N transform (one CTA, natural order)
// For N not a power of two (16 <= N <= N_MAX_ANY) one CTA holds the signal in natural order
// (slot sigma = signal index sigma) and computes the orthonormal DCT-II and DCT-III as chirp-z
// transforms (Bluestein 1970).  With W = exp(-i pi / N) and the chirp c_m = exp(i pi m^2 / 2N),
//   sum_n a_n W^{nk} = conj(c_k) sum_n (a_n conj(c_n)) c_{k-n}    (0 <= n, k < N),
// a linear convolution done by power-of-two FFTs of czt_n >= 2N - 1 points against a table
// holding the FFT of the chirp kernel (scaled by 1 / czt_n).  Then, with omega = omega_{4N},
//   DCT-II:  X_k = w_k Re(omega^k sum_n x_n W^{nk}),
//   DCT-III: x_n = Re(sum_k (w_k X_k omega^k) W^{kn}),
// and conj(c_m) = omega^{m^2 mod 4N} comes from the operator's omega_{4N} table.
__device__ __forceinline__ int sq_mod(int m, int four_n) { return (int)(((long long)m * m) % four_n); }

// A <- IFFT(FFT(A) . hat): the chirp-z convolution (B is scratch; the result lands in A).
__device__ __noinline__ void czt_conv() {
  local_fft<-1>(C.sm.A, C.sm.B, C.czt_n, C.tw2, 4 * C.czt_n);
  float2* A = shp(C.sm.A);
  const float2* hat = C.czt_hat;
  for (int k = threadIdx.x; k < C.czt_n; k += NT) A[aidx(k)] = cmul(A[aidx(k)], __ldg(hat + k));
  __syncthreads();
  local_fft<1>(C.sm.A, C.sm.B, C.czt_n, C.tw2, 4 * C.czt_n);
}

// One chirp-z DCT stage over A, whose entries' real parts hold N real values (k < N) on entry
// and on exit: TO_FREQ applies the DCT-II, TO_TIME the DCT-III.
enum CztDir : int { TO_FREQ = 0, TO_TIME = 1 };
__device__ __noinline__ void czt_stage(int dir) {
  const int N = C.g.N, Lc = C.czt_n, four_n = C.g.four_n;
  const float wk = sqrtf(2.0f / (float)N), w0 = sqrtf(1.0f / (float)N);
  {
    float2* A = shp(C.sm.A);
    const Tw tw = smem_tw();
    for (int k = threadIdx.x; k < Lc; k += NT) {
      float2 a = make_float2(0.f, 0.f);
      if (k < N) {
        const float v = A[aidx(k)].x;
        const float2 cc = tw.get<-1>(sq_mod(k, four_n));                  // conj(c_k)
        a = dir == TO_FREQ ? cscale(cc, v) : cscale(cmul(tw.get<-1>(k), cc), (k == 0 ? w0 : wk) * v);
      }
      A[aidx(k)] = a;
    }
    __syncthreads();
  }
  czt_conv();
  float2* A = shp(C.sm.A);
  const Tw tw = smem_tw();
  for (int k = threadIdx.x; k < N; k += NT) {
    const float2 o = cmul(tw.get<-1>(sq_mod(k, four_n)), A[aidx(k)]);     // conj(c_k) conv_k
    float v;
    if (dir == TO_FREQ) {
      const float2 om = tw.get<-1>(k);
      v = (k == 0 ? w0 : wk) * fmaf(om.x, o.x, -om.y * o.y);              // w_k Re(omega^k o)
    } else {
      v = o.x;
    }
    A[aidx(k)] = make_float2(v, 0.f);
  }
  __syncthreads();
}

// The sign flip d between the sparsifying basis and the DCT (operators with a basis Psi; the
// others flip the signs on the slots).
__device__ __noinline__ void psi_signs() {
  float2* A = shp(C.sm.A);
  for (int n = threadIdx.x; n < C.g.N; n += NT) {
    const uint64_t h = mix64(C.op.sign_key + (uint64_t)n + 0x9E3779B97F4A7C15ull);
    if (h >> 63) A[aidx(n)].x = -A[aidx(n)].x;
  }
  __syncthreads();
}

// The separable 2-D basis on the real parts of A, read as an n1 x n2 row-major array S:
// TO_TIME applies Psi, S -> C_{n1}^T S C_{n2} (a DCT-III along every row, then every column);
// TO_FREQ applies Psi^T, x -> C_{n1} x C_{n2}^T.  Dense products with the two small DCT-II
// matrices (n1 n2 (n1 + n2) multiply-adds), the real parts of B as the intermediate.
__device__ __noinline__ void psi2d_stage(int dir) {
  const int n1 = C.op.n1, n2 = C.op.n2, N = C.g.N;
  const float* c1 = C.op.c1;
  const float* c2 = C.op.c2;
  float2* A = shp(C.sm.A);
  float2* B = shp(C.sm.B);
  // rows: T[a][j] = sum_b S[a][b] C2[b][j] (DCT-III) or sum_b S[a][b] C2[j][b] (DCT-II)
  for (int e = threadIdx.x; e < N; e += NT) {
    const int a = e / n2, j = e - a * n2;
    float t = 0.f;
    for (int b = 0; b < n2; ++b)
      t = fmaf(A[aidx(a * n2 + b)].x, __ldg(c2 + (dir == TO_TIME ? b * n2 + j : j * n2 + b)), t);
    B[aidx(e)].x = t;
  }
  __syncthreads();
  // columns: x[i][j] = sum_a C1[a][i] T[a][j] (DCT-III) or sum_a C1[i][a] T[a][j] (DCT-II)
  for (int e = threadIdx.x; e < N; e += NT) {
    const int i = e / n2, j = e - i * n2;
    float t = 0.f;
    for (int a = 0; a < n1; ++a)
      t = fmaf(__ldg(c1 + (dir == TO_TIME ? a * n1 + i : i * n1 + a)), B[aidx(a * n2 + j)].x, t);
    A[aidx(e)] = make_float2(t, 0.f);
  }
  __syncthreads();
}

// x -> C d x (no basis) or C d Psi x (basis Psi = C^T, or the 2-D basis): the forward operator
// before the rows are picked, on the real parts of A.
__device__ __forceinline__ void generic_forward() {
  if (C.op.psi) {
    if (C.op.psi == 2) psi2d_stage(TO_TIME);
    else czt_stage(TO_TIME);
    psi_signs();
  }
  czt_stage(TO_FREQ);
}
// The transpose: C^T (no basis; the slot signs are applied by the readers) or Psi^T d C^T.
__device__ __forceinline__ void generic_inverse() {
  czt_stage(TO_TIME);
  if (C.op.psi) {
    psi_signs();
    if (C.op.psi == 2) psi2d_stage(TO_FREQ);
    else czt_stage(TO_FREQ);
  }
}

__device__ __noinline__ float transform_generic(int src, int nloc, const float* dense, const float* gin, int kind,
                                                bool inv, const float* vin, float* vout, bool fuse) {
  const int N = C.g.N, Lc = C.czt_n;
  if (threadIdx.x == 0) C.ntrans += (src != SRC_NONE ? 1 : 0) + (inv ? 1 : 0);
  if (src != SRC_NONE) {
    // the source values (times the slot signs d, which are all +1 with a basis) into A
    float2* A = shp(C.sm.A);
    const uint32_t* signw = shp(C.sm.signw);
    for (int n = threadIdx.x; n < Lc; n += NT) A[aidx(n)] = make_float2(0.f, 0.f);
    __syncthreads();
    if (src == SRC_GLOBAL_N) {
      for (int n = threadIdx.x; n < N; n += NT) A[aidx(n)].x = __ldg(gin + sig_of_slot(C.g, n)) * sgn_bits(signw, n);
    } else {
      const int* list = C.list;
      const float* vals = C.cgp;
      for (int i = threadIdx.x; i < nloc; i += NT) {
        const int n = list[i];
        A[aidx(n)].x = (src == SRC_CG ? vals[i] : dense[n]) * sgn_bits(signw, n);
      }
    }
    __syncthreads();
    generic_forward();
  }
  // the Omega step on X_k = A[k].x (0 when the forward input is zero)
  float acc = 0.f;
  {
    float2* A = shp(C.sm.A);
    const uint32_t* omask = C.omask;
    const int32_t* orank = C.orank;
    for (int k = threadIdx.x; k < N; k += NT) {
      float X = src != SRC_NONE ? A[aidx(k)].x : 0.f;
      const uint32_t wd = omask[k >> 5];
      const bool in = (wd >> (k & 31)) & 1u;
      const int rk = in ? orank[k >> 5] + __popc(wd & ((1u << (k & 31)) - 1u)) : -1;
      if (kind == MID_MASK) {
        X = in ? X : 0.f;
        acc = fmaf(X, X, acc);
      } else if (kind == MID_RESID) {
        X = in ? __ldg(vin + rk) - X : 0.f;
        acc = fmaf(X, X, acc);
      } else if (kind == MID_OUT) {
        if (in) vout[rk] = X;
      } else {   // MID_IN
        X = in ? __ldg(vin + rk) : 0.f;
      }
      A[aidx(k)] = make_float2(X, 0.f);
    }
    __syncthreads();
  }
  if (inv) {
    generic_inverse();
    const float2* A = shp(C.sm.A);
    float* S = reinterpret_cast<float*>(shp(C.sm.S));
    for (int n = threadIdx.x; n < 2 * C.g.F; n += NT) S[2 * aidx(n >> 1) + (n & 1)] = n < N ? A[aidx(n)].x : 0.f;
    __syncthreads();
  }
  if (fuse) {
    const int slot = reduce_publish(acc);
    __syncthreads();
    return reduce_collect(slot);
  }
  return acc;
}

// One application of A (forward), A^T (inverse) or A^T mask A, driven by src / kind.
//   src   SRC_NONE: the forward input is zero (skip the forward transform)
//         SRC_CG: compressed CG vector cgp on the local list (nloc entries)
//         SRC_DENSE_SLOTS: dense-by-slot array `dense` read on the local list
//         SRC_GLOBAL_N: dense signal vector `gin` of length N in global memory
//   kind  frequency step: MID_MASK keeps the Omega rows (H d), MID_RESID forms y - A x on Omega,
//         MID_OUT writes y_M = A x, MID_IN reads u_M (A^T u)
//   inv   run the DCT-III back to the signal domain (result left in the A buffer)
//   fuse  reduce the frequency step's sum of squares over the cluster through the transform's
//         own last barrier and return the total to every thread
// Returns the frequency step's sum of squares (MID_RESID: ||y - A x||^2 on Omega; MID_MASK:
// ||P_Omega A W d||^2 = d^T H d): this thread's share, or with `fuse` the cluster-wide total.
__device__ __noinline__ float transform(int src, int nloc, const float* dense, const float* gin, int kind,
                                        bool inv, const float* vin, float* vout, bool fuse = false) {
  if (C.grid) return transform_grid(src, nloc, dense, gin, kind, inv, vin, vout, fuse);
  if (C.gen) return transform_generic(src, nloc, dense, gin, kind, inv, vin, vout, fuse);
  // Each step is its own call and this function holds almost nothing live across them, so
  // every step gets the full register budget (ptxas allocates registers across calls).
  if (threadIdx.x == 0) C.ntrans += (src != SRC_NONE ? 1 : 0) + (inv ? 1 : 0);
  // B is free at the start of every transform: no other CTA reads it (both exchanges move A),
  // and this CTA's last use of it, the inverse FFT, is over; so the scatter of a sparse source
  // and the forward FFT may use it.
  if (src != SRC_NONE) {
    const bool pre2 = src != SRC_GLOBAL_N && C.g.F == F_MAX;
    scatter_fwd(src, nloc, dense, gin, pre2);
    if (pre2) fft_after_radix2<-1>(C.sm.A, C.sm.B, ctx_tw(), C.g.four_n);
    else local_fft<-1>(C.sm.A, C.sm.B, C.g.F, ctx_tw(), C.g.four_n);
    exchange_fwd();
  } else {
    cl_sync();                                    // every CTA is done with its A before any push
  }
  const float acc = freq_half(kind, src != SRC_NONE, inv, vin, vout);
  const int slot = fuse ? reduce_publish(acc) : 0;
  if (inv) {
    exchange_inv();
    cl_sync();                                    // every push into A has landed; B is scratch again
    if (fuse) {
      const float tot = reduce_collect(slot);     // the partials were published before the barrier
      local_fft<1>(C.sm.A, C.sm.B, C.g.F, ctx_tw(), C.g.four_n);
      return tot;
    }
    local_fft<1>(C.sm.A, C.sm.B, C.g.F, ctx_tw(), C.g.four_n);
  } else {
    cl_sync();                                    // nobody still reads this CTA's A
    if (fuse) return reduce_collect(slot);
  }
  return acc;
}

__device__ __forceinline__ float key_value(uint32_t k) { return k ? __uint_as_float(k - 1u) : 0.f; }

// ---------------------------------------------------------------- margins and the trace
// Selection margins as the oracle defines them: argmax (a_(1) - a_(2)) / a_(1), argmin
// (a_(2) - a_(1)) / a_(2), top-K (a_(K) - a_(K+1)) / a_(K), a comparison test
// |x - x'| / max(x, x'); a margin <= NEAR_TIE is a near-tie.
constexpr float NEAR_TIE = 1e-3f;
__device__ __forceinline__ float test_margin(float x, float xn) {
  const float big = fmaxf(x, xn);
  return big > 0.f ? fabsf(x - xn) / big : 0.f;
}

// Word offset of the next trace record if a record with `payload` words still fits, else -1.
// Every thread calls it before the barriers of the selection it records.
__device__ __forceinline__ int trace_reserve(int payload) {
  if (!C.trace || C.trace_over) return -1;
  const int off = C.trace_off;
  return off + TRACE_HEADER + payload <= C.trace_cap ? off : -1;
}

// Account for one selection or stop test (every thread calls it, after the selection's last
// barrier; cluster-uniform arguments): the near-tie statistics and, with a trace, the record's
// header at `rec` (reserved by trace_reserve, whose payload the selection has written) -- or,
// for rec == RESERVE_HERE, a record without payload reserved now.
constexpr int RESERVE_HERE = -2;
__device__ __noinline__ void note_selection(int kind, float mu, int aux, int rec, int payload) {
  if (threadIdx.x == 0) {
    if (mu <= NEAR_TIE) C.near_ties += 1;
    C.min_margin = fminf(C.min_margin, mu);
    if (C.trace && !C.trace_over) {
      if (rec == RESERVE_HERE)
        rec = C.trace_off + TRACE_HEADER + payload <= C.trace_cap ? C.trace_off : -1;
      if (rec >= 0) {
        if (C.g.c == 0) {
          uint32_t* tr = C.trace + rec;
          tr[0] = (uint32_t)kind;
          tr[1] = (uint32_t)payload;
          tr[2] = __float_as_uint(mu);
          tr[3] = (uint32_t)aux;
        }
        C.trace_off = rec + TRACE_HEADER + payload;
        C.trace_recs += 1;
      } else {
        C.trace_over = 1;
      }
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------ selection
// Radix select (8-bit digits, most significant first) of the K largest nonzero keys over the
// cluster.  On return: keys > *tau are selected and *need more are to be taken among the keys
// equal to *tau; *eq is the cluster-wide count of keys equal to *tau.
template <class KeyFn>
__device__ void radix_select(int count, int K, KeyFn key, uint32_t* tau, int* need, int* eq) {
  uint32_t prefix = 0, pmask = 0;
  int nd = K;
  int last_eq = 0;
  uint32_t* htot = shp(C.sm.htot);
  int* iscr = shp(C.sm.iscr);
  // every thread reads the histogram slot here, before the first barrier; thread 0 then keeps
  // the shared copy one pass ahead (written before each pass's last barrier)
  int hs = C.hist_slot;
  for (int shift = 24; shift >= 0; shift -= 8) {
    uint32_t* hist = shp(C.sm.hist) + 256 * hs;
    if (threadIdx.x < 256) hist[threadIdx.x] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += NT) {
      const uint32_t kk = key(i);
      if (kk != 0u && (kk & pmask) == prefix) atomicAdd(&hist[(kk >> shift) & 255u], 1u);
    }
    const bool grid = C.grid;
    const int G = C.g.P;
    uint32_t* gh = grid ? C.op.ghist + (size_t)hs * G * 256 : nullptr;
    if (grid) {
      __syncthreads();
      if (threadIdx.x < 256) gh[C.g.c * 256 + threadIdx.x] = hist[threadIdx.x];
    }
    group_sync();
    if (threadIdx.x < 256) {
      uint32_t t = 0;
      if (grid) {
        for (int r = 0; r < G; ++r) t += __ldcg(gh + r * 256 + threadIdx.x);
      } else {
        for (int r = 0; r < G; ++r) t += *cl_map(hist + threadIdx.x, r);
      }
      htot[threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // lane l owns digits [8 l, 8 l + 8); suffix sums from the top digit down
      const int lane = threadIdx.x;
      uint32_t mine = 0;
      for (int d = 0; d < 8; ++d) mine += htot[8 * lane + d];
      uint32_t suf = mine;   // inclusive suffix over lanes >= lane
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_down_sync(0xffffffffu, suf, o);
        if (lane + o < 32) suf += t;
      }
      const uint32_t above = suf - mine;   // keys with digit in higher lanes
      // the threshold digit is in the lane with above < nd <= suf
      if (above < (uint32_t)nd && (uint32_t)nd <= suf) {
        uint32_t acc = above;
        int d = 7;
        for (; d > 0; --d) {
          const uint32_t cnt = htot[8 * lane + d];
          if (acc + cnt >= (uint32_t)nd) break;
          acc += cnt;
        }
        iscr[0] = 8 * lane + d;
        iscr[1] = (int)acc;                      // keys strictly above the digit
        iscr[2] = (int)htot[8 * lane + d];       // keys equal to the digit (so far)
      }
      if (lane == 0 && suf < (uint32_t)nd) {     // fewer candidates than requested
        iscr[0] = -1;
        iscr[1] = (int)suf;
        iscr[2] = 0;
      }
    }
    __syncthreads();
    const int dig = iscr[0];
    const int above = iscr[1];
    last_eq = iscr[2];
    hs ^= 1;
    if (threadIdx.x == 0) C.hist_slot = hs;
    __syncthreads();
    if (dig < 0) {   // take every candidate (uniform decision)
      *tau = 0u; *need = 0; *eq = 0;
      return;
    }
    nd -= above;
    prefix |= (uint32_t)dig << shift;
    pmask |= 255u << shift;
  }
  *tau = prefix;
  *need = nd;
  *eq = last_eq;
}

// Select the K largest keys (ties towards the lowest signal index) and call mark(i) for each
// selected index; the second radix pass on the index only runs when the threshold is tied.
// With margins on, the boundary margin (a_(K) - a_(K+1)) / a_(K) is taken from the smallest
// selected and the largest unselected nonzero key, and a trace record stores the selected
// signal indices as an N-bit mask.
template <class KeyFn, class IdxFn, class MarkFn>
__device__ void select_topk(int count, int K, KeyFn key, IdxFn nidx, MarkFn mark) {
  const bool margins = C.want_margins;
  const int tpay = (C.g.N + 31) >> 5;
  const int rec = margins ? trace_reserve(tpay) : -1;   // read before the barriers below
  uint32_t* tbits = rec >= 0 ? C.trace + rec + TRACE_HEADER : nullptr;
  uint32_t tau;
  int need, eq;
  radix_select(count, K, key, &tau, &need, &eq);
  const bool tied = need > 0 && eq > need;
  const uint32_t N = (uint32_t)C.g.N;
  uint32_t tau2 = 0u;
  if (tied) {
    int need2, eq2;
    radix_select(
        count, need, [&](int i) { return key(i) == tau ? N - (uint32_t)nidx(i) : 0u; }, &tau2, &need2, &eq2);
  }
  uint32_t minsel = 0xffffffffu, maxun = 0u;
  for (int i = threadIdx.x; i < count; i += NT) {
    const uint32_t kk = key(i);
    const bool sel = tied ? (kk > tau || (kk == tau && N - (uint32_t)nidx(i) >= tau2)) : (kk != 0u && kk >= tau);
    if (sel) {
      mark(i);
      if (tbits) {
        const int n = nidx(i);
        atomicOr(tbits + (n >> 5), 1u << (n & 31));
      }
      minsel = min(minsel, kk);
    } else if (kk != 0u) {
      maxun = max(maxun, kk);
    }
  }
  __syncthreads();
  if (margins) {
    unsigned long long v[2] = {maxun, 0xffffffffull - minsel};
    cluster_max64(v, 2);
    const float aK = v[1] ? key_value((uint32_t)(0xffffffffull - v[1])) : 0.f;
    const float aK1 = key_value((uint32_t)v[0]);
    note_selection(TR_TOPK, aK > 0.f ? (aK - aK1) / aK : 0.f, K, rec, tpay);
  }
}

__device__ __forceinline__ uint32_t abs_key(float v) { return (__float_as_uint(v) & 0x7fffffffu) + 1u; }

// Correlation c(sigma) = d_n (C^T ...)_n held in the signal buffer.
__device__ __forceinline__ float corr_at(const SigView& sv, const uint32_t* signw, int sg) {
  return sv.at(sg) * sgn_bits(signw, sg);
}

// ------------------------------------------------------------------------------------ CG
enum R0Src : int { R0_FROM_A = 0, R0_FROM_CY = 1 };
constexpr float CG_FP32_FLOOR = 1e-6f;   // relative residual FP32 CG reaches reliably

// Algorithm 1's CG on H = W A^T A W restricted to the support in the local list (Theorem 5's
// |S|-compressed form), b = W A^T y whose by-slot values are in cy.  Start from x0 = xd[wi]
// on the list (warm) or 0, with r0 = b - H x0 taken from the A buffer (R0_FROM_A: the caller
// has just computed A^T (y - A x0)) or from cy (R0_FROM_CY, x0 = 0).  Loop while
// ||r_j|| > tol ||b|| (the printed loop test is read as its negation) and j < maxit.
__device__ __noinline__ void cg_solve(int wi, int nloc, bool warm, int r0src, float tol, int maxit) {
  float* xd = C.xd[wi];
  const float* cy = C.cy;
  const SigView A = sigview();
  const uint32_t* signw = shp(C.sm.signw);
  const int* list = C.list;
  float* cgx = C.cgx;
  float* cgr = C.cgr;
  float* cgp = C.cgp;
  float v[3] = {0.f, 0.f, threadIdx.x == 0 ? (float)nloc : 0.f};   // ||r0||^2, ||b||^2, |S|
  for (int i = threadIdx.x; i < nloc; i += NT) {
    const int sg = list[i];
    const float x0 = warm ? xd[sg] : 0.f;
    const float r0 = r0src == R0_FROM_A ? corr_at(A, signw, sg) : cy[sg];
    const float b = cy[sg];
    cgx[i] = x0;
    cgr[i] = r0;
    cgp[i] = r0;
    v[0] = fmaf(r0, r0, v[0]);
    v[1] = fmaf(b, b, v[1]);
  }
  cluster_sum(v, 3);
  float rr = v[0];
  // Algorithm 1's test on ||r_j||: absolute (the paper's xi) or relative to ||b||; maxit = 0
  // takes Theorem 5's bound of |S| steps.  An absolute xi below what FP32 CG can reach (the
  // paper's exact precision xi = 0, or xi = 1e-10) stops at the FP32 floor ||r_j|| <=
  // CG_FP32_FLOOR ||b||: past it the recursive residual no longer tracks b - H x and the
  // iterate drifts.
  const float stop2 = C.cg_abs ? fmaxf(tol * tol, CG_FP32_FLOOR * CG_FP32_FLOOR * v[1]) : tol * tol * v[1];
  if (maxit == 0) maxit = (int)v[2];
  int it = 0;
  // the cluster path folds the direction update into the next scatter (one pass over the list
  // fewer per step); the streamed and any-N paths update p here
  const bool fuse_p = !C.grid && !C.gen;
  if (threadIdx.x == 0) C.cg_beta = 0.f;   // every thread passed cluster_sum's barriers above
  if (threadIdx.x == 0) C.cg_fuse = fuse_p ? 1 : 0;
  while (it < maxit && rr > stop2) {
    // H d, with d^T H d = ||P_Omega A W d||^2 summed in the frequency step and reduced through
    // the transform's last cluster barrier (one reduction per step fewer than a dot with H d)
    // (on the cluster path the scatter first forms this step's direction p = r + beta p, with
    // the previous step's beta, 0 on the first step where p = r0 already)
    const float pq = transform(SRC_CG, nloc, nullptr, nullptr, MID_MASK, true, nullptr, nullptr, true);
    if (!(pq > 0.f)) break;   // H d = 0 in FP32: the residual is at rounding level (uniform: pq is cluster-wide)
    const float alpha = rr / pq;
    // pointers are re-read from the context after the call (nothing held live across it);
    // one pass gathers q = H d and updates x and r
    const SigView Ax = sigview();
    const uint32_t* sw = shp(C.sm.signw);
    const int* li = C.list;
    float* px = C.cgx;
    float* pr = C.cgr;
    float* pp = C.cgp;
    float rn = 0.f;
    for (int i = threadIdx.x; i < nloc; i += NT) {
      const float q = corr_at(Ax, sw, li[i]);
      px[i] = fmaf(alpha, pp[i], px[i]);
      const float r = fmaf(-alpha, q, pr[i]);
      pr[i] = r;
      rn = fmaf(r, r, rn);
    }
    cluster_sum(&rn, 1);
    const float beta = rn / rr;
    rr = rn;
    if (fuse_p) {
      if (threadIdx.x == 0) C.cg_beta = beta;   // read by the next scatter, past its first barrier
    } else {
      for (int i = threadIdx.x; i < nloc; i += NT) pp[i] = fmaf(beta, pp[i], pr[i]);
    }
    ++it;
  }
  if (threadIdx.x == 0) {
    C.cg_total += it;
    if (it >= maxit && rr > stop2) C.cg_hits += 1;
  }
  {
    const int* li = C.list;
    const float* px = C.cgx;
    float* xo = C.xd[wi];
    for (int i = threadIdx.x; i < nloc; i += NT) xo[li[i]] = px[i];
  }
  __syncthreads();
}

// Residual-correlation: A buffer <- C^T P^T (y - A xd) (unsigned slots), returns ||y - A xd||^2.
__device__ __noinline__ float resid_corr(int wi, int nloc, const float* y) {
  return transform(SRC_DENSE_SLOTS, nloc, C.xd[wi], nullptr, MID_RESID, true, y, nullptr, true);
}

// ------------------------------------------------------------------------ task execution
__device__ __noinline__ void write_recovery(const Task& t, int wi, int nloc, float rn2, int outer) {
  const Geo g = C.g;
  const int N = g.N, P = g.P;
  // zero s_out and the output bitmask (contiguous share per CTA)
  const int per = N / P;
  for (int i = threadIdx.x; i < per; i += NT) t.out[g.c * per + i] = 0.f;
  const int W = (N + 31) / 32;
  const int wper = (W + P - 1) / P;
  for (int i = threadIdx.x; i < wper; i += NT) {
    const int w = g.c * wper + i;
    if (w < W) C.bits[w] = 0u;
  }
  group_sync();
  {
    const int* list = C.list;
    const float* xd = C.xd[wi];
    for (int i = threadIdx.x; i < nloc; i += NT) {
      const int sg = list[i];
      const int n = sig_of_slot(g, sg);
      t.out[n] = xd[sg];
      atomicOr(&C.bits[n >> 5], 1u << (n & 31));
    }
  }
  group_sync();
  // sorted support: CTA c compacts words [c wper, (c+1) wper)
  int cnt = 0;
  for (int i = threadIdx.x; i < wper; i += NT) {
    const int w = g.c * wper + i;
    if (w < W) cnt += __popc(__ldcg(C.bits + w));   // written by other CTAs' atomics
  }
  float fc = (float)cnt;   // counts < 2^24: exact in FP32
  float* ring = shp(C.sm.ring);
  int* iscr = shp(C.sm.iscr);
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* wsum = shp(C.sm.wsum);
    float s = warp_sum(fc);
    if (lane == 0) wsum[warp] = s;
    __syncthreads();
    const int slot = C.ring_slot;   // only thread 0 uses and advances it here
    const bool grid = C.grid;
    float* gred = grid ? C.op.gred + (size_t)slot * P * 4 : nullptr;
    if (threadIdx.x == 0) {
      float tt = 0.f;
      for (int w = 0; w < NT / 32; ++w) tt += wsum[w];
      if (grid) gred[g.c * 4] = tt;
      else ring[4 * slot] = tt;
    }
    group_sync();
    if (threadIdx.x == 0) {
      float off = 0.f;
      for (int r = 0; r < g.c; ++r) off += grid ? __ldcg(gred + r * 4) : *cl_map(ring + 4 * slot, r);
      iscr[40] = (int)off;
      C.ring_slot = (slot + 1) & 3;
    }
    __syncthreads();
  }
  int base = iscr[40];
  __syncthreads();
  // block-ordered compaction: wper words per CTA, processed NT at a time
  for (int w0 = 0; w0 < wper; w0 += NT) {
    const int w = g.c * wper + w0 + threadIdx.x;
    const uint32_t word = (w0 + threadIdx.x < wper && w < W) ? __ldcg(C.bits + w) : 0u;
    int tot;
    int off = base + block_scan(__popc(word), &tot);
    uint32_t b = word;
    while (b) {
      const int j = __ffs(b) - 1;
      b &= b - 1;
      if (off < t.K) t.supp_out[off] = w * 32 + j;
      ++off;
    }
    base += tot;
  }
  if (g.c == 0 && threadIdx.x == 0 && t.stats) {
    cs_stats st;
    st.outer_iters = outer;
    st.cg_iters_total = C.cg_total;
    st.cg_maxit_hits = C.cg_hits;
    st.near_ties = C.near_ties;
    st.final_resid = sqrtf(rn2);
    st.min_margin = C.min_margin;
    st.status = C.grid ? *(volatile int*)C.op.gerr : CS_OK;
    st.transforms = C.ntrans;
    *t.stats = st;
  }
  if (g.c == 0 && threadIdx.x == 0 && C.trace) {
    C.trace[0] = (uint32_t)C.trace_off;
    C.trace[1] = (uint32_t)C.trace_recs;
    C.trace[2] = (uint32_t)C.trace_over;
    C.trace[3] = (uint32_t)((N + 31) >> 5);
  }
}

// A^T y into cy (dense by slot, signed) and the A buffer; returns ||y||^2.
__device__ __noinline__ float init_correlation(const float* y) {
  const float v = transform(SRC_NONE, 0, nullptr, nullptr, MID_RESID, true, y, nullptr, true);
  const SigView A = sigview();
  const uint32_t* signw = shp(C.sm.signw);
  float* cy = C.cy;
  for (int sg = threadIdx.x; sg < 2 * C.g.F; sg += NT) cy[sg] = corr_at(A, signw, sg);
  __syncthreads();
  return v;
}

__device__ void zero_mask(uint32_t* m) {
  for (int w = threadIdx.x; w < C.nwords; w += NT) m[w] = 0u;
  __syncthreads();
}

// Top-K of |c| over the local slots not in `excl` (may be null); marks into `dst`.
__device__ __noinline__ void topk_corr(int K, const uint32_t* excl, uint32_t* dst) {
  const Geo g = C.g;
  const SigView A = sigview();
  select_topk(
      C.nslots, K,
      [&](int sg) -> uint32_t {
        if (excl && mask_bit(excl, sg)) return 0u;
        return abs_key(A.at(sg));
      },
      [&](int sg) { return sig_of_slot(g, sg); },
      [&](int sg) { atomicOr(&dst[sg >> 5], 1u << (sg & 31)); });
}

// OMP argmax step: t = argmax_{j not in S} |c_j| (lowest index on ties); returns the winner's
// signal index or -1 when no candidate is left.  Adds it to the support mask (owner CTA) and
// zeroes its slot of the warm-start vector.
// This thread's largest packed key (|c| key, then the complement of the signal index, so that
// ties go to the lowest index) over its slots outside mA, skipping the key `skip` (0: none).
// NAT: the any-N path's natural slot order (the slot is the signal index).
template <bool NAT>
__device__ __forceinline__ unsigned long long argmax_key(const uint32_t* mA, unsigned long long skip) {
  const Geo g = C.g;
  const SigView A = sigview();
  const int ns = C.nslots;
  const int32_t* perm = C.op.perm;
  unsigned long long key = 0;
  for (int sg = threadIdx.x; sg < ns; sg += NT) {
    if (mask_bit(mA, sg)) continue;
    const int n0 = NAT ? sg : n_of_slot_pow2(g, sg);
    const uint32_t n = (uint32_t)(perm ? __ldg(perm + n0) : n0);   // as sig_of_slot
    const unsigned long long kk = ((unsigned long long)abs_key(A.at(sg)) << 32) | (0xffffffffu - n);
    if (kk != skip && kk > key) key = kk;
  }
  return key;
}

__device__ __noinline__ int omp_select(uint32_t* mA) {
  unsigned long long key = C.gen ? argmax_key<true>(mA, 0ull) : argmax_key<false>(mA, 0ull);
  cluster_max64(&key, 1);
  if (key == 0ull) return -1;   // no candidate left (uniform: key is cluster-reduced)
  const int n = (int)(0xffffffffu - (uint32_t)(key & 0xffffffffu));
  if (C.want_margins) {
    // runner-up over the same candidates: margin (a_(1) - a_(2)) / a_(1)
    unsigned long long k2 = C.gen ? argmax_key<true>(mA, key) : argmax_key<false>(mA, key);
    cluster_max64(&k2, 1);
    const float a1 = key_value((uint32_t)(key >> 32)), a2 = key_value((uint32_t)(k2 >> 32));
    note_selection(TR_ARGMAX, a1 > 0.f ? (a1 - a2) / a1 : 0.f, n, RESERVE_HERE, 0);
  }
  int owner, sg;
  slot_of_sig(C.g, n, owner, sg);
  if (owner == C.g.c && threadIdx.x == 0) {
    mA[sg >> 5] |= 1u << (sg & 31);
    C.xd[0][sg] = 0.f;
  }
  __syncthreads();
  return n;
}

__device__ __noinline__ void run_omp(const Task& t) {
  init_correlation(t.in);
  zero_mask(shp(C.sm.mask[0]));
  int nloc = 0;
  float rn2 = 0.f;
  for (int it = 0; it < t.K; ++it) {
    if (omp_select(shp(C.sm.mask[0])) < 0) break;
    nloc = build_list(shp(C.sm.mask[0]));
    cg_solve(0, nloc, true, R0_FROM_A, t.cg_tol, t.cg_maxit);
    rn2 = resid_corr(0, nloc, t.in);
  }
  write_recovery(t, 0, nloc, rn2, t.K);
}

// SP prune: S' = topK_{j in S~} |u_j| over the working list, marked into mW.
__device__ __noinline__ void sp_prune(int wi, int nW, int K, uint32_t* mW) {
  zero_mask(mW);
  const Geo g = C.g;
  const int* list = C.list;
  const float* xw = C.xd[wi];
  select_topk(
      nW, K, [&](int i) -> uint32_t { return abs_key(xw[list[i]]); },
      [&](int i) { return sig_of_slot(g, list[i]); },
      [&](int i) { const int sg = list[i]; atomicOr(&mW[sg >> 5], 1u << (sg & 31)); });
}

// SP merge: S~ = S u topK_{not in S} |A^T r| into mW, its list, and the warm start x0 = s on S,
// 0 on the new entries.  Returns the list length.
__device__ __noinline__ int sp_merge(int acc, int K) {
  const int wi = acc ^ 1;
  uint32_t* mW = shp(C.sm.mask[wi]);
  const uint32_t* mA = shp(C.sm.mask[acc]);
  for (int w = threadIdx.x; w < C.nwords; w += NT) mW[w] = mA[w];
  __syncthreads();
  topk_corr(K, mA, mW);
  const int nW = build_list(mW);
  const int* list = C.list;
  float* xw = C.xd[wi];
  const float* xa = C.xd[acc];
  for (int i = threadIdx.x; i < nW; i += NT) {
    const int sg = list[i];
    xw[sg] = mask_bit(mA, sg) ? xa[sg] : 0.f;
  }
  __syncthreads();
  return nW;
}

__device__ __noinline__ float mask_diff(int a, int b) {
  const uint32_t* ma = shp(C.sm.mask[a]);
  const uint32_t* mb = shp(C.sm.mask[b]);
  float diff = 0.f;
  for (int w = threadIdx.x; w < C.nwords; w += NT) diff += (float)__popc(ma[w] ^ mb[w]);
  cluster_sum(&diff, 1);
  return diff;
}

__device__ __noinline__ void run_sp(const Task& t) {
  init_correlation(t.in);
  int acc = 0;   // index of the accepted (support, solution) pair
  zero_mask(shp(C.sm.mask[0]));
  topk_corr(t.K, nullptr, shp(C.sm.mask[0]));
  int nloc = build_list(shp(C.sm.mask[0]));
  cg_solve(acc, nloc, false, R0_FROM_CY, t.cg_tol, t.cg_maxit);
  float rn2 = resid_corr(acc, nloc, t.in);
  int rounds = 0;
  while (rounds < t.outer_max) {
    ++rounds;
    const int wi = acc ^ 1;
    int nW = sp_merge(acc, t.K);                     // S~ and its warm start; r0 = c on S~
    cg_solve(wi, nW, true, R0_FROM_A, t.cg_tol, t.cg_maxit);
    sp_prune(wi, nW, t.K, shp(C.sm.mask[wi]));       // S'
    nW = build_list(shp(C.sm.mask[wi]));
    resid_corr(wi, nW, t.in);                        // r0 for x0 = u restricted to S'
    cg_solve(wi, nW, true, R0_FROM_A, t.cg_tol, t.cg_maxit);
    const float rn2_new = resid_corr(wi, nW, t.in);
    const float diff = mask_diff(wi, acc);
    const bool stop = diff == 0.f || rn2_new >= rn2;
    if (C.want_margins)
      note_selection(TR_STOP, diff == 0.f ? 1.f : test_margin(sqrtf(rn2), sqrtf(rn2_new)), stop ? 1 : 0, RESERVE_HERE, 0);
    if (stop) break;
    acc = wi;
    rn2 = rn2_new;
  }
  // the returned pair is `acc`; rebuild its list (the working list may differ)
  nloc = build_list(shp(C.sm.mask[acc]));
  write_recovery(t, acc, nloc, rn2, rounds);
}

// CoSaMP (Needell & Tropp 2009; not treated by the paper, built on the SP machinery):
// S = {}, s = 0, r = y; each round T = S u {the 2K largest |A^T r| over all indices}, b = LS(T)
// (warm-started from s), S' = the K largest |b| on T, s' = b on S' with no second solve,
// r' = y - A s'; SP's stopping rule (S' = S or ||r'|| >= ||r||) keeps (S, s).
__device__ __noinline__ void run_cosamp(const Task& t) {
  init_correlation(t.in);
  int acc = 0;
  zero_mask(shp(C.sm.mask[0]));
  float rn2 = resid_corr(acc, 0, t.in);              // ||y||^2; the A buffer holds A^T y
  int rounds = 0;
  while (rounds < t.outer_max) {
    ++rounds;
    const int wi = acc ^ 1;
    uint32_t* mW = shp(C.sm.mask[wi]);
    const uint32_t* mA = shp(C.sm.mask[acc]);
    for (int w = threadIdx.x; w < C.nwords; w += NT) mW[w] = mA[w];
    __syncthreads();
    topk_corr(2 * t.K, nullptr, mW);                 // T = S u top-2K |A^T r|
    int nW = build_list(mW);
    {
      const int* list = C.list;
      float* xw = C.xd[wi];
      const float* xa = C.xd[acc];
      for (int i = threadIdx.x; i < nW; i += NT) {
        const int sg = list[i];
        xw[sg] = mask_bit(mA, sg) ? xa[sg] : 0.f;    // warm start: s on S, 0 on the new entries
      }
      __syncthreads();
    }
    cg_solve(wi, nW, true, R0_FROM_A, t.cg_tol, t.cg_maxit);   // the A buffer holds A^T r
    sp_prune(wi, nW, t.K, mW);                        // S'
    nW = build_list(mW);
    const float rn2_new = resid_corr(wi, nW, t.in);
    const float diff = mask_diff(wi, acc);
    const bool stop = diff == 0.f || rn2_new >= rn2;
    if (C.want_margins)
      note_selection(TR_STOP, diff == 0.f ? 1.f : test_margin(sqrtf(rn2), sqrtf(rn2_new)), stop ? 1 : 0, RESERVE_HERE, 0);
    if (stop) break;
    acc = wi;
    rn2 = rn2_new;
  }
  const int nloc = build_list(shp(C.sm.mask[acc]));
  write_recovery(t, acc, nloc, rn2, rounds);
}

// OMPR replacement step: z = s + A^T r, j = argmax_{not in S} |z|, i = argmin_{in S} |z|
// (lowest index on ties).  If |z_j| > |z_i| swaps them in the support (owner CTAs), zeroes both
// slots of the warm-start vector and returns true; otherwise returns false.
__device__ __noinline__ bool ompr_swap() {
  const Geo g = C.g;
  const SigView A = sigview();
  const uint32_t* signw = shp(C.sm.signw);
  uint32_t* mA = shp(C.sm.mask[0]);
  unsigned long long key[2] = {0ull, 0ull};
  const float* xd = C.xd[0];
  for (int sg = threadIdx.x; sg < C.nslots; sg += NT) {
    const uint32_t lo = 0xffffffffu - (uint32_t)sig_of_slot(g, sg);
    if (mask_bit(mA, sg)) {
      const float z = xd[sg] + corr_at(A, signw, sg);
      const unsigned long long kk =
          ((unsigned long long)(0xffffffffu - (__float_as_uint(z) & 0x7fffffffu)) << 32) | lo;
      key[1] = kk > key[1] ? kk : key[1];
    } else {
      const unsigned long long kk = ((unsigned long long)abs_key(corr_at(A, signw, sg)) << 32) | lo;
      key[0] = kk > key[0] ? kk : key[0];
    }
  }
  cluster_max64(key, 2);
  const uint32_t zj = (uint32_t)(key[0] >> 32) - 1u;                  // |z_j| bits
  const uint32_t zi = 0xffffffffu - (uint32_t)(key[1] >> 32);         // |z_i| bits
  const bool swap = !(key[0] == 0ull || key[1] == 0ull || zj <= zi);
  const int nj = (int)(0xffffffffu - (uint32_t)(key[0] & 0xffffffffu));
  const int ni = (int)(0xffffffffu - (uint32_t)(key[1] & 0xffffffffu));
  if (C.want_margins && key[0] != 0ull && key[1] != 0ull) {
    // runners-up: the second largest |z| outside S and the second smallest inside
    unsigned long long k2[2] = {0ull, 0ull};
    for (int sg = threadIdx.x; sg < C.nslots; sg += NT) {
      const uint32_t lo = 0xffffffffu - (uint32_t)sig_of_slot(g, sg);
      if (mask_bit(mA, sg)) {
        const float z = xd[sg] + corr_at(A, signw, sg);
        const unsigned long long kk =
            ((unsigned long long)(0xffffffffu - (__float_as_uint(z) & 0x7fffffffu)) << 32) | lo;
        if (kk != key[1] && kk > k2[1]) k2[1] = kk;
      } else {
        const unsigned long long kk = ((unsigned long long)abs_key(corr_at(A, signw, sg)) << 32) | lo;
        if (kk != key[0] && kk > k2[0]) k2[0] = kk;
      }
    }
    cluster_max64(k2, 2);
    const float aj = __uint_as_float(zj), ai = __uint_as_float(zi);
    const float aj2 = key_value((uint32_t)(k2[0] >> 32));
    float mu_i = 1.f;   // a single support entry has nothing to tie with
    if (k2[1] != 0ull) {
      const float ai2 = __uint_as_float(0xffffffffu - (uint32_t)(k2[1] >> 32));
      mu_i = ai2 > 0.f ? (ai2 - ai) / ai2 : (ai2 > ai ? 1.f : 0.f);
    }
    note_selection(TR_ARGMAX, aj > 0.f ? (aj - aj2) / aj : 0.f, nj, RESERVE_HERE, 0);
    note_selection(TR_ARGMIN, mu_i, ni, RESERVE_HERE, 0);
    note_selection(TR_SWAP, test_margin(ai, aj), swap ? 1 : 0, RESERVE_HERE, 0);
  }
  if (!swap) return false;                                             // no improving swap
  int oj, sj, oi, si;
  slot_of_sig(g, nj, oj, sj);
  slot_of_sig(g, ni, oi, si);
  if (threadIdx.x == 0) {
    if (oi == g.c) { mA[si >> 5] &= ~(1u << (si & 31)); C.xd[0][si] = 0.f; }
    if (oj == g.c) { mA[sj >> 5] |= 1u << (sj & 31); C.xd[0][sj] = 0.f; }
  }
  __syncthreads();
  return true;
}

// OMPR(l) replacement step, l > 1 (Jain, Tewari & Dhillon 2011): z = s + A^T r, J = the l
// largest |z| outside S (= |A^T r| there), S' = the K largest |z| over S u J, with the
// lowest-index tie rule of every selection.  If S' != S it becomes the support (mask 0), the
// warm start keeps s on S' and starts the new entries at 0, and the function returns true.
__device__ __noinline__ bool ompr_replace(int l, int K) {
  uint32_t* mA = shp(C.sm.mask[0]);
  uint32_t* mW = shp(C.sm.mask[1]);
  for (int w = threadIdx.x; w < C.nwords; w += NT) mW[w] = mA[w];
  __syncthreads();
  topk_corr(l, mA, mW);                              // S u J
  const int nW = build_list(mW);
  {
    const SigView A = sigview();
    const uint32_t* signw = shp(C.sm.signw);
    const int* list = C.list;
    const float* xa = C.xd[0];
    float* z = C.xd[1];
    for (int i = threadIdx.x; i < nW; i += NT) {
      const int sg = list[i];
      z[sg] = (mask_bit(mA, sg) ? xa[sg] : 0.f) + corr_at(A, signw, sg);
    }
  }
  __syncthreads();
  sp_prune(1, nW, K, mW);                            // S' = topK |z| over S u J
  const bool same = mask_diff(1, 0) == 0.f;
  if (C.want_margins) note_selection(TR_STOP, 1.f, same ? 1 : 0, RESERVE_HERE, 0);   // decided by set equality
  if (same) return false;
  {
    float* xa = C.xd[0];
    for (int w = threadIdx.x; w < C.nwords; w += NT) {
      uint32_t fresh = mW[w] & ~mA[w];
      while (fresh) {
        const int b = __ffs(fresh) - 1;
        fresh &= fresh - 1;
        xa[32 * w + b] = 0.f;
      }
    }
    __syncthreads();
    for (int w = threadIdx.x; w < C.nwords; w += NT) mA[w] = mW[w];
  }
  __syncthreads();
  return true;
}

__device__ __noinline__ void run_ompr(const Task& t) {
  init_correlation(t.in);
  zero_mask(shp(C.sm.mask[0]));
  topk_corr(t.K, nullptr, shp(C.sm.mask[0]));
  int nloc = build_list(shp(C.sm.mask[0]));
  cg_solve(0, nloc, false, R0_FROM_CY, t.cg_tol, t.cg_maxit);
  float rn2 = resid_corr(0, nloc, t.in);
  int swaps = 0;
  const int l = t.ompr_l < t.op.N - t.K ? t.ompr_l : t.op.N - t.K;
  while (swaps < t.outer_max) {
    if (!(l > 1 ? ompr_replace(l, t.K) : ompr_swap())) break;
    ++swaps;
    nloc = build_list(shp(C.sm.mask[0]));
    resid_corr(0, nloc, t.in);   // r0 for x0 = s without i, 0 at j
    cg_solve(0, nloc, true, R0_FROM_A, t.cg_tol, t.cg_maxit);
    rn2 = resid_corr(0, nloc, t.in);
  }
  // a rejected OMPR(l) step leaves the working list of S u J behind: rebuild the list of S
  if (l > 1) nloc = build_list(shp(C.sm.mask[0]));
  write_recovery(t, 0, nloc, rn2, swaps);
}

// Fixed support from a sorted global index list: set the bits this CTA owns.
__device__ __noinline__ void mask_from_support(const int32_t* supp, int k, uint32_t* m) {
  zero_mask(m);
  const Geo g = C.g;
  for (int i = threadIdx.x; i < k; i += NT) {
    const int n = supp[i];
    if (n < 0 || n >= g.N) continue;
    int owner, sg;
    slot_of_sig(g, n, owner, sg);
    if (owner == g.c) atomicOr(&m[sg >> 5], 1u << (sg & 31));
  }
  __syncthreads();
}

__device__ __noinline__ void run_ls_solve(const Task& t) {
  init_correlation(t.in);
  uint32_t* m = shp(C.sm.mask[0]);
  mask_from_support(t.supp_in, t.k_in, m);
  const int nloc = build_list(m);
  cg_solve(0, nloc, false, R0_FROM_CY, t.cg_tol, t.cg_maxit);
  const Geo g = C.g;
  for (int i = threadIdx.x; i < t.k_in; i += NT) {
    const int n = t.supp_in[i];
    if (n < 0 || n >= g.N) continue;
    int owner, sg;
    slot_of_sig(g, n, owner, sg);
    if (owner == g.c) t.out[i] = C.xd[0][sg];
  }
  if (g.c == 0 && threadIdx.x == 0 && t.stats) {
    cs_stats st = {1, C.cg_total, C.cg_hits, 0, -1.f, -1.f, CS_OK, C.ntrans};
    *t.stats = st;
  }
}

__device__ __noinline__ void run_ls_backward(const Task& t) {
  uint32_t* m = shp(C.sm.mask[0]);
  mask_from_support(t.supp_in, t.k_in, m);
  const Geo g = C.g;
  // b = g placed by slot (cy doubles as the right-hand side)
  for (int i = threadIdx.x; i < t.k_in; i += NT) {
    const int n = t.supp_in[i];
    if (n < 0 || n >= g.N) continue;
    int owner, sg;
    slot_of_sig(g, n, owner, sg);
    if (owner == g.c) C.cy[sg] = t.in[i];
  }
  __syncthreads();
  const int nloc = build_list(m);
  cg_solve(0, nloc, false, R0_FROM_CY, t.cg_tol, t.cg_maxit);
  // dy = A_S z
  transform(SRC_DENSE_SLOTS, nloc, C.xd[0], nullptr, MID_OUT, false, nullptr, t.out);
  if (g.c == 0 && threadIdx.x == 0 && t.stats) {
    cs_stats st = {1, C.cg_total, C.cg_hits, 0, -1.f, -1.f, CS_OK, C.ntrans};
    *t.stats = st;
  }
}

// Per-task set-up (geometry, twiddle tables, sign bits, Omega bits) and dispatch.  The task is
// read through a pointer so no copy of it stays in registers across the calls below (ptxas
// allocates registers across calls: whatever a caller holds live is denied to its callees).
__device__ __noinline__ void run_task(const Task* tp, int P, int c, int F_alloc) {
  const OpDev& op = tp->op;
  const bool plan_ok = op.generic ? (C.plan.slot_n >= apad(op.F) && C.plan.fft_n >= op.czt_n &&
                                     C.plan.tw_hi_n >= (1 << op.hi_bits) && C.plan.tw2_lo_n >= (1 << op.tw2_lo_bits) &&
                                     C.plan.tw2_hi_n >= (1 << op.tw2_hi_bits))
                                  : C.plan.slot_n == 0;
  if (op.P != P || op.F > F_alloc || op.grid != C.grid || !plan_ok) {   // host grouping error: skip uniformly
    if (c == 0 && threadIdx.x == 0 && tp->stats) tp->stats->status = CS_ERR_INVALID_ARG;
    return;
  }
  const int nlo = 1 << op.lo_bits, nhi = 1 << op.hi_bits;
  // Twiddles, sign bits and the Omega tables depend only on the operator (and this CTA's fixed
  // rank and cluster size): consecutive tasks on one operator load them once.  Every thread
  // reads the key here, before the first barrier; thread 0 updates it after the last one.
  const bool loaded = C.setup_key == (const void*)op.omask;
  if (threadIdx.x == 0) {   // every CTA thread passed the previous task's barrier
    Geo& g = C.g;
    g.N = op.N; g.L = op.N >> 1; g.P = P; g.F = op.F; g.c = c;
    g.h = op.F / (2 * P); g.lh = __ffs(g.h) - 1; g.S2 = 2 * g.h; g.four_n = 4 * op.N;
    g.nat = op.generic;
    C.gen = op.generic;
    C.nslots = op.generic ? op.N : 2 * op.F;
    C.czt_n = op.czt_n;
    C.czt_hat = op.czt_hat;
    C.op = op;
    if (C.grid) {
      // CTA c owns rows c + lr G (lr < R); slot q = n1 R + lr is point m = q G + c, as in a
      // cluster of G CTAs holding F = R S1 points each
      g.h = 1; g.lh = 0; g.S2 = 2;   // not used by the streamed transform
      C.sig = op.gsig + (size_t)c * op.R * apad(op.S1);
      C.rmask = op.R - 1;
      C.rshift = __ffs(op.R) - 1;
      C.rowstride = apad(op.S1);
    }
    C.M = op.M;
    C.nwords = (2 * op.F + 31) / 32;
    C.omask = op.omask; C.orank = op.orank;
    C.cg_total = 0; C.cg_hits = 0; C.ntrans = 0;
    C.cg_abs = tp->cg_abs;
    const bool rec = tp->mode == MODE_RECOVER;
    C.want_margins = rec && (tp->stats != nullptr || tp->trace != nullptr);
    C.near_ties = 0;
    C.min_margin = 1.f;
    C.trace = rec && tp->trace_cap >= TRACE_HEADER ? tp->trace : nullptr;
    C.trace_cap = tp->trace_cap;
    C.trace_off = TRACE_HEADER;
    C.trace_recs = 0;
    C.trace_over = 0;
    const size_t a = 2 * (size_t)F_alloc;
    C.list = C.glist;
    C.cgx = C.gcg; C.cgr = C.gcg + a; C.cgp = C.gcg + 2 * a; C.cgq = C.gcg + 3 * a;
    C.tw.lo = C.sm.twlo; C.tw.hi = C.sm.twhi; C.tw.lo_bits = op.lo_bits; C.tw.lo_mask = nlo - 1;
    C.tw.mask4n = op.generic ? 0x7fffffff : g.four_n - 1;   // any-N: 4N is no power of two, every index is < 4N
    C.tw.qbits = op.tw_quarter ? __ffs(op.N) - 1 : 31;
    C.tw.qmask = op.tw_quarter ? op.N - 1 : 0x7fffffff;
    if (op.generic) {   // the chirp-z FFT's own table, omega_{4 czt_n}
      C.tw2.lo = C.sm.tw2lo; C.tw2.hi = C.sm.tw2hi; C.tw2.lo_bits = op.tw2_lo_bits;
      C.tw2.lo_mask = (1 << op.tw2_lo_bits) - 1; C.tw2.mask4n = 4 * op.czt_n - 1;
    }
  }
  __syncthreads();
  if (!loaded) {
    // twiddle tables and sign bits
    float2* twlo = shp(C.sm.twlo);
    float2* twhi = shp(C.sm.twhi);
    for (int i = threadIdx.x; i < nlo; i += NT) twlo[aidx(i)] = op.tw[i];
    for (int i = threadIdx.x; i < nhi; i += NT) twhi[i] = op.tw[nlo + i];
    if (op.generic) {
      float2* t2l = shp(C.sm.tw2lo);
      float2* t2h = shp(C.sm.tw2hi);
      const int n2l = 1 << op.tw2_lo_bits, n2h = 1 << op.tw2_hi_bits;
      for (int i = threadIdx.x; i < n2l; i += NT) t2l[aidx(i)] = op.tw2[i];
      for (int i = threadIdx.x; i < n2h; i += NT) t2h[i] = op.tw2[n2l + i];
    }
    uint32_t* signw = shp(C.sm.signw);
    const Geo gg = C.g;
    const int nwords = C.nwords;
    for (int w = threadIdx.x; w < nwords; w += NT) {
      uint32_t bitsw = 0u;
      for (int b = 0; b < 32; ++b) {
        const int sg = 32 * w + b;
        if (sg < 2 * op.F) {
          const uint64_t hsh = mix64(op.sign_key + (uint64_t)n_of_slot(gg, sg) + 0x9E3779B97F4A7C15ull);
          if (!op.perm && !op.psi) bitsw |= (uint32_t)(hsh >> 63) << b;   // permutation / basis: no slot signs
        }
      }
      signw[w] = bitsw;
    }
    __syncthreads();
    if (!op.generic) build_fbits();   // the any-N path reads Omega directly
    if (threadIdx.x == 0) C.setup_key = (const void*)op.omask;
  }
  const Task& t = *tp;
  switch (t.mode) {
    case MODE_APPLY:
      transform(SRC_GLOBAL_N, 0, nullptr, t.in, MID_OUT, false, nullptr, t.out);
      break;
    case MODE_APPLY_T: {
      transform(SRC_NONE, 0, nullptr, nullptr, MID_IN, true, t.in, nullptr);
      const SigView A = sigview();
      const uint32_t* signw = shp(C.sm.signw);
      const Geo gg = C.g;
      for (int sg = threadIdx.x; sg < C.nslots; sg += NT) t.out[sig_of_slot(gg, sg)] = corr_at(A, signw, sg);
      break;
    }
    case MODE_RECOVER:
      if (t.algo == CS_OMP) run_omp(t);
      else if (t.algo == CS_SP) run_sp(t);
      else if (t.algo == CS_COSAMP) run_cosamp(t);
      else run_ompr(t);
      break;
    case MODE_LS_SOLVE: run_ls_solve(t); break;
    case MODE_LS_BACKWARD: run_ls_backward(t); break;
    default: break;
  }
}

__global__ void __launch_bounds__(NT, 1) engine_kernel(const Launch lp) {
  cg::cluster_group cl = cg::this_cluster();
  const int P = (int)cl.num_blocks();
  const int c = (int)cl.block_rank();
  const int cid = blockIdx.x / P;
  const int ncl = gridDim.x / P;
  if (threadIdx.x == 0) {
    C.sm = carve(lp.plan);
    C.plan = lp.plan;
    C.grid = 0;
    C.ring_slot = 0;
    C.hist_slot = 0;
    C.cap = lp.plan.cg_cap;
    float* base = lp.scratch + (size_t)cid * lp.scratch_per_cluster + (size_t)c * scratch_floats_per_cta(lp.F_alloc);
    const size_t a = 2 * (size_t)lp.F_alloc;
    C.xd[0] = base;
    C.xd[1] = base + a;
    C.cy = base + 2 * a;
    C.glist = reinterpret_cast<int*>(base + 3 * a);
    C.gcg = base + 4 * a;
    C.rank4 = reinterpret_cast<int4*>(base + 8 * a);
    C.setup_key = nullptr;
    C.bits = lp.bits + (size_t)cid * lp.bits_per_cluster;
  }
  __syncthreads();
  if (!lp.claim) {
    for (int ti = cid; ti < lp.ntasks; ti += ncl) {
      run_task(lp.tasks ? lp.tasks + ti : &lp.single, P, c, lp.F_alloc);
      cl.sync();
    }
    return;
  }
  // dynamic claiming: rank 0 takes the next task index and every CTA reads it through DSMEM
  // between two cluster barriers (the task list is sorted by work, largest first).  The second
  // barrier also keeps rank 0 resident until every CTA has read its claim: no CTA may exit, or
  // overwrite the claim, while another still reads its shared memory.
  for (;;) {
    if (c == 0 && threadIdx.x == 0) C.next_task = atomicAdd(lp.claim, 1);
    cl.sync();
    const int ti = *cl_map(&C.next_task, 0);
    cl.sync();
    if (ti >= lp.ntasks) break;
    run_task(lp.tasks + ti, P, c, lp.F_alloc);
    cl.sync();
  }
}

// Cooperative launch of G CTAs (one per SM, co-resident) that process one signal of the
// streamed geometry; the task list is walked one task at a time by the whole grid.
__global__ void __launch_bounds__(NT, 1) grid_kernel(const Launch lp) {
  const int G = gridDim.x;
  const int c = blockIdx.x;
  if (threadIdx.x == 0) {
    C.sm = carve(lp.plan);
    C.plan = lp.plan;
    C.grid = 1;
    C.ring_slot = 0;
    C.hist_slot = 0;
    C.cap = lp.plan.cg_cap;
    float* base = lp.scratch + (size_t)c * scratch_floats_per_cta(lp.F_alloc);
    const size_t a = 2 * (size_t)lp.F_alloc;
    C.xd[0] = base;
    C.xd[1] = base + a;
    C.cy = base + 2 * a;
    C.glist = reinterpret_cast<int*>(base + 3 * a);
    C.gcg = base + 4 * a;
    C.rank4 = nullptr;
    C.setup_key = nullptr;
    C.bits = lp.bits;
    C.op = lp.tasks ? lp.tasks[0].op : lp.single.op;   // barrier state for the first task
  }
  __syncthreads();
  for (int ti = 0; ti < lp.ntasks; ++ti) {
    run_task(lp.tasks ? lp.tasks + ti : &lp.single, G, c, lp.F_alloc);
    grid_sync();
  }
}

cudaError_t launch_engine(const Launch& L, int P, int num_clusters, cudaStream_t stream) {
  const size_t smem = smem_bytes(L.plan);
  cudaError_t e = cudaFuncSetAttribute(engine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (P > 8) {
    e = cudaFuncSetAttribute(engine_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P * num_clusters);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, engine_kernel, L);
}

int max_active_clusters(int P, int F_alloc) { return max_active_plan(P, cluster_plan(F_alloc)); }

int max_active_plan(int P, const SmemPlan& plan) {
  const size_t smem = smem_bytes(plan);
  if (cudaFuncSetAttribute(engine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (P > 8 && cudaFuncSetAttribute(engine_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, engine_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_grid(const Launch& L, int G, cudaStream_t stream) {
  const size_t smem = smem_bytes(L.plan);
  cudaError_t e = cudaFuncSetAttribute(grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, grid_kernel, L);
}

int grid_fits(const OpDev& op) {
  const size_t smem = smem_bytes(grid_plan(op));
  if (smem > 227 * 1024) return 0;
  if (cudaFuncSetAttribute(grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grid_kernel, NT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * sms >= op.G ? 1 : 0;
}

// ------------------------------------------- streamed batched operator (one CTA per vector)
// A batch of A x or A^T u with 2^15 <= N <= 2^18: every CTA transforms whole vectors on its
// own, with L = F P (F = STREAM_F, P = L / F) and the decimation-in-frequency split
//   m = n1 + F n2,  k = k2 + P k1:
//   Z[k2 + P k1] = sum_n1 omega_F^{n1 k1} omega_L^{n1 k2} sum_n2 z[n1 + F n2] omega_P^{n2 k2}.
// Column pass: P-point DFTs over n2 for every n1, times omega_L^{n1 k2}, into rows T[k2][n1]
// of the CTA's global buffer (written and read back by the same CTA, L2-resident).  Row pass:
// F-point FFTs of rows k2 and P - k2 in shared memory; together they hold every pair
// (Z_k, Z_{L-k}) of the DCT step.  A^T runs the same passes in reverse order.
// Makhoul's reordering puts z[m] and z[L-1-m] in one 16-byte group of x (m < L/2):
//   x[4m .. 4m+3] = (Re z[m], Im z[L-1-m], Im z[m], Re z[L-1-m])   (times the signs d_n),
// and L-1-m = (F-1-n1) + F (P-1-n2), so a thread that owns the column pair (n1, F-1-n1)
// reads or writes x only in whole, coalesced 16-byte groups.

__device__ __forceinline__ float4 sign4(float4 q, uint32_t bits) {
  q.x = (bits & 1u) ? -q.x : q.x;
  q.y = (bits & 2u) ? -q.y : q.y;
  q.z = (bits & 4u) ? -q.z : q.z;
  q.w = (bits & 8u) ? -q.w : q.w;
  return q;
}
__device__ __forceinline__ uint32_t dbits4(const uint32_t* dbits, int m) {
  return (__ldg(dbits + (m >> 3)) >> ((4 * m) & 31)) & 0xFu;   // signs of x[4m .. 4m+3]
}

// Column pass of A x: x (one vector) -> rows T[k2][n1].
// Bulk copies (TMA) of the intermediate rows from global memory into the row buffers in shared
// memory.  A load completes on an mbarrier with a transaction count; the wait is bounded: one
// that runs out sets the status word and the pass continues, so the launch always ends (the
// caller reports the status).
constexpr long STREAM_TMA_POLLS = 1L << 20;
constexpr size_t STREAM_MBAR_OFF = sizeof(float2) * (3 * (size_t)apad(STREAM_F) + apad(1024) + 1024);
constexpr uint32_t STREAM_ROW_BYTES = sizeof(float2) * apad(STREAM_F);   // one padded row, 69 632 B

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(mbar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  for (long i = 0; i < STREAM_TMA_POLLS; ++i) {
    uint32_t done;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

template <int PT>
__device__ __forceinline__ void stream_cols_fwd(const float4* x4, const uint32_t* dbits, float2* T, const Tw& tw,
                                                int rot, int c, int nc) {
  constexpr int F = STREAM_F;
  const int rs = apad(F);
  for (int jj = c * NT + threadIdx.x; jj < F / 2; jj += nc * NT) {
    const int j = (jj + rot) & (F / 2 - 1);
    const int n1 = j, n1b = F - 1 - j;
    float2 a[PT], b[PT];   // columns n1 and n1b by n2
#pragma unroll
    for (int n2 = 0; n2 < PT / 2; ++n2) {
      const int m = n1 + F * n2, m2 = n1b + F * n2;
      const float4 q = sign4(__ldg(x4 + m), dbits4(dbits, m));
      const float4 q2 = sign4(__ldg(x4 + m2), dbits4(dbits, m2));
      a[n2] = make_float2(q.x, q.z);
      b[PT - 1 - n2] = make_float2(q.w, q.y);
      b[n2] = make_float2(q2.x, q2.z);
      a[PT - 1 - n2] = make_float2(q2.w, q2.y);
    }
    dft<PT, -1>(a);
    twiddle_powers<PT, -1>(a, tw, 8 * n1);   // a[k2] *= omega_L^{n1 k2}
    dft<PT, -1>(b);
    twiddle_powers<PT, -1>(b, tw, 8 * n1b);
#pragma unroll
    for (int k2 = 0; k2 < PT; ++k2) {
      T[k2 * rs + aidx(n1)] = a[k2];
      T[k2 * rs + aidx(n1b)] = b[k2];
    }
  }
}

// Column pass of A^T: rows T[k2][n1] -> x (one vector).
template <int PT>
__device__ __forceinline__ void stream_cols_inv(const float2* T, const uint32_t* dbits, float4* x4, const Tw& tw,
                                                int rot, int c, int nc) {
  constexpr int F = STREAM_F;
  const int rs = apad(F);
  for (int jj = c * NT + threadIdx.x; jj < F / 2; jj += nc * NT) {
    const int j = (jj + rot) & (F / 2 - 1);
    const int n1 = j, n1b = F - 1 - j;
    float2 a[PT], b[PT];
#pragma unroll
    for (int k2 = 0; k2 < PT; ++k2) {
      a[k2] = T[k2 * rs + aidx(n1)];
      b[k2] = T[k2 * rs + aidx(n1b)];
    }
    twiddle_powers<PT, 1>(a, tw, 8 * n1);   // a[k2] *= conj(omega_L^{n1 k2})
    dft<PT, 1>(a);                           // a[n2] = z[n1 + F n2]
    twiddle_powers<PT, 1>(b, tw, 8 * n1b);
    dft<PT, 1>(b);
#pragma unroll
    for (int n2 = 0; n2 < PT / 2; ++n2) {
      const int m = n1 + F * n2, m2 = n1b + F * n2;
      const float2 za = a[n2], zam = b[PT - 1 - n2];    // z[m], z[L-1-m]
      const float2 zb = b[n2], zbm = a[PT - 1 - n2];    // z[m2], z[L-1-m2]
      x4[m] = sign4(make_float4(za.x, zam.y, za.y, zam.x), dbits4(dbits, m));
      x4[m2] = sign4(make_float4(zb.x, zbm.y, zb.y, zbm.x), dbits4(dbits, m2));
    }
  }
}


__device__ __forceinline__ void copy_row(float4* dst, const float4* src) {
  for (int i = threadIdx.x; i < apad(STREAM_F) / 2; i += NT) dst[i] = src[i];
}

// Row pass of one unit: rows ra and rb = (P - ra) mod P (one row when ra is 0 or P/2).  Every
// pair (Z_k, Z_{L-k}) with k in row ra and L - k in row rb is visited once: k = ra + P k1 with
//   ra != 0, P/2:  partner (rb, F-1-k1), k1 in [0, F)
//   ra == P/2:     partner (ra, F-1-k1), k1 in [0, F/2)
//   ra == 0:       partner (0, (F-k1) mod F), k1 in [0, F/2]  (k1 = 0 and F/2 pair with themselves)
// prank holds, in this order, the rank in Omega of each of the pair's outputs (-1: not kept).
// Forward: y[rank(f)] = X_f.  Inverse: X_f = u[rank(f)] (0 off Omega), and the DCT-III
// pre-processing writes the pair back into the rows.  The global loads (ranks, and u for the
// inverse) are software-pipelined one or two steps ahead of the arithmetic.
__device__ __forceinline__ void stream_pairs(const Geo& g, int ra, float2* R0, float2* R1, const Tw& tw,
                                             const int4* prank, bool inv, const float* u, float* y, int rot) {
  constexpr int F = STREAM_F;
  const int P = g.P;
  const float wk = sqrtf(2.0f / (float)g.N), w0 = sqrtf(1.0f / (float)g.N);
  const int npairs = (ra == 0) ? F / 2 + 1 : (2 * ra == P ? F / 2 : F);
  float2* Rb = (ra == 0 || 2 * ra == P) ? R0 : R1;
  rot %= npairs;
  // pair j of this thread's sequence -> k1 (rotated start), -1 past the end
  auto k1_of = [&](int j) { return j < npairs ? (j + rot < npairs ? j + rot : j + rot - npairs) : -1; };
  auto ranks = [&](int k1) { return k1 >= 0 ? __ldg(prank + k1) : make_int4(-1, -1, -1, -1); };
  auto pair_geo = [&](int k1, int& kb, int& k, bool& self) {
    kb = ra == 0 ? ((F - k1) & (F - 1)) : F - 1 - k1;
    k = ra + P * k1;
    self = ra == 0 && (k1 == 0 || 2 * k1 == F);
  };
  if (!inv) {
    // software pipeline: the rank loads of the next U pairs are in flight during this step
    constexpr int U = 4;
    int4 rn[U];
#pragma unroll
    for (int v = 0; v < U; ++v) rn[v] = ranks(k1_of(threadIdx.x + v * NT));
    for (int j0 = threadIdx.x; j0 < npairs; j0 += U * NT) {
      int4 rc[U];
#pragma unroll
      for (int v = 0; v < U; ++v) {
        rc[v] = rn[v];
        rn[v] = ranks(k1_of(j0 + (U + v) * NT));
      }
#pragma unroll
      for (int v = 0; v < U; ++v) {
        const int k1 = k1_of(j0 + v * NT);
        if (k1 < 0) continue;
        int kb, k;
        bool self;
        pair_geo(k1, kb, k, self);
        float X[4] = {0.f, 0.f, 0.f, 0.f};
        dct2_pair(R0[aidx(k1)], Rb[aidx(kb)], k, pair_tw(tw, k), wk, w0, X);
        const int r[4] = {rc[v].x, rc[v].y, rc[v].z, rc[v].w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (r[i] >= 0) y[r[i]] = X[i];
      }
    }
  } else {
    // three stages: ranks two steps ahead, the u values they address one step ahead
    constexpr int U = 2;
    int4 r2[U], r1[U];
    float x1[U][4];
#pragma unroll
    for (int v = 0; v < U; ++v) {
      r1[v] = ranks(k1_of(threadIdx.x + v * NT));
      r2[v] = ranks(k1_of(threadIdx.x + (U + v) * NT));
    }
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int r[4] = {r1[v].x, r1[v].y, r1[v].z, r1[v].w};
#pragma unroll
      for (int i = 0; i < 4; ++i) x1[v][i] = r[i] >= 0 ? __ldg(u + r[i]) : 0.f;
    }
    for (int j0 = threadIdx.x; j0 < npairs; j0 += U * NT) {
      float xc[U][4];
#pragma unroll
      for (int v = 0; v < U; ++v) {
        const int r[4] = {r2[v].x, r2[v].y, r2[v].z, r2[v].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          xc[v][i] = x1[v][i];
          x1[v][i] = r[i] >= 0 ? __ldg(u + r[i]) : 0.f;
        }
        r2[v] = ranks(k1_of(j0 + (2 * U + v) * NT));
      }
#pragma unroll
      for (int v = 0; v < U; ++v) {
        const int k1 = k1_of(j0 + v * NT);
        if (k1 < 0) continue;
        int kb, k;
        bool self;
        pair_geo(k1, kb, k, self);
        float2 Va, Vb;
        dct3_pair(xc[v], k, self, pair_tw(tw, k), wk, w0, Va, Vb);
        R0[aidx(k1)] = Va;
        if (!self) Rb[aidx(kb)] = Vb;
      }
    }
  }
  __syncthreads();
}

// Offset of unit ra's first pair in the pair table (units in order ra = 0, 1, ..., P/2).
__host__ __device__ inline int stream_pair_base(int ra) { return ra == 0 ? 0 : STREAM_F / 2 + 1 + (ra - 1) * STREAM_F; }

// One unit of the row pass (rows ra and (P - ra) mod P), forward or inverse.
__device__ __noinline__ void stream_unit(const StreamArgs& a, int b, float2* T, int ra, int rot, uint32_t* phase) {
  constexpr int F = STREAM_F;
  float2* R0 = reinterpret_cast<float2*>(smem_raw);
  float2* R1 = R0 + apad(F);
  float2* TB = R1 + apad(F);
  const OpDev& op = a.op;
  const Tw tw = {TB + apad(F), TB + apad(F) + apad(1 << op.lo_bits), op.lo_bits, (1 << op.lo_bits) - 1, 4 * op.N - 1,
};
  Geo g;
  g.N = op.N; g.L = op.N >> 1; g.P = op.P; g.F = F; g.c = 0; g.h = 0; g.lh = 0; g.S2 = 0; g.four_n = 4 * op.N;
  const int rs = apad(F);
  const int rb = (op.P - ra) & (op.P - 1);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + STREAM_MBAR_OFF);
  if (a.mode == MODE_APPLY) {
    // rows ra (and rb) by bulk copy; R0 / R1 were last accessed by generic loads and stores
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("fence.proxy.async.global;" ::: "memory");
      mbar_expect(mbar, (rb != ra ? 2u : 1u) * STREAM_ROW_BYTES);
      bulk_g2s(R0, T + ra * rs, STREAM_ROW_BYTES, mbar);
      if (rb != ra) bulk_g2s(R1, T + rb * rs, STREAM_ROW_BYTES, mbar);
    }
    if (!mbar_wait(mbar, *phase & 1u)) atomicExch(a.err, CS_ERR_TIMEOUT);
    *phase ^= 1u;
    local_fft<-1>(R0, TB, F, tw, g.four_n);
    if (rb != ra) local_fft<-1>(R1, TB, F, tw, g.four_n);
    stream_pairs(g, ra, R0, R1, tw, a.prank + stream_pair_base(ra), false, nullptr, a.out + (size_t)b * op.M, rot);
  } else {
    stream_pairs(g, ra, R0, R1, tw, a.prank + stream_pair_base(ra), true, a.in + (size_t)b * op.M, nullptr, rot);
    local_fft<1>(R0, TB, F, tw, g.four_n);
    if (rb != ra) local_fft<1>(R1, TB, F, tw, g.four_n);
    // rows back with plain coalesced stores (a bulk store measured no faster here: R0 / R1 are
    // rewritten by the next unit right away, so its source read must be waited for at once)
    copy_row(reinterpret_cast<float4*>(T + ra * rs), reinterpret_cast<const float4*>(R0));
    if (rb != ra) copy_row(reinterpret_cast<float4*>(T + rb * rs), reinterpret_cast<const float4*>(R1));
    __syncthreads();   // R0 / R1 are rewritten by the next unit
  }
}

// Row pass share of CTA c of nc: units u = c, c + nc, ... of the P/2 units {rows 0 and P/2},
// {1, P-1}, ..., {P/2-1, P/2+1} (two rows each).
__device__ __forceinline__ void stream_rows(const StreamArgs& a, int b, float2* T, int rot, int c, int nc,
                                            uint32_t* phase) {
  const int P = a.op.P;
  for (int u = c; u < P / 2; u += nc) {
    if (u == 0) {
      stream_unit(a, b, T, 0, rot, phase);
      stream_unit(a, b, T, P / 2, rot, phase);
    } else {
      stream_unit(a, b, T, u, rot, phase);
    }
  }
}

template <int PT>
__device__ __noinline__ void stream_cols(const StreamArgs& a, int b, float2* T, int rot, int c, int nc) {
  constexpr int F = STREAM_F;
  const OpDev& op = a.op;
  float2* TB = reinterpret_cast<float2*>(smem_raw) + 2 * apad(F);
  const Tw tw = {TB + apad(F), TB + apad(F) + apad(1 << op.lo_bits), op.lo_bits, (1 << op.lo_bits) - 1, 4 * op.N - 1,
};
  if (a.mode == MODE_APPLY)
    stream_cols_fwd<PT>(reinterpret_cast<const float4*>(a.in + (size_t)b * op.N), a.dbits, T, tw, rot, c, nc);
  else
    stream_cols_inv<PT>(T, a.dbits, reinterpret_cast<float4*>(a.out + (size_t)b * op.N), tw, rot, c, nc);
}

__device__ __forceinline__ void stream_cols_any(const StreamArgs& a, int b, float2* T, int rot, int c, int nc) {
  switch (a.op.P) {
    case 2: stream_cols<2>(a, b, T, rot, c, nc); break;
    case 4: stream_cols<4>(a, b, T, rot, c, nc); break;
    case 8: stream_cols<8>(a, b, T, rot, c, nc); break;
    default: stream_cols<16>(a, b, T, rot, c, nc); break;
  }
}

// One cluster of nc CTAs per vector; the intermediate rows T of a vector live in the cluster's
// global buffer and are shared by its CTAs, with a cluster barrier between the two passes and
// after each vector (the next vector rewrites T).
__global__ void __launch_bounds__(NT, 1) stream_kernel(const StreamArgs a) {
  constexpr int F = STREAM_F;
  const OpDev& op = a.op;
  cg::cluster_group cl = cg::this_cluster();
  const int nc = (int)cl.num_blocks();
  const int c = (int)cl.block_rank();
  const int cid = blockIdx.x / nc;
  const int ncl = gridDim.x / nc;
  {
    float2* twlo = reinterpret_cast<float2*>(smem_raw) + 3 * apad(F);
    float2* twhi = twlo + apad(1 << op.lo_bits);
    const int nlo = 1 << op.lo_bits, nhi = 1 << op.hi_bits;
    for (int i = threadIdx.x; i < nlo; i += NT) twlo[aidx(i)] = op.tw[i];
    for (int i = threadIdx.x; i < nhi; i += NT) twhi[i] = op.tw[nlo + i];
  }
  if (threadIdx.x == 0) {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + STREAM_MBAR_OFF);
    mbar_init(&mbar[0]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;   // parity of the row loads' mbarrier
  float2* T = a.T + (size_t)cid * op.P * apad(F);
  // clusters walk the shared tables (sign bits, pair ranks) from different warp-aligned
  // offsets, so that concurrent clusters do not all read the same few L2 lines at once
  const int rot = (int)((cid * 37u * 32u) & (F / 2 - 1));
  for (int b = cid; b < a.B; b += ncl) {
    if (a.mode == MODE_APPLY) {
      stream_cols_any(a, b, T, rot, c, nc);
      asm volatile("fence.proxy.async.global;" ::: "memory");   // the rows are read by bulk copies
      cl.sync();   // every row of T is complete
      stream_rows(a, b, T, rot, c, nc, &phase);
    } else {
      stream_rows(a, b, T, rot, c, nc, &phase);
      cl.sync();
      stream_cols_any(a, b, T, rot, c, nc);
    }
    cl.sync();     // nobody reads T any more: the next vector may rewrite it
  }
}

size_t stream_row_floats() { return 2 * (size_t)apad(STREAM_F); }

static size_t stream_smem() {
  // rows R0, R1, the FFT ping-pong buffer, twiddle levels of up to 1024 entries each, and the
  // two mbarriers of the column pass's staging buffers (which overlay R0 and R1)
  return STREAM_MBAR_OFF + 16;
}

static cudaLaunchConfig_t stream_config(int nc, int clusters, cudaStream_t stream, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc * clusters);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = stream_smem();
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

int stream_clusters(int nc) {
  if (cudaFuncSetAttribute(stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stream_smem()) != cudaSuccess)
    return 0;
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = stream_config(nc, 1, nullptr, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, stream_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_stream(const StreamArgs& a, int nc, int clusters, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stream_smem());
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = stream_config(nc, clusters, stream, attr);
  return cudaLaunchKernelEx(&cfg, stream_kernel, a);
}

// Failure-path probe: the grid barrier's bounded wait on a flag that is set (returns at once)
// or that nothing sets (runs out after `limit` polls and reports CS_ERR_TIMEOUT).
__global__ void wait_probe_kernel(volatile unsigned* flag, unsigned long long limit, int* status) {
  if (threadIdx.x == 0) *status = spin_until_changed(flag, 0u, limit) ? (int)CS_OK : (int)CS_ERR_TIMEOUT;
}

cudaError_t launch_wait_probe(unsigned* flag, unsigned long long limit, int* status, cudaStream_t stream) {
  wait_probe_kernel<<<1, 32, 0, stream>>>(flag, limit, status);
  return cudaGetLastError();
}

}  // namespace csg
