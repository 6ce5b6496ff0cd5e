// Batched top-K support selection over |c| (Sec. II step 2 and SP's merge step): for each of B
// rows c_b of length N, the K indices of the largest |c_b[n]| outside an optional exclusion mask,
// ties to the lowest index, sorted ascending.  The stand-alone form of the selection the
// recovery kernels fuse; it streams rows that live in HBM.
//
// One CTA owns one row at a time (a persistent grid of two CTAs per SM, no waits between CTAs),
// and each of its 16 warps owns one contiguous sixteenth of the row:
//   1. a strided sample of SEL_SAMPLE keys gives a low threshold T (a lower bound of the
//      sample's r-th largest key, r set so that at least K keys of the row are >= T with
//      overwhelming probability);
//   2. one streaming pass over the row (cp.async 16-byte copies, several tiles in flight per
//      thread): every warp appends the (key, index) pairs of its range with key >= T, in index
//      order, to its own candidate segment;
//   3. an exact radix select over the candidates (11-, 11- and 10-bit digits, then the same on
//      the index among keys tied at the threshold) gives the threshold key and tie cut;
//   4. every warp compacts its chosen candidates, in order, into the output at the offset the
//      warps before it fill: the segments are in index order, so the output is sorted.
// When the sample misleads (fewer than K candidates, or a segment overflows) the CTA falls back
// to the same radix select and compaction streamed over the whole row, so the result is always
// exact; only the speed depends on the sample.  Keys are (|c| bits) + 1 (excluded: 0), so the
// unsigned order is the order of |c| and every eligible entry has a nonzero key.
#include <atomic>

#include "cs_internal.h"

namespace csg {

constexpr int SNT = 512;               // threads per CTA
constexpr int SNW = SNT / 32;          // warps per CTA, one row range and candidate segment each
constexpr int SEL_SAMPLE = SELECT_SAMPLE_MAX;   // sample keys (groups of 4 consecutive entries)
constexpr int SEL_BINS = 2048;         // 11-bit digits
constexpr int SEL_U = 4;               // scalar path: 4-entry groups per thread in registers
constexpr int SEL_DEPTH = 2;           // 16-byte path: tiles in flight per warp (cp.async)
constexpr int SEL_SU = 4;              // 16-byte copies per thread per tile
static_assert(SEL_BINS == 4 * SNT, "digit_search gives every thread four bins");
static_assert(SNW == SELECT_WARPS, "the host sizes one candidate segment per warp");

__device__ __forceinline__ uint32_t sel_key(float v) { return (__float_as_uint(v) & 0x7fffffffu) + 1u; }

struct SelShared {
  uint32_t skey[SEL_SAMPLE];
  uint32_t hist[SEL_BINS];
  uint32_t wsum[SNW];
  uint32_t wcnt[SNW];
  int res[4];
};
// the 16-byte path's copy ring: [SEL_DEPTH][SEL_SU][SNT] float4; each thread reads only the
// slots it copied itself (64 KiB, dynamic shared memory)
constexpr size_t SEL_RING_BYTES = sizeof(float4) * SEL_DEPTH * SEL_SU * SNT;
extern __shared__ float4 sel_ring[];

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// The threshold digit of one radix pass: with hist holding the counts of the digits of the
// remaining keys, the digit d with above(d) < need <= above(d) + hist[d], where above(d) counts
// the keys of higher digits.  res = {d, above(d), hist[d]}, or {-1, total, 0} when fewer than
// `need` keys remain.  Every thread calls it; the result is read after its last barrier.
__device__ void digit_search(SelShared& sh, uint32_t need) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t h[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) h[d] = sh.hist[4 * t + d];
  const uint32_t mine = h[0] + h[1] + h[2] + h[3];
  uint32_t suf = mine;   // inclusive suffix sum over the threads >= t
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_down_sync(0xffffffffu, suf, o);
    if (lane + o < 32) suf += v;
  }
  if (lane == 0) sh.wsum[w] = suf;
  __syncthreads();
  for (int w2 = w + 1; w2 < SNW; ++w2) suf += sh.wsum[w2];
  const uint32_t above = suf - mine;
  if (above < need && need <= suf) {
    uint32_t acc = above;
    int d = 3;
    for (; d > 0; --d) {
      if (acc + h[d] >= need) break;
      acc += h[d];
    }
    sh.res[0] = 4 * t + d;
    sh.res[1] = (int)acc;
    sh.res[2] = (int)h[d];
  }
  if (t == 0 && suf < need) {   // thread 0's suffix is the total
    sh.res[0] = -1;
    sh.res[1] = (int)suf;
    sh.res[2] = 0;
  }
  __syncthreads();
}

// Radix select of the K largest nonzero keys over the CTA (every thread calls it with the same
// K).  each(visit) calls visit(key) for every key this thread holds.  On return keys > *tau are
// selected and *need more are to be taken among the *eq keys equal to *tau; *tau = 0 (take every
// nonzero key) when fewer than K are nonzero.  With passes < 3 only the leading digits are
// resolved: *tau is then the threshold's prefix with the low bits zero, a lower bound of the
// K-th largest key.
template <class Each>
__device__ void block_radix_select(SelShared& sh, uint32_t K, Each each, uint32_t* tau, uint32_t* need, uint32_t* eq,
                                   int passes = 3) {
  uint32_t prefix = 0, pmask = 0, nd = K, last_eq = 0;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
    const uint32_t dmask = pass == 2 ? 1023u : 2047u;
    for (int i = threadIdx.x; i < SEL_BINS; i += SNT) sh.hist[i] = 0u;
    __syncthreads();
    each([&](uint32_t kk) {
      if (kk != 0u && (kk & pmask) == prefix) atomicAdd(&sh.hist[(kk >> shift) & dmask], 1u);
    });
    __syncthreads();
    digit_search(sh, nd);
    const int dig = sh.res[0];
    const uint32_t above = (uint32_t)sh.res[1];
    last_eq = (uint32_t)sh.res[2];
    if (dig < 0) {   // uniform
      *tau = 0u;
      *need = 0u;
      *eq = 0u;
      return;
    }
    nd -= above;
    prefix |= (uint32_t)dig << shift;
    pmask |= dmask << shift;
  }
  *tau = prefix;
  *need = nd;
  *eq = last_eq;
}

// Four consecutive entries n0 .. n0+3 of a row as keys (0 past the end or excluded).
template <bool VEC>
__device__ __forceinline__ void load4(const float* row, const uint32_t* ex, int N, int n0, uint32_t k[4]) {
  if (VEC) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(row + n0));
    k[0] = sel_key(v.x); k[1] = sel_key(v.y); k[2] = sel_key(v.z); k[3] = sel_key(v.w);
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) k[e] = n0 + e < N ? sel_key(__ldcs(row + n0 + e)) : 0u;
  }
  if (ex) {
    const uint32_t wd = __ldg(ex + (n0 >> 5)) >> (n0 & 31);   // n0 is a multiple of 4
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if ((wd >> e) & 1u) k[e] = 0u;
  }
}

// Candidate bits of four entries: bit e set when |v_e| >= tf, i.e. when |v_e| - tf has a clear
// sign bit.  The difference is never negative for |v_e| >= tf, so no entry at or above the
// threshold is lost (a NaN entry keeps a clear sign bit and stays a candidate, as its key orders
// it above +inf; a NaN threshold makes every entry a candidate).  The four sign bytes are
// gathered by byte permutes and packed into a nibble by one multiply: the shifted sign bits sit
// at bits 0, 8, 16, 24, and x 0x01020408 moves them to bits 24 .. 27 with no carries there.
__device__ __forceinline__ uint32_t cand_nibble(const float4& v, float tf) {
  const uint32_t d0 = __float_as_uint(fabsf(v.x) - tf), d1 = __float_as_uint(fabsf(v.y) - tf);
  const uint32_t d2 = __float_as_uint(fabsf(v.z) - tf), d3 = __float_as_uint(fabsf(v.w) - tf);
  const uint32_t w = __byte_perm(__byte_perm(d0, d1, 0x0073), __byte_perm(d2, d3, 0x0073), 0x5410);
  const uint32_t sgn = ((w >> 7) & 0x01010101u) * 0x01020408u >> 24;
  return ~sgn & 15u;
}

__device__ __forceinline__ uint32_t key_at(const float* row, const uint32_t* ex, int n) {
  if (ex && ((__ldg(ex + (n >> 5)) >> (n & 31)) & 1u)) return 0u;
  return sel_key(__ldcg(row + n));
}

// The warp's ordered compaction of the entries it chooses: items j < cnt (warp-uniform) in
// order, item(j) -> (key, index); writes the chosen indices at out[base ...] (below K only) and
// returns how many it chose.  COUNT: count only.
template <bool COUNT, class Item, class Chosen>
__device__ __forceinline__ uint32_t warp_compact(int cnt, Item item, Chosen chosen, int32_t* out, uint32_t base,
                                                 uint32_t K) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  constexpr int UL = 4;   // items in flight per lane
  uint32_t done = 0;
  for (int j0 = 0; j0 < cnt; j0 += 32 * UL) {
    uint2 c[UL];
#pragma unroll
    for (int e = 0; e < UL; ++e) {
      const int j = j0 + 32 * e + lane;
      c[e] = j < cnt ? item(j) : make_uint2(0u, 0u);
    }
#pragma unroll
    for (int e = 0; e < UL; ++e) {
      const int j = j0 + 32 * e + lane;
      const bool f = j < cnt && chosen(c[e].x, c[e].y);
      const uint32_t m = __ballot_sync(0xffffffffu, f);
      if (!COUNT && f) {
        const uint32_t pos = base + done + __popc(m & lt);
        if (pos < K) out[pos] = (int32_t)c[e].y;
      }
      done += __popc(m);
    }
  }
  return done;
}

template <bool VEC>
__device__ void select_row(SelShared& sh, const SelectArgs& a, int b) {
  const int N = (int)a.N;
  const uint32_t K = (uint32_t)a.K;
  const float* row = a.c + (size_t)b * a.N;
  const uint32_t* ex = a.excl ? a.excl + (size_t)b * a.W : nullptr;
  int32_t* out = a.out + (size_t)b * a.K;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int G4 = (N + 3) / 4;   // groups of four entries
  // this warp's range of groups and its candidate segment
  const int gw0 = (int)((long long)w * G4 / SNW), gw1 = (int)((long long)(w + 1) * G4 / SNW);
  const int capw = a.capw;
  uint2* seg = a.cand + ((size_t)blockIdx.x * SNW + w) * capw;

  // 1. sample: a.S / 4 groups spread evenly over the row, their r-th largest key
  const int sg4 = a.S / 4;
  constexpr int SPT = SEL_SAMPLE / 4 / SNT;   // sample groups per thread
  static_assert(SPT * 4 * SNT == SEL_SAMPLE, "whole sample groups per thread");
  {
    uint32_t k[SPT][4];
#pragma unroll
    for (int u = 0; u < SPT; ++u) {   // all loads in flight before any store
      const int j = threadIdx.x + u * SNT;
      if (j < sg4) load4<VEC>(row, ex, N, 4 * (int)((long long)j * G4 / sg4), k[u]);
    }
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int j = threadIdx.x + u * SNT;
      if (j < sg4) {
#pragma unroll
        for (int e = 0; e < 4; ++e) sh.skey[4 * j + e] = k[u][e];
      }
    }
  }
  __syncthreads();
  uint32_t tlo, need, eq;
  block_radix_select(
      sh, (uint32_t)a.r,
      [&](auto visit) {
        for (int i = threadIdx.x; i < a.S; i += SNT) visit(sh.skey[i]);
      },
      &tlo, &need, &eq, 2);   // a lower bound of the r-th largest sample key suffices
  if (tlo == 0u) tlo = 1u;   // the sample has fewer than r eligible keys: every eligible entry

  // 2. stream the row once; every warp appends the keys >= tlo of its range to its segment, in
  // index order.  Scalar path: a lane's count c <= 4 is prefix-summed over the warp from three
  // ballots of its bits, and the stores are predicated.
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t wc = 0;   // this warp's candidates so far (warp-uniform)
  auto append = [&](const uint32_t k[4], int n0) {   // warp-uniform call
    bool p[4];
    uint32_t c = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      p[e] = k[e] >= tlo;
      c += p[e] ? 1u : 0u;
    }
    const uint32_t b1 = __ballot_sync(0xffffffffu, c & 1u), b2 = __ballot_sync(0xffffffffu, c & 2u),
                   b4 = __ballot_sync(0xffffffffu, c & 4u);
    const uint32_t tot = __popc(b1) + 2u * __popc(b2) + 4u * __popc(b4);
    uint32_t pos = wc + __popc(b1 & lt) + 2u * __popc(b2 & lt) + 4u * __popc(b4 & lt);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (p[e] && pos < (uint32_t)capw) seg[pos] = make_uint2(k[e], (uint32_t)(n0 + e));
      pos += p[e] ? 1u : 0u;
    }
    wc += tot;
  };
  if (VEC) {
    // per-warp cp.async pipeline over tiles of TS = 32 SEL_SU groups, SEL_DEPTH - 1 tiles ahead
    // of the one being processed; every thread copies and later reads its own ring slots
    constexpr int TS = 32 * SEL_SU;
    const int T = (gw1 - gw0 + TS - 1) / TS;
    const float4* row4 = reinterpret_cast<const float4*>(row);
    static_assert(SEL_SU * 8 <= 32 && SEL_SU * 4 <= 32, "per-group counts (at most 32 x 4) in 8-bit fields, mask in 32 bits");
    const float tf = __uint_as_float(tlo - 1u);   // key >= tlo  <=>  |c| >= tf (bit patterns)
    // One tile: the lane's SEL_SU groups (SEL_SU x 4 entries) as a candidate mask m (bit 4u + e),
    // the counts of each group packed in 8-bit fields and prefix-summed over the warp by one
    // shuffle scan, then a loop over the lane's set bits only.  Index order is (group u, lane,
    // entry), so group u's candidates of all lanes come before group u + 1's.
    auto append_tile = [&](const float4* slot, int t) {
      uint32_t m = 0u;
#pragma unroll
      for (int u = 0; u < SEL_SU; ++u) {
        const int g = gw0 + t * TS + u * 32 + lane;
        if (g < gw1) {
          const float4 v = slot[u * SNT + threadIdx.x];
          uint32_t q = cand_nibble(v, tf);
          if (ex) q &= ~(__ldg(ex + ((4 * g) >> 5)) >> ((4 * g) & 31));
          m |= (q & 15u) << (4 * u);
        }
      }
      uint32_t packed = 0u;
#pragma unroll
      for (int u = 0; u < SEL_SU; ++u) packed |= (uint32_t)__popc((m >> (4 * u)) & 15u) << (8 * u);
      uint32_t incl = packed;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      const uint32_t excl = incl - packed;
      uint32_t gbase[SEL_SU];   // offset of group u's candidates in the segment
      uint32_t acc = wc;
#pragma unroll
      for (int u = 0; u < SEL_SU; ++u) {
        gbase[u] = acc + ((excl >> (8 * u)) & 255u);
        acc += (tot >> (8 * u)) & 255u;
      }
      uint32_t mm = m;
      while (mm) {
        const int bt = __ffs(mm) - 1;
        mm &= mm - 1u;
        const int u = bt >> 2, e = bt & 3;
        uint32_t gb = gbase[0];
#pragma unroll
        for (int uu = 1; uu < SEL_SU; ++uu) gb = u == uu ? gbase[uu] : gb;
        const uint32_t pos = gb + __popc(m & ((1u << bt) - 1u) & (15u << (4 * u)));
        const float val = reinterpret_cast<const float*>(slot + u * SNT + threadIdx.x)[e];
        const int g = gw0 + t * TS + u * 32 + lane;
        if (pos < (uint32_t)capw) seg[pos] = make_uint2(sel_key(val), (uint32_t)(4 * g + e));
      }
      wc = acc;
    };
    auto issue = [&](int t) {
      if (t < T) {
        float4* slot = sel_ring + (size_t)(t % SEL_DEPTH) * SEL_SU * SNT;
#pragma unroll
        for (int u = 0; u < SEL_SU; ++u) {
          const int g = gw0 + t * TS + u * 32 + lane;
          if (g < gw1) cp_async16(slot + u * SNT + threadIdx.x, row4 + g);
        }
      }
      cp_async_commit();   // possibly empty: keeps the group count uniform
    };
#pragma unroll
    for (int t = 0; t < SEL_DEPTH - 1; ++t) issue(t);
    for (int t = 0; t < T; ++t) {
      issue(t + SEL_DEPTH - 1);
      cp_async_wait<SEL_DEPTH - 1>();   // this thread's copies of tile t have landed
      append_tile(sel_ring + (size_t)(t % SEL_DEPTH) * SEL_SU * SNT, t);
    }
    cp_async_wait<0>();
  } else {
    for (int base = gw0; base < gw1; base += SEL_U * 32) {
      uint32_t k[SEL_U][4];
#pragma unroll
      for (int u = 0; u < SEL_U; ++u) {
        const int g = base + u * 32 + lane;
        if (g < gw1) load4<VEC>(row, ex, N, 4 * g, k[u]);
        else k[u][0] = k[u][1] = k[u][2] = k[u][3] = 0u;
      }
#pragma unroll
      for (int u = 0; u < SEL_U; ++u) append(k[u], 4 * (base + u * 32 + lane));
    }
  }
  if (lane == 0) sh.wcnt[w] = wc;
  __syncthreads();
  uint32_t nge = 0;
  bool over = false;
  for (int i = 0; i < SNW; ++i) {
    nge += sh.wcnt[i];
    over |= sh.wcnt[i] > (uint32_t)capw;
  }
  const bool fallback = over || (nge < K && tlo > 1u);
  const int cw = fallback ? 0 : (int)sh.wcnt[w];   // this warp's segment length

  // 3. exact selection: threshold key tau and, on a tie, the index cut tau2
  // candidates: every warp visits its own segment (four loads in flight per thread)
  auto each_cand = [&](auto visit) {
    for (int j0 = lane; j0 < cw; j0 += 128) {
      uint32_t kk[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) kk[e] = j0 + 32 * e < cw ? __ldcg(&seg[j0 + 32 * e].x) : 0u;
#pragma unroll
      for (int e = 0; e < 4; ++e) visit(kk[e]);
    }
  };
  auto each_row = [&](auto visit) {   // fallback: the whole row
    for (int n = threadIdx.x; n < N; n += SNT) visit(key_at(row, ex, n));
  };
  uint32_t tau, tau2 = 0u;
  if (!fallback) block_radix_select(sh, K, each_cand, &tau, &need, &eq);
  else block_radix_select(sh, K, each_row, &tau, &need, &eq);
  const bool tied = need > 0u && eq > need;
  const uint32_t N32 = (uint32_t)N;
  if (tied) {   // the `need` lowest indices among the keys equal to tau: keys N - index
    uint32_t n2, e2;
    if (!fallback) {
      block_radix_select(
          sh, need,
          [&](auto visit) {
            for (int j0 = lane; j0 < cw; j0 += 128) {
              uint2 c[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) c[e] = j0 + 32 * e < cw ? __ldcg(&seg[j0 + 32 * e]) : make_uint2(0u, 0u);
#pragma unroll
              for (int e = 0; e < 4; ++e) visit(c[e].x == tau && c[e].x != 0u ? N32 - c[e].y : 0u);
            }
          },
          &tau2, &n2, &e2);
    } else {
      block_radix_select(
          sh, need,
          [&](auto visit) {
            for (int n = threadIdx.x; n < N; n += SNT) visit(key_at(row, ex, n) == tau ? N32 - (uint32_t)n : 0u);
          },
          &tau2, &n2, &e2);
    }
  }
  auto chosen = [&](uint32_t kk, uint32_t n) {
    return tied ? (kk > tau || (kk == tau && N32 - n >= tau2)) : (kk != 0u && kk >= tau);
  };

  // 4. ordered output: count per warp, offsets in warp order, then compact
  auto cand_item = [&](int j) { return __ldcg(&seg[j]); };
  const int e0 = 4 * gw0, e1 = min(N, 4 * gw1);   // the warp's range of entries (fallback)
  auto row_item = [&](int j) { return make_uint2(key_at(row, ex, e0 + j), (uint32_t)(e0 + j)); };
  const uint32_t mine = !fallback ? warp_compact<true>(cw, cand_item, chosen, out, 0u, K)
                                  : warp_compact<true>(e1 - e0, row_item, chosen, out, 0u, K);
  if (lane == 0) sh.wsum[w] = mine;
  __syncthreads();
  uint32_t base = 0, total = 0;
  for (int i = 0; i < SNW; ++i) {
    if (i < w) base += sh.wsum[i];
    total += sh.wsum[i];
  }
  if (!fallback) warp_compact<false>(cw, cand_item, chosen, out, base, K);
  else warp_compact<false>(e1 - e0, row_item, chosen, out, base, K);
  for (uint32_t i = total + threadIdx.x; i < K; i += SNT) out[i] = -1;   // fewer than K eligible
  __syncthreads();   // sh is reused by the next row
}

__global__ void __launch_bounds__(SNT, 2) select_kernel(const SelectArgs a) {
  __shared__ SelShared sh;
  for (int b = blockIdx.x; b < a.B; b += gridDim.x) {
    if (a.vec) select_row<true>(sh, a, b);
    else select_row<false>(sh, a, b);
  }
}

// Resident CTAs per SM on the current device (0: cannot launch); the attribute and the
// occupancy query run once per device.
int select_ctas_per_sm() {
  constexpr int MAX_DEV = 64;
  static std::atomic<int> cached[MAX_DEV];   // 0: not queried yet, else CTAs per SM + 1
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) {
    cudaGetLastError();
    return 0;
  }
  const int c = cached[dev].load();
  if (c > 0) return c - 1;
  int n = 0;
  if (cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SEL_RING_BYTES) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, select_kernel, SNT, SEL_RING_BYTES) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cached[dev].store(n + 1);
  return n;
}

// The caller has obtained select_ctas_per_sm() > 0 on this device (which set the kernel's
// shared-memory attribute).
cudaError_t launch_select(const SelectArgs& a, int grid, cudaStream_t stream) {
  select_kernel<<<grid, SNT, SEL_RING_BYTES, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace csg
