// Ordering of the hash path's output by code.  The paper's output of the
// highly sparse algorithm is the hash table itself (Sec. 3.2); this library
// returns terms sorted by code like the dense path does, so the table's terms
// are ordered after compaction:
//   1. count the terms in bins of C consecutive codes (keys are distinct, so no
//      bin holds more than C terms),
//   2. exclusive scan of the bin counts,
//   3. scatter every term to its bin's range,
//   4. sort segments of whole bins, at most 2C terms each, in shared memory.
// Steps 1-3 are one counting-sort pass on the high part of the code; step 4
// orders within bins.  Two reads and two writes of the terms in total.
//
// When the code range is small enough for a bitmap of one bit per code
// (order_bitmap_bytes), a cheaper route is taken: set the bit of every key,
// prefix-popcount the bitmap, and write each term directly at its rank (the
// number of keys below it).  One read and one write of the terms, no
// contended atomics (the bit sets are fire-and-forget reductions).
#include "kr_internal.cuh"

namespace kr {

constexpr int ORD_C = 4096;              // codes per bin
constexpr int ORD_SEG = 2 * ORD_C;       // max terms per sorted segment
constexpr int ORD_THREADS = 1024;

__global__ void __launch_bounds__(256) k_bin_count(const uint64_t* __restrict__ key, int64_t n,
                                                   int64_t nb, unsigned long long* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t b = key[i] / ORD_C;
    if (b < (uint64_t)nb) atomicAdd(&cnt[b], 1ull);
  }
}

__global__ void __launch_bounds__(256) k_bin_scatter(const uint64_t* __restrict__ key,
                                                     const uint64_t* __restrict__ val, int64_t n,
                                                     int64_t nb, const int64_t* __restrict__ off,
                                                     unsigned long long* __restrict__ cur,
                                                     uint64_t* __restrict__ okey,
                                                     uint64_t* __restrict__ oval) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = key[i];
    const int64_t b = (int64_t)(k / ORD_C);
    if (b >= nb) continue;
    const int64_t pos = off[b] + (int64_t)atomicAdd(&cur[b], 1ull);
    if (pos < n) {
      okey[pos] = k;
      oval[pos] = val[i];
    }
  }
}

// One CTA per segment k: the bins whose exclusive offset lies in
// [k ORD_C, (k + 1) ORD_C); their terms form the output range
// [off[b_lo], off[b_hi]) of at most ORD_SEG terms.
__global__ void __launch_bounds__(ORD_THREADS) k_seg_sort(const uint64_t* __restrict__ key,
                                                          const uint64_t* __restrict__ val,
                                                          const int64_t* __restrict__ off, int64_t nbins,
                                                          uint64_t* __restrict__ okey,
                                                          uint64_t* __restrict__ oval) {
  extern __shared__ __align__(16) unsigned char ord_smem[];
  uint64_t* sk = (uint64_t*)ord_smem;
  uint16_t* si = (uint16_t*)(ord_smem + sizeof(uint64_t) * ORD_SEG);
  const int64_t seg = blockIdx.x;
  // lower bounds over off[0, nbins] (off[nbins] = total)
  auto lb = [&](int64_t x) {
    int64_t lo = 0, hi = nbins + 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (off[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo > nbins ? nbins : lo;
  };
  const int64_t b_lo = lb(seg * ORD_C), b_hi = lb((seg + 1) * ORD_C);
  const int64_t start = off[b_lo];
  int n = (int)(off[b_hi] - start);
  if (n > ORD_SEG) n = ORD_SEG;   // cannot happen for distinct keys; keeps smem in bounds
  if (n <= 0) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sk[i] = key[start + i];
    si[i] = (uint16_t)i;
  }
  __syncthreads();
  int N = 1;
  while (N < n) N <<= 1;
  const int pairs = N >> 1;
  for (int size = 2; size <= N; size <<= 1) {
    const int half = size >> 1;
    for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
      const int blk = p / half, o = p - blk * half;
      const int i = blk * size + o, j = blk * size + size - 1 - o;
      if (j < n && sk[i] > sk[j]) {
        const uint64_t tk = sk[i]; sk[i] = sk[j]; sk[j] = tk;
        const uint16_t ti = si[i]; si[i] = si[j]; si[j] = ti;
      }
    }
    __syncthreads();
    for (int stride = half >> 1; stride > 0; stride >>= 1) {
      for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
        const int i = (p / stride) * 2 * stride + (p % stride), j = i + stride;
        if (j < n && sk[i] > sk[j]) {
          const uint64_t tk = sk[i]; sk[i] = sk[j]; sk[j] = tk;
          const uint16_t ti = si[i]; si[i] = si[j]; si[j] = ti;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    okey[start + i] = sk[i];
    oval[start + i] = val[start + si[i]];
  }
}

// ---------------------------------------------------------------------------
// bucketed bitmap ordering (large outputs): a counting pass and a scatter put
// the terms in buckets of BK_CODES consecutive codes (bucket order, not yet
// sorted inside); then one CTA per bucket sets the bits of its keys in a
// bitmap of the bucket's codes in shared memory, turns it into per-word
// prefix counts, and writes every term at its rank.  Every random access
// (bit set, rank lookup) stays in shared memory and every write stays inside
// the bucket's own output range, where L2 combines them.
// ---------------------------------------------------------------------------
constexpr int BK_LOG2 = 20;                       // codes per bucket: 2^20
constexpr int64_t BK_CODES = int64_t(1) << BK_LOG2;
constexpr int BK_WORDS = (int)(BK_CODES / 64);    // 16384 bitmap words: 128 KB, prefixes 64 KB
constexpr int BK_THREADS = 1024;

int64_t order_buckets(int64_t krange) { return (krange + BK_CODES - 1) / BK_CODES; }

// the contiguous slice of n terms of this CTA
__device__ __forceinline__ void bk_slice(int64_t n, int64_t* a, int64_t* b) {
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  *a = min(n, (int64_t)blockIdx.x * per);
  *b = min(n, *a + per);
}

// ---------------------------------------------------------------------------
// partition ordering (the first choice for large outputs over wide code
// ranges): the terms are partitioned by the high digits of their fine bucket
// (2^F consecutive codes, F chosen for about 2048 terms a bucket) in two
// passes, each pass sorting a tile of PT_TILE terms by digit in shared memory
// so that the tile goes out as one contiguous run per digit:
//   1. super-buckets of 2^fbits fine buckets (512, or fewer when that leaves
//      under 256 super-buckets): the counts, then a scatter of every
//      CTA's slice in tiles to its reserved range of each super-bucket;
//   2. one CTA per super-bucket: its fine counts and offsets, then the
//      same tile scatter by fine bucket (back into the first arrays);
//   3. each fine bucket ranked by a bitmap of its 2^F codes in shared memory
//      and written back in order from a shared-memory copy (a bucket above
//      PT_SMAX terms is ranked into the second arrays and copied back; one
//      of at most PT_CMP_MAX terms is ranked by comparisons instead, whose
//      cost follows its terms rather than its codes).
// The result is in place.
// ---------------------------------------------------------------------------
#ifndef KR_ORDER_PARTITION
#define KR_ORDER_PARTITION 1
#endif
#ifndef KR_PT_THREADS
#define KR_PT_THREADS 1024
#endif
constexpr int PT_THREADS = KR_PT_THREADS;
constexpr int PT_TILE = 8192;                   // terms per tile: 128 KB of (key, val) in shared memory
constexpr int PT_PER = PT_TILE / PT_THREADS;    // terms per thread and tile
constexpr int PT_FINE_LOG2 = 9;                 // fine buckets per super-bucket: at most 512,
constexpr int PT_FINE = 1 << PT_FINE_LOG2;      // fewer when that leaves under PT_MIN_SUPERS
constexpr int PT_FINE_LOG2_MIN = 4;
constexpr int64_t PT_MIN_SUPERS = 256;          // CTAs of the fine pass
constexpr int64_t PT_MAX_SUPERS = 2048;
constexpr int PT_F_MIN = 10, PT_F_MAX = 17;     // fine buckets of 2^F codes: bitmaps of at most 16 KB
constexpr int PT_SMAX = 4096;                   // a fine bucket is sorted in shared memory up to this
constexpr int PT_CMP_MAX = 256;                 // and ranked by comparisons, not a bitmap, up to this

struct PtPlan {
  int F = 0;
  int fbits = PT_FINE_LOG2;   // fine buckets per super-bucket: 2^fbits
  int64_t nfb = 0, nsup = 0;
  bool ok = false;
};

static PtPlan pt_plan(int64_t n, int64_t krange) {
  PtPlan pl;
  if (n < 2 || krange < 1) return pl;
  int F = 0;
  while (F < PT_F_MAX && (double)(int64_t(1) << (F + 1)) * (double)n <= 2048.0 * (double)krange) ++F;
  if (F < PT_F_MIN) F = PT_F_MIN;
  pl.F = F;
  pl.nfb = (krange + (int64_t(1) << F) - 1) >> F;
  // narrower fine digits for outputs of few fine buckets, so that the fine
  // pass (one CTA per super-bucket) still spreads over the GPU
  int fb = PT_FINE_LOG2;
  while (fb > PT_FINE_LOG2_MIN && ((pl.nfb + (int64_t(1) << fb) - 1) >> fb) < PT_MIN_SUPERS) --fb;
  pl.fbits = fb;
  pl.nsup = (pl.nfb + (int64_t(1) << fb) - 1) >> fb;
  pl.ok = pl.nsup <= PT_MAX_SUPERS;
  return pl;
}

int64_t order_buckets_scratch(int64_t krange, int64_t n_max) {
  const int64_t nb = order_buckets(krange);
  int64_t need = 3 * (nb + 1) + scan_scratch_entries(nb);
  // partition ordering for any count n <= n_max that the plan accepts: fewer
  // terms make larger fine buckets, so n_max gives the most of them, and an
  // accepted plan has at most PT_MAX_SUPERS super-buckets of at most PT_FINE
  // fine buckets (whether or not n_max's own plan is accepted)
  const PtPlan pl = pt_plan(std::max<int64_t>(n_max, 2), krange);
  const int64_t nfb = std::min<int64_t>(pl.nfb, PT_MAX_SUPERS * PT_FINE);
  need = std::max(need, 2 * (PT_MAX_SUPERS + 1) + (nfb + 1) + scan_scratch_entries(PT_MAX_SUPERS));
  return need;
}

// Exclusive scan of cnt[0, m) into ofs[0, m) by the whole CTA of NT threads;
// wsum: NT / 32 words of scratch.
template <int NT = PT_THREADS>
__device__ __forceinline__ void pt_scan(const uint32_t* cnt, uint32_t* ofs, int m, uint32_t* wsum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (m + NT - 1) / NT;   // consecutive entries per thread
  const int a = min(m, tid * per), b = min(m, a + per);
  uint32_t t = 0;
  for (int i = a; i < b; ++i) t += cnt[i];
  uint32_t x = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < NT / 32 ? wsum[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < NT / 32) wsum[lane] = v;
  }
  __syncthreads();
  uint32_t run = (warp > 0 ? wsum[warp - 1] : 0u) + x - t;
  for (int i = a; i < b; ++i) {
    const uint32_t c = cnt[i];
    ofs[i] = run;
    run += c;
  }
  __syncthreads();
}

constexpr int PR_THREADS = 512;   // the ranking pass: several CTAs per SM

// Tile scatter shared by passes 1 and 2: the terms [t0, t1) (at most PT_TILE)
// of (key, val) go to (okey, oval) grouped by digit dig(key) in [0, m): the
// terms of digit d to base[d] + cur[d] onwards, as one run.  tcnt, tofs: m
// words; stage: PT_TILE keys then PT_TILE values.
template <typename Dig>
__device__ __forceinline__ void pt_tile(const uint64_t* __restrict__ key, const uint64_t* __restrict__ val,
                                        int64_t t0, int64_t t1, int m, Dig dig, const int64_t* base,
                                        uint32_t* cur, uint32_t* tcnt, uint32_t* tofs, uint64_t* stage,
                                        uint32_t* wsum, uint64_t* __restrict__ okey,
                                        uint64_t* __restrict__ oval) {
  const int tid = threadIdx.x;
  for (int d = tid; d < m; d += PT_THREADS) tcnt[d] = 0;
  __syncthreads();
  uint64_t k[PT_PER], v[PT_PER];
  uint32_t r[PT_PER];
#pragma unroll
  for (int q = 0; q < PT_PER; ++q) {   // every load of the tile issued before any is used
    const int64_t i = t0 + (int64_t)q * PT_THREADS + tid;
    k[q] = 0;
    v[q] = 0;
    if (i < t1) {
      k[q] = key[i];
      v[q] = val[i];
    }
  }
#pragma unroll
  for (int q = 0; q < PT_PER; ++q) {
    const int64_t i = t0 + (int64_t)q * PT_THREADS + tid;
    r[q] = i < t1 ? atomicAdd(&tcnt[dig(k[q])], 1u) : 0u;
  }
  __syncthreads();
  pt_scan(tcnt, tofs, m, wsum);
#pragma unroll
  for (int q = 0; q < PT_PER; ++q) {
    const int64_t i = t0 + (int64_t)q * PT_THREADS + tid;
    if (i < t1) {
      const uint32_t pos = tofs[dig(k[q])] + r[q];
      stage[pos] = k[q];
      stage[PT_TILE + pos] = v[q];
    }
  }
  __syncthreads();
  const int nt = (int)(t1 - t0);
  for (int j = tid; j < nt; j += PT_THREADS) {
    const uint64_t kk = stage[j];
    const int d = dig(kk);
    const int64_t g = base[d] + (int64_t)cur[d] + (j - (int64_t)tofs[d]);
    okey[g] = kk;
    oval[g] = stage[PT_TILE + j];
  }
  __syncthreads();
  for (int d = tid; d < m; d += PT_THREADS) cur[d] += tcnt[d];
  __syncthreads();
}

// The super-bucket of a key (keys lie below the code range, so the clamp
// only keeps a broken input's terms inside the arrays).
__device__ __forceinline__ int pt_sup(uint64_t k, int sh, int nsup) {
  const uint64_t d = k >> sh;
  return d < (uint64_t)nsup ? (int)d : nsup - 1;
}

// Pass 1 counts: super-bucket histograms of every CTA's slice.
__global__ void __launch_bounds__(PT_THREADS) k_pt_count(const uint64_t* __restrict__ key, int64_t n, int sh,
                                                        int nsup, unsigned long long* __restrict__ cnt) {
  extern __shared__ uint32_t ph[];
  for (int d = threadIdx.x; d < nsup; d += blockDim.x) ph[d] = 0;
  __syncthreads();
  int64_t a, e;
  bk_slice(n, &a, &e);
  for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) atomicAdd(&ph[pt_sup(key[i], sh, nsup)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < nsup; d += blockDim.x)
    if (ph[d]) atomicAdd(&cnt[d], (unsigned long long)ph[d]);
}

// Pass 1: each CTA reserves its slice's share of every super-bucket, then
// scatters the slice tile by tile into (key2, val2).
__global__ void __launch_bounds__(PT_THREADS) k_pt_super(const uint64_t* __restrict__ key,
                                                        const uint64_t* __restrict__ val, int64_t n, int sh,
                                                        int nsup, const int64_t* __restrict__ soff,
                                                        unsigned long long* __restrict__ scur,
                                                        uint64_t* __restrict__ key2, uint64_t* __restrict__ val2) {
  extern __shared__ __align__(16) unsigned char pt_smem[];
  uint64_t* stage = (uint64_t*)pt_smem;                                 // 2 * PT_TILE
  int64_t* base = (int64_t*)(pt_smem + 16 * PT_TILE);                  // [nsup]
  uint32_t* cur = (uint32_t*)(base + nsup);                             // [nsup]
  uint32_t* tcnt = cur + nsup;                                          // [nsup]
  uint32_t* tofs = tcnt + nsup;                                         // [nsup]
  __shared__ uint32_t wsum[PT_THREADS / 32];
  const int tid = threadIdx.x;
  int64_t a, e;
  bk_slice(n, &a, &e);
  for (int d = tid; d < nsup; d += PT_THREADS) tcnt[d] = 0;
  __syncthreads();
  for (int64_t i = a + tid; i < e; i += PT_THREADS) atomicAdd(&tcnt[pt_sup(key[i], sh, nsup)], 1u);
  __syncthreads();
  for (int d = tid; d < nsup; d += PT_THREADS) {
    base[d] = soff[d] + (tcnt[d] ? (int64_t)atomicAdd(&scur[d], (unsigned long long)tcnt[d]) : 0);
    cur[d] = 0;
  }
  __syncthreads();
  auto dig = [sh, nsup](uint64_t k) -> int { return pt_sup(k, sh, nsup); };
  for (int64_t t0 = a; t0 < e; t0 += PT_TILE)
    pt_tile(key, val, t0, min(e, t0 + PT_TILE), nsup, dig, base, cur, tcnt, tofs, stage, wsum, key2, val2);
}

// Pass 2: one CTA per super-bucket: its fine counts and offsets (foff, the
// fine buckets' first positions), then the tile scatter by fine bucket from
// (key2, val2) back into (key, val).
__global__ void __launch_bounds__(PT_THREADS) k_pt_fine(const uint64_t* __restrict__ key2,
                                                       const uint64_t* __restrict__ val2, int64_t n, int F,
                                                       int fbits, int64_t nfb, const int64_t* __restrict__ soff,
                                                       int64_t* __restrict__ foff, uint64_t* __restrict__ key,
                                                       uint64_t* __restrict__ val) {
  extern __shared__ __align__(16) unsigned char pt_smem[];
  uint64_t* stage = (uint64_t*)pt_smem;
  __shared__ int64_t base[PT_FINE];
  __shared__ uint32_t cur[PT_FINE], tcnt[PT_FINE], tofs[PT_FINE];
  __shared__ uint32_t wsum[PT_THREADS / 32];
  const int tid = threadIdx.x;
  const int nfine = 1 << fbits;   // at most PT_FINE
  const int64_t d = blockIdx.x;
  const int64_t s0 = soff[d], s1 = soff[d + 1];
  for (int f = tid; f < nfine; f += PT_THREADS) tcnt[f] = 0;
  __syncthreads();
  for (int64_t i = s0 + tid; i < s1; i += PT_THREADS) atomicAdd(&tcnt[(key2[i] >> F) & (nfine - 1)], 1u);
  __syncthreads();
  pt_scan(tcnt, tofs, nfine, wsum);
  for (int f = tid; f < nfine; f += PT_THREADS) {
    base[f] = s0 + tofs[f];
    cur[f] = 0;
    const int64_t fb = d * nfine + f;
    if (fb < nfb) foff[fb] = s0 + tofs[f];
  }
  if (d == gridDim.x - 1 && tid == 0) foff[nfb] = n;
  __syncthreads();
  auto dig = [F, nfine](uint64_t k) -> int { return (int)((k >> F) & (nfine - 1)); };
  for (int64_t t0 = s0; t0 < s1; t0 += PT_TILE)
    pt_tile(key2, val2, t0, min(s1, t0 + PT_TILE), nfine, dig, base, cur, tcnt, tofs, stage, wsum, key, val);
}

// Pass 3: fine buckets in ticket order; bucket b holds the terms
// [foff[b], foff[b+1]) of (key, val), codes in [b << F, (b + 1) << F).
__global__ void __launch_bounds__(PR_THREADS) k_pt_rank(uint64_t* __restrict__ key, uint64_t* __restrict__ val,
                                                       int F, int64_t nfb, const int64_t* __restrict__ foff,
                                                       unsigned long long* __restrict__ ticket,
                                                       uint64_t* __restrict__ key2, uint64_t* __restrict__ val2) {
  extern __shared__ __align__(16) unsigned char pt_smem[];
  uint64_t* stage = (uint64_t*)pt_smem;                                       // 2 * PT_SMAX
  unsigned long long* bits = (unsigned long long*)(pt_smem + 16 * PT_SMAX);   // [2^(F-6)]
  const int nw = 1 << (F - 6);
  uint32_t* pre = (uint32_t*)(bits + nw);                                     // [2^(F-6)]
  __shared__ uint32_t wsum[PR_THREADS / 32];
  __shared__ int64_t s_b;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_b = (int64_t)atomicAdd(ticket, 1ull);
    __syncthreads();
    const int64_t b = s_b;
    __syncthreads();
    if (b >= nfb) break;
    const int64_t s0 = foff[b], s1 = foff[b + 1];
    const int64_t m = s1 - s0;
    if (m < 2) continue;   // uniform across the CTA
    if (m <= PT_CMP_MAX) {
      // a small bucket: ranks by comparison (each term's rank is the number of
      // the bucket's keys below it; keys are distinct), from a shared copy
      for (int64_t j = tid; j < m; j += PR_THREADS) {
        stage[j] = key[s0 + j];
        stage[PT_SMAX + j] = val[s0 + j];
      }
      __syncthreads();
      for (int64_t j = tid; j < m; j += PR_THREADS) {
        const uint64_t k = stage[j];
        int64_t rank = 0;
        for (int64_t u = 0; u < m; ++u) rank += stage[u] < k ? 1 : 0;
        key[s0 + rank] = k;
        val[s0 + rank] = stage[PT_SMAX + j];
      }
      __syncthreads();   // stage is reused by the next bucket
      continue;
    }
    for (int w = tid; w < nw; w += PR_THREADS) bits[w] = 0ull;
    __syncthreads();
    const uint64_t lo = (uint64_t)b << F;
    const uint64_t span = uint64_t(1) << F;
    for (int64_t i = s0 + tid; i < s1; i += PR_THREADS) {
      const uint64_t c = key[i] - lo;   // < 2^F for the bucket's keys
      if (c < span) atomicOr(&bits[c >> 6], 1ull << (c & 63));
    }
    __syncthreads();
    // word prefix counts (nw <= 2048 words)
    for (int w = tid; w < nw; w += PR_THREADS) pre[w] = (uint32_t)__popcll(bits[w]);
    __syncthreads();
    pt_scan<PR_THREADS>(pre, pre, nw, wsum);   // in place: each thread reads its entries before writing them
    if (m <= PT_SMAX) {
      for (int64_t i = s0 + tid; i < s1; i += PR_THREADS) {
        const uint64_t k = key[i];
        const uint64_t c = k - lo;
        if (c >= span) continue;
        const uint32_t rank = pre[c >> 6] + (uint32_t)__popcll(bits[c >> 6] & ((1ull << (c & 63)) - 1ull));
        stage[rank] = k;
        stage[PT_SMAX + rank] = val[i];
      }
      __syncthreads();
      for (int64_t j = tid; j < m; j += PR_THREADS) {
        key[s0 + j] = stage[j];
        val[s0 + j] = stage[PT_SMAX + j];
      }
    } else {
      for (int64_t i = s0 + tid; i < s1; i += PR_THREADS) {
        const uint64_t k = key[i];
        const uint64_t c = k - lo;
        if (c >= span) continue;
        const uint32_t rank = pre[c >> 6] + (uint32_t)__popcll(bits[c >> 6] & ((1ull << (c & 63)) - 1ull));
        key2[s0 + rank] = k;
        val2[s0 + rank] = val[i];
      }
      __syncthreads();   // this CTA's writes to (key2, val2) are visible to it
      for (int64_t j = s0 + tid; j < s1; j += PR_THREADS) {
        key[j] = key2[j];
        val[j] = val2[j];
      }
    }
    __syncthreads();   // bits, pre and stage are reused by the next bucket
  }
}

static cudaError_t order_by_partition(uint64_t* key, uint64_t* val, uint64_t* key2, uint64_t* val2, int64_t n,
                                      const PtPlan& pl, int64_t* bins, cudaStream_t s) {
  const int nsup = (int)pl.nsup;
  int64_t* soff = bins;                                                   // [nsup + 1]
  unsigned long long* scur = (unsigned long long*)(bins + nsup + 1);      // [nsup], then the ticket
  int64_t* foff = bins + 2 * (nsup + 1);                                  // [nfb + 1]
  int64_t* scan = foff + pl.nfb + 1;
  cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(int64_t) * 2 * (nsup + 1), s);
  if (e != cudaSuccess) return e;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (n + 4 * PT_TILE - 1) / (4 * PT_TILE);   // slices of at least four tiles
  if (grid > sms) grid = sms;                              // one CTA per SM (128 KB of staging each)
  if (grid < 1) grid = 1;
  const size_t csm = (size_t)nsup * 4;
  const size_t ssm = (size_t)16 * PT_TILE + (size_t)nsup * 20;
  const size_t fsm = (size_t)16 * PT_TILE;
  const size_t rsm = (size_t)16 * PT_SMAX + ((size_t)1 << (pl.F - 6)) * 12;
  if ((e = raise_smem_limit((const void*)k_pt_count, csm)) != cudaSuccess ||
      (e = raise_smem_limit((const void*)k_pt_super, ssm)) != cudaSuccess ||
      (e = raise_smem_limit((const void*)k_pt_fine, fsm)) != cudaSuccess ||
      (e = raise_smem_limit((const void*)k_pt_rank, rsm)) != cudaSuccess)
    return e;
  const int sh = pl.F + pl.fbits;   // a key's super-bucket: key >> sh
  k_pt_count<<<(unsigned)grid, PT_THREADS, csm, s>>>(key, n, sh, nsup, (unsigned long long*)soff);
  if ((e = launch_scan_exclusive(soff, nsup, soff + nsup, scan, s)) != cudaSuccess) return e;
  k_pt_super<<<(unsigned)grid, PT_THREADS, ssm, s>>>(key, val, n, sh, nsup, soff, scur, key2, val2);
  k_pt_fine<<<(unsigned)nsup, PT_THREADS, fsm, s>>>(key2, val2, n, pl.F, pl.fbits, pl.nfb, soff, foff, key, val);
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pt_rank, PR_THREADS, rsm) != cudaSuccess || per < 1) {
    cudaGetLastError();
    per = 1;
  }
  k_pt_rank<<<(unsigned)(sms * per), PR_THREADS, rsm, s>>>(key, val, pl.F, pl.nfb, foff, scur + nsup, key2,
                                                         val2);
  return cudaGetLastError();
}

// Counting and scatter by bucket, each CTA over one contiguous slice of the
// terms: a shared-memory histogram of the slice, one global atomic per
// (CTA, bucket) (the per-term global atomics of a direct count would pile
// onto a few thousand counters), then in the scatter each term's place in its
// bucket is the CTA's reserved base plus a shared-memory rank.
constexpr int BK_CTA_THREADS = 512;
constexpr int BK_MAX_SMEM_BUCKETS = 8192;   // histogram in shared memory up to this many buckets


__global__ void __launch_bounds__(BK_CTA_THREADS) k_bk_count(const uint64_t* __restrict__ key, int64_t n,
                                                             int64_t nb, unsigned long long* __restrict__ cnt) {
  extern __shared__ uint32_t bh[];
  const bool local = nb <= BK_MAX_SMEM_BUCKETS;
  if (local)
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) bh[b] = 0;
  __syncthreads();
  int64_t a, e;
  bk_slice(n, &a, &e);
  for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) {
    const uint64_t b = key[i] >> BK_LOG2;
    if (b >= (uint64_t)nb) continue;
    if (local) atomicAdd(&bh[b], 1u);
    else atomicAdd(&cnt[b], 1ull);
  }
  __syncthreads();
  if (local)
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x)
      if (bh[b]) atomicAdd(&cnt[b], (unsigned long long)bh[b]);
}

__global__ void __launch_bounds__(BK_CTA_THREADS) k_bk_scatter(const uint64_t* __restrict__ key,
                                                               const uint64_t* __restrict__ val, int64_t n,
                                                               int64_t nb, const int64_t* __restrict__ off,
                                                               unsigned long long* __restrict__ cur,
                                                               uint64_t* __restrict__ okey,
                                                               uint64_t* __restrict__ oval) {
  extern __shared__ uint32_t bh[];   // [nb] slice counts, then ranks; [nb] bases (uint64 pairs)
  const bool local = nb <= BK_MAX_SMEM_BUCKETS;
  unsigned long long* base = (unsigned long long*)(bh + ((nb + 1) & ~int64_t(1)));
  int64_t a, e;
  bk_slice(n, &a, &e);
  if (local) {
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) bh[b] = 0;
    __syncthreads();
    for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) {
      const uint64_t b = key[i] >> BK_LOG2;
      if (b < (uint64_t)nb) atomicAdd(&bh[b], 1u);
    }
    __syncthreads();
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) {
      base[b] = bh[b] ? atomicAdd(&cur[b], (unsigned long long)bh[b]) : 0ull;
      bh[b] = 0;
    }
    __syncthreads();
  }
  for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) {
    const uint64_t k = key[i];
    const int64_t b = (int64_t)(k >> BK_LOG2);
    if (b >= nb) continue;
    const uint64_t r = local ? base[b] + atomicAdd(&bh[b], 1u) : atomicAdd(&cur[b], 1ull);
    const int64_t pos = off[b] + (int64_t)r;
    if (pos < off[b + 1]) {
      okey[pos] = k;
      oval[pos] = val[i];
    }
  }
}

// One CTA per bucket b: terms [off[b], off[b+1]) of (key, val), written sorted
// to the same range of (okey, oval).
__global__ void __launch_bounds__(BK_THREADS) k_bk_rank(const uint64_t* __restrict__ key,
                                                        const uint64_t* __restrict__ val,
                                                        const int64_t* __restrict__ off,
                                                        uint64_t* __restrict__ okey, uint64_t* __restrict__ oval) {
  extern __shared__ __align__(16) unsigned char bk_smem[];
  unsigned long long* bits = (unsigned long long*)bk_smem;      // [BK_WORDS]
  uint32_t* pre = (uint32_t*)(bk_smem + 8 * BK_WORDS);          // [BK_WORDS] ones before the word
  __shared__ uint32_t wsum[BK_THREADS / 32];
  const int64_t b = blockIdx.x;
  const int64_t s0 = off[b], s1 = off[b + 1];
  if (s1 <= s0) return;
  for (int w = threadIdx.x; w < BK_WORDS; w += blockDim.x) bits[w] = 0ull;
  __syncthreads();
  const uint64_t base = (uint64_t)b << BK_LOG2;
  for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
    const uint32_t c = (uint32_t)(key[i] - base);   // < BK_CODES
    atomicOr(&bits[c >> 6], 1ull << (c & 63));
  }
  __syncthreads();
  // exclusive prefix of the words' popcounts: each thread owns BK_WORDS / BK_THREADS consecutive words
  constexpr int PER = BK_WORDS / BK_THREADS;
  const int w0 = threadIdx.x * PER;
  uint32_t local[PER];
  uint32_t tsum = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    local[q] = tsum;
    tsum += (uint32_t)__popcll(bits[w0 + q]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < BK_THREADS / 32 ? wsum[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < BK_THREADS / 32) wsum[lane] = v;
  }
  __syncthreads();
  const uint32_t tbase = (warp > 0 ? wsum[warp - 1] : 0u) + x - tsum;
#pragma unroll
  for (int q = 0; q < PER; ++q) pre[w0 + q] = tbase + local[q];
  __syncthreads();
  for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
    const uint64_t k = key[i];
    const uint32_t c = (uint32_t)(k - base);
    const uint32_t w = c >> 6;
    const int64_t rank = (int64_t)pre[w] + __popcll(bits[w] & ((1ull << (c & 63)) - 1ull));
    if (s0 + rank < s1) {
      okey[s0 + rank] = k;
      oval[s0 + rank] = val[i];
    }
  }
}

// Sorts (key, val)[0, n) by key (distinct keys < krange) in place, through
// key2/val2 (n terms of scratch); bins: order_buckets_scratch(krange) int64.
cudaError_t order_by_buckets(uint64_t* key, uint64_t* val, uint64_t* key2, uint64_t* val2, int64_t n,
                             int64_t krange, int64_t* bins, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
#if KR_ORDER_PARTITION
  const PtPlan pl = pt_plan(n, krange);
  if (pl.ok) return order_by_partition(key, val, key2, val2, n, pl, bins, s);
#endif
  const int64_t nb = order_buckets(krange);
  int64_t* off = bins;                                               // [nb + 1]
  unsigned long long* cur = (unsigned long long*)(bins + nb + 1);    // [nb + 1]
  cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(int64_t) * 2 * (nb + 1), s);
  if (e != cudaSuccess) return e;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // slices of at least 4096 terms, at most a few CTAs per SM
  int64_t grid = (n + 4095) / 4096;
  if (grid > (int64_t)sms * 4) grid = (int64_t)sms * 4;
  if (grid < 1) grid = 1;
  const bool local = nb <= BK_MAX_SMEM_BUCKETS;
  const size_t csm = local ? (size_t)nb * 4 : 0;
  const size_t ssm = local ? (size_t)((nb + 1) & ~int64_t(1)) * 4 + (size_t)nb * 8 : 0;
  if ((e = raise_smem_limit((const void*)k_bk_count, csm)) != cudaSuccess ||
      (e = raise_smem_limit((const void*)k_bk_scatter, ssm)) != cudaSuccess)
    return e;
  k_bk_count<<<(unsigned)grid, BK_CTA_THREADS, csm, s>>>(key, n, nb, (unsigned long long*)off);
  e = launch_scan_exclusive(off, nb, off + nb, bins + 2 * (nb + 1), s);
  if (e != cudaSuccess) return e;
  k_bk_scatter<<<(unsigned)grid, BK_CTA_THREADS, ssm, s>>>(key, val, n, nb, off, cur, key2, val2);
  const size_t smem = (size_t)BK_WORDS * 12;
  e = raise_smem_limit((const void*)k_bk_rank, smem);
  if (e != cudaSuccess) return e;
  k_bk_rank<<<(unsigned)nb, BK_THREADS, smem, s>>>(key2, val2, off, key, val);
  return cudaGetLastError();
}

int64_t order_bins(int64_t krange) { return (krange + ORD_C - 1) / ORD_C; }
int64_t order_bins_scratch(int64_t krange) {
  const int64_t nb = order_bins(krange);
  return 2 * (nb + 1) + scan_scratch_entries(nb);
}

// ---------------------------------------------------------------------------
// bitmap rank ordering
// layout: bits[W64] (uint64), wpre[W64] (uint32: ones in the superblock before
// the word), spre[NSB + 1] (int64: ones before the superblock); a superblock
// is BM_SB words
// ---------------------------------------------------------------------------
constexpr int BM_SB = 1024;   // words per superblock (65536 codes)

static int64_t bm_words(int64_t krange) { return (krange + 63) / 64; }
static int64_t bm_sblocks(int64_t krange) { return (bm_words(krange) + BM_SB - 1) / BM_SB; }

int64_t order_bitmap_bytes(int64_t krange) {
  const int64_t w = bm_sblocks(krange) * BM_SB;
  // bitmap, word prefixes, superblock prefixes (+ total), the scan's block sums
  return w * 8 + w * 4 + (bm_sblocks(krange) + 1) * 8 + scan_scratch_entries(bm_sblocks(krange)) * 8 +
         4 * 256;
}

__global__ void __launch_bounds__(256) k_bm_set(const uint64_t* __restrict__ key, int64_t n, int64_t krange,
                                                unsigned long long* __restrict__ bits) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = key[i];
    if (k < (uint64_t)krange) atomicOr(&bits[k >> 6], 1ull << (k & 63));
  }
}

// one CTA per superblock: exclusive popcount prefix of its words, and its total
__global__ void __launch_bounds__(BM_SB) k_bm_prefix(const unsigned long long* __restrict__ bits,
                                                     uint32_t* __restrict__ wpre, int64_t* __restrict__ stot) {
  __shared__ uint32_t ws[BM_SB / 32];
  const int64_t w = (int64_t)blockIdx.x * BM_SB + threadIdx.x;
  const uint32_t c = (uint32_t)__popcll(bits[w]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = c;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = ws[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    ws[lane] = v;
  }
  __syncthreads();
  wpre[w] = (warp > 0 ? ws[warp - 1] : 0) + x - c;
  if (threadIdx.x == BM_SB - 1) stot[blockIdx.x] = (int64_t)((warp > 0 ? ws[warp - 1] : 0) + x);
}

__global__ void __launch_bounds__(256) k_bm_scatter(const uint64_t* __restrict__ key,
                                                    const uint64_t* __restrict__ val, int64_t n,
                                                    int64_t krange,
                                                    const unsigned long long* __restrict__ bits,
                                                    const uint32_t* __restrict__ wpre,
                                                    const int64_t* __restrict__ spre,
                                                    uint64_t* __restrict__ okey,
                                                    uint64_t* __restrict__ oval) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = key[i];
    if (k >= (uint64_t)krange) continue;
    const int64_t w = (int64_t)(k >> 6);
    const uint64_t below = bits[w] & ((1ull << (k & 63)) - 1ull);
    const int64_t rank = spre[w / BM_SB] + wpre[w] + __popcll(below);
    if (rank < n) {
      okey[rank] = k;
      oval[rank] = val[i];
    }
  }
}

// Sorts (key, val)[0, n) by key (distinct keys < krange) into key2/val2.
// scratch: order_bitmap_bytes(krange) bytes.
cudaError_t order_by_bitmap(const uint64_t* key, const uint64_t* val, uint64_t* key2, uint64_t* val2,
                            int64_t n, int64_t krange, void* scratch, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t nsb = bm_sblocks(krange);
  const int64_t nw = nsb * BM_SB;
  char* base = (char*)scratch;
  unsigned long long* bits = (unsigned long long*)base;
  uint32_t* wpre = (uint32_t*)(base + ((nw * 8 + 255) / 256) * 256);
  int64_t* spre = (int64_t*)((char*)wpre + ((nw * 4 + 255) / 256) * 256);
  cudaError_t e = cudaMemsetAsync(bits, 0, (size_t)nw * 8, s);
  if (e != cudaSuccess) return e;
  int64_t grid = (n + 255) / 256;
  if (grid > 152 * 16) grid = 152 * 16;
  k_bm_set<<<(unsigned)grid, 256, 0, s>>>(key, n, krange, bits);
  k_bm_prefix<<<(unsigned)nsb, BM_SB, 0, s>>>(bits, wpre, spre);
  e = launch_scan_exclusive(spre, nsb, spre + nsb, spre + nsb + 1, s);
  if (e != cudaSuccess) return e;
  k_bm_scatter<<<(unsigned)grid, 256, 0, s>>>(key, val, n, krange, bits, wpre, spre, key2, val2);
  return cudaGetLastError();
}

// Sorts (key, val)[0, n) by key, keys distinct and < krange.  Uses key2/val2
// as the binned copy and writes the sorted terms back to key/val.  bins:
// order_bins_scratch(krange) int64 of scratch.
cudaError_t order_by_bins(uint64_t* key, uint64_t* val, uint64_t* key2, uint64_t* val2, int64_t n,
                          int64_t krange, int64_t* bins, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  const int64_t nb = order_bins(krange);
  int64_t* off = bins;
  unsigned long long* cur = (unsigned long long*)(bins + nb + 1);
  cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(int64_t) * 2 * (nb + 1), s);
  if (e != cudaSuccess) return e;
  int64_t grid = (n + 255) / 256;
  if (grid > 152 * 16) grid = 152 * 16;
  k_bin_count<<<(unsigned)grid, 256, 0, s>>>(key, n, nb, (unsigned long long*)off);
  e = launch_scan_exclusive(off, nb, off + nb, bins + 2 * (nb + 1), s);
  if (e != cudaSuccess) return e;
  k_bin_scatter<<<(unsigned)grid, 256, 0, s>>>(key, val, n, nb, off, cur, key2, val2);
  const int64_t nseg = (n + ORD_C - 1) / ORD_C;
  const int smem = (int)((sizeof(uint64_t) + sizeof(uint16_t)) * ORD_SEG);
  e = raise_smem_limit((const void*)k_seg_sort, (size_t)smem);
  if (e != cudaSuccess) return e;
  k_seg_sort<<<(unsigned)nseg, ORD_THREADS, smem, s>>>(key2, val2, off, nb, key, val);
  return cudaGetLastError();
}

}  // namespace kr
