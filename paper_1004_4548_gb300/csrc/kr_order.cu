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
int64_t order_buckets_scratch(int64_t krange) {
  const int64_t nb = order_buckets(krange);
  return 3 * (nb + 1) + scan_scratch_entries(nb);
}

// Counting and scatter by bucket, each CTA over one contiguous slice of the
// terms: a shared-memory histogram of the slice, one global atomic per
// (CTA, bucket) (the per-term global atomics of a direct count would pile
// onto a few thousand counters), then in the scatter each term's place in its
// bucket is the CTA's reserved base plus a shared-memory rank.
constexpr int BK_CTA_THREADS = 512;
constexpr int BK_MAX_SMEM_BUCKETS = 8192;   // histogram in shared memory up to this many buckets

__device__ __forceinline__ void bk_slice(int64_t n, int64_t* a, int64_t* b) {
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  *a = min(n, (int64_t)blockIdx.x * per);
  *b = min(n, *a + per);
}

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
