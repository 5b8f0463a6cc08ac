// Term ordering (Sec. 3.1: the factors are sorted by ascending code so that
// the output is written in order and each block of output codes meets a
// contiguous range of each factor, the property behind the disjoint output
// intervals of Sec. 4).  Three sorts, chosen per operand by the host:
//  * bitmap: keys are distinct and their range fits an on-chip bitmap; the
//    rank of a key is the number of set bits below it (one pass, O(n + range/32));
//  * bitonic: a shared-memory bitonic network over (key << idx_bits | index)
//    words for n <= 16384 (all merges ascending, so padding to a power of two
//    needs no storage);
//  * radix: device-wide LSD radix sort of (key, payload) pairs, 8-bit digits,
//    also used for the hash-path output.
// Plus a single-CTA exclusive scan used by the compaction and the radix sort.
#include "kr_internal.cuh"

namespace kr {

// ---------------------------------------------------------------------------
// block-wide exclusive scan of int64 values held one per thread
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t s = lane < NT / 32 ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NT / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  int64_t base = warp > 0 ? warp_sums[warp - 1] : 0;
  if (total) *total = warp_sums[NT / 32 - 1];
  __syncthreads();
  return base + x - v;
}

// ---------------------------------------------------------------------------
// single-CTA exclusive scan of d[0, n); d[n] is not touched; *total = sum
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_scan_exclusive(int64_t* __restrict__ d, int64_t n,
                                                         int64_t* __restrict__ total) {
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t a = min(n, per * threadIdx.x), b = min(n, a + per);
  int64_t s = 0;
  for (int64_t i = a; i < b; ++i) s += d[i];
  int64_t tot;
  int64_t run = block_exclusive_scan<1024>(s, &tot);
  for (int64_t i = a; i < b; ++i) {
    int64_t x = d[i];
    d[i] = run;
    run += x;
  }
  if (threadIdx.x == 0 && total) *total = tot;
}

// ---------------------------------------------------------------------------
// multi-CTA exclusive scan for long arrays: block sums, a scan of the sums,
// then each block scanned with its offset.  scratch: scan_scratch_entries(n).
// ---------------------------------------------------------------------------
constexpr int SC_THREADS = 1024;
constexpr int SC_ITEMS = 8;
constexpr int64_t SC_BLOCK = (int64_t)SC_THREADS * SC_ITEMS;
constexpr int64_t SC_ONE_CTA_MAX = 65536;

int64_t scan_scratch_entries(int64_t n) { return (n + SC_BLOCK - 1) / SC_BLOCK + 1; }

__global__ void __launch_bounds__(SC_THREADS) k_scan_sums(const int64_t* __restrict__ d, int64_t n,
                                                          int64_t* __restrict__ sums) {
  const int64_t b0 = blockIdx.x * SC_BLOCK;
  int64_t s = 0;
#pragma unroll
  for (int r = 0; r < SC_ITEMS; ++r) {
    const int64_t i = b0 + (int64_t)r * SC_THREADS + threadIdx.x;
    if (i < n) s += d[i];
  }
  int64_t tot;
  block_exclusive_scan<SC_THREADS>(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_blocks(int64_t* __restrict__ d, int64_t n,
                                                            const int64_t* __restrict__ sums) {
  // each thread scans SC_ITEMS consecutive values
  const int64_t i0 = blockIdx.x * SC_BLOCK + (int64_t)threadIdx.x * SC_ITEMS;
  int64_t v[SC_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int r = 0; r < SC_ITEMS; ++r) {
    v[r] = i0 + r < n ? d[i0 + r] : 0;
    s += v[r];
  }
  int64_t run = sums[blockIdx.x] + block_exclusive_scan<SC_THREADS>(s, nullptr);
#pragma unroll
  for (int r = 0; r < SC_ITEMS; ++r) {
    if (i0 + r < n) d[i0 + r] = run;
    run += v[r];
  }
}

cudaError_t launch_scan_exclusive(int64_t* d, int64_t n, int64_t* dtotal, int64_t* scratch, cudaStream_t s) {
  if (n <= SC_ONE_CTA_MAX || !scratch) {
    k_scan_exclusive<<<1, 1024, 0, s>>>(d, n, dtotal);
    return cudaGetLastError();
  }
  const int64_t nb = (n + SC_BLOCK - 1) / SC_BLOCK;
  k_scan_sums<<<(unsigned)nb, SC_THREADS, 0, s>>>(d, n, scratch);
  k_scan_exclusive<<<1, 1024, 0, s>>>(scratch, nb, dtotal);   // offsets of the blocks, and the total
  k_scan_blocks<<<(unsigned)nb, SC_THREADS, 0, s>>>(d, n, scratch);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// bitmap rank sort (one CTA per operand).  Shared memory: the bitmap (32-bit
// words, padded to groups of 32 words) and, per 8 words, the number of set
// bits before them, so the rank of a key costs at most 8 popcounts.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_bitmap_sort(Prod* __restrict__ prods,
                                                      const OpRef* __restrict__ ops) {
  extern __shared__ uint32_t sm[];
  const OpRef r = ops[blockIdx.x];
  Prod& P = prods[r.prod];
  Operand& O = r.which ? P.g : P.f;
  const int64_t nwords = (O.key_range + 31) >> 5;
  const int64_t ngroups = (nwords + 31) >> 5;
  const int64_t nw = ngroups * 32;       // padded bitmap words
  const int64_t n8 = nw >> 3;            // 8-word blocks
  uint32_t* bits = sm;
  uint32_t* pre8 = sm + nw;
  for (int64_t w = threadIdx.x; w < nw; w += blockDim.x) bits[w] = 0;
  __syncthreads();
  uint32_t dup = 0;
  for (int64_t i = threadIdx.x; i < O.n; i += blockDim.x) {
    const uint64_t key = O.skey[i];
    const uint32_t bit = 1u << (key & 31);
    const uint32_t old = atomicOr(&bits[key >> 5], bit);
    if (old & bit) dup = 1;
  }
  __syncthreads();
  // set bits per 8-word block, each thread over a contiguous range of blocks,
  // then an exclusive scan over the threads
  const int64_t per = (n8 + blockDim.x - 1) / blockDim.x;
  const int64_t ba = min(n8, per * threadIdx.x), bb = min(n8, ba + per);
  int64_t s = 0;
  for (int64_t b = ba; b < bb; ++b) {
    const uint4 lo = *(const uint4*)&bits[8 * b];
    const uint4 hi = *(const uint4*)&bits[8 * b + 4];
    const uint32_t c = __popc(lo.x) + __popc(lo.y) + __popc(lo.z) + __popc(lo.w) +
                       __popc(hi.x) + __popc(hi.y) + __popc(hi.z) + __popc(hi.w);
    pre8[b] = c;
    s += c;
  }
  int64_t run = block_exclusive_scan<1024>(s, nullptr);
  for (int64_t b = ba; b < bb; ++b) {
    const uint32_t c = pre8[b];
    pre8[b] = (uint32_t)run;
    run += c;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < O.n; i += blockDim.x) {
    const uint64_t key = O.skey[i];
    const int64_t w = (int64_t)(key >> 5);
    uint32_t rank = pre8[w >> 3];
    for (int64_t x = w & ~(int64_t)7; x < w; ++x) rank += __popc(bits[x]);
    rank += __popc(bits[w] & ((1u << (key & 31)) - 1u));
    if (rank >= O.n) { dup = 1; continue; }
    O.skey2[rank] = key;
    O.sidx2[rank] = (uint64_t)i;
  }
  if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) atomicOr(&P.status, ST_DUP);
}

// ---------------------------------------------------------------------------
// bitonic sort of n <= 16384 packed words in shared memory (one CTA per operand)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_bitonic_sort(Prod* __restrict__ prods,
                                                       const OpRef* __restrict__ ops) {
  extern __shared__ uint64_t sk[];
  const OpRef r = ops[blockIdx.x];
  Prod& P = prods[r.prod];
  Operand& O = r.which ? P.g : P.f;
  const int n = (int)O.n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sk[i] = O.skey[i];
  __syncthreads();
  int N = 1;
  while (N < n) N <<= 1;
  const int pairs = N >> 1;
  for (int size = 2; size <= N; size <<= 1) {
    const int half = size >> 1;
    // merge two ascending runs: compare i with its mirror in the block of `size`
    for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
      const int blk = p / half, off = p - blk * half;
      const int i = blk * size + off, j = blk * size + size - 1 - off;
      if (j < n) {
        uint64_t a = sk[i], b = sk[j];
        if (a > b) { sk[i] = b; sk[j] = a; }
      }
    }
    __syncthreads();
    for (int stride = half >> 1; stride > 0; stride >>= 1) {
      for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
        const int i = (p / stride) * 2 * stride + (p % stride), j = i + stride;
        if (j < n) {
          uint64_t a = sk[i], b = sk[j];
          if (a > b) { sk[i] = b; sk[j] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) O.skey[i] = sk[i];
}

cudaError_t launch_sort_small(Prod* dprods, const OpRef* dops, int nops, int method, size_t smem,
                              cudaStream_t s) {
  if (nops <= 0) return cudaSuccess;
  if (method == SORT_BITMAP) {
    cudaError_t e = raise_smem_limit((const void*)k_bitmap_sort, (size_t)smem);
    if (e != cudaSuccess) return e;
    k_bitmap_sort<<<nops, 1024, smem, s>>>(dprods, dops);
  } else {
    cudaError_t e = raise_smem_limit((const void*)k_bitonic_sort, (size_t)smem);
    if (e != cudaSuccess) return e;
    k_bitonic_sort<<<nops, 1024, smem, s>>>(dprods, dops);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// device-wide LSD radix sort, 8-bit digits, stable
// counts layout: counts[digit * ntiles + tile]
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = RADIX_TILE / RS_THREADS;   // 16 rounds of 256 elements

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t* __restrict__ key, int64_t n,
                                                        int shift, int64_t ntiles,
                                                        int64_t* __restrict__ counts) {
  __shared__ uint32_t h[256];
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = tile * RADIX_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
      const int64_t i = base + r * RS_THREADS + threadIdx.x;
      if (i < n) atomicAdd(&h[(key[i] >> shift) & 255], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + tile] = h[threadIdx.x];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t* __restrict__ key,
                                                           const uint64_t* __restrict__ val, int64_t n,
                                                           int shift, int64_t ntiles,
                                                           const int64_t* __restrict__ offs,
                                                           uint64_t* __restrict__ key_out,
                                                           uint64_t* __restrict__ val_out) {
  constexpr int NW = RS_THREADS / 32;
  __shared__ int64_t base[256];
  __shared__ uint32_t wcount[NW][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    base[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + tile];
    const int64_t t0 = tile * RADIX_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
      for (int d = lane; d < 256; d += 32) wcount[warp][d] = 0;
      __syncthreads();
      const int64_t i = t0 + r * RS_THREADS + threadIdx.x;
      const bool ok = i < n;
      uint64_t k = 0, v = 0;
      int d = 256;
      if (ok) { k = key[i]; v = val[i]; d = (int)((k >> shift) & 255); }
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t rank = __popc(peers & lt);
      if (ok && rank == 0) wcount[warp][d] = __popc(peers);
      __syncthreads();
      {
        // per digit: exclusive offsets over the warps, advance the tile base
        const int dd = threadIdx.x;
        int64_t run = 0;
        for (int w = 0; w < NW; ++w) {
          uint32_t c = wcount[w][dd];
          wcount[w][dd] = (uint32_t)run;
          run += c;
        }
        // base[dd] is read below by every thread; advance after the reads
        __syncthreads();
        if (ok) {
          const int64_t pos = base[d] + wcount[warp][d] + rank;
          key_out[pos] = k;
          val_out[pos] = v;
        }
        __syncthreads();
        base[dd] += run;
      }
      __syncthreads();
    }
  }
}

int64_t radix_scan_entries(int64_t n) {
  const int64_t e = 256 * ((n + RADIX_TILE - 1) / RADIX_TILE);
  return e + 1 + scan_scratch_entries(e);   // digit counts, their total, the scan's block sums
}

cudaError_t radix_sort_pairs(uint64_t* key, uint64_t* val, uint64_t* key_tmp, uint64_t* val_tmp,
                             int64_t n, int bits, int64_t* dscan, cudaStream_t s,
                             bool* result_in_tmp) {
  *result_in_tmp = false;
  if (n <= 1 || bits <= 0) return cudaSuccess;
  const int64_t ntiles = (n + RADIX_TILE - 1) / RADIX_TILE;
  const int grid = (int)(ntiles < 152 * 8 ? ntiles : 152 * 8);
  uint64_t *ki = key, *vi = val, *ko = key_tmp, *vo = val_tmp;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<grid, RS_THREADS, 0, s>>>(ki, n, shift, ntiles, dscan);
    cudaError_t e = launch_scan_exclusive(dscan, 256 * ntiles, dscan + 256 * ntiles, dscan + 256 * ntiles + 1, s);
    if (e != cudaSuccess) return e;
    k_rs_scatter<<<grid, RS_THREADS, 0, s>>>(ki, vi, n, shift, ntiles, dscan, ko, vo);
    uint64_t* t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
    *result_in_tmp = !*result_in_tmp;
  }
  return cudaGetLastError();
}

}  // namespace kr
