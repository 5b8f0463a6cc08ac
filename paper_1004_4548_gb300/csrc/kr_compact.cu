// Compaction: the accumulators (dense array or hash table) -> a sparse list of
// (code, coefficient) terms with the zero coefficients dropped (the output is
// again a sparse distributed vector, Sec. 3.1).  Two passes over fixed chunks
// of every product's accumulator: count the nonzero slots, exclusive scan,
// then write each chunk's terms in slot order at its offset.  The dense
// array's slot order is code order, so the dense output comes out sorted.
#include "kr_internal.cuh"

namespace kr {

constexpr int CP_THREADS = 256;

template <int NT>
__device__ __forceinline__ int block_excl_scan_int(int v, int* total) {
  __shared__ int ws[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int s = lane < NT / 32 ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NT / 32) ws[lane] = s;
  }
  __syncthreads();
  const int base = warp > 0 ? ws[warp - 1] : 0;
  *total = ws[NT / 32 - 1];
  __syncthreads();
  return base + x - v;
}

__device__ __forceinline__ bool slot_live(const Prod& P, int64_t s, uint64_t* key, uint64_t* val) {
  if (P.path == PATH_DENSE) {
    const uint64_t v = ((const uint64_t*)P.dense)[s];
    *key = (uint64_t)s;
    *val = v;
    // int64 zero or float64 +-0.0
    return (v << 1) != 0 || (!P.f64 && v != 0);
  }
  const uint64_t k = __ldcg(P.table + 2 * s);
  const uint64_t v = __ldcg(P.table + 2 * s + 1);
  *key = k - 1;
  *val = v;
  return k != 0 && ((v << 1) != 0 || (!P.f64 && v != 0));
}

__device__ __forceinline__ int find_prod_of_chunk(const int64_t* chunk_begin, int nprod, int64_t c) {
  int lo = 0, hi = nprod - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (chunk_begin[mid] <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int64_t accum_slots(const Prod& P) {
  return P.path == PATH_DENSE ? P.krange : P.slots;
}

__global__ void __launch_bounds__(CP_THREADS) k_compact_count(const Prod* __restrict__ prods, int nprod,
                                                              const int64_t* __restrict__ chunk_begin,
                                                              int64_t* __restrict__ counts) {
  const int64_t nchunks = chunk_begin[nprod];
  __shared__ int red[CP_THREADS / 32];
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int p = find_prod_of_chunk(chunk_begin, nprod, c);
    const Prod& P = prods[p];
    int n = 0;
    if (P.status == 0) {
      const int64_t s0 = (c - chunk_begin[p]) * P.chunk;
      const int64_t s1 = min(accum_slots(P), s0 + P.chunk);
      for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        uint64_t k, v;
        n += slot_live(P, s, &k, &v) ? 1 : 0;
      }
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < CP_THREADS / 32; ++w) t += red[w];
      counts[c] = t;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(CP_THREADS) k_compact_scatter(const Prod* __restrict__ prods, int nprod,
                                                                const int64_t* __restrict__ chunk_begin,
                                                                const int64_t* __restrict__ offs,
                                                                int64_t cap,
                                                                uint64_t* __restrict__ okey,
                                                                uint64_t* __restrict__ oval) {
  const int64_t nchunks = chunk_begin[nprod];
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int p = find_prod_of_chunk(chunk_begin, nprod, c);
    const Prod& P = prods[p];
    if (P.status != 0) continue;   // uniform across the CTA
    const int64_t s0 = (c - chunk_begin[p]) * P.chunk;
    const int64_t s1 = min(accum_slots(P), s0 + P.chunk);
    int64_t run = offs[c];
    for (int64_t sb = s0; sb < s1; sb += blockDim.x) {
      const int64_t s = sb + threadIdx.x;
      uint64_t k = 0, v = 0;
      const bool live = s < s1 && slot_live(P, s, &k, &v);
      int tot;
      const int pos = block_excl_scan_int<CP_THREADS>(live ? 1 : 0, &tot);
      if (live && run + pos < cap) {
        okey[run + pos] = k;
        oval[run + pos] = v;
      }
      run += tot;
    }
  }
}

// per product: where its terms start in the output arrays and how many there are
__global__ void k_finish_counts(Prod* __restrict__ prods, int nprod,
                                const int64_t* __restrict__ chunk_begin,
                                const int64_t* __restrict__ offs, const int64_t* __restrict__ total,
                                int64_t cap) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprod) return;
  Prod& P = prods[p];
  const int64_t a = chunk_begin[p], b = chunk_begin[p + 1];
  const int64_t nch = chunk_begin[nprod];
  const int64_t start = a < nch ? offs[a] : *total;
  const int64_t end = b < nch ? offs[b] : *total;
  P.out_start = start;
  P.nout = P.status ? 0 : end - start;
  if (end > cap) P.status |= ST_OUTCAP;   // terms beyond the output arrays were not written
}

cudaError_t launch_compact(Prod* dprods, int nprod, const int64_t* dchunk_begin, int64_t nchunks,
                           int64_t* dcounts, uint64_t* okey, uint64_t* oval, int64_t cap, cudaStream_t s) {
  if (nchunks > 0) {
    const int grid = (int)(nchunks < 152 * 8 ? nchunks : 152 * 8);
    k_compact_count<<<grid, CP_THREADS, 0, s>>>(dprods, nprod, dchunk_begin, dcounts);
    cudaError_t e = launch_scan_exclusive(dcounts, nchunks, dcounts + nchunks, s);
    if (e != cudaSuccess) return e;
    k_compact_scatter<<<grid, CP_THREADS, 0, s>>>(dprods, nprod, dchunk_begin, dcounts, cap, okey, oval);
  } else {
    cudaMemsetAsync(dcounts, 0, sizeof(int64_t), s);
  }
  k_finish_counts<<<(nprod + 127) / 128, 128, 0, s>>>(dprods, nprod, dchunk_begin, dcounts,
                                                      dcounts + nchunks, cap);
  return cudaGetLastError();
}

}  // namespace kr
