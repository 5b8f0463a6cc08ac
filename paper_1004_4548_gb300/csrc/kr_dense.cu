// Dense (moderately sparse) path, Sec. 3.1: out[code_f + code_g] += C_f * C_g
// into an array indexed by code.
//
// GB300 design.  The output code range [0, W) is cut into blocks of S codes.
// Because both factors are sorted by code, the pairs (i, j) that land in the
// block [B, B + S) are, for each i, the contiguous j-range
// [lb(B - F_i), lb(B + S - F_i)) of the sorted g codes, and the i that
// contribute at all form a contiguous range too: the disjoint-interval
// argument of Sec. 4 applied to output blocks instead of input blocks.  Each
// block is accumulated by one CTA in a shared-memory slice (atomic adds on
// int64 or float64), then flushed to device memory once.  Heavy blocks are
// split into several tasks over disjoint i-ranges; their flushes combine with
// global atomic adds into a zeroed array.  Tasks are fetched dynamically by a
// persistent grid.
#include "kr_internal.cuh"

namespace kr {

constexpr int PLAN_SAMPLES = 32;   // sampled i per block for the work estimate
constexpr int MAX_SPLIT = 64;      // tasks per block at most
constexpr int ACC_THREADS = 512;

// One warp per (dense product, block): i-range by binary search, sampled work
// estimate, then 1..MAX_SPLIT tasks over equal i-slices.
__global__ void __launch_bounds__(256) k_dense_plan(const Prod* __restrict__ prods,
                                                   const int32_t* __restrict__ dense_prods,
                                                   const int64_t* __restrict__ block_begin,
                                                   int ndense, DenseTask* __restrict__ tasks,
                                                   int64_t task_cap, int64_t* __restrict__ task_count) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t total = block_begin[ndense];
  if (gw >= total) return;
  // product owning global block gw
  int lo = 0, hi = ndense - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (block_begin[mid] <= gw) lo = mid; else hi = mid - 1;
  }
  const int pid = dense_prods[lo];
  const Prod& P = prods[pid];
  if (P.status) return;
  const int64_t b = gw - block_begin[lo];
  // a truncated product's code range ends inside its last block
  const int64_t B = b * P.S, E = min(B + P.S, P.krange);
  const int64_t* F = P.f.code;
  const int64_t* G = P.g.code;
  const int64_t nf = P.f.nkeep, ng = P.g.nkeep;   // dropped terms sort last
  if (nf <= 0 || ng <= 0) return;
  const int64_t i_lo = lower_bound_i64(F, nf, B - G[ng - 1]);
  const int64_t i_hi = lower_bound_i64(F, nf, E - G[0]);
  const int32_t* gx = P.gidx;
  const int64_t gn = P.gidx_n;
  const int gsh = P.gshift;
  if (i_lo >= i_hi) return;
  const int64_t span = i_hi - i_lo;
  int64_t cnt = 0;
  const int ns = span < PLAN_SAMPLES ? (int)span : PLAN_SAMPLES;
  if (lane < ns) {
    const int64_t i = i_lo + (span * lane) / ns;
    cnt = g_lower_bound(G, ng, gx, gn, gsh, E - F[i]) - g_lower_bound(G, ng, gx, gn, gsh, B - F[i]);
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane != 0) return;
  // a zero estimate does not prove an empty block (the samples may all miss),
  // so every block with a nonempty i-range gets at least one task
  const double est = (double)cnt * (double)span / (double)ns;
  int64_t k = (int64_t)(est / (double)P.work_target) + 1;
  if (k > MAX_SPLIT) k = MAX_SPLIT;
  if (k > span) k = span;
  const int64_t base = (int64_t)atomicAdd((unsigned long long*)task_count, (unsigned long long)k);
  for (int64_t t = 0; t < k; ++t) {
    if (base + t >= task_cap) break;
    DenseTask T;
    T.prod = pid;
    T.pad = 0;
    T.block = b;
    T.i0 = i_lo + (span * t) / k;
    T.i1 = i_lo + (span * (t + 1)) / k;
    T.single = (k == 1);
    tasks[base + t] = T;
  }
}

cudaError_t launch_dense_plan(const Prod* dprods, const int32_t* ddense_prods,
                              const int64_t* dblock_begin, int ndense, int64_t nblocks_total,
                              DenseTask* dtasks, int64_t task_cap, int64_t* dtask_count,
                              cudaStream_t s) {
  if (nblocks_total <= 0) return cudaSuccess;
  const int64_t threads = nblocks_total * 32;
  const int64_t grid = (threads + 255) / 256;
  k_dense_plan<<<(unsigned)grid, 256, 0, s>>>(dprods, ddense_prods, dblock_begin, ndense, dtasks,
                                              task_cap, dtask_count);
  return cudaGetLastError();
}

// Bucket index over the sorted g codes of every dense product: bucket b
// covers codes [b << gshift, (b + 1) << gshift); gidx[b] = lower_bound(b << gshift).
// Each j writes the buckets whose lower bound it is; the buckets after the
// last code get ng.
__global__ void __launch_bounds__(256) k_build_gindex(const Prod* __restrict__ prods,
                                                     const int32_t* __restrict__ dense_prods) {
  const Prod& P = prods[dense_prods[blockIdx.y]];
  const int64_t* G = P.g.code;
  const int64_t ng = P.g.n;
  const int sh = P.gshift;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= ng;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blo = j == 0 ? 0 : (G[j - 1] >> sh) + 1;
    const int64_t bhi = j == ng ? P.gidx_n : min(G[j] >> sh, P.gidx_n);
    for (int64_t b = blo; b <= bhi; ++b) P.gidx[b] = (int32_t)j;
  }
}

cudaError_t launch_build_gindex(const Prod* dprods, const int32_t* ddense_prods, int ndense,
                                int64_t max_ng, cudaStream_t s) {
  if (ndense <= 0) return cudaSuccess;
  int64_t gx = (max_ng + 1 + 255) / 256;
  if (gx > 64) gx = 64;
  k_build_gindex<<<dim3((unsigned)gx, ndense), 256, 0, s>>>(dprods, ddense_prods);
  return cudaGetLastError();
}

template <typename T>
__device__ __forceinline__ unsigned long long to_bits(T v);
template <>
__device__ __forceinline__ unsigned long long to_bits<int64_t>(int64_t v) { return (unsigned long long)v; }
template <>
__device__ __forceinline__ unsigned long long to_bits<double>(double v) {
  return (unsigned long long)__double_as_longlong(v);
}
template <typename T>
__device__ __forceinline__ T from_bits(unsigned long long b);
template <>
__device__ __forceinline__ int64_t from_bits<int64_t>(unsigned long long b) { return (int64_t)b; }
template <>
__device__ __forceinline__ double from_bits<double>(unsigned long long b) {
  return __longlong_as_double((long long)b);
}

template <typename T>
__device__ __forceinline__ void smem_add(T* p, T v);
template <>
__device__ __forceinline__ void smem_add<int64_t>(int64_t* p, int64_t v) {
  atomicAdd((unsigned long long*)p, (unsigned long long)v);
}
template <>
__device__ __forceinline__ void smem_add<double>(double* p, double v) {
  atomicAdd(p, v);
}

// Per-chunk window table of a task, in shared memory: for the chunk's f terms,
// the slice offset of F_i (32-bit), the first j of its window, the exclusive
// prefix of the window lengths (excl[ACC_THREADS] = total) and the coefficient.
struct ChunkTable {
  int32_t f32[ACC_THREADS];
  int32_t lo[ACC_THREADS];
  int32_t excl[ACC_THREADS + 1];
  int32_t warp_sum[ACC_THREADS / 32];
  unsigned long long coef[ACC_THREADS];
};

// Accumulate the pairs of one task into the shared slice acc[0, S).
// The task's f terms are taken ACC_THREADS at a time.  Each thread finds the
// exact j-window of one f term in the sorted g codes; a block-wide prefix sum
// flattens the windows into one range of pair indices, which is cut into
// equal contiguous shares, one per warp, so that every warp reaches the
// task's barrier with the same amount of work done.  A warp walks its share
// 32 pairs at a time: consecutive lanes take consecutive g terms, and the
// slice offset a = (F_i - B) + G_j lies in [0, S) by construction (32-bit
// arithmetic is exact there; a guard keeps it in bounds regardless).
template <typename T, bool C32>
__device__ __forceinline__ T mul(T a, T b) {
  if constexpr (C32) return (T)((int64_t)(int32_t)a * (int64_t)(int32_t)b);
  else return a * b;
}

template <typename T, bool C32>
__device__ __forceinline__ void dense_task_body(const Prod& P, const DenseTask& tk, T* acc,
                                                ChunkTable& ct) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = ACC_THREADS / 32;
  constexpr unsigned FULL = 0xffffffffu;
  const int64_t S = P.S;
  const int64_t B = tk.block * S;
  // pairs land in [B, B + lim): the block, clipped to the code range
  const int64_t lim = min(S, P.krange - B);
  const int64_t* __restrict__ F = P.f.code;
  const int64_t* __restrict__ G = P.g.code;
  const int32_t* __restrict__ G32 = P.g.code32;
  const T* __restrict__ CF = (const T*)P.f.coef;
  const T* __restrict__ CG = (const T*)P.g.coef;
  const int64_t ng = P.g.n;
  for (int64_t ib = tk.i0; ib < tk.i1; ib += ACC_THREADS) {
    const int64_t i = ib + threadIdx.x;
    int32_t cnt = 0;
    if (i < tk.i1) {
      const int64_t fi = F[i] - B;
      const int64_t l = g_lower_bound(G, ng, P.gidx, P.gidx_n, P.gshift, -fi);
      const int64_t h = g_lower_bound(G, ng, P.gidx, P.gidx_n, P.gshift, lim - fi);
      ct.f32[threadIdx.x] = (int32_t)fi;
      ct.lo[threadIdx.x] = (int32_t)l;
      cnt = (int32_t)(h - l);
      ct.coef[threadIdx.x] = to_bits<T>(CF[i]);
    } else {
      ct.f32[threadIdx.x] = 0;
      ct.lo[threadIdx.x] = 0;
      ct.coef[threadIdx.x] = 0ull;
    }
    // block-wide exclusive scan of the window lengths
    int32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ct.warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int32_t w = lane < NW ? ct.warp_sum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(FULL, w, o);
        if (lane >= o) w += y;
      }
      if (lane < NW) ct.warp_sum[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const int32_t wbase = warp > 0 ? ct.warp_sum[warp - 1] : 0;
    ct.excl[threadIdx.x] = wbase + x - cnt;
    if (threadIdx.x == ACC_THREADS - 1) ct.excl[ACC_THREADS] = wbase + x;
    __syncthreads();
    const int32_t total = ct.excl[ACC_THREADS];
    // this warp's share [pb, pe) of the flattened pairs
    const int32_t pb = (int32_t)(((int64_t)total * warp) / NW);
    const int32_t pe = (int32_t)(((int64_t)total * (warp + 1)) / NW);
    if (pb < pe) {
      // k = last f term whose window starts at or before pb
      int lo_k = 0, hi_k = ACC_THREADS;
      while (hi_k - lo_k > 1) {
        const int mid = (lo_k + hi_k) >> 1;
        if (ct.excl[mid] <= pb) lo_k = mid; else hi_k = mid;
      }
      // walk this warp's windows one by one; the lanes stride the j-range
      for (int k = lo_k; k < ACC_THREADS; ++k) {
        const int32_t e0 = ct.excl[k];
        if (e0 >= pe) break;
        const int32_t e1 = ct.excl[k + 1];
        const int32_t s0 = max(pb, e0), s1 = min(pe, e1);
        if (s0 >= s1) continue;
        const int64_t jb = (int64_t)ct.lo[k] + (s0 - e0);
        const int64_t je = (int64_t)ct.lo[k] + (s1 - e0);
        const int32_t fk = ct.f32[k];
        const T ck = from_bits<T>(ct.coef[k]);
        int64_t j = jb + lane;
        for (; j + 32 < je; j += 64) {
          const int32_t a0 = fk + (G32 ? G32[j] : (int32_t)G[j]);
          const int32_t a1 = fk + (G32 ? G32[j + 32] : (int32_t)G[j + 32]);
          const T v0 = mul<T, C32>(ck, CG[j]);
          const T v1 = mul<T, C32>(ck, CG[j + 32]);
          if ((uint32_t)a0 < (uint32_t)S) smem_add<T>(&acc[a0], v0);
          if ((uint32_t)a1 < (uint32_t)S) smem_add<T>(&acc[a1], v1);
        }
        if (j < je) {
          const int32_t a0 = fk + (G32 ? G32[j] : (int32_t)G[j]);
          if ((uint32_t)a0 < (uint32_t)S) smem_add<T>(&acc[a0], mul<T, C32>(ck, CG[j]));
        }
      }
    }
    __syncthreads();   // the table is rewritten by the next chunk
  }
}

template <typename T>
__device__ __forceinline__ void dense_flush(const Prod& P, const DenseTask& tk, T* acc) {
  const int64_t S = P.S;
  const int64_t B = tk.block * S;
  const int64_t lim = min(S, P.krange - B);
  T* out = (T*)P.dense + B;
  for (int64_t s = threadIdx.x; s < lim; s += blockDim.x) {
    const T v = acc[s];
    if (v != (T)0) {
      if (tk.single) out[s] = v;
      else smem_add<T>(&out[s], v);   // generic atomicAdd works on global memory too
    }
  }
}

__global__ void __launch_bounds__(ACC_THREADS, 3) k_dense_accum(const Prod* __restrict__ prods,
                                                             const DenseTask* __restrict__ tasks,
                                                             const int64_t* __restrict__ task_count,
                                                             int64_t task_cap,
                                                             unsigned long long* __restrict__ task_next) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t s_task;
  __shared__ ChunkTable ct;
  const int64_t ntasks = min(*task_count, task_cap);
  for (;;) {
    if (threadIdx.x == 0) s_task = (int64_t)atomicAdd(task_next, 1ull);
    __syncthreads();
    const int64_t t = s_task;
    __syncthreads();
    if (t >= ntasks) break;
    const DenseTask tk = tasks[t];
    const Prod& P = prods[tk.prod];
    if (P.status) continue;
    const int64_t S = P.S;
    // zero the slice (both types are 8 bytes wide)
    int64_t* z = (int64_t*)smem_raw;
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) z[s] = 0;
    __syncthreads();
    if (P.f64) dense_task_body<double, false>(P, tk, (double*)smem_raw, ct);
    else if (P.coef32) dense_task_body<int64_t, true>(P, tk, (int64_t*)smem_raw, ct);
    else dense_task_body<int64_t, false>(P, tk, (int64_t*)smem_raw, ct);
    __syncthreads();
    if (P.f64) dense_flush<double>(P, tk, (double*)smem_raw);
    else dense_flush<int64_t>(P, tk, (int64_t*)smem_raw);
    __syncthreads();
  }
}

cudaError_t launch_dense_accum(const Prod* dprods, const DenseTask* dtasks,
                               const int64_t* dtask_count, int64_t task_cap, int64_t* dtask_next,
                               int grid, int64_t max_S, cudaStream_t s) {
  const size_t smem = (size_t)max_S * 8;
  cudaError_t e = cudaFuncSetAttribute(k_dense_accum, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  // persistent grid: every CTA that fits on the GPU at once (grid = SMs on entry)
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_accum, ACC_THREADS, smem) ==
          cudaSuccess && per_sm > 0)
    grid *= per_sm;
  else
    cudaGetLastError();
  k_dense_accum<<<grid, ACC_THREADS, smem, s>>>(dprods, dtasks, dtask_count, task_cap,
                                               (unsigned long long*)dtask_next);
  return cudaGetLastError();
}

int dense_accum_threads() { return ACC_THREADS; }
int dense_max_split() { return MAX_SPLIT; }

}  // namespace kr
