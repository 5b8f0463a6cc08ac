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
constexpr int GROUP_R = 4;         // f terms per warp step (register reuse of g loads)

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
  const int64_t B = b * P.S, E = B + P.S;
  const int64_t* F = P.f.code;
  const int64_t* G = P.g.code;
  const int64_t nf = P.f.n, ng = P.g.n;
  const int64_t i_lo = lower_bound_i64(F, nf, B - G[ng - 1]);
  const int64_t i_hi = lower_bound_i64(F, nf, E - G[0]);
  if (i_lo >= i_hi) return;
  const int64_t span = i_hi - i_lo;
  int64_t cnt = 0;
  const int ns = span < PLAN_SAMPLES ? (int)span : PLAN_SAMPLES;
  if (lane < ns) {
    const int64_t i = i_lo + (span * lane) / ns;
    cnt = lower_bound_i64(G, ng, E - F[i]) - lower_bound_i64(G, ng, B - F[i]);
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

// Accumulate the pairs of one task into the shared slice acc[0, S).
// Warps take groups of GROUP_R consecutive f terms; the lanes walk the union
// of their j-ranges, loading each g term once and testing each of the R
// output codes against the block.
template <typename T>
__device__ __forceinline__ void dense_task_body(const Prod& P, const DenseTask& tk, T* acc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = ACC_THREADS / 32;
  const int64_t S = P.S;
  const int64_t B = tk.block * S;
  const int64_t* __restrict__ F = P.f.code;
  const int64_t* __restrict__ G = P.g.code;
  const T* __restrict__ CF = (const T*)P.f.coef;
  const T* __restrict__ CG = (const T*)P.g.coef;
  const int64_t ng = P.g.n;
  const int64_t ngroups = (tk.i1 - tk.i0 + GROUP_R - 1) / GROUP_R;
  for (int64_t grp = warp; grp < ngroups; grp += NW) {
    const int64_t ia = tk.i0 + grp * GROUP_R;
    const int m = (int)min((int64_t)GROUP_R, tk.i1 - ia);
    int64_t fr[GROUP_R];
    T cr[GROUP_R];
#pragma unroll
    for (int r = 0; r < GROUP_R; ++r) {
      const int64_t i = ia + (r < m ? r : 0);
      fr[r] = F[i] - B;
      cr[r] = CF[i];
      if (r >= m) fr[r] = INT64_MIN / 4;   // never inside the block
    }
    const int64_t flast = F[ia + m - 1] - B;
    // union of the j-ranges: codes in [B, B + S) for the largest and smallest F
    const int64_t jlo = lower_bound_i64(G, ng, -flast);
    const int64_t jhi = lower_bound_i64(G, ng, S - fr[0]);
    for (int64_t j = jlo + lane; j < jhi; j += 32) {
      const int64_t gj = G[j];
      const T cg = CG[j];
#pragma unroll
      for (int r = 0; r < GROUP_R; ++r) {
        const int64_t a = fr[r] + gj;
        if ((uint64_t)a < (uint64_t)S) smem_add<T>(&acc[a], cr[r] * cg);
      }
    }
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

__global__ void __launch_bounds__(ACC_THREADS) k_dense_accum(const Prod* __restrict__ prods,
                                                             const DenseTask* __restrict__ tasks,
                                                             const int64_t* __restrict__ task_count,
                                                             int64_t task_cap,
                                                             unsigned long long* __restrict__ task_next) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t s_task;
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
    if (P.f64) dense_task_body<double>(P, tk, (double*)smem_raw);
    else dense_task_body<int64_t>(P, tk, (int64_t*)smem_raw);
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
  k_dense_accum<<<grid, ACC_THREADS, smem, s>>>(dprods, dtasks, dtask_count, task_cap,
                                               (unsigned long long*)dtask_next);
  return cudaGetLastError();
}

int dense_accum_threads() { return ACC_THREADS; }
int dense_max_split() { return MAX_SPLIT; }

}  // namespace kr
