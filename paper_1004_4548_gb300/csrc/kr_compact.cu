// Compaction: the accumulators (dense array or hash table) -> a sparse list of
// (code, coefficient) terms with the zero coefficients dropped (the output is
// again a sparse distributed vector, Sec. 3.1), over fixed chunks of every
// product's accumulator, each chunk's terms written in slot order at its
// offset: in one pass (chunk-level scan with look-back) up to
// COMPACT_ONE_PASS_MAX chunks, else in two passes (count, scan, write).  The dense array's slot order is code order, so the dense output
// comes out sorted.
#include <algorithm>

#include "kr_internal.cuh"

namespace kr {

constexpr int CP_THREADS = 256;
constexpr int CP_WARPS = CP_THREADS / 32;
constexpr unsigned CP_FULL = 0xffffffffu;

// A coefficient word is live unless it is int64 zero or float64 +-0.0.
__device__ __forceinline__ int live_word(uint64_t v, bool f64) {
  return (f64 ? (v << 1) != 0 : v != 0) ? 1 : 0;
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
  return P.path == PATH_DENSE ? P.kspan : P.slots;
}

// The chunk [s0, s1) of a product's accumulator (8192 dense slots of 8 bytes
// or 4096 hash slots of 16 bytes) is split into CP_WARPS contiguous parts, one
// per warp.  A warp holds its part in registers as CP_ROWS rows of 512 bytes,
// one 16-byte load per lane and row (a dense row: 64 slots, two per lane; a
// hash row: 32 (key + 1, value) slots, one per lane), so the accumulator is
// read from memory once per pass and every load is coalesced.
constexpr int CP_ROWS = 16;

struct Part {
  int64_t a, b;   // slots [a, b)
  ulonglong2 v[CP_ROWS];
};

template <bool STREAM>
__device__ __forceinline__ ulonglong2 ld_pair(const uint64_t* p) {
  if constexpr (STREAM) return __ldcs((const ulonglong2*)p); else return *(const ulonglong2*)p;
}

// Loads the warp's part and returns its number of live slots (in every lane).
template <bool STREAM>
__device__ __forceinline__ int load_part(const Prod& P, int64_t s0, int64_t s1, int warp, Part& pt) {
  const int lane = threadIdx.x & 31;
  const bool dense = P.path == PATH_DENSE;
  const int64_t per = P.chunk / CP_WARPS;   // CP_ROWS rows of 64 (dense) or 32 (hash) slots
  pt.a = min(s1, s0 + per * warp);
  pt.b = min(s1, pt.a + per);
  const bool f64 = P.f64;
  int n = 0;
  if (dense) {
    const uint64_t* a = (const uint64_t*)P.dense;
#pragma unroll
    for (int t = 0; t < CP_ROWS; ++t) {
      const int64_t s = pt.a + 64 * t + 2 * lane;
      ulonglong2 v = make_ulonglong2(0, 0);
      if (s + 1 < pt.b) v = ld_pair<STREAM>(a + s);
      else if (s < pt.b) v.x = a[s];
      pt.v[t] = v;
    }
#pragma unroll
    for (int t = 0; t < CP_ROWS; ++t) n += live_word(pt.v[t].x, f64) + live_word(pt.v[t].y, f64);
  } else {
#pragma unroll
    for (int t = 0; t < CP_ROWS; ++t) {
      const int64_t s = pt.a + 32 * t + lane;
      pt.v[t] = s < pt.b ? ld_pair<STREAM>(P.table + 2 * s) : make_ulonglong2(0, 0);
    }
#pragma unroll
    for (int t = 0; t < CP_ROWS; ++t) n += (pt.v[t].x != 0) & live_word(pt.v[t].y, f64);
  }
  return __reduce_add_sync(CP_FULL, (unsigned)n);
}

// Output terms [a, b) of a dense product (just written to okey / oval by
// this CTA) decoded into the caller's arrays, one term per thread.  A pass
// of its own after the chunk's writes, so that the chunk's registers are free.
__device__ __noinline__ void write_direct(const Prod& P, const DirectOut& D, int64_t a, int64_t b,
                                          const uint64_t* __restrict__ okey,
                                          const uint64_t* __restrict__ oval) {
  for (int64_t q = a + threadIdx.x; q < b; q += blockDim.x) {
    const int64_t code = (int64_t)okey[q] + P.klo;
    if (D.codes) D.codes[q] = code;
    if (D.exps) decode_poly_part(P, code, D.exps, D.ld, q);
    D.coef[q] = oval[q];
  }
}

// Writes the live slots of the warp's part in slot order from output position
// `run` (slots outside the part were loaded as zeros, which are not live).
// Keys are written relative to the product's key window (dense: the slot).
__device__ __forceinline__ void write_part(const Prod& P, const Part& pt, int64_t run, int64_t cap,
                                           uint64_t* __restrict__ okey, uint64_t* __restrict__ oval) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const bool f64 = P.f64;
  if (P.path == PATH_DENSE) {
#pragma unroll
    for (int t = 0; t < CP_ROWS; ++t) {
      const int64_t s = pt.a + 64 * t + 2 * lane;
      const int f0 = live_word(pt.v[t].x, f64), f1 = live_word(pt.v[t].y, f64);
      const unsigned b0 = __ballot_sync(CP_FULL, f0), b1 = __ballot_sync(CP_FULL, f1);
      const int64_t pos = run + __popc(b0 & lt) + __popc(b1 & lt);
      if (f0 && pos < cap) { okey[pos] = (uint64_t)s; oval[pos] = pt.v[t].x; }
      if (f1 && pos + f0 < cap) { okey[pos + f0] = (uint64_t)(s + 1); oval[pos + f0] = pt.v[t].y; }
      run += __popc(b0) + __popc(b1);
    }
  } else {
#pragma unroll
    for (int t = 0; t < CP_ROWS; ++t) {
      const int f = (pt.v[t].x != 0) & live_word(pt.v[t].y, f64);
      const unsigned b = __ballot_sync(CP_FULL, f);
      const int64_t pos = run + __popc(b & lt);
      if (f && pos < cap) { okey[pos] = pt.v[t].x - 1 - (uint64_t)P.klo; oval[pos] = pt.v[t].y; }
      run += __popc(b);
    }
  }
}

// Live slots of the warp's part, streamed (for the counting pass: a few
// registers, many warps in flight, each row read once and evicted first).
__device__ __forceinline__ int count_part(const Prod& P, int64_t s0, int64_t s1, int warp) {
  const int lane = threadIdx.x & 31;
  const int64_t per = P.chunk / CP_WARPS;
  const int64_t a0 = min(s1, s0 + per * warp), b0 = min(s1, a0 + per);
  const bool f64 = P.f64;
  int n = 0;
  if (P.path == PATH_DENSE) {
    const uint64_t* a = (const uint64_t*)P.dense;
#pragma unroll 4
    for (int64_t s = a0 + 2 * lane; s < b0; s += 64) {
      if (s + 1 < b0) {
        const ulonglong2 v = ld_pair<true>(a + s);
        n += live_word(v.x, f64) + live_word(v.y, f64);
      } else {
        n += live_word(__ldcs(a + s), f64);
      }
    }
  } else {
#pragma unroll 4
    for (int64_t s = a0 + lane; s < b0; s += 32) {
      const ulonglong2 kv = ld_pair<true>(P.table + 2 * s);
      n += (kv.x != 0) & live_word(kv.y, f64);
    }
  }
  return __reduce_add_sync(CP_FULL, (unsigned)n);
}

// Two-pass compaction, for accumulators of many chunks (several GB): a
// counting pass that streams the accumulator with many warps in flight, an
// exclusive scan of the counts, and a writing pass.
__global__ void __launch_bounds__(CP_THREADS) k_compact_count(const Prod* __restrict__ prods, int nprod,
                                                              const int64_t* __restrict__ chunk_begin,
                                                              int64_t* __restrict__ counts) {
  const int64_t nchunks = chunk_begin[nprod];
  __shared__ int red[CP_WARPS];
  const int warp = threadIdx.x >> 5;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int p = find_prod_of_chunk(chunk_begin, nprod, c);
    const Prod& P = prods[p];
    int n = 0;
    if (P.status == 0) {   // uniform across the CTA
      const int64_t s0 = (c - chunk_begin[p]) * P.chunk;
      const int64_t s1 = min(accum_slots(P), s0 + P.chunk);
      n = count_part(P, s0, s1, warp);
    }
    if ((threadIdx.x & 31) == 0) red[warp] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < CP_WARPS; ++w) t += red[w];
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
                                                                uint64_t* __restrict__ oval,
                                                                const DirectOut D) {
  const int64_t nchunks = chunk_begin[nprod];
  __shared__ int wsum[CP_WARPS];
  const int warp = threadIdx.x >> 5;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int p = find_prod_of_chunk(chunk_begin, nprod, c);
    const Prod& P = prods[p];
    if (P.status != 0) continue;   // uniform across the CTA
    const int64_t s0 = (c - chunk_begin[p]) * P.chunk;
    const int64_t s1 = min(accum_slots(P), s0 + P.chunk);
    Part pt;
    const int n = load_part<true>(P, s0, s1, warp, pt);
    if ((threadIdx.x & 31) == 0) wsum[warp] = n;
    __syncthreads();
    int64_t run = offs[c];
    for (int w = 0; w < warp; ++w) run += wsum[w];
    write_part(P, pt, run, cap, okey, oval);
    if (D.coef && P.path == PATH_DENSE) {   // uniform across the CTA
      int64_t cnt = 0;
      for (int w = 0; w < CP_WARPS; ++w) cnt += wsum[w];
      __syncthreads();   // the chunk's terms are in okey / oval
      write_direct(P, D, offs[c], min(offs[c] + cnt, min(cap, D.cap)), okey, oval);
    }
    __syncthreads();   // wsum is rewritten for the next chunk
  }
}

// Single-pass compaction (a chunk-level scan with decoupled look-back, after
// Merrill and Garland, "Single-pass parallel prefix scan with decoupled
// look-back", 2016).  CTAs take chunks in increasing order from a ticket
// counter, so every chunk before the one a CTA holds is already held by a
// running CTA.  A CTA loads its chunk into registers, counts its live slots,
// publishes the count (AGG), adds up its predecessors' published values going
// backwards until one carries an inclusive prefix (PRE), publishes its own
// inclusive prefix and writes its terms from its exclusive prefix on.  Each
// accumulator slot is read from memory once.  The wait on a predecessor is
// bounded; a CTA that gives up sets *err (the host fails the call with
// KR_ERR_TIMEOUT) and carries on without touching memory outside the output
// capacity.
constexpr uint64_t CS_AGG = 1ull << 62;
constexpr uint64_t CS_PRE = 2ull << 62;
constexpr uint64_t CS_VAL = (1ull << 62) - 1;
constexpr int CS_SPIN_LIMIT = 1 << 22;

__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Publishes chunk c's count and returns its exclusive prefix.  Called by all
// 32 lanes of one warp: the lanes read 32 predecessors at once, the nearest
// one with an inclusive prefix ends the walk, and the values up to it are
// summed; a window with an unpublished chunk before that point is read again.
__device__ __forceinline__ int64_t lookback(uint64_t* cstat, int64_t c, int64_t cnt, int64_t* err) {
  const int lane = threadIdx.x & 31;
  int64_t excl = 0;
  if (c > 0) {
    if (lane == 0) st_release(&cstat[c], CS_AGG | (uint64_t)cnt);
    int64_t q = c - 1;   // nearest predecessor of the window
    int spins = 0;
    for (;;) {
      const int64_t idx = q - lane;
      const uint64_t v = idx >= 0 ? ld_acquire(&cstat[idx]) : CS_PRE;   // before chunk 0: prefix 0
      const unsigned pre = __ballot_sync(0xffffffffu, (v & ~CS_VAL) == CS_PRE);
      const unsigned none = __ballot_sync(0xffffffffu, (v & ~CS_VAL) == 0);
      const unsigned upto = pre ? (pre & (0u - pre)) * 2u - 1u : 0xffffffffu;   // lanes up to the first prefix
      if (none & upto) {
        if (++spins > CS_SPIN_LIMIT) {
          if (lane == 0) atomicExch((unsigned long long*)err, 1ull);
          break;
        }
        __nanosleep(32);
        continue;
      }
      int64_t mine = ((1u << lane) & upto) ? (int64_t)(v & CS_VAL) : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
      excl += mine;
      if (pre) break;
      q -= 32;
    }
    excl = __shfl_sync(0xffffffffu, excl, 0);
  }
  if (lane == 0) st_release(&cstat[c], CS_PRE | (uint64_t)(excl + cnt));
  return excl;
}

// Self-test of the bounded wait: chunks 1..3 of a chain whose chunk 0 never
// publishes; chunk 1's wait must give up and set *err.
__global__ void k_lookback_selftest(uint64_t* cstat, int64_t* err, int64_t* out) {
  if (threadIdx.x >= 32) return;
  for (int64_t c = 1; c < 4; ++c) {
    const int64_t e = lookback(cstat, c, 1, err);
    if (threadIdx.x == 0) out[c] = e;
  }
}

__global__ void __launch_bounds__(CP_THREADS) k_compact(Prod* __restrict__ prods, int nprod,
                                                        const int64_t* __restrict__ chunk_begin,
                                                        uint64_t* __restrict__ cstat,
                                                        int64_t* __restrict__ offs,
                                                        unsigned long long* __restrict__ ticket,
                                                        int64_t* __restrict__ err, int64_t cap,
                                                        uint64_t* __restrict__ okey,
                                                        uint64_t* __restrict__ oval,
                                                        const DirectOut D) {
  const int64_t nchunks = chunk_begin[nprod];
  __shared__ int wsum[CP_WARPS];
  __shared__ int64_t s_c, s_excl;
  const int warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_c = (int64_t)atomicAdd(ticket, 1ull);
    __syncthreads();
    const int64_t c = s_c;
    if (c >= nchunks) break;
    const int p = find_prod_of_chunk(chunk_begin, nprod, c);
    const Prod& P = prods[p];
    const bool live = P.status == 0;   // uniform across the CTA
    const int64_t s0 = (c - chunk_begin[p]) * P.chunk;
    const int64_t s1 = min(accum_slots(P), s0 + P.chunk);
    Part pt;
    const int n = live ? load_part<true>(P, s0, s1, warp, pt) : 0;
    if ((threadIdx.x & 31) == 0) wsum[warp] = n;
    __syncthreads();
    if (warp == 0) {
      int64_t cnt = 0;
      for (int w = 0; w < CP_WARPS; ++w) cnt += wsum[w];
      const int64_t excl = lookback(cstat, c, cnt, err);
      if (threadIdx.x == 0) {
        offs[c] = excl;
        if (c == nchunks - 1) {
          offs[nchunks] = excl + cnt;
          if (nprod == 1) {   // the product's count and status (as k_finish_counts)
            Prod& Q = prods[0];
            Q.out_start = 0;
            Q.nout = Q.status ? 0 : excl + cnt;
            if (excl + cnt > cap) Q.status |= ST_OUTCAP;
          }
        }
        s_excl = excl;
      }
    }
    __syncthreads();
    if (live) {
      int64_t run = s_excl;
      for (int w = 0; w < warp; ++w) run += wsum[w];
      write_part(P, pt, run, cap, okey, oval);
    }
    if (live && D.coef && P.path == PATH_DENSE) {   // uniform across the CTA
      int64_t cnt = 0;
      for (int w = 0; w < CP_WARPS; ++w) cnt += wsum[w];
      __syncthreads();   // the chunk's terms are in okey / oval
      write_direct(P, D, s_excl, min(s_excl + cnt, min(cap, D.cap)), okey, oval);
    }
    __syncthreads();   // wsum, s_c and s_excl are rewritten for the next chunk
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
                           int64_t* dcounts, uint64_t* dcstat, int64_t* dsync, int64_t* dscan,
                           uint64_t* okey, uint64_t* oval, int64_t cap, cudaStream_t s,
                           const DirectOut& direct, int* launches) {
  *launches = 0;
  if (nchunks > 0) {
    // persistent grid: every CTA that fits on the GPU at once
    int dev = 0, sms = 152, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_compact, CP_THREADS, 0) != cudaSuccess) {
      cudaGetLastError();
      per = 2;
    }
    if (nchunks <= COMPACT_ONE_PASS_MAX) {
      const int64_t grid = std::min<int64_t>(nchunks, (int64_t)sms * std::max(per, 1));
      k_compact<<<(unsigned)grid, CP_THREADS, 0, s>>>(dprods, nprod, dchunk_begin, dcstat, dcounts,
                                                     (unsigned long long*)dsync, dsync + 1, cap, okey, oval,
                                                     direct);
      *launches += 1;
      if (nprod == 1) return cudaGetLastError();   // counted by the last chunk's CTA
    } else {
      int pc = 0, ps = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pc, k_compact_count, CP_THREADS, 0) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_compact_scatter, CP_THREADS, 0) != cudaSuccess) {
        cudaGetLastError();
        pc = ps = 2;
      }
      const int64_t gc = std::min<int64_t>(nchunks, (int64_t)sms * std::max(pc, 1));
      const int64_t gs = std::min<int64_t>(nchunks, (int64_t)sms * std::max(ps, 1));
      k_compact_count<<<(unsigned)gc, CP_THREADS, 0, s>>>(dprods, nprod, dchunk_begin, dcounts);
      cudaError_t e = launch_scan_exclusive(dcounts, nchunks, dcounts + nchunks, dscan, s);
      if (e != cudaSuccess) return e;
      k_compact_scatter<<<(unsigned)gs, CP_THREADS, 0, s>>>(dprods, nprod, dchunk_begin, dcounts, cap, okey,
                                                           oval, direct);
      *launches += 3;
    }
  } else {
    cudaMemsetAsync(dcounts, 0, sizeof(int64_t), s);
  }
  k_finish_counts<<<(nprod + 127) / 128, 128, 0, s>>>(dprods, nprod, dchunk_begin, dcounts,
                                                      dcounts + nchunks, cap);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace kr

using namespace kr;

extern "C" kr_status kr_selftest_bounded_wait(int32_t device) {
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return KR_ERR_CUDA; }
  void* buf = nullptr;
  kr_status st = KR_ERR_CUDA;
  if (cudaMalloc(&buf, 16 * sizeof(int64_t)) == cudaSuccess) {
    uint64_t* cstat = (uint64_t*)buf;            // [0, 4): the chain
    int64_t* err = (int64_t*)buf + 4;
    int64_t* out = (int64_t*)buf + 8;
    int64_t herr = 0;
    if (cudaMemset(buf, 0, 16 * sizeof(int64_t)) == cudaSuccess) {
      k_lookback_selftest<<<1, 32>>>(cstat, err, out);
      if (cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
          cudaMemcpy(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost) == cudaSuccess)
        st = herr ? KR_ERR_TIMEOUT : KR_OK;
    }
    cudaFree(buf);
  }
  cudaGetLastError();
  cudaSetDevice(prev);
  return st;
}
