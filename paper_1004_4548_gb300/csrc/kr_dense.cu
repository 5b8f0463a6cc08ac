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
// global atomic adds into the array, which the planning kernel has cleared
// for those blocks (a block with one task is written whole by its flush).
// Tasks are fetched dynamically by a persistent grid.
#include "kr_internal.cuh"

namespace kr {

constexpr int PLAN_SAMPLES = 32;   // sampled i per block for the work estimate
constexpr int MAX_SPLIT = 64;      // tasks per block at most
constexpr int ACC_THREADS = 512;

// One warp per (dense product, block): i-range by warp-wide search, sampled
// work estimate, then 1..MAX_SPLIT tasks over equal i-slices.  A block that
// gets one task is written whole by its flush; every other block (several
// tasks adding into it, or none) is zeroed here, so the accumulation array
// needs no separate clearing.
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
  const int64_t b = gw - block_begin[lo];
  // blocks tile the key window [klo, klo + kspan); its end may fall inside the last block
  const int64_t B = P.klo + b * P.S, E = min(B + P.S, P.klo + P.kspan);
  int64_t k = 0;
  const int64_t* F = P.f.code;
  const int64_t* G = P.g.code;
  const int64_t nf = P.f.nkeep, ng = P.g.nkeep;   // dropped terms sort last
  if (!P.status && nf > 0 && ng > 0) {
    int64_t i_lo, i_hi;
    warp_lower_bound2(F, nf, B - G[ng - 1], E - G[0], &i_lo, &i_hi);
    if (i_lo < i_hi) {
      const int32_t* gx = P.gidx;
      const int64_t gn = P.gidx_n;
      const int gsh = P.gshift;
      const int64_t span = i_hi - i_lo;
      int64_t cnt = 0;
      const int ns = span < PLAN_SAMPLES ? (int)span : PLAN_SAMPLES;
      if (lane < ns) {
        const int64_t i = i_lo + (span * lane) / ns;
        int64_t a, c;
        g_lower_bound2(G, ng, gx, gn, gsh, B - F[i], E - F[i], &a, &c);
        cnt = c - a;
      }
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      // a zero estimate does not prove an empty block (the samples may all miss),
      // so every block with a nonempty i-range gets at least one task
      const double est = (double)cnt * (double)span / (double)ns;
      k = (int64_t)(est / (double)P.work_target) + 1;
      if (k > MAX_SPLIT) k = MAX_SPLIT;
      if (k > span) k = span;
      int64_t base = 0;
      if (lane == 0) base = (int64_t)atomicAdd((unsigned long long*)task_count, (unsigned long long)k);
      base = __shfl_sync(0xffffffffu, base, 0);
      for (int64_t t = lane; t < k; t += 32) {
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
  }
  if (k != 1 && P.dense) {
    // 16-byte stores over the block's slots, with an 8-byte store for a slot
    // before the first 16-byte boundary and for an unpaired last slot
    uint64_t* out = (uint64_t*)P.dense + (B - P.klo);
    const int64_t len = E - B;
    const int64_t head = ((uintptr_t)out & 15) ? 1 : 0;
    if (head && lane == 0 && len > 0) out[0] = 0;
    for (int64_t s = head + 2 * lane; s + 1 < len; s += 64) *(uint4*)(out + s) = make_uint4(0, 0, 0, 0);
    if (len > head && ((len - head) & 1) && lane == 0) out[len - 1] = 0;
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
// last code get ng.  Both ends are clamped to [0, gidx_n], so codes outside
// [0, W) (a caller's broken precondition) never index outside the array.
__global__ void __launch_bounds__(256) k_build_gindex(const Prod* __restrict__ prods,
                                                     const int32_t* __restrict__ dense_prods) {
  const Prod& P = prods[dense_prods[blockIdx.y]];
  if (P.g.sort_method == SORT_CLUSTER) return;   // the cluster front end built it
  const int64_t* G = P.g.code;
  const int64_t ng = P.g.n;
  const int sh = P.gshift;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= ng;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blo = j == 0 ? 0 : max((G[j - 1] >> sh) + 1, (int64_t)0);
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

// The accumulator slice of a block in shared memory (8 bytes per code).
// int64 sums are held as two 32-bit words per slot (low words in [0, S), high
// words in [S, 2S)): a 64-bit add is a 32-bit add of the low word, whose
// returned old value gives the carry, plus a 32-bit add of high word and carry
// when that is nonzero.  The sums stay exact modulo 2^64 whatever the order of
// the adds, since each carry is seen by exactly the add that makes it.
// Shared-memory 32-bit atomics run several times faster than 64-bit ones on
// this GPU (measured chip-wide, conflict-free: 8.8 T vs 1.6 T adds/s).
// float64 sums use 64-bit atomic adds.
template <typename T>
struct Slice;

template <>
struct Slice<int64_t> {
  uint32_t* lo;
  uint32_t* hi;
  uint32_t lo_sh;    // shared-memory address of the low words
  uint32_t hi_dist;  // bytes from a low word to its high word (4 S)
  __device__ __forceinline__ Slice(void* base, int64_t S)
      : lo((uint32_t*)base), hi((uint32_t*)base + S), lo_sh((uint32_t)__cvta_generic_to_shared(base)),
        hi_dist((uint32_t)(4 * S)) {}
  __device__ __forceinline__ void add(int32_t off, int64_t v) const {
    smem_acc_split64(lo_sh + (uint32_t)off * 4u, hi_dist, (uint64_t)v);
  }
  __device__ __forceinline__ int64_t get(int64_t s) const {
    return (int64_t)(((uint64_t)hi[s] << 32) | (uint64_t)lo[s]);
  }
  // Adds the product of one chunk-table entry (slice offset x, int32
  // coefficient y, read from shared address ent) and a g term (code offset
  // gc, int32 coefficient cg) at offset x + gc, known to lie in the slice: the
  // load, the product and the add as one sequence with no range test and no
  // branch (the high-word reduction is guarded by a predicate).
  __device__ __forceinline__ void add_entry(uint32_t ent, int32_t gc, int32_t cg) const {
    asm volatile(
        "{\n\t.reg .pred q;\n\t.reg .b32 x, y, a, o, t, h, l, u;\n\t.reg .s64 v;\n\t"
        "ld.shared.v2.b32 {x, y}, [%0];\n\t"
        "add.s32 x, x, %1;\n\t"
        "mad.lo.u32 a, x, 4, %3;\n\t"
        "mul.wide.s32 v, y, %2;\n\t"
        "mov.b64 {l, u}, v;\n\t"
        "atom.shared.add.u32 o, [a], l;\n\t"
        "add.cc.u32 t, o, l;\n\t"
        "addc.u32 h, u, 0;\n\t"
        "setp.ne.u32 q, h, 0;\n\t"
        "add.u32 a, a, %4;\n\t"
        "@q red.shared.add.u32 [a], h;\n\t}"
        ::"r"(ent), "r"(gc), "r"(cg), "r"(lo_sh), "r"(hi_dist) : "memory");
  }
};

template <>
struct Slice<double> {
  double* a;
  __device__ __forceinline__ Slice(void* base, int64_t) : a((double*)base) {}
  __device__ __forceinline__ void add(int32_t off, double v) const { atomicAdd(&a[off], v); }
  __device__ __forceinline__ double get(int64_t s) const { return a[s]; }
};

// Per-chunk window table of a task, in shared memory: for the chunk's f terms,
// the slice offset of F_i (32-bit), the first j of its window, the exclusive
// prefix of the window lengths (excl[ACC_THREADS] = total) and the coefficient.
struct ChunkTable {
  int2 fc[ACC_THREADS];               // (F_i - B, coefficient as int32 when it fits) of every f term
  int32_t lo[ACC_THREADS];            // first j of the tile's window (tile owners)
  int16_t run[ACC_THREADS];           // tile length (0: not a tile owner)
  int32_t excl[ACC_THREADS + 1];
  int32_t warp_sum[ACC_THREADS / 32];
};

// f terms are taken in tiles of up to TILE_R consecutive terms whose codes
// share one aligned window of S / 8 codes; a lane multiplies one g term by
// every term of a tile, so the window search, the g loads and the walk
// bookkeeping are paid once per TILE_R term-products.  The tile's g-window is
// the union of its terms' windows, at most S / 8 codes wider than one.
#ifndef KR_FULL_TILE_FAST
#define KR_FULL_TILE_FAST 1
#endif
#ifndef KR_ACC_MIN_BLOCKS
#define KR_ACC_MIN_BLOCKS 3
#endif
#ifndef KR_TILE_R
#define KR_TILE_R 8
#endif
constexpr int TILE_R = KR_TILE_R;
static_assert(TILE_R >= 1 && (TILE_R & (TILE_R - 1)) == 0 && 32 % TILE_R == 0,
              "tiles end at warp boundaries");
#ifndef KR_DENSE_Q
#define KR_DENSE_Q 2
#endif
constexpr int DENSE_Q = KR_DENSE_Q;   // f terms examined per thread and table fill

// Accumulate the pairs of one task into the shared slice acc[0, S).
//
// The task's f terms are examined DENSE_Q * ACC_THREADS at a time; those whose
// g window in the block may hold a term (by the g bucket index) are packed
// into tables of ACC_THREADS entries.  The thread of the first entry of a
// tile (see TILE_R) finds the tile's exact g-window: the g terms
// whose product with some term of the tile can land in the block.  A
// block-wide prefix sum flattens the windows into one range of (tile, g term)
// slots, cut into equal contiguous shares, one per warp, so that every warp
// reaches the chunk's barrier with about the same work done.  A warp walks its
// share 32 consecutive slots at a time, one per lane; each lane follows the
// window its slot falls in, loads one g term and adds its products with the
// tile's f terms to the slice with shared-memory atomics (consecutive lanes of
// a window hold consecutive g terms, so one atomic instruction touches nearby
// words).  A step in which every lane holds a g term that pairs in range with
// all TILE_R terms of a full tile (most steps of a dense product) adds without
// range tests.  The slice offset a = (F_i - B) + G_j lies in [0, S) for the pairs
// this block owns; others are skipped (32-bit arithmetic is exact there, since
// the dense path keeps codes below 2^31).
template <typename T, bool C32>
__device__ __forceinline__ T mul(T a, T b) {
  if constexpr (C32) return (T)((int64_t)(int32_t)a * (int64_t)(int32_t)b);
  else return a * b;
}

template <typename T, bool C32>
__device__ __forceinline__ void dense_task_body(const Prod& P, const DenseTask& tk, const Slice<T>& acc,
                                                ChunkTable& ct) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = ACC_THREADS / 32;
  constexpr unsigned FULL = 0xffffffffu;
  const int64_t S = P.S;
  const int64_t B = P.klo + tk.block * S;
  // pairs land in [B, B + lim): the block, clipped to the key window
  const int64_t lim = min(S, P.klo + P.kspan - B);
  const int sh = 28 - __clz((int)S);   // tiles stay within aligned windows of about S / 8 codes
  const int64_t* __restrict__ F = P.f.code;
  const int64_t* __restrict__ G = P.g.code;
  const int32_t* __restrict__ G32 = P.g.code32;
  const T* __restrict__ CF = (const T*)P.f.coef;
  const T* __restrict__ CG = (const T*)P.g.coef;
  const int64_t ng = P.g.n;
  const int32_t* __restrict__ GX = P.gidx;
  const int64_t gn = P.gidx_n;
  const int gsh = P.gshift;
  // block-wide exclusive scan of one value per thread (ct.warp_sum as scratch)
  auto block_scan = [&](int32_t v, int32_t& total) -> int32_t {
    int32_t x = v;
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
    const int32_t base = warp > 0 ? ct.warp_sum[warp - 1] : 0;
    total = ct.warp_sum[NW - 1];
    __syncthreads();   // the scratch is reused by the next scan
    return base + x - v;
  };
  // The task's f terms are examined DENSE_Q * ACC_THREADS at a time: an f term
  // whose g window in the block is empty (its bucket range holds no g code)
  // takes no table entry, and the kept ones are packed into tables of
  // ACC_THREADS entries (one or more rounds).
  for (int64_t sb = tk.i0; sb < tk.i1; sb += (int64_t)ACC_THREADS * DENSE_Q) {
    int64_t fv[DENSE_Q];
    int32_t cv[DENSE_Q];
    bool keep[DENSE_Q];
    int32_t nk = 0;
#pragma unroll
    for (int q = 0; q < DENSE_Q; ++q) {
      const int64_t i = sb + (int64_t)DENSE_Q * threadIdx.x + q;
      fv[q] = 0;
      cv[q] = 0;
      if (i < tk.i1) {
        fv[q] = F[i];
        // the table keeps the int32 coefficient, or else the term's index
        if constexpr (C32) cv[q] = (int32_t)(int64_t)CF[i];
        else cv[q] = (int32_t)(i - tk.i0);
      }
    }
#pragma unroll
    for (int q = 0; q < DENSE_Q; ++q) {
      const int64_t i = sb + (int64_t)DENSE_Q * threadIdx.x + q;
      keep[q] = false;
      if (i < tk.i1) {
        // the g codes in [x1, x2) pair with this term into the block; the
        // bucket index bounds how many lie in the buckets covering that range
        const int64_t x1 = B - fv[q], x2 = B + lim - fv[q];
        int64_t below = 0, upto = 0;
        if (x1 > 0) {
          const int64_t bk = x1 >> gsh;
          below = bk >= gn ? ng : GX[bk];
        }
        if (x2 > 0) {
          const int64_t bk = (x2 - 1) >> gsh;
          upto = bk >= gn ? ng : GX[bk + 1];
        }
        keep[q] = upto > below;
      }
      nk += keep[q] ? 1 : 0;
    }
    int32_t kept;
    const int32_t pos0 = block_scan(nk, kept);
    for (int32_t r0 = 0; r0 < kept; r0 += ACC_THREADS) {
      {
        int32_t p = pos0;
#pragma unroll
        for (int q = 0; q < DENSE_Q; ++q) {
          if (keep[q]) {
            if (p >= r0 && p < r0 + ACC_THREADS) ct.fc[p - r0] = make_int2((int32_t)(fv[q] - B), cv[q]);
            ++p;
          }
        }
      }
      __syncthreads();   // the round's entries are in the table
      const int nent = min(ACC_THREADS, kept - r0);
      const int ent = threadIdx.x;
      int32_t cnt = 0, l32 = 0, r = 0;
      const bool valid = ent < nent;
      const int32_t off = valid ? ct.fc[ent].x : 0;
      const int32_t wid = off >> sh;   // floor: tiles stay within aligned windows of 2^sh codes
      const bool owner = valid && (ent == 0 || wid != (ct.fc[ent - 1].x >> sh) || (ent & (TILE_R - 1)) == 0);
      // a tile runs to the next owner (every TILE_R-th entry is one, and
      // TILE_R divides 32, so a warp's last tile ends at the warp's end) or
      // to the table's end
      const unsigned om = __ballot_sync(FULL, owner);
      if (owner) {
        const unsigned above = lane == 31 ? 0u : (om >> (lane + 1));
        const int next = above ? lane + __ffs((int)above) : 32;
        r = min(32 * warp + next, nent) - ent;
        int64_t l, h;
        g_lower_bound2(G, ng, GX, gn, gsh, -(int64_t)ct.fc[ent + r - 1].x, lim - off, &l, &h);
        l32 = (int32_t)l;
        cnt = (int32_t)(h - l);
      }
      ct.lo[ent] = l32;
      ct.run[ent] = (int16_t)r;
      int32_t wtotal;
      ct.excl[ent] = block_scan(cnt, wtotal);
      if (ent == 0) ct.excl[ACC_THREADS] = wtotal;
      __syncthreads();
      const int32_t total = ct.excl[ACC_THREADS];
      // this warp's share [pb, pe) of the flattened slots
      const int32_t pb = (int32_t)(((int64_t)total * warp) / NW);
      const int32_t pe = (int32_t)(((int64_t)total * (warp + 1)) / NW);
      if (pb < pe) {
        // k = the window of this lane's first slot (the last k with
        // excl[k] <= p); p < excl[ACC_THREADS] keeps k + 1 <= ACC_THREADS below
        int32_t p = pb + lane;
        // the window of the warp's first slot: the last k with excl[k] <= pb,
        // by two ballots over the ascending excl (16 entries a lane, then 16
        // lanes over one lane's entries); each lane then advances to its own
        // slot's window in the walk below
        int k;
        {
          constexpr int STEP = ACC_THREADS / 32;
          const unsigned le = __ballot_sync(FULL, ct.excl[lane * STEP] <= pb);   // lane 0: excl[0] = 0
          const int base = (31 - __clz((int)le)) * STEP;
          const unsigned le2 = __ballot_sync(FULL, lane < STEP && ct.excl[base + (lane < STEP ? lane : 0)] <= pb);
          k = base + 31 - __clz((int)le2);
        }
        int32_t e0 = ct.excl[k], e1 = ct.excl[k + 1];
        const int32_t lim32 = (int32_t)lim;
        const uint32_t fc_sh = (uint32_t)__cvta_generic_to_shared(&ct.fc[0]);
        // the lanes step together (uniform trip count) so that they can vote
        for (int32_t base = pb; base < pe; base += 32, p += 32) {
          const bool act = p < pe;
          int32_t gc = 0;
          T cg = (T)0;
          int rk = 0;
          if (act) {
            while (p >= e1) {   // empty windows (non-owners) are skipped here too
              ++k;
              e0 = e1;
              e1 = ct.excl[k + 1];
            }
            const int64_t j = (int64_t)ct.lo[k] + (p - e0);
            gc = G32 ? G32[j] : (int32_t)G[j];
            cg = CG[j];
            rk = ct.run[k];
          }
          if constexpr (C32) {
            // core step: in every lane a full tile and a g term in range for
            // all of the tile's f terms (offsets x_0 + gc .. x_7 + gc inside
            // [0, lim), the x_a ascending): no range tests
            bool core = false;
            if (act && rk == TILE_R) {
              const int32_t o0 = ct.fc[k].x + gc;
              core = o0 >= 0 && o0 < lim32 - (ct.fc[k + TILE_R - 1].x - ct.fc[k].x);
            }
            if (__all_sync(FULL, core)) {
              const uint32_t ent = fc_sh + (uint32_t)k * 8u;
#pragma unroll
              for (int a = 0; a < TILE_R; ++a) acc.add_entry(ent + 8u * a, gc, (int32_t)cg);
              continue;
            }
          }
          if (!act) continue;
#if KR_FULL_TILE_FAST
          if (rk == TILE_R) {   // the common case: a full tile, the loop fully unrolled
#pragma unroll
            for (int a = 0; a < TILE_R; ++a) {
              const int2 e = ct.fc[k + a];
              const int32_t off = e.x + gc;
              if ((uint32_t)off < (uint32_t)S) {
                if constexpr (C32) acc.add(off, (T)((int64_t)e.y * (int64_t)(int32_t)cg));
                else acc.add(off, mul<T, C32>(CF[tk.i0 + e.y], cg));
              }
            }
            continue;
          }
#endif
#pragma unroll 4
          for (int a = 0; a < rk; ++a) {
            const int2 e = ct.fc[k + a];
            const int32_t off = e.x + gc;
            if ((uint32_t)off < (uint32_t)S) {
              if constexpr (C32) acc.add(off, (T)((int64_t)e.y * (int64_t)(int32_t)cg));
              else acc.add(off, mul<T, C32>(CF[tk.i0 + e.y], cg));
            }
          }
        }
      }
      __syncthreads();   // the table is rewritten by the next round
    }
  }
}

// int64 sums: four slots per thread and step, their low and high words read
// by two 16-byte shared loads (the slice's halves start 16-byte aligned, S
// being a multiple of 32); a single task's block is written with 16-byte
// stores where the array is 16-byte aligned.
__device__ __forceinline__ void dense_flush_i64(const Prod& P, const DenseTask& tk, const Slice<int64_t>& acc) {
  const int64_t S = P.S;
  const int64_t B = tk.block * S;   // relative to the window
  const int64_t lim = min(S, P.kspan - B);
  unsigned long long* out = (unsigned long long*)P.dense + B;
  const bool v16 = (((uintptr_t)out) & 15) == 0;
  for (int64_t s = 4 * (int64_t)threadIdx.x; s < lim; s += 4 * (int64_t)blockDim.x) {
    const uint4 lo = *reinterpret_cast<const uint4*>(acc.lo + s);
    const uint4 hi = *reinterpret_cast<const uint4*>(acc.hi + s);
    const unsigned long long v[4] = {((unsigned long long)hi.x << 32) | lo.x, ((unsigned long long)hi.y << 32) | lo.y,
                                     ((unsigned long long)hi.z << 32) | lo.z, ((unsigned long long)hi.w << 32) | lo.w};
    if (tk.single && v16 && s + 4 <= lim) {
      *reinterpret_cast<ulonglong2*>(out + s) = make_ulonglong2(v[0], v[1]);
      *reinterpret_cast<ulonglong2*>(out + s + 2) = make_ulonglong2(v[2], v[3]);
      continue;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (s + i < lim) {
        if (tk.single) out[s + i] = v[i];   // the block's only task: every slot, zeros included
        else if (v[i] != 0) atomicAdd(&out[s + i], v[i]);
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void dense_flush(const Prod& P, const DenseTask& tk, const Slice<T>& acc) {
  const int64_t S = P.S;
  const int64_t B = tk.block * S;   // relative to the window
  const int64_t lim = min(S, P.kspan - B);
  T* out = (T*)P.dense + B;
  for (int64_t s = threadIdx.x; s < lim; s += blockDim.x) {
    const T v = acc.get(s);
    if (tk.single) out[s] = v;   // the block's only task: every slot, zeros included
    else if (v != (T)0) smem_add<T>(&out[s], v);   // generic atomicAdd works on global memory too
  }
}

__global__ void __launch_bounds__(ACC_THREADS, KR_ACC_MIN_BLOCKS) k_dense_accum(const Prod* __restrict__ prods,
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
    // zero the slice (8 bytes per code for both types)
    uint4* z = (uint4*)smem_raw;   // S * 8 bytes, S a multiple of 32
    for (int64_t s = threadIdx.x; s < S / 2; s += blockDim.x) z[s] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    if (P.f64) {
      const Slice<double> sl(smem_raw, S);
      dense_task_body<double, false>(P, tk, sl, ct);
      __syncthreads();
      dense_flush<double>(P, tk, sl);
    } else {
      const Slice<int64_t> sl(smem_raw, S);
      if (P.coef32) dense_task_body<int64_t, true>(P, tk, sl, ct);
      else dense_task_body<int64_t, false>(P, tk, sl, ct);
      __syncthreads();
      dense_flush_i64(P, tk, sl);
    }
    __syncthreads();
  }
}

cudaError_t launch_dense_accum(const Prod* dprods, const DenseTask* dtasks,
                               const int64_t* dtask_count, int64_t task_cap, int64_t* dtask_next,
                               int grid, int64_t max_S, cudaStream_t s) {
  const size_t smem = (size_t)max_S * 8;
  cudaError_t e = raise_smem_limit((const void*)k_dense_accum, (size_t)smem);
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
