// Kronecker coding kernels: exponent range scan, encoding of the operands into
// sort keys, gathering of the sorted operands, and decoding of output codes.
//
// Coding (Sec. 2, Table 2 and the equations after it): for a box
// [e_min, e_max] with widths w_k = 1 + e_k,max - e_k,min the code of e is
// sum_k c_k (e_k - e_k,min), c_0 = 1, c_k = prod_{l<k} w_l.  Each operand of a
// product is coded with the product's widths and offset by its own minimum,
// so that code_f(a) + code_g(b) = code_h(a + b) (the additivity of Eq. 5).
// Trig multipliers use the balanced form sum_k c_k t_k over the symmetric box
// |t_k| <= R_k; sums and differences of such codes are the codes of the sums
// and differences of the vectors, and the sign of a code is the sign of the
// highest-index nonzero entry, which is what the canonical form looks at.
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

#include "kr_internal.cuh"

namespace kr {

// ---------------------------------------------------------------------------
// per-operand minima / maxima of the exponents, max |t| of the multipliers,
// whether every int64 coefficient fits in int32, and (truncated products) the
// degree range.  ranges layout per operand: [0, MAXV) min, [MAXV, 2 MAXV) max,
// [2 MAXV, 3 MAXV) max|t|, then the flags described with RANGE_STRIDE.
// One launch: `split` CTAs per operand each reduce a slice of the terms to a
// partial record; the last CTA of an operand to finish (a counter per operand,
// zero at launch) combines the partials.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_SPLIT_MAX = 256;
static_assert(RS_SPLIT_MAX <= RS_THREADS, "the combine takes one partial per thread");
constexpr int RS_CTA_BUDGET = 2048;   // CTAs of one launch, about 13 per SM

struct RangePart {
  int32_t lo[MAXV], hi[MAXV], tmax[MAXV];
  int32_t fits;
  int32_t pad;
  long long dlo, dhi;
};

int range_scan_splits(int nops, int64_t max_n) {
  int64_t k = (max_n + RS_THREADS - 1) / RS_THREADS;   // one term per thread
  const int64_t budget = std::max<int64_t>(1, RS_CTA_BUDGET / std::max(1, nops));
  k = std::min<int64_t>(k, std::min<int64_t>(budget, RS_SPLIT_MAX));
  return (int)(k < 1 ? 1 : k);
}

size_t range_scan_scratch_bytes(int nops, int64_t max_n) {
  return sizeof(RangePart) * (size_t)nops * (size_t)range_scan_splits(nops, max_n);
}

__global__ void __launch_bounds__(RS_THREADS) k_range_scan(const Prod* __restrict__ prods,
                                                           const OpRef* __restrict__ ops,
                                                           RangePart* __restrict__ parts,
                                                           unsigned int* __restrict__ done,
                                                           int32_t* __restrict__ ranges) {
  const OpRef r = ops[blockIdx.y];
  const Prod& P = prods[r.prod];
  const Operand& O = r.which ? P.g : P.f;
  const int64_t i0 = O.n * blockIdx.x / gridDim.x, i1 = O.n * (blockIdx.x + 1) / gridDim.x;
  __shared__ int32_t smin[MAXV][RS_THREADS / 32], smax[MAXV][RS_THREADS / 32];
  __shared__ int sfits[RS_THREADS / 32];
  __shared__ long long sdlo[RS_THREADS / 32], sdhi[RS_THREADS / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nvar = P.np + P.nt;
  int fits = P.f64 ? 0 : 1;
  // variables four at a time, every load of a group issued before any is used
  for (int k0 = 0; k0 < max(nvar, 1); k0 += 4) {   // once at least: the coefficient check
    int32_t lo[4], hi[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) { lo[j] = INT32_MAX; hi[j] = INT32_MIN; }
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      int32_t x[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = k0 + j;
        x[j] = 0;
        if (k < P.np) x[j] = O.e[(int64_t)k * O.n + i];
        else if (k < nvar) x[j] = O.t[(int64_t)(k - P.np) * O.n + i];
      }
      if (k0 == 0 && !P.f64) {
        const int64_t c = ((const int64_t*)O.c)[i];
        if (c < INT32_MIN || c > INT32_MAX) fits = 0;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int32_t v = x[j];
        if (k0 + j >= P.np) v = v < 0 ? -v : v;
        lo[j] = min(lo[j], v);
        hi[j] = max(hi[j], v);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int32_t a = __reduce_min_sync(0xffffffffu, lo[j]);
      const int32_t b = __reduce_max_sync(0xffffffffu, hi[j]);
      if (lane == 0 && k0 + j < nvar) { smin[k0 + j][warp] = a; smax[k0 + j][warp] = b; }
    }
  }
  fits = __all_sync(0xffffffffu, fits);
  long long dlo = LLONG_MAX, dhi = LLONG_MIN;
  if (P.gmask) {
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      long long d = 0;
      for (int k = 0; k < P.np; ++k)
        if ((P.gmask >> k) & 1u) d += O.e[(int64_t)k * O.n + i];
      dlo = min(dlo, d);
      dhi = max(dhi, d);
    }
    for (int o = 16; o > 0; o >>= 1) {
      dlo = min(dlo, __shfl_xor_sync(0xffffffffu, dlo, o));
      dhi = max(dhi, __shfl_xor_sync(0xffffffffu, dhi, o));
    }
  }
  if (lane == 0) { sfits[warp] = fits; sdlo[warp] = dlo; sdhi[warp] = dhi; }
  __syncthreads();
  RangePart* pp = parts + (int64_t)blockIdx.y * gridDim.x;
  RangePart& out = pp[blockIdx.x];
  if (threadIdx.x < nvar) {
    const int k = threadIdx.x;
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    for (int w = 0; w < RS_THREADS / 32; ++w) { lo = min(lo, smin[k][w]); hi = max(hi, smax[k][w]); }
    out.lo[k] = lo;
    out.hi[k] = hi;
  }
  if (threadIdx.x == 0) {
    int f = 1;
    long long a = LLONG_MAX, b = LLONG_MIN;
    for (int w = 0; w < RS_THREADS / 32; ++w) { f &= sfits[w]; a = min(a, sdlo[w]); b = max(b, sdhi[w]); }
    out.fits = f;
    out.dlo = a;
    out.dhi = b;
  }
  // the partial is published before the count; the CTA that counts last
  // sees every partial of its operand
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&done[blockIdx.y], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the combine: thread q loads partial q (all at once, one round of loads),
  // then warp reductions and one pass over the warps' results
  const int nsplit = gridDim.x;
  const int q = threadIdx.x;   // nsplit <= RS_SPLIT_MAX == RS_THREADS
  const bool has = q < nsplit;
  int32_t plo[MAXV], phi[MAXV];
#pragma unroll
  for (int k = 0; k < MAXV; ++k) {
    plo[k] = INT32_MAX;
    phi[k] = INT32_MIN;
    if (has && k < nvar) {
      plo[k] = __ldcg(&pp[q].lo[k]);
      phi[k] = __ldcg(&pp[q].hi[k]);
    }
  }
  int pf = has ? __ldcg(&pp[q].fits) : 1;
  long long pa = has ? __ldcg(&pp[q].dlo) : LLONG_MAX, pb = has ? __ldcg(&pp[q].dhi) : LLONG_MIN;
#pragma unroll
  for (int k = 0; k < MAXV; ++k) {
    if (k < nvar) {
      const int32_t a = __reduce_min_sync(0xffffffffu, plo[k]);
      const int32_t b = __reduce_max_sync(0xffffffffu, phi[k]);
      if (lane == 0) { smin[k][warp] = a; smax[k][warp] = b; }
    }
  }
  pf = __all_sync(0xffffffffu, pf);
  for (int o = 16; o > 0; o >>= 1) {
    pa = min(pa, __shfl_xor_sync(0xffffffffu, pa, o));
    pb = max(pb, __shfl_xor_sync(0xffffffffu, pb, o));
  }
  __syncthreads();   // every warp has read its own partial record above
  if (lane == 0) { sfits[warp] = pf; sdlo[warp] = pa; sdhi[warp] = pb; }
  __syncthreads();
  int32_t* res = ranges + (int64_t)blockIdx.y * RANGE_STRIDE;
  const int k = threadIdx.x;
  if (k < nvar) {
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    for (int w = 0; w < RS_THREADS / 32; ++w) { lo = min(lo, smin[k][w]); hi = max(hi, smax[k][w]); }
    if (k < P.np) { res[k] = lo; res[MAXV + k] = hi; }
    else { res[2 * MAXV + (k - P.np)] = hi; }
  }
  if (k == 0) {
    int f = 1;
    long long a = LLONG_MAX, b = LLONG_MIN;
    for (int w = 0; w < RS_THREADS / 32; ++w) { f &= sfits[w]; a = min(a, sdlo[w]); b = max(b, sdhi[w]); }
    res[3 * MAXV] = f;
    if (P.gmask) {
      const bool over = a < INT32_MIN || b > INT32_MAX;
      res[3 * MAXV + 1] = over ? 0 : (int32_t)a;
      res[3 * MAXV + 2] = over ? 0 : (int32_t)b;
      res[3 * MAXV + 3] = over ? 1 : 0;
    }
    done[blockIdx.y] = 0;   // ready for another launch over the same counters
  }
}

cudaError_t launch_range_scan(const Prod* dprods, const OpRef* dops, int nops, int64_t max_n, void* scratch,
                              unsigned int* ddone, int32_t* dranges, cudaStream_t s) {
  if (nops > 0) {
    const int split = range_scan_splits(nops, max_n);
    k_range_scan<<<dim3(split, nops), RS_THREADS, 0, s>>>(dprods, dops, (RangePart*)scratch, ddone, dranges);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// encoding of one term of an operand into its input key
// poly:    key = code = sum_k c_k (e_k - emin_k)
// Poisson: key = ((kind * T2) + tcode) * Wp + pcode, tcode >= 0 for canonical input
// ---------------------------------------------------------------------------
struct TermCode {
  int64_t pcode;
  int64_t tcode;
  int kind;
  uint32_t bad;   // status bits
  bool drop;      // truncated product: the term's degree leaves it no partner
};

__device__ __forceinline__ TermCode encode_term(const Prod& P, const Operand& O, int64_t i) {
  TermCode tc;
  tc.pcode = 0; tc.tcode = 0; tc.kind = 0; tc.bad = 0; tc.drop = false;
  int64_t deg = 0;
#pragma unroll 4
  for (int k = 0; k < P.np; ++k) {
    int32_t e = O.e[(int64_t)k * O.n + i];
    if (P.graded) {
      if ((P.gmask >> k) & 1u) deg += e;
      if (k == P.gvar) continue;   // its digit is the degree
    }
    if (e < O.emin[k] || e > O.emax[k]) tc.bad |= ST_RANGE;
    tc.pcode += P.c[k] * (int64_t)(e - O.emin[k]);
  }
  if (P.graded) {
    const int r = P.gvar;
    if (deg < O.emin[r]) tc.bad |= ST_RANGE;
    if (deg > O.emax[r]) tc.drop = true;   // above the operand's degree limit
    else tc.pcode += P.c[r] * (deg - O.emin[r]);
  }
  if (P.nt > 0) {
#pragma unroll 4
    for (int k = 0; k < P.nt; ++k) {
      int32_t t = O.t[(int64_t)k * O.n + i];
      int32_t a = t < 0 ? -t : t;
      if (a > O.tmax[k]) tc.bad |= ST_RANGE;
      tc.tcode += P.c[P.np + k] * (int64_t)t;
    }
    tc.kind = O.k[i];
    if (tc.kind > 1) tc.bad |= ST_INVALID;
    // canonical input: highest-index nonzero multiplier positive (code > 0),
    // or the zero vector under a cosine
    if (tc.tcode < 0 || (tc.tcode == 0 && tc.kind != 0)) tc.bad |= ST_INVALID;
  }
  return tc;
}

__device__ __forceinline__ uint64_t term_key(const Prod& P, const TermCode& tc) {
  if (P.nt == 0) return (uint64_t)tc.pcode;
  return (uint64_t)(((int64_t)tc.kind * P.T2 + tc.tcode) * P.Wp + tc.pcode);
}

__global__ void __launch_bounds__(256) k_encode(Prod* __restrict__ prods, const OpRef* __restrict__ ops) {
  const OpRef r = ops[blockIdx.y];
  Prod& P = prods[r.prod];
  Operand& O = r.which ? P.g : P.f;
  uint32_t bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < O.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    TermCode tc = encode_term(P, O, i);
    bad |= tc.bad;
    uint64_t key = tc.drop ? (uint64_t)(O.sent + i) : term_key(P, tc);
    if (tc.bad) key = 0;   // keeps later kernels in bounds; the status fails the product
    if (O.sort_method == SORT_BITONIC) {
      O.skey[i] = (key << O.idx_bits) | (uint64_t)i;
    } else {
      O.skey[i] = key;
      if (O.sort_method == SORT_RADIX) ((uint64_t*)O.sidx)[i] = (uint64_t)i;
    }
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (bad && (threadIdx.x & 31) == 0) atomicOr(&P.status, bad);
}

cudaError_t launch_encode(Prod* dprods, const OpRef* dops, int nops, cudaStream_t s) {
  if (nops > 0) k_encode<<<dim3(8, nops), 256, 0, s>>>(dprods, dops);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// gather: sorted keys (+ source index) -> sorted encoded operand arrays.
// Duplicate keys are adjacent after the sort.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gather(Prod* __restrict__ prods, const OpRef* __restrict__ ops) {
  const OpRef r = ops[blockIdx.y];
  Prod& P = prods[r.prod];
  Operand& O = r.which ? P.g : P.f;
  const uint64_t mask = (O.idx_bits > 0) ? ((1ull << O.idx_bits) - 1) : 0;
  uint32_t bad = 0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < O.n;
       q += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key, prev = ~0ull;
    int64_t src;
    if (O.sort_method == SORT_BITONIC) {
      uint64_t v = O.skey[q];
      key = v >> O.idx_bits;
      src = (int64_t)(v & mask);
      if (q > 0) prev = O.skey[q - 1] >> O.idx_bits;
    } else {
      // bitmap and radix sorts leave sorted keys in skey2 and indices in sidx2
      key = O.skey2[q];
      src = (int64_t)((const uint64_t*)O.sidx2)[q];
      if (q > 0) prev = O.skey2[q - 1];
    }
    const bool dropped = key >= (uint64_t)O.sent;   // truncated away (sorted last)
    if (q > 0 && prev == key && !dropped) bad |= ST_DUP;
    if (dropped && (q == 0 || prev < (uint64_t)O.sent)) O.nkeep = q;
    if (src < 0 || src >= O.n) { bad |= ST_DUP; src = 0; }
    if (P.nt == 0) {
      O.code[q] = (int64_t)key;
      if (O.code32) O.code32[q] = (int32_t)key;
      if (P.f64) ((double*)O.coef)[q] = ((const double*)O.c)[src];
      else ((int64_t*)O.coef)[q] = ((const int64_t*)O.c)[src];
    } else {
      TermCode tc = encode_term(P, O, src);
      if (dropped) { tc.pcode = TRUNC_PSENT; tc.tcode = 0; tc.kind = 0; }
      O.code[q] = tc.pcode;
      O.tcode[q] = tc.tcode;
      O.kind[q] = (uint8_t)tc.kind;
      double c = ((const double*)O.c)[src];
      // the 1/2 of the product-to-sum identities is applied to f once here;
      // scaling by 1/2 is exact, so (c_f / 2) * c_g == (c_f * c_g) / 2
      ((double*)O.coef)[q] = r.which == 0 ? 0.5 * c : c;
    }
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (bad && (threadIdx.x & 31) == 0) atomicOr(&P.status, bad);
}

cudaError_t launch_gather(Prod* dprods, const OpRef* dops, int nops, cudaStream_t s) {
  if (nops > 0) k_gather<<<dim3(8, nops), 256, 0, s>>>(dprods, dops);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// cluster front end (SORT_CLUSTER operands): one cluster of CL_CTAS CTAs per
// operand.  The operand's key range is cut into CL_CTAS slices; CTA r holds
// slice r of the key bitmap and, per bitmap word, the number of set bits of
// the slice before it, in its shared memory.  Term i belongs to thread
// (i mod CL_CTAS * CL_THREADS) of the cluster, which holds CL_K terms at a
// time in registers (larger operands take several rounds).
//   1. each thread encodes its terms (every load issued before any is used)
//      and sets their bits in the owning CTA's slice (atomicOr through
//      distributed shared memory; a bit already set is a repeated key);
//   2. each CTA turns its slice into per-word prefix counts (block scan), and
//      the slices' totals give every slice its first rank;
//   3. each thread ranks its keys with two loads from the owning CTA (the
//      word's prefix and the word) and writes the terms in sorted position
//      (the gather); each CTA fills the dense g bucket index of its slice.
// It replaces the encode, sort and gather launches (one CTA per operand for
// the sort) by one launch whose every phase is spread over CL_CTAS SMs.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

__global__ void __cluster_dims__(CL_CTAS, 1, 1) __launch_bounds__(CL_THREADS)
    k_front_cluster(Prod* __restrict__ prods, const OpRef* __restrict__ ops) {
  extern __shared__ uint32_t csm[];
  __shared__ uint32_t wsum[CL_THREADS / 32];
  __shared__ unsigned long long s_tot, s_drop;
  __shared__ unsigned long long s_all[2][CL_CTAS];   // every slice's total and dropped count
  __shared__ int64_t s_base[CL_CTAS + 1];
  cg::cluster_group cl = cg::this_cluster();
  const unsigned me = cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const OpRef r = ops[blockIdx.x / CL_CTAS];
  Prod& P = prods[r.prod];
  Operand& O = r.which ? P.g : P.f;
  const int64_t R = O.key_range, n = O.n;
  const int64_t Lw = cluster_slice_words(R);
  const uint64_t L = (uint64_t)Lw * 32;
  uint32_t* bits = csm;
  uint32_t* pre = csm + Lw;   // set bits of the slice before each word
  for (int64_t w = tid; w < Lw; w += CL_THREADS) bits[w] = 0;
  if (tid == 0) s_drop = 0;
  cl.sync();   // every slice is clear before any thread of the cluster sets a bit
  const int64_t first = (int64_t)me * CL_THREADS + tid, stride = (int64_t)CL_CTAS * CL_THREADS;
  const int64_t round = (int64_t)CL_K * stride;
  // an operand of more than `round` terms takes several rounds, its keys
  // kept in the sort-key array between the passes (each thread reads back
  // only what it wrote); a smaller one keeps them in registers
  const bool spill = n > round;
  uint64_t key[CL_K];
  uint32_t bad = 0;
  unsigned long long ndrop = 0;
  for (int64_t base = first; base < n; base += round) {
#pragma unroll
    for (int k = 0; k < CL_K; ++k) {
      const int64_t i = base + k * stride;
      key[k] = 0;
      if (i < n) {
        TermCode tc = encode_term(P, O, i);
        uint64_t kk = tc.drop ? (uint64_t)(O.sent + i) : term_key(P, tc);
        if (!tc.bad && kk >= (uint64_t)R) tc.bad |= ST_RANGE;   // keeps the slice index in bounds
        if (tc.bad) kk = 0;   // the status fails the product
        bad |= tc.bad;
        ndrop += tc.drop ? 1 : 0;
        key[k] = kk;
      }
    }
#pragma unroll
    for (int k = 0; k < CL_K; ++k) {
      const int64_t i = base + k * stride;
      if (i < n) {
        const unsigned owner = (unsigned)(key[k] / L);
        const uint64_t off = key[k] - (uint64_t)owner * L;
        const uint32_t bit = 1u << (off & 31);
        if (atomicOr(cl.map_shared_rank(bits, owner) + (off >> 5), bit) & bit) bad |= ST_DUP;
        if (spill) O.skey[i] = key[k];
      }
    }
  }
  cl.sync();   // every key's bit is set
  // per-word prefix counts of this slice: each thread a contiguous run of words
  const int64_t per = (Lw + CL_THREADS - 1) / CL_THREADS;
  const int64_t wa = min(Lw, per * tid), wb = min(Lw, wa + per);
  uint32_t cnt = 0;
  for (int64_t w = wa; w < wb; ++w) cnt += __popc(bits[w]);
  uint32_t x = cnt;   // block exclusive scan of the counts (a slice holds < 2^32 bits)
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  for (int o = 16; o > 0; o >>= 1) ndrop += __shfl_xor_sync(0xffffffffu, ndrop, o);
  if (lane == 0 && ndrop) atomicAdd(&s_drop, ndrop);
  __syncthreads();
  if (warp == 0) {
    uint32_t v = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    wsum[lane] = v;
    if (lane == 31) s_tot = v;
  }
  __syncthreads();
  // every CTA gets this slice's total and dropped count (remote stores, seen
  // after the cluster barrier), so that no one waits on a remote load for them
  if (tid < CL_CTAS) {
    unsigned long long* dst = cl.map_shared_rank(&s_all[0][0], (unsigned)tid);
    dst[me] = s_tot;
    dst[CL_CTAS + me] = s_drop;
  }
  uint32_t run = (warp ? wsum[warp - 1] : 0) + x - cnt;
  for (int64_t w = wa; w < wb; ++w) {
    pre[w] = run;
    run += __popc(bits[w]);
  }
  cl.sync();   // every slice's prefix counts, total and dropped count are final
  if (warp == 0) {
    unsigned long long t = 0, d = 0;
    if (lane < CL_CTAS) {
      t = s_all[0][lane];
      d = s_all[1][lane];
    }
    unsigned long long inc = t;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane < CL_CTAS) s_base[lane] = (int64_t)(inc - t);
    if (lane == CL_CTAS - 1) s_base[CL_CTAS] = (int64_t)inc;
    // terms past the degree bound sort last: the kept prefix
    if (me == 0 && lane == 0) O.nkeep = n - (int64_t)d;
  }
  __syncthreads();
  for (int64_t base = first; base < n; base += round) {
    if (spill) {
#pragma unroll
      for (int k = 0; k < CL_K; ++k) key[k] = base + k * stride < n ? O.skey[base + k * stride] : 0;
    }
    int64_t q[CL_K];
#pragma unroll
    for (int k = 0; k < CL_K; ++k) {
      q[k] = n;
      if (base + k * stride < n) {
        const unsigned owner = (unsigned)(key[k] / L);
        const uint64_t off = key[k] - (uint64_t)owner * L;
        const uint32_t wv = cl.map_shared_rank(bits, owner)[off >> 5];
        const uint32_t pv = cl.map_shared_rank(pre, owner)[off >> 5];
        q[k] = s_base[owner] + pv + __popc(wv & ((1u << (off & 31)) - 1u));
      }
    }
#pragma unroll
    for (int k = 0; k < CL_K; ++k) {
      const int64_t i = base + k * stride;
      if (i >= n) continue;
      if (q[k] >= n) { bad |= ST_DUP; continue; }
      if (P.nt == 0) {
        O.code[q[k]] = (int64_t)key[k];
        if (O.code32) O.code32[q[k]] = (int32_t)key[k];
        if (P.f64) ((double*)O.coef)[q[k]] = ((const double*)O.c)[i];
        else ((int64_t*)O.coef)[q[k]] = ((const int64_t*)O.c)[i];
      } else {
        TermCode tc = encode_term(P, O, i);
        if (key[k] >= (uint64_t)O.sent) { tc.pcode = TRUNC_PSENT; tc.tcode = 0; tc.kind = 0; }
        O.code[q[k]] = tc.pcode;
        O.tcode[q[k]] = tc.tcode;
        O.kind[q[k]] = (uint8_t)tc.kind;
        const double c = ((const double*)O.c)[i];
        ((double*)O.coef)[q[k]] = r.which == 0 ? 0.5 * c : c;   // the 1/2 of the product-to-sum identities
      }
    }
  }
  // the g bucket index of a dense product: gidx[b] = number of keys below
  // b << gshift, for the buckets that start in this slice (the last CTA also
  // takes the buckets past every slice)
  if (r.which == 1 && P.nt == 0 && P.path == PATH_DENSE && P.gidx) {
    const int sh = P.gshift;
    const int64_t gn = P.gidx_n;
    const int64_t lo = (int64_t)me * (int64_t)L;
    const int64_t b0 = (lo + (int64_t(1) << sh) - 1) >> sh;
    const int64_t b1 = me == CL_CTAS - 1 ? gn + 1 : min(gn + 1, (lo + (int64_t)L + (int64_t(1) << sh) - 1) >> sh);
    for (int64_t b = b0 + tid; b < b1; b += CL_THREADS) {
      const int64_t off = (b << sh) - lo;
      int64_t v = s_base[CL_CTAS];
      if (off < (int64_t)L) {
        const int64_t w = off >> 5;
        v = s_base[me] + pre[w] + __popc(bits[w] & ((1u << (off & 31)) - 1u));
      }
      P.gidx[b] = (int32_t)v;
    }
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (bad && lane == 0) atomicOr(&P.status, bad);
  // other CTAs read this CTA's slice until here; every such read has been
  // used before its thread arrives, so the arrival needs no release
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

cudaError_t launch_front_cluster(Prod* dprods, const OpRef* dops, int nops, int64_t max_key_range,
                                 cudaStream_t s) {
  if (nops <= 0) return cudaSuccess;
  const int64_t lw = cluster_slice_words(max_key_range);
  const size_t smem = (size_t)(2 * lw) * 4;
  cudaError_t e = raise_smem_limit((const void*)k_front_cluster, (size_t)smem);
  if (e != cudaSuccess) return e;
  k_front_cluster<<<(unsigned)(nops * CL_CTAS), CL_THREADS, smem, s>>>(dprods, dops);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// decoding of output keys (inverse of the coding: mixed-radix digits)
// ---------------------------------------------------------------------------
// n: terms to decode; with dev_count, at most n of the product's device-side
// count (Prod::nout, 0 for a failed product).  vals/coef: when coef is given,
// the coefficients are copied too.
__global__ void __launch_bounds__(256) k_decode_poly(const Prod* __restrict__ prods, int prod,
                                                     const uint64_t* __restrict__ okey, int64_t n,
                                                     int32_t* __restrict__ exps, int64_t ld,
                                                     int64_t* __restrict__ codes, int dev_count,
                                                     const uint64_t* __restrict__ vals,
                                                     uint64_t* __restrict__ coef) {
  const Prod& P = prods[prod];
  if (dev_count) n = P.status ? 0 : min(n, P.nout);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t code = (int64_t)okey[q] + P.klo;   // keys are relative to the key window
    if (codes) codes[q] = code;
    if (exps) decode_poly_part(P, code, exps, ld, q);
    if (coef) coef[q] = vals[q];
  }
}

cudaError_t launch_decode_poly(const Prod* dprods, int prod, const uint64_t* okey, int64_t n,
                               int32_t* exps, int64_t ld, int64_t* codes, cudaStream_t s,
                               bool dev_count, const uint64_t* vals, uint64_t* coef) {
  if (n > 0) {
    int64_t grid = (n + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    k_decode_poly<<<(unsigned)grid, 256, 0, s>>>(dprods, prod, okey, n, exps, ld, codes, dev_count ? 1 : 0,
                                                 vals, coef);
  }
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_decode_pseries(const Prod* __restrict__ prods, int prod,
                                                        const uint64_t* __restrict__ okey, int64_t n,
                                                        int32_t* __restrict__ exps,
                                                        int32_t* __restrict__ trig,
                                                        uint8_t* __restrict__ kind, int64_t ld,
                                                        int64_t* __restrict__ codes, int dev_count,
                                                        const uint64_t* __restrict__ vals,
                                                        uint64_t* __restrict__ coef) {
  const Prod& P = prods[prod];
  if (dev_count) n = P.status ? 0 : min(n, P.nout);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t key = (int64_t)okey[q] + P.klo;   // keys are relative to the key window
    if (codes) codes[q] = key;
    if (coef) coef[q] = vals[q];
    decode_pseries_term(P, key, exps, trig, kind, ld, q);
  }
}

cudaError_t launch_decode_pseries(const Prod* dprods, int prod, const uint64_t* okey, int64_t n,
                                  int32_t* exps, int32_t* trig, uint8_t* kind, int64_t ld,
                                  int64_t* codes, cudaStream_t s, bool dev_count, const uint64_t* vals,
                                  uint64_t* coef) {
  if (n > 0) {
    int64_t grid = (n + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    k_decode_pseries<<<(unsigned)grid, 256, 0, s>>>(dprods, prod, okey, n, exps, trig, kind, ld,
                                                    codes, dev_count ? 1 : 0, vals, coef);
  }
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_decode_batch(const Prod* __restrict__ prods, int nprod,
                                                      const int64_t* __restrict__ ostart,
                                                      const ResDesc* __restrict__ rd,
                                                      const uint64_t* __restrict__ okey,
                                                      const uint64_t* __restrict__ oval, int64_t total) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nprod - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ostart[mid] <= q) lo = mid; else hi = mid - 1;
    }
    const Prod& P = prods[lo];
    const ResDesc& R = rd[lo];
    const int64_t t = q - ostart[lo];
    if (t >= R.n) continue;
    const int64_t key = (int64_t)okey[q] + P.klo;   // keys are relative to the key window
    ((uint64_t*)R.coef)[t] = oval[q];
    if (P.nt == 0) {
      decode_poly_part(P, key, R.exps, R.n, t);
    } else {
      const int64_t per_kind = P.T2 * P.Wp;
      const int64_t kd = key >= per_kind ? 1 : 0;   // keys lie below 2 * per_kind
      int64_t pc;
      const int64_t T = divmod_nn(key - kd * per_kind, P.Wp, &pc);
      R.kind[t] = (uint8_t)kd;
      if (P.np > 0) decode_poly_part(P, pc, R.exps, R.n, t);
      int64_t u = T + (P.T2 - 1);
      for (int k = 0; k < P.nt; ++k) {
        int64_t d = u;
        if (k + 1 < P.nt) u = divmod_nn(u, P.w[P.np + k], &d);
        R.trig[(int64_t)k * R.n + t] = (int32_t)(d + P.omin[P.np + k]);
      }
    }
  }
}

cudaError_t launch_decode_batch(const Prod* dprods, int nprod, const int64_t* dostart,
                                const ResDesc* drd, const uint64_t* okey, const uint64_t* oval,
                                int64_t total, cudaStream_t s) {
  if (total > 0 && nprod > 0) {
    int64_t grid = (total + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    k_decode_batch<<<(unsigned)grid, 256, 0, s>>>(dprods, nprod, dostart, drd, okey, oval, total);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// standalone coding of a box (kron_encode / kron_decode entry points)
// ---------------------------------------------------------------------------
struct Box {
  int32_t emin[MAXV];
  int32_t emax[MAXV];
  int32_t w[MAXV];
  int64_t c[MAXV];
};

__global__ void k_encode_box(const int32_t* __restrict__ exps, int64_t n, int nvars, Box b,
                             int64_t* __restrict__ codes, uint32_t* status) {
  uint32_t bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t code = 0;
    for (int k = 0; k < nvars; ++k) {
      int32_t e = exps[(int64_t)k * n + i];
      if (e < b.emin[k] || e > b.emax[k]) bad = 1;
      code += b.c[k] * (int64_t)(e - b.emin[k]);
    }
    codes[i] = code;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_RANGE);
}

__global__ void k_decode_box(const int64_t* __restrict__ codes, int64_t n, int nvars, Box b,
                             int64_t W, int32_t* __restrict__ exps, uint32_t* status) {
  uint32_t bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = codes[i];
    if (rem < 0 || rem >= W) { bad = 1; rem = 0; }
    for (int k = 0; k < nvars; ++k) {
      int64_t d = rem;
      if (k + 1 < nvars) rem = divmod_nn(rem, b.w[k], &d);
      exps[(int64_t)k * n + i] = (int32_t)(d + b.emin[k]);
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_RANGE);
}

static Box make_box(int nvars, const int32_t* emin, const int32_t* emax, const int64_t* cvec) {
  Box b;
  for (int k = 0; k < MAXV; ++k) { b.emin[k] = 0; b.emax[k] = 0; b.w[k] = 1; b.c[k] = 0; }
  for (int k = 0; k < nvars; ++k) {
    b.emin[k] = emin[k];
    b.emax[k] = emax[k];
    b.w[k] = emax[k] - emin[k] + 1;
    b.c[k] = cvec[k];
  }
  return b;
}

cudaError_t launch_encode_box(const int32_t* exps, int64_t n, int nvars, const int32_t* emin,
                              const int32_t* emax, const int64_t* cvec, int64_t* codes,
                              uint32_t* dstatus, cudaStream_t s) {
  if (n > 0) {
    int64_t grid = (n + 255) / 256;
    if (grid > 152 * 8) grid = 152 * 8;
    k_encode_box<<<(unsigned)grid, 256, 0, s>>>(exps, n, nvars, make_box(nvars, emin, emax, cvec),
                                                codes, dstatus);
  }
  return cudaGetLastError();
}

cudaError_t launch_decode_box(const int64_t* codes, int64_t n, int nvars, const int32_t* emin,
                              const int32_t* w, const int64_t* cvec, int64_t W, int32_t* exps,
                              uint32_t* dstatus, cudaStream_t s) {
  if (n > 0) {
    int32_t emax[MAXV];
    for (int k = 0; k < nvars; ++k) emax[k] = emin[k] + w[k] - 1;
    int64_t grid = (n + 255) / 256;
    if (grid > 152 * 8) grid = 152 * 8;
    k_decode_box<<<(unsigned)grid, 256, 0, s>>>(codes, n, nvars, make_box(nvars, emin, emax, cvec), W,
                                                exps, dstatus);
  }
  return cudaGetLastError();
}

}  // namespace kr
