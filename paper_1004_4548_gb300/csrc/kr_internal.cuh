// Internal declarations of libkron: the per-product plan that the host writes
// and every kernel reads, device helpers, and the kernel launchers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kron.h"

namespace kr {

constexpr int MAXV = KR_MAXV;
// per-operand range record written by k_range_scan: [0, MAXV) exponent minima,
// [MAXV, 2 MAXV) maxima, [2 MAXV, 3 MAXV) max |t|, [3 MAXV] 1 when every
// coefficient is an int64 within the int32 range; for a truncated product
// [3 MAXV + 1], [3 MAXV + 2] the least and largest degree of a term in the
// truncation variables and [3 MAXV + 3] 1 when a degree leaves the int32 range
constexpr int RANGE_STRIDE = 3 * MAXV + 4;
// code of the polynomial part of a Poisson term dropped by truncation: any
// sum of two such codes stays at or above every code range that truncation
// allows (those are at most 2^61)
constexpr int64_t TRUNC_PSENT = int64_t(1) << 61;
constexpr int PATH_DENSE = 1;
constexpr int PATH_HASH = 2;

// status bits a kernel may raise for one product (OR-ed into Prod::status)
constexpr uint32_t ST_RANGE = 1u;       // exponent outside the coding box
constexpr uint32_t ST_DUP = 2u;         // repeated input key
constexpr uint32_t ST_INVALID = 4u;     // non-canonical trig input, sine of zero vector
constexpr uint32_t ST_TABLE_FULL = 8u;  // hash probe limit reached
constexpr uint32_t ST_OUTCAP = 16u;     // compaction found more terms than reserved

// sort method chosen per operand by the host
constexpr int SORT_BITMAP = 1;   // key range fits an on-chip bitmap
constexpr int SORT_BITONIC = 2;  // n fits a shared-memory bitonic network
constexpr int SORT_RADIX = 3;    // device-wide LSD radix sort
constexpr int SORT_CLUSTER = 4;  // bitmap over a cluster's shared memory: encode, rank and
                                 // gather in one kernel (large operands, few per call)

// cluster front end: CL_CTAS CTAs per operand, each holding one slice of the
// operand's key bitmap (and per-word prefix counts) in its shared memory
constexpr int CL_CTAS = 8;
constexpr int CL_THREADS = 1024;
constexpr int CL_K = 4;              // terms per thread and round
constexpr int64_t CL_MIN_N = 2048;   // smaller operands keep the one-CTA bitmap sort
// key ranges up to this many bits: a slice's bitmap and per-word prefix
// counts (8 bytes per 32 keys) in at most 220 KB of shared memory per CTA
constexpr int64_t CL_MAX_BITS = (int64_t)CL_CTAS * 28160 * 32;
constexpr int CL_MAX_OPS = 64;       // more bitmap operands in a call: one CTA each
__host__ __device__ inline int64_t cluster_slice_words(int64_t key_range) {
  const int64_t words = (key_range + 31) >> 5;
  const int64_t per = (words + CL_CTAS - 1) / CL_CTAS;
  return (per + 7) & ~int64_t(7);
}

// One input series on the device.
struct Operand {
  const int32_t* e;     // [np][n] exponents
  const int32_t* t;     // [nt][n] trig multipliers (Poisson)
  const uint8_t* k;     // [n] kinds (Poisson)
  const void* c;        // [n] coefficients (int64 or double)
  int64_t n;
  int32_t emin[MAXV];   // this operand's exponent minima (its coding offset)
  int32_t emax[MAXV];   // declared maxima (range check)
  int32_t tmax[MAXV];   // max |t_k| of this operand (range check)
  // encoded, sorted copies in scratch
  uint64_t* skey;       // sort keys (bitonic: key << idx_bits | index, sorted in place)
  uint64_t* sidx;       // radix path: source indices
  uint64_t* skey2;      // bitmap / radix paths: sorted keys
  uint64_t* sidx2;      // bitmap / radix paths: source index of each sorted key
  int64_t* code;        // sorted: polynomial code (poly) or poly part (Poisson)
  int32_t* code32;      // dense path, g only: the sorted codes as int32 (W <= 2^31)
  int64_t* tcode;       // sorted: signed trig code (Poisson)
  uint8_t* kind;        // sorted kinds (Poisson)
  void* coef;           // sorted coefficients (Poisson f: pre-multiplied by 1/2)
  int32_t sort_method;
  int32_t idx_bits;     // bits of the index packed under the key (bitmap/bitonic)
  int64_t key_range;    // input keys lie in [0, key_range)
  // truncated products: a term that cannot reach the kept degrees gets the
  // key sent + (its index), so it sorts after every kept term; the gather
  // records how many terms are kept (the sorted prefix [0, nkeep))
  int64_t sent;
  int64_t nkeep;
  // truncation by harmonic order: the counted trig multipliers as 16-bit
  // lanes biased by 32768, two per word, rows [0, hwords) holding t and rows
  // [hwords, 2 hwords) holding -t ([2 hwords][n]), so that one sum of
  // absolute lane differences (vsadu2) per word gives |t_f - t_g| and
  // |t_f + t_g| in the counted variables
  uint32_t* hpack;
  // truncation by coefficient magnitude: sort scratch (keys, indices and
  // their ping-pong copies) and the staging of the reordered term arrays
  uint64_t* mkey;
  uint64_t* midx;
  uint64_t* mkey2;
  uint64_t* midx2;
  unsigned char* mtmp;
};

// One product, planned on the host, read by every kernel.
struct Prod {
  Operand f, g;
  int32_t np, nt;       // polynomial variables, trig variables (0: polynomial product)
  int32_t f64;          // coefficients are double
  int32_t path;         // PATH_DENSE or PATH_HASH
  int32_t coef32;       // int64 coefficients that all fit in int32 (32x32->64 multiply)
  int64_t c[MAXV];      // coding vector; poly part [0, np), trig part [np, np + nt)
  int32_t w[MAXV];      // output widths
  int32_t omin[MAXV];   // output box minimum (poly), -R_k (trig)
  // truncated product (graded coding): the degree in the variables of gmask
  // replaces variable gvar and is the most significant polynomial digit; the
  // digits are the other variables in ascending order, then the degree.
  // w[gvar], omin[gvar] describe the degree digit; gvar_min / gvar_max are
  // the output range of variable gvar itself.
  int32_t graded;
  int32_t gvar;
  uint32_t gmask;
  int32_t gvar_min, gvar_max;
  // truncation by harmonic order (Poisson series): a term is kept when the
  // sum of |t_k| over the trig variables of hmask is <= hN; hwords packed
  // words per term (Operand::hpack)
  int32_t htrunc;
  int32_t hwords;
  uint32_t hmask;
  int64_t hN;
  // truncation by coefficient magnitude (float64): a pair is kept when
  // |C_f * C_g| >= cmin as the kernels form the product (for Poisson series
  // f's coefficients are halved, and so is cmin); both operands are then in
  // order of decreasing |C| (kept terms first)
  int32_t ctrunc;
  double cmin;
  int64_t Wp;           // polynomial code range (product of poly widths)
  int64_t T2;           // canonical |trig code| values: (Wt - 1) / 2 + 1
  int64_t krange;       // output key range: Wp, or 2 * T2 * Wp for Poisson
  // the window of output keys computed: [klo, klo + kspan) (the whole range
  // unless a window was asked for).  Accumulator slots, compacted keys and
  // ordering are relative to klo; the decode adds it back.  clip: some pairs
  // produce keys outside the window (a window or a truncation), so the
  // per-pair kernels test each key.
  int64_t klo;
  int64_t kspan;
  int32_t clip;
  // dense path
  int64_t S;            // output codes per block
  int64_t nblocks;
  int64_t work_target;  // pairs per task
  void* dense;          // [kspan] accumulators (slot = key - klo)
  int32_t* gidx;        // gidx[b] = first j with g.code[j] >= b << gshift, b in [0, gidx_n]
  int64_t gidx_n;       // buckets (the last entry gidx[gidx_n] = g.n)
  int32_t gshift;
  // hash path
  uint32_t* hll;        // HyperLogLog registers of the product's output keys (HLL_M)
  double hll_est;       // estimated distinct output keys
  uint64_t* table;      // [slots][2] = (key + 1, value); key 0 = empty
  int64_t slots;        // power of two
  int32_t probe_limit;
  int32_t tile_i, tile_j;
  int64_t tiles_j;      // tiles along g
  int64_t task_begin;   // first task index of this product (hash tiles)
  int64_t ntasks;
  // compaction
  int64_t chunk;        // accumulator slots per compaction chunk
  int64_t nchunks;
  int64_t chunk_begin;  // first chunk index of this product
  int64_t out_cap;      // output terms reserved
  int64_t out_begin;    // first output slot in the batch output arrays (reserved)
  // results
  uint32_t status;
  int64_t nout;
  int64_t out_start;    // start of this product's terms in the output arrays
};

// A dense-path task: one output block, a slice of f.
struct DenseTask {
  int32_t prod;
  int32_t pad;
  int64_t block;
  int64_t i0, i1;
  int64_t single;       // 1 when the block has one task (no other writer)
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t lower_bound_i64(const int64_t* a, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// two lower_bounds over the same sorted array by a whole warp (every lane calls
// it with the same arguments and gets both answers): 32 probes per round cut
// each range 32-fold, the two searches' rounds interleaved
__device__ __forceinline__ void warp_lower_bound2(const int64_t* a, int64_t n, int64_t x1, int64_t x2,
                                                  int64_t* r1, int64_t* r2) {
  const int lane = threadIdx.x & 31;
  int64_t lo1 = 0, hi1 = n, lo2 = 0, hi2 = n;   // answers in [lo, hi]
  bool done1 = false, done2 = false;
  while ((!done1 && hi1 - lo1 > 32) || (!done2 && hi2 - lo2 > 32)) {
    const bool s1 = !done1 && hi1 - lo1 > 32, s2 = !done2 && hi2 - lo2 > 32;
    const int64_t st1 = (hi1 - lo1 + 31) >> 5, st2 = (hi2 - lo2 + 31) >> 5;
    const int64_t p1 = lo1 + lane * st1, p2 = lo2 + lane * st2;
    const bool b1 = s1 && p1 < hi1 && a[p1] < x1;
    const bool b2 = s2 && p2 < hi2 && a[p2] < x2;
    const int c1 = __popc(__ballot_sync(0xffffffffu, b1));
    const int c2 = __popc(__ballot_sync(0xffffffffu, b2));
    if (s1) {
      if (c1 == 0) { hi1 = lo1; done1 = true; }
      else {
        const int64_t pc = lo1 + (int64_t)c1 * st1;
        lo1 = lo1 + (int64_t)(c1 - 1) * st1 + 1;
        if (c1 < 32 && pc < hi1) hi1 = pc;
      }
    }
    if (s2) {
      if (c2 == 0) { hi2 = lo2; done2 = true; }
      else {
        const int64_t pc = lo2 + (int64_t)c2 * st2;
        lo2 = lo2 + (int64_t)(c2 - 1) * st2 + 1;
        if (c2 < 32 && pc < hi2) hi2 = pc;
      }
    }
  }
  const int64_t p1 = lo1 + lane, p2 = lo2 + lane;
  *r1 = lo1 + __popc(__ballot_sync(0xffffffffu, p1 < hi1 && a[p1] < x1));
  *r2 = lo2 + __popc(__ballot_sync(0xffffffffu, p2 < hi2 && a[p2] < x2));
}

// two lower_bound searches over the sorted g codes at once, each through the
// coarse bucket index (the answer for x lies in [gidx[x >> gshift],
// gidx[(x >> gshift) + 1]]), their probes interleaved so that the loads of
// both are in flight together
__device__ __forceinline__ void g_lower_bound2(const int64_t* G, int64_t ng, const int32_t* gidx,
                                               int64_t gidx_n, int gshift, int64_t x1, int64_t x2,
                                               int64_t* r1, int64_t* r2) {
  int64_t lo1 = 0, hi1 = 0, lo2 = 0, hi2 = 0;
  if (x1 > 0) {
    const int64_t b = x1 >> gshift;
    if (b >= gidx_n) lo1 = hi1 = ng; else { lo1 = gidx[b]; hi1 = gidx[b + 1]; }
  }
  if (x2 > 0) {
    const int64_t b = x2 >> gshift;
    if (b >= gidx_n) lo2 = hi2 = ng; else { lo2 = gidx[b]; hi2 = gidx[b + 1]; }
  }
  while (lo1 < hi1 || lo2 < hi2) {
    const int64_t m1 = (lo1 + hi1) >> 1, m2 = (lo2 + hi2) >> 1;
    const bool a1 = lo1 < hi1, a2 = lo2 < hi2;
    const int64_t v1 = a1 ? G[m1] : 0, v2 = a2 ? G[m2] : 0;
    if (a1) { if (v1 < x1) lo1 = m1 + 1; else hi1 = m1; }
    if (a2) { if (v2 < x2) lo2 = m2 + 1; else hi2 = m2; }
  }
  *r1 = lo1;
  *r2 = lo2;
}

// q = x / d and *r = x % d for x >= 0, d >= 1: 32-bit division when x fits
// (a 64-bit division costs several times more), which after the first digits
// of a code is almost always the case.
__device__ __forceinline__ int64_t divmod_nn(int64_t x, int64_t d, int64_t* r) {
  if ((uint64_t)x <= 0xffffffffull && d <= 0xffffffffll) {
    const uint32_t q = (uint32_t)x / (uint32_t)d;
    *r = (int64_t)((uint32_t)x - q * (uint32_t)d);
    return q;
  }
  const int64_t q = x / d;
  *r = x - q * d;
  return q;
}

// Exponents of the polynomial part of an output code (the inverse of the
// mixed-radix coding): variable k of the term goes to exps[k * ld + q].  A
// graded code holds the other variables first and the degree last; the
// exponent of gvar is the degree minus the other exponents of the mask.
__device__ __forceinline__ void decode_poly_part(const Prod& P, int64_t pc, int32_t* __restrict__ exps,
                                                 int64_t ld, int64_t q) {
  if (!P.graded) {
    for (int k = 0; k < P.np; ++k) {
      int64_t d = pc;
      if (k + 1 < P.np) pc = divmod_nn(pc, P.w[k], &d);
      exps[(int64_t)k * ld + q] = (int32_t)(d + P.omin[k]);
    }
    return;
  }
  int64_t deg_rest = 0;
  for (int k = 0; k < P.np; ++k) {
    if (k == P.gvar) continue;
    int64_t d;
    pc = divmod_nn(pc, P.w[k], &d);
    const int64_t e = d + P.omin[k];
    if ((P.gmask >> k) & 1u) deg_rest += e;
    exps[(int64_t)k * ld + q] = (int32_t)e;
  }
  exps[(int64_t)P.gvar * ld + q] = (int32_t)(pc + P.omin[P.gvar] - deg_rest);
}

// Exponents, multipliers and kind of an output key of a Poisson product
// (key = (kind * T2 + tcode) * Wp + pcode, the tcode balanced over the
// symmetric multiplier box) to term q of the output arrays (row stride ld).
__device__ __forceinline__ void decode_pseries_term(const Prod& P, int64_t key, int32_t* __restrict__ exps,
                                                    int32_t* __restrict__ trig, uint8_t* __restrict__ kind,
                                                    int64_t ld, int64_t q) {
  const int64_t per_kind = P.T2 * P.Wp;
  const int64_t kd = key >= per_kind ? 1 : 0;   // keys lie below 2 * per_kind
  int64_t pc;
  const int64_t T = divmod_nn(key - kd * per_kind, P.Wp, &pc);
  if (kind) kind[q] = (uint8_t)kd;
  if (exps) decode_poly_part(P, pc, exps, ld, q);
  if (trig) {
    int64_t u = T + (P.T2 - 1);   // T2 - 1 = sum_k c_k R_k
    for (int k = 0; k < P.nt; ++k) {
      int64_t d = u;
      if (k + 1 < P.nt) u = divmod_nn(u, P.w[P.np + k], &d);
      trig[(int64_t)k * ld + q] = (int32_t)(d + P.omin[P.np + k]);
    }
  }
}

// int64 accumulate into shared memory as two 32-bit words (the low word at
// shared address a, the high word hi_dist bytes further): a 32-bit atomic add
// of the low half returning the old value, its carry by add-with-carry, and a
// 32-bit add of high half and carry when nonzero.  Exact modulo 2^64 whatever
// the order of the adds: each carry is seen by exactly the add that makes it.
__device__ __forceinline__ void smem_acc_split64(uint32_t a, uint32_t hi_dist, uint64_t u) {
  const uint32_t l = (uint32_t)u;
  uint32_t old, h;
  asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(l) : "memory");
  asm("{\n\t.reg .u32 t;\n\tadd.cc.u32 t, %1, %2;\n\taddc.u32 %0, %3, 0;\n\t}"
      : "=r"(h) : "r"(old), "r"(l), "r"((uint32_t)(u >> 32)));
  if (h) asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a + hi_dist), "r"(h) : "memory");
}

// Harmonic orders |t_f - t_g| and |t_f + t_g| (counted variables) of term i
// of f and term j of g, from their packed multipliers (Operand::hpack).
__device__ __forceinline__ void harmonic_orders(const Prod& P, int64_t i, int64_t j, uint32_t* od,
                                                uint32_t* os) {
  const int hw = P.hwords;
  const int64_t nf = P.f.n, ng = P.g.n;
  uint32_t d = 0, sm = 0;
  for (int w = 0; w < hw; ++w) {
    const uint32_t a = __ldg(&P.f.hpack[(int64_t)w * nf + i]);
    d += __vsadu2(a, __ldg(&P.g.hpack[(int64_t)w * ng + j]));
    sm += __vsadu2(a, __ldg(&P.g.hpack[(int64_t)(hw + w) * ng + j]));
  }
  *od = d;
  *os = sm;
}

// Bytes per term of Operand::mtmp: code, coefficient, trig code, packed
// multipliers and kind, each array 8-byte aligned.
__host__ __device__ inline int64_t mag_tmp_bytes_per_term(const Prod& P) {
  return 8 + 8 + (P.nt > 0 ? 8 + 1 : 0) + (P.htrunc ? 8 * (int64_t)P.hwords : 0);
}

// The coefficient bound on a pair's product (false for NaN).
__device__ __forceinline__ bool coef_kept(const Prod& P, double prod) { return fabs(prod) >= P.cmin; }

// 64-bit mixing function (the finaliser of MurmurHash3, Appleby) for table slots
__device__ __forceinline__ uint64_t mix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// ---------------------------------------------------------------------------
// launchers (host side); each returns cudaGetLastError()
// ---------------------------------------------------------------------------
// Raises (never lowers) a kernel's dynamic shared memory limit to `bytes` on
// the current device, thread-safely; launchers call it before launching with
// more than 48 KB.
cudaError_t raise_smem_limit(const void* func, size_t bytes);

struct OpRef {      // (product, operand) pair addressed by a per-operand kernel
  int32_t prod;
  int32_t which;    // 0 = f, 1 = g
};

// Range records of every operand (min / max exponents, max |t|, flags); the
// scratch holds range_scan_scratch_bytes(nops, max_n) bytes.
size_t range_scan_scratch_bytes(int nops, int64_t max_n);
// ddone: nops counters, zero at launch (and zero again after it).
cudaError_t launch_range_scan(const Prod* dprods, const OpRef* dops, int nops, int64_t max_n, void* scratch,
                              unsigned int* ddone, int32_t* dranges, cudaStream_t s);
cudaError_t launch_encode(Prod* dprods, const OpRef* dops, int nops, cudaStream_t s);
cudaError_t launch_sort_small(Prod* dprods, const OpRef* dops, int nops, int method,
                              size_t smem, cudaStream_t s);
cudaError_t launch_gather(Prod* dprods, const OpRef* dops, int nops, cudaStream_t s);
// SORT_CLUSTER operands: encode, bitmap rank and gather (and the g bucket
// index of a dense product) in one launch of one cluster per operand
cudaError_t launch_front_cluster(Prod* dprods, const OpRef* dops, int nops, int64_t max_key_range,
                                 cudaStream_t s);

// Truncation by harmonic order: the packed multipliers of the listed operands
// (from their sorted trig codes).  Truncation by coefficient magnitude: keys
// and indices for the reorder by decreasing |C|, then (after the caller's
// sort, indices back in midx) the reorder itself, through mtmp.
cudaError_t launch_harmonic_pack(Prod* dprods, const OpRef* dops, int nops, int64_t max_n, cudaStream_t s);
cudaError_t launch_mag_keys(Prod* dprods, const OpRef* dops, int nops, int64_t max_n, cudaStream_t s);
cudaError_t launch_mag_reorder(Prod* dprods, const OpRef* dops, int nops, int64_t max_n, cudaStream_t s);

cudaError_t launch_dense_plan(const Prod* dprods, const int32_t* ddense_prods,
                              const int64_t* dblock_begin, int ndense, int64_t nblocks_total,
                              DenseTask* dtasks, int64_t task_cap, int64_t* dtask_count,
                              cudaStream_t s);
cudaError_t launch_build_gindex(const Prod* dprods, const int32_t* ddense_prods, int ndense,
                                int64_t max_ng, cudaStream_t s);
cudaError_t launch_dense_accum(const Prod* dprods, const DenseTask* dtasks,
                               const int64_t* dtask_count, int64_t task_cap, int64_t* dtask_next,
                               int grid, int64_t max_S, cudaStream_t s);
int dense_accum_threads();
// HyperLogLog cardinality estimate of every hash product's output keys
// (Flajolet, Fusy, Gandouet, Meunier 2007), from a pass over all term pairs
// that computes keys only.  2^HLL_B registers per product.
constexpr int HLL_B = 12;
constexpr int HLL_M = 1 << HLL_B;
cudaError_t launch_hll(Prod* dprods, const int32_t* dhash_prods, const int64_t* dtask_begin, int nhash,
                       int grid, cudaStream_t s);
cudaError_t launch_hll_estimate(Prod* dprods, const int32_t* dhash_prods, int nhash, cudaStream_t s);
// Histogram of the output keys of nsamples uniformly drawn term pairs of one
// product over nbins equal slices of [0, krange) (hist zeroed by the caller).
cudaError_t launch_split_sample(const Prod* dprods, int prod, int nbins, int64_t nsamples, uint64_t seed,
                                unsigned long long* dhist, cudaStream_t s);
// accumulation of every hash-path product's tiles (and Poisson tiles on the
// dense path): poly / pseries say which kinds the list holds
// Ceiling probe: updates insert-or-adds (mode 0) or plain adds (mode 1) of
// keys from `distinct` values into a zeroed table of `slots` (a power of two)
// 16-byte slots; fails counts lanes that found no slot.
cudaError_t launch_probe_table_update(uint64_t* table, uint64_t slots, int64_t distinct, int64_t updates,
                                      int mode, unsigned long long* fails, cudaStream_t s);
// (trunc: products truncated by coefficient magnitude or harmonic order, in a
// kernel of their own)
cudaError_t launch_hash_insert(Prod* dprods, const int32_t* dhash_prods, const int64_t* dtask_begin,
                               int nhash, bool poly, bool pseries, bool trunc, int grid, cudaStream_t s);
// Compaction: up to this many chunks one pass (each chunk read once, one
// launch); above it two passes, whose counting pass keeps more loads in
// flight.
constexpr int64_t COMPACT_ONE_PASS_MAX = 1024;
// Writes at most cap terms; products whose terms end beyond cap get ST_OUTCAP.
// Decoded outputs written by the compaction itself (one dense polynomial
// product whose caller's output arrays are in device memory or in pinned
// host memory, through its device mapping): term q's
// exponents to exps[k * ld + q], its code to codes[q], its coefficient to
// coef[q], for q < cap; coef == nullptr: none.
struct DirectOut {
  int32_t* exps = nullptr;
  int64_t* codes = nullptr;
  uint64_t* coef = nullptr;
  int64_t ld = 0;
  int64_t cap = 0;
};
// cstat: nchunks zeroed words of scan state; sync: two zeroed int64 (a
// ticket counter, then an error flag set when a bounded wait gave up); scan:
// scan_scratch_entries(nchunks) int64 for the two-pass form.  With one
// product compacted in one pass, the CTA of the last chunk also records the
// product's count and status (no finishing launch); returns the launches made.
cudaError_t launch_compact(Prod* dprods, int nprod, const int64_t* dchunk_begin, int64_t nchunks,
                           int64_t* dcounts, uint64_t* dcstat, int64_t* dsync, int64_t* dscan,
                           uint64_t* okey, uint64_t* oval, int64_t cap, cudaStream_t s,
                           const DirectOut& direct, int* launches);
// exclusive scan of d[0, n) in place, *dtotal = sum; long arrays use several
// CTAs and scratch of scan_scratch_entries(n) int64 (null: one CTA)
int64_t scan_scratch_entries(int64_t n);
cudaError_t launch_scan_exclusive(int64_t* d, int64_t n, int64_t* dtotal, int64_t* scratch, cudaStream_t s);

// Device-wide LSD radix sort of (key, 8-byte payload) pairs over the low
// `bits` bits of the key.  key/val and key_tmp/val_tmp ping-pong; after the
// call the sorted data is in the tmp arrays when *result_in_tmp is true.
// dscan holds radix_scan_entries(n) int64.
constexpr int RADIX_TILE = 4096;
int64_t radix_scan_entries(int64_t n);
cudaError_t radix_sort_pairs(uint64_t* key, uint64_t* val, uint64_t* key_tmp, uint64_t* val_tmp,
                             int64_t n, int bits, int64_t* dscan, cudaStream_t s,
                             bool* result_in_tmp);

// Orders (key, val)[0, n) by key (keys distinct, < krange) through bins of
// codes and shared-memory segment sorts; key2/val2 hold n terms of scratch,
// bins 2 * (order_bins(krange) + 1) int64.  Result in key/val.
constexpr int64_t ORDER_MAX_BINS = int64_t(1) << 24;
int64_t order_bins(int64_t krange);
int64_t order_bins_scratch(int64_t krange);   // int64 entries of order_by_bins' scratch
// Bitmap-rank ordering for code ranges up to ORDER_BITMAP_MAX codes: result in
// key2/val2; scratch of order_bitmap_bytes(krange).
constexpr int64_t ORDER_BITMAP_MAX = int64_t(1) << 35;
int64_t order_bitmap_bytes(int64_t krange);
cudaError_t order_by_bitmap(const uint64_t* key, const uint64_t* val, uint64_t* key2, uint64_t* val2,
                            int64_t n, int64_t krange, void* scratch, cudaStream_t s);
cudaError_t order_by_bins(uint64_t* key, uint64_t* val, uint64_t* key2, uint64_t* val2, int64_t n,
                          int64_t krange, int64_t* bins, cudaStream_t s);
// Large outputs over code ranges whose one-bit-per-code bitmap would not stay
// in L2 (above 2^30 codes, 128 MB): terms partitioned by the high digits of
// their code in two tile-sorted passes into buckets of about 2048 terms, each
// then ranked by a shared-memory bitmap (or, past 2^37 codes, bucketed by
// 2^20 codes and ranked there); sorted in place (key2/val2: n terms of
// scratch; bins: order_buckets_scratch(krange, n_max) int64 for up to n_max terms).
constexpr int64_t ORDER_BUCKET_MIN_N = int64_t(1) << 20;
constexpr int64_t ORDER_BUCKET_MIN_RANGE = int64_t(1) << 30;
constexpr int64_t ORDER_MAX_BUCKETS = int64_t(1) << 22;
int64_t order_buckets(int64_t krange);
int64_t order_buckets_scratch(int64_t krange, int64_t n_max);
cudaError_t order_by_buckets(uint64_t* key, uint64_t* val, uint64_t* key2, uint64_t* val2, int64_t n,
                             int64_t krange, int64_t* bins, cudaStream_t s);

// Decode of one product's sorted terms.  With dev_count, n is a capacity and
// the count is the product's device-side nout (0 when its status is set);
// given coef, the coefficients (vals) are copied too.
cudaError_t launch_decode_poly(const Prod* dprods, int prod, const uint64_t* okey, int64_t n,
                               int32_t* exps, int64_t ld, int64_t* codes, cudaStream_t s,
                               bool dev_count = false, const uint64_t* vals = nullptr,
                               uint64_t* coef = nullptr);
cudaError_t launch_decode_pseries(const Prod* dprods, int prod, const uint64_t* okey, int64_t n,
                                  int32_t* exps, int32_t* trig, uint8_t* kind, int64_t ld,
                                  int64_t* codes, cudaStream_t s, bool dev_count = false,
                                  const uint64_t* vals = nullptr, uint64_t* coef = nullptr);
// Where a batched decode writes one product's terms ([nvars][n] layouts).
struct ResDesc {
  int32_t* exps;
  int32_t* trig;
  uint8_t* kind;
  void* coef;
  int64_t n;
};
// Decodes the sorted terms of many products in one launch: output q belongs to
// the product p with ostart[p] <= q < ostart[p + 1] (products contiguous).
cudaError_t launch_decode_batch(const Prod* dprods, int nprod, const int64_t* dostart,
                                const ResDesc* drd, const uint64_t* okey, const uint64_t* oval,
                                int64_t total, cudaStream_t s);
cudaError_t launch_encode_box(const int32_t* exps, int64_t n, int nvars, const int32_t* emin,
                              const int32_t* emax, const int64_t* cvec, int64_t* codes,
                              uint32_t* dstatus, cudaStream_t s);
cudaError_t launch_decode_box(const int64_t* codes, int64_t n, int nvars, const int32_t* emin,
                              const int32_t* w, const int64_t* cvec, int64_t W, int32_t* exps,
                              uint32_t* dstatus, cudaStream_t s);

}  // namespace kr
