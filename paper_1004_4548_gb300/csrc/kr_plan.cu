// Host-side planning of one product: coding box, path, scratch sizes.
#include <algorithm>
#include <cmath>

#include "kr_plan.h"

// dense path: tasks per resident CTA (more: a shorter tail of the dynamic
// task queue; fewer: less zeroing and flushing of block slices)
#ifndef KR_TASKS_PER_CTA
#define KR_TASKS_PER_CTA 6
#endif

namespace kr {

int bits_for(uint64_t range) {
  int b = 0;
  if (range <= 1) return 0;
  const uint64_t top = range - 1;
  while (b < 64 && (top >> b) != 0) ++b;
  return b;
}

// Coding vector of Sec. 2: c_0 = 1, c_k = prod_{l<k} w_l; W = prod_k w_k.
kr_status coding_vector(const int64_t* w, int n, int64_t* c, int64_t* W) {
  unsigned __int128 acc = 1;
  for (int k = 0; k < n; ++k) {
    if (w[k] < 1) return KR_ERR_INVALID;
    c[k] = (int64_t)acc;
    acc *= (unsigned __int128)w[k];
    if (acc > (unsigned __int128)INT64_MAX) return KR_ERR_OVERFLOW;
  }
  *W = (int64_t)acc;
  return KR_OK;
}

static int64_t next_pow2(int64_t x) {
  int64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

static void plan_sort(Operand& op, int64_t key_range, int* passes, int64_t* radix_n) {
  op.key_range = key_range;
  op.idx_bits = 0;
  *passes = 0;
  if (key_range <= BITMAP_MAX_BITS) {
    op.sort_method = SORT_BITMAP;
  } else if (op.n <= BITONIC_MAX_N && bits_for((uint64_t)key_range) + bits_for((uint64_t)op.n) <= 63) {
    op.sort_method = SORT_BITONIC;
    op.idx_bits = bits_for((uint64_t)op.n);
  } else {
    op.sort_method = SORT_RADIX;
    *passes = (bits_for((uint64_t)key_range) + 7) / 8;
    if (op.n > *radix_n) *radix_n = op.n;
  }
}

void plan_product(const Job& job, const int32_t* rf, const int32_t* rg, int num_sms, Plan* out) {
  Plan& pl = *out;
  pl = Plan();
  Prod& P = pl.p;
  P.f = job.f;
  P.g = job.g;
  P.np = job.np;
  P.nt = job.nt;
  P.f64 = job.f64 ? 1 : 0;
  const kr_opts& o = job.opts;
  // ---- coding box of the product (output widths; each operand offset by its own minimum)
  int64_t w[MAXV], c[MAXV];
  for (int k = 0; k < P.np; ++k) {
    P.f.emin[k] = rf[k];
    P.f.emax[k] = rf[MAXV + k];
    P.g.emin[k] = rg[k];
    P.g.emax[k] = rg[MAXV + k];
    const int64_t lo = (int64_t)rf[k] + rg[k], hi = (int64_t)rf[MAXV + k] + rg[MAXV + k];
    if (lo < INT32_MIN || hi > INT32_MAX) { pl.st = KR_ERR_OVERFLOW; return; }
    P.omin[k] = (int32_t)lo;
    w[k] = hi - lo + 1;
    if (w[k] > INT32_MAX) { pl.st = KR_ERR_OVERFLOW; return; }
    P.w[k] = (int32_t)w[k];
  }
  // ---- truncation by degree (Sec. 3): graded coding.  The degree in the
  // mask's variables replaces the mask's highest-index variable r and becomes
  // the most significant digit, so "degree <= N" is "code < Wp" with Wp the
  // clipped code range.  Each operand keeps the terms whose degree leaves a
  // partner: deg_f <= N - min deg_g (and the same for g).
  P.graded = 0;
  if (o.truncate) {
    uint32_t m = o.trunc_mask ? o.trunc_mask : 0xffffffffu;
    if (P.np < 32) m &= (1u << P.np) - 1u;
    if (P.np == 0 || m == 0) { pl.st = KR_ERR_INVALID; return; }
    if (rf[3 * MAXV + 3] || rg[3 * MAXV + 3]) { pl.st = KR_ERR_OVERFLOW; return; }
    int r = 0;
    for (int k = 0; k < P.np; ++k)
      if ((m >> k) & 1u) r = k;
    const int64_t dminf = rf[3 * MAXV + 1], dmaxf = rf[3 * MAXV + 2];
    const int64_t dming = rg[3 * MAXV + 1], dmaxg = rg[3 * MAXV + 2];
    const int64_t N = o.trunc_degree;
    const int64_t dlo = dminf + dming;
    const int64_t dhi = std::min(N, dmaxf + dmaxg);
    P.graded = 1;
    P.gvar = r;
    P.gmask = m;
    P.gvar_min = P.omin[r];
    P.gvar_max = (int32_t)((int64_t)P.omin[r] + P.w[r] - 1);
    if (dhi < dlo) { pl.empty = true; return; }   // every term pair exceeds N
    if (dhi - dlo + 1 > INT32_MAX || dlo < INT32_MIN) { pl.st = KR_ERR_OVERFLOW; return; }
    w[r] = dhi - dlo + 1;
    P.w[r] = (int32_t)w[r];
    P.omin[r] = (int32_t)dlo;
    P.f.emin[r] = (int32_t)dminf;
    P.f.emax[r] = (int32_t)std::min(dmaxf, N - dming);
    P.g.emin[r] = (int32_t)dming;
    P.g.emax[r] = (int32_t)std::min(dmaxg, N - dminf);
  }
  int64_t Wp = 1;
  if (P.np > 0) {
    // digits in coding order: variable 0 first; a graded code moves the
    // degree digit (variable r's slot) to the top
    int64_t wd[MAXV], cd[MAXV];
    int ord[MAXV], nd = 0;
    for (int k = 0; k < P.np; ++k)
      if (!(P.graded && k == P.gvar)) ord[nd++] = k;
    if (P.graded) ord[nd++] = P.gvar;
    for (int q = 0; q < nd; ++q) wd[q] = w[ord[q]];
    pl.st = coding_vector(wd, nd, cd, &Wp);
    if (pl.st != KR_OK) return;
    for (int q = 0; q < nd; ++q) c[ord[q]] = cd[q];
    // room for the keys of dropped terms above the code range, and for sums
    if (P.graded && Wp > (int64_t(1) << 61)) { pl.st = KR_ERR_OVERFLOW; return; }
  }
  for (int k = 0; k < P.np; ++k) P.c[k] = c[k];
  P.Wp = Wp;
  P.T2 = 1;
  P.krange = Wp;
  if (P.nt > 0) {
    int64_t wt[MAXV], ct[MAXV], Wt = 1;
    for (int k = 0; k < P.nt; ++k) {
      P.f.tmax[k] = rf[2 * MAXV + k];
      P.g.tmax[k] = rg[2 * MAXV + k];
      const int64_t R = (int64_t)rf[2 * MAXV + k] + rg[2 * MAXV + k];
      wt[k] = 2 * R + 1;
      if (wt[k] > INT32_MAX) { pl.st = KR_ERR_OVERFLOW; return; }
      P.w[P.np + k] = (int32_t)wt[k];
      P.omin[P.np + k] = (int32_t)(-R);
    }
    pl.st = coding_vector(wt, P.nt, ct, &Wt);
    if (pl.st != KR_OK) return;
    for (int k = 0; k < P.nt; ++k) P.c[P.np + k] = ct[k];
    P.T2 = (Wt - 1) / 2 + 1;
    const unsigned __int128 kr = (unsigned __int128)2 * (unsigned __int128)P.T2 * (unsigned __int128)Wp;
    const unsigned __int128 lim = P.graded ? ((unsigned __int128)1 << 62) : (unsigned __int128)INT64_MAX;
    if (kr > lim) { pl.st = KR_ERR_OVERFLOW; return; }
    P.krange = (int64_t)kr;
  }
  // ---- truncation by harmonic order (Sec. 3), Poisson series: each emitted
  // term is tested in the kernels against the packed multipliers
  if (o.trunc_harmonic) {
    uint32_t m = o.harmonic_mask ? o.harmonic_mask : 0xffffffffu;
    if (P.nt < 32) m &= (1u << P.nt) - 1u;
    if (P.nt == 0 || m == 0) { pl.st = KR_ERR_INVALID; return; }
    int counted = 0;
    for (int k = 0; k < P.nt; ++k) {
      if (!((m >> k) & 1u)) continue;
      if (rf[2 * MAXV + k] > 32767 || rg[2 * MAXV + k] > 32767) { pl.st = KR_ERR_INVALID; return; }
      ++counted;
    }
    if (o.harmonic_order < 0) { pl.empty = true; return; }   // no term has a negative order
    P.htrunc = 1;
    P.hmask = m;
    P.hN = o.harmonic_order;
    P.hwords = (counted + 1) / 2;
  }
  // ---- truncation by coefficient magnitude (Sec. 3), float64 coefficients
  if (o.coef_min != 0.0) {
    if (!job.f64 || !(o.coef_min > 0.0) || std::isinf(o.coef_min)) { pl.st = KR_ERR_INVALID; return; }
    P.ctrunc = 1;
    // Poisson tiles form (C_f / 2) * C_g: halving both sides is exact
    P.cmin = P.nt > 0 ? o.coef_min * 0.5 : o.coef_min;
  }
  // ---- window of output keys (the whole range unless one was asked for)
  P.klo = 0;
  P.kspan = P.krange;
  P.clip = P.graded;
  if (o.code_lo > 0 || o.code_hi > 0) {
    const int64_t lo = std::max<int64_t>(0, o.code_lo);
    const int64_t hi = o.code_hi > 0 ? std::min(o.code_hi, P.krange) : P.krange;
    if (lo >= hi) { pl.empty = true; return; }
    P.klo = lo;
    P.kspan = hi - lo;
    P.clip = 1;
  }
  const int64_t nf = P.f.n, ng = P.g.n;
  const double pairs = (double)nf * (double)ng;
  P.coef32 = (!job.f64 && P.nt == 0 && rf[3 * MAXV] == 1 && rg[3 * MAXV] == 1) ? 1 : 0;
  // ---- path (Sec. 3.2: the density of the product decides)
  if (job.poisson) {
    // the lookup array of Sec. 3.1 receives both the sum and the difference
    const bool fits = (double)P.kspan * 8.0 <= (double)DENSE_POISSON_MAX_BYTES;
    if (o.path == KR_PATH_DENSE) {
      if (!fits) { pl.st = KR_ERR_INVALID; return; }
      P.path = PATH_DENSE;
    } else if (o.path == KR_PATH_HASH || P.ctrunc) {
      // a coefficient bound usually keeps a small part of the product: a
      // table sized by the estimate of the kept keys beats clearing and
      // compacting an array over the whole key range
      P.path = PATH_HASH;
    } else {
      const bool dense_enough = (double)P.krange <= DENSE_POISSON_KAPPA * 2.0 * pairs + 65536.0;
      P.path = (fits && dense_enough) ? PATH_DENSE : PATH_HASH;
    }
  } else if (P.ctrunc) {
    // a coefficient bound walks the operands by decreasing |C|, which the
    // block-by-block dense kernel (it needs code order) cannot do
    P.path = PATH_HASH;
  } else if (o.path == KR_PATH_DENSE) {
    if ((double)P.kspan * 8.0 > (double)DENSE_MAX_BYTES || P.krange > INT32_MAX) {
      pl.st = KR_ERR_INVALID;
      return;
    }
    P.path = PATH_DENSE;
  } else if (o.path == KR_PATH_HASH) {
    P.path = PATH_HASH;
  } else {
    // (the dense kernels use 32-bit offsets: codes below 2^31)
    const bool fits = (double)P.kspan * 8.0 <= (double)DENSE_MAX_BYTES && P.krange <= INT32_MAX;
    const bool dense_enough = (double)P.krange <= DENSE_KAPPA * pairs + 65536.0;
    P.path = (fits && dense_enough) ? PATH_DENSE : PATH_HASH;
  }
  // ---- operand sorts
  for (int which = 0; which < 2; ++which) {
    Operand& op = which ? P.g : P.f;
    int64_t kr;
    if (P.graded) {
      kr = P.krange + op.n;   // dropped terms get keys krange + index
    } else if (P.nt == 0) {
      int64_t span = 0;
      for (int k = 0; k < P.np; ++k) span += P.c[k] * (int64_t)(op.emax[k] - op.emin[k]);
      kr = span + 1;
    } else {
      kr = P.krange;
    }
    op.sent = P.graded ? P.krange : kr;
    op.nkeep = op.n;
    plan_sort(op, kr, which ? &pl.passes_g : &pl.passes_f, &pl.radix_sort_n);
    pl.op_bytes[which] = op.n * (8 * 7 + 1) + 8 * 256;
    if (P.htrunc) pl.op_bytes[which] += op.n * 8 * P.hwords;
    if (P.ctrunc) {
      pl.op_bytes[which] += op.n * (8 * 4 + mag_tmp_bytes_per_term(P));
      pl.radix_sort_n = std::max(pl.radix_sort_n, op.n);   // the reorder by magnitude
    }
  }
  // ---- accumulators
  if (P.path == PATH_DENSE && P.nt > 0) {
    // Poisson series on the dense path: tiles of term pairs add into the array
    P.tile_i = HASH_TILE_I;
    P.tile_j = HASH_TILE_J;
    P.tiles_j = ceil_div(ng, HASH_TILE_J);
    P.ntasks = ceil_div(nf, HASH_TILE_I) * P.tiles_j;
    pl.accum_bytes = P.kspan * 8;
    P.chunk = COMPACT_CHUNK;
    P.nchunks = ceil_div(P.kspan, P.chunk);
    pl.out_cap = (int64_t)std::min((double)P.kspan, 2.0 * pairs);
  } else if (P.path == PATH_DENSE) {
    int64_t S = o.block_slots > 0 ? o.block_slots : DEFAULT_S;
    if (S < 256) S = 256;
    if (S > MAX_S) S = MAX_S;
    S = ceil_div(S, 32) * 32;
    const int64_t kr32 = ceil_div(P.kspan, 32) * 32;
    if (S > kr32) S = kr32;
    P.S = S;
    P.nblocks = ceil_div(P.kspan, S);
    // ~6 tasks per resident CTA so the dynamic task queue evens out the
    // uneven (diamond-shaped) work per output block
    const int64_t per_sm = std::max<int64_t>(1, std::min<int64_t>(4, (227 * 1024) / (S * 8 + 11264)));
    // tasks per resident CTA: at least KR_TASKS_PER_CTA, more for large
    // products (tasks of about 50,000 term-products, at most 24 per CTA), so
    // that the last tasks, which set the run's tail, stay short
    const double ctas = (double)num_sms * (double)per_sm;
    const double per_cta = std::min(24.0, std::max((double)KR_TASKS_PER_CTA, pairs / (ctas * 5e4)));
    const double tgt = pairs / (ctas * per_cta);
    P.work_target = (int64_t)std::max(tgt, (double)(2 * S));
    pl.dense_task_cap = P.nblocks * 64;
    // bucket index over g's codes: at most 65536 buckets
    int sh = 0;
    while (((P.g.key_range >> sh) + 1) > 65535) ++sh;
    P.gshift = sh;
    P.gidx_n = (P.g.key_range >> sh) + 1;
    pl.accum_bytes = P.kspan * 8;
    P.chunk = COMPACT_CHUNK;
    P.nchunks = ceil_div(P.kspan, P.chunk);
    pl.out_cap = std::min((double)P.kspan, pairs) > 0 ? (int64_t)std::min((double)P.kspan, pairs) : 0;
  } else {
    const double m = job.poisson ? 2.0 : 1.0;
    const double upper = std::min(m * pairs, (double)P.kspan);
    const double alpha = o.load_factor > 0.0 && o.load_factor <= 0.9 ? o.load_factor : DEFAULT_LOAD;
    pl.bound_slots = next_pow2(std::max<int64_t>(1024, (int64_t)std::ceil(upper / alpha)));
    P.probe_limit = o.probe_limit > 0 ? o.probe_limit : DEFAULT_PROBES;
    P.tile_i = HASH_TILE_I;
    P.tile_j = HASH_TILE_J;
    P.tiles_j = ceil_div(ng, HASH_TILE_J);
    P.ntasks = ceil_div(nf, HASH_TILE_I) * P.tiles_j;
    P.chunk = COMPACT_CHUNK_HASH;
    // table size, chunks and output capacity follow in finish_hash_sizes
  }
}

void finish_hash_sizes(const kr_opts& o, Plan* pl) {
  Prod& P = pl->p;
  const double m = P.nt > 0 ? 2.0 : 1.0;
  const double upper = std::min(m * (double)P.f.n * (double)P.g.n, (double)P.kspan);
  const double alpha = o.load_factor > 0.0 && o.load_factor <= 0.9 ? o.load_factor : DEFAULT_LOAD;
  int64_t slots;
  if (pl->slots_override > 0) {
    slots = pl->slots_override;
  } else if (o.table_slots > 0) {
    slots = next_pow2(o.table_slots);
  } else {
    const double est = P.hll_est > 0.0 ? std::min(P.hll_est * 1.05, upper) : upper;
    slots = next_pow2(std::max<int64_t>(1024, (int64_t)std::ceil(est / alpha)));
  }
  P.slots = slots;
  P.nchunks = ceil_div(slots, P.chunk);
  pl->accum_bytes = slots * 16;
  double cap = std::min((double)slots, upper);
  // output room from the estimate (+10%, about six standard errors of the
  // 4096-register HyperLogLog); the compaction flags an overflow and the
  // product is rerun with room for a full table
  if (P.hll_est > 0.0 && !pl->outcap_full) cap = std::min(cap, P.hll_est * 1.1 + 4096.0);
  pl->out_cap = (int64_t)cap;
}

}  // namespace kr
