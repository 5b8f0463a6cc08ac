// Hash (highly sparse) path, Sec. 3.2: the schoolbook loop accumulates
// coefficient-code pairs into a hash table keyed by the code.
//
// GB300 design.  The paper's bucketed, cache-line table with an overflow
// bucket and mod-N term ordering is prior art for a cache hierarchy; here the
// table is one open-addressing array in device memory shared by the whole
// grid.  A slot is 16 bytes: (key + 1, value), key 0 meaning empty.  A thread
// claims an empty slot with a 64-bit atomicCAS on the key word and then adds
// its coefficient with an atomic add on the value word (int64 wraps, so the
// integer result does not depend on the order of the adds).  Collisions are
// resolved by linear probing (the alternative the paper names in Sec. 3.2)
// with a bounded probe count; a product that reaches the bound raises
// TABLE_FULL and the host grows the table and multiplies again (the paper's
// resize-and-rehash on a failed insert).  The home slot comes from a 64-bit
// mixing function of the key, not from key mod N, because warps insert many
// keys at once and structured codes would otherwise pile onto neighbouring
// slots.
//
// Poisson series (Sec. 2, Eq. 6 with the factor 1/2): each pair of terms
// gives one insert at the sum and one at the difference of the trig codes;
// the result kind is cos when the factors have the same kind and sin
// otherwise; the sign is - for the sum of sin*sin and for the difference of
// cos*sin.  A negative trig code is folded to its absolute value (cos is even,
// sin is odd) and a sine at code 0 is dropped.
#include "kr_internal.cuh"

namespace kr {

constexpr int HASH_THREADS = 256;
#ifndef KR_HGROUP_R
#define KR_HGROUP_R 2
#endif
constexpr int HGROUP_R = KR_HGROUP_R;   // f terms per warp step, polynomial tiles
constexpr int PGROUP_R = 2;   // f terms per warp step, Poisson tiles (two keys each)

template <typename T>
__device__ __forceinline__ void gatomic_add(T* p, T v);
template <>
__device__ __forceinline__ void gatomic_add<int64_t>(int64_t* p, int64_t v) {
  atomicAdd((unsigned long long*)p, (unsigned long long)v);
}
template <>
__device__ __forceinline__ void gatomic_add<double>(double* p, double v) {
  atomicAdd(p, v);
}

// Insert-or-add; false when probe_limit slots were all taken by other keys.
template <typename T>
__device__ __forceinline__ bool hash_add(uint64_t* __restrict__ table, uint64_t mask, int limit,
                                         uint64_t key, T val) {
  const unsigned long long stored = key + 1ull;
  uint64_t slot = mix64(key) & mask;
  for (int p = 0; p < limit; ++p) {
    unsigned long long* e = (unsigned long long*)(table + 2 * slot);
    unsigned long long k = __ldcg(e);
    if (k == 0ull) {
      k = atomicCAS(e, 0ull, stored);
      if (k == 0ull) k = stored;
    }
    if (k == stored) {
      gatomic_add<T>((T*)(e + 1), val);
      return true;
    }
    slot = (slot + 1) & mask;
  }
  return false;
}

// R independent insert-or-adds issued together so that their L2 round trips
// overlap.  Each probe claims the slot with a CAS whatever its state: an
// empty slot is taken in one round trip, a slot holding the same key is
// recognised by the value the CAS returns, any other key moves the probe on.
// The adds are fire-and-forget reductions.  Returns false if some key found
// no slot within `limit` probes.
template <int R, typename T>
struct KeyBatch {
  uint64_t key[R];
  T val[R];
};

template <int R, typename T>
__device__ __forceinline__ bool hash_add_batch(uint64_t* __restrict__ table, uint64_t mask, int limit,
                                               KeyBatch<R, T> kb, unsigned valid) {
  uint64_t slot[R];
#pragma unroll
  for (int r = 0; r < R; ++r) slot[r] = mix64(kb.key[r]) & mask;
  unsigned pend = valid;
  for (int p = 0; p < limit && pend; ++p) {
    unsigned long long got[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      got[r] = 0ull;
      if (pend & (1u << r))
        got[r] = atomicCAS((unsigned long long*)(table + 2 * slot[r]), 0ull, kb.key[r] + 1ull);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (pend & (1u << r)) {
        if (got[r] == 0ull || got[r] == kb.key[r] + 1ull) {
          gatomic_add<T>((T*)(table + 2 * slot[r] + 1), kb.val[r]);
          pend &= ~(1u << r);
        } else {
          slot[r] = (slot[r] + 1) & mask;
        }
      }
    }
  }
  return pend == 0;
}

// Whether an output key lies in the product's key window.
__device__ __forceinline__ bool in_window(const Prod& P, uint64_t key) {
  return !P.clip || key - (uint64_t)P.klo < (uint64_t)P.kspan;
}

struct HashTile {
  int pid;
  int64_t i0, i1, j0, j1;
};

__device__ __forceinline__ HashTile find_tile(const Prod* prods, const int32_t* hash_prods,
                                              const int64_t* task_begin, int nhash, int64_t t) {
  int lo = 0, hi = nhash - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (task_begin[mid] <= t) lo = mid; else hi = mid - 1;
  }
  HashTile h;
  h.pid = hash_prods[lo];
  const Prod& P = prods[h.pid];
  const int64_t local = t - task_begin[lo];
  const int64_t ti = local / P.tiles_j, tj = local - ti * P.tiles_j;
  // terms dropped by truncation sort after the kept ones: tiles stop there
  h.i0 = ti * P.tile_i;
  h.i1 = min(P.f.nkeep, h.i0 + P.tile_i);
  h.j0 = tj * P.tile_j;
  h.j1 = min(P.g.nkeep, h.j0 + P.tile_j);
  return h;
}

// CT: a coefficient bound (float64 only): both operands are in order of
// decreasing |C|, so the largest product of a tile, of a group's rows and of
// a warp step are their first pairs; whatever starts below the bound is
// skipped whole.
template <typename T, bool CT>
__device__ __forceinline__ bool poly_tile(const Prod& P, const HashTile& h) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = HASH_THREADS / 32;
  const int64_t* __restrict__ F = P.f.code;
  const int64_t* __restrict__ G = P.g.code;
  const T* __restrict__ CF = (const T*)P.f.coef;
  const T* __restrict__ CG = (const T*)P.g.coef;
  const uint64_t mask = (uint64_t)P.slots - 1;
  bool ok = true;
  if (CT && (h.i0 >= h.i1 || h.j0 >= h.j1 || !coef_kept(P, (double)CF[h.i0] * (double)CG[h.j0]))) return true;
  const int64_t ngroups = (h.i1 - h.i0 + HGROUP_R - 1) / HGROUP_R;
  for (int64_t grp = warp; grp < ngroups; grp += NW) {
    const int64_t ia = h.i0 + grp * HGROUP_R;
    const int m = (int)min((int64_t)HGROUP_R, h.i1 - ia);
    int64_t fr[HGROUP_R];
    T cr[HGROUP_R];
#pragma unroll
    for (int r = 0; r < HGROUP_R; ++r) {
      const int64_t i = ia + (r < m ? r : 0);
      fr[r] = F[i];
      cr[r] = CF[i];
    }
    const unsigned valid = (1u << m) - 1u;
    if (CT) {
      // this group's first row is its largest, later groups of the warp smaller
      if (!coef_kept(P, (double)cr[0] * (double)CG[h.j0])) break;
      // magnitude order: the window and the degree bound are masked per pair
      for (int64_t jb = h.j0; jb < h.j1; jb += 32) {
        const int64_t j = jb + lane;
        KeyBatch<HGROUP_R, T> kb;
        unsigned v = 0, big = 0;
        if (j < h.j1) {
          const int64_t gj = G[j];
          const T cg = CG[j];
#pragma unroll
          for (int r = 0; r < HGROUP_R; ++r) {
            kb.key[r] = (uint64_t)(fr[r] + gj);
            kb.val[r] = cr[r] * cg;
            if (coef_kept(P, (double)kb.val[r])) big |= 1u << r;
          }
          big &= valid;
          v = big;
#pragma unroll
          for (int r = 0; r < HGROUP_R; ++r)
            if (P.clip && (uint64_t)(fr[r] + gj - P.klo) >= (uint64_t)P.kspan) v &= ~(1u << r);
        }
        // every later step of g is smaller: once no pair of the step passes, stop
        if (!__any_sync(0xffffffffu, big != 0)) break;
        ok &= hash_add_batch<HGROUP_R, T>(P.table, mask, P.probe_limit, kb, v);
      }
      continue;
    }
    // a key window (or a truncation: codes at or above krange exceed the
    // degree bound) keeps the keys in [klo, klo + kspan).  F is ascending, so
    // the group's first term has the longest j-range below the window's end
    // and its last term the earliest start; the rest is masked per pair.
    int64_t jbeg = h.j0, jend = h.j1;
    if (P.clip) {
      int64_t flast = fr[0];
#pragma unroll
      for (int r = 1; r < HGROUP_R; ++r)
        if (r < m) flast = fr[r];
      jend = min(jend, lower_bound_i64(G, P.g.nkeep, P.klo + P.kspan - fr[0]));
      jbeg = max(jbeg, lower_bound_i64(G, P.g.nkeep, P.klo - flast));
    }
    for (int64_t j = jbeg + lane; j < jend; j += 32) {
      const int64_t gj = G[j];
      const T cg = CG[j];
      KeyBatch<HGROUP_R, T> kb;
      unsigned v = valid;
#pragma unroll
      for (int r = 0; r < HGROUP_R; ++r) {
        kb.key[r] = (uint64_t)(fr[r] + gj);
        kb.val[r] = cr[r] * cg;
        if (P.clip && (uint64_t)(fr[r] + gj - P.klo) >= (uint64_t)P.kspan) v &= ~(1u << r);
      }
      ok &= hash_add_batch<HGROUP_R, T>(P.table, mask, P.probe_limit, kb, v);
    }
  }
  return ok;
}

// The two keys (sum, difference) and values of the Poisson pair (f row r, g
// term j), with the bits of the ones to insert.  big: the pair passes the
// coefficient bound (CT), whatever the other tests say.
template <bool CT, bool HT>
__device__ __forceinline__ void pseries_pair(const Prod& P, int64_t T2Wp, int64_t i, int64_t pf, int64_t tf,
                                             int kf, double cf, int64_t j, int64_t pg, int64_t tg, int kg,
                                             double cg, uint64_t* keys, double* vals, unsigned* valid,
                                             bool* big) {
  const int64_t pc = pf + pg;
  // truncation by degree: the polynomial part's degree digit is the top one
  bool keep = !(P.graded && pc >= P.Wp);
  const double hcoef = cf * cg;   // (C_f / 2) * C_g
  *big = true;
  if (CT) {
    *big = coef_kept(P, hcoef);
    keep &= *big;
  }
  uint32_t od = 0, os = 0;
  if (HT) harmonic_orders(P, i, j, &od, &os);
  const int kd = kf ^ kg;   // cos if same kinds, sin otherwise
  // sum term
  int64_t T = tf + tg;
  double v = (kf & kg) ? -hcoef : hcoef;   // sin*sin: -cos(a+b)
  if (T < 0) { T = -T; if (kd) v = -v; }
  keys[0] = (uint64_t)(kd * T2Wp + T * P.Wp + pc);
  vals[0] = v;
  unsigned bits = 0;
  if (keep && !(T == 0 && kd) && in_window(P, keys[0]) && (!HT || os <= (uint64_t)P.hN)) bits |= 1u;
  // difference term
  T = tf - tg;
  v = (!kf && kg) ? -hcoef : hcoef;   // cos*sin: -sin(a-b)
  if (T < 0) { T = -T; if (kd) v = -v; }
  keys[1] = (uint64_t)(kd * T2Wp + T * P.Wp + pc);
  vals[1] = v;
  if (keep && !(T == 0 && kd) && in_window(P, keys[1]) && (!HT || od <= (uint64_t)P.hN)) bits |= 2u;
  *valid = bits;
}

// CT: a coefficient bound (operands in order of decreasing |C|: the first
// pair of a tile, of a row and of a warp step is its largest); HT: a
// harmonic-order bound.
template <bool CT, bool HT>
__device__ __forceinline__ bool pseries_tile(const Prod& P, const HashTile& h) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = HASH_THREADS / 32;
  const int64_t* __restrict__ PF = P.f.code;
  const int64_t* __restrict__ PG = P.g.code;
  const int64_t* __restrict__ TF = P.f.tcode;
  const int64_t* __restrict__ TG = P.g.tcode;
  const uint8_t* __restrict__ KF = P.f.kind;
  const uint8_t* __restrict__ KG = P.g.kind;
  const double* __restrict__ CF = (const double*)P.f.coef;   // already halved
  const double* __restrict__ CG = (const double*)P.g.coef;
  const uint64_t mask = (uint64_t)P.slots - 1;
  const int64_t T2Wp = P.T2 * P.Wp;
  bool ok = true;
  if (CT && (h.i0 >= h.i1 || h.j0 >= h.j1 || !coef_kept(P, CF[h.i0] * CG[h.j0]))) return true;
  const int64_t ngroups = (h.i1 - h.i0 + PGROUP_R - 1) / PGROUP_R;
  for (int64_t grp = warp; grp < ngroups; grp += NW) {
    const int64_t ia = h.i0 + grp * PGROUP_R;
    const int m = (int)min((int64_t)PGROUP_R, h.i1 - ia);
    int64_t pr[PGROUP_R], tr[PGROUP_R], ir[PGROUP_R];
    double cr[PGROUP_R];
    int kr_[PGROUP_R];
#pragma unroll
    for (int r = 0; r < PGROUP_R; ++r) {
      const int64_t i = ia + (r < m ? r : 0);
      ir[r] = i;
      pr[r] = PF[i];
      tr[r] = TF[i];
      cr[r] = CF[i];
      kr_[r] = KF[i];
    }
    if (CT && !coef_kept(P, cr[0] * CG[h.j0])) break;   // this and every later group of the warp
    // CT: warp steps in lockstep, so that the warp can stop together
    for (int64_t jb = h.j0; jb < h.j1; jb += 32) {
      const int64_t j = jb + lane;
      if (!CT && j >= h.j1) break;
      // two f terms at a time: four keys (a sum and a difference each) in flight
      KeyBatch<4, double> kb;
      unsigned valid = 0;
      bool any_big = false;
      if (j < h.j1) {
        const int64_t pg = PG[j], tg = TG[j];
        const int kg = KG[j];
        const double cg = CG[j];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          unsigned bits;
          bool big;
          pseries_pair<CT, HT>(P, T2Wp, ir[u], pr[u], tr[u], kr_[u], cr[u], j, pg, tg, kg, cg,
                               &kb.key[2 * u], &kb.val[2 * u], &bits, &big);
          if (u < m) {
            valid |= bits << (2 * u);
            any_big |= big;
          }
        }
      }
      if (CT && !__any_sync(0xffffffffu, any_big)) break;   // every later step of g is smaller
      ok &= hash_add_batch<4, double>(P.table, mask, P.probe_limit, kb, valid);
    }
  }
  return ok;
}

// Poisson series on the dense path (Sec. 3.1): both terms of a pair add into
// the array indexed by their key, with fire-and-forget float64 reductions.
template <bool CT, bool HT>
__device__ __forceinline__ void pseries_dense_tile(const Prod& P, const HashTile& h) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = HASH_THREADS / 32;
  const int64_t* __restrict__ PF = P.f.code;
  const int64_t* __restrict__ PG = P.g.code;
  const int64_t* __restrict__ TF = P.f.tcode;
  const int64_t* __restrict__ TG = P.g.tcode;
  const uint8_t* __restrict__ KF = P.f.kind;
  const uint8_t* __restrict__ KG = P.g.kind;
  const double* __restrict__ CF = (const double*)P.f.coef;   // already halved
  const double* __restrict__ CG = (const double*)P.g.coef;
  double* __restrict__ out = (double*)P.dense;   // slot = key - klo
  const int64_t T2Wp = P.T2 * P.Wp;
  const uint64_t K = (uint64_t)P.kspan, K0 = (uint64_t)P.klo;
  if (CT && (h.i0 >= h.i1 || h.j0 >= h.j1 || !coef_kept(P, CF[h.i0] * CG[h.j0]))) return;
  for (int64_t i = h.i0 + warp; i < h.i1; i += NW) {
    const int64_t pf = PF[i], tf = TF[i];
    const int kf = KF[i];
    const double cf = CF[i];
    if (CT && !coef_kept(P, cf * CG[h.j0])) break;   // this and every later row of the warp
    if (!CT && !HT) {
      for (int64_t j = h.j0 + lane; j < h.j1; j += 32) {
        const int64_t pc = pf + PG[j];
        if (P.graded && pc >= P.Wp) continue;   // above the degree bound
        const int64_t tg = TG[j];
        const int kg = KG[j];
        const double hcoef = cf * CG[j];
        const int kd = kf ^ kg;
        int64_t T = tf + tg;
        double v = (kf & kg) ? -hcoef : hcoef;
        if (T < 0) { T = -T; if (kd) v = -v; }
        if (!(T == 0 && kd)) {
          const uint64_t key = (uint64_t)(kd * T2Wp + T * P.Wp + pc) - K0;
          if (key < K) atomicAdd(&out[key], v);
        }
        T = tf - tg;
        v = (!kf && kg) ? -hcoef : hcoef;
        if (T < 0) { T = -T; if (kd) v = -v; }
        if (!(T == 0 && kd)) {
          const uint64_t key = (uint64_t)(kd * T2Wp + T * P.Wp + pc) - K0;
          if (key < K) atomicAdd(&out[key], v);
        }
      }
      continue;
    }
    for (int64_t jb = h.j0; jb < h.j1; jb += 32) {
      const int64_t j = jb + lane;
      if (!CT && j >= h.j1) break;
      bool big = false;
      if (j < h.j1) {
        uint64_t keys[2];
        double vals[2];
        unsigned bits;
        pseries_pair<CT, HT>(P, T2Wp, i, pf, tf, kf, cf, j, PG[j], TG[j], KG[j], CG[j], keys, vals, &bits,
                             &big);
        // the window test of pseries_pair is the slot test below
        if ((bits & 1u) && keys[0] - K0 < K) atomicAdd(&out[keys[0] - K0], vals[0]);
        if ((bits & 2u) && keys[1] - K0 < K) atomicAdd(&out[keys[1] - K0], vals[1]);
      }
      if (CT && !__any_sync(0xffffffffu, big)) break;   // every later step of g is smaller
    }
  }
}

// ---------------------------------------------------------------------------
// HyperLogLog pass: same tiles and keys as the inserts, no table traffic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void hll_add(uint32_t* reg, uint64_t key) {
  const uint64_t h = mix64(key);
  const uint32_t idx = (uint32_t)(h >> (64 - HLL_B));
  const uint64_t w = h << HLL_B;
  const uint32_t rho = w == 0 ? (uint32_t)(64 - HLL_B + 1) : (uint32_t)__clzll((long long)w) + 1;
  if (reg[idx] < rho) atomicMax(&reg[idx], rho);
}

// Keys (at most two) of pair (i, j) of a product truncated by coefficient
// magnitude or harmonic order, as the tiles form them: bits says which to
// count, big whether the pair passes the coefficient bound.
__device__ __forceinline__ void trunc_pair_keys(const Prod& P, int64_t i, int64_t j, uint64_t* keys,
                                                unsigned* bits, bool* big) {
  const double* CF = (const double*)P.f.coef;
  const double* CG = (const double*)P.g.coef;
  if (P.nt == 0) {
    *big = !P.ctrunc || coef_kept(P, CF[i] * CG[j]);
    keys[0] = (uint64_t)(P.f.code[i] + P.g.code[j]);
    *bits = (*big && in_window(P, keys[0])) ? 1u : 0u;
    return;
  }
  double vals[2];
  const int64_t T2Wp = P.T2 * P.Wp;
  const int64_t pf = P.f.code[i], tf = P.f.tcode[i], pg = P.g.code[j], tg = P.g.tcode[j];
  const int kf = P.f.kind[i], kg = P.g.kind[j];
  if (P.htrunc && P.ctrunc)
    pseries_pair<true, true>(P, T2Wp, i, pf, tf, kf, CF[i], j, pg, tg, kg, CG[j], keys, vals, bits, big);
  else if (P.htrunc)
    pseries_pair<false, true>(P, T2Wp, i, pf, tf, kf, CF[i], j, pg, tg, kg, CG[j], keys, vals, bits, big);
  else
    pseries_pair<true, false>(P, T2Wp, i, pf, tf, kf, CF[i], j, pg, tg, kg, CG[j], keys, vals, bits, big);
}

// The HyperLogLog pass of a truncated product: only the keys the inserts
// will make, with the same early stops under a coefficient bound.
__device__ __forceinline__ void hll_tile_trunc(const Prod& P, const HashTile& h, uint32_t* reg) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = HASH_THREADS / 32;
  const double* CF = (const double*)P.f.coef;
  const double* CG = (const double*)P.g.coef;
  if (P.ctrunc && (h.i0 >= h.i1 || h.j0 >= h.j1 || !coef_kept(P, CF[h.i0] * CG[h.j0]))) return;
  for (int64_t i = h.i0 + warp; i < h.i1; i += NW) {
    if (P.ctrunc && !coef_kept(P, CF[i] * CG[h.j0])) break;
    for (int64_t jb = h.j0; jb < h.j1; jb += 32) {
      const int64_t j = jb + lane;
      bool big = false;
      if (j < h.j1) {
        uint64_t keys[2];
        unsigned bits;
        trunc_pair_keys(P, i, j, keys, &bits, &big);
        if (bits & 1u) hll_add(reg, keys[0]);
        if (bits & 2u) hll_add(reg, keys[1]);
      }
      if (P.ctrunc && !__any_sync(0xffffffffu, big)) break;
    }
  }
}

__device__ __forceinline__ void hll_tile(const Prod& P, const HashTile& h, uint32_t* reg) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = HASH_THREADS / 32;
  if (P.ctrunc || P.htrunc) {
    hll_tile_trunc(P, h, reg);
    return;
  }
  const int64_t* __restrict__ F = P.f.code;
  const int64_t* __restrict__ G = P.g.code;
  const int64_t* __restrict__ TF = P.f.tcode;
  const int64_t* __restrict__ TG = P.g.tcode;
  const uint8_t* __restrict__ KF = P.f.kind;
  const uint8_t* __restrict__ KG = P.g.kind;
  const int64_t T2Wp = P.T2 * P.Wp;
  for (int64_t i = h.i0 + warp; i < h.i1; i += NW) {
    const int64_t fi = F[i];
    if (P.nt == 0) {
      for (int64_t j = h.j0 + lane; j < h.j1; j += 32) {
        const int64_t key = fi + G[j];
        if (in_window(P, (uint64_t)key)) hll_add(reg, (uint64_t)key);
      }
    } else {
      const int64_t ti = TF[i];
      const int ki = KF[i];
      for (int64_t j = h.j0 + lane; j < h.j1; j += 32) {
        const int64_t pc = fi + G[j];
        if (P.graded && pc >= P.Wp) continue;
        const int kd = ki ^ KG[j];
        int64_t T = ti + TG[j];
        if (T < 0) T = -T;
        uint64_t key = (uint64_t)(kd * T2Wp + T * P.Wp + pc);
        if (!(T == 0 && kd) && in_window(P, key)) hll_add(reg, key);
        T = ti - TG[j];
        if (T < 0) T = -T;
        key = (uint64_t)(kd * T2Wp + T * P.Wp + pc);
        if (!(T == 0 && kd) && in_window(P, key)) hll_add(reg, key);
      }
    }
  }
}

__global__ void __launch_bounds__(HASH_THREADS) k_hll(Prod* __restrict__ prods,
                                                      const int32_t* __restrict__ hash_prods,
                                                      const int64_t* __restrict__ task_begin, int nhash) {
  __shared__ uint32_t reg[HLL_M];
  const int64_t ntasks = task_begin[nhash];
  int cur = -1;
  for (int64_t t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const HashTile h = find_tile(prods, hash_prods, task_begin, nhash, t);
    if (h.pid != cur) {
      // flush the registers of the previous product, start the next
      __syncthreads();
      if (cur >= 0)
        for (int r = threadIdx.x; r < HLL_M; r += blockDim.x)
          if (reg[r]) atomicMax(&prods[cur].hll[r], reg[r]);
      for (int r = threadIdx.x; r < HLL_M; r += blockDim.x) reg[r] = 0;
      __syncthreads();
      cur = h.pid;
    }
    if (prods[h.pid].status == 0) hll_tile(prods[h.pid], h, reg);
  }
  __syncthreads();
  if (cur >= 0)
    for (int r = threadIdx.x; r < HLL_M; r += blockDim.x)
      if (reg[r]) atomicMax(&prods[cur].hll[r], reg[r]);
}

// ---------------------------------------------------------------------------
// Work histogram for splitting a product into key windows: uniformly drawn
// term pairs, their output keys (as the tiles form them), counted per slice
// of the key range.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_count(unsigned long long* hist, int nbins, int64_t krange,
                                            int64_t key) {
  if (key < 0 || key >= krange) return;
  int64_t b = (int64_t)(((unsigned __int128)key * (unsigned)nbins) / (unsigned __int128)krange);
  if (b >= nbins) b = nbins - 1;
  atomicAdd(&hist[b], 1ull);
}

__global__ void __launch_bounds__(256) k_split_sample(const Prod* __restrict__ prods, int prod, int nbins,
                                                      int64_t nsamples, uint64_t seed,
                                                      unsigned long long* __restrict__ hist) {
  const Prod& P = prods[prod];
  if (P.status) return;
  const int64_t nf = P.f.nkeep, ng = P.g.nkeep;
  if (nf <= 0 || ng <= 0) return;
  const int64_t T2Wp = P.T2 * P.Wp;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nsamples;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (int64_t)(mix64(seed ^ (2ull * (uint64_t)u + 1ull)) % (uint64_t)nf);
    const int64_t j = (int64_t)(mix64(seed ^ (2ull * (uint64_t)u + 2ull) ^ 0x9e3779b97f4a7c15ull) % (uint64_t)ng);
    if (P.ctrunc || P.htrunc) {
      uint64_t keys[2];
      unsigned bits;
      bool big;
      trunc_pair_keys(P, i, j, keys, &bits, &big);
      if (bits & 1u) split_count(hist, nbins, P.krange, (int64_t)keys[0]);
      if (bits & 2u) split_count(hist, nbins, P.krange, (int64_t)keys[1]);
      continue;
    }
    const int64_t pc = P.f.code[i] + P.g.code[j];
    if (P.nt == 0) {
      split_count(hist, nbins, P.krange, pc);   // truncated-away keys lie at or above krange
      continue;
    }
    if (P.graded && pc >= P.Wp) continue;
    const int kd = P.f.kind[i] ^ P.g.kind[j];
    int64_t T = P.f.tcode[i] + P.g.tcode[j];
    if (T < 0) T = -T;
    if (!(T == 0 && kd)) split_count(hist, nbins, P.krange, kd * T2Wp + T * P.Wp + pc);
    T = P.f.tcode[i] - P.g.tcode[j];
    if (T < 0) T = -T;
    if (!(T == 0 && kd)) split_count(hist, nbins, P.krange, kd * T2Wp + T * P.Wp + pc);
  }
}

cudaError_t launch_split_sample(const Prod* dprods, int prod, int nbins, int64_t nsamples, uint64_t seed,
                                unsigned long long* dhist, cudaStream_t s) {
  if (nsamples > 0) {
    int64_t grid = (nsamples + 255) / 256;
    if (grid > 152 * 8) grid = 152 * 8;
    k_split_sample<<<(unsigned)grid, 256, 0, s>>>(dprods, prod, nbins, nsamples, seed, dhist);
  }
  return cudaGetLastError();
}

// One CTA per hash product: E = alpha_m m^2 / sum 2^-M_j, with linear counting
// m ln(m / V) when E <= 5m/2 and V registers are zero.
__global__ void __launch_bounds__(256) k_hll_estimate(Prod* __restrict__ prods,
                                                      const int32_t* __restrict__ hash_prods) {
  Prod& P = prods[hash_prods[blockIdx.x]];
  __shared__ double ssum[8];
  __shared__ int szero[8];
  double sum = 0.0;
  int zeros = 0;
  for (int r = threadIdx.x; r < HLL_M; r += blockDim.x) {
    const uint32_t v = P.hll[r];
    sum += ldexp(1.0, -(int)v);
    zeros += v == 0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    zeros += __shfl_xor_sync(0xffffffffu, zeros, o);
  }
  if ((threadIdx.x & 31) == 0) { ssum[threadIdx.x >> 5] = sum; szero[threadIdx.x >> 5] = zeros; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0;
    int V = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { S += ssum[w]; V += szero[w]; }
    const double m = (double)HLL_M;
    const double alpha = 0.7213 / (1.0 + 1.079 / m);
    double E = alpha * m * m / S;
    if (E <= 2.5 * m && V > 0) E = m * log(m / (double)V);
    P.hll_est = E;
  }
}

cudaError_t launch_hll(Prod* dprods, const int32_t* dhash_prods, const int64_t* dtask_begin, int nhash,
                       int grid, cudaStream_t s) {
  if (nhash <= 0) return cudaSuccess;
  k_hll<<<grid, HASH_THREADS, 0, s>>>(dprods, dhash_prods, dtask_begin, nhash);
  return cudaGetLastError();
}

cudaError_t launch_hll_estimate(Prod* dprods, const int32_t* dhash_prods, int nhash, cudaStream_t s) {
  if (nhash <= 0) return cudaSuccess;
  k_hll_estimate<<<nhash, 256, 0, s>>>(dprods, dhash_prods);
  return cudaGetLastError();
}

// Two kernels over the same task list, each skipping the other kind's
// products: polynomial tiles need fewer registers than the Poisson tiles, so
// their kernel keeps more warps, and thus more inserts, in flight per SM.
#ifndef KR_HASH_POLY_MIN_BLOCKS
#define KR_HASH_POLY_MIN_BLOCKS 4
#endif

__global__ void __launch_bounds__(HASH_THREADS, KR_HASH_POLY_MIN_BLOCKS)
    k_hash_insert_poly(Prod* __restrict__ prods, const int32_t* __restrict__ hash_prods,
                       const int64_t* __restrict__ task_begin, int nhash) {
  const int64_t ntasks = task_begin[nhash];
  for (int64_t t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const HashTile h = find_tile(prods, hash_prods, task_begin, nhash, t);
    Prod& P = prods[h.pid];
    if (P.nt > 0) continue;
    if (*(volatile uint32_t*)&P.status) continue;   // failed product: skip its remaining tiles
    if (P.ctrunc) continue;   // k_hash_insert_trunc
    const bool ok = P.f64 ? poly_tile<double, false>(P, h) : poly_tile<int64_t, false>(P, h);
    if (!ok) atomicOr(&P.status, ST_TABLE_FULL);
  }
}

__global__ void __launch_bounds__(HASH_THREADS, 3) k_hash_insert_pseries(Prod* __restrict__ prods,
                                                                      const int32_t* __restrict__ hash_prods,
                                                                      const int64_t* __restrict__ task_begin,
                                                                      int nhash) {
  const int64_t ntasks = task_begin[nhash];
  for (int64_t t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const HashTile h = find_tile(prods, hash_prods, task_begin, nhash, t);
    Prod& P = prods[h.pid];
    if (P.nt == 0) continue;
    if (*(volatile uint32_t*)&P.status) continue;
    if (P.ctrunc || P.htrunc) continue;   // k_hash_insert_trunc
    bool ok = true;
    if (P.path == PATH_DENSE) pseries_dense_tile<false, false>(P, h);
    else ok = pseries_tile<false, false>(P, h);
    if (!ok) atomicOr(&P.status, ST_TABLE_FULL);
  }
}

// Products truncated by coefficient magnitude or harmonic order, in a kernel
// of their own so that the tests and early stops cost the plain kernels no
// registers.
__global__ void __launch_bounds__(HASH_THREADS, 2) k_hash_insert_trunc(Prod* __restrict__ prods,
                                                                    const int32_t* __restrict__ hash_prods,
                                                                    const int64_t* __restrict__ task_begin,
                                                                    int nhash) {
  const int64_t ntasks = task_begin[nhash];
  for (int64_t t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const HashTile h = find_tile(prods, hash_prods, task_begin, nhash, t);
    Prod& P = prods[h.pid];
    if (!P.ctrunc && !P.htrunc) continue;
    if (*(volatile uint32_t*)&P.status) continue;
    bool ok = true;
    if (P.nt == 0) {
      ok = poly_tile<double, true>(P, h);   // a coefficient bound (float64 only)
    } else {
      const int v = (P.ctrunc ? 1 : 0) | (P.htrunc ? 2 : 0);
      if (P.path == PATH_DENSE) {
        if (v == 1) pseries_dense_tile<true, false>(P, h);
        else if (v == 2) pseries_dense_tile<false, true>(P, h);
        else pseries_dense_tile<true, true>(P, h);
      } else {
        if (v == 1) ok = pseries_tile<true, false>(P, h);
        else if (v == 2) ok = pseries_tile<false, true>(P, h);
        else ok = pseries_tile<true, true>(P, h);
      }
    }
    if (!ok) atomicOr(&P.status, ST_TABLE_FULL);
  }
}

// Ceiling probe of the hash path: `updates` insert-or-adds of keys drawn from
// `distinct` values (a counter-based hash of the update index, so the keys
// arrive in random order), into the table as the polynomial kernel updates
// it: the same batches of HGROUP_R independent probes per lane, the same CAS
// claim and fire-and-forget add, but no term pairs to form.  mode 1 replaces
// the insert by a plain atomic add into each key's home slot (no CAS: the
// random read-modify-write alone).
__global__ void __launch_bounds__(HASH_THREADS, KR_HASH_POLY_MIN_BLOCKS)
    k_probe_table_update(uint64_t* __restrict__ table, uint64_t mask, int64_t distinct, int64_t updates,
                         uint64_t seed, int mode, unsigned long long* __restrict__ fails) {
  bool ok = true;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * HGROUP_R;
  for (int64_t u0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * HGROUP_R; u0 < updates; u0 += stride) {
    KeyBatch<HGROUP_R, int64_t> kb;
    unsigned v = 0;
#pragma unroll
    for (int r = 0; r < HGROUP_R; ++r) {
      const int64_t u = u0 + r;
      kb.key[r] = mix64(seed ^ (uint64_t)(u + 1)) % (uint64_t)distinct;
      kb.val[r] = 1;
      if (u < updates) v |= 1u << r;
    }
    if (mode == 0) {
      ok &= hash_add_batch<HGROUP_R, int64_t>(table, mask, 512, kb, v);
    } else {
#pragma unroll
      for (int r = 0; r < HGROUP_R; ++r)
        if (v & (1u << r)) gatomic_add<int64_t>((int64_t*)(table + 2 * (mix64(kb.key[r]) & mask) + 1), 1);
    }
  }
  if (!ok) atomicAdd(fails, 1ull);
}

cudaError_t launch_probe_table_update(uint64_t* table, uint64_t slots, int64_t distinct, int64_t updates,
                                      int mode, unsigned long long* fails, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_table_update, HASH_THREADS, 0);
  if (per_sm < 1) per_sm = 1;
  k_probe_table_update<<<sms * per_sm, HASH_THREADS, 0, s>>>(table, slots - 1, distinct, updates,
                                                            0x5eed5eedull, mode, fails);
  return cudaGetLastError();
}

cudaError_t launch_hash_insert(Prod* dprods, const int32_t* dhash_prods, const int64_t* dtask_begin,
                               int nhash, bool poly, bool pseries, bool trunc, int grid, cudaStream_t s) {
  if (nhash <= 0) return cudaSuccess;
  if (poly) k_hash_insert_poly<<<grid, HASH_THREADS, 0, s>>>(dprods, dhash_prods, dtask_begin, nhash);
  if (pseries) k_hash_insert_pseries<<<grid, HASH_THREADS, 0, s>>>(dprods, dhash_prods, dtask_begin, nhash);
  if (trunc) k_hash_insert_trunc<<<grid, HASH_THREADS, 0, s>>>(dprods, dhash_prods, dtask_begin, nhash);
  return cudaGetLastError();
}

}  // namespace kr
