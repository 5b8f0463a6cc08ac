// Oracle: a plain, slow CPU multiplier of sparse Laurent polynomials and
// Poisson series.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
// benchmark's CPU-baseline leg use it; the library never links or calls it.
//
// It follows the definition of the product, not the fast method:
//  * polynomials (Sec. 1, Eq. 1 with no trig part; Sec. 3.1): every term of f
//    times every term of g, exponent vectors added component-wise, coefficients
//    multiplied, equal exponent vectors accumulated;
//  * Poisson series (Sec. 1, Eq. 1; Sec. 2, Eq. 6, the product-to-sum formulas):
//    every pair of terms gives two terms with the polynomial exponents added
//    and the trig multiplier vectors added and subtracted.  Eq. 6 is printed
//    without the factor 1/2 of the trigonometric identities; the oracle uses
//    the identities (cos a cos b = 1/2 cos(a-b) + 1/2 cos(a+b), and so on).
//
// It never forms a Kronecker code.  Terms live in a std::map keyed by the
// explicit exponent vector.  The map order is the one the library's output
// uses: polynomial vectors compare from the highest-index variable down
// (reverse lexicographic, variable 0 least significant, as in Table 1 and
// Table 2); Poisson keys compare by kind (cos < sin), then trig multipliers
// from the highest index down, then polynomial exponents from the highest
// index down.
//
// Trig canonical form (the paper is silent; this is the reading used
// throughout): a multiplier vector is canonical when its highest-index nonzero
// entry is positive.  A non-canonical vector is negated; a sine term then also
// changes sign (sin(-x) = -sin x).  A sine of the zero vector vanishes and is
// dropped; a cosine of the zero vector is kept.
//
// int64 coefficients: exact sums in 128 bits, reported modulo 2^64 (the
// library's int64 arithmetic wraps), with a flag when a sum leaves the int64
// range.  float64 coefficients: each contribution is (C*D) for polynomials and
// +-((C*D)*0.5) for Poisson series, summed with Neumaier's compensated
// summation (Neumaier 1974); the sum of |contribution| per key is returned too,
// since the parity tolerance is relative to it.
//
// Truncation (Sec. 3 names truncation by the exponents of one or more
// polynomial variables): with a degree bound N over a set of polynomial
// variables, a pair of terms contributes only when the degree of its product
// term in those variables (the sum of their exponents) is at most N.  The
// oracle forms every pair and skips the ones above the bound.
//
// Parallelism: the f terms are split into contiguous slices, one map per
// thread, maps merged at the end.  An optional shard filter keeps only the
// output keys whose FNV-1a hash is congruent to shard_id modulo shard_mod, so
// a very large product can be checked one slice of its output at a time.
#include <cstdint>
#include <cstring>
#include <map>
#include <thread>
#include <vector>
#include <algorithm>
#include <type_traits>

namespace {

constexpr int MAXK = 17;   // components per key: poly vars, or 1 + trig + poly (at most 16 variables)

struct Key {
  int32_t c[MAXK];
};

struct KeyLess {
  int len;
  int order[MAXK];   // components compared in this order, most significant first
  bool operator()(const Key& a, const Key& b) const {
    for (int t = 0; t < len; ++t) {
      int k = order[t];
      if (a.c[k] != b.c[k]) return a.c[k] < b.c[k];
    }
    return false;
  }
};

struct AccI {
  unsigned __int128 s = 0;   // wrapping 128-bit sum of exact products
};

#ifndef ORC_PLANT
#define ORC_PLANT 0   // 0 = the oracle; k > 0 plants mistake k (mutation tests only)
#endif

struct AccF {
  double s = 0.0, comp = 0.0, mass = 0.0;
  void add(double x) {
    // Neumaier (1974) improved Kahan summation
    double t = s + x;
    if ((s >= 0 ? s : -s) >= (x >= 0 ? x : -x)) comp += (s - t) + x;
    else comp += (x - t) + s;
    s = t;
#if ORC_PLANT == 9
    mass += 2 * (x >= 0 ? x : -x);   // planted: every contribution counted twice in the mass
#else
    mass += (x >= 0 ? x : -x);
#endif
  }
  // adds another thread's partial sum of the same key: its running sum and
  // its compensation are two more contributions; the masses add
  void merge(const AccF& o) {
    double m = mass;
#if ORC_PLANT != 8
    add(o.s);
#endif
    add(o.comp);
#if ORC_PLANT == 10
    mass = m;   // planted: the other thread's mass dropped
#else
    mass = m + o.mass;
#endif
  }
#if ORC_PLANT == 20
  double value() const { return s; }   // planted: the compensation dropped
#else
  double value() const { return s + comp; }
#endif
};

uint64_t fnv1a(const Key& k, int len) {
  uint64_t h = 14695981039346656037ull;
  for (int t = 0; t < len; ++t) {
    h ^= (uint64_t)(uint32_t)k.c[t];
    h *= 1099511628211ull;
  }
  return h;
}

template <class Acc>
using TermMap = std::map<Key, Acc, KeyLess>;

struct Result {
  int np = 0, nt = 0;      // poly vars, trig vars (nt = 0: plain polynomial)
  bool poisson = false, is_f64 = false;
  int overflow = 0;
  std::vector<Key> keys;
  std::vector<int64_t> ci;
  std::vector<double> cf, mass;
};

KeyLess poly_order(int nv) {
  KeyLess L;
  L.len = nv;
#if ORC_PLANT == 15
  for (int t = 0; t < nv; ++t) L.order[t] = t;   // planted: variable 0 most significant
#else
  for (int t = 0; t < nv; ++t) L.order[t] = nv - 1 - t;
#endif
  return L;
}

// Poisson key layout: c[0] = kind, c[1..nt] = trig, c[1+nt..nt+np] = poly
KeyLess poisson_order(int np, int nt) {
  KeyLess L;
  L.len = 1 + nt + np;
  int t = 0;
  L.order[t++] = 0;
#if ORC_PLANT == 17
  for (int k = np - 1; k >= 0; --k) L.order[t++] = 1 + nt + k;   // planted: polynomial part before trig
  for (int k = nt - 1; k >= 0; --k) L.order[t++] = 1 + k;
#else
  for (int k = nt - 1; k >= 0; --k) L.order[t++] = 1 + k;
  for (int k = np - 1; k >= 0; --k) L.order[t++] = 1 + nt + k;
#endif
  return L;
}

bool in_shard(const Key& k, int len, int64_t mod, int64_t id) {
  if (mod <= 1) return true;
  return (int64_t)(fnv1a(k, len) % (uint64_t)mod) == id;
}

template <class F>
void run_threads(int nthreads, int64_t nf, F body) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads == 1 || nf < 2) { body(0, (int64_t)0, nf); return; }
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) {
    int64_t a = nf * t / nthreads, b = nf * (t + 1) / nthreads;
    th.emplace_back([=] { body(t, a, b); });
  }
  for (auto& x : th) x.join();
}

// Truncation (Sec. 3 lists three criteria: the exponents of polynomial
// variables, the order of the Fourier harmonics and the absolute value of the
// coefficients).  A zero flag leaves that criterion off.
//  * degree: a pair contributes only when the degree of its product term in
//    the polynomial variables of mask (the sum of their exponents) is <= N;
//  * harmonic order: a Poisson term is kept only when its harmonic order, the
//    sum of |multiplier| over the trig variables of hmask, is <= hN; it is
//    judged term by term, on each of the two terms a pair emits (the order of
//    a sum or difference of multiplier vectors is not the sum of the orders);
//  * coefficient magnitude: a pair contributes only when |C_f * C_g|, the
//    float64 product of the two coefficients (for Poisson series before the
//    1/2 of the product-to-sum identities), is >= cmin.
struct Trunc {
  int on = 0;
  uint32_t mask = 0;   // bit k: polynomial variable k counts
  int64_t N = 0;
  int hon = 0;
  uint32_t hmask = 0;  // bit k: trig variable k counts
  int64_t hN = 0;
  int con = 0;
  double cmin = 0.0;
};

// The pair (C, D) passes the coefficient bound.
bool coef_kept(const Trunc& T, double C, double D) {
  if (!T.con) return true;
  const double p = C * D;
#if ORC_PLANT == 11
  return (p >= 0 ? p : -p) > T.cmin;   // planted: the bound itself excluded
#endif
  return (p >= 0 ? p : -p) >= T.cmin;
}

// Harmonic order of the trig part key.c[1 .. nt] in the variables of hmask.
bool above_harmonic(const Trunc& T, const Key& key, int nt) {
  if (!T.hon) return false;
  int64_t o = 0;
  for (int k = 0; k < nt; ++k) {
#if ORC_PLANT == 14
    {   // planted: the mask ignored, every trig variable counts
#else
    if ((T.hmask >> k) & 1u) {
#endif
      const int64_t t = key.c[1 + k];
      o += t >= 0 ? t : -t;
    }
  }
#if ORC_PLANT == 13
  return o >= T.hN;   // planted: the bound itself excluded
#endif
  return o > T.hN;
}

// Degree of the polynomial part poly[0..np) in the truncation variables.
bool above_bound(const Trunc& T, const int32_t* poly, int np) {
  if (!T.on) return false;
  int64_t d = 0;
  for (int k = 0; k < np; ++k)
    if ((T.mask >> k) & 1u) d += poly[k];
#if ORC_PLANT == 7
  return d >= T.N;   // planted: the bound itself excluded
#endif
  return d > T.N;
}

// ---------------------------------------------------------------------------
// polynomial product
// ---------------------------------------------------------------------------
template <class Acc, class Coef>
void poly_slice(int nv, const int32_t* ef, const Coef* cf, int64_t nf, int64_t i0, int64_t i1,
                const int32_t* eg, const Coef* cg, int64_t ng, int64_t smod, int64_t sid,
                const Trunc& T, TermMap<Acc>& map) {
  Key key;
  std::memset(&key, 0, sizeof key);
  int64_t jend = ng;
#if ORC_PLANT == 5
  jend = ng - 1;   // planted: drops the last term of g
#endif
  for (int64_t i = i0; i < i1; ++i) {
    for (int64_t j = 0; j < jend; ++j) {
      for (int k = 0; k < nv; ++k) key.c[k] = ef[(int64_t)k * nf + i] + eg[(int64_t)k * ng + j];
#if ORC_PLANT == 6
      key.c[0] = ef[i] + ef[i];   // planted: uses f's first exponent twice
#endif
      if (above_bound(T, key.c, nv)) continue;
      if constexpr (std::is_same<Coef, double>::value) {
        if (!coef_kept(T, cf[i], cg[j])) continue;
      }
      if (!in_shard(key, nv, smod, sid)) continue;
      auto it = map.find(key);
      if (it == map.end()) it = map.emplace(key, Acc()).first;
      if constexpr (sizeof(Coef) == 8 && std::is_same<Coef, int64_t>::value) {
        it->second.s += (unsigned __int128)((__int128)cf[i] * (__int128)cg[j]);
      } else {
        it->second.add(cf[i] * cg[j]);
      }
    }
  }
}

Result* poly_mul(int nv, int64_t nf, const int32_t* ef, const void* cfv, int64_t ng,
                 const int32_t* eg, const void* cgv, int is_f64, int nthreads, int64_t smod,
                 int64_t sid, int keep_zero, const Trunc& T) {
  KeyLess L = poly_order(nv);
  Result* R = new Result;
  R->np = nv; R->nt = 0; R->poisson = false; R->is_f64 = is_f64 != 0;
  if (nthreads < 1) nthreads = 1;
  if (!is_f64) {
    std::vector<TermMap<AccI>> maps(nthreads, TermMap<AccI>(L));
    auto cf = (const int64_t*)cfv; auto cg = (const int64_t*)cgv;
    run_threads(nthreads, nf, [&](int t, int64_t a, int64_t b) {
      poly_slice<AccI, int64_t>(nv, ef, cf, nf, a, b, eg, cg, ng, smod, sid, T, maps[t]);
    });
    for (int t = 1; t < nthreads; ++t)
      for (auto& kv : maps[t]) maps[0][kv.first].s += kv.second.s;
    for (auto& kv : maps[0]) {
      __int128 v = (__int128)kv.second.s;
      if (v > (__int128)INT64_MAX || v < (__int128)INT64_MIN) R->overflow = 1;
      int64_t w = (int64_t)(uint64_t)kv.second.s;
#if ORC_PLANT != 16
      if (w == 0 && !keep_zero) continue;   // (planted 16: zero sums kept)
#endif
      R->keys.push_back(kv.first);
      R->ci.push_back(w);
    }
  } else {
    std::vector<TermMap<AccF>> maps(nthreads, TermMap<AccF>(L));
    auto cf = (const double*)cfv; auto cg = (const double*)cgv;
    run_threads(nthreads, nf, [&](int t, int64_t a, int64_t b) {
      poly_slice<AccF, double>(nv, ef, cf, nf, a, b, eg, cg, ng, smod, sid, T, maps[t]);
    });
    for (int t = 1; t < nthreads; ++t)
      for (auto& kv : maps[t]) maps[0][kv.first].merge(kv.second);
    for (auto& kv : maps[0]) {
      double v = kv.second.value();
      if (v == 0.0 && !keep_zero) continue;
      R->keys.push_back(kv.first);
      R->cf.push_back(v);
      R->mass.push_back(kv.second.mass);
    }
  }
  return R;
}

// ---------------------------------------------------------------------------
// Poisson series product
// ---------------------------------------------------------------------------
// Writes the canonical form of (kind, trig) into key and returns the sign the
// coefficient takes, or 0 when the term vanishes (a sine of the zero vector).
int canonicalise(Key& key, int nt) {
  int last = -1;
#if ORC_PLANT == 4
  for (int k = nt - 1; k >= 0; --k)   // planted: looks at the lowest-index nonzero
    if (key.c[1 + k] != 0) last = k;
#else
  for (int k = 0; k < nt; ++k)
    if (key.c[1 + k] != 0) last = k;
#endif
  if (last < 0) return key.c[0] == 1 ? 0 : 1;
  if (key.c[1 + last] > 0) return 1;
  for (int k = 0; k < nt; ++k) key.c[1 + k] = -key.c[1 + k];
#if ORC_PLANT == 18
  return 1;   // planted: a negated sine keeps its sign
#endif
  return key.c[0] == 1 ? -1 : 1;
}

struct PSIn {
  int64_t n;
  const int32_t* e;   // [np][n]
  const int32_t* t;   // [nt][n]
  const uint8_t* k;   // [n]
  const double* c;    // [n]
};

void emit(TermMap<AccF>& map, Key& key, int np, int nt, double coef, int64_t smod, int64_t sid,
          const Trunc& T) {
  int s = canonicalise(key, nt);
  if (s == 0) return;
  if (above_harmonic(T, key, nt)) return;
  if (!in_shard(key, 1 + nt + np, smod, sid)) return;
  auto it = map.find(key);
  if (it == map.end()) it = map.emplace(key, AccF()).first;
  it->second.add(s > 0 ? coef : -coef);
}

void poisson_slice(int np, int nt, const PSIn& F, const PSIn& G, int64_t i0, int64_t i1,
                   int64_t smod, int64_t sid, const Trunc& T, TermMap<AccF>& map) {
  Key key;
  std::memset(&key, 0, sizeof key);
  for (int64_t i = i0; i < i1; ++i) {
    for (int64_t j = 0; j < G.n; ++j) {
      if (T.on) {   // both terms of the pair share the polynomial part
        int32_t poly[MAXK];
        for (int k = 0; k < np; ++k) poly[k] = F.e[(int64_t)k * F.n + i] + G.e[(int64_t)k * G.n + j];
        if (above_bound(T, poly, np)) continue;
      }
#if ORC_PLANT == 12
      if (!coef_kept(T, F.c[i] * 0.5, G.c[j])) continue;   // planted: the bound applied after the 1/2
#else
      if (!coef_kept(T, F.c[i], G.c[j])) continue;
#endif
      double h = (F.c[i] * G.c[j]) * 0.5;
#if ORC_PLANT == 1
      h = F.c[i] * G.c[j];   // planted: the product-to-sum halves dropped
#endif
      int kf = F.k[i], kg = G.k[j];
      // (kind of the result, sign) of the difference term and of the sum term
      int kd, ks;
      double sd, ss;
      if (kf == 0 && kg == 0) { kd = 0; sd = +1; ks = 0; ss = +1; }        // cos cos
      else if (kf == 0 && kg == 1) { kd = 1; sd = -1; ks = 1; ss = +1; }   // cos sin
      else if (kf == 1 && kg == 0) { kd = 1; sd = +1; ks = 1; ss = +1; }   // sin cos
      else { kd = 0; sd = +1; ks = 0; ss = -1; }                           // sin sin
#if ORC_PLANT == 2
      if (kf == 0 && kg == 1) sd = +1;   // planted: wrong sign in cos*sin
#endif
      for (int k = 0; k < np; ++k)
        key.c[1 + nt + k] = F.e[(int64_t)k * F.n + i] + G.e[(int64_t)k * G.n + j];
#if ORC_PLANT == 19
      for (int k = 0; k < np; ++k)   // planted: the difference term's polynomial exponents subtracted
        key.c[1 + nt + k] = F.e[(int64_t)k * F.n + i] - G.e[(int64_t)k * G.n + j];
#endif
      // difference term: trig(f) - trig(g)
      key.c[0] = kd;
      for (int k = 0; k < nt; ++k)
        key.c[1 + k] = F.t[(int64_t)k * F.n + i] - G.t[(int64_t)k * G.n + j];
#if ORC_PLANT == 3
      for (int k = 0; k < nt; ++k) key.c[1 + k] = -key.c[1 + k];   // planted: g - f
#endif
      emit(map, key, np, nt, sd * h, smod, sid, T);
      // sum term: trig(f) + trig(g)
      for (int k = 0; k < np; ++k)
        key.c[1 + nt + k] = F.e[(int64_t)k * F.n + i] + G.e[(int64_t)k * G.n + j];
      key.c[0] = ks;
      for (int k = 0; k < nt; ++k)
        key.c[1 + k] = F.t[(int64_t)k * F.n + i] + G.t[(int64_t)k * G.n + j];
      emit(map, key, np, nt, ss * h, smod, sid, T);
    }
  }
}

Result* poisson_mul(int np, int nt, const PSIn& F, const PSIn& G, int nthreads, int64_t smod,
                    int64_t sid, int keep_zero, const Trunc& T) {
  KeyLess L = poisson_order(np, nt);
  Result* R = new Result;
  R->np = np; R->nt = nt; R->poisson = true; R->is_f64 = true;
  if (nthreads < 1) nthreads = 1;
  std::vector<TermMap<AccF>> maps(nthreads, TermMap<AccF>(L));
  run_threads(nthreads, F.n, [&](int t, int64_t a, int64_t b) {
    poisson_slice(np, nt, F, G, a, b, smod, sid, T, maps[t]);
  });
  for (int t = 1; t < nthreads; ++t)
    for (auto& kv : maps[t]) maps[0][kv.first].merge(kv.second);
  for (auto& kv : maps[0]) {
    double v = kv.second.value();
    if (v == 0.0 && !keep_zero) continue;
    R->keys.push_back(kv.first);
    R->cf.push_back(v);
    R->mass.push_back(kv.second.mass);
  }
  return R;
}

}  // namespace

extern "C" {

// Product of two polynomials in nv variables.  Exponents are int32 arrays laid
// out [nv][n] (one row per variable); coefficients int64 (is_f64 = 0) or
// float64 (is_f64 = 1).  Returns an owned result handle.
void* orc_poly_mul(int nv, int64_t nf, const int32_t* ef, const void* cf, int64_t ng,
                   const int32_t* eg, const void* cg, int is_f64, int nthreads,
                   int64_t shard_mod, int64_t shard_id, int keep_zero) {
  if (nv < 1 || nv > MAXK || nf < 0 || ng < 0) return nullptr;
  return poly_mul(nv, nf, ef, cf, ng, eg, cg, is_f64, nthreads, shard_mod, shard_id, keep_zero, Trunc());
}

// As orc_poly_mul, keeping only the pairs whose product term has degree at
// most max_degree in the variables of mask (bit k = variable k).
void* orc_poly_mul_trunc(int nv, int64_t nf, const int32_t* ef, const void* cf, int64_t ng,
                         const int32_t* eg, const void* cg, int is_f64, int nthreads,
                         int64_t shard_mod, int64_t shard_id, int keep_zero, uint32_t mask,
                         int64_t max_degree) {
  if (nv < 1 || nv > MAXK || nf < 0 || ng < 0) return nullptr;
  Trunc T;
  T.on = 1; T.mask = mask; T.N = max_degree;
  return poly_mul(nv, nf, ef, cf, ng, eg, cg, is_f64, nthreads, shard_mod, shard_id, keep_zero, T);
}

// Product of two Poisson series with np polynomial variables and nt trig
// variables.  kind: 0 = cos, 1 = sin.  Inputs must be canonical.
void* orc_poisson_mul(int np, int nt, int64_t nf, const int32_t* ef, const int32_t* tf,
                      const uint8_t* kf, const double* cf, int64_t ng, const int32_t* eg,
                      const int32_t* tg, const uint8_t* kg, const double* cg, int nthreads,
                      int64_t shard_mod, int64_t shard_id, int keep_zero) {
  if (np < 0 || nt < 1 || 1 + np + nt > MAXK || nf < 0 || ng < 0) return nullptr;
  PSIn F{nf, ef, tf, kf, cf}, G{ng, eg, tg, kg, cg};
  return poisson_mul(np, nt, F, G, nthreads, shard_mod, shard_id, keep_zero, Trunc());
}

// As orc_poisson_mul with the polynomial part truncated as in orc_poly_mul_trunc.
void* orc_poisson_mul_trunc(int np, int nt, int64_t nf, const int32_t* ef, const int32_t* tf,
                            const uint8_t* kf, const double* cf, int64_t ng, const int32_t* eg,
                            const int32_t* tg, const uint8_t* kg, const double* cg, int nthreads,
                            int64_t shard_mod, int64_t shard_id, int keep_zero, uint32_t mask,
                            int64_t max_degree) {
  if (np < 1 || nt < 1 || 1 + np + nt > MAXK || nf < 0 || ng < 0) return nullptr;
  PSIn F{nf, ef, tf, kf, cf}, G{ng, eg, tg, kg, cg};
  Trunc T;
  T.on = 1; T.mask = mask; T.N = max_degree;
  return poisson_mul(np, nt, F, G, nthreads, shard_mod, shard_id, keep_zero, T);
}

// Every truncation criterion at once.  deg_on / harm_on / coef_on switch the
// criteria on (see Trunc); a coefficient bound needs float64 coefficients.
struct OrcTrunc {
  int32_t deg_on;
  uint32_t deg_mask;    // 0 = every polynomial variable
  int64_t deg_max;
  int32_t harm_on;
  uint32_t harm_mask;   // 0 = every trig variable
  int64_t harm_max;
  int32_t coef_on;
  double coef_min;
};

static Trunc to_trunc(const OrcTrunc* t, int np, int nt) {
  Trunc T;
  if (!t) return T;
  T.on = t->deg_on;
  T.mask = t->deg_mask ? t->deg_mask : (np >= 32 ? 0xffffffffu : (1u << np) - 1u);
  T.N = t->deg_max;
  T.hon = t->harm_on;
  T.hmask = t->harm_mask ? t->harm_mask : (nt >= 32 ? 0xffffffffu : (1u << nt) - 1u);
  T.hN = t->harm_max;
  T.con = t->coef_on;
  T.cmin = t->coef_min;
  return T;
}

void* orc_poly_mul_tr(int nv, int64_t nf, const int32_t* ef, const void* cf, int64_t ng,
                      const int32_t* eg, const void* cg, int is_f64, int nthreads, int64_t shard_mod,
                      int64_t shard_id, int keep_zero, const OrcTrunc* tr) {
  if (nv < 1 || nv > MAXK || nf < 0 || ng < 0) return nullptr;
  if (tr && (tr->harm_on || (tr->coef_on && !is_f64))) return nullptr;
  return poly_mul(nv, nf, ef, cf, ng, eg, cg, is_f64, nthreads, shard_mod, shard_id, keep_zero,
                  to_trunc(tr, nv, 0));
}

void* orc_poisson_mul_tr(int np, int nt, int64_t nf, const int32_t* ef, const int32_t* tf,
                         const uint8_t* kf, const double* cf, int64_t ng, const int32_t* eg,
                         const int32_t* tg, const uint8_t* kg, const double* cg, int nthreads,
                         int64_t shard_mod, int64_t shard_id, int keep_zero, const OrcTrunc* tr) {
  if (np < 0 || nt < 1 || 1 + np + nt > MAXK || nf < 0 || ng < 0) return nullptr;
  if (tr && tr->deg_on && np < 1) return nullptr;
  PSIn F{nf, ef, tf, kf, cf}, G{ng, eg, tg, kg, cg};
  return poisson_mul(np, nt, F, G, nthreads, shard_mod, shard_id, keep_zero, to_trunc(tr, np, nt));
}

int64_t orc_result_nterms(const void* r) { return (int64_t)((const Result*)r)->keys.size(); }
int orc_result_overflow(const void* r) { return ((const Result*)r)->overflow; }

// Copies the result out.  Polynomial: exps [np][n], coef int64 or float64,
// mass (float64 only, may be null).  Poisson: exps [np][n], trig [nt][n],
// kind [n], coef float64, mass.  Any output pointer may be null.
void orc_result_copy(const void* rv, int32_t* exps, int32_t* trig, uint8_t* kind, void* coef,
                     double* mass) {
  const Result* R = (const Result*)rv;
  int64_t n = (int64_t)R->keys.size();
  int off = R->poisson ? 1 + R->nt : 0;
  for (int64_t i = 0; i < n; ++i) {
    const Key& k = R->keys[i];
    if (exps)
      for (int v = 0; v < R->np; ++v) exps[(int64_t)v * n + i] = k.c[off + v];
    if (R->poisson) {
      if (trig)
        for (int v = 0; v < R->nt; ++v) trig[(int64_t)v * n + i] = k.c[1 + v];
      if (kind) kind[i] = (uint8_t)k.c[0];
    }
    if (coef) {
      if (R->is_f64) ((double*)coef)[i] = R->cf[i];
      else ((int64_t*)coef)[i] = R->ci[i];
    }
    if (mass && R->is_f64) mass[i] = R->mass[i];
  }
}

void orc_result_free(void* r) { delete (Result*)r; }

// FNV-1a hash of one key, as used by the shard filter (exposed so a test can
// select the same shard of a result computed elsewhere).
uint64_t orc_key_hash(const int32_t* comps, int len) {
  Key k;
  std::memset(&k, 0, sizeof k);
  for (int t = 0; t < len && t < MAXK; ++t) k.c[t] = comps[t];
  return fnv1a(k, len);
}

int orc_plant(void) { return ORC_PLANT; }

}  // extern "C"
