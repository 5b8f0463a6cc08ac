/*
 * kron.h - C ABI of libkron: multiplication of sparse multivariate Laurent
 * polynomials and Poisson series on NVIDIA GB300 (sm_103a).
 *
 * Method (Biscani, "Multiplication of sparse Laurent polynomials and Poisson
 * series on modern hardware architectures"):
 *   1. Kronecker substitution (Sec. 2, Table 1, Table 2 and the coding
 *      equations that follow it): every exponent vector e in a box
 *      [e_min, e_max] maps to the integer code c . e - chi, with widths
 *      w_k = 1 + e_k,max - e_k,min, coding vector c = (1, w_0, w_0 w_1, ...)
 *      and chi = c . e_min.  Variable 0 is the least significant.  The map is
 *      additive, so a product of monomials is a sum of codes.
 *   2. Schoolbook product of the coded univariate polynomials (Sec. 3), with
 *      accumulation either into a dense array indexed by code (moderately
 *      sparse products, Sec. 3.1) or into a hash table keyed by code (highly
 *      sparse products, Sec. 3.2).
 *   3. Poisson series (Sec. 1, Eq. 1): each pair of terms expands, by the
 *      product-to-sum formulas of Eq. 6, into a term at the sum and a term at
 *      the difference of the trigonometric multiplier vectors.  Eq. 6 is
 *      printed without the factor 1/2 of the trigonometric identities; this
 *      library applies it (cos a cos b = 1/2 cos(a-b) + 1/2 cos(a+b), ...).
 *
 * Conventions shared by every entry point
 *   - Term arrays are "structure of arrays": exponents of a series with v
 *     variables and n terms are an int32 array [v][n] (row k holds variable k
 *     of every term, row stride n, or the output capacity for outputs).
 *   - Pointers may address device memory or host memory (pageable or pinned);
 *     the library detects which with cudaPointerGetAttributes and stages host
 *     data through device scratch, except that the terms of a dense
 *     polynomial product may be written by the GPU straight into pinned host
 *     outputs through their device mapping.  The caller owns every buffer it
 *     passes.
 *   - Every call is issued on the given stream.  Calls that return a term count
 *     synchronise that stream before returning; device outputs are complete
 *     when the call returns KR_OK only after a later synchronisation of the
 *     stream (the output decode is the last work queued).
 *   - Canonical output: terms sorted by ascending code (reverse lexicographic
 *     exponent order, variable 0 least significant; Poisson keys ordered by
 *     kind (cos < sin), then trig multipliers, then exponents), no zero
 *     coefficients; a truncated product is sorted by degree first (kr_opts).
 *     int64 coefficients use wrapping arithmetic modulo 2^64.
 *   - Trig canonical form: a multiplier vector is canonical when its
 *     highest-index nonzero entry is positive.  Inputs must be canonical and a
 *     sine may not have the zero vector (KR_ERR_INVALID otherwise).  Results
 *     are canonicalised: cos(-x) = cos x, sin(-x) = -sin x, sin 0 = 0.
 *   - No C++ exception crosses this interface.  A context is not thread safe:
 *     use one context per host thread.
 */
#ifndef KRON_H
#define KRON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KR_MAXV 16            /* max variables: poly vars + trig vars */

typedef enum {
  KR_OK = 0,
  KR_ERR_INVALID = 1,    /* bad argument, mismatched shapes, non-canonical trig input */
  KR_ERR_RANGE = 2,      /* an exponent lies outside the declared coding box */
  KR_ERR_OVERFLOW = 3,   /* the code range exceeds 2^63 - 1 (no coding exists) */
  KR_ERR_DUP = 4,        /* an input series repeats a term key */
  KR_ERR_OOM = 5,        /* device or pinned-host allocation failed */
  KR_ERR_CAPACITY = 6,   /* output buffers too small; required count returned */
  KR_ERR_TIMEOUT = 7,    /* a bounded device wait gave up (the compaction's wait on a
                            preceding chunk); the call's results are unreliable */
  KR_ERR_CUDA = 8,       /* a CUDA runtime call failed; see kr_last_error */
  KR_ERR_TABLE_FULL = 9, /* hash table full after every allowed regrowth */
  KR_ERR_TOO_LARGE = 10  /* the problem exceeds a fixed limit of the entry point */
} kr_status;

typedef enum { KR_I64 = 0, KR_F64 = 1 } kr_coef_t;

typedef enum { KR_PATH_AUTO = 0, KR_PATH_DENSE = 1, KR_PATH_HASH = 2 } kr_path;

typedef struct CUstream_st* kr_stream;   /* same type as cudaStream_t; NULL = default */
typedef struct kr_ctx kr_ctx;

/* A sparse polynomial (Sec. 3.1, "sparse distributed" representation). */
typedef struct {
  int32_t nvars;         /* 1 .. KR_MAXV */
  int64_t nterms;        /* 0 .. 2^31 - 2 */
  const int32_t* exps;   /* [nvars][nterms] */
  const void* coef;      /* int64_t or double [nterms] */
  kr_coef_t type;
} kr_poly;

/* Product buffers.  capacity: terms the buffers hold.  nterms: set on return
 * (also on KR_ERR_CAPACITY, to the count required).  exps and codes may be
 * NULL.  omin / omax: the product's coding box, set on return, for
 * kron_decode of the codes. */
typedef struct {
  int32_t nvars;
  int64_t capacity;
  int64_t nterms;
  int32_t* exps;         /* [nvars][capacity] */
  void* coef;            /* [capacity], type of the inputs */
  int64_t* codes;        /* [capacity] Kronecker codes (c . e - chi), or NULL */
  int32_t omin[KR_MAXV];
  int32_t omax[KR_MAXV];
} kr_poly_out;

/* A Poisson series (Eq. 1): sum of C x^a cos|sin(j . y). */
typedef struct {
  int32_t npoly;         /* polynomial variables, >= 0 */
  int32_t ntrig;         /* trig variables, >= 1; npoly + ntrig <= KR_MAXV */
  int64_t nterms;
  const int32_t* exps;   /* [npoly][nterms] */
  const int32_t* trig;   /* [ntrig][nterms], canonical */
  const uint8_t* kind;   /* [nterms], 0 = cos, 1 = sin */
  const double* coef;    /* [nterms] */
} kr_pseries;

typedef struct {
  int32_t npoly, ntrig;
  int64_t capacity;
  int64_t nterms;
  int32_t* exps;         /* [npoly][capacity] or NULL */
  int32_t* trig;         /* [ntrig][capacity] or NULL */
  uint8_t* kind;         /* [capacity] or NULL */
  double* coef;          /* [capacity] */
  int64_t* codes;        /* [capacity] combined keys ((kind*T2 + |t|)*Wp + p), or NULL */
} kr_pseries_out;

/* Tuning knobs.  A NULL kr_opts pointer, or a zero field, means "default". */
typedef struct {
  int32_t path;          /* kr_path; AUTO picks by density (Sec. 3.2) */
  int32_t block_slots;   /* dense path: output codes per block (shared-memory slice) */
  double load_factor;    /* hash path: target table load factor, (0, 0.9] */
  int32_t probe_limit;   /* hash path: windows probed before TABLE_FULL */
  int32_t unsorted;      /* hash path: 1 = leave the output in table order */
  int32_t max_regrow;    /* hash path: regrowths after TABLE_FULL (x4 each, the last one
                            to the term-product bound); 0 = 4, <0 = none */
  int64_t table_slots;   /* hash path: initial table slots (power of two), 0 = sized
                            from the term-product bound and load_factor */
  /* Truncated multiplication (Sec. 3: truncation by the exponents of one or
   * more polynomial variables).  With truncate = 1 the product keeps only the
   * terms whose degree in the variables of trunc_mask (the sum of their
   * exponents; bit k = polynomial variable k, 0 = all of them) is at most
   * trunc_degree, which may be negative.  Degree is additive, so these are
   * exactly the terms of the full product of that degree, and a term pair of
   * higher degree is never formed: the degree becomes the most significant
   * digit of the code (the highest-index variable of the mask is replaced by
   * the degree; the map stays one to one), the truncation becomes an upper
   * bound on the output code, and the pairs below it are, for each term of
   * f, a prefix of g's sorted codes.  Terms of an operand whose degree alone
   * leaves no partner are dropped before the multiplication.  The output is
   * sorted by that graded code: by degree first, then as usual (reverse
   * lexicographic, variable 0 least significant) over the other variables.
   * For Poisson series the degree is that of the polynomial part. */
  int32_t truncate;
  uint32_t trunc_mask;
  int64_t trunc_degree;
  /* Output key window: only the terms of the product whose key (the code of a
   * polynomial term, ((kind * T2) + |t|) * Wp + p for a Poisson term; the
   * graded code for a truncated product) lies in [code_lo, code_hi) are
   * computed; code_hi = 0 means no upper limit.  The dense path then holds an
   * array of code_hi - code_lo slots only, so a product too large for one
   * device splits into windows that run one after another or on several
   * devices, each window's terms sorted; concatenated in window order they
   * are the whole product (Sec. 4's disjoint output ranges, across calls).
   * kron_split_hist helps choose windows of equal work. */
  int64_t code_lo;
  int64_t code_hi;
  /* Truncation by the order of the Fourier harmonics (Sec. 3), Poisson series
   * only: with trunc_harmonic = 1 the product keeps only the terms whose
   * harmonic order, the sum of |t_k| over the trig variables of harmonic_mask
   * (bit k = trig variable k, 0 = all of them), is at most harmonic_order.
   * The order of a sum or a difference of multiplier vectors is not the sum
   * of the orders, so each of the two terms a pair emits is judged on its own,
   * before it reaches the accumulator; the output order is unchanged.  The
   * counted multipliers of both operands must lie in [-32767, 32767]
   * (KR_ERR_INVALID otherwise); a negative order gives the zero series. */
  int32_t trunc_harmonic;
  uint32_t harmonic_mask;
  int64_t harmonic_order;
  /* Truncation by the absolute value of the coefficients (Sec. 3), float64
   * coefficients only (KR_ERR_INVALID for int64 ones): coef_min > 0 keeps only
   * the pairs of terms with |C_f * C_g| >= coef_min, that product being the
   * float64 product of the two coefficients (for Poisson series, before the
   * 1/2 of Eq. 6).  Both operands are then walked in order of decreasing |C|,
   * so that for each term of f the kept partners are a prefix of g, and the
   * rest of the pairs is skipped without being formed (the ordering by the
   * truncation criterion that Sec. 3 proposes).  Polynomial products with a
   * bound take the hash path; 0 = no bound. */
  double coef_min;
} kr_opts;

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* Creates a context bound to CUDA device `device` (scratch arena, pinned
 * staging, status words).  Returns KR_ERR_CUDA / KR_ERR_OOM on failure. */
kr_status kr_ctx_create(int32_t device, kr_ctx** out);
/* Frees every resource of the context (synchronises its streams first). */
void kr_ctx_destroy(kr_ctx* ctx);
/* Text of the last CUDA error seen by this context ("" if none). */
const char* kr_last_error(const kr_ctx* ctx);
/* Fixed text for a status code. */
const char* kron_strerror(kr_status s);
/* Bytes of device scratch currently held by the context. */
int64_t kr_ctx_scratch_bytes(const kr_ctx* ctx);
/* Releases the context's cached scratch (device arenas, pinned staging and
 * the results of its last batch); the next call allocates what it needs.
 * Synchronises the context's device. */
kr_status kr_ctx_trim(kr_ctx* ctx);
/* Stage timing.  When enabled, every multiplication records a CUDA event on
 * its stream after each pipeline stage (range_scan, zero_accumulators, encode,
 * sort, gather, dense_plan, dense_accum, hash_insert, compact, output_sort,
 * decode, copy_out); the durations of the last call are then readable.
 * Stages that did not run are absent.  Times in milliseconds, each the
 * interval between the previous event and the stage's own. */
kr_status kr_ctx_set_profiling(kr_ctx* ctx, int32_t enable);
int32_t kr_ctx_stage_count(const kr_ctx* ctx);
/* name: static string owned by the library. */
kr_status kr_ctx_stage(const kr_ctx* ctx, int32_t i, const char** name, double* ms);
/* Kernels this context has launched since its creation (all calls). */
int64_t kr_ctx_launch_count(const kr_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Kronecker coding (Sec. 2, Table 2 and the equations after it)            */
/* ------------------------------------------------------------------------ */

/* Host-only.  For the box [emin, emax] of nvars variables writes the coding
 * vector c (cvec_out[k] = prod_{l<k} w_l) and the number of codes
 * W = prod_k w_k (range_out).  KR_ERR_OVERFLOW when W > 2^63 - 1,
 * KR_ERR_INVALID when emin > emax for some k.  Host arrays, caller-owned. */
kr_status kron_plan(const int32_t* emin, const int32_t* emax, int32_t nvars,
                    int64_t* cvec_out, int64_t* range_out);

/* codes_out[i] = sum_k c_k (exps[k][i] - emin[k]) for the box [emin, emax]
 * (host arrays).  exps: [nvars][n]; codes_out: [n].  KR_ERR_RANGE when a
 * term lies outside the box; KR_ERR_OVERFLOW as for kron_plan, and also when
 * some width w_k exceeds 2^31 - 1 (checked on the host before any device
 * work).  Synchronises the stream. */
kr_status kron_encode(kr_ctx* ctx, const int32_t* exps, int64_t n, int32_t nvars,
                      const int32_t* emin, const int32_t* emax, int64_t* codes_out,
                      kr_stream stream);

/* Inverse of kron_encode: exps_out[k][i] = (codes[i] / c_k) mod w_k + emin[k].
 * KR_ERR_RANGE when a code lies outside [0, W); KR_ERR_OVERFLOW as for
 * kron_encode.  Synchronises the stream. */
kr_status kron_decode(kr_ctx* ctx, const int64_t* codes, int64_t n, int32_t nvars,
                      const int32_t* emin, const int32_t* emax, int32_t* exps_out,
                      kr_stream stream);

/* ------------------------------------------------------------------------ */
/* Multiplication                                                            */
/* ------------------------------------------------------------------------ */

/* h = f * g for sparse Laurent polynomials (Sec. 3).  Each operand is coded in
 * the product's box (widths of the output, each operand offset by its own
 * minimum), so a code sum is the product's code.  Dense path (Sec. 3.1): the
 * output code range is split into blocks, each accumulated in on-chip shared
 * memory; hash path (Sec. 3.2): an open-addressing table in device memory.
 * Returns KR_ERR_CAPACITY with h->nterms = required when h->capacity is too
 * small: the product is kept in the context and kron_fetch_poly copies it out
 * without recomputing.  Synchronises the stream. */
kr_status poly_mul(kr_ctx* ctx, const kr_poly* f, const kr_poly* g, kr_poly_out* h,
                   const kr_opts* opts, kr_stream stream);

/* h = f * g for Poisson series (Eq. 1, Eq. 6 with the factor 1/2).  Dense
 * path (Sec. 3.1): each pair adds into an array indexed by the key of the sum
 * and of the difference term (up to 48 GiB); hash path (Sec. 3.2): both terms
 * go into the open-addressing table.  AUTO picks the dense path when the key
 * range is at most sixteen times the number of updates.
 * Polynomial exponents are coded in the product's box; trig multipliers in the
 * symmetric box |t_k| <= R_k = max|f_k| + max|g_k|, so that sums and
 * differences of codes are the codes of the sums and differences (the
 * extension of the coding vector to negated operands described in Sec. 2).
 * Capacity contract as poly_mul. */
kr_status poisson_mul(kr_ctx* ctx, const kr_pseries* f, const kr_pseries* g,
                      kr_pseries_out* h, const kr_opts* opts, kr_stream stream);

/* One product of a batch: kind 0 multiplies the polynomials f and g, kind 1
 * the Poisson series pf and pg.  opts as for poly_mul (zero = defaults). */
typedef struct {
  int32_t kind;
  kr_poly f, g;
  kr_pseries pf, pg;
  kr_opts opts;
} kr_job;

/* Result of one product of a batch.  The arrays are device memory owned by
 * the context, valid until the next kron_mul_batch on it or its destruction;
 * each is laid out [variables][nterms] (row stride nterms), sorted by code. */
typedef struct {
  kr_status status;
  int32_t path;          /* KR_PATH_DENSE or KR_PATH_HASH as run */
  int64_t nterms;
  const int32_t* exps;   /* [nvars or npoly][nterms] */
  const int32_t* trig;   /* [ntrig][nterms] (Poisson) */
  const uint8_t* kind;   /* [nterms] (Poisson) */
  const void* coef;      /* [nterms] */
} kr_result;

/* Many products of uneven sizes in one pipeline: one launch of each stage
 * (range scan, encode, sorts, gather, accumulation of every dense and hash
 * product by one persistent grid each, compaction, decode) for all products
 * of a wave.  Products are grouped into waves of at most wave_pairs
 * term-products (0 = 2^33) so that scratch stays bounded; a wave that runs
 * out of device memory is split in two.  Every product gets its own status
 * in res[i]; the call returns KR_OK unless the whole call failed (CUDA error,
 * out of memory for a single product).  Synchronises the stream. */
kr_status kron_mul_batch(kr_ctx* ctx, const kr_job* jobs, int32_t njobs, kr_result* res,
                         int64_t wave_pairs, kr_stream stream);

/* A batch prepared for repeated execution with a CUDA graph.  The first run
 * plans every product (coding boxes, paths, table sizes from the distinct-key
 * estimates, output counts) with scratch owned by the batch; the complete
 * device work of a run (encode, sorts, accumulation, compaction, ordering,
 * decode) is then captured into one CUDA graph.  Launching the batch replays
 * the graph without host planning or synchronisation.  Inputs must be device
 * buffers that keep their exponents, kinds and sizes between launches; the
 * coefficients may change.  res (optional, njobs entries) receives the first
 * run's results; result arrays are owned by the batch and overwritten by
 * every launch.  The batch holds its scratch until destroyed. */
typedef struct kr_batch kr_batch;
kr_status kron_batch_prepare(int32_t device, const kr_job* jobs, int32_t njobs, kr_batch** out,
                             kr_result* res, kr_stream stream);
/* Replays the batch on `stream` (asynchronous). */
kr_status kron_batch_launch(kr_batch* b, kr_stream stream);
/* After the launch's stream has been synchronised: statuses and result
 * pointers.  A product whose term count differs from the prepared run (its
 * coefficients now cancel differently) reports KR_ERR_CAPACITY; prepare the
 * batch again for it. */
kr_status kron_batch_results(kr_batch* b, kr_result* res, int32_t njobs);
void kron_batch_destroy(kr_batch* b);
/* Kernel launches in one replay of a prepared batch (the kernel nodes of its
 * graph), or -1 on failure. */
int64_t kron_batch_graph_kernels(const kr_batch* b);

/* Work histogram of one product for splitting it into output key windows:
 * nsamples term pairs drawn uniformly (from a counter-based hash of seed) are
 * expanded into their output keys (one per pair for polynomials, the sum and
 * difference terms for Poisson series, both with the job's truncation), and
 * hist[b] counts the keys k with floor(k * nbins / krange) = b, where krange
 * (written to *krange_out) is the product's key range: the keys of the whole
 * product lie in [0, krange).  hist: host int64 [nbins], caller-owned.  The
 * job's code window is ignored.  Equal-work windows are the quantiles of the
 * histogram.  Deterministic for fixed inputs and seed.  Synchronises the
 * stream.  KR_ERR_INVALID for an empty product or nbins < 1. */
kr_status kron_split_hist(kr_ctx* ctx, const kr_job* job, int32_t nbins, int64_t nsamples, uint64_t seed,
                          int64_t* hist, int64_t* krange_out, kr_stream stream);

/* Copy the product kept by the last poly_mul / poisson_mul of this context
 * (after KR_ERR_CAPACITY) into h.  KR_ERR_INVALID if there is none. */
kr_status kron_fetch_poly(kr_ctx* ctx, kr_poly_out* h, kr_stream stream);
kr_status kron_fetch_pseries(kr_ctx* ctx, kr_pseries_out* h, kr_stream stream);

/* Dense-path accumulation that allocates nothing.  The paper has no
 * counterpart: this entry point serves callers that cannot let a library call
 * cudaMalloc or cudaFree, because their device memory is owned by their own
 * allocator or a fixed budget, or because they cannot accept the device
 * synchronisation that an allocation or a free brings.
 *
 * Computes out[c] = sum over pairs with fcode[i] + gcode[j] = c of
 * fcoef[i] * gcoef[j] for c in [0, W), with the same planning and
 * accumulation kernels as poly_mul's dense path.
 *   fcode, gcode: device int64 [nf], [ng]: Kronecker codes of both operands in
 *     the product's box (each operand offset by its own minimum, as poly_mul
 *     codes them), ascending, without repeats, with fcode[i] + gcode[j] < W.
 *   fcoef, gcoef: device int64 or double (type) [nf], [ng].
 *   out: device int64 or double [W], written in full (zero where no term).
 * Scratch: a file-scope device array of 8 MiB (every GPU that loads the
 * library holds it until the process exits).  W > 2^24 returns
 * KR_ERR_TOO_LARGE.  No device or host memory is allocated.  The first call
 * on each device looks up the array's device address with that device
 * current (cudaGetSymbolAddress) and caches it; that first call should come
 * before any stream capture.  Every call uses the same array and leaves its
 * contents behind; the call clears what must start at zero.  Calls whose work
 * overlaps on the GPU (other streams, other host threads) race on the array:
 * order them.  Asynchronous on `stream`.  The preconditions on the codes
 * (ascending, without repeats, in [0, W), largest pair sum below W) are
 * checked on the device; inputs that break them leave out all zeros, and no
 * kernel reads or writes outside the caller's buffers. */
kr_status kron_dense_product_static(const int64_t* fcode, const void* fcoef, int64_t nf,
                                    const int64_t* gcode, const void* gcoef, int64_t ng,
                                    kr_coef_t type, int64_t W, void* out, kr_stream stream);

/* ------------------------------------------------------------------------ */
/* Measurement                                                               */
/* ------------------------------------------------------------------------ */

/* Chip-wide rate of conflict-free shared-memory 64-bit atomic adds (int64
 * when f64 = 0, float64 otherwise) on CUDA device `device`: best of `reps`
 * launches timed with CUDA events, in adds per second; < 0 on failure.  Sec. 5
 * measures a multiplication in clock cycles per monomial-by-monomial
 * multiplication and calls it optimal when that approaches the cost of one
 * coefficient multiply-add; on the dense path that step is one shared-memory
 * atomic add, so this rate is the path's ceiling.  Allocates and frees a
 * small device buffer; synchronises the device's default stream. */
double kr_probe_smem_atomic_rate(int32_t device, int32_t f64, int32_t reps);

/* Chip-wide rate of conflict-free int64 accumulates into shared memory in the
 * form the dense path's kernel uses (a 32-bit atomic add of the low word that
 * returns the old value, the carry, a 32-bit atomic add of the high word),
 * with a negative addend so that both adds happen: best of `reps` launches, in
 * accumulates per second; < 0 on failure.  The dense path's ceiling for int64
 * coefficients.  Allocates and frees a small device buffer; synchronises the
 * device's default stream. */
double kr_probe_smem_accumulate_rate(int32_t device, int32_t reps);

/* The hash path's ceiling (Sec. 3.2, the hash table; Sec. 5 measures clock
 * cycles per monomial-by-monomial multiplication, and on this path each one
 * is an insert-or-add into the table): the rate of `updates` insert-or-adds
 * (mode 0: a CAS claim of the key's slot, linear probing, then an atomic add
 * of the value, issued as the polynomial hash kernel issues them) or of plain
 * atomic adds into each key's home slot (mode 1), with keys drawn at random
 * from `distinct` values, into a zeroed table of 2^log2_slots 16-byte slots in
 * device memory; mode 2: float64 atomic adds into a zeroed array of
 * 2^log2_slots 8-byte slots at each key's hashed index (the Poisson dense
 * path's key-indexed array), on CUDA device `device`: best of `reps` launches,
 * in updates per second; < 0 on failure or bad arguments (log2_slots in
 * [10, 30], in [10, 33] for mode 2; distinct at most 0.7 of the slots).
 * Allocates and frees the table (up to 64 GiB in mode 2); synchronises the
 * device's default stream. */
double kr_probe_table_update_rate(int32_t device, int32_t log2_slots, int64_t distinct, int64_t updates,
                                  int32_t mode, int32_t reps);

/* Chip-wide arithmetic rates of the coefficient multiply-add forms the kernels
 * use (Sec. 5 calls a multiplication optimal when its cost per
 * monomial-by-monomial multiplication nears that of one coefficient
 * multiply-add): kind 0 = 64 x 64 -> 64-bit integer multiply-add (int64
 * coefficients), 1 = 32 x 32 -> 64-bit multiply-add (int64 coefficients that
 * fit 32 bits), 2 = float64 FMA; best of `reps` launches on CUDA device
 * `device`, in operations per second; < 0 on failure.  Allocates and frees
 * 8 KB; synchronises the device's default stream. */
double kr_probe_alu_rate(int32_t device, int32_t kind, int32_t reps);

/* Self-test of the library's bounded device waits (the compaction's look-back
 * over preceding chunks): runs the wait against a predecessor that never
 * publishes, on CUDA device `device`, and returns KR_ERR_TIMEOUT when the wait
 * gave up and reported it as it must (KR_OK would mean it did not; KR_ERR_CUDA
 * on a CUDA failure).  The wait ends by itself after roughly 0.1 to 1 s; the
 * device stays usable.  Allocates and frees 128 bytes; synchronises the device. */
kr_status kr_selftest_bounded_wait(int32_t device);

#ifdef __cplusplus
}
#endif
#endif /* KRON_H */
