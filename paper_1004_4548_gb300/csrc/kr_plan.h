// Host-side planning shared by the C ABI translation units: the coding box of
// a product (Sec. 2: widths, coding vector, code range with an overflow
// check), the choice between the dense and the hash path (Sec. 3.2: by the
// density of the product), and the sizes of every scratch buffer.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "kr_internal.cuh"

namespace kr {

// Upper bound on bytes the dense path may spend on its accumulator array, and
// how much larger than the number of term products the code range may be
// before the hash path is preferred (array initialisation and compaction cost
// O(W), Sec. 3.2).
constexpr int64_t DENSE_MAX_BYTES = int64_t(16) << 30;
constexpr double DENSE_KAPPA = 4.0;
// Poisson series on the dense path: the array may reach 48 GiB, and the code
// range may be sixteen times the number of updates (two per term pair)
constexpr int64_t DENSE_POISSON_MAX_BYTES = int64_t(48) << 30;
constexpr double DENSE_POISSON_KAPPA = 16.0;
constexpr int64_t BITMAP_MAX_BITS = 1600000;   // on-chip bitmap sort (<= 200 KB)
constexpr int64_t BITONIC_MAX_N = 16384;       // shared-memory bitonic sort (128 KB)
constexpr int64_t DEFAULT_S = 8192;            // dense block: 64 KB of shared memory
constexpr int64_t MAX_S = 27648;               // 216 KB slice + the 10 KB window table
// compaction chunks: 8192 dense slots (8 B) or 4096 hash slots (16 B), so that
// each of the compaction CTA's 8 warps holds 16 rows of 512 bytes
constexpr int64_t COMPACT_CHUNK = 8192;
constexpr int64_t COMPACT_CHUNK_HASH = 4096;
constexpr double DEFAULT_LOAD = 0.5;
constexpr int DEFAULT_PROBES = 512;
constexpr int HASH_TILE_I = 32;
constexpr int HASH_TILE_J = 1024;

// One product as the host sees it (device pointers to its inputs).
struct Job {
  bool poisson = false;
  bool f64 = false;
  int np = 0, nt = 0;
  Operand f{}, g{};
  kr_opts opts{};
};

// The result of planning: Prod filled except scratch pointers, plus sizes.
struct Plan {
  Prod p{};
  kr_status st = KR_OK;
  int64_t op_bytes[2] = {0, 0};
  int64_t accum_bytes = 0;   // dense array or hash table (zeroed before use)
  int64_t out_cap = 0;
  int64_t dense_task_cap = 0;
  int64_t radix_sort_n = 0;  // largest radix sort this product needs
  int64_t bound_slots = 0;   // hash: table size for the term-product bound at the load factor
  int64_t slots_override = 0;  // hash: table size forced by a regrowth
  bool outcap_full = false;    // hash: output room for a full table (after an overflow)
  bool empty = false;          // truncation or the key window leaves no term: the product is zero
  int passes_f = 0, passes_g = 0;
};

// int64 widths/codes with 128-bit overflow checks; returns KR_ERR_OVERFLOW
// when the product of the widths exceeds 2^63 - 1.
kr_status coding_vector(const int64_t* w, int n, int64_t* c, int64_t* W);

void plan_product(const Job& job, const int32_t* ranges_f, const int32_t* ranges_g, int num_sms,
                  Plan* out);

int bits_for(uint64_t range);   // bits needed for values in [0, range)

// Hash path: table size and output capacity from the HyperLogLog estimate of
// the distinct output keys (or a forced size), capped by the term-product bound.
void finish_hash_sizes(const kr_opts& o, Plan* pl);

}  // namespace kr
