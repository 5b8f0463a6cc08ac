// Operand preparation for the two truncation criteria of Sec. 3 that are not
// a bound on the code (truncation by degree is: see the graded coding of the
// planner).
//
// Harmonic order.  The order of a Poisson term is the sum of |t_k| over the
// counted trig variables.  It is not additive (|t_f + t_g| is not |t_f| +
// |t_g|), so each of the two terms a pair emits is tested on its own.  The
// kernels hold the operands' trig parts as codes; decoding two codes per pair
// would cost more than the insert it saves, so every operand term's counted
// multipliers are decoded once here into 16-bit lanes biased by 32768, two per
// 32-bit word: rows [0, hwords) hold t, rows [hwords, 2 hwords) hold -t.  Then
// |t_f - t_g|_1 is one __vsadu2 (sum of absolute differences of unsigned
// 16-bit lanes; a common bias cancels) per word of t_f and t_g, and
// |t_f + t_g|_1 the same with -t_g.
//
// Coefficient magnitude.  A pair contributes when |C_f C_g| >= eps.  Sec. 3
// proposes ordering the terms by the truncation criterion so that, while one
// term of the first factor runs over the second, everything from some point on
// can be skipped.  The float64 product's magnitude is monotone in |C_g| for a
// fixed C_f (rounding is monotone), so with g in order of decreasing |C| the
// partners a term of f keeps are a prefix of g, and with f ordered the same
// way the kept pairs form a staircase: a tile of pairs whose first pair fails
// is skipped whole, a walk along g stops at the first step where no pair
// passes.  The reorder is a stable device-wide radix sort of ~bits(|C|) (the
// bit pattern of a non-negative double orders like its value), with the terms
// dropped by a degree truncation (beyond nkeep) and NaN coefficients keyed
// last; then every term array follows the permutation.
#include "kr_internal.cuh"

namespace kr {

__global__ void __launch_bounds__(256) k_harmonic_pack(Prod* __restrict__ prods, const OpRef* __restrict__ ops) {
  const OpRef r = ops[blockIdx.y];
  const Prod& P = prods[r.prod];
  const Operand& op = r.which ? P.g : P.f;
  const int64_t n = op.n;
  const int hw = P.hwords;
  // balanced code: t = sum c_k t_k with t_k in [-R_k, R_k]; u = t + sum c_k R_k
  // has the digits t_k + R_k in the mixed radix of the widths 2 R_k + 1
  int64_t chi = 0;
  for (int k = 0; k < P.nt; ++k) chi += P.c[P.np + k] * (int64_t)(-P.omin[P.np + k]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t u = (uint64_t)(op.tcode[i] + chi);
    uint32_t pos[8], neg[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) pos[w] = neg[w] = 0x80008000u;   // bias of a zero multiplier
    int lane = 0;
    for (int k = 0; k < P.nt; ++k) {
      if (!((P.hmask >> k) & 1u)) continue;
      const uint64_t c = (uint64_t)P.c[P.np + k], w = (uint64_t)P.w[P.np + k];
      const int32_t t = (int32_t)((u / c) % w) + P.omin[P.np + k];
      const uint32_t sh = (lane & 1) * 16;
      const uint32_t keep = ~(0xffffu << sh);
      const int word = lane >> 1;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q == word) {
          pos[q] = (pos[q] & keep) | ((uint32_t)(t + 32768) << sh);
          neg[q] = (neg[q] & keep) | ((uint32_t)(32768 - t) << sh);
        }
      }
      ++lane;
    }
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      if (w < hw) {
        op.hpack[(int64_t)w * n + i] = pos[w];
        op.hpack[(int64_t)(hw + w) * n + i] = neg[w];
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_mag_keys(Prod* __restrict__ prods, const OpRef* __restrict__ ops) {
  const OpRef r = ops[blockIdx.y];
  const Prod& P = prods[r.prod];
  const Operand& op = r.which ? P.g : P.f;
  const double* C = (const double*)op.coef;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < op.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = fabs(C[i]);
    // NaN never passes the bound: it sorts last, with the dropped terms
    const bool last = i >= op.nkeep || a != a;
    op.mkey[i] = last ? ~0ull : ~(unsigned long long)__double_as_longlong(a);
    op.midx[i] = (uint64_t)i;
  }
}

// Term arrays in permuted order into mtmp (pass 0), then back (pass 1).
__global__ void __launch_bounds__(256) k_mag_move(Prod* __restrict__ prods, const OpRef* __restrict__ ops, int pass) {
  const OpRef r = ops[blockIdx.y];
  const Prod& P = prods[r.prod];
  const Operand& op = r.which ? P.g : P.f;
  const int64_t n = op.n;
  int64_t* tcode = (int64_t*)(op.mtmp);
  uint64_t* tcoef = (uint64_t*)(op.mtmp + 8 * n);
  int64_t* ttrig = (int64_t*)(op.mtmp + 16 * n);
  uint32_t* thp = (uint32_t*)(op.mtmp + 24 * n);
  uint8_t* tkind = op.mtmp + (P.nt > 0 ? 24 * n : 16 * n) + (P.htrunc ? 8 * (int64_t)P.hwords * n : 0);
  const int rows = P.htrunc ? 2 * P.hwords : 0;
  uint64_t* coef = (uint64_t*)op.coef;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    if (pass == 0) {
      const int64_t src = (int64_t)op.midx[q];
      tcode[q] = op.code[src];
      tcoef[q] = coef[src];
      if (P.nt > 0) {
        ttrig[q] = op.tcode[src];
        tkind[q] = op.kind[src];
      }
      for (int w = 0; w < rows; ++w) thp[(int64_t)w * n + q] = op.hpack[(int64_t)w * n + src];
    } else {
      op.code[q] = tcode[q];
      coef[q] = tcoef[q];
      if (P.nt > 0) {
        op.tcode[q] = ttrig[q];
        op.kind[q] = tkind[q];
      }
      for (int w = 0; w < rows; ++w) op.hpack[(int64_t)w * n + q] = thp[(int64_t)w * n + q];
    }
  }
}

static dim3 op_grid(int nops, int64_t max_n) {
  int64_t gx = (max_n + 255) / 256;
  if (gx > 1024) gx = 1024;
  if (gx < 1) gx = 1;
  return dim3((unsigned)gx, (unsigned)nops);
}

cudaError_t launch_harmonic_pack(Prod* dprods, const OpRef* dops, int nops, int64_t max_n, cudaStream_t s) {
  if (nops <= 0) return cudaSuccess;
  k_harmonic_pack<<<op_grid(nops, max_n), 256, 0, s>>>(dprods, dops);
  return cudaGetLastError();
}

cudaError_t launch_mag_keys(Prod* dprods, const OpRef* dops, int nops, int64_t max_n, cudaStream_t s) {
  if (nops <= 0) return cudaSuccess;
  k_mag_keys<<<op_grid(nops, max_n), 256, 0, s>>>(dprods, dops);
  return cudaGetLastError();
}

cudaError_t launch_mag_reorder(Prod* dprods, const OpRef* dops, int nops, int64_t max_n, cudaStream_t s) {
  if (nops <= 0) return cudaSuccess;
  k_mag_move<<<op_grid(nops, max_n), 256, 0, s>>>(dprods, dops, 0);
  k_mag_move<<<op_grid(nops, max_n), 256, 0, s>>>(dprods, dops, 1);
  return cudaGetLastError();
}

}  // namespace kr
