// Peak-rate probes for the rooflines of the dense and the hash path.  The paper measures a
// multiplication by its clock cycles per monomial-by-monomial multiplication
// (Sec. 5) and calls a kernel optimal when that count approaches the cost of
// one coefficient multiply-add.  On the GPU the dense path's multiply-add is a
// shared-memory atomic accumulate of a product, so its ceiling is the
// chip-wide rate of conflict-free accumulates, measured here: plain 64-bit
// atomic adds (int64 or float64), and the int64 accumulate in the form the
// dense kernel uses (two 32-bit atomics with a carry).
#include <algorithm>

#include "kr_internal.cuh"

namespace kr {

constexpr int PK_THREADS = 512;
constexpr int PK_SLOTS = 8192;   // 64 KB of 8-byte counters
constexpr int PK_ITERS = 1024;

template <typename T>
__global__ void __launch_bounds__(PK_THREADS) k_probe_smem_atomic(T* __restrict__ sink, T inc) {
  __shared__ T s[PK_SLOTS];
  for (int i = threadIdx.x; i < PK_SLOTS; i += blockDim.x) s[i] = (T)0;
  __syncthreads();
  // consecutive lanes hit consecutive 8-byte words: no bank conflicts, no
  // two lanes of a warp on one address
  int a = threadIdx.x;
#pragma unroll 16
  for (int it = 0; it < PK_ITERS; ++it) {
    atomicAdd(&s[a], inc);
    a = (a + PK_THREADS) & (PK_SLOTS - 1);
  }
  __syncthreads();
  T acc = (T)0;
  for (int i = threadIdx.x; i < PK_SLOTS; i += blockDim.x) acc += s[i];
  if (acc == (T)-1) sink[blockIdx.x] = acc;   // keeps the work observable
}

template <>
__global__ void __launch_bounds__(PK_THREADS) k_probe_smem_atomic<int64_t>(int64_t* __restrict__ sink,
                                                                           int64_t inc) {
  __shared__ unsigned long long s[PK_SLOTS];
  for (int i = threadIdx.x; i < PK_SLOTS; i += blockDim.x) s[i] = 0;
  __syncthreads();
  int a = threadIdx.x;
#pragma unroll 16
  for (int it = 0; it < PK_ITERS; ++it) {
    atomicAdd(&s[a], (unsigned long long)inc);
    a = (a + PK_THREADS) & (PK_SLOTS - 1);
  }
  __syncthreads();
  unsigned long long acc = 0;
  for (int i = threadIdx.x; i < PK_SLOTS; i += blockDim.x) acc += s[i];
  if (acc == ~0ull) sink[blockIdx.x] = (int64_t)acc;
}

// The dense path's int64 accumulate as the kernel performs it: a 32-bit add
// of the low word returning the old value, the carry, and a 32-bit add of the
// high word (nonzero here, as for any negative addend).
__global__ void __launch_bounds__(PK_THREADS) k_probe_smem_split64(int64_t* __restrict__ sink, int64_t inc) {
  __shared__ uint32_t s[2 * PK_SLOTS];
  for (int i = threadIdx.x; i < 2 * PK_SLOTS; i += blockDim.x) s[i] = 0;
  __syncthreads();
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(s);
  int a = threadIdx.x;
#pragma unroll 16
  for (int it = 0; it < PK_ITERS; ++it) {
    smem_acc_split64(base + 4u * (uint32_t)a, 4u * PK_SLOTS, (uint64_t)inc);
    a = (a + PK_THREADS) & (PK_SLOTS - 1);
  }
  __syncthreads();
  uint64_t acc = 0;
  for (int i = threadIdx.x; i < PK_SLOTS; i += blockDim.x) acc += ((uint64_t)s[PK_SLOTS + i] << 32) | s[i];
  if (acc == ~0ull) sink[blockIdx.x] = (int64_t)acc;
}

// Chip-wide arithmetic rates of the coefficient multiply-add forms the
// kernels use: 64 x 64 -> 64-bit integer multiply-add (int64 coefficients),
// 32 x 32 -> 64-bit multiply-add (int64 coefficients that fit 32 bits), and
// float64 FMA.  Eight independent chains per thread, so that issue, not
// latency, sets the rate.
constexpr int ALU_THREADS = 256;
constexpr int ALU_ITERS = 4096;
constexpr int ALU_CHAINS = 8;

__global__ void __launch_bounds__(ALU_THREADS) k_probe_alu(int kind, int64_t* __restrict__ sink, int64_t seed) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t acc = 0;
  if (kind == 0) {
    uint64_t x[ALU_CHAINS];
#pragma unroll
    for (int c = 0; c < ALU_CHAINS; ++c) x[c] = (uint64_t)(seed + t * ALU_CHAINS + c) | 1ull;
    // x * x (both factors unknown to the compiler): a multiply by a constant
    // would let it fold consecutive steps into one
    for (int it = 0; it < ALU_ITERS; ++it) {
#pragma unroll
      for (int c = 0; c < ALU_CHAINS; ++c) x[c] = x[c] * x[c] + (uint64_t)(2 * c + 1);
    }
#pragma unroll
    for (int c = 0; c < ALU_CHAINS; ++c) acc ^= (int64_t)x[c];
  } else if (kind == 1) {
    int64_t x[ALU_CHAINS];
    int32_t y[ALU_CHAINS];
#pragma unroll
    for (int c = 0; c < ALU_CHAINS; ++c) { x[c] = seed + t + c; y[c] = (int32_t)(seed ^ (t + 7 * c)) | 1; }
    for (int it = 0; it < ALU_ITERS; ++it) {
#pragma unroll
      for (int c = 0; c < ALU_CHAINS; ++c) x[c] += (int64_t)y[c] * (int64_t)(int32_t)x[c];
    }
#pragma unroll
    for (int c = 0; c < ALU_CHAINS; ++c) acc ^= x[c];
  } else {
    double x[ALU_CHAINS];
#pragma unroll
    for (int c = 0; c < ALU_CHAINS; ++c) x[c] = 1.0 + 1e-9 * (double)((t + c) & 1023);
    const double m = 0.999999999, a = 1e-12;
    for (int it = 0; it < ALU_ITERS; ++it) {
#pragma unroll
      for (int c = 0; c < ALU_CHAINS; ++c) x[c] = fma(x[c], m, a);
    }
    double d = 0.0;
#pragma unroll
    for (int c = 0; c < ALU_CHAINS; ++c) d += x[c];
    acc = __double_as_longlong(d);
  }
  if (acc == seed) sink[t & 1023] = acc;   // keeps the work observable
}

}  // namespace kr

using namespace kr;

extern "C" double kr_probe_alu_rate(int32_t device, int32_t kind, int32_t reps) {
  if (kind < 0 || kind > 2) return -1.0;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return -1.0; }
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_alu, ALU_THREADS, 0);
  if (per_sm < 1) per_sm = 1;
  const int grid = sms * per_sm;
  int64_t* sink = nullptr;
  if (cudaMalloc(&sink, 1024 * 8) != cudaSuccess) { cudaGetLastError(); cudaSetDevice(prev); return -1.0; }
  double best = -1.0;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int r = 0; r < (reps > 0 ? reps : 5) + 1; ++r) {
    cudaEventRecord(a, 0);
    k_probe_alu<<<grid, ALU_THREADS>>>(kind, sink, 12345);
    cudaEventRecord(b, 0);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double ops = (double)grid * ALU_THREADS * ALU_ITERS * ALU_CHAINS;
    if (r > 0 && ms > 0.f) best = std::max(best, ops / (ms * 1e-3));
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (cudaGetLastError() != cudaSuccess) best = -1.0;
  cudaSetDevice(prev);
  return best;
}

extern "C" double kr_probe_smem_accumulate_rate(int32_t device, int32_t reps) {
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return -1.0; }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_smem_split64, PK_THREADS, 0);
  if (per_sm < 1) per_sm = 1;
  const int grid = sms * per_sm;
  void* sink = nullptr;
  double best = -1.0;
  cudaEvent_t a, b;
  if (cudaMalloc(&sink, (size_t)grid * 8) != cudaSuccess) { cudaGetLastError(); cudaSetDevice(prev); return -1.0; }
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int r = 0; r < (reps > 0 ? reps : 5) + 1; ++r) {
    cudaEventRecord(a, 0);
    k_probe_smem_split64<<<grid, PK_THREADS>>>((int64_t*)sink, -1);
    cudaEventRecord(b, 0);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double ops = (double)grid * PK_THREADS * PK_ITERS;
    if (r > 0 && ms > 0.f) best = std::max(best, ops / (ms * 1e-3));
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (cudaGetLastError() != cudaSuccess) best = -1.0;
  cudaSetDevice(prev);
  return best;
}

extern "C" double kr_probe_smem_atomic_rate(int32_t device, int32_t f64, int32_t reps) {
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return -1.0; }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  int per_sm = 0;
  if (f64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_smem_atomic<double>, PK_THREADS, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_smem_atomic<int64_t>, PK_THREADS, 0);
  if (per_sm < 1) per_sm = 1;
  const int grid = sms * per_sm;
  void* sink = nullptr;
  double best = -1.0;
  cudaEvent_t a, b;
  if (cudaMalloc(&sink, (size_t)grid * 8) != cudaSuccess) { cudaGetLastError(); cudaSetDevice(prev); return -1.0; }
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int r = 0; r < (reps > 0 ? reps : 5) + 1; ++r) {
    cudaEventRecord(a, 0);
    if (f64) k_probe_smem_atomic<double><<<grid, PK_THREADS>>>((double*)sink, 1.0);
    else k_probe_smem_atomic<int64_t><<<grid, PK_THREADS>>>((int64_t*)sink, 1);
    cudaEventRecord(b, 0);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double ops = (double)grid * PK_THREADS * PK_ITERS;
    if (r > 0 && ms > 0.f) best = std::max(best, ops / (ms * 1e-3));
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (cudaGetLastError() != cudaSuccess) best = -1.0;
  cudaSetDevice(prev);
  return best;
}

// The hash path's ceiling (Sec. 3.2: the highly sparse product accumulates
// into a hash table; here an open-addressing table in device memory): random
// insert-or-adds at a given table size and key count, in the insert routine
// of the polynomial kernel, with nothing else in the loop.
// Random float64 atomic adds into a key-indexed array of 8-byte slots (the
// Poisson dense path's accumulation): update u adds 1.0 at the hashed index
// of a key drawn from [0, distinct), four updates per thread in flight.
__global__ void __launch_bounds__(256) k_probe_array_add(double* __restrict__ a, uint64_t mask,
                                                         int64_t distinct, int64_t updates, uint64_t seed) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
  for (int64_t u0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; u0 < updates; u0 += stride) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t u = u0 + r;
      if (u < updates) {
        const uint64_t key = mix64(seed ^ (uint64_t)(u + 1)) % (uint64_t)distinct;
        atomicAdd(a + (mix64(key) & mask), 1.0);
      }
    }
  }
}

extern "C" double kr_probe_table_update_rate(int32_t device, int32_t log2_slots, int64_t distinct,
                                             int64_t updates, int32_t mode, int32_t reps) {
  if (log2_slots < 10 || log2_slots > (mode == 2 ? 33 : 30) || distinct < 1 || updates < 1 ||
      mode < 0 || mode > 2 || distinct > (int64_t(1) << log2_slots) * 7 / 10)
    return -1.0;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return -1.0; }
  const uint64_t slots = uint64_t(1) << log2_slots;
  const uint64_t bytes = slots * (mode == 2 ? 8 : 16);
  uint64_t* table = nullptr;
  unsigned long long* fails = nullptr;
  if (cudaMalloc(&table, bytes) != cudaSuccess || cudaMalloc(&fails, 8) != cudaSuccess) {
    cudaGetLastError();
    if (table) cudaFree(table);
    cudaSetDevice(prev);
    return -1.0;
  }
  double best = -1.0;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  unsigned long long hf = 0;
  for (int r = 0; r < (reps > 0 ? reps : 5) + 1; ++r) {
    cudaMemset(table, 0, bytes);
    cudaMemset(fails, 0, 8);
    cudaEventRecord(a, 0);
    if (mode == 2) {
      int sms = 0, per = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_probe_array_add, 256, 0);
      k_probe_array_add<<<sms * (per > 0 ? per : 1), 256>>>((double*)table, slots - 1, distinct, updates,
                                                           0x5eed5eedull);
    } else {
      launch_probe_table_update(table, slots, distinct, updates, mode, fails, 0);
    }
    cudaEventRecord(b, 0);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaMemcpy(&hf, fails, 8, cudaMemcpyDeviceToHost);
    if (hf) { best = -1.0; break; }
    if (r > 0 && ms > 0.f) best = std::max(best, (double)updates / (ms * 1e-3));
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(table);
  cudaFree(fails);
  if (cudaGetLastError() != cudaSuccess) best = -1.0;
  cudaSetDevice(prev);
  return best;
}
