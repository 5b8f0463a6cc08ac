// An entry point that allocates nothing: the dense-path accumulation (block
// planning + shared-memory accumulation) with its scratch (the product
// descriptor, the task list and the task counters) in a file-scope device
// array instead of a context's arena.
//
// It exists for callers that cannot let a library call cudaMalloc or cudaFree:
// programs whose device memory is owned by their own allocator or a fixed
// budget, and code paths that must not pay for (or be stalled by) the device
// synchronisation an allocation or a free implies.  The caller passes every
// input and output buffer; the library's scratch is this array, which every
// GPU that loads the library holds until the process exits.
#include <algorithm>
#include <cstddef>
#include <mutex>

#include "kr_internal.cuh"

namespace kr {
int dense_max_split();

constexpr size_t STATIC_SCRATCH_BYTES = size_t(8) << 20;   // 8 MiB
constexpr int64_t STATIC_MAX_CODES = int64_t(1) << 24;     // W limit (2048 blocks of 8192 codes)
constexpr int64_t STATIC_BLOCK = 8192;
constexpr int STATIC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch per device, looked up once per device
// with that device current (in host code the symbol itself is only a host-side
// stand-in and must never be handed to a kernel).
static void* g_static_addr[STATIC_MAX_DEVICES];
static std::mutex g_static_mu;

static cudaError_t static_scratch(int device, unsigned char** out) {
  if (device < 0 || device >= STATIC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[device] = p;
  }
  *out = (unsigned char*)g_static_addr[device];
  return cudaSuccess;
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct StaticSmall {
  int32_t ids[2];
  int64_t block_begin[2];
};

// Stores the product descriptor and the planner's product list into the
// scratch array and clears the two task counters.  The descriptor travels as a
// kernel parameter (copied by value at launch), so nothing on the host stack
// has to outlive the call.
__global__ void k_static_setup(const Prod P, const StaticSmall small, Prod* __restrict__ dprod,
                               StaticSmall* __restrict__ dsmall, int64_t* __restrict__ dcnt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *dprod = P;
    *dsmall = small;
    dcnt[0] = 0;
    dcnt[1] = 0;
  }
}

// Checks the entry's preconditions on the device: both code arrays strictly
// ascending, inside [0, W), and the largest pair sum below W.  A violation
// marks the product invalid; the planner then makes no task and clears every
// block, so the output is all zeros and no kernel reads past the caller's
// arrays.
__global__ void __launch_bounds__(256) k_static_check(Prod* __restrict__ dprod, int64_t W) {
  const int64_t* F = dprod->f.code;
  const int64_t* G = dprod->g.code;
  const int64_t nf = dprod->f.n, ng = dprod->g.n;
  bool bad = false;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nf + ng;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t* A = q < nf ? F : G;
    const int64_t i = q < nf ? q : q - nf;
    const int64_t c = A[i];
    bad |= c < 0 || c >= W || (i > 0 && A[i - 1] >= c);
    if (q == 0) bad |= F[nf - 1] + G[ng - 1] >= W;   // both < W <= 2^24 here: no overflow
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&dprod->status, ST_INVALID);
}

}  // namespace kr

using namespace kr;

extern "C" kr_status kron_dense_product_static(const int64_t* fcode, const void* fcoef, int64_t nf,
                                               const int64_t* gcode, const void* gcoef, int64_t ng,
                                               kr_coef_t type, int64_t W, void* out,
                                               kr_stream stream) {
  if (W < 1 || nf < 0 || ng < 0 || !out || (type != KR_I64 && type != KR_F64)) return KR_ERR_INVALID;
  if ((nf > 0 && (!fcode || !fcoef)) || (ng > 0 && (!gcode || !gcoef))) return KR_ERR_INVALID;
  if (W > STATIC_MAX_CODES) return KR_ERR_TOO_LARGE;
  cudaStream_t s = (cudaStream_t)stream;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) { cudaGetLastError(); return KR_ERR_CUDA; }
  unsigned char* base = nullptr;
  if (static_scratch(device, &base) != cudaSuccess) { cudaGetLastError(); return KR_ERR_CUDA; }
  if (nf == 0 || ng == 0) {
    // no pair: the product is zero everywhere
    if (cudaMemsetAsync(out, 0, (size_t)W * 8, s) != cudaSuccess) { cudaGetLastError(); return KR_ERR_CUDA; }
    return KR_OK;
  }
  // Otherwise no clearing is needed: the planner clears every block that
  // several tasks (or none) add into, and a block with one task is written
  // whole by its flush.

  const int64_t S = std::min<int64_t>(STATIC_BLOCK, (W + 31) / 32 * 32);
  const int64_t nblocks = (W + S - 1) / S;
  const int64_t task_cap = nblocks * dense_max_split();
  // bucket index over g's codes (codes < W): at most 65536 buckets
  int gsh = 0;
  while (((W >> gsh) + 1) > 65535) ++gsh;
  const int64_t gidx_n = (W >> gsh) + 1;
  // layout: [Prod][ids, block_begin][counters][g index][tasks]
  const size_t off_ids = align256(sizeof(Prod));
  const size_t off_cnt = off_ids + align256(sizeof(StaticSmall));
  const size_t off_gidx = off_cnt + 256;
  const size_t off_tasks = off_gidx + align256((size_t)(gidx_n + 1) * sizeof(int32_t));
  const size_t need = off_tasks + (size_t)task_cap * sizeof(DenseTask);
  if (need > STATIC_SCRATCH_BYTES) return KR_ERR_TOO_LARGE;

  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  Prod P{};
  P.f.code = (int64_t*)fcode;
  P.f.coef = (void*)fcoef;
  P.f.n = nf;
  P.g.code = (int64_t*)gcode;
  P.g.coef = (void*)gcoef;
  P.g.n = ng;
  P.f.nkeep = nf;
  P.g.nkeep = ng;
  P.np = 1;
  P.nt = 0;
  P.f64 = type == KR_F64 ? 1 : 0;
  P.path = PATH_DENSE;
  P.krange = W;
  P.klo = 0;
  P.kspan = W;
  P.Wp = W;
  P.S = S;
  P.nblocks = nblocks;
  const double pairs = (double)nf * (double)ng;
  P.work_target = (int64_t)std::max(pairs / (double)(sms * 4), (double)(2 * S));
  P.dense = out;
  P.gidx = (int32_t*)(base + off_gidx);
  P.gidx_n = gidx_n;
  P.gshift = gsh;
  StaticSmall small{};
  small.ids[0] = 0;
  small.block_begin[0] = 0;
  small.block_begin[1] = nblocks;

  Prod* dprod = (Prod*)base;
  StaticSmall* dsmall = (StaticSmall*)(base + off_ids);
  int64_t* dcnt = (int64_t*)(base + off_cnt);
  DenseTask* dtasks = (DenseTask*)(base + off_tasks);
  k_static_setup<<<1, 32, 0, s>>>(P, small, dprod, dsmall, dcnt);
  if (cudaGetLastError() != cudaSuccess) return KR_ERR_CUDA;
  const int64_t check_blocks = std::min<int64_t>((nf + ng + 255) / 256, 4 * (int64_t)sms);
  k_static_check<<<(unsigned)check_blocks, 256, 0, s>>>(dprod, W);
  if (cudaGetLastError() != cudaSuccess) return KR_ERR_CUDA;
  if (launch_build_gindex(dprod, dsmall->ids, 1, ng, s) != cudaSuccess ||
      launch_dense_plan(dprod, dsmall->ids, dsmall->block_begin, 1, nblocks, dtasks, task_cap, dcnt, s) !=
          cudaSuccess) {
    cudaGetLastError();
    return KR_ERR_CUDA;
  }
  if (launch_dense_accum(dprod, dtasks, dcnt, task_cap, dcnt + 1, sms, S, s) != cudaSuccess) {
    cudaGetLastError();
    return KR_ERR_CUDA;
  }
  return KR_OK;
}
