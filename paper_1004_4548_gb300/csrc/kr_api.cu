// The C ABI of libkron (include/kron.h): context, scratch arenas, the
// multiplication pipeline, and the entry points.
//
// Pipeline of one call (one or many products):
//   range scan  -> [sync] host plan (coding box, path, sizes)
//   encode -> sort -> gather   (Kronecker codes of both operands, ascending)
//   dense:  block plan -> shared-memory accumulation -> flush
//   hash:   table inserts
//   compaction -> [sync] -> output sort (hash) -> decode into the caller's buffers
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include <chrono>

#include "kr_plan.h"

using namespace kr;

struct kr_ctx {
  int device = 0;
  int num_sms = 0;
  std::string err;
  void* in_arena = nullptr;
  size_t in_cap = 0;
  void* work = nullptr;
  size_t work_cap = 0;
  void* acc = nullptr;       // accumulators and outputs (phase B2)
  size_t acc_cap = 0;
  std::vector<Plan> plans;   // plans of the last pipeline run
  std::vector<void*> batch_blocks;   // result memory of the last kron_mul_batch
  // replay (prepared batches): run the device work of the saved plans again,
  // without host planning or synchronisation, so that it can be captured
  bool replay = false;
  // deferred counts: a single product whose caller decodes into device memory
  // may skip the synchronisations after phases B1 and B2 when nothing on the
  // host depends on them (no hash table to size or regrow); its term count
  // then stays on the device until the decode (ProdResult::n = -1)
  bool allow_deferred = false;
  // pointer attributes queried during the current call's staging
  std::unordered_map<const void*, cudaPointerAttributes> attr_memo;
  // a deferred dense polynomial product whose caller's outputs are all in
  // device memory or pinned host memory: the compaction decodes its terms
  // there (direct_done), and the output step only reads the count
  DirectOut direct{};
  bool direct_done = false;
  // split histogram (kron_split_hist): the pipeline stops after phase B1 and
  // samples the keys of product 0 into split_hist (host) instead
  int32_t split_nbins = 0;
  int64_t split_nsamples = 0;
  uint64_t split_seed = 0;
  int64_t* split_hist = nullptr;
  void* pinned = nullptr;
  size_t pinned_cap = 0;
  // product kept after the last multiplication (for kron_fetch_*)
  bool has_result = false;
  bool res_poisson = false;
  Prod res_prod{};
  Prod* res_dprod = nullptr;   // device copy of res_prod (in the work arena)
  const uint64_t* res_key = nullptr;
  const uint64_t* res_val = nullptr;
  int64_t res_n = 0;                    // -1 until a deferred count is read
  const int64_t* res_err = nullptr;     // deferred: the compaction's wait error word
  // stage timing (CUDA events on the call's stream) and launch counting
  bool profile = false;
  std::vector<cudaEvent_t> ev;
  std::vector<const char*> ev_name;
  int nev = 0;
  std::vector<double> stage_ms;
  std::vector<const char*> stage_name;
  int64_t launches = 0;
};

namespace {

struct CudaFail {
  cudaError_t e;
};

inline void ck(kr_ctx* ctx, cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();   // a failed allocation or launch must not be reported again by a later call
    throw CudaFail{e};
  }
}

}  // namespace

// The dynamic shared memory limit of a kernel is a property of the function
// for the whole process: a host thread lowering it between another thread's
// raise and that thread's launch would make the launch fail.  So the limit is
// only ever raised, under a lock, per function and device.
cudaError_t kr::raise_smem_limit(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limits;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limits[std::make_pair(func, dev)];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

namespace {

kr_status from_cuda(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? KR_ERR_OOM : KR_ERR_CUDA;
}

// pinned host inputs of at most this many values are read in place
#ifndef KR_ZERO_COPY_MAX
#define KR_ZERO_COPY_MAX (int64_t(1) << 18)
#endif

// Bump allocation over a base pointer; base == nullptr measures only.
struct Bump {
  char* base;
  size_t off = 0;
  explicit Bump(void* b) : base((char*)b) {}
  template <typename T>
  T* take(int64_t count, size_t align = 256) {
    off = (off + align - 1) / align * align;
    T* p = base ? (T*)(base + off) : nullptr;
    off += (size_t)std::max<int64_t>(count, 0) * sizeof(T);
    return p;
  }
};

void ensure(kr_ctx* ctx, void** buf, size_t* cap, size_t need, cudaStream_t s) {
  if (need <= *cap) return;
  ck(ctx, cudaStreamSynchronize(s), "sync before scratch growth");
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  size_t want = need + need / 4 + (1 << 20);
  ck(ctx, cudaMalloc(buf, want), "cudaMalloc scratch");
  *cap = want;
}

void ensure_pinned(kr_ctx* ctx, size_t need, cudaStream_t s) {
  if (need <= ctx->pinned_cap) return;
  ck(ctx, cudaStreamSynchronize(s), "sync before pinned growth");
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  ctx->pinned = nullptr;
  ctx->pinned_cap = 0;
  size_t want = need + need / 4 + (1 << 16);
  ck(ctx, cudaMallocHost(&ctx->pinned, want), "cudaMallocHost");
  ctx->pinned_cap = want;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A pointer through which this device's kernels may write p: p itself for
// device or managed memory, the mapped device address of pinned (page-locked)
// host memory, nullptr for pageable host memory.
void* device_view(void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  if (a.type == cudaMemoryTypeHost) return a.devicePointer;
  return nullptr;
}

// Records a stage boundary when profiling is on.
void mark(kr_ctx* ctx, cudaStream_t s, const char* name) {
  if (!ctx->profile) return;
  if (ctx->nev >= (int)ctx->ev.size()) {
    cudaEvent_t e;
    ck(ctx, cudaEventCreate(&e), "cudaEventCreate");
    ctx->ev.push_back(e);
    ctx->ev_name.push_back(nullptr);
  }
  ctx->ev_name[ctx->nev] = name;
  ck(ctx, cudaEventRecord(ctx->ev[ctx->nev], s), "cudaEventRecord");
  ctx->nev++;
}

// Host time of a planning step (profiling only), reported as a stage named
// "host_<step>" beside the device stages.
struct HostSpan {
  kr_ctx* ctx;
  const char* name;
  std::chrono::steady_clock::time_point t0;
  HostSpan(kr_ctx* c, const char* n) : ctx(c), name(n), t0(std::chrono::steady_clock::now()) {}
  void done() {
    if (!ctx || !ctx->profile) return;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    ctx->stage_ms.push_back(ms);
    ctx->stage_name.push_back(name);
    ctx = nullptr;
  }
};

// After a synchronisation: turn the recorded marks into per-stage times.
void collect_stages(kr_ctx* ctx) {
  if (!ctx->profile) return;
  for (int i = 1; i < ctx->nev; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev[i - 1], ctx->ev[i]) != cudaSuccess) {
      cudaGetLastError();
      ms = -1.f;
    }
    ctx->stage_ms.push_back(ms);
    ctx->stage_name.push_back(ctx->ev_name[i]);
  }
  ctx->nev = 0;
}

kr_status status_to_kr(uint32_t st) {
  if (st & ST_INVALID) return KR_ERR_INVALID;
  if (st & ST_RANGE) return KR_ERR_RANGE;
  if (st & ST_DUP) return KR_ERR_DUP;
  if (st & ST_TABLE_FULL) return KR_ERR_TABLE_FULL;
  if (st & ST_OUTCAP) return KR_ERR_CUDA;
  return KR_OK;
}

// Result of one product of a pipeline run.
struct ProdResult {
  kr_status st = KR_OK;
  int64_t n = 0;               // -1: the count is on the device (dprod->nout, dprod->status)
  const uint64_t* key = nullptr;
  const uint64_t* val = nullptr;
  Prod prod{};
  Prod* dprod = nullptr;
  const int64_t* err = nullptr;   // deferred: the compaction's wait error word (device)
};

// Host input of one product before staging (pointers may be host or device).
struct JobIn {
  bool poisson = false;
  bool f64 = false;
  int np = 0, nt = 0;
  const int32_t* fe = nullptr; const int32_t* ft = nullptr; const uint8_t* fk = nullptr;
  const void* fc = nullptr; int64_t nf = 0;
  const int32_t* ge = nullptr; const int32_t* gt = nullptr; const uint8_t* gk = nullptr;
  const void* gc = nullptr; int64_t ng = 0;
  kr_opts opts{};
};

// Stage host inputs into the input arena; returns device pointers.
template <typename T>
const T* stage(kr_ctx* ctx, Bump& b, const T* src, int64_t count, cudaStream_t s) {
  if (!src || count <= 0) return src;
  // one query per pointer and call (the layout passes stage every input twice)
  auto it = ctx->attr_memo.find((const void*)src);
  if (it == ctx->attr_memo.end()) {
    cudaPointerAttributes q;
    if (cudaPointerGetAttributes(&q, src) != cudaSuccess) {
      cudaGetLastError();
      q.type = cudaMemoryTypeUnregistered;
      q.devicePointer = nullptr;
    }
    it = ctx->attr_memo.emplace((const void*)src, q).first;
  }
  const cudaPointerAttributes& a = it->second;
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return src;
  // a small operand in pinned host memory is read by the kernels through its
  // device mapping (across the host link), with no staging copy
  if (a.type == cudaMemoryTypeHost && a.devicePointer && count <= KR_ZERO_COPY_MAX)
    return (const T*)a.devicePointer;
  T* dst = b.take<T>(count);
  if (b.base) ck(ctx, cudaMemcpyAsync(dst, src, (size_t)count * sizeof(T), cudaMemcpyHostToDevice, s),
                 "stage input");
  return dst;
}

// The pipeline over a set of products.  All products must have nf, ng >= 1.
//   A   staged inputs, range scan                       -> sync, host plan
//   B1  (work arena) encode, sort, gather, g index, HLL -> sync, table sizes
//   B2  (accumulator arena) zero, dense plan + accumulate, hash inserts,
//       compaction                                      -> sync
// A product whose table fills up is retried from B2 with a larger table.
void run_pipeline(kr_ctx* ctx, const std::vector<JobIn>& ins, cudaStream_t s,
                  std::vector<ProdResult>& res) {
  ctx->attr_memo.clear();
  const int nprod = (int)ins.size();
  res.assign(nprod, ProdResult());
  const int nops = 2 * nprod;
  std::vector<Job> jobs(nprod);
  HostSpan plan_span(nullptr, "host_plan");
  // ---------------- phase A: staged inputs, metadata, range scan
  if (ctx->replay) {
    for (int p = 0; p < nprod; ++p) res[p].st = ctx->plans[p].st;
  } else {
  Prod* dprods = nullptr;
  OpRef* dops = nullptr;
  int32_t* dranges = nullptr;
  char* drs = nullptr;
  unsigned int* ddone = nullptr;   // the range scan's per-operand counters, uploaded as zeros
  int64_t max_n = 1;
  for (const JobIn& in : ins) max_n = std::max(max_n, std::max(in.nf, in.ng));
  for (int pass = 0; pass < 2; ++pass) {
    Bump b(pass ? ctx->in_arena : nullptr);
    for (int p = 0; p < nprod; ++p) {
      const JobIn& in = ins[p];
      Job& J = jobs[p];
      J = Job();
      J.poisson = in.poisson;
      J.f64 = in.f64;
      J.np = in.np;
      J.nt = in.nt;
      J.opts = in.opts;
      J.f.n = in.nf;
      J.g.n = in.ng;
      J.f.e = stage(ctx, b, in.fe, (int64_t)in.np * in.nf, s);
      J.g.e = stage(ctx, b, in.ge, (int64_t)in.np * in.ng, s);
      J.f.c = (const void*)stage(ctx, b, (const uint64_t*)in.fc, in.nf, s);
      J.g.c = (const void*)stage(ctx, b, (const uint64_t*)in.gc, in.ng, s);
      if (in.poisson) {
        J.f.t = stage(ctx, b, in.ft, (int64_t)in.nt * in.nf, s);
        J.g.t = stage(ctx, b, in.gt, (int64_t)in.nt * in.ng, s);
        J.f.k = stage(ctx, b, in.fk, in.nf, s);
        J.g.k = stage(ctx, b, in.gk, in.ng, s);
      }
    }
    dprods = b.take<Prod>(nprod);
    dops = b.take<OpRef>(nops);
    ddone = b.take<unsigned int>(nops);
    dranges = b.take<int32_t>((int64_t)nops * RANGE_STRIDE);
    drs = b.take<char>((int64_t)range_scan_scratch_bytes(nops, max_n));
    if (!pass) ensure(ctx, &ctx->in_arena, &ctx->in_cap, b.off + 1, s);
  }
  ensure_pinned(ctx, (sizeof(Prod) + 2 * sizeof(OpRef) + 8 + 2 * RANGE_STRIDE * 4) * (size_t)nprod + 65536, s);
  {
    Bump hp(ctx->pinned);
    Prod* hprods = hp.take<Prod>(nprod);
    OpRef* hops = hp.take<OpRef>(nops);
    unsigned int* hdone = hp.take<unsigned int>(nops);
    memset(hdone, 0, sizeof(unsigned int) * (size_t)nops);
    int32_t* hranges = hp.take<int32_t>((int64_t)nops * RANGE_STRIDE);
    for (int p = 0; p < nprod; ++p) {
      Prod P{};
      P.f = jobs[p].f;
      P.g = jobs[p].g;
      P.np = jobs[p].np;
      P.nt = jobs[p].nt;
      P.f64 = jobs[p].f64;
      if (jobs[p].opts.truncate && P.np > 0) {
        // the range scan also measures the degree range of the mask
        uint32_t m = jobs[p].opts.trunc_mask ? jobs[p].opts.trunc_mask : 0xffffffffu;
        if (P.np < 32) m &= (1u << P.np) - 1u;
        P.gmask = m;
      }
      hprods[p] = P;
      hops[2 * p] = OpRef{p, 0};
      hops[2 * p + 1] = OpRef{p, 1};
    }
    // products, operand list and counters, laid out alike on both sides: one copy
    ck(ctx, cudaMemcpyAsync(dprods, hprods, (size_t)((char*)(ddone + nops) - (char*)dprods),
                            cudaMemcpyHostToDevice, s), "upload");
    mark(ctx, s, "begin");
    ck(ctx, launch_range_scan(dprods, dops, nops, max_n, drs, ddone, dranges, s), "range scan");
    ctx->launches += 1;
    mark(ctx, s, "range_scan");
    ck(ctx, cudaMemcpyAsync(hranges, dranges, sizeof(int32_t) * nops * RANGE_STRIDE,
                            cudaMemcpyDeviceToHost, s), "download ranges");
    ck(ctx, cudaStreamSynchronize(s), "sync ranges");
    collect_stages(ctx);
    // ---------------- host planning
    plan_span = HostSpan(ctx, "host_plan");
    std::vector<Plan> plans_tmp(nprod);
    ctx->plans.assign(nprod, Plan());
    for (int p = 0; p < nprod; ++p) {
      plan_product(jobs[p], hranges + (2 * p) * RANGE_STRIDE, hranges + (2 * p + 1) * RANGE_STRIDE,
                   ctx->num_sms, &ctx->plans[p]);
      res[p].st = ctx->plans[p].st;
    }
  }
  }   // phase A
  std::vector<Plan>& plans = ctx->plans;
  // dense_ids: polynomial products on the dense path (output-block tasks);
  // hash_ids: everything accumulated by tiles of term pairs (hash products and
  // Poisson products on the dense path); hll_ids: products with a hash table
  std::vector<int> live_ids, dense_ids, hash_ids, hll_ids;
  for (int p = 0; p < nprod; ++p) {
    if (plans[p].st != KR_OK) continue;
    if (plans[p].empty) {   // truncated to nothing: a zero product
      res[p].n = 0;
      res[p].prod = plans[p].p;
      continue;
    }
    live_ids.push_back(p);
    const bool block = plans[p].p.path == PATH_DENSE && plans[p].p.nt == 0;
    (block ? dense_ids : hash_ids).push_back(p);
    if (plans[p].p.path == PATH_HASH) hll_ids.push_back(p);
  }
  const int nlive = (int)live_ids.size();
  if (nlive == 0) return;
  std::vector<int> local(nprod, -1);
  for (int q = 0; q < nlive; ++q) local[live_ids[q]] = q;
  std::vector<int32_t> h_dense_local, h_hash_local;
  for (int p : dense_ids) h_dense_local.push_back(local[p]);
  for (int p : hash_ids) h_hash_local.push_back(local[p]);
  std::vector<int32_t> h_hll_local;
  for (int p : hll_ids) h_hll_local.push_back(local[p]);
  // deferred: one product, no hash table (nothing to size from the estimate or
  // to regrow), not a prepared or split run.  Its whole plan (phases B1 and
  // B2) goes to the device in one copy, and no step waits for the device
  // before the output count is read.
  const bool deferred = ctx->allow_deferred && !ctx->replay && !ctx->split_hist && nlive == 1 &&
                        nprod == 1 && hll_ids.empty();
  // ---------------- phase B1 layout (work arena)
  int64_t dense_tasks_total = 0, nblocks_total = 0, scan_b1 = 0, max_ng_dense = 0, max_S = 0;
  for (int p : dense_ids) {
    dense_tasks_total += plans[p].dense_task_cap;
    nblocks_total += plans[p].p.nblocks;
    max_ng_dense = std::max(max_ng_dense, plans[p].p.g.n);
    max_S = std::max(max_S, plans[p].p.S);
  }
  for (int p : live_ids) scan_b1 = std::max(scan_b1, radix_scan_entries(plans[p].radix_sort_n));
  struct B1 {
    Prod* lprods; OpRef* oplists; int32_t* dense_ids; int64_t* block_begin; int32_t* hash_ids;
    int64_t* task_begin; int64_t* scan; DenseTask* tasks; uint32_t* hll; size_t hll_bytes;
    int32_t* hll_ids; int64_t* hll_task_begin; int64_t* chunk_begin; unsigned long long* split; char* up_end;
  } A{};
  for (int pass = 0; pass < 2; ++pass) {
    Bump b(pass ? ctx->work : nullptr);
    // the arrays uploaded from the host first and contiguous: one copy
    A.lprods = b.take<Prod>(nlive);
    A.oplists = b.take<OpRef>(5 * (int64_t)nops);
    A.dense_ids = b.take<int32_t>((int64_t)dense_ids.size() + 1);
    A.block_begin = b.take<int64_t>((int64_t)dense_ids.size() + 1);
    A.hash_ids = b.take<int32_t>((int64_t)hash_ids.size() + 1);
    A.task_begin = b.take<int64_t>((int64_t)hash_ids.size() + 1);
    A.hll_ids = b.take<int32_t>((int64_t)hll_ids.size() + 1);
    A.hll_task_begin = b.take<int64_t>((int64_t)hll_ids.size() + 1);
    A.chunk_begin = b.take<int64_t>((int64_t)nlive + 1);   // used by a deferred product
    A.up_end = b.base ? b.base + b.off : nullptr;
    A.scan = b.take<int64_t>(scan_b1 + 1);
    A.tasks = b.take<DenseTask>(dense_tasks_total);
    A.hll = b.take<uint32_t>((int64_t)hll_ids.size() * HLL_M);
    A.hll_bytes = sizeof(uint32_t) * hll_ids.size() * HLL_M;
    A.split = ctx->split_hist ? b.take<unsigned long long>(ctx->split_nbins) : nullptr;
    for (int q = 0; q < (int)hll_ids.size(); ++q)
      if (pass) plans[hll_ids[q]].p.hll = A.hll + (int64_t)q * HLL_M;
    for (int p : live_ids) {
      Plan& pl = plans[p];
      for (int which = 0; which < 2; ++which) {
        Operand& op = which ? pl.p.g : pl.p.f;
        const int64_t n = op.n;
        uint64_t* ka = b.take<uint64_t>(n);
        uint64_t* kb = b.take<uint64_t>(n);
        uint64_t* ia = b.take<uint64_t>(n);
        uint64_t* ib = b.take<uint64_t>(n);
        op.skey = ka;
        op.sidx = ia;
        op.skey2 = kb;
        op.sidx2 = ib;
        const int passes = which ? pl.passes_g : pl.passes_f;
        if (op.sort_method == SORT_RADIX && passes % 2 == 0) { op.skey2 = ka; op.sidx2 = ia; }
        op.code = b.take<int64_t>(n);
        op.coef = (void*)b.take<uint64_t>(n);
        if (pl.p.nt > 0) {
          op.tcode = b.take<int64_t>(n);
          op.kind = b.take<uint8_t>(n);
        }
        if (pl.p.htrunc) op.hpack = b.take<uint32_t>(2 * (int64_t)pl.p.hwords * n);
        if (pl.p.ctrunc) {
          op.mkey = b.take<uint64_t>(n);
          op.midx = b.take<uint64_t>(n);
          op.mkey2 = b.take<uint64_t>(n);
          op.midx2 = b.take<uint64_t>(n);
          op.mtmp = b.take<unsigned char>(n * mag_tmp_bytes_per_term(pl.p));
        }
      }
      if (pl.p.path == PATH_DENSE && pl.p.nt == 0) {
        pl.p.gidx = b.take<int32_t>(pl.p.gidx_n + 1);
        pl.p.g.code32 = b.take<int32_t>(pl.p.g.n);
      }
    }
    if (!pass) ensure(ctx, &ctx->work, &ctx->work_cap, b.off + 1, s);
  }
  std::vector<int64_t> h_block_begin(dense_ids.size() + 1, 0), h_task_begin(hash_ids.size() + 1, 0);
  for (size_t q = 0; q < dense_ids.size(); ++q)
    h_block_begin[q + 1] = h_block_begin[q] + plans[dense_ids[q]].p.nblocks;
  for (size_t q = 0; q < hash_ids.size(); ++q) {
    plans[hash_ids[q]].p.task_begin = h_task_begin[q];
    h_task_begin[q + 1] = h_task_begin[q] + plans[hash_ids[q]].p.ntasks;
  }
  std::vector<int64_t> h_hll_task_begin(hll_ids.size() + 1, 0);
  for (size_t q = 0; q < hll_ids.size(); ++q)
    h_hll_task_begin[q + 1] = h_hll_task_begin[q] + plans[hll_ids[q]].p.ntasks;
  // ---------------- phase B2 layout (accumulation arena): table sizes, output
  // room, chunk ranges, accumulators; a deferred product lays it out now
  struct B2 {
    int64_t* chunk_begin; int64_t* counts; int64_t* scan; int64_t* bins; uint64_t *okey, *oval, *okey2, *oval2;
    int64_t* counters; uint64_t* cstat; char* zero; size_t zero_bytes;
  } Z{};
  int64_t out_total = 0, nchunks_total = 0, bins_total = 0, scan_b2 = 0, max_hash_out = 0;
  std::vector<int64_t> h_chunk_begin(nlive + 1, 0);
  auto layout_b2 = [&]() {
    out_total = 0, nchunks_total = 0, bins_total = 0, scan_b2 = 0, max_hash_out = 0;
    for (int p : hll_ids) {
      Plan& pl = plans[p];
      finish_hash_sizes(ins[p].opts, &pl);
      max_hash_out = std::max(max_hash_out, pl.out_cap);
      const int64_t nb = order_bins(pl.p.kspan);
      if (order_buckets(pl.p.kspan) <= ORDER_MAX_BUCKETS)
        bins_total = std::max(bins_total, order_buckets_scratch(pl.p.kspan, pl.out_cap));
      if (pl.p.kspan <= ORDER_BITMAP_MAX)
        bins_total = std::max(bins_total, (order_bitmap_bytes(pl.p.kspan) + 7) / 8);
      else if (nb <= ORDER_MAX_BINS) bins_total = std::max(bins_total, order_bins_scratch(pl.p.kspan));
      else scan_b2 = std::max(scan_b2, radix_scan_entries(pl.out_cap));
    }
    std::fill(h_chunk_begin.begin(), h_chunk_begin.end(), 0);
    for (int q = 0; q < nlive; ++q) {
      Plan& pl = plans[live_ids[q]];
      pl.p.out_cap = pl.out_cap;
      pl.p.out_begin = out_total;
      pl.p.chunk_begin = nchunks_total;
      h_chunk_begin[q] = nchunks_total;
      out_total += pl.out_cap;
      nchunks_total += pl.p.nchunks;
    }
    h_chunk_begin[nlive] = nchunks_total;
    Z = B2{};
    for (int pass = 0; pass < 2; ++pass) {
      Bump b(pass ? ctx->acc : nullptr);
      Z.chunk_begin = b.take<int64_t>(nlive + 1);
      Z.counts = b.take<int64_t>(nchunks_total + 1);
      Z.scan = b.take<int64_t>(std::max(scan_b2, scan_scratch_entries(nchunks_total)) + 1);
      Z.bins = b.take<int64_t>(bins_total);
      Z.okey = b.take<uint64_t>(out_total);
      Z.oval = b.take<uint64_t>(out_total);
      // ordering scratch: one hash product at a time
      Z.okey2 = b.take<uint64_t>(max_hash_out);
      Z.oval2 = b.take<uint64_t>(max_hash_out);
      b.off = (b.off + 255) / 256 * 256;
      const size_t zero_start = b.off;
      Z.zero = b.base ? b.base + zero_start : nullptr;
      Z.counters = b.take<int64_t>(4);   // dense task queue (2), compaction ticket and error flag
      Z.cstat = b.take<uint64_t>(nchunks_total + 1);
      for (int p : live_ids) {
        Plan& pl = plans[p];
        if (pl.p.path == PATH_DENSE && pl.p.nt > 0) pl.p.dense = (void*)b.take<uint64_t>(pl.p.kspan);
        else if (pl.p.path != PATH_DENSE) pl.p.table = b.take<uint64_t>(2 * pl.p.slots);
      }
      Z.zero_bytes = b.off - zero_start;
      // the block-accumulated arrays are cleared by the dense planning kernel
      // (the blocks that its flushes do not write whole)
      for (int p : dense_ids) plans[p].p.dense = (void*)b.take<uint64_t>(plans[p].p.kspan);
      if (!pass) ensure(ctx, &ctx->acc, &ctx->acc_cap, b.off + 1, s);
    }
  };
  if (deferred) {
    layout_b2();
    Z.chunk_begin = A.chunk_begin;   // uploaded with phase B1's plan
  }
  std::vector<OpRef> all, bm, bt;
  // large operands with key ranges of at most CL_MAX_BITS, in a call with
  // few of them: the cluster front end (encode, rank and gather by CL_CTAS
  // CTAs each); the rest: one CTA each (bitmap or bitonic) or the radix sort
  std::vector<OpRef> cl;
  int ncand = 0;
  int64_t cl_range = 0;
  auto cluster_fit = [](const Operand& op) {
    return op.sort_method == SORT_CLUSTER || (op.n >= CL_MIN_N && op.key_range <= CL_MAX_BITS);
  };
  for (int q = 0; q < nlive; ++q)
    for (int which = 0; which < 2; ++which)
      ncand += cluster_fit(which ? plans[live_ids[q]].p.g : plans[live_ids[q]].p.f);
  for (int q = 0; q < nlive; ++q) {
    Prod& P = plans[live_ids[q]].p;
    for (int which = 0; which < 2; ++which) {
      Operand& op = which ? P.g : P.f;
      if (ncand <= CL_MAX_OPS && cluster_fit(op)) op.sort_method = SORT_CLUSTER;
      if (op.sort_method == SORT_CLUSTER) {
        cl.push_back(OpRef{q, which});
        cl_range = std::max(cl_range, op.key_range);
        continue;
      }
      all.push_back(OpRef{q, which});
      if (op.sort_method == SORT_BITMAP) bm.push_back(OpRef{q, which});
      if (op.sort_method == SORT_BITONIC) bt.push_back(OpRef{q, which});
    }
  }
  bool gindex_needed = false;
  for (int p : dense_ids) gindex_needed |= plans[p].p.g.sort_method != SORT_CLUSTER;
  // operands of products truncated by harmonic order (packed multipliers) and
  // by coefficient magnitude (reorder by decreasing |C|)
  std::vector<OpRef> hops, mops;
  int64_t max_n_h = 0, max_n_m = 0;
  for (int q = 0; q < nlive; ++q) {
    const Prod& P = plans[live_ids[q]].p;
    for (int which = 0; which < 2; ++which) {
      const int64_t n = which ? P.g.n : P.f.n;
      if (P.htrunc) { hops.push_back(OpRef{q, which}); max_n_h = std::max(max_n_h, n); }
      if (P.ctrunc) { mops.push_back(OpRef{q, which}); max_n_m = std::max(max_n_m, n); }
    }
  }
  std::vector<OpRef> lists = all;
  lists.insert(lists.end(), bm.begin(), bm.end());
  lists.insert(lists.end(), bt.begin(), bt.end());
  lists.insert(lists.end(), cl.begin(), cl.end());
  lists.insert(lists.end(), hops.begin(), hops.end());
  lists.insert(lists.end(), mops.begin(), mops.end());
  ensure_pinned(ctx, sizeof(Prod) * (size_t)(nlive + 1) * 3 + sizeof(OpRef) * lists.size() +
                         16 * (h_block_begin.size() + h_task_begin.size() + 4 * (size_t)nlive) +
                         (size_t)(A.up_end - (char*)A.lprods) + 65536, s);
  Bump hb(ctx->pinned);
  Prod* hl = hb.take<Prod>(nlive);   // download area for phase B1's results
  {
    // the plan and every list, laid out in pinned memory as on the device,
    // then one copy (a handful of small copies cost more host time than data)
    char* dbase = (char*)A.lprods;
    const size_t span = (size_t)(A.up_end - dbase);
    char* st = hb.take<char>((int64_t)span);
    auto put = [&](const void* dst, const void* src, size_t bytes) {
      if (bytes) memcpy(st + ((const char*)dst - dbase), src, bytes);
    };
    for (int q = 0; q < nlive; ++q) hl[q] = plans[live_ids[q]].p;
    put(A.lprods, hl, sizeof(Prod) * nlive);
    put(A.oplists, lists.data(), sizeof(OpRef) * lists.size());
    put(A.dense_ids, h_dense_local.data(), 4 * h_dense_local.size());
    put(A.block_begin, h_block_begin.data(), 8 * h_block_begin.size());
    put(A.hash_ids, h_hash_local.data(), 4 * h_hash_local.size());
    put(A.task_begin, h_task_begin.data(), 8 * h_task_begin.size());
    put(A.hll_ids, h_hll_local.data(), 4 * h_hll_local.size());
    put(A.hll_task_begin, h_hll_task_begin.data(), 8 * h_hll_task_begin.size());
    put(A.chunk_begin, h_chunk_begin.data(), 8 * h_chunk_begin.size());
    ck(ctx, cudaMemcpyAsync(dbase, st, span, cudaMemcpyHostToDevice, s), "upload plan");
  }
  const OpRef* d_all = A.oplists;
  const OpRef* d_bm = d_all + all.size();
  const OpRef* d_bt = d_bm + bm.size();
  const OpRef* d_cl = d_bt + bt.size();
  const OpRef* d_h = d_cl + cl.size();
  const OpRef* d_m = d_h + hops.size();
  // ---------------- phase B1 device work
  plan_span.done();
  mark(ctx, s, "plan_upload");
  if (A.hll_bytes) ck(ctx, cudaMemsetAsync(A.hll, 0, A.hll_bytes, s), "memset hll");
  if (!cl.empty()) {
    ck(ctx, launch_front_cluster(A.lprods, d_cl, (int)cl.size(), cl_range, s), "cluster front end");
    ctx->launches += 1;
    mark(ctx, s, "front");
  }
  if (!all.empty()) {
    ck(ctx, launch_encode(A.lprods, d_all, (int)all.size(), s), "encode");
    ctx->launches += 1;
    mark(ctx, s, "encode");
  }
  if (!bm.empty()) {
    int64_t mx = 0;
    for (auto& r : bm) {
      const Prod& P = plans[live_ids[r.prod]].p;
      mx = std::max(mx, ((r.which ? P.g : P.f).key_range + 1023) / 1024);
    }
    ck(ctx, launch_sort_small(A.lprods, d_bm, (int)bm.size(), SORT_BITMAP, (size_t)mx * 36 * 4 + 64, s),
       "bitmap sort");
    ctx->launches += 1;
  }
  if (!bt.empty()) {
    int64_t mx = 0;
    for (auto& r : bt) {
      const Prod& P = plans[live_ids[r.prod]].p;
      mx = std::max(mx, (r.which ? P.g : P.f).n);
    }
    ck(ctx, launch_sort_small(A.lprods, d_bt, (int)bt.size(), SORT_BITONIC, (size_t)mx * 8, s),
       "bitonic sort");
    ctx->launches += 1;
  }
  for (int q = 0; q < nlive; ++q) {
    const Plan& pl = plans[live_ids[q]];
    for (int which = 0; which < 2; ++which) {
      const Operand& op = which ? pl.p.g : pl.p.f;
      if (op.sort_method != SORT_RADIX) continue;
      const int bits = bits_for((uint64_t)op.key_range);
      bool in_tmp = false;
      // keys in skey/sidx; the result ends in skey2/sidx2 (aliases skey when passes are even)
      uint64_t* tk = op.skey2 == op.skey ? (uint64_t*)op.code : op.skey2;
      uint64_t* tv = op.sidx2 == op.sidx ? (uint64_t*)op.coef : op.sidx2;
      ck(ctx, radix_sort_pairs(op.skey, op.sidx, tk, tv, op.n, bits, A.scan, s, &in_tmp),
         "radix sort operand");
      ctx->launches += 3 * ((bits + 7) / 8);
    }
  }
  if (!all.empty()) {
    mark(ctx, s, "sort");
    ck(ctx, launch_gather(A.lprods, d_all, (int)all.size(), s), "gather");
    ctx->launches += 1;
    mark(ctx, s, "gather");
  }
  if (!hops.empty()) {
    ck(ctx, launch_harmonic_pack(A.lprods, d_h, (int)hops.size(), max_n_h, s), "harmonic pack");
    ctx->launches += 1;
  }
  if (!mops.empty()) {
    ck(ctx, launch_mag_keys(A.lprods, d_m, (int)mops.size(), max_n_m, s), "magnitude keys");
    ctx->launches += 1;
    for (const OpRef& r : mops) {
      const Operand& op = r.which ? plans[live_ids[r.prod]].p.g : plans[live_ids[r.prod]].p.f;
      bool in_tmp = false;
      ck(ctx, radix_sort_pairs(op.mkey, op.midx, op.mkey2, op.midx2, op.n, 64, A.scan, s, &in_tmp),
         "magnitude sort");
      ctx->launches += 3 * 8;
      if (in_tmp)
        ck(ctx, cudaMemcpyAsync(op.midx, op.midx2, sizeof(uint64_t) * (size_t)op.n, cudaMemcpyDeviceToDevice, s),
           "magnitude order");
    }
    ck(ctx, launch_mag_reorder(A.lprods, d_m, (int)mops.size(), max_n_m, s), "magnitude reorder");
    ctx->launches += 2;
    mark(ctx, s, "magnitude_order");
  }
  if (gindex_needed) {
    ck(ctx, launch_build_gindex(A.lprods, A.dense_ids, (int)dense_ids.size(), max_ng_dense, s), "g index");
    ctx->launches += 1;
  }
  if (!hll_ids.empty()) {
    bool need_hll = false;
    for (int p : hll_ids) need_hll |= ins[p].opts.table_slots <= 0;
    if (ctx->replay) need_hll = false;   // table sizes are fixed by the prepared run
    if (need_hll) {
      ck(ctx, launch_hll(A.lprods, A.hll_ids, A.hll_task_begin, (int)hll_ids.size(), ctx->num_sms * 8, s),
         "hll");
      ck(ctx, launch_hll_estimate(A.lprods, A.hll_ids, (int)hll_ids.size(), s), "hll estimate");
      ctx->launches += 2;
      mark(ctx, s, "hll");
    }
  }
  if (!ctx->replay && !deferred) {
    ck(ctx, cudaMemcpyAsync(hl, A.lprods, sizeof(Prod) * nlive, cudaMemcpyDeviceToHost, s), "download");
    ck(ctx, cudaStreamSynchronize(s), "sync b1");
    collect_stages(ctx);
    for (int q = 0; q < nlive; ++q) {
      Plan& pl = plans[live_ids[q]];
      pl.p.status = hl[q].status;
      pl.p.hll_est = hl[q].hll_est;
      pl.p.f.nkeep = hl[q].f.nkeep;
      pl.p.g.nkeep = hl[q].g.nkeep;
    }
  }
  if (ctx->split_hist) {
    // kron_split_hist: sample the output keys of the (one) product and stop
    const size_t hb_bytes = sizeof(unsigned long long) * (size_t)ctx->split_nbins;
    ck(ctx, cudaMemsetAsync(A.split, 0, hb_bytes, s), "memset histogram");
    ck(ctx, launch_split_sample(A.lprods, 0, ctx->split_nbins, ctx->split_nsamples, ctx->split_seed,
                                A.split, s), "split sample");
    ctx->launches += 1;
    ck(ctx, cudaMemcpyAsync(ctx->split_hist, A.split, hb_bytes, cudaMemcpyDeviceToHost, s), "download");
    ck(ctx, cudaStreamSynchronize(s), "sync histogram");
    const int p = live_ids[0];
    res[p].st = status_to_kr(plans[p].p.status);
    res[p].prod = plans[p].p;
    return;
  }
  // ---------------- phase B2, repeated for products whose table filled up
  std::vector<int> regrows(nprod, 0);
  bool first_b2 = true;
  for (;;) {
    HostSpan b2_span(ctx, "host_b2");
    if (!(deferred && first_b2)) layout_b2();
    first_b2 = false;
    // a replay is captured without synchronisation: its B2 staging must not
    // overwrite B1's, so it continues after it
    Bump hb2 = (ctx->replay || deferred) ? hb : Bump(ctx->pinned);
    Prod* hl2 = hb2.take<Prod>(nlive);
    if (!deferred) {   // a deferred product's phase B2 plan went up with phase B1's
      for (int q = 0; q < nlive; ++q) hl2[q] = plans[live_ids[q]].p;
      ck(ctx, cudaMemcpyAsync(A.lprods, hl2, sizeof(Prod) * nlive, cudaMemcpyHostToDevice, s), "upload plan");
      int64_t* st = hb2.take<int64_t>(nlive + 1);
      memcpy(st, h_chunk_begin.data(), 8 * (size_t)(nlive + 1));
      ck(ctx, cudaMemcpyAsync(Z.chunk_begin, st, 8 * (size_t)(nlive + 1), cudaMemcpyHostToDevice, s),
         "upload chunks");
    }
    b2_span.done();
    mark(ctx, s, "plan_upload");
    ck(ctx, cudaMemsetAsync(Z.zero, 0, Z.zero_bytes, s), "memset accumulators");
    mark(ctx, s, "zero_accumulators");
    if (!dense_ids.empty()) {
      ck(ctx, launch_dense_plan(A.lprods, A.dense_ids, A.block_begin, (int)dense_ids.size(),
                                nblocks_total, A.tasks, dense_tasks_total, Z.counters, s),
         "dense plan");
      ctx->launches += 1;
      mark(ctx, s, "dense_plan");
      ck(ctx, launch_dense_accum(A.lprods, A.tasks, Z.counters, dense_tasks_total, Z.counters + 1,
                                 ctx->num_sms, max_S, s),
         "dense accumulate");
      ctx->launches += 1;
      mark(ctx, s, "dense_accum");
    }
    if (!hash_ids.empty()) {
      bool any_poly = false, any_pseries = false, any_trunc = false;
      for (int p : hash_ids) {
        const Prod& P = plans[p].p;
        if (P.ctrunc || P.htrunc) any_trunc = true;
        else (P.nt > 0 ? any_pseries : any_poly) = true;
      }
      ck(ctx, launch_hash_insert(A.lprods, A.hash_ids, A.task_begin, (int)hash_ids.size(), any_poly,
                                 any_pseries, any_trunc, ctx->num_sms * 8, s),
         "hash insert");
      ctx->launches += (any_poly ? 1 : 0) + (any_pseries ? 1 : 0) + (any_trunc ? 1 : 0);
      mark(ctx, s, "hash_insert");
    }
    DirectOut direct{};
    if (deferred && ctx->direct.coef) {
      const Prod& P0 = plans[live_ids[0]].p;
      // polynomials only: on the Poisson product's 596 M terms a decode pass per
      // chunk slowed the compaction more than the separate decode costs
      if (P0.path == PATH_DENSE && P0.nt == 0) {
        direct = ctx->direct;
        ctx->direct_done = true;
      }
    }
    int compact_launches = 0;
    ck(ctx, launch_compact(A.lprods, nlive, Z.chunk_begin, nchunks_total, Z.counts, Z.cstat, Z.counters + 2,
                           Z.scan, Z.okey, Z.oval, out_total, s, direct, &compact_launches),
       "compaction");
    ctx->launches += compact_launches;
    mark(ctx, s, "compact");
    if (deferred) {
      // the count, the status and the position (0: the only product) stay on
      // the device; the decode reads them there
      const int p = live_ids[0];
      res[p].st = KR_OK;
      res[p].n = -1;
      res[p].prod = plans[p].p;
      res[p].dprod = A.lprods;
      res[p].key = Z.okey;
      res[p].val = Z.oval;
      res[p].err = Z.counters + 3;
      return;
    }
    if (ctx->replay) {
      // counts and positions of the prepared run (the replayed compaction
      // writes the same ones; the caller verifies after the launch)
      for (int q = 0; q < nlive; ++q) hl2[q] = plans[live_ids[q]].p;
    } else {
      ck(ctx, cudaMemcpyAsync(hl2, A.lprods, sizeof(Prod) * nlive, cudaMemcpyDeviceToHost, s), "download");
      int64_t* herr = hb2.take<int64_t>(1);
      ck(ctx, cudaMemcpyAsync(herr, Z.counters + 3, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "download");
      ck(ctx, cudaStreamSynchronize(s), "sync results");
      collect_stages(ctx);
      if (*herr) {   // a bounded wait of the compaction gave up: no result is reliable
        ctx->err = "compaction: a wait for a preceding chunk timed out";
        for (int q = 0; q < nlive; ++q) res[live_ids[q]].st = KR_ERR_TIMEOUT;
        return;
      }
    }
    bool retry = false;
    for (int q = 0; q < nlive; ++q) {
      const int p = live_ids[q];
      Prod& P = hl2[q];
      plans[p].p.nout = P.nout;
      plans[p].p.out_start = P.out_start;
      if (!ctx->replay && (P.status & ST_OUTCAP) && !(P.status & ~ST_OUTCAP) && !plans[p].outcap_full) {
        // the estimate fell short: rerun with room for a full table
        plans[p].outcap_full = true;
        plans[p].p.status = 0;
        retry = true;
        continue;
      }
      if (!ctx->replay && (P.status & ST_TABLE_FULL)) {
        const int mr = ins[p].opts.max_regrow;
        const int allowed = mr > 0 ? mr : (mr < 0 ? 0 : 4);
        const int64_t bound = plans[p].bound_slots;
        if (regrows[p] < allowed && P.slots < bound) {
          regrows[p]++;
          plans[p].slots_override = regrows[p] == allowed ? bound : std::min(P.slots * 4, bound);
          plans[p].p.status = 0;
          retry = true;
          continue;
        }
      }
      res[p].st = status_to_kr(P.status);
      res[p].n = P.nout;
      res[p].prod = P;
      res[p].dprod = A.lprods + q;
      res[p].key = Z.okey + P.out_start;
      res[p].val = Z.oval + P.out_start;
      if (P.nout > P.out_cap) res[p].st = KR_ERR_CUDA;
    }
    if (retry) continue;   // phase B2 again, with the grown tables
    // ---------------- hash outputs: order by key
    mark(ctx, s, "begin");
    for (int q = 0; q < nlive; ++q) {
      const int p = live_ids[q];
      ProdResult& r = res[p];
      if (r.st != KR_OK || r.prod.path != PATH_HASH || r.n < 2 || ins[p].opts.unsorted) continue;
      uint64_t* k = Z.okey + r.prod.out_start;
      uint64_t* v = Z.oval + r.prod.out_start;
      uint64_t* k2 = Z.okey2;
      uint64_t* v2 = Z.oval2;
      // compacted keys are relative to the key window: they lie in [0, kspan)
      // large outputs over wide code ranges: a two-pass partition by fine
      // bucket, each bucket then ranked by a shared-memory bitmap (on the
      // 596 M-term Poisson product: 24 ms, against 77 ms for a one-pass
      // bucket scatter, 97 ms for one bitmap in device memory and 129 ms for
      // the device-wide radix sort)
      if (r.n >= ORDER_BUCKET_MIN_N && r.prod.kspan > ORDER_BUCKET_MIN_RANGE &&
          order_buckets(r.prod.kspan) <= ORDER_MAX_BUCKETS) {
        ck(ctx, order_by_buckets(k, v, k2, v2, r.n, r.prod.kspan, Z.bins, s), "output order");
        ctx->launches += 5;
      } else if (r.prod.kspan <= ORDER_BITMAP_MAX) {
        ck(ctx, order_by_bitmap(k, v, k2, v2, r.n, r.prod.kspan, Z.bins, s), "output order");
        ctx->launches += 4;
        if (nlive == 1) {
          // the only product: its ordered terms stay in the second arrays (context
          // scratch, kept until the next call like the first)
          r.key = k2;
          r.val = v2;
        } else {
          ck(ctx, cudaMemcpyAsync(k, k2, 8 * (size_t)r.n, cudaMemcpyDeviceToDevice, s), "copy");
          ck(ctx, cudaMemcpyAsync(v, v2, 8 * (size_t)r.n, cudaMemcpyDeviceToDevice, s), "copy");
        }
      } else if (order_bins(r.prod.kspan) <= ORDER_MAX_BINS) {
        ck(ctx, order_by_bins(k, v, k2, v2, r.n, r.prod.kspan, Z.bins, s), "output order");
        ctx->launches += 4;
      } else {
        const int bits = bits_for((uint64_t)r.prod.kspan);
        bool in_tmp = false;
        ck(ctx, radix_sort_pairs(k, v, k2, v2, r.n, bits, Z.scan, s, &in_tmp), "output sort");
        ctx->launches += 3 * ((bits + 7) / 8);
        if (in_tmp && nlive == 1) {
          r.key = k2;
          r.val = v2;
        } else if (in_tmp) {
          ck(ctx, cudaMemcpyAsync(k, k2, 8 * (size_t)r.n, cudaMemcpyDeviceToDevice, s), "copy");
          ck(ctx, cudaMemcpyAsync(v, v2, 8 * (size_t)r.n, cudaMemcpyDeviceToDevice, s), "copy");
        }
      }
    }
    mark(ctx, s, "output_sort");
    return;
  }
}

struct CtxGuard {
  kr_ctx* c;
  int prev = -1;
  explicit CtxGuard(kr_ctx* ctx) : c(ctx) {
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
  }
  ~CtxGuard() {
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  }
};

template <typename F>
kr_status guarded(kr_ctx* ctx, F body) {
  if (!ctx) return KR_ERR_INVALID;
  try {
    CtxGuard g(ctx);
    return body();
  } catch (const CudaFail& f) {
    return from_cuda(f.e);
  } catch (const std::bad_alloc&) {
    ctx->err = "host allocation failed";
    return KR_ERR_OOM;
  } catch (...) {
    ctx->err = "unexpected exception";
    return KR_ERR_CUDA;
  }
}

// copy n values from device src to dst (device or host)
void copy_out(kr_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!dst || bytes == 0) return;
  ck(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s), "copy output");
}

kr_status settle_deferred(kr_ctx* ctx, cudaStream_t s);

kr_status emit_poly(kr_ctx* ctx, kr_poly_out* h, cudaStream_t s) {
  const Prod& P = ctx->res_prod;
  const int64_t n = ctx->res_n;
  h->nterms = n;
  for (int k = 0; k < KR_MAXV; ++k) { h->omin[k] = 0; h->omax[k] = 0; }
  for (int k = 0; k < P.np; ++k) {
    h->omin[k] = P.omin[k];
    h->omax[k] = P.omin[k] + P.w[k] - 1;
  }
  if (P.graded) {   // a truncated product: the range of the variable itself
    h->omin[P.gvar] = P.gvar_min;
    h->omax[P.gvar] = P.gvar_max;
  }
  if (n < 0 && ctx->direct_done) {
    // the compaction has decoded the terms into the caller's arrays (device
    // memory or pinned host memory): read the count and report it
    const kr_status st = settle_deferred(ctx, s);
    h->nterms = st == KR_OK ? ctx->res_n : 0;
    if (st != KR_OK) return st;
    return ctx->res_n > h->capacity ? KR_ERR_CAPACITY : KR_OK;
  }
  if (n < 0) {
    const bool exps_dev = !h->exps || is_device_ptr(h->exps);
    const bool codes_dev = !h->codes || is_device_ptr(h->codes);
    if (exps_dev && codes_dev && is_device_ptr(h->coef)) {
      // deferred count, device outputs: decode up to the capacity, read the
      // count, then report it
      ck(ctx, launch_decode_poly(ctx->res_dprod, 0, ctx->res_key, h->capacity, h->exps, h->capacity, h->codes, s,
                                 true, ctx->res_val, (uint64_t*)h->coef),
         "decode");
      ctx->launches += 1;
      mark(ctx, s, "decode");
      const kr_status st = settle_deferred(ctx, s);
      h->nterms = st == KR_OK ? ctx->res_n : 0;
      if (st != KR_OK) return st;
      return ctx->res_n > h->capacity ? KR_ERR_CAPACITY : KR_OK;
    }
    // deferred count, host outputs: decode into device scratch with room for
    // every term the product can have (at most the capacity), read the count,
    // then copy that many terms.  The scratch is the input arena: the decode
    // runs after every kernel that reads the staged inputs, and a growth of
    // the arena waits for the stream first.
    const int64_t room = std::max<int64_t>(0, std::min<int64_t>(h->capacity, P.out_cap));
    ensure(ctx, &ctx->in_arena, &ctx->in_cap, (size_t)room * (P.np * 4 + 8) + 1024, s);
    Bump b(ctx->in_arena);
    int32_t* exps_tmp = b.take<int32_t>(room * P.np);
    int64_t* codes_tmp = b.take<int64_t>(room);
    int32_t* ex = h->exps ? (exps_dev ? h->exps : exps_tmp) : nullptr;
    int64_t* cd = h->codes ? (codes_dev ? h->codes : codes_tmp) : nullptr;
    const int64_t ld = (h->exps && !exps_dev) ? room : h->capacity;
    ck(ctx, launch_decode_poly(ctx->res_dprod, 0, ctx->res_key, room, ex, ld, cd, s, true), "decode");
    ctx->launches += 1;
    mark(ctx, s, "decode");
    const kr_status st = settle_deferred(ctx, s);
    h->nterms = st == KR_OK ? ctx->res_n : 0;
    if (st != KR_OK) return st;
    const int64_t m = ctx->res_n;
    if (m > h->capacity) return KR_ERR_CAPACITY;
    if (m > 0) {
      if (h->exps && !exps_dev)
        for (int k = 0; k < P.np; ++k)
          copy_out(ctx, h->exps + (int64_t)k * h->capacity, exps_tmp + (int64_t)k * room, (size_t)m * 4, s);
      if (h->codes && !codes_dev) copy_out(ctx, h->codes, codes_tmp, (size_t)m * 8, s);
      copy_out(ctx, h->coef, ctx->res_val, (size_t)m * 8, s);
      mark(ctx, s, "copy_out");
      ck(ctx, cudaStreamSynchronize(s), "sync output");
      collect_stages(ctx);
    }
    return KR_OK;
  }
  if (n > h->capacity) return KR_ERR_CAPACITY;
  if (n == 0) return KR_OK;
  const bool exps_dev = is_device_ptr(h->exps);
  const bool codes_dev = is_device_ptr(h->codes);
  int32_t* exps_tmp = nullptr;
  int64_t* codes_tmp = nullptr;
  int64_t ld = h->capacity;
  if ((h->exps && !exps_dev) || (h->codes && !codes_dev)) {
    // decode into the input arena, then copies (one per variable row)
    ensure(ctx, &ctx->in_arena, &ctx->in_cap, (size_t)n * (P.np * 4 + 8) + 1024, s);
    Bump b(ctx->in_arena);
    exps_tmp = b.take<int32_t>((int64_t)n * P.np);
    codes_tmp = b.take<int64_t>(n);
    if (!(h->exps && !exps_dev)) exps_tmp = nullptr;
    else ld = n;
  }
  int32_t* ex = h->exps ? (exps_dev ? h->exps : exps_tmp) : nullptr;
  int64_t* cd = h->codes ? (codes_dev ? h->codes : codes_tmp) : nullptr;
  ck(ctx, launch_decode_poly(ctx->res_dprod, 0, ctx->res_key, n, ex, ld, cd, s), "decode");
  ctx->launches += 1;
  mark(ctx, s, "decode");
  if (exps_tmp) {
    for (int k = 0; k < P.np; ++k)
      copy_out(ctx, h->exps + (int64_t)k * h->capacity, exps_tmp + (int64_t)k * n, (size_t)n * 4, s);
  }
  if (h->codes && !codes_dev) copy_out(ctx, h->codes, codes_tmp, (size_t)n * 8, s);
  copy_out(ctx, h->coef, ctx->res_val, (size_t)n * 8, s);
  mark(ctx, s, "copy_out");
  ck(ctx, cudaStreamSynchronize(s), "sync output");
  collect_stages(ctx);
  return KR_OK;
}

kr_status emit_pseries(kr_ctx* ctx, kr_pseries_out* h, cudaStream_t s) {
  const Prod& P = ctx->res_prod;
  const int64_t n = ctx->res_n;
  h->nterms = n;
  if (n < 0) {
    // deferred count (device outputs only), as in emit_poly
    ck(ctx, launch_decode_pseries(ctx->res_dprod, 0, ctx->res_key, h->capacity, h->exps, h->trig, h->kind,
                                  h->capacity, h->codes, s, true, ctx->res_val, (uint64_t*)h->coef),
       "decode");
    ctx->launches += 1;
    mark(ctx, s, "decode");
    const kr_status st = settle_deferred(ctx, s);
    h->nterms = st == KR_OK ? ctx->res_n : 0;
    if (st != KR_OK) return st;
    return ctx->res_n > h->capacity ? KR_ERR_CAPACITY : KR_OK;
  }
  if (n > h->capacity) return KR_ERR_CAPACITY;
  if (n == 0) return KR_OK;
  const bool any_host = (h->exps && !is_device_ptr(h->exps)) || (h->trig && !is_device_ptr(h->trig)) ||
                        (h->kind && !is_device_ptr(h->kind)) || (h->codes && !is_device_ptr(h->codes));
  if (!any_host) {
    ck(ctx, launch_decode_pseries(ctx->res_dprod, 0, ctx->res_key, n, h->exps, h->trig, h->kind,
                                  h->capacity, h->codes, s),
       "decode");
    ctx->launches += 1;
  } else {
    ensure(ctx, &ctx->in_arena, &ctx->in_cap, (size_t)n * (4 * (P.np + P.nt) + 1 + 8) + 1024, s);
    Bump b(ctx->in_arena);
    int32_t* ex = b.take<int32_t>((int64_t)n * P.np);
    int32_t* tr = b.take<int32_t>((int64_t)n * P.nt);
    uint8_t* kd = b.take<uint8_t>(n);
    int64_t* cd = b.take<int64_t>(n);
    ck(ctx, launch_decode_pseries(ctx->res_dprod, 0, ctx->res_key, n, ex, tr, kd, n, cd, s), "decode");
    ctx->launches += 1;
    if (h->exps)
      for (int k = 0; k < P.np; ++k)
        copy_out(ctx, h->exps + (int64_t)k * h->capacity, ex + (int64_t)k * n, (size_t)n * 4, s);
    if (h->trig)
      for (int k = 0; k < P.nt; ++k)
        copy_out(ctx, h->trig + (int64_t)k * h->capacity, tr + (int64_t)k * n, (size_t)n * 4, s);
    copy_out(ctx, h->kind, kd, (size_t)n, s);
    copy_out(ctx, h->codes, cd, (size_t)n * 8, s);
  }
  mark(ctx, s, "decode");
  copy_out(ctx, h->coef, ctx->res_val, (size_t)n * 8, s);
  mark(ctx, s, "copy_out");
  ck(ctx, cudaStreamSynchronize(s), "sync output");
  collect_stages(ctx);
  return KR_OK;
}

void keep_result(kr_ctx* ctx, const ProdResult& r, bool poisson) {
  ctx->has_result = true;
  ctx->res_poisson = poisson;
  ctx->res_prod = r.prod;
  ctx->res_dprod = r.dprod;
  ctx->res_key = r.key;
  ctx->res_val = r.val;
  ctx->res_n = r.n;
  ctx->res_err = r.err;
}

// After a deferred run: the device-side count, status and wait error of the
// kept product, read once its decode has been queued.  Synchronises.
kr_status settle_deferred(kr_ctx* ctx, cudaStream_t s) {
  ensure_pinned(ctx, 4096, s);
  Bump hp(ctx->pinned);
  Prod* hp_prod = hp.take<Prod>(1);
  int64_t* herr = hp.take<int64_t>(1);
  ck(ctx, cudaMemcpyAsync(hp_prod, ctx->res_dprod, sizeof(Prod), cudaMemcpyDeviceToHost, s), "download");
  ck(ctx, cudaMemcpyAsync(herr, ctx->res_err, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "download");
  ck(ctx, cudaStreamSynchronize(s), "sync output");
  collect_stages(ctx);
  if (*herr) {
    ctx->err = "compaction: a wait for a preceding chunk timed out";
    ctx->has_result = false;
    return KR_ERR_TIMEOUT;
  }
  if (hp_prod->status) {
    ctx->has_result = false;
    return status_to_kr(hp_prod->status);
  }
  ctx->res_n = hp_prod->nout;
  return KR_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

kr_status kr_ctx_create(int32_t device, kr_ctx** out) {
  if (!out) return KR_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return KR_ERR_CUDA;
  }
  kr_ctx* c = new (std::nothrow) kr_ctx;
  if (!c) return KR_ERR_OOM;
  c->device = device;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaSetDevice(prev);
  if (c->num_sms <= 0) c->num_sms = 1;
  *out = c;
  return KR_OK;
}

void kr_ctx_destroy(kr_ctx* ctx) {
  if (!ctx) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->in_arena) cudaFree(ctx->in_arena);
  if (ctx->work) cudaFree(ctx->work);
  if (ctx->acc) cudaFree(ctx->acc);
  for (void* b : ctx->batch_blocks) cudaFree(b);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  cudaSetDevice(prev);
  delete ctx;
}

const char* kr_last_error(const kr_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

int64_t kr_ctx_scratch_bytes(const kr_ctx* ctx) {
  return ctx ? (int64_t)(ctx->in_cap + ctx->work_cap + ctx->acc_cap) : 0;
}

kr_status kr_ctx_trim(kr_ctx* ctx) {
  if (!ctx) return KR_ERR_INVALID;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  cudaGetLastError();   // report only what the trim itself meets
  cudaDeviceSynchronize();
  if (ctx->in_arena) cudaFree(ctx->in_arena);
  if (ctx->work) cudaFree(ctx->work);
  if (ctx->acc) cudaFree(ctx->acc);
  for (void* b : ctx->batch_blocks) cudaFree(b);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  ctx->in_arena = ctx->work = ctx->acc = ctx->pinned = nullptr;
  ctx->in_cap = ctx->work_cap = ctx->acc_cap = ctx->pinned_cap = 0;
  ctx->batch_blocks.clear();
  ctx->has_result = false;
  const cudaError_t e = cudaGetLastError();
  cudaSetDevice(prev);
  return e == cudaSuccess ? KR_OK : KR_ERR_CUDA;
}

kr_status kr_ctx_set_profiling(kr_ctx* ctx, int32_t enable) {
  if (!ctx) return KR_ERR_INVALID;
  ctx->profile = enable != 0;
  ctx->nev = 0;
  return KR_OK;
}

int32_t kr_ctx_stage_count(const kr_ctx* ctx) { return ctx ? (int32_t)ctx->stage_ms.size() : 0; }

kr_status kr_ctx_stage(const kr_ctx* ctx, int32_t i, const char** name, double* ms) {
  if (!ctx || i < 0 || i >= (int32_t)ctx->stage_ms.size()) return KR_ERR_INVALID;
  if (name) *name = ctx->stage_name[i];
  if (ms) *ms = ctx->stage_ms[i];
  return KR_OK;
}

int64_t kr_ctx_launch_count(const kr_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* kron_strerror(kr_status s) {
  switch (s) {
    case KR_OK: return "ok";
    case KR_ERR_INVALID: return "invalid argument";
    case KR_ERR_RANGE: return "exponent outside the coding box";
    case KR_ERR_OVERFLOW: return "code range exceeds 2^63-1";
    case KR_ERR_DUP: return "duplicate term in an input series";
    case KR_ERR_OOM: return "out of memory";
    case KR_ERR_CAPACITY: return "output capacity too small";
    case KR_ERR_TIMEOUT: return "bounded device wait timed out";
    case KR_ERR_CUDA: return "CUDA error";
    case KR_ERR_TABLE_FULL: return "hash table full after the allowed regrowths";
    case KR_ERR_TOO_LARGE: return "problem exceeds the fixed limit of this entry point";
  }
  return "unknown status";
}

kr_status kron_plan(const int32_t* emin, const int32_t* emax, int32_t nvars, int64_t* cvec_out,
                    int64_t* range_out) {
  if (!emin || !emax || nvars < 1 || nvars > KR_MAXV) return KR_ERR_INVALID;
  int64_t w[KR_MAXV], c[KR_MAXV], W = 0;
  for (int k = 0; k < nvars; ++k) {
    if (emin[k] > emax[k]) return KR_ERR_INVALID;
    w[k] = (int64_t)emax[k] - (int64_t)emin[k] + 1;
  }
  kr_status st = coding_vector(w, nvars, c, &W);
  if (st != KR_OK) return st;
  if (cvec_out)
    for (int k = 0; k < nvars; ++k) cvec_out[k] = c[k];
  if (range_out) *range_out = W;
  return KR_OK;
}

// The standalone coding kernels keep each variable's width and offset in 32
// bits, as the product path's output boxes do: every w_k must be at most
// 2^31 - 1.
static bool widths_fit_int32(const int32_t* emin, const int32_t* emax, int32_t nvars) {
  for (int k = 0; k < nvars; ++k)
    if ((int64_t)emax[k] - (int64_t)emin[k] + 1 > (int64_t)INT32_MAX) return false;
  return true;
}

kr_status kron_encode(kr_ctx* ctx, const int32_t* exps, int64_t n, int32_t nvars, const int32_t* emin,
                      const int32_t* emax, int64_t* codes_out, kr_stream stream) {
  if (n < 0 || (n > 0 && (!exps || !codes_out))) return KR_ERR_INVALID;
  int64_t c[KR_MAXV], W;
  kr_status st = kron_plan(emin, emax, nvars, c, &W);
  if (st != KR_OK) return st;
  if (!widths_fit_int32(emin, emax, nvars)) return KR_ERR_OVERFLOW;
  if (n == 0) return KR_OK;
  return guarded(ctx, [&]() -> kr_status {
    cudaStream_t s = (cudaStream_t)stream;
    Bump b(nullptr);
    b.take<uint32_t>(1);
    const bool in_dev = is_device_ptr(exps), out_dev = is_device_ptr(codes_out);
    if (!in_dev) b.take<int32_t>(n * nvars);
    if (!out_dev) b.take<int64_t>(n);
    ensure(ctx, &ctx->in_arena, &ctx->in_cap, b.off, s);
    Bump a(ctx->in_arena);
    uint32_t* dst = a.take<uint32_t>(1);
    const int32_t* e = exps;
    if (!in_dev) {
      int32_t* t = a.take<int32_t>(n * nvars);
      ck(ctx, cudaMemcpyAsync(t, exps, (size_t)n * nvars * 4, cudaMemcpyHostToDevice, s), "copy");
      e = t;
    }
    int64_t* out = out_dev ? codes_out : a.take<int64_t>(n);
    ck(ctx, cudaMemsetAsync(dst, 0, 4, s), "memset");
    ck(ctx, launch_encode_box(e, n, nvars, emin, emax, c, out, dst, s), "encode");
    if (!out_dev) ck(ctx, cudaMemcpyAsync(codes_out, out, (size_t)n * 8, cudaMemcpyDeviceToHost, s), "copy");
    uint32_t hst = 0;
    ck(ctx, cudaMemcpyAsync(&hst, dst, 4, cudaMemcpyDeviceToHost, s), "status");
    ck(ctx, cudaStreamSynchronize(s), "sync");
    return hst ? KR_ERR_RANGE : KR_OK;
  });
}

kr_status kron_decode(kr_ctx* ctx, const int64_t* codes, int64_t n, int32_t nvars, const int32_t* emin,
                      const int32_t* emax, int32_t* exps_out, kr_stream stream) {
  if (n < 0 || (n > 0 && (!codes || !exps_out))) return KR_ERR_INVALID;
  int64_t c[KR_MAXV], W;
  kr_status st = kron_plan(emin, emax, nvars, c, &W);
  if (st != KR_OK) return st;
  if (!widths_fit_int32(emin, emax, nvars)) return KR_ERR_OVERFLOW;
  if (n == 0) return KR_OK;
  int32_t w[KR_MAXV];
  for (int k = 0; k < nvars; ++k) w[k] = emax[k] - emin[k] + 1;
  return guarded(ctx, [&]() -> kr_status {
    cudaStream_t s = (cudaStream_t)stream;
    const bool in_dev = is_device_ptr(codes), out_dev = is_device_ptr(exps_out);
    Bump b(nullptr);
    b.take<uint32_t>(1);
    if (!in_dev) b.take<int64_t>(n);
    if (!out_dev) b.take<int32_t>(n * nvars);
    ensure(ctx, &ctx->in_arena, &ctx->in_cap, b.off, s);
    Bump a(ctx->in_arena);
    uint32_t* dst = a.take<uint32_t>(1);
    const int64_t* cd = codes;
    if (!in_dev) {
      int64_t* t = a.take<int64_t>(n);
      ck(ctx, cudaMemcpyAsync(t, codes, (size_t)n * 8, cudaMemcpyHostToDevice, s), "copy");
      cd = t;
    }
    int32_t* out = out_dev ? exps_out : a.take<int32_t>(n * nvars);
    ck(ctx, cudaMemsetAsync(dst, 0, 4, s), "memset");
    ck(ctx, launch_decode_box(cd, n, nvars, emin, w, c, W, out, dst, s), "decode");
    if (!out_dev)
      ck(ctx, cudaMemcpyAsync(exps_out, out, (size_t)n * nvars * 4, cudaMemcpyDeviceToHost, s), "copy");
    uint32_t hst = 0;
    ck(ctx, cudaMemcpyAsync(&hst, dst, 4, cudaMemcpyDeviceToHost, s), "status");
    ck(ctx, cudaStreamSynchronize(s), "sync");
    return hst ? KR_ERR_RANGE : KR_OK;
  });
}

kr_status poly_mul(kr_ctx* ctx, const kr_poly* f, const kr_poly* g, kr_poly_out* h, const kr_opts* opts,
                   kr_stream stream) {
  if (!ctx || !f || !g || !h) return KR_ERR_INVALID;
  if (f->nvars < 1 || f->nvars > KR_MAXV || g->nvars != f->nvars || h->nvars != f->nvars) return KR_ERR_INVALID;
  if (f->type != g->type || (f->type != KR_I64 && f->type != KR_F64)) return KR_ERR_INVALID;
  if (f->nterms < 0 || g->nterms < 0 || h->capacity < 0) return KR_ERR_INVALID;
  if (f->nterms >= INT32_MAX || g->nterms >= INT32_MAX) return KR_ERR_INVALID;
  if ((f->nterms > 0 && (!f->exps || !f->coef)) || (g->nterms > 0 && (!g->exps || !g->coef)))
    return KR_ERR_INVALID;
  if (h->capacity > 0 && !h->coef) return KR_ERR_INVALID;
  return guarded(ctx, [&]() -> kr_status {
    cudaStream_t s = (cudaStream_t)stream;
    ctx->has_result = false;
    ctx->stage_ms.clear();
    ctx->stage_name.clear();
    ctx->nev = 0;
    if (f->nterms == 0 || g->nterms == 0) {
      h->nterms = 0;
      for (int k = 0; k < KR_MAXV; ++k) { h->omin[k] = 0; h->omax[k] = 0; }
      return KR_OK;
    }
    JobIn in;
    in.poisson = false;
    in.f64 = f->type == KR_F64;
    in.np = f->nvars;
    in.nt = 0;
    in.fe = f->exps; in.fc = f->coef; in.nf = f->nterms;
    in.ge = g->exps; in.gc = g->coef; in.ng = g->nterms;
    if (opts) in.opts = *opts;
    std::vector<ProdResult> res;
    // the term count may stay on the device until the decode (host outputs:
    // until the decode into scratch, whose terms are then copied); with every
    // output in device memory the compaction may decode into it directly
    ctx->allow_deferred = true;
    ctx->direct = DirectOut{};
    ctx->direct_done = false;
    if (h->capacity > 0) {
      // device memory, or pinned host memory through its device mapping (the
      // GPU writes the terms across the host link; no copies afterwards)
      void* cf = device_view(h->coef);
      void* ex = h->exps ? device_view(h->exps) : nullptr;
      void* cd = h->codes ? device_view(h->codes) : nullptr;
      if (cf && (!h->exps || ex) && (!h->codes || cd)) {
        ctx->direct.exps = (int32_t*)ex;
        ctx->direct.codes = (int64_t*)cd;
        ctx->direct.coef = (uint64_t*)cf;
        ctx->direct.ld = h->capacity;
        ctx->direct.cap = h->capacity;
      }
    }
    try {
      run_pipeline(ctx, {in}, s, res);
    } catch (...) {
      ctx->allow_deferred = false;
      ctx->direct = DirectOut{};
      ctx->direct_done = false;
      throw;
    }
    ctx->allow_deferred = false;
    ctx->direct = DirectOut{};
    if (res[0].st != KR_OK) {
      ctx->direct_done = false;
      return res[0].st;
    }
    keep_result(ctx, res[0], false);
    const kr_status st = emit_poly(ctx, h, s);
    ctx->direct_done = false;
    return st;
  });
}

kr_status poisson_mul(kr_ctx* ctx, const kr_pseries* f, const kr_pseries* g, kr_pseries_out* h,
                      const kr_opts* opts, kr_stream stream) {
  if (!ctx || !f || !g || !h) return KR_ERR_INVALID;
  if (f->ntrig < 1 || f->npoly < 0 || f->npoly + f->ntrig > KR_MAXV) return KR_ERR_INVALID;
  if (g->npoly != f->npoly || g->ntrig != f->ntrig || h->npoly != f->npoly || h->ntrig != f->ntrig)
    return KR_ERR_INVALID;
  if (f->nterms < 0 || g->nterms < 0 || h->capacity < 0) return KR_ERR_INVALID;
  if (f->nterms >= INT32_MAX || g->nterms >= INT32_MAX) return KR_ERR_INVALID;
  auto bad = [](const kr_pseries* p) {
    return p->nterms > 0 && ((p->npoly > 0 && !p->exps) || !p->trig || !p->kind || !p->coef);
  };
  if (bad(f) || bad(g)) return KR_ERR_INVALID;
  if (h->capacity > 0 && !h->coef) return KR_ERR_INVALID;
  return guarded(ctx, [&]() -> kr_status {
    cudaStream_t s = (cudaStream_t)stream;
    ctx->has_result = false;
    ctx->stage_ms.clear();
    ctx->stage_name.clear();
    ctx->nev = 0;
    if (f->nterms == 0 || g->nterms == 0) {
      h->nterms = 0;
      return KR_OK;
    }
    JobIn in;
    in.poisson = true;
    in.f64 = true;
    in.np = f->npoly;
    in.nt = f->ntrig;
    in.fe = f->exps; in.ft = f->trig; in.fk = f->kind; in.fc = f->coef; in.nf = f->nterms;
    in.ge = g->exps; in.gt = g->trig; in.gk = g->kind; in.gc = g->coef; in.ng = g->nterms;
    if (opts) in.opts = *opts;
    std::vector<ProdResult> res;
    ctx->allow_deferred = is_device_ptr(h->coef) && (!h->exps || is_device_ptr(h->exps)) &&
                          (!h->trig || is_device_ptr(h->trig)) && (!h->kind || is_device_ptr(h->kind)) &&
                          (!h->codes || is_device_ptr(h->codes));
    ctx->direct = DirectOut{};
    ctx->direct_done = false;
    try {
      run_pipeline(ctx, {in}, s, res);
    } catch (...) {
      ctx->allow_deferred = false;
      throw;
    }
    ctx->allow_deferred = false;
    if (res[0].st != KR_OK) return res[0].st;
    keep_result(ctx, res[0], true);
    return emit_pseries(ctx, h, s);
  });
}

namespace {

bool poly_job_ok(const kr_poly* f, const kr_poly* g) {
  if (f->nvars < 1 || f->nvars > KR_MAXV || g->nvars != f->nvars) return false;
  if (f->type != g->type || (f->type != KR_I64 && f->type != KR_F64)) return false;
  if (f->nterms < 0 || g->nterms < 0 || f->nterms >= INT32_MAX || g->nterms >= INT32_MAX) return false;
  if ((f->nterms > 0 && (!f->exps || !f->coef)) || (g->nterms > 0 && (!g->exps || !g->coef))) return false;
  return true;
}

bool pseries_job_ok(const kr_pseries* f, const kr_pseries* g) {
  if (f->ntrig < 1 || f->npoly < 0 || f->npoly + f->ntrig > KR_MAXV) return false;
  if (g->npoly != f->npoly || g->ntrig != f->ntrig) return false;
  if (f->nterms < 0 || g->nterms < 0 || f->nterms >= INT32_MAX || g->nterms >= INT32_MAX) return false;
  auto bad = [](const kr_pseries* p) {
    return p->nterms > 0 && ((p->npoly > 0 && !p->exps) || !p->trig || !p->kind || !p->coef);
  };
  return !bad(f) && !bad(g);
}

// One wave of a batch: pipeline, then one batched decode into a fresh block.
kr_status run_wave(kr_ctx* ctx, const std::vector<JobIn>& ins, const std::vector<int>& idx,
                   kr_result* res, cudaStream_t s) {
  std::vector<ProdResult> pr;
  try {
    run_pipeline(ctx, ins, s, pr);
  } catch (const CudaFail& f) {
    if (f.e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      return KR_ERR_OOM;
    }
    throw;
  }
  // live products in device order
  std::vector<int> order;
  for (int p = 0; p < (int)ins.size(); ++p)
    if (pr[p].dprod) order.push_back(p);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return pr[a].dprod < pr[b].dprod; });
  size_t bytes = 0;
  for (int p : order) {
    const int nv = pr[p].prod.np + pr[p].prod.nt;
    bytes += (size_t)pr[p].n * (4 * nv + 1 + 8) + 4 * 256;
  }
  void* block = nullptr;
  if (bytes > 0) {
    cudaError_t e = cudaMalloc(&block, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return KR_ERR_OOM;
    }
    ctx->batch_blocks.push_back(block);
  }
  const int nl = (int)order.size();
  std::vector<ResDesc> rd(nl);
  std::vector<int64_t> ostart(nl + 1, 0);
  Bump b(block);
  int64_t total = 0;
  for (int q = 0; q < nl; ++q) {
    const ProdResult& r = pr[order[q]];
    const int64_t n = r.st == KR_OK ? r.n : 0;
    rd[q].n = n;
    rd[q].coef = (void*)b.take<uint64_t>(n);
    rd[q].exps = b.take<int32_t>(n * r.prod.np);
    rd[q].trig = r.prod.nt ? b.take<int32_t>(n * r.prod.nt) : nullptr;
    rd[q].kind = r.prod.nt ? b.take<uint8_t>(n) : nullptr;
    ostart[q] = r.prod.out_start;
    total = r.prod.out_start + r.n;
  }
  if (nl > 0) ostart[nl] = total;
  for (int q = 0; q < nl; ++q) {
    const int p = order[q];
    kr_result& R = res[idx[p]];
    R.status = pr[p].st;
    R.path = pr[p].prod.path == PATH_DENSE ? KR_PATH_DENSE : KR_PATH_HASH;
    R.nterms = pr[p].st == KR_OK ? pr[p].n : 0;
    R.exps = rd[q].exps;
    R.trig = rd[q].trig;
    R.kind = rd[q].kind;
    R.coef = rd[q].coef;
  }
  for (int p = 0; p < (int)ins.size(); ++p)
    if (!pr[p].dprod) {
      kr_result& R = res[idx[p]];
      R.status = pr[p].st;
      R.nterms = 0;
    }
  if (nl == 0 || total == 0) return KR_OK;
  // the decode reads every live product's Prod from the contiguous device array
  const Prod* dbase = pr[order[0]].dprod;
  ensure_pinned(ctx, sizeof(ResDesc) * nl + 8 * (nl + 1) + 1024, s);
  Bump hp(ctx->pinned);
  ResDesc* hrd = hp.take<ResDesc>(nl);
  int64_t* host = hp.take<int64_t>(nl + 1);
  memcpy(hrd, rd.data(), sizeof(ResDesc) * nl);
  memcpy(host, ostart.data(), 8 * (size_t)(nl + 1));
  ensure(ctx, &ctx->in_arena, &ctx->in_cap, sizeof(ResDesc) * nl + 8 * (nl + 1) + 1024, s);
  Bump db(ctx->in_arena);
  ResDesc* drd = db.take<ResDesc>(nl);
  int64_t* dost = db.take<int64_t>(nl + 1);
  ck(ctx, cudaMemcpyAsync(drd, hrd, sizeof(ResDesc) * nl, cudaMemcpyHostToDevice, s), "upload");
  ck(ctx, cudaMemcpyAsync(dost, host, 8 * (size_t)(nl + 1), cudaMemcpyHostToDevice, s), "upload");
  ck(ctx, launch_decode_batch(dbase, nl, dost, drd, pr[order[0]].key - pr[order[0]].prod.out_start,
                              pr[order[0]].val - pr[order[0]].prod.out_start, total, s),
     "batched decode");
  ctx->launches += 1;
  ck(ctx, cudaStreamSynchronize(s), "sync decode");
  return KR_OK;
}

}  // namespace

kr_status kron_mul_batch(kr_ctx* ctx, const kr_job* jobs, int32_t njobs, kr_result* res,
                         int64_t wave_pairs, kr_stream stream) {
  if (!ctx || njobs < 0 || (njobs > 0 && (!jobs || !res))) return KR_ERR_INVALID;
  return guarded(ctx, [&]() -> kr_status {
    cudaStream_t s = (cudaStream_t)stream;
    ck(ctx, cudaStreamSynchronize(s), "sync");
    for (void* b : ctx->batch_blocks) cudaFree(b);
    ctx->batch_blocks.clear();
    ctx->has_result = false;
    ctx->stage_ms.clear();
    ctx->stage_name.clear();
    ctx->nev = 0;
    const double budget = wave_pairs > 0 ? (double)wave_pairs : 8589934592.0;
    std::vector<JobIn> wave;
    std::vector<int> idx;
    double wave_tp = 0.0;
    std::vector<std::pair<std::vector<JobIn>, std::vector<int>>> waves;
    for (int i = 0; i < njobs; ++i) {
      const kr_job& J = jobs[i];
      kr_result& R = res[i];
      R = kr_result{};
      JobIn in;
      if (J.kind == 0) {
        if (!poly_job_ok(&J.f, &J.g)) { R.status = KR_ERR_INVALID; continue; }
        if (J.f.nterms == 0 || J.g.nterms == 0) { R.status = KR_OK; continue; }
        in.poisson = false;
        in.f64 = J.f.type == KR_F64;
        in.np = J.f.nvars;
        in.fe = J.f.exps; in.fc = J.f.coef; in.nf = J.f.nterms;
        in.ge = J.g.exps; in.gc = J.g.coef; in.ng = J.g.nterms;
      } else if (J.kind == 1) {
        if (!pseries_job_ok(&J.pf, &J.pg)) { R.status = KR_ERR_INVALID; continue; }
        if (J.pf.nterms == 0 || J.pg.nterms == 0) { R.status = KR_OK; continue; }
        in.poisson = true;
        in.f64 = true;
        in.np = J.pf.npoly;
        in.nt = J.pf.ntrig;
        in.fe = J.pf.exps; in.ft = J.pf.trig; in.fk = J.pf.kind; in.fc = J.pf.coef; in.nf = J.pf.nterms;
        in.ge = J.pg.exps; in.gt = J.pg.trig; in.gk = J.pg.kind; in.gc = J.pg.coef; in.ng = J.pg.nterms;
      } else {
        R.status = KR_ERR_INVALID;
        continue;
      }
      in.opts = J.opts;
      const double tp = (double)in.nf * (double)in.ng;
      if (!wave.empty() && (wave_tp + tp > budget || wave.size() >= 8192)) {
        waves.emplace_back(std::move(wave), std::move(idx));
        wave.clear();
        idx.clear();
        wave_tp = 0.0;
      }
      wave.push_back(in);
      idx.push_back(i);
      wave_tp += tp;
    }
    if (!wave.empty()) waves.emplace_back(std::move(wave), std::move(idx));
    // run the waves; a wave that runs out of memory is split in two
    for (size_t w = 0; w < waves.size(); ++w) {
      kr_status st = run_wave(ctx, waves[w].first, waves[w].second, res, s);
      if (st == KR_ERR_OOM) {
        const size_t n = waves[w].first.size();
        if (n <= 1) return KR_ERR_OOM;
        std::vector<JobIn> a(waves[w].first.begin(), waves[w].first.begin() + n / 2);
        std::vector<JobIn> b2(waves[w].first.begin() + n / 2, waves[w].first.end());
        std::vector<int> ia(waves[w].second.begin(), waves[w].second.begin() + n / 2);
        std::vector<int> ib(waves[w].second.begin() + n / 2, waves[w].second.end());
        waves.insert(waves.begin() + w + 1, {std::move(b2), std::move(ib)});
        waves[w] = {std::move(a), std::move(ia)};
        --w;
        continue;
      }
      if (st != KR_OK) return st;
    }
    return KR_OK;
  });
}

}  // extern "C"

// A prepared batch: its own context (scratch that never moves), the plans of
// its first run, the result memory, and the CUDA graph of the device work.
struct kr_batch {
  kr_ctx* ctx = nullptr;
  std::vector<JobIn> ins;
  std::vector<int> idx;
  std::vector<kr_result> res;     // per job, from the prepared run
  std::vector<int> live;          // JobIn index of each decoded product, device order
  std::vector<int64_t> nout;      // expected terms per decoded product
  void* block = nullptr;          // decoded results, ResDesc array, offsets
  const Prod* dprods = nullptr;
  ResDesc* d_rd = nullptr;
  int64_t* d_ost = nullptr;
  const uint64_t* okey = nullptr;
  const uint64_t* oval = nullptr;
  int64_t total = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

kr_status kron_batch_prepare(int32_t device, const kr_job* jobs, int32_t njobs, kr_batch** out,
                             kr_result* res, kr_stream stream) {
  if (!out || njobs < 1 || !jobs) return KR_ERR_INVALID;
  *out = nullptr;
  kr_ctx* ictx = nullptr;
  kr_status st = kr_ctx_create(device, &ictx);
  if (st != KR_OK) return st;
  kr_batch* b = new (std::nothrow) kr_batch;
  if (!b) { kr_ctx_destroy(ictx); return KR_ERR_OOM; }
  b->ctx = ictx;
  b->res.assign(njobs, kr_result{});
  st = guarded(ictx, [&]() -> kr_status {
    cudaStream_t s = (cudaStream_t)stream;
    // inputs: device buffers only (the graph reads them in place)
    for (int i = 0; i < njobs; ++i) {
      const kr_job& J = jobs[i];
      JobIn in;
      auto dev_or_null = [](const void* p) { return !p || is_device_ptr(p); };
      if (J.kind == 0 && poly_job_ok(&J.f, &J.g) && J.f.nterms > 0 && J.g.nterms > 0) {
        if (!dev_or_null(J.f.exps) || !dev_or_null(J.f.coef) || !dev_or_null(J.g.exps) || !dev_or_null(J.g.coef))
          return KR_ERR_INVALID;
        in.f64 = J.f.type == KR_F64;
        in.np = J.f.nvars;
        in.fe = J.f.exps; in.fc = J.f.coef; in.nf = J.f.nterms;
        in.ge = J.g.exps; in.gc = J.g.coef; in.ng = J.g.nterms;
      } else if (J.kind == 1 && pseries_job_ok(&J.pf, &J.pg) && J.pf.nterms > 0 && J.pg.nterms > 0) {
        for (const void* p : {(const void*)J.pf.exps, (const void*)J.pf.trig, (const void*)J.pf.kind,
                              (const void*)J.pf.coef, (const void*)J.pg.exps, (const void*)J.pg.trig,
                              (const void*)J.pg.kind, (const void*)J.pg.coef})
          if (!dev_or_null(p)) return KR_ERR_INVALID;
        in.poisson = true;
        in.f64 = true;
        in.np = J.pf.npoly;
        in.nt = J.pf.ntrig;
        in.fe = J.pf.exps; in.ft = J.pf.trig; in.fk = J.pf.kind; in.fc = J.pf.coef; in.nf = J.pf.nterms;
        in.ge = J.pg.exps; in.gt = J.pg.trig; in.gk = J.pg.kind; in.gc = J.pg.coef; in.ng = J.pg.nterms;
      } else {
        b->res[i].status = KR_ERR_INVALID;   // empty or invalid: nothing to replay
        if ((J.kind == 0 && poly_job_ok(&J.f, &J.g)) || (J.kind == 1 && pseries_job_ok(&J.pf, &J.pg)))
          b->res[i].status = KR_OK;
        continue;
      }
      in.opts = J.opts;
      b->ins.push_back(in);
      b->idx.push_back(i);
    }
    if (b->ins.empty()) return KR_OK;
    // the prepared run
    std::vector<ProdResult> pr;
    run_pipeline(ictx, b->ins, s, pr);
    std::vector<int> order;
    for (int p = 0; p < (int)b->ins.size(); ++p)
      if (pr[p].dprod) order.push_back(p);
    std::sort(order.begin(), order.end(), [&](int a, int c) { return pr[a].dprod < pr[c].dprod; });
    const int nl = (int)order.size();
    size_t bytes = sizeof(ResDesc) * (nl + 1) + 8 * (nl + 2) + 512;
    for (int p : order) bytes += (size_t)pr[p].n * (4 * (pr[p].prod.np + pr[p].prod.nt) + 1 + 8) + 4 * 256;
    ck(ictx, cudaMalloc(&b->block, bytes), "cudaMalloc results");
    Bump bb(b->block);
    b->d_rd = bb.take<ResDesc>(nl);
    b->d_ost = bb.take<int64_t>(nl + 1);
    std::vector<ResDesc> rd(nl);
    std::vector<int64_t> ost(nl + 1, 0);
    for (int q = 0; q < nl; ++q) {
      const ProdResult& r = pr[order[q]];
      const int64_t n = r.st == KR_OK ? r.n : 0;
      rd[q].n = n;
      rd[q].coef = (void*)bb.take<uint64_t>(n);
      rd[q].exps = bb.take<int32_t>(n * r.prod.np);
      rd[q].trig = r.prod.nt ? bb.take<int32_t>(n * r.prod.nt) : nullptr;
      rd[q].kind = r.prod.nt ? bb.take<uint8_t>(n) : nullptr;
      ost[q] = r.prod.out_start;
      b->total = r.prod.out_start + r.n;
      b->live.push_back(order[q]);
      b->nout.push_back(r.n);
      kr_result& R = b->res[b->idx[order[q]]];
      R.status = r.st;
      R.path = r.prod.path == PATH_DENSE ? KR_PATH_DENSE : KR_PATH_HASH;
      R.nterms = n;
      R.exps = rd[q].exps; R.trig = rd[q].trig; R.kind = rd[q].kind; R.coef = rd[q].coef;
    }
    ost[nl] = b->total;
    for (int p = 0; p < (int)b->ins.size(); ++p)
      if (!pr[p].dprod) b->res[b->idx[p]].status = pr[p].st;
    if (nl == 0) return KR_OK;
    ck(ictx, cudaMemcpy(b->d_rd, rd.data(), sizeof(ResDesc) * nl, cudaMemcpyHostToDevice), "upload");
    ck(ictx, cudaMemcpy(b->d_ost, ost.data(), 8 * (size_t)(nl + 1), cudaMemcpyHostToDevice), "upload");
    b->dprods = pr[order[0]].dprod;
    b->okey = pr[order[0]].key - pr[order[0]].prod.out_start;
    b->oval = pr[order[0]].val - pr[order[0]].prod.out_start;
    ck(ictx, launch_decode_batch(b->dprods, nl, b->d_ost, b->d_rd, b->okey, b->oval, b->total, s),
       "batched decode");
    ck(ictx, cudaStreamSynchronize(s), "sync");
    // capture the device work of a replay into a graph
    ensure_pinned(ictx, ictx->pinned_cap * 2 + (1 << 20), s);
    ck(ictx, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "stream");
    ck(ictx, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed), "begin capture");
    ictx->replay = true;
    try {
      std::vector<ProdResult> pr2;
      run_pipeline(ictx, b->ins, b->cap_stream, pr2);
      ck(ictx, launch_decode_batch(b->dprods, nl, b->d_ost, b->d_rd, b->okey, b->oval, b->total,
                                   b->cap_stream), "batched decode");
    } catch (...) {
      ictx->replay = false;
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(b->cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    ictx->replay = false;
    ck(ictx, cudaStreamEndCapture(b->cap_stream, &b->graph), "end capture");
    ck(ictx, cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
    return KR_OK;
  });
  if (st != KR_OK) {
    kron_batch_destroy(b);
    return st;
  }
  if (res)
    for (int i = 0; i < njobs; ++i) res[i] = b->res[i];
  *out = b;
  return KR_OK;
}

int64_t kron_batch_graph_kernels(const kr_batch* b) {
  if (!b) return -1;
  if (!b->graph) return 0;
  size_t n = 0;
  if (cudaGraphGetNodes(b->graph, nullptr, &n) != cudaSuccess) { cudaGetLastError(); return -1; }
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(b->graph, nodes.data(), &n) != cudaSuccess) { cudaGetLastError(); return -1; }
  int64_t k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  cudaGetLastError();
  return k;
}

kr_status kron_batch_launch(kr_batch* b, kr_stream stream) {
  if (!b) return KR_ERR_INVALID;
  if (!b->exec) return KR_OK;   // nothing to recompute
  return guarded(b->ctx, [&]() -> kr_status {
    ck(b->ctx, cudaGraphLaunch(b->exec, (cudaStream_t)stream), "graph launch");
    return KR_OK;
  });
}

kr_status kron_batch_results(kr_batch* b, kr_result* res, int32_t njobs) {
  if (!b || !res || njobs != (int32_t)b->res.size()) return KR_ERR_INVALID;
  return guarded(b->ctx, [&]() -> kr_status {
    const int nl = (int)b->live.size();
    std::vector<Prod> hp(nl);
    if (nl > 0) ck(b->ctx, cudaMemcpy(hp.data(), b->dprods, sizeof(Prod) * nl, cudaMemcpyDeviceToHost), "download");
    for (int i = 0; i < njobs; ++i) res[i] = b->res[i];
    for (int q = 0; q < nl; ++q) {
      kr_result& R = res[b->idx[b->live[q]]];
      if (R.status != KR_OK) continue;
      const uint32_t stq = hp[q].status;
      if (stq) R.status = status_to_kr(stq);
      else if (hp[q].nout != b->nout[q]) R.status = KR_ERR_CAPACITY;   // counts moved: prepare again
    }
    return KR_OK;
  });
}

void kron_batch_destroy(kr_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->block) cudaFree(b->block);
  if (b->ctx) kr_ctx_destroy(b->ctx);
  delete b;
}

kr_status kron_split_hist(kr_ctx* ctx, const kr_job* job, int32_t nbins, int64_t nsamples, uint64_t seed,
                          int64_t* hist, int64_t* krange_out, kr_stream stream) {
  if (!ctx || !job || !hist || nbins < 1 || nsamples < 0) return KR_ERR_INVALID;
  const kr_job& J = *job;
  JobIn in;
  if (J.kind == 0) {
    if (!poly_job_ok(&J.f, &J.g) || J.f.nterms == 0 || J.g.nterms == 0) return KR_ERR_INVALID;
    in.poisson = false;
    in.f64 = J.f.type == KR_F64;
    in.np = J.f.nvars;
    in.fe = J.f.exps; in.fc = J.f.coef; in.nf = J.f.nterms;
    in.ge = J.g.exps; in.gc = J.g.coef; in.ng = J.g.nterms;
  } else if (J.kind == 1) {
    if (!pseries_job_ok(&J.pf, &J.pg) || J.pf.nterms == 0 || J.pg.nterms == 0) return KR_ERR_INVALID;
    in.poisson = true;
    in.f64 = true;
    in.np = J.pf.npoly;
    in.nt = J.pf.ntrig;
    in.fe = J.pf.exps; in.ft = J.pf.trig; in.fk = J.pf.kind; in.fc = J.pf.coef; in.nf = J.pf.nterms;
    in.ge = J.pg.exps; in.gt = J.pg.trig; in.gk = J.pg.kind; in.gc = J.pg.coef; in.ng = J.pg.nterms;
  } else {
    return KR_ERR_INVALID;
  }
  in.opts = J.opts;
  in.opts.code_lo = 0;
  in.opts.code_hi = 0;
  return guarded(ctx, [&]() -> kr_status {
    cudaStream_t s = (cudaStream_t)stream;
    ctx->has_result = false;
    ctx->stage_ms.clear();
    ctx->stage_name.clear();
    ctx->nev = 0;
    for (int32_t b = 0; b < nbins; ++b) hist[b] = 0;
    ctx->split_nbins = nbins;
    ctx->split_nsamples = nsamples;
    ctx->split_seed = seed;
    ctx->split_hist = hist;
    std::vector<ProdResult> res;
    try {
      run_pipeline(ctx, {in}, s, res);
    } catch (...) {
      ctx->split_hist = nullptr;
      throw;
    }
    ctx->split_hist = nullptr;
    if (krange_out) *krange_out = res[0].prod.krange;
    return res[0].st;
  });
}

kr_status kron_fetch_poly(kr_ctx* ctx, kr_poly_out* h, kr_stream stream) {
  if (!ctx || !h) return KR_ERR_INVALID;
  if (!ctx->has_result || ctx->res_poisson || h->nvars != ctx->res_prod.np) return KR_ERR_INVALID;
  return guarded(ctx, [&]() -> kr_status { return emit_poly(ctx, h, (cudaStream_t)stream); });
}

kr_status kron_fetch_pseries(kr_ctx* ctx, kr_pseries_out* h, kr_stream stream) {
  if (!ctx || !h) return KR_ERR_INVALID;
  if (!ctx->has_result || !ctx->res_poisson || h->npoly != ctx->res_prod.np ||
      h->ntrig != ctx->res_prod.nt)
    return KR_ERR_INVALID;
  return guarded(ctx, [&]() -> kr_status { return emit_pseries(ctx, h, (cudaStream_t)stream); });
}

}  // extern "C"
