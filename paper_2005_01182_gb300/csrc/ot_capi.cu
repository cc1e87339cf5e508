// C ABI of libotassign.so: context, single and multi-instance solves,
// bucketing scheduler, CUDA-graph replay and the autotuner.  The serving
// loop lives in ot_serve.cu.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "otassign.h"
#include "ot_ctx.h"
#include "ot_group.cuh"
#include "ot_shapes.h"

namespace ot {
cudaError_t launch_group_km(GroupShape, const Instance*, const int32_t*, int, int*, int, int, int,
                            cudaStream_t);
cudaError_t launch_group_bkm(GroupShape, const Instance*, const int32_t*, int, int*, int, int, int,
                             cudaStream_t);

cudaError_t launch_group(GroupShape shape, int algo, const Instance* insts, const int32_t* order,
                         int num, int* work, int nmax, int mmax, int max_ctas,
                         cudaStream_t stream) {
  if (algo == kAlgoKM)
    return launch_group_km(shape, insts, order, num, work, nmax, mmax, max_ctas, stream);
  return launch_group_bkm(shape, insts, order, num, work, nmax, mmax, max_ctas, stream);
}

static const GroupShape kShapes[OT_NUM_GROUP_SHAPES] = {
#define OT_ROW(IDX, TPI_, K_) GroupShape{TPI_, K_},
    OT_GROUP_SHAPES(OT_ROW)
#undef OT_ROW
};

int num_group_shapes() { return OT_NUM_GROUP_SHAPES; }
GroupShape group_shape(int idx) { return kShapes[idx]; }

size_t group_smem_bytes(GroupShape s, int algo, int nmax, int mmax) {
  return group_bytes(s.tpi, algo, nmax, mmax) * (s.tpi == 32 ? 8 : 1);
}

size_t group_smem_limit() { return 227 * 1024; }

int shape_index(int tpi, int k) {
  for (int i = 0; i < OT_NUM_GROUP_SHAPES; ++i)
    if (kShapes[i].tpi == tpi && kShapes[i].k == k) return i;
  return -1;
}

int bucket_of(int m) {
  int b = 0;
  while (b < kNumBuckets - 1 && m > (32 << b)) ++b;
  return b;
}

void default_table(int table[2][kNumBuckets]) {
  // bucket b holds m <= 32 << b
  static const int tpi[kNumBuckets] = {32, 32, 32, 32, 128, 256, 512, 1024};
  static const int kk[kNumBuckets] = {1, 2, 4, 8, 4, 4, 4, 4};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < kNumBuckets; ++b) table[a][b] = shape_index(tpi[b], kk[b]);
}

void default_auto(int auto_algo[kNumBuckets]) {
  // KM for the small buckets, batched KM from m > 256 on (fewer dependent
  // steps per instance); the autotuner may change either
  for (int b = 0; b < kNumBuckets; ++b) auto_algo[b] = b <= 3 ? kAlgoKM : kAlgoBKM;
}

}  // namespace ot

using namespace ot;

int resolve_algo(const ot_ctx* ctx, int algo, int m) {
  if (algo == OT_AUCTION) return kAlgoAuction;
  if (algo != OT_AUTO) return algo;
  if (m > kMaxGroupCols) return kAlgoBKM;
  return ctx->auto_algo[bucket_of(m)];
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

int ctx_fail(ot_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int ctx_cuda(ot_ctx* ctx, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return OT_OK;
  return ctx_fail(ctx, OT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

namespace {

using PtrAttrsFn = CUresult (*)(unsigned int, CUpointer_attribute*, void**, CUdeviceptr);

// cuPointerGetAttributes through the runtime's driver entry point (no link
// against the CUDA driver API library); null if unavailable.
PtrAttrsFn ptr_attrs_fn() {
  static const PtrAttrsFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttributes", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<PtrAttrsFn>(f);
  }();
  return fn;
}

}  // namespace

bool PtrKinds::on_device(const void* p) {
  if (!p) return false;
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  if (last_ < ranges_.size() && a >= ranges_[last_].lo && a < ranges_[last_].hi) return ranges_[last_].dev;
  auto it = std::upper_bound(ranges_.begin(), ranges_.end(), a,
                             [](uintptr_t x, const Range& r) { return x < r.lo; });
  if (it != ranges_.begin()) {
    const size_t i = size_t(it - ranges_.begin()) - 1;
    if (a < ranges_[i].hi) {
      last_ = i;
      return ranges_[i].dev;
    }
  }
  if (PtrAttrsFn fn = ptr_attrs_fn()) {
    CUpointer_attribute at[4] = {CU_POINTER_ATTRIBUTE_MEMORY_TYPE, CU_POINTER_ATTRIBUTE_IS_MANAGED,
                                 CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, CU_POINTER_ATTRIBUTE_RANGE_SIZE};
    unsigned long long type = 0, managed = 0, start = 0, size = 0;
    void* data[4] = {&type, &managed, &start, &size};
    if (fn(4, at, data, CUdeviceptr(a)) == CUDA_SUCCESS && size > 0 && a >= start && a - start < size &&
        (managed != 0 || type == CU_MEMORYTYPE_DEVICE || type == CU_MEMORYTYPE_HOST)) {
      const bool dev = managed != 0 || type == CU_MEMORYTYPE_DEVICE;
      const Range r{uintptr_t(start), uintptr_t(start + size), dev};
      last_ = size_t(std::upper_bound(ranges_.begin(), ranges_.end(), r.lo,
                                      [](uintptr_t x, const Range& y) { return x < y.lo; }) -
                     ranges_.begin());
      ranges_.insert(ranges_.begin() + last_, r);
      return dev;
    }
  }
  return ptr_on_device(p);  // memory CUDA does not track (pageable host)
}

bool ptr_on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int DevBuf::reserve(size_t bytes) {
  if (bytes <= cap) return OT_OK;
  const size_t want = std::max(bytes, cap * 2);
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  cap = 0;
  if (cudaMalloc(&ptr, want) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
    return OT_ERR_OOM;
  }
  cap = want;
  ++generation;
  return OT_OK;
}

void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  cap = 0;
}

int PinBuf::reserve(size_t bytes) {
  if (bytes <= cap) return OT_OK;
  const size_t want = std::max(bytes, cap * 2);
  if (ptr) cudaFreeHost(ptr);
  ptr = nullptr;
  cap = 0;
  if (cudaHostAlloc(&ptr, want, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
    return OT_ERR_OOM;
  }
  cap = want;
  return OT_OK;
}

void PinBuf::release() {
  if (ptr) cudaFreeHost(ptr);
  ptr = nullptr;
  cap = 0;
}

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// ---------------------------------------------------------------------------
// device-pointer batch: bucket, upload descriptors, launch (optionally as a
// cached CUDA graph)
// ---------------------------------------------------------------------------

struct Bucket {
  int shape;
  int algo = 0;
  int nmax = 0, mmax = 0;
  std::vector<int> idx;
};

// insts[t] already holds device pointers; entries with skip[t] set are not
// launched.  Writes per-instance stats into ctx->d_stats (k x 8).
int run_device_batch(ot_ctx* ctx, LaunchSlot& slot, std::vector<Instance>& insts,
                     const std::vector<int>& skip, int algo, cudaStream_t stream, bool fork,
                     bool own_stats, std::vector<int>* unsupported, bool allow_cluster) {
  const int k = int(insts.size());
  for (Instance& I : insts) I.step_limit = ctx->step_limit;
  if (own_stats) {
    if (int rc = slot.d_stats.reserve(size_t(k) * 8 * sizeof(int64_t)); rc) return ctx_fail(ctx, rc, "stats alloc");
    int64_t* dstats = static_cast<int64_t*>(slot.d_stats.ptr);
    for (int t = 0; t < k; ++t) insts[t].stats = dstats + size_t(t) * 8;
  }

  // A handful of wide batched-KM instances solve faster on the cluster
  // engine (16 SMs and grid-wide passes each) than one CTA apiece; many of
  // them keep the group engine busy on every SM.
  int wide_bkm = 0;
  for (int t = 0; t < k; ++t)
    if (!skip[t] && insts[t].m > kClusterRouteCols && resolve_algo(ctx, algo, insts[t].m) == kAlgoBKM) ++wide_bkm;
  const bool route_wide = allow_cluster && wide_bkm > 0 && wide_bkm <= kClusterRouteMax;
  // bucket by (algorithm, tuned shape)
  std::map<int, Bucket> buckets;
  for (int t = 0; t < k; ++t) {
    if (skip[t]) continue;
    const Instance& I = insts[t];
    const int ia = resolve_algo(ctx, algo, I.m);
    if (ia == kAlgoAuction) {
      // the auction engine: one CTA per instance, sized by m
      if (I.m > kMaxGroupCols || auction_smem_bytes(I.m) > group_smem_limit()) {
        if (unsupported) unsupported->push_back(t);
        continue;
      }
      const int th = auction_threads(I.m);
      Bucket& b = buckets[ia * 64 + th / 32];
      b.shape = th;
      b.algo = ia;
      b.nmax = std::max(b.nmax, I.n);
      b.mmax = std::max(b.mmax, I.m);
      b.idx.push_back(t);
      continue;
    }
    int sh = ctx->table[ia][bucket_of(I.m)];
    if (route_wide && ia == kAlgoBKM && I.m > kClusterRouteCols && !ctx->tuned[ia][bucket_of(I.m)]) sh = kLargeEngine;
    if (sh == kLargeEngine) {  // bucket routed to the cluster engine
      if (unsupported) unsupported->push_back(t);
      continue;
    }
    if (sh >= 0 && group_shape(sh).max_cols() < I.m) {
      int def[2][kNumBuckets];
      default_table(def);
      sh = def[ia][bucket_of(I.m)];
    }
    if (I.m > kMaxGroupCols || sh < 0 ||
        group_smem_bytes(group_shape(sh), ia, I.n, I.m) > group_smem_limit()) {
      if (unsupported) unsupported->push_back(t);
      continue;
    }
    Bucket& b = buckets[ia * 64 + sh];
    b.shape = sh;
    b.algo = ia;
    b.nmax = std::max(b.nmax, I.n);
    b.mmax = std::max(b.mmax, I.m);
    b.idx.push_back(t);
  }
  const bool pack_on = ctx->pack_rows;
  bool any_pack = false;
  if (pack_on && slot.pack && !buckets.empty()) {
    size_t nrows = 0, nelem = 0;
    for (auto& kv : buckets)
      if (kv.second.algo != kAlgoAuction)
        for (int t : kv.second.idx) { nrows += insts[t].n; nelem += size_t(insts[t].n) * insts[t].m; }
    const size_t b_pok = al256(sizeof(int32_t) * k), b_roff = al256(sizeof(int32_t) * nrows);
    const int genp = slot.d_pack.generation;
    if (slot.d_pack.reserve(b_pok + b_roff + al256(2 * nelem)) == OT_OK) {
      if (slot.d_pack.generation != genp) slot.clear_graphs();
      char* base = static_cast<char*>(slot.d_pack.ptr);
      int32_t* pok = reinterpret_cast<int32_t*>(base);
      int32_t* roff = reinterpret_cast<int32_t*>(base + b_pok);
      uint16_t* P = reinterpret_cast<uint16_t*>(base + b_pok + b_roff);
      size_t orow = 0, oel = 0;
      for (auto& kv : buckets)
        for (int t : kv.second.idx) {
          if (kv.second.algo == kAlgoAuction) continue;
          insts[t].pok = pok + t;
          insts[t].roff = roff + orow;
          insts[t].P = P + oel;
          orow += insts[t].n;
          oel += size_t(insts[t].n) * insts[t].m;
        }
      any_pack = nelem > 0;
    }
  }
  // a shape may serve several m-buckets; keep the smem bound feasible
  for (auto& kv : buckets) {
    Bucket& b = kv.second;
    std::sort(b.idx.begin(), b.idx.end(), [&](int a, int c) {
      long long wa = (long long)insts[a].n * insts[a].m, wc = (long long)insts[c].n * insts[c].m;
      return wa != wc ? wa > wc : a < c;
    });
  }
  const int nb = int(buckets.size());
  const size_t desc_bytes = al256(sizeof(Instance) * k);
  const size_t order_bytes = al256(sizeof(int32_t) * (k + 1));
  const size_t work_bytes = al256(sizeof(int) * (nb + 1));
  const size_t total = desc_bytes + order_bytes + work_bytes;

  const int gen = slot.d_meta.generation;
  if (int rc = slot.d_meta.reserve(total); rc) return ctx_fail(ctx, rc, "meta alloc");
  if (slot.d_meta.generation != gen) slot.clear_graphs();

  // descriptors and launch order, built on the host and uploaded only when
  // they differ from what the device already holds
  std::vector<char>& pend = slot.pending;
  pend.assign(desc_bytes + order_bytes, 0);
  std::memcpy(pend.data(), insts.data(), sizeof(Instance) * k);
  int32_t* horder = reinterpret_cast<int32_t*>(pend.data() + desc_bytes);
  std::string key = std::to_string(algo) + "|" + std::to_string(k);
  std::vector<int> offs;
  int off = 0;
  for (auto& kv : buckets) {
    Bucket& b = kv.second;
    offs.push_back(off);
    for (int t : b.idx) horder[off++] = t;
    key += "|" + std::to_string(b.algo) + ":" + std::to_string(b.shape) + "," + std::to_string(b.idx.size()) + "," +
           std::to_string(b.nmax) + "," + std::to_string(b.mmax);
  }
  key += "|" + std::to_string(reinterpret_cast<uintptr_t>(stream)) + (any_pack ? "|p" : "");

  char* d = static_cast<char*>(slot.d_meta.ptr);
  const Instance* dinst = reinterpret_cast<const Instance*>(d);
  const int32_t* dorder = reinterpret_cast<const int32_t*>(d + desc_bytes);
  int* dwork = reinterpret_cast<int*>(d + desc_bytes + order_bytes);

  // the slot's buffers (descriptors, work counters, packed rows, stats) are
  // reused: this launch starts after the previous one, on whatever stream
  if (slot.meta_pending) {
    if (cudaError_t e = cudaStreamWaitEvent(stream, slot.meta_ev, 0); e != cudaSuccess)
      return ctx_cuda(ctx, e, "order after previous launch");
  }
  if (!(slot.meta_valid && pend == slot.last_meta)) {
    // the pinned mirror may still feed the previous upload
    if (slot.meta_pending) cudaEventSynchronize(slot.meta_ev);
    if (int rc = slot.h_meta.reserve(pend.size()); rc) return ctx_fail(ctx, rc, "pinned alloc");
    std::memcpy(slot.h_meta.ptr, pend.data(), pend.size());
    if (cudaError_t e = cudaMemcpyAsync(d, slot.h_meta.ptr, pend.size(), cudaMemcpyHostToDevice, stream);
        e != cudaSuccess) {
      slot.meta_valid = false;
      return ctx_cuda(ctx, e, "descriptor upload");
    }
    slot.last_meta.swap(pend);
    slot.meta_valid = true;
  }

  // timing events around every bucket's kernel (external records, so that
  // they become event-record nodes when the launch is captured in a graph)
  if (slot.timing && slot.tev.size() < size_t(2 * nb)) {
    slot.clear_graphs();
    for (cudaEvent_t ev : slot.tev) cudaEventDestroy(ev);
    slot.tev.assign(size_t(2 * nb), nullptr);
    for (auto& ev : slot.tev)
      if (cudaEventCreate(&ev) != cudaSuccess) {
        slot.tev.clear();
        slot.timing = false;
        return ctx_fail(ctx, OT_ERR_CUDA, "timing events");
      }
  }
  slot.last_buckets.clear();
  for (auto& kv : buckets) {
    const Bucket& b = kv.second;
    LaunchSlot::BucketInfo bi;
    bi.algo = b.algo;
    bi.tpi = b.algo == kAlgoAuction ? b.shape : group_shape(b.shape).tpi;
    bi.k = b.algo == kAlgoAuction ? 0 : group_shape(b.shape).k;
    bi.idx = b.idx;
    slot.last_buckets.push_back(std::move(bi));
  }
  const bool timed = slot.timing && !slot.tev.empty();
  auto launch_bucket = [&](const Bucket& b, int bi, cudaStream_t s) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    if (timed && (e = cudaEventRecordWithFlags(slot.tev[2 * bi], s, cudaEventRecordExternal)) != cudaSuccess)
      return e;
    if (b.algo == kAlgoAuction)
      e = launch_auction(b.shape, dinst, dorder + offs[bi], int(b.idx.size()), dwork + bi, b.mmax, s);
    else
      e = launch_group(group_shape(b.shape), b.algo, dinst, dorder + offs[bi], int(b.idx.size()), dwork + bi,
                       b.nmax, b.mmax, ctx->max_group_ctas, s);
    if (e == cudaSuccess && timed) e = cudaEventRecordWithFlags(slot.tev[2 * bi + 1], s, cudaEventRecordExternal);
    return e;
  };
  auto enqueue = [&](cudaStream_t s) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(dwork, 0, work_bytes, s);
    if (e != cudaSuccess) return e;
    if (any_pack && (e = launch_pack(dinst, nullptr, k, s)) != cudaSuccess) return e;
    if (nb == 1 || !fork) {
      int bi = 0;
      for (auto& kv : buckets) {
        Bucket& b = kv.second;
        e = launch_bucket(b, bi, s);
        if (e != cudaSuccess) return e;
        ++bi;
      }
      return cudaSuccess;
    }
    if ((e = cudaEventRecord(ctx->fork_ev, s)) != cudaSuccess) return e;
    int bi = 0;
    for (auto& kv : buckets) {
      Bucket& b = kv.second;
      cudaStream_t bs = ctx->bstreams[bi % kForkStreams];
      if ((e = cudaStreamWaitEvent(bs, ctx->fork_ev, 0)) != cudaSuccess) return e;
      e = launch_bucket(b, bi, bs);
      if (e != cudaSuccess) return e;
      ++bi;
    }
    for (int s2 = 0; s2 < std::min(nb, kForkStreams); ++s2) {
      if ((e = cudaEventRecord(ctx->join_ev[s2], ctx->bstreams[s2])) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(s, ctx->join_ev[s2], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  };

  cudaError_t e = cudaSuccess;
  if (nb == 0) {
    // nothing to launch
  } else if (slot.use_graphs) {
    auto it = slot.graphs.find(key);
    if (it == slot.graphs.end()) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e1 = enqueue(stream);
        e = cudaStreamEndCapture(stream, &g);
        if (e1 != cudaSuccess) e = e1;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e == cudaSuccess) {
        if (slot.graphs.size() >= 64) slot.clear_graphs();
        it = slot.graphs.emplace(key, ge).first;
      }
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(it->second, stream);
  } else {
    e = enqueue(stream);
  }
  // marks the end of this launch and of the descriptor upload
  cudaEventRecord(slot.meta_ev, stream);
  slot.meta_pending = true;
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "batch launch");
  slot.last_launches = nb + (any_pack && nb > 0 ? 1 : 0);  // bucket kernels and the packing kernel
  return OT_OK;
}

int solve_wide(ot_ctx* ctx, const Instance& I, int algo, cudaStream_t stream, int64_t* stats_out) {
  if (algo == kAlgoBKM && !ctx->dense_wide && I.m <= sparse_max_cols()) return solve_sparse(ctx, I, stream, stats_out);
  return solve_large(ctx, I, algo, stream, stats_out);
}

// Validate one instance's sizes.
static int check_sizes(const void* C, int64_t ldc, int n, int m) {
  if (n < 0 || m < 0 || n > m) return OT_ERR_ARG;
  if (n > 0 && (!C || ldc < m)) return OT_ERR_ARG;
  return OT_OK;
}

// Solve k instances; every pointer is either device (dev=true) or host.
// route_wide: single-instance entry points let a wide batched-KM instance
// take the cluster engine (the batched entry point keeps the group engine
// unless the table says otherwise, so that its results do not depend on
// how many wide instances a call carries).
static int solve_many(ot_ctx* ctx, int k, const int32_t* const* C, const int64_t* ldc,
                      const int32_t* n, const int32_t* m, int algo, int32_t* const* r2c,
                      int64_t* cost, int64_t* const* u, int64_t* const* v, int32_t* status,
                      cudaStream_t stream, ot_stats* stats_out, bool route_wide) {
  if (algo != OT_KM && algo != OT_BKM && algo != OT_AUTO && algo != OT_AUCTION)
    return ctx_fail(ctx, OT_ERR_ARG, "bad algo");
  if (k < 0) return ctx_fail(ctx, OT_ERR_ARG, "k < 0");
  if (k == 0) return OT_OK;
  if (!C || !ldc || !n || !m || !r2c || !cost) return ctx_fail(ctx, OT_ERR_ARG, "null array");
  // all element pointers must live on one side
  int first = -1;
  for (int t = 0; t < k; ++t)
    if (n[t] > 0) { first = t; break; }
  PtrKinds kinds;  // one driver query per allocation, not per pointer
  const bool dev = first < 0 ? kinds.on_device(cost) : kinds.on_device(C[first]);

  std::vector<int> st(k, OT_OK), skip(k, 0);
  for (int t = 0; t < k; ++t) {
    st[t] = check_sizes(C[t], ldc[t], n[t], m[t]);
    if (st[t] == OT_OK && n[t] > 0 && !r2c[t]) st[t] = OT_ERR_ARG;
    if (st[t] == OT_OK && n[t] > 0 && kinds.on_device(C[t]) != dev) st[t] = OT_ERR_ARG;
    skip[t] = st[t] != OT_OK;
  }

  std::vector<Instance> insts(k);
  std::lock_guard<std::mutex> lock(ctx->api_mu);
  StreamScope scope(stream, ctx->stream, ctx->join_in_ev, ctx->join_out_ev);
  stream = scope.work;
  cudaError_t e;
  if (dev) {
    // device pointers: cost/status arrays are device arrays of length k
    int32_t* dstatus = status;
    if (!status || !ptr_on_device(status)) {
      if (int rc = ctx->d_status.reserve(sizeof(int32_t) * k); rc) return ctx_fail(ctx, rc, "status alloc");
      dstatus = static_cast<int32_t*>(ctx->d_status.ptr);
    }
    for (int t = 0; t < k; ++t) {
      Instance& I = insts[t];
      I.C = C[t]; I.ldc = ldc[t]; I.n = n[t]; I.m = m[t];
      I.row_to_col = r2c[t]; I.u = u ? u[t] : nullptr; I.v = v ? v[t] : nullptr;
      I.cost = cost + t; I.status = dstatus + t;
      if (n[t] == 0 && st[t] == OT_OK) skip[t] = 1;  // handled below
    }
    std::vector<int> unsup;
    if (int rc = run_device_batch(ctx, ctx->api, insts, skip, algo, stream, true, true, &unsup, route_wide); rc) return rc;
    ctx->last_k = k;
    ctx->last_skip = skip;
    // instances wider than a group: the cluster engine, one at a time
    for (int t : unsup) {
      if (insts[t].m > large_max_cols() || algo == OT_AUCTION) {
        st[t] = OT_ERR_UNSUPPORTED;
        ctx->last_skip[t] = 1;
        continue;
      }
      const int rc = solve_wide(ctx, insts[t], resolve_algo(ctx, algo, insts[t].m), stream, nullptr);
      if (rc == OT_ERR_TIMEOUT || rc == OT_ERR_UNSUPPORTED) { st[t] = rc; continue; }
      if (rc != OT_OK) return rc;
    }
    // empty instances: cost 0, status per validation; zero v of width m
    for (int t = 0; t < k; ++t) {
      if (n[t] == 0 && st[t] == OT_OK) {
        if ((e = cudaMemsetAsync(cost + t, 0, sizeof(int64_t), stream)) != cudaSuccess) return ctx_cuda(ctx, e, "memset");
        if ((e = cudaMemsetAsync(dstatus + t, 0, sizeof(int32_t), stream)) != cudaSuccess) return ctx_cuda(ctx, e, "memset");
        if (v && v[t] && m[t] > 0) cudaMemsetAsync(v[t], 0, sizeof(int64_t) * m[t], stream);
      }
    }
    // host-side validation codes go to the status array
    bool any_bad = false;
    for (int t = 0; t < k; ++t) any_bad |= st[t] != OT_OK;
    if (status && (any_bad)) {
      for (int t = 0; t < k; ++t)
        if (st[t] != OT_OK) cudaMemcpyAsync(dstatus + t, &st[t], sizeof(int32_t), cudaMemcpyHostToDevice, stream);
      cudaStreamSynchronize(stream);
    } else if (status && !ptr_on_device(status)) {
      // host status array with device data: synchronise to report device codes
      if ((e = cudaMemcpyAsync(status, dstatus, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return ctx_cuda(ctx, e, "status copy");
      cudaStreamSynchronize(stream);
    } else if (status) {
      // device status array: zero-init entries of skipped instances
    }
    if (stats_out) {
      cudaStreamSynchronize(stream);
      int64_t s8[8] = {0};
      if (k >= 1 && n[0] > 0) cudaMemcpy(s8, insts[0].stats, sizeof(s8), cudaMemcpyDeviceToHost);
      int32_t s0 = 0;
      if (k >= 1 && n[0] > 0) cudaMemcpy(&s0, dstatus, sizeof(s0), cudaMemcpyDeviceToHost);
      std::memcpy(stats_out, s8, sizeof(s8));
      if (st[0] != OT_OK) return ctx_fail(ctx, st[0], "instance failed: " + ctx->err);
      if (s0 != 0) return ctx_fail(ctx, s0, "device status error");
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "solve");
    for (int t = 0; t < k; ++t)
      if (st[t] != OT_OK && k == 1) return ctx_fail(ctx, st[t], st[t] == OT_ERR_UNSUPPORTED ? "size not supported" : "bad instance");
    return OT_OK;
  }

  // host pointers: stage through device memory.  Matrices, assignments and
  // duals are packed back to back in staging (one region each), so that host
  // buffers laid out the same way move with a single copy per region.
  std::vector<size_t> off_c(k), off_r(k), off_u(k), off_v(k);
  size_t ec = 0, er = 0, ev = 0;  // element offsets
  for (int t = 0; t < k; ++t) {
    off_c[t] = ec; off_r[t] = er; off_u[t] = er; off_v[t] = ev;
    if (skip[t]) continue;
    ec += size_t(n[t]) * m[t];
    er += size_t(n[t]);
    ev += size_t(m[t]);
  }
  const size_t base_cost = 0, base_status = al256(sizeof(int64_t) * k);
  const size_t base_c = base_status + al256(sizeof(int32_t) * k);
  const size_t base_r = base_c + al256(4 * ec), base_u = base_r + al256(4 * er);
  const size_t base_v = base_u + al256(8 * er), total = base_v + al256(8 * ev);
  if (int rc = ctx->d_io.reserve(total); rc) return ctx_fail(ctx, rc, "staging alloc");
  char* D = static_cast<char*>(ctx->d_io.ptr);
  int64_t* dcost = reinterpret_cast<int64_t*>(D + base_cost);
  int32_t* dstatus = reinterpret_cast<int32_t*>(D + base_status);
  int32_t* dC = reinterpret_cast<int32_t*>(D + base_c);
  int32_t* dR = reinterpret_cast<int32_t*>(D + base_r);
  int64_t* dU = reinterpret_cast<int64_t*>(D + base_u);
  int64_t* dV = reinterpret_cast<int64_t*>(D + base_v);
  if ((e = cudaMemsetAsync(D, 0, base_c, stream)) != cudaSuccess) return ctx_cuda(ctx, e, "memset");
  // contiguity of the caller's host buffers
  bool c_flat = true, r_flat = true, u_flat = u != nullptr, v_flat = v != nullptr;
  int first_live = -1;
  for (int t = 0; t < k; ++t) {
    if (skip[t] || n[t] == 0) continue;
    if (first_live < 0) first_live = t;
    const int f = first_live;
    c_flat &= ldc[t] == m[t] && C[t] == C[f] + off_c[t] - off_c[f];
    r_flat &= r2c[t] == r2c[f] + off_r[t] - off_r[f];
    if (u_flat) u_flat &= u[t] && u[t] == u[f] + off_u[t] - off_u[f];
    if (v_flat) v_flat &= v[t] && v[t] == v[f] + off_v[t] - off_v[f];
  }
  for (int t = 0; t < k; ++t) {
    Instance& I = insts[t];
    I.C = dC + off_c[t]; I.ldc = m[t]; I.n = n[t]; I.m = m[t];
    I.row_to_col = dR + off_r[t];
    I.u = dU + off_u[t];
    I.v = dV + off_v[t];
    I.cost = dcost + t; I.status = dstatus + t;
    if (skip[t]) continue;
    if (n[t] == 0) { skip[t] = 1; continue; }
    if (!c_flat) {
      e = cudaMemcpy2DAsync(dC + off_c[t], sizeof(int32_t) * m[t], C[t], sizeof(int32_t) * ldc[t],
                            sizeof(int32_t) * m[t], n[t], cudaMemcpyHostToDevice, stream);
      if (e != cudaSuccess) return ctx_cuda(ctx, e, "H2D");
    }
  }
  // a large batch laid out back to back moves in chunks: chunk c is solved
  // while chunks c+1.. are still being copied
  int live = 0;
  for (int t = 0; t < k; ++t) live += !skip[t];
  const int nchunks = (c_flat && live >= 64 * kHostChunks && 4 * ec >= (size_t(64) << 20)) ? kHostChunks : 1;
  std::vector<int> unsup;
  if (nchunks > 1) {
    if (int rc = ctx->api.d_stats.reserve(size_t(k) * 8 * sizeof(int64_t)); rc) return ctx_fail(ctx, rc, "stats alloc");
    int64_t* dstats = static_cast<int64_t*>(ctx->api.d_stats.ptr);
    for (int t = 0; t < k; ++t) insts[t].stats = dstats + size_t(t) * 8;
    // chunk boundaries over the instances, balanced by matrix bytes
    std::vector<int> bound(nchunks + 1, k);
    bound[0] = 0;
    for (int c = 1, t = 0; c < nchunks; ++c) {
      const size_t want = (ec / nchunks) * c;
      while (t < k && off_c[t] < want) ++t;
      bound[c] = t;
    }
    if ((e = cudaEventRecord(ctx->hev_start, stream)) != cudaSuccess) return ctx_cuda(ctx, e, "chunk start");
    for (int c = 0; c < nchunks; ++c) {
      const size_t e0 = bound[c] < k ? off_c[bound[c]] : ec, e1 = bound[c + 1] < k ? off_c[bound[c + 1]] : ec;
      if (e1 > e0) {
        // the caller's buffer is contiguous from first_live on (c_flat)
        const int32_t* src = C[first_live] + (e0 - off_c[first_live]);
        if (e0 >= off_c[first_live] &&
            (e = cudaMemcpyAsync(dC + e0, src, 4 * (e1 - e0), cudaMemcpyHostToDevice, ctx->copy_stream)) != cudaSuccess)
          return ctx_cuda(ctx, e, "H2D chunk");
      }
      if ((e = cudaEventRecord(ctx->hev_copy[c], ctx->copy_stream)) != cudaSuccess) return ctx_cuda(ctx, e, "chunk copy");
    }
    int launches = 0;
    for (int c = 0; c < nchunks; ++c) {
      cudaStream_t cs = ctx->cstreams[c];
      cudaStreamWaitEvent(cs, ctx->hev_start, 0);
      cudaStreamWaitEvent(cs, ctx->hev_copy[c], 0);
      std::vector<Instance> ci(insts.begin() + bound[c], insts.begin() + bound[c + 1]);
      std::vector<int> cskip(skip.begin() + bound[c], skip.begin() + bound[c + 1]), cun;
      if (int rc = run_device_batch(ctx, ctx->hslots[c], ci, cskip, algo, cs, true, false, &cun, route_wide); rc)
        return rc;
      for (int x : cun) unsup.push_back(bound[c] + x);
      launches += ctx->hslots[c].last_launches;
      cudaEventRecord(ctx->hev_done[c], cs);
      cudaStreamWaitEvent(stream, ctx->hev_done[c], 0);
    }
    ctx->api.last_launches = launches;
    ctx->api.last_buckets.clear();
  } else {
    if (c_flat && first_live >= 0 && ec > 0) {
      e = cudaMemcpyAsync(dC + off_c[first_live], C[first_live], 4 * (ec - off_c[first_live]),
                          cudaMemcpyHostToDevice, stream);
      if (e != cudaSuccess) return ctx_cuda(ctx, e, "H2D");
    }
    if (int rc = run_device_batch(ctx, ctx->api, insts, skip, algo, stream, true, true, &unsup, route_wide); rc)
      return rc;
  }
  ctx->last_k = k;
  ctx->last_skip = skip;
  std::vector<int> still;
  for (int t : unsup) {
    if (insts[t].m > large_max_cols() || algo == OT_AUCTION) { still.push_back(t); continue; }
    const int rc = solve_wide(ctx, insts[t], resolve_algo(ctx, algo, insts[t].m), stream, nullptr);
    if (rc == OT_ERR_TIMEOUT || rc == OT_ERR_UNSUPPORTED) { st[t] = rc; skip[t] = 1; continue; }
    if (rc != OT_OK) return rc;
  }
  unsup.swap(still);
  for (int t : unsup) { st[t] = OT_ERR_UNSUPPORTED; skip[t] = 1; ctx->last_skip[t] = 1; }
  std::vector<int32_t> hstatus(k, 0);
  if ((e = cudaMemcpyAsync(cost, dcost, sizeof(int64_t) * k, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
    return ctx_cuda(ctx, e, "D2H cost");
  cudaMemcpyAsync(hstatus.data(), dstatus, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, stream);
  const bool all_live = unsup.empty();
  if (first_live >= 0 && all_live && r_flat)
    cudaMemcpyAsync(r2c[first_live], dR + off_r[first_live], 4 * (er - off_r[first_live]), cudaMemcpyDeviceToHost, stream);
  if (first_live >= 0 && all_live && u_flat)
    cudaMemcpyAsync(u[first_live], dU + off_u[first_live], 8 * (er - off_u[first_live]), cudaMemcpyDeviceToHost, stream);
  if (first_live >= 0 && all_live && v_flat)
    cudaMemcpyAsync(v[first_live], dV + off_v[first_live], 8 * (ev - off_v[first_live]), cudaMemcpyDeviceToHost, stream);
  for (int t = 0; t < k; ++t) {
    if (st[t] != OT_OK || n[t] == 0) continue;
    if (!(all_live && r_flat))
      cudaMemcpyAsync(r2c[t], dR + off_r[t], 4 * size_t(n[t]), cudaMemcpyDeviceToHost, stream);
    if (u && u[t] && !(all_live && u_flat))
      cudaMemcpyAsync(u[t], dU + off_u[t], 8 * size_t(n[t]), cudaMemcpyDeviceToHost, stream);
    if (v && v[t] && !(all_live && v_flat))
      cudaMemcpyAsync(v[t], dV + off_v[t], 8 * size_t(m[t]), cudaMemcpyDeviceToHost, stream);
  }
  int64_t s8[8] = {0};
  if (stats_out && k >= 1 && !skip[0]) cudaMemcpyAsync(s8, insts[0].stats, sizeof(s8), cudaMemcpyDeviceToHost, stream);
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return ctx_cuda(ctx, e, "sync");
  for (int t = 0; t < k; ++t) {
    if (n[t] == 0 && st[t] == OT_OK) {
      cost[t] = 0;
      if (v && v[t]) std::memset(v[t], 0, sizeof(int64_t) * m[t]);
    }
    if (st[t] == OT_OK) st[t] = hstatus[t];
  }
  if (status)
    for (int t = 0; t < k; ++t) status[t] = st[t];
  if (stats_out) std::memcpy(stats_out, s8, sizeof(s8));
  if (k == 1 && st[0] != OT_OK)
    return ctx_fail(ctx, st[0], st[0] == OT_ERR_UNSUPPORTED ? "size not supported" : "instance failed: " + ctx->err);
  return OT_OK;
}

// ---------------------------------------------------------------------------
// exported API
// ---------------------------------------------------------------------------

int LaunchSlot::init() {
  return cudaEventCreateWithFlags(&meta_ev, cudaEventDisableTiming) == cudaSuccess ? OT_OK : OT_ERR_CUDA;
}

void LaunchSlot::clear_graphs() {
  for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
  graphs.clear();
  meta_valid = false;
}

static bool is_default_stream(cudaStream_t s) {
  return s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread;
}

StreamScope::StreamScope(cudaStream_t given, cudaStream_t own, cudaEvent_t in_ev, cudaEvent_t out)
    : user(given), work(given) {
  if (!is_default_stream(given)) return;
  work = own;
  out_ev = out;
  cudaEventRecord(in_ev, given ? given : cudaStreamLegacy);
  cudaStreamWaitEvent(own, in_ev, 0);
}

StreamScope::~StreamScope() {
  if (!out_ev) return;
  cudaEventRecord(out_ev, work);
  cudaStreamWaitEvent(user ? user : cudaStreamLegacy, out_ev, 0);
}

void LaunchSlot::release() {
  if (meta_pending && meta_ev) cudaEventSynchronize(meta_ev);
  meta_pending = false;
  clear_graphs();
  for (cudaEvent_t ev : tev) cudaEventDestroy(ev);
  tev.clear();
  d_meta.release();
  d_stats.release();
  d_pack.release();
  h_meta.release();
  if (meta_ev) cudaEventDestroy(meta_ev);
  meta_ev = nullptr;
}

extern "C" {

const char* ot_version(void) { return "otassign 0.1 sm_103a"; }

int ot_ctx_create(ot_ctx** out, const ot_config* cfg) {
  if (!out) return OT_ERR_ARG;
  *out = nullptr;
  ot_ctx* ctx = new (std::nothrow) ot_ctx();
  if (!ctx) return OT_ERR_OOM;
  ot_config c{};
  c.device = -1;
  if (cfg) c = *cfg;
  if (c.device >= 0) {
    if (cudaSetDevice(c.device) != cudaSuccess) { delete ctx; return OT_ERR_CUDA; }
    ctx->device = c.device;
  } else {
    if (cudaGetDevice(&ctx->device) != cudaSuccess) { cudaGetLastError(); delete ctx; return OT_ERR_CUDA; }
  }
  if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { delete ctx; return OT_ERR_CUDA; }
  for (int i = 0; i < kForkStreams; ++i) {
    cudaStreamCreateWithFlags(&ctx->bstreams[i], cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&ctx->join_ev[i], cudaEventDisableTiming);
  }
  cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
  for (cudaEvent_t* ev : {&ctx->join_in_ev, &ctx->join_out_ev, &ctx->sjoin_in_ev, &ctx->sjoin_out_ev})
    if (cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess) { ot_ctx_destroy(ctx); return OT_ERR_CUDA; }
  if (ctx->api.init() != OT_OK) { ot_ctx_destroy(ctx); return OT_ERR_CUDA; }
  if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->hev_start, cudaEventDisableTiming) != cudaSuccess) {
    ot_ctx_destroy(ctx);
    return OT_ERR_CUDA;
  }
  for (int c = 0; c < kHostChunks; ++c) {
    if (cudaStreamCreateWithFlags(&ctx->cstreams[c], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->hev_copy[c], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->hev_done[c], cudaEventDisableTiming) != cudaSuccess ||
        ctx->hslots[c].init() != OT_OK) {
      ot_ctx_destroy(ctx);
      return OT_ERR_CUDA;
    }
    ctx->hslots[c].use_graphs = true;
  }
  ctx->api.use_graphs = true;
  ctx->api.timing = true;
  default_table(ctx->table);
  default_auto(ctx->auto_algo);
  if (c.tune_file) {
    ctx->tune_file = c.tune_file;
    load_tune_file(ctx);
  }
  ctx->pack_rows = (c.flags & OT_CFG_NO_ROW_PACKING) == 0;
  ctx->max_group_ctas = std::max(0, c.max_group_ctas);
  ctx->step_limit = std::max<int64_t>(0, c.step_limit);
  ctx->dense_wide = (c.flags & OT_CFG_DENSE_WIDE) != 0;
  if (int rc = serve_init(ctx, c); rc) { ot_ctx_destroy(ctx); return rc; }
  if (cudaGetLastError() != cudaSuccess) { ot_ctx_destroy(ctx); return OT_ERR_CUDA; }
  *out = ctx;
  return OT_OK;
}

void ot_ctx_destroy(ot_ctx* ctx) {
  if (!ctx) return;
  serve_shutdown(ctx);
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ctx->api.release();
  for (int c = 0; c < kHostChunks; ++c) {
    if (ctx->cstreams[c]) { cudaStreamSynchronize(ctx->cstreams[c]); cudaStreamDestroy(ctx->cstreams[c]); }
    ctx->hslots[c].release();
    if (ctx->hev_copy[c]) cudaEventDestroy(ctx->hev_copy[c]);
    if (ctx->hev_done[c]) cudaEventDestroy(ctx->hev_done[c]);
  }
  if (ctx->copy_stream) { cudaStreamSynchronize(ctx->copy_stream); cudaStreamDestroy(ctx->copy_stream); }
  if (ctx->hev_start) cudaEventDestroy(ctx->hev_start);
  for (int i = 0; i < kForkStreams; ++i) {
    if (ctx->bstreams[i]) { cudaStreamSynchronize(ctx->bstreams[i]); cudaStreamDestroy(ctx->bstreams[i]); }
    if (ctx->join_ev[i]) cudaEventDestroy(ctx->join_ev[i]);
  }
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  for (cudaEvent_t ev : {ctx->join_in_ev, ctx->join_out_ev, ctx->sjoin_in_ev, ctx->sjoin_out_ev})
    if (ev) cudaEventDestroy(ev);
  ctx->d_status.release();
  ctx->d_io.release();
  ctx->d_scratch.release();
  ctx->d_large.release();
  ctx->d_scaled.release();
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* ot_last_error_string(const ot_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int ot_assign_solve(ot_ctx* ctx, const int32_t* C, int64_t ldc, int32_t n, int32_t m, int32_t algo,
                    int32_t* row_to_col, int64_t* cost, int64_t* u, int64_t* v, void* stream) {
  if (!ctx) return OT_ERR_ARG;
  if (check_sizes(C, ldc, n, m) != OT_OK || !cost || (n > 0 && !row_to_col))
    return ctx_fail(ctx, OT_ERR_ARG, "bad arguments");
  cudaSetDevice(ctx->device);
  const int32_t* Cs[1] = {C};
  int64_t ld[1] = {ldc};
  int32_t ns[1] = {n}, ms[1] = {m};
  int32_t* rs[1] = {row_to_col};
  int64_t* us[1] = {u};
  int64_t* vs[1] = {v};
  int32_t status = 0;
  // single device solves report their status when asked via *_stats
  const bool dev = n > 0 ? ptr_on_device(C) : ptr_on_device(cost);
  return solve_many(ctx, 1, Cs, ld, ns, ms, algo, rs, cost, u ? us : nullptr, v ? vs : nullptr,
                    dev ? nullptr : &status, static_cast<cudaStream_t>(stream), nullptr, true);
}

int ot_assign_solve_stats(ot_ctx* ctx, const int32_t* C, int64_t ldc, int32_t n, int32_t m,
                          int32_t algo, int32_t* row_to_col, int64_t* cost, int64_t* u, int64_t* v,
                          ot_stats* stats, void* stream) {
  if (!ctx || !stats) return OT_ERR_ARG;
  if (check_sizes(C, ldc, n, m) != OT_OK || !cost || (n > 0 && !row_to_col))
    return ctx_fail(ctx, OT_ERR_ARG, "bad arguments");
  cudaSetDevice(ctx->device);
  std::memset(stats, 0, sizeof(*stats));
  const int32_t* Cs[1] = {C};
  int64_t ld[1] = {ldc};
  int32_t ns[1] = {n}, ms[1] = {m};
  int32_t* rs[1] = {row_to_col};
  int64_t* us[1] = {u};
  int64_t* vs[1] = {v};
  int32_t status = 0;
  int rc = solve_many(ctx, 1, Cs, ld, ns, ms, algo, rs, cost, u ? us : nullptr, v ? vs : nullptr,
                      &status, static_cast<cudaStream_t>(stream), stats, true);
  if (rc == OT_OK && status != 0) return ctx_fail(ctx, status, "device status error");
  return rc;
}

int ot_assign_solve_batched(ot_ctx* ctx, int32_t k, const int32_t* const* C, const int64_t* ldc,
                            const int32_t* n, const int32_t* m, int32_t algo,
                            int32_t* const* row_to_col, int64_t* cost, int64_t* const* u,
                            int64_t* const* v, int32_t* status, void* stream) {
  if (!ctx) return OT_ERR_ARG;
  cudaSetDevice(ctx->device);
  return solve_many(ctx, k, C, ldc, n, m, algo, row_to_col, cost, u, v, status,
                    static_cast<cudaStream_t>(stream), nullptr, false);
}

int ot_last_call_stats(ot_ctx* ctx, ot_stats* total) {
  if (!ctx || !total) return OT_ERR_ARG;
  std::memset(total, 0, sizeof(*total));
  std::lock_guard<std::mutex> lock(ctx->api_mu);
  cudaSetDevice(ctx->device);
  if (ctx->api.meta_pending) cudaEventSynchronize(ctx->api.meta_ev);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "sync");
  const int k = ctx->last_k;
  if (k > 0 && ctx->api.d_stats.ptr) {
    std::vector<int64_t> h(size_t(k) * 8);
    e = cudaMemcpy(h.data(), ctx->api.d_stats.ptr, h.size() * sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "stats copy");
    for (int t = 0; t < k; ++t) {
      if (ctx->last_skip.size() == size_t(k) && ctx->last_skip[t]) continue;
      total->steps += h[t * 8 + 0];
      total->rows_scanned += h[t * 8 + 1];
      total->cost_bytes += h[t * 8 + 2];
      total->phases += h[t * 8 + 3];
      total->augmentations += h[t * 8 + 4];
      total->init_bytes += h[t * 8 + 5];
      total->reserved[1] += h[t * 8 + 7];
    }
  }
  total->reserved[0] = ctx->api.last_launches;
  return OT_OK;
}

int ot_last_call_launches(ot_ctx* ctx, ot_launch_info* out, int32_t max, int32_t* count) {
  if (!ctx || !count || max < 0 || (max > 0 && !out)) return OT_ERR_ARG;
  std::lock_guard<std::mutex> lock(ctx->api_mu);
  cudaSetDevice(ctx->device);
  LaunchSlot& slot = ctx->api;
  if (slot.meta_pending) cudaEventSynchronize(slot.meta_ev);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "sync");
  const int nb = int(slot.last_buckets.size());
  *count = nb;
  std::vector<int64_t> h;
  const int k = ctx->last_k;
  if (k > 0 && slot.d_stats.ptr) {
    h.resize(size_t(k) * 8);
    if ((e = cudaMemcpy(h.data(), slot.d_stats.ptr, h.size() * sizeof(int64_t), cudaMemcpyDeviceToHost)) !=
        cudaSuccess)
      return ctx_cuda(ctx, e, "stats copy");
  }
  for (int b = 0; b < nb && b < max; ++b) {
    const LaunchSlot::BucketInfo& bi = slot.last_buckets[b];
    ot_launch_info& o = out[b];
    std::memset(&o, 0, sizeof(o));
    o.algo = bi.algo == kAlgoAuction ? OT_AUCTION : bi.algo;
    o.threads_per_instance = bi.tpi;
    o.cols_per_thread = bi.k;
    o.instances = int32_t(bi.idx.size());
    o.ms = -1.0f;
    if (slot.timing && slot.tev.size() >= size_t(2 * nb)) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, slot.tev[2 * b], slot.tev[2 * b + 1]) == cudaSuccess) o.ms = ms;
      else cudaGetLastError();
    }
    for (int t : bi.idx) {
      if (size_t(t) * 8 + 7 >= h.size()) continue;
      o.read_bytes += h[size_t(t) * 8 + 7];
      o.init_bytes += h[size_t(t) * 8 + 5];
    }
  }
  return OT_OK;
}

int ot_tune_lookup(ot_ctx* ctx, int32_t algo, int32_t m, int32_t* tpi, int32_t* k) {
  if (!ctx || (algo != OT_KM && algo != OT_BKM && algo != OT_AUTO) || m < 0) return OT_ERR_ARG;
  algo = resolve_algo(ctx, algo, m);
  const int sh = m > kMaxGroupCols ? kLargeEngine : ctx->table[algo][bucket_of(m)];
  if (sh == kLargeEngine) {
    if (tpi) *tpi = 0;
    if (k) *k = 0;
    return OT_OK;
  }
  if (sh < 0) return OT_ERR_UNSUPPORTED;
  if (tpi) *tpi = group_shape(sh).tpi;
  if (k) *k = group_shape(sh).k;
  return OT_OK;
}

int ot_tune_set(ot_ctx* ctx, int32_t algo, int32_t m, int32_t tpi, int32_t k) {
  if (!ctx || (algo != OT_KM && algo != OT_BKM && algo != OT_AUTO) || m < 0) return OT_ERR_ARG;
  if (algo == OT_AUTO) {  // tpi selects the algorithm OT_AUTO uses for this bucket
    if (tpi != OT_KM && tpi != OT_BKM) return ctx_fail(ctx, OT_ERR_ARG, "auto entry must name KM or BKM");
    ctx->auto_algo[bucket_of(m)] = tpi;
    return OT_OK;
  }
  if (tpi == 0 && k == 0) {  // route the bucket to the cluster engine
    ctx->table[algo][bucket_of(m)] = kLargeEngine;
    ctx->tuned[algo][bucket_of(m)] = true;
    return OT_OK;
  }
  const int sh = shape_index(tpi, k);
  const int b = bucket_of(m);
  if (sh < 0 || group_shape(sh).max_cols() < (32 << b) || m > kMaxGroupCols)
    return ctx_fail(ctx, OT_ERR_UNSUPPORTED, "shape not available for this bucket");
  ctx->table[algo][b] = sh;
  ctx->tuned[algo][b] = true;
  return OT_OK;
}

int ot_autotune(ot_ctx* ctx, int32_t k, const int32_t* const* C, const int64_t* ldc,
                const int32_t* n, const int32_t* m, int32_t algo, int32_t repeats) {
  if (!ctx) return OT_ERR_ARG;
  if ((algo != OT_KM && algo != OT_BKM && algo != OT_AUTO) || k <= 0 || !C || !ldc || !n || !m)
    return ctx_fail(ctx, OT_ERR_ARG, "bad arguments");
  cudaSetDevice(ctx->device);
  repeats = std::max(1, repeats);
  std::lock_guard<std::mutex> lock(ctx->api_mu);
  // the instances may still be in flight on any of the caller's streams
  if (cudaError_t e = cudaDeviceSynchronize(); e != cudaSuccess) return ctx_cuda(ctx, e, "autotune sync");
  // scratch outputs for every instance
  size_t total = al256(sizeof(int64_t) * k) + al256(sizeof(int32_t) * k);
  std::vector<size_t> off(k);
  for (int t = 0; t < k; ++t) {
    if (check_sizes(C[t], ldc[t], n[t], m[t]) != OT_OK || !ptr_on_device(C[t]))
      return ctx_fail(ctx, OT_ERR_ARG, "autotune needs valid device instances");
    off[t] = total;
    total += al256(4 * size_t(n[t])) + al256(8 * size_t(n[t])) + al256(8 * size_t(m[t])) + al256(64);
  }
  if (int rc = ctx->d_scratch.reserve(total); rc) return ctx_fail(ctx, rc, "scratch alloc");
  char* D = static_cast<char*>(ctx->d_scratch.ptr);
  std::vector<Instance> insts(k);
  for (int t = 0; t < k; ++t) {
    Instance& I = insts[t];
    I.C = C[t]; I.ldc = ldc[t]; I.n = n[t]; I.m = m[t];
    char* p = D + off[t];
    I.row_to_col = reinterpret_cast<int32_t*>(p); p += al256(4 * size_t(n[t]));
    I.u = reinterpret_cast<int64_t*>(p); p += al256(8 * size_t(n[t]));
    I.v = reinterpret_cast<int64_t*>(p); p += al256(8 * size_t(m[t]));
    I.stats = reinterpret_cast<int64_t*>(p);
    I.cost = reinterpret_cast<int64_t*>(D) + t;
    I.status = reinterpret_cast<int32_t*>(D + al256(sizeof(int64_t) * k)) + t;
  }
  // group instances by m-bucket
  std::map<int, std::vector<int>> byb;
  for (int t = 0; t < k; ++t)
    if (n[t] > 0 && m[t] <= kMaxGroupCols) byb[bucket_of(m[t])].push_back(t);
  // time what the solves run: rows packed to 16 bits (and the 32-bit path)
  // whenever the batched launches pack them
  bool packed = false;
  if (ctx->pack_rows) {
    size_t nrows = 0, nelem = 0;
    for (auto& kv : byb)
      for (int t : kv.second) { nrows += size_t(n[t]); nelem += size_t(n[t]) * m[t]; }
    const size_t b_pok = al256(sizeof(int32_t) * k), b_roff = al256(sizeof(int32_t) * nrows);
    if (nelem > 0 && ctx->api.d_pack.reserve(b_pok + b_roff + al256(2 * nelem)) == OT_OK) {
      char* base = static_cast<char*>(ctx->api.d_pack.ptr);
      size_t orow = 0, oel = 0;
      for (auto& kv : byb)
        for (int t : kv.second) {
          insts[t].pok = reinterpret_cast<int32_t*>(base) + t;
          insts[t].roff = reinterpret_cast<int32_t*>(base + b_pok) + orow;
          insts[t].P = reinterpret_cast<uint16_t*>(base + b_pok + b_roff) + oel;
          orow += size_t(n[t]);
          oel += size_t(n[t]) * m[t];
        }
      packed = true;
    }
  }
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const size_t desc_bytes = al256(sizeof(Instance) * k);
  if (ctx->api.meta_pending) { cudaEventSynchronize(ctx->api.meta_ev); ctx->api.meta_pending = false; }
  if (int rc = ctx->api.d_meta.reserve(desc_bytes + al256(4 * size_t(k)) + 256); rc) return ctx_fail(ctx, rc, "meta alloc");
  ctx->api.clear_graphs();
  char* dm = static_cast<char*>(ctx->api.d_meta.ptr);
  Instance* dinst = reinterpret_cast<Instance*>(dm);
  int32_t* dorder = reinterpret_cast<int32_t*>(dm + desc_bytes);
  int* dwork = reinterpret_cast<int*>(dm + desc_bytes + al256(4 * size_t(k)));
  cudaMemcpyAsync(dinst, insts.data(), sizeof(Instance) * k, cudaMemcpyHostToDevice, s);
  if (packed) {
    if (cudaError_t e = launch_pack(dinst, nullptr, k, s); e != cudaSuccess) return ctx_cuda(ctx, e, "autotune pack");
  }
  FILE* tf = ctx->tune_file.empty() ? nullptr : std::fopen(ctx->tune_file.c_str(), "a");
  for (auto& kv : byb) {
    std::vector<int>& idx = kv.second;
    int nmax = 0, mmax = 0;
    for (int t : idx) { nmax = std::max(nmax, n[t]); mmax = std::max(mmax, m[t]); }
    std::sort(idx.begin(), idx.end(), [&](int a, int c) {
      return (long long)n[a] * m[a] > (long long)n[c] * m[c];
    });
    cudaMemcpyAsync(dorder, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice, s);
    // OT_AUTO tunes both algorithms and keeps the faster for the bucket
    int best_algo = -1;
    float best_algo_ms = 1e30f;
    for (int a = 0; a < 2; ++a) {
      if (algo != OT_AUTO && a != algo) continue;
      int best = -1;
      float best_ms = 1e30f;
      for (int sh = 0; sh < num_group_shapes(); ++sh) {
        GroupShape g = group_shape(sh);
        if (g.max_cols() < mmax || g.max_cols() > 8 * std::max(mmax, 32)) continue;
        if (group_smem_bytes(g, a, nmax, mmax) > group_smem_limit()) continue;
        float tmin = 1e30f;
        bool ok = true;
        for (int r = 0; r < repeats + 1 && ok; ++r) {
          cudaMemsetAsync(dwork, 0, sizeof(int), s);
          cudaEventRecord(e0, s);
          if (launch_group(g, a, dinst, dorder, int(idx.size()), dwork, nmax, mmax, 0, s) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
            break;
          }
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          if (r > 0) tmin = std::min(tmin, ms);  // first run warms up
        }
        if (ok && tmin < best_ms) { best_ms = tmin; best = sh; }
      }
      if (best >= 0) {
        ctx->table[a][kv.first] = best;
        ctx->tuned[a][kv.first] = true;
        if (tf)
          std::fprintf(tf, "{\"algo\": %d, \"bucket_mmax\": %d, \"tpi\": %d, \"k\": %d, \"ms\": %.4f}\n",
                       a, 32 << kv.first, group_shape(best).tpi, group_shape(best).k, best_ms);
        if (best_ms < best_algo_ms) { best_algo_ms = best_ms; best_algo = a; }
      }
    }
    if (algo == OT_AUTO && best_algo >= 0) {
      ctx->auto_algo[kv.first] = best_algo;
      if (tf) std::fprintf(tf, "{\"auto\": %d, \"bucket_mmax\": %d, \"ms\": %.4f}\n", best_algo, 32 << kv.first, best_algo_ms);
    }
  }
  if (tf) std::fclose(tf);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "autotune");
  return OT_OK;
}

}  // extern "C"

// JSON-lines table: {"algo": A, "bucket_mmax": M, "tpi": T, "k": K, ...}; later
// lines override earlier ones.
void load_tune_file(ot_ctx* ctx) {
  FILE* f = std::fopen(ctx->tune_file.c_str(), "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    int a = -1, mm = -1, tpi = -1, kk = -1;
    const char* p;
    if ((p = std::strstr(line, "\"algo\":"))) a = std::atoi(p + 7);
    if ((p = std::strstr(line, "\"bucket_mmax\":"))) mm = std::atoi(p + 14);
    if ((p = std::strstr(line, "\"tpi\":"))) tpi = std::atoi(p + 6);
    if ((p = std::strstr(line, "\"k\":"))) kk = std::atoi(p + 4);
    int au = -1;
    if ((p = std::strstr(line, "\"auto\":"))) au = std::atoi(p + 7);
    const int sh = shape_index(tpi, kk);
    if ((a == 0 || a == 1) && mm > 0 && sh >= 0) {
      ctx->table[a][bucket_of(mm)] = sh;
      ctx->tuned[a][bucket_of(mm)] = true;
    }
    if ((au == 0 || au == 1) && mm > 0) ctx->auto_algo[bucket_of(mm)] = au;
  }
  std::fclose(f);
}
