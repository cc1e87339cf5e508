// Serving loop of libotassign.so: continuous batching of independent solves.
//
// submit() reserves a block of a device arena (the HBM budget) for the
// request -- cost matrix, duals, assignment, counters -- and copies the cost
// matrix in; a request that does not fit yet waits in a host-side queue with
// its own copy of C.  Requests with m <= 2048 are published, as soon as
// their matrix is in the arena, to a persistent grid of solver groups that
// pull them from a ring one by one (a request starts as soon as a group is
// free, whatever else is running); wider ones are packed into waves launched
// on several streams.  Each request finishes on its own: the solver group
// writes the results and then, after a system-scope fence, a status word in
// mapped host memory, which poll() reads.  poll() copies the results out and
// frees the arena block, which lets queued requests in.  Requests on the
// persistent grid write their results (assignment, duals, cost, counters)
// straight into a slot of mapped pinned host memory, so that poll() of a
// finished grid request is a host copy with no CUDA call; when every slot
// is taken a request writes them into its arena block instead.
#include <algorithm>

#ifndef OT_SERVE_PACK
#define OT_SERVE_PACK 1
#endif
#include <chrono>
#include <cstring>

#include "ot_ctx.h"
#include "ot_group.cuh"

using namespace ot;

namespace {

constexpr int32_t kFlagPending = 0x7fffffff;
constexpr size_t kDefaultBudget = size_t(4) << 30;

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// First-fit allocator over one device slab, with coalescing frees.
struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  std::map<size_t, size_t> free_blocks;  // offset -> bytes
  int init(size_t bytes) {
    if (base) return OT_OK;
    if (cudaMalloc(&base, bytes) != cudaSuccess) {
      cudaGetLastError();
      base = nullptr;
      return OT_ERR_OOM;
    }
    size = bytes;
    free_blocks.clear();
    free_blocks[0] = bytes;
    return OT_OK;
  }
  bool alloc(size_t bytes, size_t* off) {
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t at = it->first + bytes;
      free_blocks.erase(it);
      if (rest) free_blocks[at] = rest;
      used += bytes;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    used -= bytes;
    auto it = free_blocks.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_blocks.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_blocks.erase(nx);
    }
    if (it != free_blocks.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_blocks.erase(it);
      }
    }
  }
  void destroy() {
    if (base) cudaFree(base);
    base = nullptr;
  }
};

struct Req {
  int n = 0, m = 0, algo = 0;
  size_t bytes = 0, off = 0;
  int flag = -1;                 // slot in the mapped status array
  int res = -1;                  // slot in the mapped result pool (grid requests), or -1
  bool admitted = false, launched = false;
  bool submitting = true;        // submit() has not returned the ticket yet
  bool cancelled = false;        // cancelled while its wave runs: reclaimed once finished
  std::vector<int32_t> host_C;  // packed copy while waiting for admission
};

struct Wave {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  LaunchSlot slot;
};

// offsets inside one request's arena block
struct Layout {
  size_t c, r2c, u, v, cost, stats, total;
  Layout(int n, int m) {
    c = 0;
    r2c = c + al256(4 * size_t(n) * m);
    u = r2c + al256(4 * size_t(n));
    v = u + al256(8 * size_t(n));
    cost = v + al256(8 * size_t(m));
    stats = cost + 256;
    total = stats + 256;
  }
};

// ---------------------------------------------------------------------------
// Persistent serving grid.  Resident solver groups of kPTPI threads (each
// owning kPK columns per thread, so m <= kPMaxCols) pull request
// descriptors from a ring in mapped host memory as the serving thread
// publishes them, solve each request (KM or batched KM, the group engine's
// step sequence) and write its status word, then pull the next one.  Every
// wait is bounded: a group that finds the ring empty polls with a growing
// sleep and leaves after kIdlePolls polls (the host relaunches the grid when
// new work arrives and none is resident); a stop flag ends it at once.
// ---------------------------------------------------------------------------
constexpr int kPTPI = 512, kPK = 4;
constexpr int kPMaxCols = kPTPI * kPK;
constexpr int kIdlePolls = 1 << 14;

// Mapped result pool of the persistent grid: kResSlots slots, each holding
// the results of one request of m <= kPMaxCols (41.5 KB; 42.5 MB of pinned
// host memory in all).
constexpr int kResSlots = 1024;
struct ResLayout {
  static constexpr size_t r2c = 0;
  static constexpr size_t u = r2c + 4 * size_t(kPMaxCols);
  static constexpr size_t v = u + 8 * size_t(kPMaxCols);
  static constexpr size_t cost = v + 8 * size_t(kPMaxCols);
  static constexpr size_t stats = cost + 256;
  static constexpr size_t total = stats + 256;
};
static_assert(ResLayout::total % 256 == 0, "result slots stay 256-byte aligned");

struct PQueue {                    // mapped pinned host memory
  unsigned long long tail;         // requests published (written by the host)
  int stop;                        // the host asks the grid to leave
  int pad;
};

struct PItem {                     // one published request
  Instance I;
  int algo;
  int pad;
};
static_assert(sizeof(PItem) % 8 == 0, "descriptor copied in 8-byte words");

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(kPTPI) serve_kernel(PQueue* q, const PItem* ring, int cap,
                                                      unsigned long long* head) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kWords = int(sizeof(PItem) / 8);
  __shared__ long long s_slot;
  __shared__ unsigned long long s_item[kWords];
  const int t = threadIdx.x;
  for (;;) {
    if (t == 0) {
      long long slot = -1;
      for (int poll = 0; poll < kIdlePolls && slot < 0; ++poll) {
        if (*reinterpret_cast<volatile int*>(&q->stop)) break;
        const unsigned long long tl = ld_acquire_sys(&q->tail);
        const unsigned long long h = *reinterpret_cast<volatile unsigned long long*>(head);
        if (h < tl) {
          if (atomicCAS(head, h, h + 1) == h) slot = (long long)h;
        } else {
          __nanosleep(poll < 32 ? 256 : 4096);
        }
      }
      s_slot = slot;
      if (slot >= 0) {
        // the descriptor, read past any cached copy of an earlier use of
        // the slot
        const volatile unsigned long long* src =
            reinterpret_cast<const volatile unsigned long long*>(ring + slot % cap);
        for (int x = 0; x < kWords; ++x) s_item[x] = src[x];
      }
    }
    __syncthreads();
    const long long slot = s_slot;
    if (slot < 0) break;
    const PItem& it = *reinterpret_cast<const PItem*>(s_item);
    const Instance I = it.I;
    const int algo = it.algo;
    __syncthreads();  // every thread has read s_slot and the descriptor
    if (algo == kAlgoKM) {
      const GroupSmem S = carve(smem_raw, kPTPI, kAlgoKM, kPMaxCols, kPMaxCols);
      solve_instance<kPTPI, kPK, kAlgoKM>(I, S, t);
    } else {
      const GroupSmem S = carve(smem_raw, kPTPI, kAlgoBKM, kPMaxCols, kPMaxCols);
      solve_instance<kPTPI, kPK, kAlgoBKM>(I, S, t);
    }
  }
}

}  // namespace

struct ServeState {
  ot_ctx* ctx = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::thread th;
  bool stop = false;
  bool started = false;
  Arena arena;
  size_t budget = kDefaultBudget;
  int max_inflight = 4096;
  int inflight = 0;
  std::unordered_map<uint64_t, Req> reqs;
  std::deque<uint64_t> pending, ready;
  std::vector<Wave> waves;
  int32_t* flags = nullptr;  // mapped pinned host memory
  int32_t* dflags = nullptr;
  std::vector<int> free_flags;
  uint64_t next_ticket = 1;
  cudaStream_t copy_stream = nullptr, poll_stream = nullptr;
  cudaEvent_t copy_ev = nullptr;
  int64_t n_submitted = 0, n_admitted = 0, n_completed = 0, n_waves = 0, max_busy = 0, n_refused = 0;
  int n_cancel_wait = 0;  // cancelled requests whose wave has not finished

  // persistent grid (requests with m <= kPMaxCols)
  PQueue* pq = nullptr;                 // mapped pinned host memory
  PQueue* dpq = nullptr;                // its device address
  PItem* pring = nullptr;               // mapped ring of published requests
  PItem* dpring = nullptr;
  unsigned long long* dhead = nullptr;  // requests taken by the grid (device)
  int pcap = 0;
  unsigned long long ptail = 0;         // requests published
  cudaStream_t pstream = nullptr;
  cudaEvent_t pev = nullptr;            // end of the latest grid launch
  char* hres = nullptr;                 // mapped result pool (host address)
  char* dres = nullptr;                 // its device address
  std::vector<int> free_res;
  bool prun = false;
  int pgrid = 0;
  size_t psmem = 0;
  std::vector<uint64_t> plive;          // published, status not yet seen final
  std::vector<uint64_t> watch;          // launched, not yet returned by ot_assign_completed

  int start();
  void loop();
  bool try_admit(uint64_t t, Req& r);
  Instance make_instance(const Req& r) const;
  void publish(uint64_t t, Req& r);
  void ensure_grid();
  void launch_ready();
  void release(uint64_t t, Req& r);
  void reclaim_cancelled();
};

int ServeState::start() {
  if (started) return OT_OK;
  if (int rc = arena.init(budget); rc) return rc;
  if (cudaHostAlloc(&flags, sizeof(int32_t) * max_inflight, cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return OT_ERR_OOM;
  }
  if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&dflags), flags, 0) != cudaSuccess) return OT_ERR_CUDA;
  for (int i = max_inflight - 1; i >= 0; --i) free_flags.push_back(i);
  cudaStreamCreateWithFlags(&copy_stream, cudaStreamNonBlocking);
  cudaStreamCreateWithFlags(&poll_stream, cudaStreamNonBlocking);
  cudaEventCreateWithFlags(&copy_ev, cudaEventDisableTiming);
  for (Wave& w : waves) {
    cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
    if (w.slot.init() != OT_OK) return OT_ERR_CUDA;
    // 16-bit packing of serving waves (an extra pass over each wave's
    // matrices, and the 32-bit solver path for packed instances)
    w.slot.pack = OT_SERVE_PACK != 0;
  }
  // the persistent grid's queue, ring and head counter
  pcap = max_inflight;
  if (cudaHostAlloc(&pq, sizeof(PQueue), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&pring, sizeof(PItem) * size_t(pcap), cudaHostAllocMapped) != cudaSuccess ||
      cudaMalloc(&dhead, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return OT_ERR_OOM;
  }
  std::memset(pq, 0, sizeof(PQueue));
  if (cudaHostAlloc(&hres, ResLayout::total * kResSlots, cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return OT_ERR_OOM;
  }
  if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&dres), hres, 0) != cudaSuccess) return OT_ERR_CUDA;
  for (int i = kResSlots - 1; i >= 0; --i) free_res.push_back(i);
  if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&dpq), pq, 0) != cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void**>(&dpring), pring, 0) != cudaSuccess ||
      cudaMemset(dhead, 0, sizeof(unsigned long long)) != cudaSuccess)
    return OT_ERR_CUDA;
  cudaStreamCreateWithFlags(&pstream, cudaStreamNonBlocking);
  cudaEventCreateWithFlags(&pev, cudaEventDisableTiming);
  psmem = group_bytes(kPTPI, kAlgoBKM, kPMaxCols, kPMaxCols);
  if (cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(psmem)) != cudaSuccess)
    return OT_ERR_CUDA;
  {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_kernel, kPTPI, psmem) != cudaSuccess ||
        per_sm < 1)
      return OT_ERR_CUDA;
    pgrid = per_sm * sms;
  }
  if (cudaGetLastError() != cudaSuccess) return OT_ERR_CUDA;
  started = true;
  const int dev = ctx->device;
  th = std::thread([this, dev] {
    cudaSetDevice(dev);
    loop();
  });
  return OT_OK;
}

// Caller holds mu.  Reserve arena space and a status slot for request t.
bool ServeState::try_admit(uint64_t, Req& r) {
  if (inflight >= max_inflight || free_flags.empty()) return false;
  size_t off = 0;
  if (!arena.alloc(r.bytes, &off)) return false;
  r.off = off;
  r.flag = free_flags.back();
  free_flags.pop_back();
  flags[r.flag] = kFlagPending;
  r.admitted = true;
  ++inflight;
  ++n_admitted;
  return true;
}

// The device descriptor of an admitted request (its arena block).
Instance ServeState::make_instance(const Req& r) const {
  Layout L(r.n, r.m);
  char* b = arena.base + r.off;
  Instance I = {};
  I.C = reinterpret_cast<const int32_t*>(b + L.c);
  I.ldc = r.m;
  I.n = r.n;
  I.m = r.m;
  I.row_to_col = reinterpret_cast<int32_t*>(b + L.r2c);
  I.u = reinterpret_cast<int64_t*>(b + L.u);
  I.v = reinterpret_cast<int64_t*>(b + L.v);
  I.cost = reinterpret_cast<int64_t*>(b + L.cost);
  I.stats = reinterpret_cast<int64_t*>(b + L.stats);
  I.status = dflags + r.flag;
  I.step_limit = ctx->step_limit;
  return I;
}

// Caller holds mu.  Hand request t (its matrix in the arena) to the
// persistent grid: descriptor into the ring, then the tail, with release
// order (the grid reads the tail with acquire order before the descriptor).
void ServeState::publish(uint64_t t, Req& r) {
  PItem& it = pring[ptail % static_cast<unsigned long long>(pcap)];
  Instance I = make_instance(r);
  if (!free_res.empty()) {
    r.res = free_res.back();
    free_res.pop_back();
    char* b = dres + size_t(r.res) * ResLayout::total;
    I.row_to_col = reinterpret_cast<int32_t*>(b + ResLayout::r2c);
    I.u = reinterpret_cast<int64_t*>(b + ResLayout::u);
    I.v = reinterpret_cast<int64_t*>(b + ResLayout::v);
    I.cost = reinterpret_cast<int64_t*>(b + ResLayout::cost);
    I.stats = reinterpret_cast<int64_t*>(b + ResLayout::stats);
  }
  it.I = I;
  it.algo = r.algo;
  it.pad = 0;
  ++ptail;
  __atomic_store_n(&pq->tail, ptail, __ATOMIC_RELEASE);
  r.launched = true;
  plive.push_back(t);
  watch.push_back(t);
}

// Caller holds mu.  Launch the grid unless one is resident.  (Groups that
// had already decided to leave may miss a request published meanwhile; the
// serving thread then finds it unfinished with no grid resident and
// launches again.)
void ServeState::ensure_grid() {
  if (prun && cudaEventQuery(pev) != cudaSuccess) return;  // still resident
  serve_kernel<<<pgrid, kPTPI, psmem, pstream>>>(dpq, dpring, pcap, dhead);
  cudaEventRecord(pev, pstream);
  prun = true;
  ++n_waves;
}

// Caller holds mu.  Return request t's arena block and status slot and
// forget it.
void ServeState::release(uint64_t t, Req& r) {
  if (r.admitted) {
    arena.release(r.off, r.bytes);
    free_flags.push_back(r.flag);
    --inflight;
  }
  if (r.res >= 0) free_res.push_back(r.res);
  reqs.erase(t);
}

// Caller holds mu.  Cancelled requests whose solver has written its status
// word no longer use their block.
void ServeState::reclaim_cancelled() {
  if (n_cancel_wait == 0) return;
  std::vector<uint64_t> done;
  for (auto& kv : reqs) {
    const Req& r = kv.second;
    if (r.cancelled && *reinterpret_cast<volatile int32_t*>(&flags[r.flag]) != kFlagPending) done.push_back(kv.first);
  }
  for (uint64_t t : done) {
    release(t, reqs[t]);
    --n_cancel_wait;
  }
}

// Caller holds mu.  Requests the persistent grid takes are published at
// once; every other admitted request is launched as one wave.
void ServeState::launch_ready() {
  if (ready.empty()) return;
  {
    std::deque<uint64_t> rest;
    bool any = false;
    for (uint64_t t : ready) {
      auto it = reqs.find(t);
      if (it == reqs.end()) continue;
      if (it->second.m <= kPMaxCols) {
        publish(t, it->second);
        any = true;
      } else {
        rest.push_back(t);
      }
    }
    ready.swap(rest);
    if (any) ensure_grid();
    if (ready.empty()) return;
  }
  Wave* w = nullptr;
  int busy = 0;
  for (Wave& x : waves) {
    if (x.busy && cudaEventQuery(x.done) == cudaSuccess) x.busy = false;
    busy += x.busy;
  }
  for (Wave& x : waves)
    if (!x.busy) { w = &x; break; }
  if (!w) return;
  std::vector<uint64_t> tk(ready.begin(), ready.end());
  ready.clear();
  // copies issued by the serving thread must land before the wave starts
  cudaEventRecord(copy_ev, copy_stream);
  cudaStreamWaitEvent(w->stream, copy_ev, 0);
  for (int algo = 0; algo < 2; ++algo) {
    std::vector<Instance> insts;
    std::vector<uint64_t> ids;
    for (uint64_t t : tk) {
      Req& r = reqs[t];
      if (r.algo != algo) continue;
      Layout L(r.n, r.m);
      char* b = arena.base + r.off;
      Instance I = {};
      I.C = reinterpret_cast<const int32_t*>(b + L.c);
      I.ldc = r.m;
      I.n = r.n;
      I.m = r.m;
      I.row_to_col = reinterpret_cast<int32_t*>(b + L.r2c);
      I.u = reinterpret_cast<int64_t*>(b + L.u);
      I.v = reinterpret_cast<int64_t*>(b + L.v);
      I.cost = reinterpret_cast<int64_t*>(b + L.cost);
      I.stats = reinterpret_cast<int64_t*>(b + L.stats);
      I.status = dflags + r.flag;
      insts.push_back(I);
      ids.push_back(t);
    }
    if (insts.empty()) continue;
    std::vector<int> skip(insts.size(), 0), unsup;
    int rc = run_device_batch(ctx, w->slot, insts, skip, algo, w->stream, false, false, &unsup, false);
    if (rc != OT_OK) {
      for (uint64_t t : ids) flags[reqs[t].flag] = rc;
    } else {
      for (int i : unsup) flags[reqs[ids[i]].flag] = OT_ERR_UNSUPPORTED;
    }
  }
  for (uint64_t t : tk) {
    reqs[t].launched = true;
    watch.push_back(t);
  }
  cudaEventRecord(w->done, w->stream);
  w->busy = true;
  ++n_waves;
  max_busy = std::max<int64_t>(max_busy, busy + 1);
}

void ServeState::loop() {
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    cv.wait_for(lk, std::chrono::microseconds(200));
    if (stop) break;
    // admit queued requests, oldest first, while space allows; their copies
    // go out back to back and are waited for once
    std::vector<uint64_t> admitted;
    while (!pending.empty()) {
      const uint64_t t = pending.front();
      auto it = reqs.find(t);
      if (it == reqs.end()) { pending.pop_front(); continue; }
      Req& r = it->second;
      if (!try_admit(t, r)) break;
      pending.pop_front();
      cudaMemcpyAsync(arena.base + r.off, r.host_C.data(), 4 * size_t(r.n) * r.m,
                      cudaMemcpyHostToDevice, copy_stream);
      admitted.push_back(t);
    }
    if (!admitted.empty()) {
      cudaStreamSynchronize(copy_stream);
      for (uint64_t t : admitted) {
        std::vector<int32_t>().swap(reqs[t].host_C);
        ready.push_back(t);
      }
    }
    launch_ready();
    reclaim_cancelled();
    // requests collected by poll alone stay in the completion list until a
    // completion query passes over them: keep the list bounded by the live
    // requests for clients that never call it
    if (watch.size() > 2 * reqs.size() + 1024) {
      size_t keep = 0;
      for (const uint64_t t : watch)
        if (reqs.count(t)) watch[keep++] = t;
      watch.resize(keep);
    }
    // published requests still unfinished while no grid is resident
    if (!plive.empty()) {
      std::vector<uint64_t> keep;
      for (uint64_t t : plive) {
        auto it = reqs.find(t);
        if (it == reqs.end()) continue;
        if (*reinterpret_cast<volatile int32_t*>(&flags[it->second.flag]) == kFlagPending) keep.push_back(t);
      }
      plive.swap(keep);
      if (!plive.empty()) ensure_grid();
    }
  }
}

int serve_init(ot_ctx* ctx, const ot_config& cfg) {
  ServeState* s = new (std::nothrow) ServeState();
  if (!s) return OT_ERR_OOM;
  s->ctx = ctx;
  if (cfg.hbm_budget_bytes > 0) s->budget = size_t(cfg.hbm_budget_bytes);
  if (cfg.max_inflight > 0) s->max_inflight = cfg.max_inflight;
  s->waves.resize(cfg.wave_streams > 0 ? cfg.wave_streams : 4);
  ctx->serve = s;
  return OT_OK;  // device resources are created on first submit
}

void serve_shutdown(ot_ctx* ctx) {
  ServeState* s = ctx->serve;
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  if (s->started) {
    // the persistent grid leaves at its next pull (a request being solved
    // is finished first)
    if (s->pq) __atomic_store_n(&s->pq->stop, 1, __ATOMIC_RELEASE);
    if (s->pstream) { cudaStreamSynchronize(s->pstream); cudaStreamDestroy(s->pstream); }
    if (s->pev) cudaEventDestroy(s->pev);
    if (s->dhead) cudaFree(s->dhead);
    if (s->pring) cudaFreeHost(s->pring);
    if (s->hres) cudaFreeHost(s->hres);
    if (s->pq) cudaFreeHost(s->pq);
    for (Wave& w : s->waves) {
      if (w.busy) cudaEventSynchronize(w.done);
      w.slot.release();
      if (w.done) cudaEventDestroy(w.done);
      if (w.stream) cudaStreamDestroy(w.stream);
    }
    if (s->copy_stream) { cudaStreamSynchronize(s->copy_stream); cudaStreamDestroy(s->copy_stream); }
    if (s->poll_stream) { cudaStreamSynchronize(s->poll_stream); cudaStreamDestroy(s->poll_stream); }
    if (s->copy_ev) cudaEventDestroy(s->copy_ev);
    s->arena.destroy();
    if (s->flags) cudaFreeHost(s->flags);
  }
  delete s;
  ctx->serve = nullptr;
}

extern "C" {

int ot_assign_submit(ot_ctx* ctx, const int32_t* C, int64_t ldc, int32_t n, int32_t m, int32_t algo,
                     uint64_t* ticket) {
  if (!ctx || !ticket) return OT_ERR_ARG;
  if ((algo != OT_KM && algo != OT_BKM && algo != OT_AUTO) || n <= 0 || m < n || !C || ldc < m)
    return ctx_fail(ctx, OT_ERR_ARG, "bad arguments");
  algo = resolve_algo(ctx, algo, m);
  ServeState* s = ctx->serve;
  cudaSetDevice(ctx->device);
  Layout L(n, m);
  std::unique_lock<std::mutex> lk(s->mu);
  if (!s->started) {
    if (int rc = s->start(); rc) return ctx_fail(ctx, rc, "serving start failed");
  }
  ++s->n_submitted;
  if (L.total > s->budget) {
    ++s->n_refused;
    return ctx_fail(ctx, OT_ERR_BUDGET, "request larger than the HBM budget");
  }
  const uint64_t t = s->next_ticket++;
  Req& r = s->reqs[t];
  r.n = n;
  r.m = m;
  r.algo = algo;
  r.bytes = L.total;
  const bool now = s->pending.empty() && s->try_admit(t, r);
  char* dst = now ? s->arena.base + r.off : nullptr;
  lk.unlock();
  // copy outside the lock; the caller may reuse C once submit returns.  A
  // request that could not be admitted keeps a packed host copy.
  std::vector<int32_t> hc;
  cudaError_t e;
  if (!now) hc.resize(size_t(n) * m);
  void* to = now ? static_cast<void*>(dst) : static_cast<void*>(hc.data());
  if (ldc == m)  // contiguous rows: one linear copy
    e = cudaMemcpyAsync(to, C, 4 * size_t(n) * m, cudaMemcpyDefault, s->poll_stream);
  else
    e = cudaMemcpy2DAsync(to, 4 * size_t(m), C, 4 * size_t(ldc), 4 * size_t(m), n, cudaMemcpyDefault,
                          s->poll_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->poll_stream);
  lk.lock();
  Req& rr = s->reqs[t];
  if (e != cudaSuccess) {
    if (rr.admitted) {
      s->arena.release(rr.off, rr.bytes);
      s->free_flags.push_back(rr.flag);
      --s->inflight;
    }
    s->reqs.erase(t);
    return ctx_cuda(ctx, e, "submit copy");
  }
  rr.submitting = false;
  if (now) {
    s->ready.push_back(t);
  } else {
    rr.host_C = std::move(hc);
    s->pending.push_back(t);
  }
  lk.unlock();
  s->cv.notify_one();
  *ticket = t;
  return OT_OK;
}

int ot_assign_poll(ot_ctx* ctx, uint64_t ticket, int32_t* row_to_col, int64_t* cost, int64_t* u,
                   int64_t* v) {
  if (!ctx) return OT_ERR_ARG;
  ServeState* s = ctx->serve;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return ctx_fail(ctx, OT_ERR_TICKET, "unknown ticket");
  Req& r = it->second;
  if (r.cancelled || r.submitting) return ctx_fail(ctx, OT_ERR_TICKET, "unknown ticket");
  if (!r.launched) return OT_PENDING;
  // acquire: the results, written before the status word, are visible
  const int32_t f = __atomic_load_n(&s->flags[r.flag], __ATOMIC_ACQUIRE);
  if (f == kFlagPending) return OT_PENDING;
  const int n = r.n, m = r.m;
  char* b = s->arena.base + r.off;
  const size_t off = r.off, bytes = r.bytes;
  const int flag = r.flag, res = r.res;
  lk.unlock();
  int rc = f;
  if (f == OT_OK && res >= 0) {
    // results in the mapped pool: host copies (a device destination takes
    // one synchronous copy each)
    const char* h = s->hres + size_t(res) * ResLayout::total;
    const void* src[4] = {h + ResLayout::r2c, h + ResLayout::cost, h + ResLayout::u, h + ResLayout::v};
    void* dst[4] = {row_to_col, cost, u, v};
    const size_t len[4] = {4 * size_t(n), 8, 8 * size_t(n), 8 * size_t(m)};
    for (int q = 0; q < 4 && rc == OT_OK; ++q) {
      if (!dst[q]) continue;
      cudaPointerAttributes a;
      const bool dev = cudaPointerGetAttributes(&a, dst[q]) == cudaSuccess && a.type == cudaMemoryTypeDevice;
      cudaGetLastError();
      if (!dev) {
        std::memcpy(dst[q], src[q], len[q]);
      } else {
        cudaSetDevice(ctx->device);
        const cudaError_t e = cudaMemcpy(dst[q], src[q], len[q], cudaMemcpyDefault);
        if (e != cudaSuccess) rc = ctx_cuda(ctx, e, "poll copy");
      }
    }
  } else if (f == OT_OK) {
    cudaSetDevice(ctx->device);
    Layout L(n, m);
    cudaError_t e = cudaSuccess;
    if (row_to_col) e = cudaMemcpyAsync(row_to_col, b + L.r2c, 4 * size_t(n), cudaMemcpyDefault, s->poll_stream);
    if (e == cudaSuccess && cost) e = cudaMemcpyAsync(cost, b + L.cost, 8, cudaMemcpyDefault, s->poll_stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, b + L.u, 8 * size_t(n), cudaMemcpyDefault, s->poll_stream);
    if (e == cudaSuccess && v) e = cudaMemcpyAsync(v, b + L.v, 8 * size_t(m), cudaMemcpyDefault, s->poll_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->poll_stream);
    if (e != cudaSuccess) rc = ctx_cuda(ctx, e, "poll copy");
  }
  lk.lock();
  s->arena.release(off, bytes);
  s->free_flags.push_back(flag);
  if (res >= 0) s->free_res.push_back(res);
  --s->inflight;
  s->reqs.erase(ticket);
  if (rc == OT_OK) ++s->n_completed;
  lk.unlock();
  s->cv.notify_one();
  if (rc != OT_OK && rc != OT_ERR_CUDA) return ctx_fail(ctx, rc, "request failed on the device");
  return rc;
}

int ot_assign_completed(ot_ctx* ctx, uint64_t* tickets, int32_t max, int32_t* count) {
  if (!ctx || !count || max < 0 || (max > 0 && !tickets)) return OT_ERR_ARG;
  ServeState* s = ctx->serve;
  std::lock_guard<std::mutex> g(s->mu);
  int c = 0;
  size_t keep = 0;
  for (size_t q = 0; q < s->watch.size(); ++q) {
    const uint64_t t = s->watch[q];
    auto it = s->reqs.find(t);
    if (it == s->reqs.end() || it->second.cancelled) continue;  // collected or cancelled: dropped
    // acquire: the results, written before the status word, are visible
    if (c < max && __atomic_load_n(&s->flags[it->second.flag], __ATOMIC_ACQUIRE) != kFlagPending) {
      tickets[c++] = t;
      continue;
    }
    s->watch[keep++] = t;
  }
  s->watch.resize(keep);
  *count = c;
  return OT_OK;
}

int ot_assign_cancel(ot_ctx* ctx, uint64_t ticket) {
  if (!ctx) return OT_ERR_ARG;
  ServeState* s = ctx->serve;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end() || it->second.cancelled || it->second.submitting)
    return ctx_fail(ctx, OT_ERR_TICKET, "unknown ticket");
  Req& r = it->second;
  if (!r.admitted) {
    // waiting for admission in the host queue (the queue skips it)
    s->reqs.erase(it);
    return OT_OK;
  }
  if (!r.launched) {
    // admitted, its copy landed, not yet in a wave
    s->ready.erase(std::remove(s->ready.begin(), s->ready.end(), ticket), s->ready.end());
    s->release(ticket, r);
    lk.unlock();
    s->cv.notify_one();
    return OT_OK;
  }
  // in a wave: its solver may still write into the block, which is returned
  // once the status word shows the solve has ended; the result is discarded
  r.cancelled = true;
  ++s->n_cancel_wait;
  s->reclaim_cancelled();
  lk.unlock();
  s->cv.notify_one();
  return OT_OK;
}

int ot_assign_drain(ot_ctx* ctx) {
  if (!ctx) return OT_ERR_ARG;
  ServeState* s = ctx->serve;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    {
      std::lock_guard<std::mutex> g(s->mu);
      bool all = true;
      for (auto& kv : s->reqs) {
        const Req& r = kv.second;
        if (!r.launched || *reinterpret_cast<volatile int32_t*>(&s->flags[r.flag]) == kFlagPending) {
          all = false;
          break;
        }
      }
      if (all) return OT_OK;
    }
    s->cv.notify_one();
    if (std::chrono::steady_clock::now() - t0 > std::chrono::minutes(10))
      return ctx_fail(ctx, OT_ERR_TIMEOUT, "drain timed out");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int ot_serving_counters(ot_ctx* ctx, int64_t* out8) {
  if (!ctx || !out8) return OT_ERR_ARG;
  ServeState* s = ctx->serve;
  std::lock_guard<std::mutex> g(s->mu);
  out8[0] = s->n_submitted;
  out8[1] = s->n_admitted;
  out8[2] = s->n_completed;
  out8[3] = s->n_waves;
  out8[4] = s->max_busy;
  out8[5] = int64_t(s->arena.used);
  out8[6] = int64_t(s->budget);
  out8[7] = s->n_refused;
  return OT_OK;
}

}  // extern "C"
