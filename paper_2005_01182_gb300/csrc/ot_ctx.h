// Host-side context of libotassign.so (not part of the C ABI).
#pragma once
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "otassign.h"
#include "ot_internal.h"

namespace ot {
constexpr int kNumBuckets = 8;        // bucket b: m <= 32 << b
constexpr int kMaxGroupCols = 4096;   // widest instance one group engine handles
constexpr int kForkStreams = 4;
// Host-pointer batches: matrices are copied in up to kHostChunks contiguous
// chunks, each solved as soon as its copy has landed.
constexpr int kHostChunks = 4;
constexpr int kLargeEngine = -2;  // table entry: use the cluster engine
// A batched-KM instance wider than kClusterRouteCols solved on its own
// (ot_assign_solve / _stats) goes to the cluster engine instead of one group
// unless the table entry was set explicitly.
constexpr int kClusterRouteCols = 1024;
constexpr int kClusterRouteMax = 4;
int bucket_of(int m);
int shape_index(int tpi, int k);
void default_table(int table[2][kNumBuckets]);
void default_auto(int auto_algo[kNumBuckets]);
}  // namespace ot

struct DevBuf {
  void* ptr = nullptr;
  size_t cap = 0;
  int generation = 0;
  int reserve(size_t bytes);
  void release();
};

struct PinBuf {
  void* ptr = nullptr;
  size_t cap = 0;
  int reserve(size_t bytes);
  void release();
};

struct ServeState;  // ot_serve.cu

// Descriptor upload buffers of one launcher (the API path, or one serving
// wave): pinned mirror, device copy, the event that marks the end of the
// slot's latest launch, the per-instance stats block, and cached CUDA graphs
// keyed by batch layout.  The descriptors are uploaded only when they differ
// from the ones already on the device (last_meta), so that a caller who
// re-issues the same batch never waits on the host for the previous launch.
struct LaunchSlot {
  DevBuf d_meta, d_stats, d_pack;  // d_pack: 16-bit packed rows of group-engine instances
  PinBuf h_meta;
  cudaEvent_t meta_ev = nullptr;
  bool meta_pending = false;
  std::vector<char> last_meta, pending;  // descriptor bytes on the device / being built
  bool meta_valid = false;               // last_meta matches d_meta
  bool pack = true;                      // 16-bit row packing for group-engine buckets
  // per-bucket kernel timing of the latest launch (API slot only): events
  // recorded around each bucket's kernel (event-record nodes inside graphs)
  bool timing = false;
  std::vector<cudaEvent_t> tev;  // 2 per bucket
  struct BucketInfo {
    int algo, tpi, k;
    std::vector<int> idx;
  };
  std::vector<BucketInfo> last_buckets;
  bool use_graphs = false;
  std::map<std::string, cudaGraphExec_t> graphs;
  int last_launches = 0;
  int init();
  void clear_graphs();
  void release();
};

struct ot_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t bstreams[ot::kForkStreams] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[ot::kForkStreams] = {};
  // ordering with the caller's default stream (StreamScope): one pair for
  // the calls serialised by api_mu, one for those serialised by scaled_mu
  cudaEvent_t join_in_ev = nullptr, join_out_ev = nullptr;
  cudaEvent_t sjoin_in_ev = nullptr, sjoin_out_ev = nullptr;
  std::string err;
  std::mutex api_mu;

  LaunchSlot api;
  // pipelined host-pointer batches: a copy stream, one stream, launch slot
  // and event set per chunk
  cudaStream_t copy_stream = nullptr;
  cudaStream_t cstreams[ot::kHostChunks] = {};
  LaunchSlot hslots[ot::kHostChunks];
  cudaEvent_t hev_start = nullptr, hev_copy[ot::kHostChunks] = {}, hev_done[ot::kHostChunks] = {};
  DevBuf d_status, d_io, d_scratch, d_large, d_scaled;
  std::mutex scaled_mu;

  int table[2][ot::kNumBuckets];
  bool tuned[2][ot::kNumBuckets] = {};  // entry set by ot_tune_set / ot_autotune / tune file
  int auto_algo[ot::kNumBuckets];  // algorithm OT_AUTO resolves to, per bucket
  std::string tune_file;
  bool pack_rows = true;        // 16-bit row packing of group-engine instances
  int max_group_ctas = 0;       // cap on a batched launch's persistent grid (0: none)
  long long step_limit = 0;     // per-instance step cap (failure-detection tests)
  bool dense_wide = false;      // wide batched-KM instances on the dense cluster engine

  int last_k = 0;               // instances of the most recent API call
  std::vector<int> last_skip;   // which of them were not launched

  ServeState* serve = nullptr;
};

// The stream an API call works on.  A NULL handle (or the legacy or
// per-thread default-stream handle) names the caller's default stream, on
// which graphs cannot be captured: the call then works on the context's own
// stream, which first waits for the work already queued on the default
// stream; on leaving the scope the default stream waits for the call's work.
// The events belong to the lock domain the caller holds.
struct StreamScope {
  cudaStream_t user = nullptr;  // as given
  cudaStream_t work = nullptr;  // where the call enqueues
  cudaEvent_t out_ev = nullptr;
  StreamScope(cudaStream_t given, cudaStream_t own, cudaEvent_t in_ev, cudaEvent_t out);
  ~StreamScope();
  StreamScope(const StreamScope&) = delete;
  StreamScope& operator=(const StreamScope&) = delete;
};

int ctx_fail(ot_ctx* ctx, int code, const std::string& msg);
int ctx_cuda(ot_ctx* ctx, cudaError_t e, const char* where);
bool ptr_on_device(const void* p);
// ptr_on_device for many pointers: the address range of every allocation
// met is remembered, so pointers into one allocation cost one driver query.
class PtrKinds {
 public:
  bool on_device(const void* p);

 private:
  struct Range {
    uintptr_t lo, hi;
    bool dev;
  };
  std::vector<Range> ranges_;  // sorted by lo, disjoint
  size_t last_ = 0;
};
void load_tune_file(ot_ctx* ctx);
// Bucket the instances by tuned group shape and launch them on `stream`
// (forking buckets over the context's streams when `fork`).  Entries with
// skip[t] set are not launched; instances the group engine does not take
// (too wide, routed to the cluster engine, or -- with `allow_cluster` -- a
// few wide batched-KM ones) are listed in *unsupported for the caller to
// hand to the cluster engine.  With `own_stats` the slot's stats block
// receives per-instance counters, otherwise insts[t].stats is kept.
int run_device_batch(ot_ctx* ctx, LaunchSlot& slot, std::vector<ot::Instance>& insts,
                     const std::vector<int>& skip, int algo, cudaStream_t stream, bool fork,
                     bool own_stats, std::vector<int>* unsupported, bool allow_cluster);
// Wide-instance engine (ot_large.cu): one instance on a thread-block
// cluster plus grid-wide passes; synchronises `stream`.
int solve_large(ot_ctx* ctx, const ot::Instance& I, int algo, cudaStream_t stream, int64_t* stats_out);
int large_max_cols();
// Sparse-list engine (ot_sparse.cu): one batched-KM instance with
// n <= m <= sparse_max_cols(); synchronises `stream`.
int solve_sparse(ot_ctx* ctx, const ot::Instance& I, cudaStream_t stream, int64_t* stats_out);
int sparse_max_cols();
// An instance the group engine does not take: batched KM on the sparse-list
// engine when it fits (unless the context asks for the dense cluster
// engine), everything else on the cluster engine.
int solve_wide(ot_ctx* ctx, const ot::Instance& I, int algo, cudaStream_t stream, int64_t* stats_out);
// OT_KM / OT_BKM unchanged; OT_AUTO -> the tuned algorithm of m's bucket.
int resolve_algo(const ot_ctx* ctx, int algo, int m);
int serve_init(ot_ctx* ctx, const ot_config& cfg);
void serve_shutdown(ot_ctx* ctx);
