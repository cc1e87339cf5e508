// ot_assign_solve_batched_noalloc: the multi-instance group engine launched
// without any device allocation.
//
// The batched entry point normally stages its launch metadata (one
// descriptor per instance, the per-bucket launch order and the work
// counters the persistent groups pull instances from) in buffers that the
// context allocates with cudaMalloc.  Here that scratch lives in one
// file-scope __device__ array of fixed size, so a caller that must not
// allocate device memory can still run batched solves.  The array is part
// of the loaded module: every GPU that loads the library holds it until the
// process exits.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "otassign.h"
#include "ot_ctx.h"
#include "ot_group.cuh"
#include "ot_shapes.h"

using namespace ot;

namespace {

constexpr int kNoAllocMaxInstances = OT_NOALLOC_MAX_INSTANCES;
constexpr int kNoAllocMaxBuckets = 32;

struct NoAllocScratch {
  Instance desc[kNoAllocMaxInstances];
  int32_t order[kNoAllocMaxInstances];
  int32_t status[kNoAllocMaxInstances];
  int32_t work[kNoAllocMaxBuckets];
};

// The shared scratch (about 82 KB: 72-byte descriptors, two int32 arrays).  Every call overwrites it; calls whose
// work overlaps on the GPU race on it.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoAllocScratch* g_scratch_addr[kMaxDevices] = {};

// Host-side bookkeeping of one call (about 80 KB), kept off the caller's
// stack: callers of this entry point often run on small worker-thread
// stacks.  g_mu serialises the calls that use it.
struct HostBook {
  Instance desc[kNoAllocMaxInstances];
  int32_t order[kNoAllocMaxInstances];
  int32_t bucket[kNoAllocMaxInstances];
};
HostBook g_book;

// Once per device, with that device current: the device address of the
// scratch array (its host-side name is only a stand-in, not an address a
// kernel may use).  Caller holds g_mu.
int scratch_address(int dev, NoAllocScratch** out) {
  if (dev < 0 || dev >= kMaxDevices) return OT_ERR_UNSUPPORTED;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return OT_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_scratch_addr[dev];
  return OT_OK;
}

// True when p is device (or managed) memory that device `dev` owns: a
// kernel on `dev` may then read and write through it.
bool on_device(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int ot_assign_solve_batched_noalloc(int32_t k, const int32_t* const* C, const int64_t* ldc,
                                               const int32_t* n, const int32_t* m, int32_t algo,
                                               int32_t* const* row_to_col, int64_t* cost,
                                               int64_t* const* u, int64_t* const* v, int32_t* status,
                                               void* stream) {
  if (algo != OT_KM && algo != OT_BKM && algo != OT_AUTO) return OT_ERR_ARG;
  if (k < 0 || (k > 0 && (!C || !ldc || !n || !m || !row_to_col || !cost))) return OT_ERR_ARG;
  if (k > kNoAllocMaxInstances) return OT_ERR_UNSUPPORTED;  // beyond the static scratch
  if (k == 0) return OT_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return OT_ERR_CUDA;
  }
  if (!on_device(cost, dev) || (status && !on_device(status, dev))) return OT_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The launch metadata is copied from host bookkeeping that the next call
  // overwrites, so a stream that is being captured is refused.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return OT_ERR_CUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) return OT_ERR_UNSUPPORTED;

  std::lock_guard<std::mutex> guard(g_mu);
  NoAllocScratch* S = nullptr;
  if (int rc = scratch_address(dev, &S); rc) return rc;
  Instance* hdesc = g_book.desc;
  int32_t* horder = g_book.order;
  int32_t* hbucket = g_book.bucket;
  int table[2][kNumBuckets], auto_algo[kNumBuckets];
  default_table(table);
  default_auto(auto_algo);
  // launch buckets: (algorithm, shape); empty instances (n == 0) take none
  constexpr int NB = 2 * OT_NUM_GROUP_SHAPES;
  int count[NB] = {0}, nmax[NB] = {0}, mmax[NB] = {0};
  int live = 0;
  for (int t = 0; t < k; ++t) {
    if (n[t] < 0 || m[t] < n[t]) return OT_ERR_ARG;
    hbucket[t] = -1;
    if (n[t] == 0) {
      if (v && v[t] && m[t] > 0 && !on_device(v[t], dev)) return OT_ERR_ARG;
      continue;
    }
    if (ldc[t] < m[t] || !C[t] || !row_to_col[t]) return OT_ERR_ARG;
    if (m[t] > kMaxGroupCols) return OT_ERR_UNSUPPORTED;
    // host data would need staging memory; outputs are written by the kernel
    if (!on_device(C[t], dev) || !on_device(row_to_col[t], dev)) return OT_ERR_ARG;
    if ((u && u[t] && !on_device(u[t], dev)) || (v && v[t] && !on_device(v[t], dev))) return OT_ERR_ARG;
    const int ia = algo == OT_AUTO ? auto_algo[bucket_of(m[t])] : algo;
    const int sh = table[ia][bucket_of(m[t])];
    if (group_smem_bytes(group_shape(sh), ia, n[t], m[t]) > group_smem_limit()) return OT_ERR_UNSUPPORTED;
    hbucket[t] = ia * OT_NUM_GROUP_SHAPES + sh;
    ++count[hbucket[t]];
    ++live;
    nmax[hbucket[t]] = std::max(nmax[hbucket[t]], n[t]);
    mmax[hbucket[t]] = std::max(mmax[hbucket[t]], m[t]);
    Instance& I = hdesc[t];
    I.C = C[t]; I.ldc = ldc[t]; I.n = n[t]; I.m = m[t];
    I.row_to_col = row_to_col[t];
    I.u = u ? u[t] : nullptr;
    I.v = v ? v[t] : nullptr;
    I.cost = cost + t;
    I.status = status ? status + t : S->status + t;
    I.stats = nullptr;
    I.P = nullptr;
    I.roff = nullptr;
    I.pok = nullptr;
    I.step_limit = 0;
  }
  // empty instances: cost 0 and status OK, v (when given) zero, as
  // ot_assign_solve_batched returns them
  cudaError_t e = cudaSuccess;
  for (int t = 0; t < k && e == cudaSuccess; ++t) {
    if (n[t] != 0) continue;
    e = cudaMemsetAsync(cost + t, 0, sizeof(int64_t), s);
    if (e == cudaSuccess && status) e = cudaMemsetAsync(status + t, 0, sizeof(int32_t), s);
    if (e == cudaSuccess && v && v[t] && m[t] > 0) e = cudaMemsetAsync(v[t], 0, sizeof(int64_t) * m[t], s);
  }
  if (e != cudaSuccess) return OT_ERR_CUDA;
  if (live == 0) return OT_OK;
  // launch order: bucket by bucket, largest instances first
  int off[NB + 1] = {0};
  for (int b = 0; b < NB; ++b) off[b + 1] = off[b] + count[b];
  int fill[NB];
  std::memcpy(fill, off, sizeof(fill));
  for (int t = 0; t < k; ++t)
    if (hbucket[t] >= 0) horder[fill[hbucket[t]]++] = t;
  for (int b = 0; b < NB; ++b)
    std::sort(horder + off[b], horder + off[b + 1], [&](int a, int c) {
      const long long wa = (long long)n[a] * m[a], wc = (long long)n[c] * m[c];
      return wa != wc ? wa > wc : a < c;
    });

  // Upload into the static scratch (pageable source: the runtime has staged
  // the copy before cudaMemcpyAsync returns, so the bookkeeping may be
  // reused afterwards) and clear the work counters.
  e = cudaMemcpyAsync(S->desc, hdesc, sizeof(Instance) * k, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->order, horder, sizeof(int32_t) * live, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(S->work, 0, sizeof(S->work), s);
  if (e != cudaSuccess) return OT_ERR_CUDA;
  for (int b = 0; b < NB; ++b) {
    if (!count[b]) continue;
    e = launch_group(group_shape(b % OT_NUM_GROUP_SHAPES), b / OT_NUM_GROUP_SHAPES, S->desc, S->order + off[b],
                     count[b], S->work + b, nmax[b], mmax[b], 0, s);
    if (e != cudaSuccess) return OT_ERR_CUDA;
  }
  return OT_OK;
}
