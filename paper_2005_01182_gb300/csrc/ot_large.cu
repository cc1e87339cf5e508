// Large-instance engine: one instance wider than a CTA can hold (m > 4096),
// solved by a thread-block cluster for the dependent steps plus grid-wide
// streaming passes for batched KM's forest rebuilds.
//
// Column state lives in registers of the cluster's threads (thread g of the
// cluster owns columns j = g + k * G, G = cluster threads).  One step =
// scan the rows that just joined the tree, take the cluster-wide minimum
// distance outside T (lowest column on ties) through distributed shared
// memory and one cluster barrier, then let the columns at that level join T
// (or end augmenting paths).  Row-indexed state (u, row_to_col, roots,
// levels) and the predecessor log stay in global memory (L2-resident at
// these sizes).
//
// Batched KM (paper Sec. 2.3 "Batched KM") runs phase by phase: a phase
// grows the forest of all free rows until free columns become tight, then
// augments one path per tree (lowest free column wins), applies the
// accumulated dual adjustment, and dissolves only the trees that were
// augmented.  The surviving trees keep their rows and columns; the next
// phase recomputes the distances of the columns outside T from all surviving
// rows in one grid-wide pass (large_pass), which is the HBM-bound part.
// Kuhn-Munkres runs every phase (one root row each) inside one cluster
// launch, with the same tie-breaks as the group engine.
#include <climits>
#include <cooperative_groups.h>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>

#include "ot_ctx.h"
#include "ot_group.cuh"

namespace cg = cooperative_groups;

// Cycle accounting of the step kernel, compiled in only with
// -DOT_LARGE_PROFILE (thread 0 of rank 0 measures; sections: phase setup,
// scan, CTA reduction + publication, cluster barrier, post-exchange work,
// augmentation).
#ifdef OT_LARGE_PROFILE
#define OT_PROF_DECL unsigned long long prof_acc[6] = {0, 0, 0, 0, 0, 0}; long long prof_t = clock64();
#define OT_PROF_MARK(idx)                         \
  do {                                            \
    const long long now_ = clock64();             \
    prof_acc[idx] += (unsigned long long)(now_ - prof_t); \
    prof_t = now_;                                \
  } while (0)
#define OT_PROF_FLUSH(ctl)                                               \
  do {                                                                   \
    if (g == 0) {                                                        \
      for (int q_ = 0; q_ < 6; ++q_) atomicAdd(&(ctl)->prof[q_], prof_acc[q_]); \
      atomicAdd(&(ctl)->prof[6], rows);                                  \
    }                                                                    \
  } while (0)
#else
#define OT_PROF_DECL
#define OT_PROF_MARK(idx) do {} while (0)
#define OT_PROF_FLUSH(ctl) do {} while (0)
#endif

namespace ot {

constexpr int kLargeTPB = 1024;
constexpr int kSlotMates = 32;
constexpr int kPassThreads = 256;
constexpr int kPassCols = 4 * kPassThreads;
constexpr int kMaxCluster = 16;

// ---- TMA bulk copies and mbarriers (inline PTX) ----------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> own shared memory, completing `bytes` on `bar`; 16-byte aligned
// addresses, size a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on one mbarrier phase: false if it did not complete within
// `max_polls` polls (each poll may suspend the thread for a short while).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, int max_polls) {
  for (int it = 0; it < max_polls; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
constexpr int kRingBytes = 64 * 1024;   // staged row segments per CTA

// Device-side range check: records the first violation (site, value, aux)
// and returns false so that the caller skips the access.
__device__ __forceinline__ bool in_range(int x, int hi, int* bad, int site, int aux) {
  if (x >= 0 && x < hi) return true;
  if (atomicCAS(&bad[0], 0, site) == 0) {
    bad[1] = x;
    bad[2] = aux;
  }
  return false;
}
constexpr int kMbarPolls = 1 << 22;

struct LargeCtl {
  int matched;
  int done;
  int status;
  int scount;
  int walkers;
  int bad[3];   // first out-of-range index seen by a device-side check: site, value, aux
  unsigned long long stats[8];  // steps, rows, bytes, phases, augs, init_bytes
  unsigned long long prof[8];   // cycle breakdown of the step kernel (profiling builds)
};

// A row that joins S: its index, dual and tree root, carried with the
// column exchange so that the next scan needs no dependent global load.
struct __align__(16) RowRef {
  long long u;
  int row;
  int root;
};

struct LargeWs {
  const int32_t* C;
  long long ldc;
  int n, m;
  int32_t* r2c;
  long long* u;
  long long* v;
  int* pred;             // [m] predecessor row of columns in T / path ends
  unsigned char* inT;    // [m]
  int* c2r;              // [m]
  long long* drow;       // [n] level at which a row joined S
  int* root;             // [n]
  int* slist;            // [n] rows of S (batched KM pass input)
  unsigned char* inS;    // [n]
  int* claim;            // [n] lowest free column claimed per root
  long long* part_d;     // [chunks][m]
  int* part_p;           // [chunks][m]
  RowRef* ovf;           // [2][cluster][cols per CTA] rows beyond the slot capacity
  LargeCtl* ctl;
  int chunks;
  int vec4;
  int tma;   // level rows staged with bulk copies (16-byte aligned rows, m % 4 == 0)
};

struct __align__(16) Slot {
  long long d;     // CTA minimum distance outside T
  int j;           // lowest column attaining it
  int mate;        // KM: its matched row
  int cnt;         // batched KM: matched columns at d (rows listed below)
  int nfree;       // batched KM: free columns at d
  int err;         // a bounded wait of this CTA expired
  int pad;
  long long umate; // KM: u of `mate`
  RowRef refs[kSlotMates];
};

// ---------------------------------------------------------------------------
// init: state, and for batched KM the row reduction u_i = min_j C[i][j] (B1)
// ---------------------------------------------------------------------------
__global__ void large_init(LargeWs w, int bkm) {
  const int n = w.n, m = w.m;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long j = tid; j < m; j += nth) {
    w.v[j] = 0;
    w.c2r[j] = -1;
    w.inT[j] = 0;
    w.pred[j] = -1;
  }
  for (long long i = tid; i < n; i += nth) {
    w.r2c[i] = -1;
    w.inS[i] = bkm ? 1 : 0;
    w.drow[i] = 0;
    w.root[i] = int(i);
    w.claim[i] = INT_MAX;
    w.slist[i] = int(i);
    if (!bkm) w.u[i] = 0;
  }
  if (bkm) {
    const int lane = threadIdx.x & 31;
    const long long warp = tid >> 5, nwarps = nth >> 5;
    for (long long i = warp; i < n; i += nwarps) {
      const int32_t* row = w.C + i * w.ldc;
      long long mn = kInf;
      if (w.vec4) {
        const int4* r4 = reinterpret_cast<const int4*>(row);
        for (int q = lane; q < m / 4; q += 32) {
          const int4 c = __ldcs(r4 + q);
          mn = min(mn, (long long)min(min(c.x, c.y), min(c.z, c.w)));
        }
        for (int j = (m / 4) * 4 + lane; j < m; j += 32) mn = min(mn, (long long)__ldcs(row + j));
      } else {
        for (int j = lane; j < m; j += 32) mn = min(mn, (long long)__ldcs(row + j));
      }
      mn = warp_min(mn);
      if (lane == 0) w.u[i] = mn;
    }
  }
  if (tid == 0) {
    w.ctl->matched = 0;
    w.ctl->done = n == 0;
    w.ctl->status = 0;
    w.ctl->scount = bkm ? n : 0;
    w.ctl->walkers = 0;
    w.ctl->bad[0] = w.ctl->bad[1] = w.ctl->bad[2] = 0;
    for (int q = 0; q < 8; ++q) w.ctl->stats[q] = 0;
    for (int q = 0; q < 8; ++q) w.ctl->prof[q] = 0;
    w.ctl->stats[5] = bkm ? 4ull * n * m : 0;
  }
}

// ---------------------------------------------------------------------------
// B2 pass: for every column outside T, the minimum reduced cost over the rows
// of S (lowest row on ties), as per-chunk partials.  Grid: (column tiles of
// kPassCols, row chunks); each thread owns 4 consecutive columns.
// ---------------------------------------------------------------------------
template <int VEC>
__global__ void __launch_bounds__(kPassThreads) large_pass(LargeWs w) {
  if (w.ctl->done) return;
  const int m = w.m;
  const int S = w.ctl->scount;
  const int c = blockIdx.y;
  const int r0 = int((long long)S * c / w.chunks), r1 = int((long long)S * (c + 1) / w.chunks);
  const int j0 = blockIdx.x * kPassCols + 4 * threadIdx.x;
  long long vj[4], bd[4];
  int bp[4];
  bool live[4];
  int nlive = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = j0 + q;
    live[q] = j < m && !w.inT[j];
    vj[q] = j < m ? w.v[j] : 0;
    bd[q] = kInf;
    bp[q] = INT_MAX;
    nlive += live[q];
  }
  const int32_t* C = w.C;
  const long long ldc = w.ldc;
  int r = r0;
  // four rows in flight per iteration
  for (; r + 4 <= r1; r += 4) {
    int ii[4];
    long long uu[4];
    int4 cc[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      ii[e] = w.slist[r + e];
      uu[e] = w.u[ii[e]];
      const int32_t* row = C + ii[e] * ldc;
      if (VEC && j0 + 3 < m) {
        cc[e] = __ldcs(reinterpret_cast<const int4*>(row + j0));
      } else {
        cc[e].x = j0 < m ? __ldcs(row + j0) : 0;
        cc[e].y = j0 + 1 < m ? __ldcs(row + j0 + 1) : 0;
        cc[e].z = j0 + 2 < m ? __ldcs(row + j0 + 2) : 0;
        cc[e].w = j0 + 3 < m ? __ldcs(row + j0 + 3) : 0;
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int cv[4] = {cc[e].x, cc[e].y, cc[e].z, cc[e].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long rc = (long long)cv[q] - uu[e] - vj[q];
        if (live[q] && (rc < bd[q] || (rc == bd[q] && ii[e] < bp[q]))) { bd[q] = rc; bp[q] = ii[e]; }
      }
    }
  }
  for (; r < r1; ++r) {
    const int i = w.slist[r];
    const long long ui = w.u[i];
    const int32_t* row = C + i * ldc;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!live[q]) continue;
      const long long rc = (long long)__ldcs(row + j0 + q) - ui - vj[q];
      if (rc < bd[q] || (rc == bd[q] && i < bp[q])) { bd[q] = rc; bp[q] = i; }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = j0 + q;
    if (j < m) {
      w.part_d[(long long)c * m + j] = bd[q];
      w.part_p[(long long)c * m + j] = bp[q];
    }
  }
  // algorithmic bytes: 4 per (row of S, column outside T)
  const long long wl = warp_sum((long long)nlive);
  if ((threadIdx.x & 31) == 0 && wl > 0)
    atomicAdd(&w.ctl->stats[2], (unsigned long long)(4 * wl * (r1 - r0)));
  if (blockIdx.x == 0 && threadIdx.x == 0 && r1 > r0) atomicAdd(&w.ctl->stats[1], (unsigned long long)(r1 - r0));
}


// ---------------------------------------------------------------------------
// B2 pass, bulk-copy pipeline: the same result as large_pass, with the rows'
// segments of this CTA's column tile (kTmaTileCols columns) streamed into a
// shared-memory ring by cp.async.bulk, kTmaStages stages of kTmaRows rows in
// flight, each stage completing on its own mbarrier.  Thread 0 produces,
// every thread consumes 8 columns.  Needs 16-byte aligned rows, m % 4 == 0.
// ---------------------------------------------------------------------------
constexpr int kTmaTileCols = 8 * kPassThreads;                 // 2048 columns
constexpr int kTmaRows = 4;                                   // rows per stage
constexpr int kTmaStages = 3;
constexpr int kTmaStageBytes = kTmaRows * kTmaTileCols * 4;   // 32 KB
constexpr int kTmaPassSmem = kTmaStages * kTmaStageBytes;     // 96 KB

__global__ void __launch_bounds__(kPassThreads) large_pass_tma(LargeWs w) {
  if (w.ctl->done) return;
  extern __shared__ __align__(128) int32_t ring[];
  __shared__ __align__(8) unsigned long long bars[kTmaStages];
  __shared__ int s_row[kTmaStages][kTmaRows];
  __shared__ long long s_u[kTmaStages][kTmaRows];
  const int m = w.m;
  const int S = w.ctl->scount;
  const int c = blockIdx.y;
  const int r0 = int((long long)S * c / w.chunks), r1 = int((long long)S * (c + 1) / w.chunks);
  const int tile0 = blockIdx.x * kTmaTileCols;
  const int tcols = min(kTmaTileCols, m - tile0);           // multiple of 4
  const unsigned seg_bytes = unsigned(tcols) * 4u;
  const int t = threadIdx.x;
  const int j0 = tile0 + 8 * t;
  if (t == 0) {
    for (int st = 0; st < kTmaStages; ++st) mbar_init(&bars[st], 1);
    mbar_fence_init();
  }
  long long vj[8], bd[8];
  int bp[8];
  bool live[8];
  int nlive = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int j = j0 + q;
    live[q] = j < m && !w.inT[j];
    vj[q] = j < m ? w.v[j] : 0;
    bd[q] = kInf;
    bp[q] = INT_MAX;
    nlive += live[q];
  }
  __syncthreads();
  const int nrows = r1 - r0;
  const int nstages_total = (nrows + kTmaRows - 1) / kTmaRows;
  // producer: fill stage st with rows [r0 + s*kTmaRows, ...)
  auto produce = [&](int sidx) {
    const int st = sidx % kTmaStages;
    const int rb = r0 + sidx * kTmaRows;
    const int nr = min(kTmaRows, r1 - rb);
    for (int e = 0; e < nr; ++e) {
      const int i = w.slist[rb + e];
      s_row[st][e] = i;
      s_u[st][e] = w.u[i];
    }
    mbar_arrive_expect_tx(&bars[st], seg_bytes * unsigned(nr));
    for (int e = 0; e < nr; ++e)
      bulk_g2s(ring + (st * kTmaRows + e) * kTmaTileCols, w.C + (long long)s_row[st][e] * w.ldc + tile0, seg_bytes,
               &bars[st]);
  };
  if (t == 0)
    for (int sidx = 0; sidx < min(kTmaStages, nstages_total); ++sidx) produce(sidx);
  bool failed = false;
  for (int sidx = 0; sidx < nstages_total; ++sidx) {
    const int st = sidx % kTmaStages;
    const unsigned parity = unsigned(sidx / kTmaStages) & 1u;
    if (!mbar_wait_bounded(&bars[st], parity, kMbarPolls)) { failed = true; break; }
    const int nr = min(kTmaRows, r1 - (r0 + sidx * kTmaRows));
    for (int e = 0; e < nr; ++e) {
      const int i = s_row[st][e];
      const long long ui = s_u[st][e];
      const int4* src = reinterpret_cast<const int4*>(ring + (st * kTmaRows + e) * kTmaTileCols + 8 * t);
      const int4 a = src[0], b = src[1];
      const int cv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const long long rc = (long long)cv[q] - ui - vj[q];
        if (live[q] && (rc < bd[q] || (rc == bd[q] && i < bp[q]))) { bd[q] = rc; bp[q] = i; }
      }
    }
    __syncthreads();  // stage st is free again
    if (t == 0 && sidx + kTmaStages < nstages_total) produce(sidx + kTmaStages);
  }
  if (failed) {
    // give copies still in flight a bounded chance to land before exiting
    if (t == 0) {
      w.ctl->status = kDevStepLimit;
      for (int st = 0; st < kTmaStages; ++st) mbar_wait_bounded(&bars[st], 0, 1024);
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int j = j0 + q;
    if (j < m) {
      w.part_d[(long long)c * m + j] = bd[q];
      w.part_p[(long long)c * m + j] = bp[q];
    }
  }
  const long long wl = warp_sum((long long)nlive);
  if ((threadIdx.x & 31) == 0 && wl > 0)
    atomicAdd(&w.ctl->stats[2], (unsigned long long)(4 * wl * (r1 - r0)));
  if (blockIdx.x == 0 && threadIdx.x == 0 && r1 > r0) atomicAdd(&w.ctl->stats[1], (unsigned long long)(r1 - r0));
}

// ---------------------------------------------------------------------------
// cluster step engine
// ---------------------------------------------------------------------------
template <int K, int ALGO>
__global__ void __launch_bounds__(kLargeTPB, 1) large_steps(LargeWs w) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = int(cluster.num_blocks());
  const int rank = int(cluster.block_rank());
  const int t = threadIdx.x;
  const int G = CS * kLargeTPB;
  const int g = rank * kLargeTPB + t;
  const int n = w.n, m = w.m;
  const int lane = t & 31, wid = t >> 5;
  constexpr int NW = kLargeTPB / 32;

  __shared__ Slot slots[2][kMaxCluster];
  __shared__ Best wbest[NW];
  __shared__ int s_cnt, s_nfree, s_mate;
  __shared__ long long s_umate;
  constexpr int LCAP = 256;  // rows staged per scan chunk
  __shared__ RowRef s_refs[LCAP];
  __shared__ __align__(8) unsigned long long s_bar;
  __shared__ int s_err;
  extern __shared__ __align__(128) int32_t s_ring[];  // kRingBytes: row segments
  unsigned bar_parity = 0;
  if (t == 0) {
    mbar_init(&s_bar, 1);
    mbar_fence_init();
    s_err = 0;
  }
  __syncthreads();
  __shared__ long long s_cnt_total;

  LargeCtl* ctl = w.ctl;
  if (ctl->done) return;  // uniform over the cluster
  OT_PROF_DECL

  long long dist[K], v[K];
  int pred[K], mate[K];
  int rootp[K];          // batched KM: tree root of pred[k]
  long long umate[K];    // u of mate[k]
  unsigned inT = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int j = g + k * G;
    v[k] = 0; dist[k] = kInf; pred[k] = -1; mate[k] = -1; rootp[k] = -1; umate[k] = 0;
    if (j < m) {
      v[k] = w.v[j];
      mate[k] = w.c2r[j];
      umate[k] = mate[k] >= 0 ? w.u[mate[k]] : 0;
      if (ALGO == kAlgoBKM) {
        if (w.inT[j]) {
          inT |= 1u << k;
          pred[k] = w.pred[j];
          rootp[k] = pred[k] >= 0 ? w.root[pred[k]] : -1;
          dist[k] = 0;
        } else {
          long long bd = kInf;
          int bp = INT_MAX;
          int c = 0;
          for (; c + 8 <= w.chunks; c += 8) {
            long long dd[8];
            int pp[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              dd[e] = w.part_d[(long long)(c + e) * m + j];
              pp[e] = w.part_p[(long long)(c + e) * m + j];
            }
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (dd[e] < bd || (dd[e] == bd && pp[e] < bp)) { bd = dd[e]; bp = pp[e]; }
          }
          for (; c < w.chunks; ++c) {
            const long long d = w.part_d[(long long)c * m + j];
            const int p = w.part_p[(long long)c * m + j];
            if (d < bd || (d == bd && p < bp)) { bd = d; bp = p; }
          }
          dist[k] = bd;
          pred[k] = bp == INT_MAX ? -1 : bp;
          rootp[k] = bp == INT_MAX ? -1 : w.root[bp];
        }
      }
    }
  }
  unsigned long long steps = 0, rows = 0, bytes = 0, phases = 0, augs = 0;
  int par = 0;
  int status = 0;
  int matched = ctl->matched;
  // T size at phase start (batched KM: surviving trees)
  int tcount = 0;
  if (ALGO == kAlgoBKM) {
    int mine = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) mine += (inT >> k) & 1u;
    if (t == 0) s_cnt_total = 0;
    __syncthreads();
    atomicAdd(reinterpret_cast<unsigned long long*>(&s_cnt_total), (unsigned long long)mine);
    cluster.sync();
    // every CTA adds its count into rank 0's total, then all read it
    if (t == 0 && rank != 0) {
      long long* r0 = cluster.map_shared_rank(&s_cnt_total, 0);
      atomicAdd(reinterpret_cast<unsigned long long*>(r0), (unsigned long long)s_cnt_total);
    }
    cluster.sync();
    tcount = int(*cluster.map_shared_rank(&s_cnt_total, 0));
  }

  OT_PROF_MARK(0);
  while (matched < n) {
    ++phases;
    int L;              // rows to scan this step: KM one row, batched KM from slots
    int km_row = matched;
    long long km_u = 0;  // u of km_row (0 for the root, whose u is 0 before its phase)
    long long level = 0;
    int src_mask = 0;   // batched KM: which ranks contributed rows at the last level
    if (ALGO == kAlgoKM) {
#pragma unroll
      for (int k = 0; k < K; ++k) { dist[k] = kInf; pred[k] = -1; }
      inT = 0;
      tcount = 0;
      L = 1;
    } else {
      L = 0;  // the pass already scanned every row of S
    }
    int guard = 0;
    long long D = 0;
    int jstar = -1;
    bool augment = false;
    for (;;) {
      if (++guard > m + 2) { status = kDevStepLimit; break; }
      // ---- scan the rows that joined S at `level` ----
      if (ALGO == kAlgoKM) {
        const int i = km_row;
        const long long base = level - (level == 0 ? w.u[i] : km_u);
        const int32_t* row = w.C + i * w.ldc;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int j = g + k * G;
          if (j < m && !((inT >> k) & 1u)) {
            const long long cand = base + __ldg(row + j) - v[k];
            if (cand < dist[k]) { dist[k] = cand; pred[k] = i; }
          }
        }
        bytes += 4ull * (m - tcount);
        rows += 1;
      } else if (L > 0 && w.tma) {
        // Rows of the last level, up to RB at a time: warp 0 maps each row to
        // its source slot (prefix of the per-CTA counts), records (index, u,
        // root) in shared memory and issues the bulk copies of this CTA's
        // segments of the rows into the shared ring, all completing on one
        // mbarrier; then every thread scans its columns from shared memory.
        constexpr int RB = kRingBytes / (K * kLargeTPB * 4);
        constexpr int RBW = RB < 32 ? RB : 32;  // rows staged per warp-0 round
        unsigned row_bytes = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int col0 = rank * kLargeTPB + k * G;
          if (col0 < m) row_bytes += unsigned(min(kLargeTPB, m - col0)) * 4u;
        }
        for (int b0 = 0; b0 < L; b0 += RBW) {
          const int nb = min(RBW, L - b0);
          if (wid == 0) {
            const Slot& mine = slots[par ^ 1][lane < CS ? lane : 0];
            const int mycnt = (lane < CS && ((src_mask >> lane) & 1)) ? mine.cnt : 0;
            int incl = mycnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int y = __shfl_up_sync(0xffffffffu, incl, o);
              if (lane >= o) incl += y;
            }
            const int excl = incl - mycnt;
            // lane e stages row q = b0 + e: its source CTA is the number of
            // CTAs whose inclusive prefix does not exceed q (each lane has
            // its own q, so the prefix values are broadcast one by one)
            const int q = b0 + lane;
            int src = 0;
            for (int r = 0; r < CS; ++r) src += __shfl_sync(0xffffffffu, incl, r) <= q;
            src &= 31;
            const int base_q = __shfl_sync(0xffffffffu, excl, src);
            const int cnt = __shfl_sync(0xffffffffu, mycnt, src);
            if (lane == 0 && row_bytes) mbar_arrive_expect_tx(&s_bar, row_bytes * unsigned(nb));
            __syncwarp();
            if (lane < nb) {
              const int pos = q - base_q;
              RowRef ok_rr{0, 0, 0};
              bool ok = in_range(src, CS, w.ctl->bad, 1, pos) && in_range(pos, cnt, w.ctl->bad, 2, src);
              if (ok) {
                ok_rr = cnt <= kSlotMates ? slots[par ^ 1][src].refs[pos]
                                          : w.ovf[((long long)(par ^ 1) * CS + src) * K * kLargeTPB + pos];
                ok = in_range(ok_rr.row, n, w.ctl->bad, 3, pos) && in_range(ok_rr.root, n, w.ctl->bad, 8, pos);
              }
              if (!ok) { ok_rr.row = 0; ok_rr.root = 0; s_err = 1; }
              s_refs[lane] = ok_rr;
              const int32_t* row = w.C + (long long)ok_rr.row * w.ldc;
#pragma unroll
              for (int k = 0; k < K; ++k) {
                const int col0 = rank * kLargeTPB + k * G;
                if (col0 < m)
                  bulk_g2s(s_ring + (lane * K + k) * kLargeTPB, row + col0, unsigned(min(kLargeTPB, m - col0)) * 4u,
                           &s_bar);
              }
            }
          }
          __syncthreads();
          if (row_bytes) {
            if (!mbar_wait_bounded(&s_bar, bar_parity, kMbarPolls)) s_err = 1;
            bar_parity ^= 1u;
          }
          for (int e = 0; e < nb; ++e) {
            const RowRef rr = s_refs[e];
            const long long base = level - rr.u;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const int j = g + k * G;
              if (j < m && !((inT >> k) & 1u)) {
                const long long cand = base + s_ring[(e * K + k) * kLargeTPB + t] - v[k];
                if (cand < dist[k] || (cand == dist[k] && rr.row < pred[k])) {
                  dist[k] = cand;
                  pred[k] = rr.row;
                  rootp[k] = rr.root;
                }
              }
            }
          }
          __syncthreads();  // the ring and s_refs are rewritten by the next round
        }
        bytes += 4ull * L * (m - tcount);
        rows += L;
      } else if (L > 0) {
        // Rows of the last level: staged into shared memory (index, u,
        // root) from the slots of the CTAs that had columns at that level,
        // then scanned R at a time so that R cost loads are in flight.
        constexpr int R = K >= 4 ? 1 : (K == 2 ? 2 : 8);
        for (int c0 = 0; c0 < L; c0 += LCAP) {
          const int nc = min(LCAP, L - c0);
          for (int q = t; q < nc; q += kLargeTPB) {
            int qq = c0 + q, src = 0;
            for (; src < CS; ++src) {
              if (!((src_mask >> src) & 1)) continue;
              const int cnt = slots[par ^ 1][src].cnt;
              if (qq < cnt) break;
              qq -= cnt;
            }
            const int cnt = slots[par ^ 1][src].cnt;
            s_refs[q] = cnt <= kSlotMates ? slots[par ^ 1][src].refs[qq]
                                          : w.ovf[((long long)(par ^ 1) * CS + src) * K * kLargeTPB + qq];
          }
          __syncthreads();
          for (int q0 = 0; q0 < nc; q0 += R) {
            int cc[R][K];
#pragma unroll
            for (int e = 0; e < R; ++e) {
              const int q = q0 + e;
              const int32_t* row = w.C + (long long)(q < nc ? s_refs[q].row : 0) * w.ldc;
#pragma unroll
              for (int k = 0; k < K; ++k) {
                const int j = g + k * G;
                cc[e][k] = (q < nc && j < m && !((inT >> k) & 1u)) ? __ldg(row + j) : 0;
              }
            }
#pragma unroll
            for (int e = 0; e < R; ++e) {
              const int q = q0 + e;
              if (q >= nc) break;
              const RowRef rr = s_refs[q];
              const long long base = level - rr.u;
#pragma unroll
              for (int k = 0; k < K; ++k) {
                const int j = g + k * G;
                if (j < m && !((inT >> k) & 1u)) {
                  const long long cand = base + cc[e][k] - v[k];
                  if (cand < dist[k] || (cand == dist[k] && rr.row < pred[k])) {
                    dist[k] = cand;
                    pred[k] = rr.row;
                    rootp[k] = rr.root;
                  }
                }
              }
            }
          }
          __syncthreads();
        }
        bytes += 4ull * L * (m - tcount);
        rows += L;
      }
      ++steps;
      OT_PROF_MARK(1);

      // ---- CTA minimum (dist, lowest column) outside T ----
      Best b{kInf, INT_MAX};
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int j = g + k * G;
        if (j < m && !((inT >> k) & 1u) && lex_less(dist[k], j, b.d, b.j)) b = Best{dist[k], j};
      }
      b = warp_argmin(b);
      if (lane == 0) wbest[wid] = b;
      if (t == 0) { s_cnt = 0; s_nfree = 0; s_mate = -1; s_umate = 0; }
      __syncthreads();
      const Best cb = warp_argmin(lane < NW ? wbest[lane] : Best{kInf, INT_MAX});
      // ---- my CTA's candidates at its own minimum: KM the mate of the
      // argmin column, batched KM every column at that distance ----
      Slot& my = slots[par][rank];
      if (ALGO == kAlgoKM) {
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (g + k * G == cb.j) { s_mate = mate[k]; s_umate = umate[k]; }
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int j = g + k * G;
          if (j < m && !((inT >> k) & 1u) && dist[k] == cb.d) {
            if (mate[k] < 0) {
              atomicAdd(&s_nfree, 1);
            } else {
              const int pos = atomicAdd(&s_cnt, 1);
              const RowRef rr{umate[k], mate[k], rootp[k]};
              if (pos < kSlotMates) my.refs[pos] = rr;
              w.ovf[((long long)par * CS + rank) * K * kLargeTPB + pos] = rr;
            }
          }
        }
      }
      __syncthreads();
      // ---- warp 1 asks L2 for the rows this CTA's candidates would add
      // (the winning CTA's prefetch hides most of the next scan's HBM
      // latency behind the exchange)
      if (wid == 1 && w.vec4) {
        const int nrow = ALGO == kAlgoKM ? (s_mate >= 0 ? 1 : 0) : min(s_cnt, 4);
        const int pieces = 4;  // 4 bulk prefetches per row
        const int q = lane / pieces, piece = lane % pieces;
        if (q < nrow) {
          int i = ALGO == kAlgoKM ? s_mate : my.refs[q].row;
          if (!in_range(i, n, w.ctl->bad, 4, q)) i = 0;
          const unsigned bytes = unsigned(m) * 4u;
          const unsigned chunk = ((bytes / pieces) + 15u) & ~15u;
          const unsigned off = piece * chunk;
          if (off < bytes) {
            const unsigned len = min(chunk, bytes - off) & ~15u;
            const char* src = reinterpret_cast<const char*>(w.C + (long long)i * w.ldc) + off;
            if (len) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(len) : "memory");
          }
        }
      }
      // warp r + 2 writes this CTA's slot into CTA r (all destinations in
      // parallel; warps 0 and 1 would otherwise serialise the remote stores)
      if (wid >= 2 && wid - 2 < CS) {
        const int r = wid - 2;
        const int cnt = s_cnt, ncopy = min(cnt, kSlotMates);
        Slot* dst = cluster.map_shared_rank(&slots[par][0], r) + rank;
        if (r != rank && lane < ncopy) dst->refs[lane] = my.refs[lane];
        if (lane == 0) {
          dst->d = cb.d;
          dst->j = cb.j;
          dst->mate = s_mate;
          dst->umate = s_umate;
          dst->cnt = cnt;
          dst->nfree = s_nfree;
          dst->err = s_err;
        }
      }
      OT_PROF_MARK(2);
      cluster.sync();
      OT_PROF_MARK(3);
      // ---- global minimum over the CS slots (lane r reads slot r) ----
      const Slot& sl = slots[par][lane < CS ? lane : 0];
      const bool valid = lane < CS;
      const Best gb = warp_argmin(valid ? Best{sl.d, sl.j} : Best{kInf, INT_MAX});
      D = gb.d;
      jstar = gb.j;
      if (__any_sync(0xffffffffu, valid && sl.err)) { status = kDevStepLimit; break; }
      if (jstar == INT_MAX) { status = kDevStepLimit; break; }
      if (ALGO == kAlgoKM) {
        const unsigned who = __ballot_sync(0xffffffffu, valid && sl.j == jstar);
        const int jm = __shfl_sync(0xffffffffu, valid ? sl.mate : -1, __ffs(who) - 1);
        const long long ju = __shfl_sync(0xffffffffu, valid ? sl.umate : 0ll, __ffs(who) - 1);
        // owner logs the predecessor and, if matched, moves the column into T
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (g + k * G == jstar) {
            w.pred[jstar] = pred[k];
            if (jm >= 0) inT |= 1u << k;
          }
        }
        if (jm < 0) { augment = true; break; }
        km_row = jm;
        km_u = ju;
        level = D;
        ++tcount;
        par ^= 1;
        OT_PROF_MARK(4);
        continue;
      } else {
        const bool at = valid && sl.d == D;
        const int anyfree = __any_sync(0xffffffffu, at && sl.nfree > 0);
        const int total = int(__reduce_add_sync(0xffffffffu, at ? unsigned(sl.cnt) : 0u));
        const int mask = int(__ballot_sync(0xffffffffu, at && sl.cnt > 0));
        // owners: matched columns at level D join T, their mates join S
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int j = g + k * G;
          if (j < m && !((inT >> k) & 1u) && dist[k] == D) {
            w.pred[j] = pred[k];
            if (mate[k] >= 0) {
              inT |= 1u << k;
              const int mt = mate[k];
              w.root[mt] = rootp[k];
              w.inS[mt] = 1;
              w.drow[mt] = D;
            }
          }
        }
        if (anyfree) { augment = true; break; }
        tcount += total;
        L = total;
        src_mask = mask;
        level = D;
        // The next scan reads this step's slots (now slots[par ^ 1]); they
        // are rewritten two steps later, after every CTA passed the next
        // step's cluster barrier.
        par ^= 1;
        OT_PROF_MARK(4);
        continue;
      }
    }
    OT_PROF_MARK(4);
    if (status) break;
    // ---------------- augmentation ----------------
    cluster.sync();
    if (ALGO == kAlgoBKM) {
      // one path per tree: the lowest free column at level D claims the root
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int j = g + k * G;
        if (j < m && !((inT >> k) & 1u) && dist[k] == D && mate[k] < 0 && in_range(rootp[k], n, w.ctl->bad, 5, j))
          atomicMin(&w.claim[rootp[k]], j);
      }
    }
    // accumulated dual adjustment (before the matching changes)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if ((inT >> k) & 1u) {
        const long long dd = D - dist[k];
        v[k] -= dd;
        if (ALGO == kAlgoKM) w.u[mate[k]] += dd;
      }
    }
    if (ALGO == kAlgoKM) {
      if (g == 0) w.u[matched] += D;
    } else {
      for (int i = g; i < n; i += G)
        if (w.inS[i]) w.u[i] += D - w.drow[i];
    }
    if (g == 0) ctl->walkers = 0;
    cluster.sync();
    // flip the winning alternating paths
    int walked = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      int j = g + k * G;
      if (j >= m || ((inT >> k) & 1u) || dist[k] != D || mate[k] >= 0) continue;
      if (ALGO == kAlgoKM && j != jstar) continue;
      if (ALGO == kAlgoBKM && (!in_range(rootp[k], n, w.ctl->bad, 6, j) || w.claim[rootp[k]] != j)) continue;
      int i = pred[k];
      for (int hop = 0; hop <= n; ++hop) {
        const int prev = w.r2c[i];
        w.r2c[i] = j;
        w.c2r[j] = i;
        if (prev < 0) break;
        j = prev;
        i = w.pred[j];
      }
      ++walked;
    }
    if (walked) atomicAdd(&ctl->walkers, walked);
    cluster.sync();
    const int got = ctl->walkers;
    matched += got;
    augs += got;
    if (ALGO == kAlgoBKM) {
      // dissolve the augmented trees; survivors keep S and T at level 0
      for (int i = g; i < n; i += G) {
        if (!w.inS[i]) continue;
        if (w.claim[w.root[i]] != INT_MAX) w.inS[i] = 0;
        else w.drow[i] = 0;
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (((inT >> k) & 1u) && in_range(rootp[k], n, w.ctl->bad, 7, g + k * G) && w.claim[rootp[k]] != INT_MAX)
          inT &= ~(1u << k);
      }
      cluster.sync();
      for (int i = g; i < n; i += G) w.claim[i] = INT_MAX;
      if (g == 0) ctl->scount = 0;
      cluster.sync();
      // rows of S for the next pass
      for (int i = g; i < n; i += G)
        if (w.inS[i]) w.slist[atomicAdd(&ctl->scount, 1)] = i;
      break;  // the next phase starts with a grid-wide pass
    } else {
      // refresh the mates of owned columns after the flips
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int j = g + k * G;
        if (j < m) {
          mate[k] = w.c2r[j];
          umate[k] = mate[k] >= 0 ? w.u[mate[k]] : 0;
        }
      }
      cluster.sync();
      OT_PROF_MARK(5);
    }
  }
  OT_PROF_MARK(5);
  OT_PROF_FLUSH(ctl);
  // write back column state and counters
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int j = g + k * G;
    if (j < m) {
      w.v[j] = v[k];
      w.inT[j] = (inT >> k) & 1u;
    }
  }
  if (g == 0) {
    atomicAdd(&ctl->stats[0], steps);
    atomicAdd(&ctl->stats[1], rows);
    atomicAdd(&ctl->stats[2], bytes);
    atomicAdd(&ctl->stats[3], phases);
    atomicAdd(&ctl->stats[4], augs);
    ctl->matched = matched;
    if (status) ctl->status = status;
    if (status || matched >= n) ctl->done = 1;
  }
  cluster.sync();
}

// cost = sum_i C[i][sigma(i)], counters and status into the instance
__global__ void large_final(LargeWs w, Instance I) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  long long part = 0;
  const bool ok = w.ctl->status == 0 && w.ctl->matched == w.n;
  if (ok)
    for (long long i = tid; i < w.n; i += nth) part += w.C[i * w.ldc + w.r2c[i]];
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0 && part) atomicAdd(reinterpret_cast<unsigned long long*>(I.cost), (unsigned long long)part);
  if (tid == 0) {
    if (I.status) *I.status = ok ? 0 : (w.ctl->status ? w.ctl->status : kDevStepLimit);
    if (I.stats) {
      for (int q = 0; q < 6; ++q) I.stats[q] = (long long)w.ctl->stats[q];
      I.stats[6] = 0;
      I.stats[7] = (long long)w.ctl->stats[2];  // 4-byte elements: read bytes = cost bytes
    }
  }
}

}  // namespace ot

using namespace ot;

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

template <int K, int ALGO>
static cudaError_t launch_steps(const LargeWs& w, int cs, cudaStream_t s) {
  auto kern = large_steps<K, ALGO>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kRingBytes)) != cudaSuccess)
    return e;
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(kLargeTPB, 1, 1);
  cfg.dynamicSmemBytes = kRingBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, w);
}

template <int ALGO>
static cudaError_t launch_steps_k(const LargeWs& w, int cs, int k, cudaStream_t s) {
  switch (k) {
    case 1: return launch_steps<1, ALGO>(w, cs, s);
    case 2: return launch_steps<2, ALGO>(w, cs, s);
    case 4: return launch_steps<4, ALGO>(w, cs, s);
  }
  return cudaErrorInvalidValue;
}

// Largest cluster the step engine can run with on this device (16, else 8).
static int large_cluster_size() {
  static int cached = 0;
  if (cached) return cached;
  // 16 CTAs when the device allows it (n = 16384 batched KM: 1.37 s vs
  // 1.66 s with 8)
  int best = 8;
  auto kern = large_steps<1, kAlgoBKM>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kRingBytes);
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(kLargeTPB, 1, 1);
    cfg.dynamicSmemBytes = kRingBytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) == cudaSuccess && ncl >= 1) best = 16;
  }
  cudaGetLastError();
  cached = best;
  return best;
}

int large_max_cols() { return 4 * kMaxCluster * kLargeTPB; }

// Solve one wide instance (device pointers) on `stream`.  Synchronises the
// stream between batches of phases (batched KM) and at the end.
int solve_large(ot_ctx* ctx, const Instance& I, int algo, cudaStream_t stream, int64_t* stats_out) {
  const int n = I.n, m = I.m;
  const int cs = large_cluster_size();
  int k = 1;
  while (k * cs * kLargeTPB < m) k *= 2;
  if (k > 4) return ctx_fail(ctx, OT_ERR_UNSUPPORTED, "instance too wide for the large engine");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = (m + kPassCols - 1) / kPassCols;
  int chunks = std::max(1, (4 * sms + tiles - 1) / tiles);
  chunks = std::min(chunks, std::max(1, n));

  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += a256(bytes); return o; };
  const size_t o_ctl = take(sizeof(LargeCtl));
  const size_t o_pred = take(4ull * m), o_inT = take(m), o_c2r = take(4ull * m);
  const size_t o_drow = take(8ull * n), o_root = take(4ull * n), o_slist = take(4ull * n);
  const size_t o_inS = take(n), o_claim = take(4ull * n);
  const size_t o_pd = take(8ull * chunks * m), o_pp = take(4ull * chunks * m);
  const size_t o_ovf = take(2ull * cs * k * kLargeTPB * sizeof(RowRef));
  const size_t o_u = I.u ? 0 : take(8ull * n), o_v = I.v ? 0 : take(8ull * m);
  if (int rc = ctx->d_large.reserve(off); rc) return ctx_fail(ctx, rc, "large workspace");
  char* B = static_cast<char*>(ctx->d_large.ptr);
  LargeWs w;
  w.C = I.C; w.ldc = I.ldc; w.n = n; w.m = m;
  w.r2c = I.row_to_col;
  w.u = I.u ? reinterpret_cast<long long*>(I.u) : reinterpret_cast<long long*>(B + o_u);
  w.v = I.v ? reinterpret_cast<long long*>(I.v) : reinterpret_cast<long long*>(B + o_v);
  w.pred = reinterpret_cast<int*>(B + o_pred);
  w.inT = reinterpret_cast<unsigned char*>(B + o_inT);
  w.c2r = reinterpret_cast<int*>(B + o_c2r);
  w.drow = reinterpret_cast<long long*>(B + o_drow);
  w.root = reinterpret_cast<int*>(B + o_root);
  w.slist = reinterpret_cast<int*>(B + o_slist);
  w.inS = reinterpret_cast<unsigned char*>(B + o_inS);
  w.claim = reinterpret_cast<int*>(B + o_claim);
  w.part_d = reinterpret_cast<long long*>(B + o_pd);
  w.part_p = reinterpret_cast<int*>(B + o_pp);
  w.ovf = reinterpret_cast<RowRef*>(B + o_ovf);
  w.ctl = reinterpret_cast<LargeCtl*>(B + o_ctl);
  w.chunks = chunks;
  w.vec4 = (I.ldc % 4 == 0) && (reinterpret_cast<uintptr_t>(I.C) % 16 == 0);
  w.tma = w.vec4 && (m % 4 == 0);

  cudaError_t e = cudaMemsetAsync(I.cost, 0, sizeof(int64_t), stream);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "large memset");
  large_init<<<4 * sms, 256, 0, stream>>>(w, algo == kAlgoBKM);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "large init");
  if (algo == kAlgoKM) {
    if ((e = launch_steps_k<kAlgoKM>(w, cs, k, stream)) != cudaSuccess) return ctx_cuda(ctx, e, "large steps");
  } else {
    const dim3 pgrid(tiles, chunks, 1);
    const int ttiles = (m + kTmaTileCols - 1) / kTmaTileCols;
    const int tchunks = std::max(1, std::min((2 * sms + ttiles - 1) / ttiles, chunks));
    const dim3 tgrid(ttiles, tchunks, 1);
    const bool pass_tma = w.tma;
    if (pass_tma) {
      w.chunks = tchunks;  // the step kernel reduces exactly the partials the pass writes
      if ((e = cudaFuncSetAttribute(large_pass_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaPassSmem)) !=
          cudaSuccess)
        return ctx_cuda(ctx, e, "pass attribute");
    }
    int batch = 4;
    LargeCtl h;
    for (long long launched = 0; launched < 4ll * n + 8;) {
      for (int b = 0; b < batch; ++b) {
        if (pass_tma) {
          large_pass_tma<<<tgrid, kPassThreads, kTmaPassSmem, stream>>>(w);
        } else if (w.vec4) {
          large_pass<1><<<pgrid, kPassThreads, 0, stream>>>(w);
        } else {
          large_pass<0><<<pgrid, kPassThreads, 0, stream>>>(w);
        }
        if ((e = launch_steps_k<kAlgoBKM>(w, cs, k, stream)) != cudaSuccess) return ctx_cuda(ctx, e, "large steps");
      }
      if ((e = cudaMemcpyAsync(&h, w.ctl, sizeof(h), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return ctx_cuda(ctx, e, "large ctl");
      if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return ctx_cuda(ctx, e, "large sync");
      launched += batch;
      if (h.done) break;
      if (batch < 64) batch *= 2;
    }
  }
  large_final<<<sms, 256, 0, stream>>>(w, I);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "large final");
  LargeCtl h;
  if ((e = cudaMemcpyAsync(&h, w.ctl, sizeof(h), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
    return ctx_cuda(ctx, e, "large ctl");
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return ctx_cuda(ctx, e, "large sync");
  if (stats_out)
    for (int q = 0; q < 6; ++q) stats_out[q] = (int64_t)h.stats[q];
#ifdef OT_LARGE_PROFILE
  std::fprintf(stderr, "large_steps cycles: setup %llu scan %llu reduce+publish %llu barrier %llu post %llu augment %llu (steps %llu phases %llu step-rows %llu all-rows %llu)\n",
               h.prof[0], h.prof[1], h.prof[2], h.prof[3], h.prof[4], h.prof[5], h.stats[0], h.stats[3], h.prof[6], h.stats[1]);
#endif
  if (h.bad[0])
    return ctx_fail(ctx, OT_ERR_TIMEOUT, "large engine range check " + std::to_string(h.bad[0]) + " value " +
                                             std::to_string(h.bad[1]) + " aux " + std::to_string(h.bad[2]));
  if (h.status || h.matched != n) return ctx_fail(ctx, OT_ERR_TIMEOUT, "large engine did not converge");
  return OT_OK;
}
