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

#include "ot_ctx.h"
#include "ot_group.cuh"

namespace cg = cooperative_groups;

namespace ot {

constexpr int kLargeTPB = 1024;
constexpr int kSlotMates = 32;
constexpr int kPassThreads = 256;
constexpr int kPassCols = 4 * kPassThreads;
constexpr int kMaxCluster = 16;

struct LargeCtl {
  int matched;
  int done;
  int status;
  int scount;
  int walkers;
  int pad[3];
  unsigned long long stats[8];  // steps, rows, bytes, phases, augs, init_bytes
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
  int* ovf;              // [2][cluster][cols per CTA] mates beyond the slot capacity
  LargeCtl* ctl;
  int chunks;
  int vec4;
};

struct __align__(16) Slot {
  long long d;
  int j;
  int mate;
  int cnt;
  int nfree;
  int pad[2];
  int mates[kSlotMates];
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
    for (int q = 0; q < 8; ++q) w.ctl->stats[q] = 0;
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
  __shared__ long long s_cnt_total;

  LargeCtl* ctl = w.ctl;
  if (ctl->done) return;  // uniform over the cluster

  long long dist[K], v[K];
  int pred[K], mate[K];
  unsigned inT = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int j = g + k * G;
    v[k] = 0; dist[k] = kInf; pred[k] = -1; mate[k] = -1;
    if (j < m) {
      v[k] = w.v[j];
      mate[k] = w.c2r[j];
      if (ALGO == kAlgoBKM) {
        if (w.inT[j]) {
          inT |= 1u << k;
          pred[k] = w.pred[j];
          dist[k] = 0;
        } else {
          long long bd = kInf;
          int bp = INT_MAX;
          for (int c = 0; c < w.chunks; ++c) {
            const long long d = w.part_d[(long long)c * m + j];
            const int p = w.part_p[(long long)c * m + j];
            if (d < bd || (d == bd && p < bp)) { bd = d; bp = p; }
          }
          dist[k] = bd;
          pred[k] = bp == INT_MAX ? -1 : bp;
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

  while (matched < n) {
    ++phases;
    int L;              // rows to scan this step: KM one row, batched KM from slots
    int km_row = matched;
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
        const long long base = level - w.u[i];
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
      } else if (L > 0) {
        for (int r = 0; r < CS; ++r) {
          if (!((src_mask >> r) & 1)) continue;
          const Slot& sl = slots[par ^ 1][r];
          const int cnt = sl.cnt;
          for (int q = 0; q < cnt; ++q) {
            const int i = cnt <= kSlotMates ? sl.mates[q] : w.ovf[((long long)(par ^ 1) * CS + r) * K * kLargeTPB + q];
            const long long base = level - w.u[i];
            const int32_t* row = w.C + i * w.ldc;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const int j = g + k * G;
              if (j < m && !((inT >> k) & 1u)) {
                const long long cand = base + __ldg(row + j) - v[k];
                if (cand < dist[k] || (cand == dist[k] && i < pred[k])) { dist[k] = cand; pred[k] = i; }
              }
            }
          }
        }
        bytes += 4ull * L * (m - tcount);
        rows += L;
      }
      ++steps;

      // ---- CTA minimum (dist, lowest column) outside T ----
      Best b{kInf, INT_MAX};
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int j = g + k * G;
        if (j < m && !((inT >> k) & 1u) && lex_less(dist[k], j, b.d, b.j)) b = Best{dist[k], j};
      }
      b = warp_argmin(b);
      if (lane == 0) wbest[wid] = b;
      if (t == 0) { s_cnt = 0; s_nfree = 0; s_mate = -1; }
      __syncthreads();
      Best cb = lane < NW ? wbest[lane] : Best{kInf, INT_MAX};
      cb = warp_argmin(cb);
      // ---- my CTA's candidate list at its own minimum ----
      Slot& my = slots[par][rank];
      if (ALGO == kAlgoKM) {
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (g + k * G == cb.j) s_mate = mate[k];
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int j = g + k * G;
          if (j < m && !((inT >> k) & 1u) && dist[k] == cb.d) {
            if (mate[k] < 0) {
              atomicAdd(&s_nfree, 1);
            } else {
              const int pos = atomicAdd(&s_cnt, 1);
              if (pos < kSlotMates) my.mates[pos] = mate[k];
              w.ovf[((long long)par * CS + rank) * K * kLargeTPB + pos] = mate[k];
            }
          }
        }
      }
      __syncthreads();
      if (t == 0) {
        my.d = cb.d;
        my.j = cb.j;
        my.mate = s_mate;
        my.cnt = s_cnt;
        my.nfree = s_nfree;
      }
      __syncthreads();
      // ---- publish to every CTA of the cluster, one barrier ----
      if (t < CS && t != rank) {
        Slot* dst = cluster.map_shared_rank(&slots[par][0], t);
        const int ncopy = min(my.cnt, kSlotMates);
        dst[rank].d = my.d;
        dst[rank].j = my.j;
        dst[rank].mate = my.mate;
        dst[rank].cnt = my.cnt;
        dst[rank].nfree = my.nfree;
        for (int q = 0; q < ncopy; ++q) dst[rank].mates[q] = my.mates[q];
      }
      cluster.sync();
      // ---- global minimum and the level's columns ----
      D = kInf;
      jstar = INT_MAX;
      for (int r = 0; r < CS; ++r) {
        const Slot& sl = slots[par][r];
        if (lex_less(sl.d, sl.j, D, jstar)) { D = sl.d; jstar = sl.j; }
      }
      if (jstar == INT_MAX) { status = kDevStepLimit; break; }
      if (ALGO == kAlgoKM) {
        int jm = -1;
        for (int r = 0; r < CS; ++r)
          if (slots[par][r].j == jstar) jm = slots[par][r].mate;
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
        level = D;
        ++tcount;
        par ^= 1;
        continue;
      } else {
        int anyfree = 0, total = 0, mask = 0;
        for (int r = 0; r < CS; ++r) {
          const Slot& sl = slots[par][r];
          if (sl.d == D) {
            anyfree |= sl.nfree > 0;
            total += sl.cnt;
            if (sl.cnt > 0) mask |= 1 << r;
          }
        }
        // owners: matched columns at level D join T, their mates join S
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int j = g + k * G;
          if (j < m && !((inT >> k) & 1u) && dist[k] == D) {
            w.pred[j] = pred[k];
            if (mate[k] >= 0) {
              inT |= 1u << k;
              const int mt = mate[k];
              w.root[mt] = w.root[pred[k]];
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
        par ^= 1;
        // the next scan reads slots[par ^ 1] = this step's slots; the
        // barrier of the next step protects them from being overwritten
        cluster.sync();
        continue;
      }
    }
    if (status) break;
    // ---------------- augmentation ----------------
    cluster.sync();
    if (ALGO == kAlgoBKM) {
      // one path per tree: the lowest free column at level D claims the root
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int j = g + k * G;
        if (j < m && !((inT >> k) & 1u) && dist[k] == D && mate[k] < 0)
          atomicMin(&w.claim[w.root[pred[k]]], j);
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
      if (ALGO == kAlgoBKM && w.claim[w.root[pred[k]]] != j) continue;
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
        if (((inT >> k) & 1u) && w.claim[w.root[pred[k]]] != INT_MAX) inT &= ~(1u << k);
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
        if (j < m) mate[k] = w.c2r[j];
      }
      cluster.sync();
    }
  }
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
    if (I.stats)
      for (int q = 0; q < 6; ++q) I.stats[q] = (long long)w.ctl->stats[q];
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
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(kLargeTPB, 1, 1);
  cfg.dynamicSmemBytes = 0;
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
  int best = 8;
  auto kern = large_steps<1, kAlgoBKM>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(kLargeTPB, 1, 1);
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
  const size_t o_ovf = take(8ull * cs * k * kLargeTPB);
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
  w.ovf = reinterpret_cast<int*>(B + o_ovf);
  w.ctl = reinterpret_cast<LargeCtl*>(B + o_ctl);
  w.chunks = chunks;
  w.vec4 = (I.ldc % 4 == 0) && (reinterpret_cast<uintptr_t>(I.C) % 16 == 0);

  cudaError_t e = cudaMemsetAsync(I.cost, 0, sizeof(int64_t), stream);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "large memset");
  large_init<<<4 * sms, 256, 0, stream>>>(w, algo == kAlgoBKM);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "large init");
  if (algo == kAlgoKM) {
    if ((e = launch_steps_k<kAlgoKM>(w, cs, k, stream)) != cudaSuccess) return ctx_cuda(ctx, e, "large steps");
  } else {
    const dim3 pgrid(tiles, chunks, 1);
    int batch = 4;
    LargeCtl h;
    for (int iter = 0; iter < 4 * n + 8; iter += batch) {
      for (int b = 0; b < batch; ++b) {
        if (w.vec4) large_pass<1><<<pgrid, kPassThreads, 0, stream>>>(w);
        else large_pass<0><<<pgrid, kPassThreads, 0, stream>>>(w);
        if ((e = launch_steps_k<kAlgoBKM>(w, cs, k, stream)) != cudaSuccess) return ctx_cuda(ctx, e, "large steps");
      }
      if ((e = cudaMemcpyAsync(&h, w.ctl, sizeof(h), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return ctx_cuda(ctx, e, "large ctl");
      if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return ctx_cuda(ctx, e, "large sync");
      if (h.done) break;
      batch = std::min(batch * 2, 64);
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
  if (h.status || h.matched != n) return ctx_fail(ctx, OT_ERR_TIMEOUT, "large engine did not converge");
  return OT_OK;
}
