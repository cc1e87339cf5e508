// Group engine: one cooperative thread group solves one assignment instance
// end to end on the device (Kuhn-Munkres or batched KM), many groups per
// launch pull instances from a device work counter.
//
// Layout and ownership.  A group is TPI threads (a warp when TPI == 32,
// otherwise the whole CTA).  Thread t owns columns j = t + k*TPI, k < K, and
// keeps their search state in registers: the tentative distance dist_j
// (the paper's slack, in absolute rather than decremented form), the dual
// v_j, the predecessor row, and one "in T" bit.  Row-indexed state (u,
// row_to_col, tree roots) and the column-indexed arrays that other threads
// must read (col_to_row, the predecessor log used by the augmenting walk)
// live in shared memory.  Cost rows are read straight from global memory
// with coalesced loads: at each step the group reads one row (KM) or the
// rows that just joined the tree (batched KM), only where j is outside T.
//
// Lazy duals.  Instead of touching every u_i, v_j and slack_j at every
// dual adjustment (Sec. 2.3: batched KM moves the duals across the cut of
// reached vertices as KM does), a phase keeps distances relative to the duals
// it started with and applies the accumulated adjustment once, when an
// augmenting path is found: a column that entered T at distance dist_j gets
// v_j -= D - dist_j and its matched row u += D - dist_j; every root gets
// u += D.  This yields exactly the duals of the step-by-step update (every
// comparison is the same integer comparison shifted by a common constant),
// so KM here reproduces the eager CPU reference bit for bit.
#pragma once
#include <climits>
#include <cstdint>

#include "ot_internal.h"

namespace ot {

enum { kAlgoKM = 0, kAlgoBKM = 1, kAlgoAuction = 2 };  // auction: ot_auction.cu

// status codes written by the device (match OT_ERR_* in otassign.h)
enum { kDevOk = 0, kDevStepLimit = -4 };

// (distance, column) pair of an argmin.  V = long long in general; int when
// the instance's rows are packed to 16 bits, where every distance and dual of
// the (row-shifted) problem stays below 2^31 (see solve_instance).
template <typename V>
struct BestT {
  V d;
  int j;
};
using Best = BestT<long long>;

template <typename V>
__device__ __forceinline__ constexpr V inf_of();
template <>
__device__ __forceinline__ constexpr long long inf_of<long long>() { return kInf; }
template <>
__device__ __forceinline__ constexpr int inf_of<int>() { return INT_MAX; }

template <typename V>
__device__ __forceinline__ bool lex_less(V d1, int j1, V d2, int j2) {
  return d1 < d2 || (d1 == d2 && j1 < j2);
}

// Lexicographic (d, j) minimum over the warp with three 32-bit warp
// reductions (redux.sync): flipping the sign bit makes the int64 order an
// unsigned order, then the high word, the low word among lanes holding the
// minimal high word, and the column among lanes holding the minimal key are
// reduced in turn.  Every lane receives the result.
__device__ __forceinline__ Best warp_argmin(Best b) {
  const unsigned long long key = static_cast<unsigned long long>(b.d) ^ 0x8000000000000000ull;
  const unsigned hi = unsigned(key >> 32), lo = unsigned(key);
  const unsigned mh = __reduce_min_sync(0xffffffffu, hi);
  const unsigned ml = __reduce_min_sync(0xffffffffu, hi == mh ? lo : 0xffffffffu);
  const unsigned mj = __reduce_min_sync(0xffffffffu, (hi == mh && lo == ml) ? unsigned(b.j) : 0xffffffffu);
  const unsigned long long mk = (static_cast<unsigned long long>(mh) << 32) | ml;
  return Best{static_cast<long long>(mk ^ 0x8000000000000000ull), int(mj)};
}

// The same for 32-bit distances: two warp reductions.
__device__ __forceinline__ BestT<int> warp_argmin(BestT<int> b) {
  const unsigned key = static_cast<unsigned>(b.d) ^ 0x80000000u;
  const unsigned mk = __reduce_min_sync(0xffffffffu, key);
  const unsigned mj = __reduce_min_sync(0xffffffffu, key == mk ? unsigned(b.j) : 0xffffffffu);
  return BestT<int>{static_cast<int>(mk ^ 0x80000000u), int(mj)};
}

__device__ __forceinline__ long long warp_sum(long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ long long warp_min(long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    long long y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y < x ? y : x;
  }
  return x;
}

// CTA barrier without the .aligned qualifier: each thread first waits for
// the other non-exited lanes of its warp, so the barrier stays correct when
// the warp reaches it split by the data-dependent column branches before it
// (the aligned form, __syncthreads, assumes a converged warp and may count a
// split warp as arrived before its lane 0 stored its reduction slot).
__device__ __forceinline__ void cta_sync() { asm volatile("barrier.sync 0;" ::: "memory"); }

template <int TPI>
__device__ __forceinline__ void group_sync() {
  if constexpr (TPI == 32) __syncwarp();
  else cta_sync();
}

// Shared-memory carve-up of one group.
struct GroupSmem {
  long long* u;   // [nmax] row duals
  int* r2c;       // [nmax] row -> column
  int* c2r;       // [mmax] column -> row
  int* pred;      // [mmax] predecessor row of columns that left the heap
  int* root;      // [nmax] tree root of rows in S (batched KM)
  int* claim;     // [nmax] lowest free column claimed per root (batched KM)
  int* list;      // [nmax] rows that joined S this step (batched KM)
  Best* slots;    // [2 * TPI/32] cross-warp reduction slots
  int* misc;      // [16]
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t group_bytes(int tpi, int algo, int nmax, int mmax) {
  size_t b = align16(8 * size_t(nmax)) + align16(4 * size_t(nmax)) + 2 * align16(4 * size_t(mmax));
  if (algo == kAlgoBKM) b += 3 * align16(4 * size_t(nmax));
  b += align16(2 * (tpi / 32) * sizeof(Best)) + 64;
  return b;
}

__device__ inline GroupSmem carve(unsigned char* p, int tpi, int algo, int nmax, int mmax) {
  GroupSmem s;
  s.u = reinterpret_cast<long long*>(p); p += align16(8 * size_t(nmax));
  s.r2c = reinterpret_cast<int*>(p); p += align16(4 * size_t(nmax));
  s.c2r = reinterpret_cast<int*>(p); p += align16(4 * size_t(mmax));
  s.pred = reinterpret_cast<int*>(p); p += align16(4 * size_t(mmax));
  if (algo == kAlgoBKM) {
    s.root = reinterpret_cast<int*>(p); p += align16(4 * size_t(nmax));
    s.claim = reinterpret_cast<int*>(p); p += align16(4 * size_t(nmax));
    s.list = reinterpret_cast<int*>(p); p += align16(4 * size_t(nmax));
  } else {
    s.root = s.claim = s.list = nullptr;
  }
  s.slots = reinterpret_cast<Best*>(p); p += align16(2 * (tpi / 32) * sizeof(Best));
  s.misc = reinterpret_cast<int*>(p);
  return s;
}

// Minimum (dist, column) over the group; every thread gets the result.
// The slots hold 2 x TPI/32 pairs of either width.
template <int TPI, typename V>
__device__ __forceinline__ BestT<V> group_argmin(BestT<V> b, Best* slots, int& parity) {
  b = warp_argmin(b);
  if constexpr (TPI == 32) {
    __syncwarp();
    return b;
  } else {
    constexpr int NW = TPI / 32;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    BestT<V>* s = reinterpret_cast<BestT<V>*>(slots) + parity * NW;
    parity ^= 1;
    if (l == 0) s[w] = b;
    cta_sync();
    if constexpr (NW == 2) {
      // two warps: every thread compares the two winners itself
      const BestT<V> x = s[0], y = s[1];
      return lex_less(y.d, y.j, x.d, x.j) ? y : x;
    } else {
      BestT<V> c = (l < NW) ? s[l] : BestT<V>{inf_of<V>(), INT_MAX};
      return warp_argmin(c);
    }
  }
}

template <int TPI>
__device__ __forceinline__ long long group_sum(long long x, Best* slots, int& parity) {
  x = warp_sum(x);
  if constexpr (TPI == 32) {
    return x;
  } else {
    constexpr int NW = TPI / 32;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    Best* s = slots + parity * NW;
    parity ^= 1;
    if (l == 0) s[w].d = x;
    cta_sync();
    long long y = (l < NW) ? s[l].d : 0;
    return warp_sum(y);
  }
}

// Solve one instance with the whole group.  t = thread index in the group;
// V is the type of distances and duals in registers (see solve_instance).
template <int TPI, int K, int ALGO, typename V>
__device__ __forceinline__ void solve_instance_v(const Instance& I, const GroupSmem& S, const int t,
                                                 const bool pk) {
  const int n = I.n, m = I.m;
  const int32_t* __restrict__ C = I.C;
  const long long ldc = I.ldc;
  const uint16_t* __restrict__ P = I.P;
  int rpar = 0;  // reduction-slot parity
  constexpr V kInfV = inf_of<V>();

  V dist[K], v[K];
  int pred[K];
  unsigned inT = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) { v[k] = 0; dist[k] = kInfV; pred[k] = -1; }
  // KM's open columns: owned, inside the instance and outside T (recomputed
  // per step: a mask kept in registers costs the register-bound groups more)
  const auto is_open = [&](int k) -> bool { return t + k * TPI < m && !((inT >> k) & 1u); };

  for (int i = t; i < n; i += TPI) { S.r2c[i] = -1; S.u[i] = 0; }
  for (int j = t; j < m; j += TPI) { S.c2r[j] = -1; S.pred[j] = -1; }
  if (t < 16) S.misc[t] = 0;
  group_sync<TPI>();

  long long init_bytes = 0;
  if (ALGO == kAlgoBKM && pk) {
    // B1 on the packed rows: every row minimum is 0 after the shift
    init_bytes = 4LL * n * m;
  } else if constexpr (ALGO == kAlgoBKM) {
    // B1: u_i = min_j C[i][j] (v = 0), one warp per row, lanes stride columns.
    constexpr int NW = TPI / 32;
    const int w = t >> 5, l = t & 31;
    for (int i = w; i < n; i += NW) {
      const int32_t* row = C + i * ldc;
      long long mn = kInf;
      for (int j = l; j < m; j += 32) {
        long long c = __ldg(row + j);
        mn = c < mn ? c : mn;
      }
      mn = warp_min(mn);
      if (l == 0) S.u[i] = mn;
    }
    init_bytes = 4LL * n * m;
  }
  group_sync<TPI>();

  long long steps = 0, rows = 0, bytes = 0, phases = 0, augs = 0;
  long long read_bytes = 0;  // bytes of cost elements actually loaded (2 when packed)
  int status = kDevOk;
  int matched = 0;
  int p = 0;  // list-counter parity (batched KM)

  while (matched < n) {
    ++phases;
#pragma unroll
    for (int k = 0; k < K; ++k) { dist[k] = kInfV; pred[k] = -1; }
    inT = 0;
    int L = 1;
    int km_row = matched;  // KM roots rows in index order
    V level = 0;
    int tcount = 0;

    if constexpr (ALGO == kAlgoBKM) {
      // every free row is a root of the forest; S starts as the free rows
      for (int i = t; i < n; i += TPI) {
        if (S.r2c[i] < 0) {
          int pos = atomicAdd(&S.misc[p], 1);
          S.list[pos] = i;
          S.root[i] = i;
          S.claim[i] = INT_MAX;
        }
      }
      group_sync<TPI>();
      L = S.misc[p];
    }

    // bounded: at most m + 2 steps per phase, and no more than the caller's
    // step cap allows (KM counts a phase's steps when it ends, batched KM
    // one per level as it goes: the same number of guarded iterations)
    long long glim = m + 2;
    if (I.step_limit > 0 && I.step_limit - steps < glim) glim = I.step_limit - steps;
    int guard = 0;
    for (;;) {
      if (++guard > glim) {
        status = kDevStepLimit;
        break;
      }
      if constexpr (ALGO == kAlgoBKM) {
        if (t == 0) S.misc[p ^ 1] = 0;
      }
      // A1 / B2: scan the rows that just joined the tree, columns outside T
      // (KM: fused with the thread's own minimum, A2)
      V kbd = kInfV;
      int kbj = INT_MAX;
      if constexpr (ALGO == kAlgoKM) {
        const int i = km_row;
        const V base = level - V(S.u[i]);
        V c[K];
        if (pk) {
          const uint16_t* prow = P + unsigned(i) * unsigned(m);  // n * m < 2^31 on this engine
#pragma unroll
          for (int k = 0; k < K; ++k) c[k] = is_open(k) ? V(__ldg(prow + t + k * TPI)) : V(0);
        } else {
          const int32_t* row = C + i * ldc;
#pragma unroll
          for (int k = 0; k < K; ++k) c[k] = is_open(k) ? V(__ldg(row + t + k * TPI)) : V(0);
        }
        // columns in increasing order with strict comparisons: the lowest
        // column among equal distances
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (is_open(k)) {
            const V cand = base + c[k] - v[k];
            if (cand < dist[k]) {
              dist[k] = cand;
              pred[k] = i;
            }
            if (dist[k] < kbd) {
              kbd = dist[k];
              kbj = t + k * TPI;
            }
          }
        }
      } else {
        // R rows per round so that R x K cost loads are in flight together
        // (1024-thread groups have 64 registers per thread: fewer rows)
        constexpr int R = TPI >= 1024 ? (K >= 4 ? 2 : 4) : (K >= 8 ? 2 : (K >= 4 ? 4 : (K >= 2 ? 8 : 16)));
        for (int q0 = 0; q0 < L; q0 += R) {
          int cc[R][K];
#pragma unroll
          for (int e = 0; e < R; ++e) {
            const int q = q0 + e;
            const int ri = q < L ? S.list[q] : 0;
            const int32_t* row = C + ri * ldc;
            const uint16_t* prow = P + (long long)ri * m;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const int j = t + k * TPI;
              cc[e][k] = (q < L && j < m && !((inT >> k) & 1u)) ? (pk ? int(__ldg(prow + j)) : __ldg(row + j)) : 0;
            }
          }
#pragma unroll
          for (int e = 0; e < R; ++e) {
            const int q = q0 + e;
            if (q >= L) break;
            const int i = S.list[q];
            const V base = level - V(S.u[i]);
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const int j = t + k * TPI;
              if (j < m && !((inT >> k) & 1u)) {
                const V cand = base + V(cc[e][k]) - v[k];
                if (cand < dist[k] || (cand == dist[k] && i < pred[k])) { dist[k] = cand; pred[k] = i; }
              }
            }
          }
        }
      }
      if constexpr (ALGO == kAlgoBKM) {
        ++steps;
        rows += L;
        bytes += 4LL * L * (m - tcount);
        read_bytes += (pk ? 2LL : 4LL) * L * (m - tcount);
      }

      // A2 / B4: minimum distance outside T, lowest column on ties
      BestT<V> b{kbd, kbj};
      if constexpr (ALGO == kAlgoBKM) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int j = t + k * TPI;
          if (j < m && !((inT >> k) & 1u) && lex_less(dist[k], j, b.d, b.j)) b = BestT<V>{dist[k], j};
        }
      }
      b = group_argmin<TPI, V>(b, S.slots, rpar);
      const V D = b.d;
      if (b.j == INT_MAX) { status = kDevStepLimit; break; }

      if constexpr (ALGO == kAlgoKM) {
        const int js = b.j;
        const int mate = S.c2r[js];
        if ((js % TPI) == t) {
          const int ks = js / TPI;
#pragma unroll
          for (int k = 0; k < K; ++k)
            if (k == ks) {
              S.pred[js] = pred[k];
              if (mate >= 0) inT |= 1u << k;
            }
        }
        if (mate >= 0) {
          km_row = mate;
          level = D;
          ++tcount;
          continue;
        }
        // A3: apply the accumulated dual adjustment
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if ((inT >> k) & 1u) {
            const V dd = D - dist[k];
            v[k] -= dd;
            S.u[S.c2r[t + k * TPI]] += dd;
          }
        }
        if (t == 0) S.u[matched] += D;
        group_sync<TPI>();
        // A4: flip the alternating path that ends at the free column js
        if (t == 0) {
          int j = js, i = S.pred[j];
          for (int hop = 0; hop <= n; ++hop) {
            const int prev = S.r2c[i];
            S.r2c[i] = j;
            S.c2r[j] = i;
            if (prev < 0) break;
            j = prev;
            i = S.pred[j];
          }
        }
        group_sync<TPI>();
        // KM counters once per phase: step s of the phase scanned one row
        // over m - s columns, s = 0 .. tcount
        {
          const long long S = tcount + 1;
          const long long cols = S * m - S * (S - 1) / 2;
          steps += S;
          rows += S;
          bytes += 4 * cols;
          read_bytes += (pk ? 2 : 4) * cols;
        }
        ++matched;
        ++augs;
        break;
      } else {
        // every column at the new level joins T (or ends a path if free)
        unsigned freebits = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int j = t + k * TPI;
          if (j < m && !((inT >> k) & 1u) && dist[k] == D) {
            S.pred[j] = pred[k];
            const int mate = S.c2r[j];
            if (mate < 0) {
              freebits |= 1u << k;
              S.misc[2] = 1;
            } else {
              inT |= 1u << k;
              const int pos = atomicAdd(&S.misc[p ^ 1], 1);
              S.list[pos] = mate;
              S.root[mate] = S.root[pred[k]];
              atomicAdd(&S.misc[4], 1);
            }
          }
        }
        group_sync<TPI>();
        if (S.misc[2] == 0) {
          p ^= 1;
          L = S.misc[p];
          level = D;
          tcount = S.misc[4];
          continue;
        }
        // B4: accumulated dual adjustment across the cut; roots get +D
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if ((inT >> k) & 1u) {
            const V dd = D - dist[k];
            v[k] -= dd;
            S.u[S.c2r[t + k * TPI]] += dd;
          }
        }
        for (int i = t; i < n; i += TPI)
          if (S.r2c[i] < 0) S.u[i] += D;
        // B3: one augmenting path per tree, the lowest free column wins
#pragma unroll
        for (int k = 0; k < K; ++k)
          if ((freebits >> k) & 1u) atomicMin(&S.claim[S.root[pred[k]]], t + k * TPI);
        group_sync<TPI>();
        int walked = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (!((freebits >> k) & 1u)) continue;
          int j = t + k * TPI;
          if (S.claim[S.root[pred[k]]] != j) continue;
          int i = pred[k];
          for (int hop = 0; hop <= n; ++hop) {
            const int prev = S.r2c[i];
            S.r2c[i] = j;
            S.c2r[j] = i;
            if (prev < 0) break;
            j = prev;
            i = S.pred[j];
          }
          ++walked;
        }
        if (walked) atomicAdd(&S.misc[6], walked);
        group_sync<TPI>();
        const int got = S.misc[6];
        matched += got;
        augs += got;
        group_sync<TPI>();
        if (t == 0) {
          S.misc[2] = 0;
          S.misc[4] = 0;
          S.misc[6] = 0;
          S.misc[p] = 0;
        }
        group_sync<TPI>();
        break;
      }
    }
    if (status != kDevOk) break;
    if (phases > (long long)n + 1) { status = kDevStepLimit; break; }
  }

  // A5: objective and outputs
  long long part = 0;
  if (status == kDevOk)
    for (int i = t; i < n; i += TPI) part += __ldg(C + i * ldc + S.r2c[i]);
  const long long cost = group_sum<TPI>(part, S.slots, rpar);
  for (int i = t; i < n; i += TPI) {
    I.row_to_col[i] = S.r2c[i];
    if (I.u) I.u[i] = S.u[i] + (pk ? I.roff[i] : 0);
  }
  if (I.v) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int j = t + k * TPI;
      if (j < m) I.v[j] = v[k];
    }
  }
  if (t == 0) {
    *I.cost = cost;
    if (I.stats) {
      I.stats[0] = steps;
      I.stats[1] = rows;
      I.stats[2] = bytes;
      I.stats[3] = phases;
      I.stats[4] = augs;
      I.stats[5] = init_bytes;
      I.stats[6] = 0;
      I.stats[7] = read_bytes;
    }
  }
  // results before the status word, at system scope: a host thread that
  // polls a status word in mapped host memory may then read the results
  __threadfence_system();
  group_sync<TPI>();
  if (t == 0 && I.status) *reinterpret_cast<volatile int32_t*>(I.status) = status;
  group_sync<TPI>();
}

// Packed instances run on 32-bit distances and duals.  After the row shift
// every cost lies in [0, 65535] = [0, R].  Each dual adjustment raises the
// dual objective sum(u) + sum(v) by at least the step's delta (KM: the root
// gains D and the other changes cancel pairwise; batched KM: at least one free
// root gains D), the objective never exceeds OPT <= n R and starts at 0, so
// every dual moves by at most n R in total and every distance of a phase is
// at most n R.  A candidate level - u_i + c_ij - v_j is then below
// 3 n R + R < 2^31 for n <= 8191 (the group engine has n <= m <= 4096).
template <int TPI, int K, int ALGO>
__device__ void solve_instance(const Instance& I, const GroupSmem& S, const int t) {
  const bool pk = I.P != nullptr && *I.pok != 0;
  if (pk && I.n <= 8191)
    solve_instance_v<TPI, K, ALGO, int>(I, S, t, true);
  else
    solve_instance_v<TPI, K, ALGO, long long>(I, S, t, pk);
}

// Resident warps per SM the group kernels may be compiled for (a register
// cap through __launch_bounds__); 0 leaves the register count to the
// compiler's heuristic for the block size alone.
#ifndef OT_GROUP_MIN_WARPS
#define OT_GROUP_MIN_WARPS 0
#endif
#if OT_GROUP_MIN_WARPS > 0
#define OT_GROUP_BOUNDS(TPI_)                                                                     \
  __launch_bounds__((TPI_) == 32 ? 256 : (TPI_), OT_GROUP_MIN_WARPS * 32 / ((TPI_) == 32 ? 256 : (TPI_)) > 1 \
                                                      ? OT_GROUP_MIN_WARPS * 32 / ((TPI_) == 32 ? 256 : (TPI_)) \
                                                      : 1)
#else
#define OT_GROUP_BOUNDS(TPI_) __launch_bounds__((TPI_) == 32 ? 256 : (TPI_))
#endif

template <int TPI, int K, int ALGO>
__global__ void OT_GROUP_BOUNDS(TPI)
    group_kernel(const Instance* __restrict__ insts, const int32_t* __restrict__ order, int num,
                 int* work, int nmax, int mmax, int groups_per_cta, int bytes_per_group) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int gid = (TPI == 32) ? int(threadIdx.x >> 5) : 0;
  const int t = (TPI == 32) ? int(threadIdx.x & 31) : int(threadIdx.x);
  if (gid >= groups_per_cta) return;
  const GroupSmem S = carve(smem_raw + size_t(gid) * bytes_per_group, TPI, ALGO, nmax, mmax);
  for (;;) {
    int idx;
    if constexpr (TPI == 32) {
      int x = 0;
      if (t == 0) x = atomicAdd(work, 1);
      idx = __shfl_sync(0xffffffffu, x, 0);
    } else {
      if (t == 0) S.misc[15] = atomicAdd(work, 1);
      cta_sync();
      idx = S.misc[15];
      cta_sync();
    }
    if (idx >= num) break;
    const Instance I = insts[order ? order[idx] : idx];
    solve_instance<TPI, K, ALGO>(I, S, t);
  }
}

}  // namespace ot
