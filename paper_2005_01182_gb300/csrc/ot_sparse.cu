// Sparse-list engine for one wide batched-KM instance (Sec. 2.3 "Batched
// KM"; the sparse form the paper benchmarks in Table 3).
//
// The algorithm is the cluster engine's batched KM, step for step: every
// phase grows a forest from all free rows by a multi-source search over
// reduced costs (columns join T level by level, their matched rows join S),
// stops at the first level that reaches free columns, augments one path per
// tree (the lowest free column wins), applies the accumulated dual
// adjustment and dissolves the augmented trees; surviving trees carry over.
// What changes is where the reduced costs come from.
//
// Candidate lists.  Each row keeps the columns of its kCap smallest reduced
// costs, with the bound beta_i below which the list is complete: every
// column j outside it had c_ij - u_i - v_j >= beta_i when it was built.
// Row duals only rise and column duals only fall, so after the row's dual has
// risen by a_i every unlisted reduced cost is still >= beta_i - a_i (its
// remaining budget b_i).  A row that joined S at level d therefore offers
// every unlisted column a distance >= d + b_i, and the search may take a
// level D from the lists alone while D < Lim = min over S rows of (d_i + b_i).
// When the next level reaches Lim, the rows whose bound it reached are
// scanned densely (their exact distances enter the search) and their lists
// are rebuilt around the current duals.  Levels, distances, tie-breaks and
// results are therefore exactly those of the dense search; the dense matrix
// is read once at the start and then only for rows whose budget runs out.
//
// Kernels.  sp_init: row minima (u_i, step B1) and the first lists, a warp
// per row.  Per phase, sp_relax (grid-wide, a warp per row): distances of
// the columns outside T from the lists of the rows that start the phase
// (atomic minimum of a packed (distance, row) key); every row that used half
// its budget is scanned densely and relisted (a row of S also relaxes all
// its columns).  sp_search (one CTA of 1024
// threads, column state in shared memory): the dependent level-by-level
// search -- minimum over the columns outside T, the columns at that level
// join T, their mates' lists are relaxed -- then augmentation and the dual
// update.  sp_final: objective and status.
#include <climits>
#include <cstdint>
#include <cstdio>
#include <string>

#include "ot_ctx.h"
#include "ot_group.cuh"

// Cycle accounting of the search kernel, compiled in only with
// -DOT_SPARSE_PROFILE (thread 0 measures; sections: load, minimum, rescans,
// pop, list relaxation, augmentation and phase end).
#ifdef OT_SPARSE_PROFILE
#define SP_PROF_DECL unsigned long long prof_acc[6] = {0, 0, 0, 0, 0, 0}; unsigned long long sub_acc[6] = {0, 0, 0, 0, 0, 0}; long long prof_t = clock64();
#define SP_PROF(idx)                                      \
  do {                                                    \
    const long long now_ = clock64();                     \
    prof_acc[idx] += (unsigned long long)(now_ - prof_t); \
    prof_t = now_;                                        \
  } while (0)
#define SP_PROF_FLUSH(ctl) \
  do {                     \
    if (t == 0)            \
      for (int q_ = 0; q_ < 6; ++q_) (ctl)->prof[q_] += prof_acc[q_]; \
    if (t == 0)            \
      for (int q_ = 0; q_ < 6; ++q_) (ctl)->sub[q_] += sub_acc[q_]; \
  } while (0)
// time from the start of the relax step to a point of warp 0's own work,
// after the value `dep` has arrived
#define SP_SUB(idx, dep)                                                     \
  do {                                                                       \
    if (t == 0) {                                                            \
      long long sink_;                                                       \
      asm volatile("mov.b64 %0, %1;" : "=l"(sink_) : "l"((long long)(dep)));  \
      sub_acc[idx] += (unsigned long long)(clock64() - sub_t) + (sink_ & 0); \
    }                                                                        \
  } while (0)
#define SP_SUB_START const long long sub_t = clock64();
#else
#define SP_SUB(idx, dep) do {} while (0)
#define SP_SUB_START
#define SP_PROF_DECL
#define SP_PROF(idx) do {} while (0)
#define SP_PROF_FLUSH(ctl) do {} while (0)
#endif

namespace ot {
namespace sp {

constexpr int kCap = 128;                           // list entries per row
constexpr int kRowBits = 15;                        // row bits of a packed key
constexpr unsigned long long kRowMask = (1ull << kRowBits) - 1;
// Distances saturate here.  A level is at most the dual objective's total
// rise, below n * (max C - min C) < 2^14 * 2^32 = 2^46, so a saturated key is
// never the minimum at a level the search takes.
constexpr long long kDistSat = (1LL << 48) - 1;
constexpr unsigned long long kKeyInf = ~0ull;
constexpr int kBins = 196;                          // histogram bins of reduced costs
constexpr int kSearch = 1024;                       // threads of the search CTA
constexpr int kRelaxThreads = 256;
constexpr int kRescanMax = 64;                      // rows rescanned per search round

__device__ __forceinline__ unsigned long long pack(long long d, int row) {
  d = d < 0 ? 0 : (d < kDistSat ? d : kDistSat);
  return (static_cast<unsigned long long>(d) << kRowBits) | static_cast<unsigned>(row);
}
__device__ __forceinline__ long long key_dist(unsigned long long k) { return static_cast<long long>(k >> kRowBits); }
__device__ __forceinline__ int key_row(unsigned long long k) { return static_cast<int>(k & kRowMask); }

// Reduced cost -> histogram bin: 0..15 exact, then four bins per octave.
__device__ __forceinline__ int rc_bin(long long rc) {
  if (rc < 16) return rc < 0 ? 0 : static_cast<int>(rc);
  int e = 63 - __clzll(rc);
  e = e > 47 ? 47 : e;
  return 16 + (e - 4) * 4 + static_cast<int>((rc >> (e - 2)) & 3);
}
// Smallest reduced cost of bin b.
__device__ __forceinline__ long long bin_lo(int b) {
  if (b < 16) return b;
  const int e = 4 + (b - 16) / 4, sub = (b - 16) % 4;
  return static_cast<long long>(4 + sub) << (e - 2);
}

struct Ctl {
  int matched, done, status, phase;
  int scount, sbuf;
  long long lim;                 // min remaining budget of the list-relaxed rows of S
  long long rescans;             // rows scanned densely inside the level search
  unsigned long long stats[8];   // levels, rows, bytes, phases, augs, init bytes
  unsigned long long prof[8];    // cycle accounting (profiling builds)
  unsigned long long sub[8];
};

struct Ws {
  const int32_t* C;
  long long ldc;
  int n, m;
  int32_t* r2c;
  long long* u;
  long long* v;
  int* c2r;
  int* pred;
  unsigned char* inT;
  unsigned long long* dkey;  // [m] phase-start distances (packed keys)
  long long* drow;           // [n] level at which a row joined S
  int* root;                 // [n]
  int* claim;                // [n] lowest free column claimed per root
  int* dense_ph;             // [n] phase in which the row was scanned densely
  int* sstamp;               // [n] phase in which the row is in S at phase start
  int* slist0;               // [n] rows of S at phase start (two buffers)
  int* slist1;
  int* jlist;                // [n] rows that joined S during the phase
  int* jpred;                // [n] the row each joined row was reached from
  int* ecol;                 // [n][kCap] listed columns
  int* ecst;                 // [n][kCap] their costs
  int* ecnt;                 // [n]
  long long* ubase;          // [n] u_i when the list was built
  long long* beta;           // [n] completeness bound of the list
  Ctl* ctl;
  int vec4;                  // rows 16-byte aligned with ldc % 4 == 0
};

// One pass over a cost row: load 4 consecutive costs (vector path) or
// scalars; f(j, c) is called for every column owned by thread t in a stride
// of `width` threads.  LAST marks the last pass over the row: its loads are
// evict-first, so that streaming cost rows through L2 does not push out the
// candidate lists and duals the search keeps re-reading.
template <bool LAST, typename F>
__device__ __forceinline__ void for_row(const Ws& w, const int32_t* row, int t, int width, F f) {
  const int m = w.m;
  if (w.vec4) {
    const int4* r4 = reinterpret_cast<const int4*>(row);
    const int q4 = m >> 2;
    for (int q = t; q < q4; q += width) {
      const int4 c = LAST ? __ldcs(r4 + q) : r4[q];
      const int j = q << 2;
      f(j, c.x);
      f(j + 1, c.y);
      f(j + 2, c.z);
      f(j + 3, c.w);
    }
    for (int j = (q4 << 2) + t; j < m; j += width) f(j, LAST ? __ldcs(row + j) : row[j]);
  } else {
    for (int j = t; j < m; j += width) f(j, LAST ? __ldcs(row + j) : row[j]);
  }
}

// Shared-memory minimum reductions addressed in the shared window (the
// arrays are reached through pointers the compiler cannot always place).
__device__ __forceinline__ unsigned sh_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// Accesses through 32-bit shared-window addresses.
__device__ __forceinline__ unsigned lds32(unsigned a) {
  unsigned v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts32(unsigned a, unsigned v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_min32(unsigned a, unsigned v) {
  unsigned old;
  asm volatile("atom.shared.min.u32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_min32(unsigned a, unsigned v) {
  asm volatile("red.shared.min.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sh_min_u32(unsigned* p, unsigned v) {
  asm volatile("red.shared.min.u32 [%0], %1;" ::"r"(sh_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void sh_min_s64(long long* p, long long v) {
  asm volatile("red.shared.min.s64 [%0], %1;" ::"r"(sh_addr(p)), "l"(v) : "memory");
}
// Candidate-list entries are read and written with an evict-last L2 policy:
// the search re-reads a row's list whenever the row joins S.
__device__ __forceinline__ unsigned long long keep_policy() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int ld_keep(const int* ptr, unsigned long long pol) {
  int x;
  asm volatile("ld.global.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(x) : "l"(ptr), "l"(pol));
  return x;
}
__device__ __forceinline__ void st_keep(int* ptr, int x, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.s32 [%0], %1, %2;" ::"l"(ptr), "r"(x), "l"(pol) : "memory");
}

// The exclusive bound beta of a list of at most kCap entries: the lowest
// edge of the first histogram bin at which the running count exceeds kCap,
// or `cap` when the reduced costs below cap (the only ones counted) fit.
// Called by one full warp.
__device__ __forceinline__ long long choose_beta(const int* hist, int lane, long long cap) {
  int carry = 0;
  for (int b0 = 0; b0 < kBins; b0 += 32) {
    const int b = b0 + lane;
    int x = b < kBins ? hist[b] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const unsigned over = __ballot_sync(0xffffffffu, b < kBins && carry + x > kCap);
    if (over) {
      const long long lo = bin_lo(b0 + __ffs(over) - 1);
      return lo < cap ? lo : cap;
    }
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  return cap;
}

// Upper end of the reduced costs a rebuilt list counts: a list's bound
// tends to stay near the previous one, so costs beyond a few times that
// bound are skipped (the list is then complete up to this cap at least).
__device__ __forceinline__ long long hist_cap(long long old_beta) {
  return old_beta >= (kInf >> 3) ? kInf : 4 * old_beta + 64;
}

// Lower the packed key of column j to `k` unless it is already lower (the
// plain read prunes nearly every candidate before the atomic).
__device__ __forceinline__ void relax_key(unsigned long long* key, unsigned long long k) {
  if (k < *reinterpret_cast<volatile unsigned long long*>(key)) atomicMin(key, k);
}

// ---------------------------------------------------------------------------
// init: column and row state, u_i = min_j C[i][j] (B1), first lists
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRelaxThreads) sp_init(Ws w) {
  const unsigned long long pol = keep_policy();
  __shared__ int hist[kRelaxThreads / 32][kBins];
  __shared__ int s_cnt[kRelaxThreads / 32];
  const int n = w.n, m = w.m;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long j = tid; j < m; j += nth) {
    w.v[j] = 0;
    w.c2r[j] = -1;
    w.inT[j] = 0;
    w.pred[j] = -1;
    w.dkey[j] = kKeyInf;
  }
  for (long long i = tid; i < n; i += nth) {
    w.r2c[i] = -1;
    w.drow[i] = 0;
    w.root[i] = int(i);
    w.claim[i] = INT_MAX;
    w.dense_ph[i] = -1;
    w.sstamp[i] = 0;
    w.slist0[i] = int(i);
  }
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const long long warp = tid >> 5, nwarps = nth >> 5;
  int* h = hist[wl];
  for (long long i = warp; i < n; i += nwarps) {
    const int32_t* row = w.C + i * w.ldc;
    long long mn = kInf;
    for_row<false>(w, row, lane, 32, [&](int, int c) { mn = c < mn ? c : mn; });
    mn = warp_min(mn);
    for (int b = lane; b < kBins; b += 32) h[b] = 0;
    __syncwarp();
    for_row<false>(w, row, lane, 32, [&](int, int c) { atomicAdd(&h[rc_bin((long long)c - mn)], 1); });
    __syncwarp();
    const long long beta = choose_beta(h, lane, kInf);
    if (lane == 0) s_cnt[wl] = 0;
    __syncwarp();
    int* ec = w.ecol + i * kCap;
    int* es = w.ecst + i * kCap;
    for_row<true>(w, row, lane, 32, [&](int j, int c) {
      if ((long long)c - mn < beta) {
        const int p = atomicAdd(&s_cnt[wl], 1);
        if (p < kCap) { st_keep(ec + p, j, pol); st_keep(es + p, c, pol); }
      }
    });
    __syncwarp();
    if (lane == 0) {
      w.u[i] = mn;
      w.ecnt[i] = s_cnt[wl] < kCap ? s_cnt[wl] : kCap;
      w.ubase[i] = mn;
      w.beta[i] = beta;
    }
    __syncwarp();
  }
  if (tid == 0) {
    Ctl* c = w.ctl;
    c->matched = 0;
    c->done = n == 0;
    c->status = 0;
    c->phase = 0;
    c->scount = n;
    c->sbuf = 0;
    c->lim = kInf;
    c->rescans = 0;
    for (int q = 0; q < 8; ++q) c->stats[q] = 0;
    for (int q = 0; q < 8; ++q) c->prof[q] = 0;
    for (int q = 0; q < 8; ++q) c->sub[q] = 0;
    c->stats[5] = 4ull * n * m;
  }
}

// ---------------------------------------------------------------------------
// phase start: distances of the columns outside T from the rows of S, and
// fresh lists for the rows that used half their budget
// ---------------------------------------------------------------------------
// One warp rebuilds row i's list around the current duals (and, for a row
// of S, relaxes every column outside T densely).
__device__ __forceinline__ void warp_rebuild(const Ws& w, int i, long long ui, long long old_beta, bool relax,
                                             int* h, int* cnt, int lane) {
  const unsigned long long pol = keep_policy();
  const int32_t* row = w.C + (long long)i * w.ldc;
  const long long hc = hist_cap(old_beta);
  for (int x = lane; x < kBins; x += 32) h[x] = 0;
  __syncwarp();
  for_row<false>(w, row, lane, 32, [&](int j, int c) {
    const long long rc = (long long)c - ui - __ldg(w.v + j);
    if (relax && !w.inT[j]) relax_key(w.dkey + j, pack(rc, i));
    if (rc < hc) atomicAdd(&h[rc_bin(rc)], 1);
  });
  __syncwarp();
  const long long nb = choose_beta(h, lane, hc);
  if (lane == 0) *cnt = 0;
  __syncwarp();
  int* ec = w.ecol + (long long)i * kCap;
  int* es = w.ecst + (long long)i * kCap;
  for_row<true>(w, row, lane, 32, [&](int j, int c) {
    if ((long long)c - ui - __ldg(w.v + j) < nb) {
      const int p = atomicAdd(cnt, 1);
      if (p < kCap) { st_keep(ec + p, j, pol); st_keep(es + p, c, pol); }
    }
  });
  __syncwarp();
  if (lane == 0) {
    w.ecnt[i] = *cnt < kCap ? *cnt : kCap;
    w.ubase[i] = ui;
    w.beta[i] = nb;
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kRelaxThreads) sp_relax(Ws w) {
  Ctl* ctl = w.ctl;
  if (ctl->done) return;
  const unsigned long long pol = keep_policy();
  __shared__ int hist[kRelaxThreads / 32][kBins];
  __shared__ int s_cnt[kRelaxThreads / 32];
  const int n = w.n, m = w.m;
  const int phase = ctl->phase;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long rows = 0, bytes = 0;
  long long lim = kInf;
  for (long long i = warp; i < n; i += nwarps) {
    const bool inS = w.sstamp[i] == phase;
    const long long ui = w.u[i];
    const long long beta = w.beta[i];
    const long long b = beta - (ui - w.ubase[i]);
    if (b <= 0 || b < (beta >> 1)) {
      // half the budget used: a fresh list (and, in S, exact distances)
      warp_rebuild(w, int(i), ui, beta, inS, hist[wl], &s_cnt[wl], lane);
      if (lane == 0) {
        if (inS) w.dense_ph[i] = phase;
        rows += 1;
        bytes += 4ull * m;
      }
    } else if (inS) {
      const int cnt = w.ecnt[i];
      const int* ec = w.ecol + i * kCap;
      const int* es = w.ecst + i * kCap;
      constexpr int kPer = kCap / 32;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int e = lane + 32 * q;
        if (e < cnt) {
          const int j = ld_keep(ec + e, pol);
          if (!w.inT[j]) relax_key(w.dkey + j, pack((long long)ld_keep(es + e, pol) - ui - __ldg(w.v + j), int(i)));
        }
      }
      if (lane == 0) {
        lim = b < lim ? b : lim;
        rows += 1;
        bytes += 8ull * cnt;
      }
    }
  }
  if (lane == 0) {
    if (lim < kInf) atomicMin(&ctl->lim, lim);
    if (rows) {
      atomicAdd(&ctl->stats[1], rows);
      atomicAdd(&ctl->stats[2], bytes);
    }
  }
}

// Warp minimum of a signed 64-bit value with two 32-bit warp reductions
// (redux.sync): flipping the sign bit turns the signed order into the
// unsigned order of (high word, low word).
__device__ __forceinline__ long long warp_min64(long long x) {
  const unsigned long long k = static_cast<unsigned long long>(x) ^ 0x8000000000000000ull;
  const unsigned hi = unsigned(k >> 32), lo = unsigned(k);
  const unsigned mh = __reduce_min_sync(0xffffffffu, hi);
  const unsigned ml = __reduce_min_sync(0xffffffffu, hi == mh ? lo : 0xffffffffu);
  return static_cast<long long>(((static_cast<unsigned long long>(mh) << 32) | ml) ^ 0x8000000000000000ull);
}

// Block-wide minimum of two int64 values (every thread receives both).
struct Min2 {
  long long a, b;
};
__device__ __forceinline__ Min2 block_min2(long long a, long long b, long long (*slots)[2][32], int& par) {
  a = warp_min64(a);
  b = warp_min64(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    slots[par][0][wid] = a;
    slots[par][1][wid] = b;
  }
  __syncthreads();
  a = warp_min64(slots[par][0][lane]);
  b = warp_min64(slots[par][1][lane]);
  par ^= 1;
  return Min2{a, b};
}

// ---------------------------------------------------------------------------
// the dependent search of one phase, augmentation and dual update
// ---------------------------------------------------------------------------
// Status of a phase that hands the solve to the dense cluster engine: its
// levels would leave the 32-bit distance range of the search, or the lists
// hold so few columns (heavily tied costs in a small range) that the search
// has rescanned more than n rows densely itself, on one SM.
constexpr int kToDense = -100;
constexpr unsigned kSat32 = 0xffffffffu;
constexpr unsigned kLevelMax = 0x7fffffffu;

__device__ __forceinline__ unsigned sat32(long long d) { return d < (long long)kSat32 ? unsigned(d) : kSat32; }

// Column state in shared memory: the distance (32 bits, saturating) and the
// row it was reached from (lowest row among those at that distance), the
// column's matched row, the T bits and, per warp, the smallest distance among
// its columns outside T.  All updates are native 32-bit shared atomics: a
// candidate (d, row) first takes the minimum distance (a column whose
// distance drops forgets its row), then, after a barrier, the candidates
// that reached the final distance take the minimum row.  Every distance the
// search compares at a level below 2^31 is exact; a phase whose next level
// would be 2^31 or more stops with kToDense.
__global__ void __launch_bounds__(kSearch, 1) sp_search(Ws w) {
  Ctl* ctl = w.ctl;
  if (ctl->done) return;
  const unsigned long long pol = keep_policy();
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = w.n, m = w.m;
  const int words = (m + 31) >> 5;
  const int wal = (words + 3) & ~3;
  unsigned* kd = reinterpret_cast<unsigned*>(smem);     // [m] distance
  unsigned* kr = kd + m;                                // [m] row reached from
  int* c2rs = reinterpret_cast<int*>(kr + m);           // [m] column -> row
  unsigned* tb = reinterpret_cast<unsigned*>(c2rs + m); // [words] column in T
  unsigned* t0 = tb + wal;                              // [words] column in T at phase start
  int* hist = reinterpret_cast<int*>(t0 + wal);         // [kBins]
  __shared__ long long slots[2][2][32];
  __shared__ unsigned wdist[kSearch / 32];  // smallest distance outside T per warp's columns
  __shared__ long long s_lim;
  __shared__ int s_rows[kSearch];  // rows that joined at the current level
  __shared__ int s_prs[kSearch];   // the rows they were reached from
  __shared__ int s_resc[kRescanMax];
  __shared__ int s_nnew, s_free, s_nres, s_cnt, s_walk, s_scnt;
  __shared__ long long s_beta;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int kc = (m + kSearch - 1) / kSearch;
  const int phase = ctl->phase, S = ctl->scount;
  const int* sl = ctl->sbuf ? w.slist1 : w.slist0;
  int* snext = ctl->sbuf ? w.slist0 : w.slist1;
  unsigned D = 0;  // the current level
  const unsigned a_kd = sh_addr(kd), a_kr = sh_addr(kr), a_c2r = sh_addr(c2rs), a_tb = sh_addr(tb);
  const unsigned a_wd = sh_addr(wdist);
  auto inT = [&](int j) { return (lds32(a_tb + 4u * unsigned(j >> 5)) >> (j & 31)) & 1u; };
  auto KD = [&](int j) { return lds32(a_kd + 4u * unsigned(j)); };
  // first step of a candidate: the distance
  auto lower_d = [&](int j, unsigned d) {
    const unsigned old = atom_min32(a_kd + 4u * unsigned(j), d);
    if (d < old) sts32(a_kr + 4u * unsigned(j), kSat32);
    red_min32(a_wd + 4u * unsigned((j >> 5) & 31), d);
  };
  // second step (after a barrier): the row, for candidates at the distance
  auto lower_r = [&](int j, unsigned d, int row) {
    if (KD(j) == d) red_min32(a_kr + 4u * unsigned(j), unsigned(row));
  };

  for (int j = t; j < m; j += kSearch) {
    c2rs[j] = w.c2r[j];
    if (w.inT[j]) {
      kd[j] = 0;
      kr[j] = unsigned(w.pred[j]);
    } else {
      const unsigned long long k = w.dkey[j];
      kd[j] = sat32(key_dist(k));
      kr[j] = k == kKeyInf ? kSat32 : unsigned(key_row(k));
    }
  }
  for (int q = wid; q < words; q += kSearch / 32) {
    const int j = (q << 5) + lane;
    const unsigned bits = __ballot_sync(0xffffffffu, j < m && w.inT[j]);
    if (lane == 0) tb[q] = t0[q] = bits;
  }
  if (t == 0) { s_nnew = 0; s_free = 0; s_nres = 0; s_lim = kInf; }
  __syncthreads();
  {
    unsigned md = kSat32;
    for (int k = 0; k < kc; ++k) {
      const int j = t + k * kSearch;
      if (j < m && !inT(j)) {
        const unsigned dj = KD(j);
        md = dj < md ? dj : md;
      }
    }
    md = __reduce_min_sync(0xffffffffu, md);
    if (lane == 0) wdist[wid] = md;
  }
  __syncthreads();
  SP_PROF_DECL

  long long Lim = ctl->lim;
  int par = 0;
  int jcount = 0;
  int status = 0;
  unsigned long long levels = 0, rows = 0, bytes = 0;
  long long rescans = 0;  // rows rescanned in this phase
  // candidates of this warp's first relaxed row, kept for the row step
  constexpr int kPer = kCap / 32;
  int cj[kPer];
  unsigned cd[kPer];
  for (int guard = 0;; ++guard) {
    if (guard > m + n + 4) { status = kDevStepLimit; break; }
    // ---- minimum distance outside T: over the 32 warp minima ----
    D = __reduce_min_sync(0xffffffffu, wdist[lane]);
    SP_PROF(1);
    Lim = s_lim < Lim ? s_lim : Lim;
    // every warp has read the minima (and finished the previous level's row
    // steps) before any of them changes
    __syncthreads();
    if ((long long)D >= Lim) {
      // ---- rows whose list bound the level reached: dense rescans ----
      long long nl = kInf;
      for (int q = t; q < S + jcount; q += kSearch) {
        const int i = q < S ? sl[q] : w.jlist[q - S];
        if (w.dense_ph[i] == phase) continue;
        const long long l = w.drow[i] + w.beta[i] - (w.u[i] - w.ubase[i]);
        if (l <= (long long)D) {
          const int p = atomicAdd(&s_nres, 1);
          if (p < kRescanMax) s_resc[p] = i;
          else nl = l < nl ? l : nl;  // left for the next round
        } else {
          nl = l < nl ? l : nl;
        }
      }
      __syncthreads();
      const int nr = s_nres < kRescanMax ? s_nres : kRescanMax;
      rescans += nr;
      // Lists too short for the instance (heavily tied costs in a small
      // range): more than n/4 rows rescanned here at more than 4 per level,
      // or 8 n in all.  Each rescan is a dense row pass on one SM, while the
      // dense engine scans its rows on a whole cluster; measured at
      // n = 4096, floor(C/16) of the circle/square instance needs about 25
      // rescans per level (sparse 0.25 s, dense 0.05 s), circle/square and
      // circle/triangle about 0.5 (either engine within 10 %, sparse faster
      // on circle/square), the grids none.
      {
        const long long done_rows = ctl->rescans + rescans;
        const long long done_levels = (long long)ctl->stats[0] + (long long)levels;
        if ((done_rows > n / 4 && done_rows > 4 * done_levels) || done_rows > 8ll * n) {
          status = kToDense;
          break;
        }
      }
      for (int x = 0; x < nr; ++x) {
        const int i = s_resc[x];
        const long long ui = w.u[i], dr = w.drow[i];
        const int32_t* row = w.C + (long long)i * w.ldc;
        const long long hc = hist_cap(w.beta[i]);
        for (int b = t; b < kBins; b += kSearch) hist[b] = 0;
        __syncthreads();
        for_row<false>(w, row, t, kSearch, [&](int j, int c) {
          const long long rc = (long long)c - ui - __ldg(w.v + j);
          if (!inT(j)) lower_d(j, sat32(dr + rc));
          if (rc < hc) atomicAdd(&hist[rc_bin(rc)], 1);
        });
        __syncthreads();
        if (wid == 0) {
          const long long nb = choose_beta(hist, lane, hc);
          if (lane == 0) { s_beta = nb; s_cnt = 0; }
        }
        __syncthreads();
        const long long nb = s_beta;
        int* ec = w.ecol + (long long)i * kCap;
        int* es = w.ecst + (long long)i * kCap;
        // the row step of the dense candidates, and the new list
        for_row<true>(w, row, t, kSearch, [&](int j, int c) {
          const long long rc = (long long)c - ui - __ldg(w.v + j);
          if (!inT(j)) lower_r(j, sat32(dr + rc), i);
          if (rc < nb) {
            const int p = atomicAdd(&s_cnt, 1);
            if (p < kCap) { st_keep(ec + p, j, pol); st_keep(es + p, c, pol); }
          }
        });
        __syncthreads();
        if (t == 0) {
          w.ecnt[i] = s_cnt < kCap ? s_cnt : kCap;
          w.ubase[i] = ui;
          w.beta[i] = nb;
          w.dense_ph[i] = phase;
          rows += 1;
          bytes += 4ull * m;
        }
      }
      if (t == 0) {
        s_nres = 0;
        s_lim = kInf;  // folded into nl
      }
      // the bound of the rows still on lists; the next round recomputes the
      // level with the new distances
      const Min2 r2 = block_min2(nl, kInf, slots, par);
      Lim = r2.a;
      SP_PROF(2);
      continue;
    }
    if (D > kLevelMax) { status = D == kSat32 ? kDevStepLimit : kToDense; break; }
    // ---- the columns at level D join T; free ones end augmenting paths;
    // the warps holding them recompute their minimum ----
    if (wdist[wid] == D) {
      unsigned md = kSat32;
      for (int k = 0; k < kc; ++k) {
        const int j = t + k * kSearch;
        if (j >= m || inT(j)) continue;
        const unsigned dj = KD(j);
        if (dj != D) {
          md = dj < md ? dj : md;
          continue;
        }
        const int pr = int(lds32(a_kr + 4u * unsigned(j)));
        w.pred[j] = pr;
        const int mate = int(lds32(a_c2r + 4u * unsigned(j)));
        if (mate < 0) {
          s_free = 1;
          md = dj < md ? dj : md;
        } else {
          atomicOr(tb + (j >> 5), 1u << (j & 31));
          const int p = atomicAdd(&s_nnew, 1);
          if (p < kSearch) {
            s_rows[p] = mate;
            s_prs[p] = pr;
          }
          w.jlist[jcount + p] = mate;
          w.jpred[jcount + p] = pr;
          w.drow[mate] = D;
        }
      }
      md = __reduce_min_sync(0xffffffffu, md);
      if (lane == 0) wdist[wid] = md;
    }
    __syncthreads();
    SP_PROF(3);
    ++levels;
    const int nnew = s_nnew;
    if (s_free) {
      // rows that joined at the augmenting level stay in S: their roots
      for (int x = t; x < nnew; x += kSearch) {
        const int i = x < kSearch ? s_rows[x] : w.jlist[jcount + x];
        const int pr = x < kSearch ? s_prs[x] : w.jpred[jcount + x];
        w.root[i] = w.root[pr];
      }
      jcount += nnew;
      __syncthreads();
      break;
    }
    // ---- relax the lists of the rows that joined S at level D: the
    // distance step, a barrier, the row step ----
    const int j0 = jcount;  // rows of this level: jlist[j0 .. j0 + nnew)
    auto load_row = [&](int x, int& i, int& cnt, long long& ui, int* jj, int* cc, long long* vv) {
      i = x < kSearch ? s_rows[x] : w.jlist[j0 + x];
      const int* ec = w.ecol + (long long)i * kCap;
      const int* es = w.ecst + (long long)i * kCap;
      ui = w.u[i];
      cnt = w.ecnt[i];
#pragma unroll
      for (int q = 0; q < kPer; ++q) {  // within the row's slot of kCap entries
        jj[q] = ld_keep(ec + lane + 32 * q, pol);
        cc[q] = ld_keep(es + lane + 32 * q, pol);
      }
#pragma unroll
      for (int q = 0; q < kPer; ++q) vv[q] = lane + 32 * q < cnt ? __ldg(w.v + jj[q]) : 0;
    };
    int crow = -1;
    SP_SUB_START
    for (int x = wid; x < nnew; x += kSearch / 32) {
      int i, cnt;
      long long ui;
      int jj[kPer], cc[kPer];
      long long vv[kPer];
      // the row's dual, list length and list entries, its bound and the
      // root of the row it was reached from: one round trip, then one for v
      const int pr = x < kSearch ? s_prs[x] : w.jpred[j0 + x];
      const int rt = w.root[pr];
      load_row(x, i, cnt, ui, jj, cc, vv);
      const long long lim_i = w.beta[i] - (ui - w.ubase[i]);
      const long long base = (long long)D - ui;
      if (x == 0) SP_SUB(0, ui + cnt + jj[0] + cc[kPer - 1] + rt + lim_i);
      if (x == 0) SP_SUB(1, vv[0] + vv[kPer - 1]);
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const bool live = lane + 32 * q < cnt && !inT(jj[q]);
        const unsigned d = live ? sat32(base + cc[q] - vv[q]) : kSat32;
        if (live) lower_d(jj[q], d);
        if (crow < 0) {
          cj[q] = live ? jj[q] : -1;
          cd[q] = d;
        }
      }
      if (x == 0) SP_SUB(2, cd[0]);
      if (crow < 0) crow = i;
      if (lane == 0) {
        w.root[i] = rt;
        sh_min_s64(&s_lim, (long long)D + lim_i);
        rows += 1;
        bytes += 8ull * cnt;
      }
      if (x == 0) SP_SUB(3, 0);
    }
    jcount += nnew;
    __syncthreads();
    SP_SUB(4, 0);
    // row step: the warp's first row from registers, any further rows of
    // the warp (more than 32 joined at this level) reloaded
    if (crow >= 0) {
#pragma unroll
      for (int q = 0; q < kPer; ++q)
        if (cj[q] >= 0) lower_r(cj[q], cd[q], crow);
    }
    for (int x = wid + kSearch / 32; x < nnew; x += kSearch / 32) {
      int i, cnt;
      long long ui;
      int jj[kPer], cc[kPer];
      long long vv[kPer];
      load_row(x, i, cnt, ui, jj, cc, vv);
      const long long base = (long long)D - ui;
#pragma unroll
      for (int q = 0; q < kPer; ++q)
        if (lane + 32 * q < cnt && !inT(jj[q])) lower_r(jj[q], sat32(base + cc[q] - vv[q]), i);
    }
    SP_SUB(5, 0);
    if (t == 0) s_nnew = 0;
    SP_PROF(4);
  }

  if (status == 0) {
    // ---- augmentation: one path per tree, the lowest free column wins ----
    for (int k = 0; k < kc; ++k) {
      const int j = t + k * kSearch;
      if (j >= m || inT(j) || c2rs[j] >= 0 || kd[j] != D) continue;
      atomicMin(w.claim + w.root[kr[j]], j);
    }
    // accumulated dual adjustment (before the matching changes): columns
    // carried in T since the phase started sit at distance 0
    for (int k = 0; k < kc; ++k) {
      const int j = t + k * kSearch;
      if (j >= m || !inT(j)) continue;
      const long long dd = (long long)D - (((t0[j >> 5] >> (j & 31)) & 1u) ? 0 : (long long)kd[j]);
      if (dd) {
        w.v[j] -= dd;
        w.u[c2rs[j]] += dd;
      }
    }
    for (int q = t; q < S; q += kSearch) {
      const int i = sl[q];
      if (w.r2c[i] < 0) w.u[i] += D;
    }
    if (t == 0) { s_walk = 0; s_scnt = 0; }
    __syncthreads();
    int walked = 0;
    for (int k = 0; k < kc; ++k) {
      const int j0c = t + k * kSearch;
      if (j0c >= m || inT(j0c) || c2rs[j0c] >= 0 || kd[j0c] != D) continue;
      int i = int(kr[j0c]);
      if (w.claim[w.root[i]] != j0c) continue;
      int j = j0c;
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
    if (walked) atomicAdd(&s_walk, walked);
    __syncthreads();
    // dissolve the augmented trees; the survivors start the next phase at
    // level 0 and form its S
    for (int q = t; q < S + jcount; q += kSearch) {
      const int i = q < S ? sl[q] : w.jlist[q - S];
      if (w.claim[w.root[i]] != INT_MAX) continue;
      w.drow[i] = 0;
      w.sstamp[i] = phase + 1;
      snext[atomicAdd(&s_scnt, 1)] = i;
    }
    for (int k = 0; k < kc; ++k) {
      const int j = t + k * kSearch;
      if (j >= m || !inT(j)) continue;
      if (w.claim[w.root[w.pred[j]]] != INT_MAX) atomicAnd(tb + (j >> 5), ~(1u << (j & 31)));
    }
    __syncthreads();
    for (int q = t; q < S; q += kSearch) w.claim[sl[q]] = INT_MAX;
    for (int j = t; j < m; j += kSearch) {
      w.inT[j] = inT(j);
      w.dkey[j] = kKeyInf;
    }
  }
  SP_PROF(5);
  SP_PROF_FLUSH(ctl);
  if (t == 0) {
    ctl->stats[0] += levels;
    ctl->stats[1] += rows;
    ctl->stats[2] += bytes;
    ctl->stats[3] += 1;
    ctl->rescans += rescans;
    if (status) {
      ctl->status = status;
      ctl->done = 1;
    } else {
      ctl->stats[4] += s_walk;
      ctl->matched += s_walk;
      ctl->scount = s_scnt;
      ctl->sbuf ^= 1;
      ctl->phase = phase + 1;
      ctl->lim = kInf;
      if (ctl->matched >= n) ctl->done = 1;
    }
  }
}

// cost = sum_i C[i][sigma(i)], counters and status into the instance
__global__ void sp_final(Ws w, Instance I) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const bool ok = w.ctl->status == 0 && w.ctl->matched == w.n;
  long long part = 0;
  if (ok)
    for (long long i = tid; i < w.n; i += nth) part += w.C[i * w.ldc + w.r2c[i]];
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0 && part)
    atomicAdd(reinterpret_cast<unsigned long long*>(I.cost), static_cast<unsigned long long>(part));
  if (tid == 0) {
    if (I.status) *I.status = ok ? 0 : (w.ctl->status ? w.ctl->status : kDevStepLimit);
    if (I.stats) {
      for (int q = 0; q < 6; ++q) I.stats[q] = (long long)w.ctl->stats[q];
      I.stats[6] = 0;
      I.stats[7] = (long long)w.ctl->stats[2];
    }
  }
}

}  // namespace sp
}  // namespace ot

using namespace ot;

int sparse_max_cols() { return 16384; }

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Solve one batched-KM instance (device pointers, n <= m <= 16384) on
// `stream`; synchronises the stream between batches of phases and at the end.
int solve_sparse(ot_ctx* ctx, const Instance& I, cudaStream_t stream, int64_t* stats_out) {
  using namespace ot::sp;
  const int n = I.n, m = I.m;
  if (m > sparse_max_cols() || n > m) return ctx_fail(ctx, OT_ERR_UNSUPPORTED, "instance too wide for the sparse engine");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += a256(bytes); return o; };
  const size_t o_ctl = take(sizeof(Ctl));
  const size_t o_c2r = take(4ull * m), o_pred = take(4ull * m), o_inT = take(m), o_dkey = take(8ull * m);
  const size_t o_drow = take(8ull * n), o_root = take(4ull * n), o_claim = take(4ull * n), o_dph = take(4ull * n);
  const size_t o_s0 = take(4ull * n), o_s1 = take(4ull * n), o_j = take(4ull * n), o_jp = take(4ull * n);
  const size_t o_st = take(4ull * n);
  const size_t o_ecol = take(4ull * n * kCap), o_ecst = take(4ull * n * kCap), o_ecnt = take(4ull * n);
  const size_t o_ub = take(8ull * n), o_beta = take(8ull * n);
  const size_t o_u = I.u ? 0 : take(8ull * n), o_v = I.v ? 0 : take(8ull * m);
  if (int rc = ctx->d_large.reserve(off); rc) return ctx_fail(ctx, rc, "sparse workspace");
  char* B = static_cast<char*>(ctx->d_large.ptr);
  Ws w;
  w.C = I.C; w.ldc = I.ldc; w.n = n; w.m = m;
  w.r2c = I.row_to_col;
  w.u = I.u ? reinterpret_cast<long long*>(I.u) : reinterpret_cast<long long*>(B + o_u);
  w.v = I.v ? reinterpret_cast<long long*>(I.v) : reinterpret_cast<long long*>(B + o_v);
  w.c2r = reinterpret_cast<int*>(B + o_c2r);
  w.pred = reinterpret_cast<int*>(B + o_pred);
  w.inT = reinterpret_cast<unsigned char*>(B + o_inT);
  w.dkey = reinterpret_cast<unsigned long long*>(B + o_dkey);
  w.drow = reinterpret_cast<long long*>(B + o_drow);
  w.root = reinterpret_cast<int*>(B + o_root);
  w.claim = reinterpret_cast<int*>(B + o_claim);
  w.dense_ph = reinterpret_cast<int*>(B + o_dph);
  w.slist0 = reinterpret_cast<int*>(B + o_s0);
  w.slist1 = reinterpret_cast<int*>(B + o_s1);
  w.jlist = reinterpret_cast<int*>(B + o_j);
  w.jpred = reinterpret_cast<int*>(B + o_jp);
  w.sstamp = reinterpret_cast<int*>(B + o_st);
  w.ecol = reinterpret_cast<int*>(B + o_ecol);
  w.ecst = reinterpret_cast<int*>(B + o_ecst);
  w.ecnt = reinterpret_cast<int*>(B + o_ecnt);
  w.ubase = reinterpret_cast<long long*>(B + o_ub);
  w.beta = reinterpret_cast<long long*>(B + o_beta);
  w.ctl = reinterpret_cast<Ctl*>(B + o_ctl);
  w.vec4 = (I.ldc % 4 == 0) && (reinterpret_cast<uintptr_t>(I.C) % 16 == 0);

  const int words = (m + 31) >> 5;
  const size_t smem = 3 * 4ull * m + 2 * 4ull * ((words + 3) & ~3) + 4ull * kBins;
  cudaError_t e = cudaFuncSetAttribute(sp_search, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "sparse search attribute");
  if ((e = cudaMemsetAsync(I.cost, 0, sizeof(int64_t), stream)) != cudaSuccess) return ctx_cuda(ctx, e, "sparse memset");
  sp_init<<<4 * sms, kRelaxThreads, 0, stream>>>(w);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "sparse init");
  Ctl h;
  int batch = 4;
  // every phase augments at least one path: n phases suffice
  for (long long launched = 0; launched < (long long)n + 8;) {
    for (int b = 0; b < batch; ++b) {
      sp_relax<<<2 * sms, kRelaxThreads, 0, stream>>>(w);
      sp_search<<<1, kSearch, smem, stream>>>(w);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "sparse phase");
    if ((e = cudaMemcpyAsync(&h, w.ctl, sizeof(h), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
      return ctx_cuda(ctx, e, "sparse ctl");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return ctx_cuda(ctx, e, "sparse sync");
    launched += batch;
    if (h.done) break;
    if (batch < 64) batch *= 2;
  }
  sp_final<<<sms, 256, 0, stream>>>(w, I);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "sparse final");
  if ((e = cudaMemcpyAsync(&h, w.ctl, sizeof(h), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
    return ctx_cuda(ctx, e, "sparse ctl");
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return ctx_cuda(ctx, e, "sparse sync");
  if (stats_out)
    for (int q = 0; q < 6; ++q) stats_out[q] = (int64_t)h.stats[q];
#ifdef OT_SPARSE_PROFILE
  std::fprintf(stderr, "sp_search cycles: min %llu rescan %llu pop %llu relax %llu augment+end %llu; rescanned rows %lld\n",
               h.prof[1], h.prof[2], h.prof[3], h.prof[4], h.prof[5], h.rescans);
  std::fprintf(stderr, "relax, warp 0 from the step start: loads %llu v %llu distance step %llu row done %llu "
               "barrier %llu row step %llu\n", h.sub[0], h.sub[1], h.sub[2], h.sub[3], h.sub[4], h.sub[5]);
#endif
  if (h.status == kToDense) return solve_large(ctx, I, kAlgoBKM, stream, stats_out);
  if (h.status || h.matched != n)
    return ctx_fail(ctx, OT_ERR_TIMEOUT, "sparse engine did not converge (status " + std::to_string(h.status) +
                                             ", matched " + std::to_string(h.matched) + " of " + std::to_string(n) +
                                             ", phases " + std::to_string(h.phase) + ")");
  return OT_OK;
}
