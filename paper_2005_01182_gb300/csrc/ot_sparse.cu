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
// per row.  Per phase, sp_relax (grid-wide, a warp per row of S): distances
// of the columns outside T from the lists of the rows that start the phase
// (atomic minimum of a packed (distance, row) key), rows that used half
// their budget scanned densely and relisted.  sp_search (one CTA of 1024
// threads, column state in shared memory): the dependent level-by-level
// search -- minimum over the columns outside T, the columns at that level
// join T, their mates' lists are relaxed -- then augmentation and the dual
// update.  sp_final: objective and status.
#include <climits>
#include <cstdint>
#include <string>

#include "ot_ctx.h"
#include "ot_group.cuh"

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
  unsigned long long stats[8];   // levels, rows, bytes, phases, augs, init bytes
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
  int* slist0;               // [n] rows of S at phase start (two buffers)
  int* slist1;
  int* jlist;                // [n] rows that joined S during the phase
  int* ecol;                 // [n][kCap] listed columns
  int* ecst;                 // [n][kCap] their costs
  int* ecnt;                 // [n]
  long long* ubase;          // [n] u_i when the list was built
  long long* beta;           // [n] completeness bound of the list
  Ctl* ctl;
  int vec4;                  // rows 16-byte aligned with ldc % 4 == 0
};

// The warp's view of one row: load 4 consecutive costs (vector path) or
// scalars.  f(j, c) is called for every column of the row owned by `lane`
// in a stride of `width` threads.
template <typename F>
__device__ __forceinline__ void for_row(const Ws& w, const int32_t* row, int t, int width, F f) {
  const int m = w.m;
  if (w.vec4) {
    const int4* r4 = reinterpret_cast<const int4*>(row);
    const int q4 = m >> 2;
    for (int q = t; q < q4; q += width) {
      const int4 c = r4[q];
      const int j = q << 2;
      f(j, c.x);
      f(j + 1, c.y);
      f(j + 2, c.z);
      f(j + 3, c.w);
    }
    for (int j = (q4 << 2) + t; j < m; j += width) f(j, row[j]);
  } else {
    for (int j = t; j < m; j += width) f(j, row[j]);
  }
}

// The exclusive bound beta of a list of at most kCap entries: the lowest
// edge of the first histogram bin at which the running count exceeds kCap
// (kInf when the whole row fits).  Called by one full warp.
__device__ __forceinline__ long long choose_beta(const int* hist, int lane) {
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
    if (over) return bin_lo(b0 + __ffs(over) - 1);
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  return kInf;
}

// ---------------------------------------------------------------------------
// init: column and row state, u_i = min_j C[i][j] (B1), first lists
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRelaxThreads) sp_init(Ws w) {
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
    w.slist0[i] = int(i);
  }
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const long long warp = tid >> 5, nwarps = nth >> 5;
  int* h = hist[wl];
  for (long long i = warp; i < n; i += nwarps) {
    const int32_t* row = w.C + i * w.ldc;
    long long mn = kInf;
    for_row(w, row, lane, 32, [&](int, int c) { mn = c < mn ? c : mn; });
    mn = warp_min(mn);
    for (int b = lane; b < kBins; b += 32) h[b] = 0;
    __syncwarp();
    for_row(w, row, lane, 32, [&](int, int c) { atomicAdd(&h[rc_bin((long long)c - mn)], 1); });
    __syncwarp();
    const long long beta = choose_beta(h, lane);
    if (lane == 0) s_cnt[wl] = 0;
    __syncwarp();
    int* ec = w.ecol + i * kCap;
    int* es = w.ecst + i * kCap;
    for_row(w, row, lane, 32, [&](int j, int c) {
      if ((long long)c - mn < beta) {
        const int p = atomicAdd(&s_cnt[wl], 1);
        if (p < kCap) { ec[p] = j; es[p] = c; }
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
    for (int q = 0; q < 8; ++q) c->stats[q] = 0;
    c->stats[5] = 4ull * n * m;
  }
}

// ---------------------------------------------------------------------------
// phase start: distances of the columns outside T from the rows of S
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRelaxThreads) sp_relax(Ws w) {
  Ctl* ctl = w.ctl;
  if (ctl->done) return;
  __shared__ int hist[kRelaxThreads / 32][kBins];
  __shared__ int s_cnt[kRelaxThreads / 32];
  const int m = w.m;
  const int phase = ctl->phase, S = ctl->scount;
  const int* sl = ctl->sbuf ? w.slist1 : w.slist0;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  int* h = hist[wl];
  unsigned long long rows = 0, bytes = 0;
  long long lim = kInf;
  for (long long q = warp; q < S; q += nwarps) {
    const int i = sl[q];
    const long long ui = w.u[i];
    const long long beta = w.beta[i];
    const long long b = beta - (ui - w.ubase[i]);
    if (b <= 0 || b < (beta >> 1)) {
      // half the budget used: exact distances from the dense row, new list
      const int32_t* row = w.C + (long long)i * w.ldc;
      for (int x = lane; x < kBins; x += 32) h[x] = 0;
      __syncwarp();
      for_row(w, row, lane, 32, [&](int j, int c) {
        const long long rc = (long long)c - ui - __ldg(w.v + j);
        if (!w.inT[j]) atomicMin(w.dkey + j, pack(rc, i));
        atomicAdd(&h[rc_bin(rc)], 1);
      });
      __syncwarp();
      const long long nb = choose_beta(h, lane);
      if (lane == 0) s_cnt[wl] = 0;
      __syncwarp();
      int* ec = w.ecol + (long long)i * kCap;
      int* es = w.ecst + (long long)i * kCap;
      for_row(w, row, lane, 32, [&](int j, int c) {
        if ((long long)c - ui - __ldg(w.v + j) < nb) {
          const int p = atomicAdd(&s_cnt[wl], 1);
          if (p < kCap) { ec[p] = j; es[p] = c; }
        }
      });
      __syncwarp();
      if (lane == 0) {
        w.ecnt[i] = s_cnt[wl] < kCap ? s_cnt[wl] : kCap;
        w.ubase[i] = ui;
        w.beta[i] = nb;
        w.dense_ph[i] = phase;
        rows += 1;
        bytes += 4ull * m;
      }
      __syncwarp();
    } else {
      const int cnt = w.ecnt[i];
      const int* ec = w.ecol + (long long)i * kCap;
      const int* es = w.ecst + (long long)i * kCap;
      for (int e = lane; e < cnt; e += 32) {
        const int j = ec[e];
        if (!w.inT[j]) atomicMin(w.dkey + j, pack((long long)es[e] - ui - __ldg(w.v + j), i));
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

// Block-wide minimum of two int64 values (every thread receives both).
struct Min2 {
  long long a, b;
};
__device__ __forceinline__ Min2 block_min2(long long a, long long b, long long (*slots)[2][32], int& par) {
  a = warp_min(a);
  b = warp_min(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    slots[par][0][wid] = a;
    slots[par][1][wid] = b;
  }
  __syncthreads();
  a = warp_min(slots[par][0][lane]);
  b = warp_min(slots[par][1][lane]);
  par ^= 1;
  return Min2{a, b};
}

// ---------------------------------------------------------------------------
// the dependent search of one phase, augmentation and dual update
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSearch, 1) sp_search(Ws w) {
  Ctl* ctl = w.ctl;
  if (ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = w.n, m = w.m;
  const int words = (m + 31) >> 5;
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem);
  int* c2rs = reinterpret_cast<int*>(key + m);
  unsigned* tb = reinterpret_cast<unsigned*>(c2rs + m);
  int* hist = reinterpret_cast<int*>(tb + ((words + 3) & ~3));
  __shared__ long long slots[2][2][32];
  __shared__ int s_rows[kSearch];
  __shared__ int s_resc[kRescanMax];
  __shared__ int s_nnew, s_free, s_nres, s_cnt, s_walk, s_scnt;
  __shared__ long long s_beta;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int kc = (m + kSearch - 1) / kSearch;
  const int phase = ctl->phase, S = ctl->scount;
  const int* sl = ctl->sbuf ? w.slist1 : w.slist0;
  int* snext = ctl->sbuf ? w.slist0 : w.slist1;
  auto inT = [&](int j) { return (tb[j >> 5] >> (j & 31)) & 1u; };

  for (int j = t; j < m; j += kSearch) {
    c2rs[j] = w.c2r[j];
    key[j] = w.inT[j] ? pack(0, w.pred[j]) : w.dkey[j];
  }
  for (int q = wid; q < words; q += kSearch / 32) {
    const int j = (q << 5) + lane;
    const unsigned bits = __ballot_sync(0xffffffffu, j < m && w.inT[j]);
    if (lane == 0) tb[q] = bits;
  }
  if (t == 0) { s_nnew = 0; s_free = 0; s_nres = 0; }
  __syncthreads();

  long long Lim = ctl->lim;
  int par = 0;
  int jcount = 0;
  int status = 0;
  long long D = 0;
  unsigned long long levels = 0, rows = 0, bytes = 0;
  long long my_lim = kInf;  // list bounds of the rows relaxed since the last reduction
  for (int guard = 0;; ++guard) {
    if (guard > m + n + 4) { status = kDevStepLimit; break; }
    // ---- minimum distance outside T ----
    long long lmin = kDistSat;
    for (int k = 0; k < kc; ++k) {
      const int j = t + k * kSearch;
      if (j < m && !inT(j)) {
        const long long d = key_dist(key[j]);
        lmin = d < lmin ? d : lmin;
      }
    }
    const Min2 r = block_min2(lmin, my_lim, slots, par);
    my_lim = kInf;
    D = r.a;
    Lim = r.b < Lim ? r.b : Lim;
    if (D >= kDistSat) { status = kDevStepLimit; break; }
    if (D >= Lim) {
      // ---- rows whose list bound the level reached: dense rescans ----
      long long nl = kInf;
      for (int q = t; q < S + jcount; q += kSearch) {
        const int i = q < S ? sl[q] : w.jlist[q - S];
        if (w.dense_ph[i] == phase) continue;
        const long long l = w.drow[i] + w.beta[i] - (w.u[i] - w.ubase[i]);
        if (l <= D) {
          const int p = atomicAdd(&s_nres, 1);
          if (p < kRescanMax) s_resc[p] = i;
          else nl = l < nl ? l : nl;  // left for the next round
        } else {
          nl = l < nl ? l : nl;
        }
      }
      __syncthreads();
      const int nr = s_nres < kRescanMax ? s_nres : kRescanMax;
      for (int x = 0; x < nr; ++x) {
        const int i = s_resc[x];
        const long long ui = w.u[i], dr = w.drow[i];
        const int32_t* row = w.C + (long long)i * w.ldc;
        for (int b = t; b < kBins; b += kSearch) hist[b] = 0;
        __syncthreads();
        for_row(w, row, t, kSearch, [&](int j, int c) {
          const long long rc = (long long)c - ui - __ldg(w.v + j);
          if (!inT(j)) atomicMin(key + j, pack(dr + rc, i));
          atomicAdd(&hist[rc_bin(rc)], 1);
        });
        __syncthreads();
        if (wid == 0) {
          const long long nb = choose_beta(hist, lane);
          if (lane == 0) { s_beta = nb; s_cnt = 0; }
        }
        __syncthreads();
        const long long nb = s_beta;
        int* ec = w.ecol + (long long)i * kCap;
        int* es = w.ecst + (long long)i * kCap;
        for_row(w, row, t, kSearch, [&](int j, int c) {
          if ((long long)c - ui - __ldg(w.v + j) < nb) {
            const int p = atomicAdd(&s_cnt, 1);
            if (p < kCap) { ec[p] = j; es[p] = c; }
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
      if (t == 0) s_nres = 0;
      // the bound of the rows still on lists; the next round recomputes the
      // level with the new distances
      const Min2 r2 = block_min2(nl, kInf, slots, par);
      Lim = r2.a;
      continue;
    }
    // ---- the columns at level D join T; free ones end augmenting paths ----
    if (lmin == D) {
      for (int k = 0; k < kc; ++k) {
        const int j = t + k * kSearch;
        if (j >= m || inT(j)) continue;
        const unsigned long long kj = key[j];
        if (key_dist(kj) != D) continue;
        const int pr = key_row(kj);
        w.pred[j] = pr;
        const int mate = c2rs[j];
        if (mate < 0) {
          s_free = 1;
        } else {
          atomicOr(tb + (j >> 5), 1u << (j & 31));
          const int p = atomicAdd(&s_nnew, 1);
          if (p < kSearch) s_rows[p] = mate;
          w.jlist[jcount + p] = mate;
          w.drow[mate] = D;
          w.root[mate] = w.root[pr];
        }
      }
    }
    __syncthreads();
    ++levels;
    if (s_free) break;
    const int nnew = s_nnew;
    // ---- relax the lists of the rows that joined S at level D ----
    for (int x = wid; x < nnew; x += kSearch / 32) {
      const int i = x < kSearch ? s_rows[x] : w.jlist[jcount + x];
      const long long ui = w.u[i];
      const int cnt = w.ecnt[i];
      const int* ec = w.ecol + (long long)i * kCap;
      const int* es = w.ecst + (long long)i * kCap;
      const long long base = D - ui;
      for (int e = lane; e < cnt; e += 32) {
        const int j = ec[e];
        if (!inT(j)) atomicMin(key + j, pack(base + es[e] - __ldg(w.v + j), i));
      }
      if (lane == 0) {
        const long long l = D + w.beta[i] - (ui - w.ubase[i]);
        my_lim = l < my_lim ? l : my_lim;
        rows += 1;
        bytes += 8ull * cnt;
      }
    }
    jcount += nnew;
    __syncthreads();
    if (t == 0) s_nnew = 0;
  }

  if (status == 0) {
    // ---- augmentation: one path per tree, the lowest free column wins ----
    for (int k = 0; k < kc; ++k) {
      const int j = t + k * kSearch;
      if (j >= m || inT(j) || c2rs[j] >= 0 || key_dist(key[j]) != D) continue;
      atomicMin(w.claim + w.root[key_row(key[j])], j);
    }
    // accumulated dual adjustment (before the matching changes)
    for (int k = 0; k < kc; ++k) {
      const int j = t + k * kSearch;
      if (j >= m || !inT(j)) continue;
      const long long dd = D - key_dist(key[j]);
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
      const int j0 = t + k * kSearch;
      if (j0 >= m || inT(j0) || c2rs[j0] >= 0 || key_dist(key[j0]) != D) continue;
      int i = key_row(key[j0]);
      if (w.claim[w.root[i]] != j0) continue;
      int j = j0;
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
      snext[atomicAdd(&s_scnt, 1)] = i;
    }
    for (int k = 0; k < kc; ++k) {
      const int j = t + k * kSearch;
      if (j >= m || !inT(j)) continue;
      if (w.claim[w.root[key_row(key[j])]] != INT_MAX) atomicAnd(tb + (j >> 5), ~(1u << (j & 31)));
    }
    __syncthreads();
    for (int q = t; q < S; q += kSearch) w.claim[sl[q]] = INT_MAX;
    for (int j = t; j < m; j += kSearch) {
      w.inT[j] = inT(j);
      w.dkey[j] = kKeyInf;
    }
  }
  if (t == 0) {
    ctl->stats[0] += levels;
    ctl->stats[1] += rows;
    ctl->stats[2] += bytes;
    ctl->stats[3] += 1;
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
  const size_t o_s0 = take(4ull * n), o_s1 = take(4ull * n), o_j = take(4ull * n);
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
  w.ecol = reinterpret_cast<int*>(B + o_ecol);
  w.ecst = reinterpret_cast<int*>(B + o_ecst);
  w.ecnt = reinterpret_cast<int*>(B + o_ecnt);
  w.ubase = reinterpret_cast<long long*>(B + o_ub);
  w.beta = reinterpret_cast<long long*>(B + o_beta);
  w.ctl = reinterpret_cast<Ctl*>(B + o_ctl);
  w.vec4 = (I.ldc % 4 == 0) && (reinterpret_cast<uintptr_t>(I.C) % 16 == 0);

  const int words = (m + 31) >> 5;
  const size_t smem = 8ull * m + 4ull * m + 4ull * ((words + 3) & ~3) + 4ull * kBins;
  cudaError_t e = cudaFuncSetAttribute(sp_search, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "sparse search attribute");
  if ((e = cudaMemsetAsync(I.cost, 0, sizeof(int64_t), stream)) != cudaSuccess) return ctx_cuda(ctx, e, "sparse memset");
  sp_init<<<4 * sms, kRelaxThreads, 0, stream>>>(w);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "sparse init");
  Ctl h;
  int batch = 4;
  for (int iter = 0; iter < n + 8; iter += batch) {
    for (int b = 0; b < batch; ++b) {
      sp_relax<<<2 * sms, kRelaxThreads, 0, stream>>>(w);
      sp_search<<<1, kSearch, smem, stream>>>(w);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "sparse phase");
    if ((e = cudaMemcpyAsync(&h, w.ctl, sizeof(h), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
      return ctx_cuda(ctx, e, "sparse ctl");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return ctx_cuda(ctx, e, "sparse sync");
    if (h.done) break;
    batch = std::min(batch * 2, 64);
  }
  sp_final<<<sms, 256, 0, stream>>>(w, I);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "sparse final");
  if ((e = cudaMemcpyAsync(&h, w.ctl, sizeof(h), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
    return ctx_cuda(ctx, e, "sparse ctl");
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return ctx_cuda(ctx, e, "sparse sync");
  if (stats_out)
    for (int q = 0; q < 6; ++q) stats_out[q] = (int64_t)h.stats[q];
  if (h.status || h.matched != n) return ctx_fail(ctx, OT_ERR_TIMEOUT, "sparse engine did not converge");
  return OT_OK;
}
