// Auction engine: the auction algorithm with epsilon-scaling (Sec. 2.3.3
// "The auction algorithm", Sec. 4.1 "Auction") as an exact solver, one CTA
// per instance, many instances per launch pulled from a device work counter.
//
// Method (the readings are the same as the CPU oracle's):
//   * costs are shifted to start at 0 and scaled by N + 1 (N = m bidders
//     after padding the n real rows with m - n all-zero dummy rows); bidder
//     i values object j at w_ij = C'[i][j] + p_j;
//   * every unassigned bidder bids in parallel (Jacobi rounds, the parallel
//     bidding of Sec. 2.3.3) for its lowest-w object (lowest index on ties),
//     raising its price to p + (runner-up w - lowest w) + eps; an object goes
//     to its highest bid, the lowest bidder index among equal bids, takes the
//     bid as its price and releases its previous holder;
//   * epsilon-scaling: eps_0 = max(1, R'/8) for the scaled range R', then
//     eps /= 4 (at least 1) per stage, prices kept, holders reset; the stage
//     at eps = 1 is the last, which makes the assignment exact for integer
//     costs (within N < N + 1 of the scaled optimum).
// The result of a round does not depend on the order in which bids are
// computed or resolved (maximum, then minimum index, both with atomics), so
// the device reproduces the oracle's rounds exactly.
//
// Layout.  Prices, holders, bids and the bidder list live in shared memory
// (44 bytes per column: 180 KB at m = 4096).  Warp w computes the bids of
// bidders w, w + W, ...: its lanes stride over the bidder's cost row with
// coalesced 4-byte loads, keep a per-lane (lowest w, its column, runner-up),
// and merge them with butterfly shuffles.
#include <climits>
#include <cstdint>

#include "ot_internal.h"

namespace ot {

namespace {

constexpr long long kWInf = 1LL << 61;  // above every scaled value + price
constexpr int kDevOk = 0, kDevStepLimit = -4, kDevOverflow = -6;

struct Bid {
  long long w1;  // lowest value
  int j1;        // its column (lowest index among equal values)
  long long w2;  // second-lowest value of the multiset (w1 when tied)
};

__device__ __forceinline__ Bid merge(Bid a, Bid b) {
  if (b.w1 < a.w1 || (b.w1 == a.w1 && b.j1 < a.j1)) {
    const Bid t = a;
    a = b;
    b = t;
  }
  a.w2 = min(a.w2, b.w1);
  return a;
}

__device__ __forceinline__ Bid warp_merge(Bid b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Bid x;
    x.w1 = __shfl_xor_sync(0xffffffffu, b.w1, o);
    x.j1 = __shfl_xor_sync(0xffffffffu, b.j1, o);
    x.w2 = __shfl_xor_sync(0xffffffffu, b.w2, o);
    b = merge(b, x);
  }
  return b;
}

struct AuctionSmem {
  long long* p;       // [N] prices
  long long* best;    // [N] highest bid this round (LLONG_MIN: none)
  long long* amt;     // [N] bid of bidder i
  int* winner;        // [N] lowest bidder index holding the highest bid
  int* holder;        // [N] object -> bidder, -1
  int* held;          // [N] bidder -> object, -1
  int* obj;           // [N] object bidder i bid for
  int* list;          // [N] bidders of the round
  long long* red;     // [64] block reductions
  int* misc;          // [8]
  Bid* part;          // [32] per-warp partial bids (a bidder split over warps)
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t auction_bytes(int N) {
  return 3 * al16(8 * size_t(N)) + 5 * al16(4 * size_t(N)) + 8 * 64 + 4 * 8 + 32 * sizeof(Bid);
}

__device__ AuctionSmem carve_auction(unsigned char* base, int N) {
  AuctionSmem S;
  size_t o = 0;
  S.p = reinterpret_cast<long long*>(base + o); o += al16(8 * size_t(N));
  S.best = reinterpret_cast<long long*>(base + o); o += al16(8 * size_t(N));
  S.amt = reinterpret_cast<long long*>(base + o); o += al16(8 * size_t(N));
  S.red = reinterpret_cast<long long*>(base + o); o += 8 * 64;
  S.winner = reinterpret_cast<int*>(base + o); o += al16(4 * size_t(N));
  S.holder = reinterpret_cast<int*>(base + o); o += al16(4 * size_t(N));
  S.held = reinterpret_cast<int*>(base + o); o += al16(4 * size_t(N));
  S.obj = reinterpret_cast<int*>(base + o); o += al16(4 * size_t(N));
  S.list = reinterpret_cast<int*>(base + o); o += al16(4 * size_t(N));
  S.misc = reinterpret_cast<int*>(base + o); o += 4 * 8;
  S.part = reinterpret_cast<Bid*>(base + o);
  return S;
}

// Block-wide min and max of per-thread values (results to every thread).
template <int T>
__device__ void block_minmax(long long& mn, long long& mx, long long* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    red[wid] = mn;
    red[32 + wid] = mx;
  }
  __syncthreads();
  mn = red[0];
  mx = red[32];
  for (int w = 1; w < T / 32; ++w) {
    mn = min(mn, red[w]);
    mx = max(mx, red[32 + w]);
  }
  __syncthreads();
}

template <int T>
__device__ long long block_sum(long long v, long long* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  long long s = 0;
  for (int w = 0; w < T / 32; ++w) s += red[w];
  __syncthreads();
  return s;
}

template <int T>
__device__ __forceinline__ void auction_instance(const Instance& I, const AuctionSmem& S) {
  constexpr int W = T / 32;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = I.n, N = I.m;
  const long long ldc = I.ldc;
  int status = kDevOk;
  long long stages = 0, rounds = 0, bids = 0, real_bids = 0;

  // range of the real costs (one pass over the matrix)
  long long mn = LLONG_MAX, mx = LLONG_MIN;
  for (int i = wid; i < n; i += W) {
    const int32_t* row = I.C + i * ldc;
    for (int j = lane; j < N; j += 32) {
      const long long c = __ldg(row + j);
      mn = min(mn, c);
      mx = max(mx, c);
    }
  }
  block_minmax<T>(mn, mx, S.red);
  const long long cmin = mn;
  const long long scale = (long long)N + 1;
  const long long range = (mx - mn) * scale;  // < 2^32 * 2^13: no overflow
  if (range > (1LL << 50)) status = kDevOverflow;

  for (int k = tid; k < N; k += T) S.p[k] = 0;
  long long eps = range / 8;
  if (eps < 1) eps = 1;
  const long long round_cap = 4LL * N * (N + 1) + 64;
  while (status == kDevOk) {
    ++stages;
    for (int k = tid; k < N; k += T) {
      S.holder[k] = -1;
      S.held[k] = -1;
      S.best[k] = LLONG_MIN;
      S.winner[k] = INT_MAX;
    }
    long long stage_rounds = 0;
    for (;;) {
      // bidders of this round: every unassigned bidder (any order)
      if (tid == 0) S.misc[0] = 0;
      __syncthreads();
      for (int i = tid; i < N; i += T)
        if (S.held[i] < 0) S.list[atomicAdd(&S.misc[0], 1)] = i;
      __syncthreads();
      const int U = S.misc[0];
      if (U == 0) break;
      if (++stage_rounds > round_cap) {
        status = kDevStepLimit;
        break;
      }
      ++rounds;
      bids += U;
      // bids against the round-start prices: the lanes of a warp stride the
      // bidder's row (several loads in flight), then a butterfly merge
      auto scan = [&](int i, int j0, int jstep) {
        Bid b{kWInf, INT_MAX, kWInf};
        if (i < n) {
          const int32_t* row = I.C + i * ldc;
#pragma unroll 4
          for (int j = j0; j < N; j += jstep) {
            const long long w = ((long long)__ldg(row + j) - cmin) * scale + S.p[j];
            if (w < b.w1) {
              b.w2 = b.w1;
              b.w1 = w;
              b.j1 = j;
            } else if (w < b.w2) {
              b.w2 = w;
            }
          }
        } else {
#pragma unroll 4
          for (int j = j0; j < N; j += jstep) {
            const long long w = S.p[j];
            if (w < b.w1) {
              b.w2 = b.w1;
              b.w1 = w;
              b.j1 = j;
            } else if (w < b.w2) {
              b.w2 = w;
            }
          }
        }
        return warp_merge(b);
      };
      auto place_bid = [&](int i, const Bid& b) {
        const long long w2 = N == 1 ? b.w1 : b.w2;
        const long long a = S.p[b.j1] + (w2 - b.w1) + eps;
        S.obj[i] = b.j1;
        S.amt[i] = a;
        atomicMax(&S.best[b.j1], a);
        if (i < n) ++real_bids;
      };
      if (U >= W || N < 2048) {
        // one warp per bidder
        for (int x = wid; x < U; x += W) {
          const int i = S.list[x];
          const Bid b = scan(i, lane, 32);
          if (lane == 0) place_bid(i, b);
        }
      } else {
        // fewer bidders than warps (the late rounds) on long rows: G warps
        // per bidder split its row, and one thread merges their partial bids
        // (the merge is associative, so the bid is the same as one warp's)
        int G = 1;
        while (2 * G * U <= W) G *= 2;
        const int x = wid / G, gw = wid % G;
        if (x < U) {
          const Bid b = scan(S.list[x], 32 * gw + lane, 32 * G);
          if (lane == 0) S.part[wid] = b;
        }
        __syncthreads();
        if (tid < U) {
          Bid b = S.part[tid * G];
          for (int q = 1; q < G; ++q) b = merge(b, S.part[tid * G + q]);
          place_bid(S.list[tid], b);
        }
      }
      __syncthreads();
      for (int x = tid; x < U; x += T) {
        const int i = S.list[x];
        if (S.amt[i] == S.best[S.obj[i]]) atomicMin(&S.winner[S.obj[i]], i);
      }
      __syncthreads();
      // winners take their objects at their bids; previous holders bid next round
      for (int x = tid; x < U; x += T) {
        const int i = S.list[x];
        const int j = S.obj[i];
        if (S.winner[j] == i) {
          S.p[j] = S.amt[i];
          const int old = S.holder[j];
          if (old >= 0) S.held[old] = -1;
          S.holder[j] = i;
          S.held[i] = j;
        }
      }
      __syncthreads();
      for (int x = tid; x < U; x += T) {
        const int j = S.obj[S.list[x]];
        S.best[j] = LLONG_MIN;
        S.winner[j] = INT_MAX;
      }
      // the next round's list build synchronises before these are read
    }
    if (eps == 1) break;
    eps /= 4;
    if (eps < 1) eps = 1;
    __syncthreads();
  }
  __syncthreads();

  // results
  long long part = 0;
  for (int i = tid; i < n; i += T) {
    const int j = S.held[i];
    I.row_to_col[i] = status == kDevOk ? j : -1;
    if (status == kDevOk) part += __ldg(I.C + i * ldc + j);
  }
  if (I.u)
    for (int i = tid; i < n; i += T) I.u[i] = 0;
  if (I.v)
    for (int j = tid; j < N; j += T) I.v[j] = 0;
  // real_bids was counted by the threads that placed bids
  const long long rb = block_sum<T>(real_bids, S.red);
  const long long cost = block_sum<T>(part, S.red);
  if (tid == 0) {
    *I.cost = cost;
    if (I.stats) {
      I.stats[0] = rounds;
      I.stats[1] = bids;
      I.stats[2] = 4LL * N * rb;
      I.stats[3] = stages;
      I.stats[4] = 0;
      I.stats[5] = 4LL * n * N;
      I.stats[6] = 0;
      I.stats[7] = 4LL * N * rb;
    }
  }
  __threadfence_system();
  __syncthreads();
  if (tid == 0 && I.status) *reinterpret_cast<volatile int32_t*>(I.status) = status;
  __syncthreads();
}

template <int T>
__device__ __forceinline__ void auction_loop(const Instance* __restrict__ insts, const int32_t* __restrict__ order,
                                             int num, int* work, int mmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const AuctionSmem S = carve_auction(smem_raw, mmax);
  for (;;) {
    if (threadIdx.x == 0) S.misc[1] = atomicAdd(work, 1);
    __syncthreads();
    const int idx = S.misc[1];
    __syncthreads();
    if (idx >= num) break;
    const Instance I = insts[order ? order[idx] : idx];
    auction_instance<T>(I, S);
  }
}

// Register budgets (measured): below 512 threads the compiler's choice for
// the block size alone (several CTAs per SM for small instances); at 512 a
// one-CTA-per-SM budget (the prices and bids of m = 4096 fill the shared
// memory anyway), which avoids spills in the bid scan.
template <int T>
__global__ void __launch_bounds__(T) auction_kernel(const Instance* __restrict__ insts,
                                                    const int32_t* __restrict__ order, int num, int* work,
                                                    int mmax) {
  auction_loop<T>(insts, order, num, work, mmax);
}

__global__ void __launch_bounds__(512, 1) auction_kernel_wide(const Instance* __restrict__ insts,
                                                              const int32_t* __restrict__ order, int num,
                                                              int* work, int mmax) {
  auction_loop<512>(insts, order, num, work, mmax);
}

template <int T>
cudaError_t launch_auction_t(const Instance* insts, const int32_t* order, int num, int* work, int mmax,
                             cudaStream_t stream) {
  void (*kern)(const Instance*, const int32_t*, int, int*, int) = nullptr;
  if constexpr (T >= 512)
    kern = auction_kernel_wide;
  else
    kern = auction_kernel<T>;
  const size_t smem = auction_bytes(mmax);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long cap = (long long)per_sm * sms;
  const int grid = int(num < cap ? num : cap);
  if (grid < 1) return cudaSuccess;
  kern<<<grid, T, smem, stream>>>(insts, order, num, work, mmax);
  return cudaGetLastError();
}

}  // namespace

int auction_threads(int m) {
  if (m <= 64) return 32;
  if (m <= 128) return 64;
  if (m <= 256) return 128;
  if (m <= 1024) return 256;
  return 512;
}

size_t auction_smem_bytes(int mmax) { return auction_bytes(mmax); }

cudaError_t launch_auction(int threads, const Instance* insts, const int32_t* order, int num, int* work,
                           int mmax, cudaStream_t stream) {
  switch (threads) {
    case 32: return launch_auction_t<32>(insts, order, num, work, mmax, stream);
    case 64: return launch_auction_t<64>(insts, order, num, work, mmax, stream);
    case 128: return launch_auction_t<128>(insts, order, num, work, mmax, stream);
    case 256: return launch_auction_t<256>(insts, order, num, work, mmax, stream);
    case 512: return launch_auction_t<512>(insts, order, num, work, mmax, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ot
