// Log-domain Sinkhorn (Sec. 2.2 "Matrix Scaling", Sec. 2.2.1 "Sinkhorn",
// Sec. 4.1 "Sinkhorn"): entropic OT min <X, C> - h(X)/eta over X 1 = r,
// X^T 1 = c, whose solution is X_ij = exp(f_i + g_j - eta C_ij).  One
// iteration scales every row (f_i = log r_i - LSE_j(g_j - eta C_ij)) and then
// every column (g_j = log c_j - LSE_i(f_i - eta C_ij)); the first iterate
// whose residue sum_i |r_i - (X 1)_i| (the columns are exact after their
// scaling) is at most eps * sum(r) is returned, unrounded.
//
// Each half-iteration is one streaming pass over the int32 cost matrix, the
// HBM-bound scan of the method:
//   * row pass: one warp per row, 16-byte loads, an online (max, sum)
//     log-sum-exp per lane merged by shuffles; the same pass also yields the
//     row sums and <C, X> of the previous iterate (both need exactly the
//     row's LSE against the current g), so convergence costs no extra pass;
//   * column pass: a CTA owns a tile of 4 x T columns and a block of rows,
//     keeps an online (max, sum) per column in registers while it walks its
//     rows (coalesced 16-byte loads along each row), writes one partial per
//     column, and the last CTA to finish a tile merges the partials of all
//     row blocks into g.
// Arithmetic: float32 for the exponent arguments, exponentials (__expf on
// arguments <= 0, where it is accurate to a few ulp) and sums; double for the
// residue and cost accumulators.  The iteration runs until a device flag is
// set; kernels issued after it return at once, so the host checks the flag
// only every few iterations.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "otassign.h"
#include "ot_ctx.h"

// Launch shape of the two passes (compile-time; the defaults are the ones
// measured best on GB300 for n = m = 16384).
#ifndef OT_SK_ROW_MINB
#define OT_SK_ROW_MINB 1
#endif
#ifndef OT_SK_COL_T
#define OT_SK_COL_T 128
#endif
#ifndef OT_SK_COL_CTAS
#define OT_SK_COL_CTAS 8
#endif
#ifndef OT_SK_COL_UNROLL
#define OT_SK_COL_UNROLL 8
#endif

namespace ot {
namespace {

constexpr int kColUnroll = OT_SK_COL_UNROLL;

struct SkState {
  int done;        // set when the returned iterate is final
  int iterations;  // of the returned iterate
  int final_buf;   // f buffer holding it
  int pad;
  double residue;  // sum_i |r_i - (X 1)_i| of the returned iterate
  double cost;     // <C, X> of the returned iterate
  double acc[2][2];  // per-iteration-parity accumulators: residue, cost
};

struct Lse {
  float m;  // running maximum
  float s;  // sum of exp(x - m)
  float w;  // sum of C * exp(x - m) (row pass only)
};

__device__ __forceinline__ Lse lse_merge(Lse a, Lse b) {
  if (b.s == 0.0f) return a;
  if (a.s == 0.0f) return b;
  if (b.m > a.m) {
    const Lse t = a;
    a = b;
    b = t;
  }
  const float sc = __expf(b.m - a.m);
  a.s += b.s * sc;
  a.w += b.w * sc;
  return a;
}

__device__ __forceinline__ Lse warp_lse(Lse a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Lse b;
    b.m = __shfl_xor_sync(0xffffffffu, a.m, o);
    b.s = __shfl_xor_sync(0xffffffffu, a.s, o);
    b.w = __shfl_xor_sync(0xffffffffu, a.w, o);
    a = lse_merge(a, b);
  }
  return a;
}

// Fold N values held in registers into a running log-sum-exp: one maximum
// over the chunk, one rescale of the running sums, then N independent
// exponentials (no data-dependent branch; -inf entries contribute 0).  The
// chunk must hold at least one finite value.
template <int N, bool W>
__device__ __forceinline__ void lse_chunk(Lse& a, const float (&x)[N], const float (&c)[N]) {
  float cm = x[0];
#pragma unroll
  for (int k = 1; k < N; ++k) cm = fmaxf(cm, x[k]);
  const float mn = fmaxf(a.m, cm);
  const float sc = __expf(a.m - mn);  // 0 when a.m = -inf
  float s0 = 0.0f, s1 = 0.0f, w0 = 0.0f, w1 = 0.0f;
#pragma unroll
  for (int k = 0; k < N; k += 2) {
    const float e0 = __expf(x[k] - mn);
    s0 += e0;
    if (W) w0 = fmaf(c[k], e0, w0);
    if (k + 1 < N) {
      const float e1 = __expf(x[k + 1] - mn);
      s1 += e1;
      if (W) w1 = fmaf(c[k + 1], e1, w1);
    }
  }
  a.s = fmaf(a.s, sc, s0 + s1);
  if (W) a.w = fmaf(a.w, sc, w0 + w1);
  a.m = mn;
}

// Row pass of iteration k: f_new = log r - LSE_j(g - eta C); with `check`,
// also the residue and cost of the iterate (f_old, g) into acc[k & 1].  A
// warp takes two adjacent rows (they share the loads of g); each lane keeps
// kRowChunk 16-byte loads of both rows in flight before it folds them.
constexpr int kRowChunk = 4;

template <bool VEC>
__global__ void __launch_bounds__(256, OT_SK_ROW_MINB) sk_row_pass(const int32_t* __restrict__ C, long long ldc, int n, int m,
                                                   float eta, const float* __restrict__ g,
                                                   const float* __restrict__ f_old, float* __restrict__ f_new,
                                                   const float* __restrict__ logr, const double* __restrict__ r,
                                                   SkState* st, int k, int check) {
  if (*reinterpret_cast<volatile int*>(&st->done)) return;
  __shared__ double red[2][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int warps = gridDim.x * 8;
  double res = 0.0, cost = 0.0;
  for (int i = 2 * (blockIdx.x * 8 + wid); i < n; i += 2 * warps) {
    const bool two = i + 1 < n;
    const int32_t* row0 = C + (long long)i * ldc;
    const int32_t* row1 = two ? row0 + ldc : row0;
    Lse a0{-INFINITY, 0.0f, 0.0f}, a1{-INFINITY, 0.0f, 0.0f};
    if (VEC) {
      const int nq = m >> 2;
      const int4* r0 = reinterpret_cast<const int4*>(row0);
      const int4* r1 = reinterpret_cast<const int4*>(row1);
      const float4* g4 = reinterpret_cast<const float4*>(g);
      for (int q0 = lane; q0 < nq; q0 += 32 * kRowChunk) {
        int4 c0[kRowChunk], c1[kRowChunk];
        float4 gv[kRowChunk];
#pragma unroll
        for (int u = 0; u < kRowChunk; ++u) {
          const int q = q0 + 32 * u;
          if (q < nq) {
            c0[u] = __ldg(r0 + q);
            c1[u] = __ldg(r1 + q);
            gv[u] = __ldg(g4 + q);
          } else {
            c0[u] = c1[u] = make_int4(0, 0, 0, 0);
            gv[u] = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
          }
        }
        float x[4 * kRowChunk], cf[4 * kRowChunk];
#pragma unroll
        for (int u = 0; u < kRowChunk; ++u) {
          cf[4 * u + 0] = float(c0[u].x); cf[4 * u + 1] = float(c0[u].y);
          cf[4 * u + 2] = float(c0[u].z); cf[4 * u + 3] = float(c0[u].w);
          x[4 * u + 0] = fmaf(-eta, cf[4 * u + 0], gv[u].x); x[4 * u + 1] = fmaf(-eta, cf[4 * u + 1], gv[u].y);
          x[4 * u + 2] = fmaf(-eta, cf[4 * u + 2], gv[u].z); x[4 * u + 3] = fmaf(-eta, cf[4 * u + 3], gv[u].w);
        }
        lse_chunk<4 * kRowChunk, true>(a0, x, cf);
#pragma unroll
        for (int u = 0; u < kRowChunk; ++u) {
          cf[4 * u + 0] = float(c1[u].x); cf[4 * u + 1] = float(c1[u].y);
          cf[4 * u + 2] = float(c1[u].z); cf[4 * u + 3] = float(c1[u].w);
          x[4 * u + 0] = fmaf(-eta, cf[4 * u + 0], gv[u].x); x[4 * u + 1] = fmaf(-eta, cf[4 * u + 1], gv[u].y);
          x[4 * u + 2] = fmaf(-eta, cf[4 * u + 2], gv[u].z); x[4 * u + 3] = fmaf(-eta, cf[4 * u + 3], gv[u].w);
        }
        lse_chunk<4 * kRowChunk, true>(a1, x, cf);
      }
      for (int j = (m & ~3) + lane; j < m; j += 32) {
        const float gj = __ldg(g + j);
        float x0[1], x1[1], cc0[1], cc1[1];
        cc0[0] = float(row0[j]);
        cc1[0] = float(row1[j]);
        x0[0] = fmaf(-eta, cc0[0], gj);
        x1[0] = fmaf(-eta, cc1[0], gj);
        lse_chunk<1, true>(a0, x0, cc0);
        lse_chunk<1, true>(a1, x1, cc1);
      }
    } else {
      for (int j = lane; j < m; j += 32) {
        const float gj = __ldg(g + j);
        float x0[1], x1[1], cc0[1], cc1[1];
        cc0[0] = float(__ldg(row0 + j));
        cc1[0] = float(__ldg(row1 + j));
        x0[0] = fmaf(-eta, cc0[0], gj);
        x1[0] = fmaf(-eta, cc1[0], gj);
        lse_chunk<1, true>(a0, x0, cc0);
        lse_chunk<1, true>(a1, x1, cc1);
      }
    }
    a0 = warp_lse(a0);
    a1 = warp_lse(a1);
    if (lane < 2 && (lane == 0 || two)) {
      const int ii = i + lane;
      const Lse& a = lane == 0 ? a0 : a1;
      const float L = a.m + logf(a.s);
      f_new[ii] = (logr ? logr[ii] : 0.0f) - L;
      if (check) {
        const double fo = double(f_old[ii]);
        res += fabs((r ? r[ii] : 1.0) - exp(fo + double(L)));
        cost += exp(fo + double(a.m)) * double(a.w);
      }
    }
  }
  if (!check) return;
  res += __shfl_down_sync(0xffffffffu, res, 1);
  cost += __shfl_down_sync(0xffffffffu, cost, 1);
  if (lane == 0) {
    red[0][wid] = res;
    red[1][wid] = cost;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < 8; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    atomicAdd(&st->acc[k & 1][0], s0);
    atomicAdd(&st->acc[k & 1][1], s1);
  }
}

// Column pass of iteration k.  First the convergence test of iterate k-1
// (whose residue the row pass of iteration k accumulated): when it passes, or
// when `final_k` > 0 asks for iterate final_k to be returned as it is, the
// state is recorded and nothing else happens.  Otherwise partial column
// LSEs over this CTA's rows, kColChunk rows of 16-byte loads in flight per
// thread; the last CTA of a column tile merges the partials into g.
constexpr int kColChunk = kColUnroll;

template <int T, bool VEC>
__global__ void __launch_bounds__(T) sk_col_pass(const int32_t* __restrict__ C, long long ldc, int n, int m,
                                                 float eta, const float* __restrict__ f, float* __restrict__ g,
                                                 const float* __restrict__ logc, float2* __restrict__ part,
                                                 int* __restrict__ tile_count, int rows_per_block, SkState* st,
                                                 int k, int check, double threshold, int final_k) {
  if (*reinterpret_cast<volatile int*>(&st->done)) return;
  const double res = st->acc[k & 1][0];
  if ((check && res <= threshold) || final_k > 0) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
      st->iterations = k - 1;
      st->final_buf = (k - 1) & 1;
      st->residue = res;
      st->cost = st->acc[k & 1][1];
      __threadfence();
      st->done = 1;
    }
    return;
  }
  // the next row pass accumulates into the other parity
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < 2) st->acc[(k + 1) & 1][threadIdx.x] = 0.0;

  const int nrb = gridDim.y;
  const int j0 = (blockIdx.x * T + threadIdx.x) * 4;
  const int i0 = blockIdx.y * rows_per_block;
  const int i1 = min(n, i0 + rows_per_block);
  Lse a[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) a[q] = Lse{-INFINITY, 0.0f, 0.0f};
  if (j0 < m) {
    const bool full = VEC && j0 + 3 < m;
    for (int ib = i0; ib < i1; ib += kColChunk) {
      // rows past the block end are loaded from the last row (a valid
      // address, no branch around the loads) and weighted out by f = -inf
      int4 c[kColChunk];
      float fi[kColChunk];
      if (full) {
#pragma unroll
        for (int u = 0; u < kColChunk; ++u)
          c[u] = __ldg(reinterpret_cast<const int4*>(C + (long long)min(ib + u, i1 - 1) * ldc + j0));
      } else {
#pragma unroll
        for (int u = 0; u < kColChunk; ++u) {
          const int32_t* p = C + (long long)min(ib + u, i1 - 1) * ldc + j0;
          c[u].x = __ldg(p);
          c[u].y = j0 + 1 < m ? __ldg(p + 1) : 0;
          c[u].z = j0 + 2 < m ? __ldg(p + 2) : 0;
          c[u].w = j0 + 3 < m ? __ldg(p + 3) : 0;
        }
      }
#pragma unroll
      for (int u = 0; u < kColChunk; ++u) fi[u] = ib + u < i1 ? __ldg(f + ib + u) : -INFINITY;
      float x[kColChunk], cz[kColChunk];
#pragma unroll
      for (int u = 0; u < kColChunk; ++u) { x[u] = fmaf(-eta, float(c[u].x), fi[u]); cz[u] = 0.0f; }
      lse_chunk<kColChunk, false>(a[0], x, cz);
#pragma unroll
      for (int u = 0; u < kColChunk; ++u) x[u] = fmaf(-eta, float(c[u].y), fi[u]);
      lse_chunk<kColChunk, false>(a[1], x, cz);
#pragma unroll
      for (int u = 0; u < kColChunk; ++u) x[u] = fmaf(-eta, float(c[u].z), fi[u]);
      lse_chunk<kColChunk, false>(a[2], x, cz);
#pragma unroll
      for (int u = 0; u < kColChunk; ++u) x[u] = fmaf(-eta, float(c[u].w), fi[u]);
      lse_chunk<kColChunk, false>(a[3], x, cz);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (j0 + q < m) part[(long long)blockIdx.y * m + j0 + q] = make_float2(a[q].m, a[q].s);
  }
  // last CTA of this column tile merges the row blocks
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&tile_count[blockIdx.x], 1) == nrb - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the merge is bound by L2 latency: 4 partials of each of the thread's 4
  // columns in flight per round
  Lse s[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) s[q] = Lse{-INFINITY, 0.0f, 0.0f};
  if (j0 < m) {
    for (int b0 = 0; b0 < nrb; b0 += 4) {
      float2 p[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          p[u][q] = (b0 + u < nrb && j0 + q < m) ? __ldcg(part + (long long)(b0 + u) * m + j0 + q)
                                                 : make_float2(-INFINITY, 0.0f);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) s[q] = lse_merge(s[q], Lse{p[u][q].x, p[u][q].y, 0.0f});
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (j0 + q < m) g[j0 + q] = (logc ? logc[j0 + q] : 0.0f) - (s[q].m + logf(s[q].s));
  }
  if (threadIdx.x == 0) tile_count[blockIdx.x] = 0;
}

constexpr int kColT = OT_SK_COL_T;

// ---------------------------------------------------------------------------
// Many small instances: one CTA iterates one instance to convergence (rows
// and columns of up to kBatchMaxN / kBatchMaxM), the CTAs pulling instances
// from a work counter, largest first.  Unit marginals (r = 1, c = n/m).
// Same iteration, stopping rule and float32 arithmetic as above; f (two
// buffers: the previous iterate is kept until its residue is known) and g
// live in shared memory, rows are read from global memory (L2).
// ---------------------------------------------------------------------------
constexpr int kBatchT = 128;
constexpr int kBatchMaxN = 4096, kBatchMaxM = 4096;

struct SkInstance {
  const int32_t* C;
  long long ldc;
  int n, m;
  float* f;           // [n] output
  float* g;           // [m] output
  double* cost;       // output
  double* residue;    // output
  int* iterations;    // output
};

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kBatchT / 32; ++w) t += red[w];
  return t;
}

__global__ void __launch_bounds__(kBatchT) sk_batch_kernel(const SkInstance* __restrict__ insts,
                                                           const int32_t* __restrict__ order, int num, int* work,
                                                           float eta, double eps_rel, int max_iter,
                                                           int nmax) {
  // f (two iterates) and g in dynamic shared memory sized for the batch
  extern __shared__ float sk_smem[];
  float* const gs = sk_smem + 2 * nmax;
  __shared__ double red[2][kBatchT / 32];
  __shared__ int sidx;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int W = kBatchT / 32;
  for (;;) {
    if (tid == 0) sidx = atomicAdd(work, 1);
    __syncthreads();
    const int idx = sidx;
    __syncthreads();
    if (idx >= num) break;
    const SkInstance I = insts[order[idx]];
    const int n = I.n, m = I.m;
    const float logc = logf(float(n) / float(m));
    for (int i = tid; i < n; i += kBatchT) sk_smem[i] = 0.0f;
    for (int j = tid; j < m; j += kBatchT) gs[j] = 0.0f;
    __syncthreads();
    const double threshold = eps_rel > 0.0 ? eps_rel * n : -1.0;
    int final_k = 0;
    double res = 0.0, cost = 0.0;
    for (int k = 1; k <= max_iter + 1; ++k) {
      const float* f_old = sk_smem + ((k - 1) & 1) * nmax;
      float* f_new = sk_smem + (k & 1) * nmax;
      // row pass: f_new = -LSE_j(g - eta C); residue / cost of (f_old, g)
      double pres = 0.0, pcost = 0.0;
      for (int i = wid; i < n; i += W) {
        const int32_t* row = I.C + (long long)i * I.ldc;
        Lse a{-INFINITY, 0.0f, 0.0f};
        for (int j0 = lane; j0 < m; j0 += 32 * 4) {
          float x[4], c[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = j0 + 32 * u;
            c[u] = j < m ? float(__ldg(row + j)) : 0.0f;
            x[u] = j < m ? fmaf(-eta, c[u], gs[j]) : -INFINITY;
          }
          lse_chunk<4, true>(a, x, c);
        }
        a = warp_lse(a);
        const float L = a.m + logf(a.s);
        if (lane == 0) {
          f_new[i] = -L;
          const double fo = double(f_old[i]);
          pres += fabs(1.0 - exp(fo + double(L)));
          pcost += exp(fo + double(a.m)) * double(a.w);
        }
      }
      res = block_sum_d(pres, red[0]);
      cost = block_sum_d(pcost, red[1]);
      // iterate k - 1 is returned when it meets the threshold, or when it
      // is the last one asked for
      if ((k >= 2 && threshold >= 0.0 && res <= threshold) || k == max_iter + 1) {
        final_k = k - 1;
        break;
      }
      __syncthreads();
      // column pass: g_j = log(n/m) - LSE_i(f_new - eta C), one thread per column
      for (int j = tid; j < m; j += kBatchT) {
        Lse a{-INFINITY, 0.0f, 0.0f};
        for (int i0 = 0; i0 < n; i0 += 4) {
          float x[4], cz[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = i0 + u;
            x[u] = i < n ? fmaf(-eta, float(__ldg(I.C + (long long)i * I.ldc + j)), f_new[i]) : -INFINITY;
            cz[u] = 0.0f;
          }
          lse_chunk<4, false>(a, x, cz);
        }
        gs[j] = logc - (a.m + logf(a.s));
      }
      __syncthreads();
    }
    __syncthreads();
    const float* ff = sk_smem + (final_k & 1) * nmax;
    for (int i = tid; i < n; i += kBatchT) I.f[i] = ff[i];
    for (int j = tid; j < m; j += kBatchT) I.g[j] = gs[j];
    if (tid == 0) {
      *I.cost = cost;
      *I.residue = res;
      *I.iterations = final_k;
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace ot

using namespace ot;

extern "C" int ot_sinkhorn_solve(ot_ctx* ctx, const int32_t* C, int64_t ldc, int32_t n, int32_t m,
                                 const double* r, const double* c, double eta, double eps_rel,
                                 int32_t max_iter, float* f, float* g, double* cost, double* residue,
                                 int32_t* iterations, void* stream) {
  if (!ctx) return OT_ERR_ARG;
  if (n <= 0 || m <= 0 || !C || ldc < m || !(eta > 0.0) || !std::isfinite(eta) || max_iter < 1 || !cost)
    return ctx_fail(ctx, OT_ERR_ARG, "bad arguments");
  cudaSetDevice(ctx->device);
  if (!ptr_on_device(C)) return ctx_fail(ctx, OT_ERR_ARG, "the cost matrix must be a device pointer");
  // marginals: validate, logs, total
  std::vector<double> hr(n), hc(m);
  std::vector<float> lr(n), lc(m);
  double tr = 0.0, tc = 0.0;
  for (int i = 0; i < n; ++i) {
    hr[i] = r ? r[i] : 1.0;
    if (!(hr[i] > 0.0) || !std::isfinite(hr[i])) return ctx_fail(ctx, OT_ERR_ARG, "supplies must be positive");
    lr[i] = float(std::log(hr[i]));
    tr += hr[i];
  }
  for (int j = 0; j < m; ++j) {
    hc[j] = c ? c[j] : double(n) / double(m);
    if (!(hc[j] > 0.0) || !std::isfinite(hc[j])) return ctx_fail(ctx, OT_ERR_ARG, "demands must be positive");
    lc[j] = float(std::log(hc[j]));
    tc += hc[j];
  }
  if (std::fabs(tr - tc) > 1e-9 * std::max(tr, tc)) return ctx_fail(ctx, OT_ERR_ARG, "total supply != total demand");

  std::lock_guard<std::mutex> lock(ctx->scaled_mu);
  StreamScope scope(static_cast<cudaStream_t>(stream), ctx->stream, ctx->sjoin_in_ev, ctx->sjoin_out_ev);
  cudaStream_t s = scope.work;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

  // column pass geometry: tiles of 4*T columns and enough row blocks for
  // OT_SK_COL_CTAS CTAs per SM (loads in flight), but at least 64 rows per block (the
  // merge of the partials is latency-bound in their number)
  const int tiles = (m + 4 * kColT - 1) / (4 * kColT);
  int nrb = std::max(1, std::min((n + 63) / 64, (OT_SK_COL_CTAS * sms + tiles - 1) / tiles));
  const int rows_per_block = (n + nrb - 1) / nrb;
  nrb = (n + rows_per_block - 1) / rows_per_block;

  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  const size_t o_st = off; off += al(sizeof(SkState));
  const size_t o_f0 = off; off += al(4 * size_t(n));
  const size_t o_f1 = off; off += al(4 * size_t(n));
  const size_t o_g = off; off += al(4 * size_t(m));
  const size_t o_lr = off; off += al(4 * size_t(n));
  const size_t o_lc = off; off += al(4 * size_t(m));
  const size_t o_r = off; off += al(8 * size_t(n));
  const size_t o_tc = off; off += al(4 * size_t(tiles));
  const size_t o_part = off; off += al(sizeof(float2) * size_t(nrb) * m);
  if (int rc = ctx->d_scaled.reserve(off); rc) return ctx_fail(ctx, rc, "sinkhorn workspace");
  char* B = static_cast<char*>(ctx->d_scaled.ptr);
  SkState* dst = reinterpret_cast<SkState*>(B + o_st);
  float* fb[2] = {reinterpret_cast<float*>(B + o_f0), reinterpret_cast<float*>(B + o_f1)};
  float* dg = reinterpret_cast<float*>(B + o_g);
  float* dlr = reinterpret_cast<float*>(B + o_lr);
  float* dlc = reinterpret_cast<float*>(B + o_lc);
  double* drr = reinterpret_cast<double*>(B + o_r);
  int* dtc = reinterpret_cast<int*>(B + o_tc);
  float2* dpart = reinterpret_cast<float2*>(B + o_part);
  cudaError_t e = cudaMemsetAsync(B, 0, o_lr, s);  // state, f buffers, g
  if (e == cudaSuccess) e = cudaMemsetAsync(dtc, 0, 4 * size_t(tiles), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dlr, lr.data(), 4 * size_t(n), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dlc, lc.data(), 4 * size_t(m), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(drr, hr.data(), 8 * size_t(n), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "sinkhorn setup");

  const bool vec = (ldc % 4 == 0) && (reinterpret_cast<uintptr_t>(C) % 16 == 0);
  const double threshold = eps_rel > 0.0 ? eps_rel * tr : -1.0;
  const int row_grid = std::max(1, std::min((n + 15) / 16, 8 * sms));
  const dim3 col_grid(tiles, nrb);
  // host copy of the state, polled every `chunk` iterations
  SkState h{};
  auto launch_iter = [&](int k, int check, int final_k) -> cudaError_t {
    const float* f_old = fb[(k - 1) & 1];
    float* f_new = fb[k & 1];
    if (vec)
      sk_row_pass<true><<<row_grid, 256, 0, s>>>(C, ldc, n, m, float(eta), dg, f_old, f_new, dlr, drr, dst, k,
                                                 check);
    else
      sk_row_pass<false><<<row_grid, 256, 0, s>>>(C, ldc, n, m, float(eta), dg, f_old, f_new, dlr, drr, dst, k,
                                                  check);
    if (vec)
      sk_col_pass<kColT, true><<<col_grid, kColT, 0, s>>>(C, ldc, n, m, float(eta), f_new, dg, dlc, dpart, dtc,
                                                          rows_per_block, dst, k, check, threshold, final_k);
    else
      sk_col_pass<kColT, false><<<col_grid, kColT, 0, s>>>(C, ldc, n, m, float(eta), f_new, dg, dlc, dpart, dtc,
                                                           rows_per_block, dst, k, check, threshold, final_k);
    return cudaGetLastError();
  };
  const int chunk = 8;
  bool done = false;
  for (int k = 1; k <= max_iter && !done; ++k) {
    // iteration k checks iterate k - 1 (iterate 0 is the starting point)
    if ((e = launch_iter(k, k >= 2 && threshold >= 0.0, 0)) != cudaSuccess) return ctx_cuda(ctx, e, "sinkhorn");
    if (k % chunk == 0 || k == max_iter) {
      if ((e = cudaMemcpyAsync(&h, dst, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return ctx_cuda(ctx, e, "sinkhorn poll");
      done = h.done != 0;
    }
  }
  if (!done) {
    // iterate max_iter is returned: one more row pass measures it, the
    // column pass records it (unless it converged in the meantime)
    if ((e = launch_iter(max_iter + 1, 1, max_iter + 1)) != cudaSuccess) return ctx_cuda(ctx, e, "sinkhorn");
  }
  if ((e = cudaMemcpyAsync(&h, dst, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return ctx_cuda(ctx, e, "sinkhorn result");
  if (!h.done) return ctx_fail(ctx, OT_ERR_CUDA, "sinkhorn did not record a result");
  const float* ff = fb[h.final_buf];
  if (f) {
    e = cudaMemcpyAsync(f, ff, 4 * size_t(n), ptr_on_device(f) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "sinkhorn f");
  }
  if (g) {
    e = cudaMemcpyAsync(g, dg, 4 * size_t(m), ptr_on_device(g) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "sinkhorn g");
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return ctx_cuda(ctx, e, "sinkhorn sync");
  *cost = h.cost;
  if (residue) *residue = h.residue;
  if (iterations) *iterations = h.iterations;
  return OT_OK;
}

extern "C" int ot_sinkhorn_solve_batched(ot_ctx* ctx, int32_t k, const int32_t* const* C, const int64_t* ldc,
                                         const int32_t* n, const int32_t* m, double eta, double eps_rel,
                                         int32_t max_iter, float* const* f, float* const* g, double* cost,
                                         double* residue, int32_t* iterations, void* stream) {
  if (!ctx) return OT_ERR_ARG;
  if (k < 0 || !(eta > 0.0) || !std::isfinite(eta) || max_iter < 1) return ctx_fail(ctx, OT_ERR_ARG, "bad arguments");
  if (k == 0) return OT_OK;
  if (!C || !ldc || !n || !m || !f || !g || !cost || !residue || !iterations)
    return ctx_fail(ctx, OT_ERR_ARG, "null array");
  cudaSetDevice(ctx->device);
  std::vector<SkInstance> hi(k);
  std::vector<int32_t> ord(k);
  for (int t = 0; t < k; ++t) {
    if (n[t] < 1 || m[t] < 1 || n[t] > kBatchMaxN || m[t] > kBatchMaxM || !C[t] || ldc[t] < m[t] || !f[t] || !g[t])
      return ctx_fail(ctx, n[t] > kBatchMaxN || m[t] > kBatchMaxM ? OT_ERR_UNSUPPORTED : OT_ERR_ARG,
                      "bad instance " + std::to_string(t));
    hi[t] = SkInstance{C[t], ldc[t], n[t], m[t], f[t], g[t], cost + t, residue + t, iterations + t};
    ord[t] = t;
  }
  if (!ptr_on_device(C[0]) || !ptr_on_device(cost)) return ctx_fail(ctx, OT_ERR_ARG, "device pointers expected");
  std::sort(ord.begin(), ord.end(), [&](int a, int b) {
    const long long wa = (long long)n[a] * m[a], wb = (long long)n[b] * m[b];
    return wa != wb ? wa > wb : a < b;
  });
  std::lock_guard<std::mutex> lock(ctx->scaled_mu);
  StreamScope scope(static_cast<cudaStream_t>(stream), ctx->stream, ctx->sjoin_in_ev, ctx->sjoin_out_ev);
  cudaStream_t s = scope.work;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t b_inst = al(sizeof(SkInstance) * k), b_ord = al(4 * size_t(k));
  if (int rc = ctx->d_scaled.reserve(b_inst + b_ord + 256); rc) return ctx_fail(ctx, rc, "sinkhorn batch workspace");
  char* B = static_cast<char*>(ctx->d_scaled.ptr);
  // the pinned staging of the descriptors must outlive the asynchronous copy
  std::vector<char> hbuf(b_inst + b_ord + 256, 0);
  std::memcpy(hbuf.data(), hi.data(), sizeof(SkInstance) * k);
  std::memcpy(hbuf.data() + b_inst, ord.data(), 4 * size_t(k));
  cudaError_t e = cudaMemcpyAsync(B, hbuf.data(), b_inst + b_ord + 256, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // hbuf is pageable and local
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "sinkhorn batch setup");
  int* dwork = reinterpret_cast<int*>(B + b_inst + b_ord);
  if ((e = cudaMemsetAsync(dwork, 0, sizeof(int), s)) != cudaSuccess) return ctx_cuda(ctx, e, "sinkhorn batch");
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int nmax = 0, mmax = 0;
  for (int t = 0; t < k; ++t) {
    nmax = std::max(nmax, int(n[t]));
    mmax = std::max(mmax, int(m[t]));
  }
  const size_t smem = sizeof(float) * (2 * size_t(nmax) + size_t(mmax));
  if ((e = cudaFuncSetAttribute(sk_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) != cudaSuccess)
    return ctx_cuda(ctx, e, "sinkhorn batch smem");
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sk_batch_kernel, kBatchT, smem);
  const int grid = std::max(1, std::min(k, std::max(1, per_sm) * sms));
  sk_batch_kernel<<<grid, kBatchT, smem, s>>>(reinterpret_cast<const SkInstance*>(B),
                                              reinterpret_cast<const int32_t*>(B + b_inst), k, dwork, float(eta),
                                              eps_rel, max_iter, nmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "sinkhorn batch launch");
  return OT_OK;
}
