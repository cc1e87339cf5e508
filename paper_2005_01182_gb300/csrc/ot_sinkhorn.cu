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
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "otassign.h"
#include "ot_ctx.h"

namespace ot {
namespace {

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

__device__ __forceinline__ void lse_add(Lse& a, float x, float c) {
  if (x > a.m) {
    const float sc = __expf(a.m - x);  // 0 when a.m = -inf
    a.s = a.s * sc + 1.0f;
    a.w = a.w * sc + c;
    a.m = x;
  } else {
    const float e = __expf(x - a.m);
    a.s += e;
    a.w += c * e;
  }
}

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

// Row pass of iteration k: f_new = log r - LSE_j(g - eta C); with `check`,
// also the residue and cost of the iterate (f_old, g) into acc[k & 1].
template <bool VEC>
__global__ void __launch_bounds__(256) sk_row_pass(const int32_t* __restrict__ C, long long ldc, int n, int m,
                                                   float eta, const float* __restrict__ g,
                                                   const float* __restrict__ f_old, float* __restrict__ f_new,
                                                   const float* __restrict__ logr, const double* __restrict__ r,
                                                   SkState* st, int k, int check) {
  if (*reinterpret_cast<volatile int*>(&st->done)) return;
  __shared__ double red[2][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int warps = gridDim.x * 8;
  double res = 0.0, cost = 0.0;
  for (int i = blockIdx.x * 8 + wid; i < n; i += warps) {
    const int32_t* row = C + (long long)i * ldc;
    Lse a{-INFINITY, 0.0f, 0.0f};
    if (VEC) {
      const int4* row4 = reinterpret_cast<const int4*>(row);
      const float4* g4 = reinterpret_cast<const float4*>(g);
#pragma unroll 2
      for (int q = lane; q < (m >> 2); q += 32) {
        const int4 c = __ldg(row4 + q);
        const float4 gv = __ldg(g4 + q);
        lse_add(a, fmaf(-eta, float(c.x), gv.x), float(c.x));
        lse_add(a, fmaf(-eta, float(c.y), gv.y), float(c.y));
        lse_add(a, fmaf(-eta, float(c.z), gv.z), float(c.z));
        lse_add(a, fmaf(-eta, float(c.w), gv.w), float(c.w));
      }
      for (int j = (m & ~3) + lane; j < m; j += 32) {
        const float c = float(row[j]);
        lse_add(a, fmaf(-eta, c, __ldg(g + j)), c);
      }
    } else {
      for (int j = lane; j < m; j += 32) {
        const float c = float(__ldg(row + j));
        lse_add(a, fmaf(-eta, c, __ldg(g + j)), c);
      }
    }
    a = warp_lse(a);
    const float L = a.m + logf(a.s);
    if (lane == 0) {
      f_new[i] = (logr ? logr[i] : 0.0f) - L;
      if (check) {
        const double fo = double(f_old[i]);
        res += fabs((r ? r[i] : 1.0) - exp(fo + double(L)));
        cost += exp(fo + double(a.m)) * double(a.w);
      }
    }
  }
  if (!check) return;
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
// LSEs over this CTA's rows; the last CTA of a column tile merges them into g.
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
    if (VEC && j0 + 3 < m) {
#pragma unroll 4
      for (int i = i0; i < i1; ++i) {
        const int4 c = __ldg(reinterpret_cast<const int4*>(C + (long long)i * ldc + j0));
        const float fi = __ldg(f + i);
        lse_add(a[0], fmaf(-eta, float(c.x), fi), 0.0f);
        lse_add(a[1], fmaf(-eta, float(c.y), fi), 0.0f);
        lse_add(a[2], fmaf(-eta, float(c.z), fi), 0.0f);
        lse_add(a[3], fmaf(-eta, float(c.w), fi), 0.0f);
      }
    } else {
      for (int i = i0; i < i1; ++i) {
        const int32_t* row = C + (long long)i * ldc;
        const float fi = __ldg(f + i);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (j0 + q < m) lse_add(a[q], fmaf(-eta, float(__ldg(row + j0 + q)), fi), 0.0f);
      }
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
  for (int q = 0; q < 4; ++q) {
    const int j = j0 + q;
    if (j >= m) continue;
    Lse s{-INFINITY, 0.0f, 0.0f};
    // eight partials in flight per round: the merge is bound by L2 latency
    for (int b0 = 0; b0 < nrb; b0 += 8) {
      float2 p[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        p[u] = b0 + u < nrb ? __ldcg(part + (long long)(b0 + u) * m + j) : make_float2(-INFINITY, 0.0f);
#pragma unroll
      for (int u = 0; u < 8; ++u) s = lse_merge(s, Lse{p[u].x, p[u].y, 0.0f});
    }
    g[j] = (logc ? logc[j] : 0.0f) - (s.m + logf(s.s));
  }
  if (threadIdx.x == 0) tile_count[blockIdx.x] = 0;
}

constexpr int kColT = 128;

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

  // column pass geometry: tiles of 4*T columns, enough row blocks to fill
  // the GPU, but at least 64 rows per block (the merge of the partials is
  // latency-bound in their number)
  const int tiles = (m + 4 * kColT - 1) / (4 * kColT);
  int nrb = std::max(1, std::min((n + 63) / 64, (4 * sms + tiles - 1) / tiles));
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
  const int row_grid = std::max(1, std::min((n + 7) / 8, 8 * sms));
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
