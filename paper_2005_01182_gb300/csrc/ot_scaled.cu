// Batched KM with a single scaling factor (the paper's approximate variant,
// Sec. 2.3 "Batched KM" and Table 3's 1.1-approximation): solve exactly on
// floor(C / s), report the assignment's cost under C, which lies within
// n (s - 1) of the optimum.
#include <cstring>
#include <vector>

#include "otassign.h"
#include "ot_ctx.h"

namespace ot {

// floor division (rounds toward minus infinity for negative costs)
__device__ __forceinline__ int32_t floor_div(int32_t c, int32_t s) {
  return c >= 0 ? c / s : -((-(long long)c + s - 1) / s);
}

__global__ void scale_kernel(const int32_t* __restrict__ C, long long ldc, int n, int m, int32_t s,
                             int32_t* __restrict__ out) {
  const long long total = (long long)n * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / m, j = e - i * m;
    out[e] = floor_div(__ldg(C + i * ldc + j), s);
  }
}

// cost = sum_i C[i][row_to_col[i]] (int64) into *cost (zeroed by the caller)
__global__ void true_cost_kernel(const int32_t* __restrict__ C, long long ldc, int n,
                                 const int32_t* __restrict__ r2c, unsigned long long* cost) {
  long long part = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    part += __ldg(C + (long long)i * ldc + r2c[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0 && part) atomicAdd(cost, (unsigned long long)part);
}

}  // namespace ot

using namespace ot;

extern "C" int ot_assign_solve_scaled(ot_ctx* ctx, const int32_t* C, int64_t ldc, int32_t n, int32_t m,
                                      int32_t scale, int32_t* row_to_col, int64_t* cost, int64_t* bound,
                                      void* stream) {
  if (!ctx) return OT_ERR_ARG;
  if (scale < 1 || n < 0 || m < n || (n > 0 && (!C || ldc < m || !row_to_col)) || !cost)
    return ctx_fail(ctx, OT_ERR_ARG, "bad arguments");
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> lock(ctx->scaled_mu);
  StreamScope scope(static_cast<cudaStream_t>(stream), ctx->stream, ctx->sjoin_in_ev, ctx->sjoin_out_ev);
  cudaStream_t s = scope.work;
  const bool dev = n > 0 ? ptr_on_device(C) : ptr_on_device(cost);
  if (bound) {
    const int64_t b = int64_t(n) * (scale - 1);
    if (ptr_on_device(bound)) cudaMemcpyAsync(bound, &b, sizeof(b), cudaMemcpyHostToDevice, s), cudaStreamSynchronize(s);
    else *bound = b;
  }
  if (n == 0) {
    if (dev) cudaMemsetAsync(cost, 0, sizeof(int64_t), s);
    else *cost = 0;
    return OT_OK;
  }
  // device copies: original (when C is on the host), scaled matrix, outputs
  const size_t mat = sizeof(int32_t) * size_t(n) * m;
  const size_t o_orig = 0, o_scaled = dev ? 0 : (mat + 255) & ~size_t(255);
  const size_t o_r2c = o_scaled + ((mat + 255) & ~size_t(255));
  const size_t o_u = o_r2c + ((4 * size_t(n) + 255) & ~size_t(255));
  const size_t o_v = o_u + ((8 * size_t(n) + 255) & ~size_t(255));
  const size_t o_cost = o_v + ((8 * size_t(m) + 255) & ~size_t(255));
  const size_t total = o_cost + 256;
  if (int rc = ctx->d_scaled.reserve(total); rc) return ctx_fail(ctx, rc, "scaled workspace");
  char* B = static_cast<char*>(ctx->d_scaled.ptr);
  const int32_t* Cd = C;
  long long ld = ldc;
  cudaError_t e;
  if (!dev) {
    e = cudaMemcpy2DAsync(B + o_orig, 4 * size_t(m), C, 4 * size_t(ldc), 4 * size_t(m), n,
                          cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "scaled H2D");
    Cd = reinterpret_cast<const int32_t*>(B + o_orig);
    ld = m;
  }
  int32_t* Cs = reinterpret_cast<int32_t*>(B + o_scaled);
  int32_t* r2c = dev ? row_to_col : reinterpret_cast<int32_t*>(B + o_r2c);
  int64_t* du = reinterpret_cast<int64_t*>(B + o_u);
  int64_t* dv = reinterpret_cast<int64_t*>(B + o_v);
  int64_t* dcost = reinterpret_cast<int64_t*>(B + o_cost);
  int dv_id = 0, sms = 0;
  cudaGetDevice(&dv_id);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dv_id);
  scale_kernel<<<4 * sms, 256, 0, s>>>(Cd, ld, n, m, scale, Cs);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "scale kernel");
  // exact batched KM on the scaled costs (scaled cost into dcost, discarded)
  ot_stats st;
  int rc = ot_assign_solve_stats(ctx, Cs, m, n, m, OT_BKM, r2c, dcost, du, dv, &st, s);
  if (rc != OT_OK) return rc;
  // cost of that assignment under the original costs
  unsigned long long* tc = reinterpret_cast<unsigned long long*>(dcost);
  cudaMemsetAsync(tc, 0, sizeof(*tc), s);
  true_cost_kernel<<<(n + 255) / 256, 256, 0, s>>>(Cd, ld, n, r2c, tc);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "true cost");
  if (dev) {
    e = cudaMemcpyAsync(cost, tc, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  } else {
    e = cudaMemcpyAsync(cost, tc, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(row_to_col, r2c, 4 * size_t(n), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "scaled results");
  return OT_OK;
}
