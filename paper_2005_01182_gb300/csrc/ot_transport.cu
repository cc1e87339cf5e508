// Optimal transport with integer supplies and demands (Eq. 1 with integer r
// and c, the Hitchcock-Koopmans case of Sec. 1) by vertex replication: row i
// appears supply[i] times and column j demand[j] times, in index order, in an
// assignment problem, whose matching is folded back into a flow matrix.
#include <cstring>
#include <vector>

#include "otassign.h"
#include "ot_ctx.h"

namespace ot {

__global__ void expand_kernel(const int32_t* __restrict__ C, long long ldc, const int32_t* __restrict__ rowmap,
                              const int32_t* __restrict__ colmap, int R, int M, int32_t* __restrict__ out) {
  const long long total = (long long)R * M;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / M, c = e - r * M;
    out[e] = __ldg(C + (long long)rowmap[r] * ldc + colmap[c]);
  }
}

__global__ void fold_kernel(const int32_t* __restrict__ r2c, const int32_t* __restrict__ rowmap,
                            const int32_t* __restrict__ colmap, int R, int m, int32_t* __restrict__ flow) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x)
    atomicAdd(&flow[(long long)rowmap[r] * m + colmap[r2c[r]]], 1);
}

}  // namespace ot

using namespace ot;

extern "C" int ot_transport_solve(ot_ctx* ctx, const int32_t* C, int64_t ldc, int32_t n, int32_t m,
                                  const int32_t* supply, const int32_t* demand, int32_t algo, int64_t* cost,
                                  int32_t* flow, void* stream) {
  if (!ctx) return OT_ERR_ARG;
  if (n < 0 || m < 0 || !cost || (n > 0 && (!C || ldc < m || !supply || !flow)) || (m > 0 && !demand) ||
      (algo != OT_KM && algo != OT_BKM && algo != OT_AUTO))
    return ctx_fail(ctx, OT_ERR_ARG, "bad arguments");
  long long R = 0, M = 0;
  for (int i = 0; i < n; ++i) {
    if (supply[i] < 0) return ctx_fail(ctx, OT_ERR_ARG, "negative supply");
    R += supply[i];
  }
  for (int j = 0; j < m; ++j) {
    if (demand[j] < 0) return ctx_fail(ctx, OT_ERR_ARG, "negative demand");
    M += demand[j];
  }
  if (R > M) return ctx_fail(ctx, OT_ERR_ARG, "total supply exceeds total demand");
  if (M > 65536 || R * M > (1LL << 30))
    return ctx_fail(ctx, OT_ERR_UNSUPPORTED, "replicated problem too large");
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> lock(ctx->scaled_mu);
  StreamScope scope(static_cast<cudaStream_t>(stream), ctx->stream, ctx->sjoin_in_ev, ctx->sjoin_out_ev);
  cudaStream_t s = scope.work;
  const bool dev = n > 0 ? ptr_on_device(C) : false;
  const bool dflow = n > 0 && ptr_on_device(flow);
  if (R == 0) {
    if (n > 0 && m > 0) {
      if (dflow) cudaMemsetAsync(flow, 0, sizeof(int32_t) * size_t(n) * m, s), cudaStreamSynchronize(s);
      else std::memset(flow, 0, sizeof(int32_t) * size_t(n) * m);
    }
    if (ptr_on_device(cost)) cudaMemsetAsync(cost, 0, sizeof(int64_t), s), cudaStreamSynchronize(s);
    else *cost = 0;
    return OT_OK;
  }
  std::vector<int32_t> rowmap(R), colmap(M);
  for (int i = 0, r = 0; i < n; ++i)
    for (int q = 0; q < supply[i]; ++q) rowmap[r++] = i;
  for (int j = 0, c = 0; j < m; ++j)
    for (int q = 0; q < demand[j]; ++q) colmap[c++] = j;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t b_c = dev ? 0 : al(4 * size_t(n) * m);
  size_t off = 0;
  const size_t o_c = off; off += b_c;
  const size_t o_rep = off; off += al(4 * size_t(R) * M);
  const size_t o_rm = off; off += al(4 * size_t(R));
  const size_t o_cm = off; off += al(4 * size_t(M));
  const size_t o_r2c = off; off += al(4 * size_t(R));
  const size_t o_u = off; off += al(8 * size_t(R));
  const size_t o_v = off; off += al(8 * size_t(M));
  const size_t o_flow = off; off += al(4 * size_t(n) * m);
  const size_t o_cost = off; off += 256;
  if (int rc = ctx->d_scaled.reserve(off); rc) return ctx_fail(ctx, rc, "transport workspace");
  char* B = static_cast<char*>(ctx->d_scaled.ptr);
  const int32_t* Cd = C;
  long long ld = ldc;
  cudaError_t e;
  if (!dev) {
    e = cudaMemcpy2DAsync(B + o_c, 4 * size_t(m), C, 4 * size_t(ldc), 4 * size_t(m), n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "transport H2D");
    Cd = reinterpret_cast<const int32_t*>(B + o_c);
    ld = m;
  }
  int32_t* rep = reinterpret_cast<int32_t*>(B + o_rep);
  int32_t* drm = reinterpret_cast<int32_t*>(B + o_rm);
  int32_t* dcm = reinterpret_cast<int32_t*>(B + o_cm);
  int32_t* r2c = reinterpret_cast<int32_t*>(B + o_r2c);
  int64_t* du = reinterpret_cast<int64_t*>(B + o_u);
  int64_t* dv = reinterpret_cast<int64_t*>(B + o_v);
  int32_t* dflowbuf = dflow ? flow : reinterpret_cast<int32_t*>(B + o_flow);
  int64_t* dcost = reinterpret_cast<int64_t*>(B + o_cost);
  e = cudaMemcpyAsync(drm, rowmap.data(), 4 * size_t(R), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dcm, colmap.data(), 4 * size_t(M), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "transport maps");
  int dv_id = 0, sms = 0;
  cudaGetDevice(&dv_id);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dv_id);
  expand_kernel<<<4 * sms, 256, 0, s>>>(Cd, ld, drm, dcm, int(R), int(M), rep);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "expand");
  ot_stats st;
  int rc = ot_assign_solve_stats(ctx, rep, M, int(R), int(M), algo, r2c, dcost, du, dv, &st, s);
  if (rc != OT_OK) return rc;
  if ((e = cudaMemsetAsync(dflowbuf, 0, sizeof(int32_t) * size_t(n) * m, s)) != cudaSuccess)
    return ctx_cuda(ctx, e, "flow memset");
  fold_kernel<<<(int(R) + 255) / 256, 256, 0, s>>>(r2c, drm, dcm, int(R), m, dflowbuf);
  if ((e = cudaGetLastError()) != cudaSuccess) return ctx_cuda(ctx, e, "fold");
  if (!dflow) e = cudaMemcpyAsync(flow, dflowbuf, sizeof(int32_t) * size_t(n) * m, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cost, dcost, sizeof(int64_t), ptr_on_device(cost) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ctx_cuda(ctx, e, "transport results");
  return OT_OK;
}
