// Row packing for the group engine: each cost row is stored as 16-bit
// offsets from its minimum when its range allows, halving the bytes every
// dependent step loads and the L2 footprint of a batch (the solver runs on
// the row-shifted problem; see Instance::P).
#include <climits>

#include "ot_internal.h"

namespace ot {

constexpr int kPackRegs = 8;  // rows up to 256 columns are packed from registers

__global__ void __launch_bounds__(256) pack_kernel(const Instance* __restrict__ insts,
                                                   const int32_t* __restrict__ order, int num) {
  const Instance I = insts[order ? order[blockIdx.x] : blockIdx.x];
  if (I.P == nullptr) return;  // not packed (uniform over the CTA)
  __shared__ int ok;
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int n = I.n, m = I.m;
  uint16_t* P = const_cast<uint16_t*>(I.P);
  int32_t* roff = const_cast<int32_t*>(I.roff);
  if (m <= 32 * kPackRegs) {
    // the row stays in registers: all its loads in flight at once, one read
    for (int i = warp; i < n; i += nwarps) {
      const int32_t* row = I.C + (long long)i * I.ldc;
      int c[kPackRegs];
#pragma unroll
      for (int q = 0; q < kPackRegs; ++q) {
        const int j = lane + 32 * q;
        c[q] = j < m ? __ldg(row + j) : 0;
      }
      int mn = INT_MAX, mx = INT_MIN;
#pragma unroll
      for (int q = 0; q < kPackRegs; ++q)
        if (lane + 32 * q < m) {
          mn = min(mn, c[q]);
          mx = max(mx, c[q]);
        }
      mn = __reduce_min_sync(0xffffffffu, mn);
      mx = __reduce_max_sync(0xffffffffu, mx);
      if ((long long)mx - (long long)mn > 65535) {
        if (lane == 0) ok = 0;
        continue;
      }
      uint16_t* prow = P + (long long)i * m;
#pragma unroll
      for (int q = 0; q < kPackRegs; ++q) {
        const int j = lane + 32 * q;
        if (j < m) prow[j] = static_cast<uint16_t>(c[q] - mn);
      }
      if (lane == 0) roff[i] = mn;
    }
    __syncthreads();
    if (threadIdx.x == 0) *const_cast<int32_t*>(I.pok) = ok;
    return;
  }
  for (int i = warp; i < n; i += nwarps) {
    const int32_t* row = I.C + (long long)i * I.ldc;
    int mn = INT_MAX, mx = INT_MIN;
    for (int j = lane; j < m; j += 32) {
      const int c = __ldg(row + j);
      mn = min(mn, c);
      mx = max(mx, c);
    }
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((long long)mx - (long long)mn > 65535) {
      if (lane == 0) ok = 0;
      continue;
    }
    uint16_t* prow = P + (long long)i * m;
    for (int j = lane; j < m; j += 32) prow[j] = static_cast<uint16_t>(__ldg(row + j) - mn);
    if (lane == 0) roff[i] = mn;
  }
  __syncthreads();
  if (threadIdx.x == 0) *const_cast<int32_t*>(I.pok) = ok;
}

cudaError_t launch_pack(const Instance* insts, const int32_t* order, int num, cudaStream_t stream) {
  if (num <= 0) return cudaSuccess;
  pack_kernel<<<num, 256, 0, stream>>>(insts, order, num);
  return cudaGetLastError();
}

}  // namespace ot
