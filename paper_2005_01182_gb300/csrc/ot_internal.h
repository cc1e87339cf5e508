// Internal types shared by the CUDA translation units of libotassign.so.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ot {

constexpr long long kInf = 1LL << 62;

// One instance as the device engines see it.  All pointers are device
// pointers; stats/status may be null.
struct Instance {
  const int32_t* C;   // row-major, ldc elements per row
  int64_t ldc;
  int32_t n, m;
  int32_t* row_to_col;  // [n]
  int64_t* u;           // [n]
  int64_t* v;           // [m]
  int64_t* cost;        // [1]
  int32_t* status;      // [1]
  int64_t* stats;       // [8], laid out as ot_stats
  // Optional 16-bit copy of C made by pack_rows: C[i][j] = P[i*m + j] +
  // roff[i] when *pok != 0 (every row's range fits 16 bits).  The solver then
  // runs on the row-shifted problem, which has the same assignment and the
  // same column duals; row duals are shifted back by roff at the end.
  // (plain struct: every constructor of an Instance sets these, nullptr
  // when not packed)
  const uint16_t* P;
  const int32_t* roff;
  const int32_t* pok;
  // Dependent steps the instance may take before its status becomes the
  // step-limit code (0: only the built-in guards apply).
  long long step_limit;
};

// Pack the rows of `num` instances (insts[order[t]], P/roff/pok set) into
// 16-bit offsets from each row's minimum; one CTA per instance.
cudaError_t launch_pack(const Instance* insts, const int32_t* order, int num, cudaStream_t stream);

// Shape of a solver group: TPI threads cooperate on one instance, each
// owning K columns (j = t + k*TPI).  TPI == 32 packs several warps per CTA.
struct GroupShape {
  int tpi;
  int k;
  int max_cols() const { return tpi * k; }
};

// Launch the group engine over `num` instances listed in `order` (indices
// into `insts`), pulling work from `work_counter` (device int, zeroed by
// the caller).  algo: 0 = KM, 1 = batched KM.  nmax/mmax bound the sizes of
// the listed instances.  Returns a CUDA error code.
cudaError_t launch_group(GroupShape shape, int algo, const Instance* insts,
                         const int32_t* order, int num, int* work_counter, int nmax,
                         int mmax, int max_ctas, cudaStream_t stream);

// Shapes compiled into the library, smallest first.
int num_group_shapes();
GroupShape group_shape(int idx);
// Dynamic shared memory the group engine needs per CTA for these bounds.
size_t group_smem_bytes(GroupShape shape, int algo, int nmax, int mmax);
size_t group_smem_limit();

// Auction engine (ot_auction.cu): one CTA of auction_threads(m) threads
// per instance; `num` instances listed in `order`, pulled from `work`.
int auction_threads(int m);
size_t auction_smem_bytes(int mmax);
cudaError_t launch_auction(int threads, const Instance* insts, const int32_t* order, int num, int* work,
                           int mmax, cudaStream_t stream);

}  // namespace ot
