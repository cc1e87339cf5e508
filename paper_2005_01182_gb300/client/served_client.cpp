// Open-loop client of the serving entry points (ot_assign_submit,
// ot_assign_completed, ot_assign_poll), so that a served stream can be
// measured without an interpreter in the loop.  One host thread submits each
// request once its arrival time has passed, collects the requests the
// completion query returns, and records when each one completed and its
// cost.  Built beside libotassign.so as libotclient.so; it holds no solver
// code of its own.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <thread>
#include <unordered_map>
#include <vector>

#include "otassign.h"

extern "C" {

// Replay a stream of nreq requests over nmat host matrices (request r uses
// matrix r % nmat: C[q] row-major n[q] x m[q], contiguous).  arrival_s[r]:
// arrival time of request r in seconds from the start, non-decreasing (all
// zero: submit as fast as the window allows).  At most `window` requests
// are outstanding (submitted, not yet collected).  Outputs: done_s[r], the
// time request r was collected; cost[r], its optimal cost; *total_s, the
// time the last one was collected.  Returns OT_OK or the first error code of
// the serving calls.
int otc_replay(ot_ctx* ctx, int32_t nmat, const int32_t* const* C, const int32_t* n, const int32_t* m,
               int32_t nreq, const double* arrival_s, int32_t window, int32_t algo, double* done_s, int64_t* cost,
               double* total_s) {
  if (!ctx || nmat <= 0 || nreq < 0 || !C || !n || !m || window <= 0 || !total_s ||
      (nreq > 0 && (!arrival_s || !done_s || !cost)))
    return OT_ERR_ARG;
  int nmax = 1;
  for (int q = 0; q < nmat; ++q) nmax = std::max(nmax, int(n[q]));
  std::vector<int32_t> r2c(static_cast<size_t>(nmax));
  std::vector<uint64_t> fin(4096);
  std::unordered_map<uint64_t, int32_t> out;
  out.reserve(static_cast<size_t>(std::min(window, nreq)) * 2 + 16);
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  auto since = [&] { return std::chrono::duration<double>(clk::now() - t0).count(); };
  int32_t nxt = 0;
  while (nxt < nreq || !out.empty()) {
    while (nxt < nreq && arrival_s[nxt] <= since() && static_cast<int32_t>(out.size()) < window) {
      const int q = nxt % nmat;
      uint64_t tk = 0;
      const int rc = ot_assign_submit(ctx, C[q], m[q], n[q], m[q], algo, &tk);
      if (rc != OT_OK) return rc;
      out.emplace(tk, nxt);
      ++nxt;
    }
    int32_t cnt = 0;
    int rc = ot_assign_completed(ctx, fin.data(), static_cast<int32_t>(fin.size()), &cnt);
    if (rc != OT_OK) return rc;
    for (int x = 0; x < cnt; ++x) {
      const auto it = out.find(fin[x]);
      if (it == out.end()) return OT_ERR_TICKET;
      const int32_t r = it->second;
      rc = ot_assign_poll(ctx, fin[x], r2c.data(), &cost[r], nullptr, nullptr);
      if (rc != OT_OK) return rc;
      done_s[r] = since();
      out.erase(it);
    }
    if (cnt == 0) {
      // nothing finished: wait up to 20 us, not past the next arrival (a
      // yielding spin: a sleep of that length lasts several times longer)
      double until = since() + 20e-6;
      if (nxt < nreq && static_cast<int32_t>(out.size()) < window) until = std::min(until, arrival_s[nxt]);
      while (since() < until) std::this_thread::yield();
    }
  }
  *total_s = since();
  return OT_OK;
}

}  // extern "C"
