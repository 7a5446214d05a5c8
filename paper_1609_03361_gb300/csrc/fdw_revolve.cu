// Binomial checkpoint schedules for the reverse (adjoint) sweep of the FWI
// gradient when only `nslots` checkpoint pairs fit in memory: Griewank's
// binomial checkpointing (A. Griewank, Optimization Methods and Software 1,
// 1992; A. Griewank and A. Walther, ACM TOMS 26, 2000, "revolve"), applied
// to the k-step segments of the gradient pass (the paper's gradient workload,
// Sec. 5.4, stores wavefields; this trades memory for recomputation).
//
// Model.  Time is cut into nseg segments.  Reversing a segment needs the
// forward state (u^{a}, u^{a-1}) at its start; the state at segment 0 is zero
// and needs no slot.  Actions:
//   ADVANCE b   run the forward steps from the current segment start to b's
//   TAKESHOT s  store the current state in slot s
//   RESTORE s   make slot s (or -1: the zero state) the current state
//   REVERSE j   recompute segment j from the current state (which must be j's
//               start) and run its adjoint steps
// Reversing l segments whose start state is held, with c free slots, costs at
// least F(l, c) segment advances; with s = c + 1 and r the smallest integer
// with C(s + r, s) >= l,
//   F(l, c) = r l - C(s + r, s + 1)         (c >= 1),   F(l, 0) = l (l - 1) / 2,
// and the schedule below attains it: it advances j segments, stores that
// state, reverses the right part with one slot fewer and then the left part,
// with j the smallest minimiser of j + F(l - j, c - 1) + F(j, c).
#include <cstdint>
#include <vector>

#include "fdw_internal.h"
#include "fdwave.h"

namespace fdw {
namespace {

// C(n, k), saturating at 2^62.
long long binom(long long n, long long k) {
  if (k < 0 || n < 0 || k > n) return 0;
  if (k > n - k) k = n - k;
  const long long cap = 1LL << 62;
  long long v = 1;
  for (long long i = 1; i <= k; ++i) {
    // v * (n - k + i) / i stays exact: v * (n-k+i) is divisible by i
    const long long f = n - k + i;
    if (v > cap / f) return cap;
    v = v * f / i;
  }
  return v;
}

struct Builder {
  std::vector<CkptAction> out;
  long long cur = 0;  // segment whose start state is current
  void advance(long long b) {
    out.push_back({kCkptAdvance, (int)b});
    cur = b;
  }
  void ensure(long long a, int hold) {
    if (cur != a) {
      out.push_back({kCkptRestore, hold});
      cur = a;
    }
  }
  void rev(long long a, long long l, std::vector<int>& freeslots, int hold) {
    if (l <= 0) return;
    if (l == 1) {
      ensure(a, hold);
      out.push_back({kCkptReverse, (int)a});
      return;
    }
    const int c = (int)freeslots.size();
    if (c == 0) {  // no slot: re-advance from the held state for every segment
      for (long long i = l - 1; i >= 0; --i) {
        ensure(a, hold);
        if (i > 0) advance(a + i);
        out.push_back({kCkptReverse, (int)(a + i)});
      }
      return;
    }
    long long bj = 1, best = -1;
    for (long long j = 1; j < l; ++j) {
      const long long t = j + revolve_cost(l - j, c - 1) + revolve_cost(j, c);
      if (best < 0 || t < best) {
        best = t;
        bj = j;
      }
    }
    ensure(a, hold);
    advance(a + bj);
    const int slot = freeslots.back();
    freeslots.pop_back();
    out.push_back({kCkptTakeshot, slot});
    rev(a + bj, l - bj, freeslots, slot);
    freeslots.push_back(slot);
    rev(a, bj, freeslots, hold);
  }
};

}  // namespace

long long revolve_cost(long long l, int c) {
  if (l <= 1) return 0;
  if (c <= 0) return l * (l - 1) / 2;
  const long long s = c + 1;
  long long r = 0;
  while (binom(s + r, s) < l) ++r;
  return r * l - binom(s + r, s + 1);
}

std::vector<CkptAction> revolve_schedule(int nseg, int nslots) {
  Builder b;
  std::vector<int> freeslots;
  for (int i = nslots - 1; i >= 0; --i) freeslots.push_back(i);
  b.rev(0, nseg, freeslots, -1);
  return b.out;
}

}  // namespace fdw

extern "C" int fdw_checkpoint_schedule(int nseg, int nslots, int* actions, int cap) {
  if (nseg < 1 || nslots < 0 || cap < 0 || (cap > 0 && !actions)) return -1;
  const std::vector<fdw::CkptAction> v = fdw::revolve_schedule(nseg, nslots);
  if ((long long)v.size() > cap) return (int)v.size();
  for (size_t i = 0; i < v.size(); ++i) {
    actions[2 * i] = v[i].op;
    actions[2 * i + 1] = v[i].arg;
  }
  return (int)v.size();
}
