// k_listsched.cuh -- makespan of a mapping on a fixed number of workers per side (a list schedule).
//
// The testbed of Sec. IV.A runs the kernels on 3 CPU worker cores and 1 GPU worker.  Given a split,
// the schedule is simulated event by event in time order:
//   - a task v runs without preemption on one worker of side part[v] for its cost on that side;
//   - its data are there at r(v) = max over in-entries u->v of finish(u) (+ w(u,v) when u sits on the
//     other side; every parallel entry counts, transfers do not compete); r = 0 for a source;
//   - at each time t, every running task that ends at or before t ends (its worker becomes idle, and a
//     successor whose last predecessor this was is released); then, on each side, while a worker is
//     idle and a released task with r <= t waits, the waiting task with the smallest (r, id) starts;
//     t moves to the next end of a running task or, on a side with an idle worker, to the smallest r
//     among its waiting tasks.
// The simulation is one event after another, so its data-parallel form is across graphs: one warp
// simulates one graph (a persistent grid takes graphs from an atomic queue, largest first).  Within a
// warp:
//   - workers are lanes: lane i < Pc is CPU worker i, Pc <= i < Pc + Pg a GPU worker; a worker lane
//     holds its running task, its end time and the task's out-row bounds in registers (the bounds are
//     loaded when the task starts, so they have arrived when it ends);
//   - the waiting tasks of a side are an unordered array of (r, id, cost) records; the next task to
//     start is found by a warp-wide scan and shuffle reduction (the records are 16 bytes, one vector
//     load per lane per 32 records), and taken out by moving the last record, which the scan left in
//     the registers of one lane, into its slot;
//   - when a task ends, the warp walks its out-row 32 entries at a time; every lane loads its
//     successor's record {ready time, pending count, side, cost on that side} (16 bytes), lanes that
//     hit the same successor (parallel entries) are grouped with __match_any_sync, and the group's
//     leader writes the updated record back (plain store: only this warp touches the graph) and
//     appends the successor to its side's waiting array once the count reaches 0.
// A task's path through the loop is thus three dependent memory round trips: its predecessor's
// out-row entries, its own record, and the scan that starts it.
// The result does not depend on the order in which tasks ending at the same time are processed, nor
// on which idle worker of a side takes a task.
#pragma once
#include "gp_internal.cuh"

namespace gp {

constexpr int kLsMaxWorkers = 32;  // workers of both sides together (one lane each)

struct __align__(16) LsRec {  // per vertex
  long long ready;   // r(v) so far (max over the predecessors that have ended)
  int pending;       // predecessors (in-entries) not ended yet
  unsigned sc;       // side << 31 | cost on that side (costs are validated to be non-negative int32)
};
struct __align__(16) LsWait {  // a waiting task
  long long r;
  int v;
  int cost;  // on its side
};

struct LsJob {       // one graph
  int64_t n;
  const int64_t* off;      // out-CSR
  const int32_t* cols;
  const int32_t* w;
  const int32_t* cC;
  const int32_t* cG;
  const int64_t* in_off;   // in-degrees from the vertex-indexed in-CSR
  const uint8_t* part;
  LsRec* rec;              // n records
  LsWait* wait;            // 2n records: side 0 at [0, n), side 1 at [n, 2n)
  long long* fin;          // n finish times
};

struct LsOut {
  long long makespan;
  int status;  // bit 0: a part value > 1; bit 1: the event loop exceeded its iteration bound
  int pad;
};

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ bool ls_less(long long ra, int va, long long rb, int vb) {
  return ra < rb || (ra == rb && va < vb);
}

// Warp-wide minimum of a non-negative 64-bit value (its high and low words order it as unsigned).
__device__ __forceinline__ long long ls_min(long long x) {
  const unsigned hi = (unsigned)((unsigned long long)x >> 32), lo = (unsigned)(unsigned long long)x;
  const unsigned mhi = __reduce_min_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_min_sync(0xffffffffu, hi == mhi ? lo : 0xffffffffu);
  return (long long)(((unsigned long long)mhi << 32) | mlo);
}

// A side's waiting array and the smallest record its last scan found (warp-uniform).
struct LsSide {
  LsWait* W;
  int len;
  bool clean;  // the array is unchanged since that scan: br, bv, bi, bc still hold
  long long br;
  int bv, bi, bc;
};

// Starts on one side at time t: while a worker of the side is idle (mine: this lane is one of the
// side's workers) and the waiting task with the smallest (r, id) has r <= t, it starts on the lowest
// idle worker, which loads the task's out-row bounds.  On return, cand = that smallest r if a worker
// stayed idle and tasks wait (else unchanged).  The array is scanned only when it changed since the
// last scan.
__device__ __forceinline__ void ls_starts(LsSide& S, bool mine, long long t, const int64_t* off, bool& busy,
                                          bool& pf, long long& wend, int64_t& we0, int64_t& we1, long long& ms,
                                          long long* fin, long long& cand) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    const unsigned idle = __ballot_sync(0xffffffffu, mine && !busy);
    if (!idle || S.len == 0) return;
    const int last = S.len - 1;
    LsWait y{0, 0, 0};  // the last record, when this call scanned
    const bool fresh = !S.clean;
    if (fresh) {
      long long br = LLONG_MAX;
      int bv = INT_MAX, bi = -1, bc = 0;
      LsWait xl{0, 0, 0};  // the last record this lane read
      for (int i = lane; i < S.len; i += 32) {
        const LsWait x = S.W[i];
        xl = x;
        if (ls_less(x.r, x.v, br, bv)) {
          br = x.r;
          bv = x.v;
          bi = i;
          bc = x.cost;
        }
      }
      // the smallest (r, id) of the warp: r by ls_min, then the smallest id among the lanes holding it
      const long long mr = ls_min(br);
      const unsigned mv = __reduce_min_sync(0xffffffffu, br == mr ? (unsigned)bv : 0xffffffffu);
      const int wl = __ffs(__ballot_sync(0xffffffffu, br == mr && (unsigned)bv == mv)) - 1;
      S.br = mr;
      S.bv = (int)mv;
      S.bi = __shfl_sync(0xffffffffu, bi, wl);
      S.bc = __shfl_sync(0xffffffffu, bc, wl);
      S.clean = true;
      // lane last % 32 read the last record in its final scan step
      y.r = __shfl_sync(0xffffffffu, xl.r, last & 31);
      y.v = __shfl_sync(0xffffffffu, xl.v, last & 31);
      y.cost = __shfl_sync(0xffffffffu, xl.cost, last & 31);
    }
    if (S.br > t) {
      cand = S.br;
      return;
    }
    // take it out: the last record moves into its slot
    if (lane == 0 && S.bi != last) S.W[S.bi] = fresh ? y : S.W[last];
    S.len--;
    S.clean = false;
    __syncwarp();
    if (lane == __ffs(idle) - 1) {
      busy = true;
      pf = true;
      wend = t + (long long)S.bc;
      we0 = off[S.bv];
      we1 = off[S.bv + 1];
      fin[S.bv] = wend;
      ms = wend > ms ? wend : ms;
    }
  }
}

// One warp, one graph.
__device__ void ls_graph(const LsJob& J, int Pc, int Pg, LsOut* out) {
  const int lane = threadIdx.x & 31;
  const int64_t n = J.n;
  int bad = 0;
  // records: pending = in-degree, ready = 0, side and cost on it; sources into the waiting arrays
  int len0 = 0, len1 = 0;
  for (int64_t base = 0; base < n; base += 32) {
    const int64_t v = base + lane;
    bool src = false;
    int side = 0, cost = 0;
    if (v < n) {
      const int deg = (int)(J.in_off[v + 1] - J.in_off[v]);
      const uint8_t p = J.part[v];
      bad |= p > 1;
      side = p & 1;
      cost = side ? J.cG[v] : J.cC[v];
      LsRec r;
      r.ready = 0;
      r.pending = deg;
      r.sc = ((unsigned)side << 31) | ((unsigned)cost & 0x7fffffffu);
      J.rec[v] = r;
      src = deg == 0;
    }
    const unsigned m0 = __ballot_sync(0xffffffffu, src && side == 0);
    const unsigned m1 = __ballot_sync(0xffffffffu, src && side == 1);
    const unsigned lt = (1u << lane) - 1u;
    if (src) {
      LsWait x;
      x.r = 0;
      x.v = (int)v;
      x.cost = cost;
      if (side == 0)
        J.wait[len0 + __popc(m0 & lt)] = x;
      else
        J.wait[n + len1 + __popc(m1 & lt)] = x;
    }
    len0 += __popc(m0);
    len1 += __popc(m1);
  }
  bad = __any_sync(0xffffffffu, bad);
  if (bad) {
    if (lane == 0) {
      out->makespan = 0;
      out->status = 1;
    }
    return;
  }
  __syncwarp();
  // worker lanes
  const bool is_worker = lane < Pc + Pg;
  const int wside = lane < Pc ? 0 : 1;
  bool busy = false;
  long long wend = 0;
  int64_t we0 = 0, we1 = 0;  // the running task's out-row
  bool pf = false;           // that row is still to be prefetched
  LsSide S0{J.wait, len0, false, 0, 0, 0, 0}, S1{J.wait + n, len1, false, 0, 0, 0, 0};
  long long ms = 0;
  long long t = 0;
  const long long kInf = LLONG_MAX;
  // every iteration ends a task, starts one or moves t to an end or a ready time: 4n + 8 is a bound
  const int64_t max_iter = 4 * n + 8;
  int64_t iter = 0;
  for (;; iter++) {
    if (iter > max_iter) {
      bad = 2;
      break;
    }
    // the first out-entries of the task this lane started in the previous iteration (its row bounds have
    // arrived by now) are fetched into L1, to be there when the task ends
    if (pf) {
      pf = false;
      const int64_t last = (we1 - we0 > 32 ? we0 + 32 : we1) - 1;
      if (last >= we0) {
        prefetch_l1(J.cols + we0);
        prefetch_l1(J.cols + last);
        prefetch_l1(J.w + we0);
        prefetch_l1(J.w + last);
      }
    }
    // ---- ends at or before t
    unsigned endm = __ballot_sync(0xffffffffu, is_worker && busy && wend <= t);
    while (endm) {
      const int wl = __ffs(endm) - 1;
      endm &= endm - 1;
      const long long fu = __shfl_sync(0xffffffffu, wend, wl);
      const int64_t e0 = __shfl_sync(0xffffffffu, we0, wl), e1 = __shfl_sync(0xffffffffu, we1, wl);
      const unsigned pu = wl < Pc ? 0u : 1u;
      if (lane == wl) busy = false;
      for (int64_t b = e0; b < e1; b += 32) {
        const int64_t e = b + lane;
        const bool valid = e < e1;
        int v = -1;
        long long arrive = 0;
        LsRec rv{0, 0, 0u};
        if (valid && GP_IN(J.cols[e], n, 13)) {
          v = J.cols[e];
          const int32_t we = J.w[e];
          rv = J.rec[v];
          arrive = fu + ((rv.sc >> 31) != pu ? (long long)we : 0ll);
        }
        const unsigned pv = rv.sc >> 31;
        // lanes holding the same successor form one group; its leader applies the group's update
        const unsigned grp = __match_any_sync(0xffffffffu, v);
        long long amax = arrive;
        int cnt = 0;
        for (unsigned gm = grp; gm; gm &= gm - 1) {
          const int src = __ffs(gm) - 1;
          const long long a = __shfl_sync(grp, arrive, src);
          amax = a > amax ? a : amax;
          cnt++;
        }
        const bool leader = v >= 0 && lane == __ffs(grp) - 1;
        bool released = false;
        if (leader) {
          rv.ready = amax > rv.ready ? amax : rv.ready;
          rv.pending -= cnt;
          J.rec[v] = rv;
          released = rv.pending == 0;
        }
        const unsigned m0 = __ballot_sync(0xffffffffu, released && pv == 0);
        const unsigned m1 = __ballot_sync(0xffffffffu, released && pv == 1);
        const unsigned lt = (1u << lane) - 1u;
        if (released) {
          LsWait x;
          x.r = rv.ready;
          x.v = v;
          x.cost = (int)(rv.sc & 0x7fffffffu);
          if (pv == 0)
            S0.W[S0.len + __popc(m0 & lt)] = x;
          else
            S1.W[S1.len + __popc(m1 & lt)] = x;
        }
        if (m0) {
          S0.len += __popc(m0);
          S0.clean = false;
        }
        if (m1) {
          S1.len += __popc(m1);
          S1.clean = false;
        }
        __syncwarp();  // the next chunk may update a successor this chunk updated
      }
    }
    // ---- starts at t, side by side; cand = the smallest waiting r of a side with an idle worker
    long long cand0 = kInf, cand1 = kInf;
    ls_starts(S0, is_worker && wside == 0, t, J.off, busy, pf, wend, we0, we1, ms, J.fin, cand0);
    ls_starts(S1, is_worker && wside == 1, t, J.off, busy, pf, wend, we0, we1, ms, J.fin, cand1);
    // ---- next time
    if (__any_sync(0xffffffffu, is_worker && busy && wend <= t)) continue;  // a task of cost 0 ended at t
    long long nx = ls_min((is_worker && busy) ? wend : kInf);
    nx = cand0 < nx ? cand0 : nx;
    nx = cand1 < nx ? cand1 : nx;
    if (nx == kInf) break;
    t = nx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long q = __shfl_xor_sync(0xffffffffu, ms, o);
    ms = q > ms ? q : ms;
  }
  if (lane == 0) {
    out->makespan = ms;
    out->status = bad;
  }
}

// Persistent: each warp takes graphs from `queue` (graph ids in `order`, largest first).
__global__ void __launch_bounds__(256, 2) k_listsched(int count, const LsJob* __restrict__ jobs,
                                                   const int* __restrict__ order, int Pc, int Pg,
                                                   unsigned* queue, LsOut* out) {
  const int lane = threadIdx.x & 31;
  unsigned long long bytes = 0;
  for (;;) {
    unsigned q = 0;
    if (lane == 0) q = atomicAdd(queue, 1u);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= (unsigned)count) break;
    const int gi = order[q];
    const LsJob J = jobs[gi];
    ls_graph(J, Pc, Pg, &out[gi]);
    if (lane == 0) bytes += (unsigned long long)J.n * 69 + (unsigned long long)(J.off[J.n] - J.off[0]) * 9;
  }
  if (lane == 0 && bytes) atomicAdd(&d_alg_bytes[F_LISTSCHED], bytes);
}

}  // namespace gp
