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
//     holds its running task and its end time in registers;
//   - the waiting tasks of a side are an unordered array of (r, id) records; the next task to start
//     is found by a warp-wide scan and shuffle reduction (the records are 16 bytes, one vector load
//     per lane per 32 records), and taken out by moving the last record into its slot;
//   - when a task ends, the warp walks its out-row 32 entries at a time; lanes that hit the same
//     successor (parallel entries) are grouped with __match_any_sync, and the group's leader updates
//     the successor's {ready time, pending count} record (16 bytes, plain load and store: only this
//     warp touches the graph) and appends it to its side's waiting array once the count reaches 0.
// The result does not depend on the order in which tasks ending at the same time are processed, nor
// on which idle worker of a side takes a task.
#pragma once
#include "gp_internal.cuh"

namespace gp {

constexpr int kLsMaxWorkers = 32;  // workers of both sides together (one lane each)

struct __align__(16) LsRec {  // per vertex
  long long ready;   // r(v) so far (max over the predecessors that have ended)
  int pending;       // predecessors (in-entries) not ended yet
  int pad;
};
struct __align__(16) LsWait {  // a waiting task
  long long r;
  int v;
  int pad;
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

__device__ __forceinline__ bool ls_less(long long ra, int va, long long rb, int vb) {
  return ra < rb || (ra == rb && va < vb);
}

// Starts on one side at time t: while a worker of the side is idle (mine: this lane is one of the
// side's workers) and the waiting task with the smallest (r, id) has r <= t, it starts on the lowest
// idle worker.  On return, cand = that smallest r if a worker stayed idle and tasks wait (else
// unchanged).
__device__ __forceinline__ void ls_starts(LsWait* W, int& len, bool mine, long long t,
                                          const int32_t* cost, bool& busy, int& wtask, long long& wend,
                                          long long& ms, long long* fin, long long& cand) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    const unsigned idle = __ballot_sync(0xffffffffu, mine && !busy);
    if (!idle || len == 0) return;
    long long br = LLONG_MAX;
    int bv = INT_MAX, bi = -1;
    for (int i = lane; i < len; i += 32) {
      const LsWait x = W[i];
      if (ls_less(x.r, x.v, br, bv)) {
        br = x.r;
        bv = x.v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long r2 = __shfl_xor_sync(0xffffffffu, br, o);
      const int v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ls_less(r2, v2, br, bv)) {
        br = r2;
        bv = v2;
        bi = i2;
      }
    }
    if (br > t) {
      cand = br;
      return;
    }
    // take it out (the last record moves into its slot) and start it on the lowest idle worker
    if (lane == 0) {
      const int last = len - 1;
      if (bi != last) W[bi] = W[last];
    }
    len--;
    __syncwarp();
    if (lane == __ffs(idle) - 1) {
      busy = true;
      wtask = bv;
      wend = t + (long long)cost[bv];
      fin[bv] = wend;
      ms = wend > ms ? wend : ms;
    }
  }
}

// One warp, one graph.
__device__ void ls_graph(const LsJob& J, int Pc, int Pg, LsOut* out) {
  const int lane = threadIdx.x & 31;
  const int64_t n = J.n;
  int bad = 0;
  // records: pending = in-degree, ready = 0; sources into the waiting arrays
  int len0 = 0, len1 = 0;
  for (int64_t base = 0; base < n; base += 32) {
    const int64_t v = base + lane;
    bool src = false;
    int side = 0;
    if (v < n) {
      const int deg = (int)(J.in_off[v + 1] - J.in_off[v]);
      LsRec r;
      r.ready = 0;
      r.pending = deg;
      r.pad = 0;
      J.rec[v] = r;
      const uint8_t p = J.part[v];
      bad |= p > 1;
      side = p & 1;
      src = deg == 0;
    }
    const unsigned m0 = __ballot_sync(0xffffffffu, src && side == 0);
    const unsigned m1 = __ballot_sync(0xffffffffu, src && side == 1);
    const unsigned lt = (1u << lane) - 1u;
    if (src) {
      LsWait x;
      x.r = 0;
      x.v = (int)v;
      x.pad = 0;
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
  int wtask = -1;
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
    // ---- ends at or before t
    unsigned endm = __ballot_sync(0xffffffffu, is_worker && busy && wend <= t);
    while (endm) {
      const int wl = __ffs(endm) - 1;
      endm &= endm - 1;
      const int u = __shfl_sync(0xffffffffu, wtask, wl);
      const long long fu = __shfl_sync(0xffffffffu, wend, wl);
      if (lane == wl) busy = false;
      const uint8_t pu = J.part[u];
      const int64_t e0 = J.off[u], e1 = J.off[u + 1];
      for (int64_t b = e0; b < e1; b += 32) {
        const int64_t e = b + lane;
        const bool valid = e < e1;
        int v = -1;
        long long arrive = 0;
        uint8_t pv = 0;
        if (valid && GP_IN(J.cols[e], n, 13)) {
          v = J.cols[e];
          pv = J.part[v];
          arrive = fu + (pv != pu ? (long long)J.w[e] : 0ll);
        }
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
        long long rdy = 0;
        if (leader) {
          LsRec r = J.rec[v];
          r.ready = amax > r.ready ? amax : r.ready;
          r.pending -= cnt;
          J.rec[v] = r;
          released = r.pending == 0;
          rdy = r.ready;
        }
        const unsigned m0 = __ballot_sync(0xffffffffu, released && pv == 0);
        const unsigned m1 = __ballot_sync(0xffffffffu, released && pv == 1);
        const unsigned lt = (1u << lane) - 1u;
        if (released) {
          LsWait x;
          x.r = rdy;
          x.v = v;
          x.pad = 0;
          if (pv == 0)
            J.wait[len0 + __popc(m0 & lt)] = x;
          else
            J.wait[n + len1 + __popc(m1 & lt)] = x;
        }
        len0 += __popc(m0);
        len1 += __popc(m1);
        __syncwarp();  // the next chunk may update a successor this chunk updated
      }
    }
    // ---- starts at t, side by side; cand = the smallest waiting r of a side with an idle worker
    long long cand0 = kInf, cand1 = kInf;
    ls_starts(J.wait, len0, is_worker && wside == 0, t, J.cC, busy, wtask, wend, ms, J.fin, cand0);
    ls_starts(J.wait + n, len1, is_worker && wside == 1, t, J.cG, busy, wtask, wend, ms, J.fin, cand1);
    // ---- next time
    if (__any_sync(0xffffffffu, is_worker && busy && wend <= t)) continue;  // a task of cost 0 ended at t
    long long nx = (is_worker && busy) ? wend : kInf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long q = __shfl_xor_sync(0xffffffffu, nx, o);
      nx = q < nx ? q : nx;
    }
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
__global__ void __launch_bounds__(256) k_listsched(int count, const LsJob* __restrict__ jobs,
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
