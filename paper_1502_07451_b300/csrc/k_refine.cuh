// k_refine.cuh -- uncoarsening: projection, balance round, synchronous gain rounds.
//
// gain(v) = W(v, other side) - W(v, own side).  Gain round r moves vertices from side r mod 2: the
// candidates are that side's vertices with gain > 0; in (gain desc, id asc) order, the longest
// prefix whose added weight keeps the destination within its bound moves, all at once.  A balance
// round (only when the split is infeasible) orders all of the over-bound side's vertices the same
// way and moves the shortest prefix that brings that side within its bound while the other side
// stays within its bound, else the longest prefix that keeps the other side within its bound.
// Rounds stop after two consecutive rounds without moves.
//
// The ordered prefix is found without sorting: the candidates' keys
// ((gmax - gain) << idbits | id, unique, ascending = gain desc, id asc) are radix-selected by
// their cumulative weight (8-bit digits, most significant first) in one CTA.  All round control
// lives in a device block (Ctl), so a level's rounds run without host round trips: the levels of a
// partition go through three launches of k_refine_tail (one CTA, one cluster, one cooperative grid,
// by level size), and the launch-per-step kernels (whose rounds after the stop return at once)
// remain for devices without cooperative launch.  Fixed vertices (g.fix) are never candidates.
#pragma once
#include "gp_internal.cuh"
#include "k_coarsen.cuh"
#include "k_makespan.cuh"  // grid_wait_bounded

namespace gp {

typedef unsigned __int128 u128;

struct CandCounters {
  unsigned long long ncand;
  unsigned long long cost_dst, cost_src;
  long long gmax, gmin;
};

// device control block of one partition call
struct Ctl {
  long long BC, BG, LC, LG;
  CandCounters cc[2];          // candidates of the current round, double-buffered by round parity
  int32_t sel_round;           // round whose selection ran last (-1 balance, -2 none)
  int32_t accept;              // 0 none, 1 all, 2 keys below thr
  unsigned long long thr_hi, thr_lo;
  long long sel_gmax;
  int32_t idbits, side_src;
  int32_t done, streak, rounds, balanced, bal_active, pad;
  long long moves, bal_moves, take;
  unsigned long long ndirty[2];  // vertices whose gain a round's moves changed, double-buffered
  long long sLC, sLG;            // the loads at the start of a round (the grid refinement's local selection)
};

struct Cands {
  int32_t* id;
  long long* gain;
  long long* cd;  // weight joining the destination
  long long* cs;  // weight leaving the source
  long long* gainv;   // current gain of every vertex of the level
  int32_t* stamp;     // round tag of the last round whose moves made the vertex's gain stale
  int32_t* dirty[2];  // the vertices stamped by a round, double-buffered by round parity
};

// tag of round r (-1 = balance) at level l; stamps start at -1
__host__ __device__ __forceinline__ int32_t round_tag(int level, int r) { return (level << 4) | (r + 2); }

__device__ __forceinline__ u128 cand_key(long long gmax, long long gain, int32_t id, int idbits) {
  return ((u128)(unsigned long long)(gmax - gain) << idbits) | (u128)(uint32_t)id;
}

// The round bodies below take the calling thread's index and the thread count of the range that
// shares the work: the whole grid for the single-graph kernels, one CTA in the batch path (where
// the control block lives in shared memory).
__device__ void ref_loads(const LevelGraph& g, const uint8_t* __restrict__ part, Ctl* ctl, int64_t tid,
                          int64_t stride) {
  __shared__ long long sh[32];
  long long c = 0, gg = 0;
  for (int64_t v = tid; v < g.n; v += stride) {
    if (part[v] == 0)
      c += g.vC[v];
    else
      gg += g.vG[v];
  }
  c = block_sum<long long>(c, sh);
  gg = block_sum<long long>(gg, sh);
  if (threadIdx.x == 0) {
    if (c) atomicAdd((unsigned long long*)&ctl->LC, (unsigned long long)c);
    if (gg) atomicAdd((unsigned long long*)&ctl->LG, (unsigned long long)gg);
  }
}
__global__ void k_ref_loads(LevelGraph g, const uint8_t* __restrict__ part, Ctl* ctl) {
  ref_loads(g, part, ctl, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

__device__ __forceinline__ void reset_counters(CandCounters& c) {
  c.ncand = 0;
  c.cost_dst = 0;
  c.cost_src = 0;
  c.gmax = LLONG_MIN;
  c.gmin = LLONG_MAX;
}

__device__ void ref_begin(Ctl* ctl, int idbits) {  // one thread
  Ctl& c = *ctl;
  c.done = 0;
  c.streak = 0;
  c.rounds = 0;
  c.balanced = 0;
  c.moves = 0;
  c.bal_moves = 0;
  c.sel_round = -2;
  c.idbits = idbits;
  c.ndirty[0] = 0;
  c.ndirty[1] = 0;
  reset_counters(c.cc[0]);
  reset_counters(c.cc[1]);
  const bool overC = c.LC > c.BC, overG = c.LG > c.BG;
  c.bal_active = (overC || overG) ? 1 : 0;
  if (overC && overG) {
    const __int128 lhs = (__int128)(c.LC - c.BC) * (__int128)c.BG;
    const __int128 rhs = (__int128)(c.LG - c.BG) * (__int128)c.BC;
    c.side_src = (lhs >= rhs) ? 0 : 1;
  } else {
    c.side_src = overC ? 0 : 1;
  }
}
__global__ void k_ref_begin(Ctl* ctl, int idbits) { ref_begin(ctl, idbits); }

// gain of every vertex (a group of G lanes per row), once per level
template <int G>
__device__ void gain_all(const LevelGraph& g, const uint8_t* __restrict__ part, long long* __restrict__ gainv,
                         int64_t tid, int64_t stride, int fam = F_GAIN) {
  __shared__ unsigned long long sacc[32];
  const int64_t group = tid / G, ngroups = stride / G;
  const int sub = threadIdx.x % G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G));
  unsigned long long bytes = 0;
  const int64_t nfull = (g.n + ngroups - 1) / ngroups * ngroups;  // every group runs the same trips
  for (int64_t v = group; v < nfull; v += ngroups) {
    long long acc = 0;
    if (v < g.n) {
      const uint8_t p = part[v];
      const int64_t b = g.start[v];
      const int32_t d = g.deg[v];
      for (int32_t k0 = sub; k0 < d; k0 += 4 * G) {  // four entries per lane in flight
        int32_t us[4];
        long long ws[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int32_t k = k0 + q * G;
          us[q] = k < d ? g.adj[b + k] : -1;
          ws[q] = k < d ? g.W[b + k] : 0;
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (us[q] >= 0 && GP_IN(us[q], g.n, 6)) acc += (part[us[q]] == p) ? -ws[q] : ws[q];
      }
      if (sub == 0) bytes += 21ull + 13ull * (unsigned long long)d;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(gmask, acc, o, G);
    if (v < g.n && sub == 0) gainv[v] = acc;
  }
  account(fam, bytes, sacc);
}
template <int G>
__global__ void __launch_bounds__(256)
    k_gain_all(LevelGraph g, const uint8_t* __restrict__ part, long long* __restrict__ gainv) {
  gain_all<G>(g, part, gainv, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

__device__ __forceinline__ void push_cand(CandCounters* cc, const Cands& cand, int32_t v, long long gain,
                                          long long cdv, long long csv, unsigned long long& sum_cd,
                                          unsigned long long& sum_cs, long long& gmax, long long& gmin) {
  const unsigned long long slot = atomicAdd(&cc->ncand, 1ull);
  cand.id[slot] = v;
  cand.gain[slot] = gain;
  cand.cd[slot] = cdv;
  cand.cs[slot] = csv;
  sum_cd += (unsigned long long)cdv;
  sum_cs += (unsigned long long)csv;
  gmax = gain > gmax ? gain : gmax;
  gmin = gain < gmin ? gain : gmin;
}

// Candidates of round r (-1 = balance): from the stored gains, except for the vertices the previous
// round's moves made stale (stamp == prev_tag), whose gains are recomputed here by a warp each and
// stored back.  Both parts write disjoint vertices.
__device__ void ref_cands(const LevelGraph& g, const uint8_t* __restrict__ part, Ctl* ctl, int r, int32_t prev_tag,
                          const Cands& cand, int64_t tid, int64_t stride, int fam = F_GAIN) {
  __shared__ long long sh[32];
  __shared__ unsigned long long shu[32];
  __shared__ unsigned long long sacc[32];
  __shared__ int s_src, s_skip;
  __shared__ unsigned long long s_nd;
  if (threadIdx.x == 0) {
    s_skip = (r < 0) ? !ctl->bal_active : ctl->done;
    s_src = (r < 0) ? ctl->side_src : (r & 1);
    s_nd = (r < 0) ? 0ull : ctl->ndirty[r & 1];
  }
  __syncthreads();
  if (s_skip) return;
  const int src = s_src;
  const int par = (r < 0) ? 1 : (r & 1);
  CandCounters* cc = &ctl->cc[par];
  const int64_t* cdst = src == 0 ? g.vG : g.vC;
  const int64_t* csrc = src == 0 ? g.vC : g.vG;
  unsigned long long sum_cd = 0, sum_cs = 0, bytes = 0;
  long long gmax = LLONG_MIN, gmin = LLONG_MAX;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  // whole warps step together (v = warp base + lane), so that a warp reserves its candidates' slots
  // with one atomic
  for (int64_t vb = tid - lane; vb < g.n; vb += stride) {
    const int64_t v = vb + lane;
    bool want = false;
    long long gain = 0;
    if (v < g.n) {
      bytes += 1;
      if (part[v] == src) {
        bytes += 12;
        if (cand.stamp[v] != prev_tag) {  // stale ones are recomputed below
          gain = cand.gainv[v];
          want = (r < 0 || gain > 0) && !(g.fix && g.fix[v] >= 0);  // a fixed vertex never moves
        }
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) continue;
    unsigned long long slot0 = 0;
    if (lane == __ffs(m) - 1) slot0 = atomicAdd(&cc->ncand, (unsigned long long)__popc(m));
    slot0 = __shfl_sync(0xffffffffu, slot0, __ffs(m) - 1);
    if (want) {
      const unsigned long long slot = slot0 + __popc(m & lt);
      const long long cdv = cdst[v], csv = csrc[v];
      cand.id[slot] = (int32_t)v;
      cand.gain[slot] = gain;
      cand.cd[slot] = cdv;
      cand.cs[slot] = csv;
      sum_cd += (unsigned long long)cdv;
      sum_cs += (unsigned long long)csv;
      gmax = gain > gmax ? gain : gmax;
      gmin = gain < gmin ? gain : gmin;
      bytes += 44;
    }
  }
  const int32_t* dl = cand.dirty[(r < 0) ? 0 : (r & 1)];
  for (int64_t k = tid >> 5; k < (int64_t)s_nd; k += stride >> 5) {
    const int32_t v = dl[k];
    const uint8_t p = part[v];
    const int64_t b = g.start[v];
    const int32_t d = g.deg[v];
    long long acc = 0;
    for (int32_t q = lane; q < d; q += 32) {
      const long long w = g.W[b + q];
      const int32_t u = g.adj[b + q];
      if (GP_IN(u, g.n, 7)) acc += (part[u] == p) ? -w : w;
    }
    acc = warp_sum64(acc);
    if (lane == 0) {
      cand.gainv[v] = acc;
      bytes += 29ull + 13ull * (unsigned long long)d;
      if (p == src && (r < 0 || acc > 0) && !(g.fix && g.fix[v] >= 0)) {
        push_cand(cc, cand, v, acc, cdst[v], csrc[v], sum_cd, sum_cs, gmax, gmin);
        bytes += 44;
      }
    }
  }
  sum_cd = block_sum<unsigned long long>(sum_cd, shu);
  sum_cs = block_sum<unsigned long long>(sum_cs, shu);
  {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long a = __shfl_xor_sync(0xffffffffu, gmax, o);
      const long long b = __shfl_xor_sync(0xffffffffu, gmin, o);
      gmax = a > gmax ? a : gmax;
      gmin = b < gmin ? b : gmin;
    }
    if (lane == 0) sh[threadIdx.x >> 5] = gmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long mx = LLONG_MIN;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) mx = sh[w] > mx ? sh[w] : mx;
      if (mx != LLONG_MIN) atomicMax(&cc->gmax, mx);
    }
    __syncthreads();
    if (lane == 0) sh[threadIdx.x >> 5] = gmin;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long mn = LLONG_MAX;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) mn = sh[w] < mn ? sh[w] : mn;
      if (mn != LLONG_MAX) atomicMin(&cc->gmin, mn);
      if (sum_cd) atomicAdd(&cc->cost_dst, sum_cd);
      if (sum_cs) atomicAdd(&cc->cost_src, sum_cs);
    }
  }
  account(fam, bytes, sacc);
}
__global__ void __launch_bounds__(256)
    k_ref_cands(LevelGraph g, const uint8_t* __restrict__ part, Ctl* ctl, int r, int32_t prev_tag, Cands cand) {
  ref_cands(g, part, ctl, r, prev_tag, cand, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
            (int64_t)gridDim.x * blockDim.x);
}

// Among the candidates in key order, the first one at which the running weight exceeds T (T >= 0).
// which: 0 = destination weight, 1 = source weight, 2 = one per candidate.
// Returns 1 and its key / rank (candidates with smaller keys) in shared memory, else 0.
struct SelOut {
  int found;
  u128 key;
  long long rank;
};

__device__ void block_select(const Cands& cand, unsigned long long N, int which, long long T, long long gmax,
                             int idbits, int keybits, SelOut* out, unsigned long long* hw,
                             unsigned long long* hc) {
  __shared__ u128 s_prefix;
  __shared__ long long s_T, s_rank;
  __shared__ int s_found;
  const int KB = ((keybits + 7) / 8) * 8;
  if (threadIdx.x == 0) {
    s_prefix = 0;
    s_T = T;
    s_rank = 0;
    s_found = 1;
  }
  __syncthreads();
  for (int shift = KB - 8; shift >= 0; shift -= 8) {
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
      hw[d] = 0;
      hc[d] = 0;
    }
    __syncthreads();
    const u128 prefix = s_prefix;
    for (unsigned long long i = threadIdx.x; i < N; i += blockDim.x) {
      const u128 k = cand_key(gmax, cand.gain[i], cand.id[i], idbits);
      if ((k >> (shift + 8)) != prefix) continue;
      const int d = (int)((k >> shift) & 255);
      const unsigned long long w = which == 0 ? (unsigned long long)cand.cd[i]
                                   : which == 1 ? (unsigned long long)cand.cs[i] : 1ull;
      atomicAdd(&hw[d], w);
      atomicAdd(&hc[d], 1ull);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long cum = 0;
      int chosen = -1;
      for (int d = 0; d < 256; d++) {
        if (cum + (long long)hw[d] > s_T) {
          chosen = d;
          break;
        }
        cum += (long long)hw[d];
        s_rank += (long long)hc[d];
      }
      if (chosen < 0) {
        s_found = 0;
      } else {
        s_T -= cum;
        s_prefix = (s_prefix << 8) | (u128)chosen;
      }
    }
    __syncthreads();
    if (!s_found) break;
  }
  if (threadIdx.x == 0) {
    out->found = s_found;
    out->key = s_prefix;
    out->rank = s_rank;
  }
  __syncthreads();
}

__device__ __forceinline__ int bits_of(unsigned long long x) {  // bits needed to hold x (>= 1)
  return x == 0 ? 1 : 64 - __clzll((long long)x);
}

__device__ void ref_select(Ctl* ctl, int r, const Cands& cand) {  // one block
  __shared__ unsigned long long hw[256], hc[256];
  __shared__ SelOut so;
  __shared__ int s_skip;
  Ctl& c = *ctl;
  if (threadIdx.x == 0) s_skip = (r < 0) ? !c.bal_active : c.done;
  __syncthreads();
  if (s_skip) return;
  const int par = (r < 0) ? 1 : (r & 1);
  const CandCounters cc = c.cc[par];
  const unsigned long long N = cc.ncand;
  const int idbits = c.idbits;
  const long long gmax = cc.gmax;
  const int keybits = N ? bits_of((unsigned long long)(cc.gmax - cc.gmin)) + idbits : 1;
  long long k = 0;
  int accept = 0;  // 0 none, 1 all, 2 below threshold
  u128 thr = 0;
  if (r >= 0) {
    const int dst = 1 - (r & 1);
    const long long Ld = dst == 0 ? c.LC : c.LG, Bd = dst == 0 ? c.BC : c.BG;
    if (N == 0 || Ld > Bd) {
      k = 0;
    } else if ((long long)cc.cost_dst <= Bd - Ld) {
      k = (long long)N;
      accept = 1;
    } else {
      block_select(cand, N, 0, Bd - Ld, gmax, idbits, keybits, &so, hw, hc);
      k = so.rank;
      thr = so.key;
      accept = k > 0 ? 2 : 0;
    }
  } else {
    const int s = c.side_src;
    const long long Ls = s == 0 ? c.LC : c.LG, Bs = s == 0 ? c.BC : c.BG;
    const long long Lo = s == 0 ? c.LG : c.LC, Bo = s == 0 ? c.BG : c.BC;
    const long long E = Ls - Bs;  // > 0
    const long long INF = LLONG_MAX;
    long long k1 = INF, k2;
    if ((long long)cc.cost_src >= E && N > 0) {
      block_select(cand, N, 1, E - 1, gmax, idbits, keybits, &so, hw, hc);
      k1 = so.rank + 1;
    }
    const long long T2 = Bo - Lo;
    if (T2 < 0) {
      k2 = -1;
    } else if ((long long)cc.cost_dst <= T2) {
      k2 = (long long)N;
    } else {
      block_select(cand, N, 0, T2, gmax, idbits, keybits, &so, hw, hc);
      k2 = so.rank;
    }
    k = (k1 <= k2) ? k1 : (k2 > 0 ? k2 : 0);
    if (k == 0) {
      accept = 0;
    } else if (k == (long long)N) {
      accept = 1;
    } else {
      block_select(cand, N, 2, k, gmax, idbits, keybits, &so, hw, hc);  // the candidate of rank k
      thr = so.key;
      accept = 2;
    }
  }
  if (threadIdx.x == 0) {
    c.sel_round = r;
    c.accept = accept;
    c.thr_hi = (unsigned long long)(thr >> 64);
    c.thr_lo = (unsigned long long)thr;
    c.sel_gmax = gmax;
    c.take = k;
    if (r >= 0) {
      c.rounds += 1;
      c.moves += k;
      c.streak = (k == 0) ? c.streak + 1 : 0;
      if (c.streak == 2) c.done = 1;
      reset_counters(c.cc[par ^ 1]);  // the next round's counters (last read by round r-1)
      c.ndirty[(r + 1) & 1] = 0;      // this round's apply stamps into it (last read by round r-1)
    } else {
      c.balanced = 1;
      c.bal_moves = k;
      c.ndirty[0] = 0;
    }
  }
}
__global__ void __launch_bounds__(1024) k_ref_select(Ctl* ctl, int r, Cands cand) { ref_select(ctl, r, cand); }

// A round's selection as the moves need it.
struct SelParams {
  int go, accept, src, idbits;
  unsigned long long N, hi, lo;
  long long gmax;
};

__device__ void ref_apply_body(const SelParams sp, Ctl* ctl, int r, const LevelGraph& g, uint8_t* __restrict__ part,
                               int32_t tag, const Cands& cand, int64_t tid, int64_t stride, int fam);

__device__ void ref_apply(Ctl* ctl, int r, const LevelGraph& g, uint8_t* __restrict__ part, int32_t tag,
                          const Cands& cand, int64_t tid, int64_t stride, int fam = F_APPLY) {
  __shared__ SelParams s_sp;
  if (threadIdx.x == 0) {
    const Ctl& c = *ctl;
    s_sp.go = (c.sel_round == r) && c.accept != 0;
    s_sp.accept = c.accept;
    s_sp.src = (r < 0) ? c.side_src : (r & 1);
    s_sp.idbits = c.idbits;
    s_sp.N = c.cc[(r < 0) ? 1 : (r & 1)].ncand;
    s_sp.hi = c.thr_hi;
    s_sp.lo = c.thr_lo;
    s_sp.gmax = c.sel_gmax;
  }
  __syncthreads();
  const SelParams sp = s_sp;
  ref_apply_body(sp, ctl, r, g, part, tag, cand, tid, stride, fam);
}

// Moves the accepted candidates and stamps them and their neighbours as stale for the next round
// (a warp per candidate; atomicExch on the stamp lists each stale vertex once).  sp is the same in
// every thread.
__device__ void ref_apply_body(const SelParams sp, Ctl* ctl, int r, const LevelGraph& g, uint8_t* __restrict__ part,
                               int32_t tag, const Cands& cand, int64_t tid, int64_t stride, int fam) {
  __shared__ long long sh[32];
  __shared__ unsigned long long sacc[32];
  if (!sp.go) return;
  const int s_accept = sp.accept, s_src = sp.src, s_idbits = sp.idbits;
  const unsigned long long s_N = sp.N, s_hi = sp.hi, s_lo = sp.lo;
  const long long s_gmax = sp.gmax;
  const int dst = 1 - s_src;
  const u128 thr = ((u128)s_hi << 64) | (u128)s_lo;
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  unsigned long long* nd = &ctl->ndirty[(r + 1) & 1];
  int32_t* dl = cand.dirty[(r + 1) & 1];
  long long dC = 0, dG = 0;
  unsigned long long bytes = 0;
  const int64_t gw = tid >> 5;
  const int64_t nw = stride >> 5;
  for (int64_t i = gw; i < (int64_t)s_N; i += nw) {
    const int32_t v = cand.id[i];
    if (s_accept == 2 && !(cand_key(s_gmax, cand.gain[i], v, s_idbits) < thr)) continue;
    if (lane == 0) {
      part[v] = (uint8_t)dst;
      const long long c = g.vC[v], gg = g.vG[v];
      if (dst == 1) {
        dC -= c;
        dG += gg;
      } else {
        dC += c;
        dG -= gg;
      }
      if (atomicExch(&cand.stamp[v], tag) != tag) dl[atomicAdd(nd, 1ull)] = v;
      bytes += 29;
    }
    const int64_t b = g.start[v];
    const int32_t d = g.deg[v];
    for (int32_t qb = 0; qb < d; qb += 32) {  // the warp reserves its new stale entries with one atomic
      const int32_t q = qb + lane;
      int32_t u = -1;
      bool fresh = false;
      if (q < d) {
        u = g.adj[b + q];
        fresh = GP_IN(u, g.n, 8) && atomicExch(&cand.stamp[u], tag) != tag;
      }
      const unsigned m = __ballot_sync(0xffffffffu, fresh);
      if (!m) continue;
      unsigned long long p0 = 0;
      if (lane == __ffs(m) - 1) p0 = atomicAdd(nd, (unsigned long long)__popc(m));
      p0 = __shfl_sync(0xffffffffu, p0, __ffs(m) - 1);
      if (fresh) dl[p0 + __popc(m & lt)] = u;
    }
    if (lane == 0) bytes += 12ull + 8ull * (unsigned long long)d;
  }
  dC = block_sum<long long>(dC, sh);
  dG = block_sum<long long>(dG, sh);
  if (threadIdx.x == 0) {
    if (dC) atomicAdd((unsigned long long*)&ctl->LC, (unsigned long long)dC);
    if (dG) atomicAdd((unsigned long long*)&ctl->LG, (unsigned long long)dG);
  }
  account(fam, bytes, sacc);
}
__global__ void __launch_bounds__(256)
    k_ref_apply(Ctl* ctl, int r, LevelGraph g, uint8_t* __restrict__ part, int32_t tag, Cands cand) {
  ref_apply(ctl, r, g, part, tag, cand, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
            (int64_t)gridDim.x * blockDim.x);
}

// per-level record: rounds, moves, balanced, balance moves
__global__ void k_ref_end(const Ctl* ctl, int level, int32_t* t_rounds, long long* t_moves, int32_t* t_bal,
                          long long* t_balmoves) {
  t_rounds[level] = ctl->rounds;
  t_moves[level] = ctl->moves;
  t_bal[level] = ctl->balanced;
  t_balmoves[level] = ctl->bal_moves;
}

__global__ void k_project(int64_t n, const int32_t* __restrict__ cmap, const uint8_t* __restrict__ pc,
                          uint8_t* __restrict__ pf) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    pf[v] = pc[cmap[v]];
}

static inline int idbits_for(int64_t n) {
  int b = 1;
  while (b < 31 && (int64_t(1) << b) < n) b++;
  return b;
}

void project(int64_t n, const int32_t* cmap, const uint8_t* part_c, uint8_t* part_f, cudaStream_t s) {
  GP_LAUNCH(F_PROJECT, k_project, grid_for(n, 256), 256, 0, s, n, cmap, part_c, part_f);
  GP_CHECK_LAUNCH();
}

// zero LC / LG and recompute them from part
void refine_loads(const LevelGraph& g, const uint8_t* part, Ctl* ctl, cudaStream_t s) {
  GP_CUDA(cudaMemsetAsync(&ctl->LC, 0, 2 * sizeof(long long), s));
  GP_LAUNCH(F_MISC, k_ref_loads, grid_for(g.n, 256, 4), 256, 0, s, g, part, ctl);
  GP_CHECK_LAUNCH();
}

static inline int group_for_degree(double avg) {
  if (avg <= 3.0) return 2;
  if (avg <= 6.0) return 4;
  if (avg <= 12.0) return 8;
  if (avg <= 24.0) return 16;
  return 32;
}

// The coarse end of the uncoarsening in ONE CTA: levels hi (the coarsest) down to lo, each projected
// from the level above (except hi), then refined exactly as refine_level_run does (the same round
// bodies over the CTA's threads, __syncthreads() between steps, and no rounds after the stop), and its
// record written.  Replaces ~31 launches per level where the levels are small.
constexpr int kTailMaxLevels = 48;
constexpr int64_t kTailMaxVertices = 4096;  // measured on the 1M workload: 2,048-4,096 best (12.56 vs 13.07 ms)
constexpr int64_t kClusterTailMaxVertices = 16384;  // one cluster up to here (1M workload: 10.95 -> 10.81 ms;
                                                     // 65,536 measured slower, 11.26 ms)
struct TailLevel {
  LevelGraph g;
  const int32_t* cmap;  // level l -> level l + 1 (unused at hi)
  uint8_t* part;
  int32_t G;            // lanes per row of the gain pass
  int32_t idbits;
};
struct TailArgs {
  int32_t lo, hi;
  const uint8_t* top_part;        // split of level hi + 1, projected onto level hi (null: hi is the coarsest)
  TailLevel lev[kTailMaxLevels];  // lev[l - lo]
};

// MODE kTailCluster: the same over one thread-block cluster (the cluster's threads share each step, the
// cluster barrier separates the steps, the one-block selection runs in rank 0), for levels a little
// larger.  MODE kTailGrid: the same over a cooperative grid (one CTA per SM at most, all resident), for
// the large levels: a grid barrier of its own separates the steps (a counter that every CTA increments
// and polls, the wait bounded by the global timer at 0.5 s; on expiry the CTA stops, sets *err, and the
// other CTAs' waits then expire too), replacing ~31 launches per level.
constexpr int kTailCta = 0, kTailCluster = 1, kTailGrid = 2;

__device__ __forceinline__ bool tail_grid_sync(unsigned* bar, unsigned& epoch, int* err) {
  __syncthreads();
  bool ok = true;
  epoch += 1;
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's writes before its arrival
    atomicAdd(bar, 1u);
    ok = grid_wait_bounded(bar, epoch * gridDim.x);
    if (!ok) atomicOr(err, 1);
    __threadfence();
  }
  return __syncthreads_or(!ok) == 0;
}

// Failure-path self-check of the grid barrier: CTA 1 returns without arriving, so CTA 0's wait runs out
// (0.5 s), sets *err and returns.
__global__ void k_grid_wait_selftest(unsigned* bar, int* err) {
  if (blockIdx.x != 0) return;
  unsigned epoch = 0;
  tail_grid_sync(bar, epoch, err);
}

template <int MODE>
__global__ void __launch_bounds__(1024, 1)
    k_refine_tail(TailArgs A, Ctl* ctl, Cands cand, int32_t* t_rounds, long long* t_moves, int32_t* t_bal,
                  long long* t_balmoves, unsigned* bar, int* err) {
  uint32_t rank = 0, nranks = 1;
  if (MODE == kTailCluster) {
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(nranks));
  } else if (MODE == kTailGrid) {
    rank = blockIdx.x;
    nranks = gridDim.x;
  }
  const int64_t tid = (int64_t)rank * blockDim.x + threadIdx.x, stride = (int64_t)nranks * blockDim.x;
  const bool lead = rank == 0 && threadIdx.x == 0;
  unsigned epoch = 0;
  auto sync = [&]() -> bool {
    if (MODE == kTailCluster) {
      cluster_sync();
      return true;
    }
    if (MODE == kTailGrid) return tail_grid_sync(bar, epoch, err);
    __syncthreads();
    return true;
  };
  for (int l = A.hi; l >= A.lo; l--) {
    const TailLevel& T = A.lev[l - A.lo];
    const LevelGraph& g = T.g;
    const uint8_t* pc = l < A.hi ? A.lev[l + 1 - A.lo].part : A.top_part;
    if (pc)
      for (int64_t v = tid; v < g.n; v += stride) T.part[v] = pc[T.cmap[v]];
    if (lead) ref_begin(ctl, T.idbits);
    if (!sync()) return;
    switch (T.G) {
      case 2: gain_all<2>(g, T.part, cand.gainv, tid, stride, F_REFINE); break;
      case 4: gain_all<4>(g, T.part, cand.gainv, tid, stride, F_REFINE); break;
      case 8: gain_all<8>(g, T.part, cand.gainv, tid, stride, F_REFINE); break;
      case 16: gain_all<16>(g, T.part, cand.gainv, tid, stride, F_REFINE); break;
      default: gain_all<32>(g, T.part, cand.gainv, tid, stride, F_REFINE); break;
    }
    if (!sync()) return;
    int32_t prev = round_tag(l, -2);
    for (int r = -1; r < kRefineRounds; r++) {
      if (MODE == kTailGrid && r >= 0 && lead) {
        // ahead of the selection (which may then run in every CTA): the next round's counters and stale
        // list (last used by the previous round), and the loads the selection compares against
        reset_counters(ctl->cc[(r & 1) ^ 1]);
        ctl->ndirty[(r + 1) & 1] = 0;
        ctl->sLC = ctl->LC;
        ctl->sLG = ctl->LG;
      }
      ref_cands(g, T.part, ctl, r, prev, cand, tid, stride, F_REFINE);
      if (!sync()) return;
      // a gain round whose selection takes all candidates or none needs no histogram: every CTA decides
      // it from the round's counters (unchanged until the next barrier), CTA 0 records it, and the moves
      // follow without the barrier a selection in one CTA needs
      bool local = false;
      SelParams sp{};
      if (MODE == kTailGrid && r >= 0) {
        const CandCounters* cc = &ctl->cc[r & 1];
        const unsigned long long N = __ldcg(&cc->ncand);
        const long long cost_dst = (long long)__ldcg(&cc->cost_dst);
        const int dst = 1 - (r & 1);
        const long long Ld = __ldcg(dst == 0 ? &ctl->sLC : &ctl->sLG);
        const long long Bd = dst == 0 ? ctl->BC : ctl->BG;
        long long k = -1;
        if (N == 0 || Ld > Bd)
          k = 0;
        else if (cost_dst <= Bd - Ld)
          k = (long long)N;
        if (k >= 0) {
          local = true;
          sp.go = k > 0;
          sp.accept = k > 0 ? 1 : 0;
          sp.src = r & 1;
          sp.idbits = ctl->idbits;
          sp.N = N;
          sp.gmax = __ldcg(&cc->gmax);
          if (lead) {  // what the one-CTA selection records for the same round
            Ctl& c = *ctl;
            c.sel_round = r;
            c.accept = sp.accept;
            c.thr_hi = 0;
            c.thr_lo = 0;
            c.sel_gmax = sp.gmax;
            c.take = k;
            c.rounds += 1;
            c.moves += k;
            c.streak = (k == 0) ? c.streak + 1 : 0;
            if (c.streak == 2) c.done = 1;
          }
        }
      }
      if (local) {
        ref_apply_body(sp, ctl, r, g, T.part, round_tag(l, r), cand, tid, stride, F_REFINE);
      } else {
        if (rank == 0) ref_select(ctl, r, cand);
        if (!sync()) return;
        ref_apply(ctl, r, g, T.part, round_tag(l, r), cand, tid, stride, F_REFINE);
      }
      if (!sync()) return;
      prev = round_tag(l, r);
      if (*(volatile int32_t*)&ctl->done) break;  // later rounds would return at once (uniform: read after the barrier)
    }
    if (lead) {
      t_rounds[l] = ctl->rounds;
      t_moves[l] = ctl->moves;
      t_bal[l] = ctl->balanced;
      t_balmoves[l] = ctl->bal_moves;
    }
    if (!sync()) return;
  }
}

// One level: gains of all vertices, then the balance round and up to 8 gain rounds, enqueued without
// host round trips (rounds after the stop return at once).  avg_deg selects the row group size.
void refine_level_run(const LevelGraph& g, uint8_t* part, Ctl* ctl, const Cands& cand, int level, double avg_deg,
                      cudaStream_t s) {
  const int64_t n = g.n;
  const unsigned vgrid = grid_for(n, 256, 8);
  const unsigned agrid = grid_for(n, 256, 4);
  const int G = group_for_degree(avg_deg * 0.25);  // about six row entries per lane (measured best)
  switch (G) {
#define GP_GA(GG) \
  case GG: GP_LAUNCH(F_GAIN, k_gain_all<GG>, grid_for(n * GG, 256), 256, 0, s, g, part, cand.gainv); break;
    GP_GA(2) GP_GA(4) GP_GA(8) GP_GA(16) GP_GA(32)
#undef GP_GA
  }
  GP_LAUNCH(F_MISC, k_ref_begin, 1, 1, 0, s, ctl, idbits_for(n));
  int32_t prev = round_tag(level, -2);  // no stale vertices before the balance round
  for (int r = -1; r < kRefineRounds; r++) {
    GP_LAUNCH(F_GAIN, k_ref_cands, vgrid, 256, 0, s, g, part, ctl, r, prev, cand);
    GP_LAUNCH(F_SELECT, k_ref_select, 1, 1024, 0, s, ctl, r, cand);
    GP_LAUNCH(F_APPLY, k_ref_apply, agrid, 256, 0, s, ctl, r, g, part, round_tag(level, r), cand);
    prev = round_tag(level, r);
  }
  GP_CHECK_LAUNCH();
}

// The levels of `ta` in one cooperative grid launch of k_refine_tail<kTailGrid> (one CTA of 1,024 threads per
// SM, all resident).  *bar and *err must be zero.  `wait_for` (nullable): work that may still hold SMs on
// another stream (a deferred creation's level traversal), waited for first.  Returns false, having
// launched nothing, where the device cannot hold the whole grid; the caller then runs a launch per step.
static bool launch_refine_grid(const TailArgs& ta, Ctl* ctl, const Cands& cand, int32_t* t_rounds,
                               long long* t_moves, int32_t* t_bal, long long* t_balmoves, unsigned* bar, int* err,
                               cudaEvent_t wait_for, cudaStream_t s) {
  static int grid_blocks = -1;  // resident CTAs of the grid (0: no cooperative launch)
  if (grid_blocks < 0) {
    int coop = 0, dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refine_tail<kTailGrid>, 1024, 0) ==
                    cudaSuccess)
      grid_blocks = per_sm > 0 ? num_sms() * per_sm : 0;
    else
      grid_blocks = 0;
    cudaGetLastError();
  }
  if (grid_blocks <= 0) return false;
  if (wait_for) GP_CUDA(cudaStreamWaitEvent(s, wait_for, 0));
  TailArgs a = ta;
  Ctl* c = ctl;
  Cands cd = cand;
  void* args[] = {(void*)&a, (void*)&c, (void*)&cd, (void*)&t_rounds, (void*)&t_moves,
                  (void*)&t_bal, (void*)&t_balmoves, (void*)&bar, (void*)&err};
  launch_begin(F_REFINE, s);
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_refine_tail<kTailGrid>, dim3(grid_blocks),
                                                    dim3(1024), args, 0, s);
  launch_end(F_REFINE, s);
  if (e != cudaSuccess) {  // no room for the whole grid (e.g. a shared or partitioned device)
    cudaGetLastError();
    grid_blocks = 0;
    return false;
  }
  return true;
}

}  // namespace gp
