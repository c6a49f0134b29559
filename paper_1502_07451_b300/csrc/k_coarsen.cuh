// k_coarsen.cuh -- coarsening: handshake heavy-edge matching, two-hop pairing, contraction.
//
// Matching round (synchronous): every unmatched vertex v picks, among its unmatched neighbours u
// whose merged weights stay within the caps, the edge with the largest key
// (W desc, h(seed, min, max) desc, min asc, max asc); v and u match when they picked each other.
// Two-hop pairing: each vertex still unmatched names its best neighbour under the same key (its
// anchor); walking each anchor's row in ascending neighbour order, consecutive anchored vertices
// are paired unless their merged weights exceed the caps (a failed pair leaves the newer one
// pending).  Contraction: representatives (unmatched vertices and the smaller end of each pair)
// are numbered in vertex order; a coarse row is the union of both members' rows mapped through
// cmap, without the coarse vertex itself, equal neighbours added up.
// Fixed vertices (g.fix non-null): two vertices pinned to different sides never merge, in either
// step; a coarse vertex is pinned where one of its members is.
#pragma once
#include "gp_internal.cuh"
#include "k_graph.cuh"
#include "k_rows.cuh"
#include "k_scan.cuh"

namespace gp {

__global__ void k_match_init(int64_t n, const int64_t* __restrict__ vC, const int64_t* __restrict__ vG,
                             int64_t capC, int64_t capG, int32_t* __restrict__ mate,
                             int32_t* __restrict__ pick, uint8_t* __restrict__ alive) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    mate[v] = -1;
    pick[v] = -1;
    // a vertex over a cap on its own can never merge (weights are >= 0)
    alive[v] = (vC[v] <= capC && vG[v] <= capG) ? 1 : 0;
  }
}

// max vertex weights of the level (vC, vG >= 0): a vertex v with vC[v] + maxC <= capC and
// vG[v] + maxG <= capG fits the caps with any neighbour, so its picks skip the weight gathers.
__global__ void k_max_weights(int64_t n, const int64_t* __restrict__ vC, const int64_t* __restrict__ vG,
                              long long* mx) {
  long long a = 0, b = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    a = vC[v] > a ? vC[v] : a;
    b = vG[v] > b ? vG[v] : b;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long x = __shfl_xor_sync(0xffffffffu, a, o), y = __shfl_xor_sync(0xffffffffu, b, o);
    a = x > a ? x : a;
    b = y > b ? y : b;
  }
  if ((threadIdx.x & 31) == 0) {
    if (a) atomicMax(&mx[0], a);
    if (b) atomicMax(&mx[1], b);
  }
}

__device__ __forceinline__ EdgeKey group_best_key(EdgeKey k, unsigned gmask, int G) {
  for (int o = G / 2; o > 0; o >>= 1) {
    EdgeKey q;
    q.W = __shfl_xor_sync(gmask, k.W, o, G);
    q.h = __shfl_xor_sync(gmask, k.h, o, G);
    q.nm = __shfl_xor_sync(gmask, k.nm, o, G);
    if (key_better(q, k)) k = q;
  }
  return k;
}

__device__ __forceinline__ unsigned group_mask(int G) {
  return (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G));
}

// Running best edge of one lane under the matching key.  Edge weights are compared first; the
// tie-break hash is computed only when two offered edges have equal W (rare for summed weights).
struct LazyKey {
  int64_t W = -1;  // -1: nothing offered (weights are >= 0)
  uint32_t u = 0;
  bool hashed = false;
  EdgeKey k;
  __device__ __forceinline__ void offer(int64_t w, uint32_t uu, uint64_t seed, uint32_t v) {
    if (w > W) {
      W = w;
      u = uu;
      hashed = false;
    } else if (w == W) {
      if (!hashed) {
        k = make_key(W, seed, v, u);
        hashed = true;
      }
      const EdgeKey kn = make_key(w, seed, v, uu);
      if (key_better(kn, k)) {
        k = kn;
        u = uu;
      }
    }
  }
  __device__ __forceinline__ EdgeKey key(uint64_t seed, uint32_t v) const {
    if (W < 0) return key_none();
    return hashed ? k : make_key(W, seed, v, u);
  }
};

// One handshake round, picks: a group of G lanes per unmatched vertex.  `tid` / `stride`: the
// calling thread and the number of threads sharing the level (grid or one CTA).  Returns, per
// thread, whether it recorded a pick.  FIX: g.fix is set (a separate instance: the check costs the
// plain picks 10 registers).
template <int G, bool FIX = false, bool LIST = false>
__device__ bool match_pick(const LevelGraph& g, int64_t capC, int64_t capG, uint64_t seed, long long mC, long long mG,
                           const int32_t* __restrict__ mate, int32_t* __restrict__ pick,
                           uint8_t* __restrict__ alive, int64_t tid, int64_t stride, bool all_free = false,
                           const int32_t* __restrict__ list = nullptr, int64_t count = 0) {
  __shared__ unsigned long long sacc[32];
  const int64_t group = tid / G, ngroups = stride / G;
  const int sub = threadIdx.x % G;
  const unsigned gmask = group_mask(G);
  unsigned long long bytes = 0;
  bool picked = false;
  // every vertex, or (LIST) the vertices of `list`: those still unmatched and alive after the previous round
  const int64_t nv = LIST ? count : g.n;
  for (int64_t i = group; i < nv; i += ngroups) {
    const int64_t v = LIST ? (int64_t)list[i] : i;
    if (sub == 0) bytes += LIST ? 9 : 5;
    if (mate[v] != -1 || !alive[v]) continue;  // same v across the group: uniform
    const int64_t b = g.start[v];
    const int32_t d = g.deg[v];
    const int64_t cv = g.vC[v], gv = g.vG[v];
    const bool nocap = cv + mC <= capC && gv + mG <= capG;
    const int8_t fv = FIX ? g.fix[v] : (int8_t)-1;  // a free v is compatible with every neighbour
    LazyKey lk;
    // four entries per lane in flight: ids and weights, then the neighbours' match state
    for (int32_t k0 = sub; k0 < d; k0 += 4 * G) {
      int32_t us[4];
      int64_t ws[4];
      bool ok[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int32_t k = k0 + q * G;
        ok[q] = k < d;
        us[q] = ok[q] ? g.adj[b + k] : 0;
        ws[q] = ok[q] ? g.W[b + k] : 0;
        ok[q] = ok[q] && GP_IN(us[q], g.n, 1);
      }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        if (!ok[q]) continue;
        bytes += all_free ? 12 : 16;
        if (!all_free) ok[q] = mate[us[q]] == -1;  // the first round: nobody is matched yet
      }
      if (!nocap) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
          if (!ok[q]) continue;
          bytes += 16;
          ok[q] = cv + g.vC[us[q]] <= capC && gv + g.vG[us[q]] <= capG;
        }
      }
      if (FIX && fv >= 0) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
          if (!ok[q]) continue;
          bytes += 1;
          const int8_t fu = g.fix[us[q]];
          ok[q] = fu < 0 || fu == fv;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; q++)
        if (ok[q]) lk.offer(ws[q], (uint32_t)us[q], seed, (uint32_t)v);
    }
    const EdgeKey best = group_best_key(lk.key(seed, (uint32_t)v), gmask, G);
    if (sub == 0) {
      bytes += 12 + 16 + 4;
      if (best.W < 0) {
        pick[v] = -1;
        alive[v] = 0;  // no eligible neighbour now means none later: neighbours only get matched
      } else {
        pick[v] = key_other(best, (uint32_t)v);
        picked = true;
      }
    }
  }
  account(F_MATCH_PICK, bytes, sacc);
  return picked;
}
template <int G, bool FIX, bool LIST>
__global__ void __launch_bounds__(256, 5)  // 5 blocks per SM: at most 51 registers
    k_match_pick(LevelGraph g, int64_t capC, int64_t capG, uint64_t seed, const long long* __restrict__ maxw,
                 const int32_t* __restrict__ mate, int32_t* __restrict__ pick, uint8_t* __restrict__ alive,
                 int all_free, const int32_t* __restrict__ list, const unsigned* list_cnt) {
  match_pick<G, FIX, LIST>(g, capC, capG, seed, maxw[0], maxw[1], mate, pick, alive,
                           (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x,
                           all_free != 0, list, LIST ? (int64_t)*list_cnt : 0);
}

// Handshakes of a round: v and u are matched when each picked the other.  Over every vertex, or over
// `list_in` (launched with 256 threads); with `list_out`, the vertices that stay unmatched and alive
// (with keep_dead: every unmatched vertex, for the two-hop anchors) are appended there for the next
// round, whose picks then run on whole groups of such vertices instead of skipping the matched ones
// (the list's order does not matter: a pick depends only on the state at the start of its round).
__global__ void __launch_bounds__(256)
    k_match_confirm(int64_t n, int32_t* __restrict__ mate, const int32_t* __restrict__ pick,
                    const uint8_t* __restrict__ alive, const int32_t* __restrict__ list_in, const unsigned* cnt_in,
                    int32_t* __restrict__ list_out, unsigned* cnt_out, int keep_dead) {
  const int64_t nv = list_in ? (int64_t)*cnt_in : n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  // whole blocks (of 8 warps) step together, so that a block appends its survivors with one atomic
  __shared__ unsigned s_wc[8], s_base;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t bb = (int64_t)blockIdx.x * blockDim.x; bb < nv; bb += stride) {
    const int64_t i = bb + threadIdx.x;
    bool keep = false;
    int32_t v = -1;
    if (i < nv) {
      v = list_in ? list_in[i] : (int32_t)i;
      if (mate[v] == -1) {
        const int32_t u = pick[v];
        if (u >= 0 && GP_IN(u, n, 2) && pick[u] == v)
          mate[v] = u;
        else
          keep = keep_dead || alive[v] != 0;
      }
    }
    if (list_out) {
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) s_wc[wid] = __popc(m);
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned tot = 0;
        for (int q = 0; q < 8; q++) tot += s_wc[q];
        s_base = tot ? atomicAdd(cnt_out, tot) : 0;
      }
      unsigned before = 0;
      for (int q = 0; q < wid; q++) before += s_wc[q];
      __syncthreads();
      if (keep) list_out[s_base + before + __popc(m & lt)] = v;
      __syncthreads();  // s_wc and s_base are rewritten by the next step
    }
  }
}

// anchor of every unmatched vertex: its best neighbour under the matching key (no filters)
template <int G, bool LIST = false>
__device__ void match_anchor(const LevelGraph& g, uint64_t seed, const int32_t* __restrict__ mate,
                             int32_t* __restrict__ anchor, uint8_t* __restrict__ is_anchor, int64_t tid,
                             int64_t stride, int32_t* __restrict__ scnt = nullptr,
                             const int32_t* __restrict__ list = nullptr, int64_t count = 0) {
  __shared__ unsigned long long sacc[32];
  const int64_t group = tid / G, ngroups = stride / G;
  const int sub = threadIdx.x % G;
  const unsigned gmask = group_mask(G);
  unsigned long long bytes = 0;
  // every vertex, or (LIST) the vertices of `list`: the unmatched ones, whose anchors are still -1
  const int64_t nv = LIST ? count : g.n;
  for (int64_t i = group; i < nv; i += ngroups) {
    const int64_t v = LIST ? (int64_t)list[i] : i;
    if (!LIST && mate[v] != -1) {
      if (sub == 0) {
        anchor[v] = -1;
        bytes += 8;
      }
      continue;
    }
    const int64_t b = g.start[v];
    const int32_t d = g.deg[v];
    LazyKey lk;
    for (int32_t k0 = sub; k0 < d; k0 += 4 * G) {  // four entries per lane in flight
      int32_t us[4];
      int64_t ws[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int32_t k = k0 + q * G;
        us[q] = k < d ? g.adj[b + k] : -1;
        ws[q] = k < d ? g.W[b + k] : 0;
      }
#pragma unroll
      for (int q = 0; q < 4; q++)
        if (us[q] >= 0 && GP_IN(us[q], g.n, 3)) {
          lk.offer(ws[q], (uint32_t)us[q], seed, (uint32_t)v);
          bytes += 12;
        }
    }
    const EdgeKey best = group_best_key(lk.key(seed, (uint32_t)v), gmask, G);
    if (sub == 0) {
      bytes += 20;
      if (best.W < 0) {
        anchor[v] = -1;
      } else {
        const int32_t a = key_other(best, (uint32_t)v);
        anchor[v] = a;
        if (is_anchor) is_anchor[a] = 1;
        if (scnt) atomicAdd(&scnt[a], 1);  // the anchor's bucket size
      }
    }
  }
  account(F_TWOHOP, bytes, sacc);
}
template <int G, bool LIST>
__global__ void __launch_bounds__(256)
    k_anchor(LevelGraph g, uint64_t seed, const int32_t* __restrict__ mate, int32_t* __restrict__ anchor,
             uint8_t* __restrict__ is_anchor, int32_t* __restrict__ scnt, const int32_t* __restrict__ list,
             const unsigned* list_cnt) {
  match_anchor<G, LIST>(g, seed, mate, anchor, is_anchor, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                        (int64_t)gridDim.x * blockDim.x, scnt, list, LIST ? (int64_t)*list_cnt : 0);
}

// every anchored vertex into its anchor's bucket: sat[soff[a] .. soff[a + 1]) (in no particular order;
// scnt, the bucket sizes, counts down to zero)
__global__ void k_sat_scatter(int64_t n, const int32_t* __restrict__ anchor, const int64_t* __restrict__ soff,
                              int32_t* __restrict__ scnt, int32_t* __restrict__ sat) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = anchor[v];
    if (a >= 0) sat[soff[a] + atomicSub(&scnt[a], 1) - 1] = (int32_t)v;
  }
}

// Pairs the vertices anchored at h in ascending vertex order.  Sequentially: a vertex joins the
// pending one when the caps allow (pair formed, nothing pending), else it becomes pending.  With
// P_i = "item i is pending after its turn" and ok_i = "caps allow item i-1 with item i":
// P_i = !(P_{i-1} && ok_i), so P flips along runs of ok and resets to true where ok fails; item i is
// paired with item i-1 exactly when P_i is false.  A warp evaluates this 32 items at a time with a
// max-scan of the last reset position, carrying the last item across chunks.
// `items` holds the anchored vertices sorted ascending; `nitems` of them.
__device__ void pair_sorted(const LevelGraph& g, int64_t capC, int64_t capG, const int32_t* items, int64_t nitems,
                            int32_t* __restrict__ mate, unsigned long long& bytes) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  int32_t p_id = -1;  // carried last item
  int64_t p_c = 0, p_g = 0;
  int p_f = -1;
  bool p_pend = false;
  for (int64_t base = 0; base < nitems; base += 32) {
    const bool flag = base + lane < nitems;
    const int32_t v = flag ? items[base + lane] : -1;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    int64_t vc = 0, vg = 0;
    int vf = -1;
    if (flag) {
      vc = g.vC[v];
      vg = g.vG[v];
      bytes += 20;
      if (g.fix) vf = g.fix[v];
    }
    const unsigned below = m & lt;
    const int pred_lane = below ? 31 - __clz(below) : -1;
    const int srcl = pred_lane >= 0 ? pred_lane : lane;
    int32_t q_id = __shfl_sync(0xffffffffu, v, srcl);
    int64_t q_c = __shfl_sync(0xffffffffu, vc, srcl);
    int64_t q_g = __shfl_sync(0xffffffffu, vg, srcl);
    int q_f = __shfl_sync(0xffffffffu, vf, srcl);
    if (pred_lane < 0) {
      q_id = p_id;
      q_c = p_c;
      q_g = p_g;
      q_f = p_f;
    }
    const bool okprev = flag && q_id >= 0 && (q_c + vc <= capC) && (q_g + vg <= capG) &&
                        (q_f < 0 || vf < 0 || q_f == vf);
    const int sidx = __popc(below);
    int scan = (flag && !okprev) ? sidx : INT_MIN;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, scan, o);
      if (lane >= o) scan = y > scan ? y : scan;
    }
    const int r0 = (p_id >= 0 && p_pend) ? -1 : -2;
    const int lr = scan > r0 ? scan : r0;
    const bool P = ((sidx - lr) & 1) == 0;
    if (flag && !P) {
      mate[v] = q_id;
      mate[q_id] = v;
      bytes += 8;
    }
    const int last = 31 - __clz(m);
    p_id = __shfl_sync(0xffffffffu, v, last);
    p_c = __shfl_sync(0xffffffffu, vc, last);
    p_g = __shfl_sync(0xffffffffu, vg, last);
    p_f = __shfl_sync(0xffffffffu, vf, last);
    p_pend = __shfl_sync(0xffffffffu, P, last);
  }
}

__device__ __forceinline__ void warp_bitonic_keys(int32_t* K, int P, int lane) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int32_t a = K[i], b = K[ixj];
          if ((a > b) == ((i & k) == 0)) {
            K[i] = b;
            K[ixj] = a;
          }
        }
      }
      __syncwarp();
    }
  }
}

constexpr int kSatCap = 1024;  // anchored vertices a warp sorts in shared memory
constexpr int kTwohopWarps = 4;

// Sorts k <= 32 keys held one per lane (ascending; lanes >= k hold INT32_MAX).
__device__ __forceinline__ int32_t warp_sort32(int32_t x, int lane) {
#pragma unroll
  for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      const int32_t y = __shfl_xor_sync(0xffffffffu, x, j);
      const bool keep_min = ((lane & j) == 0) == ((lane & kk) == 0);
      x = keep_min ? (x < y ? x : y) : (x > y ? x : y);
    }
  }
  return x;
}

// Stable LSD radix sort of k keys in [0, 2^nbits) by one warp (8-bit digits), ping-ponging between
// A and B; returns the buffer holding the sorted keys.
__device__ int32_t* warp_radix_keys(int32_t* A, int32_t* B, int k, int nbits, int* hist) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  for (int shift = 0; shift < nbits; shift += 8) {
    for (int d = lane; d < 256; d += 32) hist[d] = 0;
    __syncwarp();
    for (int i = lane; i < k; i += 32) atomicAdd(&hist[(A[i] >> shift) & 255], 1);
    __syncwarp();
    int loc[8], sum = 0;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      loc[q] = hist[8 * lane + q];
      sum += loc[q];
    }
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    int run = inc - sum;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      hist[8 * lane + q] = run;
      run += loc[q];
    }
    __syncwarp();
    for (int base = 0; base < k; base += 32) {
      const int i = base + lane;
      const bool valid = i < k;
      const int32_t key = valid ? A[i] : 0;
      const int d = (key >> shift) & 255;
      const unsigned act = __ballot_sync(0xffffffffu, valid);
      unsigned peers = 0;
      int pos0 = 0, rank = 0;
      if (valid) {
        peers = __match_any_sync(act, d);
        rank = __popc(peers & lt);
        pos0 = hist[d];
      }
      __syncwarp();
      if (valid) {
        B[pos0 + rank] = key;
        if (rank == 0) hist[d] = pos0 + __popc(peers);
      }
      __syncwarp();
    }
    int32_t* t = A;
    A = B;
    B = t;
  }
  return A;
}

// Warp per anchor, from the anchors' buckets (sat[soff[h] .. soff[h + 1])): loads its bucket, sorts it and
// pairs it in ascending vertex order (pair_sorted).
// Buckets of more than `cap` go to the list `big`.  `gw` / `nw`: this warp and the number of warps
// sharing the level; S0 / S1 (cap keys each) and hist (256) are the warp's shared-memory buffers.
template <class Off>
__device__ void twohop_bucket_warps(const LevelGraph& g, int64_t capC, int64_t capG, const Off* __restrict__ soff,
                                    const int32_t* __restrict__ sat, int32_t* __restrict__ mate,
                                    int32_t* __restrict__ big, unsigned* big_cnt, int nbits, int64_t gw, int64_t nw,
                                    int32_t* S0, int32_t* S1, int* hist, int cap, unsigned long long& bytes) {
  const int lane = threadIdx.x & 31;
  for (int64_t hb = gw * 32; hb < g.n; hb += nw * 32) {
    const int64_t h0 = hb + lane;
    const int64_t lo = h0 < g.n ? (int64_t)soff[h0] : 0, hi = h0 < g.n ? (int64_t)soff[h0 + 1] : 0;
    unsigned am = __ballot_sync(0xffffffffu, hi > lo);
    while (am) {
      const int src = __ffs(am) - 1;
      am &= am - 1;
      const int64_t h = hb + src;
      const int64_t b = __shfl_sync(0xffffffffu, lo, src);
      const int k = (int)(__shfl_sync(0xffffffffu, hi, src) - b);
      if (k > cap) {
        if (lane == 0) big[atomicAdd(big_cnt, 1u)] = (int32_t)h;
        continue;
      }
      for (int q = lane; q < k; q += 32) S0[q] = sat[b + q];
      bytes += 4ull * (unsigned long long)k;
      __syncwarp();
      const int32_t* sorted = S0;
      if (k <= 32) {
        const int32_t x = warp_sort32(lane < k ? S0[lane] : INT32_MAX, lane);
        __syncwarp();
        S0[lane] = x;
        __syncwarp();
      } else {
        sorted = warp_radix_keys(S0, S1, k, nbits, hist);
      }
      pair_sorted(g, capC, capG, sorted, k, mate, bytes);
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(kTwohopWarps * 32)
    k_twohop_b(LevelGraph g, int64_t capC, int64_t capG, const int64_t* __restrict__ soff,
               const int32_t* __restrict__ sat, int32_t* __restrict__ mate, int32_t* __restrict__ big,
               unsigned* big_cnt, int nbits) {
  __shared__ int32_t sbuf[kTwohopWarps][2][kSatCap];
  __shared__ int hist_all[kTwohopWarps][256];
  __shared__ unsigned long long sacc[32];
  const int wib = threadIdx.x >> 5;
  unsigned long long bytes = 0;
  twohop_bucket_warps<int64_t>(g, capC, capG, soff, sat, mate, big, big_cnt, nbits,
                               (int64_t)blockIdx.x * kTwohopWarps + wib, (int64_t)gridDim.x * kTwohopWarps,
                               sbuf[wib][0], sbuf[wib][1], hist_all[wib], kSatCap, bytes);
  account(F_TWOHOP, bytes, sacc);
}

// Block per anchor with more than kSatCap anchored vertices: gather them into scratch (the anchor's
// row region, or its bucket when soff is given), LSD radix sort by vertex id (8-bit digits), then one
// warp pairs them.
__global__ void __launch_bounds__(1024)
    k_twohop_big(LevelGraph g, int64_t capC, int64_t capG, const int32_t* __restrict__ anchor,
                 int32_t* __restrict__ mate, const int32_t* __restrict__ big, const unsigned* big_cnt,
                 int32_t* __restrict__ ta, int32_t* __restrict__ tb, int nbits,
                 const int64_t* __restrict__ soff = nullptr, const int32_t* __restrict__ sat = nullptr) {
  __shared__ unsigned s_k;
  __shared__ unsigned hist[256];
  __shared__ unsigned binbase[256];
  __shared__ int wcnt[32][256];
  __shared__ unsigned long long sacc[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const unsigned lt = lanemask_lt();
  unsigned long long bytes = 0;
  const unsigned nbig = *big_cnt;
  for (unsigned bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
    const int32_t h = big[bi];
    const int64_t b = soff ? soff[h] : g.start[h];
    const int32_t d = soff ? (int32_t)(soff[h + 1] - b) : g.deg[h];
    if (threadIdx.x == 0) s_k = soff ? (unsigned)d : 0u;
    __syncthreads();
    if (soff) {
      for (int32_t q = threadIdx.x; q < d; q += blockDim.x) ta[b + q] = sat[b + q];
    } else {
      for (int32_t q = threadIdx.x; q < d; q += blockDim.x) {
        const int32_t v = g.adj[b + q];
        if (GP_IN(v, g.n, 4) && anchor[v] == h) ta[b + atomicAdd(&s_k, 1u)] = v;
      }
    }
    __syncthreads();
    const int64_t N = s_k;
    int32_t* src = ta + b;
    int32_t* dst = tb + b;
    for (int shift = 0; shift < nbits; shift += 8) {
      for (int x = threadIdx.x; x < 256; x += blockDim.x) hist[x] = 0;
      __syncthreads();
      for (int64_t i = threadIdx.x; i < N; i += blockDim.x) atomicAdd(&hist[(src[i] >> shift) & 255], 1u);
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int x = 0; x < 256; x++) {
          binbase[x] = run;
          run += hist[x];
        }
      }
      __syncthreads();
      for (int64_t tile = 0; tile < N; tile += blockDim.x) {
        const int64_t i = tile + threadIdx.x;
        const bool valid = i < N;
        for (int x = lane; x < 256; x += 32) wcnt[wid][x] = 0;
        __syncwarp();
        int32_t key = 0;
        int dg = 0, rank = 0;
        if (valid) {
          key = src[i];
          dg = (key >> shift) & 255;
        }
        const unsigned act = __ballot_sync(0xffffffffu, valid);
        if (valid) {
          const unsigned peers = __match_any_sync(act, dg);
          rank = __popc(peers & lt);
          if (rank == 0) wcnt[wid][dg] = __popc(peers);
        }
        __syncthreads();
        unsigned tilecnt = 0;
        if (threadIdx.x < 256) {
          int run = 0;
          for (int w = 0; w < nwarps; w++) {
            const int c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += c;
          }
          tilecnt = (unsigned)run;
        }
        __syncthreads();
        if (valid) dst[binbase[dg] + wcnt[wid][dg] + rank] = key;
        __syncthreads();
        if (threadIdx.x < 256) binbase[threadIdx.x] += tilecnt;
        __syncthreads();
      }
      int32_t* t = src;
      src = dst;
      dst = t;
    }
    if (wid == 0) pair_sorted(g, capC, capG, src, N, mate, bytes);
    if (threadIdx.x == 0) bytes += 12ull * (unsigned long long)d;
    __syncthreads();
  }
  account(F_TWOHOP, bytes, sacc);
}

__global__ void k_rep_flags(int64_t n, const int32_t* __restrict__ mate, uint8_t* __restrict__ rep) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = mate[v];
    rep[v] = (u < 0 || v < u) ? 1 : 0;
  }
}

// cmap holds the exclusive scan of the representative flags; complete it and set up the coarse
// vertices: members, summed weights, raw row length.
__device__ void cmap_fill(const LevelGraph& g, const int32_t* __restrict__ mate, int32_t* __restrict__ cmap,
                          int32_t* __restrict__ rep_of, int32_t* __restrict__ mate_of, int64_t* __restrict__ cvC,
                          int64_t* __restrict__ cvG, int64_t* __restrict__ rawlen, int64_t tid, int64_t stride,
                          int8_t* __restrict__ cfix = nullptr) {
  for (int64_t v = tid; v < g.n; v += stride) {
    const int32_t u = mate[v];
    if (!GP_IN(u + 1, g.n + 1, 5)) continue;  // a partner id, or -1
    if (u < 0 || v < u) {
      const int32_t c = cmap[v];
      rep_of[c] = (int32_t)v;
      mate_of[c] = u;
      cvC[c] = g.vC[v] + (u >= 0 ? g.vC[u] : 0);
      cvG[c] = g.vG[v] + (u >= 0 ? g.vG[u] : 0);
      if (cfix) {  // members are compatible: at most one side among them
        const int8_t a = g.fix[v], b = u >= 0 ? g.fix[u] : (int8_t)-1;
        cfix[c] = a > b ? a : b;
      }
      rawlen[c] = (int64_t)g.deg[v] + (u >= 0 ? (int64_t)g.deg[u] : 0);
    } else {
      cmap[v] = cmap[u];
    }
  }
}
__global__ void k_cmap_fill(LevelGraph g, const int32_t* __restrict__ mate, int32_t* __restrict__ cmap,
                            int32_t* __restrict__ rep_of, int32_t* __restrict__ mate_of,
                            int64_t* __restrict__ cvC, int64_t* __restrict__ cvG, int64_t* __restrict__ rawlen,
                            int8_t* __restrict__ cfix) {
  cmap_fill(g, mate, cmap, rep_of, mate_of, cvC, cvG, rawlen, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
            (int64_t)gridDim.x * blockDim.x, cfix);
}

static inline unsigned grid_for(int64_t work, int per_block, int max_per_sm = 16) {
  const int64_t want = (work + per_block - 1) / per_block;
  const int64_t cap = (int64_t)num_sms() * max_per_sm;
  return (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
}

static inline int group_for_avg(double avg) {
  if (avg <= 3.0) return 2;
  if (avg <= 6.0) return 4;
  if (avg <= 12.0) return 8;
  if (avg <= 24.0) return 16;
  return 32;
}
// matching rounds: about sixteen row entries per lane (fewer lanes per vertex: less key-reduction work
// per vertex; measured on the 1M workload, 12.05 -> 11.35 ms per partition with eight against two per
// lane, then picks 2.28 -> 2.18 ms per step with sixteen against eight, and 29.8 -> 28.8 ms on the 16M
// workload; four and thirty-two measured slower)
static inline int group_for_match(double avg) { return group_for_avg(avg * 0.0625); }

void match_level(const LevelGraph& g, int64_t capC, int64_t capG, uint64_t seed, int rounds, bool twohop,
                 int32_t* mate, cudaStream_t s) {
  const int64_t n = g.n;
  if (n <= 0) return;
  int32_t* pick = dnew<int32_t>(n, s);
  uint8_t* alive = dnew<uint8_t>(n, s);
  long long* maxw = dnew<long long>(2, s);
  const int G = group_for_match((double)(g.a > 0 ? g.a : g.cap) / (double)n);
  GP_CUDA(cudaMemsetAsync(maxw, 0, 2 * sizeof(long long), s));
  GP_LAUNCH(F_MISC, k_match_init, grid_for(n, 256), 256, 0, s, n, g.vC, g.vG, capC, capG, mate, pick, alive);
  GP_LAUNCH(F_MISC, k_max_weights, grid_for(n, 256, 4), 256, 0, s, n, g.vC, g.vG, maxw);
  // round 0 picks over every vertex; each later round over the list of the vertices the previous
  // round's handshakes left unmatched and alive (two lists, used in turn; a counter per round)
  int32_t* lists[2] = {dnew<int32_t>(n, s), dnew<int32_t>(n, s)};
  unsigned* cnts = dnew<unsigned>(rounds > 0 ? rounds : 1, s);
  GP_CUDA(cudaMemsetAsync(cnts, 0, sizeof(unsigned) * (size_t)(rounds > 0 ? rounds : 1), s));
  for (int r = 0; r < rounds; r++) {
    const int32_t* lin = r == 0 ? nullptr : lists[(r - 1) & 1];
    const unsigned* cin = r == 0 ? nullptr : cnts + (r - 1);
    // the last round lists every vertex it leaves unmatched, alive or not, for the two-hop anchors
    const bool last_for_anchors = twohop && r + 1 == rounds;
    int32_t* lout = (r + 1 < rounds || last_for_anchors) ? lists[r & 1] : nullptr;
    unsigned* cout = (r + 1 < rounds || last_for_anchors) ? cnts + r : nullptr;
    switch (G) {
#define GP_MP1(GG, FX, LS)                                                                               \
  GP_LAUNCH(F_MATCH_PICK, (k_match_pick<GG, FX, LS>), grid_for(n * GG, 256), 256, 0, s, g, capC, capG, seed, \
            (const long long*)maxw, mate, pick, alive, r == 0 ? 1 : 0, lin, cin)
#define GP_MP(GG)                                 \
  case GG:                                        \
    if (g.fix) {                                  \
      if (lin)                                    \
        GP_MP1(GG, true, true);                   \
      else                                        \
        GP_MP1(GG, true, false);                  \
    } else {                                      \
      if (lin)                                    \
        GP_MP1(GG, false, true);                  \
      else                                        \
        GP_MP1(GG, false, false);                 \
    }                                             \
    break;
      GP_MP(2) GP_MP(4) GP_MP(8) GP_MP(16) GP_MP(32)
#undef GP_MP
#undef GP_MP1
    }
    // (the last round's confirm then runs over every vertex: those that died in earlier rounds are
    // unmatched too, and the two-hop pairing anchors them as well)
    GP_LAUNCH(F_MATCH_CONFIRM, k_match_confirm, grid_for(n, 256), 256, 0, s, n, mate, pick,
              (const uint8_t*)alive, last_for_anchors ? nullptr : lin, last_for_anchors ? nullptr : cin, lout, cout,
              last_for_anchors ? 1 : 0);
  }
  const int32_t* alist = (twohop && rounds > 0) ? lists[(rounds - 1) & 1] : nullptr;
  const unsigned* acnt = (twohop && rounds > 0) ? cnts + (rounds - 1) : nullptr;
  if (twohop) {
    // every unmatched vertex into the bucket of its anchor (count, scan, scatter), then a warp per
    // anchor pairs its bucket; buckets of more than kSatCap vertices, a block each
    int32_t* anchor = pick;  // reuse
    int32_t* scnt = dnew<int32_t>(n, s);
    int64_t* soff = dnew<int64_t>(n + 1, s);
    int32_t* sat = dnew<int32_t>(n, s);
    unsigned* big_cnt = dnew<unsigned>(1, s);
    int32_t* big = dnew<int32_t>(n, s);
    int32_t* ta = dnew<int32_t>(n, s);
    int32_t* tb = dnew<int32_t>(n, s);
    GP_CUDA(cudaMemsetAsync(scnt, 0, sizeof(int32_t) * (size_t)n, s));
    GP_CUDA(cudaMemsetAsync(big_cnt, 0, sizeof(unsigned), s));
    if (alist) GP_CUDA(cudaMemsetAsync(anchor, 0xff, sizeof(int32_t) * (size_t)n, s));  // -1: no anchor
    switch (G) {
#define GP_AN(GG)                                                                                         \
  case GG:                                                                                               \
    if (alist)                                                                                           \
      GP_LAUNCH(F_TWOHOP, (k_anchor<GG, true>), grid_for(n * GG, 256), 256, 0, s, g, seed, mate, anchor,   \
                (uint8_t*)nullptr, scnt, alist, acnt);                                                   \
    else                                                                                                 \
      GP_LAUNCH(F_TWOHOP, (k_anchor<GG, false>), grid_for(n * GG, 256), 256, 0, s, g, seed, mate, anchor,  \
                (uint8_t*)nullptr, scnt, (const int32_t*)nullptr, (const unsigned*)nullptr);             \
    break;
      GP_AN(2) GP_AN(4) GP_AN(8) GP_AN(16) GP_AN(32)
#undef GP_AN
    }
    scan_i32_to_i64(scnt, soff, n, s);
    GP_LAUNCH(F_TWOHOP, k_sat_scatter, grid_for(n, 256), 256, 0, s, n, (const int32_t*)anchor,
              (const int64_t*)soff, scnt, sat);
    int nbits = 1;
    while (nbits < 31 && (int64_t(1) << nbits) < n) nbits++;
    GP_LAUNCH(F_TWOHOP, k_twohop_b, grid_for(n, kTwohopWarps * 32, 16), kTwohopWarps * 32, 0, s, g, capC, capG,
              (const int64_t*)soff, (const int32_t*)sat, mate, big, big_cnt, nbits);
    GP_LAUNCH(F_TWOHOP, k_twohop_big, (unsigned)num_sms(), 1024, 0, s, g, capC, capG, (const int32_t*)anchor, mate,
              (const int32_t*)big, (const unsigned*)big_cnt, ta, tb, nbits, (const int64_t*)soff,
              (const int32_t*)sat);
    dfree(scnt, s);
    dfree(soff, s);
    dfree(sat, s);
    dfree(big_cnt, s);
    dfree(big, s);
    dfree(ta, s);
    dfree(tb, s);
  }
  dfree(lists[0], s);
  dfree(lists[1], s);
  dfree(cnts, s);
  GP_CHECK_LAUNCH();
  dfree(pick, s);
  dfree(alive, s);
  dfree(maxw, s);
}

void coarse_count(const LevelGraph& g, const int32_t* mate, int32_t* cmap, int64_t* /*unused*/, cudaStream_t s) {
  const int64_t n = g.n;
  uint8_t* rep = dnew<uint8_t>(n, s);
  GP_LAUNCH(F_CMAP, k_rep_flags, grid_for(n, 256), 256, 0, s, n, mate, rep);
  scan_u8_to_i32(rep, cmap, n, s);  // cmap[n] = number of coarse vertices
  dfree(rep, s);
}

// Requires cg.n = number of coarse vertices and cg.cap >= sum of the fine degrees; allocates the
// coarse arrays.
void contract_level(const LevelGraph& g, const int32_t* mate, int32_t* cmap, LevelGraph& cg, cudaStream_t s) {
  const int64_t nc = cg.n;
  int32_t* rep_of = dnew<int32_t>(nc, s);
  int32_t* mate_of = dnew<int32_t>(nc, s);
  int64_t* rawlen = dnew<int64_t>(nc, s);
  cg.start = dnew<int64_t>(nc + 1, s);
  cg.deg = dnew<int32_t>(nc, s);
  cg.vC = dnew<int64_t>(nc, s);
  cg.vG = dnew<int64_t>(nc, s);
  cg.adj = dnew<int32_t>(cg.cap, s);
  cg.W = dnew<int64_t>(cg.cap, s);
  cg.fix = g.fix ? dnew<int8_t>(nc, s) : nullptr;
  GP_LAUNCH(F_CMAP, k_cmap_fill, grid_for(g.n, 256), 256, 0, s, g, mate, cmap, rep_of, mate_of, cg.vC, cg.vG,
            rawlen, cg.fix);
  scan_i64(rawlen, cg.start, nc, s);
  TwoSrc src{};
  src.a_start = g.start;
  src.a_deg = g.deg;
  src.a_col = g.adj;
  src.a_w64 = g.W;
  src.b_start = g.start;
  src.b_deg = g.deg;
  src.b_col = g.adj;
  src.b_w64 = g.W;
  src.row_a = rep_of;
  src.row_b = mate_of;
  src.map = cmap;
  src.map_n = g.n;
  src.drop_self = 1;
  merge_rows_unordered(src, nc, nc, cg.start, cg.deg, cg.adj, cg.W, F_CONTRACT_MERGE, cg.cap, s);
  dfree(rep_of, s);
  dfree(mate_of, s);
  dfree(rawlen, s);
}

}  // namespace gp
