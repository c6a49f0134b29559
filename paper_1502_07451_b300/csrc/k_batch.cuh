// k_batch.cuh -- many graphs in one persistent launch.
//
// A CTA takes the next graph from a queue (largest graphs first) and runs the whole bipartitioner
// on it: handshake matching and two-hop pairing, contraction, greedy growing on the coarsest level,
// projection and refinement back to level 0, the cut and, when asked, the makespan.  The steps are
// those of the single-graph path: where that path launches a kernel over the grid, the CTA runs the
// same round body with itself as the grid (the shared bodies of k_coarsen.cuh / k_refine.cuh), and
// __syncthreads() takes the place of the kernel boundary; the rest (scans, contraction merge, greedy
// growing, cut, makespan) are CTA-scope versions of the same definitions.  Every result of a graph
// is therefore the single-graph result.
//
// Each CTA owns a slot of global memory and carves a graph's scratch and coarse levels out of it
// with a bump allocator.  A graph whose levels do not fit is abandoned and reported as deferred; the
// host partitions it afterwards with the single-graph path.
//
// A schedule (threads per CTA, CTAs per SM, lanes per row, warp hash-table size) only changes how
// the work of one graph is spread over its CTA, never a result.
#pragma once
#include "gp_internal.cuh"
#include "k_coarsen.cuh"
#include "k_initial.cuh"
#include "k_refine.cuh"
#include "k_propose.cuh"

namespace gp {

// One graph of a batch (device copy).
struct BatchGraph {
  // level 0: the symmetrised graph in padded CSR
  const int64_t* start;
  const int32_t* deg;
  const int32_t* adj;
  const int64_t* W;
  const int64_t* vC;
  const int64_t* vG;
  int64_t n, a0;
  int64_t BC, BG, SC, SG;
  uint64_t seed;
  const float* logits;  // not null: the learned path (proposal from these logits, refinement of level 0)
  // directed out-CSR (cut)
  const int64_t* off;
  const int32_t* cols;
  const int32_t* w;
  // topological levels and the level-ordered in-CSR (makespan)
  const int64_t* lev_ptr;
  const int32_t* lev_vtx;
  const int64_t* lo_off;
  const int32_t* lo_src;
  const int32_t* lo_w;
  const int32_t* lo_cC;
  const int32_t* lo_cG;
  int32_t nlev;
  int32_t want_makespan;
  uint8_t* part;  // level-0 split, n bytes of device memory
};

constexpr int32_t kBatchDone = 0, kBatchDeferred = 1;

struct BatchOut {
  long long cut, LC, LG, makespan;
  int32_t status, feasible, levels, rounds, coarsest_n, trial;
};

struct BatchSched {
  int32_t gshift;    // lanes per row: the degree rule's choice times 2^gshift, clamped to 2..32
  int32_t hash_cap;  // entries of a warp's contraction hash table (power of two, 64..256)
};

constexpr int kBatchWarpSmem = 3072;  // dynamic shared memory per warp

// POD view of one level (shared memory holds the table of a graph's levels).
struct LevRec {
  int64_t n, a;  // vertices, entries
  int64_t* start;
  int32_t* deg;
  int32_t* adj;
  int64_t* W;
  int64_t* vC;
  int64_t* vG;
  int32_t* cmap;  // to the next coarser level (n + 1 entries)
  uint8_t* part;
};

__device__ __forceinline__ LevelGraph lev_view(const LevRec& r) {
  LevelGraph g;
  g.n = r.n;
  g.cap = r.a;
  g.start = r.start;
  g.deg = r.deg;
  g.adj = r.adj;
  g.W = r.W;
  g.vC = r.vC;
  g.vG = r.vG;
  return g;
}

// Bump allocator over a CTA's slot; every thread of the CTA holds an identical copy.
struct SlotArena {
  char* base;
  unsigned long long size, used;
  bool fail;
  template <class T>
  __device__ __forceinline__ T* get(int64_t count) {
    const unsigned long long a = (used + 255ull) & ~255ull;
    const unsigned long long need = a + sizeof(T) * (unsigned long long)(count > 0 ? count : 1);
    if (fail || need > size) {
      fail = true;
      return nullptr;
    }
    used = need;
    return (T*)(base + a);
  }
};

__device__ __forceinline__ int lanes_for_degree(int64_t a, int64_t n, int shift) {
  const int64_t nn = n > 0 ? n : 1;
  int G;
  if (a <= 3 * nn) G = 2;
  else if (a <= 6 * nn) G = 4;
  else if (a <= 12 * nn) G = 8;
  else if (a <= 24 * nn) G = 16;
  else G = 32;
  if (shift > 0) G <<= shift;
  if (shift < 0) G >>= -shift;
  return G < 2 ? 2 : (G > 32 ? 32 : G);
}

__device__ __forceinline__ int bits_for(int64_t n) {
  int b = 1;
  while (b < 31 && (int64_t(1) << b) < n) b++;
  return b;
}

// ------------------------------------------------------------------------------------------------
// CTA-scope primitives
// ------------------------------------------------------------------------------------------------
// Inclusive scan of one value per thread; `tot` gets the CTA total.  `sh` needs 32 slots.
template <class T>
__device__ __forceinline__ T cta_scan_incl(T x, T* sh, T& tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T s = lane < nw ? sh[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) sh[lane] = s;
  }
  __syncthreads();
  const T before = wid ? sh[wid - 1] : T(0);
  tot = sh[nw - 1];
  __syncthreads();
  return x + before;
}

template <class T>
__device__ __forceinline__ T cta_max(T x, T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  __syncthreads();
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  T r = sh[0];
  for (int w = 1; w < nw; w++) r = sh[w] > r ? sh[w] : r;
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------------------------------------
// Coarsening of one level: handshake rounds, two-hop pairing.  mate gets the matching.
// ------------------------------------------------------------------------------------------------
template <int G>
__device__ void b_pick_round(const LevelGraph& g, long long capC, long long capG, uint64_t seed, long long mC,
                             long long mG, const int32_t* mate, int32_t* pick, uint8_t* alive, int* s_flag) {
  const bool picked = match_pick<G>(g, capC, capG, seed, mC, mG, mate, pick, alive, threadIdx.x, blockDim.x);
  if (picked) *s_flag = 1;
}
template <int G>
__device__ void b_anchor(const LevelGraph& g, uint64_t seed, const int32_t* mate, int32_t* anchor, int32_t* scnt) {
  match_anchor<G>(g, seed, mate, anchor, nullptr, threadIdx.x, blockDim.x, scnt);
}

__device__ void b_match(const LevelGraph& g, long long capC, long long capG, uint64_t seed, int G, int32_t* mate,
                        int32_t* pick, uint8_t* alive, int32_t* biglist, int32_t* sat, uint32_t* bits,
                        unsigned char* dsm, int* s_flag, unsigned* s_cnt, long long* s_red, int32_t* scnt,
                        int32_t* soff, int32_t* bucket) {
  const int64_t n = g.n;
  long long mC = 0, mG = 0;
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
    const long long c = g.vC[v], q = g.vG[v];
    mate[v] = -1;
    pick[v] = -1;
    alive[v] = (c <= capC && q <= capG) ? 1 : 0;  // over a cap on its own: never merges
    mC = c > mC ? c : mC;
    mG = q > mG ? q : mG;
  }
  mC = cta_max<long long>(mC, s_red);
  mG = cta_max<long long>(mG, s_red);
  for (int r = 0; r < kMatchRounds; r++) {
    if (threadIdx.x == 0) *s_flag = 0;
    __syncthreads();
    switch (G) {
      case 2: b_pick_round<2>(g, capC, capG, seed, mC, mG, mate, pick, alive, s_flag); break;
      case 4: b_pick_round<4>(g, capC, capG, seed, mC, mG, mate, pick, alive, s_flag); break;
      case 8: b_pick_round<8>(g, capC, capG, seed, mC, mG, mate, pick, alive, s_flag); break;
      case 16: b_pick_round<16>(g, capC, capG, seed, mC, mG, mate, pick, alive, s_flag); break;
      default: b_pick_round<32>(g, capC, capG, seed, mC, mG, mate, pick, alive, s_flag); break;
    }
    __syncthreads();
    if (*s_flag == 0) break;  // nobody picked: later rounds pick nothing either
    __syncthreads();
    if (threadIdx.x == 0) *s_flag = 0;
    __syncthreads();
    bool matched = false;
    for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
      if (mate[v] != -1) continue;
      const int32_t u = pick[v];
      if (u >= 0 && pick[u] == (int32_t)v) {
        mate[v] = u;
        matched = true;
      }
    }
    if (matched) *s_flag = 1;
    __syncthreads();
    if (*s_flag == 0) break;  // no new pair: the next round would see the same state
    __syncthreads();
  }
  // two-hop pairing, from anchor buckets: each unmatched vertex counts itself into its anchor's bucket,
  // a scan gives the buckets' offsets, the vertices are scattered into them, and a warp per anchor
  // pairs its bucket (scnt / soff / bucket: n, n + 1 and n entries of scratch)
  int32_t* anchor = pick;
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) scnt[v] = 0;
  __syncthreads();
  switch (G) {
    case 2: b_anchor<2>(g, seed, mate, anchor, scnt); break;
    case 4: b_anchor<4>(g, seed, mate, anchor, scnt); break;
    case 8: b_anchor<8>(g, seed, mate, anchor, scnt); break;
    case 16: b_anchor<16>(g, seed, mate, anchor, scnt); break;
    default: b_anchor<32>(g, seed, mate, anchor, scnt); break;
  }
  __syncthreads();
  {
    long long run = 0;
    for (int64_t b0 = 0; b0 < n; b0 += blockDim.x) {
      const int64_t v = b0 + threadIdx.x;
      const long long x = v < n ? scnt[v] : 0;
      long long tot;
      const long long inc = cta_scan_incl<long long>(x, s_red, tot);
      if (v < n) soff[v] = (int32_t)(run + inc - x);
      run += tot;
    }
    if (threadIdx.x == 0) {
      soff[n] = (int32_t)run;
      *s_cnt = 0;
    }
  }
  __syncthreads();
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
    const int32_t a = anchor[v];
    if (a >= 0) bucket[soff[a] + atomicSub(&scnt[a], 1) - 1] = (int32_t)v;
  }
  __syncthreads();
  const int nbits = bits_for(n);
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long bytes = 0;
  {
    int32_t* S0 = (int32_t*)(dsm + (size_t)wib * kBatchWarpSmem);
    int32_t* S1 = S0 + 256;
    int* hist = (int*)(S0 + 512);
    twohop_bucket_warps<int32_t>(g, capC, capG, soff, bucket, mate, biglist, s_cnt, nbits, wib, blockDim.x >> 5, S0,
                                 S1, hist, 256, bytes);
  }
  __syncthreads();
  const unsigned nbig = *s_cnt;
  const int64_t nwords = (n + 31) >> 5;
  for (unsigned bi = 0; bi < nbig; bi++) {
    // anchors with many anchored vertices: a bitmap over the vertex ids gives them in ascending order
    const int32_t h = biglist[bi];
    for (int64_t q = threadIdx.x; q < nwords; q += blockDim.x) bits[q] = 0u;
    __syncthreads();
    const int32_t b = soff[h];
    const int32_t d = soff[h + 1] - b;
    for (int32_t q = threadIdx.x; q < d; q += blockDim.x) {  // the bucket's vertices, as a bitmap
      const int32_t v = bucket[b + q];
      atomicOr(&bits[v >> 5], 1u << (v & 31));
    }
    bytes += 4ull * (unsigned long long)((d + (int)blockDim.x - 1 - (int)threadIdx.x) / (int)blockDim.x);
    __syncthreads();
    if (wib == 0) {
      int64_t k = 0;
      for (int64_t q0 = 0; q0 < nwords; q0 += 32) {
        const int64_t q = q0 + lane;
        uint32_t wv = q < nwords ? bits[q] : 0u;
        const int c = __popc(wv);
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += y;
        }
        int64_t pos = k + inc - c;
        while (wv) {
          const int bit = __ffs(wv) - 1;
          wv &= wv - 1;
          sat[pos++] = (int32_t)(q * 32 + bit);
        }
        k += __shfl_sync(0xffffffffu, inc, 31);
      }
      __syncwarp();
      pair_sorted(g, capC, capG, sat, k, mate, bytes);
    }
    __syncthreads();
  }
  __shared__ unsigned long long sacc[32];
  account(F_TWOHOP, bytes, sacc);
}

// ------------------------------------------------------------------------------------------------
// Contraction of level f into c (c.n, c.start..c.part allocated; cap of c's rows = f.a).
// ------------------------------------------------------------------------------------------------
// Merges the rows of `src` (nrows of them; row r written at start[r], merged length to deg[r], in no
// particular order): a per-warp shared-memory hash table (hash_cap entries), then one table over the
// whole dynamic shared memory for longer rows, then a dense accumulator (acc = 0, mark = -1 on entry
// and on exit, indexed by the mapped column) for the longest.
__device__ void b_merge_rows(const TwoSrc& src, int64_t nrows, const int64_t* start, int32_t* deg, int32_t* adj,
                             int64_t* W, int32_t* biglist, int64_t* acc, int32_t* mark, int hash_cap,
                             unsigned char* dsm, int dsm_bytes, unsigned* s_cnt, int fam) {
  if (threadIdx.x == 0) *s_cnt = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned lt = lanemask_lt();
  unsigned long long bytes = 0;
  // warp tier: a hash table of hash_cap entries per warp
  {
    unsigned long long* V = (unsigned long long*)(dsm + (size_t)wib * kBatchWarpSmem);
    int32_t* K = (int32_t*)(V + hash_cap);
    for (int64_t r = wib; r < nrows; r += nw) {
      const RowView rv = row_view(src, r);
      const int64_t len = rv.a_len + rv.b_len;
      if (2 * len > hash_cap) {
        if (lane == 0) biglist[atomicAdd(s_cnt, 1u)] = (int32_t)r;
        continue;
      }
      int T = 32;
      while (T < 2 * len) T <<= 1;
      const int shift = 32 - (31 - __clz(T));
      for (int i = lane; i < T; i += 32) {
        K[i] = kEmptyKey;
        V[i] = 0ull;
      }
      __syncwarp();
      for (int64_t i = lane; i < len; i += 32) {
        int32_t col;
        int64_t w;
        row_entry(src, rv, i, col, w);
        bytes += 16;
        if (src.drop_self && col == (int32_t)r) continue;
        unsigned slot = ((uint32_t)col * 0x9E3779B1u) >> shift;
        for (;;) {
          const int32_t old = atomicCAS(&K[slot], kEmptyKey, col);
          if (old == kEmptyKey || old == col) {
            atomicAdd(&V[slot], (unsigned long long)w);
            break;
          }
          slot = (slot + 1) & (unsigned)(T - 1);
        }
      }
      __syncwarp();
      const int64_t ob = start[r];
      int out = 0;
      for (int base = 0; base < T; base += 32) {
        const int32_t k = K[base + lane];
        const bool has = k != kEmptyKey;
        const unsigned m = __ballot_sync(0xffffffffu, has);
        if (has) {
          const int pos = out + __popc(m & lt);
          adj[ob + pos] = k;
          W[ob + pos] = (int64_t)V[base + lane];
        }
        out += __popc(m);
      }
      if (lane == 0) {
        deg[r] = out;
        bytes += 12ull * (unsigned long long)out + 24ull;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  const unsigned nbig = *s_cnt;
  __syncthreads();
  // block tier: one table over the whole dynamic shared memory; beyond it, a dense accumulator
  // indexed by coarse id (acc = 0 and mark = -1 between rows)
  int TB = 32;
  while ((TB << 1) * 12 <= dsm_bytes) TB <<= 1;
  unsigned long long* V = (unsigned long long*)dsm;
  int32_t* K = (int32_t*)(V + TB);
  for (unsigned bi = 0; bi < nbig; bi++) {
    const int32_t r = biglist[bi];
    const RowView rv = row_view(src, r);
    const int64_t len = rv.a_len + rv.b_len;
    const int64_t ob = start[r];
    if (threadIdx.x == 0) *s_cnt = 0;
    if (2 * len <= TB) {
      int T = 32;
      while (T < 2 * len) T <<= 1;
      const int shift = 32 - (31 - __clz(T));
      for (int i = threadIdx.x; i < T; i += blockDim.x) {
        K[i] = kEmptyKey;
        V[i] = 0ull;
      }
      __syncthreads();
      for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        int32_t col;
        int64_t w;
        row_entry(src, rv, i, col, w);
        bytes += 16;
        if (src.drop_self && col == r) continue;
        unsigned slot = ((uint32_t)col * 0x9E3779B1u) >> shift;
        for (;;) {
          const int32_t old = atomicCAS(&K[slot], kEmptyKey, col);
          if (old == kEmptyKey || old == col) {
            atomicAdd(&V[slot], (unsigned long long)w);
            break;
          }
          slot = (slot + 1) & (unsigned)(T - 1);
        }
      }
      __syncthreads();
      for (int base = 0; base < T; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const bool has = i < T && K[i] != kEmptyKey;
        const unsigned m = __ballot_sync(0xffffffffu, has);
        unsigned wpos = 0;
        if (lane == 0 && m) wpos = atomicAdd(s_cnt, (unsigned)__popc(m));
        wpos = __shfl_sync(0xffffffffu, wpos, 0);
        if (has) {
          const unsigned pos = wpos + __popc(m & lt);
          adj[ob + pos] = K[i];
          W[ob + pos] = (int64_t)V[i];
        }
      }
      __syncthreads();
    } else {
      __syncthreads();
      for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        int32_t col;
        int64_t w;
        row_entry(src, rv, i, col, w);
        bytes += 16;
        if (src.drop_self && col == r) continue;
        atomicAdd((unsigned long long*)&acc[col], (unsigned long long)w);
        if (atomicExch(&mark[col], r) != r) adj[ob + atomicAdd(s_cnt, 1u)] = col;
      }
      __syncthreads();
      const unsigned k = *s_cnt;
      for (unsigned i = threadIdx.x; i < k; i += blockDim.x) {
        const int32_t col = adj[ob + i];
        W[ob + i] = acc[col];
        acc[col] = 0;
        mark[col] = -1;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      deg[r] = (int32_t)*s_cnt;
      bytes += 12ull * (unsigned long long)*s_cnt + 24ull;
    }
    __syncthreads();
  }
  __shared__ unsigned long long sacc[32];
  account(fam, bytes, sacc);
}

__device__ void b_contract(const LevelGraph& f, const int32_t* mate, int32_t* cmap, int32_t* rep_of,
                           int32_t* mate_of, long long* rawlen, int32_t* biglist, int64_t* acc, int32_t* mark,
                           const LevRec& c, int hash_cap, unsigned char* dsm, int dsm_bytes, unsigned* s_cnt,
                           long long* s_red) {
  const int64_t n = f.n, nc = c.n;
  // coarse ids: representatives (unmatched vertices, smaller end of a pair) in vertex order
  long long run = 0;
  for (int64_t b = 0; b < n; b += blockDim.x) {
    const int64_t v = b + threadIdx.x;
    int flag = 0;
    if (v < n) {
      const int32_t u = mate[v];
      flag = (u < 0 || v < u) ? 1 : 0;
    }
    long long tot;
    const long long inc = cta_scan_incl<long long>((long long)flag, s_red, tot);
    if (flag) cmap[v] = (int32_t)(run + inc - 1);
    run += tot;
  }
  __syncthreads();
  cmap_fill(f, mate, cmap, rep_of, mate_of, c.vC, c.vG, (int64_t*)rawlen, threadIdx.x, blockDim.x);
  __syncthreads();
  // row starts: exclusive scan of the raw lengths
  run = 0;
  for (int64_t b = 0; b < nc; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const long long x = i < nc ? rawlen[i] : 0;
    long long tot;
    const long long inc = cta_scan_incl<long long>(x, s_red, tot);
    if (i < nc) c.start[i] = run + inc - x;
    run += tot;
  }
  if (threadIdx.x == 0) {
    c.start[nc] = run;
    *s_cnt = 0;
  }
  __syncthreads();
  TwoSrc src{};
  src.a_start = f.start;
  src.a_deg = f.deg;
  src.a_col = f.adj;
  src.a_w64 = f.W;
  src.b_start = f.start;
  src.b_deg = f.deg;
  src.b_col = f.adj;
  src.b_w64 = f.W;
  src.row_a = rep_of;
  src.row_b = mate_of;
  src.map = cmap;
  src.drop_self = 1;
  b_merge_rows(src, nc, c.start, c.deg, c.adj, c.W, biglist, acc, mark, hash_cap, dsm, dsm_bytes, s_cnt,
               F_CONTRACT_MERGE);
}

// ------------------------------------------------------------------------------------------------
// Greedy growing: one warp per trial.  side / toC / adjC: the trial's arrays (shared or global).
// ------------------------------------------------------------------------------------------------
__device__ void warp_grow(const LevelGraph& g, long long BC, long long BG, long long SG, int64_t start,
                          const int64_t* wsum, uint8_t* side, long long* toC, int32_t* adjC, long long* cut_out,
                          int* feas_out) {
  const int lane = threadIdx.x & 31;
  const int64_t n = g.n;
  for (int64_t v = lane; v < n; v += 32) {
    side[v] = 1;
    toC[v] = 0;
    adjC[v] = 0;
  }
  long long LC = 0, LG = SG;
  int32_t x = (g.vC[start] <= BC) ? (int32_t)start : -1;
  __syncwarp();
  for (;;) {
    if (x >= 0) {
      LC += g.vC[x];
      LG -= g.vG[x];
      if (lane == 0) side[x] = 0;
      const int64_t b = g.start[x];
      const int32_t d = g.deg[x];
      for (int32_t k = lane; k < d; k += 32) {  // rows hold distinct neighbours
        const int32_t u = g.adj[b + k];
        toC[u] += g.W[b + k];
        adjC[u] += 1;
      }
      __syncwarp();
    }
    if (LG <= BG) break;
    GrowKey best{0, 0, -1};
    for (int64_t v = lane; v < n; v += 32) {
      if (side[v] != 1 || LC + g.vC[v] > BC) continue;
      const GrowKey k{adjC[v] > 0 ? 1 : 0, 2 * toC[v] - wsum[v], (int32_t)v};
      if (grow_better(k, best)) best = k;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      GrowKey q;
      q.a = __shfl_xor_sync(0xffffffffu, best.a, o);
      q.g = __shfl_xor_sync(0xffffffffu, best.g, o);
      q.v = __shfl_xor_sync(0xffffffffu, best.v, o);
      if (grow_better(q, best)) best = q;
    }
    x = best.v;
    if (x < 0) break;
  }
  long long cut = 0;
  for (int64_t v = lane; v < n; v += 32)
    if (side[v] == 0) cut += wsum[v] - toC[v];
  cut = warp_sum64(cut);
  if (lane == 0) {
    *cut_out = cut;
    *feas_out = (LC <= BC && LG <= BG) ? 1 : 0;
  }
}

// ------------------------------------------------------------------------------------------------
// The learned proposal at CTA scope: vertices by (logit desc, id asc); the first
// k = min(kC, kG) go to the CPU (kC: longest prefix within B_C; kG: shortest prefix after which the
// GPU load is within B_G), found by the refinement's weighted radix selection over the keys
// ((max - float_key(logit)) << idbits | id).  Returns false on a NaN logit.
// ------------------------------------------------------------------------------------------------
__device__ bool b_propose(const BatchGraph& B, const Cands& cand, uint8_t* part, long long* s_red,
                          unsigned long long* s_redu) {
  __shared__ unsigned long long hw[256], hc[256];
  __shared__ SelOut so;
  __shared__ int s_nan;
  const int64_t n = B.n;
  if (threadIdx.x == 0) s_nan = 0;
  __syncthreads();
  long long gmax = LLONG_MIN, gmin = LLONG_MAX;
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
    const float z = B.logits[v];
    if (isnan(z)) s_nan = 1;
    const long long k = (long long)float_order_key(z);
    cand.id[v] = (int32_t)v;
    cand.gain[v] = k;
    cand.cd[v] = B.vC[v];
    cand.cs[v] = B.vG[v];
    gmax = k > gmax ? k : gmax;
    gmin = k < gmin ? k : gmin;
  }
  gmax = cta_max<long long>(gmax, s_red);
  gmin = -cta_max<long long>(-gmin, s_red);
  if (s_nan) return false;
  const int idbits = bits_for(n);
  const int keybits = bits_of((unsigned long long)(gmax - gmin)) + idbits;
  const unsigned long long N = (unsigned long long)n;
  int64_t kC = n, kG = 0;
  if (B.SC > B.BC) {
    block_select(cand, N, 0, B.BC, gmax, idbits, keybits, &so, hw, hc);
    kC = so.found ? so.rank : n;
  }
  const long long D = B.SG - B.BG;
  if (D > 0) {
    block_select(cand, N, 1, D - 1, gmax, idbits, keybits, &so, hw, hc);
    kG = so.found ? so.rank + 1 : n;
  }
  const int64_t k = kC < kG ? kC : kG;
  if (k <= 0 || k >= n) {
    for (int64_t v = threadIdx.x; v < n; v += blockDim.x) part[v] = k <= 0 ? 1 : 0;
  } else {
    block_select(cand, N, 2, k, gmax, idbits, keybits, &so, hw, hc);  // the candidate of rank k
    const u128 thr = so.key;
    for (int64_t v = threadIdx.x; v < n; v += blockDim.x)
      part[v] = cand_key(gmax, cand.gain[v], (int32_t)v, idbits) < thr ? 0 : 1;
  }
  __syncthreads();
  return true;
}

// ------------------------------------------------------------------------------------------------
// One graph.
// ------------------------------------------------------------------------------------------------
template <int G>
__device__ void b_gain_all(const LevelGraph& g, const uint8_t* part, long long* gainv) {
  gain_all<G>(g, part, gainv, threadIdx.x, blockDim.x);
}

__device__ void batch_graph(const BatchGraph& B, BatchOut* out, char* slot, unsigned long long slot_bytes,
                            unsigned char* dsm, int dsm_bytes, const BatchSched& sch) {
  __shared__ LevRec s_lev[kMaxLevels + 1];
  __shared__ Ctl s_ctl;
  __shared__ long long s_red[32];
  __shared__ unsigned long long s_redu[32];
  __shared__ int s_flag;
  __shared__ unsigned s_cnt;
  __shared__ long long s_tcut[kTrials];
  __shared__ int s_tfeas[kTrials];
  __shared__ int s_best;
  const int64_t n0 = B.n;
  if (n0 == 0) {
    if (threadIdx.x == 0) {
      BatchOut o{};
      o.status = kBatchDone;
      o.feasible = 1;
      o.trial = -1;
      *out = o;
    }
    __syncthreads();
    return;
  }
  SlotArena A{slot, slot_bytes, 0ull, false};
  int32_t* mate = A.get<int32_t>(n0);
  int32_t* pick = A.get<int32_t>(n0);
  uint8_t* alive = A.get<uint8_t>(n0);
  int32_t* rep_of = A.get<int32_t>(n0);
  int32_t* mate_of = A.get<int32_t>(n0);
  int32_t* biglist = A.get<int32_t>(n0);
  int32_t* sat = A.get<int32_t>(n0);
  uint32_t* bits = A.get<uint32_t>((n0 + 31) / 32);
  int64_t* acc = A.get<int64_t>(n0);
  int32_t* mark = A.get<int32_t>(n0);
  Cands cand;
  cand.id = A.get<int32_t>(n0);
  cand.gain = A.get<long long>(n0);
  cand.cd = A.get<long long>(n0);
  cand.cs = A.get<long long>(n0);
  cand.gainv = A.get<long long>(n0);
  cand.stamp = A.get<int32_t>(n0);
  cand.dirty[0] = A.get<int32_t>(n0);
  cand.dirty[1] = A.get<int32_t>(n0);
  unsigned long long* fp = B.want_makespan ? A.get<unsigned long long>(n0) : nullptr;
  if (A.fail) {
    if (threadIdx.x == 0) out->status = kBatchDeferred;
    __syncthreads();
    return;
  }
  for (int64_t v = threadIdx.x; v < n0; v += blockDim.x) {
    acc[v] = 0;
    mark[v] = -1;
    cand.stamp[v] = -1;
  }
  if (threadIdx.x == 0) {
    LevRec r0;
    r0.n = n0;
    r0.a = B.a0;
    r0.start = const_cast<int64_t*>(B.start);
    r0.deg = const_cast<int32_t*>(B.deg);
    r0.adj = const_cast<int32_t*>(B.adj);
    r0.W = const_cast<int64_t*>(B.W);
    r0.vC = const_cast<int64_t*>(B.vC);
    r0.vG = const_cast<int64_t*>(B.vG);
    r0.cmap = nullptr;
    r0.part = B.part;
    s_lev[0] = r0;
  }
  __syncthreads();
  const long long BC = B.BC, BG = B.BG;
  const long long capC = BC / kCapDiv, capG = BG / kCapDiv;
  int L = 0;
  if (B.logits) {
    // ---- learned proposal at level 0 (no coarsening, no growing)
    if (!b_propose(B, cand, B.part, s_red, s_redu)) {
      if (threadIdx.x == 0) out->status = kBatchDeferred;  // the single-graph path reports the NaN
      __syncthreads();
      return;
    }
    if (threadIdx.x == 0) s_best = -1;
  }
  // ---- coarsening
  for (;;) {
    if (B.logits) break;
    const LevRec f = s_lev[L];
    if (!(f.n > kCoarsest && L < kMaxLevels)) break;
    const LevelGraph g = lev_view(f);
    const int G = lanes_for_degree(f.a, f.n, sch.gshift);
    // scratch of the two-hop buckets: arrays the refinement uses later (idle while coarsening)
    b_match(g, capC, capG, B.seed, G, mate, pick, alive, biglist, sat, bits, dsm, &s_flag, &s_cnt, s_red,
            cand.dirty[0], (int32_t*)cand.cd, cand.dirty[1]);
    __syncthreads();
    long long reps = 0;
    for (int64_t v = threadIdx.x; v < f.n; v += blockDim.x) {
      const int32_t u = mate[v];
      reps += (u < 0 || v < u) ? 1 : 0;
    }
    const long long nc = block_sum<long long>(reps, s_red);
    if (nc * kStallDen > f.n * kStallNum) break;  // the matching keeps too many vertices
    LevRec c;
    c.n = nc;
    c.a = 0;
    c.start = A.get<int64_t>(nc + 1);
    c.deg = A.get<int32_t>(nc);
    c.vC = A.get<int64_t>(nc);
    c.vG = A.get<int64_t>(nc);
    c.adj = A.get<int32_t>(f.a);
    c.W = A.get<int64_t>(f.a);
    c.part = A.get<uint8_t>(nc);
    c.cmap = nullptr;
    int32_t* cmap = A.get<int32_t>(f.n + 1);
    if (A.fail) {
      if (threadIdx.x == 0) out->status = kBatchDeferred;
      __syncthreads();
      return;
    }
    b_contract(g, mate, cmap, rep_of, mate_of, cand.gain, biglist, acc, mark, c, sch.hash_cap, dsm, dsm_bytes,
               &s_cnt, s_red);
    long long a = 0;
    for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) a += c.deg[i];
    a = block_sum<long long>(a, s_red);
    if (threadIdx.x == 0) {
      c.a = a;
      s_lev[L].cmap = cmap;
      s_lev[L + 1] = c;
    }
    __syncthreads();
    L++;
  }
  // ---- greedy growing on the coarsest level
  if (!B.logits) {
    const LevRec f = s_lev[L];
    const LevelGraph g = lev_view(f);
    const int64_t n = f.n;
    if (B.SG <= BG) {
      for (int64_t v = threadIdx.x; v < n; v += blockDim.x) f.part[v] = 1;
      if (threadIdx.x == 0) s_best = -1;
    } else {
      const size_t per = ((size_t)n * 13 + 64 + 15) & ~(size_t)15;  // toC | adjC | side, 16-byte aligned
      unsigned char* tmem;
      int64_t* wsum = acc;  // free between levels; restored to zero below
      if ((size_t)kTrials * per <= (size_t)dsm_bytes) {
        tmem = dsm;
      } else {
        tmem = (unsigned char*)A.get<unsigned char>((int64_t)(kTrials * per));
        if (A.fail) {
          if (threadIdx.x == 0) out->status = kBatchDeferred;
          __syncthreads();
          return;
        }
      }
      const int lane = threadIdx.x & 31;
      for (int64_t v = threadIdx.x >> 5; v < n; v += blockDim.x >> 5) {
        const int64_t b = f.start[v];
        const int32_t d = f.deg[v];
        int64_t s = 0;
        for (int32_t k = lane; k < d; k += 32) s += f.W[b + k];
        s = warp_sum64(s);
        if (lane == 0) wsum[v] = s;
      }
      __syncthreads();
      const int wib = threadIdx.x >> 5;
      if (wib < kTrials) {
        unsigned char* base = tmem + (size_t)wib * per;
        long long* toC = (long long*)base;
        int32_t* adjC = (int32_t*)(base + 8 * (size_t)n);
        uint8_t* side = base + 12 * (size_t)n;
        const int64_t s0 = (int64_t)(pair_hash(B.seed, 0xFFFFFFFFu, (uint32_t)wib) % (uint64_t)n);
        warp_grow(g, BC, BG, B.SG, s0, wsum, side, toC, adjC, &s_tcut[wib], &s_tfeas[wib]);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int bt = 0;
        for (int t = 1; t < kTrials; t++)
          if (s_tfeas[t] > s_tfeas[bt] || (s_tfeas[t] == s_tfeas[bt] && s_tcut[t] < s_tcut[bt])) bt = t;
        s_best = bt;
      }
      __syncthreads();
      const uint8_t* side = tmem + (size_t)s_best * per + 12 * (size_t)n;
      for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
        f.part[v] = side[v];
        wsum[v] = 0;
      }
    }
    __syncthreads();
  }
  // ---- refinement, coarsest to finest
  int32_t rounds_total = 0;
  if (threadIdx.x == 0) {
    memset(&s_ctl, 0, sizeof(Ctl));
    s_ctl.BC = BC;
    s_ctl.BG = BG;
  }
  __syncthreads();
  for (int l = L; l >= 0; l--) {
    const LevRec f = s_lev[l];
    const LevelGraph g = lev_view(f);
    if (l < L) {
      const uint8_t* pc = s_lev[l + 1].part;
      for (int64_t v = threadIdx.x; v < f.n; v += blockDim.x) f.part[v] = pc[f.cmap[v]];
    }
    if (threadIdx.x == 0) {
      s_ctl.LC = 0;
      s_ctl.LG = 0;
    }
    __syncthreads();
    ref_loads(g, f.part, &s_ctl, threadIdx.x, blockDim.x);
    __syncthreads();
    if (threadIdx.x == 0) ref_begin(&s_ctl, bits_for(f.n));
    const int G = lanes_for_degree(f.a, f.n, sch.gshift);
    switch (G) {
      case 2: b_gain_all<2>(g, f.part, cand.gainv); break;
      case 4: b_gain_all<4>(g, f.part, cand.gainv); break;
      case 8: b_gain_all<8>(g, f.part, cand.gainv); break;
      case 16: b_gain_all<16>(g, f.part, cand.gainv); break;
      default: b_gain_all<32>(g, f.part, cand.gainv); break;
    }
    __syncthreads();
    int32_t prev = round_tag(l, -2);
    for (int r = -1; r < kRefineRounds; r++) {
      ref_cands(g, f.part, &s_ctl, r, prev, cand, threadIdx.x, blockDim.x);
      __syncthreads();
      ref_select(&s_ctl, r, cand);
      __syncthreads();
      ref_apply(&s_ctl, r, g, f.part, round_tag(l, r), cand, threadIdx.x, blockDim.x);
      __syncthreads();
      prev = round_tag(l, r);
      if (s_ctl.done) break;  // later rounds would return at once
    }
    rounds_total += s_ctl.rounds;
    __syncthreads();
  }
  // ---- cut over the directed edges
  const uint8_t* part = B.part;
  unsigned long long cut = 0;
  for (int64_t u = threadIdx.x; u < n0; u += blockDim.x) {
    const uint8_t pu = part[u];
    for (int64_t e = B.off[u]; e < B.off[u + 1]; e++)
      if (part[B.cols[e]] != pu) cut += (unsigned long long)B.w[e];
  }
  cut = block_sum<unsigned long long>(cut, s_redu);
  // ---- makespan: level by level of the topological order
  unsigned long long ms = 0;
  if (B.want_makespan) {
    const int Gm = lanes_for_degree(B.lo_off[n0], n0, 0);
    const int sub = threadIdx.x % Gm;
    const int64_t group = threadIdx.x / Gm, ngroups = blockDim.x / Gm;
    const unsigned gmask = group_mask(Gm);
    for (int32_t l = 0; l < B.nlev; l++) {
      const int64_t beg = B.lev_ptr[l], end = B.lev_ptr[l + 1];
      const int64_t trips = (end - beg + ngroups - 1) / ngroups;  // every group runs the same trips
      for (int64_t t = 0; t < trips; t++) {
        const int64_t i = beg + t * ngroups + group;
        unsigned long long best = 0;
        uint8_t p = 0;
        int32_t cost = 0;
        if (i < end) {
          const int32_t v = B.lev_vtx[i];
          p = part[v];
          cost = p ? B.lo_cG[i] : B.lo_cC[i];
          for (int64_t e = B.lo_off[i] + sub; e < B.lo_off[i + 1]; e += Gm) {
            const unsigned long long fv = fp[B.lo_src[e]];
            const unsigned long long tv =
                (fv >> 1) + (((uint8_t)(fv & 1ull) != p) ? (unsigned long long)B.lo_w[e] : 0ull);
            best = tv > best ? tv : best;
          }
        }
        for (int o = Gm / 2; o > 0; o >>= 1) {
          const unsigned long long q = __shfl_xor_sync(gmask, best, o, Gm);
          best = q > best ? q : best;
        }
        if (i < end && sub == 0) {
          const unsigned long long fin = best + (unsigned long long)cost;
          fp[i] = (fin << 1) | (unsigned long long)p;
          ms = fin > ms ? fin : ms;
        }
      }
      __syncthreads();
    }
    ms = cta_max<unsigned long long>(ms, s_redu);
  }
  if (threadIdx.x == 0) {
    BatchOut o;
    o.cut = (long long)cut;
    o.LC = s_ctl.LC;
    o.LG = s_ctl.LG;
    o.makespan = (long long)ms;
    o.status = kBatchDone;
    o.feasible = (s_ctl.LC <= BC && s_ctl.LG <= BG) ? 1 : 0;
    o.levels = L;
    o.rounds = rounds_total;
    o.coarsest_n = (int32_t)s_lev[L].n;
    o.trial = s_best;
    *out = o;
  }
  __syncthreads();
}

// The persistent kernel: CTAs pop graph ids from the queue (order = largest first) until it runs
// dry.  Only the queue head is shared between CTAs.
template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_batch(const BatchGraph* __restrict__ graphs, const int32_t* __restrict__ order, int32_t count,
            unsigned* queue, char* ws, unsigned long long slot_bytes, BatchOut* out, BatchSched sch) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ int s_next;
  char* slot = ws + (size_t)blockIdx.x * slot_bytes;
  const int dsm_bytes = (NT / 32) * kBatchWarpSmem;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned q = atomicAdd(queue, 1u);
      s_next = q < (unsigned)count ? order[q] : -1;
    }
    __syncthreads();
    const int gi = s_next;
    __syncthreads();
    if (gi < 0) break;
    batch_graph(graphs[gi], out + gi, slot, slot_bytes, dsm, dsm_bytes, sch);
  }
}

}  // namespace gp
