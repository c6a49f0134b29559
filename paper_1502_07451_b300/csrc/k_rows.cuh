// k_rows.cuh -- per-row gather, sort by column and segmented reduction of equal columns.
//
// Used twice on the path:
//   * symmetrisation (graph creation): row v = out-row(v) + in-row(v); every directed entry adds its
//     transfer cost to the undirected weight of both endpoints (Sec. III.B: transfer time does not
//     depend on the direction);
//   * contraction: coarse row c = row(rep) + row(mate) mapped through cmap, without c itself.
// Rows are bucketed by raw length: a warp sorts rows of <= kWarpCap entries in shared memory, a
// block sorts rows of <= kBlockCap entries, and longer rows are radix-sorted by a block through a
// global scratch buffer.  The output row r starts at out_start[r] (capacity = raw length); its merged
// length goes to deg_out[r].  Row order within the output is ascending column.
#pragma once
#include "gp_internal.cuh"
#include "k_scan.cuh"

namespace gp {

constexpr int kWarpCap = 256;
constexpr int kBlockCap = 8192;
constexpr int kMergeWarps = 8;  // warps per block of the warp tier

struct RowView {
  int64_t a_beg, a_len, b_beg, b_len;
};

__device__ __forceinline__ RowView row_view(const TwoSrc& s, int64_t r) {
  RowView v;
  const int64_t ra = s.row_a ? (int64_t)s.row_a[r] : r;
  v.a_beg = s.a_start[ra];
  v.a_len = s.a_deg ? (int64_t)s.a_deg[ra] : s.a_start[ra + 1] - s.a_start[ra];
  v.b_beg = 0;
  v.b_len = 0;
  if (s.b_col) {
    const int64_t rb = s.row_b ? (int64_t)s.row_b[r] : r;
    if (rb >= 0) {
      v.b_beg = s.b_start[rb];
      v.b_len = s.b_deg ? (int64_t)s.b_deg[rb] : s.b_start[rb + 1] - s.b_start[rb];
    }
  }
  return v;
}

__device__ __forceinline__ void row_entry(const TwoSrc& s, const RowView& v, int64_t i, int32_t& col,
                                          int64_t& w) {
  if (i < v.a_len) {
    const int64_t e = v.a_beg + i;
    col = s.a_col[e];
    w = s.a_w64 ? s.a_w64[e] : (int64_t)s.a_w32[e];
  } else {
    const int64_t e = v.b_beg + (i - v.a_len);
    col = s.b_col[e];
    w = s.b_w64 ? s.b_w64[e] : (int64_t)s.b_w32[e];
  }
#ifdef GP_CHECKED
  if (s.map && s.map_n > 0 && !GP_IN(col, s.map_n, 12)) col = 0;  // recorded; an in-range id instead
#endif
  if (s.map) col = s.map[col];
}

// Row entries read once and merged rows written once by the hash tiers go through the cache with an
// evict-first policy (ld.global.cs / st.global.cs), so that on graphs larger than the L2 they do not
// push out the coarse-id map, which every row gathers from.
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
  return __ldcs(p);
}
template <typename T>
__device__ __forceinline__ void st_stream(T* p, T v) {
  __stcs(p, v);
}
__device__ __forceinline__ void row_entry_stream(const TwoSrc& s, const RowView& v, int64_t i, int32_t& col,
                                                 int64_t& w) {
  if (i < v.a_len) {
    const int64_t e = v.a_beg + i;
    col = ld_stream(s.a_col + e);
    w = s.a_w64 ? ld_stream(s.a_w64 + e) : (int64_t)ld_stream(s.a_w32 + e);
  } else {
    const int64_t e = v.b_beg + (i - v.a_len);
    col = ld_stream(s.b_col + e);
    w = s.b_w64 ? ld_stream(s.b_w64 + e) : (int64_t)ld_stream(s.b_w32 + e);
  }
#ifdef GP_CHECKED
  if (s.map && s.map_n > 0 && !GP_IN(col, s.map_n, 12)) col = 0;
#endif
  if (s.map) col = s.map[col];
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned long long entry_bytes(const TwoSrc& s, bool from_a) {
  const bool w64 = from_a ? (s.a_w64 != nullptr) : (s.b_w64 != nullptr);
  return 4ull + (w64 ? 8ull : 4ull) + (s.map ? 4ull : 0ull);
}

// ------------------------------------------------------------------------------------------------
// warp tier
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void warp_bitonic(int32_t* K, int64_t* V, int P, int lane) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int32_t a = K[i], b = K[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            K[i] = b;
            K[ixj] = a;
            const int64_t t = V[i];
            V[i] = V[ixj];
            V[ixj] = t;
          }
        }
      }
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(kMergeWarps * 32)
    k_merge_warp(TwoSrc s, int64_t nrows, const int64_t* __restrict__ out_start,
                 int32_t* __restrict__ deg_out, int32_t* __restrict__ adj_out, int64_t* __restrict__ W_out,
                 int32_t* __restrict__ list_mid, unsigned* cnt_mid, int32_t* __restrict__ list_huge,
                 unsigned* cnt_huge, int fam) {
  __shared__ int32_t skey[kMergeWarps][kWarpCap];
  __shared__ int64_t sval[kMergeWarps][kWarpCap];
  __shared__ unsigned long long sacc[32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* K = skey[wib];
  int64_t* V = sval[wib];
  const unsigned lt = lanemask_lt();
  unsigned long long bytes = 0;
  for (int64_t r = (int64_t)blockIdx.x * kMergeWarps + wib; r < nrows; r += (int64_t)gridDim.x * kMergeWarps) {
    const RowView v = row_view(s, r);
    const int64_t len = v.a_len + v.b_len;
    if (len > kWarpCap) {
      if (lane == 0) {
        if (len > kBlockCap)
          list_huge[atomicAdd(cnt_huge, 1u)] = (int32_t)r;
        else
          list_mid[atomicAdd(cnt_mid, 1u)] = (int32_t)r;
      }
      continue;
    }
    int cnt = 0;
    for (int64_t base = 0; base < len; base += 32) {
      const int64_t i = base + lane;
      int32_t col = INT32_MAX;
      int64_t w = 0;
      bool keep = false;
      if (i < len) {
        row_entry(s, v, i, col, w);
        keep = !(s.drop_self && col == (int32_t)r);
        bytes += entry_bytes(s, i < v.a_len);
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int pos = cnt + __popc(m & lt);
        K[pos] = col;
        V[pos] = w;
      }
      cnt += __popc(m);
    }
    int P = 32;
    while (P < cnt) P <<= 1;
    for (int i = cnt + lane; i < P; i += 32) {
      K[i] = INT32_MAX;
      V[i] = 0;
    }
    __syncwarp();
    warp_bitonic(K, V, P, lane);
    const int64_t ob = out_start[r];
    int out = 0;
    for (int base = 0; base < cnt; base += 32) {
      const int i = base + lane;
      const bool head = i < cnt && (i == 0 || K[i - 1] != K[i]);
      int64_t sum = 0;
      if (head) {
        const int32_t k = K[i];
        for (int q = i; q < cnt && K[q] == k; q++) sum += V[q];
      }
      const unsigned m = __ballot_sync(0xffffffffu, head);
      if (head) {
        const int pos = out + __popc(m & lt);
        adj_out[ob + pos] = K[i];
        W_out[ob + pos] = sum;
      }
      out += __popc(m);
    }
    if (lane == 0) deg_out[r] = out;
    if (lane == 0) bytes += 12ull * (unsigned long long)out + 24ull;
    __syncwarp();
  }
  account(fam, bytes, sacc);
}

// ------------------------------------------------------------------------------------------------
// block tier (rows of kWarpCap < raw <= kBlockCap entries)
// ------------------------------------------------------------------------------------------------
constexpr int kMergeBlockThreads = 1024;
constexpr size_t kMergeBlockSmem = (size_t)kBlockCap * (sizeof(int32_t) + sizeof(int64_t));

__global__ void __launch_bounds__(kMergeBlockThreads)
    k_merge_block(TwoSrc s, const int32_t* __restrict__ list, const unsigned* cnt,
                  const int64_t* __restrict__ out_start, int32_t* __restrict__ deg_out,
                  int32_t* __restrict__ adj_out, int64_t* __restrict__ W_out, int fam) {
  extern __shared__ __align__(16) unsigned char smem[];
  int64_t* V = (int64_t*)smem;
  int32_t* K = (int32_t*)(V + kBlockCap);
  __shared__ int s_n;
  __shared__ int sh[33];
  __shared__ unsigned long long sacc[32];
  const unsigned nlist = *cnt;
  unsigned long long bytes = 0;
  for (unsigned li = blockIdx.x; li < nlist; li += gridDim.x) {
    const int64_t r = list[li];
    const RowView v = row_view(s, r);
    const int64_t len = v.a_len + v.b_len;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
      int32_t col;
      int64_t w;
      row_entry(s, v, i, col, w);
      bytes += entry_bytes(s, i < v.a_len);
      if (!(s.drop_self && col == (int32_t)r)) {
        const int pos = atomicAdd(&s_n, 1);
        K[pos] = col;
        V[pos] = w;
      }
    }
    __syncthreads();
    const int cnt = s_n;
    int P = 2;
    while (P < cnt) P <<= 1;
    for (int i = cnt + threadIdx.x; i < P; i += blockDim.x) {
      K[i] = INT32_MAX;
      V[i] = 0;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const int32_t a = K[i], b = K[ixj];
            const bool up = (i & k) == 0;
            if ((a > b) == up) {
              K[i] = b;
              K[ixj] = a;
              const int64_t t = V[i];
              V[i] = V[ixj];
              V[ixj] = t;
            }
          }
        }
        __syncthreads();
      }
    }
    const int64_t ob = out_start[r];
    int running = 0;
    for (int base = 0; base < cnt; base += blockDim.x) {
      const int i = base + threadIdx.x;
      const bool head = i < cnt && (i == 0 || K[i - 1] != K[i]);
      int64_t sum = 0;
      if (head) {
        const int32_t k = K[i];
        for (int q = i; q < cnt && K[q] == k; q++) sum += V[q];
      }
      int tot;
      const int ex = block_exclusive_scan<int>(head ? 1 : 0, sh, &tot);
      if (head) {
        adj_out[ob + running + ex] = K[i];
        W_out[ob + running + ex] = sum;
      }
      running += tot;
    }
    if (threadIdx.x == 0) {
      deg_out[r] = running;
      bytes += 12ull * (unsigned long long)running + 24ull;
    }
    __syncthreads();
  }
  account(fam, bytes, sacc);
}

// ------------------------------------------------------------------------------------------------
// huge tier (raw > kBlockCap): LSD radix sort by one block through scratch, then merge.
// ------------------------------------------------------------------------------------------------
constexpr int kHugeThreads = 1024;

__global__ void __launch_bounds__(kHugeThreads)
    k_merge_huge(TwoSrc s, const int32_t* __restrict__ list, const unsigned* cnt,
                 const int64_t* __restrict__ out_start, int32_t* __restrict__ deg_out,
                 int32_t* __restrict__ adj_out, int64_t* __restrict__ W_out, int32_t* __restrict__ tk,
                 int64_t* __restrict__ tv, int nbits, int fam) {
  __shared__ unsigned long long s_n;
  __shared__ unsigned long long hist[256];
  __shared__ long long binbase[256];
  __shared__ int wcnt[kHugeThreads / 32][256];
  __shared__ long long sh[33];
  __shared__ unsigned long long sacc[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned lt = lanemask_lt();
  const unsigned nlist = *cnt;
  unsigned long long bytes = 0;
  for (unsigned li = blockIdx.x; li < nlist; li += gridDim.x) {
    const int64_t r = list[li];
    const RowView v = row_view(s, r);
    const int64_t len = v.a_len + v.b_len;
    const int64_t ob = out_start[r];
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
      int32_t col;
      int64_t w;
      row_entry(s, v, i, col, w);
      bytes += entry_bytes(s, i < v.a_len);
      if (!(s.drop_self && col == (int32_t)r)) {
        const unsigned long long pos = atomicAdd(&s_n, 1ull);
        tk[ob + pos] = col;
        tv[ob + pos] = w;
      }
    }
    __syncthreads();
    const int64_t N = (int64_t)s_n;
    int32_t* srcK = tk + ob;
    int64_t* srcV = tv + ob;
    int32_t* dstK = adj_out + ob;
    int64_t* dstV = W_out + ob;
    for (int shift = 0; shift < nbits; shift += 8) {
      for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d] = 0;
      __syncthreads();
      for (int64_t i = threadIdx.x; i < N; i += blockDim.x) atomicAdd(&hist[(srcK[i] >> shift) & 255], 1ull);
      __syncthreads();
      if (threadIdx.x == 0) {
        long long run = 0;
        for (int d = 0; d < 256; d++) {
          binbase[d] = run;
          run += (long long)hist[d];
        }
      }
      __syncthreads();
      for (int64_t tile = 0; tile < N; tile += blockDim.x) {
        const int64_t i = tile + threadIdx.x;
        const bool valid = i < N;
        int32_t key = 0;
        int64_t val = 0;
        int d = 0;
        for (int q = lane; q < 256; q += 32) wcnt[wid][q] = 0;
        __syncwarp();
        unsigned peers = 0;
        int rank = 0;
        if (valid) {
          key = srcK[i];
          val = srcV[i];
          d = (key >> shift) & 255;
        }
        const unsigned act = __ballot_sync(0xffffffffu, valid);
        if (valid) {
          peers = __match_any_sync(act, d);
          rank = __popc(peers & lt);
          if (rank == 0) wcnt[wid][d] = __popc(peers);
        }
        __syncthreads();
        long long tilecnt = 0;
        if (threadIdx.x < 256) {
          int run = 0;
          for (int w = 0; w < nw; w++) {
            const int c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += c;
          }
          tilecnt = run;
        }
        __syncthreads();
        if (valid) {
          const long long pos = binbase[d] + wcnt[wid][d] + rank;
          dstK[pos] = key;
          dstV[pos] = val;
        }
        __syncthreads();
        if (threadIdx.x < 256) binbase[threadIdx.x] += tilecnt;
        __syncthreads();
      }
      int32_t* tK = srcK;
      srcK = dstK;
      dstK = tK;
      int64_t* tV = srcV;
      srcV = dstV;
      dstV = tV;
    }
    // sorted data is in src; merge equal columns into dst
    long long running = 0;
    for (int64_t base = 0; base < N; base += blockDim.x) {
      const int64_t i = base + threadIdx.x;
      const bool head = i < N && (i == 0 || srcK[i - 1] != srcK[i]);
      int64_t sum = 0;
      int32_t k = 0;
      if (head) {
        k = srcK[i];
        for (int64_t q = i; q < N && srcK[q] == k; q++) sum += srcV[q];
      }
      long long tot;
      const long long ex = block_exclusive_scan<long long>(head ? 1 : 0, sh, &tot);
      if (head) {
        dstK[running + ex] = k;
        dstV[running + ex] = sum;
      }
      running += tot;
    }
    __syncthreads();
    if (dstK != adj_out + ob) {
      for (int64_t i = threadIdx.x; i < running; i += blockDim.x) {
        adj_out[ob + i] = dstK[i];
        W_out[ob + i] = dstV[i];
      }
    }
    if (threadIdx.x == 0) {
      deg_out[r] = (int32_t)running;
      bytes += 12ull * (unsigned long long)running + 24ull;
    }
    __syncthreads();
  }
  account(fam, bytes, sacc);
}

// ------------------------------------------------------------------------------------------------
// Unordered merge (contraction): duplicates are combined in a per-warp shared-memory hash table and
// the distinct (column, summed weight) pairs are written in no particular order.  Every consumer of
// coarse rows is independent of their order (sums, maxima under a total order, sets); the two-hop
// pairing sorts what it walks.  Rows longer than TMAX / 2 raw entries are deferred to the next tier.
// The table is emptied once per warp; a row's inserts remember the slots they claimed (one per lane
// and pass, in registers), and after the row only those slots are read out and emptied again, so a
// row costs work in its distinct entries, not in the table size.
// ------------------------------------------------------------------------------------------------
constexpr int32_t kEmptyKey = -1;

template <int TMAX>
__device__ __forceinline__ int table_shift() {  // slot = (col * golden) >> shift covers [0, TMAX)
  return 32 - (31 - __clz(TMAX));
}

template <int TMAX, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
    k_merge_hash(TwoSrc s, int64_t nrows, const int32_t* __restrict__ list, const unsigned* list_cnt,
                 const int64_t* __restrict__ out_start, int32_t* __restrict__ deg_out,
                 int32_t* __restrict__ adj_out, int64_t* __restrict__ W_out, int32_t* __restrict__ dl1,
                 unsigned* dc1, int64_t split1, int32_t* __restrict__ dl2, unsigned* dc2, int64_t split2,
                 int32_t* __restrict__ dl3, unsigned* dc3, int fam) {
  constexpr int kPasses = TMAX / 64;  // a row holds at most TMAX / 2 raw entries, 32 per pass
  extern __shared__ __align__(16) unsigned char smem_h[];
  __shared__ unsigned long long sacc[32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned long long* V = (unsigned long long*)smem_h + (size_t)wib * TMAX;
  int32_t* K = (int32_t*)((unsigned long long*)smem_h + (size_t)WARPS * TMAX) + (size_t)wib * TMAX;
  const unsigned lt = lanemask_lt();
  const int shift = table_shift<TMAX>();
  const int64_t total = list ? (int64_t)*list_cnt : nrows;
  unsigned long long bytes = 0;
  for (int i = lane; i < TMAX; i += 32) {
    K[i] = kEmptyKey;
    V[i] = 0ull;
  }
  __syncwarp();
  for (int64_t it = (int64_t)blockIdx.x * WARPS + wib; it < total; it += (int64_t)gridDim.x * WARPS) {
    const int64_t r = list ? (int64_t)list[it] : it;
    const RowView v = row_view(s, r);
    const int64_t len = v.a_len + v.b_len;
    if (2 * len > TMAX) {
      if (lane == 0) {
        if (len <= split1)
          dl1[atomicAdd(dc1, 1u)] = (int32_t)r;
        else if (len <= split2)
          dl2[atomicAdd(dc2, 1u)] = (int32_t)r;
        else
          dl3[atomicAdd(dc3, 1u)] = (int32_t)r;
      }
      continue;
    }
    int slot[kPasses];
    unsigned claimed = 0;  // bit p: this lane's entry of pass p took a new slot
#pragma unroll
    for (int p = 0; p < kPasses; p++) {
      slot[p] = 0;
      if (p * 32 >= len) break;
      const int64_t i = p * 32 + lane;
      if (i >= len) continue;
      int32_t col;
      int64_t w;
      row_entry_stream(s, v, i, col, w);
      bytes += entry_bytes(s, i < v.a_len);
      if (s.drop_self && col == (int32_t)r) continue;
      unsigned sl = ((uint32_t)col * 0x9E3779B1u) >> shift;
      for (;;) {
        const int32_t old = atomicCAS(&K[sl], kEmptyKey, col);
        if (old == kEmptyKey || old == col) {
          atomicAdd(&V[sl], (unsigned long long)w);
          if (old == kEmptyKey) claimed |= 1u << p;
          break;
        }
        sl = (sl + 1) & (unsigned)(TMAX - 1);
      }
      slot[p] = (int)sl;
    }
    __syncwarp();
    // each distinct column is read out (and its slot emptied) by the lane that claimed its slot
    const int64_t ob = out_start[r];
    int out = 0;
#pragma unroll
    for (int p = 0; p < kPasses; p++) {
      if (p * 32 >= len) break;
      const bool c = (claimed >> p) & 1u;
      const unsigned m = __ballot_sync(0xffffffffu, c);
      if (c) {
        const int pos = out + __popc(m & lt);
        st_stream(adj_out + ob + pos, K[slot[p]]);
        st_stream(W_out + ob + pos, (int64_t)V[slot[p]]);
        K[slot[p]] = kEmptyKey;
        V[slot[p]] = 0ull;
      }
      out += __popc(m);
    }
    if (lane == 0) {
      deg_out[r] = out;
      bytes += 12ull * (unsigned long long)out + 24ull;
    }
    __syncwarp();
  }
  account(fam, bytes, sacc);
}

// Warp per row of at most 32 raw entries, without a table: each lane holds one entry, __match_any_sync
// finds the lanes holding the same column, and the lowest of them sums their weights and writes the
// merged entry (at its rank among those lowest lanes).  Longer rows go to the list of their tier.
__global__ void __launch_bounds__(256)
    k_merge_match(TwoSrc s, int64_t nrows, const int64_t* __restrict__ out_start, int32_t* __restrict__ deg_out,
                  int32_t* __restrict__ adj_out, int64_t* __restrict__ W_out, int32_t* __restrict__ dl1,
                  unsigned* dc1, int64_t split1, int32_t* __restrict__ dl2, unsigned* dc2, int64_t split2,
                  int32_t* __restrict__ dl3, unsigned* dc3, int64_t split3, int32_t* __restrict__ dl4,
                  unsigned* dc4, int fam) {
  __shared__ unsigned long long sacc[32];
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long bytes = 0;
  // 32 rows per warp step: every lane measures one row, the long ones go to their tier's list with one
  // atomic per tier and step, then the warp merges the short ones one after another
  for (int64_t rb = gw * 32; rb < nrows; rb += nw * 32) {
    const int64_t rl = rb + lane;
    RowView mv{0, 0, 0, 0};
    int64_t mlen = -1;
    if (rl < nrows) {
      mv = row_view(s, rl);
      mlen = mv.a_len + mv.b_len;
    }
    const int tier = mlen < 0 ? -1 : mlen <= 32 ? 0 : mlen <= split1 ? 1 : mlen <= split2 ? 2 : mlen <= split3 ? 3 : 4;
#pragma unroll
    for (int t = 1; t <= 4; t++) {
      const unsigned m = __ballot_sync(0xffffffffu, tier == t);
      if (!m) continue;
      int32_t* dl = t == 1 ? dl1 : t == 2 ? dl2 : t == 3 ? dl3 : dl4;
      unsigned* dc = t == 1 ? dc1 : t == 2 ? dc2 : t == 3 ? dc3 : dc4;
      unsigned p0 = 0;
      if (lane == __ffs(m) - 1) p0 = atomicAdd(dc, (unsigned)__popc(m));
      p0 = __shfl_sync(0xffffffffu, p0, __ffs(m) - 1);
      if (tier == t) dl[p0 + __popc(m & lt)] = (int32_t)rl;
    }
    for (unsigned sm = __ballot_sync(0xffffffffu, tier == 0); sm; sm &= sm - 1) {
      const int src = __ffs(sm) - 1;
      const int64_t r = rb + src;
      RowView v;
      v.a_beg = __shfl_sync(0xffffffffu, mv.a_beg, src);
      v.a_len = __shfl_sync(0xffffffffu, mv.a_len, src);
      v.b_beg = __shfl_sync(0xffffffffu, mv.b_beg, src);
      v.b_len = __shfl_sync(0xffffffffu, mv.b_len, src);
      const int64_t len = v.a_len + v.b_len;
      int32_t col = -1;
      int64_t w = 0;
      if (lane < len) {
        row_entry(s, v, lane, col, w);
        bytes += entry_bytes(s, lane < v.a_len);
        if (s.drop_self && col == (int32_t)r) col = -1;
      }
      const bool has = col >= 0;
      const unsigned hm = __ballot_sync(0xffffffffu, has);
      const unsigned peers = __match_any_sync(0xffffffffu, col) & hm;  // lanes with this lane's column
      const bool lead = has && (peers & lt) == 0;                      // the lowest of them
      unsigned long long sum = 0;
      for (unsigned q = peers; q; q &= q - 1) {  // the column's weights, summed in every peer lane
        const int sl = __ffs(q) - 1;
        sum += (unsigned long long)__shfl_sync(peers, (long long)w, sl);
      }
      const unsigned leads = __ballot_sync(0xffffffffu, lead);
      const int64_t ob = out_start[r];
      if (lead) {
        const int pos = __popc(leads & lt);
        adj_out[ob + pos] = col;
        W_out[ob + pos] = (int64_t)sum;
      }
      if (lane == 0) {
        const int out = __popc(leads);
        deg_out[r] = out;
        bytes += 12ull * (unsigned long long)out + 24ull;
      }
    }
  }
  account(fam, bytes, sacc);
}

// Block per row: one hash table over the block's dynamic shared memory (TMAX entries), rows of up to
// TMAX / 2 raw entries, taken from `list`; output positions come from a block counter (any order).
// As in the warp tier, the table is emptied once and each row empties the slots it claimed.
template <int TMAX, int THREADS>
__global__ void __launch_bounds__(THREADS)
    k_merge_hash_blk(TwoSrc s, const int32_t* __restrict__ list, const unsigned* list_cnt,
                     const int64_t* __restrict__ out_start, int32_t* __restrict__ deg_out,
                     int32_t* __restrict__ adj_out, int64_t* __restrict__ W_out, int fam) {
  constexpr int kPasses = TMAX / 2 / THREADS;
  extern __shared__ __align__(16) unsigned char smem_b[];
  __shared__ unsigned long long sacc[32];
  __shared__ unsigned s_out;
  unsigned long long* V = (unsigned long long*)smem_b;
  int32_t* K = (int32_t*)(V + TMAX);
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const int shift = table_shift<TMAX>();
  const int64_t total = (int64_t)*list_cnt;
  unsigned long long bytes = 0;
  if (total <= (int64_t)blockIdx.x) return;  // no row for this block (uniform)
  for (int i = threadIdx.x; i < TMAX; i += THREADS) {
    K[i] = kEmptyKey;
    V[i] = 0ull;
  }
  for (int64_t it = blockIdx.x; it < total; it += gridDim.x) {
    const int64_t r = list[it];
    const RowView v = row_view(s, r);
    const int64_t len = v.a_len + v.b_len;
    if (threadIdx.x == 0) s_out = 0;
    __syncthreads();
    int slot[kPasses];
    unsigned claimed = 0;
#pragma unroll
    for (int p = 0; p < kPasses; p++) {
      slot[p] = 0;
      if ((int64_t)p * THREADS >= len) break;
      const int64_t i = (int64_t)p * THREADS + threadIdx.x;
      if (i >= len) continue;
      int32_t col;
      int64_t w;
      row_entry_stream(s, v, i, col, w);
      bytes += entry_bytes(s, i < v.a_len);
      if (s.drop_self && col == (int32_t)r) continue;
      unsigned sl = ((uint32_t)col * 0x9E3779B1u) >> shift;
      for (;;) {
        const int32_t old = atomicCAS(&K[sl], kEmptyKey, col);
        if (old == kEmptyKey || old == col) {
          atomicAdd(&V[sl], (unsigned long long)w);
          if (old == kEmptyKey) claimed |= 1u << p;
          break;
        }
        sl = (sl + 1) & (unsigned)(TMAX - 1);
      }
      slot[p] = (int)sl;
    }
    __syncthreads();
    const int64_t ob = out_start[r];
#pragma unroll
    for (int p = 0; p < kPasses; p++) {
      if ((int64_t)p * THREADS >= len) break;
      const bool c = (claimed >> p) & 1u;
      const unsigned m = __ballot_sync(0xffffffffu, c);
      unsigned wpos = 0;
      if (lane == 0 && m) wpos = atomicAdd(&s_out, (unsigned)__popc(m));
      wpos = __shfl_sync(0xffffffffu, wpos, 0);
      if (c) {
        const unsigned pos = wpos + __popc(m & lt);
        st_stream(adj_out + ob + pos, K[slot[p]]);
        st_stream(W_out + ob + pos, (int64_t)V[slot[p]]);
        K[slot[p]] = kEmptyKey;
        V[slot[p]] = 0ull;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      deg_out[r] = (int32_t)s_out;
      bytes += 12ull * (unsigned long long)s_out + 24ull;
    }
  }
  account(fam, bytes, sacc);
}

constexpr int kHashT1 = 256, kHashW1 = 8;    // rows of <= 128 raw entries
constexpr int kHashT2 = 2048, kHashW2 = 4;   // rows of <= 1024 raw entries
constexpr size_t kHashSmem1 = (size_t)kHashT1 * kHashW1 * 12;
constexpr size_t kHashSmem2 = (size_t)kHashT2 * kHashW2 * 12;

void merge_rows(const TwoSrc& src, int64_t nrows, int64_t ncols, const int64_t* out_start,
                int32_t* deg_out, int32_t* adj_out, int64_t* W_out, int family, int64_t raw_bound,
                cudaStream_t s) {
  if (nrows <= 0) return;
  static bool attr_set = false;
  if (!attr_set) {
    GP_CUDA(cudaFuncSetAttribute(k_merge_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMergeBlockSmem));
    attr_set = true;
  }
  unsigned* cnts = dnew<unsigned>(2, s);
  GP_CUDA(cudaMemsetAsync(cnts, 0, 2 * sizeof(unsigned), s));
  int32_t* list_mid = dnew<int32_t>(nrows, s);
  int32_t* list_huge = dnew<int32_t>(nrows, s);
  const int sms = num_sms();
  const int64_t want = (nrows + kMergeWarps - 1) / kMergeWarps;
  const unsigned grid = (unsigned)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
  GP_LAUNCH(family, k_merge_warp, grid, kMergeWarps * 32, 0, s, src, nrows, out_start, deg_out, adj_out,
            W_out, list_mid, cnts, list_huge, cnts + 1, family);
  GP_LAUNCH(family, k_merge_block, (unsigned)(2 * sms), kMergeBlockThreads, kMergeBlockSmem, s, src,
            list_mid, cnts, out_start, deg_out, adj_out, W_out, family);
  int nbits = 1;
  while (nbits < 31 && (int64_t(1) << nbits) < ncols) nbits++;
  int32_t* tk = dnew<int32_t>(raw_bound, s);
  int64_t* tv = dnew<int64_t>(raw_bound, s);
  GP_LAUNCH(family, k_merge_huge, (unsigned)sms, kHugeThreads, 0, s, src, list_huge, cnts + 1, out_start,
            deg_out, adj_out, W_out, tk, tv, nbits, family);
  GP_CHECK_LAUNCH();
  dfree(tk, s);
  dfree(tv, s);
  dfree(list_mid, s);
  dfree(list_huge, s);
  dfree(cnts, s);
}

// Unordered merge (symmetrisation, contraction): rows in no particular order.  Tiers by raw length: a
// warp with the entries in registers (<= 32; only when the rows average at most 20 raw entries), a warp
// and a 256-entry table (<= 128), a block of 256 threads and a 2,048-entry table (<= 1,024), a block of
// 1,024 threads and a 16,384-entry table (<= 8,192), then the radix tier.
constexpr int kHashTB2 = 2048, kHashTB3 = 16384;
constexpr size_t kHashSmemB2 = (size_t)kHashTB2 * 12, kHashSmemB3 = (size_t)kHashTB3 * 12;
void merge_rows_unordered(const TwoSrc& src, int64_t nrows, int64_t ncols, const int64_t* out_start,
                          int32_t* deg_out, int32_t* adj_out, int64_t* W_out, int family, int64_t raw_bound,
                          cudaStream_t s) {
  if (nrows <= 0) return;
  static bool attr_set = false;
  if (!attr_set) {
    GP_CUDA(cudaFuncSetAttribute(k_merge_hash_blk<kHashTB3, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kHashSmemB3));
    attr_set = true;
  }
  unsigned* cnts = dnew<unsigned>(4, s);  // tier-2 list, tier-3 list, huge list, tier-1 list
  GP_CUDA(cudaMemsetAsync(cnts, 0, 4 * sizeof(unsigned), s));
  int32_t* l1 = dnew<int32_t>(nrows, s);
  int32_t* l2 = dnew<int32_t>(nrows, s);
  int32_t* l3 = dnew<int32_t>(nrows, s);
  int32_t* lh = dnew<int32_t>(nrows, s);
  const int sms = num_sms();
  if (raw_bound <= 20 * nrows) {
    // short rows on average (the symmetrisation: out-row + in-row): tier 0 merges rows of <= 32 raw
    // entries in registers (a warp each, 32 rows measured per warp step) and lists the others by tier;
    // tier 1 (a warp and a 256-entry table per row) takes its list
    const int64_t want0 = (nrows + 255) / 256;
    const unsigned grid0 = (unsigned)(want0 < (int64_t)sms * 16 ? want0 : (int64_t)sms * 16);
    GP_LAUNCH(family, k_merge_match, grid0, 256, 0, s, src, nrows, out_start, deg_out, adj_out, W_out, l1,
              cnts + 3, (int64_t)kHashT1 / 2, l2, cnts, (int64_t)kHashT2 / 2, l3, cnts + 1, (int64_t)kBlockCap, lh,
              cnts + 2, family);
    GP_LAUNCH(family, (k_merge_hash<kHashT1, kHashW1>), (unsigned)(sms * 16), kHashW1 * 32, kHashSmem1, s, src,
              nrows, (const int32_t*)l1, (const unsigned*)(cnts + 3), out_start, deg_out, adj_out, W_out, l2, cnts,
              (int64_t)kHashT2 / 2, l3, cnts + 1, (int64_t)kBlockCap, lh, cnts + 2, family);
  } else {
    // longer rows (the contraction): tier 1 over every row, longer ones to their tier's list
    const int64_t want = (nrows + kHashW1 - 1) / kHashW1;
    const unsigned grid1 = (unsigned)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
    GP_LAUNCH(family, (k_merge_hash<kHashT1, kHashW1>), grid1, kHashW1 * 32, kHashSmem1, s, src, nrows,
              (const int32_t*)nullptr, (const unsigned*)nullptr, out_start, deg_out, adj_out, W_out, l2, cnts,
              (int64_t)kHashT2 / 2, l3, cnts + 1, (int64_t)kBlockCap, lh, cnts + 2, family);
  }
  GP_LAUNCH(family, (k_merge_hash_blk<kHashTB2, 256>), (unsigned)(8 * sms), 256, kHashSmemB2, s, src,
            (const int32_t*)l2, (const unsigned*)cnts, out_start, deg_out, adj_out, W_out, family);
  GP_LAUNCH(family, (k_merge_hash_blk<kHashTB3, 1024>), (unsigned)sms, 1024, kHashSmemB3, s, src,
            (const int32_t*)l3, (const unsigned*)(cnts + 1), out_start, deg_out, adj_out, W_out, family);
  int nbits = 1;
  while (nbits < 31 && (int64_t(1) << nbits) < ncols) nbits++;
  int32_t* tk = dnew<int32_t>(raw_bound, s);
  int64_t* tv = dnew<int64_t>(raw_bound, s);
  GP_LAUNCH(family, k_merge_huge, (unsigned)sms, kHugeThreads, 0, s, src, lh, cnts + 2, out_start, deg_out, adj_out,
            W_out, tk, tv, nbits, family);
  GP_CHECK_LAUNCH();
  dfree(tk, s);
  dfree(tv, s);
  dfree(l1, s);
  dfree(l2, s);
  dfree(l3, s);
  dfree(lh, s);
  dfree(cnts, s);
}

}  // namespace gp
