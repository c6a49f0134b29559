// k_graph.cuh -- graph creation: validation, transpose, topological levels, symmetrisation inputs.
#pragma once
#include "gp_internal.cuh"
#include "k_scan.cuh"

namespace gp {

enum : int { VF_INVALID = 1, VF_SELFLOOP = 2 };

// 64-bit add into a 128-bit (lo, hi) accumulator.
__device__ __forceinline__ void add_u128(unsigned long long* acc, unsigned long long x) {
  if (x == 0) return;
  const unsigned long long old = atomicAdd(acc, x);
  if (old + x < old) atomicAdd(acc + 1, 1ull);
}

// Checks offsets, ids, costs; sums edge / CPU / GPU costs into sums[0..5] (three 128-bit values).
__global__ void __launch_bounds__(256)
    k_validate(int64_t n, int64_t m, const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
               const int32_t* __restrict__ w, const int32_t* __restrict__ cC,
               const int32_t* __restrict__ cG, int* flags, unsigned long long* sums) {
  __shared__ unsigned long long sh[32];
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int bad = 0;
  unsigned long long sw = 0, sc = 0, sg = 0;
  if (tid == 0 && (off[0] != 0 || off[n] != m)) bad = 1;
  for (int64_t v = tid; v < n; v += stride) {
    if (off[v + 1] < off[v]) bad = 1;
    const int32_t a = cC[v], b = cG[v];
    if (a < 0 || b < 0) bad = 1;
    sc += (unsigned long long)(a < 0 ? 0 : a);
    sg += (unsigned long long)(b < 0 ? 0 : b);
  }
  for (int64_t e = tid; e < m; e += stride) {
    const int32_t c = cols[e], x = w[e];
    if (c < 0 || c >= n || x < 0) bad = 1;
    sw += (unsigned long long)(x < 0 ? 0 : x);
  }
  if (bad) atomicOr(flags, VF_INVALID);
  sw = block_sum<unsigned long long>(sw, sh);
  sc = block_sum<unsigned long long>(sc, sh);
  sg = block_sum<unsigned long long>(sg, sh);
  if (threadIdx.x == 0) {
    add_u128(sums + 0, sw);
    add_u128(sums + 2, sc);
    add_u128(sums + 4, sg);
  }
}

__global__ void k_indeg(int64_t m, const int32_t* __restrict__ cols, int32_t* __restrict__ indeg) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&indeg[cols[e]], 1);
}

// in-CSR fill (G lanes per source row); also detects self-loops.  Blocks take chunks of consecutive
// source rows in order from a counter (`next`, zero at launch), so the whole grid works on neighbouring
// rows at any time: on a DAG whose edges stay near their source in id order, the in-rows the rows
// scatter to stay in L2 while their sectors fill up (a static grid-stride split lets the blocks drift
// apart, and the window of in-rows being written grows beyond the L2).
template <int G>  // lanes per row
__global__ void __launch_bounds__(256)
    k_fill_in(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
              const int32_t* __restrict__ w, const int64_t* __restrict__ in_off, int32_t* cursor,
              int32_t* __restrict__ in_src, int32_t* __restrict__ in_w, int* flags, unsigned long long* next) {
  constexpr int kGroups = 256 / G, kRows = 4 * kGroups;  // rows per chunk: four per group
  __shared__ long long s_base;
  const int sub = threadIdx.x % G, group = threadIdx.x / G;
  for (;;) {
    if (threadIdx.x == 0) s_base = (long long)atomicAdd(next, (unsigned long long)kRows);
    __syncthreads();
    const int64_t base = s_base;
    __syncthreads();  // every thread has read the chunk before thread 0 takes the next
    if (base >= n) break;
    const int64_t end = base + kRows < n ? base + kRows : n;
    for (int64_t u = base + group; u < end; u += kGroups) {
      const int64_t b = off[u], e_end = off[u + 1];
      for (int64_t e = b + sub; e < e_end; e += G) {
        const int32_t v = cols[e];
        if (v == (int32_t)u) atomicOr(flags, VF_SELFLOOP);
        const int64_t pos = in_off[v] + atomicAdd(&cursor[v], 1);
        in_src[pos] = (int32_t)u;
        in_w[pos] = w[e];
      }
    }
  }
}

// Kahn's algorithm, level-synchronous.  Level l holds the vertices whose longest path from a source
// has l edges: lev_vtx[lev_ptr[l] .. lev_ptr[l+1]).  Every placed vertex also gets a frontier record
// frec[pos] = (row start, vertex << 32 | row length).  Three kernels share the work:
//   k_levels_init   (grid)      in-degree counters, the sources as level 0, L2 prefetch of the rows;
//   k_levels_cta    (one CTA)   levels up to max_width vertices, one __syncthreads() per level (one SM
//                               issues every gather and counter decrement of a level, so it only
//                               pays on narrow levels: the host sets max_width to about 1,300
//                               out-entries' worth of vertices);
//   k_levels        (cluster)   resumes where the CTA kernel stopped (a wider level), if it did.
// New frontier vertices of level l+1 are appended after level l with counter cnt[(l+1) % 3]; the
// counter of level l+2 is cleared during level l, after every thread has read it as the size of level
// l-1, so one barrier per level suffices.  cnt[3] receives the number of vertices placed (n exactly
// when the graph is acyclic).  resume = {level, begin, end, done}.
__global__ void k_levels_init(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                              const int64_t* __restrict__ in_off, int32_t* rem, int32_t* lev_vtx, int32_t* level,
                              unsigned long long* cnt, longlong2* frec) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  prefetch_l2(off, sizeof(int64_t) * (size_t)(n + 1));  // the level loop chases these: keep them in L2
  prefetch_l2(cols, sizeof(int32_t) * (size_t)off[n]);
  for (int64_t v = tid; v < n; v += stride) {
    const int32_t d = (int32_t)(in_off[v + 1] - in_off[v]);
    rem[v] = d;
    if (d == 0) {
      const unsigned long long pos = atomicAdd(&cnt[0], 1ull);
      lev_vtx[pos] = (int32_t)v;
      level[v] = 0;
      frec[pos] = make_longlong2(off[v], ((long long)v << 32) | (long long)(off[v + 1] - off[v]));
    }
  }
}

constexpr int kLevCap = 4096;            // frontier records of a level kept in shared memory
constexpr int kLevK = 8;                 // out-entries per lane in flight
constexpr size_t kLevCtaSmem = 2 * kLevCap * sizeof(longlong2);

// One CTA of 1,024 threads; requires m < 2^31.  A warp takes 32 frontier vertices, and its lanes split
// their out-entries evenly (a lane's share is contiguous in the concatenation of the 32 rows), kLevK
// at a time: the column ids are loaded together, then the counter decrements are issued together with
// the loads of the successors' row ranges, so that a level costs two dependent round trips.
__global__ void __launch_bounds__(1024, 1)
    k_levels_cta(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ cols, int32_t* rem,
                 int32_t* lev_vtx, int64_t* lev_ptr, int32_t* level, unsigned long long* cnt, int32_t* nlev_out,
                 longlong2* frec, int64_t* resume, int64_t max_width) {
  extern __shared__ __align__(16) unsigned char lev_smem[];
  longlong2* buf = (longlong2*)lev_smem;  // [2][kLevCap]
  __shared__ unsigned int s_cnt[3];
  __shared__ int32_t s_incl[32][32];
  __shared__ int32_t s_eb[32][32];
  __shared__ unsigned long long sacc[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long bytes = 0;
  if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
  int64_t beg = 0, end = (int64_t)__ldcg(&cnt[0]);
  int32_t lev = 0;
  __syncthreads();
  while (end > beg) {
    if (end - beg > max_width) {  // uniform: every thread holds the same bounds
      if (threadIdx.x == 0) {
        resume[0] = lev;
        resume[1] = beg;
        resume[2] = end;
        resume[3] = 0;
        cnt[(lev + 1) % 3] = 0;
        cnt[(lev + 2) % 3] = 0;
      }
      account(F_LEVELS, bytes, sacc);
      return;
    }
    if (threadIdx.x == 0) {
      lev_ptr[lev] = beg;
      s_cnt[(lev + 2) % 3] = 0;
    }
    unsigned int* app = &s_cnt[(lev + 1) % 3];
    const longlong2* cur = buf + (size_t)(lev & 1) * kLevCap;
    longlong2* nxt = buf + (size_t)((lev + 1) & 1) * kLevCap;
    for (int64_t base = beg + (int64_t)warp * 32; base < end; base += 1024) {
      const int64_t i = base + lane;
      int32_t eb = 0, len = 0;
      if (i < end) {
        const longlong2 rec = (lev > 0 && i - beg < kLevCap) ? cur[i - beg] : __ldcg(frec + i);
        eb = (int32_t)rec.x;
        len = (int32_t)(rec.y & 0xFFFFFFFFll);
        bytes += 48ull + 12ull * (unsigned long long)len;
      }
      int32_t incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
      s_incl[warp][lane] = incl;
      s_eb[warp][lane] = eb;
      __syncwarp();
      const int32_t per = (total + 31) >> 5;
      int32_t k = lane * per < total ? lane * per : total;
      const int32_t k_end = k + per < total ? k + per : total;
      // the row holding entry k: first j with incl[j] > k
      int32_t j = 0;
      if (k < k_end) {
        int32_t lo = 0, hi = 31;
        while (lo < hi) {
          const int32_t mid = (lo + hi) >> 1;
          if (s_incl[warp][mid] > k) hi = mid;
          else lo = mid + 1;
        }
        j = lo;
      }
      while (k < k_end) {
        int32_t w[kLevK];
#pragma unroll
        for (int q = 0; q < kLevK; q++) {
          w[q] = -1;
          if (k < k_end) {
            while (s_incl[warp][j] <= k) j++;
            const int32_t excl = j ? s_incl[warp][j - 1] : 0;  // entries of the rows before row j
            w[q] = cols[s_eb[warp][j] + (k - excl)];
            k++;
          }
        }
        int32_t r[kLevK], ub[kLevK], ue[kLevK];
#pragma unroll
        for (int q = 0; q < kLevK; q++) {
          r[q] = 0;
          if (w[q] >= 0) {
            r[q] = atomicSub(&rem[w[q]], 1);
            ub[q] = (int32_t)off[w[q]];  // in flight with the decrement
            ue[q] = (int32_t)off[w[q] + 1];
          }
        }
#pragma unroll
        for (int q = 0; q < kLevK; q++) {
          if (w[q] >= 0 && r[q] == 1) {
            const unsigned int a = atomicAdd(app, 1u);
            const int64_t pos = end + (int64_t)a;
            const longlong2 rec = make_longlong2((long long)ub[q], ((long long)w[q] << 32) | (long long)(ue[q] - ub[q]));
            lev_vtx[pos] = w[q];
            level[w[q]] = lev + 1;
            frec[pos] = rec;
            if (a < (unsigned int)kLevCap) nxt[a] = rec;
            if (ue[q] > ub[q]) asm volatile("prefetch.global.L2 [%0];" ::"l"(cols + ub[q]));
          }
        }
      }
      __syncwarp();
    }
    __syncthreads();
    beg = end;
    end = beg + (int64_t)*(volatile unsigned int*)app;
    lev++;
  }
  if (threadIdx.x == 0) {
    lev_ptr[lev] = beg;
    *nlev_out = lev;
    cnt[3] = (unsigned long long)beg;
    resume[3] = 1;
  }
  account(F_LEVELS, bytes, sacc);
}

// The cluster kernel: continues from resume = {level, begin, end, done} (nothing to do when done).
template <int G>
__global__ void __launch_bounds__(1024)
    k_levels(const int64_t* __restrict__ off, const int32_t* __restrict__ cols, int32_t* rem, int32_t* lev_vtx,
             int64_t* lev_ptr, int32_t* level, unsigned long long* cnt, int32_t* nlev_out, longlong2* frec,
             const int64_t* resume) {
  __shared__ unsigned long long sacc[32];
  if (__ldcg(resume + 3)) return;  // the CTA kernel placed every level
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t group = tid / G, ngroups = stride / G;
  const int sub = (int)(tid % G);
  // algorithmic bytes: per vertex its in-range (16), counter init (4), frontier slot (4), row range
  // (16), level-order slot and level (8); per out-entry the id (4) and the counter decrement (8)
  unsigned long long bytes = 0;
  // where the CTA kernel stopped; when it did not run, level 0 as the init kernel left it
  const int64_t r_end = __ldcg(resume + 2);
  int64_t beg = __ldcg(resume + 1), end = r_end ? r_end : (int64_t)__ldcg(&cnt[0]);
  int32_t lev = (int32_t)__ldcg(resume + 0);
  while (end > beg) {
    if (tid == 0) {
      lev_ptr[lev] = beg;
      cnt[(lev + 2) % 3] = 0;
    }
    unsigned long long* app = &cnt[(lev + 1) % 3];
    for (int64_t i = beg + group; i < end; i += ngroups) {
      // the record its producer wrote (row range loaded there, under that level's barrier)
      const longlong2 rec = __ldcg(frec + i);  // written by other CTAs: bypass L1
      const int64_t eb = rec.x, ee = eb + (rec.y & 0xFFFFFFFFll);
      if (sub == 0) bytes += 48ull + 12ull * (unsigned long long)(ee - eb);
      // two out-entries per lane at a time: both decrements are in flight together, and with them the
      // successors' row ranges (needed by the one whose count reaches zero)
      for (int64_t e = eb + sub; e < ee; e += 2 * G) {
        const bool two = e + G < ee;
        const int32_t u1 = cols[e];
        const int32_t u2 = two ? cols[e + G] : -1;
        const int r1 = atomicSub(&rem[u1], 1);
        const int r2 = two ? atomicSub(&rem[u2], 1) : 0;
        const int64_t ub1 = off[u1], ue1 = off[u1 + 1];
        int64_t ub2 = 0, ue2 = 0;
        if (two) {
          ub2 = off[u2];
          ue2 = off[u2 + 1];
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
          const int32_t u = q ? u2 : u1;
          if ((q ? r2 : r1) == 1) {
            const int64_t ub = q ? ub2 : ub1, ue = q ? ue2 : ue1;
            // warp-aggregated append: one atomic per set of lanes that got here together
            const unsigned act = __activemask();
            const int lane = threadIdx.x & 31;
            const int leader = __ffs(act) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(app, (unsigned long long)__popc(act));
            base = __shfl_sync(act, base, leader);
            const unsigned long long k = base + (unsigned long long)__popc(act & ((1u << lane) - 1u));
            lev_vtx[end + (int64_t)k] = u;
            level[u] = lev + 1;
            frec[end + (int64_t)k] = make_longlong2(ub, ((long long)u << 32) | (long long)(ue - ub));
          }
        }
      }
    }
    cluster_sync();
    beg = end;
    end = beg + (int64_t) * (volatile unsigned long long*)app;
    lev++;
  }
  if (tid == 0) {
    lev_ptr[lev] = beg;
    *nlev_out = lev;
    cnt[3] = (unsigned long long)beg;
  }
  account(F_LEVELS, bytes, sacc);
}

// {vertices placed, levels, widest level} of a traversal (one block)
__global__ void k_level_summary(const unsigned long long* placed, const int32_t* nlev, const int64_t* lev_ptr,
                                int64_t* out) {
  __shared__ long long sh[32];
  const int32_t L = *nlev;
  long long mw = 0;
  for (int32_t l = threadIdx.x; l < L; l += blockDim.x) {
    const long long w = lev_ptr[l + 1] - lev_ptr[l];
    mw = w > mw ? w : mw;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long q = __shfl_xor_sync(0xffffffffu, mw, o);
    mw = q > mw ? q : mw;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mw;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = sh[w] > m ? sh[w] : m;
    out[0] = (int64_t)*placed;
    out[1] = L;
    out[2] = m;
  }
}

// position i of the level order: vertex, in-degree, costs (positions a cyclic graph left unplaced hold
// -1 when the level order was cleared first, and get no entries)
__global__ void k_lo_prep(int64_t n, const int32_t* __restrict__ lev_vtx, const int64_t* __restrict__ in_off,
                          const int32_t* __restrict__ cC, const int32_t* __restrict__ cG,
                          int32_t* __restrict__ pos_of, int32_t* __restrict__ lo_deg,
                          int32_t* __restrict__ lo_cC, int32_t* __restrict__ lo_cG) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = lev_vtx[i];
    if (v < 0) {
      lo_deg[i] = 0;
      lo_cC[i] = 0;
      lo_cG[i] = 0;
      continue;
    }
    pos_of[v] = (int32_t)i;
    lo_deg[i] = (int32_t)(in_off[v + 1] - in_off[v]);
    lo_cC[i] = cC[v];
    lo_cG[i] = cG[v];
  }
}

template <int G>  // lanes per position
__global__ void __launch_bounds__(256)
    k_lo_fill(int64_t n, const int32_t* __restrict__ lev_vtx, const int64_t* __restrict__ in_off,
              const int32_t* __restrict__ in_src, const int32_t* __restrict__ in_w,
              const int32_t* __restrict__ pos_of, const int64_t* __restrict__ lo_off,
              int32_t* __restrict__ lo_src, int32_t* __restrict__ lo_w) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sub = threadIdx.x % G;
  const int64_t gw = tid / G, nw = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t i = gw; i < n; i += nw) {
    const int32_t v = lev_vtx[i];
    if (v < 0) continue;  // unplaced (cyclic graph): no entries
    const int64_t b = in_off[v], d = in_off[v + 1] - b, o = lo_off[i];
    for (int64_t k = sub; k < d; k += G) {
      lo_src[o + k] = pos_of[in_src[b + k]];
      lo_w[o + k] = in_w[b + k];
    }
  }
}

__global__ void k_rawlen_sym(int64_t n, const int64_t* __restrict__ off, const int64_t* __restrict__ in_off,
                             int64_t* __restrict__ rawlen) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    rawlen[v] = (off[v + 1] - off[v]) + (in_off[v + 1] - in_off[v]);
}

__global__ void k_widen(int64_t n, const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                        int64_t* __restrict__ wa, int64_t* __restrict__ wb) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    wa[v] = a[v];
    wb[v] = b[v];
  }
}

__global__ void k_sum_deg(int64_t n, const int32_t* __restrict__ deg, unsigned long long* out) {
  __shared__ unsigned long long sh[32];
  unsigned long long s = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    s += (unsigned long long)deg[v];
  s = block_sum<unsigned long long>(s, sh);
  if (threadIdx.x == 0 && s) atomicAdd(out, s);
}

__global__ void k_sum_i64(int64_t n, const int64_t* __restrict__ x, unsigned long long* out) {
  __shared__ unsigned long long sh[32];
  unsigned long long s = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    s += (unsigned long long)x[v];
  s = block_sum<unsigned long long>(s, sh);
  if (threadIdx.x == 0 && s) atomicAdd(out, s);
}

// sum of non-negative int64 values into *out (zeroed here)
void sum_i64(const int64_t* x, int64_t n, long long* out, cudaStream_t s) {
  GP_CUDA(cudaMemsetAsync(out, 0, sizeof(long long), s));
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  GP_LAUNCH(F_MISC, k_sum_i64, (unsigned)(want < 1 ? 1 : (want < cap ? want : cap)), 256, 0, s, n, x,
            (unsigned long long*)out);
  GP_CHECK_LAUNCH();
}

// padded CSR -> compact CSR copy (warp per row); coff must hold the exclusive scan of deg
__global__ void __launch_bounds__(256)
    k_compact_rows(int64_t n, const int64_t* __restrict__ start, const int32_t* __restrict__ deg,
                   const int32_t* __restrict__ adj, const int64_t* __restrict__ W,
                   const int64_t* __restrict__ coff, int32_t* __restrict__ cadj, int64_t* __restrict__ cW) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = gw; v < n; v += nw) {
    const int64_t b = start[v], o = coff[v];
    const int32_t d = deg[v];
    for (int32_t k = lane; k < d; k += 32) {
      cadj[o + k] = adj[b + k];
      cW[o + k] = W[b + k];
    }
  }
}

// compact CSR -> (start, deg) view
__global__ void k_deg_from_off(int64_t n, const int64_t* __restrict__ off, int32_t* __restrict__ deg) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    deg[v] = (int32_t)(off[v + 1] - off[v]);
}

__global__ void k_fill_u8(int64_t n, uint8_t* p, uint8_t x) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    p[v] = x;
}

// fixed-vertex values outside {-1, 0, 1} set *bad
__global__ void k_fix_check(int64_t n, const int8_t* __restrict__ fix, int* bad) {
  bool b = false;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    b |= fix[v] < -1 || fix[v] > 1;
  if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) *bad = 1;
}

}  // namespace gp
