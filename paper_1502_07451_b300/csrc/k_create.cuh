// k_create.cuh -- graph creation for many DAGs in one persistent launch.
//
// A CTA takes the next DAG from a queue (largest first) and builds what gp_graph_create builds for
// it, with the same checks in the same precedence: validation and exact sums, the transpose (in-CSR)
// and the self-loop check, the topological levels by Kahn's algorithm (one __syncthreads per level),
// the level-ordered in-CSR of the makespan, and the symmetrised level 0 (out-row + in-row of every
// vertex, merged by the batch kernel's hash tiers).  Scratch comes from the CTA's slot; the outputs go
// to the arrays the host laid out for the handle.
#pragma once
#include "gp_internal.cuh"
#include "k_batch.cuh"
#include "k_graph.cuh"

namespace gp {

struct CreateJob {
  int64_t n, m;
  const int64_t* off;  // device copies of the inputs
  const int32_t* cols;
  const int32_t* w;
  const int32_t* cC;
  const int32_t* cG;
  int64_t* in_off;
  int32_t* in_src;
  int32_t* in_w;
  int32_t* lev_vtx;
  int64_t* lev_ptr;
  int32_t* level;
  int64_t* lo_off;
  int32_t* lo_src;
  int32_t* lo_w;
  int32_t* lo_cC;
  int32_t* lo_cG;
  int64_t* start;  // level 0
  int32_t* deg;
  int32_t* adj;
  int64_t* W;
  int64_t* vC;
  int64_t* vG;
};

struct CreateOut {
  int32_t status, nlev;
  long long SC, SG, a0, max_width;
};

// exclusive scan of x(i) for i < N into out(i); returns the total
template <class F, class O>
__device__ long long cta_scan_excl(int64_t N, F x_of, O store, long long* sh) {
  long long run = 0;
  for (int64_t b = 0; b < N; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const long long x = i < N ? x_of(i) : 0;
    long long tot;
    const long long inc = cta_scan_incl<long long>(x, sh, tot);
    if (i < N) store(i, run + inc - x);
    run += tot;
  }
  return run;
}

__device__ void create_graph(const CreateJob& J, CreateOut* out, char* slot, unsigned long long slot_bytes,
                             unsigned char* dsm, int dsm_bytes) {
  __shared__ long long s_red[32];
  __shared__ unsigned long long s_redu[32];
  __shared__ int s_bad, s_self;
  __shared__ unsigned long long s_tail, s_end;
  __shared__ unsigned s_cnt;
  const int64_t n = J.n, m = J.m;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  CreateOut o{};
  if (threadIdx.x == 0) {
    s_bad = 0;
    s_self = 0;
  }
  __syncthreads();
  // ---- validation and exact sums (each cost < 2^31 and n, m < 2^31: the sums fit 64 bits)
  unsigned long long sw = 0, sc = 0, sg = 0;
  if (threadIdx.x == 0 && (J.off[0] != 0 || J.off[n] != m)) s_bad = 1;
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
    const int32_t a = J.cC[v], b = J.cG[v];
    if (J.off[v + 1] < J.off[v] || a < 0 || b < 0) s_bad = 1;
    sc += (unsigned long long)(a < 0 ? 0 : a);
    sg += (unsigned long long)(b < 0 ? 0 : b);
  }
  for (int64_t e = threadIdx.x; e < m; e += blockDim.x) {
    const int32_t c = J.cols[e], x = J.w[e];
    if (c < 0 || c >= n || x < 0) s_bad = 1;
    sw += (unsigned long long)(x < 0 ? 0 : x);
  }
  sw = block_sum<unsigned long long>(sw, s_redu);
  sc = block_sum<unsigned long long>(sc, s_redu);
  sg = block_sum<unsigned long long>(sg, s_redu);
  if (s_bad) {
    if (threadIdx.x == 0) {
      o.status = GP_ERR_INVALID;
      *out = o;
    }
    __syncthreads();
    return;
  }
  const unsigned long long lim = (unsigned long long)kSumLimit;
  if (sw > lim || sc > lim || sg > lim) {
    if (threadIdx.x == 0) {
      o.status = GP_ERR_OVERFLOW;
      *out = o;
    }
    __syncthreads();
    return;
  }
  o.SC = (long long)sc;
  o.SG = (long long)sg;
  // ---- slot scratch
  SlotArena A{slot, slot_bytes, 0ull, false};
  int32_t* cursor = A.get<int32_t>(n);
  int32_t* rem = A.get<int32_t>(n);
  int32_t* pos_of = A.get<int32_t>(n);
  int32_t* lo_deg = A.get<int32_t>(n);
  long long* rawlen = A.get<long long>(n);
  int32_t* biglist = A.get<int32_t>(n);
  int64_t* acc = A.get<int64_t>(n);
  int32_t* mark = A.get<int32_t>(n);
  if (A.fail) {  // the host sizes the slots for the largest graph: not reached
    if (threadIdx.x == 0) {
      o.status = GP_ERR_OOM;
      *out = o;
    }
    __syncthreads();
    return;
  }
  // ---- transpose and self-loop check (warp per source row)
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
    cursor[v] = 0;
    acc[v] = 0;
    mark[v] = -1;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < m; e += blockDim.x) atomicAdd(&cursor[J.cols[e]], 1);
  __syncthreads();
  {
    const long long tot = cta_scan_excl(
        n, [&](int64_t i) { return (long long)cursor[i]; }, [&](int64_t i, long long x) { J.in_off[i] = x; },
        s_red);
    if (threadIdx.x == 0) J.in_off[n] = tot;
  }
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) cursor[v] = 0;
  __syncthreads();
  for (int64_t u = wib; u < n; u += nw) {
    const int64_t b = J.off[u], e_end = J.off[u + 1];
    for (int64_t e = b + lane; e < e_end; e += 32) {
      const int32_t v = J.cols[e];
      if (v == (int32_t)u) s_self = 1;
      const int64_t pos = J.in_off[v] + atomicAdd(&cursor[v], 1);
      J.in_src[pos] = (int32_t)u;
      J.in_w[pos] = J.w[e];
    }
  }
  __syncthreads();
  if (s_self) {
    if (threadIdx.x == 0) {
      o.status = GP_ERR_NOT_DAG;
      *out = o;
    }
    __syncthreads();
    return;
  }
  // ---- Kahn's algorithm: one __syncthreads per level, a group of 4 lanes per frontier vertex
  if (threadIdx.x == 0) s_tail = 0;
  __syncthreads();
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
    const int32_t d = (int32_t)(J.in_off[v + 1] - J.in_off[v]);
    rem[v] = d;
    if (d == 0) {
      J.lev_vtx[atomicAdd(&s_tail, 1ull)] = (int32_t)v;
      J.level[v] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) s_end = s_tail;
  __syncthreads();
  int64_t beg = 0, end = (int64_t)s_end, maxw = 0;
  int32_t lev = 0;
  constexpr int G = 4;
  const int64_t group = threadIdx.x / G, ngroups = blockDim.x / G;
  const int sub = threadIdx.x % G;
  while (end > beg) {
    if (threadIdx.x == 0) J.lev_ptr[lev] = beg;
    maxw = (end - beg) > maxw ? (end - beg) : maxw;
    for (int64_t i = beg + group; i < end; i += ngroups) {
      const int32_t v = J.lev_vtx[i];
      for (int64_t e = J.off[v] + sub; e < J.off[v + 1]; e += G) {
        const int32_t w = J.cols[e];
        if (atomicSub(&rem[w], 1) == 1) {
          J.lev_vtx[atomicAdd(&s_tail, 1ull)] = w;
          J.level[w] = lev + 1;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_end = s_tail;
    __syncthreads();
    beg = end;
    end = (int64_t)s_end;
    lev++;
  }
  if (threadIdx.x == 0) J.lev_ptr[lev] = beg;
  if (beg != n) {
    if (threadIdx.x == 0) {
      o.status = GP_ERR_NOT_DAG;
      *out = o;
    }
    __syncthreads();
    return;
  }
  // ---- level-ordered in-CSR (sources by level position)
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int32_t v = J.lev_vtx[i];
    pos_of[v] = (int32_t)i;
    lo_deg[i] = (int32_t)(J.in_off[v + 1] - J.in_off[v]);
    J.lo_cC[i] = J.cC[v];
    J.lo_cG[i] = J.cG[v];
  }
  __syncthreads();
  {
    const long long tot = cta_scan_excl(
        n, [&](int64_t i) { return (long long)lo_deg[i]; }, [&](int64_t i, long long x) { J.lo_off[i] = x; }, s_red);
    if (threadIdx.x == 0) J.lo_off[n] = tot;
  }
  __syncthreads();
  for (int64_t i = wib; i < n; i += nw) {
    const int32_t v = J.lev_vtx[i];
    const int64_t b = J.in_off[v], d = J.in_off[v + 1] - b, o2 = J.lo_off[i];
    for (int64_t k = lane; k < d; k += 32) {
      J.lo_src[o2 + k] = pos_of[J.in_src[b + k]];
      J.lo_w[o2 + k] = J.in_w[b + k];
    }
  }
  // ---- symmetrised level 0: row v = out-row(v) + in-row(v), merged
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
    rawlen[v] = (J.off[v + 1] - J.off[v]) + (J.in_off[v + 1] - J.in_off[v]);
    J.vC[v] = J.cC[v];
    J.vG[v] = J.cG[v];
  }
  __syncthreads();
  {
    const long long tot = cta_scan_excl(
        n, [&](int64_t i) { return rawlen[i]; }, [&](int64_t i, long long x) { J.start[i] = x; }, s_red);
    if (threadIdx.x == 0) J.start[n] = tot;
  }
  __syncthreads();
  TwoSrc src{};
  src.a_start = J.off;
  src.a_col = J.cols;
  src.a_w32 = J.w;
  src.b_start = J.in_off;
  src.b_col = J.in_src;
  src.b_w32 = J.in_w;
  src.drop_self = 0;
  b_merge_rows(src, n, J.start, J.deg, J.adj, J.W, biglist, acc, mark, 256, dsm, dsm_bytes, &s_cnt, F_SYM_MERGE);
  long long a0 = 0;
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) a0 += J.deg[v];
  a0 = block_sum<long long>(a0, s_red);
  if (threadIdx.x == 0) {
    o.status = GP_OK;
    o.nlev = lev;
    o.a0 = a0;
    o.max_width = maxw;
    *out = o;
  }
  __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT, 2)
    k_create_batch(const CreateJob* __restrict__ jobs, const int32_t* __restrict__ order, int32_t count,
                   unsigned* queue, char* ws, unsigned long long slot_bytes, CreateOut* out) {
  extern __shared__ __align__(16) unsigned char dsm_c[];
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
    create_graph(jobs[gi], out + gi, slot, slot_bytes, dsm_c, dsm_bytes);
  }
}

// copies every graph's five input arrays from the caller's device buffers (block per graph)
struct CopyJob {
  int64_t n, m;
  const int64_t* off;
  const int32_t* cols;
  const int32_t* w;
  const int32_t* cC;
  const int32_t* cG;
  int64_t* d_off;
  int32_t* d_cols;
  int32_t* d_w;
  int32_t* d_cC;
  int32_t* d_cG;
};
__global__ void k_copy_inputs(const CopyJob* __restrict__ J, int count) {
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const CopyJob c = J[i];
    for (int64_t v = threadIdx.x; v <= c.n; v += blockDim.x) c.d_off[v] = c.off[v];
    for (int64_t v = threadIdx.x; v < c.n; v += blockDim.x) {
      c.d_cC[v] = c.cC[v];
      c.d_cG[v] = c.cG[v];
    }
    for (int64_t e = threadIdx.x; e < c.m; e += blockDim.x) {
      c.d_cols[e] = c.cols[e];
      c.d_w[e] = c.w[e];
    }
  }
}

}  // namespace gp
