// k_makespan.cuh -- makespan of a CPU/GPU mapping (max-plus longest path) and the cut.
//
// finish(v) = t_side(v)(v) + max over entries u->v of (finish(u) + [side(u) != side(v)] w(u,v)),
// the max over no entries being 0, and makespan = max_v finish(v).  Vertices are visited level by
// level of the topological order (one thread-block cluster, the hardware cluster barrier between
// levels); within a level, a group of G lanes reduces one vertex's in-entries.  finish is kept by level position,
// packed with the side bit (2 finish + side) so one gather gives both.
#pragma once
#include "gp_internal.cuh"

namespace gp {

// The static data of a group's first vertex in a level (vertex, side, in-entry range, the lane's
// first in-entry, own time), loaded one level ahead so that after the barrier only the predecessor
// finish times remain on the critical path.
struct MsItem {
  int64_t i, eb, ee;
  int32_t v, src, w, src2, w2, cost;
  uint8_t p;
  bool valid;
};

template <int G>
__device__ __forceinline__ void ms_load(MsItem& it, int64_t i, int64_t end, int sub, const int32_t* lev_vtx,
                                        const int64_t* lo_off, const int32_t* lo_src, const int32_t* lo_w,
                                        const int32_t* lo_cC, const int32_t* lo_cG, const uint8_t* part) {
  it.valid = i < end;
  it.i = i;
  if (!it.valid) return;
  it.v = lev_vtx[i];
  it.eb = lo_off[i];
  it.ee = lo_off[i + 1];
  it.p = part[it.v];
  it.cost = it.p ? lo_cG[i] : lo_cC[i];
  const int64_t e = it.eb + sub;
  it.src = -1;
  it.w = 0;
  it.src2 = -1;
  it.w2 = 0;
  if (e < it.ee) {
    it.src = lo_src[e];
    it.w = lo_w[e];
  }
  if (e + G < it.ee) {  // a second entry per lane covers in-degrees up to 2G without a dependent load
    it.src2 = lo_src[e + G];
    it.w2 = lo_w[e + G];
  }
}

template <int G>
__global__ void __launch_bounds__(1024)
    k_makespan(int32_t nlev, const int64_t* __restrict__ lev_ptr, const int32_t* __restrict__ lev_vtx,
               const int64_t* __restrict__ lo_off, const int32_t* __restrict__ lo_src,
               const int32_t* __restrict__ lo_w, const int32_t* __restrict__ lo_cC,
               const int32_t* __restrict__ lo_cG, const uint8_t* __restrict__ part,
               unsigned long long* fp, unsigned long long* ms_out, int* bad_part,
               int64_t* __restrict__ finish_out) {
  __shared__ unsigned long long sh[32];
  __shared__ unsigned long long sacc[32];
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t group = tid / G, ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int sub = threadIdx.x % G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G));
  unsigned long long local_max = 0, bytes = 0;
  // one vertex of a level: finish = own time + max over in-entries (predecessor finish, plus the
  // transfer time when the sides differ); `first` carries the prefetched first entry of the lane
  auto finish_of = [&](const MsItem& it) {
    unsigned long long best = 0;
    const unsigned long long f1 = it.src >= 0 ? __ldcg(fp + it.src) : 0ull;  // written by other CTAs
    const unsigned long long f2 = it.src2 >= 0 ? __ldcg(fp + it.src2) : 0ull;
    if (it.src >= 0) best = (f1 >> 1) + (((uint8_t)(f1 & 1ull) != it.p) ? (unsigned long long)it.w : 0ull);
    if (it.src2 >= 0) {
      const unsigned long long t = (f2 >> 1) + (((uint8_t)(f2 & 1ull) != it.p) ? (unsigned long long)it.w2 : 0ull);
      best = t > best ? t : best;
    }
    for (int64_t e = it.eb + sub + 2 * G; e < it.ee; e += G) {
      const unsigned long long f = __ldcg(fp + lo_src[e]);
      const unsigned long long t = (f >> 1) + (((uint8_t)(f & 1ull) != it.p) ? (unsigned long long)lo_w[e] : 0ull);
      best = t > best ? t : best;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const unsigned long long q = __shfl_xor_sync(gmask, best, o, G);
      best = q > best ? q : best;
    }
    if (sub == 0) {
      if (it.p > 1) atomicOr(bad_part, 1);
      const unsigned long long fin = best + (unsigned long long)it.cost;
      fp[it.i] = (fin << 1) | (unsigned long long)(it.p & 1);
      local_max = fin > local_max ? fin : local_max;
      if (finish_out) finish_out[it.v] = (int64_t)fin;
      bytes += 4ull + 1ull + 16ull + (unsigned long long)(it.ee - it.eb) * 16ull + 4ull + 8ull;
    }
  };
  // static data of the group's first vertex two levels ahead: a level's dependent prefetch chain
  // (vertex -> side, row -> first entry) then has a whole level to complete
  MsItem cur, nx1, nx2;
  int64_t beg = lev_ptr[0], end = nlev > 0 ? lev_ptr[1] : 0;
  int64_t end1 = nlev > 1 ? lev_ptr[2] : end;  // end of level l+1
  ms_load<G>(cur, beg + group, end, sub, lev_vtx, lo_off, lo_src, lo_w, lo_cC, lo_cG, part);
  if (nlev > 1) ms_load<G>(nx1, end + group, end1, sub, lev_vtx, lo_off, lo_src, lo_w, lo_cC, lo_cG, part);
  for (int32_t l = 0; l < nlev; l++) {
    const int64_t end2 = (l + 2 < nlev) ? lev_ptr[l + 3] : end1;  // end of level l+2
    if (cur.valid) finish_of(cur);
    for (int64_t i = beg + group + ngroups; i < end; i += ngroups) {  // levels wider than the groups
      MsItem it;
      ms_load<G>(it, i, end, sub, lev_vtx, lo_off, lo_src, lo_w, lo_cC, lo_cG, part);
      finish_of(it);
    }
    cluster_arrive();
    if (l + 2 < nlev) ms_load<G>(nx2, end1 + group, end2, sub, lev_vtx, lo_off, lo_src, lo_w, lo_cC, lo_cG, part);
    cluster_wait();
    cur = nx1;
    nx1 = nx2;
    beg = end;
    end = end1;
    end1 = end2;
  }
  // block max
  {
    unsigned long long x = local_max;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long q = __shfl_xor_sync(0xffffffffu, x, o);
      x = q > x ? q : x;
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long mx = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) mx = sh[w] > mx ? sh[w] : mx;
      if (mx) atomicMax(ms_out, mx);
    }
  }
  account(F_MAKESPAN, bytes, sacc);
}

// cut over the directed out-CSR (warp per row)
__global__ void __launch_bounds__(256)
    k_cut(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
          const int32_t* __restrict__ w, const uint8_t* __restrict__ part, unsigned long long* cut,
          int* bad_part) {
  __shared__ unsigned long long sh[32];
  __shared__ unsigned long long sacc[32];
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long s = 0, bytes = 0;
  for (int64_t u = gw; u < n; u += nw) {
    const uint8_t pu = part[u];
    if (pu > 1 && lane == 0) atomicOr(bad_part, 1);
    const int64_t b = off[u], e_end = off[u + 1];
    for (int64_t e = b + lane; e < e_end; e += 32)
      if (part[cols[e]] != pu) s += (unsigned long long)w[e];
    if (lane == 0) bytes += 17ull + (unsigned long long)(e_end - b) * 9ull;
  }
  s = block_sum<unsigned long long>(s, sh);
  if (threadIdx.x == 0 && s) atomicAdd(cut, s);
  account(F_CUT, bytes, sacc);
}

}  // namespace gp
