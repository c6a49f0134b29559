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
  for (int32_t l = 0; l < nlev; l++) {
    const int64_t beg = lev_ptr[l], end = lev_ptr[l + 1];
    // all lanes of a group share i, so they run the same iterations and the group shuffle is safe
    for (int64_t i = beg + group; i < end; i += ngroups) {
      unsigned long long best = 0;
      const int32_t v = lev_vtx[i];
      const uint8_t p = part[v];
      if (p > 1) atomicOr(bad_part, 1);
      const int64_t eb = lo_off[i], ee = lo_off[i + 1];
      for (int64_t e = eb + sub; e < ee; e += G) {
        const unsigned long long f = __ldcg(fp + lo_src[e]);  // written by other blocks: bypass L1
        const unsigned long long t = (f >> 1) + (((uint8_t)(f & 1ull) != p) ? (unsigned long long)lo_w[e] : 0ull);
        best = t > best ? t : best;
      }
      if (sub == 0) bytes += 4ull + 1ull + 16ull + (unsigned long long)(ee - eb) * 16ull + 4ull + 8ull;
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        const unsigned long long q = __shfl_xor_sync(gmask, best, o, G);
        best = q > best ? q : best;
      }
      if (sub == 0) {
        const unsigned long long fin = best + (unsigned long long)(p ? lo_cG[i] : lo_cC[i]);
        fp[i] = (fin << 1) | (unsigned long long)p;
        local_max = fin > local_max ? fin : local_max;
        if (finish_out) finish_out[lev_vtx[i]] = (int64_t)fin;
      }
    }
    cluster_sync();
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
