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

// cut over the directed out-CSR: a group of G lanes per row (G from the average out-degree, about one
// entry per lane), so that a warp has 32 / G rows' loads in flight
template <int G>
__global__ void __launch_bounds__(256)
    k_cut(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
          const int32_t* __restrict__ w, const uint8_t* __restrict__ part, unsigned long long* cut,
          int* bad_part) {
  __shared__ unsigned long long sh[32];
  __shared__ unsigned long long sacc[32];
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t group = tid / G, ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int sub = threadIdx.x % G;
  unsigned long long s = 0, bytes = 0;
  for (int64_t u = group; u < n; u += ngroups) {
    const uint8_t pu = part[u];
    if (pu > 1 && sub == 0) atomicOr(bad_part, 1);
    const int64_t b = off[u], e_end = off[u + 1];
    for (int64_t e = b + sub; e < e_end; e += G)
      if (GP_IN(cols[e], n, 11) && part[cols[e]] != pu) s += (unsigned long long)w[e];
    if (sub == 0) bytes += 17ull + (unsigned long long)(e_end - b) * 9ull;
  }
  s = block_sum<unsigned long long>(s, sh);
  if (threadIdx.x == 0 && s) atomicAdd(cut, s);
  account(F_CUT, bytes, sacc);
}

}  // namespace gp

namespace gp {

// ------------------------------------------------------------------------------------------------
// The same recurrence with the predecessor finish times in distributed shared memory.  Every CTA of
// the cluster keeps a ring of the packed finish times of the last kMsR level positions.  A vertex's
// value goes to the ring of every CTA with st.async, whose completion counts bytes on that CTA's
// mbarrier for the level (two mbarriers alternate between even and odd levels); a CTA starts level
// l + 1 once its mbarrier has seen every value of level l.  No cluster barrier separates the levels,
// so a level costs one one-way remote store plus the vertex work.  A predecessor further back than
// the ring is read from the global copy, which the writing lane stores before its st.async (whose
// mbarrier completion releases it at cluster scope; the wait acquires at cluster scope).  A CTA is
// at most one level ahead of another's reads, so a level never overwrites a ring slot still needed
// when levels are at most kMsR wide.  Every wait is bounded: on expiry the kernel sets bit 1 of
// *bad_part, stops, and still meets the cluster barrier at its end.
// ------------------------------------------------------------------------------------------------
constexpr int kMsR = 8192;
constexpr size_t kMsRingBytes = (size_t)kMsR * sizeof(unsigned long long);

__device__ __forceinline__ uint32_t cluster_nranks() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void st_cluster_u64(uint32_t local_addr, uint32_t rank, unsigned long long v) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(local_addr), "r"(rank));
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(ra), "l"(v) : "memory");
}

// The lookahead of the distributed-shared-memory kernel, in two stages so that no load waits on
// another load of the same level: stage A (two levels ahead) loads what the position alone addresses
// (in-entry range, vertex, both costs); stage B (one level ahead) what stage A's values address (side,
// the lane's first two in-entries).  32-bit positions and in-entry indices.
struct MsA {
  int32_t i, eb, ee, v, cC, cG;
  bool valid;
};
struct MsB {
  int32_t i, eb, ee, src, w, src2, w2, cC, cG;
  uint8_t p;
  bool valid;
};

__device__ __forceinline__ void ms_load_a(MsA& a, int32_t i, int32_t end, const int32_t* lev_vtx, const int64_t* lo_off,
                                          const int32_t* lo_cC, const int32_t* lo_cG) {
  a.valid = i < end;
  a.i = i;
  if (!a.valid) return;
  a.eb = (int32_t)lo_off[i];
  a.ee = (int32_t)lo_off[i + 1];
  a.v = lev_vtx[i];
  a.cC = lo_cC[i];
  a.cG = lo_cG[i];
}

// st.async of one u64 into CTA `rank`'s shared memory at the offset of `local_addr`, counted (8 bytes)
// on that CTA's mbarrier at the offset of `local_bar`
__device__ __forceinline__ void st_async_u64(uint32_t local_addr, uint32_t rank, unsigned long long v,
                                             uint32_t local_bar) {
  uint32_t ra, rb;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(local_addr), "r"(rank));
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rb) : "r"(local_bar), "r"(rank));
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.u64 [%0], %1, [%2];" ::"r"(ra), "l"(v), "r"(rb)
               : "memory");
}
__device__ __forceinline__ void mbar_init_cluster(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// this thread's arrival on the phase plus the bytes the phase waits for
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// wait (acquire, cluster scope) for the phase of the given parity to complete; false after ~0.5 s
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  unsigned long long t0 = 0;
  for (uint32_t k = 0;; k++) {
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((k & 255u) == 0) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (k == 0) t0 = t;
      else if (t - t0 > 500000000ull) return false;
    }
  }
}

template <int G>
__device__ __forceinline__ void ms_load_b(MsB& b, const MsA& a, int sub, const int32_t* lo_src, const int32_t* lo_w,
                                          const uint8_t* part) {
  b.valid = a.valid;
  b.i = a.i;
  if (!a.valid) return;
  b.eb = a.eb;
  b.ee = a.ee;
  b.p = part[a.v];
  b.cC = a.cC;  // the side picks the cost when the vertex is computed (b.p may still be in flight)
  b.cG = a.cG;
  const int32_t e = a.eb + sub;
  b.src = -1;
  b.w = 0;
  b.src2 = -1;
  b.w2 = 0;
  if (e < a.ee) {
    b.src = lo_src[e];
    b.w = lo_w[e];
  }
  if (e + G < a.ee) {
    b.src2 = lo_src[e + G];
    b.w2 = lo_w[e + G];
  }
}

template <int G>
__global__ void __launch_bounds__(1024)
    k_makespan_dsm(int32_t nlev, const int64_t* __restrict__ lev_ptr, const int32_t* __restrict__ lev_vtx,
                   const int64_t* __restrict__ lo_off, const int32_t* __restrict__ lo_src,
                   const int32_t* __restrict__ lo_w, const int32_t* __restrict__ lo_cC,
                   const int32_t* __restrict__ lo_cG, const uint8_t* __restrict__ part,
                   unsigned long long* fp, unsigned long long* ms_out, int* bad_part,
                   int64_t* __restrict__ finish_out) {
  extern __shared__ __align__(16) unsigned long long ms_ring[];
  __shared__ __align__(8) unsigned long long ms_bar[2];
  __shared__ unsigned long long sh[32];
  __shared__ unsigned long long sacc[32];
  const int32_t tid = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  const int32_t group = tid / G, ngroups = (int32_t)(gridDim.x * blockDim.x) / G;
  const int sub = threadIdx.x % G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G));
  const uint32_t nranks = cluster_nranks();
  const uint32_t ring_base = (uint32_t)__cvta_generic_to_shared(ms_ring);
  const uint32_t bar_base = (uint32_t)__cvta_generic_to_shared(ms_bar);
  unsigned long long local_max = 0, bytes = 0;
  int32_t ring_lo = 0;
  auto pred = [&](int32_t sp) -> unsigned long long {
    return sp >= ring_lo ? ms_ring[sp & (kMsR - 1)] : __ldcg(fp + sp);
  };
  // packed finish (2 finish + side) of one vertex, in every lane of its group
  auto value_of = [&](const MsB& b) -> unsigned long long {
    const uint8_t p = b.p;
    unsigned long long best = 0;
    const int32_t e = b.eb + sub;
    if (b.src >= 0) {
      const unsigned long long f = pred(b.src);
      best = (f >> 1) + (((uint8_t)(f & 1ull) != p) ? (unsigned long long)b.w : 0ull);
    }
    if (b.src2 >= 0) {
      const unsigned long long f = pred(b.src2);
      const unsigned long long t = (f >> 1) + (((uint8_t)(f & 1ull) != p) ? (unsigned long long)b.w2 : 0ull);
      best = t > best ? t : best;
    }
    for (int32_t x = e + 2 * G; x < b.ee; x += G) {
      const unsigned long long f = pred(lo_src[x]);
      const unsigned long long t = (f >> 1) + (((uint8_t)(f & 1ull) != p) ? (unsigned long long)lo_w[x] : 0ull);
      best = t > best ? t : best;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const unsigned long long q = __shfl_xor_sync(gmask, best, o, G);
      best = q > best ? q : best;
    }
    const unsigned long long fin = best + (unsigned long long)(p ? b.cG : b.cC);
    if (sub == 0) {
      if (p > 1) atomicOr(bad_part, 1);
      local_max = fin > local_max ? fin : local_max;
      bytes += 4ull + 1ull + 16ull + (unsigned long long)(b.ee - b.eb) * 16ull + 4ull + 8ull;
    }
    return (fin << 1) | (unsigned long long)(p & 1);
  };
  // the value into the global copy and the ring of every CTA of the cluster, counted on that CTA's
  // mbarrier of the level's parity (the group's lanes share the ranks; each stores the global copy
  // before its remote stores, so that their release covers it)
  auto publish = [&](int32_t i, unsigned long long packed, uint32_t parity_bar) {
    fp[i] = packed;
    const uint32_t a = ring_base + (uint32_t)(i & (kMsR - 1)) * 8u;
    for (uint32_t r = (uint32_t)sub; r < nranks; r += G) st_async_u64(a, r, packed, parity_bar);
  };
  auto lp = [&](int32_t l) -> int32_t { return (int32_t)lev_ptr[l < nlev ? l : nlev]; };
  // level l's bounds [beg, end); end1, end2 = ends of levels l + 1, l + 2; end3 loaded one level ahead
  int32_t beg = lp(0), end = lp(1), end1 = lp(2), end2 = lp(3), end3 = lp(4);
  MsA a1, a2;
  MsB cur, b1;
  {
    MsA a0;
    ms_load_a(a0, beg + group, end, lev_vtx, lo_off, lo_cC, lo_cG);
    ms_load_a(a1, end + group, end1, lev_vtx, lo_off, lo_cC, lo_cG);
    ms_load_b<G>(cur, a0, sub, lo_src, lo_w, part);
  }
  if (threadIdx.x == 0) {
    mbar_init_cluster(bar_base, 1);
    mbar_init_cluster(bar_base + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (nlev > 0) mbar_expect(bar_base, 8u * (uint32_t)(end - beg));  // level 0's values
  }
  cluster_sync();  // every CTA's mbarriers are initialised before the first remote store
  bool failed = false;
  for (int32_t l = 0; l < nlev; l++) {
    // level l + 1's values are expected before this CTA sends any of level l's (so before any CTA
    // can send level l + 1's); the mbarrier's previous phase (level l - 1) has completed here
    if (threadIdx.x == 0 && !failed && l + 1 < nlev)
      mbar_expect(bar_base + 8u * ((l + 1) & 1), 8u * (uint32_t)(end1 - end));
    if (__syncthreads_or(failed)) break;  // a wait gave up somewhere in this CTA: stop together
    ring_lo = end - kMsR;
    const uint32_t bar_l = bar_base + 8u * (l & 1);
    if (cur.valid) {
      const unsigned long long pk = value_of(cur);
      publish(cur.i, pk, bar_l);
      if (finish_out && sub == 0) finish_out[lev_vtx[cur.i]] = (int64_t)(pk >> 1);
    }
    for (int32_t i = beg + group + ngroups; i < end; i += ngroups) {  // levels wider than the groups
      MsA a;
      MsB b;
      ms_load_a(a, i, end, lev_vtx, lo_off, lo_cC, lo_cG);
      ms_load_b<G>(b, a, sub, lo_src, lo_w, part);
      const unsigned long long pk = value_of(b);
      publish(i, pk, bar_l);
      if (finish_out && sub == 0) finish_out[a.v] = (int64_t)(pk >> 1);
    }
    // lookahead while the level's values travel: stage B of level l + 1 from stage A's registers,
    // stage A of level l + 2 from its bounds
    ms_load_b<G>(b1, a1, sub, lo_src, lo_w, part);
    ms_load_a(a2, end1 + group, end2, lev_vtx, lo_off, lo_cC, lo_cG);
    const int32_t end4 = lp(l + 5);
    if (!mbar_wait_bounded(bar_l, (uint32_t)((l >> 1) & 1))) {
      failed = true;
      atomicOr(bad_part, 2);
    }
    cur = b1;
    a1 = a2;
    beg = end;
    end = end1;
    end1 = end2;
    end2 = end3;
    end3 = end4;
  }
  cluster_sync();  // no CTA leaves while remote stores to it may be in flight
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

}  // namespace gp

namespace gp {

// ------------------------------------------------------------------------------------------------
// The same recurrence for DAGs whose levels are wider than the ring: one cooperative grid of up to one
// CTA per SM, so that a lane group has about one vertex per level, with the two-stage lookahead of
// k_makespan_dsm and predecessors read from the global copy (L2).  Levels are separated by a grid
// barrier of this kernel's own: every CTA's thread 0, after its CTA's stores and a fence, adds one to
// bar[0]; it then waits until bar[0] reaches (level + 1) x CTAs and fences again.  The waits are bounded
// by the global timer (0.5 s): on expiry the thread sets bit 1 of *bad_part, and its CTA (deciding
// together through __syncthreads_or) stops; the other CTAs' waits then expire too.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ bool grid_wait_bounded(const unsigned* bar, unsigned target) {
  unsigned long long t0 = 0;
  for (uint32_t k = 0;; k++) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
    if (v >= target) return true;
    if ((k & 63u) == 0) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (k == 0) t0 = t;
      else if (t - t0 > 500000000ull) return false;
    }
  }
}

template <int G>
__global__ void __launch_bounds__(1024, 1)
    k_makespan_grid(int32_t nlev, const int64_t* __restrict__ lev_ptr, const int32_t* __restrict__ lev_vtx,
                    const int64_t* __restrict__ lo_off, const int32_t* __restrict__ lo_src,
                    const int32_t* __restrict__ lo_w, const int32_t* __restrict__ lo_cC,
                    const int32_t* __restrict__ lo_cG, const uint8_t* __restrict__ part,
                    unsigned long long* fp, unsigned long long* ms_out, int* bad_part,
                    int64_t* __restrict__ finish_out, unsigned* bar) {
  __shared__ unsigned long long sh[32];
  __shared__ unsigned long long sacc[32];
  const int32_t tid = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  const int32_t group = tid / G, ngroups = (int32_t)(gridDim.x * blockDim.x) / G;
  const int sub = threadIdx.x % G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G));
  unsigned long long local_max = 0, bytes = 0;
  auto value_of = [&](const MsB& b) -> unsigned long long {
    const uint8_t p = b.p;
    unsigned long long best = 0;
    const int32_t e = b.eb + sub;
    if (b.src >= 0) {
      const unsigned long long f = __ldcg(fp + b.src);
      best = (f >> 1) + (((uint8_t)(f & 1ull) != p) ? (unsigned long long)b.w : 0ull);
    }
    if (b.src2 >= 0) {
      const unsigned long long f = __ldcg(fp + b.src2);
      const unsigned long long t = (f >> 1) + (((uint8_t)(f & 1ull) != p) ? (unsigned long long)b.w2 : 0ull);
      best = t > best ? t : best;
    }
    for (int32_t x = e + 2 * G; x < b.ee; x += G) {
      const unsigned long long f = __ldcg(fp + lo_src[x]);
      const unsigned long long t = (f >> 1) + (((uint8_t)(f & 1ull) != p) ? (unsigned long long)lo_w[x] : 0ull);
      best = t > best ? t : best;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const unsigned long long q = __shfl_xor_sync(gmask, best, o, G);
      best = q > best ? q : best;
    }
    const unsigned long long fin = best + (unsigned long long)(p ? b.cG : b.cC);
    if (sub == 0) {
      if (p > 1) atomicOr(bad_part, 1);
      local_max = fin > local_max ? fin : local_max;
      bytes += 4ull + 1ull + 16ull + (unsigned long long)(b.ee - b.eb) * 16ull + 4ull + 8ull;
    }
    return (fin << 1) | (unsigned long long)(p & 1);
  };
  auto lp = [&](int32_t l) -> int32_t { return (int32_t)lev_ptr[l < nlev ? l : nlev]; };
  int32_t beg = lp(0), end = lp(1), end1 = lp(2), end2 = lp(3), end3 = lp(4);
  MsA a1, a2;
  MsB cur, b1;
  {
    MsA a0;
    ms_load_a(a0, beg + group, end, lev_vtx, lo_off, lo_cC, lo_cG);
    ms_load_a(a1, end + group, end1, lev_vtx, lo_off, lo_cC, lo_cG);
    ms_load_b<G>(cur, a0, sub, lo_src, lo_w, part);
  }
  bool failed = false;
  for (int32_t l = 0; l < nlev; l++) {
    if (__syncthreads_or(failed)) break;  // a wait gave up: this CTA stops (the others' waits expire)
    if (cur.valid) {
      const unsigned long long pk = value_of(cur);
      if (sub == 0) {
        fp[cur.i] = pk;
        if (finish_out) finish_out[lev_vtx[cur.i]] = (int64_t)(pk >> 1);
      }
    }
    for (int32_t i = beg + group + ngroups; i < end; i += ngroups) {  // levels wider than the groups
      MsA a;
      MsB b;
      ms_load_a(a, i, end, lev_vtx, lo_off, lo_cC, lo_cG);
      ms_load_b<G>(b, a, sub, lo_src, lo_w, part);
      const unsigned long long pk = value_of(b);
      if (sub == 0) {
        fp[i] = pk;
        if (finish_out) finish_out[a.v] = (int64_t)(pk >> 1);
      }
    }
    // lookahead, then the grid barrier
    ms_load_b<G>(b1, a1, sub, lo_src, lo_w, part);
    ms_load_a(a2, end1 + group, end2, lev_vtx, lo_off, lo_cC, lo_cG);
    const int32_t end4 = lp(l + 5);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // this CTA's finish times before its arrival
      atomicAdd(bar, 1u);
      if (!grid_wait_bounded(bar, (unsigned)(l + 1) * gridDim.x)) {
        failed = true;
        atomicOr(bad_part, 2);
      }
      __threadfence();
    }
    cur = b1;
    a1 = a2;
    beg = end;
    end = end1;
    end1 = end2;
    end2 = end3;
    end3 = end4;
  }
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

}  // namespace gp
