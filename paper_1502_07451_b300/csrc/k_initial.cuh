// k_initial.cuh -- initial bipartition by greedy graph growing on the coarsest graph.
//
// All vertices start on the GPU.  Trial t grows a CPU region from s_t = h(seed, 0xFFFFFFFF, t) mod n
// (moved first if its CPU weight fits B_C): while the GPU load exceeds B_G, among GPU-side vertices
// whose CPU weight still fits, the ones adjacent to the region are preferred (all of them when none
// is adjacent) and the one with the largest gain W(to CPU) - W(to GPU), smallest id on ties, moves.
// One CTA runs one trial; each step is a block-wide argmax.  The best trial is the feasible one with
// the smallest cut, then the smallest t.  All-GPU is chosen without trials when sum vG <= B_G.
// Fixed vertices (g.fix non-null): the CPU-pinned ones start in the CPU region, only free vertices
// move, and the pre-check is on the split with every free vertex on the GPU (decided in the kernel:
// every trial then reports it, flagged 2, and the pick records trial -1).
#pragma once
#include "gp_internal.cuh"
#include "k_coarsen.cuh"

namespace gp {

constexpr int kGggpThreads = 512;

__global__ void __launch_bounds__(256) k_wsum(LevelGraph g, int64_t* __restrict__ wsum) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = gw; v < g.n; v += nw) {
    const int64_t b = g.start[v];
    const int32_t d = g.deg[v];
    int64_t s = 0;
    for (int32_t k = lane; k < d; k += 32) s += g.W[b + k];
    s = warp_sum64(s);
    if (lane == 0) wsum[v] = s;
  }
}

struct GrowKey {
  int a;          // adjacent to the CPU region
  long long g;    // gain
  int32_t v;      // vertex, -1 = none
};
__device__ __forceinline__ bool grow_better(const GrowKey& x, const GrowKey& y) {
  if (x.v < 0) return false;
  if (y.v < 0) return true;
  if (x.a != y.a) return x.a > y.a;
  if (x.g != y.g) return x.g > y.g;
  return x.v < y.v;
}

__global__ void __launch_bounds__(kGggpThreads)
    k_gggp(LevelGraph g, long long BC, long long BG, long long SG, uint64_t seed, long long start_override,
           const int64_t* __restrict__ wsum, uint8_t* __restrict__ side_all, long long* __restrict__ toC_all,
           int32_t* __restrict__ adjC_all, long long* __restrict__ res) {
  __shared__ long long s_LC, s_LG;
  __shared__ int32_t s_x;
  __shared__ int s_pre;
  __shared__ GrowKey s_best[kGggpThreads / 32];
  __shared__ long long sh[32];
  __shared__ unsigned long long sacc[32];
  const int t = blockIdx.x;
  const int64_t n = g.n;
  uint8_t* side = side_all + (int64_t)t * n;
  long long* toC = toC_all + (int64_t)t * n;
  int32_t* adjC = adjC_all + (int64_t)t * n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long bytes = 0;
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
    side[v] = (g.fix && g.fix[v] == 0) ? 0 : 1;
    toC[v] = 0;
    adjC[v] = 0;
  }
  long long LC0 = 0, LG0 = SG;
  if (g.fix) {  // the CPU-pinned vertices form the initial region
    __syncthreads();
    long long c = 0, gg = 0;
    for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
      if (g.fix[v] != 0) continue;
      c += g.vC[v];
      gg += g.vG[v];
      for (int64_t e = g.start[v]; e < g.start[v] + g.deg[v]; e++) {
        atomicAdd((unsigned long long*)&toC[g.adj[e]], (unsigned long long)g.W[e]);
        atomicAdd(&adjC[g.adj[e]], 1);
      }
    }
    LC0 = block_sum<long long>(c, sh);
    LG0 = SG - block_sum<long long>(gg, sh);
  }
  if (threadIdx.x == 0) {
    const int64_t s = start_override >= 0 ? start_override
                                          : (int64_t)(pair_hash(seed, 0xFFFFFFFFu, (uint32_t)t) % (uint64_t)n);
    s_LC = LC0;
    s_LG = LG0;
    s_pre = g.fix != nullptr && LC0 <= BC && LG0 <= BG;
    const bool sfree = !g.fix || g.fix[s] < 0;
    s_x = (!s_pre && sfree && LC0 + g.vC[s] <= BC) ? (int32_t)s : -1;
  }
  __syncthreads();
  for (;;) {
    const int32_t x = s_x;
    if (x >= 0) {
      if (threadIdx.x == 0) {
        side[x] = 0;
        s_LC += g.vC[x];
        s_LG -= g.vG[x];
      }
      const int64_t b = g.start[x];
      const int32_t d = g.deg[x];
      for (int32_t k = threadIdx.x; k < d; k += blockDim.x) {
        const int32_t u = g.adj[b + k];  // rows hold distinct neighbours: no two threads share u
        toC[u] += g.W[b + k];
        adjC[u] += 1;
      }
      bytes += 24ull * (unsigned long long)((d + blockDim.x - 1 - threadIdx.x) / blockDim.x);
    }
    __syncthreads();
    if (s_LG <= BG) break;
    const long long LC = s_LC;
    GrowKey best{0, 0, -1};
    for (int64_t v = threadIdx.x; v < n; v += blockDim.x) {
      if (side[v] != 1 || (g.fix && g.fix[v] >= 0) || LC + g.vC[v] > BC) continue;
      const GrowKey k{adjC[v] > 0 ? 1 : 0, 2 * toC[v] - wsum[v], (int32_t)v};
      if (grow_better(k, best)) best = k;
    }
    bytes += 22ull * (unsigned long long)((n + blockDim.x - 1 - threadIdx.x) / blockDim.x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      GrowKey q;
      q.a = __shfl_xor_sync(0xffffffffu, best.a, o);
      q.g = __shfl_xor_sync(0xffffffffu, best.g, o);
      q.v = __shfl_xor_sync(0xffffffffu, best.v, o);
      if (grow_better(q, best)) best = q;
    }
    if (lane == 0) s_best[wid] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      GrowKey bb = s_best[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); w++)
        if (grow_better(s_best[w], bb)) bb = s_best[w];
      s_x = bb.v;
    }
    __syncthreads();
    if (s_x < 0) break;
  }
  long long cut = 0;
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x)
    if (side[v] == 0) cut += wsum[v] - toC[v];
  cut = block_sum<long long>(cut, sh);
  if (threadIdx.x == 0) {
    res[4 * t + 0] = cut;
    res[4 * t + 1] = s_pre ? 2 : (s_LC <= BC && s_LG <= BG) ? 1 : 0;
    res[4 * t + 2] = s_LC;
    res[4 * t + 3] = s_LG;
  }
  account(F_GGGP, bytes, sacc);
}

__global__ void k_gggp_pick(int64_t n, int ntrials, const long long* __restrict__ res,
                            const uint8_t* __restrict__ side_all, uint8_t* __restrict__ part, int32_t* trial_out) {
  __shared__ int s_t;
  if (threadIdx.x == 0) {
    int bt = 0;
    for (int t = 1; t < ntrials; t++) {
      const long long f = res[4 * t + 1], bf = res[4 * bt + 1];
      if (f > bf || (f == bf && res[4 * t] < res[4 * bt])) bt = t;
    }
    s_t = bt;
    *trial_out = res[4 * bt + 1] == 2 ? -1 : bt;  // 2: the pre-check's split (every trial holds it)
  }
  __syncthreads();
  const uint8_t* side = side_all + (int64_t)s_t * n;
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) part[v] = side[v];
}

__global__ void k_set_i32(int32_t* p, int32_t x) { *p = x; }

void gggp(const LevelGraph& g, int64_t BC, int64_t BG, int64_t SG, uint64_t seed, uint8_t* part, int32_t* trial_dev,
          cudaStream_t s) {
  const int64_t n = g.n;
  if (n <= 0) return;
  if (!g.fix && SG <= BG) {
    GP_LAUNCH(F_GGGP, k_fill_u8, grid_for(n, 256), 256, 0, s, n, part, (uint8_t)1);
    GP_LAUNCH(F_MISC, k_set_i32, 1, 1, 0, s, trial_dev, -1);
    GP_CHECK_LAUNCH();
    return;
  }
  int64_t* wsum = dnew<int64_t>(n, s);
  uint8_t* side_all = dnew<uint8_t>(n * kTrials, s);
  long long* toC_all = dnew<long long>(n * kTrials, s);
  int32_t* adjC_all = dnew<int32_t>(n * kTrials, s);
  long long* res = dnew<long long>(4 * kTrials, s);
  GP_LAUNCH(F_GGGP, k_wsum, grid_for(n * 32, 256), 256, 0, s, g, wsum);
  GP_LAUNCH(F_GGGP, k_gggp, kTrials, kGggpThreads, 0, s, g, (long long)BC, (long long)BG, (long long)SG, seed,
            -1ll, wsum, side_all, toC_all, adjC_all, res);
  GP_LAUNCH(F_GGGP, k_gggp_pick, 1, 256, 0, s, n, kTrials, res, side_all, part, trial_dev);
  GP_CHECK_LAUNCH();
  dfree(wsum, s);
  dfree(side_all, s);
  dfree(toC_all, s);
  dfree(adjC_all, s);
  dfree(res, s);
}

void gggp_grow_one(const LevelGraph& g, int64_t BC, int64_t BG, int64_t start, uint8_t* part, int64_t* cut_dev,
                   cudaStream_t s) {
  const int64_t n = g.n;
  int64_t* wsum = dnew<int64_t>(n, s);
  long long* toC = dnew<long long>(n, s);
  int32_t* adjC = dnew<int32_t>(n, s);
  long long* res = dnew<long long>(4, s);
  long long* sg = dnew<long long>(1, s);
  GP_LAUNCH(F_GGGP, k_wsum, grid_for(n * 32, 256), 256, 0, s, g, wsum);
  sum_i64(g.vG, n, sg, s);  // SG of this graph
  long long SG = 0;
  GP_CUDA(cudaMemcpyAsync(&SG, sg, sizeof(long long), cudaMemcpyDeviceToHost, s));
  GP_CUDA(cudaStreamSynchronize(s));
  GP_LAUNCH(F_GGGP, k_gggp, 1, kGggpThreads, 0, s, g, (long long)BC, (long long)BG, SG, 0ull, (long long)start,
            wsum, part, toC, adjC, res);
  GP_CUDA(cudaMemcpyAsync(cut_dev, res, sizeof(long long), cudaMemcpyDeviceToDevice, s));
  GP_CHECK_LAUNCH();
  dfree(wsum, s);
  dfree(toC, s);
  dfree(adjC, s);
  dfree(res, s);
  dfree(sg, s);
}

}  // namespace gp
