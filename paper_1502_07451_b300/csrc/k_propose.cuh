// k_propose.cuh -- the learned proposal's split: vertices ordered by (logit desc, id asc), the first
// k = min(kC, kG) to the CPU (kC: longest prefix whose CPU load fits B_C; kG: shortest prefix after
// which the GPU load fits B_G).  No sort: two weighted radix selections (8-bit digits, most
// significant first) over the 64-bit keys (~float_key(logit) << 32 | id) find the first key of each
// prefix that crosses its threshold, run side by side in the same passes.
#pragma once
#include "gp_internal.cuh"

namespace gp {

__device__ __forceinline__ uint32_t float_order_key(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

struct PropSel {
  unsigned long long prefix[2];  // selected high digits (C, G)
  long long rem[2];              // remaining threshold within the prefix
  unsigned long long less[2];    // keys below the prefix region
  int found[2];                  // 0 while the running weight has not crossed the threshold
  int active[2];
  int bad;                       // a NaN logit was seen
};

__global__ void k_prop_keys(int64_t n, const float* __restrict__ logit, unsigned long long* __restrict__ key,
                            PropSel* sel) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float z = logit[v];
    if (isnan(z)) sel->bad = 1;
    key[v] = ((unsigned long long)(~float_order_key(z)) << 32) | (unsigned long long)(uint32_t)v;
  }
}

// histograms (weight and count per digit) of the keys inside each selection's current prefix
__global__ void __launch_bounds__(256) k_prop_hist(int64_t n, const unsigned long long* __restrict__ key,
                                                   const int64_t* __restrict__ vC, const int64_t* __restrict__ vG,
                                                   const PropSel* __restrict__ sel, int shift,
                                                   unsigned long long* __restrict__ hist /* [2][2][256] */) {
  __shared__ unsigned long long h[2][2][256];
  __shared__ unsigned long long s_pre[2];
  __shared__ int s_act[2];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) (&h[0][0][0])[i] = 0ull;
  if (threadIdx.x < 2) {
    s_pre[threadIdx.x] = sel->prefix[threadIdx.x];
    s_act[threadIdx.x] = sel->active[threadIdx.x];
  }
  __syncthreads();
  const unsigned long long hi_mask = shift >= 56 ? 0ull : (~0ull << (shift + 8));
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = key[v];
    const int d = (int)((k >> shift) & 255ull);
    const int64_t id = (int64_t)(k & 0xFFFFFFFFull);
    if (s_act[0] && (k & hi_mask) == s_pre[0]) {
      atomicAdd(&h[0][0][d], (unsigned long long)vC[id]);
      atomicAdd(&h[0][1][d], 1ull);
    }
    if (s_act[1] && (k & hi_mask) == s_pre[1]) {
      atomicAdd(&h[1][0][d], (unsigned long long)vG[id]);
      atomicAdd(&h[1][1][d], 1ull);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
    const unsigned long long x = (&h[0][0][0])[i];
    if (x) atomicAdd(&hist[i], x);
  }
}

// one thread: choose each selection's digit (the first where the running weight exceeds rem)
__global__ void k_prop_pick(PropSel* sel, int shift, unsigned long long* __restrict__ hist) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int q = 0; q < 2; q++) {
    if (!sel->active[q]) continue;
    const unsigned long long* w = hist + q * 512;
    const unsigned long long* c = w + 256;
    long long cum = 0;
    unsigned long long below = 0;
    int chosen = -1;
    for (int d = 0; d < 256; d++) {
      if (cum + (long long)w[d] > sel->rem[q]) {
        chosen = d;
        break;
      }
      cum += (long long)w[d];
      below += c[d];
    }
    if (chosen < 0) {  // the whole region fits: no crossing key
      sel->active[q] = 0;
      sel->found[q] = 0;
      continue;
    }
    sel->prefix[q] |= (unsigned long long)chosen << shift;
    sel->rem[q] -= cum;
    sel->less[q] += below;
    sel->found[q] = 1;
  }
  for (int i = 0; i < 1024; i++) hist[i] = 0ull;
}

// part[v] = 0 (CPU) for the first k keys: key < thr, or key <= thr when inclusive; all / none by mode
__global__ void k_prop_assign(int64_t n, const unsigned long long* __restrict__ key, unsigned long long thr, int mode,
                              uint8_t* __restrict__ part) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = key[v];
    bool cpu;
    if (mode == 0)
      cpu = false;
    else if (mode == 1)
      cpu = true;
    else if (mode == 2)
      cpu = k < thr;
    else
      cpu = k <= thr;
    part[(int64_t)(k & 0xFFFFFFFFull)] = cpu ? 0 : 1;
  }
}

}  // namespace gp
