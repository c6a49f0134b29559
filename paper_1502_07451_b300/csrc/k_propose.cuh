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

// Each selection's digit: the first where the running weight exceeds rem.  Warp q serves selection q:
// lane l sums digits 8l..8l+7, a warp scan gives the weight before each lane's digits, and the first lane
// whose digits pass rem walks them.  Then the histogram is cleared for the next digit (64 threads).
__global__ void __launch_bounds__(64) k_prop_pick(PropSel* sel, int shift, unsigned long long* __restrict__ hist) {
  const int q = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (sel->active[q]) {
    const unsigned long long* w = hist + q * 512;
    const unsigned long long* c = w + 256;
    long long w8 = 0;
    unsigned long long c8 = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
      w8 += (long long)w[8 * l + k];
      c8 += c[8 * l + k];
    }
    long long wi = w8;
    unsigned long long ci = c8;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long a = __shfl_up_sync(0xffffffffu, wi, o);
      const unsigned long long b = __shfl_up_sync(0xffffffffu, ci, o);
      if (l >= o) {
        wi += a;
        ci += b;
      }
    }
    const long long rem = sel->rem[q];
    const unsigned pass = __ballot_sync(0xffffffffu, wi > rem);
    if (pass == 0) {  // the whole region fits: no crossing key
      if (l == 0) {
        sel->active[q] = 0;
        sel->found[q] = 0;
      }
    } else if (l == __ffs(pass) - 1) {
      long long cum = wi - w8;
      unsigned long long below = ci - c8;
      int d = 8 * l;
      for (;; d++) {
        if (cum + (long long)w[d] > rem) break;
        cum += (long long)w[d];
        below += c[d];
      }
      sel->prefix[q] |= (unsigned long long)d << shift;
      sel->rem[q] -= cum;
      sel->less[q] += below;
      sel->found[q] = 1;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) hist[i] = 0ull;
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
